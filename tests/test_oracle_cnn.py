"""Pins of the FP64 MultiScale, SmallScale and MonoScale CNN oracle (Sec. 3.1): library special cases
(torch conv2d / pooling / interpolation in FP64 on CPU, used only here to pin
the oracle), adjointness, finite differences, the parameter counts and the
embedding of the SmallScale in a zero-padded MultiScale."""
import numpy as np
import pytest

from oracle import cnn as C

torch = pytest.importorskip("torch")
F = torch.nn.functional


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).double()


def test_parameter_count():
    assert C.param_count() == 372643


def test_conv3x3_replicate_matches_library():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 9, 11))
    w = rng.standard_normal((7, 5, 3, 3))
    b = rng.standard_normal(7)
    ref = F.conv2d(F.pad(T(x)[None], (1, 1, 1, 1), mode="replicate"), T(w), T(b))[0].numpy()
    assert np.allclose(C.conv3x3(x, w, b), ref, atol=1e-12)


def test_conv3x3_backward_matches_autograd():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((4, 6, 7))
    w = rng.standard_normal((3, 4, 3, 3))
    b = rng.standard_normal(3)
    gy = rng.standard_normal((3, 6, 7))
    xt, wt, bt = (T(a).requires_grad_() for a in (x, w, b))
    y = F.conv2d(F.pad(xt[None], (1, 1, 1, 1), mode="replicate"), wt, bt)[0]
    y.backward(T(gy))
    gx, gw, gb = C.conv3x3_backward(x, w, gy)
    assert np.allclose(gx, xt.grad.numpy(), atol=1e-12)
    assert np.allclose(gw, wt.grad.numpy(), atol=1e-12)
    assert np.allclose(gb, bt.grad.numpy(), atol=1e-12)


def test_avgpool_is_bilinear_half_and_matches_library():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 8, 12))
    p = C.avgpool2(x)
    assert np.allclose(p, F.avg_pool2d(T(x)[None], 2)[0].numpy(), atol=1e-14)
    bil = F.interpolate(T(x)[None], scale_factor=0.5, mode="bilinear", align_corners=False)
    assert np.allclose(p, bil[0].numpy(), atol=1e-14)


def test_upsample_matches_library_and_is_adjoint():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 5, 7))
    up = C.upsample2(x)
    ref = F.interpolate(T(x)[None], scale_factor=2, mode="bilinear", align_corners=False)
    assert np.allclose(up, ref[0].numpy(), atol=1e-14)
    y = rng.standard_normal(up.shape)
    assert np.isclose(np.sum(up * y), np.sum(x * C.upsample2_backward(y)), rtol=1e-13)
    gp = rng.standard_normal((2, 4, 6))
    xx = rng.standard_normal((2, 8, 12))
    assert np.isclose(np.sum(C.avgpool2(xx) * gp), np.sum(xx * C.avgpool2_backward(gp)),
                      rtol=1e-13)


def test_network_gradients_by_central_differences():
    rng = np.random.default_rng(4)
    params = C.init_params(seed=1)
    # small random biases so that ReLU masks are not degenerate
    params = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in params]
    n = 8
    div = rng.standard_normal((n, n))
    fl = (rng.random((n, n)) < 0.2).astype(np.uint8)
    gout = rng.standard_normal((n, n))
    out, tape = C.forward(params, div, fl, keep=True)
    grads = C.backward(params, tape, gout)
    eps = 1e-6
    checked = 0
    for li in [0, 3, 4, 5, 9, 11, 12, 18]:
        w, b = params[li]
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in w.shape)
            wp = [(ww.copy(), bb) for ww, bb in params]
            wm = [(ww.copy(), bb) for ww, bb in params]
            wp[li][0][idx] += eps
            wm[li][0][idx] -= eps
            fd = (np.sum(C.forward(wp, div, fl) * gout) - np.sum(C.forward(wm, div, fl) * gout)) / (2 * eps)
            assert np.isclose(grads[li][0][idx], fd, rtol=1e-5, atol=1e-8), (li, idx)
            checked += 1
        j = int(rng.integers(0, b.shape[0]))
        bp = [(ww, bb.copy()) for ww, bb in params]
        bm = [(ww, bb.copy()) for ww, bb in params]
        bp[li][1][j] += eps
        bm[li][1][j] -= eps
        fd = (np.sum(C.forward(bp, div, fl) * gout) - np.sum(C.forward(bm, div, fl) * gout)) / (2 * eps)
        assert np.isclose(grads[li][1][j], fd, rtol=1e-5, atol=1e-8)
    assert checked == 24


def test_forward_shapes_and_scale_structure():
    params = C.init_params(seed=2)
    assert len(params) == 5 + 7 + 7
    out = C.forward(params, np.zeros((16, 16)), np.zeros((16, 16), np.uint8))
    assert out.shape == (16, 16)


def test_smallscale_parameter_count():
    # about three times fewer parameters than the MultiScale (Sec. 3.1)
    assert C.param_count("smallscale") == 123491
    assert 2.5 < C.param_count() / C.param_count("smallscale") < 3.5
    shapes = C.param_shapes("smallscale")
    assert len(shapes) == len(C.param_shapes()) == 19
    assert max(ws[0] for _, _, ws, _ in shapes) == 32


def embed_small_in_multiscale(small):
    """MultiScale parameters that compute the SmallScale network: its weights
    in the first channels of every layer, zeros on the extra channels (their
    pre-activations are 0, ReLU keeps them 0, and no later weight reads them)."""
    out = []
    for (_, _, ws, bs), (w, b) in zip(C.param_shapes(), small):
        W_ = np.zeros(ws)
        B_ = np.zeros(bs)
        W_[:w.shape[0], :w.shape[1]] = w
        B_[:b.shape[0]] = b
        out.append((W_, B_))
    return out


def test_smallscale_is_a_zero_padded_multiscale():
    rng = np.random.default_rng(7)
    small = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in
             C.init_params(seed=3, arch="smallscale")]
    big = embed_small_in_multiscale(small)
    n = 16
    div = rng.standard_normal((n, n))
    fl = (rng.random((n, n)) < 0.2).astype(np.uint8)
    gout = rng.standard_normal((n, n))
    o_s, tape_s = C.forward(small, div, fl, keep=True)
    o_b, tape_b = C.forward(big, div, fl, keep=True)
    assert np.array_equal(o_s, o_b)
    g_s = C.backward(small, tape_s, gout)
    g_b = C.backward(big, tape_b, gout)
    for (gw, gb), (hw, hb) in zip(g_s, g_b):
        assert np.allclose(gw, hw[:gw.shape[0], :gw.shape[1]], rtol=1e-12, atol=1e-14)
        assert np.allclose(gb, hb[:gb.shape[0]], rtol=1e-12, atol=1e-14)
    # flatten / unflatten round trip in the SmallScale layout
    flat = C.flatten(small)
    assert flat.size == C.param_count("smallscale")
    back = C.unflatten(flat, "smallscale")
    assert all(np.array_equal(a, c) and np.array_equal(b, d)
               for (a, b), (c, d) in zip(small, back))


def test_smallscale_gradients_by_central_differences():
    rng = np.random.default_rng(8)
    params = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in
              C.init_params(seed=4, arch="smallscale")]
    n = 8
    div = rng.standard_normal((n, n))
    fl = (rng.random((n, n)) < 0.2).astype(np.uint8)
    gout = rng.standard_normal((n, n))
    _, tape = C.forward(params, div, fl, keep=True)
    grads = C.backward(params, tape, gout)
    eps = 1e-6
    for li in [1, 2, 7, 14]:
        w = params[li][0]
        idx = tuple(rng.integers(0, s) for s in w.shape)
        wp = [(ww.copy(), bb) for ww, bb in params]
        wm = [(ww.copy(), bb) for ww, bb in params]
        wp[li][0][idx] += eps
        wm[li][0][idx] -= eps
        fd = (np.sum(C.forward(wp, div, fl) * gout) - np.sum(C.forward(wm, div, fl) * gout)) / (2 * eps)
        assert np.isclose(grads[li][0][idx], fd, rtol=1e-5, atol=1e-8), (li, idx)


def test_monoscale_parameter_count_and_structure():
    shapes = C.param_shapes("monoscale")
    assert len(shapes) == 9 and all(sc == 1 for sc, _, _, _ in shapes)
    assert C.param_count("monoscale") == 222497
    assert shapes[0][2][1] == 2 and shapes[-1][2][0] == 1
    with pytest.raises(ValueError):
        C.arch_of([(np.zeros((4, 2, 3, 3)), np.zeros(4))])


def test_monoscale_is_a_chain_of_library_convolutions():
    """The MonoScale is a plain feed-forward chain: replicate padding,
    convolution, ReLU except after the last two (torch FP64 on CPU)."""
    rng = np.random.default_rng(9)
    params = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in
              C.init_params(seed=5, arch="monoscale")]
    n = 12
    div = rng.standard_normal((n, 2 * n))
    fl = (rng.random((n, 2 * n)) < 0.2).astype(np.uint8)
    h = torch.stack([T(div), T(fl.astype(np.float64))])[None]
    for l, (w, b) in enumerate(params):
        h = F.conv2d(F.pad(h, (1, 1, 1, 1), mode="replicate"), T(w), T(b))
        if l < len(params) - 2:
            h = torch.relu(h)
    assert C.arch_of(params) == "monoscale"
    assert np.allclose(C.forward(params, div, fl), h[0, 0].numpy(), rtol=1e-12, atol=1e-12)


def test_monoscale_gradients_by_central_differences():
    rng = np.random.default_rng(10)
    params = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in
              C.init_params(seed=6, arch="monoscale")]
    n = 8
    div = rng.standard_normal((n, n))
    fl = (rng.random((n, n)) < 0.2).astype(np.uint8)
    gout = rng.standard_normal((n, n))
    _, tape = C.forward(params, div, fl, keep=True)
    grads = C.backward(params, tape, gout)
    eps = 1e-6
    for li in [0, 3, 6, 8]:
        w, b = params[li]
        idx = tuple(rng.integers(0, s) for s in w.shape)
        wp = [(ww.copy(), bb) for ww, bb in params]
        wm = [(ww.copy(), bb) for ww, bb in params]
        wp[li][0][idx] += eps
        wm[li][0][idx] -= eps
        fd = (np.sum(C.forward(wp, div, fl) * gout) - np.sum(C.forward(wm, div, fl) * gout)) / (2 * eps)
        assert np.isclose(grads[li][0][idx], fd, rtol=1e-5, atol=1e-8), (li, idx)
        j = int(rng.integers(0, b.shape[0]))
        bp = [(ww, bb.copy()) for ww, bb in params]
        bm = [(ww, bb.copy()) for ww, bb in params]
        bp[li][1][j] += eps
        bm[li][1][j] -= eps
        fd = (np.sum(C.forward(bp, div, fl) * gout) - np.sum(C.forward(bm, div, fl) * gout)) / (2 * eps)
        assert np.isclose(grads[li][1][j], fd, rtol=1e-5, atol=1e-8)


def test_unet_parameter_count_and_structure():
    shapes = C.param_shapes("unet")
    assert len(shapes) == 20 and C.param_count("unet") == 388545
    # five scales; the last layer is the 1 x 1 convolution 32 -> 1
    assert sorted({sc for sc, _, _, _ in shapes}) == [1, 2, 4, 8, 16]
    assert shapes[-1][2] == (1, 32, 1, 1)
    assert C.arch_of(C.init_params(0, "unet")) == "unet"


def test_maxpool_matches_library():
    rng = np.random.default_rng(11)
    x = rng.standard_normal((3, 8, 12))
    assert np.array_equal(C.maxpool2(x), F.max_pool2d(T(x)[None], 2)[0].numpy())


def test_unet_is_a_chain_of_library_operations():
    """Encoder (replicate-padded 3 x 3 convolutions, ReLU, 2 x 2 max pooling),
    decoder ([bilinear x 2 of the coarser features, skip features], 3 x 3
    convolutions), 1 x 1 output; ReLU after every convolution except the last
    two (torch FP64 on CPU)."""
    rng = np.random.default_rng(12)
    params = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in C.init_params(6, "unet")]
    n = 32
    div = rng.standard_normal((n, n))
    fl = (rng.random((n, n)) < 0.2).astype(np.uint8)
    ws = iter(enumerate(params))

    def conv(h):
        l, (w, b) = next(ws)
        pad = (1, 1, 1, 1) if w.shape[2] == 3 else (0, 0, 0, 0)
        h = F.conv2d(F.pad(h, pad, mode="replicate"), T(w), T(b))
        return torch.relu(h) if l < len(params) - 2 else h

    h = torch.stack([T(div), T(fl.astype(np.float64))])[None]
    skips = []
    for level in range(4):
        if level > 0:
            h = F.max_pool2d(h, 2)
        h = conv(conv(h))
        skips.append(h)
    h = conv(conv(conv(F.max_pool2d(h, 2))))
    for level in (3, 2, 1, 0):
        up = F.interpolate(h, scale_factor=2, mode="bilinear", align_corners=False)
        h = conv(conv(torch.cat([up, skips[level]], dim=1)))
    h = conv(h)
    assert np.allclose(C.forward(params, div, fl), h[0, 0].numpy(), rtol=1e-12, atol=1e-12)


def test_unet_gradients_match_library_autograd():
    """The oracle backward of the Unet against torch autograd of the same
    chain of library operations (FP64 on CPU; random inputs, so no ties in the
    max pooling)."""
    rng = np.random.default_rng(13)
    params = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in C.init_params(7, "unet")]
    n = 32
    div = rng.standard_normal((n, n))
    fl = (rng.random((n, n)) < 0.2).astype(np.uint8)
    gout = rng.standard_normal((n, n))
    tw = [(T(w).requires_grad_(), T(b).requires_grad_()) for w, b in params]
    ws = iter(enumerate(tw))

    def conv(h):
        l, (w, b) = next(ws)
        pad = (1, 1, 1, 1) if w.shape[2] == 3 else (0, 0, 0, 0)
        h = F.conv2d(F.pad(h, pad, mode="replicate"), w, b)
        return torch.relu(h) if l < len(tw) - 2 else h

    h = torch.stack([T(div), T(fl.astype(np.float64))])[None]
    skips = []
    for level in range(4):
        if level > 0:
            h = F.max_pool2d(h, 2)
        h = conv(conv(h))
        skips.append(h)
    h = conv(conv(conv(F.max_pool2d(h, 2))))
    for level in (3, 2, 1, 0):
        up = F.interpolate(h, scale_factor=2, mode="bilinear", align_corners=False)
        h = conv(conv(torch.cat([up, skips[level]], dim=1)))
    (conv(h)[0, 0] * T(gout)).sum().backward()
    out, tape = C.forward(params, div, fl, keep=True)
    grads = C.backward(params, tape, gout)
    for (gw, gb), (w, b) in zip(grads, tw):
        assert np.allclose(gw, w.grad.numpy(), rtol=1e-10, atol=1e-12)
        assert np.allclose(gb, b.grad.numpy(), rtol=1e-10, atol=1e-12)


def test_unet_gradients_by_central_differences():
    rng = np.random.default_rng(14)
    params = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in C.init_params(8, "unet")]
    n = 16
    div = rng.standard_normal((n, n))
    fl = (rng.random((n, n)) < 0.2).astype(np.uint8)
    gout = rng.standard_normal((n, n))
    _, tape = C.forward(params, div, fl, keep=True)
    grads = C.backward(params, tape, gout)
    eps = 1e-6
    for li in [0, 5, 9, 12, 17, 19]:
        w = params[li][0]
        idx = tuple(rng.integers(0, s) for s in w.shape)
        wp = [(ww.copy(), bb) for ww, bb in params]
        wm = [(ww.copy(), bb) for ww, bb in params]
        wp[li][0][idx] += eps
        wm[li][0][idx] -= eps
        fd = (np.sum(C.forward(wp, div, fl) * gout) - np.sum(C.forward(wm, div, fl) * gout)) / (2 * eps)
        assert np.isclose(grads[li][0][idx], fd, rtol=1e-5, atol=1e-8), (li, idx)


def test_maxpool_backward_routes_to_the_first_maximum():
    x = np.array([[[1.0, 3.0, 2.0, 2.0], [3.0, 0.0, 2.0, 2.0]]])
    g = np.array([[[5.0, 7.0]]])
    gx = C.maxpool2_backward(x, g)
    # ties go to the first maximum in the order (0, 0), (0, 1), (1, 0), (1, 1)
    assert np.array_equal(gx, [[[0.0, 5.0, 7.0, 0.0], [0.0, 0.0, 0.0, 0.0]]])


def test_round_bf16_matches_an_independent_conversion():
    # torch's CPU float32 -> bfloat16 conversion (round to nearest even) on
    # random values across the exponent range, exact ties, subnormals and
    # values at the top of the range (which round to infinity)
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    rand = (rng.standard_normal(20000) * np.exp2(rng.integers(-130, 127, 20000))).astype(np.float32)
    base = rng.integers(0, 1 << 15, 4000).astype(np.uint32) << 16
    ties = (base | 0x8000).view(np.float32)            # exactly half way
    above = (base | 0x8001).view(np.float32)
    below = (base | 0x7FFF).view(np.float32)
    sub = (rng.integers(1, 1 << 23, 2000).astype(np.uint32)).view(np.float32)
    top = np.array([3.3895314e38, 3.3961776e38, 3.4028235e38, -3.4028235e38, 0.0, -0.0,
                    np.float32(1.0) + np.float32(2 ** -8)], np.float32)
    x = np.concatenate([rand, ties, -ties, above, below, sub, -sub, top]).astype(np.float32)
    x = x[np.isfinite(x)]
    exp = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    got = C.round_bf16(x)
    assert np.array_equal(np.isinf(got), np.isinf(exp))
    fin = np.isfinite(exp)
    assert np.array_equal(got[fin], exp[fin])
    assert np.array_equal(np.signbit(got), np.signbit(exp))
