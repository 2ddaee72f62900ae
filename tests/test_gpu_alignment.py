"""The vector paths of the streaming kernels (rows a multiple of four cells,
16-byte aligned arrays) and their one-cell fallbacks give the same results:
every call here runs once on aligned tensors and once on views that start 4
bytes (float) or 1 byte (flags) past an aligned address, which the library
must route to the scalar kernels.  Elementwise results are bit-identical; the
norms' sums within their FP32 rounding; the network input (pooled in FP32 on
the vector path, in FP64 on the scalar one) within its BF16 rounding."""
import numpy as np
import pytest

from paper_2109_09363_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hp = pytest.importorskip("paper_2109_09363_gb300")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09363_gb300 import build
    build.build()
    return torch.device("cuda:0")


def shifted(t, off):
    """A copy of t in a buffer of the same dtype that starts `off` elements
    past the buffer's (aligned) start."""
    base = torch.zeros(t.numel() + off, dtype=t.dtype, device=t.device)
    view = base[off:off + t.numel()].view(t.shape)
    view.copy_(t)
    assert view.data_ptr() % 16 != 0
    return view


def case(B, ny, nx, seed):
    us, vs, fs = [], [], []
    for b in range(B):
        u, v = W.vortex_velocity(ny, nx, seed + b, n_vortices=6, width=(2.0, 8.0))
        us.append(u); vs.append(v)
        fs.append(W.random_obstacles(ny, nx, seed + 50 + b, rect_side=(3, 12), disc_radius=(2, 8)))
    return (torch.from_numpy(np.stack(us).astype(np.float32)),
            torch.from_numpy(np.stack(vs).astype(np.float32)),
            torch.from_numpy(np.stack(fs)))


@pytest.mark.parametrize("B,ny,nx", [(2, 37, 264), (1, 16, 64)])
def test_stencil_calls_match_their_scalar_fallbacks(dev, B, ny, nx):
    u, v, fl = (t.to(dev) for t in case(B, ny, nx, 11))
    div_a = hp.hp_divergence(u, v, fl)
    mask_a = hp.hp_face_mask(fl)
    div_b = hp.hp_divergence(shifted(u, 1), shifted(v, 1), shifted(fl, 1))
    mask_b = hp.hp_face_mask(shifted(fl, 1))
    assert torch.equal(div_a, div_b)
    assert torch.equal(mask_a, mask_b)
    ctx = hp.Context(B, ny, nx)
    e1a, eia = hp.hp_div_norms(ctx, u, v, fl)
    e1b, eib = hp.hp_div_norms(ctx, shifted(u, 1), shifted(v, 1), shifted(fl, 1))
    assert torch.allclose(e1a, e1b, rtol=1e-6, atol=0)
    assert torch.equal(eia, eib)
    # the projection: mask and divergence, correction and norms on both paths
    prm = hp.ProjectParams(threshold=1e-3, max_iters=500)
    ua, va = u.clone(), v.clone()
    oa = hp.hp_project(ctx, ua, va, fl, prm)
    ub, vb, fb = shifted(u, 1), shifted(v, 1), shifted(fl, 1)
    ob = hp.hp_project(ctx, ub, vb, fb, prm)
    torch.cuda.synchronize()
    assert torch.equal(oa["iters"], ob["iters"])
    assert torch.equal(ua, ub) and torch.equal(va, vb)
    assert torch.equal(oa["p"], ob["p"])
    assert torch.allclose(oa["e1"], ob["e1"], rtol=1e-6, atol=0)
    ctx.check()


@pytest.mark.parametrize("off", [1, 2, 3])
@pytest.mark.parametrize("B,ny,nx", [(2, 37, 264), (3, 5, 516)])
def test_misaligned_u_alone_stays_on_the_vector_path(dev, B, ny, nx, off):
    # u may start at any float (its rows of nx + 1 values start at every
    # offset anyway): with v and the flags aligned the vector kernels run and
    # give the results of aligned u bit for bit
    u, v, fl = (t.to(dev) for t in case(B, ny, nx, 17))
    us = shifted(u, off)
    assert torch.equal(hp.hp_divergence(u, v, fl), hp.hp_divergence(us, v, fl))
    ctx = hp.Context(B, ny, nx)
    e1a, eia = hp.hp_div_norms(ctx, u, v, fl)
    e1b, eib = hp.hp_div_norms(ctx, us, v, fl)
    assert torch.equal(e1a, e1b) and torch.equal(eia, eib)
    prm = hp.ProjectParams(threshold=1e-3, max_iters=300)
    ua, va = u.clone(), v.clone()
    vb = v.clone()
    oa = hp.hp_project(ctx, ua, va, fl, prm)
    ob = hp.hp_project(ctx, us, vb, fl, prm)
    torch.cuda.synchronize()
    assert torch.equal(oa["iters"], ob["iters"])
    assert torch.equal(ua, us) and torch.equal(va, vb)
    assert torch.equal(oa["e1"], ob["e1"])
    ctx.check()


def test_network_input_matches_its_scalar_fallback(dev):
    from paper_2109_09363_gb300 import training as T
    B, n = 2, 64
    u, v, fl = (t.to(dev) for t in case(B, n, n, 21))
    div = hp.hp_divergence(u, v, fl)
    cnn = hp.CNN(B, n, n, params=T.init_params(seed=5))
    pa, sa = hp.hp_cnn_forward(cnn, div, fl)
    pb, sb = hp.hp_cnn_forward(cnn, shifted(div, 1), shifted(fl, 1))
    torch.cuda.synchronize()
    assert torch.equal(sa, sb)
    scale = pa.abs().max().item()
    assert (pa - pb).abs().max().item() <= 2e-2 * scale
    assert cnn.check() == 0
