"""FP64 oracle of the MultiScale CNN and of its narrower SmallScale variant
(Sec. 3.1, network architectures), numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings of the paper (listed in the design notes): every convolution is 3 x 3
with replication padding; scale 1/4 is 2 -> 32 -> 64 -> 64 -> 32 -> 1 (5
convolutions), scales 1/2 and 1 are 3 -> 32 -> 64 -> 64 -> 64 -> 64 -> 32 -> 1
(7 convolutions) with input [div/s, flags, upsampled coarser output]; ReLU
after every convolution of a branch except its last two; down-sampling is 2 x
2 (4 x 4) average pooling, which equals bilinear down-sampling by 1/2 at
half-pixel centres; up-sampling is bilinear x 2 at half-pixel centres with the
edge sample repeated.  372,643 parameters.

SmallScale (Sec. 3.1): the same structure with fewer filters per layer, about
three times fewer parameters.  Reading: every 64-channel layer has 32
channels, 2 -> 32 -> 32 -> 32 -> 32 -> 1 and 3 -> 32 -> 32 -> 32 -> 32 -> 32
-> 32 -> 1; 123,491 parameters (3.02 times fewer).

MonoScale (Sec. 3.1): one feed-forward branch of 9 convolutions at full
resolution with replicated borders on [div/s, flags].  Reading: 3 x 3 kernels
only, 2 -> 32 -> 64 -> 64 -> 64 -> 64 -> 64 -> 64 -> 32 -> 1, ReLU after every
convolution except the last two; 222,497 parameters.

Unet (Sec. 3.1: five scales, max pooling down, bilinear up, skip connections,
3 x 3 and 1 x 1 kernels; the widths are in a figure that is not recoverable).
Reading: encoder levels at n, n/2, n/4, n/8 end in 32 channels (the skip
features): 2 -> 32 -> 32, then after each 2 x 2 max pooling 32 -> 64 -> 32;
the bottom (n/16) 32 -> 64 -> 64 -> 32; each decoder level takes
[up(coarser), skip] (64 channels) through 64 -> 64 -> 32, the last one
64 -> 32 -> 32 and a 1 x 1 convolution 32 -> 1.  ReLU after every
convolution except the last two; 388,545 parameters.

Layout: activations [C][H][W] (one grid), weights [Cout][Cin][3][3].
"""
from __future__ import annotations

import numpy as np

BRANCH_WIDTHS = {
    4: [2, 32, 64, 64, 32, 1],               # scale 1/4
    2: [3, 32, 64, 64, 64, 64, 32, 1],       # scale 1/2
    1: [3, 32, 64, 64, 64, 64, 32, 1],       # full scale
}
SMALL_WIDTHS = {
    4: [2, 32, 32, 32, 32, 1],
    2: [3, 32, 32, 32, 32, 32, 32, 1],
    1: [3, 32, 32, 32, 32, 32, 32, 1],
}
SCALES = (4, 2, 1)
# every architecture as its branches in network order: (scale, widths); the
# input of a branch is [div_s, flags] at its scale, followed by the
# up-sampled output of the branch before it when there is one
ARCHS = {
    "multiscale": [(sc, BRANCH_WIDTHS[sc]) for sc in SCALES],
    "smallscale": [(sc, SMALL_WIDTHS[sc]) for sc in SCALES],
    "monoscale": [(1, [2, 32, 64, 64, 64, 64, 64, 64, 32, 1])],
}


# the Unet's layers in network order: (scale, cin, cout, kernel size)
UNET_LAYERS = ([(1, 2, 32, 3), (1, 32, 32, 3)] +
               [(sc, c, o, 3) for sc in (2, 4, 8) for c, o in ((32, 64), (64, 32))] +
               [(16, 32, 64, 3), (16, 64, 64, 3), (16, 64, 32, 3)] +
               [(sc, c, o, 3) for sc in (8, 4, 2) for c, o in ((64, 64), (64, 32))] +
               [(1, 64, 32, 3), (1, 32, 32, 3), (1, 32, 1, 1)])


def param_shapes(arch="multiscale"):
    """[(scale, layer, (Cout, Cin, k, k), (Cout,))] in network order."""
    if arch == "unet":
        return [(sc, l, (o, c, k, k), (o,)) for l, (sc, c, o, k) in enumerate(UNET_LAYERS)]
    out = []
    for sc, w in ARCHS[arch]:
        for l in range(len(w) - 1):
            out.append((sc, l, (w[l + 1], w[l], 3, 3), (w[l + 1],)))
    return out


def param_count(arch="multiscale"):
    return sum(int(np.prod(ws)) + int(np.prod(bs)) for _, _, ws, bs in param_shapes(arch))


def arch_of(params):
    """The architecture whose layer shapes the parameter list has."""
    shapes = [(tuple(np.shape(w)), tuple(np.shape(b))) for w, b in params]
    for name in list(ARCHS) + ["unet"]:
        if shapes == [(ws, bs) for _, _, ws, bs in param_shapes(name)]:
            return name
    raise ValueError("parameters of no known architecture")


def relu_after(l, nl):
    """ReLU after every convolution of a branch of nl layers except its last
    two."""
    return l < nl - 2


def init_params(seed=0, arch="multiscale"):
    """He-uniform weights, zero biases (a deterministic starting point)."""
    g = np.random.Generator(np.random.PCG64(seed))
    params = []
    for sc, l, ws, bs in param_shapes(arch):
        fan_in = ws[1] * ws[2] * ws[3]
        lim = np.sqrt(6.0 / fan_in)
        params.append((g.uniform(-lim, lim, ws), np.zeros(bs)))
    return params


# ------------------------------------------------------------- primitives

def conv3x3(x, w, b):
    """y[o, i, j] = b[o] + sum_{c, dy, dx} w[o, c, dy, dx] x_pad[c, i + dy, j + dx],
    x_pad = x with one replicated ghost cell on each side."""
    C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)), mode="edge")
    y = np.zeros((w.shape[0], H, W))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("oc,chw->ohw", w[:, :, dy, dx], xp[:, dy:dy + H, dx:dx + W])
    return y + b[:, None, None]


def conv3x3_backward(x, w, gy):
    """Gradients of conv3x3 w.r.t. x, w and b given gy = dL/dy."""
    C, H, W = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)), mode="edge")
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gw[:, :, dy, dx] = np.einsum("ohw,chw->oc", gy, xp[:, dy:dy + H, dx:dx + W])
            gxp[:, dy:dy + H, dx:dx + W] += np.einsum("oc,ohw->chw", w[:, :, dy, dx], gy)
    # transpose of the replication padding: ghost gradients go to the edge
    gxp[:, 1, :] += gxp[:, 0, :]
    gxp[:, H, :] += gxp[:, H + 1, :]
    gxp[:, :, 1] += gxp[:, :, 0]
    gxp[:, :, W] += gxp[:, :, W + 1]
    return gxp[:, 1:H + 1, 1:W + 1], gw, gy.sum(axis=(1, 2))


def maxpool2(x):
    """2 x 2 max pooling of [C][H][W] (H, W even)."""
    return np.maximum(np.maximum(x[:, 0::2, 0::2], x[:, 0::2, 1::2]),
                      np.maximum(x[:, 1::2, 0::2], x[:, 1::2, 1::2]))


def conv1x1(x, w, b):
    """y[o] = b[o] + sum_i w[o, i] x[i]; w [Cout][Cin][1][1]."""
    return np.einsum("oi,ihw->ohw", w[:, :, 0, 0], x) + b[:, None, None]


def avgpool2(x):
    C, H, W = x.shape
    return x.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def avgpool2_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) / 4.0


def _up1d(x, axis):
    """Bilinear x 2 along one axis, half-pixel centres, edge repeated:
    out[2i] = 3/4 x[i] + 1/4 x[i-1], out[2i+1] = 3/4 x[i] + 1/4 x[i+1]."""
    n = x.shape[axis]
    idx = np.arange(n)
    prev = np.take(x, np.maximum(idx - 1, 0), axis=axis)
    nxt = np.take(x, np.minimum(idx + 1, n - 1), axis=axis)
    even = 0.75 * x + 0.25 * prev
    odd = 0.75 * x + 0.25 * nxt
    out = np.stack([even, odd], axis=axis + 1)
    shape = list(x.shape)
    shape[axis] = 2 * n
    return out.reshape(shape)


def upsample2(x):
    return _up1d(_up1d(x, 1), 2)


def _up1d_backward(g, axis):
    """Transpose of _up1d along `axis`."""
    g = np.moveaxis(g, axis, 0)
    ge, go = g[0::2], g[1::2]
    n = ge.shape[0]
    gx = 0.75 * (ge + go)
    idx = np.arange(n)
    np.add.at(gx, np.maximum(idx - 1, 0), 0.25 * ge)
    np.add.at(gx, np.minimum(idx + 1, n - 1), 0.25 * go)
    return np.moveaxis(gx, 0, axis)


def upsample2_backward(g):
    return _up1d_backward(_up1d_backward(g, 2), 1)


# --------------------------------------------------------------- network

def round_bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as FP64."""
    f = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    f = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, div, flags, keep=False, act_round=None):
    """phi_hat = network([div_s, flags]) for one grid (H, W divisible by 4);
    the architecture is the one the parameters have.

    div_s is the already scaled divergence (the caller divides by s and
    multiplies the output by s).  With keep=True returns (out, tape) for
    backward.  act_round (e.g. round_bf16) is applied to every branch input
    and to every activation that feeds another convolution, to model a
    reduced-precision storage of activations; the arithmetic stays FP64."""
    rnd = act_round if act_round is not None else (lambda a: a)
    x0 = np.stack([np.asarray(div, np.float64), (np.asarray(flags) != 0).astype(np.float64)])
    if arch_of(params) == "unet":
        out, tape = _forward_unet(params, x0, rnd)
        return (out, tape) if keep else out
    xin = {1: x0, 2: avgpool2(x0)}
    xin[4] = avgpool2(xin[2])
    tape = []
    p = iter(params)
    prev = None
    for sc, widths in ARCHS[arch_of(params)]:
        h = xin[sc] if prev is None else np.concatenate([xin[sc], upsample2(prev)], axis=0)
        h = rnd(h)
        nl = len(widths) - 1
        for l in range(nl):
            w, b = next(p)
            pre = conv3x3(h, w, b)
            out = np.maximum(pre, 0.0) if relu_after(l, nl) else pre
            tape.append((sc, l, h, pre))
            h = rnd(out) if l < nl - 1 else out
        prev = h
    return (prev[0], tape) if keep else prev[0]


def _forward_unet(params, x0, rnd):
    """The Unet of the reading above on x0 = [div_s, flags] (H, W divisible by
    16); rnd models the storage rounding of every stored activation.  Returns
    (output, tape): per layer its input and pre-activation, and the skip
    features (the inputs of the max poolings)."""
    nl = len(params)
    it = iter(enumerate(params))
    convs = []

    def conv(h):
        l, (w, b) = next(it)
        pre = conv1x1(h, w, b) if w.shape[2] == 1 else conv3x3(h, w, b)
        convs.append((h, pre))
        out = np.maximum(pre, 0.0) if relu_after(l, nl) else pre
        return rnd(out) if l < nl - 1 else out

    h = rnd(x0)
    skips = []
    for level in range(4):
        if level > 0:
            h = maxpool2(h)
        h = conv(conv(h))
        skips.append(h)
    h = conv(conv(conv(maxpool2(h))))
    for level in (3, 2, 1, 0):
        h = conv(conv(np.concatenate([rnd(upsample2(h)), skips[level]], axis=0)))
    out = conv(h)[0]
    return out, {"unet": True, "convs": convs, "skips": skips}


def maxpool2_backward(x, g):
    """Transpose of maxpool2 at x: each gradient goes to the first maximum of
    its window in the order (0, 0), (0, 1), (1, 0), (1, 1)."""
    gx = np.zeros_like(x)
    m = maxpool2(x)
    taken = np.zeros(m.shape, bool)
    for dy in (0, 1):
        for dx in (0, 1):
            hit = (x[:, dy::2, dx::2] == m) & ~taken
            gx[:, dy::2, dx::2] = np.where(hit, g, 0.0)
            taken |= hit
    return gx


def conv1x1_backward(x, w, gy):
    """(gx, gw, gb) of conv1x1."""
    gx = np.einsum("oi,ohw->ihw", w[:, :, 0, 0], gy)
    gw = np.einsum("ohw,ihw->oi", gy, x)[:, :, None, None]
    return gx, gw, gy.sum(axis=(1, 2))


def _backward_unet(params, tape, g_out):
    """Gradients of the Unet's output w.r.t. every parameter (the forward's
    rounding taken as the identity, as for the other networks)."""
    nl = len(params)
    convs, skips = tape["convs"], tape["skips"]
    grads = [None] * nl
    state = {"l": nl - 1}

    def conv_back(g):
        l = state["l"]
        h, pre = convs[l]
        if relu_after(l, nl):
            g = g * (pre > 0)
        w = params[l][0]
        gx, gw, gb = conv1x1_backward(h, w, g) if w.shape[2] == 1 else conv3x3_backward(h, w, g)
        grads[l] = (gw, gb)
        state["l"] = l - 1
        return gx

    g = conv_back(g_out[None].astype(np.float64))
    g_skip = [None] * 4
    for level in (0, 1, 2, 3):
        g_cat = conv_back(conv_back(g))
        g_skip[level] = g_cat[32:]
        g = upsample2_backward(g_cat[:32])
    g = conv_back(conv_back(conv_back(g)))  # bottom, down to the pooled skip 3
    for level in (3, 2, 1, 0):
        g = g_skip[level] + maxpool2_backward(skips[level], g)
        g = conv_back(conv_back(g))
    return grads


def flatten(params):
    """Flat FP32-order vector: per layer weights [cout][cin][3][3], then bias."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def unflatten(flat, arch="multiscale"):
    out, k = [], 0
    for _, _, ws, bs in param_shapes(arch):
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append((np.asarray(flat[k:k + nw], np.float64).reshape(ws),
                    np.asarray(flat[k + nw:k + nw + nb], np.float64)))
        k += nw + nb
    return out


def backward(params, tape, g_out):
    """Gradients of the network output (given dL/dphi_hat) w.r.t. every
    parameter, as a list aligned with params: [(gw, gb), ...]."""
    if isinstance(tape, dict) and tape.get("unet"):
        return _backward_unet(params, tape, g_out)
    grads = [None] * len(params)
    g = g_out[None].astype(np.float64)
    idx = len(params) - 1
    g_prev_up = None
    branches = ARCHS[arch_of(params)]
    for k in reversed(range(len(branches))):
        nl = len(branches[k][1]) - 1
        if g_prev_up is not None:
            g = g_prev_up
        for l in reversed(range(nl)):
            _, _, h, pre = tape[idx]
            if relu_after(l, nl):
                g = g * (pre > 0)
            gx, gw, gb = conv3x3_backward(h, params[idx][0], g)
            grads[idx] = (gw, gb)
            g = gx
            idx -= 1
        # g is the gradient of this branch's input [x_sc(, upsampled coarser)]
        g_prev_up = upsample2_backward(g[2:3]) if k > 0 else None
    return grads
