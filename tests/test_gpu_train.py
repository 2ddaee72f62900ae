"""Training of the MultiScale CNN: the GPU gradient (hand-written backward
kernels) against the FP64 oracle backward, and what training gains: the
hybrid projection with the trained network needs fewer Jacobi sweeps than
plain Jacobi at the same threshold on held-out grids."""
import numpy as np
import pytest

import oracle
from oracle import cnn as C
from oracle import train as TR
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
    oracle.build()
    return torch.device("cuda:0")


def oracle_gradient(params, phi_gpu, div, fl, tgt, s, lam, act_round):
    """Oracle gradient of the batch loss, the loss gradient taken at the GPU's
    own output phi_gpu (isolates the backward kernels from forward rounding)."""
    B = div.shape[0]
    pw = [(C.round_bf16(w), b.astype(np.float32).astype(np.float64)) for w, b in params]
    total = [(np.zeros_like(w), np.zeros_like(b)) for w, b in pw]
    L = 0.0
    for b in range(B):
        d = div[b].astype(np.float64)
        _, tape = C.forward(pw, d / s[b], fl[b], keep=True, act_round=act_round)
        lb, gphi = TR.loss_and_grad(phi_gpu[b], tgt[b], d, fl[b], s[b], lam)
        L += lb / B
        gr = C.backward(pw, tape, gphi / B)
        total = [(tw + gw, tb + gb) for (tw, tb), (gw, gb) in zip(total, gr)]
    return L, total


@pytest.mark.parametrize("lam", [0.0, 1.0])
def test_gradient_matches_oracle_backward(dev, lam):
    B, n = 2, 32
    rng = np.random.default_rng(0)
    params = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in C.init_params(seed=11)]
    u, v, fl = W.training_case(B, n, 100)
    ud = torch.from_numpy(u.astype(np.float32)).to(dev)
    vd = torch.from_numpy(v.astype(np.float32)).to(dev)
    fd = torch.from_numpy(fl).to(dev)
    div = hp.hp_divergence(ud, vd, fd)
    tgt = torch.from_numpy(rng.standard_normal((B, n, n)).astype(np.float32)).to(dev)
    cnn = hp.CNN(B, n, n, params=C.flatten(params))
    tr = hp.Trainer(cnn, B, n, n)
    g, loss = tr.gradient(div, fd, tgt, lambda_div=lam)
    phi_gpu, s = hp.hp_cnn_forward(cnn, div, fd)
    torch.cuda.synchronize()
    args = (phi_gpu.cpu().numpy(), div.cpu().numpy(), fl, tgt.cpu().numpy(),
            [float(x) for x in s.cpu()], lam)
    L, ref = oracle_gradient(params, *args, act_round=C.round_bf16)
    assert np.isclose(float(loss.item()), L, rtol=1e-4)
    # sensitivity of the gradient to the BF16 storage of activations
    _, ref64 = oracle_gradient(params, *args, act_round=None)
    flat = g.cpu().numpy()
    k = 0
    for (w, b), (w64, b64) in zip(ref, ref64):
        nw, nb = w.size, b.size
        gw, gb = flat[k:k + nw], flat[k + nw:k + nw + nb]
        scale = max(np.abs(w).max(), np.abs(b).max())
        sens = max(np.abs(w - w64).max(), np.abs(b - b64).max())
        bar = max(5e-2 * scale, 3.0 * sens) + 1e-9
        assert np.abs(gw - w.ravel()).max() <= bar, (k, np.abs(gw - w.ravel()).max(), scale, sens)
        assert np.abs(gb - b.ravel()).max() <= bar
        k += nw + nb


@pytest.mark.parametrize("B,ny,nx", [(2, 128, 128), (1, 64, 160)])
def test_tensor_core_backward_matches_oracle(dev, B, ny, nx):
    """Sizes where every branch is at least 32 pixels wide, so that every
    32/64-channel layer takes the tensor-core backward (BF16 gradients, the
    replicated-border terms added separately); 160 = one full and one partial
    128-pixel segment."""
    rng = np.random.default_rng(B + nx)
    params = [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in C.init_params(seed=13)]
    u, v, fl = W.training_case(1, max(ny, nx), 700)
    u, v, fl = u[:, :ny, :nx + 1], v[:, :ny + 1, :nx], fl[:, :ny, :nx]
    u, v, fl = np.repeat(u, B, 0), np.repeat(v, B, 0), np.ascontiguousarray(np.repeat(fl, B, 0))
    if B > 1:  # a different field on the second grid
        u[1] = np.roll(u[1], 17, axis=1)
        v[1] = np.roll(v[1], 29, axis=0)
    ud = torch.from_numpy(np.ascontiguousarray(u, np.float32)).to(dev)
    vd = torch.from_numpy(np.ascontiguousarray(v, np.float32)).to(dev)
    fd = torch.from_numpy(fl).to(dev)
    div = hp.hp_divergence(ud, vd, fd)
    tgt = torch.from_numpy(rng.standard_normal((B, ny, nx)).astype(np.float32)).to(dev)
    cnn = hp.CNN(B, ny, nx, params=C.flatten(params))
    tr = hp.Trainer(cnn, B, ny, nx)
    lam = 1.0
    g, loss = tr.gradient(div, fd, tgt, lambda_div=lam)
    phi_gpu, s = hp.hp_cnn_forward(cnn, div, fd)
    torch.cuda.synchronize()
    args = (phi_gpu.cpu().numpy(), div.cpu().numpy(), fl, tgt.cpu().numpy(),
            [float(x) for x in s.cpu()], lam)
    L, ref = oracle_gradient(params, *args, act_round=C.round_bf16)
    assert np.isclose(float(loss.item()), L, rtol=1e-4)
    _, ref64 = oracle_gradient(params, *args, act_round=None)
    flat = g.cpu().numpy()
    k = 0
    for (w, b), (w64, b64) in zip(ref, ref64):
        nw, nb = w.size, b.size
        gw, gb = flat[k:k + nw], flat[k + nw:k + nw + nb]
        scale = max(np.abs(w).max(), np.abs(b).max())
        sens = max(np.abs(w - w64).max(), np.abs(b - b64).max())
        bar = max(5e-2 * scale, 3.0 * sens) + 1e-9
        assert np.abs(gw - w.ravel()).max() <= bar, (k, np.abs(gw - w.ravel()).max(), scale, sens)
        assert np.abs(gb - b.ravel()).max() <= bar, (k, np.abs(gb - b.ravel()).max(), scale)
        k += nw + nb


def test_training_reduces_loss_and_jacobi_sweeps(dev):
    from paper_2109_09363_gb300 import training as T
    n = 64
    data = T.generate_pairs(1024, n, seed0=0, sweeps=16000, device=dev)
    cnn = hp.CNN(64, n, n, params=C.flatten(C.init_params(seed=1)))
    losses = T.train(cnn, data, epochs=30, batch=64, lr=1e-3, lambda_div=1.0)
    assert np.mean(losses[-10:]) < 0.5 * np.mean(losses[:10])
    # held-out grids: hybrid vs plain at the same threshold
    u, v, fl = W.training_case(32, n, 50000)
    thr, cap = 1e-3, 4000
    ctx = hp.Context(32, n, n)
    cnn_eval = hp.CNN(32, n, n, params=cnn.get_params())
    res = {}
    for mode in ("plain", "hybrid"):
        ud = torch.from_numpy(u.astype(np.float32)).to(dev)
        vd = torch.from_numpy(v.astype(np.float32)).to(dev)
        fd = torch.from_numpy(fl).to(dev)
        prm = hp.ProjectParams(threshold=thr, max_iters=cap)
        out = (hp.hp_project(ctx, ud, vd, fd, prm) if mode == "plain"
               else hp.hp_project_hybrid(ctx, cnn_eval, ud, vd, fd, prm))
        res[mode] = out["iters"].cpu().numpy()
    # measured: about 5x fewer sweeps at 1e-3 after this much training
    assert res["hybrid"].mean() < 0.5 * res["plain"].mean(), res
