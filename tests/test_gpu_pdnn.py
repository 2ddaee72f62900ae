"""Physics-driven training (Sec. 3.2, Eq. 4) on the GPU:
1. the gradient of the loss (hp_trainer_pdnn_gradient) against the FP64
   oracle loss (which corrects the velocity and takes its divergence) chained
   into the oracle backward of the network, for both norms and unequal grid
   weights; the loss gradient is taken at the GPU's own network output, as in
   the supervised training test;
2. the rollout of the training solver step by step against the oracle
   (teacher-forced: each step starts from the GPU's previous state);
3. training on the physics-driven loss lowers it;
4. argument checks of the new entry points."""
import numpy as np
import pytest

import oracle
from oracle import adjoint as AD
from oracle import advect as A
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


def t32(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev)


def oracle_pdnn_gradient(params, phi_gpu, u, v, fl, s, w, norm, act_round):
    """Oracle loss and parameter gradient at the GPU's network output."""
    pw = [(C.round_bf16(wt), b.astype(np.float32).astype(np.float64)) for wt, b in params]
    total = [(np.zeros_like(wt), np.zeros_like(b)) for wt, b in pw]
    L = 0.0
    for b in range(fl.shape[0]):
        d = oracle.divergence(u[b][None], v[b][None], fl[b][None])[0]
        _, tape = C.forward(pw, d / s[b], fl[b], keep=True, act_round=act_round)
        lb, gphi = TR.pdnn_loss_and_grad(phi_gpu[b], u[b], v[b], fl[b], s[b], w[b], norm)
        L += lb
        gr = C.backward(pw, tape, gphi)
        total = [(tw + gw, tb + gb) for (tw, tb), (gw, gb) in zip(total, gr)]
    return L, total


@pytest.mark.parametrize("norm", [1, 2])
def test_pdnn_gradient_matches_oracle_backward(dev, norm):
    B, n = 3, 32
    rng = np.random.default_rng(5 + norm)
    params = [(wt, 0.05 * rng.standard_normal(b.shape)) for wt, b in C.init_params(seed=12)]
    u, v, fl = W.training_case(B, n, 400)
    u = u.astype(np.float32).astype(np.float64)
    v = v.astype(np.float32).astype(np.float64)
    ud, vd, fd = t32(u, dev), t32(v, dev), torch.from_numpy(fl).to(dev)
    div = hp.hp_divergence(ud, vd, fd)
    w = np.array([0.5, 1.25, 2.0], np.float32)
    cnn = hp.CNN(B, n, n, params=C.flatten(params))
    tr = hp.Trainer(cnn, B, n, n)
    g, loss = tr.pdnn_gradient(div, fd, t32(w, dev), norm=norm)
    phi_gpu, s = hp.hp_cnn_forward(cnn, div, fd)
    torch.cuda.synchronize()
    args = (phi_gpu.cpu().numpy(), u, v, fl, [float(x) for x in s.cpu()],
            w.astype(np.float64), norm)
    L, ref = oracle_pdnn_gradient(params, *args, act_round=C.round_bf16)
    assert np.isclose(float(loss.item()), L, rtol=1e-5), (float(loss.item()), L)
    # sensitivity of the gradient to the BF16 storage of activations
    _, ref64 = oracle_pdnn_gradient(params, *args, act_round=None)
    flat = g.cpu().numpy()
    k = 0
    for (wr, br), (w64, b64) in zip(ref, ref64):
        nw, nb = wr.size, br.size
        gw, gb = flat[k:k + nw], flat[k + nw:k + nw + nb]
        scale = max(np.abs(wr).max(), np.abs(br).max())
        sens = max(np.abs(wr - w64).max(), np.abs(br - b64).max())
        bar = max(5e-2 * scale, 3.0 * sens) + 1e-9
        assert np.abs(gw - wr.ravel()).max() <= bar, (k, np.abs(gw - wr.ravel()).max(), scale)
        assert np.abs(gb - br.ravel()).max() <= bar
        k += nw + nb


def test_pdnn_rollout_matches_oracle_step_by_step(dev):
    from paper_2109_09363_gb300 import training as T
    B, n, steps, dt, tol = 2, 64, 3, 0.1, 1e-5
    u, v, fl = W.training_case(B, n, 500)
    ud, vd, fd = t32(u, dev), t32(v, dev), torch.from_numpy(fl).to(dev)
    cnn = hp.CNN(B, n, n, params=C.flatten(C.init_params(seed=4)))
    ctx = hp.Context(B, n, n)
    trace = []
    ul, vl = T.pdnn_rollout(cnn, ctx, ud, vd, fd, steps, dt, trace=trace)
    torch.cuda.synchronize()
    assert len(trace) == steps
    assert torch.equal(ud, t32(u, dev))  # inputs untouched
    for k, (us, vs, up, vp) in enumerate(trace):
        # projection from the network's guess (the network itself is checked
        # against the oracle in the CNN tests)
        div = hp.hp_divergence(us, vs, fd)
        phi_hat, s = hp.hp_cnn_forward(cnn, div, fd)
        phi0 = phi_hat.cpu().numpy().astype(np.float64) * s.cpu().numpy()[:, None, None]
        su, sv = us.cpu().numpy().astype(np.float64), vs.cpu().numpy().astype(np.float64)
        eu, ev, _ = AD.project_fixed(su, sv, phi0, fl, 0)
        umax = max(np.abs(eu).max(), np.abs(ev).max())
        assert np.abs(up.cpu().numpy() - eu).max() <= tol * umax, k
        assert np.abs(vp.cpu().numpy() - ev).max() <= tol * umax, k
        # advection without buoyancy, into the next step's input
        nu, nv = (trace[k + 1][0], trace[k + 1][1]) if k + 1 < steps else (ul, vl)
        for b in range(B):
            au, av, _ = A.advect_step(up.cpu().numpy()[b].astype(np.float64),
                                      vp.cpu().numpy()[b].astype(np.float64),
                                      np.ones((n, n)), fl[b], dt, gravity=0.0)
            amax = max(np.abs(au).max(), np.abs(av).max())
            assert np.abs(nu.cpu().numpy()[b] - au).max() <= tol * amax, (k, b)
            assert np.abs(nv.cpu().numpy()[b] - av).max() <= tol * amax, (k, b)


def test_pdnn_training_lowers_the_loss(dev):
    from paper_2109_09363_gb300 import training as T
    N, n, batch = 128, 64, 16
    u, v, fl = W.training_case(N, n, 600)
    data = (t32(u, dev), t32(v, dev), torch.from_numpy(fl).to(dev))
    cnn = hp.CNN(2 * batch, n, n, params=T.init_params(seed=2))
    losses, ns = T.train_pdnn(cnn, data, steps=150, batch=batch, lr=1e-3, norm=2, seed=1)
    assert set(ns) <= {4, 16}
    assert all(np.isfinite(losses))
    first, last = np.mean(losses[:10]), np.mean(losses[-10:])
    assert last < 0.5 * first, (first, last)


def test_pdnn_argument_checks(dev):
    B, n = 2, 32
    cnn = hp.CNN(B, n, n, params=C.flatten(C.init_params(seed=1)))
    with pytest.raises(hp.HprojError):
        hp.Trainer(cnn, B + 1, n, n)  # larger than the network's workspace
    tr = hp.Trainer(cnn, B, n, n)
    fd = torch.zeros((B, n, n), dtype=torch.uint8, device=dev)
    div = torch.zeros((B, n, n), dtype=torch.float32, device=dev)
    w = torch.ones(B, dtype=torch.float32, device=dev)
    for bad in (0, 3):
        with pytest.raises(hp.HprojError):
            tr.pdnn_gradient(div, fd, w, norm=bad)
    # zero divergence and a zero guess: zero loss, zero gradient
    cnn0 = hp.CNN(B, n, n, params=np.zeros(hp.CNN.param_count(), np.float32))
    tr0 = hp.Trainer(cnn0, B, n, n)
    g, loss = tr0.pdnn_gradient(div, fd, w, norm=1)
    torch.cuda.synchronize()
    assert float(loss.item()) == 0.0
    assert float(g.abs().max().item()) == 0.0
