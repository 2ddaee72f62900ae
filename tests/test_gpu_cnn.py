"""MultiScale CNN forward (hp_cnn_forward) and the hybrid projection
(hp_project_hybrid) against the FP64 oracle.

The oracle network runs in FP64 from the same BF16-rounded weights, with its
activations rounded to BF16 where the GPU stores them (branch inputs and every
activation that feeds another convolution).  Bar for the network output:
|phi_hat_gpu - phi_hat| <= 2e-2 * max|phi_hat| (FP32 accumulation order flips
BF16 roundings, which then propagate through up to 7 layers).  The hybrid
projection is compared with the oracle projection started from the GPU's
own guess (bit-identical FP32 phi_0), under the usual projection bars."""
import numpy as np
import pytest

import oracle
from oracle import cnn as C
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


def random_params(seed):
    rng = np.random.default_rng(seed)
    params = C.init_params(seed=seed)
    return [(w, 0.05 * rng.standard_normal(b.shape)) for w, b in params]


def bf16_weights(params):
    return [(C.round_bf16(w), b.astype(np.float32).astype(np.float64)) for w, b in params]


def case(B, n, seed):
    us, vs, fs = [], [], []
    for b in range(B):
        u, v = W.vortex_velocity(n, n, 40 + seed + b, n_vortices=8, width=(n / 32, n / 8))
        fs.append(W.random_obstacles(n, n, 50 + seed + b, rect_side=(n / 16, n / 4),
                                     disc_radius=(n / 32, n / 8)))
        us.append(u); vs.append(v)
    return (np.stack(us).astype(np.float32), np.stack(vs).astype(np.float32), np.stack(fs))


@pytest.mark.parametrize("B,n", [(2, 64), (1, 128)])
def test_cnn_forward_matches_oracle(dev, B, n):
    params = random_params(3)
    flat = C.flatten(params)
    u, v, fl = case(B, n, 1)
    cnn = hp.CNN(B, n, n, params=flat)
    ud, vd, fd = (torch.from_numpy(a).to(dev) for a in (u, v, fl))
    div = hp.hp_divergence(ud, vd, fd)
    phi_hat, s = hp.hp_cnn_forward(cnn, div, fd)
    torch.cuda.synchronize()
    cnn.check()  # no tensor-core wait gave up
    pw = bf16_weights(params)
    for b in range(B):
        d = div[b].cpu().numpy().astype(np.float64)
        sb = float(s[b].cpu())
        fluid = fl[b] == 0
        s_ref = np.abs(d[fluid]).mean()
        assert np.isclose(sb, s_ref, rtol=1e-6)
        ref = C.forward(pw, d / sb, fl[b], act_round=C.round_bf16)
        got = phi_hat[b].cpu().numpy()
        assert np.abs(got - ref).max() <= 2e-2 * np.abs(ref).max(), np.abs(got - ref).max()


def test_hybrid_projection_matches_oracle_from_the_same_guess(dev):
    B, n, thr, cap = 2, 64, 1e-3, 3000
    params = random_params(5)
    u, v, fl = case(B, n, 7)
    cnn = hp.CNN(B, n, n, params=C.flatten(params))
    ctx = hp.Context(B, n, n)
    ud, vd, fd = (torch.from_numpy(a).to(dev) for a in (u, v, fl))
    div = hp.hp_divergence(ud, vd, fd)
    phi_hat, s = hp.hp_cnn_forward(cnn, div, fd)
    phi0 = (phi_hat.cpu().numpy() * s.cpu().numpy()[:, None, None]).astype(np.float32)
    out = hp.hp_project_hybrid(ctx, cnn, ud, vd, fd, hp.ProjectParams(threshold=thr, max_iters=cap))
    torch.cuda.synchronize()
    ref = oracle.project(u.astype(np.float64), v.astype(np.float64), fl, thr, cap,
                         phi0=phi0.astype(np.float64), hist_len=cap + 2)
    gi = out["iters"].cpu().numpy()
    for b in range(B):
        if gi[b] != ref["iters"][b]:
            eh = ref["e_hist"][b]
            lo, hi = sorted((int(gi[b]), int(ref["iters"][b])))
            assert np.all(np.abs(eh[lo:hi + 1] - thr) / thr <= 5e-5)
        else:
            gu = ud.cpu().numpy()[b]
            umax = np.abs(ref["u"][b]).max()
            assert np.abs(gu - ref["u"][b]).max() <= 1e-5 * umax
    # the guess enters: E_0 of the hybrid equals the oracle's E(phi_0)
    e0 = oracle.mean_abs_residual(phi0.astype(np.float64) * (oracle.face_mask(fl) > 0),
                                  oracle.divergence(*oracle.zero_closed_faces(
                                      u.astype(np.float64), v.astype(np.float64), fl), fl), fl)
    assert np.allclose(ref["e_hist"][:, 0], e0, rtol=1e-12)
