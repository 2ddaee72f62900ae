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


def check_against_oracle(gi, gu, gv, ref, i, u, v, fl, thr, cap, phi0):
    """Grid i of an oracle result against the GPU's: the same iteration count,
    or a stop one side of a near tie (E within 5e-5 of E_t where both
    histories exist; the oracle's ends at its own stop), in which case the
    oracle is run again for exactly the GPU's count; then the corrected
    velocity within 1e-5 of the largest."""
    if gi != ref["iters"][i]:
        eh = ref["e_hist"][i]
        lo, hi = sorted((int(gi), int(ref["iters"][i])))
        seg = eh[lo:hi + 1]
        seg = seg[np.isfinite(seg)]
        assert seg.size >= 1 and np.all(np.abs(seg - thr) / thr <= 5e-5), (gi, ref["iters"][i])
        ref = oracle.project(u[None].astype(np.float64), v[None].astype(np.float64), fl[None],
                             0.0, 0, phi0=phi0[None].astype(np.float64), fixed_iters=int(gi))
        i = 0
    umax = max(np.abs(ref["u"][i]).max(), np.abs(ref["v"][i]).max())
    assert np.abs(gu - ref["u"][i]).max() <= 1e-5 * umax
    assert np.abs(gv - ref["v"][i]).max() <= 1e-5 * umax


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
    gu, gv = ud.cpu().numpy(), vd.cpu().numpy()
    for b in range(B):
        check_against_oracle(gi[b], gu[b], gv[b], ref, b, u[b], v[b], fl[b], thr, cap, phi0[b])
    # the guess enters: E_0 of the hybrid equals the oracle's E(phi_0)
    e0 = oracle.mean_abs_residual(phi0.astype(np.float64) * (oracle.face_mask(fl) > 0),
                                  oracle.divergence(*oracle.zero_closed_faces(
                                      u.astype(np.float64), v.astype(np.float64), fl), fl), fl)
    assert np.allclose(ref["e_hist"][:, 0], e0, rtol=1e-12)


def test_hybrid_projection_at_the_benchmark_size_sampled(dev):
    """The hybrid projection on the benchmark's batch (16 x 512^2 vortex
    grids with obstacles, E_t = 1e-4, cap 5000) with a MultiScale of random
    weights; four grids checked in full against the oracle projection from
    the same FP32 guess (iteration counts, or a near tie at E_t, and the
    corrected velocity)."""
    B, n, thr, cap = 16, 512, 1e-4, 5000
    u64, v64, fl = W.batched_vortex_case(B, n)
    u, v = u64.astype(np.float32), v64.astype(np.float32)
    cnn = hp.CNN(B, n, n, params=C.flatten(random_params(11)))
    ctx = hp.Context(B, n, n)
    ud, vd, fd = (torch.from_numpy(a).to(dev) for a in (u, v, fl))
    div = hp.hp_divergence(ud, vd, fd)
    phi_hat, s = hp.hp_cnn_forward(cnn, div, fd)
    phi0 = (phi_hat.cpu().numpy() * s.cpu().numpy()[:, None, None]).astype(np.float32)
    out = hp.hp_project_hybrid(ctx, cnn, ud, vd, fd, hp.ProjectParams(threshold=thr, max_iters=cap))
    torch.cuda.synchronize()
    assert cnn.check() == 0
    gi = out["iters"].cpu().numpy()
    gu, gv = ud.cpu().numpy(), vd.cpu().numpy()
    oracle.set_threads(0)
    sample = [0, 6, 11, 15]
    ref = oracle.project(u[sample].astype(np.float64), v[sample].astype(np.float64), fl[sample],
                         thr, cap, phi0=phi0[sample].astype(np.float64), hist_len=cap + 2)
    for i, b in enumerate(sample):
        check_against_oracle(gi[b], gu[b], gv[b], ref, i, u[b], v[b], fl[b], thr, cap, phi0[b])
