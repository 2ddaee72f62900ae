"""Full-size workload checks beyond the benchmark grids.

1. An 8-step rollout of fixed-count projections (k = 20) on 8 grids of 256^2
   with obstacles: the loss sums mean(div(u_t)^2) and 0.1 * mean((p_t -
   p_ref_t)^2) over the steps, with a fixed forcing added to the projected
   velocity between steps.  Gradients w.r.t. the initial velocity and every
   step's initial guess phi_0 (what a network would output) come from
   torch.autograd chaining the library's adjoint eight times; they are
   compared with the same chain composed by hand from the FP64 oracle's
   forward and adjoint (the oracle adjoint is pinned by central differences
   and the dense Jacobian in the oracle tests).
2. The 1024^2 plume with a solid disc of radius 64 centred 256 cells above a
   128-cell inlet: three driver steps teacher-forced against the oracle
   (advection and projection at E_t = 1e-8; at the raw E_t = 1e-3 this plume
   needs no sweeps), then one hybrid projection from a randomly initialised
   network's guess against the oracle projection from the same guess.
3. The 2048^2 plume with 8 random discs: two driver steps
   teacher-forced, then a hybrid projection with the Unet from its guess."""
import numpy as np
import pytest

import oracle
from oracle import adjoint as AD
from oracle import advect as A
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


def div_t(u, v):
    """Forward-difference divergence of every cell (closed faces are zero
    after a projection, so this equals the masked divergence)."""
    return (u[:, :, 1:] - u[:, :, :-1]) + (v[:, 1:, :] - v[:, :-1, :])


def div_np(u, v):
    return (u[:, :, 1:] - u[:, :, :-1]) + (v[:, 1:, :] - v[:, :-1, :])


def div_adjoint_np(g, shape_u, shape_v):
    """Transpose of div_np applied to a cell field g."""
    gu = np.zeros(shape_u)
    gv = np.zeros(shape_v)
    gu[:, :, 1:] += g
    gu[:, :, :-1] -= g
    gv[:, 1:, :] += g
    gv[:, :-1, :] -= g
    return gu, gv


def test_rollout_gradient_8_steps_256(dev):
    from paper_2109_09363_gb300.autograd import project_fixed
    B, n, k, steps, dt, rho0 = 8, 256, 20, 8, 0.1, 1.0
    u64, v64, fl = W.batched_vortex_case(B, n, seed0=300, n_vortices=16)
    rng = np.random.default_rng(11)
    fu = [0.01 * rng.standard_normal(u64.shape) for _ in range(steps)]
    fv = [0.01 * rng.standard_normal(v64.shape) for _ in range(steps)]
    phi0 = [0.1 * rng.standard_normal((B, n, n)) for _ in range(steps)]
    pref = [0.1 * rng.standard_normal((B, n, n)) for _ in range(steps)]
    cells = B * n * n

    # GPU: autograd through the library's forward and adjoint
    ctx = hp.Context(B, n, n)
    f32 = lambda a: torch.from_numpy(np.asarray(a, np.float32)).to(dev)
    u0 = f32(u64).requires_grad_()
    v0 = f32(v64).requires_grad_()
    g_phi = [f32(p).requires_grad_() for p in phi0]
    fd = torch.from_numpy(fl).to(dev)
    us, vs = u0, v0
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    for t in range(steps):
        uo, vo, po = project_fixed(us, vs, g_phi[t], fd, ctx, k, dt, rho0)
        d = div_t(uo, vo)
        loss = loss + (d.double() ** 2).sum() / cells + \
            0.1 * ((po.double() - f32(pref[t]).double()) ** 2).sum() / cells
        us, vs = uo + f32(fu[t]), vo + f32(fv[t])
    loss.backward()

    # oracle: the same chain in FP64, backward composed by hand
    su, sv = [], []
    out = []
    cu, cv = u64.copy(), v64.copy()
    L = 0.0
    for t in range(steps):
        su.append(cu); sv.append(cv)
        ou, ov, op = AD.project_fixed(cu, cv, phi0[t].astype(np.float32).astype(np.float64),
                                      fl, k, dt, rho0)
        out.append((ou, ov, op))
        dd = div_np(ou, ov)
        L += (dd ** 2).sum() / cells + 0.1 * ((op - pref[t].astype(np.float32)) ** 2).sum() / cells
        cu, cv = ou + fu[t].astype(np.float32), ov + fv[t].astype(np.float32)
    assert np.isclose(float(loss.item()), L, rtol=1e-5)
    gu_next = np.zeros(u64.shape)
    gv_next = np.zeros(v64.shape)
    g_phi_ref = [None] * steps
    for t in reversed(range(steps)):
        ou, ov, op = out[t]
        gdu, gdv = div_adjoint_np(2.0 * div_np(ou, ov) / cells, u64.shape, v64.shape)
        gu = gdu + gu_next
        gv = gdv + gv_next
        gp = 0.2 * (op - pref[t].astype(np.float32)) / cells
        gu_star, gv_star, gphi = AD.project_fixed_adjoint(gu, gv, gp, fl, k, dt, rho0)
        g_phi_ref[t] = gphi
        gu_next, gv_next = gu_star, gv_star

    # FP32 sweeps chained over 8 steps: 5e-5 of the largest entry
    def close(got, exp):
        g = got.detach().cpu().numpy().astype(np.float64)
        scale = max(np.abs(exp).max(), 1e-30)
        return np.abs(g - exp).max() <= 5e-5 * scale, np.abs(g - exp).max() / scale

    ok, err = close(u0.grad, gu_next)
    assert ok, err
    ok, err = close(v0.grad, gv_next)
    assert ok, err
    for t in range(steps):
        ok, err = close(g_phi[t].grad, g_phi_ref[t])
        assert ok, (t, err)


def test_plume_1024_cylinder_and_hybrid_step(dev):
    from paper_2109_09363_gb300.plume import Plume, PlumeConfig
    n, thr, cap, tol = 1024, 1e-8, 1500, 1e-5
    u0, v0, rho0 = W.plume_initial_state(n, seed=0)
    fl = W.plume_flags(n, cylinder_radius=64, cylinder_height=256)[None]
    x0, x1 = W.inlet_columns(n)
    assert (x0, x1) == (448, 576)
    cfg = PlumeConfig(ny=n, nx=n, dt=0.1, inlet=(x0, x1), threshold=thr, max_iters=cap)
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sim = Plume(cfg, t32(u0[None].astype(np.float32)), t32(v0[None].astype(np.float32)),
                t32(rho0[None].astype(np.float32)), t32(fl))
    oracle.set_threads(0)
    swept = 0
    for step in range(3):
        su, sv, sr = (x.cpu().numpy()[0].astype(np.float64) for x in (sim.u, sim.v, sim.rho))
        sim.advect()
        eu, ev, er = A.advect_step(su, sv, sr, fl[0], cfg.dt, inlet=(x0, x1))
        gu, gv, gr = (x.cpu().numpy()[0] for x in (sim.u, sim.v, sim.rho))
        umax = max(np.abs(eu).max(), np.abs(ev).max(), 1e-30)
        assert np.abs(gu - eu).max() <= tol * umax, step
        assert np.abs(gv - ev).max() <= tol * umax, step
        assert np.abs(gr - er).max() <= tol * np.abs(er).max(), step
        ustar = (gu.astype(np.float64), gv.astype(np.float64))
        out = sim.project()
        torch.cuda.synchronize()
        kg = int(out["iters"].cpu()[0])
        swept += kg
        ref = oracle.project(ustar[0][None], ustar[1][None], fl, thr, cap, dt=cfg.dt,
                             hist_len=cap + 2)
        ko = int(ref["iters"][0])
        if kg != ko:
            eh = ref["e_hist"][0]
            lo, hi = sorted((kg, ko))
            seg = eh[lo:hi + 1]
            seg = seg[np.isfinite(seg)]  # the oracle's history ends at its own stop
            assert seg.size and np.all(np.abs(seg - thr) / thr <= 5e-5), (step, kg, ko)
            ref = oracle.project(ustar[0][None], ustar[1][None], fl, thr, cap, dt=cfg.dt,
                                 fixed_iters=kg)
        pu, pv = sim.u.cpu().numpy()[0], sim.v.cpu().numpy()[0]
        umax = max(np.abs(ref["u"]).max(), np.abs(ref["v"]).max(), 1e-30)
        assert np.abs(pu - ref["u"][0]).max() <= tol * umax, step
        assert np.abs(pv - ref["v"][0]).max() <= tol * umax, step
    assert swept > 0

    # one hybrid projection of the next u* from a random network's guess
    sim.advect()
    us, vs = sim.u.clone(), sim.v.clone()
    ctx = hp.Context(1, n, n)
    cnn = hp.CNN(1, n, n, params=C.flatten(C.init_params(seed=3)))
    fd = t32(fl)
    div = hp.hp_divergence(us, vs, fd)
    phi_hat, s = hp.hp_cnn_forward(cnn, div, fd)
    phi0 = (phi_hat.cpu().numpy() * s.cpu().numpy()[:, None, None]).astype(np.float64)
    assert np.all(np.isfinite(phi0))
    uh, vh = us.clone(), vs.clone()
    out = hp.hp_project_hybrid(ctx, cnn, uh, vh, fd, hp.ProjectParams(
        threshold=thr, max_iters=cap, dt=cfg.dt))
    torch.cuda.synchronize()
    ref = oracle.project(us.cpu().numpy().astype(np.float64), vs.cpu().numpy().astype(np.float64),
                         fl, thr, cap, dt=cfg.dt, phi0=phi0, hist_len=cap + 2)
    kg, ko = int(out["iters"].cpu()[0]), int(ref["iters"][0])
    if kg != ko:
        eh = ref["e_hist"][0]
        lo, hi = sorted((kg, ko))
        seg = eh[lo:hi + 1]
        seg = seg[np.isfinite(seg)]  # the oracle's history ends at its own stop
        assert seg.size and np.all(np.abs(seg - thr) / thr <= 5e-5), (kg, ko)
    else:
        umax = max(np.abs(ref["u"]).max(), np.abs(ref["v"]).max(), 1e-30)
        assert np.abs(uh.cpu().numpy()[0] - ref["u"][0]).max() <= tol * umax
        assert np.abs(vh.cpu().numpy()[0] - ref["v"][0]).max() <= tol * umax


def test_plume_2048_eight_cylinders_and_unet_hybrid(dev):
    """The large evaluation geometry at its size: the 2048^2 plume (inlet
    256 cells) with 8 non-overlapping discs of radius U(32, 128), two driver
    steps teacher-forced against the oracle (the temporally blocked sweeps
    serve grids of this size), then one hybrid projection with the Unet from
    its own guess against the oracle projection from the same guess."""
    from paper_2109_09363_gb300.plume import Plume, PlumeConfig
    n, thr, cap, tol = 2048, 1e-10, 800, 1e-5
    u0, v0, rho0 = W.plume_initial_state(n, seed=5)
    x0, x1 = W.inlet_columns(n)
    fl = W.random_cylinders(n, 8, 5, radius=(32, 128), inlet=(x0, x1))[None]
    cfg = PlumeConfig(ny=n, nx=n, dt=0.1, inlet=(x0, x1), threshold=thr, max_iters=cap)
    t32 = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    sim = Plume(cfg, t32(u0[None].astype(np.float32)), t32(v0[None].astype(np.float32)),
                t32(rho0[None].astype(np.float32)), t32(fl))
    oracle.set_threads(0)

    def check(ustar, kg, pu, pv, phi0=None):
        ref = oracle.project(ustar[0][None], ustar[1][None], fl, thr, cap, dt=cfg.dt,
                             phi0=phi0, hist_len=cap + 2)
        ko = int(ref["iters"][0])
        if kg != ko:
            eh = ref["e_hist"][0]
            lo, hi = sorted((kg, ko))
            seg = eh[lo:hi + 1]
            seg = seg[np.isfinite(seg)]  # the oracle's history ends at its own stop
            assert seg.size and np.all(np.abs(seg - thr) / thr <= 5e-5), (kg, ko)
            ref = oracle.project(ustar[0][None], ustar[1][None], fl, thr, cap, dt=cfg.dt,
                                 phi0=phi0, fixed_iters=kg)
        umax = max(np.abs(ref["u"]).max(), np.abs(ref["v"]).max(), 1e-30)
        assert np.abs(pu - ref["u"][0]).max() <= tol * umax
        assert np.abs(pv - ref["v"][0]).max() <= tol * umax

    for step in range(2):
        su, sv, sr = (x.cpu().numpy()[0].astype(np.float64) for x in (sim.u, sim.v, sim.rho))
        sim.advect()
        eu, ev, er = A.advect_step(su, sv, sr, fl[0], cfg.dt, inlet=(x0, x1))
        gu, gv, gr = (x.cpu().numpy()[0] for x in (sim.u, sim.v, sim.rho))
        umax = max(np.abs(eu).max(), np.abs(ev).max(), 1e-30)
        assert np.abs(gu - eu).max() <= tol * umax, step
        assert np.abs(gv - ev).max() <= tol * umax, step
        assert np.abs(gr - er).max() <= tol * np.abs(er).max(), step
        ustar = (gu.astype(np.float64), gv.astype(np.float64))
        out = sim.project()
        torch.cuda.synchronize()
        check(ustar, int(out["iters"].cpu()[0]), sim.u.cpu().numpy()[0], sim.v.cpu().numpy()[0])
        assert hp.hp_resident_clusters(sim.ctx, 1, n, n) == 0   # the blocked kernel ran

    sim.advect()
    us, vs = sim.u.clone(), sim.v.clone()
    ctx = hp.Context(1, n, n)
    cnn = hp.CNN(1, n, n, params=C.flatten(C.init_params(seed=8, arch="unet")), arch="unet")
    fd = t32(fl)
    div = hp.hp_divergence(us, vs, fd)
    phi_hat, s = hp.hp_cnn_forward(cnn, div, fd)
    phi0 = (phi_hat.cpu().numpy() * s.cpu().numpy()[:, None, None]).astype(np.float64)
    assert np.all(np.isfinite(phi0))
    uh, vh = us.clone(), vs.clone()
    out = hp.hp_project_hybrid(ctx, cnn, uh, vh, fd, hp.ProjectParams(
        threshold=thr, max_iters=cap, dt=cfg.dt))
    torch.cuda.synchronize()
    assert cnn.check() == 0
    check((us.cpu().numpy()[0].astype(np.float64), vs.cpu().numpy()[0].astype(np.float64)),
          int(out["iters"].cpu()[0]), uh.cpu().numpy()[0], vh.cpu().numpy()[0], phi0=phi0)
    ctx.check()
