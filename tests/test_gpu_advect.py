"""GPU parity of the plume driver step (hp_advect_step) and of the plume
loop (advect + project, configuration: 128^2 closed box, 16-cell inlet with
rho = 1.1, g = -0.002, dt = 0.1, 50 steps) against the FP64 oracle, with the
oracle restarted from the GPU state every step (teacher forcing)."""
import numpy as np
import pytest

import oracle
from oracle import advect as A
from paper_2109_09363_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hp = pytest.importorskip("paper_2109_09363_gb300")

TOL = 1e-5  # relative to the field's max, per face / cell


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09363_gb300 import build
    build.build()
    oracle.build()
    return torch.device("cuda:0")


def t(a, dev):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


@pytest.mark.parametrize("shape,dt", [((1, 16, 16), 0.1), ((2, 67, 130), 0.5), ((1, 128, 96), 2.5)])
def test_advect_step_matches_oracle(dev, shape, dt):
    B, ny, nx = shape
    rng = np.random.default_rng(ny + nx)
    us, vs, rs, fs = [], [], [], []
    for b in range(B):
        u, v = W.vortex_velocity(ny, nx, 7 + b, n_vortices=6, width=(3, 12))
        us.append(u); vs.append(v)
        rs.append(1.0 + 0.05 * rng.standard_normal((ny, nx)))
        fs.append(W.random_obstacles(ny, nx, 9 + b, rect_side=(3, 12), disc_radius=(2, 6)))
    u = np.stack(us).astype(np.float32); v = np.stack(vs).astype(np.float32)
    rho = np.stack(rs).astype(np.float32); fl = np.stack(fs)
    inlet = (nx // 2 - 4, nx // 2 + 4)
    pp = hp.PlumeParams(dt=dt, inlet_x0=inlet[0], inlet_x1=inlet[1])
    uo, vo, ro = hp.hp_advect_step(t(u, dev), t(v, dev), t(rho, dev), t(fl, dev), pp)
    torch.cuda.synchronize()
    uo, vo, ro = uo.cpu().numpy(), vo.cpu().numpy(), ro.cpu().numpy()
    for b in range(B):
        eu, ev, er = A.advect_step(u[b], v[b], rho[b], fl[b], dt, inlet=inlet)
        umax = max(np.abs(eu).max(), np.abs(ev).max())
        assert np.abs(uo[b] - eu).max() <= TOL * umax
        assert np.abs(vo[b] - ev).max() <= TOL * umax
        assert np.abs(ro[b] - er).max() <= TOL * np.abs(er).max()


@pytest.mark.parametrize("threshold", [1e-3, 1e-7])
def test_plume_128_teacher_forced(dev, threshold):
    from paper_2109_09363_gb300.plume import Plume, PlumeConfig
    n = 128
    u0, v0, rho0 = W.plume_initial_state(n, seed=0)
    fl = W.plume_flags(n)[None]
    x0, x1 = W.inlet_columns(n)
    cfg = PlumeConfig(ny=n, nx=n, dt=0.1, inlet=(x0, x1), threshold=threshold, max_iters=2000)
    sim = Plume(cfg, t(u0[None].astype(np.float32), dev), t(v0[None].astype(np.float32), dev),
                t(rho0[None].astype(np.float32), dev), t(fl, dev))
    swept = 0
    for step in range(50):
        su, sv, sr = (x.cpu().numpy()[0].astype(np.float64) for x in (sim.u, sim.v, sim.rho))
        sim.advect()
        eu, ev, er = A.advect_step(su, sv, sr, fl[0], cfg.dt, inlet=(x0, x1))
        gu, gv, gr = (x.cpu().numpy()[0] for x in (sim.u, sim.v, sim.rho))
        umax = max(np.abs(eu).max(), np.abs(ev).max(), 1e-12)
        assert np.abs(gu - eu).max() <= TOL * umax, step
        assert np.abs(gv - ev).max() <= TOL * umax, step
        assert np.abs(gr - er).max() <= TOL * np.abs(er).max(), step
        ustar = (gu.astype(np.float64), gv.astype(np.float64))
        out = sim.project()
        torch.cuda.synchronize()
        ref = oracle.project(ustar[0], ustar[1], fl, threshold, 2000, dt=cfg.dt,
                             hist_len=2002)
        kg = int(out["iters"].cpu()[0])
        ko = int(ref["iters"][0])
        swept += kg
        if kg != ko:
            eh = ref["e_hist"][0]
            lo, hi = min(kg, ko), max(kg, ko)
            seg = eh[lo:hi + 1]
            seg = seg[np.isfinite(seg)]  # the oracle's history ends at its own stop
            assert seg.size and np.all(np.abs(seg - threshold) / threshold <= 5e-5), (step, kg, ko)
            ref = oracle.project(ustar[0], ustar[1], fl, threshold, 2000, dt=cfg.dt,
                                 fixed_iters=kg)
        pu, pv = sim.u.cpu().numpy()[0], sim.v.cpu().numpy()[0]
        umax = max(np.abs(ref["u"]).max(), np.abs(ref["v"]).max(), 1e-12)
        assert np.abs(pu - ref["u"][0]).max() <= TOL * umax, step
        assert np.abs(pv - ref["v"][0]).max() <= TOL * umax, step
    if threshold < 1e-5:
        assert swept > 0
    # the light fluid rises: negative v above the inlet
    assert sim.v.cpu().numpy()[0][n - 2, n // 2] < 0


@pytest.mark.parametrize("shape,dt", [((1, 16, 16), 0.1), ((2, 67, 130), 0.5), ((1, 128, 96), 2.5)])
def test_maccormack_step_matches_oracle(dev, shape, dt):
    B, ny, nx = shape
    rng = np.random.default_rng(ny + nx + 1)
    us, vs, rs, fs = [], [], [], []
    for b in range(B):
        u, v = W.vortex_velocity(ny, nx, 17 + b, n_vortices=6, width=(3, 12))
        us.append(u); vs.append(v)
        rs.append(1.0 + 0.05 * rng.standard_normal((ny, nx)))
        fs.append(W.random_obstacles(ny, nx, 19 + b, rect_side=(3, 12), disc_radius=(2, 6)))
    u = np.stack(us).astype(np.float32); v = np.stack(vs).astype(np.float32)
    rho = np.stack(rs).astype(np.float32); fl = np.stack(fs)
    inlet = (nx // 2 - 4, nx // 2 + 4)
    pp = hp.PlumeParams(dt=dt, inlet_x0=inlet[0], inlet_x1=inlet[1], scheme=1)
    uo, vo, ro = hp.hp_advect_step(t(u, dev), t(v, dev), t(rho, dev), t(fl, dev), pp)
    torch.cuda.synchronize()
    uo, vo, ro = uo.cpu().numpy(), vo.cpu().numpy(), ro.cpu().numpy()
    for b in range(B):
        eu, ev, er = A.advect_step(u[b], v[b], rho[b], fl[b], dt, inlet=inlet,
                                   scheme="maccormack")
        umax = max(np.abs(eu).max(), np.abs(ev).max())
        assert np.abs(uo[b] - eu).max() <= TOL * umax
        assert np.abs(vo[b] - ev).max() <= TOL * umax
        assert np.abs(ro[b] - er).max() <= TOL * np.abs(er).max()
        # and it is not the first-order result
        su, sv, sr = A.advect_step(u[b], v[b], rho[b], fl[b], dt, inlet=inlet)
        assert np.abs(er - sr).max() > 100 * TOL * np.abs(er).max()
    with pytest.raises(hp.HprojError):
        hp.hp_advect_step(t(u, dev), t(v, dev), t(rho, dev), t(fl, dev),
                          hp.PlumeParams(dt=dt, scheme=2))


def test_maccormack_fast_flow_matches_oracle(dev):
    """A displacement dt |vel| of up to 4.4 cells: the backward sample's
    corners fall inside the forward field's shared-memory window (up to two
    samples away) for most samples and outside it for the rest, where the
    kernel evaluates the forward field where it needs it."""
    B, ny, nx, dt = 2, 70, 100, 8.0
    rng = np.random.default_rng(5)
    us, vs, rs, fs = [], [], [], []
    for b in range(B):
        u, v = W.vortex_velocity(ny, nx, 3 + b, n_vortices=6, width=(3, 12))
        us.append(u); vs.append(v)
        rs.append(1.0 + 0.05 * rng.standard_normal((ny, nx)))
        fs.append(W.random_obstacles(ny, nx, 29 + b, rect_side=(3, 12), disc_radius=(2, 6)))
    u = np.stack(us).astype(np.float32); v = np.stack(vs).astype(np.float32)
    far = dt * np.abs(u) >= 2.0
    assert 0.02 < far.mean() < 0.5
    rho = np.stack(rs).astype(np.float32); fl = np.stack(fs)
    inlet = (nx // 2 - 4, nx // 2 + 4)
    pp = hp.PlumeParams(dt=dt, inlet_x0=inlet[0], inlet_x1=inlet[1], scheme=1)
    uo, vo, ro = hp.hp_advect_step(t(u, dev), t(v, dev), t(rho, dev), t(fl, dev), pp)
    torch.cuda.synchronize()
    uo, vo, ro = uo.cpu().numpy(), vo.cpu().numpy(), ro.cpu().numpy()
    for b in range(B):
        eu, ev, er = A.advect_step(u[b], v[b], rho[b], fl[b], dt, inlet=inlet,
                                   scheme="maccormack")
        umax = max(np.abs(eu).max(), np.abs(ev).max())
        assert np.abs(uo[b] - eu).max() <= TOL * umax
        assert np.abs(vo[b] - ev).max() <= TOL * umax
        assert np.abs(ro[b] - er).max() <= TOL * np.abs(er).max()


def test_plume_head_matches_oracle(dev):
    n = 96
    rng = np.random.default_rng(4)
    rho = np.ones((3, n, n), np.float32)
    rho[0] += (0.02 * rng.standard_normal((n, n))).astype(np.float32)
    rho[1, 60:90, 20:31] = 1.1
    rho[1, 40, 70] = 0.9
    g = torch.from_numpy(rho).to(dev)
    for contrast in (0.0, 0.01, 0.03, 0.05, 0.2):
        got = hp.hp_plume_head(g, 1.0, contrast).cpu().numpy()
        for b in range(3):
            assert tuple(got[b]) == A.plume_head(rho[b], 1.0, contrast), (contrast, b)


def test_plume_maccormack_paper_geometry_teacher_forced(dev):
    """The paper's plume with the cylinder (Sec. 2.1) at 128^2, MacCormack
    advection, every step checked against the oracle from the GPU state."""
    from paper_2109_09363_gb300.plume import Plume, PlumeConfig
    n, thr = 128, 1e-7
    fl, (x0, x1) = W.paper_plume_geometry(n)
    fl = fl[None]
    u0, v0, rho0 = W.plume_initial_state(n, seed=1)
    cfg = PlumeConfig(ny=n, nx=n, dt=0.5, gravity=-0.05, inlet=(x0, x1), threshold=thr,
                      max_iters=3000, scheme=1)
    sim = Plume(cfg, t(u0[None].astype(np.float32), dev), t(v0[None].astype(np.float32), dev),
                t(rho0[None].astype(np.float32), dev), t(fl, dev))
    for step in range(12):
        su, sv, sr = (x.cpu().numpy()[0].astype(np.float64) for x in (sim.u, sim.v, sim.rho))
        sim.advect()
        eu, ev, er = A.advect_step(su, sv, sr, fl[0], cfg.dt, gravity=cfg.gravity,
                                   inlet=(x0, x1), scheme="maccormack")
        gu, gv, gr = (x.cpu().numpy()[0] for x in (sim.u, sim.v, sim.rho))
        umax = max(np.abs(eu).max(), np.abs(ev).max(), 1e-12)
        assert np.abs(gu - eu).max() <= TOL * umax, step
        assert np.abs(gv - ev).max() <= TOL * umax, step
        assert np.abs(gr - er).max() <= TOL * np.abs(er).max(), step
        sim.project()
        torch.cuda.synchronize()
    hy, _, _ = sim.head()
    assert float(hy[0]) > 0.0
