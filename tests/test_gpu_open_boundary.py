"""Velocity injection at the plume inlet (U_in, Sec. 2.1 and 4.1) with an open
top (reading: the exterior beyond the top wall at p = 0), on the GPU against
the FP64 oracle (oracle/boundary.py, oracle/advect.py):

- the projection with open_top and a prescribed inflow, every sweep kernel,
  ragged multi-tile shapes with obstacles: iteration counts exact (or a near
  tie), corrected velocity within 1e-5 of max|u|, closed faces exactly zero,
  the prescribed faces unchanged, E_k history within 2e-5;
- the hybrid projection from the network's guess under the same boundary;
- the injected plume teacher-forced step by step (advection with injection,
  then projection), and its volume balance: inflow = outflow through the top.
"""
import numpy as np
import pytest

import oracle
from oracle import advect as AV
from oracle import boundary as BD
from paper_2109_09363_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
hp = pytest.importorskip("paper_2109_09363_gb300")

NEAR_TIE = 5e-5
U_TOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2109_09363_gb300 import build
    build.build()
    oracle.build()
    return torch.device("cuda:0")


def to_dev(dev, *arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrays]


def injected_case(B, ny, nx, seed, u_in=0.2):
    us, vs, fs = [], [], []
    x0, x1 = W.inlet_columns(nx)
    for b in range(B):
        u, v = W.vortex_velocity(ny, nx, 300 + seed + b, n_vortices=max(4, ny * nx // 8192),
                                 width=(max(2.0, nx / 64), max(4.0, nx / 16)), amp=(-0.2, 0.2))
        fl = W.random_obstacles(ny, nx, 400 + seed + b, rect_side=(nx / 32, nx / 6),
                                disc_radius=(nx / 64, nx / 12))
        fl[ny - 3:, :] = 0          # the inlet row stays fluid
        v = v.copy()
        v[ny, x0:x1] = -u_in
        us.append(u); vs.append(v); fs.append(fl)
    return (np.stack(us).astype(np.float32), np.stack(vs).astype(np.float32), np.stack(fs),
            (x0, x1))


def compare(g, u, v, fl, inflow, thr, cap, phi0=None, dt=1.0):
    u64, v64 = u.astype(np.float64), v.astype(np.float64)
    for b in range(fl.shape[0]):
        ref = BD.project(u64[b], v64[b], fl[b], thr, cap, open_top=True, inflow=inflow,
                         phi0=None if phi0 is None else phi0[b], dt=dt)
        kg, ko = int(g["iters"][b]), int(ref["iters"])
        eh = np.array(ref["e_hist"])
        if kg != ko:
            lo, hi = min(kg, ko), max(kg, ko)
            # the oracle's history ends at its own stop
            seg = eh[lo:min(hi + 1, eh.size)]
            seg = seg[np.isfinite(seg)]
            margins = np.abs(seg - thr) / thr
            assert seg.size and np.all(margins <= NEAR_TIE), (b, kg, ko, margins)
            ref = BD.project(u64[b], v64[b], fl[b], 0.0, 0, open_top=True, inflow=inflow,
                             phi0=None if phi0 is None else phi0[b], fixed_iters=kg, dt=dt)
        else:
            assert int(g["converged"][b]) == int(ref["converged"])
            n = min(eh.size, g["e_hist"].shape[1], kg + 1)
            gh = g["e_hist"][b, :n]
            assert np.all(np.abs(gh - eh[:n]) <= 2e-5 * np.abs(eh[:n]) + 1e-30), b
        umax = max(np.abs(ref["u"]).max(), np.abs(ref["v"]).max())
        assert np.abs(g["u"][b] - ref["u"]).max() <= U_TOL * umax, b
        assert np.abs(g["v"][b] - ref["v"]).max() <= U_TOL * umax, b
        pmax = max(np.abs(ref["p"]).max(), 1e-30)
        assert np.abs(g["p"][b] - ref["p"]).max() <= U_TOL * pmax, b
        # closed faces exactly zero, prescribed faces unchanged
        ou, ov, pv = BD.faces(fl[b], True, inflow)
        assert np.all(g["u"][b][~ou] == 0.0)
        assert np.all(g["v"][b][~(ov | pv)] == 0.0)
        assert np.array_equal(g["v"][b][pv], v[b][pv])


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("B,ny,nx", [(2, 64, 64), (1, 67, 130), (1, 130, 257)])
def test_open_top_projection_matches_the_oracle(dev, kernel, B, ny, nx):
    u, v, fl, inflow = injected_case(B, ny, nx, ny + nx)
    thr = 2e-4
    cap = 3000
    prm = hp.ProjectParams(threshold=thr, max_iters=cap, sweep_kernel=kernel, open_top=1,
                           inflow=inflow)
    ctx = hp.Context(B, ny, nx)
    ud, vd, fd = to_dev(dev, u, v, fl)
    out = hp.hp_project(ctx, ud, vd, fd, prm, hist_len=cap + 2)
    torch.cuda.synchronize()
    g = {k: t.cpu().numpy() for k, t in out.items()}
    g["u"], g["v"] = ud.cpu().numpy(), vd.cpu().numpy()
    compare(g, u, v, fl, inflow, thr, cap)
    if kernel == 0 and ny <= 512 and nx <= 512:
        assert hp.hp_resident_clusters(ctx, B, ny, nx) > 0


def div32(u, v, fl, inflow):
    """The divergence in FP32 with the library's operation order
    ((u_e - u_w) + (v_s - v_n), each step rounded to FP32), open top and
    prescribed inflow faces included: the same bits as the GPU's."""
    out = []
    for b in range(fl.shape[0]):
        ou, ov, pv = BD.faces(fl[b], True, inflow)
        uf = np.where(ou, u[b], np.float32(0)).astype(np.float32)
        vf = np.where(ov | pv, v[b], np.float32(0)).astype(np.float32)
        d = (uf[:, 1:] - uf[:, :-1]) + (vf[1:, :] - vf[:-1, :])
        out.append(np.where(fl[b] == 0, d, np.float32(0)).astype(np.float32))
    return np.stack(out)


def test_open_top_hybrid_from_the_networks_guess(dev):
    from oracle import cnn as C
    B, n = 2, 64
    u, v, fl, inflow = injected_case(B, n, n, 9)
    cnn = hp.CNN(B, n, n, params=C.flatten(C.init_params(seed=4)))
    ctx = hp.Context(B, n, n)
    prm = hp.ProjectParams(threshold=2e-4, max_iters=3000, open_top=1, inflow=inflow)
    # the guess the hybrid starts from: the network on this boundary's
    # divergence (the same FP32 bits as inside the hybrid projection)
    dd, fd = to_dev(dev, div32(u, v, fl, inflow), fl)
    phi_hat, s = hp.hp_cnn_forward(cnn, dd, fd)
    phi0 = (phi_hat * s[:, None, None]).cpu().numpy().astype(np.float64)
    ud, vd = to_dev(dev, u, v)
    out = hp.hp_project_hybrid(ctx, cnn, ud, vd, fd, prm, hist_len=3002)
    torch.cuda.synchronize()
    assert cnn.check() == 0
    g = {k: t.cpu().numpy() for k, t in out.items()}
    g["u"], g["v"] = ud.cpu().numpy(), vd.cpu().numpy()
    compare(g, u, v, fl, inflow, 2e-4, 3000, phi0=phi0)


def test_injected_plume_teacher_forced(dev):
    """128^2 plume, inlet 16 cells injecting at U_in = 0.05 with rho = 1.1,
    open top, g = -0.002, dt = 0.1: per step the GPU advection (with
    injection) against the oracle's from the same state, then the GPU
    projection of the GPU's u* against the oracle's projection of the same
    u*; the projected field carries the inflow out through the top."""
    n, steps, u_in, thr, cap = 128, 12, 0.05, 1e-6, 4000
    x0, x1 = W.inlet_columns(n)
    fl = W.plume_flags(n)
    u0, v0, rho0 = W.plume_initial_state(n, seed=4)
    pp = hp.PlumeParams(dt=0.1, gravity=-0.002, inlet_x0=x0, inlet_x1=x1, u_in=u_in, open_top=1)
    prm = hp.ProjectParams(threshold=thr, max_iters=cap, dt=0.1, open_top=1, inflow=(x0, x1))
    ctx = hp.Context(1, n, n)
    fd = to_dev(dev, fl[None])[0]
    u, v, rho = (a.astype(np.float32) for a in (u0, v0, rho0))
    sweeps = 0
    for k in range(steps):
        ud, vd, rd = to_dev(dev, u[None], v[None], rho[None])
        us, vs, rs = hp.hp_advect_step(ud, vd, rd, fd, pp)
        ua, va, ra = AV.advect_step(u, v, rho, fl, 0.1, inlet=(x0, x1), u_in=u_in, open_top=True)
        torch.cuda.synchronize()
        for got, ref in ((us, ua), (vs, va), (rs, ra)):
            gg = got[0].cpu().numpy()
            assert np.abs(gg - ref).max() <= 1e-5 * max(np.abs(ref).max(), 1e-30), k
        ustar, vstar = us.cpu().numpy(), vs.cpu().numpy()
        assert np.all(vstar[0, n, x0:x1] == np.float32(-u_in))
        out = hp.hp_project(ctx, us, vs, fd, prm, hist_len=cap + 2)
        torch.cuda.synchronize()
        g = {kk: t.cpu().numpy() for kk, t in out.items()}
        g["u"], g["v"] = us.cpu().numpy(), vs.cpu().numpy()
        compare(g, ustar, vstar, fl[None], (x0, x1), thr, cap, dt=0.1)
        sweeps += int(g["iters"][0])
        u, v, rho = g["u"][0], g["v"][0], rs[0].cpu().numpy()
        # volume balance: what enters at the bottom leaves through the top
        top, bottom = v[0, :].astype(np.float64).sum(), v[n, :].astype(np.float64).sum()
        assert bottom == pytest.approx(-u_in * (x1 - x0), rel=1e-6)
        assert abs(top - bottom) <= n * n * float(g["e1"][0]) * 1.01 + 1e-6
    assert sweeps > 0
