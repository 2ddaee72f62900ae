"""FP64 oracle of the projection with an open top and a prescribed inflow,
numpy.  TEST INFRASTRUCTURE ONLY (see the package docstring).

The plume of the paper injects the light fluid at the speed U_in through an
inlet in the bottom wall (Sec. 2.1 and 4.1); the injected volume has to
leave the box.  Reading (the paper gives no outflow boundary): the top wall
is open to an exterior at pressure p = 0, and the inlet faces carry the
prescribed inflow velocity.  On the staggered grid (row 0 at the top, v
positive downwards):

  - open faces: the interior faces between two fluid cells, and with an open
    top the v faces of row 0 above fluid cells (to an exterior ghost cell
    with phi = 0);
  - prescribed faces: the bottom-boundary v faces of the inflow columns
    under fluid cells; they keep the given velocity, enter the divergence of
    the cell above them and are closed for the pressure;
  - every other face is closed and carries zero velocity.

The projection then follows the paper's steps as the closed-box oracle does
(oracle.c): zero the closed faces, divergence over open and prescribed faces
(Eq. 3), masked Jacobi sweeps (Sec. 2.2) with the open faces' neighbours
(the exterior counts as phi = 0), E_k = mean |r(phi_k)| over all cells with
the stop test before every sweep (Sec. 3.3 and 4.1), the correction of the
open faces (Eq. 2), and the norms of the corrected velocity.  With the top
closed and no inflow it is the closed-box projection.
"""
from __future__ import annotations

import numpy as np


def faces(flags, open_top=False, inflow=(0, 0)):
    """(open_u [ny][nx+1], open_v [ny+1][nx], prescribed_v [ny+1][nx]) as
    boolean arrays for one grid."""
    fluid = np.asarray(flags) == 0
    ny, nx = fluid.shape
    ou = np.zeros((ny, nx + 1), bool)
    ou[:, 1:nx] = fluid[:, :-1] & fluid[:, 1:]
    ov = np.zeros((ny + 1, nx), bool)
    ov[1:ny, :] = fluid[:-1, :] & fluid[1:, :]
    if open_top:
        ov[0, :] = fluid[0, :]
    pv = np.zeros((ny + 1, nx), bool)
    x0, x1 = max(inflow[0], 0), min(inflow[1], nx)
    if x1 > x0:
        pv[ny, x0:x1] = fluid[ny - 1, x0:x1]
    return ou, ov, pv


def divergence(u, v, ou, ov, pv):
    """Forward difference over the open and the prescribed faces."""
    uf = np.where(ou, u, 0.0)
    vf = np.where(ov | pv, v, 0.0)
    return (uf[:, 1:] - uf[:, :-1]) + (vf[1:, :] - vf[:-1, :])


def neighbours_and_count(phi, ou, ov):
    """(sum over the open faces of the neighbour's phi, number of open faces)
    per cell; the exterior beyond an open top face holds phi = 0."""
    ny, nx = phi.shape
    s = np.zeros_like(phi)
    n = np.zeros_like(phi)
    w, e = ou[:, :-1], ou[:, 1:]            # west / east faces of each cell
    no, so = ov[:-1, :], ov[1:, :]          # north / south faces of each cell
    s[:, 1:] += np.where(w[:, 1:], phi[:, :-1], 0.0)
    s[:, :-1] += np.where(e[:, :-1], phi[:, 1:], 0.0)
    s[1:, :] += np.where(no[1:, :], phi[:-1, :], 0.0)
    s[:-1, :] += np.where(so[:-1, :], phi[1:, :], 0.0)
    n += w.astype(np.float64) + e + no + so   # counts (bool + bool would be OR)
    return s, n


def residual(phi, div, ou, ov):
    """r = div - sum over open faces of (phi_nb - phi_c)."""
    s, n = neighbours_and_count(phi, ou, ov)
    return div - (s - n * phi)


def jacobi_sweep(phi, div, ou, ov):
    """phi' = (sum over open faces of phi_nb - div) / n; 0 where n = 0."""
    s, n = neighbours_and_count(phi, ou, ov)
    return np.where(n > 0, (s - div) / np.maximum(n, 1), 0.0)


def correct(u, v, phi, ou, ov, pv):
    """Eq. 2 on the open faces (the exterior phi = 0 beyond the top), the
    prescribed faces unchanged, every other face zero."""
    ny, nx = phi.shape
    gu = np.zeros_like(u)
    gu[:, 1:nx] = phi[:, 1:] - phi[:, :-1]
    pad = np.vstack([np.zeros((1, nx)), phi])      # row 0: the exterior
    gv = np.zeros_like(v)
    gv[:ny, :] = pad[1:, :] - pad[:-1, :]
    uo = np.where(ou, u - gu, 0.0)
    vo = np.where(ov, v - gv, np.where(pv, v, 0.0))
    return uo, vo


def project(u, v, flags, threshold, max_iters, open_top=False, inflow=(0, 0), dt=1.0,
            rho0=1.0, phi0=None, fixed_iters=0):
    """The projection of every grid of a batch ([B][ny][nx+1] etc. or one
    grid); returns a dict of u, v, p, iters, e1, einf, converged, e_hist
    (per grid the list of E_k up to the stop)."""
    fl = np.asarray(flags)
    single = fl.ndim == 2
    fl = fl.reshape((-1,) + fl.shape[-2:])
    B, ny, nx = fl.shape
    u = np.asarray(u, np.float64).reshape(B, ny, nx + 1)
    v = np.asarray(v, np.float64).reshape(B, ny + 1, nx)
    out = {k: [] for k in ("u", "v", "p", "iters", "e1", "einf", "converged", "e_hist")}
    cells = float(nx * ny)
    for b in range(B):
        ou, ov, pv = faces(fl[b], open_top, inflow)
        ub = np.where(ou, u[b], 0.0)
        vb = np.where(ov | pv, v[b], 0.0)
        div = divergence(ub, vb, ou, ov, pv)
        has_face = neighbours_and_count(np.zeros((ny, nx)), ou, ov)[1] > 0
        phi = np.zeros((ny, nx)) if phi0 is None else np.where(
            has_face, np.asarray(phi0, np.float64).reshape(B, ny, nx)[b], 0.0)
        cap = fixed_iters if fixed_iters > 0 else max_iters
        hist = []
        k, conv = 0, 0
        while True:
            e = np.abs(residual(phi, div, ou, ov)).sum() / cells
            hist.append(e)
            if fixed_iters <= 0 and e <= threshold:
                conv = 1
                break
            if k >= cap or not np.isfinite(e):
                conv = 1 if fixed_iters > 0 else 0
                break
            phi = jacobi_sweep(phi, div, ou, ov)
            k += 1
        uo, vo = correct(ub, vb, phi, ou, ov, pv)
        dc = np.where(np.asarray(fl[b]) == 0, divergence(uo, vo, ou, ov, pv), 0.0)
        out["u"].append(uo)
        out["v"].append(vo)
        out["p"].append(phi * rho0 / dt)
        out["iters"].append(k)
        out["e1"].append(np.abs(dc).sum() / cells)
        out["einf"].append(np.abs(dc).max())
        out["converged"].append(conv)
        out["e_hist"].append(hist)
    res = {k: (np.array(vv) if k != "e_hist" else vv) for k, vv in out.items()}
    if single:
        res = {k: vv[0] for k, vv in res.items()}
    return res
