"""FP64 oracle of the plume driver step (advection and buoyancy), numpy.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.2 of the paper advects the density and the velocity with a
semi-Lagrangian scheme and adds the external forces with forward Euler,
giving u*; the projection follows.  This oracle takes the first-order
semi-Lagrangian form (one Euler backtrace, bilinear interpolation) and the
Boussinesq buoyancy of the plume case:

  1. inlet: rho = rho_in on the inlet cells (bottom row, columns [x0, x1));
  2. every quantity q (rho at cell centres, u and v at their faces) is
     sampled at the departure point x - dt * vel(x), with vel the velocity at
     the start of the step (u^n, v^n) interpolated bilinearly per component;
     sample positions are clamped to the span of the quantity's grid;
  3. buoyancy on the interior v faces: v += dt * g * (rho_face - rho_amb) with
     rho_face the mean of the two adjacent advected cell densities;
  4. the velocity of every closed face is set to zero.

Positions: cell (i, j) centred at (i + 1/2, j + 1/2); u face (j, i) at
(i, j + 1/2); v face (j, i) at (i + 1/2, j); row 0 is the top of the image,
so a negative v points up.

With scheme="maccormack" step 2 is the MacCormack semi-Lagrangian method the
paper names (Sec. 2.2, after Selle et al. 2008) for rho, u and v alike: the
forward semi-Lagrangian result q_f, the backward semi-Lagrangian result q_b
(q_f sampled at x + dt * vel(x)), q_f + (q - q_b) / 2, clamped to the
smallest and largest of the four samples of q that the forward step
interpolated (the limiter that keeps the scheme stable).
"""
from __future__ import annotations

import numpy as np

import oracle


def bilinear(q, x, y, ox, oy):
    """Bilinear sample of q[j][i] (sample (j, i) at (i + ox, j + oy)) at
    points (x, y); positions outside the sample span are clamped to it."""
    My, Mx = q.shape
    tx = np.clip(x - ox, 0.0, Mx - 1.0)
    ty = np.clip(y - oy, 0.0, My - 1.0)
    i0 = np.minimum(np.floor(tx).astype(np.int64), max(Mx - 2, 0))
    j0 = np.minimum(np.floor(ty).astype(np.int64), max(My - 2, 0))
    fx = tx - i0
    fy = ty - j0
    i1 = np.minimum(i0 + 1, Mx - 1)
    j1 = np.minimum(j0 + 1, My - 1)
    top = q[j0, i0] * (1.0 - fx) + q[j0, i1] * fx
    bot = q[j1, i0] * (1.0 - fx) + q[j1, i1] * fx
    return top * (1.0 - fy) + bot * fy


def stencil_range(q, x, y, ox, oy):
    """(min, max) of the four samples of q that bilinear(q, x, y, ox, oy)
    interpolates."""
    My, Mx = q.shape
    tx = np.clip(x - ox, 0.0, Mx - 1.0)
    ty = np.clip(y - oy, 0.0, My - 1.0)
    i0 = np.minimum(np.floor(tx).astype(np.int64), max(Mx - 2, 0))
    j0 = np.minimum(np.floor(ty).astype(np.int64), max(My - 2, 0))
    i1 = np.minimum(i0 + 1, Mx - 1)
    j1 = np.minimum(j0 + 1, My - 1)
    c = np.stack([q[j0, i0], q[j0, i1], q[j1, i0], q[j1, i1]])
    return c.min(axis=0), c.max(axis=0)


def advect_quantity(q, x, y, ox, oy, vx, vy, dt, scheme):
    """q [My][Mx] (sample (j, i) at (i + ox, j + oy)) advected to its own
    sample points (x, y) with the velocity (vx, vy) there."""
    xd, yd = x - dt * vx, y - dt * vy
    fwd = bilinear(q, xd, yd, ox, oy)
    if scheme == "sl":
        return fwd
    if scheme != "maccormack":
        raise ValueError(scheme)
    back = bilinear(fwd, x + dt * vx, y + dt * vy, ox, oy)
    lo, hi = stencil_range(q, xd, yd, ox, oy)
    return np.clip(fwd + 0.5 * (q - back), lo, hi)


def velocity_at(u, v, x, y):
    """(u, v) at points (x, y): each component interpolated on its own faces."""
    return bilinear(u, x, y, 0.0, 0.5), bilinear(v, x, y, 0.5, 0.0)


def advect_step(u, v, rho, flags, dt, gravity=-0.002, rho_amb=1.0, rho_in=1.1, inlet=None,
                scheme="sl", u_in=0.0, open_top=False):
    """One driver step on one grid; returns (u*, v*, rho) in FP64.

    u [ny][nx+1], v [ny+1][nx], rho, flags [ny][nx]; inlet = (x0, x1) columns
    of the bottom-row density source or None; scheme "sl" (first-order
    semi-Lagrangian) or "maccormack".  Velocity injection (the plume's inlet
    speed U_in of Sec. 4.1): the bottom-boundary v faces of the inlet columns
    under fluid cells get v = -u_in (upwards) after the step; with open_top
    the top-boundary v faces of fluid cells keep their advected velocity (the
    outflow) instead of being closed.
    """
    u = np.asarray(u, np.float64)
    v = np.asarray(v, np.float64)
    rho = np.array(rho, np.float64)
    ny, nx = rho.shape
    if inlet is not None:
        rho[ny - 1, inlet[0]:inlet[1]] = rho_in
    # departure points of the cell centres, u faces and v faces
    jc, ic = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    xc, yc = ic + 0.5, jc + 0.5
    ju, iu = np.meshgrid(np.arange(ny), np.arange(nx + 1), indexing="ij")
    xu, yu = iu.astype(np.float64), ju + 0.5
    jv, iv = np.meshgrid(np.arange(ny + 1), np.arange(nx), indexing="ij")
    xv, yv = iv + 0.5, jv.astype(np.float64)

    vx, vy = velocity_at(u, v, xc, yc)
    rho_new = advect_quantity(rho, xc, yc, 0.5, 0.5, vx, vy, dt, scheme)
    vx, vy = velocity_at(u, v, xu, yu)
    u_new = advect_quantity(u, xu, yu, 0.0, 0.5, vx, vy, dt, scheme)
    vx, vy = velocity_at(u, v, xv, yv)
    v_new = advect_quantity(v, xv, yv, 0.5, 0.0, vx, vy, dt, scheme)
    # Boussinesq buoyancy on interior v faces (forward Euler)
    rho_face = 0.5 * (rho_new[:-1, :] + rho_new[1:, :])
    v_new[1:ny, :] += dt * gravity * (rho_face - rho_amb)
    uz, vz = oracle.zero_closed_faces(u_new, v_new, flags)
    uz, vz = uz[0], vz[0]
    fluid = np.asarray(flags).reshape(ny, nx) == 0
    if open_top:
        vz[0, fluid[0]] = v_new[0, fluid[0]]
    if inlet is not None and u_in != 0.0:
        cols = np.zeros(nx, bool)
        cols[max(inlet[0], 0):max(min(inlet[1], nx), 0)] = True
        vz[ny, cols & fluid[ny - 1]] = -u_in
    return uz, vz, rho_new


def plume_head(rho, rho_amb=1.0, contrast=0.01):
    """Plume head of one grid (Sec. 4.1: the highest point of the plume and
    its horizontal extent): (smallest row, smallest column, largest column) of
    the cells with |rho - rho_amb| >= contrast, (ny, nx, -1) if there is none.
    The comparison is made in FP32, as in the library, so that both take the
    same decision for every cell."""
    r = np.asarray(rho, np.float32)
    m = np.abs(r - np.float32(rho_amb)) >= np.float32(contrast)
    ny, nx = r.shape
    if not m.any():
        return ny, nx, -1
    rows, cols = np.nonzero(m)
    return int(rows.min()), int(cols.min()), int(cols.max())
