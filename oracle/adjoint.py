"""FP64 oracle of the adjoint of the fixed-count projection, numpy + the C
oracle.  TEST INFRASTRUCTURE ONLY (see the package docstring).

Forward (Eq. 2-3 with k Jacobi sweeps, Sec. 2.2):
    div = D(Z u*)                    Z zeroes closed faces, D the open-face divergence
    phi_k = J^k(phi_0; div)          k masked Jacobi sweeps
    u = Z u* - G phi_k,  p = phi_k rho0 / dt
The paper notes that the gradient of the correction is known (Sec. 3.2); the
transposes follow from the forward definitions:
    dL/dphi_k = D(g_u) + (rho0 / dt) g_p          since G^T = -D on open faces
    (dL/dphi_0, dL/ddiv) = (J^k)^T dL/dphi_k      (oracle.jacobi_adjoint)
    dL/du* = Z g_u - G dL/ddiv                    = oracle.correct(g_u, dL/ddiv)
"""
from __future__ import annotations

import numpy as np

import oracle


def project_fixed(u, v, phi0, flags, k, dt=1.0, rho0=1.0):
    r = oracle.project(u, v, flags, 0.0, 0, dt=dt, rho0=rho0, phi0=phi0, fixed_iters=k)
    return r["u"], r["v"], r["p"]


def project_fixed_adjoint(gu, gv, gp, flags, k, dt=1.0, rho0=1.0):
    """(dL/du*, dL/dv*, dL/dphi_0) given dL/du, dL/dv, dL/dp."""
    lam = oracle.divergence(gu, gv, flags)
    if gp is not None:
        lam = lam + (rho0 / dt) * np.asarray(gp, np.float64).reshape(lam.shape)
    g_phi0, g_div = oracle.jacobi_adjoint(lam, flags, k)
    # the forward sets phi_0 to zero on cells without an open face, so the
    # gradient of those entries is zero (also for k = 0)
    g_phi0 = g_phi0 * (oracle.face_mask(flags) > 0)
    gus, gvs = oracle.correct(gu, gv, g_div, flags)
    return gus, gvs, g_phi0
