"""FP64 oracle of the training losses of the MultiScale CNN, numpy.
TEST INFRASTRUCTURE ONLY (see the package docstring).

1. loss_and_grad: the supervised loss with a divergence term (below).
2. pdnn_loss_and_grad: the physics-driven loss of Sec. 3.2 (Eq. 4).
3. adam_step: the optimiser (Sec. 3.2 trains with a gradient-descent
   algorithm; Adam as published by Kingma and Ba, 2015, Algorithm 1).
4. training_target: the pressure target of a training pair (the plain
   solver's iterates, reading below).

Reading (the paper trains on the divergence of the corrected field, Sec. 3.2,
and this build also supervises on pressures from the plain solver); both terms
are relative, so that neither dominates through the scale of its units:
    t = phi*/s, d = div/s, e = phi_hat - t
    sup = sum_fluid (e - mean_fluid e)^2 / sum_fluid (t - mean_fluid t)^2
    div = lambda * sum_all r^2 / sum_all d^2,  r = d - L phi_hat (0 on solid)
per grid; the batch loss is the mean over grids.
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import adjoint as AD


def loss_and_grad(phi_hat, target, div, flags, s, lam):
    """(loss, dloss/dphi_hat) for one grid."""
    phi_hat = np.asarray(phi_hat, np.float64)
    fluid = np.asarray(flags) == 0
    t = np.asarray(target, np.float64) / s
    d = np.asarray(div, np.float64) / s
    e = phi_hat - t
    g = np.zeros_like(phi_hat)
    loss = 0.0
    if fluid.any():
        vt = ((t - t[fluid].mean())[fluid] ** 2).sum()
        if vt > 0:
            ebar = e[fluid].mean()
            loss += ((e - ebar)[fluid] ** 2).sum() / vt
            g[fluid] = 2.0 * (e - ebar)[fluid] / vt
    d2 = (d ** 2).sum()
    if d2 > 0:
        r = oracle.residual(phi_hat, d, flags)[0]
        loss += lam * (r ** 2).sum() / d2
        # d(sum r^2)/dphi = -2 L r, and L r = -residual(r, 0)
        lr = -oracle.residual(r, np.zeros_like(r), flags)[0]
        g += -2.0 * lam / d2 * lr
    return loss, g


def forward_divergence(u, v):
    """Forward-difference divergence of every cell from all of its faces."""
    return (u[..., :, 1:] - u[..., :, :-1]) + (v[..., 1:, :] - v[..., :-1, :])


def forward_divergence_adjoint(g, nx, ny):
    """Transpose of forward_divergence for a cell field g [ny][nx]."""
    gu = np.zeros((ny, nx + 1))
    gv = np.zeros((ny + 1, nx))
    gu[:, 1:] += g
    gu[:, :-1] -= g
    gv[1:, :] += g
    gv[:-1, :] -= g
    return gu, gv


def pdnn_loss_and_grad(phi_hat, u_star, v_star, flags, s, weight, norm):
    """(loss, dloss/dphi_hat) of the physics-driven loss (Sec. 3.2, Eq. 4) for
    one grid whose network output is phi_hat.

    During training the network alone solves the Poisson problem: its guess
    phi = s * phi_hat (s the input scale of the network) corrects u* by Eq. 2
    without any Jacobi sweep, and the loss is the mean over all nx * ny cells
    of |div u|^norm times weight; norm = 1 is the printed Eq. 4, norm = 2 the
    mean squared error that the text names.  Here u comes from the projection
    oracle (zero closed faces, correct) and div u from all faces; the gradient
    runs the chain backwards: divergence transpose, the adjoint of the
    zero-sweep projection, the factor s.  sign(0) is taken as 0."""
    if norm not in (1, 2):
        raise ValueError("norm must be 1 or 2")
    fl = np.asarray(flags)[None]
    ny, nx = fl.shape[1:]
    phi0 = s * np.asarray(phi_hat, np.float64).reshape(1, ny, nx)
    u, v, _ = AD.project_fixed(np.asarray(u_star, np.float64).reshape(1, ny, nx + 1),
                               np.asarray(v_star, np.float64).reshape(1, ny + 1, nx),
                               phi0, fl, 0)
    d = forward_divergence(u[0], v[0])
    cells = nx * ny
    if norm == 1:
        loss = weight * np.abs(d).sum() / cells
        gd = weight * np.sign(d) / cells
    else:
        loss = weight * (d ** 2).sum() / cells
        gd = 2.0 * weight * d / cells
    gu, gv = forward_divergence_adjoint(gd, nx, ny)
    _, _, g_phi0 = AD.project_fixed_adjoint(gu[None], gv[None], None, fl, 0)
    return loss, s * g_phi0[0]


def adam_step(theta, m, v, g, t, lr, beta1, beta2, eps):
    """One Adam update at step t >= 1 (Kingma and Ba, 2015, Algorithm 1), in
    FP64; returns the new (theta, m, v):
        m <- beta1 m + (1 - beta1) g,  v <- beta2 v + (1 - beta2) g^2
        m_hat = m / (1 - beta1^t),     v_hat = v / (1 - beta2^t)
        theta <- theta - lr m_hat / (sqrt(v_hat) + eps)
    (eps outside the square root, both moments bias-corrected)."""
    theta, m, v, g = (np.asarray(a, np.float64) for a in (theta, m, v, g))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def training_target(div, flags, n):
    """Pressure target of a training pair: n masked Jacobi sweeps (Sec. 2.2)
    from phi_0 = 0 on the right-hand side div, then the mean of phi_n and
    phi_{n+1} (reading: the mean cancels the period-2 component that plain
    Jacobi never damps, so the networks do not learn it).  div, flags
    [B][ny][nx] or [ny][nx]; returns FP64 of the same shape."""
    div = np.asarray(div, np.float64)
    phi = np.zeros_like(div)
    for _ in range(n):
        phi = oracle.jacobi_sweep(phi, div, flags).reshape(div.shape)
    nxt = oracle.jacobi_sweep(phi, div, flags).reshape(div.shape)
    return 0.5 * (phi + nxt)
