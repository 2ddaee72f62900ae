"""FP64 oracle of the training loss of the MultiScale CNN, numpy.
TEST INFRASTRUCTURE ONLY (see the package docstring).

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
