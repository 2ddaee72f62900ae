"""Pins of the training-loss oracles: central differences of their
gradients, the residual identity, an exact guess, gauge invariance."""
import numpy as np
import pytest

import oracle
from oracle import train as TR


def test_loss_gradient_by_central_differences():
    rng = np.random.default_rng(0)
    n = 10
    fl = (rng.random((n, n)) < 0.15).astype(np.uint8)
    phi = rng.standard_normal((n, n))
    tgt = rng.standard_normal((n, n))
    div = rng.standard_normal((n, n)) * (fl == 0)
    s, lam = 0.7, 0.3
    L, g = TR.loss_and_grad(phi, tgt, div, fl, s, lam)
    eps = 1e-6
    for _ in range(20):
        idx = tuple(rng.integers(0, n, 2))
        p, m = phi.copy(), phi.copy()
        p[idx] += eps
        m[idx] -= eps
        fd = (TR.loss_and_grad(p, tgt, div, fl, s, lam)[0] -
              TR.loss_and_grad(m, tgt, div, fl, s, lam)[0]) / (2 * eps)
        assert np.isclose(g[idx], fd, rtol=1e-6, atol=1e-9)


def test_loss_is_gauge_invariant_in_the_supervised_term():
    rng = np.random.default_rng(1)
    n = 8
    fl = np.zeros((n, n), np.uint8)
    phi = rng.standard_normal((n, n))
    tgt = rng.standard_normal((n, n))
    div = np.zeros((n, n))
    a = TR.loss_and_grad(phi, tgt, div, fl, 1.0, 0.0)[0]
    b = TR.loss_and_grad(phi + 3.0, tgt, div, fl, 1.0, 0.0)[0]
    assert np.isclose(a, b, rtol=1e-12)


def _pdnn_case(n, seed, solid_frac=0.15):
    rng = np.random.default_rng(seed)
    fl = (rng.random((n, n)) < solid_frac).astype(np.uint8)
    u = rng.standard_normal((n, n + 1))
    v = rng.standard_normal((n + 1, n))
    phi = rng.standard_normal((n, n))
    return rng, fl, u, v, phi


@pytest.mark.parametrize("norm", [1, 2])
def test_pdnn_loss_is_the_residual_of_the_scaled_guess(norm):
    """div(u* - grad(s phi_hat)) equals s * r(phi_hat; div(u*)/s) on every cell
    (the identity behind the fused stop test, Eq. 2-3), so the loss computed
    through the corrected velocity equals the one written with the residual."""
    _, fl, u, v, phi = _pdnn_case(12, 3)
    s, w = 0.37, 1.7
    L, _ = TR.pdnn_loss_and_grad(phi, u, v, fl, s, w, norm)
    d = oracle.divergence(u[None], v[None], fl[None])[0]
    r = s * oracle.residual(phi, d / s, fl)[0]
    assert np.isclose(L, w * (np.abs(r) ** norm).sum() / fl.size, rtol=1e-12)


@pytest.mark.parametrize("norm", [1, 2])
def test_pdnn_gradient_by_central_differences(norm):
    rng, fl, u, v, phi = _pdnn_case(10, 4)
    s, w = 0.8, 0.6
    L, g = TR.pdnn_loss_and_grad(phi, u, v, fl, s, w, norm)
    # central differences are exact for a quadratic and, away from its kinks,
    # for a piecewise linear loss: eps only has to beat cancellation
    eps = 1e-5
    pr = oracle.project(u[None], v[None], fl[None], 0.0, 0, phi0=s * phi[None])
    d0 = TR.forward_divergence(pr["u"][0], pr["v"][0])
    # the L1 loss is smooth only away from div = 0: keep every perturbed
    # divergence on its side of zero (cells without an open face stay at 0)
    open_ = oracle.face_mask(fl[None])[0] > 0
    assert np.all(d0[~open_] == 0.0)
    assert np.abs(d0[open_]).min() > 4 * s * eps
    for _ in range(25):
        idx = tuple(rng.integers(0, 10, 2))
        p, m = phi.copy(), phi.copy()
        p[idx] += eps
        m[idx] -= eps
        fd = (TR.pdnn_loss_and_grad(p, u, v, fl, s, w, norm)[0] -
              TR.pdnn_loss_and_grad(m, u, v, fl, s, w, norm)[0]) / (2 * eps)
        assert np.isclose(g[idx], fd, rtol=1e-7, atol=1e-9), (idx, g[idx], fd)


def test_pdnn_exact_guess_removes_the_divergence():
    """u* = grad(psi) on open faces: phi_hat = psi / s makes the corrected
    field zero, so both losses vanish and the L2 gradient too."""
    rng, fl, _, _, psi = _pdnn_case(14, 5, solid_frac=0.2)
    z = np.zeros((1, 14, 15)), np.zeros((1, 15, 14))
    u, v = oracle.correct(z[0], z[1], -psi[None], fl[None])
    assert np.abs(u).max() > 0.1
    s = 0.45
    for norm in (1, 2):
        L, g = TR.pdnn_loss_and_grad(psi / s, u[0], v[0], fl, s, 1.0, norm)
        assert L < 1e-13
        if norm == 2:
            assert np.abs(g).max() < 1e-13


def test_pdnn_loss_is_gauge_invariant():
    _, fl, u, v, phi = _pdnn_case(9, 6, solid_frac=0.0)
    a = TR.pdnn_loss_and_grad(phi, u, v, fl, 0.5, 1.0, 2)[0]
    b = TR.pdnn_loss_and_grad(phi - 2.5, u, v, fl, 0.5, 1.0, 2)[0]
    assert np.isclose(a, b, rtol=1e-12)
