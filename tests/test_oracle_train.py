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


# ------------------------------------------------------------- value pins

def test_supervised_loss_value_by_hand():
    # 3 x 3 grid, centre solid: the 8 fluid cells form a ring (each corner
    # and edge cell has its two ring neighbours).  s = 2, lambda = 0.5.
    #   phi_hat = 1 at (0, 0), 0 elsewhere; target phi* = 4 at (0, 0)
    #   (t = phi*/s = 2 there), the solid centre holds values the loss ignores.
    #   e = phi_hat - t = -1 at (0, 0): sum (e - mean e)^2 = 49/64 + 7/64 = 7/8
    #   sum (t - mean t)^2 = (7/4)^2 + 7 (1/4)^2 = 7/2  ->  supervised 1/4
    #   div = 2 at (0, 0), -2 at (0, 1): d = div/s = 1, -1, sum d^2 = 2
    #   L phi_hat: -2 at (0, 0), +1 at its ring neighbours (0, 1) and (1, 0)
    #   r = d - L phi_hat = 3, -2, -1: sum r^2 = 14  ->  0.5 * 14 / 2 = 3.5
    fl = np.zeros((3, 3), np.uint8)
    fl[1, 1] = 1
    phi_hat = np.zeros((3, 3)); phi_hat[0, 0] = 1.0; phi_hat[1, 1] = 5.0
    target = np.zeros((3, 3)); target[0, 0] = 4.0; target[1, 1] = 7.0
    div = np.zeros((3, 3)); div[0, 0] = 2.0; div[0, 1] = -2.0
    loss, _ = TR.loss_and_grad(phi_hat, target, div, fl, 2.0, 0.5)
    assert loss == pytest.approx(0.25 + 3.5, abs=1e-14)
    # each term alone
    assert TR.loss_and_grad(phi_hat, target, div, fl, 2.0, 0.0)[0] == pytest.approx(0.25, abs=1e-15)
    # phi_hat = t exactly: no supervised error; L t = -4, +2, +2 at (0, 0) and
    # its two ring neighbours, r = 1 + 4, -1 - 2, 0 - 2, sum r^2 = 38
    assert TR.loss_and_grad(target / 2.0, target, div, fl, 2.0, 0.5)[0] == pytest.approx(
        0.5 * 38 / 2.0, abs=1e-14)


def test_adam_two_steps_by_hand():
    # theta_0 = 1, gradients 0.5 then -0.25, lr 0.1, beta 0.9 / 0.999, eps 1e-8
    #   t = 1: m = 0.05, v = 2.5e-4, m_hat = 0.5, v_hat = 0.25,
    #          theta = 1 - 0.1 * 0.5 / (0.5 + 1e-8)
    #   t = 2: m = 0.045 - 0.025 = 0.02, v = 2.4975e-4 + 6.25e-5 = 3.1225e-4,
    #          m_hat = 0.02 / 0.19 = 2/19, v_hat = 3.1225e-4 / 1.999e-3,
    #          theta = theta_1 - 0.1 * m_hat / (sqrt(v_hat) + 1e-8)
    th, m, v = TR.adam_step(1.0, 0.0, 0.0, 0.5, 1, 0.1, 0.9, 0.999, 1e-8)
    assert float(m) == pytest.approx(0.05, rel=1e-15)
    assert float(v) == pytest.approx(2.5e-4, rel=1e-14)
    assert float(th) == pytest.approx(0.90000000199999996, abs=1e-15)
    th, m, v = TR.adam_step(th, m, v, -0.25, 2, 0.1, 0.9, 0.999, 1e-8)
    assert float(m) == pytest.approx(0.02, rel=1e-14)
    assert float(v) == pytest.approx(3.1225e-4, rel=1e-14)
    assert float(th) == pytest.approx(0.87336629870784616, abs=1e-14)


def test_adam_without_memory_is_normalised_descent():
    # beta1 = beta2 = 0: m_hat = g, v_hat = g^2, the step is lr g / (|g| + eps)
    g = np.array([3.0, -0.5, 0.0, 1e-9])
    th, m, v = TR.adam_step(np.ones(4), np.zeros(4), np.zeros(4), g, 5, 0.01, 0.0, 0.0, 1e-8)
    assert np.allclose(th, 1.0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-16)
    assert np.array_equal(m, g) and np.array_equal(v, g * g)


def test_training_target_matches_dense_matrix_powers():
    # phi_{k+1} = D^-1 (W phi_k - div) from phi_0 = 0, built densely here
    n, sweeps = 8, 7
    fl = np.zeros((n, n), np.uint8)
    fl[2:4, 3:6] = 1
    fl[6, 1] = 1
    div = np.random.default_rng(9).standard_normal((n, n)) * (fl == 0)
    Wm = np.zeros((n * n, n * n))
    for j in range(n):
        for i in range(n):
            for dj, di in ((0, -1), (0, 1), (-1, 0), (1, 0)):
                jj, ii = j + dj, i + di
                if 0 <= jj < n and 0 <= ii < n and fl[j, i] == 0 and fl[jj, ii] == 0:
                    Wm[j * n + i, jj * n + ii] = 1.0
    cnt = Wm.sum(axis=1)
    dinv = np.where(cnt > 0, 1.0 / np.maximum(cnt, 1), 0.0)
    phi = np.zeros(n * n)
    it = []
    for _ in range(sweeps + 1):
        phi = dinv * (Wm @ phi - div.ravel())
        it.append(phi)
    exp = 0.5 * (it[sweeps - 1] + it[sweeps])
    got = TR.training_target(div, fl, sweeps)
    assert np.allclose(got.ravel(), exp, rtol=0, atol=1e-13)
    # n = 0: the mean of phi_0 = 0 and one sweep
    assert np.allclose(TR.training_target(div, fl, 0).ravel(), 0.5 * it[0], rtol=0, atol=1e-14)
