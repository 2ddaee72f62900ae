"""Pin of the training-loss oracle: central differences of its gradient."""
import numpy as np

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
