"""Pins of the FP64 advection/buoyancy oracle (driver step of Sec. 2.2):
identity at rest, exact integer shifts, exactness on linear fields, a
library interpolator, and the buoyancy increment."""
import numpy as np

from oracle import advect as A


def test_bilinear_matches_scipy_regular_grid_interpolator():
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(0)
    q = rng.standard_normal((9, 13))
    ox, oy = 0.5, 0.0
    x = rng.uniform(ox, 12 + ox, 200)
    y = rng.uniform(oy, 8 + oy, 200)
    f = RegularGridInterpolator((np.arange(9) + oy, np.arange(13) + ox), q, method="linear")
    assert np.allclose(A.bilinear(q, x, y, ox, oy), f(np.stack([y, x], axis=1)), atol=1e-13)


def test_bilinear_is_exact_on_linear_fields_and_clamps():
    jj, ii = np.meshgrid(np.arange(7), np.arange(11), indexing="ij")
    q = 0.3 * (ii + 0.5) - 1.7 * (jj + 0.5) + 2.0
    rng = np.random.default_rng(1)
    x = rng.uniform(0.5, 10.5, 100)
    y = rng.uniform(0.5, 6.5, 100)
    assert np.allclose(A.bilinear(q, x, y, 0.5, 0.5), 0.3 * x - 1.7 * y + 2.0, atol=1e-13)
    # outside the span: clamped to the edge sample
    assert A.bilinear(q, np.array([-5.0]), np.array([0.5]), 0.5, 0.5)[0] == q[0, 0]


def test_rest_state_is_unchanged_and_inlet_is_set():
    n = 16
    rho = 1.0 + np.zeros((n, n))
    u, v = np.zeros((n, n + 1)), np.zeros((n + 1, n))
    fl = np.zeros((n, n), np.uint8)
    u2, v2, r2 = A.advect_step(u, v, rho, fl, dt=0.1, gravity=0.0, inlet=(6, 10))
    assert np.all(u2 == 0) and np.all(v2 == 0)
    exp = rho.copy()
    exp[n - 1, 6:10] = 1.1
    assert np.array_equal(r2, exp)


def test_uniform_velocity_integer_shift_is_exact_in_the_interior():
    n, U, dt = 24, 5.0, 0.4  # dt * U = 2 cells
    rng = np.random.default_rng(2)
    rho = rng.standard_normal((n, n))
    u = np.full((n, n + 1), U)
    v = np.zeros((n + 1, n))
    fl = np.zeros((n, n), np.uint8)
    _, _, r2 = A.advect_step(u, v, rho, fl, dt=dt, gravity=0.0)
    assert np.allclose(r2[:, 2:], rho[:, :-2], atol=1e-14, rtol=0)
    # v moves the field down by 3 rows
    u0 = np.zeros((n, n + 1))
    vv = np.full((n + 1, n), 7.5)
    _, _, r3 = A.advect_step(u0, vv, rho, fl, dt=dt, gravity=0.0)
    assert np.allclose(r3[3:, :], rho[:-3, :], atol=1e-14, rtol=0)


def test_buoyancy_increment():
    n, dt, g = 12, 0.1, -0.002
    rng = np.random.default_rng(3)
    rho = 1.0 + 0.1 * rng.random((n, n))
    u, v = np.zeros((n, n + 1)), np.zeros((n + 1, n))
    fl = np.zeros((n, n), np.uint8)
    _, v2, r2 = A.advect_step(u, v, rho, fl, dt=dt, gravity=g)
    assert np.array_equal(r2, rho)
    exp = dt * g * (0.5 * (rho[:-1, :] + rho[1:, :]) - 1.0)
    assert np.allclose(v2[1:n, :], exp, rtol=1e-15, atol=0)
    assert np.all(v2[0] == 0) and np.all(v2[n] == 0)


def test_closed_faces_are_zeroed():
    n = 10
    rng = np.random.default_rng(4)
    u = rng.standard_normal((n, n + 1))
    v = rng.standard_normal((n + 1, n))
    fl = np.zeros((n, n), np.uint8)
    fl[4:6, 4:6] = 1
    u2, v2, _ = A.advect_step(u, v, np.ones((n, n)), fl, dt=0.05)
    assert np.all(u2[:, 0] == 0) and np.all(u2[:, n] == 0)
    assert np.all(v2[0, :] == 0) and np.all(v2[n, :] == 0)
    assert np.all(u2[4:6, 4:7] == 0) and np.all(v2[4:7, 4:6] == 0)


# --- MacCormack (Sec. 2.2, after Selle et al. 2008) ---------------------------------

def _uniform(n, U, V):
    return np.full((n, n + 1), U), np.full((n + 1, n), V)


def test_maccormack_rest_state_and_integer_shift():
    n = 24
    rng = np.random.default_rng(3)
    rho = rng.standard_normal((n, n))
    fl = np.zeros((n, n), np.uint8)
    u, v = _uniform(n, 0.0, 0.0)
    _, _, r0 = A.advect_step(u, v, rho, fl, dt=0.1, gravity=0.0, scheme="maccormack")
    assert np.array_equal(r0, rho)
    # two cells to the right: the forward step is exact, the backward step
    # returns the input exactly, so the correction vanishes where both stay inside
    u, v = _uniform(n, 5.0, 0.0)
    _, _, r2 = A.advect_step(u, v, rho, fl, dt=0.4, gravity=0.0, scheme="maccormack")
    assert np.allclose(r2[:, 2:n - 2], rho[:, :n - 4], atol=1e-14, rtol=0)


def _monotone_field(n, x, y):
    w = n / 6.0
    return np.tanh((x - 0.45 * n) / w) + 0.5 * np.tanh((y - 0.55 * n) / w)


def _translation_errors(n, dx, dy):
    """Max error of one step of each scheme translating a smooth field with
    no interior extremum by (dx, dy) cells, away from the boundary."""
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    xc, yc = ii + 0.5, jj + 0.5
    rho = _monotone_field(n, xc, yc)
    exact = _monotone_field(n, xc - dx, yc - dy)
    fl = np.zeros((n, n), np.uint8)
    u, v = _uniform(n, dx / 0.1, dy / 0.1)
    m = slice(4, n - 4)
    err = {}
    for sc in ("sl", "maccormack"):
        _, _, r = A.advect_step(u, v, rho, fl, dt=0.1, gravity=0.0, scheme=sc)
        err[sc] = np.abs(r - exact)[m, m].max()
    return err


def test_maccormack_is_higher_order_than_semi_lagrangian():
    """One step of a fractional translation: the first-order scheme's error
    is the bilinear interpolation error, O(h^2) per step; MacCormack cancels
    its leading term (O(h^3) per step).  Halving h (the field twice as wide
    in cells, the same displacement in cells) must cut the MacCormack error by
    about 8 and the semi-Lagrangian error by about 4."""
    e1 = _translation_errors(48, 0.37, -0.21)
    e2 = _translation_errors(96, 0.37, -0.21)
    assert e1["maccormack"] < 0.2 * e1["sl"]
    assert 3.0 < e1["sl"] / e2["sl"] < 5.0
    assert e1["maccormack"] / e2["maccormack"] > 6.0


def test_maccormack_exact_on_linear_fields():
    n = 20
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    rho = 0.4 * (ii + 0.5) - 0.9 * (jj + 0.5)
    fl = np.zeros((n, n), np.uint8)
    u, v = _uniform(n, 3.1, -1.7)  # (0.31, -0.17) cells per step
    _, _, r = A.advect_step(u, v, rho, fl, dt=0.1, gravity=0.0, scheme="maccormack")
    exact = 0.4 * (ii + 0.5 - 0.31) - 0.9 * (jj + 0.5 + 0.17)
    assert np.allclose(r[2:-2, 2:-2], exact[2:-2, 2:-2], atol=1e-12, rtol=0)


def test_maccormack_limiter_creates_no_new_extrema():
    n = 32
    rho = np.zeros((n, n))
    rho[:, 10:20] = 1.0
    fl = np.zeros((n, n), np.uint8)
    u, v = _uniform(n, 4.3, 1.9)
    _, _, r_sl = A.advect_step(u, v, rho, fl, dt=0.1, gravity=0.0, scheme="sl")
    _, _, r_mc = A.advect_step(u, v, rho, fl, dt=0.1, gravity=0.0, scheme="maccormack")
    assert r_mc.min() >= 0.0 and r_mc.max() <= 1.0
    assert np.abs(r_mc - r_sl).max() > 0.05  # the correction acts at the fronts
    # each value lies within the four samples its forward step interpolated
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    lo, hi = A.stencil_range(rho, ii + 0.5 - 0.43, jj + 0.5 - 0.19, 0.5, 0.5)
    assert np.all(r_mc >= lo - 1e-15) and np.all(r_mc <= hi + 1e-15)


def test_plume_head_of_constructed_fields():
    n = 40
    rho = np.ones((n, n))
    assert A.plume_head(rho, 1.0, 0.01) == (n, n, -1)
    # a light blob: rows 12..20, columns 7..30 (a disc clipped by a box)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    blob = ((ii - 18.5) ** 2 / 12.0 ** 2 + (jj - 16.0) ** 2 / 4.5 ** 2 <= 1.0)
    rho[blob] = 1.05
    rows, cols = np.nonzero(blob)
    assert A.plume_head(rho, 1.0, 0.01) == (rows.min(), cols.min(), cols.max())
    # heavier fluid counts by its contrast too; below the contrast it does not
    rho[35, 2] = 0.98
    assert A.plume_head(rho, 1.0, 0.01) == (rows.min(), 2, cols.max())
    assert A.plume_head(rho, 1.0, 0.03) == (rows.min(), cols.min(), cols.max())
    assert A.plume_head(rho, 1.0, 0.06) == (n, n, -1)
