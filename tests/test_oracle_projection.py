"""Pins of the FP64 oracle's projection path against facts that do not come
from the oracle itself: closed forms, exact identities, a dense direct solve,
dense matrix powers, brute force on tiny grids and a hand-derived fixture.

Each test names the part of the method it pins (Eq. 2, Eq. 3, the Jacobi
iteration of Sec. 2.2, E_1 of Sec. 4.1, the stop rule of Sec. 3.3).
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2109_09363_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
# Independent dense constructions (Python loops over cells and neighbours,
# never calling the oracle).

def _nbrs(fl, j, i):
    ny, nx = fl.shape
    out = []
    for dj, di in ((0, -1), (0, 1), (-1, 0), (1, 0)):
        jj, ii = j + dj, i + di
        if 0 <= jj < ny and 0 <= ii < nx and fl[j, i] == 0 and fl[jj, ii] == 0:
            out.append(jj * nx + ii)
    return out


def dense_adjacency(fl):
    """W (open-face adjacency) and n (open-face count) of one grid."""
    ny, nx = fl.shape
    Wm = np.zeros((ny * nx, ny * nx))
    for j in range(ny):
        for i in range(nx):
            for q in _nbrs(fl, j, i):
                Wm[j * nx + i, q] = 1.0
    return Wm, Wm.sum(axis=1)


def dense_laplacian(fl):
    Wm, n = dense_adjacency(fl)
    return Wm - np.diag(n)


def small_case(n=8, seed=3, solid=True):
    u, v = W.vortex_velocity(n, n, seed, n_vortices=4, width=(1.5, 4.0))
    fl = np.zeros((n, n), np.uint8)
    if solid:
        fl[2:4, 3:6] = 1
        fl[6, 1] = 1
    return u, v, fl


def cos_mode(n, k, l):
    i = np.arange(n) + 0.5
    return np.outer(np.cos(np.pi * l * i / n), np.cos(np.pi * k * i / n))


def cos_eig(n, k, l):
    return -4 * np.sin(np.pi * k / (2 * n)) ** 2 - 4 * np.sin(np.pi * l / (2 * n)) ** 2


# ------------------------------------------------------------ face mask

def test_face_mask_brute_force():
    rng = np.random.default_rng(0)
    for shape in [(1, 1), (1, 5), (4, 4), (5, 7), (9, 3)]:
        fl = (rng.random(shape) < 0.3).astype(np.uint8)
        got = oracle.face_mask(fl)[0]
        ny, nx = shape
        for j in range(ny):
            for i in range(nx):
                exp = 0
                if fl[j, i] == 0:
                    if i > 0 and fl[j, i - 1] == 0: exp |= 1
                    if i < nx - 1 and fl[j, i + 1] == 0: exp |= 2
                    if j > 0 and fl[j - 1, i] == 0: exp |= 4
                    if j < ny - 1 and fl[j + 1, i] == 0: exp |= 8
                assert got[j, i] == exp


# ----------------------------------------------------------- divergence

def test_divergence_of_linear_field_interior():
    n, a, b = 10, 0.7, -0.3
    xu = np.broadcast_to(np.arange(n + 1, dtype=float), (n, n + 1))
    yv = np.broadcast_to(np.arange(n + 1, dtype=float)[:, None], (n + 1, n))
    fl = np.zeros((n, n), np.uint8)
    d = oracle.divergence(a * xu, b * yv, fl)[0]
    assert np.allclose(d[1:-1, 1:-1], a + b, atol=1e-14, rtol=0)


def test_divergence_telescopes_in_closed_box():
    u, v = W.vortex_velocity(32, 32, 7)
    fl = W.random_obstacles(32, 32, 8, disc_radius=(2, 6), rect_side=(3, 9))
    d = oracle.divergence(u, v, fl)
    assert abs(d.sum()) < 1e-12 * np.abs(d).sum()


def test_divergence_of_stream_function_field_is_zero():
    rng = np.random.default_rng(5)
    n = 12
    psi = rng.standard_normal((n + 1, n + 1))
    psi[0, :] = psi[-1, :] = psi[:, 0] = psi[:, -1] = 0.0
    u = psi[1:, :] - psi[:-1, :]           # [n][n+1]
    v = -(psi[:, 1:] - psi[:, :-1])        # [n+1][n]
    d = oracle.divergence(u, v, np.zeros((n, n), np.uint8))
    assert np.abs(d).max() < 1e-14


def test_zero_closed_faces():
    u, v, fl = small_case()
    uz, vz = oracle.zero_closed_faces(u, v, fl)
    m = oracle.face_mask(fl)[0]
    n = fl.shape[0]
    for j in range(n):
        for i in range(n + 1):
            op = 0 < i < n and fl[j, i - 1] == 0 and fl[j, i] == 0
            assert (uz[0, j, i] == u[j, i]) if op else (uz[0, j, i] == 0.0)
    assert m.shape == (n, n)


# ------------------------------------------------- Laplacian and sweep

def test_residual_of_neumann_cosine_modes_is_zero():
    n = 16
    fl = np.zeros((n, n), np.uint8)
    for k, l in [(1, 0), (0, 3), (2, 5), (7, 7)]:
        mode = cos_mode(n, k, l)
        div = cos_eig(n, k, l) * mode
        r = oracle.residual(mode, div, fl)
        assert np.abs(r).max() < 1e-13
        # a fixed point of the Jacobi sweep
        assert np.allclose(oracle.jacobi_sweep(mode, div, fl)[0], mode, atol=1e-14, rtol=0)


def test_sweep_matches_dense_jacobi_matrix():
    u, v, fl = small_case(8)
    uz, vz = oracle.zero_closed_faces(u, v, fl)
    div = oracle.divergence(uz, vz, fl)[0].ravel()
    Wm, n = dense_adjacency(fl)
    Dinv = np.where(n > 0, 1.0 / np.maximum(n, 1), 0.0)
    phi = np.random.default_rng(1).standard_normal(64)
    exp = Dinv * (Wm @ phi - div)
    got = oracle.jacobi_sweep(phi.reshape(8, 8), div.reshape(8, 8), fl)[0].ravel()
    assert np.allclose(got, exp, atol=1e-14, rtol=0)
    # residual = div - L phi on fluid cells
    r = oracle.residual(phi.reshape(8, 8), div.reshape(8, 8), fl)[0].ravel()
    L = dense_laplacian(fl)
    fluid = fl.ravel() == 0
    assert np.allclose(r[fluid], (div - L @ phi)[fluid], atol=1e-13, rtol=0)
    assert np.all(r[~fluid] == 0)


def test_jacobi_matrix_has_plus_and_minus_one_eigenvalues():
    fl = np.zeros((8, 8), np.uint8)
    Wm, n = dense_adjacency(fl)
    ev = np.linalg.eigvals(Wm / n[:, None])
    assert np.min(np.abs(ev - 1.0)) < 1e-12
    assert np.min(np.abs(ev + 1.0)) < 1e-12
    assert np.max(np.abs(ev)) < 1 + 1e-12


def test_long_jacobi_converges_to_cosine_mode():
    n = 16
    fl = np.zeros((n, n), np.uint8)
    mode = cos_mode(n, 1, 1)
    div = cos_eig(n, 1, 1) * mode
    phi = np.zeros((n, n))
    for _ in range(4000):
        phi = oracle.jacobi_sweep(phi, div, fl)[0]
    nxt = oracle.jacobi_sweep(phi, div, fl)[0]
    # the cosine mode is an eigenvector of L but not of D^-1 W at the walls, so
    # the non-decaying eigenvalue -1 component alternates between iterates; the
    # mean of two consecutive iterates cancels it
    avg = 0.5 * (phi + nxt)
    assert np.allclose(avg - avg.mean(), mode, atol=1e-9, rtol=0)
    assert not np.allclose(phi - phi.mean(), mode, atol=1e-9, rtol=0)


# ---------------------------------------------- correction and projection

def test_gradient_is_minus_adjoint_of_divergence():
    u, v, fl = small_case(8)
    rng = np.random.default_rng(2)
    phi = rng.standard_normal((8, 8))
    uz, vz = oracle.zero_closed_faces(u, v, fl)
    # correct(0, phi) = -grad phi on open faces
    gu, gv = oracle.correct(np.zeros_like(u), np.zeros_like(v), phi, fl)
    lhs = -(np.sum(gu[0] * uz[0]) + np.sum(gv[0] * vz[0]))   # <grad phi, u>
    rhs = -np.sum(phi * oracle.divergence(uz, vz, fl)[0])      # -<phi, div u>
    assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_dense_direct_solve_gives_divergence_free_velocity():
    for seed in range(3):
        u, v = W.vortex_velocity(16, 16, seed, n_vortices=6, width=(2, 6))
        fl = W.random_obstacles(16, 16, 10 + seed, disc_radius=(2, 4), rect_side=(2, 5))
        uz, vz = oracle.zero_closed_faces(u, v, fl)
        div = oracle.divergence(uz, vz, fl)[0].ravel()
        L = dense_laplacian(fl)
        phi = np.linalg.lstsq(L, div, rcond=None)[0].reshape(16, 16)
        uc, vc = oracle.correct(uz, vz, phi, fl)
        assert np.abs(oracle.divergence(uc, vc, fl)).max() < 1e-10
        # the iterative projection approaches the same (gauge-free) velocity;
        # plain Jacobi keeps a period-2 component (eigenvalue -1 of D^-1 W on
        # the bipartite grid graph), which the mean of two consecutive sweep
        # counts cancels (the correction is affine in phi)
        ra = oracle.project(u, v, fl, threshold=0.0, max_iters=0, fixed_iters=60000)
        rb = oracle.project(u, v, fl, threshold=0.0, max_iters=0, fixed_iters=60001)
        assert np.abs(0.5 * (ra["u"][0] + rb["u"][0]) - uc[0]).max() < 1e-8
        assert np.abs(0.5 * (ra["v"][0] + rb["v"][0]) - vc[0]).max() < 1e-8


def test_projection_leaves_closed_faces_exactly_zero():
    u, v, fl = small_case(8)
    res = oracle.project(u, v, fl, threshold=1e-3, max_iters=500)
    n = 8
    for j in range(n):
        for i in range(n + 1):
            if not (0 < i < n and fl[j, i - 1] == 0 and fl[j, i] == 0):
                assert res["u"][0, j, i] == 0.0
    for j in range(n + 1):
        for i in range(n):
            if not (0 < j < n and fl[j - 1, i] == 0 and fl[j, i] == 0):
                assert res["v"][0, j, i] == 0.0


def test_projection_is_idempotent():
    u, v, fl = small_case(8)
    r1 = oracle.project(u, v, fl, threshold=5e-3, max_iters=100000)
    assert r1["converged"][0] == 1
    r2 = oracle.project(r1["u"], r1["v"], fl, threshold=5e-3, max_iters=100000)
    # the corrected field already meets the threshold: zero sweeps, unchanged u
    assert r2["iters"][0] == 0
    assert np.array_equal(r2["u"], r1["u"]) and np.array_equal(r2["v"], r1["v"])
    assert np.all(r2["phi"] == 0)


def test_iteration_count_matches_dense_matrix_powers():
    u, v, fl = small_case(8, seed=11)
    uz, vz = oracle.zero_closed_faces(u, v, fl)
    div = oracle.divergence(uz, vz, fl)[0].ravel()
    Wm, n = dense_adjacency(fl)
    Dinv = np.where(n > 0, 1.0 / np.maximum(n, 1), 0.0)
    L = Wm - np.diag(n)
    fluid = fl.ravel() == 0
    phi = np.zeros(64)
    hist = []
    for _ in range(300):
        r = np.where(fluid, div - L @ phi, 0.0)
        hist.append(np.abs(r).sum() / 64)
        phi = Dinv * (Wm @ phi - div)
    hist = np.array(hist)
    for thr in [hist[0] * 1.01, hist[5] * 0.999, hist[40], hist[120] * 1.0001]:
        k_dense = int(np.argmax(hist <= thr))
        res = oracle.project(u, v, fl, threshold=thr, max_iters=1000, hist_len=300)
        assert res["iters"][0] == k_dense
        assert np.allclose(res["e_hist"][0, :k_dense + 1], hist[:k_dense + 1], rtol=1e-12,
                           atol=1e-15)


def test_cap_and_fixed_iteration_modes():
    u, v, fl = small_case(8)
    res = oracle.project(u, v, fl, threshold=0.0, max_iters=0)
    assert res["iters"][0] == 0 and res["converged"][0] == 0
    res = oracle.project(u, v, fl, threshold=0.0, max_iters=7)
    assert res["iters"][0] == 7 and res["converged"][0] == 0
    res = oracle.project(u, v, fl, threshold=1e9, max_iters=7)
    assert res["iters"][0] == 0 and res["converged"][0] == 1
    uz, vz = oracle.zero_closed_faces(u, v, fl)
    div = oracle.divergence(uz, vz, fl)
    phi = np.zeros((1, 8, 8))
    for _ in range(5):
        phi = oracle.jacobi_sweep(phi, div, fl)
    res = oracle.project(u, v, fl, threshold=0.0, max_iters=0, fixed_iters=5)
    assert np.array_equal(res["phi"], phi) and res["iters"][0] == 5


def test_initial_guess_counts_and_is_zeroed_on_solid_cells():
    u, v, fl = small_case(8)
    uz, vz = oracle.zero_closed_faces(u, v, fl)
    div = oracle.divergence(uz, vz, fl)[0].ravel()
    exact = np.linalg.lstsq(dense_laplacian(fl), div, rcond=None)[0].reshape(1, 8, 8)
    guess = exact.copy()
    guess[0][fl == 1] = 123.0      # garbage on solid cells is ignored
    res = oracle.project(u, v, fl, threshold=1e-9, max_iters=10, phi0=guess)
    assert res["iters"][0] == 0 and res["converged"][0] == 1
    assert np.all(res["phi"][0][fl == 1] == 0.0)


def test_p_is_scaled_phi():
    u, v, fl = small_case(8)
    res = oracle.project(u, v, fl, threshold=1e-4, max_iters=1000, dt=0.1, rho0=2.0)
    assert np.allclose(res["p"], res["phi"] * 2.0 / 0.1, rtol=1e-15, atol=0)


def test_e1_einf_of_corrected_velocity():
    u, v, fl = small_case(8)
    res = oracle.project(u, v, fl, threshold=1e-4, max_iters=1000)
    d = oracle.divergence(res["u"], res["v"], fl)[0]
    assert np.isclose(res["e1"][0], np.abs(d).mean(), rtol=1e-14)
    assert res["einf"][0] == np.abs(d).max()


def test_golden_path3_hand_derivation():
    g = json.load(open(os.path.join(GOLDEN, "path3_jacobi.json")))
    fl = np.zeros((g["ny"], g["nx"]), np.uint8)
    u = np.array(g["u_star"]); v = np.array(g["v_star"])
    div = oracle.divergence(u, v, fl)[0]
    assert np.array_equal(div, np.array(g["div"]))
    phi = np.zeros_like(div)
    for k, it in enumerate(g["jacobi_iterates"]):
        assert np.array_equal(phi, np.array(it))
        assert np.isclose(oracle.mean_abs_residual(phi, div, fl)[0], g["E1_of_iterates"][k],
                          rtol=1e-15)
        phi = oracle.jacobi_sweep(phi, div, fl)[0]
    ex = np.array(g["exact_phi_up_to_constant"])
    uc, vc = oracle.correct(u, v, ex, fl)
    assert np.array_equal(uc[0], np.array(g["exact_corrected_u"]))


def test_batched_grids_are_independent():
    u, v, fl = W.batched_vortex_case(3, 16)
    res = oracle.project(u, v, fl, threshold=1e-3, max_iters=300)
    for b in range(3):
        one = oracle.project(u[b], v[b], fl[b], threshold=1e-3, max_iters=300)
        assert one["iters"][0] == res["iters"][b]
        assert np.array_equal(one["u"][0], res["u"][b])


def test_plain_jacobi_error_floor_closed_form():
    """On the bipartite grid graph D^-1 W has the eigenvalue -1 with the
    checkerboard eigenvector s = (-1)^(i+j); its component never decays, and
    E_k tends to sum over fluid components of |sum_c s_c div_c| / (nx ny)."""
    from scipy import ndimage
    for seed, n in [(3, 8), (4, 12)]:
        u, v, fl = small_case(n, seed=seed)
        uz, vz = oracle.zero_closed_faces(u, v, fl)
        div = oracle.divergence(uz, vz, fl)[0]
        lab, ncomp = ndimage.label(fl == 0)
        s = (-1.0) ** np.add.outer(np.arange(n), np.arange(n))
        floor = sum(abs(np.sum((s * div)[lab == c])) for c in range(1, ncomp + 1)) / (n * n)
        res = oracle.project(u, v, fl, threshold=0.0, max_iters=40000, hist_len=40001)
        assert np.isclose(res["e_hist"][0, 40000], floor, rtol=1e-9)
        assert np.isclose(res["e_hist"][0, 39999], floor, rtol=1e-9)
