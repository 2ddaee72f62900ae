"""Pins of the open-top / prescribed-inflow projection oracle
(oracle/boundary.py): it reduces to the closed-box C oracle, its Jacobi
iteration converges to an independent dense direct solve (the exterior at
p = 0 makes the problem non-singular: no constant mode and no checkerboard
floor), the corrected field balances the inflow with the outflow through the
top (the discrete divergence theorem), and the prescribed faces are kept."""
import numpy as np
import pytest

import oracle
from oracle import boundary as BD
from paper_2109_09363_gb300 import workloads as W


def case(n=16, seed=3):
    u, v = W.vortex_velocity(n, n, seed, n_vortices=4, width=(1.5, n / 4))
    fl = np.zeros((n, n), np.uint8)
    fl[n // 4:n // 4 + 3, n // 3:n // 3 + 4] = 1
    fl[n - 4, 2] = 1
    return u, v, fl


def test_closed_box_is_the_c_oracle():
    u, v, fl = case(16)
    a = BD.project(u, v, fl, 1e-3, 500)
    b = oracle.project(u, v, fl, 1e-3, 500)
    assert a["iters"] == int(b["iters"][0])
    assert np.allclose(a["u"], b["u"][0], atol=1e-12, rtol=0)
    assert np.allclose(a["v"], b["v"][0], atol=1e-12, rtol=0)
    assert np.allclose(a["p"], b["p"][0], atol=1e-12, rtol=0)
    assert a["e1"] == pytest.approx(float(b["e1"][0]), rel=1e-10)


def dense_open_top(fl):
    """Dense Laplacian with the exterior beyond the top at phi = 0, built by
    loops over cells: A[c][c] = -(open faces), A[c][nb] = 1 per open face to
    a fluid neighbour."""
    ny, nx = fl.shape
    A = np.zeros((ny * nx, ny * nx))
    for j in range(ny):
        for i in range(nx):
            if fl[j, i]:
                A[j * nx + i, j * nx + i] = 1.0   # solid: phi = 0 there
                continue
            c = j * nx + i
            if j == 0:
                A[c, c] -= 1.0                   # open top face, exterior phi = 0
            for jj, ii in ((j, i - 1), (j, i + 1), (j - 1, i), (j + 1, i)):
                if 0 <= jj < ny and 0 <= ii < nx and not fl[jj, ii]:
                    A[c, c] -= 1.0
                    A[c, jj * nx + ii] += 1.0
    return A


def test_open_top_jacobi_converges_to_the_dense_solve():
    n = 12
    u, v, fl = case(n, 5)
    inflow = (4, 8)
    v = v.copy()
    v[n, 4:8] = -0.3
    ou, ov, pv = BD.faces(fl, True, inflow)
    ub, vb = np.where(ou, u, 0.0), np.where(ov | pv, v, 0.0)
    div = BD.divergence(ub, vb, ou, ov, pv)
    phi_exact = np.linalg.solve(dense_open_top(fl), np.where(fl == 0, div, 0.0).ravel())
    r = BD.project(u, v, fl, 0.0, 0, open_top=True, inflow=inflow, fixed_iters=16000)
    assert np.abs(r["p"].ravel() - phi_exact).max() < 1e-9 * np.abs(phi_exact).max()
    # no floor: E falls to roundoff, and the corrected field is divergence-free
    assert r["e_hist"][-1] < 1e-12
    assert r["e1"] < 1e-12


def test_inflow_leaves_through_the_top_and_prescribed_faces_are_kept():
    n = 16
    u, v, fl = case(n, 7)
    v = v.copy()
    v[n, 5:11] = -0.25            # injected upwards at U_in = 0.25
    r = BD.project(u, v, fl, 1e-12, 20000, open_top=True, inflow=(5, 11))
    assert r["converged"] == 1
    # sum of div over the box = bottom-boundary flux - top-boundary flux
    assert np.sum(r["v"][0, :]) == pytest.approx(np.sum(r["v"][n, :]), abs=n * n * 1e-11)
    assert np.sum(r["v"][n, :]) == pytest.approx(-0.25 * 6)
    assert np.array_equal(r["v"][n, 5:11], v[n, 5:11])
    assert not r["v"][n, :5].any() and not r["v"][n, 11:].any()
    # the top faces carry the outflow, the side walls stay closed
    assert np.all(r["u"][:, 0] == 0) and np.all(r["u"][:, n] == 0)
    assert np.sum(r["v"][0, :]) < 0


def test_correction_is_the_gradient_with_the_exterior_at_zero():
    n = 10
    u, v, fl = case(n, 9)
    phi = np.random.default_rng(2).standard_normal((n, n)) * (fl == 0)
    ou, ov, pv = BD.faces(fl, True, (2, 5))
    uo, vo = BD.correct(u, v, phi, ou, ov, pv)
    j, i = 0, 4
    assert fl[j, i] == 0 and ov[0, i]
    assert vo[0, i] == pytest.approx(v[0, i] - phi[0, i])
    j, i = 5, 6
    if ou[j, i]:
        assert uo[j, i] == pytest.approx(u[j, i] - (phi[j, i] - phi[j, i - 1]))
    assert vo[n, 3] == v[n, 3]
