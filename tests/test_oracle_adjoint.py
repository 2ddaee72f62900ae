"""Pins of the projection adjoint oracle: central differences of a scalar
loss in FP64 and the transpose of the dense Jacobian of the forward map."""
import numpy as np

import oracle
from oracle import adjoint as AD
from paper_2109_09363_gb300 import workloads as W


def setup(n, seed):
    u, v = W.vortex_velocity(n, n, seed, n_vortices=5, width=(1.5, n / 4))
    fl = np.zeros((n, n), np.uint8)
    fl[n // 4:n // 2, n // 3:n // 2 + 1] = 1
    phi0 = np.random.default_rng(seed).standard_normal((n, n)) * (fl == 0)
    return u, v, fl, phi0


def loss(u, v, phi0, fl, a, b, c, k, dt, rho0):
    uo, vo, po = AD.project_fixed(u, v, phi0, fl, k, dt, rho0)
    return np.sum(uo * a) + np.sum(vo * b) + np.sum(po * c)


def test_adjoint_matches_central_differences():
    n, k, dt, rho0 = 12, 20, 0.1, 1.3
    u, v, fl, phi0 = setup(n, 3)
    rng = np.random.default_rng(4)
    a, b, c = (rng.standard_normal(s) for s in [(n, n + 1), (n + 1, n), (n, n)])
    gus, gvs, gphi = AD.project_fixed_adjoint(a[None], b[None], c[None], fl, k, dt, rho0)
    eps = 1e-6
    for _ in range(12):
        which = rng.integers(0, 3)
        arr = [u, v, phi0][which]
        idx = tuple(rng.integers(0, s) for s in arr.shape)
        ap, am = arr.copy(), arr.copy()
        ap[idx] += eps
        am[idx] -= eps
        args_p = [u, v, phi0]; args_p[which] = ap
        args_m = [u, v, phi0]; args_m[which] = am
        fd = (loss(*args_p, fl, a, b, c, k, dt, rho0) - loss(*args_m, fl, a, b, c, k, dt, rho0)) / (2 * eps)
        g = [gus[0], gvs[0], gphi[0]][which][idx]
        assert np.isclose(g, fd, rtol=1e-6, atol=1e-7), (which, idx, g, fd)


import pytest


@pytest.mark.parametrize("k", [0, 1, 7])
def test_adjoint_is_the_dense_jacobian_transpose(k):
    n, dt, rho0 = 6, 1.0, 1.0
    u, v, fl, phi0 = setup(n, 5)
    sizes = [u.size, v.size, phi0.size]
    nin = sum(sizes)
    base = np.concatenate([u.ravel(), v.ravel(), phi0.ravel()])

    def fwd(x):
        uu = x[:sizes[0]].reshape(u.shape)
        vv = x[sizes[0]:sizes[0] + sizes[1]].reshape(v.shape)
        pp = x[sizes[0] + sizes[1]:].reshape(phi0.shape)
        uo, vo, po = AD.project_fixed(uu, vv, pp, fl, k, dt, rho0)
        return np.concatenate([uo.ravel(), vo.ravel(), po.ravel()])

    f0 = fwd(base)
    J = np.zeros((f0.size, nin))
    for i in range(nin):
        e = base.copy()
        e[i] += 1.0
        J[:, i] = fwd(e) - f0   # the map is affine: exact columns
    rng = np.random.default_rng(6)
    g = rng.standard_normal(f0.size)
    gu = g[:u.size].reshape(u.shape)[None]
    gv = g[u.size:u.size + v.size].reshape(v.shape)[None]
    gp = g[u.size + v.size:].reshape(phi0.shape)[None]
    gus, gvs, gphi = AD.project_fixed_adjoint(gu, gv, gp, fl, k, dt, rho0)
    got = np.concatenate([gus.ravel(), gvs.ravel(), gphi.ravel()])
    exp = J.T @ g
    # including phi_0 on cells without an open face, whose column is zero
    assert np.allclose(got, exp, atol=1e-10)


def _dense_divergence(fl):
    """D (cells x faces, u faces then v faces in row-major order) of the
    open-face divergence, and the open-face indicator; built here by loops."""
    ny, nx = fl.shape
    nu = ny * (nx + 1)
    D = np.zeros((ny * nx, nu + (ny + 1) * nx))
    open_f = np.zeros(D.shape[1], bool)
    for j in range(ny):
        for i in range(1, nx):
            if fl[j, i - 1] == 0 and fl[j, i] == 0:
                f = j * (nx + 1) + i
                D[j * nx + i - 1, f] += 1.0   # east face of the left cell
                D[j * nx + i, f] -= 1.0       # west face of the right cell
                open_f[f] = True
    for j in range(1, ny):
        for i in range(nx):
            if fl[j - 1, i] == 0 and fl[j, i] == 0:
                f = nu + j * nx + i
                D[(j - 1) * nx + i, f] += 1.0
                D[j * nx + i, f] -= 1.0
                open_f[f] = True
    return D, open_f


def _components(fl):
    """Connected fluid components (4-neighbour flood fill) as cell lists."""
    ny, nx = fl.shape
    seen = np.zeros_like(fl, bool)
    comps = []
    for j0 in range(ny):
        for i0 in range(nx):
            if fl[j0, i0] or seen[j0, i0]:
                continue
            stack, cells = [(j0, i0)], []
            seen[j0, i0] = True
            while stack:
                j, i = stack.pop()
                cells.append((j, i))
                for jj, ii in ((j, i - 1), (j, i + 1), (j - 1, i), (j + 1, i)):
                    if 0 <= jj < ny and 0 <= ii < nx and not fl[jj, ii] and not seen[jj, ii]:
                        seen[jj, ii] = True
                        stack.append((jj, ii))
            comps.append(cells)
    return comps


def test_adjoint_tends_to_the_dense_solve_gradient():
    # As k grows, u = Z u* - G phi_k tends to the exact projection
    # (I - D^T (D D^T)^+ D) Z u* (G = -D^T on open faces), so dL/du* tends to
    # Z (I - D^T (D D^T)^+ D) g (the dense solve below).  Plain Jacobi never damps the checkerboard
    # mode (eigenvalue -1 on the bipartite grid graph), so g is taken
    # orthogonal to D^T s of every component's checkerboard s: the adjoint
    # sweeps then do not excite that mode and converge.
    n = 8
    fl = np.zeros((n, n), np.uint8)
    fl[2:4, 3:5] = 1
    fl[6, 1] = 1
    D, open_f = _dense_divergence(fl)
    g = np.random.default_rng(12).standard_normal(D.shape[1])
    for cells in _components(fl):
        s = np.zeros(n * n)
        for j, i in cells:
            s[j * n + i] = (-1.0) ** (i + j)
        a = D.T @ s
        if a @ a > 0:
            g -= (g @ a) / (a @ a) * a
    # minimum-norm least-squares solve of the singular Poisson system
    phi = np.linalg.lstsq(D @ D.T, D @ g, rcond=None)[0]
    assert np.abs(D @ D.T @ phi - D @ g).max() < 1e-12
    exact = open_f * (g - D.T @ phi)
    nu = n * (n + 1)
    gu = g[:nu].reshape(1, n, n + 1)
    gv = g[nu:].reshape(1, n + 1, n)
    err = []
    for k in (50, 400, 3000):
        gus, gvs, _ = AD.project_fixed_adjoint(gu, gv, None, fl, k)
        got = np.concatenate([gus.ravel(), gvs.ravel()])
        err.append(np.abs(got - exact).max())
    assert err[0] > err[1] > err[2]          # converging with k
    assert err[2] < 1e-10 * np.abs(exact).max()
