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
