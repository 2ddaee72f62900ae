"""FP64 CPU oracle for the pressure projection of arXiv 2109.09363.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library in ``paper_2109_09363_gb300`` and never imports it.

The projection itself (mask, divergence, Jacobi to threshold, correction) is
plain C in ``oracle.c`` (built by :func:`build`); the networks, the advection
step, the adjoint and the training losses and optimiser are plain numpy
(``cnn.py``, ``advect.py``, ``adjoint.py``, ``train.py``).  All arithmetic is
FP64.

Functions that have no independent pin say so in their docstring ("parity
unpinned"); every other function is pinned by ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (gcc, OpenMP, -O2)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", src, "-o", _SO, "-lm"]
        subprocess.run(cmd, check=True)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_SO)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _u8(a):
    return np.ascontiguousarray(a, dtype=np.uint8)


def _shape(flags):
    flags = np.asarray(flags)
    if flags.ndim == 2:
        flags = flags[None]
    return flags.shape


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 = leave it); returns the count in use."""
    lib = _load()
    lib.or_set_threads.restype = ctypes.c_int
    return int(lib.or_set_threads(ctypes.c_int(n)))


def face_mask(flags):
    """Open-face bits per cell: 1 west, 2 east, 4 north (row j-1), 8 south (row j+1).

    A face is open when it is not on the domain boundary and both adjacent
    cells are fluid (Sec. 2.2: boolean geometry field, closed walls).
    """
    lib = _load()
    fl = _u8(flags).reshape(_shape(flags))
    B, ny, nx = fl.shape
    out = np.empty_like(fl)
    lib.or_face_mask(_p(fl), B, ny, nx, _p(out))
    return out


def zero_closed_faces(u, v, flags):
    """Copies of (u, v) with every closed face set to zero."""
    lib = _load()
    fl = _u8(flags).reshape(_shape(flags))
    B, ny, nx = fl.shape
    u = _f64(u).reshape(B, ny, nx + 1).copy()
    v = _f64(v).reshape(B, ny + 1, nx).copy()
    lib.or_zero_closed_faces(_p(u), _p(v), _p(fl), B, ny, nx)
    return u, v


def divergence(u, v, flags):
    """Forward-difference divergence of the open-face velocities (Eq. 3 right-hand side)."""
    lib = _load()
    fl = _u8(flags).reshape(_shape(flags))
    B, ny, nx = fl.shape
    u = _f64(u).reshape(B, ny, nx + 1)
    v = _f64(v).reshape(B, ny + 1, nx)
    out = np.empty((B, ny, nx))
    lib.or_divergence(_p(u), _p(v), _p(fl), B, ny, nx, _p(out))
    return out


def jacobi_sweep(phi, div, flags):
    """One Jacobi sweep of the masked Poisson operator (Sec. 2.2)."""
    lib = _load()
    fl = _u8(flags).reshape(_shape(flags))
    B, ny, nx = fl.shape
    phi = _f64(phi).reshape(B, ny, nx)
    div = _f64(div).reshape(B, ny, nx)
    out = np.empty((B, ny, nx))
    lib.or_jacobi_sweep(_p(phi), _p(div), _p(fl), B, ny, nx, _p(out))
    return out


def residual(phi, div, flags):
    """r = div - L phi on fluid cells, 0 on solid cells."""
    lib = _load()
    fl = _u8(flags).reshape(_shape(flags))
    B, ny, nx = fl.shape
    phi = _f64(phi).reshape(B, ny, nx)
    div = _f64(div).reshape(B, ny, nx)
    out = np.empty((B, ny, nx))
    lib.or_residual(_p(phi), _p(div), _p(fl), B, ny, nx, _p(out))
    return out


def mean_abs_residual(phi, div, flags):
    """E(phi) = sum |r| / (nx ny) per grid (E_1 of Sec. 4.1 for the corrected field)."""
    lib = _load()
    fl = _u8(flags).reshape(_shape(flags))
    B, ny, nx = fl.shape
    phi = _f64(phi).reshape(B, ny, nx)
    div = _f64(div).reshape(B, ny, nx)
    out = np.empty(B)
    lib.or_mean_abs_residual(_p(phi), _p(div), _p(fl), B, ny, nx, _p(out))
    return out


def correct(u, v, phi, flags):
    """u = u* - grad phi on open faces, 0 on closed ones (Eq. 2 with phi = dt p / rho0)."""
    lib = _load()
    fl = _u8(flags).reshape(_shape(flags))
    B, ny, nx = fl.shape
    u = _f64(u).reshape(B, ny, nx + 1).copy()
    v = _f64(v).reshape(B, ny + 1, nx).copy()
    phi = _f64(phi).reshape(B, ny, nx)
    lib.or_correct(_p(u), _p(v), _p(phi), _p(fl), B, ny, nx)
    return u, v


def div_norms(u, v, flags):
    """(E_1, E_inf) = (mean |div u|, max |div u|) per grid (Sec. 4.1)."""
    lib = _load()
    fl = _u8(flags).reshape(_shape(flags))
    B, ny, nx = fl.shape
    u = _f64(u).reshape(B, ny, nx + 1)
    v = _f64(v).reshape(B, ny + 1, nx)
    e1 = np.empty(B)
    einf = np.empty(B)
    lib.or_div_norms(_p(u), _p(v), _p(fl), B, ny, nx, _p(e1), _p(einf))
    return e1, einf


def project(u, v, flags, threshold, max_iters, dt=1.0, rho0=1.0, phi0=None, fixed_iters=0,
            hist_len=0):
    """Pressure projection of B grids (Sec. 2.2 and the hybrid rule of Sec. 3.3).

    Returns a dict with the corrected ``u``, ``v``, the scaled pressure ``phi``
    (= dt p / rho0), ``p``, ``iters`` (k*), ``converged``, ``e1``/``einf`` of the
    corrected velocity and, with ``hist_len`` > 0, ``e_hist`` = E_k for k <
    hist_len (NaN after the stop).
    """
    lib = _load()
    fl = _u8(flags).reshape(_shape(flags))
    B, ny, nx = fl.shape
    u = _f64(u).reshape(B, ny, nx + 1).copy()
    v = _f64(v).reshape(B, ny + 1, nx).copy()
    phi0a = None if phi0 is None else _f64(phi0).reshape(B, ny, nx)
    p = np.empty((B, ny, nx))
    phi = np.empty((B, ny, nx))
    iters = np.empty(B, np.int32)
    e1 = np.empty(B)
    einf = np.empty(B)
    conv = np.empty(B, np.uint8)
    hist = np.empty((B, max(hist_len, 1)))
    lib.or_project(_p(u), _p(v), _p(fl), B, ny, nx, ctypes.c_double(threshold),
                   ctypes.c_int(max_iters), ctypes.c_int(fixed_iters), ctypes.c_double(dt),
                   ctypes.c_double(rho0), _p(phi0a), _p(p), _p(phi), _p(iters), _p(e1),
                   _p(einf), _p(conv), _p(hist) if hist_len > 0 else None,
                   ctypes.c_int(hist_len))
    out = dict(u=u, v=v, p=p, phi=phi, iters=iters, e1=e1, einf=einf, converged=conv)
    if hist_len > 0:
        out["e_hist"] = hist
    return out


def jacobi_adjoint(g_phik, flags, k):
    """Transpose of the k-sweep map (phi_0, div) -> phi_k applied to g_phik.

    Returns (g_phi0, g_div).  The paper only says the gradient of the
    correction is known (Sec. 3.2); the transposes are derived from the
    forward sweep and pinned by finite differences and by a dense transpose.
    """
    lib = _load()
    fl = _u8(flags).reshape(_shape(flags))
    B, ny, nx = fl.shape
    g = _f64(g_phik).reshape(B, ny, nx)
    g_phi0 = np.empty((B, ny, nx))
    g_div = np.zeros((B, ny, nx))
    lib.or_jacobi_adjoint(_p(g), _p(fl), B, ny, nx, ctypes.c_int(k), _p(g_phi0), _p(g_div))
    return g_phi0, g_div
