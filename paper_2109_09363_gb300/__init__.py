"""GB300 (sm_103a) pressure projection of the hybrid CNN + Jacobi solver of
arXiv 2109.09363: Python binding of the C ABI declared in ``include/hproj.h``.

This module only marshals arguments: every step of the projection runs in the
CUDA kernels of ``libhproj.so``.  Arrays are torch tensors on the CUDA device
(PyTorch supplies device memory and the current stream); the functions keep
the names of the C entry points.  There is no CPU fallback: without the built
library or without a GB300 device the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
# HPROJ_LIBRARY selects another build of the same C ABI (e.g. a debug build)
LIB_PATH = os.environ.get("HPROJ_LIBRARY") or os.path.join(HERE, "libhproj.so")

_lib = None


class HprojError(RuntimeError):
    pass


HP_ERR_TIMEOUT = 7
HP_WARN_CNN_NONFINITE = 100


class hp_shape(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int32), ("ny", ctypes.c_int32), ("nx", ctypes.c_int32)]


class hp_project_params(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("fixed_iters", ctypes.c_int32), ("dt", ctypes.c_float), ("rho0", ctypes.c_float),
                ("temporal_block", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("sweep_kernel", ctypes.c_int32), ("open_top", ctypes.c_int32),
                ("inflow_x0", ctypes.c_int32), ("inflow_x1", ctypes.c_int32)]


class hp_plume_params(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_float), ("gravity", ctypes.c_float), ("rho_amb", ctypes.c_float),
                ("rho_in", ctypes.c_float), ("inlet_x0", ctypes.c_int32),
                ("inlet_x1", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("u_in", ctypes.c_float), ("open_top", ctypes.c_int32)]


_P = ctypes.c_void_p
_SIGS = {
    "hp_ctx_create": (ctypes.c_int, [ctypes.POINTER(_P), hp_shape, ctypes.c_int]),
    "hp_ctx_destroy": (None, [_P]),
    "hp_ctx_check": (ctypes.c_int, [_P]),
    "hp_trainer_check": (ctypes.c_int, [_P]),
    "hp_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "hp_last_cuda_error": (ctypes.c_char_p, []),
    "hp_face_mask": (ctypes.c_int, [_P, _P, hp_shape, _P]),
    "hp_divergence": (ctypes.c_int, [_P, _P, _P, _P, hp_shape, _P]),
    "hp_div_norms": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, hp_shape, _P]),
    "hp_project": (ctypes.c_int, [_P, _P, _P, _P, hp_shape, ctypes.POINTER(hp_project_params),
                                  _P, _P, _P, _P, _P, _P, _P, ctypes.c_int32, _P]),
    "hp_jacobi_sweeps": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int32, _P, hp_shape, _P]),
    "hp_jacobi_target": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32, _P, hp_shape, _P]),
    "hp_div_norms_noalloc": (ctypes.c_int, [_P, _P, _P, _P, _P, hp_shape, _P]),
    "hp_resident_clusters": (ctypes.c_int32, [_P, hp_shape]),
    "hp_advect_step": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, hp_shape,
                                      ctypes.POINTER(hp_plume_params), _P]),
    "hp_plume_head": (ctypes.c_int, [_P, hp_shape, ctypes.c_float, ctypes.c_float, _P, _P]),
    "hp_conv3x3_bf16": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, _P, _P]),
    "hp_project_adjoint": (ctypes.c_int, [_P, _P, _P, _P, _P, hp_shape, ctypes.c_int32,
                                          ctypes.c_float, ctypes.c_float, _P, _P, _P, _P]),
    "hp_trainer_create": (ctypes.c_int, [ctypes.POINTER(_P), _P, hp_shape]),
    "hp_trainer_destroy": (None, [_P]),
    "hp_trainer_gradient": (ctypes.c_int, [_P, _P, _P, _P, hp_shape, ctypes.c_float, _P, _P, _P]),
    "hp_trainer_step": (ctypes.c_int, [_P, _P, _P, _P, hp_shape, ctypes.c_void_p, _P, _P]),
    "hp_trainer_sync_params": (ctypes.c_int, [_P]),
    "hp_trainer_get_state": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_int64)]),
    "hp_trainer_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "hp_trainer_load": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "hp_cnn_save": (ctypes.c_int, [_P, ctypes.c_char_p]),
    "hp_cnn_load": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_char_p, hp_shape, ctypes.c_int]),
    "hp_trainer_pdnn_gradient": (ctypes.c_int, [_P, _P, _P, _P, hp_shape, ctypes.c_int32, _P,
                                                _P, _P]),
    "hp_trainer_pdnn_step": (ctypes.c_int, [_P, _P, _P, _P, hp_shape, ctypes.c_int32,
                                            ctypes.c_void_p, _P, _P]),
    "hp_cnn_param_count": (ctypes.c_int64, []),
    "hp_cnn_arch_param_count": (ctypes.c_int64, [ctypes.c_int32]),
    "hp_cnn_create": (ctypes.c_int, [ctypes.POINTER(_P), hp_shape, ctypes.c_int]),
    "hp_cnn_create_arch": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int32, hp_shape,
                                          ctypes.c_int]),
    "hp_cnn_get_arch": (ctypes.c_int32, [_P]),
    "hp_cnn_destroy": (None, [_P]),
    "hp_cnn_set_params": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "hp_cnn_check": (ctypes.c_int, [_P]),
    "hp_cnn_set_wait_limit": (ctypes.c_int, [_P, ctypes.c_uint32]),
    "hp_cnn_get_params": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
    "hp_cnn_forward": (ctypes.c_int, [_P, _P, _P, _P, _P, hp_shape, _P]),
    "hp_project_hybrid": (ctypes.c_int, [_P, _P, _P, _P, _P, hp_shape,
                                         ctypes.POINTER(hp_project_params), _P, _P, _P, _P, _P,
                                         _P, ctypes.c_int32, _P]),
}


def load_library(path: str = LIB_PATH):
    """Load libhproj.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise HprojError(f"{path} is missing: run __graft_entry__.build() first")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int):
    if rc != 0:
        lib = load_library()
        msg = lib.hp_status_string(rc).decode()
        err = lib.hp_last_cuda_error().decode()
        raise HprojError(f"hproj status {rc} ({msg}) {err}")


def _torch():
    import torch
    return torch


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise HprojError("hproj takes CUDA tensors only")
    if not t.is_contiguous():
        raise HprojError("hproj takes contiguous tensors only")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _shape_of_flags(flags):
    if flags.dim() != 3:
        raise HprojError("flags must be [B][ny][nx]")
    B, ny, nx = flags.shape
    return hp_shape(B, ny, nx)


def _check_dtype(t, dtype, shape, name):
    if t is None:
        return
    if t.dtype != dtype:
        raise HprojError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise HprojError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")


class Context:
    """Workspaces for grids up to (batch, ny, nx); owns device memory."""

    def __init__(self, batch: int, ny: int, nx: int, device: int | None = None):
        torch = _torch()
        lib = load_library()
        dev = torch.cuda.current_device() if device is None else device
        self.device = dev
        self._h = _P()
        _check(lib.hp_ctx_create(ctypes.byref(self._h), hp_shape(batch, ny, nx), dev))

    @property
    def handle(self):
        return self._h

    def check(self):
        """Raise if a kernel wrote into a guard zone past one of this
        context's workspaces (synchronises the device)."""
        _check(load_library().hp_ctx_check(self._h))

    def close(self):
        if self._h:
            load_library().hp_ctx_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class ProjectParams:
    threshold: float = 1e-3
    max_iters: int = 2000
    fixed_iters: int = 0
    dt: float = 1.0
    rho0: float = 1.0
    temporal_block: int = 0
    use_graph: int = 1
    sweep_kernel: int = 0
    open_top: int = 0      # 1: the top boundary is open to p = 0 (outflow)
    inflow: tuple = (0, 0)  # bottom-boundary v faces of these columns keep their velocity

    def c(self):
        return hp_project_params(self.threshold, self.max_iters, self.fixed_iters, self.dt,
                                 self.rho0, self.temporal_block, self.use_graph,
                                 self.sweep_kernel, self.open_top, self.inflow[0],
                                 self.inflow[1])


def hp_face_mask(flags, mask_out=None, stream=None):
    torch = _torch()
    s = _shape_of_flags(flags)
    _check_dtype(flags, torch.uint8, flags.shape, "flags")
    if mask_out is None:
        mask_out = torch.empty_like(flags)
    _check(load_library().hp_face_mask(_ptr(flags), _ptr(mask_out), s, _stream(stream)))
    return mask_out


def hp_divergence(u, v, flags, div_out=None, stream=None):
    torch = _torch()
    s = _shape_of_flags(flags)
    B, ny, nx = flags.shape
    _check_dtype(u, torch.float32, (B, ny, nx + 1), "u")
    _check_dtype(v, torch.float32, (B, ny + 1, nx), "v")
    if div_out is None:
        div_out = torch.empty((B, ny, nx), dtype=torch.float32, device=u.device)
    _check(load_library().hp_divergence(_ptr(u), _ptr(v), _ptr(flags), _ptr(div_out), s,
                                        _stream(stream)))
    return div_out


def hp_resident_clusters(ctx: Context, batch: int, ny: int, nx: int) -> int:
    """Grids of this shape the grid-resident sweep kernel (sweep_kernel = 4)
    holds at once; 0 when it cannot run the shape (hp_project then uses the
    temporally blocked kernel)."""
    return int(load_library().hp_resident_clusters(ctx.handle, hp_shape(batch, ny, nx)))


def hp_div_norms(ctx: Context, u, v, flags, stream=None):
    torch = _torch()
    s = _shape_of_flags(flags)
    B, ny, nx = flags.shape
    _check_dtype(u, torch.float32, (B, ny, nx + 1), "u")
    _check_dtype(v, torch.float32, (B, ny + 1, nx), "v")
    e1 = torch.empty(B, dtype=torch.float64, device=u.device)
    einf = torch.empty(B, dtype=torch.float64, device=u.device)
    _check(load_library().hp_div_norms(ctx.handle, _ptr(u), _ptr(v), _ptr(flags), _ptr(e1),
                                       _ptr(einf), s, _stream(stream)))
    return e1, einf


def hp_div_norms_noalloc(u, v, flags, e1_out=None, einf_out=None, stream=None):
    """E_1 and E_inf like hp_div_norms, without a context: for callers that
    cannot allocate device memory for workspaces.  The library keeps a fixed
    scratch array on each device instead; calls that overlap on the GPU race.
    The output tensors may be passed in so that the call allocates nothing."""
    torch = _torch()
    s = _shape_of_flags(flags)
    B, ny, nx = flags.shape
    _check_dtype(u, torch.float32, (B, ny, nx + 1), "u")
    _check_dtype(v, torch.float32, (B, ny + 1, nx), "v")
    if e1_out is None:
        e1_out = torch.empty(B, dtype=torch.float64, device=u.device)
    if einf_out is None:
        einf_out = torch.empty(B, dtype=torch.float64, device=u.device)
    _check(load_library().hp_div_norms_noalloc(_ptr(u), _ptr(v), _ptr(flags), _ptr(e1_out),
                                               _ptr(einf_out), s, _stream(stream)))
    return e1_out, einf_out


def hp_project(ctx: Context, u, v, flags, params: ProjectParams, phi0=None, p_out=None,
               hist_len: int = 0, stream=None, out=None):
    """Project (u, v) in place; returns a dict of device tensors
    p, iters, e1, einf, converged (and e_hist when hist_len > 0)."""
    torch = _torch()
    s = _shape_of_flags(flags)
    B, ny, nx = flags.shape
    _check_dtype(u, torch.float32, (B, ny, nx + 1), "u")
    _check_dtype(v, torch.float32, (B, ny + 1, nx), "v")
    _check_dtype(phi0, torch.float32, (B, ny, nx), "phi0")
    dev = u.device
    if out is None:
        out = {
            "p": p_out if p_out is not None else torch.empty((B, ny, nx), dtype=torch.float32,
                                                             device=dev),
            "iters": torch.empty(B, dtype=torch.int32, device=dev),
            "e1": torch.empty(B, dtype=torch.float64, device=dev),
            "einf": torch.empty(B, dtype=torch.float64, device=dev),
            "converged": torch.empty(B, dtype=torch.uint8, device=dev),
        }
        if hist_len > 0:
            out["e_hist"] = torch.full((B, hist_len), float("nan"), dtype=torch.float64,
                                       device=dev)
    prm = params.c()
    hist = out.get("e_hist")
    _check(load_library().hp_project(
        ctx.handle, _ptr(u), _ptr(v), _ptr(flags), s, ctypes.byref(prm), _ptr(phi0),
        _ptr(out["p"]), _ptr(out["iters"]), _ptr(out["e1"]), _ptr(out["einf"]),
        _ptr(out["converged"]), _ptr(hist), ctypes.c_int32(hist.shape[1] if hist is not None
                                                           else 0), _stream(stream)))
    return out


def hp_jacobi_sweeps(ctx: Context, phi_in, div, flags, n: int, phi_out=None, with_e=False,
                     stream=None):
    torch = _torch()
    s = _shape_of_flags(flags)
    B, ny, nx = flags.shape
    _check_dtype(phi_in, torch.float32, (B, ny, nx), "phi_in")
    _check_dtype(div, torch.float32, (B, ny, nx), "div")
    if phi_out is None:
        phi_out = torch.empty_like(phi_in)
    e = torch.empty((B, n), dtype=torch.float64, device=phi_in.device) if with_e else None
    _check(load_library().hp_jacobi_sweeps(ctx.handle, _ptr(phi_in), _ptr(div), _ptr(flags),
                                           _ptr(phi_out), ctypes.c_int32(n), _ptr(e), s,
                                           _stream(stream)))
    return (phi_out, e) if with_e else phi_out


def hp_jacobi_target(ctx: Context, div, flags, n: int, target_out=None, stream=None):
    """Training target of the plain solver: n Jacobi sweeps from zero on the
    right-hand side div, then the mean of phi_n and phi_{n+1}."""
    torch = _torch()
    s = _shape_of_flags(flags)
    B, ny, nx = flags.shape
    _check_dtype(div, torch.float32, (B, ny, nx), "div")
    if target_out is None:
        target_out = torch.empty_like(div)
    _check(load_library().hp_jacobi_target(ctx.handle, _ptr(div), _ptr(flags), ctypes.c_int32(n),
                                           _ptr(target_out), s, _stream(stream)))
    return target_out


@dataclass
class PlumeParams:
    dt: float = 0.1
    gravity: float = -0.002
    rho_amb: float = 1.0
    rho_in: float = 1.1
    inlet_x0: int = 0
    inlet_x1: int = 0
    scheme: int = 0  # 0 first-order semi-Lagrangian, 1 MacCormack
    u_in: float = 0.0  # injection speed on the inlet faces (upwards)
    open_top: int = 0  # 1: the top boundary is open (outflow)

    def c(self):
        return hp_plume_params(self.dt, self.gravity, self.rho_amb, self.rho_in, self.inlet_x0,
                               self.inlet_x1, self.scheme, self.u_in, self.open_top)


def hp_advect_step(u, v, rho, flags, params: PlumeParams, u_out=None, v_out=None, rho_out=None,
                   stream=None):
    """Driver step (inlet, semi-Lagrangian advection, buoyancy); returns
    (u*, v*, rho) as new device tensors unless outputs are given."""
    torch = _torch()
    s = _shape_of_flags(flags)
    B, ny, nx = flags.shape
    _check_dtype(u, torch.float32, (B, ny, nx + 1), "u")
    _check_dtype(v, torch.float32, (B, ny + 1, nx), "v")
    _check_dtype(rho, torch.float32, (B, ny, nx), "rho")
    u_out = torch.empty_like(u) if u_out is None else u_out
    v_out = torch.empty_like(v) if v_out is None else v_out
    rho_out = torch.empty_like(rho) if rho_out is None else rho_out
    prm = params.c()
    _check(load_library().hp_advect_step(_ptr(u), _ptr(v), _ptr(rho), _ptr(flags), _ptr(u_out),
                                         _ptr(v_out), _ptr(rho_out), s, ctypes.byref(prm),
                                         _stream(stream)))
    return u_out, v_out, rho_out


def hp_plume_head(rho, rho_amb: float = 1.0, contrast: float = 0.01, out=None, stream=None):
    """Plume head per grid: int32 [B][3] = (smallest row, smallest column,
    largest column) of the cells with |rho - rho_amb| >= contrast; (ny, nx, -1)
    when there is none."""
    torch = _torch()
    if rho.dim() != 3:
        raise HprojError("rho must be [B][ny][nx]")
    _check_dtype(rho, torch.float32, tuple(rho.shape), "rho")
    B, ny, nx = rho.shape
    out = torch.empty((B, 3), dtype=torch.int32, device=rho.device) if out is None else out
    _check(load_library().hp_plume_head(_ptr(rho), hp_shape(B, ny, nx), float(rho_amb),
                                        float(contrast), _ptr(out), _stream(stream)))
    return out


def hp_conv3x3_bf16(x, w, bias, relu: bool, y=None, err=None, stream=None):
    """y = [relu](conv3x3_replicate(x, w) + bias) on the tensor cores.
    x: bf16 [B][H][W][Cin]; w: bf16 [3][3][Cout][Cin]; bias: float32 [Cout]."""
    torch = _torch()
    B, H, W, cin = x.shape
    cout = w.shape[2]
    if x.dtype != torch.bfloat16 or w.dtype != torch.bfloat16 or bias.dtype != torch.float32:
        raise HprojError("x, w must be bfloat16 and bias float32")
    if tuple(w.shape) != (3, 3, cout, cin):
        raise HprojError("w must be [3][3][cout][cin]")
    if y is None:
        y = torch.empty((B, H, W, cout), dtype=torch.bfloat16, device=x.device)
    _check(load_library().hp_conv3x3_bf16(_ptr(x), _ptr(w), _ptr(bias), _ptr(y), B, H, W, cin,
                                          cout, int(bool(relu)), _ptr(err), _stream(stream)))
    return y


def hp_project_adjoint(ctx: Context, gu, gv, gp, flags, k: int, dt: float = 1.0,
                       rho0: float = 1.0, stream=None):
    """(dL/du*, dL/dv*, dL/dphi_0) of the fixed-count projection."""
    torch = _torch()
    s = _shape_of_flags(flags)
    B, ny, nx = flags.shape
    _check_dtype(gu, torch.float32, (B, ny, nx + 1), "gu")
    _check_dtype(gv, torch.float32, (B, ny + 1, nx), "gv")
    _check_dtype(gp, torch.float32, (B, ny, nx), "gp")
    gus, gvs = torch.empty_like(gu), torch.empty_like(gv)
    gphi = torch.empty((B, ny, nx), dtype=torch.float32, device=gu.device)
    _check(load_library().hp_project_adjoint(ctx.handle, _ptr(gu), _ptr(gv), _ptr(gp),
                                             _ptr(flags), s, int(k), float(dt), float(rho0),
                                             _ptr(gus), _ptr(gvs), _ptr(gphi), _stream(stream)))
    return gus, gvs, gphi


CNN_ARCHS = {"multiscale": 0, "smallscale": 1, "monoscale": 2, "unet": 3}  # hp_cnn_arch


class CNN:
    """CNN weights and workspace on the device (hp_cnn): the MultiScale, its
    narrower SmallScale variant, the feed-forward MonoScale or the Unet (Sec.
    3.1; forward and hybrid projection only, grid sizes multiples of 16)."""

    def __init__(self, batch: int, ny: int, nx: int, device: int | None = None, params=None,
                 arch: str = "multiscale", path: str | None = None):
        """A new network; with `path`, the architecture and parameters of a
        checkpoint file (hp_cnn_load) instead of `arch` and `params`."""
        torch = _torch()
        lib = load_library()
        dev = torch.cuda.current_device() if device is None else device
        self._h = _P()
        if path is not None:
            _check(lib.hp_cnn_load(ctypes.byref(self._h), os.fsencode(path),
                                   hp_shape(batch, ny, nx), dev))
            code = int(lib.hp_cnn_get_arch(self._h))
            arch = next(a for a, c in CNN_ARCHS.items() if c == code)
        elif arch not in CNN_ARCHS:
            raise ValueError(f"arch must be one of {sorted(CNN_ARCHS)}")
        else:
            _check(lib.hp_cnn_create_arch(ctypes.byref(self._h), CNN_ARCHS[arch],
                                          hp_shape(batch, ny, nx), dev))
        self.arch = arch
        self.n_params = CNN.param_count(arch)
        if params is not None:
            self.set_params(params)

    def save(self, path: str):
        """Checkpoint file of the architecture and parameters (hp_cnn_save)."""
        _check(load_library().hp_cnn_save(self._h, os.fsencode(path)))

    @staticmethod
    def param_count(arch: str = "multiscale") -> int:
        if arch not in CNN_ARCHS:
            raise ValueError(f"arch must be one of {sorted(CNN_ARCHS)}")
        return int(load_library().hp_cnn_arch_param_count(CNN_ARCHS[arch]))

    @property
    def handle(self):
        return self._h

    def set_params(self, flat):
        import numpy as np
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(load_library().hp_cnn_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p),
                                                a.size))

    def check(self):
        """Raise if a tensor-core wait of this network's kernels timed out
        since the last check (synchronises the device).  Returns
        HP_WARN_CNN_NONFINITE (100) when a hybrid projection replaced a
        non-finite guess by zero since the last check, else 0."""
        rc = load_library().hp_cnn_check(self._h)
        if rc == HP_WARN_CNN_NONFINITE:
            return rc
        _check(rc)
        return 0

    def set_wait_limit(self, polls: int):
        """Polls of each bounded pipeline wait of the tensor-core kernels
        (0 = the compiled limit)."""
        _check(load_library().hp_cnn_set_wait_limit(self._h, int(polls)))

    def get_params(self):
        import numpy as np
        a = np.empty(self.n_params, dtype=np.float32)
        _check(load_library().hp_cnn_get_params(self._h, a.ctypes.data_as(ctypes.c_void_p),
                                                a.size))
        return a

    def close(self):
        if self._h:
            load_library().hp_cnn_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class hp_train_params(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float), ("lambda_div", ctypes.c_float)]


class Trainer:
    """Adam training of a CNN on the device (hp_trainer)."""

    def __init__(self, cnn: CNN, batch: int, ny: int, nx: int):
        self.cnn = cnn
        self._h = _P()
        _check(load_library().hp_trainer_create(ctypes.byref(self._h), cnn.handle,
                                                hp_shape(batch, ny, nx)))

    def gradient(self, div, flags, target, lambda_div=0.1, stream=None):
        torch = _torch()
        s = _shape_of_flags(flags)
        g = torch.empty(self.cnn.n_params, dtype=torch.float32, device=div.device)
        loss = torch.empty(1, dtype=torch.float64, device=div.device)
        _check(load_library().hp_trainer_gradient(self._h, _ptr(div), _ptr(flags), _ptr(target),
                                                  s, float(lambda_div), _ptr(g), _ptr(loss),
                                                  _stream(stream)))
        return g, loss

    def step(self, div, flags, target, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
             lambda_div=0.1, loss_out=None, stream=None):
        torch = _torch()
        s = _shape_of_flags(flags)
        if loss_out is None:
            loss_out = torch.empty(1, dtype=torch.float64, device=div.device)
        prm = hp_train_params(lr, beta1, beta2, eps, lambda_div)
        _check(load_library().hp_trainer_step(self._h, _ptr(div), _ptr(flags), _ptr(target), s,
                                              ctypes.cast(ctypes.byref(prm), ctypes.c_void_p),
                                              _ptr(loss_out), _stream(stream)))
        return loss_out

    def pdnn_gradient(self, div, flags, weight, norm=1, stream=None):
        """Gradient and value of the physics-driven loss (Sec. 3.2, Eq. 4):
        sum_b weight[b] * mean |div u_b|^norm, u_b corrected by the network."""
        torch = _torch()
        s = _shape_of_flags(flags)
        _check_dtype(weight, torch.float32, (flags.shape[0],), "weight")
        g = torch.empty(self.cnn.n_params, dtype=torch.float32, device=div.device)
        loss = torch.empty(1, dtype=torch.float64, device=div.device)
        _check(load_library().hp_trainer_pdnn_gradient(self._h, _ptr(div), _ptr(flags),
                                                       _ptr(weight), s, int(norm), _ptr(g),
                                                       _ptr(loss), _stream(stream)))
        return g, loss

    def pdnn_step(self, div, flags, weight, norm=1, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                  loss_out=None, stream=None):
        torch = _torch()
        s = _shape_of_flags(flags)
        _check_dtype(weight, torch.float32, (flags.shape[0],), "weight")
        if loss_out is None:
            loss_out = torch.empty(1, dtype=torch.float64, device=div.device)
        prm = hp_train_params(lr, beta1, beta2, eps, 0.0)
        _check(load_library().hp_trainer_pdnn_step(self._h, _ptr(div), _ptr(flags), _ptr(weight),
                                                   s, int(norm),
                                                   ctypes.cast(ctypes.byref(prm), ctypes.c_void_p),
                                                   _ptr(loss_out), _stream(stream)))
        return loss_out

    def sync_params(self):
        _check(load_library().hp_trainer_sync_params(self._h))

    def check(self):
        """Raise on overwritten guard zones of the trainer's or its network's
        workspaces or a timed-out wait (synchronises the device)."""
        rc = load_library().hp_trainer_check(self._h)
        if rc != HP_WARN_CNN_NONFINITE:
            _check(rc)

    def state(self):
        """(masters, m, v, step): the FP32 masters, the Adam moments (numpy,
        network parameter order) and the number of Adam steps taken."""
        import numpy as np
        n = self.cnn.n_params
        w, m, v = (np.empty(n, dtype=np.float32) for _ in range(3))
        step = ctypes.c_int64(0)
        _check(load_library().hp_trainer_get_state(
            self._h, w.ctypes.data_as(ctypes.c_void_p), m.ctypes.data_as(ctypes.c_void_p),
            v.ctypes.data_as(ctypes.c_void_p), ctypes.byref(step)))
        return w, m, v, int(step.value)

    def save(self, path: str):
        """Checkpoint file of the masters, Adam moments and step (hp_trainer_save)."""
        _check(load_library().hp_trainer_save(self._h, os.fsencode(path)))

    def load(self, path: str):
        """Restore masters, moments and step from a checkpoint (hp_trainer_load)."""
        _check(load_library().hp_trainer_load(self._h, os.fsencode(path)))

    def close(self):
        if self._h:
            load_library().hp_trainer_destroy(self._h)
            self._h = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hp_cnn_forward(cnn: CNN, div, flags, phi_hat=None, s_out=None, stream=None):
    torch = _torch()
    s = _shape_of_flags(flags)
    B, ny, nx = flags.shape
    _check_dtype(div, torch.float32, (B, ny, nx), "div")
    phi_hat = torch.empty_like(div) if phi_hat is None else phi_hat
    s_out = torch.empty(B, dtype=torch.float32, device=div.device) if s_out is None else s_out
    _check(load_library().hp_cnn_forward(cnn.handle, _ptr(div), _ptr(flags), _ptr(phi_hat),
                                         _ptr(s_out), s, _stream(stream)))
    return phi_hat, s_out


def hp_project_hybrid(ctx: Context, cnn: CNN, u, v, flags, params: ProjectParams, hist_len=0,
                      stream=None, out=None):
    torch = _torch()
    s = _shape_of_flags(flags)
    B, ny, nx = flags.shape
    _check_dtype(u, torch.float32, (B, ny, nx + 1), "u")
    _check_dtype(v, torch.float32, (B, ny + 1, nx), "v")
    dev = u.device
    if out is None:
        out = {"p": torch.empty((B, ny, nx), dtype=torch.float32, device=dev),
               "iters": torch.empty(B, dtype=torch.int32, device=dev),
               "e1": torch.empty(B, dtype=torch.float64, device=dev),
               "einf": torch.empty(B, dtype=torch.float64, device=dev),
               "converged": torch.empty(B, dtype=torch.uint8, device=dev)}
        if hist_len > 0:
            out["e_hist"] = torch.full((B, hist_len), float("nan"), dtype=torch.float64,
                                       device=dev)
    prm = params.c()
    hist = out.get("e_hist")
    _check(load_library().hp_project_hybrid(
        ctx.handle, cnn.handle, _ptr(u), _ptr(v), _ptr(flags), s, ctypes.byref(prm),
        _ptr(out["p"]), _ptr(out["iters"]), _ptr(out["e1"]), _ptr(out["einf"]),
        _ptr(out["converged"]), _ptr(hist), ctypes.c_int32(hist.shape[1] if hist is not None
                                                           else 0), _stream(stream)))
    return out


def exported_symbols():
    """Names of the functions declared in include/hproj.h (parsed from the header)."""
    import re
    hdr = os.path.join(HERE, "..", "include", "hproj.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:hp_status|void|int64_t|int32_t|const char \*)\s*(hp_\w+)\s*\(",
                                 txt, re.M)))
