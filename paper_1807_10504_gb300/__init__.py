"""GB300 (sm_103a) immersed-boundary projection library: Python binding.

Argument marshalling only: every step of the path runs in the CUDA library
``libibgb300.so`` (C ABI in ``include/ib.h``).  Torch tensors provide device
memory and the stream.  There is no CPU fallback: if the library is missing or
no GPU is present, calls raise.

Names follow the C ABI: ``ib_init``, ``ib_interp``, ``ib_spread``,
``mg_setup``, ``mg_solve``, ``ns_step`` and the ``ib_op_*`` verification
operators.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libibgb300.so")

IB_OK, IB_EINVAL, IB_ENOMEM, IB_ENOTCONV, IB_ENAN, IB_EMARKER, IB_ECUDA = range(7)
STATUS = {0: "IB_OK", 1: "IB_EINVAL", 2: "IB_ENOMEM", 3: "IB_ENOTCONV", 4: "IB_ENAN",
          5: "IB_EMARKER", 6: "IB_ECUDA"}
FIELDS = {"u": 0, "v": 1, "p": 2, "H": 3, "rho": 4, "bx": 5, "by": 6, "Fx": 7, "Fy": 8,
          "b": 9, "mu": 10, "us": 11, "vs": 12}

EXPORTS = [
    "ib_init", "ib_destroy", "ib_last_error", "ib_set_markers", "ib_get_markers",
    "ib_num_markers", "ib_get_field", "ib_set_field", "ib_marker_geometry", "ib_marker_sort",
    "ib_interp", "ib_spread", "ib_heaviside", "ib_relocate", "mg_setup", "mg_solve",
    "ns_step", "ib_last_solve", "ib_save", "ib_load", "ib_op_coeffs", "ib_op_residual",
    "ib_op_rbgs", "ib_op_restrict_residual", "ib_op_prolong_add", "ib_op_coarsen_beta",
    "ib_op_rhs", "ib_op_correct", "ib_op_predictor", "ib_launch_count", "ib_profile_begin",
    "ib_profile_end", "ib_bench_kernel", "mg_solve_noalloc", "cnn_init", "cnn_destroy", "cnn_num_params",
    "cnn_get_params", "cnn_set_params", "cnn_grad", "cnn_train_step", "cnn_infer",
    "ib_attach_cnn", "ib_use_graphs", "cnn_set_scale", "cnn_get_scale", "cnn_set_coarsen",
    "ib_op_predictor_axi", "ib_op_rhs_axi", "ib_op_axi_weights", "ib_frame_state",
    "ib_mass_correct", "ib_op_cn_solve", "ns_step_io", "mg_solve_noalloc_error",
    "ib_debug_stall_staging", "ib_probe_fp64", "cnn_fit_scale", "cnn_train",
    "cnn_set_tensor_path",
]


class IBError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ib_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("h", C.c_double), ("x0", C.c_double),
                ("y0", C.c_double), ("rho_g", C.c_double), ("rho_l", C.c_double),
                ("mu_g", C.c_double), ("mu_l", C.c_double), ("sigma", C.c_double),
                ("gx", C.c_double), ("gy", C.c_double), ("kernel", C.c_int32),
                ("spread", C.c_int32), ("precision", C.c_int32), ("tol", C.c_double),
                ("max_cycles", C.c_int32), ("nu1", C.c_int32), ("nu2", C.c_int32),
                ("relocate_every", C.c_int32), ("axisym", C.c_int32), ("frame", C.c_int32),
                ("c1", C.c_double), ("c2", C.c_double), ("mass_every", C.c_int32),
                ("mass_tol", C.c_double), ("viscous", C.c_int32), ("cn_sweeps", C.c_int32),
                ("indicator", C.c_int32)]


_lib = None
_P = C.c_void_p
_i32, _d = C.c_int32, C.c_double


def build(force=False):
    from . import _build
    return _build.build(force=force)


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise IBError(IB_ECUDA, f"CUDA library not built: {LIB_PATH} (run build())")
        L = C.CDLL(LIB_PATH)
        sig = {
            "ib_init": [C.POINTER(_P), C.POINTER(ib_config), _P, _P, _P, _i32, _P],
            "ib_set_markers": [_P, _P, _P, C.c_int], "ib_get_markers": [_P, _P, _P, C.c_int],
            "ib_get_field": [_P, C.c_int, _P, C.c_int], "ib_set_field": [_P, C.c_int, _P, C.c_int],
            "ib_marker_geometry": [_P, _P, _P, _P, _P], "ib_marker_sort": [_P, _P, _P, _P],
            "ib_interp": [_P, _P, _P, _P, _P], "ib_spread": [_P, C.c_int, _P, _P, _P, _P],
            "ib_heaviside": [_P, _P], "ib_relocate": [_P], "mg_setup": [_P, _P, _P],
            "mg_solve": [_P, _P, _P, C.c_int, _d, C.c_int, C.POINTER(C.c_int), C.POINTER(_d)],
            "ns_step": [_P, _d, C.c_int, C.c_int],
            "ns_step_io": [_P, _d, C.c_int, _P, _P, _P, _P, _P],
            "ib_last_solve": [_P, C.POINTER(C.c_int), C.POINTER(_d)],
            "ib_save": [_P, C.c_char_p], "ib_load": [_P, C.c_char_p],
            "ib_op_coeffs": [_i32, _i32, _d, _d, _d, _d, _P, _P, _P, _P, _P, _P],
            "ib_op_residual": [_i32, _i32, _d, _P, _P, _P, _P, _P, _P],
            "ib_op_rbgs": [_i32, _i32, _d, _P, _P, _P, _P, _i32, _P],
            "ib_op_restrict_residual": [_i32, _i32, _d, _P, _P, _P, _P, _P, _P],
            "ib_op_prolong_add": [_i32, _i32, _P, _P, _P],
            "ib_op_coarsen_beta": [_i32, _i32, _P, _P, _P, _P, _P],
            "ib_op_rhs": [_i32, _i32, _d, _d, _P, _P, _P, _P, _P, _P, _P, _P],
            "ib_op_correct": [_i32, _i32, _d, _d, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
            "mg_solve_noalloc": [_i32, _i32, _d, _P, _P, _P, _P, C.c_int, _d, C.c_int, C.c_int,
                                 C.c_int, C.POINTER(C.c_int), C.POINTER(_d), _P],
            "cnn_init": [C.POINTER(_P), _i32, _i32, C.c_uint64, _P],
            "cnn_get_params": [_P, _P, C.c_int64], "cnn_set_params": [_P, _P, C.c_int64],
            "cnn_grad": [_P, _i32, _i32, _d, _P, _P, _P, C.POINTER(C.c_float), _P, _P],
            "cnn_train_step": [_P, _i32, _i32, _d, _P, _P, _P, C.c_float, C.POINTER(C.c_float),
                               _P],
            "cnn_infer": [_P, _i32, _i32, _d, _P, _P, _P, _P],
            "cnn_fit_scale": [_P, _i32, _i32, _d, _P, _P, C.POINTER(_d), _P],
            "cnn_train": [_P, _i32, _i32, _d, _P, _P, _P, _i32, _i32, C.c_float, C.c_uint64, _P,
                          _P],
            "cnn_set_scale": [_P, _d], "cnn_set_coarsen": [_P, _i32],
            "cnn_set_tensor_path": [_P, _i32],
            "ib_bench_kernel": [_P, C.c_int, C.c_int, C.c_int, _P, _P],
            "ib_attach_cnn": [_P, _P], "ib_use_graphs": [_P, C.c_int],
            "ib_op_predictor": [_i32, _i32, _d, _d, _P, _P, _P, _P, _P, _P, _i32, _d, _d, _P,
                                _P, _P, _P, _P],
            "ib_op_predictor_axi": [_i32, _i32, _d, _d, _P, _P, _P, _P, _P, _P, _i32, _d, _P,
                                    _P, _P, _P, _P, _P],
            "ib_frame_state": [_P, _P], "ib_mass_correct": [_P, _P],
            "ib_op_cn_solve": [_i32, _i32, _d, _d, _P, _P, _i32, _i32, _P, _P, _P, _P, _P],
            "ib_op_rhs_axi": [_i32, _i32, _d, _d, _P, _P, _P, _P, _P, _P, _P, _P],
            "ib_op_axi_weights": [_i32, _i32, _d, _P, _P, _P, _P, _P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.ib_destroy.argtypes = [_P]
        L.ib_destroy.restype = None
        L.ib_last_error.argtypes = [_P]
        L.ib_last_error.restype = C.c_char_p
        L.mg_solve_noalloc_error.argtypes = []
        L.mg_solve_noalloc_error.restype = C.c_char_p
        L.ib_probe_fp64.argtypes = [_P, C.POINTER(_d)]
        L.ib_probe_fp64.restype = C.c_int
        L.ib_debug_stall_staging.argtypes = [C.c_int]
        L.ib_debug_stall_staging.restype = C.c_int
        L.ib_profile_begin.argtypes = [C.c_int]
        L.ib_profile_begin.restype = C.c_int
        L.ib_profile_end.argtypes = [C.POINTER(_d), C.POINTER(C.c_int)]
        L.ib_profile_end.restype = C.c_int
        L.ib_launch_count.argtypes = []
        L.ib_launch_count.restype = C.c_ulonglong
        L.cnn_destroy.argtypes = [_P]
        L.cnn_destroy.restype = None
        L.cnn_get_scale.argtypes = [_P]
        L.cnn_get_scale.restype = _d
        L.cnn_num_params.argtypes = [_P]
        L.cnn_num_params.restype = C.c_int64
        L.ib_num_markers.argtypes = [_P]
        L.ib_num_markers.restype = _i32
        _lib = L
    return _lib


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise IBError(IB_ECUDA, "no CUDA device: this library has no CPU path")
    return torch


def _ptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise IBError(IB_EINVAL, "expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise IBError(IB_EINVAL, f"expected {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _check(st, ctx=None, what=""):
    if st != IB_OK:
        msg = lib().ib_last_error(ctx).decode() if ctx else what
        raise IBError(st, msg)


# -------------------------------------------------------------- context API
@dataclass
class Config:
    nx: int
    ny: int
    h: float
    x0: float = 0.0
    y0: float = 0.0
    rho_g: float = 1e-3
    rho_l: float = 1.0
    mu_g: float = 1e-4
    mu_l: float = 1e-2
    sigma: float = 1.0
    gx: float = 0.0
    gy: float = 0.0
    kernel: int = 0
    spread: int = 1
    precision: int = 0
    tol: float = 1e-10
    max_cycles: int = 100
    nu1: int = 2
    nu2: int = 2
    relocate_every: int = 10
    axisym: int = 0
    frame: int = 0
    c1: float = 0.1
    c2: float = 0.1
    mass_every: int = 0
    mass_tol: float = 1e-6
    viscous: int = 0
    cn_sweeps: int = 20
    indicator: int = 0

    def c(self) -> ib_config:
        return ib_config(**{k: getattr(self, k) for k, _ in ib_config._fields_})


class Context:
    """Owns an ``ib_ctx``: fields, markers and the multigrid hierarchy live in
    device memory allocated by the library; calls run on the current torch
    stream at construction."""

    def __init__(self, cfg: Config, X, Y, drop_start):
        torch = _torch()
        self.cfg = cfg
        X = np.ascontiguousarray(X, np.float64)
        Y = np.ascontiguousarray(Y, np.float64)
        ds = np.ascontiguousarray(drop_start, np.int32)
        self.M = int(ds[-1])
        self._h = C.c_void_p()
        self._cfg = cfg.c()
        self._stream = torch.cuda.current_stream()
        st = lib().ib_init(C.byref(self._h), C.byref(self._cfg), X.ctypes.data, Y.ctypes.data,
                           ds.ctypes.data, len(ds) - 1, C.c_void_p(self._stream.cuda_stream))
        _check(st, None, "ib_init")
        self.ndrops = len(ds) - 1

    def __del__(self):
        try:
            if self._h:
                lib().ib_destroy(self._h)
                self._h = C.c_void_p()
        except Exception:
            pass

    def close(self):
        self.__del__()

    # shapes
    def shape(self, name):
        nx, ny = self.cfg.nx, self.cfg.ny
        return {"u": (ny, nx + 1), "us": (ny, nx + 1), "bx": (ny, nx + 1), "Fx": (ny, nx + 1),
                "v": (ny + 1, nx), "vs": (ny + 1, nx), "by": (ny + 1, nx),
                "Fy": (ny + 1, nx)}.get(name, (ny, nx))

    def get(self, name):
        torch = _torch()
        out = torch.empty(self.shape(name), dtype=torch.float64, device="cuda")
        _check(lib().ib_get_field(self._h, FIELDS[name], _ptr(out), 1), self._h)
        return out

    def get_host(self, name, out: np.ndarray | None = None):
        out = np.empty(self.shape(name)) if out is None else out
        _check(lib().ib_get_field(self._h, FIELDS[name], out.ctypes.data, 0), self._h)
        return out

    def set(self, name, t):
        _check(lib().ib_set_field(self._h, FIELDS[name], _ptr(t, _torch().float64), 1), self._h)

    def markers(self):
        torch = _torch()
        X = torch.empty(self.M, dtype=torch.float64, device="cuda")
        Y = torch.empty_like(X)
        _check(lib().ib_get_markers(self._h, _ptr(X), _ptr(Y), 1), self._h)
        return X, Y

    def set_markers_host(self, X: np.ndarray, Y: np.ndarray):
        _check(lib().ib_set_markers(self._h, X.ctypes.data, Y.ctypes.data, 0), self._h)

    def get_markers_host(self, X: np.ndarray, Y: np.ndarray):
        _check(lib().ib_get_markers(self._h, X.ctypes.data, Y.ctypes.data, 0), self._h)

    def set_markers(self, X, Y):
        _check(lib().ib_set_markers(self._h, _ptr(X), _ptr(Y), 1), self._h)

    def geometry(self):
        torch = _torch()
        outs = [torch.empty(self.M, dtype=torch.float64, device="cuda") for _ in range(4)]
        _check(lib().ib_marker_geometry(self._h, *[_ptr(o) for o in outs]), self._h)
        return outs

    def marker_sort(self):
        torch = _torch()
        keys = torch.empty(self.M, dtype=torch.int32, device="cuda")
        ids = torch.empty(self.M, dtype=torch.int32, device="cuda")
        cs = torch.empty(self.cfg.nx * self.cfg.ny + 1, dtype=torch.int32, device="cuda")
        _check(lib().ib_marker_sort(self._h, _ptr(keys), _ptr(ids), _ptr(cs)), self._h)
        return keys, ids, cs

    def interp(self, u, v):
        torch = _torch()
        U = torch.empty(self.M, dtype=torch.float64, device="cuda")
        V = torch.empty_like(U)
        _check(lib().ib_interp(self._h, _ptr(u, torch.float64), _ptr(v, torch.float64), _ptr(U),
                               _ptr(V)), self._h)
        return U, V

    def spread(self, mode, fmag=None, want_H=False):
        torch = _torch()
        Fx = torch.empty(self.shape("Fx"), dtype=torch.float64, device="cuda")
        Fy = torch.empty(self.shape("Fy"), dtype=torch.float64, device="cuda")
        H = torch.empty(self.shape("H"), dtype=torch.float64, device="cuda") if want_H else None
        _check(lib().ib_spread(self._h, mode, _ptr(fmag, torch.float64), _ptr(Fx), _ptr(Fy),
                               _ptr(H)), self._h)
        return (Fx, Fy, H) if want_H else (Fx, Fy)

    def heaviside(self):
        torch = _torch()
        H = torch.empty(self.shape("H"), dtype=torch.float64, device="cuda")
        _check(lib().ib_heaviside(self._h, _ptr(H)), self._h)
        return H

    def relocate(self):
        _check(lib().ib_relocate(self._h), self._h)

    def mass_correct(self):
        """Section 2.5 measure correction of the current markers; returns the
        normal offset of each drop (0 where none was needed)."""
        eps = np.zeros(self.ndrops)
        _check(lib().ib_mass_correct(self._h, eps.ctypes.data), self._h)
        return eps

    def frame_state(self):
        """(centre of mass, next acceleration S, frame velocity Vf, boundary
        velocity) of the non-inertial frame."""
        out = np.zeros(4)
        _check(lib().ib_frame_state(self._h, out.ctypes.data), self._h)
        return tuple(float(x) for x in out)

    def mg_setup(self, bx, by):
        torch = _torch()
        _check(lib().mg_setup(self._h, _ptr(bx, torch.float64), _ptr(by, torch.float64)),
               self._h)

    def mg_solve(self, rhs, p, precision=0, tol=1e-10, max_cycles=100, check=True):
        torch = _torch()
        cyc, rr = C.c_int(0), C.c_double(0.0)
        st = lib().mg_solve(self._h, _ptr(rhs, torch.float64), _ptr(p, torch.float64), precision,
                            tol, max_cycles, C.byref(cyc), C.byref(rr))
        if check and st not in (IB_OK,):
            _check(st, self._h)
        return st, cyc.value, rr.value

    def ns_step(self, dt, nsteps=1, warm=1):
        _check(lib().ns_step(self._h, dt, nsteps, warm), self._h)
        cyc, rr = C.c_int(0), C.c_double(0.0)
        lib().ib_last_solve(self._h, C.byref(cyc), C.byref(rr))
        return cyc.value, rr.value

    def ns_step_io(self, dt, warm=1, X=None, Y=None, p_out=None, X_out=None, Y_out=None):
        """One time step with host numpy buffers (see ns_step_io): optional
        markers in, optional pressure and markers out; returns (cycles,
        relative residual) of the step's solve."""
        def ptr(a):
            if a is None:
                return None
            if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
                raise ValueError("host buffers must be C-contiguous float64")
            return a.ctypes.data
        _check(lib().ns_step_io(self._h, dt, warm, ptr(X), ptr(Y), ptr(p_out), ptr(X_out),
                                ptr(Y_out)), self._h)
        cyc, rr = C.c_int(0), C.c_double(0.0)
        lib().ib_last_solve(self._h, C.byref(cyc), C.byref(rr))
        return cyc.value, rr.value

    def bench_kernel(self, which: int, reps: int = 50, level: int = 0):
        """(us per launch, work units per launch) of `reps` back-to-back
        launches of one kernel on the current data (see ib_bench_kernel)."""
        us, units = C.c_double(0.0), C.c_double(0.0)
        _check(lib().ib_bench_kernel(self._h, which, level, reps, C.byref(us), C.byref(units)),
               self._h)
        return us.value, units.value

    def use_graphs(self, enable: bool):
        _check(lib().ib_use_graphs(self._h, int(enable)), self._h)

    def attach(self, net):
        """Use `net` (a Net) for ns_step(..., warm=2); None detaches."""
        self._net = net
        _check(lib().ib_attach_cnn(self._h, net._h if net is not None else None), self._h)

    def save(self, path):
        _check(lib().ib_save(self._h, str(path).encode()), self._h)

    def load(self, path):
        _check(lib().ib_load(self._h, str(path).encode()), self._h)


# -------------------------------------------------------------- learned warm start
class Net:
    """The warm-start CNN (``cnn_*`` entry points): BF16 tensor-core forward
    and backward kernels, FP32 master weights and Adam state on the device."""

    def __init__(self, seed=0, c1=16, c2=32):
        torch = _torch()
        self._h = C.c_void_p()
        st = lib().cnn_init(C.byref(self._h), c1, c2, seed,
                            C.c_void_p(torch.cuda.current_stream().cuda_stream))
        _check(st, None, "cnn_init")
        self.nparam = int(lib().cnn_num_params(self._h))

    def __del__(self):
        try:
            if self._h:
                lib().cnn_destroy(self._h)
                self._h = C.c_void_p()
        except Exception:
            pass

    def get_params(self) -> np.ndarray:
        out = np.empty(self.nparam, np.float32)
        _check(lib().cnn_get_params(self._h, out.ctypes.data, self.nparam), None, "cnn_get_params")
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        _check(lib().cnn_set_params(self._h, flat.ctypes.data, self.nparam), None, "cnn_set_params")

    @property
    def scale(self) -> float:
        return float(lib().cnn_get_scale(self._h))

    @scale.setter
    def scale(self, c: float):
        _check(lib().cnn_set_scale(self._h, float(c)), None, "cnn_set_scale")

    def grad(self, rhs, rho, p, h=None):
        B, N = rhs.shape[0], rhs.shape[-1]
        h = 1.0 / N if h is None else h
        loss = C.c_float(0.0)
        g = np.empty(self.nparam, np.float32)
        _check(lib().cnn_grad(self._h, B, N, h, _ptr(rhs), _ptr(rho), _ptr(p), C.byref(loss),
                              g.ctypes.data, _stream()), None, "cnn_grad")
        return loss.value, g

    def train_step(self, rhs, rho, p, lr=1e-3, h=None):
        B, N = rhs.shape[0], rhs.shape[-1]
        h = 1.0 / N if h is None else h
        loss = C.c_float(0.0)
        _check(lib().cnn_train_step(self._h, B, N, h, _ptr(rhs), _ptr(rho), _ptr(p), lr,
                                    C.byref(loss), _stream()), None, "cnn_train_step")
        return loss.value

    def fit_scale(self, rhs, p, h=None) -> float:
        """Set (and return) the pressure scale c from samples (B, N, N) of the
        right-hand side and the pressure (cnn_fit_scale)."""
        B, N = rhs.shape[0], rhs.shape[-1]
        h = 1.0 / N if h is None else h
        c = C.c_double(0.0)
        _check(lib().cnn_fit_scale(self._h, B, N, h, _ptr(rhs), _ptr(p), C.byref(c), _stream()),
               None, "cnn_fit_scale")
        return c.value

    def train(self, rhs, rho, p, steps, batch=16, lr=2e-3, seed=0, h=None):
        """A training run on samples (n, N, N) (cnn_train): the scale fit,
        then `steps` Adam steps on random mini-batches with the learning rate
        decaying tenfold; returns the list of batch losses."""
        n, N = rhs.shape[0], rhs.shape[-1]
        h = 1.0 / N if h is None else h
        losses = np.empty(steps, np.float32)
        _check(lib().cnn_train(self._h, n, N, h, _ptr(rhs), _ptr(rho), _ptr(p), steps, batch, lr,
                               seed, losses.ctypes.data, _stream()), None, "cnn_train")
        return losses.tolist()

    def set_tensor_path(self, mode: int):
        """0: the warp-level mma.sync kernel everywhere; 1 (default): tcgen05
        for the layer shapes where it is faster; 2: tcgen05 for every layer
        whose width is a multiple of 128 (see cnn_set_tensor_path)."""
        _check(lib().cnn_set_tensor_path(self._h, int(mode)), None, "cnn_set_tensor_path")

    def set_coarsen(self, levels: int):
        """Run inference on the grid coarsened by 2^levels (inputs averaged,
        estimate interpolated back); 0 = the solve grid itself."""
        _check(lib().cnn_set_coarsen(self._h, int(levels)), None, "cnn_set_coarsen")

    def infer(self, rhs, rho, h=None, out=None):
        """Pressure estimate for a batch (B, N, N) of right-hand sides and
        densities; written to ``out`` when given (repeated calls with the same
        arguments replay a recorded CUDA graph of the launches)."""
        torch = _torch()
        B, N = rhs.shape[0], rhs.shape[-1]
        h = 1.0 / N if h is None else h
        p0 = torch.empty((B, N, N), dtype=torch.float64, device="cuda") if out is None else out
        _check(lib().cnn_infer(self._h, B, N, h, _ptr(rhs), _ptr(rho), _ptr(p0), _stream()),
               None, "cnn_infer")
        return p0


# -------------------------------------------------------------- no-allocation solve
def mg_solve_noalloc(bx, by, rhs, p, h, precision=0, tol=1e-10, max_cycles=100, nu1=2, nu2=2):
    """Pressure solve through ``mg_solve_noalloc``: scratch comes from a fixed
    device array inside the library, so nothing is allocated (for callers that
    cannot allocate device memory).  ``p`` is updated in place.  Returns
    (status, cycles, relative residual); ``noalloc_error()`` gives the
    library's message for a failed call.  Arrays of the wrong shape raise
    IBError(IB_EINVAL) before the call."""
    torch = _torch()
    ny, nx = p.shape
    for name, a, shape in (("bx", bx, (ny, nx + 1)), ("by", by, (ny + 1, nx)),
                           ("rhs", rhs, (ny, nx))):
        if tuple(a.shape) != shape:
            raise IBError(IB_EINVAL, f"{name} has shape {tuple(a.shape)}, expected {shape}")
    cyc, rr = C.c_int(0), C.c_double(0.0)
    st = lib().mg_solve_noalloc(nx, ny, h, _ptr(bx, torch.float64), _ptr(by, torch.float64),
                                _ptr(rhs, torch.float64), _ptr(p, torch.float64), precision, tol,
                                max_cycles, nu1, nu2, C.byref(cyc), C.byref(rr), _stream())
    return st, cyc.value, rr.value


def probe_fp64() -> float:
    """Measured FP64 FMA throughput of the current GPU in TFLOP/s."""
    t = C.c_double(0.0)
    _check(lib().ib_probe_fp64(_stream(), C.byref(t)), None, "ib_probe_fp64")
    return t.value


def noalloc_error() -> str:
    return lib().mg_solve_noalloc_error().decode()


def debug_stall_staging(enable: bool) -> None:
    """Test hook: make every TMA-staged FP32 smoother block's bounded wait
    run out (see ib_debug_stall_staging), or restore normal operation."""
    _check(lib().ib_debug_stall_staging(1 if enable else 0), None, "ib_debug_stall_staging")


# -------------------------------------------------------------- measurement
PROF_SWEEP64, PROF_SWEEP32, PROF_RESNORM, PROF_PROLONG32 = 0, 1, 2, 3
PROF_PRE, PROF_SOLVE, PROF_POST = 4, 5, 6  # the parts of ns_step


def launch_count() -> int:
    return int(lib().ib_launch_count())


def profile_begin(kind: int):
    _check(lib().ib_profile_begin(kind), None, "ib_profile_begin")


def profile_end():
    t, n = C.c_double(0.0), C.c_int(0)
    _check(lib().ib_profile_end(C.byref(t), C.byref(n)), None, "ib_profile_end")
    return t.value, n.value


# -------------------------------------------------------------- operators
def _op(name, *args):
    st = getattr(lib(), name)(*args, _stream())
    _check(st, None, name)


def ib_op_coeffs(H, rho_g, rho_l, mu_g, mu_l):
    torch = _torch()
    ny, nx = H.shape
    rho, mu = torch.empty_like(H), torch.empty_like(H)
    bx = torch.empty((ny, nx + 1), dtype=torch.float64, device="cuda")
    by = torch.empty((ny + 1, nx), dtype=torch.float64, device="cuda")
    _op("ib_op_coeffs", nx, ny, rho_g, rho_l, mu_g, mu_l, _ptr(H), _ptr(rho), _ptr(mu),
        _ptr(bx), _ptr(by))
    return rho, mu, bx, by


def ib_op_residual(bx, by, b, p, h):
    ny, nx = p.shape
    r = _torch().empty_like(p)
    _op("ib_op_residual", nx, ny, h, _ptr(bx), _ptr(by), _ptr(b), _ptr(p), _ptr(r))
    return r


def ib_op_rbgs(bx, by, b, p, h, nsweeps=1):
    ny, nx = p.shape
    p = p.clone()
    _op("ib_op_rbgs", nx, ny, h, _ptr(bx), _ptr(by), _ptr(b), _ptr(p), nsweeps)
    return p


def ib_op_restrict_residual(bx, by, b, p, h):
    ny, nx = p.shape
    rc = _torch().empty((ny // 2, nx // 2), dtype=p.dtype, device=p.device)
    _op("ib_op_restrict_residual", nx, ny, h, _ptr(bx), _ptr(by), _ptr(b), _ptr(p), _ptr(rc))
    return rc


def ib_op_prolong_add(ec, ef):
    nyc, nxc = ec.shape
    ef = ef.clone()
    _op("ib_op_prolong_add", nxc, nyc, _ptr(ec), _ptr(ef))
    return ef


def ib_op_coarsen_beta(bx, by):
    torch = _torch()
    ny, nx = bx.shape[0], by.shape[1]
    bxc = torch.empty((ny // 2, nx // 2 + 1), dtype=torch.float64, device="cuda")
    byc = torch.empty((ny // 2 + 1, nx // 2), dtype=torch.float64, device="cuda")
    _op("ib_op_coarsen_beta", nx, ny, _ptr(bx), _ptr(by), _ptr(bxc), _ptr(byc))
    return bxc, byc


def ib_op_rhs(us, vs, Fx, Fy, bx, by, h, dt):
    ny, nx = us.shape[0], vs.shape[1]
    b = _torch().empty((ny, nx), dtype=us.dtype, device=us.device)
    _op("ib_op_rhs", nx, ny, h, dt, _ptr(us), _ptr(vs), _ptr(Fx), _ptr(Fy), _ptr(bx), _ptr(by),
        _ptr(b))
    return b


def ib_op_correct(us, vs, p, Fx, Fy, bx, by, h, dt):
    ny, nx = p.shape
    u, v = _torch().empty_like(us), _torch().empty_like(vs)
    _op("ib_op_correct", nx, ny, h, dt, _ptr(us), _ptr(vs), _ptr(p), _ptr(Fx), _ptr(Fy),
        _ptr(bx), _ptr(by), _ptr(u), _ptr(v))
    return u, v


def ib_op_predictor_axi(rho, mu, u, v, h, dt, au_prev=None, av_prev=None, gy=0.0, S=None,
                        wb=None):
    """Axisymmetric predictor; S (extra axial acceleration) and wb (axial
    velocity of the z boundaries and the outer wall) go in a frame record."""
    torch = _torch()
    ny, nx = rho.shape
    us, vs, au, av = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(u),
                      torch.empty_like(v))
    have = au_prev is not None
    frame = None
    if S is not None or wb is not None:
        frame = torch.zeros(8, dtype=torch.float64, device=u.device)
        frame[3] = float(S or 0.0)
        frame[5] = float(wb or 0.0)
    _op("ib_op_predictor_axi", nx, ny, h, dt, _ptr(rho), _ptr(mu), _ptr(u), _ptr(v),
        _ptr(au_prev), _ptr(av_prev), int(have), float(gy), _ptr(frame), _ptr(us), _ptr(vs),
        _ptr(au), _ptr(av))
    return us, vs, au, av


def ib_op_rhs_axi(us, vs, Fx, Fy, bx, by, h, dt):
    ny, nx = us.shape[0], vs.shape[1]
    b = _torch().empty((ny, nx), dtype=us.dtype, device=us.device)
    _op("ib_op_rhs_axi", nx, ny, h, dt, _ptr(us), _ptr(vs), _ptr(Fx), _ptr(Fy), _ptr(bx),
        _ptr(by), _ptr(b))
    return b


def ib_op_cn_solve(rho, mu, ue, ve, h, dt, nsweeps, axisym=0):
    torch = _torch()
    ny, nx = rho.shape
    us, vs = torch.empty_like(ue), torch.empty_like(ve)
    _op("ib_op_cn_solve", nx, ny, h, dt, _ptr(rho), _ptr(mu), int(axisym), int(nsweeps), _ptr(ue),
        _ptr(ve), _ptr(us), _ptr(vs))
    return us, vs


def ib_op_axi_weights(bx, by, h):
    ny, nx = bx.shape[0], by.shape[1]
    bxa, bya = _torch().empty_like(bx), _torch().empty_like(by)
    _op("ib_op_axi_weights", nx, ny, h, _ptr(bx), _ptr(by), _ptr(bxa), _ptr(bya))
    return bxa, bya


def ib_op_predictor(rho, mu, u, v, h, dt, au_prev=None, av_prev=None, g=(0.0, 0.0)):
    torch = _torch()
    ny, nx = rho.shape
    us, vs, au, av = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(u),
                      torch.empty_like(v))
    have = au_prev is not None
    _op("ib_op_predictor", nx, ny, h, dt, _ptr(rho), _ptr(mu), _ptr(u), _ptr(v),
        _ptr(au_prev), _ptr(av_prev), int(have), float(g[0]), float(g[1]), _ptr(us), _ptr(vs),
        _ptr(au), _ptr(av))
    return us, vs, au, av
