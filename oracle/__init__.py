"""Plain FP64 CPU oracle for the immersed-boundary projection method of
Ong & Miura (arXiv 1807.10504).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it.  The arithmetic lives in
``ib_oracle.c`` (built with ``-O3 -ffp-contract=off``; a second build adds
``-fopenmp`` for the timed CPU baseline on all host cores); this module is argument
marshalling plus the composition of one time step (Section 2.1 fractional
step with the force in the projection, Section 3.2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ib_oracle.c")
_SRC_AXI = os.path.join(_HERE, "ib_oracle_axi.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")

IB_OK, IB_EINVAL, IB_ENOMEM, IB_ENOTCONV, IB_ENAN, IB_EMARKER = 0, 1, 2, 3, 4, 5


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain gcc, -O3, no
    multiply-add contraction).  With ``openmp``, the same source with
    ``-fopenmp`` into ``oracle/liboracle_omp.so``: its loops over independent
    cells, faces or markers run on all host cores, with results identical bit
    for bit (every sum keeps its serial order).  Returns the library path, or
    raises if the compiler fails."""
    out = _LIB_OMP if openmp else _LIB
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(
        os.path.getmtime(_SRC), os.path.getmtime(_SRC_AXI),
        os.path.getmtime(os.path.join(_HERE, "ib_oracle.h"))
    ):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O3", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
             *(["-fopenmp"] if openmp else []), "-o", tmp, _SRC, _SRC_AXI, "-lm"]
        )
        os.replace(tmp, out)
    return out


def set_threads(openmp: bool) -> None:
    """Route every following oracle call to the serial library (default) or
    to its OpenMP build (all host cores; same results)."""
    global _variant
    _variant = "omp" if openmp else "serial"


def threads() -> int:
    """Host threads the current variant uses."""
    if _variant == "serial":
        return 1
    return int(os.environ.get("OMP_NUM_THREADS", "0")) or (os.cpu_count() or 1)


_libs = {}
_variant = "serial"
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i, _d = C.c_int, C.c_double


def lib():
    L = _libs.get(_variant)
    if L is None:
        L = C.CDLL(build(openmp=_variant == "omp"))
        sig = {
            "or_phi": (_d, [_i, _d]),
            "or_heaviside_profile": (_d, [_d]),
            "or_coeffs": (None, [_i, _i, _d, _d, _d, _d, _D, _D, _D, _D, _D]),
            "or_apply_A": (None, [_i, _i, _d, _D, _D, _D, _D]),
            "or_residual": (None, [_i, _i, _d, _D, _D, _D, _D, _D]),
            "or_rbgs": (None, [_i, _i, _d, _D, _D, _D, _D, _i]),
            "or_restrict": (None, [_i, _i, _D, _D]),
            "or_coarsen_beta": (None, [_i, _i, _D, _D, _D, _D]),
            "or_prolong_add": (None, [_i, _i, _D, _D]),
            "or_mg_levels": (_i, [_i, _i, _I32, _I32, _i]),
            "or_dense_solve": (_i, [_i, _i, _d, _D, _D, _D, _D]),
            "or_mg_solve": (_i, [_i, _i, _d, _D, _D, _D, _D, _i, _d, _i, _i, _i,
                                 C.POINTER(_i), C.POINTER(_d), _D]),
            "or_rhs": (None, [_i, _i, _d, _d, _D, _D, _D, _D, _D, _D, _D]),
            "or_correct": (None, [_i, _i, _d, _d, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
            "or_divergence": (None, [_i, _i, _d, _D, _D, _D]),
            "or_predictor": (None, [_i, _i, _d, _d, _D, _D, _D, _D, _D, _D, _i, _d, _d,
                                    _D, _D, _D, _D]),
            "or_cell_keys": (None, [_i, _D, _D, _d, _d, _d, _i, _i, _U32]),
            "or_marker_sort": (None, [_i, _U32, _U32]),
            "or_interp": (None, [_i, _i, _i, _d, _d, _d, _D, _D, _i, _D, _D, _D, _D]),
            "or_spread_conv": (None, [_i, _i, _i, _d, _d, _d, _i, _D, _D, _D, _D, _D, _D,
                                      _D, _D]),
            "or_curvature": (None, [_i, _D, _D, _i, _I32, _D, _D, _D, _D]),
            "or_inside": (None, [_i, _i, _d, _d, _d, _i, _D, _D, _i, _I32, _D]),
            "or_inside_cell": (_d, [_i, _i, _d, _d, _d, _i, _D, _D, _i, _I32]),
            "or_heaviside": (None, [_i, _i, _d, _d, _d, _i, _D, _D, _i, _I32, _D]),
            "or_heaviside_cell": (_d, [_i, _i, _d, _d, _d, _i, _D, _D, _i, _I32, _d]),
            "or_spread_irrot": (None, [_i, _i, _d, _d, _d, _i, _D, _D, _i, _I32, _D, _D,
                                       _D, _D]),
            "or_bspline_relocate": (_i, [_i, _D, _D, _i, _I32, _d, _D, _D]),
            "or_apply_A_axi": (None, [_i, _i, _d, _D, _D, _D, _D]),
            "or_axi_weights": (None, [_i, _i, _d, _D, _D, _D, _D]),
            "or_divergence_axi": (None, [_i, _i, _d, _D, _D, _D]),
            "or_rhs_axi": (None, [_i, _i, _d, _d, _D, _D, _D, _D, _D, _D, _D]),
            "or_predictor_axi": (None, [_i, _i, _d, _d, _D, _D, _D, _D, _D, _D, _i, _d, _d,
                                        _d, _D, _D, _D, _D]),
            "or_curvature_axi": (None, [_i, _D, _D, _i, _I32, _D, _D, _D, _D]),
            "or_spread_conv_axi": (None, [_i, _i, _i, _d, _i, _D, _D, _D, _D, _D, _D, _D,
                                          _D]),
            "or_interp_axi": (None, [_i, _i, _i, _d, _D, _D, _i, _D, _D, _D, _D]),
            "or_drop_com_axi": (None, [_i, _D, _D, _I32, _i, C.POINTER(_d), C.POINTER(_d)]),
            "or_drop_measure": (_d, [_i, _D, _D, _i]),
            "or_cn_solve": (None, [_i, _i, _d, _d, _D, _D, _i, _d, _i, _D, _D]),
            "or_mass_correct": (_i, [_i, _D, _D, _i, _I32, _D, _i, _d, _d, _D, _D, _D]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _libs[_variant] = L
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ds(drop_start):
    return np.ascontiguousarray(drop_start, dtype=np.int32)


# --------------------------------------------------------------------------
# Kernels and profiles (Section 2.2 Eq. (cherby), Section 3.2 Eq. (new_hea))
def phi(r, kernel: int = 0):
    return np.vectorize(lambda x: lib().or_phi(kernel, float(x)))(np.asarray(r, float))


def heaviside_profile(r):
    return np.vectorize(lambda x: lib().or_heaviside_profile(float(x)))(np.asarray(r, float))


# --------------------------------------------------------------------------
# Grid operators (Section 2.1)
def coeffs(H, rho_g, rho_l, mu_g, mu_l):
    ny, nx = H.shape
    rho, mu = np.empty((ny, nx)), np.empty((ny, nx))
    bx, by = np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    lib().or_coeffs(nx, ny, rho_g, rho_l, mu_g, mu_l, _f64(H), rho, mu, bx, by)
    return rho, mu, bx, by


def apply_A(bx, by, p, h):
    ny, nx = p.shape
    out = np.empty((ny, nx))
    lib().or_apply_A(nx, ny, h, _f64(bx), _f64(by), _f64(p), out)
    return out


def residual(bx, by, b, p, h):
    ny, nx = p.shape
    r = np.empty((ny, nx))
    lib().or_residual(nx, ny, h, _f64(bx), _f64(by), _f64(b), _f64(p), r)
    return r


def rbgs(bx, by, b, p, h, nsweeps=1):
    p = _f64(p).copy()
    ny, nx = p.shape
    lib().or_rbgs(nx, ny, h, _f64(bx), _f64(by), _f64(b), p, nsweeps)
    return p


def restrict(r):
    ny, nx = r.shape
    rc = np.empty((ny // 2, nx // 2))
    lib().or_restrict(nx, ny, _f64(r), rc)
    return rc


def coarsen_beta(bx, by):
    ny, nx1 = bx.shape
    nx = nx1 - 1
    bxc, byc = np.empty((ny // 2, nx // 2 + 1)), np.empty((ny // 2 + 1, nx // 2))
    lib().or_coarsen_beta(nx, ny, _f64(bx), _f64(by), bxc, byc)
    return bxc, byc


def prolong_add(ec, ef):
    ef = _f64(ef).copy()
    nyc, nxc = ec.shape
    lib().or_prolong_add(nxc, nyc, _f64(ec), ef)
    return ef


def mg_levels(nx, ny):
    a, b = np.zeros(32, np.int32), np.zeros(32, np.int32)
    L = lib().or_mg_levels(nx, ny, a, b, 32)
    return [(int(a[k]), int(b[k])) for k in range(L)]


def dense_solve(bx, by, b, h):
    ny, nx = b.shape
    p = np.empty((ny, nx))
    st = lib().or_dense_solve(nx, ny, h, _f64(bx), _f64(by), _f64(b), p)
    if st != 0:
        raise RuntimeError("singular dense system")
    return p


@dataclass
class MGResult:
    p: np.ndarray
    status: int
    cycles: int
    relres: float
    hist: np.ndarray


def mg_solve(bx, by, b, h, p0=None, precision=0, tol=1e-10, max_cycles=100,
             nu1=2, nu2=2) -> MGResult:
    ny, nx = b.shape
    p = np.zeros((ny, nx)) if p0 is None else _f64(p0).copy()
    cyc, rel = _i(0), _d(0.0)
    hist = np.zeros(max_cycles + 2)
    st = lib().or_mg_solve(nx, ny, h, _f64(bx), _f64(by), _f64(b), p, precision, tol,
                           max_cycles, nu1, nu2, C.byref(cyc), C.byref(rel), hist)
    return MGResult(p, st, cyc.value, rel.value, hist[: cyc.value + 1])


def rhs(us, vs, Fx, Fy, bx, by, h, dt):
    ny, nx = us.shape[0], vs.shape[1]
    b = np.empty((ny, nx))
    lib().or_rhs(nx, ny, h, dt, _f64(us), _f64(vs), _f64(Fx), _f64(Fy), _f64(bx),
                 _f64(by), b)
    return b


def correct(us, vs, p, Fx, Fy, bx, by, h, dt):
    ny, nx = p.shape
    u, v = np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    lib().or_correct(nx, ny, h, dt, _f64(us), _f64(vs), _f64(p), _f64(Fx), _f64(Fy),
                     _f64(bx), _f64(by), u, v)
    return u, v


def divergence(u, v, h):
    ny, nx = u.shape[0], v.shape[1]
    d = np.empty((ny, nx))
    lib().or_divergence(nx, ny, h, _f64(u), _f64(v), d)
    return d


def predictor(rho, mu, u, v, h, dt, au_prev=None, av_prev=None, g=(0.0, 0.0)):
    ny, nx = rho.shape
    have = au_prev is not None
    aup = _f64(au_prev) if have else np.zeros((ny, nx + 1))
    avp = _f64(av_prev) if have else np.zeros((ny + 1, nx))
    us, vs = np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    au, av = np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    lib().or_predictor(nx, ny, h, dt, _f64(rho), _f64(mu), _f64(u), _f64(v), aup, avp,
                       int(have), float(g[0]), float(g[1]), us, vs, au, av)
    return us, vs, au, av


# --------------------------------------------------------------------------
# Markers (Sections 2.2, 3, 4)
def cell_keys(X, Y, x0, y0, h, nx, ny):
    key = np.empty(len(X), np.uint32)
    lib().or_cell_keys(len(X), _f64(X), _f64(Y), x0, y0, h, nx, ny, key)
    return key


def marker_sort(key):
    order = np.empty(len(key), np.uint32)
    lib().or_marker_sort(len(key), np.ascontiguousarray(key, np.uint32), order)
    return order


def interp(u, v, X, Y, h, x0=0.0, y0=0.0, kernel=0):
    ny, nx = u.shape[0], v.shape[1]
    U, V = np.empty(len(X)), np.empty(len(X))
    lib().or_interp(kernel, nx, ny, h, x0, y0, _f64(u), _f64(v), len(X), _f64(X), _f64(Y),
                    U, V)
    return U, V


def curvature(X, Y, drop_start):
    M = len(X)
    k, nxm, nym, ds = (np.empty(M) for _ in range(4))
    lib().or_curvature(M, _f64(X), _f64(Y), len(drop_start) - 1, _ds(drop_start), k, nxm,
                       nym, ds)
    return k, nxm, nym, ds


def spread_conv(X, Y, fmag, nxm, nym, ds, nx, ny, h, x0=0.0, y0=0.0, kernel=0):
    Fx, Fy = np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    lib().or_spread_conv(kernel, nx, ny, h, x0, y0, len(X), _f64(X), _f64(Y), _f64(fmag),
                         _f64(nxm), _f64(nym), _f64(ds), Fx, Fy)
    return Fx, Fy


def inside(X, Y, drop_start, nx, ny, h, x0=0.0, y0=0.0):
    chi = np.empty((ny, nx))
    lib().or_inside(nx, ny, h, x0, y0, len(X), _f64(X), _f64(Y), len(drop_start) - 1,
                    _ds(drop_start), chi)
    return chi


def inside_cell(i, j, X, Y, drop_start, h, x0=0.0, y0=0.0):
    return lib().or_inside_cell(int(i), int(j), h, x0, y0, len(X), _f64(X), _f64(Y),
                                len(drop_start) - 1, _ds(drop_start))


def heaviside(X, Y, drop_start, nx, ny, h, x0=0.0, y0=0.0):
    H = np.empty((ny, nx))
    lib().or_heaviside(nx, ny, h, x0, y0, len(X), _f64(X), _f64(Y), len(drop_start) - 1,
                       _ds(drop_start), H)
    return H


def heaviside_cell(i, j, X, Y, drop_start, h, chi, x0=0.0, y0=0.0):
    return lib().or_heaviside_cell(int(i), int(j), h, x0, y0, len(X), _f64(X), _f64(Y),
                                   len(drop_start) - 1, _ds(drop_start), float(chi))


def spread_irrot(X, Y, drop_start, fmag, H, h, x0=0.0, y0=0.0):
    ny, nx = H.shape
    Fx, Fy = np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    lib().or_spread_irrot(nx, ny, h, x0, y0, len(X), _f64(X), _f64(Y), len(drop_start) - 1,
                          _ds(drop_start), _f64(fmag), _f64(H), Fx, Fy)
    return Fx, Fy


def bspline_relocate(X, Y, drop_start, h):
    Xo, Yo = np.empty(len(X)), np.empty(len(X))
    st = lib().or_bspline_relocate(len(X), _f64(X), _f64(Y), len(drop_start) - 1,
                                   _ds(drop_start), h, Xo, Yo)
    if st != 0:
        raise RuntimeError("B-spline least-squares system not positive definite")
    return Xo, Yo


# --------------------------------------------------------------------------
# Axisymmetric (r, z) form (ib_oracle_axi.c): x = r from the axis, the drop
# given as its full closed meridian curve (right half and mirror image).
def apply_A_axi(bx, by, p, h):
    ny, nx = p.shape
    out = np.empty((ny, nx))
    lib().or_apply_A_axi(nx, ny, h, _f64(bx), _f64(by), _f64(p), out)
    return out


def axi_weights(bx, by, h):
    ny, nx = bx.shape[0], by.shape[1]
    bxa, bya = np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    lib().or_axi_weights(nx, ny, h, _f64(bx), _f64(by), bxa, bya)
    return bxa, bya


def divergence_axi(u, v, h):
    ny, nx = u.shape[0], v.shape[1]
    d = np.empty((ny, nx))
    lib().or_divergence_axi(nx, ny, h, _f64(u), _f64(v), d)
    return d


def rhs_axi(us, vs, Fx, Fy, bx, by, h, dt):
    ny, nx = us.shape[0], vs.shape[1]
    b = np.empty((ny, nx))
    lib().or_rhs_axi(nx, ny, h, dt, _f64(us), _f64(vs), _f64(Fx), _f64(Fy), _f64(bx),
                     _f64(by), b)
    return b


def predictor_axi(rho, mu, u, v, h, dt, au_prev=None, av_prev=None, g=(0.0, 0.0), wb=0.0):
    ny, nx = rho.shape
    have = au_prev is not None
    aup = _f64(au_prev) if have else np.zeros((ny, nx + 1))
    avp = _f64(av_prev) if have else np.zeros((ny + 1, nx))
    us, vs = np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    au, av = np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    lib().or_predictor_axi(nx, ny, h, dt, _f64(rho), _f64(mu), _f64(u), _f64(v), aup, avp,
                           int(have), float(g[0]), float(g[1]), float(wb), us, vs, au, av)
    return us, vs, au, av


def curvature_axi(X, Y, drop_start):
    M = len(X)
    k, nxm, nym, ds = (np.empty(M) for _ in range(4))
    lib().or_curvature_axi(M, _f64(X), _f64(Y), len(drop_start) - 1, _ds(drop_start), k,
                           nxm, nym, ds)
    return k, nxm, nym, ds


def spread_conv_axi(X, Y, fmag, nxm, nym, ds, nx, ny, h, kernel=0):
    Fx, Fy = np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    lib().or_spread_conv_axi(kernel, nx, ny, h, len(X), _f64(X), _f64(Y), _f64(fmag),
                             _f64(nxm), _f64(nym), _f64(ds), Fx, Fy)
    return Fx, Fy


def interp_axi(u, v, X, Y, h, kernel=0):
    ny, nx = u.shape[0], v.shape[1]
    U, V = np.empty(len(X)), np.empty(len(X))
    lib().or_interp_axi(kernel, nx, ny, h, _f64(u), _f64(v), len(X), _f64(X), _f64(Y), U, V)
    return U, V


def drop_com_axi(X, Y, drop_start, d=0):
    vol, zc = _d(0.0), _d(0.0)
    lib().or_drop_com_axi(len(X), _f64(X), _f64(Y), _ds(drop_start), int(d), C.byref(vol),
                          C.byref(zc))
    return vol.value, zc.value


def indicator_poisson(X, Y, drop_start, nx, ny, h, x0=0.0, y0=0.0, kernel=0, axisym=0,
                      tol=1e-12):
    """Section 2.2 Eq. (ind_psn): the indicator I of the conventional scheme,
    div grad I = div(delta vector), the delta vector being the conventional
    spreading (Eq. (delta)) of the markers' inward unit normals times their
    arc weights (ring-weighted in the axisymmetric form, where the equation is
    the r-weighted one).  Neumann walls; the free constant makes the mean of
    the cells along the walls zero (the axis is not a wall); clipped to [0, 1] (reading: I is a volume
    fraction).  Returns I."""
    k, nxm, nym, ds = curvature(X, Y, drop_start)
    ones = np.ones(len(X))
    if axisym:
        Gx, Gy = spread_conv_axi(X, _f64(Y) - y0, ones, nxm, nym, ds, nx, ny, h, kernel)
    else:
        Gx, Gy = spread_conv(X, Y, ones, nxm, nym, ds, nx, ny, h, x0, y0, kernel)
    bx = np.ones((ny, nx + 1))
    by = np.ones((ny + 1, nx))
    bx[:, [0, -1]] = 0.0
    by[[0, -1], :] = 0.0
    zx, zy = np.zeros_like(bx), np.zeros_like(by)
    if axisym:
        b = rhs_axi(Gx, Gy, zx, zy, bx, by, h, 1.0)
        bxa, bya = axi_weights(bx, by, h)
        r = (np.arange(nx) + 0.5) * h
        res = mg_solve(bxa, bya, b * r[None, :], h, tol=tol, max_cycles=300)
    else:
        b = rhs(Gx, Gy, zx, zy, bx, by, h, 1.0)
        res = mg_solve(bx, by, b, h, tol=tol, max_cycles=300)
    I = res.p
    # the cells along the walls (the axis column is not a wall)
    ring = np.concatenate([I[0], I[-1], I[1:-1, -1]] + ([] if axisym else [I[1:-1, 0]]))
    return np.clip(I - ring.mean(), 0.0, 1.0)


def cn_solve(rho, mu, ue, ve, h, dt, nsweeps, axisym=0, wb=0.0):
    """Section 2.1 Crank-Nicolson: nsweeps red-black sweeps on
    u* - dt / (2 rho_f) D(u*) = u_e per component."""
    ny, nx = rho.shape
    us, vs = _f64(ue).copy(), _f64(ve).copy()
    lib().or_cn_solve(nx, ny, h, dt, _f64(rho), _f64(mu), int(axisym), float(wb), int(nsweeps),
                      us, vs)
    return us, vs


def drop_measures(X, Y, drop_start, axisym=0):
    """Section 2.5: enclosed area (planar) or volume of revolution of each drop."""
    ds_ = _ds(drop_start)
    X, Y = _f64(X), _f64(Y)
    return np.array([lib().or_drop_measure(int(ds_[d + 1] - ds_[d]),
                                           np.ascontiguousarray(X[ds_[d]:ds_[d + 1]]),
                                           np.ascontiguousarray(Y[ds_[d]:ds_[d + 1]]), int(axisym))
                     for d in range(len(ds_) - 1)])


def mass_correct(X, Y, drop_start, A0, h, axisym=0, tol=1e-6):
    """Section 2.5: bisection offset along the inward normals restoring each
    drop's initial measure A0 where it drifted by more than tol.  Returns
    (X, Y, eps per drop)."""
    M = len(X)
    Xo, Yo = np.empty(M), np.empty(M)
    eps = np.empty(len(drop_start) - 1)
    lib().or_mass_correct(M, _f64(X), _f64(Y), len(drop_start) - 1, _ds(drop_start), _f64(A0),
                          int(axisym), float(tol), float(h), Xo, Yo, eps)
    return Xo, Yo, eps


def symmetrise(X, Y, drop_start):
    """Mirror symmetry of each drop's closed meridian curve about r = 0:
    marker k of a drop of n (n even) pairs with marker (n - k) mod n; each
    pair is replaced by its symmetric mean (markers 0 and n/2 land on the
    axis)."""
    X, Y = _f64(X).copy(), _f64(Y).copy()
    ds_ = _ds(drop_start)
    for d in range(len(ds_) - 1):
        s, e = int(ds_[d]), int(ds_[d + 1])
        n = e - s
        k = np.arange(n)
        p = (n - k) % n
        x, y = X[s:e].copy(), Y[s:e].copy()
        X[s:e] = 0.5 * (x - x[p])
        Y[s:e] = 0.5 * (y + y[p])
    return X, Y


# --------------------------------------------------------------------------
# One time step (Section 2.1 fractional step, force in the projection as in
# Section 3.2 Eq. (ns2_new)); the order of the stages is that of the method:
# relocate markers (every `relocate_every` steps), curvature, Heaviside and
# properties at the current marker positions, predictor, spreading,
# pressure solve, correction, marker advection by interpolated velocity.
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
    kernel: int = 0          # 0 cosine (Eq. cherby), 1 Peskin 4-point
    spread: int = 1          # 0 conventional (Eq. delta_vec), 1 irrotational
    precision: int = 0       # 0 FP64 multigrid, 1 FP32 cycles in FP64 refinement
    tol: float = 1e-10
    max_cycles: int = 100
    nu1: int = 2
    nu2: int = 2
    relocate_every: int = 10  # 0 = never
    axisym: int = 0           # 1: (r, z) with x = r from the axis (x0 = 0)
    mass_every: int = 0       # Section 2.5 measure check period in steps, 0 = never
    mass_tol: float = 1e-6
    viscous: int = 0          # 0 explicit, 1 Crank-Nicolson (Section 2.1)
    indicator: int = 0        # properties from 0: polygon Heaviside, 1: Eq. (ind_psn)
    cn_sweeps: int = 20       # red-black sweeps of the Crank-Nicolson solve
    frame: int = 0            # 1: non-inertial frame following drop 0 (axisym only)
    c1: float = 0.1           # Section 2.4 Eq. (fictitious) constants
    c2: float = 0.1


@dataclass
class State:
    u: np.ndarray
    v: np.ndarray
    p: np.ndarray
    X: np.ndarray
    Y: np.ndarray
    drop_start: np.ndarray
    au: np.ndarray | None = None
    av: np.ndarray | None = None
    frame: dict | None = None  # non-inertial frame: com0, com_prev, S, Vf
    A0: np.ndarray | None = None  # initial drop measures (Section 2.5)
    step: int = 0
    last: dict = field(default_factory=dict)


def init_state(cfg: Config, X, Y, drop_start) -> State:
    return State(u=np.zeros((cfg.ny, cfg.nx + 1)), v=np.zeros((cfg.ny + 1, cfg.nx)),
                 p=np.zeros((cfg.ny, cfg.nx)), X=_f64(X).copy(), Y=_f64(Y).copy(),
                 drop_start=_ds(drop_start).copy(),
                 A0=drop_measures(X, Y, drop_start, cfg.axisym))


def _markers_update(cfg: Config, st: State):
    """Marker upkeep at the start of a step: B-spline relocation (every
    relocate_every steps), then the Section 2.5 measure correction (every
    mass_every steps after the first); axisymmetric curves re-symmetrised."""
    if cfg.relocate_every > 0 and st.step % cfg.relocate_every == 0:
        st.X, st.Y = bspline_relocate(st.X, st.Y, st.drop_start, cfg.h)
        if cfg.axisym:
            st.X, st.Y = symmetrise(st.X, st.Y, st.drop_start)
    if cfg.mass_every > 0 and st.step > 0 and st.step % cfg.mass_every == 0:
        st.X, st.Y, _ = mass_correct(st.X, st.Y, st.drop_start, st.A0, cfg.h, cfg.axisym,
                                     cfg.mass_tol)
        if cfg.axisym:
            st.X, st.Y = symmetrise(st.X, st.Y, st.drop_start)


def ns_step(cfg: Config, st: State, dt: float) -> State:
    if cfg.axisym:
        return _ns_step_axi(cfg, st, dt)
    h = cfg.h
    _markers_update(cfg, st)
    kap, nxm, nym, ds = curvature(st.X, st.Y, st.drop_start)
    fmag = cfg.sigma * kap
    H = heaviside(st.X, st.Y, st.drop_start, cfg.nx, cfg.ny, h, cfg.x0, cfg.y0)
    Ip = H if not cfg.indicator else indicator_poisson(st.X, st.Y, st.drop_start, cfg.nx,
                                                        cfg.ny, h, cfg.x0, cfg.y0, cfg.kernel)
    rho, mu, bx, by = coeffs(Ip, cfg.rho_g, cfg.rho_l, cfg.mu_g, cfg.mu_l)
    if cfg.viscous:
        us, vs, au, av = predictor(rho, 0.5 * mu, st.u, st.v, h, dt, st.au, st.av,
                                   (cfg.gx, cfg.gy))
        us, vs = cn_solve(rho, mu, us, vs, h, dt, cfg.cn_sweeps)
    else:
        us, vs, au, av = predictor(rho, mu, st.u, st.v, h, dt, st.au, st.av, (cfg.gx, cfg.gy))
    if cfg.spread == 0:
        Fx, Fy = spread_conv(st.X, st.Y, fmag, nxm, nym, ds, cfg.nx, cfg.ny, h, cfg.x0,
                             cfg.y0, cfg.kernel)
    else:
        Fx, Fy = spread_irrot(st.X, st.Y, st.drop_start, fmag, H, h, cfg.x0, cfg.y0)
    b = rhs(us, vs, Fx, Fy, bx, by, h, dt)
    res = mg_solve(bx, by, b, h, st.p, cfg.precision, cfg.tol, cfg.max_cycles, cfg.nu1,
                   cfg.nu2)
    u, v = correct(us, vs, res.p, Fx, Fy, bx, by, h, dt)
    U, V = interp(u, v, st.X, st.Y, h, cfg.x0, cfg.y0, cfg.kernel)
    st.u, st.v, st.p, st.au, st.av = u, v, res.p, au, av
    st.X = st.X + dt * U
    st.Y = st.Y + dt * V
    st.step += 1
    st.last = dict(H=H, rho=rho, bx=bx, by=by, Fx=Fx, Fy=Fy, b=b, cycles=res.cycles,
                   relres=res.relres, status=res.status, kappa=kap)
    return st


def _ns_step_axi(cfg: Config, st: State, dt: float) -> State:
    """The same stages in the axisymmetric form: the meridian curve is kept
    mirror-symmetric (after relocation and after advection), curvature adds
    the azimuthal term, the Heaviside and the irrotational force are the
    planar ones of the full curve on the real cells, the conventional force
    is ring-weighted, and the pressure equation is solved as the symmetric
    r-weighted system (coefficients r_face beta, right-hand side r_i b)."""
    h = cfg.h
    if cfg.frame and st.frame is None:
        c0 = drop_com_axi(st.X, st.Y, st.drop_start, 0)[1]
        st.frame = dict(com0=c0, com_prev=c0, S=0.0, Vf=0.0)
    S = st.frame["S"] if cfg.frame else 0.0
    wb = -st.frame["Vf"] if cfg.frame else 0.0
    _markers_update(cfg, st)
    kap, nxm, nym, ds = curvature_axi(st.X, st.Y, st.drop_start)
    fmag = cfg.sigma * kap
    H = heaviside(st.X, st.Y, st.drop_start, cfg.nx, cfg.ny, h, 0.0, cfg.y0)
    Ip = H if not cfg.indicator else indicator_poisson(st.X, st.Y, st.drop_start, cfg.nx,
                                                        cfg.ny, h, 0.0, cfg.y0, cfg.kernel, 1)
    rho, mu, bx, by = coeffs(Ip, cfg.rho_g, cfg.rho_l, cfg.mu_g, cfg.mu_l)
    if cfg.viscous:
        us, vs, au, av = predictor_axi(rho, 0.5 * mu, st.u, st.v, h, dt, st.au, st.av,
                                       (0.0, cfg.gy + S), wb)
        us, vs = cn_solve(rho, mu, us, vs, h, dt, cfg.cn_sweeps, 1, wb)
    else:
        us, vs, au, av = predictor_axi(rho, mu, st.u, st.v, h, dt, st.au, st.av,
                                       (0.0, cfg.gy + S), wb)
    if cfg.spread == 0:
        Fx, Fy = spread_conv_axi(st.X, st.Y - cfg.y0, fmag, nxm, nym, ds, cfg.nx, cfg.ny, h,
                                 cfg.kernel)
    else:
        Fx, Fy = spread_irrot(st.X, st.Y, st.drop_start, fmag, H, h, 0.0, cfg.y0)
    b = rhs_axi(us, vs, Fx, Fy, bx, by, h, dt)
    bxa, bya = axi_weights(bx, by, h)
    r = (np.arange(cfg.nx) + 0.5) * h
    res = mg_solve(bxa, bya, b * r[None, :], h, st.p, cfg.precision, cfg.tol, cfg.max_cycles,
                   cfg.nu1, cfg.nu2)
    u, v = correct(us, vs, res.p, Fx, Fy, bx, by, h, dt)
    v[0, :] = wb      # the z boundaries keep their prescribed axial velocity
    v[-1, :] = wb
    U, V = interp_axi(u, v, st.X, st.Y - cfg.y0, h, cfg.kernel)
    st.u, st.v, st.p, st.au, st.av = u, v, res.p, au, av
    st.X, st.Y = symmetrise(st.X + dt * U, st.Y + dt * V, st.drop_start)
    if cfg.frame:
        # Section 2.4 Eqs. (fictitious), (fic_1), (fic_2), read as a restoring
        # law on drop 0's centre of mass: the acceleration all fluid feels in
        # the next step, S = (c1 (COM_o - COM_n) - c2 (COM_n - COM_{n-1})) / dt^2;
        # the frame velocity changed by -S dt during this step.
        f = st.frame
        com = drop_com_axi(st.X, st.Y, st.drop_start, 0)[1]
        f["Vf"] = f["Vf"] - f["S"] * dt
        f["S"] = (cfg.c1 * (f["com0"] - com) - cfg.c2 * (com - f["com_prev"])) / (dt * dt)
        f["com_prev"] = com
    st.step += 1
    st.last = dict(H=H, rho=rho, bx=bx, by=by, Fx=Fx, Fy=Fy, b=b, cycles=res.cycles,
                   relres=res.relres, status=res.status, kappa=kap)
    return st
