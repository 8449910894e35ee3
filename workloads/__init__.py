"""Seeded synthetic inputs shared by the CUDA path's tests and benchmark and by
the oracle's tests.

This module holds input generation only (marker polylines, random fields):
none of the method's arithmetic.  Every generator is deterministic in its seed.

Workload recipes (the paper's static, oscillating and multi-drop setups,
Section 5; physical constants where the paper leaves them open: liquid
rho = 1, mu = 1e-2; gas rho = 1e-3, mu = 1e-4 for density ratio 1000 and
viscosity ratio 100; sigma = 1):
  static_drop_64     64 x 64 unit box, one drop R = 0.25 at (0.5, 0.5),
                     128 equispaced markers.
  oscillating_256    256 x 256 unit box, r(theta) = 0.2 (1 + 0.05 cos 2 theta)
                     about (0.5, 0.5), 512 markers, radial jitter uniform in
                     +-1e-3 (seed 1808).
  multidrop_N        N x N unit box (N = 1024, 2048), 64 non-overlapping drops,
                     radii U[0.01, 0.03], 256 markers each (seed 1811), drops at
                     least 8 cells from the walls and 8 cells apart.
  axisymmetric drops (x = r from the axis, y = z): the drop's full closed
                     meridian curve, marker 0 on the axis at the bottom, n/2 on
                     the axis at the top, marker k and n - k mirror images.
  freefall_axi       256 x 1024 cells over 4D x 16D (D = 1 mm), water drop
                     (rho 1000, mu 1e-3) in air (rho 1.2, mu 1.8e-5),
                     sigma = 0.072, g = 9.81, drop centre 4D above the bottom,
                     1024 markers on the full meridian (512 on the half profile).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Markers:
    X: np.ndarray
    Y: np.ndarray
    drop_start: np.ndarray  # int32, ndrops + 1 offsets

    @property
    def M(self) -> int:
        return len(self.X)

    @property
    def ndrops(self) -> int:
        return len(self.drop_start) - 1


def polar_drop(cx, cy, radius_fn, n, theta0=0.0):
    """Counter-clockwise closed polyline r(theta) about (cx, cy), n markers."""
    th = theta0 + 2.0 * np.pi * np.arange(n) / n
    r = radius_fn(th)
    return cx + r * np.cos(th), cy + r * np.sin(th)


def circle(cx, cy, R, n, theta0=0.0):
    return polar_drop(cx, cy, lambda t: np.full_like(t, R), n, theta0)


def join(drops) -> Markers:
    X = np.concatenate([d[0] for d in drops]).astype(np.float64)
    Y = np.concatenate([d[1] for d in drops]).astype(np.float64)
    starts = np.zeros(len(drops) + 1, np.int32)
    starts[1:] = np.cumsum([len(d[0]) for d in drops])
    return Markers(X, Y, starts)


def static_drop(n_cells=64, R=0.25, n_markers=128) -> Markers:
    return join([circle(0.5, 0.5, R, n_markers)])


def oscillating_drop(n_markers=512, r0=0.2, eps=0.05, jitter=1e-3, seed=1808) -> Markers:
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-jitter, jitter, n_markers)
    th = 2.0 * np.pi * np.arange(n_markers) / n_markers
    r = r0 * (1.0 + eps * np.cos(2.0 * th)) + jit
    return join([(0.5 + r * np.cos(th), 0.5 + r * np.sin(th))])


def elliptic_drop(cx, cy, r, beta, n_markers) -> Markers:
    """Section 5.2 Eq. (osc): x = cx + r cos(t) beta, y = cy + r sin(t) / beta."""
    th = 2.0 * np.pi * np.arange(n_markers) / n_markers
    return join([(cx + r * np.cos(th) * beta, cy + r * np.sin(th) / beta)])


def axi_drop(zc, radius_fn, n) -> Markers:
    """Axisymmetric drop centred on the axis at height zc: its full meridian
    curve r(theta) (counter-clockwise from the bottom axis point, theta =
    -pi/2 + 2 pi k / n, n even), markers k and n - k mirror images."""
    assert n % 2 == 0
    th = -0.5 * np.pi + 2.0 * np.pi * np.arange(n // 2 + 1) / n
    r = radius_fn(th)
    x, y = r * np.cos(th), zc + r * np.sin(th)
    x[0] = x[-1] = 0.0
    return join([_mirror(x, y)])


def _mirror(x, y):
    """Full closed curve from its right half (axis point to axis point):
    markers n - k are the reflections of markers k."""
    return np.concatenate([x, -x[-2:0:-1]]), np.concatenate([y, y[-2:0:-1]])


def axi_sphere(zc, R, n) -> Markers:
    return axi_drop(zc, lambda t: np.full_like(t, R), n)


def axi_elliptic_drop(zc, r, beta, n) -> Markers:
    """Section 5.2 Eq. (osc) about (0, zc): r' = r cos(t) beta, z = zc + r sin(t) / beta."""
    assert n % 2 == 0
    th = -0.5 * np.pi + 2.0 * np.pi * np.arange(n // 2 + 1) / n
    x, y = r * np.cos(th) * beta, zc + r * np.sin(th) / beta
    x[0] = x[-1] = 0.0
    return join([_mirror(x, y)])


def freefall_axi(n_markers=1024):
    """The free-fall water drop (SI units): returns (markers, constants)."""
    D = 1e-3
    nr, nz = 256, 1024
    h = 4 * D / nr
    mk = axi_sphere(4 * D, 0.5 * D, n_markers)
    const = dict(nx=nr, ny=nz, h=h, rho_l=1000.0, rho_g=1.2, mu_l=1e-3, mu_g=1.8e-5,
                 sigma=0.072, g=9.81)
    return mk, const


def multidrop(n_cells=1024, ndrops=64, rmin=0.01, rmax=0.03, n_per_drop=256,
              seed=1811, gap_cells=8) -> Markers:
    rng = np.random.default_rng(seed)
    h = 1.0 / n_cells
    gap = gap_cells * h
    centres, radii = [], []
    tries = 0
    while len(centres) < ndrops:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place drops")
        R = rng.uniform(rmin, rmax)
        c = rng.uniform(R + gap, 1.0 - R - gap, 2)
        ok = all(np.hypot(*(c - c2)) >= R + R2 + gap for c2, R2 in zip(centres, radii))
        if ok:
            centres.append(c)
            radii.append(R)
    drops = [circle(c[0], c[1], R, n_per_drop, theta0=rng.uniform(0, 2 * np.pi))
             for c, R in zip(centres, radii)]
    return join(drops)


def random_H(nx, ny, seed, smooth=True):
    """A smooth field in [0, 1] with sharp-ish transitions (a stand-in for a
    Heaviside field with several drops)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    Xg, Yg = np.meshgrid(x, y)
    H = np.zeros((ny, nx))
    for _ in range(4):
        cx, cy = rng.uniform(0.2, 0.8, 2)
        R = rng.uniform(0.08, 0.2)
        d = np.hypot(Xg - cx, Yg - cy) - R
        w = 1.5 / nx if smooth else 1e-9
        H = np.maximum(H, 0.5 * (1.0 - np.tanh(d / w)))
    return np.clip(H, 0.0, 1.0)


def random_faces(nx, ny, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-scale, scale, (ny, nx + 1))
    v = rng.uniform(-scale, scale, (ny + 1, nx))
    u[:, 0] = u[:, -1] = 0.0
    v[0, :] = v[-1, :] = 0.0
    return u, v


def random_cells(nx, ny, seed, scale=1.0):
    return np.random.default_rng(seed).uniform(-scale, scale, (ny, nx))


def capillary_dt(h, rho_l, rho_g, sigma, mu_l=None, mu_g=None, umax=0.0):
    """Time step: the capillary limit of Brackbill et al. (cited in Section 1),
    the explicit viscous limit and an advective CFL limit."""
    dt = 0.5 * np.sqrt((rho_l + rho_g) * h ** 3 / (4.0 * np.pi * sigma))
    if mu_l is not None and mu_g is not None:
        dt = min(dt, 0.25 * h * h * min(rho_l / mu_l, rho_g / mu_g))
    if umax > 0.0:
        dt = min(dt, 0.5 * h / umax)
    return float(dt)
