"""Pins of the oracle's time integration and of its variable-density
advection against facts the paper and the mathematics fix, independent of
how the oracle writes them:

* the oscillation period of a slightly elliptic drop, run through the
  oracle's own composed time step (Section 2.1 fractional step with the force
  in the projection, Section 3.2), against the closed forms Eq. (osc_p)
  (planar) and Eq. (aosc_p) (axisymmetric), within the discrepancy the
  paper's own table of periods (Section 5.2) prints for that grid spacing;
* momentum conservation of the flux-form advection of Section 2.1
  Eq. (ad_bf) with a random density field: the interior fluxes cancel in
  pairs, so with the fluid next to the walls at rest the total advective
  change of each momentum component is zero to roundoff;
* second-order consistency of that advection with the continuous operator
  div(rho u u) on smooth fields (planar and cylindrical), the derivatives
  of the continuous fluxes taken numerically from their analytic forms.
"""
import json
import os

import numpy as np
import pytest

import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


def _table(geometry, dx):
    rows = json.load(open(GOLD))["oscillation_period_table"]["rows"]
    return next(r for r in rows if r["geometry"] == geometry and r["dx"] == dx)


def _first_cycle_period(ts, ext, T):
    """Time of the first maximum of the deformation after t = 0.75 T (the
    drop starts at a maximum), by a parabola through the seven samples
    around the largest one."""
    k0 = int(np.searchsorted(ts, 0.75 * T))
    i = k0 + int(np.argmax(ext[k0:]))
    assert 3 <= i < len(ext) - 3, "no maximum inside the run"
    a, b, _ = np.polyfit(ts[i - 3:i + 4], ext[i - 3:i + 4], 2)
    return -b / (2 * a)


# Drop density 1, ambient 0.01 (the densities that reproduce the printed
# periods), viscosities 0.01 / 1e-5, sigma 1, R = 0.2 deformed by Eq. (osc)
# with beta = 1.03, n = 2 mode, B-spline relocation every 10 steps.
RHO_D, RHO_A, MU_D, MU_A, R0, BETA = 1.0, 0.01, 1e-2, 1e-5, 0.2, 1.03


@pytest.mark.parametrize("spread", [0, 1])
def test_planar_oscillation_period_of_the_oracle(O, spread):
    # Delta x = 0.02 on a 1.28 x 1.28 box (walls 3.2 radii from the centre;
    # 64 cells coarsen to 4).  Eq. (osc_p): T = 2 pi sqrt((rho_d + rho_a)
    # r^3 / ((n^3 - n) sigma)) = 0.23057.
    h, n = 0.02, 64
    mk = W.elliptic_drop(0.64, 0.64, R0, BETA, 128)
    cfg = O.Config(nx=n, ny=n, h=h, spread=spread, relocate_every=10, rho_l=RHO_D, rho_g=RHO_A,
                   mu_l=MU_D, mu_g=MU_A)
    st = O.init_state(cfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, RHO_D, RHO_A, 1.0, MU_D, MU_A)
    T = 2 * np.pi * np.sqrt((RHO_D + RHO_A) * R0 ** 3 / ((2 ** 3 - 2) * 1.0))
    assert abs(T - json.load(open(GOLD))["oscillation_period_2d"]["period"]) < 1e-5
    ts, ext = [], []
    for k in range(int(1.15 * T / dt)):
        O.ns_step(cfg, st, dt)
        assert st.last["status"] == 0
        ts.append((k + 1) * dt)
        ext.append((st.X.max() - st.X.min()) - (st.Y.max() - st.Y.min()))
    Tsim = _first_cycle_period(np.array(ts), np.array(ext), T)
    row = _table("2D", 0.02)
    # the paper's larger discrepancy at this grid spacing (new scheme, 4.57 %)
    tol = max(row["conventional"], row["new"])
    assert abs(Tsim - T) / T <= tol, (Tsim, T, abs(Tsim - T) / T)


@pytest.mark.parametrize("spread", [0, 1])
def test_axisymmetric_oscillation_period_of_the_oracle(O, spread):
    # Delta x = 0.02 on r in [0, 0.64], z in [0, 1.28]: 32 x 64 cells
    # (coarsen to 2 x 4).  Eq. (aosc_p): T = 2 pi sqrt(((n + 1) rho_d + n rho_a)
    # r^3 / (n (n - 1)(n + 1)(n + 2) sigma)) = 0.19935.
    h, nx, ny = 0.02, 32, 64
    mk = W.axi_elliptic_drop(0.64, R0, BETA, 128)
    cfg = O.Config(nx=nx, ny=ny, h=h, axisym=1, spread=spread, relocate_every=10, rho_l=RHO_D,
                   rho_g=RHO_A, mu_l=MU_D, mu_g=MU_A)
    st = O.init_state(cfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, RHO_D, RHO_A, 1.0, MU_D, MU_A)
    T = 2 * np.pi * np.sqrt((3 * RHO_D + 2 * RHO_A) * R0 ** 3 / (2 * 1 * 3 * 4 * 1.0))
    assert abs(T - json.load(open(GOLD))["oscillation_period_axisym"]["period"]) < 1e-5
    ts, ext = [], []
    for k in range(int(1.15 * T / dt)):
        O.ns_step(cfg, st, dt)
        assert st.last["status"] == 0
        ts.append((k + 1) * dt)
        ext.append((st.X.max() - st.X.min()) - (st.Y.max() - st.Y.min()))
    Tsim = _first_cycle_period(np.array(ts), np.array(ext), T)
    row = _table("axisymmetric", 0.02)
    tol = max(row["conventional"], row["new"])  # 4.84 %
    assert abs(Tsim - T) / T <= tol, (Tsim, T, abs(Tsim - T) / T)


# ----------------------------------------------------------------- advection
def _random_flow(nx, ny, seed):
    """Random positive density and random velocities that vanish on the
    faces next to every wall (faces 0, 1, n-1, n in the normal direction), so
    that no momentum flux crosses the boundary of the interior control
    volumes."""
    rng = np.random.default_rng(seed)
    rho = 10.0 ** rng.uniform(-3.0, 0.0, (ny, nx))  # density ratio up to 1000
    u = rng.standard_normal((ny, nx + 1))
    v = rng.standard_normal((ny + 1, nx))
    u[:, [0, 1, -2, -1]] = 0.0
    v[[0, 1, -2, -1], :] = 0.0
    return rho, u, v


def test_planar_advection_conserves_momentum(O):
    nx, ny, h = 24, 20, 0.05
    rho, u, v = _random_flow(nx, ny, 61)
    _, _, au, av = O.predictor(rho, np.zeros_like(rho), u, v, h, 1e-3)
    # total change of x and y momentum over the u- and v-control volumes (area h^2)
    for a in (au, av):
        assert abs(a.sum() * h * h) <= 1e-13 * np.abs(a).sum() * h * h


def test_axisymmetric_advection_conserves_momentum(O):
    # ring control volumes r0 h^2 per radian: r0 the radius of the face
    nx, ny, h = 24, 20, 0.05
    rho, u, v = _random_flow(nx, ny, 62)
    _, _, au, av = O.predictor_axi(rho, np.zeros_like(rho), u, v, h, 1e-3)
    ru = (np.arange(nx + 1) * h)[None, :]
    rv = ((np.arange(nx) + 0.5) * h)[None, :]
    for a, r in ((au, ru), (av, rv)):
        w = a * r * h * h
        assert abs(w.sum()) <= 1e-13 * np.abs(w).sum()


def _d(f, x, y, axis, d=1e-3):
    """Fourth-order central difference of an analytic function."""
    if axis == 0:
        return (-f(x + 2 * d, y) + 8 * f(x + d, y) - 8 * f(x - d, y) + f(x - 2 * d, y)) / (12 * d)
    return (-f(x, y + 2 * d) + 8 * f(x, y + d) - 8 * f(x, y - d) + f(x, y - 2 * d)) / (12 * d)


PI = np.pi
# smooth fields on the unit square, zero on every wall (no-slip), density
# varying by a factor of about 2.5
U = lambda x, y: np.sin(PI * x) * np.sin(PI * y) * (1 + 0.3 * x)
V = lambda x, y: np.sin(PI * x) * np.sin(PI * y) * (0.5 - 0.4 * y)
RHO = lambda x, y: 1.5 + 0.5 * np.cos(PI * x) * np.cos(2 * PI * y) + 0.2 * x


def _planar_errors(O, n):
    h = 1.0 / n
    xc, xf = (np.arange(n) + 0.5) * h, np.arange(n + 1) * h
    XU, YU = np.meshgrid(xf, xc)
    XV, YV = np.meshgrid(xc, xf)
    rho = RHO(*np.meshgrid(xc, xc))
    _, _, au, av = O.predictor(rho, np.zeros_like(rho), U(XU, YU), V(XV, YV), h, 1e-3)
    # div(rho u u): x-component at the u-faces, y-component at the v-faces
    Ax = _d(lambda x, y: RHO(x, y) * U(x, y) ** 2, XU, YU, 0) + \
        _d(lambda x, y: RHO(x, y) * U(x, y) * V(x, y), XU, YU, 1)
    Ay = _d(lambda x, y: RHO(x, y) * U(x, y) * V(x, y), XV, YV, 0) + \
        _d(lambda x, y: RHO(x, y) * V(x, y) ** 2, XV, YV, 1)
    return np.abs(au - Ax)[:, 1:-1].max(), np.abs(av - Ay)[1:-1, :].max()


def test_planar_advection_is_second_order_consistent(O):
    e = [_planar_errors(O, n) for n in (16, 32, 64)]
    for c in (0, 1):
        for k in range(2):
            assert e[k][c] / e[k + 1][c] > 3.6, e  # error falls as h^2
    assert max(e[-1]) < 2e-2


# cylindrical (r, z) fields on [0, 1]^2: u odd in r and zero on the axis and
# the outer wall, w even in r, both zero at z = 0, 1; density even in r
UA = lambda r, z: np.sin(PI * r) * (1 + 0.3 * r * r) * np.sin(PI * z)
WA = lambda r, z: 0.5 * (1 + np.cos(PI * r)) * np.sin(PI * z) * (0.5 - 0.4 * z)
RHOA = lambda r, z: 1.5 + 0.5 * np.cos(PI * r) * np.cos(2 * PI * z) + 0.2 * r * r


def _axi_errors(O, n):
    h = 1.0 / n
    xc, xf = (np.arange(n) + 0.5) * h, np.arange(n + 1) * h
    XU, YU = np.meshgrid(xf, xc)
    XV, YV = np.meshgrid(xc, xf)
    rho = RHOA(*np.meshgrid(xc, xc))
    u, w = UA(XU, YU), WA(XV, YV)
    _, _, au, av = O.predictor_axi(rho, np.zeros_like(rho), u, w, h, 1e-3)
    # radial: (1/r) d(r rho u^2)/dr + d(rho u w)/dz, compared where r >= 1/4
    # (near the axis a ring volume's average and its face value differ at
    # first order); axial: (1/r) d(r rho u w)/dr + d(rho w^2)/dz everywhere
    rs = np.where(XU > 0, XU, 1.0)
    Ar = _d(lambda r, z: r * RHOA(r, z) * UA(r, z) ** 2, XU, YU, 0) / rs + \
        _d(lambda r, z: RHOA(r, z) * UA(r, z) * WA(r, z), XU, YU, 1)
    Az = _d(lambda r, z: r * RHOA(r, z) * UA(r, z) * WA(r, z), XV, YV, 0) / XV + \
        _d(lambda r, z: RHOA(r, z) * WA(r, z) ** 2, XV, YV, 1)
    far = (XU >= 0.25) & (XU < 1.0)
    e_r, e_z = np.abs(au - Ar)[far].max(), np.abs(av - Az)[1:-1, :].max()
    # every radial face, the axis included, against the exact ring-volume
    # average of the radial part: the flux r rho u^2 taken exactly at the
    # volume's two radii, their difference over r0 h (w = 0 isolates it)
    _, _, au0, _ = O.predictor_axi(rho, np.zeros_like(rho), u, 0 * w, h, 1e-3)
    F = lambda r, z: r * RHOA(r, z) * UA(r, z) ** 2
    cv = (F(XU + h / 2, YU) - F(XU - h / 2, YU)) / (rs * h)
    e_cv = np.abs(au0 - cv)[:, 1:-1].max()
    return e_r, e_z, e_cv


def test_axisymmetric_advection_is_second_order_consistent(O):
    e = [_axi_errors(O, n) for n in (16, 32, 64)]
    for c in range(3):
        for k in range(2):
            assert e[k][c] / e[k + 1][c] > 3.6, e
    assert max(e[-1]) < 2e-2
