"""GPU parity of the axisymmetric (r, z) path against the oracle on the same
seeded inputs: marker geometry with the azimuthal curvature, the Heaviside
and face forces of the full meridian curve folded onto the real grid,
mirrored interpolation, the ring-volume predictor and right-hand side, and
composed time steps (static sphere: Laplace jump 2 sigma / R; deforming
ellipsoid: both spreadings with relocation and re-symmetrisation)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def T():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch


@pytest.fixture(scope="module")
def ib():
    import paper_1807_10504_gb300 as ib
    ib.lib()
    return ib


def ctx_axi(ib, nx, ny, h, mk, **kw):
    cfg = ib.Config(nx=nx, ny=ny, h=h, axisym=1, **kw)
    return ib.Context(cfg, mk.X, mk.Y, mk.drop_start), cfg


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_geometry_matches_oracle(T, ib, O):
    mk = W.axi_elliptic_drop(1.0, 0.3, 1.2, 160)
    ctx, _ = ctx_axi(ib, 32, 64, 1 / 32, mk)
    k, nxm, nym, ds = (a.cpu().numpy() for a in ctx.geometry())
    ko, nxo, nyo, dso = O.curvature_axi(mk.X, mk.Y, mk.drop_start)
    assert rel(k, ko) <= 1e-13 and rel(nxm, nxo) <= 1e-14 and rel(ds, dso) <= 1e-14
    # a sphere: 2/R at every marker, the two axis markers included
    sp = W.axi_sphere(1.0, 0.25, 128)
    ctx2, _ = ctx_axi(ib, 32, 64, 1 / 32, sp)
    k2 = ctx2.geometry()[0].cpu().numpy()
    assert np.abs(k2 - 8.0).max() < 1e-11


@pytest.mark.parametrize("nx,ny", [(32, 64), (40, 56)])
def test_heaviside_matches_oracle(T, ib, O, nx, ny):
    h = 1.0 / 32
    mk = W.axi_elliptic_drop(0.9, 0.35, 1.15, 200)
    ctx, _ = ctx_axi(ib, nx, ny, h, mk)
    H = ctx.heaviside().cpu().numpy()
    Ho = O.heaviside(mk.X, mk.Y, mk.drop_start, nx, ny, h, 0.0, 0.0)
    assert np.abs(H - Ho).max() <= 1e-13 + 8 * max(nx, ny) * 2.0**-53
    assert H.min() >= -1e-14 and H.max() <= 1 + 1e-14


def test_interp_matches_oracle(T, ib, O):
    nx, ny, h = 32, 64, 1 / 32
    mk = W.axi_elliptic_drop(1.0, 0.3, 1.2, 160)
    ctx, _ = ctx_axi(ib, nx, ny, h, mk)
    u, v = W.random_faces(nx, ny, 31)
    u[:, 0] = 0.0
    d = lambda a: T.from_numpy(np.ascontiguousarray(a)).cuda()
    for kernel in (0, 1):
        ctx.close()
        ctx, _ = ctx_axi(ib, nx, ny, h, mk, kernel=kernel)
        U, V = (a.cpu().numpy() for a in ctx.interp(d(u), d(v)))
        Uo, Vo = O.interp_axi(u, v, mk.X, mk.Y, h, kernel)
        assert rel(U, Uo) <= 1e-13 and rel(V, Vo) <= 1e-13


@pytest.mark.parametrize("kernel", [0, 1])
def test_spreading_matches_oracle(T, ib, O, kernel):
    nx, ny, h = 32, 64, 1 / 32
    mk = W.axi_elliptic_drop(1.0, 0.3, 1.2, 160)
    ctx, cfg = ctx_axi(ib, nx, ny, h, mk, kernel=kernel)
    k, nxm, nym, ds = O.curvature_axi(mk.X, mk.Y, mk.drop_start)
    fmag = cfg.sigma * k
    Fx, Fy = (a.cpu().numpy() for a in ctx.spread(0))
    Fxo, Fyo = O.spread_conv_axi(mk.X, mk.Y, fmag, nxm, nym, ds, nx, ny, h, kernel)
    scale = max(np.abs(Fxo).max(), np.abs(Fyo).max())
    assert np.abs(Fx - Fxo).max() <= 1e-12 * scale and np.abs(Fy - Fyo).max() <= 1e-12 * scale
    Fx, Fy, H = (a.cpu().numpy() for a in ctx.spread(1, want_H=True))
    Ho = O.heaviside(mk.X, mk.Y, mk.drop_start, nx, ny, h, 0.0, 0.0)
    Fxo, Fyo = O.spread_irrot(mk.X, mk.Y, mk.drop_start, fmag, Ho, h, 0.0, 0.0)
    scale = max(np.abs(Fxo).max(), np.abs(Fyo).max())
    assert np.abs(Fx - Fxo).max() <= 1e-11 * scale and np.abs(Fy - Fyo).max() <= 1e-11 * scale


def test_predictor_rhs_weights_match_oracle(T, ib, O):
    nx, ny, h, dt = 40, 72, 1 / 40, 2e-4
    H = W.random_H(nx, ny, 41)
    rho, mu, bx, by = O.coeffs(H, 1e-3, 1.0, 1e-4, 1e-2)
    u, v = W.random_faces(nx, ny, 42)
    aup, avp = W.random_faces(nx, ny, 43)
    Fx, Fy = W.random_faces(nx, ny, 44, scale=20.0)
    d = lambda a: T.from_numpy(np.ascontiguousarray(a)).cuda()
    for have in (False, True):
        us, vs, au, av = ib.ib_op_predictor_axi(d(rho), d(mu), d(u), d(v), h, dt,
                                                d(aup) if have else None,
                                                d(avp) if have else None, gy=-9.81)
        o = O.predictor_axi(rho, mu, u, v, h, dt, aup if have else None, avp if have else None,
                            (0.0, -9.81))
        for g, r in zip((us, vs, au, av), o):
            assert np.abs(g.cpu().numpy() - r).max() <= 1e-12 * max(np.abs(r).max(), 1.0)
    # with a frame record: extra axial acceleration S, moving boundaries wb
    us, vs, au, av = ib.ib_op_predictor_axi(d(rho), d(mu), d(u), d(v), h, dt, d(aup), d(avp),
                                            gy=-9.81, S=0.37, wb=0.21)
    o = O.predictor_axi(rho, mu, u, v, h, dt, aup, avp, (0.0, -9.81 + 0.37), 0.21)
    for g, r in zip((us, vs, au, av), o):
        assert np.abs(g.cpu().numpy() - r).max() <= 1e-12 * max(np.abs(r).max(), 1.0)
    assert np.all(vs.cpu().numpy()[[0, -1]] == 0.21)
    us, vs = W.random_faces(nx, ny, 45)
    us[:, 0] = 0.0
    b = ib.ib_op_rhs_axi(d(us), d(vs), d(Fx), d(Fy), d(bx), d(by), h, dt).cpu().numpy()
    r = (np.arange(nx) + 0.5) * h
    bo = r[None, :] * O.rhs_axi(us, vs, Fx, Fy, bx, by, h, dt)
    assert rel(b, bo) <= 1e-13
    bxa, bya = (a.cpu().numpy() for a in ib.ib_op_axi_weights(d(bx), d(by), h))
    bxo, byo = O.axi_weights(bx, by, h)
    assert np.array_equal(bxa, bxo) and np.array_equal(bya, byo)


def test_static_sphere_step_matches_oracle(T, ib, O):
    nx, ny, R = 32, 64, 0.25
    h = 1.0 / nx
    mk = W.axi_sphere(1.0, R, 128)
    ctx, cfg = ctx_axi(ib, nx, ny, h, mk, spread=1, relocate_every=0, tol=1e-12)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    cyc, rr = ctx.ns_step(dt, 1, 1)
    ocfg = O.Config(nx=nx, ny=ny, h=h, spread=1, relocate_every=0, axisym=1, tol=1e-12)
    st = O.init_state(ocfg, mk.X, mk.Y, mk.drop_start)
    O.ns_step(ocfg, st, dt)
    p = ctx.get("p").cpu().numpy()
    assert rel(p, st.p) <= 1e-10
    jump = p[32, 1] - p[2, nx - 2]
    assert abs(jump - 2.0 / R) < 1e-9 * (2.0 / R)
    assert max(np.abs(ctx.get("u").cpu().numpy()).max(), np.abs(ctx.get("v").cpu().numpy()).max()) < 1e-9


@pytest.mark.parametrize("spread,precision", [(0, 0), (1, 0), (1, 2)])
def test_steps_match_oracle(T, ib, O, spread, precision):
    # A deforming ellipsoid (Section 5.2 Eq. (osc) about the axis, beta 1.1):
    # relocation every 2 steps (with re-symmetrisation), 4 steps; the FP64
    # path to 1e-10 of the oracle (p relative to max |p|, u and w relative to
    # the inertial-capillary velocity sqrt(sigma / (rho_l R))), the
    # mixed-precision path (refined to the same residual) to 1e-6.
    nx, ny = 32, 64
    h = 1.0 / nx
    mk = W.axi_elliptic_drop(1.0, 0.25, 1.1, 128)
    kw = dict(spread=spread, relocate_every=2, tol=1e-11)
    ctx, cfg = ctx_axi(ib, nx, ny, h, mk, precision=precision, **kw)
    ocfg = O.Config(nx=nx, ny=ny, h=h, axisym=1, precision=0, **kw)
    st = O.init_state(ocfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    for _ in range(4):
        ctx.ns_step(dt, 1, 1)
        O.ns_step(ocfg, st, dt)
    tol = 1e-10 if precision == 0 else 1e-6
    X, Y = (a.cpu().numpy() for a in ctx.markers())
    xtol = 1e-12 if precision == 0 else 1e-9
    assert np.abs(X - st.X).max() <= xtol and np.abs(Y - st.Y).max() <= xtol
    n = len(X)
    k = np.arange(n)
    assert np.array_equal(X, -X[(n - k) % n]) and np.array_equal(Y, Y[(n - k) % n])
    U = np.sqrt(1.0 / (1.0 * 0.25))
    ep = rel(ctx.get("p").cpu().numpy(), st.p)
    assert ep <= tol, ep
    for name, ref in (("u", st.u), ("v", st.v)):
        e = np.abs(ctx.get(name).cpu().numpy() - ref).max() / U
        assert e <= tol, (name, e)


def test_rejects_curves_that_are_not_meridians(T, ib):
    mk = W.axi_sphere(1.0, 0.25, 64)
    X = mk.X.copy()
    X[5] += 1e-9  # not mirror-symmetric
    with pytest.raises(ib.IBError):
        ib.Context(ib.Config(nx=32, ny=64, h=1 / 32, axisym=1), X, mk.Y, mk.drop_start)
    with pytest.raises(ib.IBError):  # odd marker count
        ib.Context(ib.Config(nx=32, ny=64, h=1 / 32, axisym=1), mk.X[:63], mk.Y[:63],
                   np.array([0, 63], np.int32))
    with pytest.raises(ib.IBError):  # the axis must be at x0 = 0
        ib.Context(ib.Config(nx=32, ny=64, h=1 / 32, axisym=1, x0=0.1), mk.X, mk.Y,
                   mk.drop_start)


def test_free_fall_frame_matches_oracle(T, ib, O):
    # Gravity and the non-inertial frame (Section 2.4): 40 steps of a dense
    # sphere released from rest; the frame record, the fields and the markers
    # follow the oracle's: p within 1e-10 of max |p|, u and w within 1e-10 of
    # the inertial-capillary velocity (measured: ~2e-13 and ~6e-13).  The
    # frame's acceleration divides centre-of-mass differences by dt^2 (~6e-7
    # here), which lifts rounding differences of the positions (~1e-16) to
    # ~1e-10 in S; S itself is compared at 1e-6.
    nx, ny, h, R = 32, 96, 1 / 32, 0.25
    mk = W.axi_sphere(1.0, R, 96)
    kw = dict(axisym=1, frame=1, gy=-1.0, relocate_every=10, spread=1, tol=1e-11)
    ctx = ib.Context(ib.Config(nx=nx, ny=ny, h=h, **kw), mk.X, mk.Y, mk.drop_start)
    ocfg = O.Config(nx=nx, ny=ny, h=h, **kw)
    st = O.init_state(ocfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    for _ in range(40):
        ctx.ns_step(dt, 1, 1)
        O.ns_step(ocfg, st, dt)
    com, S, vf, wb = ctx.frame_state()
    f = st.frame
    assert abs(vf - f["Vf"]) <= 1e-7 * abs(f["Vf"]) and abs(wb + vf) == 0.0
    assert abs(com - f["com_prev"]) <= 1e-12
    assert abs(S - f["S"]) <= 1e-6 * max(abs(f["S"]), 1.0)
    ep = rel(ctx.get("p").cpu().numpy(), st.p)
    U = np.sqrt(1.0 / (1.0 * R))
    eu = max(np.abs(ctx.get(n).cpu().numpy() - r).max() for n, r in (("u", st.u), ("v", st.v))) / U
    assert ep <= 1e-10 and eu <= 1e-10, (ep, eu)
    X, Y = (a.cpu().numpy() for a in ctx.markers())
    assert np.abs(X - st.X).max() <= 1e-12 and np.abs(Y - st.Y).max() <= 1e-12
    with pytest.raises(ib.IBError):  # the frame needs the axisymmetric form
        ib.Context(ib.Config(nx=32, ny=32, h=1 / 32, frame=1), *W.circle(0.5, 0.5, 0.2, 32),
                   np.array([0, 32], np.int32))


def test_axisymmetric_oscillation_period(T, ib):
    # Section 5.2's axisymmetric oscillating drop at the paper's grid 0.01 (the
    # domain 1.28 x 2.56 instead of 2 x 2, so that the multigrid coarsens to
    # 4 x 8 cells; the walls stay 5 radii away), R = 0.2 about the axis
    # deformed by Eq. (osc) with beta = 1.03, drop
    # density 1 and ambient 0.01 (the densities that reproduce the printed
    # periods), viscosities 0.01 / 1e-5, sigma 1, irrotational spreading with
    # B-spline relocation.  The first extremum of the r-extent minus the
    # z-extent falls at half the closed-form n = 2 period of Eq. (aosc_p),
    # 2 pi sqrt(((n+1) rho_d + n rho_a) r^3 / (n (n-1)(n+1)(n+2) sigma)) =
    # 0.19935, within 5 % (the paper's own discrepancy at this grid: 1.53 %).
    h = 0.01
    mk = W.axi_elliptic_drop(1.28, 0.2, 1.03, 256)
    cfg = ib.Config(nx=128, ny=256, h=h, axisym=1, rho_l=1.0, rho_g=0.01, mu_l=0.01, mu_g=1e-5,
                    sigma=1.0, spread=1, relocate_every=10, precision=2, tol=1e-10,
                    max_cycles=200)
    ctx = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, 1.0, 0.01, 1.0, 0.01, 1e-5)
    ext, ts = [], []
    for k in range(110):
        ctx.ns_step(dt, 10, 1)
        X, Y = ctx.markers()
        ext.append(float(X.max() - X.min()) - float(Y.max() - Y.min()))
        ts.append(10 * (k + 1) * dt)
    ext = np.array(ext)
    i = int(np.argmin(ext))  # starts wider in r than tall in z: first minimum at T/2
    assert 0 < i < len(ext) - 1
    a, b, c = np.polyfit(np.array(ts[i - 1:i + 2]), ext[i - 1:i + 2], 2)
    t_half = -b / (2 * a)
    Ta = 2 * np.pi * np.sqrt((3 * 1.0 + 2 * 0.01) * 0.2 ** 3 / (2 * 1 * 3 * 4 * 1.0))
    assert abs(Ta - 0.19935) < 1e-5
    assert abs(2 * t_half - Ta) <= 0.05 * Ta, (2 * t_half, Ta)
