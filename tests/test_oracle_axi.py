"""Pins of the axisymmetric (r, z) oracle against what the mathematics fixes:
polynomial exactness of the ring finite-volume operators, the r-weighted
symmetric form against a dense solve of the direct finite-volume operator,
a discretely divergence-free projection, the curvature of a sphere (Section
4 Eq. (curv_ax)), exact ring-force conservation, mirror interpolation of
linear fields, the volume and centre of mass of revolution against brute
force, and the Laplace jump 2 sigma / R of a static sphere (Section 5.1)."""
import numpy as np
import pytest

import workloads as W


def _walls(bx, by):
    bx[:, 0] = bx[:, -1] = 0.0
    by[0, :] = by[-1, :] = 0.0
    return bx, by


def _unit_beta(nx, ny):
    return _walls(np.ones((ny, nx + 1)), np.ones((ny + 1, nx)))


def test_pressure_operator_is_exact_on_quadratics(O):
    # (1/r) d/dr (r dp/dr) of r^2 is 4 and d2/dz2 of z^2 is 2; the ring
    # finite-volume operator reproduces both exactly away from the walls
    # (the axis needs no exclusion: its face has zero area).
    nx, ny, h = 12, 10, 0.1
    bx, by = _unit_beta(nx, ny)
    r = (np.arange(nx) + 0.5) * h
    z = (np.arange(ny) + 0.5) * h
    R, Z = np.meshgrid(r, z)
    a = O.apply_A_axi(bx, by, R**2, h)
    assert np.abs(a[:, : nx - 1] - 4.0).max() < 1e-11
    b = O.apply_A_axi(bx, by, Z**2 + 3.0 * R**2 - 7.0, h)
    assert np.abs(b[1:-1, : nx - 1] - 14.0).max() < 1e-11


def test_weighted_form_is_r_times_the_operator(O):
    nx, ny, h = 16, 12, 1 / 16
    H = W.random_H(nx, ny, 4)
    rho, mu, bx, by = O.coeffs(H, 1e-3, 1.0, 1e-4, 1e-2)
    p = W.random_cells(nx, ny, 5)
    bxa, bya = O.axi_weights(bx, by, h)
    r = (np.arange(nx) + 0.5) * h
    lhs = O.apply_A(bxa, bya, p, h)
    rhs = r[None, :] * O.apply_A_axi(bx, by, p, h)
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(rhs).max()
    assert np.all(bxa[:, 0] == 0.0)  # the axis face has zero area


@pytest.mark.parametrize("nx,ny", [(8, 8), (12, 16)])
def test_multigrid_on_weighted_form_matches_dense_fv_solve(O, nx, ny):
    # Dense matrix of the direct ring finite-volume operator (columns by
    # applying it to unit vectors), solved by least squares with the mean of
    # p fixed to zero, against multigrid on the symmetric weighted form.
    h = 1.0 / nx
    H = W.random_H(nx, ny, 6)
    rho, mu, bx, by = O.coeffs(H, 1e-3, 1.0, 1e-4, 1e-2)
    n = nx * ny
    A = np.empty((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = O.apply_A_axi(bx, by, e.reshape(ny, nx), h).ravel()
    r = (np.arange(nx) + 0.5) * h
    b = W.random_cells(nx, ny, 7)
    rw = np.tile(r, ny)
    b = b - (rw @ b.ravel()) / rw.sum()   # compatible: sum r b = 0
    M = np.vstack([A, np.ones((1, n))])
    pd = np.linalg.lstsq(M, np.concatenate([b.ravel(), [0.0]]), rcond=None)[0].reshape(ny, nx)
    assert np.abs(A @ pd.ravel() - b.ravel()).max() < 1e-8 * np.abs(b).max()
    bxa, bya = O.axi_weights(bx, by, h)
    res = O.mg_solve(bxa, bya, b * r[None, :], h, tol=1e-13, max_cycles=300)
    assert res.status == 0
    assert np.abs(res.p - pd).max() <= 1e-9 * np.abs(pd).max()


def test_projection_is_discretely_divergence_free(O):
    nx, ny, h, dt = 24, 32, 1 / 24, 1e-3
    H = W.random_H(nx, ny, 8)
    rho, mu, bx, by = O.coeffs(H, 1e-3, 1.0, 1e-4, 1e-2)
    us, vs = W.random_faces(nx, ny, 9)
    Fx, Fy = W.random_faces(nx, ny, 10, scale=30.0)
    us[:, 0] = 0.0  # no flow through the axis
    b = O.rhs_axi(us, vs, Fx, Fy, bx, by, h, dt)
    r = (np.arange(nx) + 0.5) * h
    bxa, bya = O.axi_weights(bx, by, h)
    res = O.mg_solve(bxa, bya, b * r[None, :], h, tol=1e-13, max_cycles=300)
    assert res.status == 0
    u, v = O.correct(us, vs, res.p, Fx, Fy, bx, by, h, dt)
    d0 = np.abs(O.divergence_axi(us, vs, h)).max()
    assert np.abs(O.divergence_axi(u, v, h)).max() < 1e-9 * d0
    assert np.all(u[:, 0] == 0.0)


def test_viscous_terms_exact_on_textbook_fields(O):
    # Vector diffusion in cylindrical coordinates: u_r = r is harmonic
    # ((1/r)(r u')' - u/r^2 = 0) and w = r^2 has (1/r)(r w')' = 4.  The
    # difference of two predictor steps with mu = 1 and mu = 0 isolates the
    # viscous term; both identities hold exactly in the discrete operator.
    nx, ny, h, dt = 10, 8, 0.1, 1e-3
    rho = np.ones((ny, nx))
    r_face = np.arange(nx + 1) * h
    r_cell = (np.arange(nx) + 0.5) * h
    u = np.tile(r_face, (ny, 1))
    u[:, -1] = 0.0
    v = np.tile(r_cell**2, (ny + 1, 1))
    outs = {}
    for m in (0.0, 1.0):
        us, vs, _, _ = O.predictor_axi(rho, np.full((ny, nx), m), u, v, h, dt)
        outs[m] = (us, vs)
    du = (outs[1.0][0] - outs[0.0][0]) / dt
    dv = (outs[1.0][1] - outs[0.0][1]) / dt
    assert np.abs(du[1:-1, 1 : nx - 1]).max() < 1e-9
    assert np.abs(dv[1:-1, : nx - 1] - 4.0).max() < 1e-9


def test_sphere_curvature_is_two_over_R(O):
    for R, n in ((0.25, 128), (0.3, 64)):
        mk = W.axi_sphere(0.5, R, n)
        k, nxm, nym, ds = O.curvature_axi(mk.X, mk.Y, mk.drop_start)
        assert np.abs(k - 2.0 / R).max() < 1e-11 * (2.0 / R)


def test_volume_and_centre_of_mass_of_revolution(O):
    # A cylinder r <= a, b <= z <= c (its meridian rectangle, both halves):
    # V = pi a^2 (c - b), z_c = (b + c) / 2 exactly.
    a, b, c = 0.3, 0.2, 0.9
    x = np.array([0.0, a, a, 0.0])
    y = np.array([b, b, c, c])
    X = np.concatenate([x, -x[-2:0:-1]])
    Y = np.concatenate([y, y[-2:0:-1]])
    vol, zc = O.drop_com_axi(X, Y, np.array([0, len(X)], np.int32))
    assert abs(vol - np.pi * a * a * (c - b)) < 1e-14 and abs(zc - 0.5 * (b + c)) < 1e-14
    # an ellipse meridian against brute-force sampling of 2 pi r over the
    # cells of a fine (r, z) lattice inside the polygon
    mk = W.axi_elliptic_drop(0.6, 0.2, 1.3, 96)
    vol, zc = O.drop_com_axi(mk.X, mk.Y, mk.drop_start)
    ng = 1200
    rr = (np.arange(ng) + 0.5) * (0.3 / ng)
    zz = 0.4 + (np.arange(ng) + 0.5) * (0.4 / ng)
    Rg, Zg = np.meshgrid(rr, zz)
    inside = _inside(mk.X, mk.Y, Rg.ravel(), Zg.ravel()).reshape(Rg.shape)
    dA = (0.3 / ng) * (0.4 / ng)
    vb = 2 * np.pi * (Rg * inside).sum() * dA
    zb = (Rg * Zg * inside).sum() / (Rg * inside).sum()
    assert abs(vol - vb) < 3e-3 * vb and abs(zc - zb) < 1e-4


def _inside(X, Y, px, py):
    # crossing number, vectorised over the query points
    cnt = np.zeros(px.shape, int)
    n = len(X)
    for m in range(n):
        ax, ay, bx, by = X[m], Y[m], X[(m + 1) % n], Y[(m + 1) % n]
        cross = (ay > py) != (by > py)
        with np.errstate(divide="ignore", invalid="ignore"):
            xc = ax + (py - ay) * (bx - ax) / (by - ay)
        cnt += cross & (xc > px)
    return (cnt & 1).astype(float)


def test_ring_force_spreading_conserves_the_axial_force(O):
    # Sum over the real y-faces of F_z r_f h^2 = (1/2) sum over all markers of
    # f_z ds |r_m| (each mirror pair shares its kernel weight between the
    # real faces and their mirror images).
    nx, ny, h = 24, 32, 1 / 24
    mk = W.axi_elliptic_drop(0.6, 0.3, 1.1, 80)
    k, nxm, nym, ds = O.curvature_axi(mk.X, mk.Y, mk.drop_start)
    Fx, Fy = O.spread_conv_axi(mk.X, mk.Y, k, nxm, nym, ds, nx, ny, h, kernel=1)
    r = (np.arange(nx) + 0.5) * h
    lhs = (Fy * r[None, :]).sum() * h * h
    rhs = 0.5 * (k * nym * ds * np.abs(mk.X)).sum()
    assert abs(lhs - rhs) < 1e-12 * np.abs(k * nym * ds * np.abs(mk.X)).sum()
    assert np.all(Fx[:, 0] == 0.0) and np.all(Fx[:, -1] == 0.0)


def test_mirror_interpolation_of_linear_fields(O):
    # u = r (odd continuation r) and w = z (even continuation z): the Peskin
    # kernel (zero first moment) reproduces linear fields exactly, on both
    # halves of the curve, markers on the axis included.
    nx, ny, h = 16, 24, 1 / 16
    u = np.tile(np.arange(nx + 1) * h, (ny, 1))
    v = np.tile((np.arange(ny + 1) * h)[:, None], (1, nx))
    mk = W.axi_elliptic_drop(0.75, 0.3, 1.2, 64)
    U, V = O.interp_axi(u, v, mk.X, mk.Y, h, kernel=1)
    assert np.abs(U - mk.X).max() < 1e-13 and np.abs(V - mk.Y).max() < 1e-13


def test_static_sphere_laplace_jump(O):
    # One step of the static sphere with the irrotational force and no
    # relocation: the exact curvature 2/R is constant along the interface,
    # the force is a discrete gradient, the velocity stays zero to roundoff
    # and the pressure jump is 2 sigma / R.
    nx, ny, R = 32, 64, 0.25
    h = 1.0 / nx
    mk = W.axi_sphere(1.0, R, 128)
    cfg = O.Config(nx=nx, ny=ny, h=h, spread=1, relocate_every=0, axisym=1, tol=1e-12)
    st = O.init_state(cfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    O.ns_step(cfg, st, dt)
    assert st.last["status"] == 0
    assert max(np.abs(st.u).max(), np.abs(st.v).max()) < 1e-9
    p = st.p
    jump = p[32, 1] - p[2, nx - 2]   # centre of the drop vs far corner
    assert abs(jump - 2.0 / R) < 1e-9 * (2.0 / R)


def test_free_fall_frame_follows_the_released_drop(O):
    # A dense sphere released from rest accelerates at g (rho_d - rho_a) /
    # (rho_d + rho_a / 2) (buoyancy and added mass; drag is negligible at
    # first).  The non-inertial frame (Section 2.4) keeps the drop's centre
    # of mass at its start while the frame velocity carries the fall: after
    # 150 steps Vf is within 1 % of that closed form and the centre moved by
    # less than 1e-4 R.
    nx, ny, h, R, g = 32, 96, 1 / 32, 0.25, -1.0
    mk = W.axi_sphere(1.0, R, 96)
    cfg = O.Config(nx=nx, ny=ny, h=h, axisym=1, frame=1, gy=g, relocate_every=10, spread=1)
    st = O.init_state(cfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    for _ in range(150):
        O.ns_step(cfg, st, dt)
        assert st.last["status"] == 0
    gp = g * (1.0 - 1e-3) / (1.0 + 0.5e-3)
    assert abs(st.frame["Vf"] / (gp * 150 * dt) - 1.0) < 1e-2
    assert abs(st.frame["com_prev"] - st.frame["com0"]) < 1e-4 * R
    # the ambient fluid streams in at the bottom and out at the top with -Vf
    assert np.abs(st.v[0] - st.v[-1]).max() == 0.0 and st.v[0, 0] > 0.0
