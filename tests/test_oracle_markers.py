"""Pins of the oracle's marker routines: binning/sort (brute force),
interpolation and conventional spreading (Section 2.2 Eq. (jump_condu),
Section 3.1 Eq. (delta_vec)) against moment closed forms and adjointness,
curvature (Section 4 Eq. (ten_f)) against circles, the polygon Heaviside
(Section 3.2) against sub-cell sampling, and the least-squares B-spline
relocation (Section 4) against an independent library fit."""
import numpy as np
import pytest

import workloads as W


def test_keys_and_sort_brute_force(O):
    rng = np.random.default_rng(0)
    nx, ny, h, x0, y0 = 40, 30, 0.025, -0.3, 0.2
    X = rng.uniform(x0, x0 + nx * h, 500)
    Y = rng.uniform(y0, y0 + ny * h, 500)
    X[:50] = x0 + h * rng.integers(0, nx, 50)       # exactly on cell edges
    X[50:60] = X[60:70]; Y[50:60] = Y[60:70]         # duplicate keys
    key = O.cell_keys(X, Y, x0, y0, h, nx, ny)
    ref = [int(np.floor((y - y0) / h)) * nx + int(np.floor((x - x0) / h)) for x, y in zip(X, Y)]
    assert np.array_equal(key, np.array(ref, np.uint32))
    order = O.marker_sort(key)
    assert np.array_equal(order, np.lexsort((np.arange(500), key)).astype(np.uint32))


@pytest.mark.parametrize("kernel", [0, 1])
def test_interp_linear_field_first_moment(O, kernel):
    # u = a + b x on x-faces: U(X) = a + b X + b h m1(frac), with m1 the first
    # moment of the kernel (closed form for the cosine kernel, 0 for Peskin's).
    nx = ny = 32
    h = 1 / 32
    a, bcoef = 0.4, 1.7
    xf = np.arange(nx + 1) * h
    u = np.tile(a + bcoef * xf, (ny, 1))
    v = np.zeros((ny + 1, nx))
    rng = np.random.default_rng(1)
    X, Y = rng.uniform(0.3, 0.7, 64), rng.uniform(0.3, 0.7, 64)
    U, V = O.interp(u, v, X, Y, h, kernel=kernel)
    s = X / h
    r = s - np.floor(s)
    # sum_k (k - s) phi(k - s) over the support: closed form in r = frac(s)
    m1 = 0.25 * (2 - 4 * r + 2 * np.sin(np.pi * r / 2) - 2 * np.cos(np.pi * r / 2)) if kernel == 0 else 0 * r
    assert np.abs(U - (a + bcoef * X + bcoef * h * m1)).max() < 1e-13
    assert np.abs(V).max() == 0.0


def test_spread_total_force_and_adjointness(O):
    n, h = 48, 1 / 48
    mk = W.join([W.circle(0.45, 0.55, 0.2, 97)])
    k, nxm, nym, ds = O.curvature(mk.X, mk.Y, mk.drop_start)
    rng = np.random.default_rng(2)
    fmag = rng.uniform(0.5, 2.0, mk.M)
    for kernel in (0, 1):
        Fx, Fy = O.spread_conv(mk.X, mk.Y, fmag, nxm, nym, ds, n, n, h, kernel=kernel)
        # partition of unity: the grid total equals the marker total
        assert abs(Fx.sum() * h * h - (fmag * nxm * ds).sum()) < 1e-13
        assert abs(Fy.sum() * h * h - (fmag * nym * ds).sum()) < 1e-13
        # spreading is the adjoint of interpolation with the same kernel
        u, v = W.random_faces(n, n, 3)
        U, V = O.interp(u, v, mk.X, mk.Y, h, kernel=kernel)
        lhs = ((u * Fx).sum() + (v * Fy).sum()) * h * h
        rhs = (U * fmag * nxm * ds + V * fmag * nym * ds).sum()
        assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_curvature_on_circles(O):
    for R, n, th0 in [(0.25, 128, 0.0), (0.013, 256, 0.3), (2.0, 37, 1.0)]:
        mk = W.join([W.circle(0.5, -0.2, R, n, th0)])
        k, nxm, nym, ds = O.curvature(mk.X, mk.Y, mk.drop_start)
        assert np.abs(k * R - 1).max() < 1e-10  # rounding of positions / turning angle
        # inward unit normals point to the centre
        cx, cy = 0.5 - mk.X, -0.2 - mk.Y
        assert np.abs(nxm - cx / R).max() < 1e-11 and np.abs(nym - cy / R).max() < 1e-11
        chord = 2 * R * np.sin(np.pi / n)
        assert np.abs(ds - chord).max() < 1e-13 * max(R, 1)
    # clockwise order flips the sign
    X, Y = W.circle(0.5, 0.5, 0.2, 64)
    mk = W.join([(X[::-1].copy(), Y[::-1].copy())])
    assert np.all(O.curvature(mk.X, mk.Y, mk.drop_start)[0] < 0)


def test_curvature_ellipse_converges(O):
    # curvature of x = a cos t, y = b sin t is ab / (a^2 sin^2 t + b^2 cos^2 t)^{3/2}
    errs = []
    for n in (64, 128, 256):
        mk = W.elliptic_drop(0.0, 0.0, 0.2, 1.3, n)
        k = O.curvature(mk.X, mk.Y, mk.drop_start)[0]
        t = 2 * np.pi * np.arange(n) / n
        a, b = 0.2 * 1.3, 0.2 / 1.3
        ke = a * b / (a**2 * np.sin(t)**2 + b**2 * np.cos(t)**2)**1.5
        errs.append(np.abs(k - ke).max() / ke.max())
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_inside_test_circle(O):
    n, h = 40, 1 / 40
    mk = W.join([W.circle(0.5, 0.5, 0.3, 400)])
    chi = O.inside(mk.X, mk.Y, mk.drop_start, n, n, h)
    c = (np.arange(n) + 0.5) * h
    d = np.hypot(*np.meshgrid(c - 0.5, c - 0.5)) - 0.3
    far = np.abs(d) > 0.002  # farther than the polygon-to-circle gap
    assert np.array_equal(chi[far], (d[far] < 0).astype(float))


def _point_in_quad(px, py, qx, qy):
    s = []
    for k in range(4):
        ax, ay, bx, by = qx[k], qy[k], qx[(k + 1) % 4], qy[(k + 1) % 4]
        s.append((bx - ax) * (py - ay) - (by - ay) * (px - ax))
    s = np.array(s)
    return np.all(s >= 0, axis=0) | np.all(s <= 0, axis=0)


def test_heaviside_against_subcell_sampling(O):
    # Brute force: sample points in a cell, give each the strip value of the
    # strip polygon that contains it (built here from the definition: offsets
    # k-2.5 .. k-1.5 cells along the marker normals) or the cell's inside
    # flag when no strip contains it, and average.
    n, h = 32, 1 / 32
    mk = W.join([W.circle(0.47, 0.52, 0.23, 60, 0.1)])
    H = O.heaviside(mk.X, mk.Y, mk.drop_start, n, n, h)
    chi = O.inside(mk.X, mk.Y, mk.drop_start, n, n, h)
    k_, nxm, nym, ds = O.curvature(mk.X, mk.Y, mk.drop_start)
    Hk = O.heaviside_profile(np.arange(-2, 3, dtype=float))
    S = 300
    g = (np.arange(S) + 0.5) / S
    gx, gy = np.meshgrid(g, g)
    rng = np.random.default_rng(4)
    band = np.argwhere((H > 1e-12) & (H < 1 - 1e-12))
    for (j, i) in band[rng.choice(len(band), 12, replace=False)]:
        px, py = (i + gx).ravel(), (j + gy).ravel()
        val = np.full(px.shape, np.nan)
        for m in range(mk.M):
            m2 = (m + 1) % mk.M
            for kk in range(5):
                a, b = kk - 2.5, kk - 1.5
                qx = np.array([mk.X[m] / h + a * nxm[m], mk.X[m2] / h + a * nxm[m2],
                               mk.X[m2] / h + b * nxm[m2], mk.X[m] / h + b * nxm[m]])
                qy = np.array([mk.Y[m] / h + a * nym[m], mk.Y[m2] / h + a * nym[m2],
                               mk.Y[m2] / h + b * nym[m2], mk.Y[m] / h + b * nym[m]])
                if qx.max() < i or qx.min() > i + 1 or qy.max() < j or qy.min() > j + 1:
                    continue
                inq = _point_in_quad(px, py, qx, qy) & np.isnan(val)
                val[inq] = Hk[kk]
        val[np.isnan(val)] = chi[j, i]
        assert abs(val.mean() - H[j, i]) < 4.0 / S
        assert abs(O.heaviside_cell(i, j, mk.X, mk.Y, mk.drop_start, h, chi[j, i]) - H[j, i]) < 1e-14


def test_heaviside_bounds_symmetry_and_area(O):
    n, h = 64, 1 / 64
    mk = W.join([W.circle(0.5, 0.5, 0.25, 128)])
    H = O.heaviside(mk.X, mk.Y, mk.drop_start, n, n, h)
    assert H.min() >= -1e-15 and H.max() <= 1 + 1e-15
    assert np.abs(H - H.T).max() < 1e-13           # x <-> y mirror of the marker set
    assert np.abs(H - H[:, ::-1]).max() < 1e-13    # x mirror
    poly_area = 0.5 * 128 * 0.25**2 * np.sin(2 * np.pi / 128)
    assert abs(H.sum() * h * h - poly_area) < 0.05 * h * 2 * np.pi * 0.25  # O(h * perimeter * h/R)
    # a square drop with long straight edges: the band integrates exactly along
    # the edges, so the area error comes from the four corners only
    side, per = 0.5, 100
    t = np.linspace(0, 1, per, endpoint=False)
    xs = np.concatenate([0.25 + side * t, np.full(per, 0.75), 0.75 - side * t, np.full(per, 0.25)])
    ys = np.concatenate([np.full(per, 0.25), 0.25 + side * t, np.full(per, 0.75), 0.75 - side * t])
    sq = W.join([(xs, ys)])
    Hs = O.heaviside(sq.X, sq.Y, sq.drop_start, n, n, h)
    assert abs(Hs.sum() * h * h - side**2) < 4 * 6 * h * h


def test_irrotational_spread_is_discrete_gradient(O):
    # Section 3.2: with constant f the face force is f grad_h H, so every node
    # curl vanishes and the total force is zero (H = 0 at the walls).
    n, h = 64, 1 / 64
    mk = W.join([W.circle(0.5, 0.5, 0.2, 126)])
    H = O.heaviside(mk.X, mk.Y, mk.drop_start, n, n, h)
    Fx, Fy = O.spread_irrot(mk.X, mk.Y, mk.drop_start, np.ones(mk.M), H, h)
    curl = (Fy[1:-1, 1:] - Fy[1:-1, :-1]) - (Fx[1:, 1:-1] - Fx[:-1, 1:-1])
    assert np.abs(curl).max() < 1e-12 * np.abs(Fx).max()
    assert abs(Fx.sum()) < 1e-10 and abs(Fy.sum()) < 1e-10
    # the conventional splitting is rotational (Section 3.1, Fig. Heaviside_curl)
    k, nxm, nym, ds = O.curvature(mk.X, mk.Y, mk.drop_start)
    Gx, Gy = O.spread_conv(mk.X, mk.Y, np.ones(mk.M), nxm, nym, ds, n, n, h)
    curl_c = (Gy[1:-1, 1:] - Gy[1:-1, :-1]) - (Gx[1:, 1:-1] - Gx[:-1, 1:-1])
    assert np.abs(curl_c).max() > 1e-3 * np.abs(Gx).max()


def test_irrotational_face_force_takes_nearest_segment_value(O):
    n, h = 48, 1 / 48
    mk = W.join([W.circle(0.5, 0.5, 0.2, 100)])
    H = O.heaviside(mk.X, mk.Y, mk.drop_start, n, n, h)
    f = np.full(mk.M, 3.5)
    Fx, Fy = O.spread_irrot(mk.X, mk.Y, mk.drop_start, f, H, h)
    dHx = np.diff(H, axis=1) / h
    assert np.abs(Fx[:, 1:-1] - 3.5 * dHx).max() < 1e-12 * np.abs(Fx).max()
    # a marker-dependent f: a face right at a marker takes that marker's value
    f2 = np.arange(mk.M, dtype=float)
    Fx2, _ = O.spread_irrot(mk.X, mk.Y, mk.drop_start, f2, H, h)
    nz = np.argwhere(dHx != 0)
    j, i = nz[len(nz) // 3]
    q = np.array([(i + 1) * h, (j + 0.5) * h])
    d = np.hypot(mk.X - q[0], mk.Y - q[1])
    m = int(np.argmin(d))
    assert f2.min() <= Fx2[j, i + 1] / dHx[j, i] <= f2.max()
    assert abs(Fx2[j, i + 1] / dHx[j, i] - m) <= 1.0 + 1e-9


def _periodic_fit_scipy(X, Y, h):
    from scipy.interpolate import BSpline
    n = len(X)
    seg = np.hypot(np.roll(X, -1) - X, np.roll(Y, -1) - Y)
    s = np.concatenate([[0.0], np.cumsum(seg)[:-1]])
    L = seg.sum()
    g = max(4, min(n, int(np.floor(L / (1.5 * h) + 0.5))))
    tau = L / g
    t = np.arange(-3, g + 4) * tau
    Bm = BSpline.design_matrix(s, t, 3, extrapolate=False).toarray()  # g+3 basis fns
    Bp = Bm[:, :g].copy()
    Bp[:, :3] += Bm[:, g:g + 3]                                        # periodic wrap
    cx = np.linalg.lstsq(Bp, X, rcond=None)[0]
    cy = np.linalg.lstsq(Bp, Y, rcond=None)[0]
    full = lambda c: BSpline(t, np.concatenate([c, c[:3]]), 3)
    return full(cx), full(cy), L, g


def _project(sx, sy, s, x, y):
    # Newton on |C(s) - P|^2 with the library spline's own derivatives
    for _ in range(30):
        dx, dy = sx(s) - x, sy(s) - y
        d1x, d1y, d2x, d2y = sx(s, 1), sy(s, 1), sx(s, 2), sy(s, 2)
        s = s - (dx * d1x + dy * d1y) / (d1x * d1x + d1y * d1y + dx * d2x + dy * d2y)
    return float(s), float(np.hypot(sx(s) - x, sy(s) - y))


def test_bspline_relocation_against_library_fit(O):
    pytest.importorskip("scipy")
    from scipy.integrate import quad
    h = 1 / 64
    mk = W.oscillating_drop(n_markers=90, r0=0.2, eps=0.05, jitter=2e-3, seed=11)
    Xo, Yo = O.bspline_relocate(mk.X, mk.Y, mk.drop_start, h)
    sx, sy, L, g = _periodic_fit_scipy(mk.X, mk.Y, h)
    ss = np.linspace(0, L, 20001)
    cx, cy = sx(ss), sy(ss)
    # every relocated marker lies on the independently fitted curve
    for x, y in zip(Xo, Yo):
        k = np.argmin(np.hypot(cx - x, cy - y))
        sp_, dist = _project(sx, sy, ss[k], x, y)
        assert dist < 1e-12
    # first marker at parameter 0, and equal arc length between markers
    assert abs(Xo[0] - sx(0.0)) < 1e-12 and abs(Yo[0] - sy(0.0)) < 1e-12
    speed = lambda s: np.hypot(sx(s, 1), sy(s, 1))
    total = sum(quad(speed, k * L / g, (k + 1) * L / g, epsabs=1e-14)[0] for k in range(g))
    par = []
    for x, y in zip(Xo, Yo):
        k = np.argmin(np.hypot(cx - x, cy - y))
        par.append(_project(sx, sy, ss[k], x, y)[0])
    par = np.array(par)
    tau = L / g
    spans = np.cumsum([0.0] + [quad(speed, k * tau, (k + 1) * tau, epsabs=1e-15)[0] for k in range(g)])

    def arc(p):  # piecewise over knot spans, where the speed is smooth
        q = min(int(p // tau), g - 1)
        return spans[q] + quad(speed, q * tau, p, epsabs=1e-15)[0]

    arcs = np.array([arc(p) for p in par])
    target = total * np.arange(len(Xo)) / len(Xo)
    assert np.abs(arcs - target).max() < 1e-11


def test_bspline_relocation_circle_and_equivariance(O):
    h = 1 / 128
    mk = W.join([W.circle(0.5, 0.5, 0.2, 200, 0.2)])
    Xo, Yo = O.bspline_relocate(mk.X, mk.Y, mk.drop_start, h)
    r = np.hypot(Xo - 0.5, Yo - 0.5)
    assert np.abs(r - 0.2).max() < 1e-6
    d = np.hypot(np.diff(np.append(Xo, Xo[0])), np.diff(np.append(Yo, Yo[0])))
    assert d.std() / d.mean() < 1e-6
    Xs, Ys = O.bspline_relocate(mk.X + 0.125, mk.Y - 0.25, mk.drop_start, h)
    assert np.abs(Xs - 0.125 - Xo).max() < 1e-12 and np.abs(Ys + 0.25 - Yo).max() < 1e-12


def test_row_inside_equals_pointwise_crossing_number(O):
    n, h = 80, 1 / 80
    mk = W.multidrop(80, ndrops=5, rmin=0.06, rmax=0.12, n_per_drop=70, seed=9, gap_cells=6)
    chi = O.inside(mk.X, mk.Y, mk.drop_start, n, n, h)
    for j in range(0, n, 3):
        for i in range(n):
            assert chi[j, i] == O.inside_cell(i, j, mk.X, mk.Y, mk.drop_start, h)


def test_mass_correction_restores_the_measure(O):
    # Section 2.5: a regular polygon offset inward along its normals by 0.3 h
    # stays regular with the same normals; the bisection correction towards
    # the original area (planar) or volume of revolution (axisymmetric)
    # recovers the original markers and measure.
    h = 1 / 64
    for axisym in (0, 1):
        mk = W.axi_sphere(0.5, 0.25, 128) if axisym else W.static_drop(64, 0.25, 128)
        A0 = O.drop_measures(mk.X, mk.Y, mk.drop_start, axisym)
        if axisym:
            assert abs(A0[0] - 4 / 3 * np.pi * 0.25**3) < 2e-3 * A0[0]
        else:
            assert abs(A0[0] - np.pi * 0.25**2) < 1e-3 * A0[0]
        k, nxm, nym, ds = O.curvature(mk.X, mk.Y, mk.drop_start)
        Xs, Ys = mk.X + 0.3 * h * nxm, mk.Y + 0.3 * h * nym
        assert O.drop_measures(Xs, Ys, mk.drop_start, axisym)[0] < A0[0]
        Xc, Yc, eps = O.mass_correct(Xs, Ys, mk.drop_start, A0, h, axisym)
        assert abs(eps[0] + 0.3 * h) < 1e-12 * h
        assert np.abs(Xc - mk.X).max() < 1e-13 and np.abs(Yc - mk.Y).max() < 1e-13
        A = O.drop_measures(Xc, Yc, mk.drop_start, axisym)[0]
        assert abs(A - A0[0]) < 1e-12 * A0[0]
        # within the tolerance nothing moves
        Xn, Yn, e0 = O.mass_correct(mk.X, mk.Y, mk.drop_start, A0 * (1 + 5e-7), h, axisym)
        assert e0[0] == 0.0 and np.array_equal(Xn, mk.X)


@pytest.mark.parametrize("axisym", [0, 1])
def test_indicator_poisson_is_the_drop_indicator(O, axisym):
    # Eq. (ind_psn): I from div grad I = div(delta vector) is 1 deep inside a
    # drop and 0 far outside, and its integral (area, or volume of
    # revolution) is the drop's measure to O(h^2); its discrete gradient
    # differs from the delta vector by a divergence-free field only.
    n, h, R = 64, 1 / 64, 0.25
    if axisym:
        mk = W.axi_sphere(0.5, R, 128)
        I = O.indicator_poisson(mk.X, mk.Y, mk.drop_start, 32, 64, h, axisym=1)
        r = (np.arange(32) + 0.5) * h
        meas = 2 * np.pi * (I * r[None, :]).sum() * h * h
        exact = 4 / 3 * np.pi * R**3
        inside, outside = I[32, 2], I[2, 30]
    else:
        mk = W.static_drop(n, R, 128)
        I = O.indicator_poisson(mk.X, mk.Y, mk.drop_start, n, n, h)
        meas = I.sum() * h * h
        exact = np.pi * R**2
        inside, outside = I[32, 32], I[3, 3]
    assert abs(inside - 1.0) < 1e-3 and outside < 1e-3
    assert abs(meas - exact) < 1e-2 * exact
    assert I.min() >= 0.0 and I.max() <= 1.0
