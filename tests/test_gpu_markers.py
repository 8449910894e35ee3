"""GPU parity of the marker kernels against the oracle: binning and order
(bit-exact), curvature, interpolation, both spreadings, the polygon Heaviside
and B-spline relocation, plus sampled checks at the 1024^2 / 64-drop size."""
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


def htol(n):
    """Absolute tolerance on H: both sides form cell-local polygon coordinates
    from grid coordinates of size up to n, so each clip carries an absolute
    rounding of a few n * 2^-53; a cell sums a handful of such areas."""
    return 1e-13 + 8 * n * 2.0 ** -53


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = {
    "static64": (64, W.static_drop(64, 0.25, 128)),
    "osc96": (96, W.oscillating_drop(300, 0.2, 0.05, 1e-3, 1808)),
    "multi200": (200, W.multidrop(200, ndrops=6, rmin=0.05, rmax=0.12, n_per_drop=160, seed=3,
                                  gap_cells=12)),
}


def make(ib, n, mk, **kw):
    cfg = ib.Config(nx=n, ny=n, h=1.0 / n, **kw)
    return cfg, ib.Context(cfg, mk.X, mk.Y, mk.drop_start)


@pytest.mark.parametrize("case", list(CASES))
def test_sort_bit_exact(T, ib, O, case):
    n, mk = CASES[case]
    cfg, ctx = make(ib, n, mk)
    keys, ids, cs = ctx.marker_sort()
    okey = O.cell_keys(mk.X, mk.Y, 0.0, 0.0, 1.0 / n, n, n)
    order = O.marker_sort(okey)
    assert np.array_equal(ids.cpu().numpy().astype(np.uint32), order)
    assert np.array_equal(keys.cpu().numpy().astype(np.uint32), okey[order])
    ref_cs = np.searchsorted(okey[order], np.arange(n * n + 1), side="left")
    assert np.array_equal(cs.cpu().numpy(), ref_cs)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("kernel", [0, 1])
def test_geometry_interp_spread_conv(T, ib, O, case, kernel):
    n, mk = CASES[case]
    cfg, ctx = make(ib, n, mk, kernel=kernel, sigma=0.7)
    k, nxm, nym, ds = ctx.geometry()
    ok, onx, ony, ods = O.curvature(mk.X, mk.Y, mk.drop_start)
    for a, b in ((k, ok), (nxm, onx), (nym, ony), (ds, ods)):
        assert rel(a, b) <= 1e-13
    u, v = W.random_faces(n, n, 21)
    U, V = ctx.interp(T.from_numpy(u).cuda(), T.from_numpy(v).cuda())
    oU, oV = O.interp(u, v, mk.X, mk.Y, 1.0 / n, kernel=kernel)
    assert rel(U, oU) <= 1e-13 and rel(V, oV) <= 1e-13
    Fx, Fy = ctx.spread(0)
    oFx, oFy = O.spread_conv(mk.X, mk.Y, 0.7 * ok, onx, ony, ods, n, n, 1.0 / n, kernel=kernel)
    assert rel(Fx, oFx) <= 1e-12 and rel(Fy, oFy) <= 1e-12
    f = T.from_numpy(np.linspace(0.5, 2.0, mk.M)).cuda()
    Fx, Fy = ctx.spread(0, fmag=f)
    oFx, oFy = O.spread_conv(mk.X, mk.Y, f.cpu().numpy(), onx, ony, ods, n, n, 1.0 / n,
                             kernel=kernel)
    assert rel(Fx, oFx) <= 1e-12 and rel(Fy, oFy) <= 1e-12


@pytest.mark.parametrize("case", list(CASES))
def test_heaviside_and_irrotational_spread(T, ib, O, case):
    n, mk = CASES[case]
    cfg, ctx = make(ib, n, mk, sigma=1.3)
    H = ctx.heaviside().cpu().numpy()
    oH = O.heaviside(mk.X, mk.Y, mk.drop_start, n, n, 1.0 / n)
    assert np.abs(H - oH).max() <= htol(n)
    Fx, Fy, H2 = ctx.spread(1, want_H=True)
    assert np.abs(H2.cpu().numpy() - oH).max() <= htol(n)
    ok = O.curvature(mk.X, mk.Y, mk.drop_start)[0]
    oFx, oFy = O.spread_irrot(mk.X, mk.Y, mk.drop_start, 1.3 * ok, oH, 1.0 / n)
    assert rel(Fx, oFx) <= 1e-11 and rel(Fy, oFy) <= 1e-11


def test_heaviside_folded_strips(T, ib, O):
    """A drop of radius 2 cells: the inner strips of every polygon fold over
    the centre (non-convex quadrilaterals), which the band kernel clips
    quadrilateral by quadrilateral instead of by half-planes."""
    n = 64
    mk = W.join([W.circle(0.5, 0.5, 2.0 / n, 16, theta0=0.1), W.circle(0.27, 0.3, 0.1, 48)])
    cfg, ctx = make(ib, n, mk, sigma=1.0)
    H = ctx.heaviside().cpu().numpy()
    oH = O.heaviside(mk.X, mk.Y, mk.drop_start, n, n, 1.0 / n)
    assert np.abs(H - oH).max() <= htol(n)


@pytest.mark.parametrize("case", list(CASES))
def test_relocation(T, ib, O, case):
    n, mk = CASES[case]
    cfg, ctx = make(ib, n, mk)
    ctx.relocate()
    X, Y = ctx.markers()
    oX, oY = O.bspline_relocate(mk.X, mk.Y, mk.drop_start, 1.0 / n)
    assert np.abs(X.cpu().numpy() - oX).max() <= 1e-12
    assert np.abs(Y.cpu().numpy() - oY).max() <= 1e-12


def test_relocation_many_markers(T, ib, O):
    """The 1024^2 workload's 64 drops (16384 markers): the placement kernel
    takes one thread per marker at this count (eight lanes per marker below
    4096 markers, as in the cases above); every relocated marker against the
    oracle."""
    n = 1024
    mk = W.multidrop(n)
    assert mk.X.size >= 4096
    cfg, ctx = make(ib, n, mk)
    ctx.relocate()
    X, Y = ctx.markers()
    oX, oY = O.bspline_relocate(mk.X, mk.Y, mk.drop_start, 1.0 / n)
    assert np.abs(X.cpu().numpy() - oX).max() <= 1e-12
    assert np.abs(Y.cpu().numpy() - oY).max() <= 1e-12


def test_marker_errors(T, ib):
    X, Y = W.circle(0.5, 0.5, 0.2, 40)
    cfg = ib.Config(nx=32, ny=32, h=1 / 32)
    with pytest.raises(ib.IBError) as e:
        ib.Context(cfg, X[::-1].copy(), Y[::-1].copy(), [0, 40])  # clockwise
    assert e.value.status == ib.IB_EMARKER
    with pytest.raises(ib.IBError) as e:
        ib.Context(cfg, X + 0.4, Y, [0, 40])  # too close to the wall
    assert e.value.status == ib.IB_EMARKER
    with pytest.raises(ib.IBError) as e:
        ib.Context(cfg, X[:2], Y[:2], [0, 2])  # degenerate drop
    assert e.value.status == ib.IB_EINVAL
    with pytest.raises(ib.IBError) as e:
        ib.Context(ib.Config(nx=1030, ny=1030, h=1 / 1030), X, Y, [0, 40])  # coarsest 515^2
    assert e.value.status == ib.IB_EINVAL
    ctx = ib.Context(cfg, X, Y, [0, 40])
    bad = T.from_numpy(np.full(40, 0.01)).cuda()
    with pytest.raises(ib.IBError) as e:
        ctx.set_markers(bad, bad)
    assert e.value.status == ib.IB_EMARKER


def test_full_size_multidrop_sampled(T, ib, O):
    # 1024^2, 64 drops x 256 markers: sort bit-exact, interpolation and
    # curvature everywhere, Heaviside on sampled band cells, conventional
    # spreading on sampled faces, irrotational force on sampled faces.
    n = 1024
    mk = W.multidrop(n)
    cfg, ctx = make(ib, n, mk)
    keys, ids, cs = ctx.marker_sort()
    okey = O.cell_keys(mk.X, mk.Y, 0.0, 0.0, 1.0 / n, n, n)
    order = O.marker_sort(okey)
    assert np.array_equal(ids.cpu().numpy().astype(np.uint32), order)
    k, nxm, nym, ds = ctx.geometry()
    ok, onx, ony, ods = O.curvature(mk.X, mk.Y, mk.drop_start)
    assert rel(k, ok) <= 1e-12
    u, v = W.random_faces(n, n, 5)
    U, V = ctx.interp(T.from_numpy(u).cuda(), T.from_numpy(v).cuda())
    oU, oV = O.interp(u, v, mk.X, mk.Y, 1.0 / n)
    assert rel(U, oU) <= 1e-13 and rel(V, oV) <= 1e-13
    H = ctx.heaviside().cpu().numpy()
    band = np.argwhere((H > 0) & (H < 1))
    rng = np.random.default_rng(0)
    h = 1.0 / n
    for (j, i) in band[rng.choice(len(band), 40, replace=False)]:
        chi = O.inside_cell(i, j, mk.X, mk.Y, mk.drop_start, h)
        assert abs(H[j, i] - O.heaviside_cell(i, j, mk.X, mk.Y, mk.drop_start, h, chi)) <= htol(n)
    for (j, i) in rng.integers(0, n, (40, 2)):
        if 0 < H[j, i] < 1:
            continue
        assert H[j, i] == O.inside_cell(i, j, mk.X, mk.Y, mk.drop_start, h)
    Fx, Fy = ctx.spread(0)
    oFx, oFy = O.spread_conv(mk.X, mk.Y, ok, onx, ony, ods, n, n, 1.0 / n)
    assert rel(Fx, oFx) <= 1e-12 and rel(Fy, oFy) <= 1e-12
