"""GPU parity of the Section 2.5 measure (mass) correction with the oracle:
the bisection offset along the inward normals for several drops offset by
different amounts (planar areas and axisymmetric volumes), and composed
steps with the correction every few steps."""
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


@pytest.mark.parametrize("axisym", [0, 1])
def test_correction_matches_oracle(T, ib, O, axisym):
    if axisym:
        n, ny, h = 32, 64, 1 / 32
        mk = W.axi_elliptic_drop(1.0, 0.3, 1.2, 160)
        offs = [0.27 * h]
    else:
        n, ny, h = 128, 128, 1 / 128
        mk = W.multidrop(128, ndrops=5, rmin=0.05, rmax=0.12, n_per_drop=120, seed=7,
                         gap_cells=12)
        offs = [0.31 * h, -0.22 * h, 0.0, 1e-9 * h, 0.45 * h]
    cfg = ib.Config(nx=n, ny=ny, h=h, axisym=axisym)
    ctx = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
    A0 = O.drop_measures(mk.X, mk.Y, mk.drop_start, axisym)
    k, nxm, nym, ds = O.curvature(mk.X, mk.Y, mk.drop_start)
    Xs, Ys = mk.X.copy(), mk.Y.copy()
    for d, e in enumerate(offs):
        s, t = mk.drop_start[d], mk.drop_start[d + 1]
        Xs[s:t] += e * nxm[s:t]
        Ys[s:t] += e * nym[s:t]
    if axisym:
        Xs, Ys = O.symmetrise(Xs, Ys, mk.drop_start)
    ctx.set_markers_host(np.ascontiguousarray(Xs), np.ascontiguousarray(Ys))
    eps = ctx.mass_correct()
    Xo, Yo, eo = O.mass_correct(Xs, Ys, mk.drop_start, A0, h, axisym)
    if axisym:
        Xo, Yo = O.symmetrise(Xo, Yo, mk.drop_start)
    X, Y = (a.cpu().numpy() for a in ctx.markers())
    assert np.abs(eps - eo).max() <= 1e-13 * h
    assert np.abs(X - Xo).max() <= 1e-14 and np.abs(Y - Yo).max() <= 1e-14
    # drops within the tolerance (offset 0 and 1e-9 h) did not move
    for d, e in enumerate(offs):
        if abs(e) < 1e-6 * h:
            assert eps[d] == 0.0
        else:
            assert abs(eps[d] + e) < 1e-3 * h
    A = O.drop_measures(X, Y, mk.drop_start, axisym)
    moved = eps != 0.0
    assert np.all(np.abs(A - A0)[moved] <= 1e-11 * A0[moved])


def test_steps_with_correction_match_oracle(T, ib, O):
    # planar oscillating drop, relocation every 3 steps and the measure
    # correction every 2: six steps against the oracle
    n, h = 64, 1 / 64
    mk = W.elliptic_drop(0.5, 0.5, 0.22, 1.15, 128)
    kw = dict(spread=1, relocate_every=3, mass_every=2, mass_tol=1e-9, tol=1e-11)
    ctx = ib.Context(ib.Config(nx=n, ny=n, h=h, **kw), mk.X, mk.Y, mk.drop_start)
    ocfg = O.Config(nx=n, ny=n, h=h, **kw)
    st = O.init_state(ocfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    for _ in range(6):
        ctx.ns_step(dt, 1, 1)
        O.ns_step(ocfg, st, dt)
    X, Y = (a.cpu().numpy() for a in ctx.markers())
    assert np.abs(X - st.X).max() <= 1e-12 and np.abs(Y - st.Y).max() <= 1e-12
    p = ctx.get("p").cpu().numpy()
    assert np.abs(p - st.p).max() <= 1e-10 * np.abs(st.p).max(), np.abs(p - st.p).max()
