"""GPU parity of the Crank-Nicolson viscous step (Section 2.1) with the
oracle: the red-black solve itself (planar and axisymmetric, same sweeps in
the same order) and composed time steps with the implicit viscous half."""
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
@pytest.mark.parametrize("nx,ny", [(64, 48), (33, 70)])
def test_cn_solve_matches_oracle(T, ib, O, axisym, nx, ny):
    h, dt = 1.0 / 64, 2e-4
    H = W.random_H(nx, ny, 61)
    rho, mu, bx, by = O.coeffs(H, 1e-3, 1.0, 1e-4, 1e-2)
    mu = mu * 5.0
    ue, ve = W.random_faces(nx, ny, 62)
    ue[:, [0, -1]] = 0.0
    ve[[0, -1], :] = 0.0
    d = lambda a: T.from_numpy(np.ascontiguousarray(a)).cuda()
    us, vs = ib.ib_op_cn_solve(d(rho), d(mu), d(ue), d(ve), h, dt, 20, axisym)
    uo, vo = O.cn_solve(rho, mu, ue, ve, h, dt, 20, axisym)
    assert np.abs(us.cpu().numpy() - uo).max() <= 1e-13 * np.abs(uo).max()
    assert np.abs(vs.cpu().numpy() - vo).max() <= 1e-13 * np.abs(vo).max()


@pytest.mark.parametrize("axisym", [0, 1])
def test_cn_steps_match_oracle(T, ib, O, axisym):
    # an oscillating drop (planar ellipse, or the axisymmetric ellipsoid under
    # gravity in the non-inertial frame), Crank-Nicolson viscous steps
    if axisym:
        nx, ny, h = 32, 96, 1 / 32
        mk = W.axi_elliptic_drop(1.5, 0.25, 1.1, 96)
        kw = dict(axisym=1, frame=1, gy=-1.0)
    else:
        nx, ny, h = 64, 64, 1 / 64
        mk = W.elliptic_drop(0.5, 0.5, 0.22, 1.15, 128)
        kw = {}
    kw.update(spread=1, relocate_every=3, viscous=1, cn_sweeps=20, tol=1e-11)
    ctx = ib.Context(ib.Config(nx=nx, ny=ny, h=h, **kw), mk.X, mk.Y, mk.drop_start)
    ocfg = O.Config(nx=nx, ny=ny, h=h, **kw)
    st = O.init_state(ocfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    for _ in range(5):
        ctx.ns_step(dt, 1, 1)
        O.ns_step(ocfg, st, dt)
    # p within 1e-10 of max |p|; u, v within 1e-10 of the inertial-capillary
    # velocity sqrt(sigma / (rho_l R)) (the viscous solve's sweeps are the
    # oracle's, so only rounding separates them)
    U = np.sqrt(1.0 / (1.0 * 0.25))
    got = ctx.get("p").cpu().numpy()
    assert np.abs(got - st.p).max() <= 1e-10 * np.abs(st.p).max(), np.abs(got - st.p).max()
    for name, ref in (("u", st.u), ("v", st.v)):
        got = ctx.get(name).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * U, (name, np.abs(got - ref).max())
    X, Y = (a.cpu().numpy() for a in ctx.markers())
    assert np.abs(X - st.X).max() <= 1e-12 and np.abs(Y - st.Y).max() <= 1e-12
