"""GPU parity of the grid operators (through the C ABI) against the oracle on
seeded inputs whose sizes span several 64x16 tiles with ragged tails."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

SIZES = [(70, 52), (130, 34), (8, 8), (64, 16)]


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


def dev(T, a):
    return T.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


def rel(a, b):
    a = a.cpu().numpy() if hasattr(a, "cpu") else a
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def setup(O, nx, ny, seed):
    H = W.random_H(nx, ny, seed)
    rho, mu, bx, by = O.coeffs(H, 1e-3, 1.0, 1e-4, 1e-2)
    return H, rho, mu, bx, by


@pytest.mark.parametrize("nx,ny", SIZES)
def test_coeffs(T, ib, O, nx, ny):
    H, rho, mu, bx, by = setup(O, nx, ny, 1)
    g = ib.ib_op_coeffs(dev(T, H), 1e-3, 1.0, 1e-4, 1e-2)
    for a, b in zip(g, (rho, mu, bx, by)):
        assert rel(a, b) <= 1e-15


@pytest.mark.parametrize("nx,ny", SIZES)
def test_residual_rbgs_restrict_prolong(T, ib, O, nx, ny):
    h = 1.0 / nx
    H, rho, mu, bx, by = setup(O, nx, ny, 2)
    b = W.random_cells(nx, ny, 3)
    p = W.random_cells(nx, ny, 4)
    dbx, dby, db, dp = dev(T, bx), dev(T, by), dev(T, b), dev(T, p)
    assert rel(ib.ib_op_residual(dbx, dby, db, dp, h), O.residual(bx, by, b, p, h)) <= 1e-12
    for ns in (1, 3):
        assert rel(ib.ib_op_rbgs(dbx, dby, db, dp, h, ns), O.rbgs(bx, by, b, p, h, ns)) <= 1e-12
    if nx % 2 == 0 and ny % 2 == 0:
        ref = O.restrict(O.residual(bx, by, b, p, h))
        assert rel(ib.ib_op_restrict_residual(dbx, dby, db, dp, h), ref) <= 1e-12
        bxc, byc = O.coarsen_beta(bx, by)
        gx, gy = ib.ib_op_coarsen_beta(dbx, dby)
        assert rel(gx, bxc) == 0 and rel(gy, byc) == 0
        ec = W.random_cells(nx // 2, ny // 2, 5)
        assert rel(ib.ib_op_prolong_add(dev(T, ec), dp), O.prolong_add(ec, p)) <= 1e-14


def test_rbgs_ignores_wall_coefficients(T, ib, O):
    nx = ny = 40
    h = 1 / 40
    H, rho, mu, bx, by = setup(O, nx, ny, 6)
    bx2, by2 = bx.copy(), by.copy()
    bx2[:, 0] = bx2[:, -1] = 7.0
    by2[0] = by2[-1] = 9.0
    b, p = W.random_cells(nx, ny, 7), W.random_cells(nx, ny, 8)
    g = ib.ib_op_rbgs(dev(T, bx2), dev(T, by2), dev(T, b), dev(T, p), h, 2)
    assert rel(g, O.rbgs(bx, by, b, p, h, 2)) <= 1e-12


@pytest.mark.parametrize("nx,ny", SIZES)
def test_rhs_correct_predictor(T, ib, O, nx, ny):
    h, dt = 1.0 / nx, 3e-4
    H, rho, mu, bx, by = setup(O, nx, ny, 9)
    us, vs = W.random_faces(nx, ny, 10)
    Fx, Fy = W.random_faces(nx, ny, 11, scale=30)
    p = W.random_cells(nx, ny, 12)
    d = lambda a: dev(T, a)
    assert rel(ib.ib_op_rhs(d(us), d(vs), d(Fx), d(Fy), d(bx), d(by), h, dt),
               O.rhs(us, vs, Fx, Fy, bx, by, h, dt)) <= 1e-13
    gu, gv = ib.ib_op_correct(d(us), d(vs), d(p), d(Fx), d(Fy), d(bx), d(by), h, dt)
    ou, ov = O.correct(us, vs, p, Fx, Fy, bx, by, h, dt)
    assert rel(gu, ou) <= 1e-13 and rel(gv, ov) <= 1e-13
    u, v = W.random_faces(nx, ny, 13)
    g1 = ib.ib_op_predictor(d(rho), d(mu), d(u), d(v), h, dt, g=(0.1, -9.8))
    o1 = O.predictor(rho, mu, u, v, h, dt, g=(0.1, -9.8))
    for a, b in zip(g1, o1):
        assert rel(a, b) <= 1e-12
    g2 = ib.ib_op_predictor(d(rho), d(mu), d(u), d(v), h, dt, g1[2], g1[3], g=(0.1, -9.8))
    o2 = O.predictor(rho, mu, u, v, h, dt, o1[2], o1[3], g=(0.1, -9.8))
    for a, b in zip(g2, o2):
        assert rel(a, b) <= 1e-12
