"""Pins of the oracle's pressure operator and multigrid (Section 2.1 Eq. (ps),
solved by multigrid) against textbook eigenvectors, exact constant-flux
solutions, invariants and a dense direct solve."""
import numpy as np
import pytest

import workloads as W


def _betas(n, seed, ratio=1000.0):
    H = W.random_H(n, n, seed)
    import oracle as O
    return O.coeffs(H, 1.0 / ratio, 1.0, 1e-4, 1e-2)


def test_coeffs_small_case_by_hand(O):
    H = np.array([[0.0, 1.0], [0.5, 0.25]])
    rho, mu, bx, by = O.coeffs(H, 0.1, 2.0, 0.01, 0.5)
    assert np.allclose(rho, 0.1 + 1.9 * H, rtol=0, atol=1e-15)
    assert np.allclose(mu, 0.01 + 0.49 * H, rtol=0, atol=1e-15)
    # x-faces: walls zero, interior = 1 / mean of the two neighbours
    assert bx[0, 0] == 0 and bx[0, 2] == 0 and bx[1, 0] == 0 and bx[1, 2] == 0
    assert abs(bx[0, 1] - 1 / (0.5 * (0.1 + 2.0))) < 1e-15
    assert abs(by[1, 0] - 1 / (0.5 * (0.1 + 0.1 + 1.9 * 0.5))) < 1e-15
    assert np.all(by[0] == 0) and np.all(by[2] == 0)


@pytest.mark.parametrize("nx,ny", [(8, 8), (16, 12), (10, 6)])
def test_constant_beta_textbook_eigenvectors(O, nx, ny):
    # Constant beta reduces A to the 5-point Neumann Laplacian, whose
    # eigenvectors are cos(k pi (i+1/2)/nx) cos(l pi (j+1/2)/ny) with
    # eigenvalues -(4/h^2)(sin^2(k pi/2nx) + sin^2(l pi/2ny)).
    h = 0.1
    bx = np.ones((ny, nx + 1)); bx[:, 0] = bx[:, -1] = 0
    by = np.ones((ny + 1, nx)); by[0] = by[-1] = 0
    i, j = np.arange(nx) + 0.5, np.arange(ny) + 0.5
    for k, l in [(0, 1), (1, 0), (2, 3), (nx - 1, ny - 1)]:
        v = np.outer(np.cos(l * np.pi * j / ny), np.cos(k * np.pi * i / nx))
        lam = -(4 / h**2) * (np.sin(k * np.pi / (2 * nx))**2 + np.sin(l * np.pi / (2 * ny))**2)
        Av = O.apply_A(bx, by, v, h)
        assert np.abs(Av - lam * v).max() < 1e-11 * max(1.0, abs(lam))


def test_variable_beta_constant_flux_solution(O):
    # 1-D structure: beta varies along x only and p_i - p_{i-1} = C / beta_i.
    # Then the flux is C on every interior face, so A p = 0 in interior cells
    # and = +-C/h^2 in the first/last column (walls carry no flux).
    nx, ny, h, C = 12, 5, 0.25, 0.7
    rng = np.random.default_rng(0)
    bcol = rng.uniform(0.5, 1000.0, nx + 1); bcol[0] = bcol[-1] = 0
    bx = np.tile(bcol, (ny, 1))
    by = np.ones((ny + 1, nx)); by[0] = by[-1] = 0
    p1 = np.concatenate([[0.0], np.cumsum(C / bcol[1:-1])])
    p = np.tile(p1, (ny, 1))
    Ap = O.apply_A(bx, by, p, h)
    assert np.abs(Ap[:, 1:-1]).max() < 1e-12
    assert np.allclose(Ap[:, 0], C / h**2, rtol=1e-12)
    assert np.allclose(Ap[:, -1], -C / h**2, rtol=1e-12)
    # the same along y (transposed roles)
    brow = rng.uniform(0.5, 1000.0, ny + 1); brow[0] = brow[-1] = 0
    by2 = np.tile(brow[:, None], (1, nx))
    bx2 = np.ones((ny, nx + 1)); bx2[:, 0] = bx2[:, -1] = 0
    q1 = np.concatenate([[0.0], np.cumsum(C / brow[1:-1])])
    q = np.tile(q1[:, None], (1, nx))
    Aq = O.apply_A(bx2, by2, q, h)
    assert np.abs(Aq[1:-1]).max() < 1e-12
    assert np.allclose(Aq[0], C / h**2, rtol=1e-12) and np.allclose(Aq[-1], -C / h**2, rtol=1e-12)


def test_operator_symmetric_and_annihilates_constants(O):
    n, h = 16, 1 / 16
    rho, mu, bx, by = _betas(n, 3)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    xAy, yAx = (x * O.apply_A(bx, by, y, h)).sum(), (y * O.apply_A(bx, by, x, h)).sum()
    assert abs(xAy - yAx) < 1e-12 * abs(xAy)
    assert np.abs(O.apply_A(bx, by, np.full((n, n), 3.0), h)).max() == 0.0
    assert (x * O.apply_A(bx, by, x, h)).sum() < 0  # negative semi-definite


def test_rbgs_zeroes_residual_of_last_colour(O):
    n, h = 12, 1 / 12
    rho, mu, bx, by = _betas(n, 4)
    b = W.random_cells(n, n, 5)
    p = O.rbgs(bx, by, b, W.random_cells(n, n, 6), h, 1)
    r = O.residual(bx, by, b, p, h)
    black = (np.add.outer(np.arange(n), np.arange(n)) % 2) == 1
    assert np.abs(r[black]).max() < 1e-9 * np.abs(b).max() * 1e3
    assert np.abs(r[~black]).max() > 1e-3  # red cells moved by the black half-sweep


def test_restrict_and_prolong_exactness(O):
    rng = np.random.default_rng(2)
    r = rng.standard_normal((8, 12))
    rc = O.restrict(r)
    assert abs(4 * rc.sum() - r.sum()) < 1e-13
    assert np.allclose(O.restrict(np.full((8, 12), 2.5)), 2.5, rtol=0, atol=0)
    # bilinear prolongation reproduces linear functions away from the walls:
    # coarse centre I sits at fine coordinate 2I + 1/2.
    nxc, nyc = 6, 5
    I, J = np.meshgrid(np.arange(nxc), np.arange(nyc))
    ec = 0.3 * I - 0.7 * J + 1.1
    ef = O.prolong_add(ec, np.zeros((2 * nyc, 2 * nxc)))
    i, j = np.meshgrid(np.arange(2 * nxc), np.arange(2 * nyc))
    ref = 0.3 * (i - 0.5) / 2 - 0.7 * (j - 0.5) / 2 + 1.1
    assert np.abs((ef - ref)[1:-1, 1:-1]).max() < 1e-14
    assert np.allclose(O.prolong_add(np.full((nyc, nxc), 4.0), np.ones((2 * nyc, 2 * nxc))), 5.0)


def test_coarsen_beta_is_mean_of_fine_faces(O):
    rng = np.random.default_rng(3)
    bx, by = rng.uniform(1, 2, (8, 11)), rng.uniform(1, 2, (9, 10))
    bxc, byc = O.coarsen_beta(bx, by)
    assert bxc.shape == (4, 6) and byc.shape == (5, 5)
    assert abs(bxc[1, 2] - 0.5 * (bx[2, 4] + bx[3, 4])) < 1e-15
    assert abs(byc[3, 4] - 0.5 * (by[6, 8] + by[6, 9])) < 1e-15


@pytest.mark.parametrize("n", [8, 16, 32])
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_mg_matches_dense_direct_solve(O, n, precision):
    h = 1 / n
    rho, mu, bx, by = _betas(n, 7 + n)
    b = W.random_cells(n, n, 8)
    pd = O.dense_solve(bx, by, b, h)
    res = O.mg_solve(bx, by, b, h, precision=precision, tol=1e-13, max_cycles=200)
    assert res.status == 0
    assert np.abs(res.p - pd).max() <= 1e-10 * np.abs(pd).max()
    assert abs(res.p.mean()) < 1e-12 * np.abs(pd).max()


def test_dense_solve_constant_beta_eigenvector(O):
    n, h = 16, 1 / 16
    bx = np.ones((n, n + 1)); bx[:, 0] = bx[:, -1] = 0
    by = np.ones((n + 1, n)); by[0] = by[-1] = 0
    c = np.cos(np.pi * (np.arange(n) + 0.5) / n)
    v = np.outer(c, c)
    lam = -(4 / h**2) * 2 * np.sin(np.pi / (2 * n))**2
    p = O.dense_solve(bx, by, lam * v, h)
    assert np.abs(p - v).max() < 1e-11


def test_mg_status_codes(O):
    n, h = 16, 1 / 16
    rho, mu, bx, by = _betas(n, 9)
    b = W.random_cells(n, n, 10)
    r = O.mg_solve(bx, by, b, h, tol=1e-14, max_cycles=1)
    assert r.status == 3 and r.cycles == 1
    b2 = b.copy(); b2[3, 3] = np.nan
    assert O.mg_solve(bx, by, b2, h).status == 4
    z = O.mg_solve(bx, by, np.full((n, n), 2.0), h)  # constant rhs -> zero after mean removal
    assert z.status == 0 and z.cycles == 0 and np.all(z.p == 0)
    r = O.mg_solve(bx, by, b, h, tol=1e-10)
    assert np.all(np.diff(r.hist) < 0)


def test_mg_levels_rule(O):
    # halve while both sides are even and the level has more than 16 cells
    assert O.mg_levels(64, 64) == [(64, 64), (32, 32), (16, 16), (8, 8), (4, 4)]
    assert O.mg_levels(256, 1024)[-1] == (2, 8)
    assert O.mg_levels(12, 12) == [(12, 12), (6, 6), (3, 3)]
    assert O.mg_levels(20, 12) == [(20, 12), (10, 6), (5, 3)]
    assert O.mg_levels(16, 2) == [(16, 2), (8, 1)] and O.mg_levels(8, 2) == [(8, 2)]


def test_two_inner_cycles_per_fp64_residual(O):
    # precision 2 runs FP32 V-cycles in pairs between FP64 residuals: an even
    # cycle count, no residual formed after the first cycle of a pair, and the
    # iterate after 2k cycles equals k outer steps of one-cycle defect
    # correction only in the limit (both converge to the dense solution).
    n, h = 32, 1 / 32
    rho, mu, bx, by = _betas(n, 41)
    b = W.random_cells(n, n, 42)
    r2 = O.mg_solve(bx, by, b, h, precision=2, tol=1e-12, max_cycles=200)
    r1 = O.mg_solve(bx, by, b, h, precision=1, tol=1e-12, max_cycles=200)
    assert r2.status == 0 and r2.cycles % 2 == 0
    assert np.all(np.isnan(r2.hist[1::2])) and np.all(np.isfinite(r2.hist[0::2]))
    # per V-cycle the pair contracts like two single cycles
    assert r2.cycles <= r1.cycles + 2
    pd = O.dense_solve(bx, by, b, h)
    assert np.abs(r2.p - pd).max() <= 1e-9 * np.abs(pd).max()
