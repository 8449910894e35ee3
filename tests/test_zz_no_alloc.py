"""The no-allocation pressure solve (mg_solve_noalloc) for callers that cannot
allocate device memory: through the C ABI it must give the same solution as
the regular context solve (mg_setup + mg_solve) on the same inputs, on two
calls in a row (its scratch array persists between calls), and reject grids
above its fixed limit.  Kept last in collection order so that a failure here
does not stop the rest of a -x run."""
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


def _system(n, seed):
    import oracle as O
    O.build()
    H = W.random_H(n, n, seed)
    rho, mu, bx, by = O.coeffs(H, 1e-3, 1.0, 1e-4, 1e-2)
    return bx, by, W.random_cells(n, n, seed + 1)


def _reference(ib, T, n, bx, by, b, precision):
    R = min(0.2, 0.45 - 3.0 / n)
    X, Y = W.circle(0.5, 0.5, R, 16)
    ctx = ib.Context(ib.Config(nx=n, ny=n, h=1.0 / n), X, Y, [0, 16])
    d = lambda a: T.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx.mg_setup(d(bx), d(by))
    p = T.zeros((n, n), dtype=T.float64, device="cuda")
    st, cyc, rr = ctx.mg_solve(d(b), p, precision, 1e-10, 200)
    assert st == 0
    return p.cpu().numpy(), cyc


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_noalloc_matches_context_solve_twice(T, precision):
    import paper_1807_10504_gb300 as ib
    d = lambda a: T.from_numpy(np.ascontiguousarray(a)).cuda()
    for n, seed in ((64, 31), (256, 41)):  # two calls in a row, different systems
        bx, by, b = _system(n, seed)
        ref, rcyc = _reference(ib, T, n, bx, by, b, precision)
        p = T.zeros((n, n), dtype=T.float64, device="cuda")
        st, cyc, rr = ib.mg_solve_noalloc(d(bx), d(by), d(b), p, 1.0 / n, precision, 1e-10, 200)
        assert st == ib.IB_OK and rr <= 1e-10 and cyc == rcyc
        assert np.abs(p.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()
    # the same system again: stale scratch contents must not leak in
    p = T.zeros((n, n), dtype=T.float64, device="cuda")
    st, cyc, rr = ib.mg_solve_noalloc(d(bx), d(by), d(b), p, 1.0 / n, precision, 1e-10, 200)
    assert st == ib.IB_OK and cyc == rcyc
    assert np.abs(p.cpu().numpy() - ref).max() <= 1e-10 * np.abs(ref).max()


def test_noalloc_rejects_grids_above_the_limit(T):
    import paper_1807_10504_gb300 as ib
    n = 512  # 262144 cells > 65536
    z = T.zeros((n, n), dtype=T.float64, device="cuda")
    bx = T.zeros((n, n + 1), dtype=T.float64, device="cuda")
    by = T.zeros((n + 1, n), dtype=T.float64, device="cuda")
    st, _, _ = ib.mg_solve_noalloc(bx, by, z, z.clone(), 1.0 / n)
    assert st == ib.IB_EINVAL
    assert "IB_NOALLOC_MAX_CELLS" in ib.noalloc_error()
    # arrays of the wrong shape are refused before the library reads them
    m = 64
    p = T.zeros((m, m), dtype=T.float64, device="cuda")
    bad = T.zeros((m, m), dtype=T.float64, device="cuda")  # beta_x needs m x (m + 1)
    byg = T.zeros((m + 1, m), dtype=T.float64, device="cuda")
    with pytest.raises(ib.IBError) as e:
        ib.mg_solve_noalloc(bad, byg, p.clone(), p, 1.0 / m)
    assert e.value.status == ib.IB_EINVAL
