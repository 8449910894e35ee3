"""The multigrid smoother's failure path, exercised without a GPU fault: the
test hook ib_debug_stall_staging makes every TMA-staged FP32 smoother block
wait, after its copies have landed, on a barrier phase that nothing
completes.  Its wait is bounded (50 ms of global time), so the block skips its
tile and raises the solve's fault word; the solve must return IB_ECUDA with
the time-out named, through the solve graph, the host-driven loop and the
no-allocation entry point alike, and the next solve (hook off) must give the
normal result again."""
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


def _system(O, n, seed):
    H = W.random_H(n, n, seed)
    _, _, bx, by = O.coeffs(H, 1e-3, 1.0, 1e-4, 1e-2)
    return bx, by, W.random_cells(n, n, seed + 1)


def test_staging_time_out_is_reported_and_the_solver_recovers(T, O):
    import paper_1807_10504_gb300 as ib
    d = lambda a: T.from_numpy(np.ascontiguousarray(a)).cuda()
    n = 256  # levels 256^2 and 128^2 are TMA-staged; 64^2 and below form the tail
    bx, by, b = _system(O, n, 71)
    X, Y = W.circle(0.5, 0.5, 0.2, 16)
    ctx = ib.Context(ib.Config(nx=n, ny=n, h=1.0 / n), X, Y, [0, 16])
    ctx.mg_setup(d(bx), d(by))
    bd = d(b)
    zeros = lambda m: T.zeros((m, m), dtype=T.float64, device="cuda")
    ref = zeros(n)
    st, cyc_ref, _ = ctx.mg_solve(bd, ref, 2, 1e-10, 200)
    assert st == ib.IB_OK
    # the no-allocation solve on a grid within its limit
    m = 128
    bx2, by2, b2 = _system(O, m, 81)
    ref2 = zeros(m)
    st, _, _ = ib.mg_solve_noalloc(d(bx2), d(by2), d(b2), ref2, 1.0 / m, 2, 1e-10, 200)
    assert st == ib.IB_OK
    ib.debug_stall_staging(True)
    try:
        for graphs in (True, False):
            ctx.use_graphs(graphs)
            with pytest.raises(ib.IBError) as e:
                ctx.mg_solve(bd, zeros(n), 2, 1e-10, 2)
            assert e.value.status == ib.IB_ECUDA
            assert "staging wait timed out" in str(e.value)
        st, _, _ = ib.mg_solve_noalloc(d(bx2), d(by2), d(b2), zeros(m), 1.0 / m, 1, 1e-10, 2)
        assert st == ib.IB_ECUDA
        assert "staging wait timed out" in ib.noalloc_error()
    finally:
        ib.debug_stall_staging(False)
    T.cuda.synchronize()
    # hook off: the same solves give the same results as before, bit for bit
    for graphs in (True, False):
        ctx.use_graphs(graphs)
        p = zeros(n)
        st, cyc, rr = ctx.mg_solve(bd, p, 2, 1e-10, 200)
        assert st == ib.IB_OK and cyc == cyc_ref and rr <= 1e-10
        assert T.equal(p, ref)
    p2 = zeros(m)
    st, _, rr = ib.mg_solve_noalloc(d(bx2), d(by2), d(b2), p2, 1.0 / m, 2, 1e-10, 200)
    assert st == ib.IB_OK and rr <= 1e-10 and T.equal(p2, ref2)
    assert ib.noalloc_error() == ""
    ctx.close()
