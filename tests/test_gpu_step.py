"""GPU parity of the composed time step (ns_step through the C ABI) against
the oracle's step on the static-drop (64^2) and oscillating-drop (256^2)
workloads, checkpoint/resume bit-identity and run-to-run determinism."""
import os

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


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def run_pair(ib, O, n, mk, steps, tol=1e-12, **kw):
    h = 1.0 / n
    cfg = ib.Config(nx=n, ny=n, h=h, tol=tol, max_cycles=200, **kw)
    ctx = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
    ocfg = O.Config(nx=n, ny=n, h=h, tol=tol, max_cycles=200,
                    **{k: v for k, v in kw.items() if k != "precision"})
    st = O.init_state(ocfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    for _ in range(steps):
        ctx.ns_step(dt, 1, 1)
        O.ns_step(ocfg, st, dt)
    return ctx, st


def u_scale(sigma, rho_l, R):
    """Inertial-capillary velocity sqrt(sigma / (rho_l R)) of a drop of radius
    R: the physical scale of surface-tension-driven flow, against which
    velocity differences are measured (the balanced static drop's own
    velocity is roundoff, so its maximum is no scale)."""
    return float(np.sqrt(sigma / (rho_l * R)))


@pytest.mark.parametrize("spread", [0, 1])
def test_static_drop_steps_match_oracle(T, ib, O, spread):
    # the FP64 path: p within 1e-10 of max |p|, u, v within 1e-10 of the
    # capillary velocity scale, markers within 1e-12, after 3 steps
    mk = W.static_drop(64, 0.25, 128)
    ctx, st = run_pair(ib, O, 64, mk, 3, spread=spread, relocate_every=10)
    U = u_scale(1.0, 1.0, 0.25)
    assert rel(ctx.get_host("p"), st.p) <= 1e-10
    for name, ref in (("u", st.u), ("v", st.v)):
        assert np.abs(ctx.get_host(name) - ref).max() <= 1e-10 * U, name
    X, Y = ctx.markers()
    assert np.abs(X.cpu().numpy() - st.X).max() <= 1e-12
    assert np.abs(Y.cpu().numpy() - st.Y).max() <= 1e-12


def test_oscillating_drop_precisions_match_oracle_over_2000_steps(T, ib, O):
    """The 256^2 oscillating-drop workload (r = 0.2 (1 + 0.05 cos 2 theta),
    512 markers with +-1e-3 jitter, density ratio 1000, viscosity ratio 100,
    relocation every 10 steps, pressure to 1e-10): each precision path of
    the GPU step against the oracle's FP64 step at steps 1, 10, 100, 500 and
    2000.  FP64: p within 1e-10 of max |p| and u, v within 1e-10 of the
    capillary velocity scale; FP32 smoothing in FP64 defect correction (one or
    two V-cycles per FP64 residual): within 1e-6 after refinement; markers
    within 1e-12 for all.  The oracle runs its OpenMP build (bit-identical to
    the serial one)."""
    n, h = 256, 1.0 / 256
    mk = W.oscillating_drop()
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    kw = dict(nx=n, ny=n, h=h, tol=1e-10, max_cycles=200, spread=1, relocate_every=10)
    ctxs = {p: ib.Context(ib.Config(precision=p, **kw), mk.X, mk.Y, mk.drop_start)
            for p in (0, 1, 2)}
    ocfg = O.Config(precision=0, **kw)
    st = O.init_state(ocfg, mk.X, mk.Y, mk.drop_start)
    U = u_scale(1.0, 1.0, 0.2)
    worst = {p: 0.0 for p in ctxs}
    O.set_threads(True)
    try:
        for k in range(1, 2001):
            O.ns_step(ocfg, st, dt)
            for c in ctxs.values():
                c.ns_step(dt, 1, 1)
            if k not in (1, 10, 100, 500, 2000):
                continue
            for p, c in ctxs.items():
                ep = rel(c.get_host("p"), st.p)
                eu = max(np.abs(c.get_host("u") - st.u).max(),
                         np.abs(c.get_host("v") - st.v).max()) / U
                X, Y = (a.cpu().numpy() for a in c.markers())
                em = max(np.abs(X - st.X).max(), np.abs(Y - st.Y).max())
                bound = 1e-10 if p == 0 else 1e-6
                assert ep <= bound and eu <= bound and em <= 1e-12, (p, k, ep, eu, em)
                worst[p] = max(worst[p], ep, eu)
    finally:
        O.set_threads(False)
        for c in ctxs.values():
            c.close()
    print("worst relative difference from the FP64 oracle by precision:", worst)


def test_oscillating_drop_step_fields_match_oracle(T, ib, O):
    # the step's intermediate fields (Heaviside and face force) after two steps
    mk = W.oscillating_drop()
    ctx, st = run_pair(ib, O, 256, mk, 2, tol=1e-12, spread=1, relocate_every=10)
    for name, ref in (("H", st.last["H"]), ("Fx", st.last["Fx"]), ("Fy", st.last["Fy"])):
        assert rel(ctx.get_host(name), ref) <= 1e-11, name
    assert rel(ctx.get_host("p"), st.p) <= 1e-10


def test_checkpoint_resume_and_determinism(T, ib, tmp_path):
    mk = W.oscillating_drop(200, seed=5)
    n = 96
    cfg = ib.Config(nx=n, ny=n, h=1.0 / n, relocate_every=3)
    dt = W.capillary_dt(1.0 / n, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    a = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
    a.ns_step(dt, 2, 1)
    path = os.path.join(tmp_path, "ck.bin")
    a.save(path)
    a.ns_step(dt, 3, 1)
    b = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
    b.load(path)
    b.ns_step(dt, 3, 1)
    c = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
    c.ns_step(dt, 5, 1)
    for name in ("u", "v", "p"):
        ua, ub, uc = a.get_host(name), b.get_host(name), c.get_host(name)
        assert np.array_equal(ua, ub) and np.array_equal(ua, uc), name
    assert T.equal(a.markers()[0], b.markers()[0])


def test_step_errors(T, ib):
    mk = W.static_drop(32, 0.25, 64)
    cfg = ib.Config(nx=32, ny=32, h=1 / 32)
    ctx = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
    with pytest.raises(ib.IBError) as e:
        ctx.ns_step(-1.0)
    assert e.value.status == ib.IB_EINVAL
    # a huge time step throws markers out of the domain: reported, no fault
    u = T.full((32, 33), 50.0, dtype=T.float64, device="cuda")
    u[:, 0] = 0
    u[:, -1] = 0
    ctx.set("u", u)
    with pytest.raises(ib.IBError) as e:
        ctx.ns_step(0.05, 1, 1)
    assert e.value.status == ib.IB_EMARKER


def test_oscillating_drop_precisions_and_period(T, ib):
    # The 256^2 oscillating drop (r = 0.2 (1 + 0.05 cos 2 theta), density
    # ratio 1000, viscosity ratio 100, sigma 1, 512 markers, relocation every
    # 10 steps): (1) after 2000 steps the FP32-smoothing path agrees with the
    # FP64 path to 1e-6 on u, v and p; (2) the first extremum of the x-extent
    # falls at half the n = 2 capillary period of the closed form, 2 pi
    # sqrt((rho_d + rho_a) r^3 / ((n^3 - n) sigma)), within 5 %.
    n, h = 256, 1.0 / 256
    mk = W.oscillating_drop()
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    res = {}
    for prec in (0, 1):
        cfg = ib.Config(nx=n, ny=n, h=h, precision=prec, tol=1e-10, max_cycles=200, spread=1,
                        relocate_every=10)
        ctx = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
        ctx.ns_step(dt, 2000, 1)
        res[prec] = {k: ctx.get_host(k) for k in ("u", "v", "p")}
        if prec == 1:
            ext, ts = [], []
            for k in range(150):
                ctx.ns_step(dt, 20, 1)
                X, Y = ctx.markers()
                ext.append(float(X.max() - X.min()) - float(Y.max() - Y.min()))
                ts.append((2000 + 20 * (k + 1)) * dt)
        ctx.close()
    for k in ("u", "v", "p"):
        scale = np.abs(res[0][k]).max()
        assert np.abs(res[1][k] - res[0][k]).max() <= 1e-6 * scale, k
    ext = np.array(ext)
    i = int(np.argmin(ext))  # the drop starts elongated in x: first minimum at T/2
    assert 0 < i < len(ext) - 1
    a, b, c = np.polyfit(np.array(ts[i - 1:i + 2]), ext[i - 1:i + 2], 2)
    t_half = -b / (2 * a)
    T2 = 2 * np.pi * np.sqrt((1.0 + 1e-3) * 0.2 ** 3 / (6 * 1.0))
    assert abs(2 * t_half - T2) <= 0.05 * T2, (2 * t_half, T2)


def test_extrapolated_warm_start_reaches_the_same_solution(T, ib):
    # warm = 3 starts each pressure solve from 2 p^n - p^(n-1): the solution
    # after each step is the one from the previous-pressure start (same
    # tolerance) and no more V-cycles are needed.
    import numpy as np
    n, h = 128, 1 / 128
    mk = W.oscillating_drop(n_markers=256)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    out = {}
    for warm in (1, 3):
        cfg = ib.Config(nx=n, ny=n, h=h, precision=2, tol=1e-11, spread=1, relocate_every=10)
        ctx = ib.Context(cfg, mk.X, mk.Y, mk.drop_start)
        cyc = []
        for _ in range(30):
            c, rr = ctx.ns_step(dt, 1, warm)
            assert rr <= 1e-11
            cyc.append(c)
        out[warm] = (ctx.get_host("p"), ctx.get_host("u"), sum(cyc[5:]))
        ctx.close()
    p1, p3 = out[1][0], out[3][0]
    assert np.abs(p1 - p3).max() <= 1e-7 * np.abs(p1).max()
    assert out[3][2] <= out[1][2]


def test_ns_step_io_matches_separate_calls(T, ib):
    """ns_step_io (markers in, step, pressure and markers out, one host
    synchronisation) against ib_set_markers + ns_step + ib_get_field +
    ib_get_markers on an identical context: bit-identical results, including
    a relocation step; an unpaired marker buffer is rejected."""
    n = 64
    mk = W.oscillating_drop(128, 0.2, 0.05, 1e-3, 1808)
    dt = W.capillary_dt(1.0 / n, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    ctxs = [ib.Context(ib.Config(nx=n, ny=n, h=1.0 / n, relocate_every=2, precision=2, tol=1e-10),
                       mk.X, mk.Y, mk.drop_start) for _ in range(2)]
    pin = lambda shape: T.empty(shape, dtype=T.float64).pin_memory().numpy()
    M = ctxs[0].M
    Xa, Ya, Xb, Yb = pin(M), pin(M), pin(M), pin(M)
    pa, pb = pin((n, n)), pin((n, n))
    ctxs[0].get_markers_host(Xa, Ya)
    ctxs[1].get_markers_host(Xb, Yb)
    for _ in range(3):
        ctxs[0].set_markers_host(Xa, Ya)
        ctxs[0].ns_step(dt, 1, 1)
        ctxs[0].get_host("p", pa)
        ctxs[0].get_markers_host(Xa, Ya)
        ctxs[1].ns_step_io(dt, 1, Xb, Yb, pb, Xb, Yb)
        assert np.array_equal(pa, pb)
        assert np.array_equal(Xa, Xb) and np.array_equal(Ya, Yb)
    with pytest.raises(ib.IBError) as e:
        ctxs[1].ns_step_io(dt, 1, Xb, None)
    assert e.value.status == ib.IB_EINVAL
    for c in ctxs:
        c.close()


def test_static_drop_100_steps_parasitic_currents_and_laplace_jump(T, ib):
    """The Laplace test (Section 5.1): the 64^2 static drop after 100 FP64 steps.
    With markers as placed (curvature exactly 1/R) the irrotational force is
    a discrete gradient balanced by the pressure: no parasitic current to
    roundoff and the jump of Eq. (sd_pres_diff) equal to sigma / R = 4; the
    conventional spreading drives parasitic currents.  With B-spline
    relocation the fitted curvature varies slightly and the irrotational
    currents stay two orders of magnitude below the conventional ones."""
    import bench
    rep = bench.static_drop_report(ib, 100)
    irr, conv = rep["irrotational_relocate0"], rep["conventional_relocate0"]
    assert irr["max_u"] < 1e-9 and irr["jump_rel_err"] < 1e-9, irr
    assert conv["max_u"] > 1e-4 and conv["jump_rel_err"] < 0.05, conv
    assert rep["irrotational_relocate10"]["max_u"] < 1e-2 * rep["conventional_relocate10"]["max_u"]
    print("static drop, 100 steps:", rep)


def test_step_reports_its_solve_status_after_the_launches_that_follow_it(T, ib):
    """ns_step queues the pressure solve and the launches after it without a
    host wait and reads the solve's status at the step's final
    synchronisation.  A solve stopped by its cycle cap still reports
    IB_ENOTCONV (and its cycle count) through the recorded graphs as through
    direct launches; a solve whose smoother blocks time out (the staging
    test hook, bounded waits) reports IB_ECUDA with the time-out named, ahead
    of any marker flag the step's later launches may raise."""
    n = 256  # levels 256^2 and 128^2 are TMA-staged
    mk = W.static_drop(n, 0.25, 256)
    kw = dict(nx=n, ny=n, h=1.0 / n, precision=2, tol=1e-15, max_cycles=2, relocate_every=0)
    got = []
    for graphs in (True, False):
        ctx = ib.Context(ib.Config(**kw), mk.X, mk.Y, mk.drop_start)
        ctx.use_graphs(graphs)
        res = []
        for _ in range(3):  # the first step runs direct, the next ones replay graphs
            with pytest.raises(ib.IBError) as e:
                ctx.ns_step(1e-4, 1, 1)
            assert e.value.status == ib.IB_ENOTCONV
            cyc, rr = C_last(ib, ctx)
            assert cyc == 2 and rr > 1e-15
            res.append(rr)
        got.append(res)
        ctx.close()
    assert got[0] == got[1]
    ctx = ib.Context(ib.Config(**kw), mk.X, mk.Y, mk.drop_start)
    with pytest.raises(ib.IBError):
        ctx.ns_step(1e-4, 1, 1)  # cycle cap, as above; the graphs are recorded
    ib.debug_stall_staging(True)
    try:
        with pytest.raises(ib.IBError) as e:
            ctx.ns_step(1e-4, 1, 1)
        assert e.value.status == ib.IB_ECUDA
        assert "staging wait timed out" in str(e.value)
    finally:
        ib.debug_stall_staging(False)
    T.cuda.synchronize()
    ctx.close()


def C_last(ib, ctx):
    import ctypes
    cyc, rr = ctypes.c_int(0), ctypes.c_double(0.0)
    ib.lib().ib_last_solve(ctx._h, ctypes.byref(cyc), ctypes.byref(rr))
    return cyc.value, rr.value
