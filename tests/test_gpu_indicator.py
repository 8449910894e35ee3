"""GPU parity of the indicator function of Section 2.2 Eq. (ind_psn) (the
conventional scheme's density and viscosity field) with the oracle: composed
steps whose properties come from the Poisson indicator instead of the
polygon Heaviside, planar and axisymmetric."""
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
def test_indicator_steps_match_oracle(T, ib, O, axisym):
    if axisym:
        nx, ny, h = 32, 64, 1 / 32
        mk = W.axi_elliptic_drop(1.0, 0.25, 1.1, 128)
        kw = dict(axisym=1)
    else:
        nx, ny, h = 64, 64, 1 / 64
        mk = W.elliptic_drop(0.5, 0.5, 0.22, 1.15, 128)
        kw = {}
    kw.update(spread=0, relocate_every=0, indicator=1, tol=1e-11)
    ctx = ib.Context(ib.Config(nx=nx, ny=ny, h=h, **kw), mk.X, mk.Y, mk.drop_start)
    ocfg = O.Config(nx=nx, ny=ny, h=h, **kw)
    st = O.init_state(ocfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, 1.0, 1e-3, 1.0, 1e-2, 1e-4)
    for _ in range(3):
        ctx.ns_step(dt, 1, 1)
        O.ns_step(ocfg, st, dt)
    rho = ctx.get("rho").cpu().numpy()
    assert np.abs(rho - st.last["rho"]).max() <= 1e-10
    # the property field is the smooth indicator, not the polygon Heaviside
    H = ctx.get("H").cpu().numpy()
    assert np.abs((rho - 1e-3) / (1 - 1e-3) - H).max() > 1e-3
    # p within 1e-10 of max |p|; u, v within 1e-10 of the inertial-capillary
    # velocity sqrt(sigma / (rho_l R))
    U = np.sqrt(1.0 / (1.0 * 0.22))
    got = ctx.get("p").cpu().numpy()
    assert np.abs(got - st.p).max() <= 1e-10 * np.abs(st.p).max(), np.abs(got - st.p).max()
    for name, ref in (("u", st.u), ("v", st.v)):
        got = ctx.get(name).cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-10 * U, (name, np.abs(got - ref).max())
