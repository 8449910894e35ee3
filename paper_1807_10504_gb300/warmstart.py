"""Training data and training loop of the learned warm start.

The solver generates its own training pairs: seeded time-step runs on small
grids with 1-8 drops (radii U[0.03, 0.1], density ratio U[100, 1000], viscosity
ratio 100, sigma 1) are advanced with ``ns_step``; every ``every`` steps the
right-hand side b, the cell density rho and the converged pressure p of the
step are copied into device tensors.  The network (``Net``) is then trained on
random mini-batches with its own forward/backward kernels and Adam.  All of it
runs on the GPU through the C ABI; this module only sequences the calls.
"""
from __future__ import annotations

import numpy as np

import workloads as W

from . import Config, Context, Net, _torch


def _drops(n_cells, rng):
    k = int(rng.integers(1, 9))
    h = 1.0 / n_cells
    gap = 8 * h
    centres, radii = [], []
    tries = 0
    while len(centres) < k and tries < 2000:
        tries += 1
        R = rng.uniform(0.03, 0.1)
        c = rng.uniform(R + gap, 1.0 - R - gap, 2)
        if all(np.hypot(*(c - c2)) >= R + R2 + gap for c2, R2 in zip(centres, radii)):
            centres.append(c)
            radii.append(R)
    per = max(24, int(2 * np.pi * max(radii) / (0.75 * h)))
    return W.join([W.circle(c[0], c[1], R, max(24, int(per * R / max(radii))),
                            theta0=rng.uniform(0, 2 * np.pi)) for c, R in zip(centres, radii)])


def generate(n_samples, n_cells=128, seed=0, every=5, steps_per_run=40, precision=1):
    """Returns device tensors (b, rho, p) of shape (n_samples, n_cells, n_cells)."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    B = torch.empty((n_samples, n_cells, n_cells), dtype=torch.float64, device="cuda")
    R = torch.empty_like(B)
    P = torch.empty_like(B)
    got = 0
    h = 1.0 / n_cells
    while got < n_samples:
        mk = _drops(n_cells, rng)
        ratio = rng.uniform(100.0, 1000.0)
        cfg = Config(nx=n_cells, ny=n_cells, h=h, rho_l=1.0, rho_g=1.0 / ratio, mu_l=1e-2,
                     mu_g=1e-2 / 100.0, sigma=1.0, precision=precision, relocate_every=10)
        ctx = Context(cfg, mk.X, mk.Y, mk.drop_start)
        dt = W.capillary_dt(h, cfg.rho_l, cfg.rho_g, cfg.sigma, cfg.mu_l, cfg.mu_g)
        for s in range(steps_per_run):
            try:
                ctx.ns_step(dt, 1, 1)
            except Exception:
                break  # a drop reached a wall: start the next run
            if (s + 1) % every == 0 and got < n_samples:
                B[got] = ctx.get("b")
                R[got] = ctx.get("rho")
                P[got] = ctx.get("p")
                got += 1
        ctx.close()
    return B, R, P


def train(net: Net, data, steps=1000, batch=16, lr=2e-3, seed=0):
    """One training run on the solver-generated samples (``cnn_train``: the
    pressure scale fitted from the data, then Adam on random mini-batches with
    the learning rate decaying tenfold); returns the list of batch losses."""
    B, R, P = data
    return net.train(B, R, P, steps, batch, lr, seed)


def evaluate(net: Net, n_cells=512, ndrops=8, seed=1810, steps=6, precision=1, reps=5):
    """Pressure solves of one seeded multi-drop system from three starting
    points: zero (cold), the previous step's pressure, and the network's
    estimate; each solved to 1e-10 with the given precision.  Returns
    {start: {"cycles", "ms", "relres"}} (ms = median over `reps`, CUDA events,
    the network's inference included in its time)."""
    torch = _torch()
    h = 1.0 / n_cells
    mk = W.multidrop(n_cells, ndrops=ndrops, rmin=0.03, rmax=0.1, n_per_drop=256, seed=seed,
                     gap_cells=12)
    cfg = Config(nx=n_cells, ny=n_cells, h=h, precision=precision, relocate_every=10)
    ctx = Context(cfg, mk.X, mk.Y, mk.drop_start)
    dt = W.capillary_dt(h, cfg.rho_l, cfg.rho_g, cfg.sigma, cfg.mu_l, cfg.mu_g)
    ctx.ns_step(dt, steps - 1, 1)
    p_prev = ctx.get("p")
    ctx.ns_step(dt, 1, 1)
    b, rho = ctx.get("b"), ctx.get("rho")
    out = {}
    for name in ("cold", "prev", "cnn"):
        times, cyc, rr = [], None, None
        for _ in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            if name == "cold":
                p = torch.zeros_like(b)
            elif name == "prev":
                p = p_prev.clone()
            else:
                p = net.infer(b[None], rho[None])[0]
            st, cyc, rr = ctx.mg_solve(b, p, precision, 1e-10, 200)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        out[name] = {"cycles": cyc, "ms": float(np.median(times[1:])), "relres": rr}
    ctx.close()
    return out
