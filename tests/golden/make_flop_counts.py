"""Record the algorithmic operation counts of the oracle (flop_counts.json).

Runs the op-counting build of the oracle (oracle/opcount.py: the oracle's own
arithmetic, common subexpressions shared and constants folded) on seeded
smooth states, where no admissibility fallback fires, so every count is
that of the general case.  flops = add/sub + mul + div (an FMA is 2);
transcendentals (exp, erfc, sqrt, tanh) are one op each and kept apart.
The benchmark takes its roofline numerators from this file.

    python tests/golden/make_flop_counts.py
"""
from __future__ import annotations

import json
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from oracle import opcount  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "flop_counts.json")
TRANS = ("exp", "erfc", "sqrt", "tanh")


def smooth_state(dim, n, seed):
    """Smooth periodic state with a small seeded perturbation (no fallback)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    axes = np.meshgrid(*[(np.arange(n) + 0.5) * h] * dim, indexing="ij")[::-1]  # x, y, z
    ph = sum((a + 1) * x for a, x in enumerate(axes))
    rho = 1.0 + 0.2 * np.sin(2 * math.pi * ph) + 0.02 * rng.random(axes[0].shape)
    vel = [0.3 * np.cos(2 * math.pi * (ph + 0.1 * a)) for a in range(dim)]
    p = 1.0 + 0.1 * np.cos(2 * math.pi * ph)
    W = np.stack([rho] + [rho * u for u in vel] + [p / 0.4 + 0.5 * rho * sum(u * u for u in vel)])
    G = 0.1 * rng.normal(size=(dim,) + W.shape)
    return W, G, h


def summary(r, per=1.0):
    d = {k: r[k] / per for k in ("add", "mul", "div") + TRANS}
    d["flops"] = (r["add"] + r["mul"] + r["div"]) / per
    d["transcendental"] = sum(r[k] for k in TRANS) / per
    return d


def diff(a, b, per):
    return summary({k: a[k] - b[k] for k in ("add", "mul", "div") + TRANS}, per)


def random_prim_state(rng, m):
    rho = rng.uniform(0.4, 1.8)
    vel = rng.uniform(-0.9, 0.9, size=m)
    p = rng.uniform(0.4, 1.8)
    return np.array([rho] + list(rho * vel) + [p / 0.4 + 0.5 * rho * vel @ vel])


def main():
    rng = np.random.default_rng(20461)
    out = {"convention": "flops = add/sub + mul + div (FMA = 2); transcendentals exp, erfc, sqrt, tanh one op each, "
                         "kept apart; common subexpressions shared and constants folded (oracle/opcount.hpp)"}
    # gas-kinetic flux at one face Gauss point (face frame), Euler and Navier-Stokes
    for m in (1, 2, 3):
        for tm, mu in ((0, 0.0), (2, 0.01)):
            if m == 1 and tm == 2:
                continue
            cases = [(random_prim_state(rng, m), random_prim_state(rng, m), rng.normal(size=(m, m + 2)),
                      rng.normal(size=(m, m + 2)), 0.01) for _ in range(3)]
            rs = opcount.gks_point(m, cases, tau_mode=tm, mu=mu)
            assert all(r["status"] == 0 for r in rs)
            assert all(r == rs[0] for r in rs), "data-independent count"
            out[f"gks_point_{m}d" + ("_ns" if tm == 2 else "")] = summary(rs[0])
    # blended cubic of one (cell, variable), GENO / WENO-Z / TENO
    for dim in (2, 3):
        for lim in (0, 2, 3):
            nin = 1 + dim + 2 * dim * (1 + dim)
            rs = opcount.genomd_cells(dim, [rng.normal(size=nin) for _ in range(64)], limiter=lim)
            if lim != 3:
                assert all(r == rs[0] for r in rs), "data-independent count"
            # TENO cuts candidates (products with a zero weight fold away): mean over the sample
            mean = {k: float(np.mean([r[k] for r in rs])) for k in ("add", "mul", "div") + TRANS}
            out[f"cubic_cell_var_{dim}d_limiter{lim}"] = summary(mean)
    # whole grids: one stage's interface states, one stage's fluxes, one step
    for dim, n in ((2, 16), (3, 6)):
        W, G, h = smooth_state(dim, n, 7 + dim)
        cfg = O.make_cfg(dim, (n,) * dim, h, bc=0)
        dt = 0.4 * h / O.max_wavespeed(cfg, W)
        rec = opcount.step(dim, (n,) * dim, h, dt, W, G, what="recon")
        flx = opcount.step(dim, (n,) * dim, h, dt, W, G, what="flux")
        stp = opcount.step(dim, (n,) * dim, h, dt, W, G, what="step")
        cells = n**dim
        ngp = dim * cells * (2 if dim == 2 else 4)  # unique face Gauss points (periodic)
        fit = out[f"cubic_cell_var_{dim}d_limiter0"]
        nv = dim + 2
        fits = {k: fit[k] * nv * cells for k in ("add", "mul", "div") + TRANS}
        out[f"face_states_gp_{dim}d"] = diff(rec, fits, ngp)
        out[f"flux_stage_cell_{dim}d"] = summary(flx, cells)
        out[f"step_cell_update_{dim}d"] = summary(stp, cells)
        two = {k: 2 * flx[k] for k in ("add", "mul", "div") + TRANS}
        out[f"update_cell_stage_{dim}d"] = diff(stp, two, 2 * cells)
        out[f"grid_{dim}d"] = {"n": n, "cells": cells, "unique_gauss_points": ngp, "seed": 7 + dim}
    # 1D non-compact GENO (order 5 / 6), HLLC, classical RK4: one step of a
    # smooth periodic grid, per cell-update (the face kernel evaluates each
    # face once per RK stage)
    n = 64
    W1, _, h1 = smooth_state(1, n, 5)
    cfg1 = O.make_cfg(1, (n,), h1, bc=0)
    dt1 = 0.4 * h1 / O.max_wavespeed(cfg1, W1)
    for order in (5, 6):
        r = opcount.nc_step(order, n, h1, dt1, W1)
        assert r["status"] == 0
        out[f"nc_step_cell_update_1d_order{order}"] = summary(r, n)
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps({k: v.get("flops") for k, v in out.items() if isinstance(v, dict)}, indent=1))


if __name__ == "__main__":
    main()
