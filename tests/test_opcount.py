"""The op-counting build of the oracle (no GPU): the counting scalar counts
what it says on expressions with known answers, and the recorded counts the
benchmark's roofline numerators come from (golden/flop_counts.json, written
by golden/make_flop_counts.py) are what the oracle counts today."""
import json
import os

import numpy as np
import pytest

from oracle import opcount

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "flop_counts.json")))
KEYS = ("add", "mul", "div", "exp", "erfc", "sqrt", "tanh")


def test_counting_scalar_on_known_expressions():
    want = {
        "a*b+c": dict(add=1, mul=1),
        "(a+b)*(b+a)": dict(add=1, mul=1),  # the sum is shared (commutative)
        "a^7": dict(mul=4),  # binary exponentiation
        "a*1+0-0*b": {},  # identities fold away
        "exp(a)+exp(a)": dict(exp=1, add=1),  # shared
        "(2*3)*a/-1": dict(mul=1),  # constants fold, negation is free
        "|a-b|/(a+b)+sqrt+erfc+tanh": dict(add=5, div=1, sqrt=1, erfc=1, tanh=1, absminmax=1),
    }
    got = {r["what"]: r for r in opcount.self_test()}
    assert set(got) == set(want)
    for k, w in want.items():
        for key in KEYS + ("absminmax",):
            assert got[k][key] == w.get(key, 0), (k, key, got[k])


def _state(rng, m):
    rho = rng.uniform(0.4, 1.8)
    vel = rng.uniform(-0.9, 0.9, size=m)
    p = rng.uniform(0.4, 1.8)
    return np.array([rho] + list(rho * vel) + [p / 0.4 + 0.5 * rho * vel @ vel])


@pytest.mark.parametrize("m", [1, 2, 3])
def test_flux_count_matches_record(m):
    rng = np.random.default_rng(3 + m)
    cases = [(_state(rng, m), _state(rng, m), rng.normal(size=(m, m + 2)), rng.normal(size=(m, m + 2)), 0.02)]
    r = opcount.gks_point(m, cases)[0]
    g = GOLD[f"gks_point_{m}d"]
    for k in KEYS:
        assert r[k] == g[k], (k, r[k], g[k])


@pytest.mark.parametrize("dim", [2, 3])
def test_cubic_count_matches_record(dim):
    rng = np.random.default_rng(dim)
    nin = 1 + dim + 2 * dim * (1 + dim)
    r = opcount.genomd_cells(dim, [rng.normal(size=nin)])[0]
    g = GOLD[f"cubic_cell_var_{dim}d_limiter0"]
    for k in KEYS:
        assert r[k] == g[k], (k, r[k], g[k])


def test_step_count_per_cell_update_is_grid_independent():
    """On a periodic grid every cell and face is unique, so the count per
    cell-update of an 8^2 grid equals the recorded 16^2 one, and it splits
    into two stages of fluxes plus the two updates."""
    import sys

    sys.path.insert(0, os.path.join(os.path.dirname(__file__), "golden"))
    import make_flop_counts as M

    import oracle as O

    n = 8
    W, G, h = M.smooth_state(2, n, 11)
    cfg = O.make_cfg(2, (n, n), h, bc=0)
    dt = 0.4 * h / O.max_wavespeed(cfg, W)
    r = opcount.step(2, (n, n), h, dt, W, G, what="step")
    per = (r["add"] + r["mul"] + r["div"]) / (n * n)
    assert per == GOLD["step_cell_update_2d"]["flops"]
    parts = 2 * GOLD["flux_stage_cell_2d"]["flops"] + 2 * GOLD["update_cell_stage_2d"]["flops"]
    assert parts == pytest.approx(per, rel=1e-12)
    # one stage's fluxes = the cubics of its cells + 4 face Gauss points per cell
    flux = GOLD["flux_stage_cell_2d"]["flops"]
    gp = GOLD["gks_point_2d"]["flops"] + GOLD["face_states_gp_2d"]["flops"]
    assert flux == pytest.approx(4 * GOLD["cubic_cell_var_2d_limiter0"]["flops"] + 4 * gp, rel=1e-12)
