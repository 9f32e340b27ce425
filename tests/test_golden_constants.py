"""The constants and the accuracy-test data printed in the paper (golden
fixture with citations) against the oracle's defaults and the input
generators (no GPU)."""
import json
import math
import os

import numpy as np

from paper_2507_20461_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_oracle_defaults_are_the_papers(oracle):
    cfg = oracle.make_cfg(1, (8,), 0.1)
    assert cfg.C == GOLD["C"]["value"]
    assert cfg.eps == GOLD["eps"]["value"]
    assert cfg.C0 == GOLD["C0"]["value"]
    assert cfg.teno_ct == GOLD["teno_ct"]["value"]


def test_oracle_uses_r2_in_1d_and_r3_in_multid(oracle):
    """alpha^H = 1 + (IS^tau / (IS^H + eps))^r: recover r from chi on a
    crafted 1D point and a multi-D cell."""
    # 1D: any data, recompute chi with r = 2 from the returned indicators
    cfg = oracle.make_cfg(1, (8,), 0.1)
    rng = np.random.default_rng(0)
    for _ in range(20):
        o = oracle.geno1d_point(cfg, rng.normal(size=5), rng.normal(size=5) * 0.1, 0)
        r = GOLD["r_structured"]["value"]
        aH = 1 + (o["IStau"] / (o["ISH"] + 1e-15)) ** r
        aL = 1 + (o["IStau"] / (o["ISL"] + 1e-15)) ** r
        chi = math.tanh(GOLD["C"]["value"] * 2 * aH / (aH + aL)) / math.tanh(GOLD["C"]["value"])
        assert abs(chi - o["chi"]) < 1e-12
    cfg = oracle.make_cfg(2, (8, 8), 0.1)
    for _ in range(20):
        o = oracle.genomd_cell(cfg, 0.3, rng.normal(size=2), rng.normal(size=4), rng.normal(size=(4, 2)))
        r = GOLD["r_unstructured"]["value"]
        aH = 1 + (o["IStau"] / (o["ISH"] + 1e-15)) ** r
        aL = 1 + (o["IStau"] / (o["ISL"] + 1e-15)) ** r
        chi = math.tanh(GOLD["C"]["value"] * 2 * aH / (aH + aL)) / math.tanh(GOLD["C"]["value"])
        assert abs(chi - o["chi"]) < 1e-12


def test_accuracy_ic_matches_paper():
    g = GOLD["accuracy_1d"]
    n = 64
    W, G, h = I.sine_wave(1, n)
    x = (np.arange(n) + 0.5) * h
    assert h == (g["domain"][1] - g["domain"][0]) / n
    # cell averages converge to the point values of the printed IC
    np.testing.assert_allclose(W[0], 1 + g["rho_amp"] * np.sin(math.pi * x), atol=2e-3)
    np.testing.assert_allclose(W[1] / W[0], g["U"])
    p = 0.4 * (W[2] - 0.5 * W[1] ** 2 / W[0])
    np.testing.assert_allclose(p, g["p"], rtol=1e-13)
