"""Conditioning of the mixed-precision parity cases (oracle only, no GPU).

The admissibility fallback (reading R9) replaces a reconstructed face state
by its cell's average when its rho or p is not above delta = 0.3 times the
cell's.  It is a switch: a face whose ratio sits near delta goes one way or
the other under a tiny change of the state.  The mixed-precision path takes
the decision on FP32 face states (relative rounding of order 1e-5 where
p = (gamma - 1)(E - rho |u|^2 / 2) cancels), the oracle on FP64 ones, so a
mean-L1 bar of 1e-5 against the oracle only tests the FP32 arithmetic on a
case with no decision that close to its threshold.

Pinned here, by moving delta in the oracle:
* the smooth Fourier case (config 3's modes without shocks, drifting at
  (0.5, 0.25)) and the 1D Riemann case are unchanged, bit for bit, under a
  relative 3e-3 change of delta;
* the 64^2 Fourier + shock case is not: a relative 1e-4 change moves its
  20-step density by more than 1e-4 in the mean, so its GPU test is held to
  that spread rather than to 1e-5.
"""
import numpy as np

from paper_2507_20461_gb300 import inputs as I

STEPS = 20


def _run(oracle, dim, n, h, bc, W, G, adm):
    cfg = oracle.make_cfg(dim, (n,) * dim, h, bc=bc, adm_delta=adm)
    W, G = W.copy(), G.copy()
    for _ in range(STEPS):
        dt = 0.4 * h / oracle.max_wavespeed(cfg, W)
        assert oracle.step(cfg, dt, W, G) == 0
    return W


def test_smooth_fourier_case_has_no_decision_near_threshold(oracle):
    W, G, h = I.fourier_shocks_2d(64, seed=20463, nshocks=0, drift=(0.5, 0.25))
    ref = _run(oracle, 2, 64, h, 0, W, G, 0.3)
    for r in (-3e-3, 3e-3):
        assert np.array_equal(_run(oracle, 2, 64, h, 0, W, G, 0.3 * (1 + r)), ref)


def test_riemann_1d_case_has_no_decision_near_threshold(oracle):
    W, G, h, _ = I.riemann_1d(200, seed=20461)
    ref = _run(oracle, 1, 200, h, 1, W, G, 0.3)
    for r in (-3e-3, 3e-3):
        assert np.array_equal(_run(oracle, 1, 200, h, 1, W, G, 0.3 * (1 + r)), ref)


def test_shock_case_has_a_decision_within_fp32_rounding(oracle):
    W, G, h = I.fourier_shocks_2d(64, seed=20463)
    ref = _run(oracle, 2, 64, h, 0, W, G, 0.3)
    moved = _run(oracle, 2, 64, h, 0, W, G, 0.3 * (1 + 1e-4))
    assert np.abs(moved[0] - ref[0]).mean() > 1e-4
    # the drift-free smooth variant keeps its modes: the generator's draws
    # are those of the shock case
    Ws, _, _ = I.fourier_shocks_2d(64, seed=20463, nshocks=0)
    assert np.allclose(Ws[0].mean(), 1.0) and Ws[0].std() > 0.01
