"""Pins of the oracle's WENO-Z and TENO weight variants (no GPU).

Sec. 5.1 defines the WENO-Z weights (Eq. wgt-WENO-Z) and the TENO weights
(Eq. wgt-TENO-1 with the exponent 7, Eq. wgt-TENO-2 with the cut-off
C_T = 1e-6).  The paper runs them in its compact schemes by replacing the
nonlinear weights of its earlier (unprinted) combination; here they act on
GENO's candidates in the adaptive-order combination (reading R14):

    R = (w0/d0) q^H + sum_k (w_k - (w0/d0) d_k) p_k,   d0 = 0.85.

What fixes it independently of the oracle's arithmetic:
* consistency: when every candidate is the same polynomial, R is that
  polynomial whatever the weights (the combination's coefficients sum to 1);
* the ENO property at a jump: TENO's cut keeps exactly the smooth candidates,
  WENO-Z's weights on the others vanish to rounding;
* TENO keeps every candidate on resolved smooth 1D data, so it is the
  linear scheme there; at smooth extrema in multi-D it cuts the high-order
  candidate (Sec. 5.2), and the errors order as GENO < WENO-Z < TENO;
* the paper's accuracy comparison (Sec. 6.1, 8th-order compact GKS): on the
  coarsest mesh the GENO result is the best of the three.
"""
import numpy as np
import pytest

from paper_2507_20461_gb300 import inputs as I


def _quadratic_cells(a, b, c):
    """averages and cell-unit averaged derivatives of a + b xi + c xi^2 on cells -2..2"""
    k = np.arange(-2, 3, dtype=np.float64)
    w = a + b * k + c * (k * k + 1.0 / 12.0)
    d = b + 2 * c * k
    return w, d


@pytest.mark.parametrize("limiter", [2, 3])
def test_equal_candidates_reproduce_the_polynomial(oracle, limiter):
    cfg = oracle.make_cfg(1, (8,), 0.1, limiter=limiter)
    for a, b, c in ((1.0, 0.3, -0.2), (2.0, -1.0, 0.5), (0.5, 0.0, 0.0)):
        w, d = _quadratic_cells(a, b, c)
        left = oracle.geno1d_point(cfg, w, d, 0)
        assert left["val"] == pytest.approx(a + b / 2 + c / 4, rel=1e-14, abs=1e-14)
        assert left["der"] == pytest.approx(b + c, rel=1e-13, abs=1e-13)
        right = oracle.geno1d_point(cfg, w, d, 1)
        assert right["val"] == pytest.approx(a - b / 2 + c / 4, rel=1e-14, abs=1e-14)


def test_step_keeps_only_the_smooth_candidates_1d(oracle):
    """Left state at the face j+1/2 with a jump between cells j+1 and j+2: the
    sub-stencils {j-1, j} and {j-1, j, j+1} are smooth (constant 0)."""
    w = np.array([0.0, 0.0, 0.0, 0.0, 1.0])
    d = np.zeros(5)
    teno = oracle.geno1d_point(oracle.make_cfg(1, (8,), 0.1, limiter=3), w, d, 0)
    assert teno["val"] == 0.0 and teno["der"] == 0.0 and teno["chi"] == 0.0
    wz = oracle.geno1d_point(oracle.make_cfg(1, (8,), 0.1, limiter=2), w, d, 0)
    assert abs(wz["val"]) <= 1e-12 and wz["chi"] <= 1e-12
    # the linear scheme overshoots there (the pin is not vacuous)
    lin = oracle.geno1d_point(oracle.make_cfg(1, (8,), 0.1, limiter=1), w, d, 0)
    assert abs(lin["val"]) > 1e-3


@pytest.mark.parametrize("m", [2, 3])
def test_step_keeps_only_the_smooth_candidates_multid(oracle, m):
    """A jump across the +x face only: TENO cuts the cubic and the +x linear
    polynomial; the kept linear polynomials are flat, so the blended
    polynomial is exactly the cell average."""
    W0, D0 = 0.0, [0.0] * m
    Wn = [0.0] * (2 * m)
    Wn[1] = 1.0  # q = 2 e + (side > 0): +x is q = 1
    Dn = [[0.0] * m for _ in range(2 * m)]
    teno = oracle.genomd_cell(oracle.make_cfg(m, (8,) * m, 0.1, limiter=3), W0, D0, Wn, Dn)
    assert np.all(teno["coef"] == 0.0) and teno["chi"] == 0.0
    wz = oracle.genomd_cell(oracle.make_cfg(m, (8,) * m, 0.1, limiter=2), W0, D0, Wn, Dn)
    assert np.abs(wz["coef"]).max() <= 1e-12
    lin = oracle.genomd_cell(oracle.make_cfg(m, (8,) * m, 0.1, limiter=1), W0, D0, Wn, Dn)
    assert np.abs(lin["coef"]).max() > 1e-3


def _run(oracle, dim, n, limiter, t_end, cfl=0.4):
    W, G, h = I.sine_wave(dim, n)
    cfg = oracle.make_cfg(dim, (n,) * dim, h, bc=0, limiter=limiter)
    t = 0.0
    while t < t_end - 1e-12:
        dt = min(cfl * h / oracle.max_wavespeed(cfg, W), t_end - t)
        assert oracle.step(cfg, dt, W, G) == 0
        t += dt
    return W, I.sine_exact_rho(dim, n, t_end)


def test_teno_is_linear_on_resolved_smooth_data_1d(oracle):
    Wt, _ = _run(oracle, 1, 16, 3, 2.0)
    Wl, _ = _run(oracle, 1, 16, 1, 2.0)
    assert np.abs(Wt - Wl).max() <= 1e-12
    # WENO-Z's weights move away from the linear ones (tau_Z > 0)
    Wz, _ = _run(oracle, 1, 16, 2, 2.0)
    assert np.abs(Wz - Wl).max() > 1e-12


def test_smooth_extrema_ordering_multid(oracle):
    """Sec. 5.2, smooth extrema: GENO keeps the linear reconstruction, WENO-Z
    deviates a little, TENO switches to the low-order candidates once the
    indicator ratio passes its cut.  On the advected diagonal wave (24^2
    cells) the errors are ordered GENO < WENO-Z < TENO, and GENO equals the
    linear scheme."""
    err = {}
    for lim in (0, 1, 2, 3):
        W, ex = _run(oracle, 2, 24, lim, 0.1)
        err[lim] = np.abs(W[0] - ex).mean()
    assert err[0] == pytest.approx(err[1], rel=1e-9)
    assert err[0] < err[2] < err[3], err


def test_geno_is_best_on_the_coarsest_mesh(oracle):
    """Sec. 6.1: advected density wave rho = 1 + 0.2 sin(pi x) on [0, 2] with
    4 cells (the compact scheme's coarsest mesh), t = 20: the GENO result is
    the most accurate of GENO, WENO-Z and TENO."""
    err = {}
    for lim in (0, 2, 3):
        W, ex = _run(oracle, 1, 4, lim, 20.0)
        err[lim] = np.abs(W[0] - ex).mean()
    assert err[0] < err[2] and err[0] < err[3], err
