"""Pins of the closed-form linearity analysis (oracle/geno_analysis.py, no GPU).

The paper states what the curves of Sec. 3.1 and Sec. 5.2 show; these
properties, and limits worked out by hand from the weight definitions, fix
the module:
* the path function runs from chi(0) = 0 to chi(1) = 1 and keeps chi within
  1e-10 of one for alpha above 0.6 (the "linearity preserving" plateau);
* smooth extrema (tau ~ IS^min): GENO keeps the linear reconstruction for
  every phi; WENO-Z leaves it at once and tends to 3/5; TENO switches from 1
  to 0 at the phi where the scale-separation indicator reaches C_T;
* discontinuities (tau ~ IS^max): all three tend to 0 as phi grows; for
  small phi (fine meshes) GENO and TENO keep the linear reconstruction.
"""
import math

import numpy as np
import pytest

from oracle import geno_analysis as A


def test_path_function_endpoints_and_plateau():
    a = np.linspace(0.0, 1.0, 1001)
    chi = A.path_function(a)
    assert chi[0] == 0.0 and chi[-1] == 1.0
    assert np.all(np.diff(chi) >= 0)
    assert np.all(1.0 - chi[a >= 0.6] <= 1e-10)
    # steep start: chi(0.05) = tanh(1) / tanh(20)
    assert A.path_function(0.05) == pytest.approx(math.tanh(1.0))


def test_ultimate_indicator_bounds():
    rng = np.random.default_rng(2)
    for _ in range(200):
        ISL, ISH = sorted(rng.uniform(1e-6, 10.0, size=2))
        tau = rng.uniform(0.0, 20.0)
        a = A.ultimate_indicator(tau, ISH, ISL, 2)
        assert 0.0 < a <= 1.0 + 1e-15


@pytest.mark.parametrize("phi", [1.0, 10.0, 1e3, 1e6, 1e12])
def test_smooth_extrema_scenario(phi):
    # GENO: alpha = 2 (1 + phi^-2) / (3 + phi^-2) >= 2/3, so chi >= tanh(40/3) / tanh(20)
    g = A.geno_linearity(phi, "min")
    assert g >= math.tanh(40.0 / 3.0) / math.tanh(20.0) - 1e-15
    # WENO-Z: chi = 3 (1 + 1/phi) / ((1 + 1/phi) + 4), below 1 as soon as phi > 1
    wz = A.weights_linearity(2, phi, "min")
    assert wz == pytest.approx(3 * (1 + 1 / phi) / ((1 + 1 / phi) + 4), rel=1e-12)


def test_wenoz_limit_and_teno_switch():
    assert A.weights_linearity(2, 1e15, "min") == pytest.approx(0.6, rel=1e-9)
    # TENO: gamma_max = phi^-7 / (phi^-7 + 2) <= 1e-6 from phi* = ((1 - 1e-6) / 2e-6)^(1/7)
    phi_star = ((1 - 1e-6) / 2e-6) ** (1 / 7)
    assert A.weights_linearity(3, phi_star * 0.999, "min") == 1.0
    assert A.weights_linearity(3, phi_star * 1.001, "min") == 0.0
    # TENO's cut ignores tau: the same switch in both scenarios
    assert A.weights_linearity(3, phi_star * 1.001, "max") == 0.0


def test_discontinuity_scenario():
    # large phi: every method leaves the linear reconstruction
    for lim in (2, 3):
        assert A.weights_linearity(lim, 1e8, "max") < 1e-7
    assert A.geno_linearity(1e8, "max") < 1e-6
    # GENO: alpha = 4 / (3 + phi^2); small phi keeps chi at 1
    assert A.geno_linearity(1.0, "max") == 1.0
    assert A.geno_linearity(1.2, "max") == pytest.approx(
        math.tanh(20 * 4 / (3 + 1.44)) / math.tanh(20), rel=1e-14)
    # WENO-Z: chi = 6 / (2 + 2 (1 + phi)) -> about 3 / phi
    assert A.weights_linearity(2, 1e4, "max") == pytest.approx(6 / (2 + 2 * (1 + 1e4)), rel=1e-12)
