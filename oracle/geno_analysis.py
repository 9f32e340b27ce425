"""Closed-form analysis of the nonlinear reconstructions (test infrastructure).

Plain restatements, in FP64 numpy, of the paper's analysis of how much of
the high-order linear reconstruction each nonlinear method keeps:

* the GENO path function chi(alpha) = tanh(C alpha) / tanh(C)
  (Sec. 3.1, Eq. HLP-weight; Fig. HLP-path-function);
* the ultimate smoothness indicator alpha (Sec. 3.2, Eq. HLP-sp);
* the linearity parameter of WENO-Z and TENO, chi = min_k w_k / d_k
  (Sec. 5.2, Eq. linearity-paprameter), with the WENO-Z weights
  (Eq. wgt-WENO-Z) and the TENO weights (Eq. wgt-TENO-1, Eq. wgt-TENO-2);
* the two scenarios of Sec. 5.2: IS^max = phi IS^min with tau ~ IS^max or
  tau ~ IS^min, three sub-stencils with d_k = 1/3.

Reading for the scenarios (the paper gives the figures, not the indicator
sets): one candidate sits at IS^max and the others at IS^min = 1; GENO takes
IS^H = IS^max and IS^L = IS^min with r = 2 (structured meshes); eps is
negligible next to the indicators.

Only tests may import this module.
"""
from __future__ import annotations

import numpy as np


def path_function(alpha, C=20.0):
    """chi(alpha), Eq. HLP-weight."""
    alpha = np.asarray(alpha, dtype=np.float64)
    return np.tanh(C * alpha) / np.tanh(C)


def ultimate_indicator(IS_tau, IS_H, IS_L, r, eps=1e-15):
    """alpha = 2 alpha^H / (alpha^H + alpha^L), Eq. HLP-sp."""
    aH = 1.0 + (IS_tau / (IS_H + eps)) ** r
    aL = 1.0 + (IS_tau / (IS_L + eps)) ** r
    return 2.0 * aH / (aH + aL)


def scenario_indicators(phi, scenario, k0=3, n_max=1):
    """Indicator set of the Sec. 5.2 scenarios: n_max candidates at
    IS^max = phi, the others at IS^min = 1; tau = IS^max (scenario 'max',
    discontinuity) or IS^min (scenario 'min', smooth extremum).
    Returns (IS[k0], tau)."""
    IS = np.ones(k0)
    IS[:n_max] = phi
    tau = phi if scenario == "max" else 1.0
    return IS, tau


def geno_linearity(phi, scenario, r=2, C=20.0, eps=1e-15, k0=3, n_max=1):
    """chi of GENO for one phi: IS^H = max IS_k, IS^L = min IS_k (Eq. IS-highorder-2,
    Eq. HLP-IS-loworder-2), IS^tau = tau."""
    IS, tau = scenario_indicators(phi, scenario, k0, n_max)
    return float(path_function(ultimate_indicator(tau, IS.max(), IS.min(), r, eps), C))


def wenoz_weights(IS, tau, d, eps=1e-15):
    """Eq. wgt-WENO-Z."""
    wt = d * (1.0 + tau / (IS + eps))
    return wt / wt.sum()


def teno_weights(IS, d, ct=1e-6, eps=1e-15, q=7):
    """Eq. wgt-TENO-1 (exponent q = 7) and Eq. wgt-TENO-2 (cut-off ct)."""
    g = (1.0 / (IS + eps)) ** q
    gamma = g / g.sum()
    keep = (gamma > ct).astype(np.float64)
    wt = keep * d
    return wt / wt.sum()


def weights_linearity(limiter, phi, scenario, ct=1e-6, eps=1e-15, k0=3, n_max=1):
    """min_k w_k / d_k (Eq. linearity-paprameter) for WENO-Z (limiter 2) or
    TENO (limiter 3) with d_k = 1 / k0."""
    IS, tau = scenario_indicators(phi, scenario, k0, n_max)
    d = np.full(k0, 1.0 / k0)
    w = wenoz_weights(IS, tau, d, eps) if limiter == 2 else teno_weights(IS, d, ct, eps)
    return float((w / d).min())
