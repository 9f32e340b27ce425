"""The reconstruction's nonlinear-weight device code (GENO path function,
WENO-Z and TENO weights) against the closed-form linearity analysis of
Sec. 3.1 and Sec. 5.2 (oracle/geno_analysis.py), through geno_linearity on
cuda:0, in FP64 and FP32."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import geno_analysis as A
from paper_2507_20461_gb300 import binding as B

pytestmark = pytest.mark.gpu
DEV = "cuda:0"

PHI_STAR = ((1 - 1e-6) / 2e-6) ** (1 / 7)  # TENO's switch for one large of three indicators


def _phis():
    phi = np.logspace(0.0, 8.0, 321)
    # keep clear of TENO's switch, where rounding decides the cut
    return phi[np.abs(phi / PHI_STAR - 1) > 1e-3]


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("scenario", ["min", "max"])
@pytest.mark.parametrize("limiter", [0, 2, 3])
def test_linearity_curves(limiter, scenario, precision):
    phi = _phis()
    IS = np.stack([A.scenario_indicators(p, scenario)[0] for p in phi])
    tau = np.array([A.scenario_indicators(p, scenario)[1] for p in phi])
    if limiter == 0:
        want = np.array([A.geno_linearity(p, scenario) for p in phi])
    else:
        want = np.array([A.weights_linearity(limiter, p, scenario) for p in phi])
    ISd = torch.from_numpy(np.ascontiguousarray(IS)).to(DEV)
    taud = torch.from_numpy(tau).to(DEV)
    chi = torch.zeros(len(phi), dtype=torch.float64, device=DEV)
    B.geno_linearity(ISd, taud, chi, limiter, r=2, precision=precision)
    got = chi.cpu().numpy()
    tol = 1e-12 if precision == 0 else 2e-6
    np.testing.assert_allclose(got, want, rtol=0, atol=tol)


def test_unstructured_exponent_and_bad_arguments():
    """r = 3 (unstructured meshes) on GENO's indicators, and argument checks."""
    rng = np.random.default_rng(4)
    IS = rng.uniform(1e-4, 10.0, size=(64, 4))
    tau = rng.uniform(0.0, 5.0, size=64)
    want = A.path_function(A.ultimate_indicator(tau, IS.max(axis=1), IS.min(axis=1), 3))
    ISd = torch.from_numpy(IS).to(DEV)
    taud = torch.from_numpy(tau).to(DEV)
    chi = torch.zeros(64, dtype=torch.float64, device=DEV)
    B.geno_linearity(ISd, taud, chi, 0, r=3)
    np.testing.assert_allclose(chi.cpu().numpy(), want, rtol=0, atol=1e-12)
    with pytest.raises(B.GksError):
        B.geno_linearity(ISd, taud, chi, 0, r=4)
