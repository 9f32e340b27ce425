"""The library's gas-kinetic interface flux (csrc/gks_device.cuh, gks_point),
compiled for the CPU through the test-only stand-in of tests/hostshim,
against the oracle's flux at single interface points in the face frame:

* FP64: the Euler flux (physical collision time 0) and the Navier-Stokes
  flux (tau = mu / p0) in 1D, 2D and 3D, to the same bars as the GPU flux
  parity test (1e-12 of the scale for F and W(dt/2), 1e-10 of
  |dF/dt| + |F| / dt for dF/dt);
* FP32: the same formulas with the two initial Maxwellians evaluated on
  left/right lane pairs (the packed two-lane path of the Euler flux) and
  the scalar path of the Navier-Stokes flux, to FP32 accuracy.  A lane mix-up
  (a side's state, slope or half-space sign in the other lane) would move the
  flux by O(1).
The states are random admissible face states with random slopes on both
sides along every axis, unequal left and right."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2507_20461_gb300", "csrc")
GAMMA, C1, C2 = 1.4, 0.05, 1.0

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("gp") / "gks_point_check")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-I", os.path.join(HERE, "hostshim"), "-I", CSRC,
                        os.path.join(HERE, "gks_point_check.cpp"), "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _state(rng, m):
    rho = rng.uniform(0.5, 2.0)
    u = rng.uniform(-0.5, 0.5, size=m)
    p = rng.uniform(0.5, 2.0)
    return np.array([rho, *(rho * u), p / (GAMMA - 1) + 0.5 * rho * (u @ u)])


def _cases(m, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        Wl, Wr = _state(rng, m), _state(rng, m)
        dWl = rng.normal(scale=0.2, size=(m, m + 2))
        dWr = rng.normal(scale=0.2, size=(m, m + 2))
        dt = rng.uniform(0.002, 0.02)
        out.append((Wl, Wr, dWl, dWr, dt))
    return out


def _host(exe, m, ns, prec, mu, cases):
    lines = [str(len(cases))]
    for Wl, Wr, dWl, dWr, dt in cases:
        vals = [m, ns, prec, GAMMA, C1, C2, mu, dt, *Wl, *Wr, *dWl.ravel(), *dWr.ravel()]
        lines.append(" ".join(repr(float(v)) if i > 2 else str(int(v)) for i, v in enumerate(vals)))
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    res = []
    for ln in r.stdout.strip().splitlines():
        v = [float(x) for x in ln.split()]
        nv = m + 2
        res.append((int(v[0]), np.array(v[1:1 + nv]), np.array(v[1 + nv:1 + 2 * nv]), np.array(v[1 + 2 * nv:])))
    return res


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("ns", [0, 1])
def test_fp64_flux_matches_oracle(exe, oracle, m, ns):
    mu = 0.01 if ns else 0.0
    cases = _cases(m, 25, 100 * m + ns)
    got = _host(exe, m, ns, 0, mu, cases)
    for (Wl, Wr, dWl, dWr, dt), (ok, F, Ft, Wh) in zip(cases, got):
        assert ok == 1
        Fo, Fto, Who = oracle.gks_point(m, GAMMA, dt, Wl, Wr, dWl, dWr, c1=C1, c2=C2, tau_mode=2 if ns else 0, mu=mu)
        s = np.abs(Fo).max()
        np.testing.assert_allclose(F, Fo, rtol=0, atol=1e-12 * s)
        np.testing.assert_allclose(Ft, Fto, rtol=0, atol=1e-10 * (np.abs(Fto).max() + s / dt))
        np.testing.assert_allclose(Wh, Who, rtol=0, atol=1e-12 * np.abs(Who).max())


@pytest.mark.parametrize("m", [1, 2, 3])
@pytest.mark.parametrize("ns", [0, 1])
def test_fp32_flux_matches_oracle(exe, oracle, m, ns):
    """FP32 rounding of the inputs alone moves the flux by about 1e-7 of
    its scale; the bars leave two orders of magnitude for the arithmetic."""
    mu = 0.01 if ns else 0.0
    cases = _cases(m, 25, 200 * m + ns)
    got = _host(exe, m, ns, 1, mu, cases)
    worst = 0.0
    for (Wl, Wr, dWl, dWr, dt), (ok, F, Ft, Wh) in zip(cases, got):
        assert ok == 1
        Fo, Fto, Who = oracle.gks_point(m, GAMMA, dt, Wl, Wr, dWl, dWr, c1=C1, c2=C2, tau_mode=2 if ns else 0, mu=mu)
        s = np.abs(Fo).max()
        worst = max(worst, np.abs(F - Fo).max() / s)
        np.testing.assert_allclose(F, Fo, rtol=0, atol=2e-5 * s)
        np.testing.assert_allclose(Ft, Fto, rtol=0, atol=2e-4 * (np.abs(Fto).max() + s / dt))
        np.testing.assert_allclose(Wh, Who, rtol=0, atol=2e-5 * np.abs(Who).max())
    assert worst > 0.0  # the FP32 path really ran in FP32


def test_inadmissible_side_is_reported(exe):
    """A side with negative pressure: the flux reports it (both precisions)."""
    m = 2
    (Wl, Wr, dWl, dWr, dt), = _cases(m, 1, 7)
    Wr = Wr.copy()
    Wr[-1] = 0.1 * Wr[-1] - 10.0
    for prec in (0, 1):
        (ok, *_), = _host(exe, m, 0, prec, 0.0, [(Wl, Wr, dWl, dWr, dt)])
        assert ok == 0
