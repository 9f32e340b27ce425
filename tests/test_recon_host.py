"""The library's per-cell GENO blend (csrc/kernels.cuh, blend_cubic: the
least-squares cubic, its indicators, the 2m linear sub-polynomials, the path
function and the blend; WENO-Z / TENO in the adaptive-order combination),
compiled for the CPU through the test-only CUDA stand-in of tests/hostshim,
against the oracle's per-cell reconstruction (or_genomd_cell) on random
crosses in 2D and 3D, for the linear scheme, GENO, WENO-Z and TENO:
FP64 to 1e-12 of the coefficients' scale, FP32 to FP32 accuracy.  The
states mix smooth crosses (chi near 1) with jumps (chi well below 1), so the
path function and the sub-polynomial weights both act."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2507_20461_gb300", "csrc")

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("rc") / "recon_check")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-I", os.path.join(HERE, "hostshim"), "-I", CSRC,
                        os.path.join(HERE, "recon_check.cpp"), "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _product_monomials(m):
    text = open(os.path.join(CSRC, "geno_coeffs.cuh")).read()
    lines = re.findall(r"Monomials \(coefficient order\): ([^*]*)\*/", text)
    return [tuple(int(p) for p in re.findall(r"\^(\d)", t)) for t in lines[m - 2].split(",")]


def _cross(rng, m, jump):
    """own average, own gradient, the 2m neighbours' averages and gradients
    (cell units): a smooth field, plus a jump across one face if asked"""
    W0 = rng.uniform(0.5, 2.0)
    g = rng.normal(scale=0.2, size=m)
    Wn, Dn = [], []
    for e in range(m):
        for s in (-1, 1):
            w = W0 + s * g[e] + rng.normal(scale=0.02)
            if jump and e == 0 and s == 1:
                w += jump
            Wn.append(w)
            Dn.append(g + rng.normal(scale=0.05, size=m))
    return W0, g + rng.normal(scale=0.05, size=m), Wn, Dn


def _host(exe, m, lim, prec, crosses):
    lines = [str(len(crosses))]
    for W0, D0, Wn, Dn in crosses:
        d = []
        for q in range(2 * m):
            d += [Wn[q] - W0, *Dn[q]]
        d += list(D0)
        lines.append(" ".join(repr(float(x)) for x in d))
    r = subprocess.run([exe, str(m), str(lim), str(prec)], input="\n".join(lines) + "\n", capture_output=True,
                       text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    return np.array([[float(x) for x in ln.split()] for ln in r.stdout.strip().splitlines()])


@pytest.mark.parametrize("m", [2, 3])
@pytest.mark.parametrize("lim", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_blend_matches_oracle(exe, oracle, m, lim, prec):
    rng = np.random.default_rng(1000 * m + 10 * lim + prec)
    crosses = [_cross(rng, m, jump) for jump in [0.0] * 10 + list(rng.uniform(0.2, 1.5, size=10))]
    got = _host(exe, m, lim, prec, crosses)
    cfg = oracle.make_cfg(m, (4,) * m, 1.0, limiter=lim)
    oexp = [tuple(int(x) for x in e[:m]) for e in oracle.monomials(m, 3)]
    pexp = [e[:m] for e in _product_monomials(m)]
    chis = []
    for (W0, D0, Wn, Dn), b in zip(crosses, got):
        o = oracle.genomd_cell(cfg, W0, D0, Wn, Dn)
        chis.append(o["chi"])
        ref = dict(zip(oexp, o["coef"]))
        want = np.array([ref[e] for e in pexp])
        # the oracle states the polynomial in raw monomials, constant
        # included, the kernel as P - W0 = sum_k c_k (mono_k - <mono_k>): the
        # same c_k, and the oracle's constant is W0 - sum_k c_k <mono_k>
        assert sorted(set(oexp) - set(pexp)) == [(0,) * m]
        avg0 = np.array([np.prod([0.0 if p % 2 else 0.5**p / (p + 1) for p in e]) for e in pexp])
        assert abs(ref[(0,) * m] - (W0 - want @ avg0)) <= 1e-12 * abs(W0)
        scale = np.abs(want).max()
        tol = 1e-12 if prec == 0 else 2e-5
        np.testing.assert_allclose(b, want, rtol=0, atol=tol * scale)
    if lim == 0:
        assert min(chis) < 0.5 < max(chis)  # both regimes of the path function were exercised
