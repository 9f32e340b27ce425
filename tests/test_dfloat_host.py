"""The double-float arithmetic of the mixed-precision update (csrc/kernels.cuh),
compiled for the CPU through the test-only CUDA stand-in of tests/hostshim,
checked exactly with rationals:

* TwoSum (Knuth) and FastTwoSum (Dekker): s + e equals a + b exactly;
* the face-sum accumulation (two_sum_acc): s + e equals the exact sum of the
  face values up to the rounding of the error term alone;
* the double-float product and sum carry about 48 bits;
* the stage constants of the two-stage fourth-order update (make_updc) are
  the scheme's coefficients (stage 1: -dt/2, -dt^2/8, and for the carried
  accumulator -dt, -dt^2/6; stage 2: -dt^2/3, each times 1/(h NG)), split
  into two floats whose sum holds them to 2^-48."""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2507_20461_gb300", "csrc")

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("df") / "dfloat_check")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(HERE, "hostshim"),
                        "-I", CSRC, os.path.join(HERE, "dfloat_check.cpp"), "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _run(exe, args, text=""):
    r = subprocess.run([exe, *args], input=text, capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    return [[Fraction(float.fromhex(t)) for t in ln.split()] for ln in r.stdout.strip().splitlines()]


def _f32(x):
    return np.float32(x).item()


def _floats(rng, n):
    """floats over many binades, both signs"""
    return [_f32(rng.choice([-1, 1]) * 10.0 ** rng.uniform(-6, 6) * rng.uniform(1, 2)) for _ in range(n)]


def test_two_sum_is_exact(exe):
    rng = np.random.default_rng(1)
    a, b = _floats(rng, 2000), _floats(rng, 2000)
    rows = _run(exe, ["twosum"], f"{len(a)}\n" + "\n".join(f"{x!r} {y!r}" for x, y in zip(a, b)) + "\n")
    for x, y, (s, e, fs, fe) in zip(a, b, rows):
        exact = Fraction(x) + Fraction(y)
        assert s + e == exact
        assert fs + fe == exact
        assert s == Fraction(_f32(x + y)) or abs(e) <= abs(s) * Fraction(1, 2**23)


def test_face_sum_accumulation(exe):
    """2m (+/-) face values of mixed size, as the update sums them: the
    error of s + e is the rounding of e alone, far below 2^-40 of the
    values' magnitude"""
    rng = np.random.default_rng(2)
    n, length = 500, 12
    seqs = [[_f32(v) for v in rng.normal(size=length) * 10.0 ** rng.uniform(-3, 3, size=length)] for _ in range(n)]
    text = f"{n} {length}\n" + "\n".join(" ".join(repr(x) for x in s) for s in seqs) + "\n"
    rows = _run(exe, ["acc"], text)
    for s_in, (s, e) in zip(seqs, rows):
        exact = sum(Fraction(x) for x in s_in)
        mag = sum(abs(Fraction(x)) for x in s_in)
        assert abs(s + e - exact) <= mag * Fraction(1, 2**40)


def test_double_float_product_and_sum(exe):
    rng = np.random.default_rng(3)
    cases = []
    for _ in range(2000):
        k, x = rng.uniform(0.5, 2.0) * 10.0 ** rng.uniform(-4, 4), rng.uniform(0.5, 2.0) * 10.0 ** rng.uniform(-4, 4)
        kh, xh = _f32(k), _f32(x)
        cases.append((kh, _f32(k - kh), xh, _f32(x - xh)))
    rows = _run(exe, ["mul"], f"{len(cases)}\n" + "\n".join(" ".join(repr(v) for v in c) for c in cases) + "\n")
    for (kh, kl, xh, xl), (ph, pl, sh, sl) in zip(cases, rows):
        K, X = Fraction(kh) + Fraction(kl), Fraction(xh) + Fraction(xl)
        assert abs(ph + pl - K * X) <= abs(K * X) * Fraction(1, 2**44)
        assert abs(sh + sl - (K + X)) <= abs(K + X) * Fraction(1, 2**44)


@pytest.mark.parametrize("dt,cw", [(0.01, 512.0), (1.3e-4, 1024.0 / 4), (0.25, 0.5)])
def test_stage_constants(exe, dt, cw):
    rows = _run(exe, ["updc", repr(dt), repr(cw)])
    want = [-dt / 2 * cw, -dt * dt / 8 * cw, -dt * cw, -dt * dt / 6 * cw, -dt * dt / 3 * cw]
    for (hi, lo), w in zip(rows, want):
        assert abs(float(hi + lo) - w) <= abs(w) * 2.0**-47
        assert abs(lo) <= abs(hi) * 2.0**-23
    # the two stages combine to the fourth-order step: dt L(F) + dt^2/6 (L(Ft) + 2 L(Ft*)), L = -cw S
    k2, k3, k4 = (float(h + l) for h, l in rows[2:])
    assert abs(k4 - 2 * k3) <= abs(k4) * 2.0**-45 and abs(k2 + dt * cw) <= abs(k2) * 2.0**-45
