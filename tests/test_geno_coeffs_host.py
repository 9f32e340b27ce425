"""The generated reconstruction code of the product path (csrc/geno_coeffs.cuh,
written by csrc/gen_coeffs.py), compiled for the CPU, against what the
mathematics fixes (no GPU, no oracle):

* the least-squares cubic (Sec. 4.3 on Cartesian cells) reproduces any cubic
  exactly from its neighbours' averages and averaged gradients (the cubic
  lies in the fitted space, so the least-squares residual is zero);
* the face Gauss-point evaluations give the cubic's value minus the cell
  average and its gradient at the points (face at +-1/2, tangential
  coordinates -+1/(2 sqrt 3));
* the indicators are the integrals of the squared derivatives of order 1..3
  (IS^H) and of order 3 (IS^tau) over the cell, each multi-index once;
* p^7 of the compact 1D stencil reproduces every polynomial of degree 7 at
  the face x_{j+1/2} (Sec. 4.2).
All in cell units; the reconstruction cell is [-1/2, 1/2]^m."""
import itertools
import math
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
    out = str(tmp_path_factory.mktemp("gc") / "geno_coeffs_check")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-I", CSRC, os.path.join(HERE, "geno_coeffs_check.cpp"), "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _run(exe, args, cases):
    text = f"{len(cases)}\n" + "\n".join(" ".join(repr(float(x)) for x in c) for c in cases) + "\n"
    r = subprocess.run([exe, *args], input=text, capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    return np.array([[float(x) for x in ln.split()] for ln in r.stdout.strip().splitlines()])


def _monomials(m):
    """The coefficient order the header states, as exponent tuples."""
    text = open(os.path.join(CSRC, "geno_coeffs.cuh")).read()
    lines = re.findall(r"Monomials \(coefficient order\): ([^*]*)\*/", text)
    exps = [tuple(int(p) for p in re.findall(r"\^(\d)", t)) for t in lines[m - 2].split(",")]
    return [e[:m] for e in exps]


def _avg1(p, o):
    return ((o + 0.5) ** (p + 1) - (o - 0.5) ** (p + 1)) / (p + 1)


def _avg(e, off):
    return math.prod(_avg1(p, o) for p, o in zip(e, off))


def _davg(e, a, off):
    """average of d/dx_a of the monomial e over the cell at off"""
    if e[a] == 0:
        return 0.0
    f = list(e)
    f[a] -= 1
    return e[a] * _avg(tuple(f), off)


def _value(e, x):
    return math.prod(xi ** p for xi, p in zip(x, e))


def _dvalue(e, a, x):
    if e[a] == 0:
        return 0.0
    f = list(e)
    f[a] -= 1
    return e[a] * _value(tuple(f), x)


def _data(m, mons, c):
    zero = (0,) * m
    d = np.zeros(2 * m * (1 + m) + m)
    for e in range(m):
        for side in (-1, 1):
            q = 2 * e + (side > 0)
            off = tuple(side if a == e else 0 for a in range(m))
            d[q * (1 + m)] = sum(ck * (_avg(mk, off) - _avg(mk, zero)) for ck, mk in zip(c, mons))
            for a in range(m):
                d[q * (1 + m) + 1 + a] = sum(ck * _davg(mk, a, off) for ck, mk in zip(c, mons))
    for a in range(m):
        d[2 * m * (1 + m) + a] = sum(ck * _davg(mk, a, zero) for ck, mk in zip(c, mons))
    return d


@pytest.mark.parametrize("m", [2, 3])
def test_fit_reproduces_cubics(exe, m):
    mons = _monomials(m)
    assert len(mons) == (9 if m == 2 else 18) and len(set(mons)) == len(mons)
    assert all(1 <= sum(e) <= 3 for e in mons)
    rng = np.random.default_rng(10 + m)
    cs = [rng.normal(size=len(mons)) for _ in range(20)]
    got = _run(exe, ["fit", str(m)], [_data(m, mons, c) for c in cs])
    for c, g in zip(cs, got):
        np.testing.assert_allclose(g, c, rtol=0, atol=1e-12 * np.abs(c).max())


@pytest.mark.parametrize("m", [2, 3])
def test_gauss_point_evaluation(exe, m):
    mons = _monomials(m)
    ng = 2 if m == 2 else 4
    g0 = math.sqrt(3.0) / 6.0
    zero = (0,) * m
    rng = np.random.default_rng(20 + m)
    cs = [rng.normal(size=len(mons)) for _ in range(6)]
    for d in range(m):
        tang = [a for a in range(m) if a != d]
        for s in (0, 1):
            for g in range(ng):
                x = [0.0] * m
                x[d] = 0.5 if s else -0.5
                for ti, a in enumerate(tang):
                    x[a] = g0 if (g >> ti) & 1 else -g0
                got = _run(exe, ["eval", str(m), str(d), str(s), str(g)], cs)
                for c, o in zip(cs, got):
                    val = sum(ck * (_value(mk, x) - _avg(mk, zero)) for ck, mk in zip(c, mons))
                    grad = [sum(ck * _dvalue(mk, a, x) for ck, mk in zip(c, mons)) for a in range(m)]
                    np.testing.assert_allclose(o, [val, *grad], rtol=0, atol=1e-12 * np.abs(c).max())


def _poly_mul(p, q):
    r = {}
    for e1, c1 in p.items():
        for e2, c2 in q.items():
            e = tuple(a + b for a, b in zip(e1, e2))
            r[e] = r.get(e, 0.0) + c1 * c2
    return r


def _poly_deriv(p, l):
    r = {}
    for e, c in p.items():
        f = list(e)
        k = c
        for a, la in enumerate(l):
            for _ in range(la):
                if f[a] == 0:
                    k = 0.0
                    break
                k *= f[a]
                f[a] -= 1
        if k:
            r[tuple(f)] = r.get(tuple(f), 0.0) + k
    return r


def _cell_integral(p):
    """integral over [-1/2, 1/2]^m"""
    return sum(c * math.prod(0.0 if k % 2 else 2 * 0.5 ** (k + 1) / (k + 1) for k in e) for e, c in p.items())


@pytest.mark.parametrize("m", [2, 3])
def test_indicators_are_derivative_integrals(exe, m):
    mons = _monomials(m)
    rng = np.random.default_rng(30 + m)
    cs = [rng.normal(size=len(mons)) for _ in range(10)]
    got = _run(exe, ["ind", str(m)], cs)
    for c, (ish, ist) in zip(cs, got):
        P = {mk: ck for ck, mk in zip(c, mons)}  # the constant part has no derivatives
        h = t = 0.0
        for l in itertools.product(range(4), repeat=m):
            if 1 <= sum(l) <= 3:
                dp = _poly_deriv(P, l)
                v = _cell_integral(_poly_mul(dp, dp))
                h += v
                if sum(l) == 3:
                    t += v
        assert abs(ish - h) <= 1e-12 * max(1.0, h), (ish, h)
        assert abs(ist - t) <= 1e-12 * max(1.0, t), (ist, t)


def test_p7_reproduces_degree_7(exe):
    rng = np.random.default_rng(40)
    cases, want = [], []
    for _ in range(20):
        a = rng.normal(size=8)
        P = np.polynomial.Polynomial(a)
        dP = P.deriv()
        iP, idP = P.integ(), dP.integ()
        w = [iP(q + 0.5) - iP(q - 0.5) for q in (-1, 0, 1, 2)]
        d = [idP(q + 0.5) - idP(q - 0.5) for q in (-1, 0, 1, 2)]
        cases.append(w + d)
        want.append((P(0.5), dP(0.5)))
    got = _run(exe, ["p7"], cases)
    for (v, dv), (gv, gd) in zip(want, got):
        scale = 1.0 + abs(v) + abs(dv)
        assert abs(gv - v) <= 1e-12 * scale and abs(gd - dv) <= 1e-12 * scale
