"""Pins of the oracle's GENO reconstruction against what the paper and the
mathematics fix (no GPU).

P1  exactness: the 1D p^7 of the compact stencil (Sec. 4.2) reproduces every
    polynomial of degree <= 7; the three sub-stencil quadratics reproduce
    degree <= 2; the multi-D compact cubic (Sec. 4.3, Cartesian reading)
    reproduces every cubic of its space; linear sub-polynomials reproduce
    linear data.
P2  closed forms of the smoothness indicators: IS_k of a quadratic is
    a1^2 + 13/3 a2^2 (Eq. IS-highorder-1 with |l| <= 2 in cell units);
    multi-D IS^H / IS^tau are integrals of squared derivatives of the cubic
    (Eq. IS-highorder-1, Eq. IS-highorder-2, Eq. IS-tau), checked here by
    Gauss-Legendre quadrature; IS_k of a linear sub-polynomial is |g_k|^2
    with g_k in closed form.
P3  the path function: chi = 1 whenever IS^tau = 0 (Eq. HLP-sp, HLP-weight),
    chi -> 0 at a jump with the ENO sub-polynomial selected (Sec. 3.3).
"""
import itertools
import math

import numpy as np
import pytest
from numpy.polynomial import polynomial as P

GL_X, GL_W = np.polynomial.legendre.leggauss(12)
GL_X = GL_X / 2.0
GL_W = GL_W / 2.0  # nodes/weights on [-1/2, 1/2]


def _avg1d(coef, c):
    """Exact average over [c - 1/2, c + 1/2] of the 1D polynomial with coefficients coef."""
    I = P.polyint(coef)
    return P.polyval(c + 0.5, I) - P.polyval(c - 0.5, I)


@pytest.mark.parametrize("side", [0, 1])
@pytest.mark.parametrize("deg", [0, 1, 3, 5, 7])
def test_p7_exact_for_degree_le_7(oracle, side, deg):
    rng = np.random.default_rng(100 + deg + 10 * side)
    cfg = oracle.make_cfg(1, (8,), 0.1, limiter=1)  # chi = 1: R = p^7
    for _ in range(5):
        coef = rng.normal(size=deg + 1)
        dcoef = P.polyder(coef) if deg > 0 else np.zeros(1)
        w5 = [_avg1d(coef, q) for q in range(-2, 3)]
        d5 = [P.polyval(q + 0.5, coef) - P.polyval(q - 0.5, coef) for q in range(-2, 3)]
        x = 0.5 if side == 0 else -0.5
        o = oracle.geno1d_point(cfg, w5, d5, side)
        scale = 1.0 + np.abs(coef).sum()
        assert abs(o["val"] - P.polyval(x, coef)) <= 1e-13 * scale
        assert abs(o["der"] - P.polyval(x, dcoef)) <= 1e-12 * scale


def test_p8_not_exact_for_degree_8(oracle):
    """The fit is exactly eighth order: a degree-8 polynomial is not reproduced."""
    cfg = oracle.make_cfg(1, (8,), 0.1, limiter=1)
    coef = np.zeros(9)
    coef[8] = 1.0
    w5 = [_avg1d(coef, q) for q in range(-2, 3)]
    d5 = [P.polyval(q + 0.5, coef) - P.polyval(q - 0.5, coef) for q in range(-2, 3)]
    o = oracle.geno1d_point(cfg, w5, d5, 0)
    assert abs(o["val"] - 0.5**8) > 1e-6


@pytest.mark.parametrize("side", [0, 1])
def test_geno1d_quadratic_exact_and_indicators(oracle, side):
    """On quadratic data every candidate equals the quadratic, so R is exact for
    any weights; IS_k = a1^2 + 13/3 a2^2 (coefficients about the cell centre),
    IS^tau = 0 and therefore chi = 1."""
    rng = np.random.default_rng(7 + side)
    cfg = oracle.make_cfg(1, (8,), 0.1)
    for _ in range(10):
        coef = rng.normal(size=3)
        w5 = [_avg1d(coef, q) for q in range(-2, 3)]
        d5 = [P.polyval(q + 0.5, coef) - P.polyval(q - 0.5, coef) for q in range(-2, 3)]
        x = 0.5 if side == 0 else -0.5
        o = oracle.geno1d_point(cfg, w5, d5, side)
        assert abs(o["val"] - P.polyval(x, coef)) < 1e-13
        assert abs(o["der"] - P.polyval(x, P.polyder(coef))) < 1e-12
        js = coef[1] ** 2 + 13.0 / 3.0 * coef[2] ** 2
        for k in ("IS1", "IS2", "IS3"):
            assert abs(o[k] - js) <= 1e-13 * (1 + js)
        assert o["IStau"] <= 1e-13 * (1 + js)
        assert o["chi"] == pytest.approx(1.0, abs=1e-15)


def test_geno1d_jump_selects_eno(oracle):
    """A jump between the reconstruction cell and its right neighbour: chi -> 0
    and the left interface value stays at the smooth side (no overshoot)."""
    cfg = oracle.make_cfg(1, (8,), 0.1)
    w5 = [0.0, 0.0, 0.0, 1.0, 1.0]
    d5 = [0.0] * 5
    o = oracle.geno1d_point(cfg, w5, d5, 0)
    assert o["chi"] < 1e-3
    assert abs(o["val"]) < 1e-6
    # the mirrored right state at the same face sits on the other side of the jump
    w5r = [0.0, 0.0, 1.0, 1.0, 1.0]
    o = oracle.geno1d_point(cfg, w5r, d5, 1)
    assert o["chi"] < 1e-3
    assert abs(o["val"] - 1.0) < 1e-6


def test_geno1d_chi_in_unit_interval(oracle):
    cfg = oracle.make_cfg(1, (8,), 0.1)
    rng = np.random.default_rng(3)
    for _ in range(200):
        w5 = rng.normal(size=5) * rng.choice([1e-6, 1.0, 1e3])
        d5 = rng.normal(size=5)
        for side in (0, 1):
            o = oracle.geno1d_point(cfg, w5, d5, side)
            assert 0.0 <= o["chi"] <= 1.0 + 1e-15
            assert o["ISL"] <= o["ISH"]


# ---------------------------------------------------------------- multi-D
def _mono_space(oracle, m):
    return oracle.monomials(m, 3)


def _cell_avg_md(e, off, m, dax=-1):
    """Average over cell `off` of the monomial with exponents e (optionally
    differentiated along dax) by tensor Gauss-Legendre quadrature."""
    e = list(e)
    fac = 1.0
    if dax >= 0:
        if e[dax] == 0:
            return 0.0
        fac = e[dax]
        e[dax] -= 1
    for a in range(m):
        fac *= float(np.sum(GL_W * (GL_X + off[a]) ** e[a]))
    return fac


def _data_for_poly(oracle, m, coefs, E):
    """Cell averages and averaged gradients of sum_k coefs[k] mono_k on the cross."""

    def avg(off, dax=-1):
        return sum(c * _cell_avg_md(E[k], off, m, dax) for k, c in enumerate(coefs))

    zero = [0, 0, 0]
    W0 = avg(zero)
    D0 = [avg(zero, a) for a in range(m)]
    Wn, Dn = [], []
    for e in range(m):
        for s in (-1, 1):
            off = [0, 0, 0]
            off[e] = s
            Wn.append(avg(off))
            Dn.append([avg(off, a) for a in range(m)])
    return W0, D0, Wn, Dn


@pytest.mark.parametrize("m", [2, 3])
def test_cubic_lsq_exact(oracle, m):
    E = _mono_space(oracle, m)
    assert len(E) == (10 if m == 2 else 19)
    if m == 3:
        assert not any((e == [1, 1, 1]).all() for e in E)
    cfg = oracle.make_cfg(m, (8,) * m, 0.1, limiter=1)
    rng = np.random.default_rng(11 * m)
    for _ in range(5):
        coefs = rng.normal(size=len(E))
        W0, D0, Wn, Dn = _data_for_poly(oracle, m, coefs, E)
        o = oracle.genomd_cell(cfg, W0, D0, Wn, Dn)
        np.testing.assert_allclose(o["coef"], coefs, rtol=0, atol=1e-12)


def test_3d_trilinear_is_invisible():
    """xi eta zeta has zero average and zero averaged gradient on every cell of
    the seven-cell cross: the reason the 3D compact cubic omits it."""
    e = [1, 1, 1]
    offs = [[0, 0, 0]] + [[s if a == d else 0 for a in range(3)] for d in range(3) for s in (-1, 1)]
    for off in offs:
        assert abs(_cell_avg_md(e, off, 3)) < 1e-15
        for dax in range(3):
            assert abs(_cell_avg_md(e, off, 3, dax)) < 1e-15


@pytest.mark.parametrize("m", [2, 3])
def test_linear_data_reproduced_by_geno(oracle, m):
    """Linear data: every sub-polynomial and the cubic are exact, so R is exact
    for any chi; IS_k = |g|^2 for every sub-stencil."""
    E = _mono_space(oracle, m)
    cfg = oracle.make_cfg(m, (8,) * m, 0.1)
    rng = np.random.default_rng(5)
    for _ in range(5):
        coefs = np.zeros(len(E))
        coefs[: 1 + m] = rng.normal(size=1 + m)
        W0, D0, Wn, Dn = _data_for_poly(oracle, m, coefs, E)
        o = oracle.genomd_cell(cfg, W0, D0, Wn, Dn)
        np.testing.assert_allclose(o["coef"], coefs, atol=1e-13)
        g2 = float(np.sum(coefs[1 : 1 + m] ** 2))
        np.testing.assert_allclose(o["IS"], g2, rtol=1e-13)


def _deriv_sq_integral(m, E, coefs, l):
    """int over the unit cell of (D^l p)^2 by tensor Gauss-Legendre quadrature."""
    pts = np.array(list(itertools.product(GL_X, repeat=m)))
    wts = np.prod(np.array(list(itertools.product(GL_W, repeat=m))), axis=1)
    val = np.zeros(len(pts))
    for k, c in enumerate(coefs):
        e = list(E[k])
        f = c
        ok = True
        for a in range(m):
            for _ in range(l[a]):
                if e[a] == 0:
                    ok = False
                    break
                f *= e[a]
                e[a] -= 1
        if not ok:
            continue
        term = np.full(len(pts), f)
        for a in range(m):
            term = term * pts[:, a] ** e[a]
        val += term
    return float(np.sum(wts * val * val))


@pytest.mark.parametrize("m", [2, 3])
def test_multid_indicators_are_derivative_integrals(oracle, m):
    E = _mono_space(oracle, m)
    cfg = oracle.make_cfg(m, (8,) * m, 0.1)
    rng = np.random.default_rng(17 + m)
    for _ in range(3):
        coefs = rng.normal(size=len(E))
        W0, D0, Wn, Dn = _data_for_poly(oracle, m, coefs, E)
        o = oracle.genomd_cell(cfg, W0, D0, Wn, Dn)
        ISH = 0.0
        IStau = 0.0
        for l in itertools.product(range(4), repeat=m):
            s = sum(l)
            if 1 <= s <= 3:
                v = _deriv_sq_integral(m, E, coefs, l)
                ISH += v
                if s == 3:
                    IStau += v
        assert o["ISH"] == pytest.approx(ISH, rel=1e-12)
        assert o["IStau"] == pytest.approx(IStau, rel=1e-11, abs=1e-13)
        # IS^L: trimmed mean of the linear sub-stencil indicators (Eq. HLP-IS-loworder-3)
        IS = np.sort(o["IS"])
        assert o["ISL"] == pytest.approx(IS[1:-1].mean(), rel=1e-13)
        # linear sub-polynomials in closed form: g_d = (s dW + D_{n,d}) / 2, g_t = D_{n,t}
        for q in range(2 * m):
            d, s = q // 2, (1 if q % 2 else -1)
            g = np.array(Dn[q], dtype=float)
            g[d] = 0.5 * (s * (Wn[q] - W0) + Dn[q][d])
            assert o["IS"][q] == pytest.approx(float(g @ g), rel=1e-12)


@pytest.mark.parametrize("m", [2, 3])
def test_multid_quadratic_keeps_chi_one(oracle, m):
    """A quadratic has no third derivatives, so IS^tau = 0 and chi = 1."""
    E = _mono_space(oracle, m)
    cfg = oracle.make_cfg(m, (8,) * m, 0.1)
    rng = np.random.default_rng(23)
    deg = E.sum(axis=1)
    coefs = np.where(deg <= 2, rng.normal(size=len(E)), 0.0)
    W0, D0, Wn, Dn = _data_for_poly(oracle, m, coefs, E)
    o = oracle.genomd_cell(cfg, W0, D0, Wn, Dn)
    assert o["IStau"] < 1e-13
    assert o["chi"] == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(o["coef"], coefs, atol=1e-12)


@pytest.mark.parametrize("m", [2, 3])
def test_multid_jump_lowers_chi(oracle, m):
    """A jump across the +x face: chi -> 0 and R is dominated by the smooth
    linear sub-polynomials (no growth of the +x face value beyond the data)."""
    cfg = oracle.make_cfg(m, (8,) * m, 0.1)
    D0 = [0.0] * m
    Wn = [0.0] * (2 * m)
    Wn[1] = 1.0  # +x neighbour
    Dn = [[0.0] * m for _ in range(2 * m)]
    o = oracle.genomd_cell(cfg, 0.0, D0, Wn, Dn)
    assert o["chi"] < 0.05
    # value at the +x face centre stays between the two data values
    E = _mono_space(oracle, m)
    x = np.zeros(3)
    x[0] = 0.5
    val = sum(c * np.prod([x[a] ** E[k][a] for a in range(m)]) for k, c in enumerate(o["coef"]))
    assert -1e-3 < val < 0.5
