"""Pins of the oracle's 1D non-compact GENO schemes (Sec. 4.1) with the HLLC
flux and classical RK4 (no GPU).

What fixes them independently of the oracle's fits:
* the high-order polynomials reproduce every polynomial of degree < order
  (averages in, point value at the face out), GENO every quadratic;
* the 5th-order sub-stencil indicators equal Jiang and Shu's closed forms;
  the 6th-order cubic indicators equal the derivative integrals of the data's
  own cubic (numpy polynomial calculus);
* HLLC keeps a stationary contact exactly (an HLL flux would smear it) and
  reduces to the Euler flux for equal states;
* design order 5 and 6 on the advected density wave (Sec. 6.1), fourth order
  in time, conservation, mirror symmetry, convergence to exact Riemann
  solutions;
* the paper's comparison (Sec. 6.1): the compact 8th-order GKS on 4 cells is
  more accurate than the non-compact schemes on 6.
"""
import numpy as np
import pytest
from numpy.polynomial import polynomial as Pn

from oracle import riemann
from paper_2507_20461_gb300 import inputs as I

GAMMA = 1.4


def _avgs(coef, offsets):
    """cell averages of sum coef[k] xi^k over [o - 1/2, o + 1/2]"""
    P = Pn.polyint(coef)
    return np.array([Pn.polyval(o + 0.5, P) - Pn.polyval(o - 0.5, P) for o in offsets])


@pytest.mark.parametrize("order", [5, 6])
def test_linear_reconstruction_reproduces_polynomials(oracle, order):
    cfg = oracle.make_cfg(1, (8,), 0.1, limiter=1)
    rng = np.random.default_rng(order)
    for deg in range(order):
        coef = rng.normal(size=deg + 1)
        u = _avgs(coef, range(-2, 4))
        assert oracle.nc_point(cfg, order, u)["val"] == pytest.approx(Pn.polyval(0.5, coef), rel=1e-12, abs=1e-12)
    coef = np.zeros(order + 1)
    coef[order] = 1.0
    u = _avgs(coef, range(-2, 4))
    assert abs(oracle.nc_point(cfg, order, u)["val"] - 0.5**order) > 1e-6


@pytest.mark.parametrize("order", [5, 6])
def test_geno_reproduces_quadratics(oracle, order):
    cfg = oracle.make_cfg(1, (8,), 0.1)
    coef = np.array([0.7, -0.4, 0.9])
    r = oracle.nc_point(cfg, order, _avgs(coef, range(-2, 4)))
    assert r["val"] == pytest.approx(Pn.polyval(0.5, coef), rel=1e-13)
    assert np.allclose(r["p"], Pn.polyval(0.5, coef), rtol=1e-13)


def test_fifth_order_indicators_are_jiang_shu(oracle):
    cfg = oracle.make_cfg(1, (8,), 0.1)
    rng = np.random.default_rng(11)
    for _ in range(20):
        u = rng.normal(size=6)
        a, b, c, d, e = u[:5]  # offsets -2..2
        js = [
            13 / 12 * (a - 2 * b + c) ** 2 + 0.25 * (a - 4 * b + 3 * c) ** 2,
            13 / 12 * (b - 2 * c + d) ** 2 + 0.25 * (b - d) ** 2,
            13 / 12 * (c - 2 * d + e) ** 2 + 0.25 * (3 * c - 4 * d + e) ** 2,
        ]
        np.testing.assert_allclose(oracle.nc_point(cfg, 5, u)["IS"], js, rtol=1e-12, atol=1e-13)


def test_sixth_order_cubic_indicators(oracle):
    """Cubic data: the two cubic sub-stencils reproduce it, so their
    indicators are sum_(l=1..3) int_cell (d^l p)^2 of the data's own cubic."""
    cfg = oracle.make_cfg(1, (8,), 0.1)
    coef = np.array([0.2, 1.1, -0.6, 0.8])
    u = _avgs(coef, range(-2, 4))
    want = 0.0
    for l in range(1, 4):
        dl = Pn.polyder(coef, l)
        sq = Pn.polyint(Pn.polymul(dl, dl))
        want += Pn.polyval(0.5, sq) - Pn.polyval(-0.5, sq)
    IS = oracle.nc_point(cfg, 6, u)["IS"]
    assert IS[2] == pytest.approx(want, rel=1e-12)
    assert IS[3] == pytest.approx(want, rel=1e-12)


def _run(oracle, order, W, cfg, t_end, cfl):
    t = 0.0
    h = cfg.h
    while t < t_end - 1e-12:
        dt = min(cfl * h / oracle.max_wavespeed(cfg, W), t_end - t)
        assert oracle.nc_step(cfg, order, dt, W) == 0
        t += dt
    return W


@pytest.mark.parametrize("order", [5, 6])
def test_stationary_contact_is_kept_exactly(oracle, order):
    n = 24
    x = (np.arange(n) + 0.5) / n
    rho = np.where(x < 0.5, 1.0, 0.125)
    W = np.stack([rho, np.zeros(n), np.full(n, 1.0 / (GAMMA - 1))])
    cfg = oracle.make_cfg(1, (n,), 1.0 / n, bc=1)
    W1 = _run(oracle, order, W.copy(), cfg, 0.2, 0.4)
    np.testing.assert_allclose(W1, W, rtol=0, atol=1e-13)
    # equal states: the Euler flux
    F = oracle.nc_flux(cfg, order, np.stack([np.full(n, 1.3), np.full(n, 1.3 * 0.4), np.full(n, 2.0)]))
    u, p = 0.4, (GAMMA - 1) * (2.0 - 0.5 * 1.3 * 0.16)
    np.testing.assert_allclose(F[:, 5], [1.3 * u, 1.3 * u * u + p, u * (2.0 + p)], rtol=1e-14)


@pytest.mark.parametrize("order,min_order", [(5, 4.7), (6, 5.7)])
def test_design_order(oracle, order, min_order):
    """Sec. 6.1 advected density wave; dt ~ h^1.5 keeps the RK4 error below the
    spatial one."""
    err = []
    for n in (8, 16, 32):
        W, G, h = I.sine_wave(1, n)
        cfg = oracle.make_cfg(1, (n,), h, bc=0)
        W = _run(oracle, order, W, cfg, 2.0, 0.4 * (8 / n) ** 0.5)
        err.append(np.abs(W[0] - I.sine_exact_rho(1, n, 2.0)).mean())
    rates = [np.log2(err[i] / err[i + 1]) for i in range(2)]
    assert min(rates) >= min_order, rates


def test_rk4_is_fourth_order_in_time(oracle):
    n, order = 32, 6
    W0, G, h = I.sine_wave(1, n)
    cfg = oracle.make_cfg(1, (n,), h, bc=0)
    ref = _run(oracle, order, W0.copy(), cfg, 0.5, 0.025)
    err = [np.abs(_run(oracle, order, W0.copy(), cfg, 0.5, c)[0] - ref[0]).max() for c in (0.4, 0.2)]
    assert np.log2(err[0] / err[1]) >= 3.7, err


@pytest.mark.parametrize("order", [5, 6])
def test_conservation_and_mirror_symmetry(oracle, order):
    n = 40
    W, G, h, _ = I.riemann_1d(n, seed=3)
    Wp = np.ascontiguousarray(np.concatenate([W, W[:, ::-1] * np.array([[1], [-1], [1]])], axis=1))
    cfg = oracle.make_cfg(1, (2 * n,), h, bc=0)
    tot0 = Wp.sum(axis=1)
    W1 = _run(oracle, order, Wp.copy(), cfg, 0.05, 0.4)
    np.testing.assert_allclose(W1.sum(axis=1), tot0, rtol=1e-13, atol=1e-12)
    # the mirror image x -> -x, u -> -u stays a mirror image
    np.testing.assert_allclose(W1[:, ::-1] * np.array([[1], [-1], [1]]), W1, rtol=1e-12, atol=1e-12)


def test_converges_to_exact_riemann(oracle):
    L = (1.0, 0.0, 1.0)
    R = (0.125, 0.0, 0.1)
    errs = []
    for n in (32, 64, 128):
        x = (np.arange(n) + 0.5) / n
        rho = np.where(x < 0.5, L[0], R[0])
        p = np.where(x < 0.5, L[2], R[2])
        W = np.stack([rho, np.zeros(n), p / (GAMMA - 1)])
        cfg = oracle.make_cfg(1, (n,), 1.0 / n, bc=1)
        W = _run(oracle, 6, W, cfg, 0.15, 0.4)
        ex = riemann.cell_averages(L, R, n, 0.15)
        errs.append(np.abs(W[0] - ex[0]).mean())
    assert errs[0] > errs[1] > errs[2], errs
    assert np.log2(errs[0] / errs[2]) / 2 >= 0.5, errs


def test_compact_beats_noncompact_on_coarse_meshes(oracle):
    """Sec. 6.1: the compact scheme reaches a smaller error with fewer cells:
    8th-order compact GKS on 4 cells against the 5th/6th-order non-compact
    schemes on 6 cells, t = 2."""
    W, G, h = I.sine_wave(1, 4)
    cfg = oracle.make_cfg(1, (4,), h, bc=0)
    t = 0.0
    while t < 2.0 - 1e-12:
        dt = min(0.4 * h / oracle.max_wavespeed(cfg, W), 2.0 - t)
        assert oracle.step(cfg, dt, W, G) == 0
        t += dt
    e_compact = np.abs(W[0] - I.sine_exact_rho(1, 4, 2.0)).mean()
    for order in (5, 6):
        W6, G6, h6 = I.sine_wave(1, 6)
        cfg6 = oracle.make_cfg(1, (6,), h6, bc=0)
        W6 = _run(oracle, order, W6, cfg6, 2.0, 0.4)
        assert e_compact < np.abs(W6[0] - I.sine_exact_rho(1, 6, 2.0)).mean()


@pytest.mark.parametrize("order", [5, 6])
def test_blast_wave(oracle, order):
    """Woodward-Colella blast wave (Sec. 6.6) with reflecting walls, N = 400,
    CFL 0.4, to t = 0.038: both schemes stay admissible (the 6th-order one
    only with IS^tau over the outer and centred sub-stencils, R16)."""
    n = 400
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    W = np.stack([np.ones(n), np.zeros(n), p / (GAMMA - 1)])
    cfg = oracle.make_cfg(1, (n,), h, bc=2)
    W = _run(oracle, order, W, cfg, 0.038, 0.4)
    assert W[0].min() > 0 and abs(W[0].sum() * h - 1.0) < 1e-12


def test_sixth_order_sees_a_jump_at_the_stencil_end(oracle):
    """A jump between offsets 2 and 3 lies only in S_0 and S_4: the path
    function must still leave the high-order polynomial."""
    cfg = oracle.make_cfg(1, (8,), 0.1)
    r = oracle.nc_point(cfg, 6, np.array([0.0, 0.0, 0.0, 0.0, 0.0, 1.0]))
    assert r["chi"] < 1e-10 and abs(r["val"]) < 1e-10
