"""Brute-force pin of the oracle's multi-dimensional gas-kinetic flux (no GPU).

The paper takes the interface flux from the BGK solution of the gas-kinetic
scheme and defers its formulas (Sec. 2).  The oracle evaluates that solution
with closed-form half-space moments and products of velocity polynomials.
This test evaluates it from its definition instead, with nothing shared:

  * velocity integrals by tensor quadrature of the Maxwellians themselves:
    Gauss-Legendre over each half line of the normal velocity u (the split at
    u = 0 is where the two initial states meet), Gauss-Hermite over the
    tangential velocities v (and w), chi-square moments for the K internal
    degrees of freedom;
  * micro-slopes a_e (one per face axis e, normal and tangential) of each
    Maxwellian from its own quadrature moment matrix <psi psi^T> (numpy
    solve), time slopes A from the compatibility condition
    <(sum_e a_e u_e + A) psi> = 0;
  * the equilibrium's relaxation integral (1/tau) int_0^t g0 (...) e^{-(t-s)/tau} ds
    and the time integrals of the flux over [0, dt/2] and [0, dt] by
    Gauss-Legendre quadrature in s and t.

The states differ on the two sides and both sides carry non-zero normal and
tangential slopes, so the tangential transport terms of each side (and which
side they belong to) enter the result.  A control case swaps the two sides'
tangential slopes and must move the result far beyond the tolerance.

The BGK solution at the interface (x = 0) for t >= 0, with numerical collision
time tau (relaxation) and tau0 the collision time of the Chapman-Enskog parts
(0 for the Euler flux, tau itself for the plain BGK solution, mu / p0 for the
Navier-Stokes flux):

  f(0, t) = (1/tau) int_0^t g0 [1 - (t - s) sum_e a0_e u_e + s A0] e^{-(t-s)/tau} ds
          + [tau0 != tau] (tau - tau0) (1 - e^{-t/tau}) (sum_e a0_e u_e + A0) g0
          + e^{-t/tau} [1 - t sum_e a_e u_e - tau0 (sum_e a_e u_e + A)] g_{l|r},

the last term with g_l, a_l, A_l for u > 0 and g_r, a_r, A_r for u < 0.
"""
import math

import numpy as np
import pytest
from scipy import stats

GAMMA = 1.4


def _state(rng, m):
    rho = rng.uniform(0.4, 1.8)
    vel = rng.uniform(-0.9, 0.9, size=m)
    p = rng.uniform(0.4, 1.8)
    return np.array([rho] + list(rho * vel) + [p / (GAMMA - 1) + 0.5 * rho * vel @ vel])


def _prim(W, m):
    rho = W[0]
    U = W[1 : 1 + m] / rho
    p = (GAMMA - 1) * (W[m + 1] - 0.5 * rho * U @ U)
    return rho, U, rho / (2 * p), p


class Maxwellian:
    """Quadrature nodes of rho^-1 g over the velocity space (or over the half
    space u > 0 / u < 0), and E[(xi^2)^j] of the internal degrees of freedom."""

    def __init__(self, W, m, half):
        self.m = m
        self.rho, self.U, self.lam, self.p = _prim(W, m)
        sig = 1.0 / math.sqrt(2.0 * self.lam)  # standard deviation per velocity component
        U0 = self.U[0]
        if half == 0:
            x, w = np.polynomial.hermite_e.hermegauss(40)
            un, uw = U0 + sig * x, w / math.sqrt(2 * math.pi)
        else:
            # Gauss-Legendre over [0, U0 + 16 sig] or [U0 - 16 sig, 0] of the normal density
            a, b = (0.0, max(U0 + 16 * sig, 1e-3)) if half > 0 else (min(U0 - 16 * sig, -1e-3), 0.0)
            x, w = np.polynomial.legendre.leggauss(600)
            un = 0.5 * (b - a) * (x + 1) + a
            uw = 0.5 * (b - a) * w * np.exp(-((un - U0) ** 2) / (2 * sig * sig)) / (math.sqrt(2 * math.pi) * sig)
        xs, ws = np.polynomial.hermite_e.hermegauss(16)
        axes, wts = [un], [uw]
        for a_ in range(1, m):
            axes.append(self.U[a_] + sig * xs)
            wts.append(ws / math.sqrt(2 * math.pi))
        grids = np.meshgrid(*axes, indexing="ij")
        wgrid = np.prod(np.meshgrid(*wts, indexing="ij"), axis=0)
        self.u = [g.ravel() for g in grids]  # u_0 (normal), u_1, u_2
        self.w = wgrid.ravel()
        K = 2.0 / (GAMMA - 1) - m
        ch = stats.chi2(K)
        self.xi = np.array([1.0] + [ch.moment(j) / (2 * self.lam) ** j for j in range(1, 5)])

    def mean(self, poly):
        """E[poly] for poly = [c_0, c_1, ...]: coefficients (arrays over the
        nodes) of powers of xi^2."""
        return float(sum(np.sum(self.w * c) * self.xi[j] for j, c in enumerate(poly)))


def _zero(n):
    return [np.zeros(n) for _ in range(4)]


def _mul(a, b):
    out = _zero(a[0].size)
    for i, ai in enumerate(a):
        for j, bj in enumerate(b):
            if i + j < 4:
                out[i + j] = out[i + j] + ai * bj
    return out


def _add(a, b, cb=1.0):
    return [x + cb * y for x, y in zip(a, b)]


def _const(g, c):
    z = _zero(g.w.size)
    z[0] = z[0] + c
    return z


def _psi(g, b):
    """psi_b: 1, u_1 .. u_m, (|u|^2 + xi^2) / 2."""
    m = g.m
    z = _zero(g.w.size)
    if b == 0:
        z[0] = z[0] + 1.0
    elif b <= m:
        z[0] = g.u[b - 1].copy()
    else:
        z[0] = 0.5 * sum(x * x for x in g.u)
        z[1] = z[1] + 0.5
    return z


def _vel(g, e):
    z = _zero(g.w.size)
    z[0] = g.u[e].copy()
    return z


def _coef_poly(g, s):
    """sum_b s_b psi_b."""
    out = _zero(g.w.size)
    for b in range(g.m + 2):
        out = _add(out, _psi(g, b), s[b])
    return out


def _moment_matrix(g):
    nv = g.m + 2
    return np.array([[g.mean(_mul(_psi(g, a), _psi(g, b))) for b in range(nv)] for a in range(nv)])


def _slopes(W, dW, m):
    """Micro-slopes a_e (coefficients on psi) of the full-space Maxwellian of W
    for the physical derivatives dW[e] along face axis e, <a_e psi> = dW_e / rho;
    and the time slope A from <(sum_e a_e u_e + A) psi> = 0."""
    g = Maxwellian(W, m, 0)
    Mm = _moment_matrix(g)
    s = [np.linalg.solve(Mm, dW[e] / g.rho) for e in range(m)]
    T = _zero(g.w.size)
    for e in range(m):
        T = _add(T, _mul(_coef_poly(g, s[e]), _vel(g, e)))
    rhs = np.array([-g.mean(_mul(T, _psi(g, b))) for b in range(m + 2)])
    A = np.linalg.solve(Mm, rhs)
    return s, A


def _moments(g, s, A, with_u):
    """rho <u^k psi_b>, rho <u^k psi_b sum_e a_e u_e>, rho <u^k psi_b A> (k = with_u)
    against the (half- or full-space) Maxwellian g."""
    m = g.m
    T = _zero(g.w.size)
    for e in range(m):
        T = _add(T, _mul(_coef_poly(g, s[e]), _vel(g, e)))
    Ap = _coef_poly(g, A)
    out = np.zeros((3, m + 2))
    for b in range(m + 2):
        ps = _psi(g, b)
        if with_u:
            ps = _mul(ps, _vel(g, 0))
        out[0, b] = g.rho * g.mean(ps)
        out[1, b] = g.rho * g.mean(_mul(ps, T))
        out[2, b] = g.rho * g.mean(_mul(ps, Ap))
    return out


def brute_force(m, Wl, Wr, dWl, dWr, dt, c1, c2, tau_mode, mu):
    """F, dF/dt and W(dt/2) of the BGK solution above by quadrature."""
    gl_h, gr_h = Maxwellian(Wl, m, +1), Maxwellian(Wr, m, -1)
    # equilibrium: the two half streams collide
    W0 = np.array([gl_h.rho * gl_h.mean(_psi(gl_h, b)) + gr_h.rho * gr_h.mean(_psi(gr_h, b)) for b in range(m + 2)])
    sl, Al = _slopes(Wl, dWl, m)
    sr, Ar = _slopes(Wr, dWr, m)
    s0, A0 = _slopes(W0, 0.5 * (np.asarray(dWl) + np.asarray(dWr)), m)
    g0 = Maxwellian(W0, m, 0)
    pl, pr, p0 = gl_h.p, gr_h.p, g0.p
    tau = c1 * dt + c2 * abs(pl - pr) / (pl + pr) * dt
    tau_p = mu / p0
    if tau_mode == 2:
        tau += tau_p
    tau0 = {0: 0.0, 1: tau, 2: tau_p}[tau_mode]
    # velocity moments of every velocity function the solution is built from
    Mom = {}
    for k in (0, 1):
        Mom["0", k] = _moments(g0, s0, A0, k)
        Mom["l", k] = _moments(gl_h, sl, Al, k)
        Mom["r", k] = _moments(gr_h, sr, Ar, k)
    sn, sw = np.polynomial.legendre.leggauss(48)

    def f_mom(t, k):
        """rho <u^k psi f(0, t)> for every psi."""
        ss = 0.5 * t * (sn + 1)
        ws = 0.5 * t * sw
        ker = ws * np.exp(-(t - ss) / tau) / tau
        I0, I1, I2 = ker.sum(), (ker * (t - ss)).sum(), (ker * ss).sum()
        e0 = Mom["0", k]
        out = I0 * e0[0] - I1 * e0[1] + I2 * e0[2]
        et = math.exp(-t / tau)
        if tau_mode != 1:
            out = out + (tau - tau0) * (1 - et) * (e0[1] + e0[2])
        for side in ("l", "r"):
            M_ = Mom[side, k]
            out = out + et * (M_[0] - t * M_[1] - tau0 * (M_[1] + M_[2]))
        return out

    tn, tw = np.polynomial.legendre.leggauss(40)

    def F_int(delta):
        return sum(w * 0.5 * delta * f_mom(0.5 * delta * (x + 1), 1) for x, w in zip(tn, tw))

    F1, F2 = F_int(0.5 * dt), F_int(dt)
    return (4 * F1 - F2) / dt, 4 * (F2 - 2 * F1) / dt**2, f_mom(0.5 * dt, 0)


def _case(rng, m):
    Wl, Wr = _state(rng, m), _state(rng, m)
    dWl = rng.normal(size=(m, m + 2)) * 0.6
    dWr = rng.normal(size=(m, m + 2)) * 0.6
    return Wl, Wr, dWl, dWr


def _close(a, b, tol):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() <= tol * scale


@pytest.mark.parametrize("tau_mode", [0, 1, 2])
@pytest.mark.parametrize("m", [2, 3])
def test_bgk_brute_force_multid(oracle, m, tau_mode):
    """Unequal states, non-zero normal and tangential slopes on both sides:
    the oracle's F, dF/dt and W(dt/2) equal the quadrature of the BGK
    solution to 1e-10 of each vector's scale."""
    rng = np.random.default_rng(900 + 10 * m + tau_mode)
    dt, c1, c2 = 0.04, 0.5, 1.0
    mu = 0.02 if tau_mode == 2 else 0.0
    for _ in range(2):
        Wl, Wr, dWl, dWr = _case(rng, m)
        F, Ft, Wh = oracle.gks_point(m, GAMMA, dt, Wl, Wr, dWl, dWr, c1=c1, c2=c2, tau_mode=tau_mode, mu=mu)
        Fb, Ftb, Whb = brute_force(m, Wl, Wr, dWl, dWr, dt, c1, c2, tau_mode, mu)
        assert _close(F, Fb, 1e-10), (F, Fb)
        assert _close(Ft, Ftb, 1e-10), (Ft, Ftb)
        assert _close(Wh, Whb, 1e-10), (Wh, Whb)


@pytest.mark.parametrize("m", [2, 3])
def test_bgk_brute_force_sees_the_tangential_slopes(oracle, m):
    """Control: the brute force with the two sides' tangential slopes swapped
    (or the tangential slopes dropped) is far from the oracle, so the pin
    above decides which side each tangential transport term belongs to."""
    rng = np.random.default_rng(950 + m)
    dt = 0.04
    Wl, Wr, dWl, dWr = _case(rng, m)
    F, Ft, Wh = oracle.gks_point(m, GAMMA, dt, Wl, Wr, dWl, dWr, c1=0.5)
    swl, swr = dWl.copy(), dWr.copy()
    swl[1:], swr[1:] = dWr[1:], dWl[1:]
    Fs, Fts, Whs = brute_force(m, Wl, Wr, swl, swr, dt, 0.5, 1.0, 0, 0.0)
    assert not _close(F, Fs, 1e-6) or not _close(Wh, Whs, 1e-6)
    zl, zr = dWl.copy(), dWr.copy()
    zl[1:] = 0.0
    zr[1:] = 0.0
    Fz, Ftz, Whz = brute_force(m, Wl, Wr, zl, zr, dt, 0.5, 1.0, 0, 0.0)
    assert not _close(F, Fz, 1e-6) or not _close(Wh, Whz, 1e-6)
