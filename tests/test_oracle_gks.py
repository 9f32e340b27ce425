"""Pins of the oracle's gas-kinetic flux (no GPU).

The paper defers the GKS flux to earlier work (Sec. 2); the oracle uses the
BGK solution with a kinetic collision of the left/right states.  What fixes it
independently of the oracle's moment algebra:

P6a free stream: equal states and no slopes give the exact Euler flux, no time
    derivative, and the unchanged interface state, for any collision time;
P6b at tau = 0 with equal states the flux is the Euler flux, its time
    derivative is F'(W) dW/dt with dW/dt = -sum_e A_e dW/dx_e
    (Cauchy-Kovalevskaya, Jacobians by complex-step differentiation), and
    W(dt/2) = W + dt/2 dW/dt;
P6c brute force: the BGK integral solution along characteristics, integrated
    numerically in time and velocity (chi-square moments for the internal
    degrees of freedom), matches the oracle's F, dF/dt and W(dt/2) with
    unequal states, unequal slopes and tau > 0;
P7  half-space moments match numerical quadrature and add up to the full-space
    moments; the moment matrix matches quadrature; the micro-slope solve has
    a residual at round-off.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

GAMMA = 1.4


def euler_flux(W, m, d, gamma=GAMMA):
    rho = W[0]
    vel = [W[1 + a] / rho for a in range(m)]
    E = W[m + 1]
    p = (gamma - 1) * (E - 0.5 * rho * sum(v * v for v in vel))
    F = [rho * vel[d]] + [W[1 + a] * vel[d] + (p if a == d else 0.0) for a in range(m)] + [vel[d] * (E + p)]
    return np.array(F)


def jacobian(W, m, d, gamma=GAMMA):
    nv = m + 2
    J = np.zeros((nv, nv))
    hstep = 1e-30
    for j in range(nv):
        Wc = W.astype(complex)
        Wc[j] += 1j * hstep
        J[:, j] = np.imag(euler_flux(Wc, m, d, gamma)) / hstep
    return J


def random_state(rng, m, gamma=GAMMA):
    rho = rng.uniform(0.3, 2.0)
    vel = rng.uniform(-1.0, 1.0, size=m)
    p = rng.uniform(0.3, 2.0)
    return np.array([rho] + list(rho * vel) + [p / (gamma - 1) + 0.5 * rho * vel @ vel])


@pytest.mark.parametrize("m", [1, 2, 3])
def test_free_stream_flux(oracle, m):
    rng = np.random.default_rng(m)
    for tau_c1 in (0.0, 0.7):
        W = random_state(rng, m)
        z = np.zeros((m, m + 2))
        F, Ft, Wh = oracle.gks_point(m, GAMMA, 0.01, W, W, z, z, c1=tau_c1)
        np.testing.assert_allclose(F, euler_flux(W, m, 0), rtol=1e-13, atol=1e-14)
        np.testing.assert_allclose(Ft, 0.0, atol=1e-10)
        np.testing.assert_allclose(Wh, W, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("c1", [0.0, 0.05, 0.5])
@pytest.mark.parametrize("m", [1, 2, 3])
def test_tau0_cauchy_kovalevskaya(oracle, m, c1):
    rng = np.random.default_rng(10 + m)
    dt = 0.02
    for _ in range(4):
        W = random_state(rng, m)
        dW = rng.normal(size=(m, m + 2)) * 0.3
        F, Ft, Wh = oracle.gks_point(m, GAMMA, dt, W, W, dW, dW, c1=c1, c2=1.0)
        Wt = -sum(jacobian(W, m, e) @ dW[e] for e in range(m))
        np.testing.assert_allclose(F, euler_flux(W, m, 0), rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(Ft, jacobian(W, m, 0) @ Wt, rtol=1e-10, atol=1e-11)
        np.testing.assert_allclose(Wh, W + 0.5 * dt * Wt, rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------ brute force 1D
def _prim(W):
    rho = W[0]
    U = W[1] / rho
    p = (GAMMA - 1) * (W[2] - 0.5 * rho * U * U)
    return rho, U, rho / (2 * p), p


def _xi_moments(K, lam, jmax=3):
    """E[(xi^2)^j] for K internal degrees of freedom, each of variance 1/(2 lam)."""
    ch = stats.chi2(K)
    return np.array([1.0] + [ch.moment(j) / (2 * lam) ** j for j in range(1, jmax + 1)])


def _poly_psi(u):
    """psi_a = 1, u, (u^2 + xi^2)/2 as coefficient arrays in powers of xi^2 (per u node)."""
    one = np.ones_like(u)
    z = np.zeros_like(u)
    return [np.stack([one, z, z]), np.stack([u, z, z]), np.stack([0.5 * u * u, 0.5 * one, z])]


def _slope_poly(s, u):
    """a = s0 + s1 u + s2 (u^2 + xi^2)/2 in powers of xi^2."""
    return np.stack([s[0] + s[1] * u + 0.5 * s[2] * u * u, 0.5 * s[2] * np.ones_like(u), np.zeros_like(u)])


def _mul(a, b):
    """product of two polynomials in xi^2 (degree <= 2 kept)."""
    out = np.zeros_like(a)
    for i in range(3):
        for j in range(3 - i):
            out[i + j] += a[i] * b[j]
    return out


def _quad_moment(oracle_ignored, W, poly_fn, half):
    """rho^-1 int poly(u, xi) g du dxi over u>0 (half=1), u<0 (-1) or all (0), numerically."""
    rho, U, lam, _ = _prim(W)
    K = 2 / (GAMMA - 1) - 1
    xm = _xi_moments(K, lam)
    lo, hi = U - 14 / math.sqrt(lam), U + 14 / math.sqrt(lam)
    if half > 0:
        lo = max(lo, 0.0)
    if half < 0:
        hi = min(hi, 0.0)
    if hi <= lo:
        return 0.0

    def integrand(u):
        c = poly_fn(np.array([u]))
        return float(sum(c[j][0] * xm[j] for j in range(3))) * math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)

    return integrate.quad(integrand, lo, hi, epsabs=1e-14, epsrel=1e-13, limit=200)[0]


@pytest.mark.parametrize("tau_mode", [1, 0, 2])
def test_bgk_brute_force_1d(oracle, tau_mode):
    """tau_mode 1: plain BGK solution with one collision time tau_n.
    tau_mode 0 (Euler): the initial state carries no Chapman-Enskog part and
    the equilibrium's Chapman-Enskog terms use the physical tau = 0, which
    equals the BGK(tau_n) solution plus tau_n (1 - e^{-t/tau_n}) (a0 u + A0) g0.
    tau_mode 2 (Navier-Stokes): physical tau_p = mu / p0 in the Chapman-Enskog
    terms of the initial states and of the equilibrium, relaxation with
    tau_n = tau_p + c1 dt + ...: the BGK(tau_n) solution whose initial states
    carry tau_p, plus (tau_n - tau_p) (1 - e^{-t/tau_n}) (a0 u + A0) g0."""
    rng = np.random.default_rng(42)
    dt = 0.05
    c1 = 0.6
    mu = 0.03 if tau_mode == 2 else 0.0
    for case in range(3):
        Wl = random_state(rng, 1)
        Wr = random_state(rng, 1)
        dWl = rng.normal(size=3) * 0.5
        dWr = rng.normal(size=3) * 0.5
        F, Ft, Wh = oracle.gks_point(1, GAMMA, dt, Wl, Wr, dWl, dWr, c1=c1, c2=1.0, tau_mode=tau_mode, mu=mu)
        rl, Ul, laml, pl = _prim(Wl)
        rr, Ur, lamr, pr = _prim(Wr)
        tau = c1 * dt + abs(pl - pr) / (pl + pr) * dt
        # equilibrium state by numerical half-space quadrature
        W0 = np.array([
            rl * _quad_moment(None, Wl, lambda u, a=a: _poly_psi(u)[a], +1)
            + rr * _quad_moment(None, Wr, lambda u, a=a: _poly_psi(u)[a], -1)
            for a in range(3)
        ])
        r0, U0, lam0, p0 = _prim(W0)
        tau_p = mu / p0  # physical collision time (tau_mode 2)
        if tau_mode == 2:
            tau += tau_p
        # micro-slopes: oracle's slope solve (pinned below by its residual)
        sl = oracle.slope_solve(1, GAMMA, Wl, dWl / rl)
        sr = oracle.slope_solve(1, GAMMA, Wr, dWr / rr)
        s0 = oracle.slope_solve(1, GAMMA, W0, 0.5 * (dWl + dWr) / r0)

        # time coefficients from <(a u + A) psi> = 0, moments by quadrature
        def Acoef(W, s, rho):
            rhs = np.array([
                -_quad_moment(None, W, lambda u, a=a: _mul(_mul(_slope_poly(s, u), np.stack([u, 0 * u, 0 * u])), _poly_psi(u)[a]), 0)
                for a in range(3)
            ])
            return oracle.slope_solve(1, GAMMA, W, rhs)

        Al, Ar, A0 = Acoef(Wl, sl, rl), Acoef(Wr, sr, rr), Acoef(W0, s0, r0)
        K = 2 / (GAMMA - 1) - 1
        xm = {k: _xi_moments(K, lam) for k, lam in (("l", laml), ("r", lamr), ("0", lam0))}
        gs, gws = np.polynomial.legendre.leggauss(40)

        def gauss_u(U, lam):
            return lambda u: math.sqrt(lam / math.pi) * np.exp(-lam * (u - U) ** 2)

        # velocity nodes on both half lines
        lo = min(Ul, Ur, U0) - 14 / math.sqrt(min(laml, lamr, lam0))
        hi = max(Ul, Ur, U0) + 14 / math.sqrt(min(laml, lamr, lam0))
        un, uw = np.polynomial.legendre.leggauss(400)
        uneg = lo / 2 * (un + 1)  # [lo, 0]
        wneg = uw * (-lo) / 2
        upos = hi / 2 * (un + 1)  # [0, hi]
        wpos = uw * hi / 2
        u = np.concatenate([uneg, upos])
        wu = np.concatenate([wneg, wpos])
        pos = u > 0

        def f_moments(t, with_u):
            """int psi_a (u) f(0, t, u, xi) du dxi for a = 0..2."""
            # equilibrium part: (1/tau) int_0^t g0 (1 + a0 x + A0 s) e^{-(t-s)/tau} ds, x = -u (t - s)
            s_nodes = t / 2 * (gs + 1)
            s_w = gws * t / 2
            a0p = _slope_poly(s0, u)
            A0p = _slope_poly(A0, u)
            eq = np.zeros((3, u.size))
            for s, w in zip(s_nodes, s_w):
                k = w * math.exp(-(t - s) / tau) / tau
                eq[0] += k
                eq += k * (a0p * (-u * (t - s)) + A0p * s)
            et = math.exp(-t / tau)
            # collision time of the Chapman-Enskog parts
            tau0 = {0: 0.0, 1: tau, 2: tau_p}[tau_mode]
            if tau_mode != 1:
                eq += (tau - tau0) * (1 - et) * (_mul(a0p, np.stack([u, 0 * u, 0 * u])) + A0p)
            neq = {}
            for key, s_, A_ in (("l", sl, Al), ("r", sr, Ar)):
                ap = _slope_poly(s_, u)
                Ap = _slope_poly(A_, u)
                base = np.zeros((3, u.size))
                base[0] = 1.0
                neq[key] = et * (base + ap * (-u * t) - tau0 * (_mul(ap, np.stack([u, 0 * u, 0 * u])) + Ap))
            out = np.zeros(3)
            for a in range(3):
                ps = _poly_psi(u)[a]
                if with_u:
                    ps = _mul(ps, np.stack([u, 0 * u, 0 * u]))
                pe = _mul(eq, ps)
                pl_ = _mul(neq["l"], ps)
                pr_ = _mul(neq["r"], ps)
                ve = r0 * gauss_u(U0, lam0)(u) * sum(pe[j] * xm["0"][j] for j in range(3))
                vl = rl * gauss_u(Ul, laml)(u) * sum(pl_[j] * xm["l"][j] for j in range(3))
                vr = rr * gauss_u(Ur, lamr)(u) * sum(pr_[j] * xm["r"][j] for j in range(3))
                out[a] = float(np.sum(wu * (ve + np.where(pos, vl, vr))))
            return out

        def F_int(delta):
            tn, tw = np.polynomial.legendre.leggauss(30)
            return sum(w * delta / 2 * f_moments(delta / 2 * (x + 1), True) for x, w in zip(tn, tw))

        F1, F2 = F_int(dt / 2), F_int(dt)
        Fb = (4 * F1 - F2) / dt
        Ftb = 4 * (F2 - 2 * F1) / dt**2
        Whb = f_moments(dt / 2, False)
        np.testing.assert_allclose(F, Fb, rtol=1e-9, atol=1e-10)
        np.testing.assert_allclose(Ft, Ftb, rtol=1e-7, atol=1e-7)
        np.testing.assert_allclose(Wh, Whb, rtol=1e-9, atol=1e-10)


# ------------------------------------------------------------------- P7
@pytest.mark.parametrize("U", [-1.3, -0.2, 0.0, 0.4, 2.1])
@pytest.mark.parametrize("lam", [0.3, 1.0, 4.0])
def test_half_moments_quadrature(oracle, U, lam):
    dens = lambda u: math.sqrt(lam / math.pi) * math.exp(-lam * (u - U) ** 2)
    for n in range(0, 8):
        qp = integrate.quad(lambda u: u**n * dens(u), 0, np.inf, epsabs=1e-15, epsrel=1e-14)[0]
        qm = integrate.quad(lambda u: u**n * dens(u), -np.inf, 0, epsabs=1e-15, epsrel=1e-14)[0]
        mp = oracle.mom_half(n, U, lam, +1)
        mm = oracle.mom_half(n, U, lam, -1)
        scale = 1.0 + abs(qp) + abs(qm)
        assert abs(mp - qp) <= 1e-12 * scale
        assert abs(mm - qm) <= 1e-12 * scale
        full = stats.norm(loc=U, scale=math.sqrt(1 / (2 * lam))).moment(n)
        assert abs(mp + mm - full) <= 1e-12 * (1 + abs(full))


@pytest.mark.parametrize("m", [1, 2, 3])
def test_moment_matrix_quadrature(oracle, m):
    rng = np.random.default_rng(30 + m)
    W = random_state(rng, m)
    M = oracle.moment_matrix(m, GAMMA, W)
    rho = W[0]
    vel = W[1 : 1 + m] / rho
    p = (GAMMA - 1) * (W[m + 1] - 0.5 * rho * vel @ vel)
    lam = rho / (2 * p)
    K = 2 / (GAMMA - 1) - m
    # Monte-Carlo-free check: Gauss-Hermite tensor quadrature over the m velocities,
    # chi-square moments for the internal degrees of freedom
    gh_x, gh_w = np.polynomial.hermite.hermgauss(12)
    sig = 1 / math.sqrt(lam)
    xm = _xi_moments(K, lam, 4)
    grids = np.meshgrid(*([gh_x] * m), indexing="ij")
    wts = np.prod(np.meshgrid(*([gh_w] * m), indexing="ij"), axis=0) / math.pi ** (m / 2)
    us = [vel[a] + sig * grids[a] for a in range(m)]
    u2 = sum(x * x for x in us)
    # psi as coefficients in powers of xi^2
    psis = [(np.ones_like(u2), 0 * u2)] + [(x, 0 * u2) for x in us] + [(0.5 * u2, 0.5 + 0 * u2)]
    nv = m + 2
    Mq = np.zeros((nv, nv))
    for i in range(nv):
        for j in range(nv):
            a0, a1 = psis[i]
            b0, b1 = psis[j]
            val = a0 * b0 + (a0 * b1 + a1 * b0) * xm[1] + a1 * b1 * xm[2]
            Mq[i, j] = float(np.sum(wts * val))
    np.testing.assert_allclose(M, Mq, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_slope_solve_residual(oracle, m):
    rng = np.random.default_rng(50 + m)
    for _ in range(5):
        W = random_state(rng, m)
        rhs = rng.normal(size=m + 2)
        s = oracle.slope_solve(m, GAMMA, W, rhs)
        M = oracle.moment_matrix(m, GAMMA, W)
        np.testing.assert_allclose(M @ s, rhs, rtol=1e-13, atol=1e-13)


def test_mirror_symmetry_of_flux(oracle):
    """x -> -x, u -> -u: swapping the sides and mirroring states and slopes
    mirrors the flux (mass and energy fluxes change sign, momentum flux not)."""
    rng = np.random.default_rng(77)
    for m in (1, 2, 3):
        Wl, Wr = random_state(rng, m), random_state(rng, m)
        dWl = rng.normal(size=(m, m + 2)) * 0.3
        dWr = rng.normal(size=(m, m + 2)) * 0.3
        F, Ft, Wh = oracle.gks_point(m, GAMMA, 0.03, Wl, Wr, dWl, dWr)

        def mir(W):
            W = W.copy()
            W[1] = -W[1]
            return W

        def mird(dW):
            dW = dW.copy()
            dW[0] = -dW[0]  # normal derivative flips
            dW[:, 1] = -dW[:, 1]  # normal momentum flips
            return dW

        Fm, Ftm, Whm = oracle.gks_point(m, GAMMA, 0.03, mir(Wr), mir(Wl), mird(dWr), mird(dWl))
        sgn = np.ones(m + 2)
        sgn[0] = sgn[-1] = -1
        sgn[2 : 1 + m] = -1  # tangential momentum fluxes (u_t u_n) change sign with u_n
        np.testing.assert_allclose(Fm, sgn * F, rtol=1e-12, atol=1e-13)
        np.testing.assert_allclose(Ftm, sgn * Ft, rtol=1e-10, atol=1e-11)
        np.testing.assert_allclose(Whm, mir(Wh), rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------------- P8
# Navier-Stokes (tau_mode 2, Prandtl number 1): for continuous data the BGK
# solution is the Chapman-Enskog one, whose flux is the Euler flux plus the
# Newtonian stress and Fourier heat flux with mu = tau p and conductivity
# kappa = mu c_p, c_p = gamma / (gamma - 1) (R = 1, T = p / rho).


@pytest.mark.parametrize("m", [2, 3])
def test_ns_shear_stress_closed_form(oracle, m):
    """Linear shear V(x) = V0 + s x at rest normally (U = 0), uniform rho, p:
    F = (0, p, -mu s, [0,] -mu s V0) (stress tau_xy = mu dV/dx and its work),
    for any dt and numerical collision time."""
    rho, p, V0, s_, mu = 1.3, 0.8, 0.35, 0.7, 0.02
    W = np.zeros(m + 2)
    W[0] = rho
    W[2] = rho * V0
    W[m + 1] = p / (GAMMA - 1) + 0.5 * rho * V0 * V0
    dW = np.zeros((m, m + 2))
    dW[0, 2] = rho * s_
    dW[0, m + 1] = rho * V0 * s_
    for dt, c1 in ((0.01, 0.05), (0.2, 0.6)):
        F, Ft, Wh = oracle.gks_point(m, GAMMA, dt, W, W, dW, dW, c1=c1, tau_mode=2, mu=mu)
        want = np.zeros(m + 2)
        want[1] = p
        want[2] = -mu * s_
        want[m + 1] = -mu * s_ * V0
        np.testing.assert_allclose(F, want, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("m", [1, 2, 3])
def test_ns_heat_flux_closed_form(oracle, m):
    """Fluid at rest at uniform pressure with a density gradient r along the
    normal: F = (0, p, 0.., -kappa dT/dx) with T = p / rho,
    dT/dx = -p r / rho^2, kappa = mu gamma / (gamma - 1)."""
    rho, p, r, mu = 0.9, 1.7, 0.45, 0.015
    W = np.zeros(m + 2)
    W[0] = rho
    W[m + 1] = p / (GAMMA - 1)
    dW = np.zeros((m, m + 2))
    dW[0, 0] = r
    F, Ft, Wh = oracle.gks_point(m, GAMMA, 0.02, W, W, dW, dW, tau_mode=2, mu=mu)
    want = np.zeros(m + 2)
    want[1] = p
    want[m + 1] = mu * GAMMA / (GAMMA - 1) * p * r / rho**2
    np.testing.assert_allclose(F, want, rtol=1e-12, atol=1e-13)


def test_ns_zero_viscosity_is_euler(oracle):
    rng = np.random.default_rng(7)
    for m in (1, 2, 3):
        Wl, Wr = random_state(rng, m), random_state(rng, m)
        dWl, dWr = rng.normal(size=(m, m + 2)), rng.normal(size=(m, m + 2))
        a = oracle.gks_point(m, GAMMA, 0.03, Wl, Wr, dWl, dWr, tau_mode=0)
        b = oracle.gks_point(m, GAMMA, 0.03, Wl, Wr, dWl, dWr, tau_mode=2, mu=0.0)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
