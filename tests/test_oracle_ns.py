"""Pins of the oracle's Navier-Stokes scheme (no GPU).

The paper applies the compact GKS to viscous flow (Sec. 2: the flux is the
total convective plus viscous flux; Sec. 6.9 and the Taylor-Green vortex:
Prandtl number 1, dynamic viscosity mu).  The BGK model's Chapman-Enskog
limit fixes the transport coefficients independently of the oracle: shear
viscosity mu = tau p, longitudinal (normal-stress) viscosity 2 mu (N - 1) / N
for N = 2 / (gamma - 1) degrees of freedom, heat conductivity
kappa = mu c_p with c_p = (N + 2) / 2 (R = 1).

P9  small-amplitude Fourier modes on a periodic grid follow the linearised
    Navier-Stokes equations with those coefficients, solved exactly here
    (3x3 matrix exponential): the entropy (heat-conduction) mode, the damped
    acoustic mode, and the transverse shear mode exp(-nu k^2 t).  The BGK flux
    carries no time derivative of its viscous part, so the viscous terms are
    first order in time; the bars are taken at small CFL numbers where that
    error is far below the effect of a wrong coefficient (a c_v for c_p, the
    3D-monatomic 4/3 mu for the normal stress, nu = mu / p: each changes the
    measured amplitudes by more than 1 %);
P10 the viscous time-step limit cfl h^2 / (2 (m - 1) nu).

All runs stay in the continuum regime (mean free path tau c far below the
cell size), where the Navier-Stokes equations hold.
"""
import math

import numpy as np
import pytest
from scipy.linalg import expm

GAMMA = 1.4
K = 2 * math.pi


def linear_ns(rho0, p0, mu, t, x0):
    """Exact amplitudes (rho', u', T') at time t of the mode
    Re(x e^{ikx}), k = 2 pi, of the linearised Navier-Stokes equations about
    rest with the BGK transport coefficients."""
    N = 2 / (GAMMA - 1)
    T0 = p0 / rho0
    cv = N / 2
    kappa = mu * (N + 2) / 2
    muL = 2 * mu * (N - 1) / N
    k = K
    A = np.array(
        [
            [0, -1j * k * rho0, 0],
            [-1j * k * T0 / rho0, -muL * k * k / rho0, -1j * k],
            [0, -1j * k * p0 / (rho0 * cv), -kappa * k * k / (rho0 * cv)],
        ]
    )
    return expm(A * t) @ x0


def _cell_avgs(n):
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    s = (np.cos(K * (x - h / 2)) - np.cos(K * (x + h / 2))) / (K * h)
    c = (np.sin(K * (x + h / 2)) - np.sin(K * (x - h / 2))) / (K * h)
    return x, h, s, c


def _mode_state(mode, dim, n, ny, p0, amp):
    """Cell averages and averaged gradients of the mode (first order in amp):
    entropy: rho' = amp sin kx at uniform pressure; acoustic: u' = amp sin kx;
    shear: transverse velocity v' = amp sin kx (dim >= 2)."""
    x, h, s, c = _cell_avgs(n)
    z = np.zeros(n)
    r, u, v, T = z, z, z, z
    dr, du, dv, dT = z, z, z, z
    if mode == "entropy":
        r, T = amp * s, -amp * p0 * s
        dr, dT = amp * K * c, -amp * p0 * K * c
    elif mode == "acoustic":
        u, du = amp * s, amp * K * c
    else:
        v, dv = amp * s, amp * K * c
    rho = 1 + r
    p = rho * (p0 + T)
    dp = dr * (p0 + T) + rho * dT
    nv = dim + 2
    shp = (n,) if dim == 1 else (ny, n)
    W = np.zeros((nv,) + shp)
    G = np.zeros((dim, nv) + shp)
    ke = 0.5 * rho * (u * u + v * v)
    W[0], W[1], W[nv - 1] = rho, rho * u, p / (GAMMA - 1) + ke
    G[0, 0], G[0, 1] = dr, dr * u + rho * du
    G[0, nv - 1] = dp / (GAMMA - 1) + 0.5 * dr * (u * u + v * v) + rho * (u * du + v * dv)
    if dim >= 2:
        W[2], G[0, 2] = rho * v, dr * v + rho * dv
    return W, G, x, h


def _project(W, x, h, comp):
    """sin / cos coefficient of a cell-averaged field (divided by the cell
    averaging factor, exact for a single mode)."""
    if comp == "rho":
        q = W[0] - 1.0
    elif comp == "u":
        q = W[1] / W[0]
    else:
        q = W[2] / W[0]
    if q.ndim == 2:
        q = q.mean(axis=0)
    S = math.sin(K * h / 2) / (K * h / 2)
    return 2 * np.mean(q * np.sin(K * x)) / S


def _run(oracle, mode, dim, n, cfl, mu=0.01, p0=100.0, amp=1e-3, t_end=0.25, ny=2):
    W, G, x, h = _mode_state(mode, dim, n, ny, p0, amp)
    cfg = oracle.make_cfg(dim, (n,) if dim == 1 else (n, ny), h, bc=0, mu=mu)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(oracle.cfl_dt(cfg, W, cfl), t_end - t)
        assert oracle.step(cfg, dt, W, G) == 0
        t += dt
    return W, x, h


@pytest.mark.parametrize("dim", [1, 2])
def test_entropy_mode_heat_conduction(oracle, dim):
    amp, p0, mu, t_end = 1e-3, 100.0, 0.01, 0.25
    W, x, h = _run(oracle, "entropy", dim, 32, 0.1, mu=mu, p0=p0, amp=amp, t_end=t_end)
    x0 = -1j * np.array([amp, 0.0, -amp * p0])  # sin kx = Re(-i e^{ikx})
    want = -linear_ns(1.0, p0, mu, t_end, x0)[0].imag
    got = _project(W, x, h, "rho")
    # decayed by ~10 %; a c_v in place of c_p would leave it 4 % off
    assert abs(got / want - 1) <= 1e-4, (got, want)


@pytest.mark.parametrize("dim", [1, 2])
def test_acoustic_mode_damping(oracle, dim):
    amp, p0, mu, t_end = 1e-3, 100.0, 0.01, 0.25
    W, x, h = _run(oracle, "acoustic", dim, 64, 0.2, mu=mu, p0=p0, amp=amp, t_end=t_end)
    want = -linear_ns(1.0, p0, mu, t_end, -1j * np.array([0.0, amp, 0.0]))[1].imag
    got = _project(W, x, h, "u")
    # a normal-stress viscosity of 4/3 mu (instead of 1.6 mu) moves it by 1.3 %
    assert abs(got / want - 1) <= 2e-3, (got, want)


def test_shear_mode_decay(oracle):
    amp, p0, mu, t_end = 1e-3, 100.0, 0.01, 0.25
    W, x, h = _run(oracle, "shear", 2, 32, 0.4, mu=mu, p0=p0, amp=amp, t_end=t_end)
    want = amp * math.exp(-mu * K * K * t_end)
    got = _project(W, x, h, "v")
    assert abs(got / want - 1) <= 2e-4, (got, want)


def test_inviscid_limit_has_no_decay(oracle):
    """mu = 0: the shear mode is a steady Euler solution; what decays is the
    scheme's own dissipation (the reconstructed face states differ at the
    truncation level), far below the 4 % the viscosity 0.01 gives here."""
    amp = 1e-3
    W, x, h = _run(oracle, "shear", 2, 16, 0.4, mu=0.0, amp=amp, t_end=0.1)
    assert abs(_project(W, x, h, "v") / amp - 1) <= 1e-4


def test_viscous_time_step(oracle):
    """dt = min(cfl h / max(|u| + c), cfl h^2 / (2 (m - 1) nu_max)),
    nu_max = mu / min rho (2 nu in 1D)."""
    rng = np.random.default_rng(3)
    for dim, mu in ((1, 0.05), (2, 0.05), (3, 0.05), (2, 1e-6)):
        n = (8,) * dim
        h = 1.0 / 8
        nv = dim + 2
        rho = rng.uniform(0.5, 2.0, size=n)
        vel = rng.uniform(-0.3, 0.3, size=(dim,) + n)
        p = rng.uniform(0.5, 2.0, size=n)
        W = np.zeros((nv,) + n)
        W[0] = rho
        W[1 : dim + 1] = rho * vel
        W[nv - 1] = p / (GAMMA - 1) + 0.5 * rho * (vel * vel).sum(axis=0)
        cfg = oracle.make_cfg(dim, n, h, bc=0, mu=mu)
        smax = (np.abs(vel).max(axis=0) + np.sqrt(GAMMA * p / rho)).max()
        want = min(0.4 * h / smax, 0.4 * h * h / (2 * max(dim - 1, 1) * mu / rho.min()))
        assert oracle.cfl_dt(cfg, W, 0.4) == pytest.approx(want, rel=1e-13)


def test_taylor_green_initial_decay(oracle):
    """Taylor-Green vortex (u0 = 1, Ma 0.1): the initial field is a single
    Stokes mode with |k|^2 = 3 per component and the inviscid dynamics keeps
    the kinetic energy, so E_k(t) / E_k(0) = exp(-6 nu t) up to O(nu t^3) and
    the Mach-number effects; 12^3 cells, Re = 100 with L0 = 2 pi (mu = 0.0628)."""
    from paper_2507_20461_gb300 import inputs as I

    n, mu, t_end = 12, 2 * math.pi / 100, 0.06
    W, G, h = I.taylor_green_3d(n)
    cfg = oracle.make_cfg(3, (n, n, n), h, bc=0, mu=mu)

    def ek(W):
        return float(np.mean(0.5 * (W[1] ** 2 + W[2] ** 2 + W[3] ** 2) / W[0]))

    E0 = ek(W)
    assert E0 == pytest.approx(0.125, rel=2e-3)  # <|u|^2 / 2> = 1/8 (cell-centre sampling)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(oracle.cfl_dt(cfg, W, 0.4), t_end - t)
        assert oracle.step(cfg, dt, W, G) == 0
        t += dt
    ratio = ek(W) / E0
    want = math.exp(-6 * mu * t_end)
    # the decay is 2.2 %; a viscosity off by 10 % would miss by 2e-3
    assert abs(ratio / want - 1) <= 1e-3, (ratio, want)
