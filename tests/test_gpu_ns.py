"""Navier-Stokes path (opts.mu > 0) of the CUDA library against the oracle,
on cuda:0, through the C ABI.

Bars as for the Euler path: FP64 fluxes element-wise to 1e-12 of the
variable's scale (1e-10 for dF/dt), FP64 steps to a relative L1 residual of
1e-12 per step, mixed precision to a mean |d rho| of 1e-5.  The viscosities
span the continuum regime (tau / dt << 1) and tau / dt of order ten, where
the tau terms of the flux dominate."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2507_20461_gb300 import binding as B

from test_gpu_parity import CASES, _dev, _random_smooth, _rel_l1, _solver

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("mu", [1e-3, 0.05])
@pytest.mark.parametrize("dim,n", CASES)
def test_ns_flux_parity(dim, n, mu):
    bc = 0
    W, G, h = _random_smooth(dim, n, 40 + dim, bc)
    cfg = O.make_cfg(dim, n, h, bc=bc, mu=mu)
    dt = 0.3 * h / O.max_wavespeed(cfg, W)
    ref = O.flux(cfg, dt, W, G)
    s = _solver(dim, n, h, bc, mu=mu)
    s.set_state(_dev(W), _dev(G))
    out = torch.zeros(ref.size, dtype=torch.float64, device=DEV)
    s.flux(dt, out)
    got = out.cpu().numpy().reshape(ref.shape)
    for v in range(dim + 2):
        Fs = np.abs(ref[0, v]).max() + 1e-300
        np.testing.assert_allclose(got[0, v], ref[0, v], rtol=0, atol=1e-12 * Fs)
        np.testing.assert_allclose(got[1, v], ref[1, v], rtol=0, atol=1e-10 * (np.abs(ref[1, v]).max() + Fs / dt))
        np.testing.assert_allclose(got[2, v], ref[2, v], rtol=0, atol=1e-12 * (np.abs(ref[2, v]).max() + 1e-300))
    s.close()



@pytest.mark.parametrize("bc", [0, 3])
@pytest.mark.parametrize("dim,n", CASES)
def test_ns_steps_parity(dim, n, bc):
    """Five FP64 steps with mu = 0.01: relative L1 residual <= 1e-12 per step
    (checked after each step), gradients to 1e-9 of their scale."""
    mu = 0.01
    W, G, h = _random_smooth(dim, n, 50 + dim, bc)
    cfg = O.make_cfg(dim, n, h, bc=bc, mu=mu)
    s = _solver(dim, n, h, bc, mu=mu)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    Wo, Go = W.copy(), G.copy()
    for _ in range(5):
        dt = O.cfl_dt(cfg, Wo, 0.4)
        assert O.step(cfg, dt, Wo, Go) == 0
        s.step(dt)
        s.get_state(Wd, Gd)
        Wg, Gg = Wd.cpu().numpy(), Gd.cpu().numpy()
        assert _rel_l1(Wg, Wo).max() <= 1e-12
        for d in range(dim):
            np.testing.assert_allclose(Gg[d], Go[d], rtol=0, atol=1e-9 * np.abs(Go[d]).max())
        # continue both from the oracle's state so that each step is compared alone
        Wd.copy_(_dev(Wo))
        Gd.copy_(_dev(Go))
        s.set_state(Wd, Gd)
    s.close()


@pytest.mark.parametrize("dim,n", [(1, (40,)), (2, (24, 20)), (3, (10, 8, 6))])
def test_ns_viscous_time_step(dim, n):
    """gks_step_cfl with the viscous limit binding (mu large for the grid):
    one step equals the oracle's step with its cfl_dt."""
    mu = 0.2
    bc = 0
    W, G, h = _random_smooth(dim, n, 60 + dim, bc)
    cfg = O.make_cfg(dim, n, h, bc=bc, mu=mu)
    dt = O.cfl_dt(cfg, W, 0.4)
    assert dt < 0.4 * h / O.max_wavespeed(cfg, W)  # the viscous limit binds
    Wo, Go = W.copy(), G.copy()
    assert O.step(cfg, dt, Wo, Go) == 0
    s = _solver(dim, n, h, bc, mu=mu)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    s.step_cfl(0.4, 1)
    s.get_state(Wd, Gd)
    assert _rel_l1(Wd.cpu().numpy(), Wo).max() <= 1e-12
    s.close()


def test_ns_mixed_precision():
    """2D, mu = 0.005, 20 CFL steps in mixed precision against the FP64 oracle."""
    dim, n, bc, mu = 2, (48, 40), 0, 0.005
    W, G, h = _random_smooth(dim, n, 70, bc)
    cfg = O.make_cfg(dim, n, h, bc=bc, mu=mu)
    s = _solver(dim, n, h, bc, precision=1, mu=mu)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    Wo, Go = W.copy(), G.copy()
    for _ in range(20):
        dt = O.cfl_dt(cfg, Wo, 0.4)
        assert O.step(cfg, dt, Wo, Go) == 0
        s.step(dt)
    s.get_state(Wd, Gd)
    d = np.abs(Wd.cpu().numpy()[0] - Wo[0])
    assert d.mean() <= 1e-5, d.mean()
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_ns_shear_wave_decay(precision):
    """Transverse shear wave v = a sin(2 pi x) on a 128 x 4 periodic grid
    decays as exp(-nu k^2 t) (linearised Navier-Stokes), through gks_step_cfl."""
    n, ny, mu, amp, p0, t_end = 128, 4, 0.01, 1e-3, 100.0, 0.1
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    k = 2 * math.pi
    s_avg = (np.cos(k * (x - h / 2)) - np.cos(k * (x + h / 2))) / (k * h)
    c_avg = (np.sin(k * (x + h / 2)) - np.sin(k * (x - h / 2))) / (k * h)
    W = np.zeros((4, ny, n))
    G = np.zeros((2, 4, ny, n))
    v = amp * s_avg
    W[0], W[2], W[3] = 1.0, v, p0 / 0.4 + 0.5 * v * v
    G[0, 2] = amp * k * c_avg
    G[0, 3] = v * amp * k * c_avg
    cfg = O.make_cfg(2, (n, ny), h, bc=0, mu=mu)
    dt = O.cfl_dt(cfg, W, 0.4)
    nsteps = int(round(t_end / dt))
    s = _solver(2, (n, ny), h, 0, precision=precision, mu=mu)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    for _ in range(nsteps):
        s.step(dt)
    s.get_state(Wd, Gd)
    Wn = Wd.cpu().numpy()
    got = 2 * np.mean((Wn[2] / Wn[0]).mean(axis=0) * np.sin(k * x)) / (math.sin(k * h / 2) / (k * h / 2))
    want = amp * math.exp(-mu * k * k * nsteps * dt)
    assert abs(got / want - 1) <= 5e-4, (got, want)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_taylor_green_decay(precision):
    """Taylor-Green vortex on 32^3 cells, Re = 100 (L0 = 2 pi), t = 0.1:
    E_k(t) / E_k(0) = exp(-6 nu t) (single Stokes mode, energy-conserving
    inviscid dynamics), through gks_step_cfl."""
    from paper_2507_20461_gb300 import inputs as I

    n, mu, cfl = 32, 2 * math.pi / 100, 0.4
    W, G, h = I.taylor_green_3d(n)
    cfg = O.make_cfg(3, (n, n, n), h, bc=0, mu=mu)
    dt = O.cfl_dt(cfg, W, cfl)
    nsteps = 10
    s = B.Solver((n, n, n), lo=[-math.pi] * 3, hi=[math.pi] * 3, bc=B.BC_PERIODIC, precision=precision, mu=mu)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    for _ in range(nsteps):
        s.step(dt)
    s.get_state(Wd, Gd)
    Wn = Wd.cpu().numpy()

    def ek(W):
        return float(np.mean(0.5 * (W[1] ** 2 + W[2] ** 2 + W[3] ** 2) / W[0]))

    ratio = ek(Wn) / ek(W)
    want = math.exp(-6 * mu * nsteps * dt)
    assert abs(ratio / want - 1) <= 3e-4, (ratio, want)
    s.close()


def test_viscous_shock_tube():
    """Viscous shock tube (Sec. 6.9), 80 x 40 cells, no-slip walls on three
    sides and a slip symmetry line on top, mu = 0.005: ten FP64 steps match the
    oracle step by step; FP64 and mixed runs of 80 CFL steps stay admissible
    and conserve mass (closed box)."""
    from paper_2507_20461_gb300 import inputs as I

    nx, mu = 80, 0.005
    sides = (3, 3, 3, 2, 0, 0)
    W, G, h = I.viscous_shock_tube(nx)
    n = (nx, nx // 2)
    cfg = O.make_cfg(2, n, h, bc=sides, mu=mu)
    s = B.Solver(n, lo=[0, 0], hi=[1.0, 0.5], bc=sides, precision=0, mu=mu)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    Wo, Go = W.copy(), G.copy()
    for _ in range(10):
        dt = O.cfl_dt(cfg, Wo, 0.4)
        assert O.step(cfg, dt, Wo, Go) == 0
        s.step(dt)
    s.get_state(Wd, Gd)
    assert _rel_l1(Wd.cpu().numpy(), Wo).max() <= 1e-11
    s.close()
    mass0 = W[0].sum()
    for precision in (0, 1):
        s = B.Solver(n, lo=[0, 0], hi=[1.0, 0.5], bc=sides, precision=precision, mu=mu)
        Wd, Gd = _dev(W), _dev(G)
        s.set_state(Wd, Gd)
        s.step_cfl(0.4, 80)
        s.get_state(Wd, Gd)
        rho = Wd.cpu().numpy()[0]
        assert np.isfinite(rho).all() and rho.min() > 0
        assert abs(rho.sum() / mass0 - 1) <= 1e-12
        s.close()
