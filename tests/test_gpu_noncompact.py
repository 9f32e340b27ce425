"""1D non-compact GENO schemes (order 5 and 6, Sec. 4.1) with the HLLC flux
and classical RK4, through the C ABI on cuda:0, against the oracle.

Bars as for the compact path: FP64 face states and fluxes element-wise to
1e-12 of the variable's scale, steps to a relative L1 residual of 1e-12."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2507_20461_gb300 import binding as B
from paper_2507_20461_gb300 import inputs as I

from test_gpu_parity import _dev, _rel_l1

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
GAMMA = 1.4


def _solver(n, h, bc, order, **kw):
    return B.Solver((n,), lo=[0.0], hi=[n * h], gamma=GAMMA, bc=bc, precision=0, order=order, **kw)


def _state(n, seed):
    W, G, h, _ = I.riemann_1d(n, seed=seed)
    rng = np.random.default_rng(seed)
    W = W * (1 + 0.02 * rng.random(W.shape))
    return np.ascontiguousarray(W), np.zeros_like(G), h


@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("order", [5, 6])
def test_states_and_fluxes(order, bc):
    n = 137
    W, G, h = _state(n, 40 + order + bc)
    cfg = O.make_cfg(1, (n,), h, bc=bc)
    ref = O.nc_reconstruct(cfg, order, W)
    s = _solver(n, h, bc, order)
    s.set_state(_dev(W), _dev(G))
    out = torch.zeros(2 * 3 * 2 * (n + 1), dtype=torch.float64, device=DEV)
    s.reconstruct(out)
    got = out.cpu().numpy().reshape(2, 3, 2, n + 1)
    for v in range(3):
        scale = np.abs(W[v]).max()
        np.testing.assert_allclose(got[:, v, 0], ref[:, v], rtol=0, atol=1e-12 * scale)
        assert np.all(got[:, v, 1] == 0.0)
    Fref = O.nc_flux(cfg, order, W)
    ff = torch.zeros(3 * 3 * (n + 1), dtype=torch.float64, device=DEV)
    s.flux(1e-3, ff)
    F = ff.cpu().numpy().reshape(3, 3, n + 1)
    for v in range(3):
        np.testing.assert_allclose(F[0, v], Fref[v], rtol=0, atol=1e-12 * (np.abs(Fref[v]).max() + 1e-300))
    assert np.all(F[1:] == 0.0)
    s.close()


@pytest.mark.parametrize("bc", [0, 1, 2])
@pytest.mark.parametrize("order", [5, 6])
def test_rk4_steps(order, bc):
    """Ten RK4 steps, each compared with the oracle's step from the same state."""
    n = 200
    W, G, h = _state(n, 50 + order + bc)
    cfg = O.make_cfg(1, (n,), h, bc=bc)
    s = _solver(n, h, bc, order)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    Wo = W.copy()
    for _ in range(10):
        dt = 0.4 * h / O.max_wavespeed(cfg, Wo)
        assert O.nc_step(cfg, order, dt, Wo) == 0
        s.step(dt)
        s.get_state(Wd, Gd)
        assert _rel_l1(Wd.cpu().numpy(), Wo).max() <= 1e-12
        Wd.copy_(_dev(Wo))
        s.set_state(Wd, Gd)
    s.close()


def test_step_cfl_and_blast_wave():
    """Woodward-Colella blast wave (Sec. 6.6), N = 400, reflecting walls, CFL
    0.4 through gks_step_cfl: admissible, mass conserved between the walls,
    and the first steps equal the oracle's."""
    n = 400
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    W = np.ascontiguousarray(np.stack([np.ones(n), np.zeros(n), p / (GAMMA - 1)]))
    G = np.zeros((1, 3, n))
    for order in (5, 6):
        cfg = O.make_cfg(1, (n,), h, bc=2)
        s = _solver(n, h, 2, order)
        Wd, Gd = _dev(W), _dev(G)
        s.set_state(Wd, Gd)
        Wo = W.copy()
        for _ in range(3):
            dt = 0.4 * h / O.max_wavespeed(cfg, Wo)
            assert O.nc_step(cfg, order, dt, Wo) == 0
        s.step_cfl(0.4, 3)
        s.get_state(Wd, Gd)
        assert _rel_l1(Wd.cpu().numpy(), Wo).max() <= 1e-11
        s.step_cfl(0.4, 1600)
        s.get_state(Wd, Gd)
        rho = Wd.cpu().numpy()[0]
        assert rho.min() > 0 and abs(rho.sum() * h - 1.0) < 1e-12
        s.close()


def _gauss_avgs(n, L, x0, b, t):
    """cell averages of 1 + 0.5 exp(-ln2 (x - t)^2 / b^2) on a periodic [x0, x0 + L)"""
    h = L / n
    edges = x0 + np.arange(n + 1) * h
    k = math.sqrt(math.log(2.0)) / b
    from scipy.special import erf

    out = np.zeros(n)
    for shift in (-L, 0.0, L):
        c = t + shift
        out += 0.5 * (math.sqrt(math.pi) / (2 * k)) * (erf(k * (edges[1:] - c)) - erf(k * (edges[:-1] - c))) / h
    return 1.0 + out


def test_entropy_wave_long_run():
    """Entropy wave (Sec. 6.2): rho = 1 + 0.5 exp(-ln2 x^2 / b^2), b = 1.5,
    u = 1, p = 1 on [-800, 1000] with 1800 cells, t = 400 (about 133 periods
    of the 2b-wide wave), CFL 0.4.  The compact 8th-order GKS and the
    non-compact 6th-order scheme, both with GENO, keep the wave (L1 below
    1e-3 of the exact averages, no new extrema); the linear compact scheme
    (chi = 1) does not: GENO is what keeps the long run bounded.  (The paper
    also reports the compact scheme more accurate than the non-compact one;
    under the readings here it is not: 9.3e-4 against 5.9e-4.)"""
    n, L, x0, b, t_end = 1800, 1800.0, -800.0, 1.5, 400.0
    h = L / n
    rho = _gauss_avgs(n, L, x0, b, 0.0)
    edges = x0 + np.arange(n + 1) * h
    # averaged derivative of rho: (rho(x_{j+1/2}) - rho(x_{j-1/2})) / h
    pt = 1.0 + 0.5 * np.exp(-math.log(2.0) * edges**2 / b**2)
    drho = (pt[1:] - pt[:-1]) / h
    W = np.ascontiguousarray(np.stack([rho, rho, 1.0 / (GAMMA - 1) + 0.5 * rho]))
    G = np.ascontiguousarray(np.stack([drho, drho, 0.5 * drho])[None])
    exact = _gauss_avgs(n, L, x0, b, t_end)
    err, peak = {}, {}
    for order, lim in ((8, 0), (6, 0), (8, 1)):
        s = B.Solver((n,), lo=[x0], hi=[x0 + L], gamma=GAMMA, bc=B.BC_PERIODIC, precision=0, order=order, limiter=lim)
        Wd, Gd = _dev(W), _dev(G)
        s.set_state(Wd, Gd)
        t = 0.0
        while t < t_end - 1e-9:
            dt = min(0.4 * h / s.max_wavespeed(), t_end - t)
            s.step(dt)
            t += dt
        s.get_state(Wd, Gd)
        r = Wd.cpu().numpy()[0]
        err[(order, lim)] = np.abs(r - exact).mean()
        peak[(order, lim)] = r.max()
        assert abs(r.sum() / rho.sum() - 1) <= 1e-13
        s.close()
    for key in ((8, 0), (6, 0)):
        assert err[key] < 1e-3 and peak[key] < 1.5, (key, err, peak)
    assert err[(8, 0)] < err[(8, 1)] and peak[(8, 1)] > 1.5, (err, peak)
