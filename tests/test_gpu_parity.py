"""Parity of the CUDA library (through its C ABI) with the oracle, on cuda:0.

Bars (the tolerances are written in each test, with the arithmetic behind them):
  - FP64 interface states and fluxes: element-wise, relative 1e-12 of the
    variable's scale (values) and 1e-10 (derivatives, time derivatives);
  - FP64 one step: per-variable relative L1 residual <= 1e-12;
  - FP64 after a full run: relative L1 <= 1e-9 per variable;
  - mixed precision (FP32 reconstruction/flux, FP64 accumulation): mean
    |rho_gpu - rho_oracle| <= 1e-5 where no admissibility decision sits
    within FP32 rounding of its threshold, and on the 2048^2 workload.
Sizes span several thread blocks and a ragged tail; the full-size cases use
the launch path the benchmark times (gks_step_cfl) and compare sampled
windows, whose centres depend on nothing outside the window.
"""
import functools
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2507_20461_gb300 import binding as B
from paper_2507_20461_gb300 import inputs as I

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _random_smooth(dim, n, seed, bc):
    """Smooth state with a random perturbation of the averages and gradients."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(n))
    h = 1.0 / n[0]
    grids = np.meshgrid(*[(np.arange(k) + 0.5) * h for k in reversed(n)], indexing="ij")
    phase = sum((a + 1) * g for a, g in enumerate(reversed(grids)))
    rho = 1.0 + 0.3 * np.sin(2 * math.pi * phase) + 0.05 * rng.random(shape)
    vel = [0.3 * np.cos(2 * math.pi * (phase + 0.1 * a)) + 0.05 * rng.random(shape) for a in range(dim)]
    p = 1.0 + 0.2 * np.cos(2 * math.pi * phase) + 0.05 * rng.random(shape)
    ke = sum(u * u for u in vel)
    W = np.stack([rho] + [rho * u for u in vel] + [p / 0.4 + 0.5 * rho * ke])
    G = 0.5 * rng.normal(size=(dim,) + W.shape)
    return W, G, h


def _solver(dim, n, h, bc, precision=0, **kw):
    hi = [k * h for k in n]
    return B.Solver(tuple(n), lo=[0.0] * dim, hi=hi, gamma=1.4, bc=bc, precision=precision, **kw)


CASES = [
    (1, (53,)),
    (2, (37, 29)),
    (3, (11, 9, 7)),
]


@pytest.mark.parametrize("bc", [0, 1, 2, 3])
@pytest.mark.parametrize("dim,n", CASES)
def test_reconstruct_parity(dim, n, bc):
    W, G, h = _random_smooth(dim, n, 1 + dim, bc)
    cfg = O.make_cfg(dim, n, h, bc=bc)
    ref = O.reconstruct(cfg, W, G)
    s = _solver(dim, n, h, bc)
    s.set_state(_dev(W), _dev(G))
    out = torch.zeros(ref.size, dtype=torch.float64, device=DEV)
    s.reconstruct(out)
    got = out.cpu().numpy().reshape(ref.shape)
    nv = dim + 2
    for v in range(nv):
        scale = np.abs(W[v]).max() + 1e-300
        np.testing.assert_allclose(got[:, v, 0], ref[:, v, 0], rtol=0, atol=1e-12 * scale)
        dscale = np.abs(ref[:, v, 1:]).max() + scale / h
        np.testing.assert_allclose(got[:, v, 1:], ref[:, v, 1:], rtol=0, atol=1e-11 * dscale)
    s.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_fallback_states_parity(precision):
    """The admissibility fallback in both branches: the oracle tests' state
    where every candidate polynomial carries the same steep slope, at
    thresholds 0.3 and 0.6 (about a thousand replaced states each, and the
    kept states' margins of at least 10% decide alike in FP32).  The GPU
    replaces exactly the states the oracle does, and the values agree
    element-wise (FP64: 1e-12 of the scale; mixed: FP32 rounding)."""
    from test_oracle_admissibility import _steep_gradient

    n = (24, 20)
    W, G, h = _steep_gradient(n)
    for delta in (0.3, 0.6):
        ref = O.reconstruct(O.make_cfg(2, n, h, bc=0, adm_delta=delta), W, G)
        s = _solver(2, n, h, 0, precision=precision, adm_delta=delta)
        s.set_state(_dev(W), _dev(G))
        out = torch.zeros(ref.size, dtype=torch.float64, device=DEV)
        s.reconstruct(out)
        got = out.cpu().numpy().reshape(ref.shape)
        s.close()
        # replaced states: zero slopes in every variable
        ref_fb = np.all(ref[:, :, 1:] == 0.0, axis=(1, 2))
        got_fb = np.all(got[:, :, 1:] == 0.0, axis=(1, 2))
        assert ref_fb.sum() >= 1000 and np.array_equal(got_fb, ref_fb)
        tol = 1e-12 if precision == 0 else 2e-6
        for v in range(4):
            scale = np.abs(W[v]).max()
            np.testing.assert_allclose(got[:, v, 0], ref[:, v, 0], rtol=0, atol=tol * scale)
            dscale = np.abs(ref[:, v, 1:]).max() + scale / h
            np.testing.assert_allclose(got[:, v, 1:], ref[:, v, 1:], rtol=0, atol=10 * tol * dscale)


@pytest.mark.parametrize("dim,n", CASES)
def test_flux_parity(dim, n):
    bc = 1
    W, G, h = _random_smooth(dim, n, 10 + dim, bc)
    cfg = O.make_cfg(dim, n, h, bc=bc)
    dt = 0.3 * h / O.max_wavespeed(cfg, W)
    ref = O.flux(cfg, dt, W, G)
    s = _solver(dim, n, h, bc)
    s.set_state(_dev(W), _dev(G))
    out = torch.zeros(ref.size, dtype=torch.float64, device=DEV)
    s.flux(dt, out)
    got = out.cpu().numpy().reshape(ref.shape)
    for v in range(dim + 2):
        Fs = np.abs(ref[0, v]).max() + 1e-300
        np.testing.assert_allclose(got[0, v], ref[0, v], rtol=0, atol=1e-12 * Fs)
        # dF/dt: recovered from time integrals, oracle rounding ~ eps |F| / dt
        np.testing.assert_allclose(got[1, v], ref[1, v], rtol=0, atol=1e-10 * (np.abs(ref[1, v]).max() + Fs / dt))
        np.testing.assert_allclose(got[2, v], ref[2, v], rtol=0, atol=1e-12 * (np.abs(ref[2, v]).max() + 1e-300))
    s.close()


def _rel_l1(a, b):
    nv = a.shape[0]
    return np.array([np.abs(a[v] - b[v]).sum() / (np.abs(b[v]).sum() + 1e-300) for v in range(nv)])


@pytest.mark.parametrize("bc", [0, 1, 2, 3])
@pytest.mark.parametrize("dim,n", CASES)
def test_one_step_parity(dim, n, bc):
    W, G, h = _random_smooth(dim, n, 20 + dim, bc)
    cfg = O.make_cfg(dim, n, h, bc=bc)
    dt = 0.4 * h / O.max_wavespeed(cfg, W)
    Wo, Go = W.copy(), G.copy()
    assert O.step(cfg, dt, Wo, Go) == 0
    s = _solver(dim, n, h, bc)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    s.step(dt)
    s.get_state(Wd, Gd)
    Wg, Gg = Wd.cpu().numpy(), Gd.cpu().numpy()
    assert _rel_l1(Wg, Wo).max() <= 1e-12
    for d in range(dim):
        np.testing.assert_allclose(Gg[d], Go[d], rtol=0, atol=1e-9 * np.abs(Go[d]).max())
    s.close()


def _run_pair(dim, n, h, bc, W, G, nsteps, cfl=0.4, precision=0, stage_kernels=0):
    """nsteps on both sides with the oracle's CFL time steps fed to the GPU."""
    cfg = O.make_cfg(dim, n, h, bc=bc)
    s = _solver(dim, n, h, bc, precision=precision, stage_kernels=stage_kernels)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    Wo, Go = W.copy(), G.copy()
    for _ in range(nsteps):
        dt = cfl * h / O.max_wavespeed(cfg, Wo)
        assert O.step(cfg, dt, Wo, Go) == 0
        s.step(dt)
    s.get_state(Wd, Gd)
    out = (Wd.cpu().numpy(), Gd.cpu().numpy(), Wo, Go)
    s.close()
    return out


def test_config1_full_run_parity():
    """1D Euler, gamma 1.4, N = 400 on [0, 1], seeded two-state Riemann IC,
    transmissive, CFL 0.4, 200 steps.

    GENO's nonlinear weights amplify rounding differences on this run (about
    e^0.14 per step after the discontinuities interact; the linear scheme does
    not), so no two implementations that round differently can agree to 1e-9
    after 200 steps.  The bar is therefore relative to the oracle's own
    sensitivity: the GPU-oracle difference must not exceed 10x the difference
    between two oracle runs whose initial states differ by 1e-14 relative, and
    the first 40 steps (before the amplification) must agree to 1e-10."""
    n = 400
    W, G, h, _ = I.riemann_1d(n, seed=20461)
    Wg40, _, Wo40, _ = _run_pair(1, (n,), h, 1, W, G, 40)
    assert _rel_l1(Wg40, Wo40).max() <= 1e-10
    Wg, Gg, Wo, Go = _run_pair(1, (n,), h, 1, W, G, 200)
    # oracle sensitivity to a 1e-14 relative perturbation of the initial state
    cfg = O.make_cfg(1, (n,), h, bc=1)
    Wp = W * (1 + 1e-14 * np.sin(np.arange(n)))
    Gp = G.copy()
    Wr = W.copy()
    Gr = G.copy()
    for _ in range(200):
        dt = 0.4 * h / O.max_wavespeed(cfg, Wr)
        assert O.step(cfg, dt, Wr, Gr) == 0
        assert O.step(cfg, dt, Wp, Gp) == 0
    sens = _rel_l1(Wp, Wr)
    gap = _rel_l1(Wg, Wo)
    assert (gap <= 10 * sens + 1e-12).all(), (gap, sens)


def test_2d_quadrants_multistep_parity():
    """Config-2-type four-quadrant IC (transmissive) on a ragged 45 x 38 grid, 25 steps."""
    W, G, h = I.quadrants_2d(38, seed=20462, nx=45)
    Wg, Gg, Wo, Go = _run_pair(2, (45, 38), h, 1, W, G, 25)
    assert _rel_l1(Wg, Wo).max() <= 1e-9


def test_3d_multistep_parity():
    W, G, h = I.turbulence_3d(12, seed=20465)
    Wg, Gg, Wo, Go = _run_pair(3, (12, 12, 12), h, 0, W, G, 4)
    assert _rel_l1(Wg, Wo).max() <= 1e-10


# Mixed precision against the FP64 oracle.  The admissibility fallback
# (reading R9) is a switch on rho and p of each reconstructed face state
# relative to its cell, and the mixed path decides it on FP32 face states.
# Where a face sits within FP32 rounding of the threshold the two paths may
# decide differently, and the run then moves by O(1e-3) around that face.
# The 1e-5 bar is therefore applied to cases that the oracle tests pin as
# having no decision within 3e-3 of its threshold
# (test_oracle_conditioning.py); the shock case, which has decisions within
# 1e-4, is held to the oracle's own spread under such a change of the
# threshold; the full-size workload carries the bar over 4 M cells.
MIXED_SMOOTH_2D = dict(n=64, seed=20463, nshocks=0, drift=(0.5, 0.25))


# the 2D mixed-precision step runs either as three kernels (stage_kernels 0)
# or as the fused stage kernel (1); the mixed-precision bars hold for both
SK = [0, 1]


@pytest.mark.parametrize("sk", SK)
@pytest.mark.parametrize("case", ["fourier_smooth_2d", "riemann_1d"])
def test_mixed_precision_density_l1(case, sk):
    """FP32 reconstruction/flux with FP64 accumulation against the FP64 oracle,
    20 steps: mean |rho_gpu - rho_oracle| <= 1e-5."""
    if case == "riemann_1d" and sk:
        pytest.skip("the fused stage kernel is 2D")
    if case == "fourier_smooth_2d":
        c = MIXED_SMOOTH_2D
        W, G, h = I.fourier_shocks_2d(c["n"], seed=c["seed"], nshocks=c["nshocks"], drift=c["drift"])
        dim, n, bc = 2, (c["n"], c["n"]), 0
    else:
        W, G, h, _ = I.riemann_1d(200, seed=20461)
        dim, n, bc = 1, (200,), 1
    Wg, Gg, Wo, Go = _run_pair(dim, n, h, bc, W, G, 20, precision=1, stage_kernels=sk)
    err = np.abs(Wg[0] - Wo[0]).mean()
    assert err <= 1e-5, err


@pytest.mark.parametrize("sk", SK)
def test_mixed_precision_shock_case_within_switch_spread(sk):
    """64^2 Fourier modes + 4 shocks, 20 steps: the mixed result lies within
    1e-5 of the oracle plus the oracle's own spread when the admissibility
    threshold moves by a relative 1e-4 (the FP32 face states' rounding)."""
    n = 64
    W, G, h = I.fourier_shocks_2d(n, seed=20463)
    Wg, Gg, Wo, Go = _run_pair(2, (n, n), h, 0, W, G, 20, precision=1, stage_kernels=sk)
    spread = 0.0
    for r in (-1e-4, 1e-4):
        cfg = O.make_cfg(2, (n, n), h, bc=0, adm_delta=0.3 * (1 + r))
        Wp, Gp = W.copy(), G.copy()
        for _ in range(20):
            dt = 0.4 * h / O.max_wavespeed(cfg, Wp)
            assert O.step(cfg, dt, Wp, Gp) == 0
        spread = max(spread, np.abs(Wp[0] - Wo[0]).mean())
    err = np.abs(Wg[0] - Wo[0]).mean()
    assert err <= 1e-5 + spread, (err, spread)


def _window_check(Wfull, Gfull, Wnew, Gnew, dim, n, h, dt, rng, nwin=6, r=4, pad=4, tol=1e-12, per_var=False,
                  **cfg_kw):
    """Oracle step on (2(r+pad)+1)^dim windows around random cells of a periodic
    grid; the centre (radius pad... 0) is exact because a step reaches r cells.
    per_var: scale each variable's tolerances by its own magnitude in the
    window, the momenta by the momentum vector's (else all by the largest).  cfg_kw: further oracle options (mu for the
    Navier-Stokes path)."""
    w = 2 * (r + pad) + 1
    for _ in range(nwin):
        c = [int(rng.integers(0, k)) for k in n]
        idx = [np.arange(ci - r - pad, ci + r + pad + 1) % k for ci, k in zip(c, n)]
        sl = np.ix_(*reversed(idx))
        Ww = np.ascontiguousarray(Wfull[(slice(None),) + sl])
        Gw = np.ascontiguousarray(Gfull[(slice(None), slice(None)) + sl])
        cfg = O.make_cfg(dim, (w,) * dim, h, bc=1, **cfg_kw)
        assert O.step(cfg, dt, Ww, Gw) == 0
        ctr = (r + pad,) * dim
        ref_w = Ww[(slice(None),) + ctr]
        got_w = Wnew[(slice(None),) + tuple(reversed(c))]
        np.testing.assert_allclose(got_w, ref_w, rtol=tol, atol=tol)
        ref_g = Gw[(slice(None), slice(None)) + ctr]
        got_g = Gnew[(slice(None), slice(None)) + tuple(reversed(c))]
        # gradients are differences of interface states over h: tolerance tol |W| / h
        geps = 1e-9 if tol < 1e-9 else tol
        if per_var:
            nv = ref_w.shape[0]
            for v in range(nv):
                # a momentum component's rounding is at the scale of the momentum
                # vector (the moments mix the components), so the momenta share one
                wscale = np.abs(Ww[1:nv - 1]).max() if 1 <= v <= nv - 2 else np.abs(Ww[v]).max()
                np.testing.assert_allclose(got_g[:, v], ref_g[:, v], rtol=0,
                                           atol=geps * wscale / h + 1e-9 * np.abs(ref_g[:, v]).max())
        else:
            gtol = geps * (np.abs(ref_w).max() / h)
            np.testing.assert_allclose(got_g, ref_g, rtol=0, atol=gtol + 1e-9 * np.abs(ref_g).max())


@pytest.mark.parametrize("precision,tol,sk", [(0, 1e-12, 0), (1, 2e-5, 0), (1, 2e-5, 1)])
def test_config3_full_size_sampled(precision, tol, sk):
    """2D 2048^2 periodic Fourier modes + 4 shocks (the benchmark workload),
    one step through gks_step_cfl (dt computed on the device); sampled windows
    compared with the oracle."""
    n = 2048
    W, G, h = I.fourier_shocks_2d(n, seed=20463)
    s = _solver(2, (n, n), h, 0, precision=precision, stage_kernels=sk)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    smax = s.max_wavespeed()
    cfg = O.make_cfg(2, (8, 8), h)
    dt = 0.4 * h / smax
    s.step_cfl(0.4, 1)
    s.get_state(Wd, Gd)
    Wn, Gn = Wd.cpu().numpy(), Gd.cpu().numpy()
    rng = np.random.default_rng(5)
    _window_check(W, G, Wn, Gn, 2, (n, n), h, dt, rng, tol=tol)
    s.close()


@pytest.mark.parametrize("sk", SK)
def test_config3_mixed_l1_full_size(sk):
    """The mixed-precision bar on the workload it is stated for: 2048^2
    periodic Fourier modes + 4 shocks, 20 steps with the same time steps on
    the mixed and the FP64 path (the FP64 path matches the oracle to 1e-12
    per step, test_config3_full_size_sampled): mean |d rho| <= 1e-5.

    20 steps, because the colliding shocks amplify rounding-level
    differences by about e^0.3 per step: the FP64 path started from an input
    perturbed by a relative 2^-24 leaves its unperturbed run by 1.6e-6 at
    step 20 and by 3.4e-4 at step 100, where no FP32 pipeline can meet
    1e-5."""
    n = 2048
    W, G, h = I.fourier_shocks_2d(n, seed=20463)
    s64 = _solver(2, (n, n), h, 0, precision=0)
    s32 = _solver(2, (n, n), h, 0, precision=1, stage_kernels=sk)
    W64, G64 = _dev(W), _dev(G)
    W32, G32 = _dev(W), _dev(G)
    s64.set_state(W64, G64)
    s32.set_state(W32, G32)
    for _ in range(20):
        dt = 0.4 * h / s64.max_wavespeed()
        s64.step(dt)
        s32.step(dt)
    s64.get_state(W64, G64)
    s32.get_state(W32, G32)
    err = (W32[0] - W64[0]).abs().mean().item()
    s64.close()
    s32.close()
    assert err <= 1e-5, err


@functools.lru_cache(maxsize=2)
def _ics_3d(case):
    if case == "turbulence":
        W, G, h = I.turbulence_3d(256, seed=20465)
        return W, G, h, [0.0] * 3, [1.0] * 3, 0.0
    W, G, h = I.taylor_green_3d(256)
    return W, G, h, [-math.pi] * 3, [math.pi] * 3, 2 * math.pi / 1600.0


@pytest.mark.parametrize("case,precision,tol", [("turbulence", 1, 2e-5), ("turbulence", 0, 1e-12),
                                                ("taylor_green", 1, 2e-5)])
def test_3d_full_size_sampled(case, precision, tol):
    """The 3D workloads the benchmark times, at full size (256^3 periodic):
    the solenoidal turbulence field (Euler; one step through gks_step_cfl,
    dt computed on the device) and the Taylor-Green vortex (Navier-Stokes,
    Re 1600; one step of the oracle's CFL time step).  Sampled 17^3 windows
    compared with the oracle."""
    n = 256
    W, G, h, lo, hi, mu = _ics_3d(case)
    s = B.Solver((n, n, n), lo=lo, hi=hi, gamma=1.4, bc=B.BC_PERIODIC, precision=precision, mu=mu)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    if mu == 0.0:
        dt = 0.4 * h / s.max_wavespeed()
        s.step_cfl(0.4, 1)
    else:
        dt = O.cfl_dt(O.make_cfg(3, (n, n, n), h, bc=0, mu=mu), W, 0.4)
        s.step(dt)
    s.get_state(Wd, Gd)
    assert s.status() == 0
    Wn, Gn = Wd.cpu().numpy(), Gd.cpu().numpy()
    s.close()
    del Wd, Gd
    rng = np.random.default_rng(11)
    _window_check(W, G, Wn, Gn, 3, (n, n, n), h, dt, rng, nwin=3, tol=tol, per_var=True, mu=mu)


def test_config2_full_size_sampled():
    """2D 512^2 four-quadrant IC (transmissive), one FP64 step at full size, windows
    away from the boundary compared with the oracle; plus 100 steps stay admissible."""
    n = 512
    W, G, h = I.quadrants_2d(n, seed=20462)
    s = _solver(2, (n, n), h, 1)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    dt = 0.4 * h / s.max_wavespeed()
    s.step(dt)
    s.get_state(Wd, Gd)
    Wn, Gn = Wd.cpu().numpy(), Gd.cpu().numpy()
    rng = np.random.default_rng(6)
    # windows around the quadrant corner and interfaces (all interior, >= 9 cells from the edge)
    for c in ([256, 256], [255, 300], [100, 256], [256, 40], [300, 470]):
        r, pad = 4, 4
        idx = [np.arange(ci - r - pad, ci + r + pad + 1) for ci in c]
        sl = np.ix_(idx[1], idx[0])
        Ww = np.ascontiguousarray(W[(slice(None),) + sl])
        Gw = np.ascontiguousarray(G[(slice(None), slice(None)) + sl])
        cfg = O.make_cfg(2, (17, 17), h, bc=1)
        assert O.step(cfg, dt, Ww, Gw) == 0
        np.testing.assert_allclose(Wn[:, c[1], c[0]], Ww[:, 8, 8], rtol=1e-12, atol=1e-12)
    s.step_cfl(0.4, 100)
    assert s.status() == 0
    s.close()


def test_config2_late_window_multistep():
    """2D 512^2 four-quadrant IC (transmissive, FP64, CFL 0.4 on the device),
    the configuration's 500 steps: the GPU runs steps 1-490, then steps
    491-500 with the time steps it takes read back; the oracle runs the same
    ten steps on 100^2 windows of the step-490 state.  One step moves
    information by at most 4 cells, so the 20^2 centre of a window depends on
    nothing outside it after ten steps; there the GPU's step-500 state agrees
    with the oracle to a relative L1 of 1e-9 per variable (the final-L1 bar)
    and element-wise to 1e-10 of the variable's scale."""
    n = 512
    W, G, h = I.quadrants_2d(n, seed=20462)
    s = _solver(2, (n, n), h, 1)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    s.step_cfl(0.4, 490)
    assert s.status() == 0
    s.get_state(Wd, Gd)
    W490, G490 = Wd.cpu().numpy(), Gd.cpu().numpy()
    dts = []
    for _ in range(10):
        dts.append(0.4 * h / s.max_wavespeed())
        s.step(dts[-1])
    s.get_state(Wd, Gd)
    assert s.status() == 0
    W500 = Wd.cpu().numpy()
    s.close()
    R, C = 50, 10  # window half-width, compared centre half-width
    for cx, cy in ((256, 256), (150, 380)):
        ix = np.arange(cx - R, cx + R)
        iy = np.arange(cy - R, cy + R)
        sl = np.ix_(iy, ix)
        Ww = np.ascontiguousarray(W490[(slice(None),) + sl])
        Gw = np.ascontiguousarray(G490[(slice(None), slice(None)) + sl])
        cfg = O.make_cfg(2, (2 * R, 2 * R), h, bc=1)
        for dt in dts:
            assert O.step(cfg, dt, Ww, Gw) == 0
        got = W500[:, cy - C:cy + C, cx - C:cx + C]
        ref = Ww[:, R - C:R + C, R - C:R + C]
        rel = np.abs(got - ref).sum(axis=(1, 2)) / np.abs(ref).sum(axis=(1, 2))
        assert rel.max() <= 1e-9, rel
        for v in range(4):
            np.testing.assert_allclose(got[v], ref[v], rtol=0, atol=1e-10 * np.abs(ref[v]).max())


def test_free_stream_preserved():
    for dim, n in CASES:
        h = 1.0 / n[0]
        shape = tuple(reversed(n))
        W = np.zeros((dim + 2,) + shape)
        W[0] = 1.3
        for a in range(dim):
            W[1 + a] = 1.3 * (0.2 + 0.1 * a)
        W[dim + 1] = 2.0 / 0.4 + 0.5 * 1.3 * sum((0.2 + 0.1 * a) ** 2 for a in range(dim))
        G = np.zeros((dim,) + W.shape)
        s = _solver(dim, n, h, 0)
        Wd, Gd = _dev(W), _dev(G)
        s.set_state(Wd, Gd)
        for _ in range(3):
            s.step(0.2 * h)
        s.get_state(Wd, Gd)
        np.testing.assert_allclose(Wd.cpu().numpy(), W, rtol=1e-14, atol=1e-14)
        assert np.abs(Gd.cpu().numpy()).max() < 1e-12
        s.close()


def test_periodic_conservation_gpu():
    n = (64, 48)
    W, G, h = _random_smooth(2, n, 31, 0)
    s = _solver(2, n, h, 0)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    s.step_cfl(0.4, 20)
    s.get_state(Wd, Gd)
    Wg = Wd.cpu().numpy()
    np.testing.assert_allclose(Wg.sum(axis=(1, 2)), W.sum(axis=(1, 2)), rtol=1e-13)
    s.close()


def test_tiny_grids():
    """Degenerate sizes: single-cell and two-cell axes run and agree with the oracle."""
    for dim, n, bc in [(1, (2,), 0), (1, (1,), 1), (2, (1, 5), 0), (2, (3, 2), 1), (3, (2, 1, 3), 1)]:
        W, G, h = _random_smooth(dim, n, 40, bc)
        G *= 0.1
        cfg = O.make_cfg(dim, n, h, bc=bc)
        dt = 0.2 * h / O.max_wavespeed(cfg, W)
        Wo, Go = W.copy(), G.copy()
        assert O.step(cfg, dt, Wo, Go) == 0
        s = _solver(dim, n, h, bc)
        Wd, Gd = _dev(W), _dev(G)
        s.set_state(Wd, Gd)
        s.step(dt)
        s.get_state(Wd, Gd)
        assert _rel_l1(Wd.cpu().numpy(), Wo).max() <= 1e-12, (dim, n, bc)
        s.close()


def test_nonphysical_state_reported():
    n = (16, 16)
    W, G, h = _random_smooth(2, n, 50, 0)
    W[3, 5, 5] = 0.1 * W[3, 5, 5] - 10.0  # negative pressure in one cell
    s = _solver(2, n, h, 0)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    s.step(1e-4)
    with pytest.raises(B.GksError) as e:
        s.get_state(Wd, Gd)
    assert e.value.code == B.ERR_NONPHYSICAL
    s.close()


def test_bad_arguments():
    s = _solver(2, (8, 8), 1.0 / 8, 0)
    with pytest.raises(B.GksError) as e:
        s.step(-1.0)
    assert e.value.code == B.ERR_ARG
    with pytest.raises(B.GksError) as e:
        s.step(float("nan"))
    assert e.value.code == B.ERR_ARG
    s.close()


def test_blast_wave_reflective():
    """Woodward-Colella blast wave (Sec. 6.6): rho = 1, u = 0, p = 1000 | 0.01 | 100
    at x < 0.1 | 0.1 <= x < 0.9 | x >= 0.9, reflecting walls, N = 400, t = 0.038.
    FP64 and mixed runs stay admissible; the first steps match the oracle.
    CFL 0.2: without the temporal limiting at strong shocks that the paper
    takes from earlier work (and does not state), the oracle itself loses
    positivity near t = 0.011 at CFL 0.4 and completes at CFL 0.2."""
    n = 400
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    p = np.where(x < 0.1, 1000.0, np.where(x < 0.9, 0.01, 100.0))
    W = np.stack([np.ones(n), np.zeros(n), p / 0.4])
    G = np.zeros((1, 3, n))
    Wg, Gg, Wo, Go = _run_pair(1, (n,), h, 2, W, G, 20, cfl=0.2)
    assert _rel_l1(Wg, Wo).max() <= 1e-10
    for prec in (0, 1):
        s = _solver(1, (n,), h, 2, precision=prec)
        Wd, Gd = _dev(W), _dev(G)
        s.set_state(Wd, Gd)
        t = 0.0
        while t < 0.038 - 1e-12:
            dt = min(0.2 * h / s.max_wavespeed(), 0.038 - t)
            s.step(dt)
            t += dt
        s.get_state(Wd, Gd)
        rho = Wd[0].cpu().numpy()
        assert rho.min() > 0 and np.isfinite(rho).all()
        assert abs(rho.sum() * h - 1.0) < 1e-9  # mass is conserved between reflecting walls
        s.close()


SIDES = [
    (2, (37, 29), (3, 2, 1, 3, 0, 0)),
    (2, (24, 31), (0, 0, 3, 3, 0, 0)),
    (3, (11, 9, 7), (3, 3, 0, 0, 2, 1)),
    (1, (53,), (3, 1, 0, 0, 0, 0)),
]


@pytest.mark.parametrize("dim,n,sides", SIDES)
def test_per_side_bc_parity(dim, n, sides):
    """Boundary conditions chosen per side (geno_gks_create_sides): interface
    states and one FP64 step against the oracle, Euler and Navier-Stokes."""
    W, G, h = _random_smooth(dim, n, 80 + dim, 1)
    cfg = O.make_cfg(dim, n, h, bc=sides)
    ref = O.reconstruct(cfg, W, G)
    s = _solver(dim, n, h, sides)
    s.set_state(_dev(W), _dev(G))
    out = torch.zeros(ref.size, dtype=torch.float64, device=DEV)
    s.reconstruct(out)
    got = out.cpu().numpy().reshape(ref.shape)
    for v in range(dim + 2):
        scale = np.abs(W[v]).max() + 1e-300
        np.testing.assert_allclose(got[:, v, 0], ref[:, v, 0], rtol=0, atol=1e-12 * scale)
    s.close()
    for mu in (0.0, 0.01):
        cfg = O.make_cfg(dim, n, h, bc=sides, mu=mu)
        dt = O.cfl_dt(cfg, W, 0.4)
        Wo, Go = W.copy(), G.copy()
        assert O.step(cfg, dt, Wo, Go) == 0
        s = _solver(dim, n, h, sides, mu=mu)
        Wd, Gd = _dev(W), _dev(G)
        s.set_state(Wd, Gd)
        s.step(dt)
        s.get_state(Wd, Gd)
        assert _rel_l1(Wd.cpu().numpy(), Wo).max() <= 1e-12
        s.close()


def test_per_side_bc_rejects_unpaired_periodic():
    with pytest.raises(B.GksError) as e:
        _solver(2, (8, 8), 1.0 / 8, (0, 1, 1, 1, 0, 0))
    assert e.value.code == B.ERR_ARG


@pytest.mark.parametrize("precision,sk", [(0, 0), (1, 0), (1, 1)])
@pytest.mark.parametrize("dim,n", [(2, (256, 256)), (3, (48, 40, 32))])
def test_conservation_periodic(dim, n, precision, sk):
    """Periodic grids: the summed cell averages of every conserved variable stay
    fixed to FP64 rounding in both precisions (the face fluxes of a cell are
    accumulated exactly, so each face's flux leaves one cell and enters the
    other without a rounding of its own)."""
    if sk and dim != 2:
        pytest.skip("the fused stage kernel is 2D")
    W, G, h = _random_smooth(dim, n, 90 + dim, 0)
    s = _solver(dim, n, h, 0, precision=precision, stage_kernels=sk)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    s.step_cfl(0.4, 40)
    s.get_state(Wd, Gd)
    Wn = Wd.cpu().numpy()
    nv = dim + 2
    ax = tuple(range(1, dim + 1))
    tot0, tot = W.sum(axis=ax), Wn.sum(axis=ax)
    scale = np.abs(W).sum(axis=ax)
    drift = np.abs(tot - tot0) / scale
    assert drift.max() <= 1e-13, drift


@pytest.mark.parametrize("limiter", [2, 3])
@pytest.mark.parametrize("dim,n", CASES)
def test_limiter_variants_parity(dim, n, limiter):
    """WENO-Z (2) and TENO (3) weights: interface states element-wise and one
    FP64 step against the oracle."""
    bc = 1
    W, G, h = _random_smooth(dim, n, 100 + dim, bc)
    cfg = O.make_cfg(dim, n, h, bc=bc, limiter=limiter)
    ref = O.reconstruct(cfg, W, G)
    s = _solver(dim, n, h, bc, limiter=limiter)
    s.set_state(_dev(W), _dev(G))
    out = torch.zeros(ref.size, dtype=torch.float64, device=DEV)
    s.reconstruct(out)
    got = out.cpu().numpy().reshape(ref.shape)
    for v in range(dim + 2):
        scale = np.abs(W[v]).max() + 1e-300
        np.testing.assert_allclose(got[:, v, 0], ref[:, v, 0], rtol=0, atol=1e-12 * scale)
        dscale = np.abs(ref[:, v, 1:]).max() + scale / h
        np.testing.assert_allclose(got[:, v, 1:], ref[:, v, 1:], rtol=0, atol=1e-11 * dscale)
    dt = 0.4 * h / O.max_wavespeed(cfg, W)
    Wo, Go = W.copy(), G.copy()
    assert O.step(cfg, dt, Wo, Go) == 0
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    s.step(dt)
    s.get_state(Wd, Gd)
    assert _rel_l1(Wd.cpu().numpy(), Wo).max() <= 1e-12
    s.close()


@pytest.mark.parametrize("sk", SK)
@pytest.mark.parametrize("limiter", [2, 3])
def test_limiter_variants_mixed(limiter, sk):
    """Mixed precision with WENO-Z / TENO weights, 2D quadrants, 10 steps:
    mean |d rho| against the FP64 oracle within the mixed-precision bar."""
    n = (40, 36)
    W, G, h = I.quadrants_2d(36, seed=31, nx=40)
    cfg = O.make_cfg(2, n, h, bc=1, limiter=limiter)
    s = _solver(2, n, h, 1, precision=1, limiter=limiter, stage_kernels=sk)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    Wo, Go = W.copy(), G.copy()
    for _ in range(10):
        dt = 0.4 * h / O.max_wavespeed(cfg, Wo)
        assert O.step(cfg, dt, Wo, Go) == 0
        s.step(dt)
    s.get_state(Wd, Gd)
    d = np.abs(Wd.cpu().numpy()[0] - Wo[0])
    assert d.mean() <= 1e-5, d.mean()
    s.close()


@pytest.mark.parametrize("sk", SK)
def test_mixed_smooth_flow_tracks_fp64_sensitivity(sk):
    """The 16-mode smooth variant of the 2048^2 workload (no shocks, drifting
    at (0.5, 0.25), periodic) at 256^2 with a fixed time step: the mixed path
    meets the 1e-5 bar after 20 steps (mean |d rho| against the FP64 path,
    which matches the oracle to 1e-12 per step), and after 300 steps stays
    within 3x of the FP64 path's own divergence from an input perturbed by a
    relative 2^-24 (measured 1.3x).  Even this flow amplifies rounding-level
    differences (the linear scheme, chi = 1, amplifies them more than GENO):
    the perturbed FP64 run differs by 3e-8 at step 20 and by 8e-5 at step
    300, so an absolute bar at that horizon would measure the scheme's
    sensitivity, not the precision split."""
    n = 256
    W, G, h = I.fourier_shocks_2d(n, seed=20463, nshocks=0, drift=(0.5, 0.25))
    cfg = O.make_cfg(2, (n, n), h, bc=0)
    dt = 0.35 * h / O.max_wavespeed(cfg, W)
    Wp = W * (1 + 2.0**-24 * np.random.default_rng(3).uniform(-1, 1, size=W.shape))

    def run(W0, prec, skk):
        s = _solver(2, (n, n), h, 0, precision=prec, stage_kernels=skk)
        Wd, Gd = _dev(W0), _dev(G)
        s.set_state(Wd, Gd)
        out = {}
        for k in range(1, 301):
            s.step(dt)
            if k in (20, 300):
                s.get_state(Wd, Gd)
                out[k] = Wd[0].cpu().numpy().copy()
        assert s.status() == 0
        s.close()
        return out

    r64, rmx, rpt = run(W, 0, 0), run(W, 1, sk), run(Wp, 0, 0)
    assert np.abs(rmx[20] - r64[20]).mean() <= 1e-5
    spread = np.abs(rpt[300] - r64[300]).mean()
    assert np.abs(rmx[300] - r64[300]).mean() <= 3.0 * spread, (np.abs(rmx[300] - r64[300]).mean(), spread)
