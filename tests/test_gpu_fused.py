"""The fused 2D stage kernel (one kernel per stage: reconstruction, flux and
update of a tile in shared memory) against the three-kernel path and the
oracle, on cuda:0.

Both paths run the same FP32 reconstruction and flux formulas and the same
exact face sums and double-float accumulation; only where the intermediate
values live differs.  The compiler fuses multiplies and adds differently in
the two kernels, so the FP32 values differ at rounding level: on smooth
states the averages agree to 1e-6 of their scale after a few steps (one
step moves a cell by about dt/h = 0.3 of an FP32-rounded flux difference)
and the gradients, differences of FP32 interface states over h, to 1e-4 of
|W| / h (the GENO weights amplify rounding differences: the path function's
slope is up to C = 20, and near a wall a few steps of that reach about a
hundred FP32 ulps of an interface state).  A face on a tile edge is evaluated by both tiles that touch it;
the periodic conservation check shows that both evaluations agree (a
difference would leave the summed averages drifting by the FP32 size of
that difference).  The three-kernel path is itself held to the oracle by the mixed-precision
parity tests (test_gpu_parity.py).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_20461_gb300 import binding as B
from paper_2507_20461_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(DEV)


def _state(nx, ny, seed, amp=0.3):
    """Smooth state with a seeded random perturbation, non-zero gradients."""
    rng = np.random.default_rng(seed)
    h = 1.0 / max(nx, ny)
    y, x = np.meshgrid((np.arange(ny) + 0.5) * h, (np.arange(nx) + 0.5) * h, indexing="ij")
    ph = x + 2 * y
    rho = 1.0 + amp * np.sin(2 * math.pi * ph) + 0.05 * rng.random(x.shape)
    u = 0.3 * np.cos(2 * math.pi * ph) + 0.05 * rng.random(x.shape)
    v = 0.2 * np.sin(2 * math.pi * (x - y)) + 0.05 * rng.random(x.shape)
    p = 1.0 + 0.2 * np.cos(2 * math.pi * ph) + 0.05 * rng.random(x.shape)
    W = np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])
    G = 0.3 * rng.normal(size=(2,) + W.shape)
    return W, G, h


def _agree(a, b, W, h):
    """the two paths' (W, G) after the same steps, within FP32 rounding"""
    sc = np.abs(W).max()  # the flux terms are of the size of the largest variable
    np.testing.assert_allclose(a[0], b[0], rtol=0, atol=1e-6 * sc)
    np.testing.assert_allclose(a[1], b[1], rtol=0, atol=1e-4 * sc / h)


def _run(W, G, h, steps, stage_kernels, bc=B.BC_PERIODIC, limiter=0, mu=0.0, cfl=0.4):
    """bc: one type for every side, or six (x lo, x hi, y lo, y hi, z lo, z hi)."""
    ny, nx = W.shape[1:]
    kw = dict(mu=mu) if mu else {}
    s = B.Solver((nx, ny), lo=[0, 0], hi=[nx * h, ny * h], bc=bc, precision=1, limiter=limiter,
                 stage_kernels=stage_kernels, **kw)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    s.step_cfl(cfl, steps)
    s.get_state(Wd, Gd)
    st = s.status()
    s.close()
    return Wd.cpu().numpy(), Gd.cpu().numpy(), st


@pytest.mark.parametrize("nx,ny", [(32, 8), (37, 29), (64, 64), (100, 17), (5, 3), (1, 9), (33, 1), (130, 70)])
@pytest.mark.parametrize("bc", [B.BC_PERIODIC, B.BC_TRANSMISSIVE, B.BC_REFLECTIVE, B.BC_NOSLIP])
def test_fused_equals_three_kernel_path(nx, ny, bc):
    """Tiles smaller than, equal to and ragged against the 32 x 8 tile, grids
    one cell wide (ghosts mirrored or wrapped several times), every boundary
    type: the fused stage kernel agrees with the three-kernel path."""
    W, G, h = _state(nx, ny, 100 + nx + 7 * ny + bc)
    a = _run(W, G, h, 4, 1, bc=bc)
    b = _run(W, G, h, 4, 0, bc=bc)
    assert a[2] == b[2] == 0
    _agree(a, b, W, h)


@pytest.mark.parametrize("sides", [[B.BC_NOSLIP, B.BC_REFLECTIVE, 0, 0, 0, 0], [1, 1, B.BC_NOSLIP, B.BC_REFLECTIVE, 0, 0]])
def test_fused_equals_three_kernel_path_per_side(sides):
    """Different walls on the two sides of an axis, periodic across."""
    W, G, h = _state(70, 45, 3)
    a = _run(W, G, h, 4, 1, bc=sides)
    b = _run(W, G, h, 4, 0, bc=sides)
    _agree(a, b, W, h)


def _smooth_exact(nx, ny, seed):
    """A smooth periodic state with its exact cell-averaged gradients (the
    point values and derivatives at cell centres): no weight sits at a cut."""
    rng = np.random.default_rng(seed)
    h = 1.0 / max(nx, ny)
    y, x = np.meshgrid((np.arange(ny) + 0.5) / ny, (np.arange(nx) + 0.5) / nx, indexing="ij")
    a = rng.uniform(0, 2 * np.pi)
    k = 2 * np.pi
    ph = k * (x + y) + a
    rho, drho = 1 + 0.2 * np.sin(ph), 0.2 * np.cos(ph)
    u, du = 0.3 * np.cos(ph), -0.3 * np.sin(ph)
    v, dv = 0.2 * np.sin(ph), 0.2 * np.cos(ph)
    p, dp = 1 + 0.1 * np.cos(ph), -0.1 * np.sin(ph)
    W = np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])
    dW = np.stack([drho, drho * u + rho * du, drho * v + rho * dv,
                   dp / 0.4 + 0.5 * drho * (u * u + v * v) + rho * (u * du + v * dv)])
    G = np.stack([k * dW, k * dW])  # d/dx = d/dy = k d/dph
    return W, G, 1.0 / nx


@pytest.mark.parametrize("limiter", [1, 2, 3])
def test_fused_equals_three_kernel_path_limiters(limiter):
    """GENO (tested above), the linear scheme and WENO-Z on a noisy state;
    TENO on a smooth state with exact gradients, because its cut is a switch:
    on noisy data a rounding-level difference between the two kernels can
    drop a candidate in one and keep it in the other."""
    if limiter == 3:
        W, G, h = _smooth_exact(48, 48, 11)
    else:
        W, G, h = _state(45, 38, 7 + limiter)
    a = _run(W, G, h, 5, 1, limiter=limiter)
    b = _run(W, G, h, 5, 0, limiter=limiter)
    _agree(a, b, W, h)


def test_fused_equals_three_kernel_path_navier_stokes():
    W, G, h = _state(48, 40, 21)
    a = _run(W, G, h, 5, 1, mu=2e-3, cfl=0.2)
    b = _run(W, G, h, 5, 0, mu=2e-3, cfl=0.2)
    _agree(a, b, W, h)


def test_fused_equals_three_kernel_path_shocks():
    """The 2D 2048^2 workload's recipe at 256^2 (modes + Mach 1.5-3 shocks,
    where the admissibility fallback fires), 10 steps: the density agrees to
    the mixed-precision bar, mean |d rho| <= 1e-5 (a rounding-level
    difference can flip an admissibility decision near its threshold)."""
    W, G, h = I.fourier_shocks_2d(256, 20463)
    a = _run(W, G, h, 10, 1)
    b = _run(W, G, h, 10, 0)
    assert a[2] == b[2] == 0
    err = np.abs(a[0][0] - b[0][0]).mean()
    assert err <= 1e-5, err


def test_fused_against_oracle_20_steps():
    """The 16-mode smooth variant of the 2048^2 workload at 64^2 (drifting
    gas, no admissibility decision near its threshold) through the fused
    kernel against the FP64 oracle, 20 steps: mean |rho - rho_oracle| <= 1e-5,
    the mixed-precision bar."""
    import oracle as O

    n = 64
    W, G, h = I.fourier_shocks_2d(n, seed=20463, nshocks=0, drift=(0.5, 0.25))
    cfg = O.make_cfg(2, (n, n), h, bc=0)
    s = B.Solver((n, n), bc=B.BC_PERIODIC, precision=1, stage_kernels=1)
    Wd, Gd = _dev(W), _dev(G)
    s.set_state(Wd, Gd)
    Wo, Go = W.copy(), G.copy()
    for _ in range(20):
        dt = 0.4 * h / O.max_wavespeed(cfg, Wo)
        assert O.step(cfg, dt, Wo, Go) == 0
        s.step(dt)
    s.get_state(Wd, Gd)
    assert s.status() == 0
    s.close()
    err = np.abs(Wd.cpu().numpy()[0] - Wo[0]).mean()
    assert err <= 1e-5, err


def test_fused_conserves_periodic_sums():
    """Periodic 200 x 120 (ragged against the tile), 40 CFL steps: every
    summed conserved variable keeps its value to 1e-13 of its scale."""
    W, G, h = _state(200, 120, 5)
    W1, _, st = _run(W, G, h, 40, 1)
    assert st == 0
    s0 = W.sum(axis=(1, 2))
    s1 = W1.sum(axis=(1, 2))
    scale = np.abs(W).sum(axis=(1, 2))
    assert np.all(np.abs(s1 - s0) <= 1e-13 * scale), (s1 - s0) / scale
