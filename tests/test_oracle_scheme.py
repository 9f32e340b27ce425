"""Scheme-level pins of the oracle (no GPU).

P3  GENO preserves the linear scheme on smooth waves (Sec. 3.1, linearity
    preserving): results equal the chi = 1 run to round-off; on a jump they
    differ (the pin is not vacuous).
P4  design order on the advected density sine wave (Sec. 6.1, Sec. 6.10):
    eighth order in 1D with dt ~ h^3 (so the time error is below the spatial
    one), fourth order in 2D with dt ~ h^2.
P5  conservation: with periodic boundaries the sums of the cell averages are
    constant (Eq. semifvs, telescoping fluxes); the sums of the cell-averaged
    gradients vanish (Eq. slope, telescoping interface states).
P8  symmetries: mirror x -> -x, transposition x <-> y, the 3D axis cycle
    x -> y -> z -> x, and invariance of y-independent data.
P9  convergence to the exact Riemann solution of seeded two-state problems.
"""
import math

import numpy as np
import pytest

from paper_2507_20461_gb300 import inputs as I


def _run(oracle, cfg, W, G, dt, nsteps):
    W = np.ascontiguousarray(W, dtype=np.float64).copy()
    G = np.ascontiguousarray(G, dtype=np.float64).copy()
    for _ in range(nsteps):
        r = oracle.step(cfg, dt, W, G)
        assert r == 0, r
    return W, G


def test_geno_equals_linear_on_smooth_1d(oracle):
    W, G, h = I.sine_wave(1, 32)
    res = []
    for lim in (0, 1):
        cfg = oracle.make_cfg(1, (32,), h, limiter=lim)
        res.append(_run(oracle, cfg, W, G, 0.2 * h, 10))
    assert np.max(np.abs(res[0][0] - res[1][0])) < 1e-13
    assert np.max(np.abs(res[0][1] - res[1][1])) < 1e-11


def test_geno_equals_linear_on_smooth_2d(oracle):
    W, G, h = I.sine_wave(2, 12)
    res = []
    for lim in (0, 1):
        cfg = oracle.make_cfg(2, (12, 12), h, limiter=lim)
        res.append(_run(oracle, cfg, W, G, 0.2 * h, 3))
    assert np.max(np.abs(res[0][0] - res[1][0])) < 1e-13


def test_geno_differs_from_linear_on_jump(oracle):
    W, G, h, _ = I.riemann_1d(32, seed=1)
    res = []
    for lim in (0, 1):
        cfg = oracle.make_cfg(1, (32,), h, bc=1, limiter=lim)
        res.append(_run(oracle, cfg, W, G, 0.02 * h, 3))
    assert np.max(np.abs(res[0][0] - res[1][0])) > 1e-6


def _order_run(oracle, dim, n, dt_fn, T):
    W, G, h = I.sine_wave(dim, n)
    cfg = oracle.make_cfg(dim, (n,) * dim, h)
    nst = int(math.ceil(T / dt_fn(h)))
    W, G = _run(oracle, cfg, W, G, T / nst, nst)
    return float(np.mean(np.abs(W[0] - I.sine_exact_rho(dim, n, T))))


def test_design_order_1d(oracle):
    """E1 of Sec. 6.1 (rho = 1 + 0.2 sin(pi x), U = p = 1 on [0, 2], periodic)."""
    e = [_order_run(oracle, 1, n, lambda h: 0.2 * h**3, 0.05) for n in (8, 16, 32)]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(2)]
    assert orders[-1] >= 7.5, (e, orders)


def test_design_order_2d(oracle):
    """Cartesian counterpart of the accuracy test of Sec. 6.10 in 2D."""
    e = [_order_run(oracle, 2, n, lambda h: 0.1 * h**2, 0.1) for n in (8, 16)]
    order = math.log2(e[0] / e[1])
    assert order >= 3.6, (e, order)


def test_design_order_3d(oracle):
    e = [_order_run(oracle, 3, n, lambda h: 0.1 * h**2, 0.05) for n in (4, 8)]
    order = math.log2(e[0] / e[1])
    assert order >= 3.6, (e, order)


@pytest.mark.parametrize("dim,n", [(1, 24), (2, 10), (3, 5)])
def test_conservation_periodic(oracle, dim, n):
    rng = np.random.default_rng(dim)
    W, G, h = I.sine_wave(dim, n)
    # perturb to a generic smooth-ish state
    W = W * (1 + 0.05 * rng.random(W.shape))
    G = G + 0.1 * rng.normal(size=G.shape)
    cfg = oracle.make_cfg(dim, (n,) * dim, h)
    s0 = W.reshape(dim + 2, -1).sum(axis=1)
    W1, G1 = _run(oracle, cfg, W, G, 0.1 * h, 4)
    s1 = W1.reshape(dim + 2, -1).sum(axis=1)
    np.testing.assert_allclose(s1, s0, rtol=1e-13)
    gs = G1.reshape(dim, dim + 2, -1).sum(axis=2)
    np.testing.assert_allclose(gs, 0.0, atol=1e-10 * np.abs(G1).max() * G1[0, 0].size)


def test_mirror_symmetry_1d(oracle):
    n = 40
    W, G, h, _ = I.riemann_1d(n, seed=3)
    W = W + 0.01 * np.sin(np.arange(n))[None, :]
    cfg = oracle.make_cfg(1, (n,), h, bc=1)

    def mirror(W, G):
        Wm = W[:, ::-1].copy()
        Wm[1] *= -1
        Gm = -G[:, :, ::-1].copy()
        Gm[:, 1] *= -1
        return Wm, Gm

    W1, G1 = _run(oracle, cfg, W, G, 0.05 * h, 3)
    Wm, Gm = mirror(W, G)
    W2, G2 = _run(oracle, cfg, Wm, Gm, 0.05 * h, 3)
    W2b, G2b = mirror(W2, G2)
    np.testing.assert_allclose(W2b, W1, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(G2b, G1, rtol=1e-11, atol=1e-11)


def test_transpose_symmetry_2d(oracle):
    n = 10
    W, G, h = I.quadrants_2d(n, seed=4)
    rng = np.random.default_rng(4)
    W = W * (1 + 0.02 * rng.random(W.shape))
    cfg = oracle.make_cfg(2, (n, n), h, bc=1)

    def transpose(W, G):
        Wt = np.transpose(W, (0, 2, 1)).copy()
        Wt[[1, 2]] = Wt[[2, 1]]
        Gt = np.transpose(G, (0, 1, 3, 2)).copy()
        Gt = Gt[[1, 0]]
        Gt[:, [1, 2]] = Gt[:, [2, 1]]
        return Wt, Gt

    W1, G1 = _run(oracle, cfg, W, G, 0.05 * h, 2)
    Wt, Gt = transpose(W, G)
    W2, G2 = _run(oracle, cfg, Wt, Gt, 0.05 * h, 2)
    W2b, G2b = transpose(W2, G2)
    np.testing.assert_allclose(W2b, W1, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(G2b, G1, rtol=1e-10, atol=1e-10)


def test_axis_cycle_symmetry_3d(oracle):
    """The rotation x' = y, y' = z, z' = x: on a non-cubic grid with data
    varying in every component, stepping the rotated state and rotating back
    gives the original run (the face frames' transverse axes, the tangential
    slopes and the transverse moments must follow the axes)."""
    rng = np.random.default_rng(6)
    nx, ny, nz = 6, 7, 8
    h = 1.0 / nx
    shape = (nz, ny, nx)
    rho = 1.0 + 0.2 * rng.random(shape)
    vel = [0.3 * (rng.random(shape) - 0.5) for _ in range(3)]
    p = 1.0 + 0.2 * rng.random(shape)
    ke = sum(u * u for u in vel)
    W = np.stack([rho] + [rho * u for u in vel] + [p / 0.4 + 0.5 * rho * ke])
    G = 0.3 * rng.normal(size=(3,) + W.shape)

    def cycle(W, G):
        """new [v][z'][y'][x'] = old [v][x][z][y]; u' = v, v' = w, w' = u;
        d/dx' = d/dy, d/dy' = d/dz, d/dz' = d/dx"""
        Wc = np.transpose(W, (0, 3, 1, 2))[[0, 2, 3, 1, 4]].copy()
        Gc = np.transpose(G, (0, 1, 4, 2, 3))[:, [0, 2, 3, 1, 4]][[1, 2, 0]].copy()
        return Wc, Gc

    dt = 0.05 * h
    W1, G1 = _run(oracle, oracle.make_cfg(3, (nx, ny, nz), h, bc=1), W, G, dt, 2)
    Wc, Gc = cycle(W, G)
    W2, G2 = _run(oracle, oracle.make_cfg(3, (ny, nz, nx), h, bc=1), Wc, Gc, dt, 2)
    W2b, G2b = cycle(*cycle(W2, G2))
    np.testing.assert_allclose(W2b, W1, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(G2b, G1, rtol=1e-10, atol=1e-10)
    # not vacuous: rotating the axes but not the momentum components breaks it
    Wx = np.transpose(W, (0, 3, 1, 2)).copy()
    Gx = np.transpose(G, (0, 1, 4, 2, 3))[[1, 2, 0]].copy()
    W3, G3 = _run(oracle, oracle.make_cfg(3, (ny, nz, nx), h, bc=1), Wx, Gx, dt, 2)
    W3b = np.transpose(W3, (0, 2, 3, 1))
    assert np.abs(W3b[[0, 4]] - W1[[0, 4]]).max() > 1e-6


def test_y_invariant_stays_y_invariant(oracle):
    n1, ny = 24, 6
    W1d, G1d, h, _ = I.riemann_1d(n1, seed=5)
    W = np.zeros((4, ny, n1))
    W[0] = W1d[0]
    W[1] = W1d[1]
    W[3] = W1d[2]
    G = np.zeros((2, 4, ny, n1))
    cfg = oracle.make_cfg(2, (n1, ny), h, bc=0)
    W, G = _run(oracle, cfg, W, G, 0.05 * h, 2)
    assert np.max(np.abs(W - W[:, :1, :])) < 1e-13
    assert np.max(np.abs(W[2])) < 1e-13
    assert np.max(np.abs(G[1])) < 1e-11


def test_converges_to_exact_riemann(oracle):
    """Seeded two-state problems of the config-1 family (rho, p ~ U[0.1, 1],
    u ~ U[-0.5, 0.5], transmissive ends, run until the fastest wave is 0.43
    from the centre).  L1 density distance to the exact solution (cell
    averages by 64-point sampling): for every seed the N = 256 error is below
    the N = 32 error, and the median rate over seeds is >= 0.45.  (Convergence
    is slow for some seeds: post-shock noise, which the temporal limiting at
    strong discontinuities that the paper defers to earlier work would damp.)"""
    from oracle import riemann

    rates = []
    for seed in range(6):
        errs = []
        for n in (32, 256):
            W, G, h, st = I.riemann_1d(n, seed)
            cfg = oracle.make_cfg(1, (n,), h, bc=1)
            t = 0.45 / oracle.max_wavespeed(cfg, W) / 1.05
            tt = 0.0
            W = W.copy()
            G = G.copy()
            while tt < t - 1e-14:
                dt = min(0.4 * h / oracle.max_wavespeed(cfg, W), t - tt)
                assert oracle.step(cfg, dt, W, G) == 0
                tt += dt
            ex = riemann.cell_averages(st[0], st[1], n, t)
            errs.append(float(np.mean(np.abs(W[0] - ex[0]))))
        assert errs[1] < errs[0], (seed, errs)
        rates.append(math.log2(errs[0] / errs[1]) / 3)
    assert float(np.median(rates)) >= 0.45, rates


def _contact_overshoot(oracle, limiter):
    n = 64
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    rho = np.where(x < 0.5, 1.0, 0.5)
    u = 0.5 * np.ones(n)
    p = np.ones(n)
    W = np.stack([rho, rho * u, p / 0.4 + 0.5 * rho * u * u])
    G = np.zeros((1, 3, n))
    cfg = oracle.make_cfg(1, (n,), h, bc=1, limiter=limiter)
    worst = 0.0
    for _ in range(40):
        dt = 0.4 * h / oracle.max_wavespeed(cfg, W)
        assert oracle.step(cfg, dt, W, G) == 0
        worst = max(worst, W[0].max() - 1.0, 0.5 - W[0].min())
    return worst


def test_contact_overshoot_below_linear(oracle):
    """An isolated contact (u = 0.5, p = 1, rho 1 | 0.5): GENO keeps the density
    overshoot under half of the linear scheme's and under 3% of the data.
    (Component-wise blending of conservative variables perturbs the pressure at
    a contact, so GENO is essentially, not strictly, non-oscillatory here.)"""
    geno = _contact_overshoot(oracle, 0)
    lin = _contact_overshoot(oracle, 1)
    assert geno <= 0.5 * lin, (geno, lin)
    assert geno <= 0.03, geno


def _mirror_1d(W, G):
    """Mirror image about the right end: reversed, momentum negated; gradients
    of even variables negated, of the (odd) momentum kept."""
    Wm = W[:, ::-1].copy()
    Wm[1] *= -1
    Gm = -G[:, :, ::-1].copy()
    Gm[:, 1] *= -1
    return Wm, Gm


def test_reflective_equals_symmetric_periodic_1d(oracle):
    """A reflective wall at both ends of [0, 1] is the mirror-symmetric periodic
    problem on [0, 2] (R8 reading of the reflecting boundaries of Sec. 6.6)."""
    n = 40
    W, G, h, _ = I.riemann_1d(n, seed=7)
    rng = np.random.default_rng(7)
    W = W * (1 + 0.02 * rng.random(W.shape))
    W[1] += 0.1
    G = 0.3 * rng.normal(size=G.shape)
    Wm, Gm = _mirror_1d(W, G)
    W2 = np.ascontiguousarray(np.concatenate([W, Wm], axis=1))
    G2 = np.ascontiguousarray(np.concatenate([G, Gm], axis=2))
    cfg_r = oracle.make_cfg(1, (n,), h, bc=2)
    cfg_p = oracle.make_cfg(1, (2 * n,), h, bc=0)
    dt = 0.3 * h / oracle.max_wavespeed(cfg_p, W2)
    Wr, Gr = _run(oracle, cfg_r, W, G, dt, 5)
    Wp, Gp = _run(oracle, cfg_p, W2, G2, dt, 5)
    np.testing.assert_allclose(Wr, Wp[:, :n], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Gr, Gp[:, :, :n], rtol=1e-9, atol=1e-9)
    # the transmissive result differs (the pin is not vacuous)
    Wt, _ = _run(oracle, oracle.make_cfg(1, (n,), h, bc=1), W, G, dt, 5)
    assert np.abs(Wt - Wr).max() > 1e-6


def test_reflective_equals_symmetric_periodic_2d(oracle):
    nx, ny = 8, 6
    W, G, h = I.quadrants_2d(ny, seed=9, nx=nx)
    rng = np.random.default_rng(9)
    W = W * (1 + 0.02 * rng.random(W.shape))
    G = 0.2 * rng.normal(size=G.shape)

    def mirror_x(W, G):
        Wm = W[:, :, ::-1].copy()
        Wm[1] *= -1
        Gm = G[:, :, :, ::-1].copy()
        Gm[0] *= -1  # d/dx of even variables flips
        Gm[:, 1] *= -1  # x-momentum is odd
        return Wm, Gm

    def mirror_y(W, G):
        Wm = W[:, ::-1, :].copy()
        Wm[2] *= -1
        Gm = G[:, :, ::-1, :].copy()
        Gm[1] *= -1
        Gm[:, 2] *= -1
        return Wm, Gm

    Wx, Gx = mirror_x(W, G)
    Wa = np.concatenate([W, Wx], axis=2)
    Ga = np.concatenate([G, Gx], axis=3)
    Wy, Gy = mirror_y(Wa, Ga)
    W4 = np.ascontiguousarray(np.concatenate([Wa, Wy], axis=1))
    G4 = np.ascontiguousarray(np.concatenate([Ga, Gy], axis=2))
    cfg_r = oracle.make_cfg(2, (nx, ny), h, bc=2)
    cfg_p = oracle.make_cfg(2, (2 * nx, 2 * ny), h, bc=0)
    dt = 0.3 * h / oracle.max_wavespeed(cfg_p, W4)
    Wr, Gr = _run(oracle, cfg_r, W, G, dt, 3)
    Wp, Gp = _run(oracle, cfg_p, W4, G4, dt, 3)
    np.testing.assert_allclose(Wr, Wp[:, :ny, :nx], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Gr, Gp[:, :, :ny, :nx], rtol=1e-9, atol=1e-9)


def _y_uniform_channel_state(nx, ny, seed):
    """y-independent state with nonzero normal and tangential velocity near the
    x-walls (averages and x-gradients; no y-gradients)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / nx
    x = (np.arange(nx) + 0.5) * h
    rho = 1.0 + 0.2 * np.sin(3 * x) + 0.02 * rng.random(nx)
    u = 0.1 * np.cos(2 * x) + 0.01 * rng.random(nx)
    v = 0.3 * np.sin(5 * x) + 0.01 * rng.random(nx)
    p = 1.0 + 0.1 * np.cos(4 * x)
    W1 = np.stack([rho, rho * u, rho * v, p / 0.4 + 0.5 * rho * (u * u + v * v)])
    G1 = 0.3 * rng.normal(size=(4, nx))
    W = np.ascontiguousarray(np.repeat(W1[:, None, :], ny, axis=1))
    G = np.zeros((2, 4, ny, nx))
    G[0] = np.repeat(G1[:, None, :], ny, axis=1)
    return W, G, h


@pytest.mark.parametrize("mu", [0.0, 0.01])
def test_noslip_walls_equal_point_symmetric_periodic(oracle, mu):
    """No-slip walls at x = 0, 1 (y periodic) for a y-independent state are the
    periodic problem on [0, 2] with the point-symmetric extension
    (x -> -x, u -> -u, v -> -v), a symmetry of the equations for such states;
    per-side boundary conditions (R8), Euler and Navier-Stokes."""
    nx, ny = 12, 3
    W, G, h = _y_uniform_channel_state(nx, ny, 11)
    Wm = W[:, :, ::-1].copy()
    Wm[1:3] *= -1
    Gm = G[:, :, :, ::-1].copy()
    Gm[0] *= -1
    Gm[:, 1:3] *= -1
    W2 = np.ascontiguousarray(np.concatenate([W, Wm], axis=2))
    G2 = np.ascontiguousarray(np.concatenate([G, Gm], axis=3))
    cfg_w = oracle.make_cfg(2, (nx, ny), h, bc=(3, 3, 0, 0, 0, 0), mu=mu)
    cfg_p = oracle.make_cfg(2, (2 * nx, ny), h, bc=0, mu=mu)
    dt = 0.3 * h / oracle.max_wavespeed(cfg_p, W2)
    Ww, Gw = _run(oracle, cfg_w, W, G, dt, 4)
    Wp, Gp = _run(oracle, cfg_p, W2, G2, dt, 4)
    np.testing.assert_allclose(Ww, Wp[:, :, :nx], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(Gw, Gp[:, :, :, :nx], rtol=1e-9, atol=1e-9)
    # a slip wall gives another result (the tangential momentum is even there)
    Ws, _ = _run(oracle, oracle.make_cfg(2, (nx, ny), h, bc=(2, 2, 0, 0, 0, 0), mu=mu), W, G, dt, 4)
    assert np.abs(Ws - Ww).max() > 1e-6


def test_noslip_channel_mode_decay(oracle):
    """Shear mode v = a sin(pi x) between no-slip walls at x = 0, 1 decays as
    exp(-nu pi^2 t) (linearised Navier-Stokes, Sec. 6.9's wall condition)."""
    nx, ny, mu, amp, p0, t_end = 32, 2, 0.01, 1e-3, 100.0, 0.5
    h = 1.0 / nx
    x = (np.arange(nx) + 0.5) * h
    k = np.pi
    s_avg = (np.cos(k * (x - h / 2)) - np.cos(k * (x + h / 2))) / (k * h)
    c_avg = (np.sin(k * (x + h / 2)) - np.sin(k * (x - h / 2))) / (k * h)
    v = amp * s_avg
    W = np.zeros((4, ny, nx))
    G = np.zeros((2, 4, ny, nx))
    W[0], W[2], W[3] = 1.0, v, p0 / 0.4 + 0.5 * v * v
    G[0, 2] = amp * k * c_avg
    G[0, 3] = v * amp * k * c_avg
    cfg = oracle.make_cfg(2, (nx, ny), h, bc=(3, 3, 0, 0, 0, 0), mu=mu)
    t = 0.0
    while t < t_end - 1e-14:
        dt = min(oracle.cfl_dt(cfg, W, 0.4), t_end - t)
        assert oracle.step(cfg, dt, W, G) == 0
        t += dt
    got = 2 * np.mean((W[2] / W[0]).mean(axis=0) * np.sin(k * x)) / (np.sin(k * h / 2) / (k * h / 2))
    want = amp * np.exp(-mu * k * k * t_end)
    assert abs(got / want - 1) <= 2e-4, (got, want)


def test_per_side_bc_plumbing(oracle):
    n = (10, 8)
    W, G, h = I.quadrants_2d(8, seed=3, nx=10)
    dt = 0.3 * h / oracle.max_wavespeed(oracle.make_cfg(2, n, h, bc=1), W)
    a, _ = _run(oracle, oracle.make_cfg(2, n, h, bc=1), W, G, dt, 2)
    b, _ = _run(oracle, oracle.make_cfg(2, n, h, bc=(1, 1, 1, 1, 0, 0)), W, G, dt, 2)
    np.testing.assert_array_equal(a, b)
    # periodic on one side only is rejected
    bad = oracle.make_cfg(2, n, h, bc=(0, 1, 1, 1, 0, 0))
    assert oracle.step(bad, dt, W.copy(), G.copy()) != 0


@pytest.mark.parametrize("mu", [0.0, 0.005])
def test_closed_box_conserves_mass_and_energy(oracle, mu):
    """Viscous shock tube box (Sec. 6.9): no-slip walls on three sides, a slip
    symmetry line on top.  Nothing but momentum crosses a wall, so the summed
    mass and energy stay fixed to rounding (R8: a no-slip wall face carries no
    mass or energy flux)."""
    nx = 24
    W, G, h = I.viscous_shock_tube(nx)
    cfg = oracle.make_cfg(2, (nx, nx // 2), h, bc=(3, 3, 3, 2, 0, 0), mu=mu)
    m0, e0 = W[0].sum(), W[3].sum()
    for _ in range(8):
        assert oracle.step(cfg, oracle.cfl_dt(cfg, W, 0.4), W, G) == 0
    assert abs(W[0].sum() / m0 - 1) <= 1e-14
    assert abs(W[3].sum() / e0 - 1) <= 1e-14
