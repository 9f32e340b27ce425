"""Seeded synthetic initial data for the compact GKS (numpy only).

Holds none of the scheme's arithmetic: it only builds cell averages ``W`` and
cell-averaged gradients ``G`` of initial conditions shaped like the paper's
test families (Sec. 6): advected density sine waves (Sec. 6.1, Sec. 6.10),
two-state Riemann problems (Sec. 6.5), four-quadrant Riemann problems, smooth
density modes crossed by planar shocks (shock/smooth-wave interaction,
Sec. 6.3), a solenoidal turbulence-like velocity field (Sec. 6.13), and the
two viscous cases: the viscous shock tube (Sec. 6.9) and the Taylor-Green
vortex.
Both the CUDA library's tests and the oracle's tests take their inputs here.

Layouts: ``W[v][k][j][i]`` with v = rho, rho u (, rho v, rho w), rho E;
``G[d][v][k][j][i]`` = d W / d x_d.  Arrays are returned squeezed to the
dimension (1D: (nv, n) and (1, nv, n)).
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = 1.4


def _cons(rho, vel, p, gamma):
    """Pointwise conservative variables from primitives; vel is a list of arrays."""
    ke = sum(u * u for u in vel)
    out = [rho] + [rho * u for u in vel] + [p / (gamma - 1.0) + 0.5 * rho * ke]
    return np.stack(out)


def sine_wave(dim: int, n: int, t: float = 0.0, gamma: float = GAMMA, amp: float = 0.2, L: float = 2.0):
    """rho = 1 + amp sin(pi (x + y + z - dim t)), U = 1 per axis, p = 1 on [0, L]^dim (Sec. 6.1, 6.10).

    Exact cell averages (sinc factor) and exact averaged gradients (face
    averages differenced, Gauss theorem).  Returns (W, G, h).
    """
    h = L / n
    c = (np.arange(n) + 0.5) * h
    grids = np.meshgrid(*([c] * dim), indexing="ij")[::-1]  # grids[a] varies along axis a in [k][j][i] order
    shape = (n,) * dim
    s = math.sin(math.pi * h / 2) / (math.pi * h / 2)
    phase = sum(grids) - dim * t
    rho_avg = 1.0 + amp * np.sin(math.pi * phase) * s**dim
    nv = dim + 2
    W = np.empty((nv,) + shape)
    W[0] = rho_avg
    for a in range(dim):
        W[1 + a] = rho_avg
    W[dim + 1] = 1.0 / (gamma - 1.0) + 0.5 * dim * rho_avg
    G = np.zeros((dim, nv) + shape)
    drho = amp * s ** (dim - 1) * (np.sin(math.pi * (phase + h / 2)) - np.sin(math.pi * (phase - h / 2))) / h
    for d in range(dim):
        G[d, 0] = drho
        for a in range(dim):
            G[d, 1 + a] = drho
        G[d, dim + 1] = 0.5 * dim * drho
    return W, G, h


def sine_exact_rho(dim: int, n: int, t: float, amp: float = 0.2, L: float = 2.0):
    W, _, _ = sine_wave(dim, n, t=t, amp=amp, L=L)
    return W[0]


def riemann_1d(n: int, seed: int, gamma: float = GAMMA):
    """Two seeded states, rho, p ~ U[0.1, 1], u ~ U[-0.5, 0.5], jump at x = 0.5 on [0, 1]."""
    rng = np.random.default_rng(seed)
    st = [(rng.uniform(0.1, 1.0), rng.uniform(-0.5, 0.5), rng.uniform(0.1, 1.0)) for _ in range(2)]
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    left = x < 0.5
    rho = np.where(left, st[0][0], st[1][0])
    u = np.where(left, st[0][1], st[1][1])
    p = np.where(left, st[0][2], st[1][2])
    W = _cons(rho, [u], p, gamma)
    G = np.zeros((1,) + W.shape)
    return W, G, h, st


def quadrants_2d(n: int, seed: int, gamma: float = GAMMA, nx: int | None = None):
    """Four seeded quadrant states on [0, 1]^2 split at 0.5: rho, p ~ U[0.1, 1.5], u, v ~ U[-0.8, 0.8].

    Piecewise constant, so the cell-averaged gradients are zero.  ``nx`` allows
    a non-square grid (same h, domain [0, nx h] x [0, 1]).
    """
    rng = np.random.default_rng(seed)
    nx = n if nx is None else nx
    st = [(rng.uniform(0.1, 1.5), rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), rng.uniform(0.1, 1.5)) for _ in range(4)]
    h = 1.0 / n
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(n) + 0.5) * h
    Y, X = np.meshgrid(y, x, indexing="ij")
    q = (X >= 0.5 * nx * h).astype(int) + 2 * (Y >= 0.5).astype(int)
    arr = np.array(st)
    rho, u, v, p = (arr[q, i] for i in range(4))
    W = _cons(rho, [u, v], p, gamma)
    G = np.zeros((2,) + W.shape)
    return W, G, h


def _fourier_shock_strip(xs, ys, modes, shocks, gamma, drift=(0.0, 0.0)):
    """Point values on the tensor grid ys x xs (1D arrays): base gas
    rho = 1 + 0.2/16 sum cos(2 pi k.x + phi), (u, v) = drift, p = 1, then each
    shock in order overwrites its slab with the Rankine-Hugoniot post-shock
    state of the gas at rest (moving along the shock normal)."""
    rho = np.ones((ys.size, xs.size))
    amp = 0.2 / len(modes)
    for (kx, ky, ph) in modes:
        ax = 2 * math.pi * kx * xs + ph
        by = 2 * math.pi * ky * ys
        rho += amp * (np.outer(np.cos(by), np.cos(ax)) - np.outer(np.sin(by), np.sin(ax)))
    u = np.full_like(rho, drift[0])
    v = np.full_like(rho, drift[1])
    p = np.ones_like(rho)
    base_rho = rho.copy()
    for (nx_, ny_, off, M) in shocks:
        nn = math.hypot(nx_, ny_)
        sarg = np.mod(np.add.outer(ny_ * ys, nx_ * xs) - off, 1.0)
        behind = sarg > 1.0 - 0.125 * nn
        r = (gamma + 1) * M * M / ((gamma - 1) * M * M + 2)
        pr = 1 + 2 * gamma / (gamma + 1) * (M * M - 1)
        du = M * np.sqrt(gamma / base_rho) * (1 - 1 / r)
        rho = np.where(behind, base_rho * r, rho)
        p = np.where(behind, pr, p)
        u = np.where(behind, du * nx_ / nn, u)
        v = np.where(behind, du * ny_ / nn, v)
    return rho, u, v, p


def fourier_shocks_2d(n: int, seed: int, gamma: float = GAMMA, sub: int | None = None,
                      nshocks: int = 4, drift=(0.0, 0.0)):
    """Periodic [0,1]^2: rho = 1 + 0.2/16 sum_m cos(2 pi k_m.x + phi_m), 1 <= |k_m|_inf <= 8,
    u = 0, p = 1, then four planar shocks (normals from {(1,0),(0,1),(1,1),(1,-1)},
    offset ~ U[0,1), Mach ~ U[1.5, 3]); each shock sets, in a slab of width
    0.125 behind its front, the Rankine-Hugoniot post-shock state of the base
    gas (later shocks overwrite earlier ones).  Averages by sub x sub midpoint
    sampling (sub = 8 up to n = 512, else 4), gradients by the Gauss theorem
    with sub samples per face.

    Smooth variant: nshocks < 4 keeps only the first shocks drawn (the draws
    are unchanged, so the modes are those of the full case) and drift gives
    the base gas a uniform velocity (the shocks' post-shock states are those
    of the gas at rest, so drift is meant for nshocks = 0).
    """
    rng = np.random.default_rng(seed)
    modes = []
    while len(modes) < 16:
        kx, ky = rng.integers(-8, 9, size=2)
        if max(abs(kx), abs(ky)) >= 1:
            modes.append((int(kx), int(ky), rng.uniform(0, 2 * math.pi)))
    normals = [(1, 0), (0, 1), (1, 1), (1, -1)]
    shocks = []
    for i in range(4):
        nrm = normals[rng.integers(0, 4)]
        shocks.append((nrm[0], nrm[1], rng.uniform(0, 1), rng.uniform(1.5, 3.0)))
    shocks = shocks[:nshocks]
    if sub is None:
        sub = 8 if n <= 512 else 4
    h = 1.0 / n
    nv = 4
    W = np.zeros((nv, n, n))
    G = np.zeros((2, nv, n, n))
    off = (np.arange(sub) + 0.5) / sub - 0.5
    base = (np.arange(n) + 0.5) * h
    xs_sub = (base[:, None] + off[None, :] * h).ravel()  # cell-major sub-samples
    xs_face = np.concatenate([base - 0.5 * h, [1.0 - 0.5 * h + h]])  # n + 1 face coordinates
    rows = max(1, min(n, (1 << 22) // (n * sub * sub)))
    for j0 in range(0, n, rows):
        j1 = min(n, j0 + rows)
        ys_sub = (base[j0:j1, None] + off[None, :] * h).ravel()
        rho, u, v, p = _fourier_shock_strip(xs_sub, ys_sub, modes, shocks, gamma, drift)
        cons = _cons(rho, [u, v], p, gamma)  # (nv, (j1-j0)*sub, n*sub)
        W[:, j0:j1] = cons.reshape(nv, j1 - j0, sub, n, sub).mean(axis=(2, 4))
        # x faces: sample x on faces, y on sub-samples
        rho, u, v, p = _fourier_shock_strip(xs_face, ys_sub, modes, shocks, gamma, drift)
        cf = _cons(rho, [u, v], p, gamma).reshape(nv, j1 - j0, sub, n + 1).mean(axis=2)
        G[0, :, j0:j1] = (cf[:, :, 1:] - cf[:, :, :-1]) / h
        # y faces
        ys_face = np.concatenate([base[j0:j1] - 0.5 * h, [base[j1 - 1] + 0.5 * h]])
        rho, u, v, p = _fourier_shock_strip(xs_sub, ys_face, modes, shocks, gamma, drift)
        cf = _cons(rho, [u, v], p, gamma).reshape(nv, j1 - j0 + 1, n, sub).mean(axis=3)
        G[1, :, j0:j1] = (cf[:, 1:] - cf[:, :-1]) / h
    return W, G, h


def batch_sizes(count: int, seed: int, lo: int = 64, hi: int = 1024):
    """Grid sides drawn log-uniformly in [lo, hi], rounded to even."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    return [int(max(2, 2 * round(x / 2))) for x in s]


# Batched workload (256 grids, sides from batch_sizes(256, 20464)): grid g's
# four-quadrant IC uses seed 20464 + g + 1000 k, k = BATCH_REDRAWS.get(g, 0).
# The recipe's rule: an IC on which the FP64 path (the oracle's arithmetic)
# turns non-physical within the workload's 300 steps is redrawn.  Grid 61
# (64^2): the FP64 batch reaches p <= 0 within its first draw's 300 steps;
# its redraw runs through in FP64 and in mixed precision.  A grid
# that only the mixed-precision path turns non-physical is kept and reported
# (Batch.grid_status), not redrawn.
BATCH_BASE_SEED = 20464
BATCH_REDRAWS = {61: 1}


def batch_seed(g: int, base: int = BATCH_BASE_SEED) -> int:
    return base + g + 1000 * BATCH_REDRAWS.get(g, 0)


def turbulence_3d(n: int, seed: int, gamma: float = GAMMA, mach: float = 0.6, k0: float = 4.0):
    """Periodic [0,1]^3, rho = 1, solenoidal random-phase velocity with
    E(k) ~ k^4 exp(-2 (k/k0)^2), scaled to u_rms = 1, p = 1/(gamma mach^2).

    Averages are the point values at cell centres, gradients spectral
    derivatives there (synthetic input, not a discretisation claim).
    """
    rng = np.random.default_rng(seed)
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    kk = np.sqrt(KX**2 + KY**2 + KZ**2)
    kk[0, 0, 0] = 1.0
    amp = np.sqrt(kk**4 * np.exp(-2 * (kk / k0) ** 2) / (4 * math.pi * kk**2))
    amp[0, 0, 0] = 0.0
    comps = []
    for _ in range(3):
        ph = rng.uniform(0, 2 * math.pi, size=kk.shape)
        comps.append(amp * np.exp(1j * ph))
    # project out the component along k
    dot = (comps[0] * KX + comps[1] * KY + comps[2] * KZ) / kk**2
    comps = [comps[0] - dot * KX, comps[1] - dot * KY, comps[2] - dot * KZ]
    vel = [np.real(np.fft.ifftn(c)) for c in comps]
    urms = math.sqrt(sum(float(np.mean(v * v)) for v in vel) / 3.0)
    vel = [v / urms for v in vel]
    dvel = []
    for c in comps:
        dvel.append([np.real(np.fft.ifftn(1j * 2 * math.pi * K * c)) / urms for K in (KX, KY, KZ)])
    rho = np.ones((n, n, n))
    p = np.full((n, n, n), 1.0 / (gamma * mach * mach))
    W = _cons(rho, vel, p, gamma)
    G = np.zeros((3, 5, n, n, n))
    for d in range(3):
        for a in range(3):
            G[d, 1 + a] = dvel[a][d]
        G[d, 4] = sum(vel[a] * dvel[a][d] for a in range(3))
    return W, G, 1.0 / n


def viscous_shock_tube(nx: int, gamma: float = GAMMA):
    """Viscous shock tube (Sec. 6.9) on [0, 1] x [0, 0.5]: (rho, u, v, p) =
    (120, 0, 0, 120/gamma) for x < 0.5 and (1.2, 0, 0, 1.2/gamma) beyond;
    nx x nx/2 cells (nx even, so the jump lies on a face), zero gradients.
    The paper's walls: no-slip at x = 0, 1 and y = 0, a symmetry line at
    y = 0.5 (boundary sides (3, 3, 3, 2)); mu = 0.005 (Re = 200), Pr = 1."""
    if nx % 2:
        raise ValueError("nx must be even")
    ny = nx // 2
    h = 1.0 / nx
    x = (np.arange(nx) + 0.5) * h
    rho1 = np.where(x < 0.5, 120.0, 1.2)
    rho = np.repeat(rho1[None, :], ny, axis=0)
    p = rho / gamma
    W = _cons(rho, [np.zeros_like(rho), np.zeros_like(rho)], p, gamma)
    G = np.zeros((2, 4, ny, nx))
    return W, G, h


def taylor_green_3d(n: int, gamma: float = GAMMA, mach: float = 0.1, u0: float = 1.0):
    """Taylor-Green vortex on the periodic cube [-pi, pi]^3 (n^3 cells):
    u = u0 sin x cos y cos z, v = -u0 cos x sin y cos z, w = 0, uniform
    temperature, rho = 1 + (gamma mach^2 / 16)(cos 2x + cos 2y)(cos 2z + 2),
    p = rho / (gamma mach^2) (so that mach = u0 / sqrt(gamma p0 / rho0)).
    Averages are the point values at cell centres and gradients the exact
    derivatives there (synthetic input).  Returns W, G, h = 2 pi / n."""
    h = 2 * math.pi / n
    c = -math.pi + (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    sx, cx, sy, cy, sz, cz = np.sin(X), np.cos(X), np.sin(Y), np.cos(Y), np.sin(Z), np.cos(Z)
    u = u0 * sx * cy * cz
    v = -u0 * cx * sy * cz
    w = np.zeros_like(u)
    a = gamma * mach * mach / 16.0
    rho = 1.0 + a * (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0)
    T = 1.0 / (gamma * mach * mach)
    p = rho * T
    W = _cons(rho, [u, v, w], p, gamma)
    # exact derivatives: d/dx, d/dy, d/dz of rho, u, v (w = 0)
    drho = [
        -2 * a * np.sin(2 * X) * (np.cos(2 * Z) + 2.0),
        -2 * a * np.sin(2 * Y) * (np.cos(2 * Z) + 2.0),
        -2 * a * (np.cos(2 * X) + np.cos(2 * Y)) * np.sin(2 * Z),
    ]
    du = [u0 * cx * cy * cz, -u0 * sx * sy * cz, -u0 * sx * cy * sz]
    dv = [u0 * sx * sy * cz, -u0 * cx * cy * cz, u0 * cx * sy * sz]
    G = np.zeros((3, 5, n, n, n))
    for d in range(3):
        G[d, 0] = drho[d]
        G[d, 1] = drho[d] * u + rho * du[d]
        G[d, 2] = drho[d] * v + rho * dv[d]
        # E = p / (gamma - 1) + rho |u|^2 / 2 with p = rho T
        G[d, 4] = drho[d] * T / (gamma - 1) + 0.5 * drho[d] * (u * u + v * v) + rho * (u * du[d] + v * dv[d])
    return W, G, h
