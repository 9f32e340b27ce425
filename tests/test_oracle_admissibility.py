"""Pins of the oracle's admissibility fallback (reading R9), no GPU.

The reading: a reconstructed interface state whose density or pressure is
not above delta times that of its own cell's average is replaced, for that
side and Gauss point, by the cell average with zero slopes.  The paper
prints no value for delta (0.3 here), so the constant stays a reading; what
is pinned is the rule itself, checked on the oracle's output without its
code:
* every interface state either passes the test against its own cell or is
  exactly that cell's average with zero derivatives;
* both branches occur, on a state built so that every candidate polynomial
  carries the same steep slope (the pin is not vacuous);
* with delta near 0 no state with positive rho and p falls back, and raising
  delta only adds fallbacks.
"""
import numpy as np

GAMMA = 1.4


def _pressure(U, m):
    rho = U[0]
    ke = sum(U[1 + a] ** 2 for a in range(m)) / rho
    return (GAMMA - 1.0) * (U[m + 1] - 0.5 * ke)


def _own_cells(dim, n):
    """For every face of a periodic grid (x faces first, then y faces), the
    flat index (k, j, i order) of its side-0 and side-1 cell."""
    nx = n[0]
    ny = n[1] if dim >= 2 else 1
    out = []
    # x faces: (n0 + 1) x n1, i fastest
    for j in range(ny):
        for i in range(nx + 1):
            out.append(((j * nx + (i - 1) % nx), (j * nx + i % nx)))
    if dim >= 2:
        for j in range(ny + 1):
            for i in range(nx):
                out.append((((j - 1) % ny) * nx + i, (j % ny) * nx + i))
    return out


def _states(oracle, dim, n, W, G, h, delta):
    cfg = oracle.make_cfg(dim, n, h, bc=0, adm_delta=delta)
    return oracle.reconstruct(cfg, W, G)


def _classify(dim, n, W, fs, delta, fs_raw=None):
    """Per (side, gauss, face): 'fallback' if the state is exactly its own
    cell's average with zero derivatives (no cell of the test data has zero
    slopes, so no reconstruction lands there by itself), else 'pass', which
    must meet the test against its own cell.  With fs_raw (the states for a
    threshold near 0, i.e. the reconstruction before the rule wherever that
    has positive rho and p): a passing state equals its unfiltered state, and
    a fallback's unfiltered state fails the test (or was replaced already)."""
    m = dim
    nv = m + 2
    Wf = W.reshape(nv, -1)
    cells = _own_cells(dim, n)
    assert fs.shape[-1] == len(cells)
    kinds = {"pass": 0, "fallback": 0}
    for f, (c0, c1) in enumerate(cells):
        for side, c in ((0, c0), (1, c1)):
            Uc = Wf[:, c]
            pc = _pressure(Uc, m)
            for g in range(fs.shape[3]):
                U = fs[side, :, 0, g, f]
                if np.array_equal(U, Uc) and np.all(fs[side, :, 1:, g, f] == 0.0):
                    kinds["fallback"] += 1
                    if fs_raw is not None:
                        R = fs_raw[side, :, 0, g, f]
                        replaced_raw = np.array_equal(R, Uc) and np.all(fs_raw[side, :, 1:, g, f] == 0.0)
                        assert replaced_raw or not (R[0] > delta * Uc[0] and _pressure(R, m) > delta * pc), (f, side, g)
                else:
                    assert U[0] > delta * Uc[0] and _pressure(U, m) > delta * pc, (f, side, g, U, Uc)
                    if fs_raw is not None:
                        assert np.array_equal(fs[side, :, :, g, f], fs_raw[side, :, :, g, f]), (f, side, g)
                    kinds["pass"] += 1
    return kinds


def _steep_gradient(n=(24, 20), slope=5.0):
    """Nearly flat, dilute averages (rho ~ p ~ 0.1, at rest) on a periodic grid, with
    the same steep y-derivative of the density in every cell,
    h d(rho)/dy = slope 0.1 (pressure gradient zero).  Every candidate
    polynomial then carries a slope (the linear ones take their tangential
    slope from the averaged gradients; the least-squares cubic a compromise
    with the flat averages), so GENO has no flat candidate: for slope 5 the
    side above each y face reaches a slightly negative density and must fall
    back, while the x faces' Gauss points (about 0.034 and 0.17) pass."""
    nx, ny = n
    h = 1.0 / nx
    W = np.zeros((4, ny, nx))
    # alternate the density by 5% along x, so that a fallback to a
    # neighbour's average would differ from one to the cell's own
    W[0] = 0.1 * (1.0 + 0.05 * (np.arange(nx) % 2))[None, :]
    W[3] = 0.1 / (GAMMA - 1.0)
    G = np.zeros((2, 4, ny, nx))
    G[1, 0] = slope * 0.1 / h
    return W, G, h


def test_every_state_passes_or_is_its_cell_average(oracle):
    n = (24, 20)
    W, G, h = _steep_gradient(n)
    raw = _states(oracle, 2, n, W, G, h, 1e-12)
    delta = 0.3
    kinds = _classify(2, n, W, _states(oracle, 2, n, W, G, h, delta), delta, raw)
    assert kinds["pass"] > 0 and kinds["fallback"] > 0, kinds


def test_delta_orders_the_fallbacks(oracle):
    """The set of replaced states grows with delta; with delta near 0 only
    states with rho <= 0 or p <= 0 are replaced, and every returned state has
    positive rho and p."""
    n = (24, 20)
    W, G, h = _steep_gradient(n)
    raw = _states(oracle, 2, n, W, G, h, 1e-12)
    for side in (0, 1):
        for g in range(raw.shape[3]):
            U = raw[side, :, 0, g, :]
            assert np.all(U[0] > 0) and np.all(_pressure(U, 2) > 0)
    counts = [_classify(2, n, W, _states(oracle, 2, n, W, G, h, d), d, raw)["fallback"] for d in (1e-12, 0.1, 0.3, 0.6)]
    assert counts == sorted(counts) and counts[-1] > counts[0], counts
