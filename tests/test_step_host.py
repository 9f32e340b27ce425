"""The library's FP64 step, assembled on the CPU from the very item functions
the GPU kernels run (csrc/kernels.cuh: cell_poly_item, face_flux_item,
update_item) through the test-only CUDA stand-in of tests/hostshim, against
the oracle's step: 2D and 3D, every boundary type, the weight variants, to
the GPU path's bar (per-variable relative L1 <= 1e-12)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2507_20461_gb300", "csrc")

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("st") / "step_check")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-I", os.path.join(HERE, "hostshim"), "-I", CSRC,
                        os.path.join(HERE, "step_check.cpp"), "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _state(n, seed):
    """smooth random state on [0,1]^m (cell centres) and a perturbed gradient"""
    m = len(n)
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(n))  # arrays are [z][y][x]
    axes = [(np.arange(k) + 0.5) / k for k in reversed(n)]
    X = np.meshgrid(*axes, indexing="ij")
    rho = 1.0 + 0.2 * sum(np.sin(2 * np.pi * x + rng.uniform(0, 6)) for x in X)
    vel = [0.3 * np.cos(2 * np.pi * X[-1 - a] + rng.uniform(0, 6)) for a in range(m)]
    p = 1.0 + 0.1 * sum(np.cos(2 * np.pi * x + rng.uniform(0, 6)) for x in X)
    W = np.array([rho, *(rho * v for v in vel), p / 0.4 + 0.5 * rho * sum(v * v for v in vel)])
    h = 1.0 / n[0]
    G = np.array([np.gradient(W, h, axis=1 + (m - 1 - a)) for a in range(m)])
    G = G + rng.normal(scale=0.02, size=G.shape)
    return W.reshape(m + 2, -1), G.reshape(m, m + 2, -1), h, shape


CASES = [((12, 10), 0, 0), ((12, 10), 1, 0), ((12, 10), 2, 0), ((12, 10), 3, 0), ((9, 11), 1, 2), ((9, 11), 0, 3),
         ((6, 5, 4), 0, 0), ((6, 5, 4), 1, 0), ((6, 5, 4), 2, 0), ((5, 4, 6), 3, 1)]


@pytest.mark.parametrize("n,bc,lim", CASES)
def test_host_step_matches_oracle(exe, oracle, n, bc, lim):
    m = len(n)
    W, G, h, shape = _state(n, 17 * sum(n) + bc + 5 * lim)
    Wf, Gf = W.reshape((m + 2,) + shape), G.reshape((m, m + 2) + shape)
    cfg = oracle.make_cfg(m, n, h, bc=bc, limiter=lim)
    dt = 0.3 * h / oracle.max_wavespeed(cfg, np.ascontiguousarray(Wf))
    text = repr(dt) + "\n" + " ".join(repr(float(v)) for v in W.ravel()) + "\n" + \
        " ".join(repr(float(v)) for v in G.ravel()) + "\n"
    n3 = list(n) + [1] * (3 - m)
    r = subprocess.run([exe, str(m), *map(str, n3), repr(h), str(bc), str(lim)], input=text, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    Wg = np.array([float(t) for t in lines[0].split()]).reshape(W.shape)
    Gg = np.array([float(t) for t in lines[1].split()]).reshape(G.shape)
    assert int(lines[2]) == 0
    Wo, Go = np.ascontiguousarray(Wf.copy()), np.ascontiguousarray(Gf.copy())
    assert oracle.step(cfg, dt, Wo, Go) == 0
    Wo, Go = Wo.reshape(W.shape), Go.reshape(G.shape)
    assert np.abs(Wo - W).sum() > 1e-6 * np.abs(W).sum()  # the step moved the state
    for v in range(m + 2):
        assert np.abs(Wg[v] - Wo[v]).sum() <= 1e-12 * np.abs(Wo[v]).sum(), v
    for a in range(m):
        for v in range(m + 2):
            assert np.abs(Gg[a, v] - Go[a, v]).sum() <= 1e-11 * (np.abs(Go[a, v]).sum() + np.abs(Go).sum() * 1e-3)


@pytest.mark.parametrize("seed", [3, 11])
def test_host_step_quadrants_matches_oracle(exe, oracle, seed):
    """The four-quadrant Riemann state of the batched workload (jumps: GENO's
    weights far from linear, the admissibility fallback in play), 20^2,
    transmissive: the host step against the oracle's at the same bar."""
    from paper_2507_20461_gb300 import inputs as I

    n = 20
    W, G, h = I.quadrants_2d(n, seed=seed)
    cfg = oracle.make_cfg(2, (n, n), h, bc=1)
    dt = 0.4 * h / oracle.max_wavespeed(cfg, W)
    text = repr(dt) + "\n" + " ".join(repr(float(v)) for v in W.ravel()) + "\n" + \
        " ".join(repr(float(v)) for v in G.ravel()) + "\n"
    r = subprocess.run([exe, "2", str(n), str(n), "1", repr(h), "1", "0"], input=text, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    Wg = np.array([float(t) for t in lines[0].split()]).reshape(W.shape)
    assert int(lines[2]) == 0
    Wo, Go = W.copy(), G.copy()
    assert oracle.step(cfg, dt, Wo, Go) == 0
    for v in range(4):
        assert np.abs(Wg[v] - Wo[v]).sum() <= 1e-12 * np.abs(Wo[v]).sum(), v


@pytest.mark.parametrize("n,bc", [((12, 10), 0), ((10, 9), 3), ((6, 5, 4), 1)])
def test_host_navier_stokes_step_matches_oracle(exe, oracle, n, bc):
    """The Navier-Stokes flux (physical collision time mu / p0 added to the
    numerical one) through the same host-built step, against the oracle's
    viscous step (tau_mode 2): periodic, no-slip walls and 3D."""
    m = len(n)
    mu = 0.01
    W, G, h, shape = _state(n, 31 * sum(n) + bc)
    Wf, Gf = W.reshape((m + 2,) + shape), G.reshape((m, m + 2) + shape)
    cfg = oracle.make_cfg(m, n, h, bc=bc, tau_mode=2, mu=mu)
    dt = 0.3 * h / oracle.max_wavespeed(cfg, np.ascontiguousarray(Wf))
    text = repr(dt) + "\n" + " ".join(repr(float(v)) for v in W.ravel()) + "\n" + \
        " ".join(repr(float(v)) for v in G.ravel()) + "\n"
    n3 = list(n) + [1] * (3 - m)
    r = subprocess.run([exe, str(m), *map(str, n3), repr(h), str(bc), "0", repr(mu)], input=text,
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.strip().splitlines()
    Wg = np.array([float(t) for t in lines[0].split()]).reshape(W.shape)
    assert int(lines[2]) == 0
    Wo, Go = np.ascontiguousarray(Wf.copy()), np.ascontiguousarray(Gf.copy())
    assert oracle.step(cfg, dt, Wo, Go) == 0
    Wo = Wo.reshape(W.shape)
    for v in range(m + 2):
        assert np.abs(Wg[v] - Wo[v]).sum() <= 1e-12 * np.abs(Wo[v]).sum(), v
