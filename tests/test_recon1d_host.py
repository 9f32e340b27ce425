"""The library's 1D compact reconstruction (csrc/kernels.cuh, recon1d_face:
p^7 on {j-1 .. j+2}, the three sub-stencil quadratics of each side, the
GENO / WENO-Z / TENO blend, ghost cells by index mapping), compiled for the
CPU through the test-only CUDA stand-in of tests/hostshim, against the
oracle's interface states on whole 1D grids: every boundary type, every
weight variant, smooth states and states with jumps; FP64 to 1e-12 of the
variable's scale, FP32 to FP32 accuracy."""
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
    out = str(tmp_path_factory.mktemp("r1") / "recon1d_check")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-I", os.path.join(HERE, "hostshim"), "-I", CSRC,
                        os.path.join(HERE, "recon1d_check.cpp"), "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


def _state(n, seed, jumps):
    rng = np.random.default_rng(seed)
    x = (np.arange(n) + 0.5) / n
    rho = 1.0 + 0.3 * np.sin(2 * np.pi * x + rng.uniform(0, 6))
    u = 0.2 * np.cos(2 * np.pi * x + rng.uniform(0, 6))
    p = 1.0 + 0.2 * np.sin(4 * np.pi * x + rng.uniform(0, 6))
    if jumps:
        rho = rho + 0.8 * (x > 0.45)
        p = p + 0.5 * (x > 0.7)
    W = np.array([rho, rho * u, p / 0.4 + 0.5 * rho * u * u])
    G = np.gradient(W, 1.0 / n, axis=1) + rng.normal(scale=0.05, size=W.shape)
    return W, G


@pytest.mark.parametrize("bc", [0, 1, 2, 3])
@pytest.mark.parametrize("lim", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("jumps", [False, True])
def test_recon1d_matches_oracle(exe, oracle, bc, lim, prec, jumps):
    n = 40
    W, G = _state(n, 10 * bc + lim, jumps)
    text = " ".join(repr(float(v)) for v in W.ravel()) + "\n" + " ".join(repr(float(v)) for v in G.ravel()) + "\n"
    r = subprocess.run([exe, str(n), str(bc), str(lim), str(prec)], input=text, capture_output=True, text=True,
                       timeout=60)
    assert r.returncode == 0, r.stderr
    got = np.array([[float(t) for t in ln.split()] for ln in r.stdout.strip().splitlines()]).reshape(n + 1, 2, 3, 2)
    cfg = oracle.make_cfg(1, (n,), 1.0 / n, bc=bc, limiter=lim)
    ref = oracle.reconstruct(cfg, W, G)  # [side][v][comp][gauss][face]
    tol = 1e-12 if prec == 0 else 2e-5
    for s in range(2):
        for v in range(3):
            for c in range(2):
                want = ref[s, v, c, 0, :]
                scale = np.abs(ref[s, v, c, 0, :]).max() + (np.abs(W[v]).max() if c == 0 else 0.0)
                np.testing.assert_allclose(got[:, s, v, c], want, rtol=0, atol=tol * scale)
