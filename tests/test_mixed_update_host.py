"""The library's mixed-precision stage update (csrc/kernels.cuh,
update_item<float, M, S>, 2D and 3D), compiled for the CPU through the test-only CUDA
stand-in of tests/hostshim, on random FP32 face sums, checked against exact
rational arithmetic of the two-stage update (stage 1: W* = W + k0 S(F) +
k1 S(Ft), Acc = k2 S(F) + k3 S(Ft); stage 2: W^{n+1} = W + Acc + k4 S(Ft*),
with S the sum over directions of (upper face - lower face) and
k = (-dt/2, -dt^2/8, -dt, -dt^2/6, -dt^2/3) / (h NG)):

* the face sums are accumulated exactly and the stage combination carries
  about 48 bits (the double-float FP32 arithmetic);
* stage 2 adds its increment to the FP64 state with FP64 roundings only,
  and the new FP32 shadow is the exact split of the new FP64 state;
* the gradients are the FP32 Gauss-theorem differences of the W(dt/2) face
  sums."""
import os
import shutil
import subprocess
from fractions import Fraction as Fr

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2507_20461_gb300", "csrc")

pytestmark = pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("mu") / "mixed_update_check")
    r = subprocess.run(["g++", "-O1", "-std=c++17", "-ffp-contract=off", "-I", os.path.join(HERE, "hostshim"),
                        "-I", CSRC, os.path.join(HERE, "mixed_update_check.cpp"), "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return out


@pytest.mark.parametrize("n", [(7, 5), (4, 5, 3)])
def test_mixed_update_matches_exact_arithmetic(exe, n):
    m = len(n)
    nv, ng = m + 2, (2 if m == 2 else 4)
    h, dt = 1.0 / 64, 2.3e-3
    nx, ny = n[0], n[1]
    nz = n[2] if m == 3 else 1
    nc = nx * ny * nz
    nfd = [(nx + (d == 0)) * (ny + (d == 1)) * (nz + (d == 2)) for d in range(m)]
    foff = [sum(nfd[:d]) for d in range(m)]
    nf = sum(nfd)
    rng = np.random.default_rng(12 + m)
    W = 1.0 + 0.3 * rng.normal(size=(nv, nc))
    W[1:m + 1] *= 0.1

    def faces():
        mag = 10.0 ** rng.uniform(-2, 2, size=(3, nv, nf))
        return (rng.uniform(-1, 1, size=(3, nv, nf)) * mag).astype(np.float32)

    ff1, ff2 = faces(), faces()
    text = "\n".join(" ".join(repr(float(x)) for x in a.ravel()) for a in (W, ff1, ff2)) + "\n"
    r = subprocess.run([exe, str(nx), str(ny), str(n[2] if m == 3 else 0), repr(h), repr(dt)], input=text,
                       capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    rows = r.stdout.strip().splitlines()
    arr = [[Fr(float.fromhex(t)) for t in ln.split()] for ln in rows[:8]]
    h1, l1, g1, acc, Wn, h0, l0, g0 = arr
    # (the random face sums make some states non-physical, so the status
    # word is set; the arithmetic is what is checked here)

    cw = 1.0 / h / ng  # 1 / (h NG)
    k = [Fr(-0.5 * dt * cw), Fr(-0.125 * dt * dt * cw), Fr(-dt * cw), Fr(-dt * dt / 6.0 * cw), Fr(-dt * dt / 3.0 * cw)]

    def face(ff, q, v, d, idx, plus):
        e = [nx + (d == 0), ny + (d == 1), nz + (d == 2)]
        c = list(idx)
        c[d] += plus
        return Fr(float(ff[q, v, foff[d] + (c[2] * e[1] + c[1]) * e[0] + c[0]]))

    def S(ff, q, v, idx):
        return sum(face(ff, q, v, d, idx, 1) - face(ff, q, v, d, idx, 0) for d in range(m))

    def mag(ff, q, v, idx):
        """sum of the face values' magnitudes: the scale of the error term of
        an exact (double-float) face sum, whatever the cancellation"""
        return sum(abs(face(ff, q, v, d, idx, 1)) + abs(face(ff, q, v, d, idx, 0)) for d in range(m))

    e45 = Fr(1, 2**45)
    for v in range(nv):
        for kz in range(nz):
            for j in range(ny):
                for i in range(nx):
                    idx = (i, j, kz)
                    c = (kz * ny + j) * nx + i
                    w = Fr(float(W[v, c]))
                    sF, sT = S(ff1, 0, v, idx), S(ff1, 1, v, idx)
                    mF, mT = mag(ff1, 0, v, idx), mag(ff1, 1, v, idx)
                    ws = w + k[0] * sF + k[1] * sT
                    assert abs(h1[v * nc + c] + l1[v * nc + c] - ws) <= e45 * (abs(w) + abs(k[0]) * mF + abs(k[1]) * mT)
                    A = k[2] * sF + k[3] * sT
                    a = acc[v * nc + c] + acc[(nv + v) * nc + c]
                    assert abs(a - A) <= e45 * (abs(k[2]) * mF + abs(k[3]) * mT)
                    for d in range(m):
                        gd = (face(ff1, 2, v, d, idx, 1) - face(ff1, 2, v, d, idx, 0)) * Fr(float(np.float32(cw)))
                        got = g1[(d * nv + v) * nc + c]
                        assert abs(got - gd) <= Fr(1, 2**21) * abs(gd) + Fr(1, 2**100)
                    # stage 2 from the carried accumulator
                    sT2 = S(ff2, 1, v, idx)
                    wn = w + a + k[4] * sT2
                    got = Wn[v * nc + c]
                    assert abs(got - wn) <= Fr(1, 2**51) * abs(wn) + e45 * (abs(a) + abs(k[4]) * mag(ff2, 1, v, idx))
                    # the new shadow is the exact split of the new FP64 state
                    hh = np.float32(float(got))
                    assert h0[v * nc + c] == Fr(float(hh))
                    assert l0[v * nc + c] == Fr(float(np.float32(float(got) - float(hh))))
