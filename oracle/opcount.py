"""Operation counts of the oracle (TEST INFRASTRUCTURE ONLY).

The oracle's C source is compiled once more as C++ with every
floating-point type replaced by the counting scalar of ``opcount.hpp``
(common subexpressions shared, constants folded; see that header), together
with the main program ``opcount_main.cpp``.  The counts are the algorithmic work of
the method as the oracle states it: flops = add/sub + mul + div (a fused
multiply-add counts 2), and the transcendentals exp, erfc, sqrt, tanh one
each, reported apart.  Used by tests and by the script that records the
counts the benchmark's roofline numerators come from.
"""
from __future__ import annotations

import json
import os
import re
import struct
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geno_gks_oracle.c")
_BUILD = os.path.join(_HERE, "_opcount")
_EXE = os.path.join(_BUILD, "opcount")


def _inputs():
    return [_SRC, os.path.join(_HERE, "opcount.hpp"), os.path.join(_HERE, "opcount_main.cpp"), __file__]


def build(force: bool = False) -> str:
    """Translate the oracle to the counting scalar and compile the main program."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_EXE) and os.path.getmtime(_EXE) >= max(os.path.getmtime(f) for f in _inputs()):
        return _EXE
    src = open(_SRC).read()
    src = "\n".join(l for l in src.splitlines() if not l.lstrip().startswith("#pragma omp"))
    src = re.sub(r"\blong double\b", "ocn", src)
    src = re.sub(r"\bdouble\b", "ocn", src)
    gen = os.path.join(_BUILD, "oracle_ocn.inc")
    with open(gen + ".tmp", "w") as f:
        f.write(src)
    os.replace(gen + ".tmp", gen)
    tmp = _EXE + f".{os.getpid()}.tmp"
    cmd = ["g++", "-std=gnu++17", "-O1", "-w", "-I", _HERE, "-I", _BUILD, "-o", tmp,
           os.path.join(_HERE, "opcount_main.cpp")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"op-count build failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, _EXE)
    return _EXE


def _run(args, payload: bytes) -> list[dict]:
    exe = build()
    r = subprocess.run([exe, *map(str, args)], input=payload, capture_output=True, timeout=3600)
    if r.returncode != 0:
        raise RuntimeError(f"op-count run failed ({r.returncode}): {r.stderr.decode()[-2000:]}")
    return [json.loads(l) for l in r.stdout.decode().splitlines() if l.strip()]


def _f64(a) -> bytes:
    return np.ascontiguousarray(a, dtype="<f8").tobytes()


def self_test() -> list[dict]:
    """Counts of small expressions with known answers (see opcount_main.cpp)."""
    return _run(["selftest"], b"")


def gks_point(m: int, cases, gamma=1.4, c1=0.05, c2=1.0, tau_mode=0, mu=0.0) -> list[dict]:
    """Counts of one or_gks_point call per case (Wl, Wr, dWl[m][nv], dWr[m][nv], dt)."""
    nv = m + 2
    buf = bytearray()
    for Wl, Wr, dWl, dWr, dt in cases:
        buf += _f64(Wl) + _f64(Wr) + _f64(np.reshape(dWl, (m, nv))) + _f64(np.reshape(dWr, (m, nv))) + _f64([dt])
    return _run(["gks", m, len(cases), gamma, c1, c2, tau_mode, mu], bytes(buf))


def step(dim: int, n, h: float, dt: float, W, G, gamma=1.4, bc=0, what="step", limiter=0) -> dict:
    """Counts of one oracle call on a whole grid: what = "step" (or_step, both
    stages), "flux" (or_flux: reconstruction + flux of one stage) or "recon"
    (or_reconstruct: the interface states of one stage)."""
    nn = list(n) + [1] * (3 - len(n))
    payload = _f64(W) + _f64(G)
    return _run([what, dim, nn[0], nn[1], nn[2], repr(h), repr(dt), gamma, bc, limiter], payload)[0]


def genomd_cells(dim: int, cells, limiter=0) -> list[dict]:
    """Counts of the multi-D GENO cubic of one cell per entry (or_genomd_cell
    inputs: W0, D0[m], then per face neighbour Wn, Dn[m]; cell units)."""
    buf = bytearray()
    for c in cells:
        buf += _f64(c)
    return _run(["cell", dim, len(cells), limiter], bytes(buf))


def nc_step(order: int, n: int, h: float, dt: float, W, gamma=1.4, bc=0) -> dict:
    """Counts of one classical RK4 step of the 1D non-compact GENO scheme of
    the given order (5 or 6) with the HLLC flux on n cells (or_nc_step)."""
    return _run(["ncstep", order, n, repr(h), repr(dt), gamma, bc], _f64(W))[0]
