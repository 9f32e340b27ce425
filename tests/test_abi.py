"""The C-ABI library loads and exports every function include/*.h declares;
host-side argument checks and size queries work without a GPU."""
import ctypes as C
import glob
import json
import os
import re

import pytest

from paper_2507_20461_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(\w+)\s*\(([^;{]*)\)\s*;", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "return", "sizeof"):
                names.add(name)
    return names


def test_every_declared_symbol_is_exported():
    lib = B.lib()
    names = _declared()
    assert {"geno_gks_create", "geno_reconstruct", "gks_flux", "gks_step", "gks_destroy"} <= names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_default_opts_are_the_papers_constants():
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))
    o = B.default_opts()
    assert o.C == gold["C"]["value"]
    assert o.eps == gold["eps"]["value"]
    assert o.C0 == gold["C0"]["value"]
    assert o.teno_ct == gold["teno_ct"]["value"]
    assert o.precision == 0 and o.limiter == 0


def test_sizes_without_gpu():
    g = B.make_grid((10, 7), [0, 0], [1.0, 0.7])
    assert B.face_count(g) == 11 * 7 + 10 * 8
    assert B.workspace_bytes(g, 0) > B.workspace_bytes(g, 1) > 0
    g1 = B.make_grid((400,))
    assert B.face_count(g1) == 401
    g3 = B.make_grid((4, 5, 6), [0, 0, 0], [0.4, 0.5, 0.6])
    assert B.face_count(g3) == 5 * 5 * 6 + 4 * 6 * 6 + 4 * 5 * 7


@pytest.mark.parametrize(
    "n,lo,hi,order,gamma,bc",
    [
        ((0, 4), None, None, 4, 1.4, 0),        # empty axis
        ((4, 4), [0, 0], [1.0, 2.0], 4, 1.4, 0),  # unequal cell size
        ((8,), None, None, 4, 1.4, 0),          # 1D is order 8
        ((8, 8), None, None, 8, 1.4, 0),        # 2D is order 4
        ((8, 8), None, None, 4, 1.0, 0),        # gamma must exceed 1
        ((8, 8), None, None, 4, 1.4, 7),        # unknown boundary condition
    ],
)
def test_create_rejects_bad_arguments(n, lo, hi, order, gamma, bc):
    g = B.make_grid(n, lo, hi)
    h = C.c_void_p()
    r = B.lib().geno_gks_create(C.byref(g), gamma, order, bc, None, C.byref(h))
    assert r in (B.ERR_ARG, B.ERR_UNSUPPORTED)
    assert not h.value
    assert B.gks_last_error(None)


def test_null_handles_are_rejected():
    L = B.lib()
    assert L.gks_step(None, 0.1) == B.ERR_ARG
    assert L.gks_status(None) == B.ERR_ARG
    assert L.gks_destroy(None) == B.OK
    assert L.gks_batch_run(None, 0.4, 1) == B.ERR_ARG
    st = (C.c_int * 4)()
    assert L.gks_batch_grid_status(None, st, 4) == B.ERR_ARG


def test_fast_division_formula():
    """The kernels divide 32-bit indices by launch-fixed divisors as
    floor(M n / 2^64) with M = ceil(2^64 / d) (Lemire, Kaser and Kurz 2019,
    Theorem 1); the host computes M as floor((2^64 - 1) / d) + 1.  Exact for
    every n, d < 2^32 (checked here on edges and random samples)."""
    import random

    rng = random.Random(5)
    ds = [2, 3, 5, 7, 10, 64, 1000, 2049, 2050, 4097, 65535, 65536, 2**31 - 1, 2**31, 2**32 - 1]
    ds += [rng.randrange(2, 2**32) for _ in range(300)]
    for d in ds:
        M = (2**64 - 1) // d + 1
        ns = [0, 1, d - 1, d, d + 1, 2**32 - 1, (2**32 - 1) // d * d, (2**32 - 1) // d * d - 1]
        ns += [rng.randrange(0, 2**32) for _ in range(200)]
        for n in ns:
            if 0 <= n < 2**32:
                assert (M * n) >> 64 == n // d, (d, n)


def _static_flux():
    f = B.lib().gks_flux_2d_static
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_void_p,
                  C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
    return f


def _bad_opts(**kw):
    o = B.default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize(
    "nx,ny,h,opts",
    [
        (2**31 - 2, 10, 0.1, None),     # (nx + 2) wraps in 32-bit arithmetic
        (10, 2**31 - 2, 0.1, None),
        (2**31 - 1, 2**31 - 1, 0.1, None),
        (200, 200, 0.005, None),        # beyond the static scratch
        (10, 10, float("inf"), None),
        (10, 10, 0.1, dict(C=0.0)),     # 1 / tanh(0)
        (10, 10, 0.1, dict(eps=0.0)),
        (10, 10, 0.1, dict(C0=-1.0)),
        (10, 10, 0.1, dict(c1_tau=-0.1)),
        (10, 10, 0.1, dict(adm_delta=1.0)),
    ],
)
def test_static_flux_rejects_before_any_launch(nx, ny, h, opts):
    """gks_flux_2d_static turns sizes and constants it cannot use into
    GKS_ERR_ARG on the host, before it touches a GPU (so this runs without
    one); the pointers are never dereferenced."""
    o = C.byref(_bad_opts(**opts)) if opts else None
    p = C.c_void_p(256)
    r = _static_flux()(nx, ny, h, 1.4, B.BC_PERIODIC, o, p, p, 1e-3, p, None)
    assert r == B.ERR_ARG
