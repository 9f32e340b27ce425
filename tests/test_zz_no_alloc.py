"""gks_flux_2d_static: the flux entry point for callers that cannot allocate
device memory (its only scratch is a static device array inside the library)
must give the same face fluxes as gks_flux, call after call.

Collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2507_20461_gb300 import binding as B
from paper_2507_20461_gb300 import inputs as I

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _static_fn():
    f = B.lib().gks_flux_2d_static
    f.restype = C.c_int
    f.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_void_p,
                  C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]
    return f


def _state(nx, ny, seed):
    W, G, h = I.quadrants_2d(ny, seed=seed, nx=nx)
    rng = np.random.default_rng(seed)
    W = W * (1 + 0.01 * rng.random(W.shape))
    G = 0.2 * rng.normal(size=G.shape)
    return W, G, h


def _reference(nx, ny, h, bc, W, G, dt, limiter=0):
    s = B.Solver((nx, ny), lo=[0, 0], hi=[nx * h, ny * h], bc=bc, precision=0, limiter=limiter)
    s.set_state(torch.from_numpy(W).to(DEV), torch.from_numpy(G).to(DEV))
    out = torch.zeros(3 * 4 * 2 * s.nfaces, dtype=torch.float64, device=DEV)
    s.flux(dt, out)
    s.close()
    return out.cpu().numpy()


def _opts(limiter):
    o = B.default_opts()
    o.limiter = limiter
    return o


def test_static_flux_matches_gks_flux_twice():
    f = _static_fn()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(37, 29, 3, B.BC_TRANSMISSIVE, 0.002), (64, 50, 4, B.BC_PERIODIC, 0.001)]
    for nx, ny, seed, bc, dt in cases:  # two calls in a row, different sizes and states
        W, G, h = _state(nx, ny, seed)
        ref = _reference(nx, ny, h, bc, W, G, dt)
        Wd = torch.from_numpy(W).to(DEV)
        Gd = torch.from_numpy(G).to(DEV)
        out = torch.full((ref.size,), float("nan"), dtype=torch.float64, device=DEV)
        r = f(nx, ny, h, 1.4, bc, None, Wd.data_ptr(), Gd.data_ptr(), dt, out.data_ptr(), stream)
        assert r == B.OK
        got = out.cpu().numpy()
        scale = np.abs(ref).max()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * scale)


def test_static_flux_rejects_oversized_grid():
    f = _static_fn()
    W = torch.zeros(4 * 200 * 200, dtype=torch.float64, device=DEV)
    G = torch.zeros(2 * 4 * 200 * 200, dtype=torch.float64, device=DEV)
    out = torch.zeros(10, dtype=torch.float64, device=DEV)
    r = f(200, 200, 0.005, 1.4, B.BC_PERIODIC, None, W.data_ptr(), G.data_ptr(), 1e-3, out.data_ptr(), None)
    assert r == B.ERR_ARG


@pytest.mark.parametrize("bc,limiter", [(B.BC_REFLECTIVE, 0), (B.BC_NOSLIP, 0), (B.BC_TRANSMISSIVE, 2),
                                        (B.BC_PERIODIC, 3)])
def test_static_flux_walls_and_weight_variants(bc, limiter):
    """Slip and no-slip walls (mirrored ghosts with sign flips) and the
    WENO-Z / TENO weights go through the same kernels as gks_flux."""
    f = _static_fn()
    stream = torch.cuda.current_stream().cuda_stream
    nx, ny, dt = 33, 27, 0.0015
    W, G, h = _state(nx, ny, 11 + limiter + 3 * bc)
    ref = _reference(nx, ny, h, bc, W, G, dt, limiter)
    o = _opts(limiter)
    Wd, Gd = torch.from_numpy(W).to(DEV), torch.from_numpy(G).to(DEV)  # kept alive across the call
    for _ in range(2):
        out = torch.full((ref.size,), float("nan"), dtype=torch.float64, device=DEV)
        r = f(nx, ny, h, 1.4, bc, C.byref(o), Wd.data_ptr(), Gd.data_ptr(), dt, out.data_ptr(), stream)
        assert r == B.OK
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_static_flux_reports_a_nonphysical_state():
    """A block of cells at negative pressure leaves face states the flux
    cannot use: the call says so, and a later valid call is unaffected (the
    status word is cleared per call)."""
    f = _static_fn()
    stream = torch.cuda.current_stream().cuda_stream
    nx, ny, dt = 20, 16, 0.002
    W, G, h = _state(nx, ny, 5)
    Wbad = W.copy()
    # E below the kinetic energy: p < 0 in a 3 x 3 block
    ke = 0.5 * (Wbad[1] ** 2 + Wbad[2] ** 2) / Wbad[0]
    Wbad[3, 6:9, 8:11] = ke[6:9, 8:11] - 1.0
    out = torch.zeros(3 * 4 * 2 * ((nx + 1) * ny + nx * (ny + 1)), dtype=torch.float64, device=DEV)
    Wb, Gd = torch.from_numpy(Wbad).to(DEV), torch.from_numpy(G).to(DEV)  # kept alive across the calls
    r = f(nx, ny, h, 1.4, B.BC_PERIODIC, None, Wb.data_ptr(), Gd.data_ptr(), dt, out.data_ptr(), stream)
    assert r == B.ERR_NONPHYSICAL
    ref = _reference(nx, ny, h, B.BC_PERIODIC, W, G, dt)
    Wd = torch.from_numpy(W).to(DEV)
    r = f(nx, ny, h, 1.4, B.BC_PERIODIC, None, Wd.data_ptr(), Gd.data_ptr(), dt, out.data_ptr(), stream)
    assert r == B.OK
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())
