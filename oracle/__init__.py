"""Oracle: plain FP64 CPU restatement of the compact GKS with GENO reconstruction.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU
baseline of the benchmark import this package.  It shares no code with the
CUDA library (``paper_2507_20461_gb300``); neither imports the other.

The arithmetic lives in ``geno_gks_oracle.c`` (plain C, long double for the
polynomial fits, double elsewhere), compiled here into ``liboracle.so`` by
:func:`build`.  The exact Riemann solver used by pin P9 is ``riemann.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "geno_gks_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK = 0
ERR_ARG = -1
ERR_NONPHYSICAL = -4


class Cfg(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("n", C.c_int * 3),
        ("h", C.c_double),
        ("gamma", C.c_double),
        ("bc", C.c_int),
        ("C", C.c_double),
        ("eps", C.c_double),
        ("C0", C.c_double),
        ("c1_tau", C.c_double),
        ("c2_tau", C.c_double),
        ("limiter", C.c_int),
        ("tau_mode", C.c_int),
        ("adm_delta", C.c_double),
        ("mu", C.c_double),
        ("bcs", C.c_int * 6),
        ("ao_d0", C.c_double),
        ("teno_ct", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (-O2, OpenMP, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        dp = C.POINTER(C.c_double)
        cp = C.POINTER(Cfg)
        L.or_face_total.argtypes = [cp]
        L.or_face_total.restype = C.c_long
        L.or_reconstruct.argtypes = [cp, dp, dp, dp]
        L.or_flux.argtypes = [cp, C.c_double, dp, dp, dp]
        L.or_step.argtypes = [cp, C.c_double, dp, dp]
        L.or_max_wavespeed.argtypes = [cp, dp]
        L.or_max_wavespeed.restype = C.c_double
        L.or_geno1d_point.argtypes = [cp, dp, dp, C.c_int, dp]
        L.or_genomd_cell.argtypes = [cp, dp, dp]
        L.or_monomials.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int)]
        L.or_gks_point.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_int, C.c_double, C.c_double, dp, dp, dp, dp, dp, dp, dp]
        L.or_max_kin_viscosity.argtypes = [cp, dp]
        L.or_max_kin_viscosity.restype = C.c_double
        L.or_slope_solve.argtypes = [C.c_int, C.c_double, dp, dp, dp]
        L.or_nc_reconstruct.argtypes = [cp, C.c_int, dp, dp]
        L.or_nc_flux.argtypes = [cp, C.c_int, dp, dp]
        L.or_nc_step.argtypes = [cp, C.c_int, C.c_double, dp]
        L.or_nc_point.argtypes = [cp, C.c_int, dp, dp]
        L.or_moment_matrix.argtypes = [C.c_int, C.c_double, dp, dp]
        L.or_mom_half.argtypes = [C.c_int, C.c_double, C.c_double, C.c_int]
        L.or_mom_half.restype = C.c_double
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_cfg(dim, n, h, gamma=1.4, bc=0, C_=20.0, eps=1e-15, C0=8.0, c1_tau=0.05, c2_tau=1.0, limiter=0, tau_mode=0, adm_delta=0.3, mu=0.0, ao_d0=0.85, teno_ct=1e-6) -> Cfg:
    nn = list(n) + [1] * (3 - len(n))
    if mu > 0.0 and tau_mode == 0:
        tau_mode = 2
    # bc: one code for every side, or six (x lo, x hi, y lo, y hi, z lo, z hi)
    sides = [int(bc)] * 6 if np.isscalar(bc) else [int(b) for b in bc]
    if len(sides) != 6:
        raise ValueError("per-side boundary conditions need six entries")
    return Cfg(dim, (C.c_int * 3)(*nn), h, gamma, sides[0], C_, eps, C0, c1_tau, c2_tau, limiter, tau_mode, adm_delta,
               mu, (C.c_int * 6)(*sides), ao_d0, teno_ct)


def ngauss(dim: int) -> int:
    return {1: 1, 2: 2, 3: 4}[dim]


def face_total(cfg: Cfg) -> int:
    return int(lib().or_face_total(C.byref(cfg)))


def reconstruct(cfg: Cfg, W: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Interface states [side][var][comp][gauss][face] (comp 0 value, 1+e d/dx_e)."""
    m = cfg.dim
    nv = m + 2
    out = np.zeros((2, nv, m + 1, ngauss(m), face_total(cfg)))
    W = np.ascontiguousarray(W, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    r = lib().or_reconstruct(C.byref(cfg), _p(W), _p(G), _p(out))
    if r != OK:
        raise RuntimeError(f"oracle reconstruct failed: {r}")
    return out


def flux(cfg: Cfg, dt: float, W: np.ndarray, G: np.ndarray) -> np.ndarray:
    """Face quantities [q][var][gauss][face], q = F, dF/dt, W(dt/2)."""
    m = cfg.dim
    nv = m + 2
    out = np.zeros((3, nv, ngauss(m), face_total(cfg)))
    W = np.ascontiguousarray(W, dtype=np.float64)
    G = np.ascontiguousarray(G, dtype=np.float64)
    r = lib().or_flux(C.byref(cfg), float(dt), _p(W), _p(G), _p(out))
    if r != OK:
        raise RuntimeError(f"oracle flux failed: {r}")
    return out


def step(cfg: Cfg, dt: float, W: np.ndarray, G: np.ndarray) -> int:
    """One two-stage step in place; returns the status code."""
    assert W.dtype == np.float64 and W.flags.c_contiguous
    assert G.dtype == np.float64 and G.flags.c_contiguous
    return int(lib().or_step(C.byref(cfg), float(dt), _p(W), _p(G)))


def max_wavespeed(cfg: Cfg, W: np.ndarray) -> float:
    W = np.ascontiguousarray(W, dtype=np.float64)
    return float(lib().or_max_wavespeed(C.byref(cfg), _p(W)))


def max_kin_viscosity(cfg: Cfg, W: np.ndarray) -> float:
    W = np.ascontiguousarray(W, dtype=np.float64)
    return float(lib().or_max_kin_viscosity(C.byref(cfg), _p(W)))


def cfl_dt(cfg: Cfg, W: np.ndarray, cfl: float) -> float:
    """CFL time step with the viscous limit cfl h^2 / (2 (m - 1) nu) (Sec. 6;
    2 nu in 1D) when mu > 0."""
    dt = cfl * cfg.h / max_wavespeed(cfg, W)
    if cfg.mu > 0.0:
        nu = max_kin_viscosity(cfg, W)
        dt = min(dt, cfl * cfg.h * cfg.h / (2.0 * max(cfg.dim - 1, 1) * nu))
    return dt


def nc_reconstruct(cfg: Cfg, order: int, W: np.ndarray) -> np.ndarray:
    """1D non-compact GENO face states [side][v][face] (Sec. 4.1)."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros((2, 3, cfg.n[0] + 1))
    if lib().or_nc_reconstruct(C.byref(cfg), int(order), _p(W), _p(out)) != OK:
        raise RuntimeError("nc_reconstruct failed")
    return out


def nc_point(cfg: Cfg, order: int, u6) -> dict:
    """left value at x_{j+1/2} from averages at offsets -2..3, with its parts"""
    u6 = np.ascontiguousarray(u6, dtype=np.float64)
    out = np.zeros(11)
    if lib().or_nc_point(C.byref(cfg), int(order), _p(u6), _p(out)) != OK:
        raise RuntimeError("nc_point failed")
    k = 3 if order == 5 else 4
    return {"val": out[0], "qH": out[1], "chi": out[2], "p": out[3 : 3 + k].copy(), "IS": out[7 : 7 + k].copy()}


def nc_flux(cfg: Cfg, order: int, W: np.ndarray) -> np.ndarray:
    """HLLC fluxes [v][face] of the non-compact GENO states."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    out = np.zeros((3, cfg.n[0] + 1))
    r = lib().or_nc_flux(C.byref(cfg), int(order), _p(W), _p(out))
    if r != OK:
        raise RuntimeError(f"nc_flux failed ({r})")
    return out


def nc_step(cfg: Cfg, order: int, dt: float, W: np.ndarray) -> int:
    """One classical RK4 step of the non-compact scheme, in place."""
    assert W.flags.c_contiguous and W.dtype == np.float64
    return lib().or_nc_step(C.byref(cfg), int(order), float(dt), _p(W))


def geno1d_point(cfg: Cfg, w5, d5, side: int) -> dict:
    w5 = np.ascontiguousarray(w5, dtype=np.float64)
    d5 = np.ascontiguousarray(d5, dtype=np.float64)
    out = np.zeros(9)
    r = lib().or_geno1d_point(C.byref(cfg), _p(w5), _p(d5), int(side), _p(out))
    if r != OK:
        raise RuntimeError("geno1d failed")
    keys = ["val", "der", "chi", "IS1", "IS2", "IS3", "ISH", "ISL", "IStau"]
    return dict(zip(keys, out.tolist()))


def monomials(m: int, deg: int = 3) -> np.ndarray:
    e = (C.c_int * 300)()
    n = lib().or_monomials(m, deg, e)
    return np.array(e[: 3 * n]).reshape(n, 3)


def genomd_cell(cfg: Cfg, W0, D0, Wn, Dn) -> dict:
    m = cfg.dim
    inp = [W0] + list(D0)
    for q in range(2 * m):
        inp += [Wn[q]] + list(Dn[q])
    inp = np.array(inp, dtype=np.float64)
    out = np.zeros(40)
    nm = lib().or_genomd_cell(C.byref(cfg), _p(inp), _p(out))
    if nm < 0:
        raise RuntimeError("genomd failed")
    return {
        "coef": out[:nm].copy(),
        "chi": out[nm],
        "ISH": out[nm + 1],
        "ISL": out[nm + 2],
        "IStau": out[nm + 3],
        "IS": out[nm + 4 : nm + 4 + 2 * m].copy(),
    }


def gks_point(m, gamma, dt, Wl, Wr, dWl, dWr, c1=0.05, c2=1.0, tau_mode=0, mu=0.0):
    nv = m + 2
    Wl = np.ascontiguousarray(Wl, dtype=np.float64)
    Wr = np.ascontiguousarray(Wr, dtype=np.float64)
    dWl = np.ascontiguousarray(np.reshape(dWl, (m, nv)), dtype=np.float64)
    dWr = np.ascontiguousarray(np.reshape(dWr, (m, nv)), dtype=np.float64)
    F = np.zeros(nv)
    Ft = np.zeros(nv)
    Wh = np.zeros(nv)
    r = lib().or_gks_point(m, gamma, c1, c2, int(tau_mode), float(mu), dt, _p(Wl), _p(Wr), _p(dWl), _p(dWr), _p(F), _p(Ft), _p(Wh))
    if r != OK:
        raise RuntimeError("gks_point failed")
    return F, Ft, Wh


def slope_solve(m, gamma, W, rhs):
    W = np.ascontiguousarray(W, dtype=np.float64)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    s = np.zeros(m + 2)
    if lib().or_slope_solve(m, gamma, _p(W), _p(rhs), _p(s)) != OK:
        raise RuntimeError("slope solve failed")
    return s


def moment_matrix(m, gamma, W):
    W = np.ascontiguousarray(W, dtype=np.float64)
    M = np.zeros((m + 2, m + 2))
    if lib().or_moment_matrix(m, gamma, _p(W), _p(M)) != OK:
        raise RuntimeError("moment matrix failed")
    return M


def mom_half(n: int, U: float, lam: float, sign: int) -> float:
    return float(lib().or_mom_half(n, U, lam, sign))
