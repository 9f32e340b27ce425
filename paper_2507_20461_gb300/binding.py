"""Thin ctypes binding of ``libgenogks.so`` (the C ABI in include/genogks.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Arrays may be torch CUDA tensors (device pointers, on the
current torch stream) or numpy / CPU arrays (host pointers).  There is no
CPU fallback: if the library cannot be loaded every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

OK = 0
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NONPHYSICAL, ERR_UNSUPPORTED = -1, -2, -3, -4, -6
ST_RHO, ST_P, ST_NAN, ST_FLUX = 1, 2, 4, 8
BC_PERIODIC, BC_TRANSMISSIVE, BC_REFLECTIVE, BC_NOSLIP = 0, 1, 2, 3
LIMITER_GENO, LIMITER_LINEAR, LIMITER_WENOZ, LIMITER_TENO = 0, 1, 2, 3


class GksError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"genogks error {code}: {msg}")
        self.code = code


class Grid(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class Opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("limiter", C.c_int),
        ("C", C.c_double),
        ("eps", C.c_double),
        ("C0", C.c_double),
        ("c1_tau", C.c_double),
        ("c2_tau", C.c_double),
        ("adm_delta", C.c_double),
        ("stream", C.c_void_p),
        ("workspace", C.c_void_p),
        ("workspace_bytes", C.c_size_t),
        ("mu", C.c_double),
        ("ao_d0", C.c_double),
        ("teno_ct", C.c_double),
        ("stage_kernels", C.c_int),
    ]


_OPT_CONSTS = ("C", "eps", "C0", "c1_tau", "c2_tau", "adm_delta", "mu", "ao_d0", "teno_ct")


def _set_consts(o: Opts, consts: dict) -> None:
    """Scheme constants by keyword (an unknown name is an error, not a new
    Python attribute of the ctypes structure)."""
    for k, v in consts.items():
        if k not in _OPT_CONSTS:
            raise TypeError(f"unknown scheme constant {k!r} (expected one of {_OPT_CONSTS})")
        setattr(o, k, float(v))


_lib = None


def lib(build: bool = True):
    """Load (building first if needed) the in-tree library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libgenogks.so not found at {path}; run __graft_entry__.build()")
    L = C.CDLL(path)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    gp, op = C.POINTER(Grid), C.POINTER(Opts)
    sig = {
        "gks_default_opts": (None, [op]),
        "gks_workspace_bytes": (C.c_size_t, [gp, C.c_int]),
        "gks_face_count": (C.c_long, [gp]),
        "geno_gks_create": (C.c_int, [gp, C.c_double, C.c_int, C.c_int, op, C.POINTER(vp)]),
        "geno_gks_create_sides": (C.c_int, [gp, C.c_double, C.c_int, C.POINTER(C.c_int), op, C.POINTER(vp)]),
        "gks_set_state": (C.c_int, [vp, vp, vp, C.c_int]),
        "gks_get_state": (C.c_int, [vp, vp, vp, C.c_int]),
        "geno_reconstruct": (C.c_int, [vp, vp, C.c_int]),
        "gks_flux": (C.c_int, [vp, C.c_double, vp, C.c_int]),
        "gks_step": (C.c_int, [vp, C.c_double]),
        "gks_step_cfl": (C.c_int, [vp, C.c_double, C.c_int]),
        "gks_max_wavespeed": (C.c_int, [vp, dp]),
        "gks_status": (C.c_int, [vp]),
        "gks_destroy": (C.c_int, [vp]),
        "gks_profile_enable": (C.c_int, [vp, C.c_int, C.c_int]),
        "gks_profile_read": (C.c_int, [vp, C.c_int, C.POINTER(C.c_long), dp]),
        "gks_last_error": (C.c_char_p, [vp]),
        "gks_batch_create": (C.c_int, [C.c_int, ip, ip, dp, C.c_double, C.c_int, op, C.POINTER(vp)]),
        "gks_batch_set_state": (C.c_int, [vp, C.c_int, vp, vp, C.c_int]),
        "gks_batch_get_state": (C.c_int, [vp, C.c_int, vp, vp, C.c_int]),
        "gks_batch_run": (C.c_int, [vp, C.c_double, C.c_int]),
        "gks_batch_status": (C.c_int, [vp]),
        "gks_batch_grid_status": (C.c_int, [vp, C.POINTER(C.c_int), C.c_int]),
        "gks_batch_destroy": (C.c_int, [vp]),
        "gks_batch_last_error": (C.c_char_p, [vp]),
        "gks_batch_tuning": (C.c_char_p, [vp]),
        "geno_linearity": (C.c_int, [op, C.c_int, C.c_int, C.c_int, C.c_long, vp, vp, vp, vp]),
        "gks_pipe_probe": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_double), vp]),
    }
    for name, (res, args) in sig.items():
        if hasattr(L, name):
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
    _lib = L
    return L


def _ptr(a):
    """(pointer, on_device) of a torch tensor or numpy array of float64."""
    try:
        import torch

        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                raise ValueError("tensors must be contiguous float64")
            return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    except ImportError:
        pass
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags.c_contiguous:
        raise ValueError("arrays must be C-contiguous float64")
    return C.c_void_p(a.ctypes.data), 0


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch

            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    return C.c_void_p(getattr(stream, "cuda_stream", stream))


def default_opts() -> Opts:
    o = Opts()
    lib().gks_default_opts(C.byref(o))
    return o


def make_grid(n, lo=None, hi=None) -> Grid:
    dim = len(n)
    nn = list(n) + [1] * (3 - dim)
    lo = list(lo) if lo is not None else [0.0] * dim
    hi = list(hi) if hi is not None else [1.0] * dim
    lo += [0.0] * (3 - dim)
    hi += [1.0] * (3 - dim)
    return Grid(dim, (C.c_int * 3)(*nn), (C.c_double * 3)(*lo), (C.c_double * 3)(*hi))


def _check(h, r, fn="gks_last_error"):
    if r < 0:
        msg = getattr(lib(), fn)(h)
        raise GksError(r, msg.decode() if msg else "")
    return r


def face_count(grid: Grid) -> int:
    return int(lib().gks_face_count(C.byref(grid)))


def workspace_bytes(grid: Grid, precision: int = 0) -> int:
    return int(lib().gks_workspace_bytes(C.byref(grid), precision))


def geno_linearity(IS, tau, chi, limiter: int, r: int = 2, precision: int = 0, stream=None, **consts):
    """chi[i] of the nonlinear weights for the indicator sets IS[i, :] and
    IS^tau = tau[i] on the device (see include/genogks.h); device float64
    tensors IS (n x k), tau (n), chi (n)."""
    o = default_opts()
    o.precision = precision
    _set_consts(o, consts)
    n, k = IS.shape
    pi, di = _ptr(IS)
    pt, dt_ = _ptr(tau)
    pc, dc = _ptr(chi)
    if not (di and dt_ and dc):
        raise ValueError("IS, tau and chi must be device tensors")
    sp = _stream_ptr(stream)
    r_ = lib().geno_linearity(C.byref(o), int(limiter), int(r), int(k), int(n), pi, pt, pc, sp)
    _check(None, r_)


def geno_gks_create(grid: Grid, gamma: float, order: int, bc, opts: Opts | None = None):
    """bc: one boundary type for every side, or six (x lo, x hi, y lo, y hi,
    z lo, z hi) through geno_gks_create_sides."""
    h = C.c_void_p()
    op = C.byref(opts) if opts is not None else None
    if isinstance(bc, (int, np.integer)):
        r = lib().geno_gks_create(C.byref(grid), gamma, order, int(bc), op, C.byref(h))
    else:
        sides = [int(b) for b in bc]
        if len(sides) != 6:
            raise ValueError("per-side boundary conditions need six entries")
        r = lib().geno_gks_create_sides(C.byref(grid), gamma, order, (C.c_int * 6)(*sides), op, C.byref(h))
    _check(None, r)
    return h


def gks_set_state(h, W, G):
    pw, dw = _ptr(W)
    pg, dg = _ptr(G)
    if dw != dg:
        raise ValueError("W and G must both be on the device or both on the host")
    return _check(h, lib().gks_set_state(h, pw, pg, dw))


def gks_get_state(h, W, G):
    pw, dw = _ptr(W)
    pg, dg = _ptr(G)
    if dw != dg:
        raise ValueError("W and G must both be on the device or both on the host")
    return _check(h, lib().gks_get_state(h, pw, pg, dw))


def geno_reconstruct(h, out):
    p, d = _ptr(out)
    return _check(h, lib().geno_reconstruct(h, p, d))


def gks_flux(h, dt: float, out):
    p, d = _ptr(out)
    return _check(h, lib().gks_flux(h, float(dt), p, d))


def gks_step(h, dt: float):
    return _check(h, lib().gks_step(h, float(dt)))


def gks_step_cfl(h, cfl: float, nsteps: int):
    return _check(h, lib().gks_step_cfl(h, float(cfl), int(nsteps)))


def gks_max_wavespeed(h) -> float:
    s = C.c_double()
    _check(h, lib().gks_max_wavespeed(h, C.byref(s)))
    return s.value


def gks_status(h) -> int:
    return _check(h, lib().gks_status(h))


KC_RECON, KC_FACE, KC_UPDATE, KC_DT, KC_STAGE = 0, 1, 2, 3, 4


def gks_profile_enable(h, on: bool = True, reset: bool = True):
    return _check(h, lib().gks_profile_enable(h, int(on), int(reset)))


def gks_profile_read(h, kernel_class: int):
    n = C.c_long()
    ms = C.c_double()
    _check(h, lib().gks_profile_read(h, kernel_class, C.byref(n), C.byref(ms)))
    return n.value, ms.value


def gks_destroy(h):
    return lib().gks_destroy(h)


def gks_last_error(h) -> str:
    m = lib().gks_last_error(h)
    return m.decode() if m else ""


def gks_batch_create(nx, ny, hs, gamma: float, bc: int, opts: Opts | None = None):
    nb = len(nx)
    ax = (C.c_int * nb)(*nx)
    ay = (C.c_int * nb)(*ny)
    ah = (C.c_double * nb)(*hs)
    h = C.c_void_p()
    r = lib().gks_batch_create(nb, ax, ay, ah, gamma, bc, C.byref(opts) if opts is not None else None, C.byref(h))
    _check(None, r, "gks_batch_last_error")
    return h


def gks_batch_set_state(b, grid: int, W, G):
    pw, dw = _ptr(W)
    pg, dg = _ptr(G)
    if dw != dg:
        raise ValueError("W and G must both be on the device or both on the host")
    return _check(b, lib().gks_batch_set_state(b, grid, pw, pg, dw), "gks_batch_last_error")


def gks_batch_get_state(b, grid: int, W, G):
    pw, dw = _ptr(W)
    pg, dg = _ptr(G)
    if dw != dg:
        raise ValueError("W and G must both be on the device or both on the host")
    return _check(b, lib().gks_batch_get_state(b, grid, pw, pg, dw), "gks_batch_last_error")


def gks_batch_run(b, cfl: float, nsteps: int):
    return _check(b, lib().gks_batch_run(b, float(cfl), int(nsteps)), "gks_batch_last_error")


def gks_batch_status(b) -> int:
    return _check(b, lib().gks_batch_status(b), "gks_batch_last_error")


def gks_batch_grid_status(b, n: int) -> list:
    out = (C.c_int * n)()
    _check(b, lib().gks_batch_grid_status(b, out, n), "gks_batch_last_error")
    return list(out)


def gks_batch_tuning(b) -> str:
    m = lib().gks_batch_tuning(b)
    return m.decode() if m else ""


def gks_batch_destroy(b):
    return lib().gks_batch_destroy(b)


class Batch:
    """Handle wrapper of the batched 2D mode."""

    def __init__(self, nx, ny, hs, gamma=1.4, bc=BC_TRANSMISSIVE, precision=1, limiter=0, stream=None, **consts):
        o = default_opts()
        o.precision = precision
        o.limiter = limiter
        _set_consts(o, consts)
        sp = _stream_ptr(stream)
        o.stream = sp.value if sp is not None else None
        self.nx, self.ny = list(nx), list(ny)
        self.h = gks_batch_create(self.nx, self.ny, hs, gamma, bc, o)

    def set_state(self, g, W, G):
        gks_batch_set_state(self.h, g, W, G)

    def get_state(self, g, W, G):
        gks_batch_get_state(self.h, g, W, G)

    def run(self, cfl, nsteps):
        gks_batch_run(self.h, cfl, nsteps)

    def status(self):
        return gks_batch_status(self.h)

    def grid_status(self):
        """Status word of every grid (0: its states stayed admissible)."""
        return gks_batch_grid_status(self.h, len(self.nx))

    def tuning(self):
        return gks_batch_tuning(self.h)

    def close(self):
        if self.h is not None:
            gks_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Handle wrapper: ``Solver(n=(nx, ny), lo, hi, gamma, bc, precision)``."""

    def __init__(self, n, lo=None, hi=None, gamma=1.4, bc=BC_PERIODIC, precision=0, limiter=0, stream=None, order=None,
                 stage_kernels=0, **consts):
        self.grid = make_grid(n, lo, hi)
        self.dim = len(n)
        self.nv = self.dim + 2
        self.n = tuple(n)
        o = default_opts()
        o.precision = precision
        o.limiter = limiter
        o.stage_kernels = stage_kernels
        _set_consts(o, consts)
        sp = _stream_ptr(stream)
        o.stream = sp.value if sp is not None else None
        self.opts = o
        if order is None:
            order = 8 if self.dim == 1 else 4
        self.order = order
        self.h = geno_gks_create(self.grid, gamma, order, bc, o)

    @property
    def shape(self):
        return tuple(reversed(self.n))

    @property
    def nfaces(self):
        return face_count(self.grid)

    @property
    def ngauss(self):
        return {1: 1, 2: 2, 3: 4}[self.dim]

    def set_state(self, W, G):
        gks_set_state(self.h, W, G)

    def get_state(self, W, G):
        gks_get_state(self.h, W, G)

    def reconstruct(self, out):
        geno_reconstruct(self.h, out)

    def flux(self, dt, out):
        gks_flux(self.h, dt, out)

    def step(self, dt):
        gks_step(self.h, dt)

    def step_cfl(self, cfl, nsteps=1):
        gks_step_cfl(self.h, cfl, nsteps)

    def max_wavespeed(self):
        return gks_max_wavespeed(self.h)

    def status(self):
        return gks_status(self.h)

    def profile(self, on=True, reset=True):
        gks_profile_enable(self.h, on, reset)

    def profile_read(self, kernel_class):
        return gks_profile_read(self.h, kernel_class)

    def close(self):
        if self.h is not None:
            gks_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PIPE_FFMA, PIPE_DFMA, PIPE_MUFU, PIPE_FFMA2 = 0, 1, 2, 3


def pipe_probe(kind: int, iters: int, stream=None) -> float:
    """Measured throughput (flops or ops per second) of one arithmetic pipe:
    PIPE_FFMA, PIPE_DFMA (2 flops per FMA), PIPE_MUFU (1 op per ex2) or
    PIPE_FFMA2 (packed two-lane FP32 FMA, 4 flops per instruction)."""
    out = C.c_double()
    sp = _stream_ptr(stream)
    _check(None, lib().gks_pipe_probe(int(kind), int(iters), C.byref(out), sp))
    return float(out.value)
