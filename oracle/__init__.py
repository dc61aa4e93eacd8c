"""Plain double-precision CPU oracle for the ultra-relativistic lattice
Boltzmann step (Mohseni, Mendoza, Succi, Herrmann, arXiv:1302.1125).

TEST INFRASTRUCTURE ONLY.  This package is the reference that the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library (``paper_1302_1125_gb300``) and never imports it.

``rlb_oracle.c`` holds the arithmetic (plain C, FP64, -ffp-contract=off);
this module only compiles it and marshals numpy arrays through ctypes.
``riemann.py`` is the exact ideal-fluid Riemann solver used as a pin.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

BC_PERIODIC, BC_OUTFLOW, BC_INLET = 0, 1, 2
LIMITER_MINMOD, LIMITER_NONE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over cells, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "rlb_oracle.h"))
    ):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC",
           "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3)]


class _Params(C.Structure):
    _fields_ = [("g", _Grid), ("dt", C.c_double), ("eta_over_s", C.c_double),
                ("zeta_over_s", C.c_double), ("tau_override", C.c_double),
                ("alpha_override", C.c_double), ("inlet_n", C.c_double),
                ("inlet_T", C.c_double), ("inlet_u", C.c_double * 3),
                ("limiter", C.c_int), ("euler_mode", C.c_int), ("model", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # RLB_ORACLE_LIB points the test suite's mutation check at a copy of
        # the oracle compiled with a planted mistake
        path = os.environ.get("RLB_ORACLE_LIB") or build()
        _lib = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        _lib.orc_lattice.restype = C.c_double
        _lib.orc_lattice.argtypes = [C.POINTER(C.c_int), dp, dp, dp]
        _lib.orc_feq.argtypes = [C.c_double, dp, dp]
        _lib.orc_heq.argtypes = [C.c_double, dp, dp]
        _lib.orc_moments.argtypes = [dp, dp, dp]
        _lib.orc_recover.argtypes = [dp, dp]
        _lib.orc_recover.restype = C.c_int
        _lib.orc_tau.argtypes = [C.POINTER(_Params), C.c_double, C.c_double]
        _lib.orc_tau.restype = C.c_double
        _lib.orc_alpha.argtypes = [C.POINTER(_Params)]
        _lib.orc_alpha.restype = C.c_double
        _lib.orc_minmod.argtypes = [C.c_double, C.c_double]
        _lib.orc_minmod.restype = C.c_double
        _lib.orc_stream.argtypes = [C.POINTER(_Params), dp, C.c_double, dp, C.c_double, dp]
        _lib.orc_laplacian.argtypes = [C.POINTER(_Params), dp, C.c_double, dp]
        _lib.orc_init.argtypes = [C.POINTER(_Params)] + [dp] * 8
        _lib.orc_step.argtypes = [C.POINTER(_Params)] + [dp] * 5
        _lib.orc_step.restype = C.c_long
        _lib.orc_step_cells.argtypes = [C.POINTER(_Params), C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int, C.c_long, C.POINTER(C.c_long), dp, dp, dp]
        _lib.orc_step_cells.restype = C.c_long
        _lib.orc_solid_reset.argtypes = [C.POINTER(_Params), C.c_void_p, C.c_double, C.c_double, dp, dp, dp]
        _lib.orc_solid_reset.restype = None
        _lib.orc_macroscopic.argtypes = [C.POINTER(_Params), dp, dp, dp]
        _lib.orc_macroscopic.restype = C.c_long
        _lib.orc_nu.restype = C.c_double
        _lib.orc_set_model.argtypes = [C.c_int]
        _lib.orc_get_model.restype = C.c_int
        _lib.orc_set_threads.argtypes = [C.c_int]
        _lib.orc_get_threads.restype = C.c_int
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def set_model(model: int) -> None:
    """lattice used by the functions without Params: 0 extended, 1 basic"""
    lib().orc_set_model(int(model))


def nu(model: int = 0) -> float:
    """the lattice constant nu = c/c_s: sqrt(13) (extended), sqrt(19) (basic)"""
    set_model(model)
    return float(lib().orc_nu())


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


@dataclass
class Params:
    nx: int
    ny: int = 1
    nz: int = 1
    bc_lo: tuple = (BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC)
    bc_hi: tuple = (BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC)
    dt: float = 0.25
    eta_over_s: float = 0.1
    zeta_over_s: float = 0.0
    tau_override: float = 0.0
    alpha_override: float = -1.0
    inlet_n: float = 1.0
    inlet_T: float = 1.0
    inlet_u: tuple = (0.0, 0.0, 0.0)
    limiter: int = LIMITER_MINMOD
    euler_mode: int = 0
    model: int = 0          # 0 extended lattice (Sec. II.A), 1 basic lattice (Sec. II)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def c(self) -> _Params:
        g = _Grid(self.nx, self.ny, self.nz, (C.c_int * 3)(*self.bc_lo), (C.c_int * 3)(*self.bc_hi))
        return _Params(g, self.dt, self.eta_over_s, self.zeta_over_s, self.tau_override,
                       self.alpha_override, self.inlet_n, self.inlet_T,
                       (C.c_double * 3)(*self.inlet_u), self.limiter, self.euler_mode, self.model)


def lattice(model: int = 0):
    """(e[19,3] int, c[19,3], w[19], wh[19], xi0) as the oracle builds them."""
    set_model(model)
    e = np.zeros((19, 3), np.int32)
    c = np.zeros((19, 3))
    w = np.zeros(19)
    wh = np.zeros(19)
    xi0 = lib().orc_lattice(e.ctypes.data_as(C.POINTER(C.c_int)), _p(c), _p(w), _p(wh))
    return e, c, w, wh, xi0


def feq(P: float, up, model: int = 0) -> np.ndarray:
    set_model(model)
    out = np.zeros(19)
    lib().orc_feq(float(P), _p(np.ascontiguousarray(up, np.float64)), _p(out))
    return out


def heq(n: float, up, model: int = 0) -> np.ndarray:
    set_model(model)
    out = np.zeros(19)
    lib().orc_heq(float(n), _p(np.ascontiguousarray(up, np.float64)), _p(out))
    return out


def moments(f, h, model: int = 0) -> np.ndarray:
    set_model(model)
    out = np.zeros(5)
    lib().orc_moments(_p(np.ascontiguousarray(f, np.float64)),
                      _p(np.ascontiguousarray(h, np.float64)), _p(out))
    return out


def recover(mom, model: int = 0):
    set_model(model)
    out = np.zeros(5)
    bad = lib().orc_recover(_p(np.ascontiguousarray(mom, np.float64)), _p(out))
    return out, bool(bad)


def tau(p: Params, P: float, n: float) -> float:
    cp = p.c()
    return lib().orc_tau(C.byref(cp), float(P), float(n))


def alpha(p: Params) -> float:
    cp = p.c()
    return lib().orc_alpha(C.byref(cp))


def minmod(X: float, Y: float) -> float:
    return lib().orc_minmod(float(X), float(Y))


def stream(p: Params, q: np.ndarray, pa, k: float, ghost: float = 0.0) -> np.ndarray:
    q = np.ascontiguousarray(q, np.float64).reshape(-1)
    out = np.zeros_like(q)
    cp = p.c()
    lib().orc_stream(C.byref(cp), _p(q), float(ghost), _p(np.asarray(pa, np.float64)),
                     float(k), _p(out))
    return out


def laplacian(p: Params, q: np.ndarray, ghost: float = 0.0) -> np.ndarray:
    q = np.ascontiguousarray(q, np.float64).reshape(-1)
    out = np.zeros_like(q)
    cp = p.c()
    lib().orc_laplacian(C.byref(cp), _p(q), float(ghost), _p(out))
    return out


@dataclass
class State:
    p: Params
    f: np.ndarray = field(repr=False)
    h: np.ndarray = field(repr=False)
    prev: np.ndarray = field(repr=False)
    nonphysical: int = 0
    solid: tuple = None     # (mask uint8[N], n, T): cells held at equilibrium


def init(p: Params, n, T, ux, uy, uz) -> State:
    N = p.N
    arrs = [np.ascontiguousarray(np.broadcast_to(a, (N,)), np.float64) for a in (n, T, ux, uy, uz)]
    f = np.zeros(19 * N)
    h = np.zeros(19 * N)
    prev = np.zeros(5 * N)
    cp = p.c()
    lib().orc_init(C.byref(cp), *[_p(a) for a in arrs], _p(f), _p(h), _p(prev))
    return State(p, f, h, prev)


def step(s: State, nsteps: int = 1) -> State:
    """Advance ``nsteps`` time steps in place (double-buffered internally)."""
    cp = s.p.c()
    fo = np.empty_like(s.f)
    ho = np.empty_like(s.h)
    for _ in range(int(nsteps)):
        s.nonphysical += lib().orc_step(C.byref(cp), _p(s.f), _p(s.h), _p(s.prev), _p(fo), _p(ho))
        s.f, fo = fo, s.f
        s.h, ho = ho, s.h
        if s.solid is not None:
            _solid_reset(s)
    return s


def _solid_reset(s: State):
    mask, n, T = s.solid
    cp = s.p.c()
    lib().orc_solid_reset(C.byref(cp), mask.ctypes.data, float(n), float(T), _p(s.f), _p(s.h), _p(s.prev))


def set_solid(s: State, mask, n: float, T: float) -> State:
    """Hold the cells where mask != 0 at the equilibrium of (n, T, u = 0):
    applied now and after every step (orc_solid_reset)."""
    m = np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0, np.uint8)
    assert m.size == s.p.N
    s.solid = (m, float(n), float(T))
    _solid_reset(s)
    return s


def step_cells(p: Params, f, h, prev, cells) -> tuple:
    """One update of the listed cells only, from full-size float32 or float64
    state (as laid out above).  Returns (f[k,19], h[k,19], macros[k,5], bad)."""
    f = np.ascontiguousarray(f).reshape(-1)
    h = np.ascontiguousarray(h).reshape(-1)
    prev = np.ascontiguousarray(prev).reshape(-1)
    assert f.dtype == h.dtype == prev.dtype and f.dtype in (np.float32, np.float64)
    cells = np.ascontiguousarray(cells, np.int64)
    k = cells.size
    fo = np.zeros((k, 19))
    ho = np.zeros((k, 19))
    mo = np.zeros((k, 5))
    cp = p.c()
    bad = lib().orc_step_cells(C.byref(cp), f.ctypes.data, h.ctypes.data, prev.ctypes.data,
                               int(f.dtype == np.float32), k,
                               cells.ctypes.data_as(C.POINTER(C.c_long)),
                               _p(fo), _p(ho), _p(mo))
    return fo, ho, mo, bad


def macroscopic(s: State) -> np.ndarray:
    """(6, N): n, e, u_x, u_y, u_z, gamma."""
    out = np.zeros(6 * s.p.N)
    cp = s.p.c()
    lib().orc_macroscopic(C.byref(cp), _p(s.f), _p(s.h), _p(out))
    return out.reshape(6, s.p.N)
