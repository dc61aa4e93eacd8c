"""Thin ctypes binding of librlb (include/rlb.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels of librlb.so.  The functions below carry the names of the C ABI;
``Grid`` wraps one context for convenience.  Device buffers are torch CUDA
tensors (PyTorch provides device memory and streams), host buffers are
numpy arrays or CPU tensors.  There is no CPU fallback: if librlb.so is
missing or no GPU is present the calls fail with an error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librlb.so")

RLB_OK, RLB_E_INVALID, RLB_E_NOMEM, RLB_E_CUDA = 0, -1, -2, -3
RLB_E_UNSTABLE, RLB_E_NONPHYSICAL, RLB_E_TIMEOUT = -4, -5, -6
LIMITER_MINMOD, LIMITER_NONE = 0, 1
BC_PERIODIC, BC_OUTFLOW, BC_INLET = 0, 1, 2
FP64, FP32_STORAGE = 0, 1
MODEL_EXTENDED, MODEL_BASIC = 0, 1
# rlb_options.thread_mapping; MAPPING_BULK_TILES: tiles staged by block-wide bulk copies
MAPPING_AUTO, MAPPING_TILES, MAPPING_LINEAR, MAPPING_BULK_TILES = 0, 1, 2, 3
Q = 19


class rlb_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("bc_lo", C.c_int * 3), ("bc_hi", C.c_int * 3),
                ("inlet_n", C.c_double), ("inlet_T", C.c_double), ("inlet_u", C.c_double * 3)]


class rlb_options(C.Structure):
    _fields_ = [("dt_over_dx", C.c_double), ("tau_override", C.c_double),
                ("alpha_override", C.c_double), ("euler_mode", C.c_int),
                ("precision", C.c_int), ("cuda_stream", C.c_void_p), ("symmetry_1d", C.c_int),
                ("model", C.c_int), ("thread_mapping", C.c_int), ("symmetry_2d", C.c_int),
                ("recovery_fp64", C.c_int), ("slab_rows", C.c_int)]


class rlb_batch_tuning(C.Structure):
    _fields_ = [("threads", C.c_int), ("bound", C.c_int), ("cluster", C.c_int),
                ("pairs_per_thread", C.c_int), ("ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class RLBError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status


_lib = None


def lib() -> C.CDLL:
    """Load librlb.so (built in-tree by paper_1302_1125_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run `python -m paper_1302_1125_gb300.build` "
                               "(the CUDA library is required, there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, dp = C.c_void_p, C.POINTER(C.c_double)
        ctxp = C.c_void_p
        L.rlb_default_options.argtypes = [C.POINTER(rlb_options)]
        L.rlb_default_options.restype = None
        L.rlb_check_config.argtypes = [C.POINTER(rlb_grid), C.c_int, C.c_double, C.c_double, C.c_int,
                                       C.POINTER(rlb_options)]
        L.rlb_check_config.restype = C.c_int
        L.rlb_create.argtypes = [C.POINTER(rlb_grid), C.c_int, C.c_double, C.c_double, C.c_int,
                                 C.POINTER(rlb_options), C.POINTER(ctxp)]
        L.rlb_create.restype = C.c_int
        L.rlb_init.argtypes = [ctxp, vp, vp, vp, vp, vp, C.c_int]
        L.rlb_init.restype = C.c_int
        L.rlb_step.argtypes = [ctxp, C.c_longlong]
        L.rlb_step.restype = C.c_int
        L.rlb_macroscopic.argtypes = [ctxp, vp, C.c_int]
        L.rlb_macroscopic.restype = C.c_int
        L.rlb_conserved_totals.argtypes = [ctxp, dp]
        L.rlb_conserved_totals.restype = C.c_int
        L.rlb_state_bytes.argtypes = [ctxp]
        L.rlb_state_bytes.restype = C.c_size_t
        L.rlb_get_state.argtypes = [ctxp, vp, C.c_size_t, C.c_int]
        L.rlb_get_state.restype = C.c_int
        L.rlb_set_state.argtypes = [ctxp, vp, C.c_size_t, C.c_int]
        L.rlb_set_state.restype = C.c_int
        L.rlb_set_stream.argtypes = [ctxp, vp]
        L.rlb_set_stream.restype = C.c_int
        L.rlb_launch_count.argtypes = [ctxp]
        L.rlb_launch_count.restype = C.c_longlong
        L.rlb_destroy.argtypes = [ctxp]
        L.rlb_destroy.restype = None
        L.rlb_last_error.argtypes = [ctxp]
        L.rlb_last_error.restype = C.c_char_p
        L.rlb_status_string.argtypes = [C.c_int]
        L.rlb_status_string.restype = C.c_char_p
        L.rlb_step_kernel.argtypes = [C.c_void_p]
        L.rlb_step_kernel.restype = C.c_char_p
        L.rlb_set_solid.argtypes = [ctxp, vp, C.c_double, C.c_double, C.c_int]
        L.rlb_set_solid.restype = C.c_int
        L.rlb_conserved_totals_noalloc.argtypes = [vp, vp, C.c_int, C.c_longlong, C.c_int, vp, vp]
        L.rlb_conserved_totals_noalloc.restype = C.c_int
        ip, llp, tp = C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(rlb_batch_tuning)
        L.rlb_batch_create.argtypes = [C.c_int, ip, dp, dp, C.c_int, C.POINTER(rlb_options), C.POINTER(vp)]
        L.rlb_batch_create.restype = C.c_int
        L.rlb_batch_init.argtypes = [vp, vp, vp, vp, C.c_int]
        L.rlb_batch_init.restype = C.c_int
        L.rlb_batch_step.argtypes = [vp, llp]
        L.rlb_batch_step.restype = C.c_int
        L.rlb_batch_macroscopic.argtypes = [vp, vp, C.c_int]
        L.rlb_batch_macroscopic.restype = C.c_int
        L.rlb_batch_totals.argtypes = [vp, dp]
        L.rlb_batch_totals.restype = C.c_int
        L.rlb_batch_plan.argtypes = [C.c_int, ip, llp, tp, C.c_int, ip, ip, ip, ip, llp]
        L.rlb_batch_plan.restype = C.c_int
        L.rlb_batch_autotune.argtypes = [vp, llp, C.c_int, tp, C.c_int, ip, tp]
        L.rlb_batch_autotune.restype = C.c_int
        L.rlb_batch_set_tuning.argtypes = [vp, tp]
        L.rlb_batch_set_tuning.restype = C.c_int
        L.rlb_batch_get_tuning.argtypes = [vp, tp, ip]
        L.rlb_batch_get_tuning.restype = C.c_int
        L.rlb_batch_set_stream.argtypes = [vp, vp]
        L.rlb_batch_set_stream.restype = C.c_int
        L.rlb_batch_total_cells.argtypes = [vp]
        L.rlb_batch_total_cells.restype = C.c_longlong
        L.rlb_batch_launch_count.argtypes = [vp]
        L.rlb_batch_launch_count.restype = C.c_longlong
        L.rlb_batch_destroy.argtypes = [vp]
        L.rlb_batch_destroy.restype = None
        L.rlb_batch_last_error.argtypes = [vp]
        L.rlb_batch_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().rlb_status_string(int(status)).decode()


def rlb_step_kernel(ctx) -> str:
    return lib().rlb_step_kernel(ctx).decode()


def last_error(ctx=None) -> str:
    return lib().rlb_last_error(ctx).decode()


def _check(status: int, ctx=None):
    if status != RLB_OK:
        raise RLBError(status, last_error(ctx))


def make_grid(nx, ny=1, nz=1, bc_lo=(BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC),
              bc_hi=(BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC), inlet=(1.0, 1.0, (0.0, 0.0, 0.0))):
    n, T, u = inlet
    return rlb_grid(int(nx), int(ny), int(nz), (C.c_int * 3)(*bc_lo), (C.c_int * 3)(*bc_hi),
                    float(n), float(T), (C.c_double * 3)(*u))


def make_options(dt_over_dx=0.25, tau_override=0.0, alpha_override=-1.0, euler_mode=0,
                 precision=FP64, cuda_stream=None, symmetry_1d=0, model=MODEL_EXTENDED,
                 thread_mapping=MAPPING_AUTO, symmetry_2d=0, recovery_fp64=0, slab_rows=0):
    return rlb_options(float(dt_over_dx), float(tau_override), float(alpha_override),
                       int(euler_mode), int(precision), cuda_stream, int(symmetry_1d), int(model),
                       int(thread_mapping), int(symmetry_2d), int(recovery_fp64), int(slab_rows))


def rlb_check_config(grid, Q, eta_over_s, zeta_over_s, limiter, opts) -> int:
    return lib().rlb_check_config(C.byref(grid), int(Q), float(eta_over_s), float(zeta_over_s),
                                  int(limiter), C.byref(opts) if opts is not None else None)


def rlb_create(grid, Q, eta_over_s, zeta_over_s, limiter, opts):
    ctx = C.c_void_p()
    st = lib().rlb_create(C.byref(grid), int(Q), float(eta_over_s), float(zeta_over_s),
                          int(limiter), C.byref(opts) if opts is not None else None, C.byref(ctx))
    _check(st)
    return ctx


def _torch():
    import torch
    return torch


def _current_stream():
    try:
        torch = _torch()
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def _as_f64(a, N):
    """(pointer, on_device, keepalive) for an N-vector of float64"""
    if hasattr(a, "is_cuda"):
        torch = _torch()
        t = a.reshape(-1).to(torch.float64).contiguous()
        if t.numel() != N:
            raise ValueError(f"field has {t.numel()} values, expected {N}")
        if t.is_cuda:
            return t.data_ptr(), 1, t
        arr = t.numpy()
    else:
        arr = np.ascontiguousarray(np.broadcast_to(np.asarray(a, np.float64), (N,)))
    return arr.ctypes.data, 0, arr


def rlb_init(ctx, n, T, ux, uy, uz, N):
    ptrs, keep = [], []
    ondev = None
    for a in (n, T, ux, uy, uz):
        p, d, k = _as_f64(a, N)
        ondev = d if ondev is None else ondev
        if d != ondev:
            raise ValueError("all fields must be on the same side (host or device)")
        ptrs.append(p)
        keep.append(k)
    _check(lib().rlb_init(ctx, *ptrs, ondev), ctx)


def rlb_step(ctx, nsteps: int):
    _check(lib().rlb_step(ctx, int(nsteps)), ctx)


def rlb_macroscopic(ctx, out, on_device: int):
    ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
    _check(lib().rlb_macroscopic(ctx, ptr, int(on_device)), ctx)


def rlb_conserved_totals(ctx) -> np.ndarray:
    out = np.zeros(5)
    _check(lib().rlb_conserved_totals(ctx, out.ctypes.data_as(C.POINTER(C.c_double))), ctx)
    return out


def rlb_conserved_totals_noalloc(f_ptr, h_ptr, N, plane_stride, precision, out_ptr, stream=None):
    """Allocation-free grid totals from caller device buffers (see rlb.h):
    f_ptr, h_ptr, out_ptr are device addresses (ints); raises on error."""
    st = lib().rlb_conserved_totals_noalloc(f_ptr, h_ptr, int(N), int(plane_stride), int(precision),
                                             out_ptr, stream)
    _check(st)


def rlb_state_bytes(ctx) -> int:
    return int(lib().rlb_state_bytes(ctx))


def _state_buffer(buf, nbytes: int) -> int:
    """address of a contiguous numpy array or torch tensor holding at least
    nbytes; raises rather than let the library overrun a short buffer"""
    if hasattr(buf, "data_ptr"):
        size, contiguous, ptr = buf.numel() * buf.element_size(), buf.is_contiguous(), buf.data_ptr()
    else:
        size, contiguous, ptr = buf.nbytes, buf.flags.c_contiguous, buf.ctypes.data
    if not contiguous:
        raise ValueError("the state buffer must be contiguous")
    if size < nbytes:
        raise ValueError(f"the state buffer holds {size} bytes; the state needs {nbytes}")
    return ptr


def rlb_get_state(ctx, buf, on_device: int):
    nbytes = rlb_state_bytes(ctx)
    _check(lib().rlb_get_state(ctx, _state_buffer(buf, nbytes), nbytes, int(on_device)), ctx)


def rlb_set_state(ctx, buf, on_device: int):
    nbytes = rlb_state_bytes(ctx)
    _check(lib().rlb_set_state(ctx, _state_buffer(buf, nbytes), nbytes, int(on_device)), ctx)


def rlb_set_stream(ctx, stream):
    _check(lib().rlb_set_stream(ctx, stream), ctx)


def rlb_launch_count(ctx) -> int:
    return int(lib().rlb_launch_count(ctx))


def rlb_destroy(ctx):
    lib().rlb_destroy(ctx)


class Grid:
    """One simulation context: a grid, its populations and parameters.

    The keyword arguments are the fields of rlb_grid and rlb_options
    (include/rlb.h): boundaries per face (bc_lo, bc_hi; the inlet state for
    RLB_BC_INLET faces), eta/s and zeta/s, the limiter, dt/dx, the tau and
    alpha overrides, Euler mode, the precision (FP64 or FP32_STORAGE), the
    lattice (model), the CUDA stream ("current": torch's current stream),
    the thread mapping of the grid kernels (MAPPING_AUTO, MAPPING_TILES,
    MAPPING_LINEAR; the results are the same) and the exact symmetry
    reductions (symmetry_1d on grids with ny = nz = 1, symmetry_2d on grids
    with nz = 1; viscous step), and for FP32_STORAGE the FP64 Landau-frame
    recovery (recovery_fp64 = 1) and the block order of the 3-D tiles
    (slab_rows; 0 automatic; the results are the same)."""

    def __init__(self, nx, ny=1, nz=1, *, bc_lo=(BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC),
                 bc_hi=(BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC), inlet=(1.0, 1.0, (0.0, 0.0, 0.0)),
                 eta_over_s=0.1, zeta_over_s=0.0, limiter=LIMITER_MINMOD, dt_over_dx=0.25,
                 tau_override=0.0, alpha_override=-1.0, euler_mode=0, precision=FP64,
                 model=MODEL_EXTENDED, stream="current", thread_mapping=0, symmetry_1d=0, symmetry_2d=0,
                 recovery_fp64=0, slab_rows=0):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.precision = int(precision)
        s = _current_stream() if stream == "current" else stream
        self._grid = make_grid(nx, ny, nz, bc_lo, bc_hi, inlet)
        self._opts = make_options(dt_over_dx, tau_override, alpha_override, euler_mode, precision, s,
                                  symmetry_1d=symmetry_1d, model=model, thread_mapping=thread_mapping,
                                  symmetry_2d=symmetry_2d, recovery_fp64=recovery_fp64,
                                  slab_rows=slab_rows)
        self.ctx = rlb_create(self._grid, Q, eta_over_s, zeta_over_s, limiter, self._opts)

    @classmethod
    def from_workload(cls, w, precision=None, **kw):
        return cls(w.nx, w.ny, w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, inlet=w.inlet,
                   eta_over_s=w.eta_over_s, zeta_over_s=w.zeta_over_s, dt_over_dx=w.dt_over_dx,
                   tau_override=w.tau_override, alpha_override=w.alpha_override,
                   euler_mode=w.euler_mode,
                   precision=w.precision if precision is None else precision, **kw)

    def init(self, n, T, ux, uy, uz):
        rlb_init(self.ctx, n, T, ux, uy, uz, self.N)
        return self

    def step(self, nsteps=1):
        rlb_step(self.ctx, nsteps)
        return self

    @property
    def step_kernel(self) -> str:
        """name of the step kernel this grid's steps launch (rlb_step_kernel)"""
        return rlb_step_kernel(self.ctx)

    def set_solid(self, mask, n, T):
        """hold the cells where mask != 0 at the equilibrium of (n, T, u = 0)
        (mask: N values, numpy or torch CUDA; None removes the solid cells)"""
        if mask is None:
            _check(lib().rlb_set_solid(self.ctx, None, 1.0, 1.0, 0), self.ctx)
            return self
        if hasattr(mask, "is_cuda") and mask.is_cuda:
            torch = _torch()
            m = (mask.reshape(-1) != 0).to(torch.uint8).contiguous()
            if m.numel() != self.N:
                raise ValueError(f"mask has {m.numel()} values, expected {self.N}")
            _check(lib().rlb_set_solid(self.ctx, m.data_ptr(), float(n), float(T), 1), self.ctx)
        else:
            m = np.ascontiguousarray(np.asarray(mask).reshape(-1) != 0, np.uint8)
            if m.size != self.N:
                raise ValueError(f"mask has {m.size} values, expected {self.N}")
            _check(lib().rlb_set_solid(self.ctx, m.ctypes.data, float(n), float(T), 0), self.ctx)
        return self

    def macroscopic(self, device=True):
        """(6, N) float64: n, e, u_x, u_y, u_z, gamma (torch CUDA tensor or numpy)"""
        if device:
            torch = _torch()
            out = torch.empty((6, self.N), dtype=torch.float64, device="cuda")
            rlb_macroscopic(self.ctx, out, 1)
            return out
        out = np.empty((6, self.N))
        rlb_macroscopic(self.ctx, out, 0)
        return out

    def totals(self):
        return rlb_conserved_totals(self.ctx)

    def state_dtype(self):
        return np.float32 if self.precision == FP32_STORAGE else np.float64

    def get_state(self):
        """host numpy copy: (f[19, N], h[19, N], prev[5, N])"""
        buf = np.empty(43 * self.N, self.state_dtype())
        rlb_get_state(self.ctx, buf, 0)
        return buf[:19 * self.N].reshape(19, self.N), buf[19 * self.N:38 * self.N].reshape(19, self.N), \
            buf[38 * self.N:].reshape(5, self.N)

    def set_state(self, f, h, prev):
        buf = np.ascontiguousarray(np.concatenate([np.ravel(f), np.ravel(h), np.ravel(prev)]),
                                   self.state_dtype())
        rlb_set_state(self.ctx, buf, 0)
        return self

    @property
    def launches(self) -> int:
        return rlb_launch_count(self.ctx)

    def close(self):
        if self.ctx:
            rlb_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Batched tubes
# ---------------------------------------------------------------------------

def batch_last_error(b=None) -> str:
    return lib().rlb_batch_last_error(b).decode()


def _bcheck(status: int, b=None):
    if status != RLB_OK:
        raise RLBError(status, batch_last_error(b))


def _i32(a):
    return np.ascontiguousarray(a, np.int32)


def _i64(a):
    return np.ascontiguousarray(a, np.int64)


def rlb_batch_plan(nx, nsteps, tuning, nclusters):
    """Host-side job plan (see rlb.h): (order, jobs[njobs, 4], cl_start, critical)."""
    nx = _i32(nx)
    B = nx.size
    st = _i64(np.broadcast_to(np.asarray(nsteps, np.int64), (B,)))   # the library reads B counts
    order = np.zeros(B, np.int32)
    jobs = np.zeros(4 * B, np.int32)
    cl = np.zeros(int(nclusters) + 1, np.int32)
    nj, crit = C.c_int(), C.c_longlong()
    ip, llp = C.POINTER(C.c_int), C.POINTER(C.c_longlong)
    _bcheck(lib().rlb_batch_plan(B, nx.ctypes.data_as(ip), st.ctypes.data_as(llp), C.byref(tuning),
                                 int(nclusters), order.ctypes.data_as(ip), jobs.ctypes.data_as(ip),
                                 C.byref(nj), cl.ctypes.data_as(ip), C.byref(crit)))
    return order, jobs[:4 * nj.value].reshape(-1, 4), cl, crit.value


class Batch:
    """B independent 1-D tubes advanced by one persistent launch (FP32 storage)."""

    def __init__(self, nx, eta_over_s, zeta_over_s, *, limiter=LIMITER_MINMOD, dt_over_dx=0.15,
                 tau_override=0.0, alpha_override=-1.0, symmetry_1d=0, stream="current"):
        self.nx = _i32(nx)
        self.B = int(self.nx.size)
        # one value per tube (a scalar applies to all); the library reads B of each
        self.eta = np.ascontiguousarray(np.broadcast_to(np.asarray(eta_over_s, np.float64), (self.B,)))
        self.zeta = np.ascontiguousarray(np.broadcast_to(np.asarray(zeta_over_s, np.float64), (self.B,)))
        s = _current_stream() if stream == "current" else stream
        self._opts = make_options(dt_over_dx, tau_override, alpha_override, 0, FP32_STORAGE, s, symmetry_1d)
        h = C.c_void_p()
        dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
        _bcheck(lib().rlb_batch_create(self.B, self.nx.ctypes.data_as(ip), self.eta.ctypes.data_as(dp),
                                       self.zeta.ctypes.data_as(dp), int(limiter), C.byref(self._opts),
                                       C.byref(h)))
        self.b = h
        self.total = int(lib().rlb_batch_total_cells(self.b))
        self.offsets = np.zeros(self.B + 1, np.int64)
        self.offsets[1:] = np.cumsum(self.nx)

    @classmethod
    def from_spec(cls, spec, **kw):
        return cls(spec.nx, spec.eta_over_s, spec.zeta_over_s, dt_over_dx=spec.dt_over_dx,
                   alpha_override=spec.alpha, **kw)

    def init(self, n, T, ux):
        ptrs, keep, ondev = [], [], None
        for a in (n, T, ux):
            p, d, k = _as_f64(a, self.total)
            ondev = d if ondev is None else ondev
            if d != ondev:
                raise ValueError("all fields must be on the same side (host or device)")
            ptrs.append(p)
            keep.append(k)
        _bcheck(lib().rlb_batch_init(self.b, *ptrs, ondev), self.b)
        return self

    def step(self, nsteps):
        st = _i64(np.broadcast_to(np.asarray(nsteps, np.int64), (self.B,)))
        _bcheck(lib().rlb_batch_step(self.b, st.ctypes.data_as(C.POINTER(C.c_longlong))), self.b)
        return self

    def macroscopic(self, device=True):
        """(6, total) float64, packed: n, e, u_x, u_y, u_z, gamma"""
        if device:
            torch = _torch()
            out = torch.empty((6, self.total), dtype=torch.float64, device="cuda")
            _bcheck(lib().rlb_batch_macroscopic(self.b, out.data_ptr(), 1), self.b)
            return out
        out = np.empty((6, self.total))
        _bcheck(lib().rlb_batch_macroscopic(self.b, out.ctypes.data, 0), self.b)
        return out

    def totals(self):
        """(B, 5): per-tube T^00, T^0x, T^0y, T^0z, N^0"""
        out = np.zeros(5 * self.B)
        _bcheck(lib().rlb_batch_totals(self.b, out.ctypes.data_as(C.POINTER(C.c_double))), self.b)
        return out.reshape(self.B, 5)

    def tuning(self):
        t, n = rlb_batch_tuning(), C.c_int()
        _bcheck(lib().rlb_batch_get_tuning(self.b, C.byref(t), C.byref(n)), self.b)
        return t, n.value

    def set_tuning(self, threads, bound, cluster, pairs_per_thread=1):
        t = rlb_batch_tuning(int(threads), int(bound), int(cluster), int(pairs_per_thread), 0.0)
        _bcheck(lib().rlb_batch_set_tuning(self.b, C.byref(t)), self.b)

    def autotune(self, nsteps, divisor=16, max_trials=64):
        st = _i64(np.broadcast_to(np.asarray(nsteps, np.int64), (self.B,)))
        trials = (rlb_batch_tuning * max_trials)()
        n, best = C.c_int(), rlb_batch_tuning()
        _bcheck(lib().rlb_batch_autotune(self.b, st.ctypes.data_as(C.POINTER(C.c_longlong)), int(divisor),
                                         trials, int(max_trials), C.byref(n), C.byref(best)), self.b)
        return best, [trials[i] for i in range(min(n.value, max_trials))]

    @property
    def launches(self) -> int:
        return int(lib().rlb_batch_launch_count(self.b))

    def close(self):
        if self.b:
            lib().rlb_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
