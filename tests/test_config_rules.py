"""rlb_check_config against the rules include/rlb.h states, on random
configurations (CPU, no device):

* RLB_E_INVALID for a bad argument: Q != 19, a dimension < 1, N >= 2^31, an
  unknown boundary, limiter, precision or mode, an inlet on a y or z face or
  with n <= 0, T <= 0, |u| >= 1; eta/s or zeta/s negative or not finite;
  dt/dx not positive and finite; non-finite overrides; a symmetry reduction
  on a grid or inlet it does not fit, with Euler mode, or both at once;
  recovery_fp64 other than 0 or 1, or 1 without FP32 storage, with Euler
  mode, the basic lattice, a symmetry reduction, the linear mapping or odd
  nx;
* else RLB_E_UNSTABLE when dt/dx times the largest sum over moving axes of
  |c_ia| c0/c_t exceeds 1, or 2 d (c0 nu/c_t) dt alpha exceeds 1, with d the
  number of axes with more than one cell (at least 1) and alpha the override
  or 27 (zeta/s)/nu^6 (Eq. 56 at the reference state);
* else RLB_OK.

The model below restates those rules; a status the library gives that the
model does not predict is a mismatch between the header and the code.
"""
import math

import pytest

from paper_1302_1125_gb300 import rlb

hyp = pytest.importorskip("hypothesis")
st = hyp.strategies

LATTICE = {0: (math.sqrt(13.0), 2), 1: (math.sqrt(19.0), 1)}   # nu, |c_ia| of a diagonal


def expected(nx, ny, nz, lo, hi, inlet_n, inlet_T, inlet_u, eta, zeta, limiter, o, Q=19):
    invalid = False
    invalid |= Q != 19
    invalid |= min(nx, ny, nz) < 1
    invalid |= nx * ny * nz > 2 ** 31 - 1
    bcs = list(lo) + list(hi)
    invalid |= any(b not in (0, 1, 2) for b in bcs)
    invalid |= any(b == 2 for a, b in enumerate(lo) if a != 0) or any(b == 2 for a, b in enumerate(hi) if a != 0)
    has_inlet = 2 in (lo[0], hi[0])
    if has_inlet:
        u2 = sum(v * v for v in inlet_u)
        invalid |= not (inlet_n > 0 and inlet_T > 0 and u2 < 1 and math.isfinite(inlet_n * inlet_T))
    invalid |= not (eta >= 0 and math.isfinite(eta)) or not (zeta >= 0 and math.isfinite(zeta))
    invalid |= limiter not in (0, 1)
    invalid |= not (o["dt"] > 0 and math.isfinite(o["dt"]))
    invalid |= o["precision"] not in (0, 1) or o["euler"] not in (0, 1) or o["model"] not in (0, 1)
    invalid |= o["precision"] == 1 and nx * ny * nz >= 2 ** 30
    invalid |= o["sym1"] not in (0, 1) or o["sym2"] not in (0, 1) or o["mapping"] not in (0, 1, 2, 3)
    if o["sym1"] == 1:
        invalid |= o["euler"] != 0 or ny != 1 or nz != 1 or (has_inlet and (inlet_u[1] != 0 or inlet_u[2] != 0))
    if o["sym2"] == 1:
        invalid |= o["euler"] != 0 or nz != 1 or ny < 2 or (has_inlet and inlet_u[2] != 0)
    invalid |= o["sym1"] == 1 and o["sym2"] == 1
    invalid |= o["rec64"] not in (0, 1)
    if o["rec64"] == 1:
        invalid |= (o["precision"] != 1 or o["euler"] != 0 or o["model"] != 0 or o["sym1"] != 0
                    or o["sym2"] != 0 or o["mapping"] == 2 or nx % 2 != 0)
    invalid |= not (math.isfinite(o["tau"]) and math.isfinite(o["alpha"]))
    if invalid:
        return rlb.RLB_E_INVALID
    nu, dmag = LATTICE[o["model"]]
    c0ct = nu / math.sqrt(27.0)
    d = max((nx > 1) + (ny > 1) + (nz > 1), 1)
    if o["dt"] * (2 if d >= 2 else 1) * dmag * c0ct > 1.0:
        return rlb.RLB_E_UNSTABLE
    alpha = o["alpha"] if o["alpha"] >= 0 else 27.0 * zeta / nu ** 6
    if 2 * d * c0ct * nu * o["dt"] * alpha > 1.0:
        return rlb.RLB_E_UNSTABLE
    return rlb.RLB_OK


dims = st.sampled_from([0, 1, 2, 3, 64])
bc = st.sampled_from([0, 1, 2, 3])
real = st.sampled_from([-0.1, 0.0, 0.05, 0.1, 0.5, 3.0, math.inf, math.nan])
vel = st.sampled_from([0.0, 0.3, -0.6, 0.9, 1.0])


@hyp.settings(max_examples=3000, deadline=None, derandomize=True)
@hyp.given(nx=dims, ny=dims, nz=dims, lo=st.tuples(bc, bc, bc), hi=st.tuples(bc, bc, bc),
           inlet_n=real, inlet_T=real, inlet_u=st.tuples(vel, vel, vel), eta=real, zeta=real,
           limiter=st.sampled_from([0, 1, 2]),
           dt=st.sampled_from([0.0, 0.05, 0.15, 0.25, 0.3, 0.4, 0.6, math.nan]),
           precision=st.sampled_from([0, 1, 2]), euler=st.sampled_from([0, 1, 2]),
           sym1=st.sampled_from([0, 1, 2]), sym2=st.sampled_from([0, 1, 2]),
           model=st.sampled_from([0, 1, 2]), mapping=st.sampled_from([-1, 0, 1, 2, 3, 4]),
           tau=st.sampled_from([0.0, 0.8, math.inf]),
           alpha=st.sampled_from([-1.0, 0.0, 0.05, 0.2, 0.5, math.nan]),
           rec64=st.sampled_from([0, 0, 1, 1, 2]))
def test_check_config_follows_the_documented_rules(nx, ny, nz, lo, hi, inlet_n, inlet_T, inlet_u, eta,
                                                   zeta, limiter, dt, precision, euler, sym1, sym2,
                                                   model, mapping, tau, alpha, rec64):
    o = dict(dt=dt, precision=precision, euler=euler, sym1=sym1, sym2=sym2, model=model,
             mapping=mapping, tau=tau, alpha=alpha, rec64=rec64)
    g = rlb.make_grid(nx, ny, nz, lo, hi, (inlet_n, inlet_T, inlet_u))
    opts = rlb.make_options(dt, tau, alpha, euler, precision, None, symmetry_1d=sym1, model=model,
                            thread_mapping=mapping, symmetry_2d=sym2, recovery_fp64=rec64)
    got = rlb.rlb_check_config(g, 19, eta, zeta, limiter, opts)
    assert got == expected(nx, ny, nz, lo, hi, inlet_n, inlet_T, inlet_u, eta, zeta, limiter, o)


@pytest.mark.parametrize("Q", [0, 18, 20, 27])
def test_check_config_wants_19_populations(Q):
    g = rlb.make_grid(8, 1, 1, (1, 0, 0), (1, 0, 0), (1.0, 1.0, (0.0, 0.0, 0.0)))
    assert rlb.rlb_check_config(g, Q, 0.1, 0.0, 0, rlb.make_options()) == rlb.RLB_E_INVALID
    assert rlb.rlb_check_config(g, 19, 0.1, 0.0, 0, rlb.make_options()) == rlb.RLB_OK


def test_check_config_counts_cells_in_64_bits():
    big = 1 << 11        # 2^33 cells
    g = rlb.make_grid(big, big, big, (0, 0, 0), (0, 0, 0), (1.0, 1.0, (0.0, 0.0, 0.0)))
    assert rlb.rlb_check_config(g, 19, 0.1, 0.0, 0, rlb.make_options()) == rlb.RLB_E_INVALID
    g = rlb.make_grid(1291, 1291, 1291, (0, 0, 0), (0, 0, 0), (1.0, 1.0, (0.0, 0.0, 0.0)))   # 2^31 + 4.2e6
    assert rlb.rlb_check_config(g, 19, 0.1, 0.0, 0, rlb.make_options()) == rlb.RLB_E_INVALID
    g = rlb.make_grid(1290, 1290, 1290, (0, 0, 0), (0, 0, 0), (1.0, 1.0, (0.0, 0.0, 0.0)))   # 2^31 - 7.9e5
    assert rlb.rlb_check_config(g, 19, 0.1, 0.0, 0, rlb.make_options()) == rlb.RLB_OK
    g = rlb.make_grid(1024, 1024, 1024, (0, 0, 0), (0, 0, 0), (1.0, 1.0, (0.0, 0.0, 0.0)))   # 2^30
    assert rlb.rlb_check_config(g, 19, 0.1, 0.0, 0, rlb.make_options(dt_over_dx=0.15)) == rlb.RLB_OK


def batch_expected(nx, eta, zeta, limiter, o):
    """the statuses rlb_batch_create may return under the header's rules
    (their order is not specified, so both when both kinds apply); a valid
    batch reaches the device and, without one, fails with RLB_E_CUDA"""
    B = len(nx)
    invalid = not (1 <= B <= 65535)
    invalid |= o["precision"] != 1 or o["euler"] != 0 or o["sym1"] not in (0, 1) or o["model"] != 0
    invalid |= o.get("rec64", 0) != 0
    invalid |= limiter not in (0, 1)
    invalid |= not (o["dt"] > 0 and math.isfinite(o["dt"]))
    invalid |= not (math.isfinite(o["tau"]) and math.isfinite(o["alpha"]))
    invalid |= any(n < 1 for n in nx)
    invalid |= any(not (v >= 0 and math.isfinite(v)) for v in list(eta) + list(zeta))
    invalid |= sum(-(-max(n, 0) // 32) * 32 for n in nx) > 2 ** 30
    nu = math.sqrt(13.0)
    c0ct = nu / math.sqrt(27.0)
    unstable = False
    if math.isfinite(o["dt"]) and o["dt"] > 0:
        unstable |= 2 * c0ct * o["dt"] > 1.0
        for z in zeta:
            alpha = o["alpha"] if o["alpha"] >= 0 else 27.0 * z / nu ** 6
            unstable |= 2 * c0ct * nu * o["dt"] * alpha > 1.0
    got = set()
    if invalid:
        got.add(rlb.RLB_E_INVALID)
    if unstable:
        got.add(rlb.RLB_E_UNSTABLE)
    return got or {rlb.RLB_E_CUDA}


@hyp.settings(max_examples=2000, deadline=None, derandomize=True)
@hyp.given(nx=st.lists(st.sampled_from([0, 1, 33, 800, 8192]), min_size=0, max_size=4),
           eta=st.sampled_from([-0.1, 0.0, 0.1, math.inf, math.nan]),
           zeta=st.sampled_from([0.0, 0.05, 1e4, 1e6, -1.0, math.nan]),
           limiter=st.sampled_from([0, 1, 2]),
           dt=st.sampled_from([0.0, 0.15, 0.25, 0.5, 0.8, math.nan]),
           precision=st.sampled_from([0, 1]), euler=st.sampled_from([0, 1]),
           sym1=st.sampled_from([0, 1, 2]), model=st.sampled_from([0, 1]),
           tau=st.sampled_from([0.0, 0.8, math.inf]),
           alpha=st.sampled_from([-1.0, 0.0, 0.2, 2.0, math.nan]))
def test_batch_create_follows_the_documented_rules(nx, eta, zeta, limiter, dt, precision, euler, sym1,
                                                   model, tau, alpha):
    import ctypes as C
    import numpy as np
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a valid batch would allocate on the device")
    o = dict(dt=dt, precision=precision, euler=euler, sym1=sym1, model=model, tau=tau, alpha=alpha)
    B = len(nx)
    n_arr = np.asarray(nx if B else [1], np.int32)
    e_arr = np.full(max(B, 1), eta, np.float64)
    z_arr = np.full(max(B, 1), zeta, np.float64)
    opts = rlb.make_options(dt, tau, alpha, euler, precision, None, symmetry_1d=sym1, model=model)
    h = C.c_void_p()
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
    got = rlb.lib().rlb_batch_create(B, n_arr.ctypes.data_as(ip), e_arr.ctypes.data_as(dp),
                                     z_arr.ctypes.data_as(dp), limiter, C.byref(opts), C.byref(h))
    assert h.value is None
    assert got in batch_expected(nx, [eta] * B, [zeta] * B, limiter, o)


@pytest.mark.parametrize("B,n,expect", [(65536, 1, rlb.RLB_E_INVALID), (2, 1 << 29, rlb.RLB_E_CUDA),
                                        (3, 1 << 29, rlb.RLB_E_INVALID), (2, (1 << 29) + 1, rlb.RLB_E_INVALID)])
def test_batch_create_size_limits(B, n, expect):
    """B <= 65535; at most 2^30 stored cells, each tube rounded up to 32 cells"""
    import ctypes as C
    import numpy as np
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a valid batch would allocate on the device")
    nx = np.full(B, n, np.int32)
    eta = np.full(B, 0.1)
    zeta = np.zeros(B)
    opts = rlb.make_options(dt_over_dx=0.15, precision=rlb.FP32_STORAGE)
    h = C.c_void_p()
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
    got = rlb.lib().rlb_batch_create(B, nx.ctypes.data_as(ip), eta.ctypes.data_as(dp), zeta.ctypes.data_as(dp),
                                     0, C.byref(opts), C.byref(h))
    assert got == expect and h.value is None
