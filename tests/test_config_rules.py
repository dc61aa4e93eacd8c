"""rlb_check_config against the rules include/rlb.h states, on random
configurations (CPU, no device):

* RLB_E_INVALID for a bad argument: Q != 19, a dimension < 1, N >= 2^31, an
  unknown boundary, limiter, precision or mode, an inlet on a y or z face or
  with n <= 0, T <= 0, |u| >= 1; eta/s or zeta/s negative or not finite;
  dt/dx not positive and finite; non-finite overrides; a symmetry reduction
  on a grid or inlet it does not fit, with Euler mode, or both at once;
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
    invalid |= o["sym1"] not in (0, 1) or o["sym2"] not in (0, 1) or o["mapping"] not in (0, 1, 2)
    if o["sym1"] == 1:
        invalid |= o["euler"] != 0 or ny != 1 or nz != 1 or (has_inlet and (inlet_u[1] != 0 or inlet_u[2] != 0))
    if o["sym2"] == 1:
        invalid |= o["euler"] != 0 or nz != 1 or ny < 2 or (has_inlet and inlet_u[2] != 0)
    invalid |= o["sym1"] == 1 and o["sym2"] == 1
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
           model=st.sampled_from([0, 1, 2]), mapping=st.sampled_from([-1, 0, 1, 2, 3]),
           tau=st.sampled_from([0.0, 0.8, math.inf]),
           alpha=st.sampled_from([-1.0, 0.0, 0.05, 0.2, 0.5, math.nan]))
def test_check_config_follows_the_documented_rules(nx, ny, nz, lo, hi, inlet_n, inlet_T, inlet_u, eta,
                                                   zeta, limiter, dt, precision, euler, sym1, sym2,
                                                   model, mapping, tau, alpha):
    o = dict(dt=dt, precision=precision, euler=euler, sym1=sym1, sym2=sym2, model=model,
             mapping=mapping, tau=tau, alpha=alpha)
    g = rlb.make_grid(nx, ny, nz, lo, hi, (inlet_n, inlet_T, inlet_u))
    opts = rlb.make_options(dt, tau, alpha, euler, precision, None, symmetry_1d=sym1, model=model,
                            thread_mapping=mapping, symmetry_2d=sym2)
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
