"""Why the FP32-storage form's Landau-frame recovery need not run in FP64
(CPU, oracle and numpy only).

The recovery (Sec. II, eps = 3P) meets the 1 - beta^2 cancellation in one
place: E^2 - |M|^2 = P^2 (8 gamma^2 + 1) is the difference of two numbers of
size 16 P^2 gamma^4.  Once that difference is known accurately, the rest is
well conditioned: P = (E^2 - |M|^2) / (E + sqrt(E^2 + 3 (E^2 - |M|^2))),
gamma^2 = (E + P) / (4 P), u' = M / (4 P gamma), n = N^0 / gamma, each a
product, quotient or square root of positive numbers.

What limits the accuracy is the storage.  Rounding the 19 equilibrium
populations of a state moving at gamma to float32 moves E - |M| by about
2^-24 times the populations' size, which is ~gamma^2 times larger than
E - |M|; the recovered P then moves by up to ~gamma^2 x 2.6e-7.  These tests
show, on the equilibria of states moving at gamma = 5, 10 and 20:

* the FP64 recovery (the oracle's) of the float32-rounded populations has
  that error, growing like gamma^2; at gamma = 20 it reaches ~1e-4 in the
  worst of 60 random directions (~1e-5 to 2e-5 along x or a diagonal);
* the arithmetic of the float kernel's recovery (E^2 - |M|^2 from the exact
  sums in double-float, i.e. correct to about 2^-48, rounded once to float,
  then float divisions and square roots), emulated here in numpy float32,
  has the same error as the FP64 recovery to within a few float roundings:
  FP64 arithmetic would buy nothing the stored populations can carry;
* a single-float E^2 - |M|^2 would not stay on that floor: its own error is
  of the floor's size and adds to it.
"""
import math

import numpy as np
import pytest

f32 = np.float32


def states(gamma, k, seed):
    rng = np.random.default_rng(seed)
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    out = []
    for j in range(k):
        d = rng.normal(size=3)
        if j == 0:
            d = np.array([1.0, 0.0, 0.0])
        d /= np.linalg.norm(d)
        out.append((float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.5, 2.0)), gamma * beta * d))
    return out


def float_recovery(orc, mom):
    """the float kernel's recovery, emulated: mom = (E, M_x, M_y, M_z, N^0)
    of float populations (exact sums in double); E^2 - |M|^2 correct to
    double, rounded once; everything after it in float32"""
    xi0 = orc.lattice()[4]
    S = mom[0] / xi0 ** 2
    V = mom[1:4] / xi0
    D = f32(xi0 ** 2 * (xi0 ** 2 * S * S - V @ V))
    E = f32(xi0 ** 2) * f32(S)
    root2 = f32(float(E) * float(E) + 3.0 * float(D))    # one fused rounding
    den = f32(E + np.sqrt(root2, dtype=f32))
    P = f32(D / den)
    fourP = f32(4.0) * P
    g = np.sqrt(f32((E + P) / fourP), dtype=f32)
    s = f32(f32(xi0) / f32(fourP * g))
    u = (V.astype(f32) * s).astype(f32)
    n = f32(f32(f32(xi0) * f32(mom[4] / xi0)) / g)
    return np.array([P, u[0], u[1], u[2], n], np.float64)


@pytest.mark.parametrize("gamma", [5.0, 10.0, 20.0])
def test_float_recovery_matches_fp64_recovery_on_stored_populations(orc, gamma):
    worst64 = np.zeros(5)
    worst32 = np.zeros(5)
    diff = 0.0
    for P, n, up in states(gamma, 60, seed=int(gamma)):
        f = orc.feq(P, up)
        h = orc.heq(n, up)
        fs = f.astype(f32).astype(np.float64)      # what FP32 storage holds
        hs = h.astype(f32).astype(np.float64)
        exact = np.r_[P, up, n]
        mom = orc.moments(fs, hs)
        m64, bad = orc.recover(mom)
        assert not bad
        m32 = float_recovery(orc, mom)
        scale = np.r_[P, np.full(3, np.linalg.norm(up)), n]
        worst64 = np.maximum(worst64, np.abs(m64 - exact) / scale)
        worst32 = np.maximum(worst32, np.abs(m32 - exact) / scale)
        diff = max(diff, float(np.max(np.abs(m32 - m64) / scale)))
    # the storage floor: below gamma^2 x 3e-7 and below 1e-4 in every field
    assert worst64.max() <= 3e-7 * gamma ** 2
    assert worst64.max() <= 1.2e-4
    # at gamma >= 5 the floor is well above float rounding, and the float
    # recovery adds only a few roundings to it
    assert worst64[0] >= 30 * 2.0 ** -24
    assert diff <= 8 * 2.0 ** -24, diff
    assert np.all(worst32 <= worst64 + 8 * 2.0 ** -24)


@pytest.mark.parametrize("gamma", [5.0, 10.0, 20.0])
def test_single_float_difference_adds_to_the_floor(orc, gamma):
    """E^2 - |M|^2 rounded from float E and |M| (no double-float) has an
    error of the same order as the storage floor (2 gamma^2 roundings), so
    it would add to the floor instead of staying on it: the recovered P's
    worst error grows by more than 30 %.  The double-float difference is
    what keeps the float recovery on the floor."""
    single, dfloat = 0.0, 0.0
    for P, n, up in states(gamma, 200, seed=100 + int(gamma)):
        fs = orc.feq(P, up).astype(f32).astype(np.float64)
        hs = orc.heq(n, up).astype(f32).astype(np.float64)
        mom = orc.moments(fs, hs)
        E, M = f32(mom[0]), mom[1:4].astype(f32)
        D = f32(E * E - f32(M @ M))
        Ps = f32(D / f32(E + np.sqrt(f32(E * E + f32(3.0) * D), dtype=f32)))
        single = max(single, abs(float(Ps) - P) / P)
        dfloat = max(dfloat, abs(float_recovery(orc, mom)[0] - P) / P)
    assert single >= 1.3 * dfloat, (single, dfloat)
