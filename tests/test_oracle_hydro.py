"""Pins of the oracle's step by the hydrodynamics it must reproduce and by
statements of Sec. II.B and Sec. III, not by its own formulas:

* Linear acoustics of the e = 3P gas: a small pressure pulse splits into two
  halves that move at the speed of sound c_s = 1/sqrt(3) (c_s^2 = dP/de), and
  in each half the flow velocity is u = +-c_s de / (e + P) =
  +-(sqrt(3)/4) dP / P0 (the acoustic impedance).  Euler mode and a
  low-viscosity run.
* The number distribution h follows Eq. 57 without the lambda_i (bulk)
  term (Sec. II.B): after one viscous step h does not depend on alpha,
  while f does.
* An inlet face holding the gas's own state (Sec. III) is invisible: a
  uniform moving state next to it stays uniform.
"""
import math

import numpy as np
import pytest

CS = 1.0 / math.sqrt(3.0)
D_G = 16.0


def n_eq(T):
    return D_G * np.asarray(T) ** 3 / math.pi ** 2


@pytest.mark.parametrize("euler,eta,tol", [(1, 0.0, 0.1), (0, 0.01, 0.5)])
def test_sound_pulse(orc, euler, eta, tol):
    nx, x0, sig, amp, dt, steps = 600, 300.0, 8.0, 1e-3, 0.25, 480
    x = np.arange(nx)
    T = (1.0 + amp * np.exp(-(x - x0) ** 2 / (2 * sig ** 2))) ** 0.25   # P = n_eq(T) T: dP/P0 = amp
    z = np.zeros(nx)
    p = orc.Params(nx=nx, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, eta_over_s=eta,
                   alpha_override=0.0, euler_mode=euler)
    s = orc.init(p, n_eq(T), T, z, z, z)
    P0 = float(n_eq(1.0))
    orc.step(s, steps)
    assert s.nonphysical == 0
    m = orc.macroscopic(s)
    dP = m[1] / 3.0 - P0
    u = m[2]
    t = steps * dt
    for side, sign in ((x > x0, 1.0), (x < x0, -1.0)):
        centroid = (x[side] * dP[side]).sum() / dP[side].sum()
        assert abs(centroid - (x0 + sign * CS * t)) < tol, (centroid, x0 + sign * CS * t)
        ratio = (u[side] * dP[side]).sum() / (dP[side] ** 2).sum()
        assert ratio == pytest.approx(sign * math.sqrt(3.0) / (4.0 * P0), rel=5e-3)
    # each half carries half the pulse and the peak has split
    assert dP[x > x0].sum() == pytest.approx(dP[x < x0].sum(), rel=1e-9)
    assert dP.max() < 0.55 * amp * P0


def test_number_distribution_has_no_bulk_term(orc):
    from paper_1302_1125_gb300 import workloads as W
    w = W.periodic_box(7, 6, 5, seed=11, amp=0.3)
    out = {}
    for alpha in (0.0, 0.3):
        p = orc.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt=0.2,
                       tau_override=0.8, alpha_override=alpha)
        s = orc.init(p, *w.fields())
        orc.step(s, 1)
        out[alpha] = (s.f.copy(), s.h.copy())
    assert np.array_equal(out[0.0][1], out[0.3][1])
    df = np.abs(out[0.0][0] - out[0.3][0]).reshape(19, -1)
    assert np.all(df[0] == 0.0)             # lambda_0 = 0
    assert df[1:].max() > 1e-4 * np.abs(out[0.0][0]).max()


@pytest.mark.parametrize("dims,u", [((40, 1, 1), (0.4, 0.0, 0.0)), ((24, 6, 1), (0.35, 0.2, 0.0)),
                                    ((40, 1, 1), (-0.3, 0.0, 0.0))])
def test_inlet_at_the_gas_state_is_invisible(orc, dims, u):
    nx, ny, nz = dims
    N = nx * ny * nz
    n, T = 0.8, 1.7
    p = orc.Params(nx=nx, ny=ny, nz=nz, bc_lo=(2, 0, 0), bc_hi=(1, 0, 0), dt=0.15, eta_over_s=0.05,
                   alpha_override=0.2, inlet_n=n, inlet_T=T, inlet_u=u)
    s = orc.init(p, np.full(N, n), np.full(N, T), np.full(N, u[0]), np.full(N, u[1]), np.full(N, u[2]))
    f0, h0 = s.f.copy(), s.h.copy()
    orc.step(s, 30)
    assert np.allclose(s.f, f0, rtol=0, atol=1e-13 * np.abs(f0).max())
    assert np.allclose(s.h, h0, rtol=0, atol=1e-13 * np.abs(h0).max())
    # a different inlet state does reach the gas
    p.inlet_T = 1.0
    s = orc.init(p, np.full(N, n), np.full(N, T), np.full(N, u[0]), np.full(N, u[1]), np.full(N, u[2]))
    orc.step(s, 5)
    assert np.abs(s.f - f0).max() > 1e-3 * np.abs(f0).max()
