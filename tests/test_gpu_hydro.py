"""The CUDA step, through the C ABI, against hydrodynamics and against
statements of Sec. II.B and Sec. III, in both precisions (the oracle's
pins of the same properties are in test_oracle_hydro.py):

* linear acoustics of the e = 3P gas: a small pressure pulse splits into
  halves moving at c_s = 1/sqrt(3) with u = +-(sqrt(3)/4) dP / P0;
* the number distribution h has no bulk (lambda_i) term: after one viscous
  step h is bit for bit the same for any alpha, while f is not (and its rest
  population is, lambda_0 = 0);
* an inlet holding the gas's own moving state is invisible.
"""
import math

import numpy as np
import pytest

from paper_1302_1125_gb300 import rlb
from paper_1302_1125_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
CS = 1.0 / math.sqrt(3.0)
PRECISIONS = [rlb.FP64, rlb.FP32_STORAGE]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1302_1125_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("euler,eta,tol", [(1, 0.0, 0.15), (0, 0.01, 0.5)])
def test_sound_pulse(precision, euler, eta, tol):
    nx, x0, sig, amp, dt, steps = 600, 300.0, 8.0, 1e-3, 0.25, 480
    x = np.arange(nx)
    T = (1.0 + amp * np.exp(-(x - x0) ** 2 / (2 * sig ** 2))) ** 0.25
    z = np.zeros(nx)
    g = rlb.Grid(nx, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), eta_over_s=eta, dt_over_dx=dt,
                 alpha_override=0.0, euler_mode=euler, precision=precision)
    g.init(W.n_eq(T), T, z, z, z).step(steps)
    m = g.macroscopic(device=False)
    g.close()
    P = m[1] / 3.0
    far = (x < 100) | (x >= 500)                 # not reached by the pulses
    P0 = float(np.median(P[far]))
    assert P0 == pytest.approx(float(W.n_eq(1.0)), rel=1e-6)
    dP = P - P0
    u = m[2]
    t = steps * dt
    for side, sign in ((x > x0, 1.0), (x < x0, -1.0)):
        centroid = (x[side] * dP[side]).sum() / dP[side].sum()
        assert abs(centroid - (x0 + sign * CS * t)) < tol, (centroid, x0 + sign * CS * t)
        ratio = (u[side] * dP[side]).sum() / (dP[side] ** 2).sum()
        assert ratio == pytest.approx(sign * math.sqrt(3.0) / (4.0 * P0), rel=1e-2)
    assert dP.max() < 0.55 * amp * P0


@pytest.mark.parametrize("precision", PRECISIONS)
def test_number_distribution_has_no_bulk_term(precision):
    w = W.periodic_box(16, 12, 10, seed=11, amp=0.3)
    out = {}
    for alpha in (0.0, 0.3):
        g = rlb.Grid(w.nx, w.ny, w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt_over_dx=0.2,
                     tau_override=0.8, alpha_override=alpha, precision=precision)
        g.init(*w.fields()).step(1)
        f, h, _ = g.get_state()
        out[alpha] = (np.array(f, copy=True), np.array(h, copy=True))
        g.close()
    assert np.array_equal(out[0.0][1], out[0.3][1])
    df = np.abs(out[0.0][0].astype(np.float64) - out[0.3][0].astype(np.float64))
    assert np.all(df[0] == 0.0)
    assert df[1:].max() > 1e-4 * np.abs(out[0.0][0]).max()


@pytest.mark.parametrize("precision,tol", [(rlb.FP64, 1e-13), (rlb.FP32_STORAGE, 1e-5)])
@pytest.mark.parametrize("dims,u", [((40, 1, 1), (0.4, 0.0, 0.0)), ((24, 6, 1), (0.35, 0.2, 0.0)),
                                    ((40, 1, 1), (-0.3, 0.0, 0.0))])
def test_inlet_at_the_gas_state_is_invisible(precision, tol, dims, u):
    nx, ny, nz = dims
    N = nx * ny * nz
    n, T = 0.8, 1.7
    fields = (np.full(N, n), np.full(N, T), np.full(N, u[0]), np.full(N, u[1]), np.full(N, u[2]))
    g = rlb.Grid(nx, ny, nz, bc_lo=(2, 0, 0), bc_hi=(1, 0, 0), inlet=(n, T, u), eta_over_s=0.05,
                 dt_over_dx=0.15, alpha_override=0.2, precision=precision)
    g.init(*fields)
    m0 = g.macroscopic(device=False)
    g.step(30)
    m = g.macroscopic(device=False)
    g.close()
    for k in (0, 1, 2, 3, 5):
        assert np.abs(m[k] - m0[k]).max() <= tol * max(np.abs(m0[k]).max(), 1.0), k
