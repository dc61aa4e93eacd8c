"""Initialisation and macroscopic output of the FP32-storage form (float and
double-float arithmetic, two cells per thread), against the oracle cell by
cell.

* rlb_init: every stored population is the oracle's f^eq / h^eq (Eqs. 43-46)
  of the input state within 16 units of float rounding of its plane's scale
  (64 near the light cone; the oracle's equilibria carry the moments of Eq. 36 exactly); the stored
  previous level is the raw sums of the stored populations.
* rlb_macroscopic: the oracle's moments and Landau-frame recovery of the same
  stored populations, within 8 units of float rounding per field scale.
* Both lattices, odd cell counts (the last thread holds one cell), velocities
  close to the light cone, and an odd number of solid cells.
"""
import math

import numpy as np
import pytest

from paper_1302_1125_gb300 import rlb
from paper_1302_1125_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1302_1125_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def fields(nx, seed, beta_max=0.9):
    rng = np.random.default_rng(seed)
    n = rng.uniform(0.2, 3.0, nx)
    T = rng.uniform(0.1, 2.0, nx)
    d = rng.normal(size=(3, nx))
    d /= np.linalg.norm(d, axis=0)
    v = d * rng.uniform(0.0, beta_max, nx)
    return n, T, v[0].copy(), v[1].copy(), v[2].copy()


def grid(nx, model):
    per = (rlb.BC_PERIODIC,) * 3
    return rlb.Grid(nx, bc_lo=per, bc_hi=per, dt_over_dx=0.25, eta_over_s=0.1, alpha_override=0.0,
                    precision=rlb.FP32_STORAGE, model=model)


@pytest.mark.parametrize("model", [rlb.MODEL_EXTENDED, rlb.MODEL_BASIC])
@pytest.mark.parametrize("nx,beta_max,units", [(4097, 0.9, 16), (301, 0.999, 64)])
def test_init_populations_are_the_oracle_equilibria(orc, model, nx, beta_max, units):
    # near the light cone (gamma ~ 22) the terms of a population are ~gamma^2
    # times their sum, and their float roundings with them
    n, T, ux, uy, uz = fields(nx, 31 + nx, beta_max)
    g = grid(nx, model).init(n, T, ux, uy, uz)
    f, h, prev = g.get_state()
    g.close()
    _, c, _, _, xi0 = orc.lattice(model)
    gam = 1.0 / np.sqrt(1.0 - (ux * ux + uy * uy + uz * uz))
    up = gam * np.vstack([ux, uy, uz])
    fo = np.array([orc.feq(n[i] * T[i], up[:, i], model) for i in range(nx)]).T
    ho = np.array([orc.heq(n[i], up[:, i], model) for i in range(nx)]).T
    for got, ref in ((f, fo), (h, ho)):
        for k in range(19):
            scale = np.abs(ref[k]).max()
            assert np.abs(got[k] - ref[k]).max() <= units * U * scale, k
    f64, h64 = f.astype(np.float64), h.astype(np.float64)
    fa, ha = np.abs(f64), np.abs(h64)
    # previous level: raw sums of the stored populations, one float rounding
    # (the double-float accumulation adds ~2^-44 of the absolute sum)
    sums = np.vstack([f64.sum(0), c.T @ f64, h64.sum(0)])
    asum = np.vstack([fa.sum(0), np.abs(c).T @ fa, ha.sum(0)])
    assert np.all(np.abs(prev - sums) <= U * np.abs(sums) + 2.0 ** -40 * asum)


@pytest.mark.parametrize("model", [rlb.MODEL_EXTENDED, rlb.MODEL_BASIC])
def test_macroscopic_is_the_oracle_recovery_of_the_stored_state(orc, model):
    w = W.periodic_box(41, 7, 7, seed=5, gamma_max=2.0, tau_override=0.7, alpha_override=0.1,
                       precision=rlb.FP32_STORAGE)
    assert w.N % 2 == 1
    g = rlb.Grid.from_workload(w, model=model).init(*w.fields())
    g.step(25)                        # populations off equilibrium
    f, h, _ = g.get_state()
    m = g.macroscopic(device=False)
    g.close()
    ref = np.zeros((6, w.N))
    for i in range(w.N):
        mac, bad = orc.recover(orc.moments(f[:, i].astype(np.float64), h[:, i].astype(np.float64), model), model)
        assert not bad
        P, u, nn = mac[0], mac[1:4], mac[4]
        gam = math.sqrt(1.0 + u @ u)
        ref[:, i] = [nn, 3 * P, u[0] / gam, u[1] / gam, u[2] / gam, gam]
    for k in range(6):
        scale = np.abs(ref[k]).max() if k in (0, 1, 5) else 1.0
        assert np.abs(m[k] - ref[k]).max() <= 8 * U * scale, k


def test_odd_solid_cell_count_holds_the_state():
    w = W.sphere_cloud("beta02", scale=8, viscous=True)
    mask = w.solid_mask().copy()
    idx = np.flatnonzero(mask)
    if idx.size % 2 == 0:
        mask[idx[-1]] = 0
    assert mask.sum() % 2 == 1
    n1, T1 = 0.7, 0.8
    g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE).init(*w.fields())
    g.set_solid(mask, n1, T1).step(5)
    m = g.macroscopic(device=False)
    f, h, _ = g.get_state()
    g.close()
    sol = np.flatnonzero(mask)
    # every solid cell holds the same populations, those rlb_init writes for the state
    ref = rlb.Grid(3, precision=rlb.FP32_STORAGE).init(np.full(3, n1), np.full(3, T1), np.zeros(3),
                                                      np.zeros(3), np.zeros(3))
    fr, hr, _ = ref.get_state()
    ref.close()
    assert np.array_equal(f[:, sol], np.repeat(fr[:, :1], sol.size, 1))
    assert np.array_equal(h[:, sol], np.repeat(hr[:, :1], sol.size, 1))
    assert np.abs(m[0, sol] / n1 - 1).max() <= 4 * U
    assert np.abs(m[2:5, sol]).max() <= 4 * U
