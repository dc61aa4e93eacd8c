"""Solid cells on the GPU (rlb_set_solid; Sec. III, the astrophysical run's
cloud held at the equilibrium of (n1, T1, u = 0)).

* FP64 form against the oracle within 1e-10 relative (max norm) on the
  paper's sphere-cloud run shrunk 4x per axis, and on a cloud whose state
  differs from the gas around it.
* FP32-storage form: L1 relative error against the oracle <= 1e-4.
* The solid cells read back exactly their state; a reset launch follows
  every step; removing the solid cells restores the plain step.
* The full 200 x 100 x 100 run, 1000 steps, in both forms: FP32 against FP64
  within the L1 bound, solid cells in their state.
"""
import numpy as np
import pytest

from paper_1302_1125_gb300 import rlb
from paper_1302_1125_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1302_1125_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def oparams(orc, w):
    return orc.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt=w.dt_over_dx,
                      eta_over_s=w.eta_over_s, zeta_over_s=w.zeta_over_s, tau_override=w.tau_override,
                      alpha_override=w.alpha_override, inlet_n=w.inlet[0], inlet_T=w.inlet[1],
                      inlet_u=tuple(w.inlet[2]), euler_mode=w.euler_mode)


def run_gpu(w, steps, precision, solid=None):
    g = rlb.Grid.from_workload(w, precision=precision)
    g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
    mask, n1, T1 = solid if solid is not None else (w.solid_mask(), w.solid[1], w.solid[2])
    g.set_solid(mask, n1, T1)
    l0 = g.launches
    g.step(steps)
    assert g.launches == l0 + 2 * steps       # step kernel + solid reset per step
    return g, g.macroscopic(device=False)


def run_oracle(orc, w, steps, solid=None):
    s = orc.init(oparams(orc, w), *w.fields())
    mask, n1, T1 = solid if solid is not None else (w.solid_mask(), w.solid[1], w.solid[2])
    orc.set_solid(s, mask, n1, T1)
    orc.step(s, steps)
    assert s.nonphysical == 0
    return orc.macroscopic(s)


def relinf(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def l1rel(a, b):
    return float(np.sum(np.abs(a - b)) / max(np.sum(np.abs(b)), 1e-300))


def odd_cloud(w):
    """a cloud state unlike the gas around it"""
    return w.solid_mask(), 0.7 * float(W.n_eq(0.8)), 0.8


@pytest.mark.parametrize("which", ["paper", "odd_state"])
def test_fp64_sphere_cloud_matches_oracle(orc, which):
    w = W.sphere_cloud("beta02", scale=4, viscous=True, precision=rlb.FP64)
    solid = odd_cloud(w) if which == "odd_state" else None
    steps = 250 if which == "paper" else 120
    g, mg = run_gpu(w, steps, rlb.FP64, solid)
    mo = run_oracle(orc, w, steps, solid)
    for k in (0, 1, 2, 3, 4, 5):
        assert relinf(mg[k], mo[k]) <= 1e-10, (k, relinf(mg[k], mo[k]))
    g.close()


def test_fp32_sphere_cloud_l1(orc):
    w = W.sphere_cloud("beta02", scale=4, viscous=True)
    g, mg = run_gpu(w, 250, rlb.FP32_STORAGE)
    mo = run_oracle(orc, w, 250)
    errs = [l1rel(mg[k], mo[k]) for k in (0, 1, 2)]
    assert max(errs) <= 1e-4, errs
    g.close()


@pytest.mark.parametrize("precision,tol", [(rlb.FP64, 1e-13), (rlb.FP32_STORAGE, 2e-6)])
def test_solid_cells_hold_their_state(precision, tol):
    w = W.sphere_cloud("beta02", scale=4, viscous=True)
    mask, n1, T1 = odd_cloud(w)
    g, m = run_gpu(w, 60, precision, (mask, n1, T1))
    sol = mask.nonzero()[0]
    assert sol.size > 0
    assert relinf(m[0, sol], np.full(sol.size, n1)) <= tol
    assert relinf(m[1, sol], np.full(sol.size, 3 * n1 * T1)) <= tol
    assert np.max(np.abs(m[2:5, sol])) <= tol
    # a device mask gives the same cells; None removes them
    g2 = rlb.Grid.from_workload(w, precision=precision)
    g2.init(*w.fields())
    g2.set_solid(torch.as_tensor(mask, device="cuda"), n1, T1)
    g2.step(60)
    assert np.array_equal(g2.macroscopic(device=False), m)
    g2.set_solid(None, 1.0, 1.0)
    l0 = g2.launches
    g2.step(2)
    assert g2.launches == l0 + 2
    g.close()
    g2.close()


def test_bad_solid_state_is_rejected():
    w = W.sphere_cloud("beta02", scale=8, viscous=True)
    g = rlb.Grid.from_workload(w).init(*w.fields())
    with pytest.raises(rlb.RLBError) as e:
        g.set_solid(w.solid_mask(), -1.0, 1.0)
    assert e.value.status == rlb.RLB_E_INVALID
    g.step(1)
    g.close()


def test_full_size_sphere_cloud_fp32_vs_fp64():
    """the paper's 200 x 100 x 100 run (beta ~ 0.2, viscous, tau = 1), 1000 steps"""
    w = W.sphere_cloud("beta02", viscous=True)
    _, m32 = run_gpu(w, w.steps, rlb.FP32_STORAGE)
    _, m64 = run_gpu(w, w.steps, rlb.FP64)
    errs = [l1rel(m32[k], m64[k]) for k in (0, 1)]
    errs.append(float(np.sum(np.abs(m32[2] - m64[2])) / np.sum(np.abs(m64[5]))))
    assert max(errs) <= 1e-4, errs
    sol = w.solid_mask().nonzero()[0]
    assert relinf(m64[0, sol], np.full(sol.size, w.solid[1])) <= 1e-13
    # the shock has reached and passed the cloud: velocity around it is not zero
    assert 0.15 < np.max(m64[2]) < 0.3
