"""The exact 1-D symmetry reduction on grids (rlb_options.symmetry_1d with
ny = nz = 1), FP32 storage and FP64: with u_y = u_z = 0 the step keeps one
plane per class of equal populations (7 per distribution), as the batched
tubes do.

* Against the FP64 oracle: the FP32 L1 bound (1e-4) on the shock tubes of
  the benchmark's 1-D configurations and on an odd-length tube.
* Against the 19-population FP32 step: the same state up to the rounding
  order of the moment sums (L1 <= 1e-5 after thousands of steps, where the
  shocks amplify that order), the same conserved totals, and in the state
  read back every class member equals its representative.
* rlb_init rejects u_y or u_z != 0; rlb_set_state rejects unequal class
  members and resumes a symmetric state bit for bit.
* The FP64 form under the reduction meets the 1e-10 bar against the oracle.
"""
import numpy as np
import pytest

from paper_1302_1125_gb300 import rlb
from paper_1302_1125_gb300 import workloads as W

from norms import l1_fields

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
MEMBERS = [(3, 4), (3, 5), (3, 6), (7, 8), (7, 11), (7, 12), (9, 10), (9, 13), (9, 14), (15, 16), (15, 17),
           (15, 18)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1302_1125_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def l1rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def run(w, steps, sym):
    g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, symmetry_1d=sym)
    g.init(*w.fields())
    l0 = g.launches
    g.step(steps)
    assert g.launches == l0 + steps
    return g


CASES = {
    "tube_800": (lambda: W.tube_800(), 2000),
    "tube_8192a_2048": (lambda: W.tube_8192("a", nx=2048), 1500),
    "tube_8192b_1024": (lambda: W.tube_8192("b", nx=1024), 800),
    "odd_tube_203": (lambda: W.riemann_tube(203, 16.0, 2.0, eta_over_s=0.05), 400),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_reduced_tube_matches_oracle(orc, name):
    make, steps = CASES[name]
    w = make()
    g = run(w, steps, 1)
    mg = g.macroscopic(device=False)
    g.close()
    p = orc.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt=w.dt_over_dx,
                   eta_over_s=w.eta_over_s, zeta_over_s=w.zeta_over_s, tau_override=w.tau_override,
                   alpha_override=w.alpha_override)
    s = orc.init(p, *w.fields())
    orc.step(s, steps)
    assert s.nonphysical == 0
    mo = orc.macroscopic(s)
    errs = list(l1_fields(mg, mo).values())
    assert max(errs) <= 1e-4, errs
    assert np.abs(mg[3:5]).max() == 0.0


@pytest.mark.parametrize("name", sorted(CASES))
def test_reduced_tube_equals_full_step(name):
    make, steps = CASES[name]
    w = make()
    full, red = run(w, steps, 0), run(w, steps, 1)
    mf, mr = full.macroscopic(device=False), red.macroscopic(device=False)
    for k in (0, 1, 5):
        assert l1rel(mr[k], mf[k]) <= 1e-5, k
    assert np.abs(mr[2] - mf[2]).sum() / np.abs(mf[5]).sum() <= 1e-5
    tf, tr = full.totals(), red.totals()
    assert np.allclose(tr, tf, rtol=1e-6, atol=1e-6 * abs(tf[0]))
    f, h, prev = red.get_state()
    for a, b in MEMBERS:
        assert np.array_equal(f[a], f[b]) and np.array_equal(h[a], h[b]), (a, b)
    assert np.all(prev[2] == 0.0) and np.all(prev[3] == 0.0)
    full.close()
    red.close()


def test_short_run_equals_full_step_closely():
    """a few steps: the rounding-order difference has not been amplified"""
    w = W.tube_800()
    full, red = run(w, 20, 0), run(w, 20, 1)
    mf, mr = full.macroscopic(device=False), red.macroscopic(device=False)
    for k in (0, 1, 5):
        assert np.abs(mr[k] - mf[k]).max() <= 1e-6 * np.abs(mf[k]).max(), k
    full.close()
    red.close()


def test_init_rejects_transverse_motion():
    w = W.tube_800()
    n, T, ux, uy, uz = w.fields()
    for bad in ("uy", "uz"):
        v = np.zeros_like(ux)
        v[17] = 1e-3
        args = (n, T, ux, v, uz) if bad == "uy" else (n, T, ux, uy, v)
        g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, symmetry_1d=1)
        with pytest.raises(rlb.RLBError) as e:
            g.init(*args)
        assert e.value.status == rlb.RLB_E_INVALID
        assert "mirror image" in rlb.last_error(g.ctx)
        g.init(*w.fields()).step(2)          # the context stays usable
        g.close()


def test_set_state_checks_the_classes():
    w = W.tube_800()
    g = run(w, 5, 1)
    f, h, prev = (a.copy() for a in g.get_state())
    g.step(5)
    ref = g.get_state()
    g2 = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, symmetry_1d=1)
    bad = h.copy()
    bad[17, 400] *= 1.0001
    with pytest.raises(rlb.RLBError) as e:
        g2.set_state(f, bad, prev)
    assert e.value.status == rlb.RLB_E_INVALID
    g2.set_state(f, h, prev).step(5)
    for a, b in zip(g2.get_state(), ref):
        assert np.array_equal(a, b)
    g.close()
    g2.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_reduced_tube_matches_oracle(orc, name):
    """the FP64 form under the reduction: the 1e-10 bar against the oracle"""
    make, steps = CASES[name]
    w = make()
    g = rlb.Grid.from_workload(w, precision=rlb.FP64, symmetry_1d=1)
    g.init(*w.fields()).step(steps)
    mg = g.macroscopic(device=False)
    f, h, prev = g.get_state()
    g.close()
    p = orc.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt=w.dt_over_dx,
                   eta_over_s=w.eta_over_s, zeta_over_s=w.zeta_over_s, tau_override=w.tau_override,
                   alpha_override=w.alpha_override)
    s = orc.init(p, *w.fields())
    orc.step(s, steps)
    mo = orc.macroscopic(s)
    for k in (0, 1, 5):
        assert np.abs(mg[k] - mo[k]).max() <= 1e-10 * np.abs(mo[k]).max(), k
    assert np.abs(mg[2] - mo[2]).max() <= 1e-10 * np.abs(mo[2]).max()
    assert np.abs(mg[3:5]).max() == 0.0
    for a, b in MEMBERS:
        assert np.array_equal(f[a], f[b]) and np.array_equal(h[a], h[b]), (a, b)
    assert np.all(prev[2] == 0.0) and np.all(prev[3] == 0.0)


def test_fp64_set_state_checks_the_classes():
    w = W.tube_800()
    g = rlb.Grid.from_workload(w, precision=rlb.FP64, symmetry_1d=1).init(*w.fields()).step(5)
    f, h, prev = (a.copy() for a in g.get_state())
    bad = f.copy()
    bad[11, 100] *= 1.0 + 1e-12
    with pytest.raises(rlb.RLBError) as e:
        g.set_state(bad, h, prev)
    assert e.value.status == rlb.RLB_E_INVALID
    g.set_state(f, h, prev).step(2)
    g.close()
