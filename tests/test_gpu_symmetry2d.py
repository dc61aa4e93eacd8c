"""The exact 2-D symmetry reduction of the grid step (rlb_options.symmetry_2d),
FP32 storage and FP64: on a grid with nz = 1 and u_z = 0 the state is its
own mirror image in z, so the step keeps one plane per class of mirror-image
populations (14 per distribution).

* Against the FP64 oracle: the FP32 L1 bound (1e-4) on the 2-D shock-cloud
  (inlet, outflow, periodic y) and on periodic boxes.
* Against the 19-population FP32 step: the same state up to the rounding order
  of the moment sums (L1 <= 1e-6), the same conserved totals, and in the
  state read back every mirror image equals its class representative.
* Odd nx (no aligned pairs), both thread mappings, solid cells.
* rlb_init rejects u_z != 0; rlb_set_state rejects a state whose mirror images
  differ and takes a symmetric one.
* The FP64 form under the reduction meets the 1e-10 bar against the oracle.
"""
import numpy as np
import pytest

from paper_1302_1125_gb300 import rlb
from paper_1302_1125_gb300 import workloads as W

from norms import l1_fields

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
MIRRORS = [(5, 6), (11, 12), (13, 14), (15, 16), (17, 18)]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1302_1125_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def l1rel(a, b):
    return float(np.abs(a - b).sum() / np.abs(b).sum())


def run(w, steps, sym, **kw):
    g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, symmetry_2d=sym, **kw)
    g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
    l0 = g.launches
    g.step(steps)
    assert g.launches == l0 + steps
    return g


def oracle_macro(orc, w, steps):
    p = orc.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt=w.dt_over_dx,
                   eta_over_s=w.eta_over_s, zeta_over_s=w.zeta_over_s, tau_override=w.tau_override,
                   alpha_override=w.alpha_override, inlet_n=w.inlet[0], inlet_T=w.inlet[1],
                   inlet_u=tuple(w.inlet[2]))
    s = orc.init(p, *w.fields())
    orc.step(s, steps)
    assert s.nonphysical == 0
    return orc.macroscopic(s)


CASES = {
    "cloud_2d_s16": (lambda: W.cloud_2d(scale=16), 300),
    "box_2d": (lambda: W.periodic_box(48, 40, 1, seed=11, tau_override=0.0, alpha_override=0.1,
                                      precision=rlb.FP32_STORAGE), 150),
    "odd_box_2d": (lambda: W.periodic_box(45, 19, 1, seed=2, tau_override=0.0, alpha_override=0.05,
                                          precision=rlb.FP32_STORAGE), 120),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_reduced_step_matches_oracle(orc, name):
    make, steps = CASES[name]
    w = make()
    assert np.all(w.fields()[4] == 0.0)
    g = run(w, steps, 1)
    mg = g.macroscopic(device=False)
    g.close()
    mo = oracle_macro(orc, w, steps)
    errs = list(l1_fields(mg, mo).values())
    assert max(errs) <= 1e-4, errs
    assert np.abs(mg[4]).max() == 0.0          # u_z stays exactly zero


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("mapping", [rlb.MAPPING_TILES, rlb.MAPPING_LINEAR])
def test_reduced_step_equals_full_step(name, mapping):
    make, steps = CASES[name]
    w = make()
    full = run(w, steps, 0, thread_mapping=mapping)
    red = run(w, steps, 1, thread_mapping=mapping)
    mf, mr = full.macroscopic(device=False), red.macroscopic(device=False)
    for k in (0, 1, 5):
        assert l1rel(mr[k], mf[k]) <= 1e-6, k
    for k in (2, 3):
        assert np.abs(mr[k] - mf[k]).sum() / np.abs(mf[5]).sum() <= 1e-6, k
    tf, tr = full.totals(), red.totals()
    assert np.allclose(tr, tf, rtol=1e-6, atol=1e-6 * abs(tf[0]))
    f, h, prev = red.get_state()
    for a, b in MIRRORS:
        assert np.array_equal(f[a], f[b]) and np.array_equal(h[a], h[b]), (a, b)
    assert np.all(prev[3] == 0.0)
    full.close()
    red.close()


def test_mirror_refresh_launches_once_per_read():
    w = CASES["box_2d"][0]()
    g = run(w, 10, 1)
    l0 = g.launches
    g.macroscopic(device=False)
    l1 = g.launches
    g.totals()
    g.get_state()
    assert l1 - l0 == 2                      # refresh + output
    assert g.launches - l1 == 2              # totals' two kernels, no second refresh
    g.close()


def test_reduced_step_with_solid_cells():
    w = W.cloud_2d(scale=16)
    mask = np.zeros(w.N, np.uint8)
    yy, xx = np.divmod(np.arange(w.N), w.nx)
    mask[(xx - 60) ** 2 + (yy - 32) ** 2 <= 36] = 1
    out = []
    for sym in (0, 1):
        g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, symmetry_2d=sym)
        g.init(*w.fields()).set_solid(mask, 2.0, 0.5).step(80)
        out.append(g.macroscopic(device=False))
        g.close()
    for k in (0, 1):
        assert l1rel(out[1][k], out[0][k]) <= 1e-6
    sol = mask.nonzero()[0]
    assert np.abs(out[1][0, sol] / 2.0 - 1).max() <= 1e-6


def test_init_rejects_motion_in_z():
    w = CASES["box_2d"][0]()
    n, T, ux, uy, uz = w.fields()
    uz = uz.copy()
    uz[7] = 1e-3
    g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, symmetry_2d=1)
    with pytest.raises(rlb.RLBError) as e:
        g.init(n, T, ux, uy, uz)
    assert e.value.status == rlb.RLB_E_INVALID
    assert "mirror image" in rlb.last_error(g.ctx)
    g.init(*w.fields()).step(2)              # the context stays usable
    g.close()


def test_set_state_checks_the_symmetry():
    w = CASES["box_2d"][0]()
    g = run(w, 5, 1)
    f, h, prev = (a.copy() for a in g.get_state())
    g.step(5)
    ref = g.get_state()
    g2 = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, symmetry_2d=1)
    bad = f.copy()
    bad[12, 3] *= 1.0001
    with pytest.raises(rlb.RLBError) as e:
        g2.set_state(bad, h, prev)
    assert e.value.status == rlb.RLB_E_INVALID
    g2.set_state(f, h, prev).step(5)
    for a, b in zip(g2.get_state(), ref):
        assert np.array_equal(a, b)
    g.close()
    g2.close()


def test_full_size_cloud_2d_reduced_equals_full():
    """the benchmark's 2048 x 1024 2-D shock-cloud: 40 steps with and without
    the reduction, compared over the whole grid"""
    w = W.cloud_2d()
    full = run(w, 40, 0)
    red = run(w, 40, 1)
    mf, mr = full.macroscopic(device=False), red.macroscopic(device=False)
    for k in (0, 1, 5):
        assert l1rel(mr[k], mf[k]) <= 1e-6, k
        assert np.abs(mr[k] - mf[k]).max() <= 1e-5 * np.abs(mf[k]).max(), k
    for k in (2, 3):
        assert np.abs(mr[k] - mf[k]).sum() / np.abs(mf[5]).sum() <= 1e-6, k
    assert np.abs(mr[4]).max() == 0.0
    full.close()
    red.close()


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_reduced_step_matches_oracle(orc, name):
    """the FP64 form under the reduction: the 1e-10 bar against the oracle"""
    make, steps = CASES[name]
    w = make()
    g = rlb.Grid.from_workload(w, precision=rlb.FP64, symmetry_2d=1)
    g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()]).step(steps)
    mg = g.macroscopic(device=False)
    f, h, prev = g.get_state()
    g.close()
    mo = oracle_macro(orc, w, steps)
    for k in (0, 1, 5):
        assert np.abs(mg[k] - mo[k]).max() <= 1e-10 * np.abs(mo[k]).max(), k
    for k in (2, 3):
        assert np.abs(mg[k] - mo[k]).max() <= 1e-10 * np.abs(mo[2:4]).max(), k
    assert np.abs(mg[4]).max() == 0.0
    for a, b in MIRRORS:
        assert np.array_equal(f[a], f[b]) and np.array_equal(h[a], h[b]), (a, b)
    assert np.all(prev[3] == 0.0)
