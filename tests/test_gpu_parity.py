"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 form: every macroscopic field within 1e-10 relative (max-norm over the
grid, normalised by the field's max) of the oracle after the same number of
steps on the same seeded inputs.  FP32-storage form: per-field L1 relative
error against the FP64 oracle <= 1e-4 and conservation drift <= 1e-6.  At
the full 512 x 256 x 256 size the oracle recomputes a sample of cells one
by one from the GPU's own input state and the GPU's output must match.
"""
import math

import numpy as np
import pytest

from paper_1302_1125_gb300 import rlb
from paper_1302_1125_gb300 import workloads as W

from norms import l1_fields

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP64_TOL = 1e-10
FP32_L1_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1302_1125_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def oparams(orc, w, **kw):
    p = orc.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt=w.dt_over_dx,
                   eta_over_s=w.eta_over_s, zeta_over_s=w.zeta_over_s,
                   tau_override=w.tau_override, alpha_override=w.alpha_override,
                   inlet_n=w.inlet[0], inlet_T=w.inlet[1], inlet_u=tuple(w.inlet[2]),
                   euler_mode=w.euler_mode)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def run_gpu(w, steps, precision, limiter=0):
    g = rlb.Grid(w.nx, w.ny, w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, inlet=w.inlet,
                 eta_over_s=w.eta_over_s, zeta_over_s=w.zeta_over_s, limiter=limiter,
                 dt_over_dx=w.dt_over_dx, tau_override=w.tau_override,
                 alpha_override=w.alpha_override, euler_mode=w.euler_mode, precision=precision)
    g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
    launches = g.launches
    g.step(steps)
    assert g.launches == launches + steps
    return g, g.macroscopic(device=False)


def run_oracle(orc, w, steps, limiter=0):
    s = orc.init(oparams(orc, w, limiter=limiter), *w.fields())
    orc.step(s, steps)
    assert s.nonphysical == 0
    return s, orc.macroscopic(s)


def relinf(a, b):
    scale = np.abs(b).max()
    return np.abs(a - b).max() / scale if scale > 0 else np.abs(a - b).max()


def l1rel(a, b):
    return np.abs(a - b).sum() / np.abs(b).sum()


def assert_fp64_parity(mg, mo, fields=(0, 1, 2, 3, 4, 5)):
    names = ["n", "e", "u_x", "u_y", "u_z", "gamma"]
    for k in fields:
        if k in (2, 3, 4):
            err = np.abs(mg[k] - mo[k]).max() / max(np.abs(mo[2:5]).max(), 1e-300)
        else:
            err = relinf(mg[k], mo[k])
        assert err <= FP64_TOL, f"{names[k]}: {err:.3e}"


def _box(nx, ny, nz, seed, **kw):
    return W.periodic_box(nx, ny, nz, seed=seed, **kw)


FP64_CASES = {
    "tube_800_full": (lambda: W.tube_800(), 2000, 0),
    "tube_8192a_full_nx": (lambda: W.tube_8192("a"), 300, 0),
    "tube_8192b": (lambda: W.tube_8192("b", nx=1024), 500, 0),
    "cloud_2d_s16": (lambda: W.cloud_2d(scale=16, precision=0), 200, 0),
    "cloud_3d_s16": (lambda: W.cloud_3d(scale=16, precision=0), 100, 0),
    "ragged_3d_box": (lambda: _box(37, 13, 11, 1, tau_override=0.0, alpha_override=0.1), 60, 0),
    "ragged_2d_box": (lambda: _box(45, 19, 1, 2, tau_override=0.0, alpha_override=0.05), 100, 0),
    "ragged_1d_tube": (lambda: W.riemann_tube(203, 16.0, 2.0, eta_over_s=0.05), 400, 0),
    "first_order_upwind": (lambda: W.riemann_tube(123, 16.0, 2.0, eta_over_s=0.05), 300, 1),
    "tiny_1x1x1": (lambda: _box(1, 1, 1, 3), 20, 0),
    "tiny_2x1x1": (lambda: _box(2, 1, 1, 4), 20, 0),
    "tiny_3x3x3": (lambda: _box(3, 3, 3, 5), 20, 0),
    "tiny_2x3x1": (lambda: _box(2, 3, 1, 6), 20, 0),
}


@pytest.mark.parametrize("name", sorted(FP64_CASES))
def test_fp64_matches_oracle(orc, name):
    make, steps, limiter = FP64_CASES[name]
    w = make()
    w.precision = 0
    g, mg = run_gpu(w, steps, rlb.FP64, limiter)
    _, mo = run_oracle(orc, w, steps, limiter)
    assert_fp64_parity(mg, mo)


def test_fp64_outflow_on_every_face(orc):
    w = _box(20, 12, 10, 8, tau_override=0.0, alpha_override=0.1)
    w.bc_lo = w.bc_hi = (1, 1, 1)
    w.eta_over_s = 0.05
    g, mg = run_gpu(w, 40, rlb.FP64)
    _, mo = run_oracle(orc, w, 40)
    assert_fp64_parity(mg, mo)


@pytest.mark.parametrize("dims", [(203, 1, 1), (29, 17, 1), (17, 9, 7)])
def test_fp64_euler_mode_matches_oracle(orc, dims):
    if dims[1] == 1:
        w = W.riemann_tube(dims[0], 1000.0, 1000.0 ** 0.25, dt_over_dx=0.15, alpha_override=0.2)
    else:
        w = _box(*dims, seed=9, tau_override=0.0, alpha_override=0.1)
    w.euler_mode = 1
    g, mg = run_gpu(w, 150, rlb.FP64)
    _, mo = run_oracle(orc, w, 150)
    assert_fp64_parity(mg, mo)


def test_fp64_single_step_populations_match(orc):
    # one step from the same state: every population and the stored macros
    w = W.cloud_3d(scale=16, precision=0)
    g, _ = run_gpu(w, 5, rlb.FP64)
    f0, h0, p0 = g.get_state()
    g.step(1)
    f1, h1, p1 = g.get_state()
    cells = np.arange(w.N)
    fo, ho, mo, bad = orc.step_cells(oparams(orc, w), f0, h0, p0, cells)
    assert bad == 0
    for a, b in ((f1, fo.T), (h1, ho.T), (p1, mo.T)):
        for k in range(a.shape[0]):
            assert relinf(a[k], b[k]) <= 1e-12


def test_fp32_form_l1_error_against_fp64_oracle(orc):
    report = {}
    for name, make, steps in (("tube_800", lambda: W.tube_800(), 2000),
                              ("tube_8192a", lambda: W.tube_8192("a", nx=2048), 2000),
                              ("cloud_2d_s16", lambda: W.cloud_2d(scale=16), 300),
                              # the headline shock-cloud, shrunk 8x per axis (64 x 32 x 32)
                              ("cloud_3d_s8", lambda: W.cloud_3d(scale=8), 200)):
        w = make()
        _, mg = run_gpu(w, steps, rlb.FP32_STORAGE)
        _, mo = run_oracle(orc, w, steps)
        errs = l1_fields(mg, mo)
        report[name] = errs
        assert max(errs.values()) <= FP32_L1_TOL, (name, errs)
    print("FP32 L1 errors (n, e, u_x):", report)


def _euler(w):
    w.euler_mode = 1
    return w


def _all_outflow(w):
    w.bc_lo = w.bc_hi = (1, 1, 1)
    w.eta_over_s = 0.05
    return w


# the FP32-storage kernel's other paths: staging with wrap-around in x, y and
# z (even nx), the unstaged path (odd nx), Euler mode (unstaged), open faces
FP32_CASES = {
    "even_3d_periodic_box": (lambda: _box(36, 14, 10, 12, tau_override=0.0, alpha_override=0.1), 80),
    "ragged_3d_box": (lambda: _box(37, 13, 11, 1, tau_override=0.0, alpha_override=0.1), 60),
    "outflow_every_face": (lambda: _all_outflow(_box(20, 12, 10, 8, tau_override=0.0, alpha_override=0.1)), 40),
    "euler_tube": (lambda: _euler(W.riemann_tube(400, 1000.0, 1000.0 ** 0.25, dt_over_dx=0.15,
                                                 alpha_override=0.2)), 300),
    "euler_3d_box": (lambda: _euler(_box(18, 10, 8, 9, tau_override=0.0, alpha_override=0.1)), 80),
    "tiny_2x1x1": (lambda: _box(2, 1, 1, 4), 20),
}


@pytest.mark.parametrize("name", sorted(FP32_CASES))
def test_fp32_paths_l1_error_against_fp64_oracle(orc, name):
    make, steps = FP32_CASES[name]
    w = make()
    _, mg = run_gpu(w, steps, rlb.FP32_STORAGE)
    _, mo = run_oracle(orc, w, steps)
    errs = l1_fields(mg, mo)
    assert max(errs.values()) <= FP32_L1_TOL, (name, errs)


@pytest.mark.parametrize("make", [
    lambda: _box(37, 13, 11, 1, tau_override=0.0, alpha_override=0.1),      # odd nx: single-cell pairs
    lambda: _box(36, 14, 10, 12, tau_override=0.0, alpha_override=0.1),
    lambda: _all_outflow(_box(20, 12, 10, 8, tau_override=0.0, alpha_override=0.1)),
    lambda: _box(200, 9, 1, 3, tau_override=0.0, alpha_override=0.1),       # 2-D, rows break inside warps
    lambda: _box(128, 8, 3, 5, tau_override=0.0, alpha_override=0.1),       # tiles fill: both take every lane
    lambda: W.sphere_cloud("beta02", scale=4, viscous=True),                # inlet face, 50 x 25 x 25
])
@pytest.mark.parametrize("precision", [rlb.FP32_STORAGE, rlb.FP64])
def test_thread_mappings_agree_bit_for_bit(make, precision):
    """tiles and the linear order cover the same cells with the same
    per-cell code: the states are equal bit for bit"""
    w = make()
    states = []
    for mapping in (rlb.MAPPING_TILES, rlb.MAPPING_LINEAR, rlb.MAPPING_AUTO):
        g = rlb.Grid.from_workload(w, precision=precision, thread_mapping=mapping)
        g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
        g.step(15)
        states.append(g.get_state())
        g.close()
    for other in states[1:]:
        for a, b in zip(states[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("precision,tol", [(rlb.FP64, 1e-13), (rlb.FP32_STORAGE, 1e-6)])
def test_conservation_drift(precision, tol):
    w = _box(48, 40, 1, 11, tau_override=0.8, alpha_override=0.15)
    g = rlb.Grid.from_workload(w, precision=precision)
    g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
    t0 = g.totals()
    g.step(2000)
    t1 = g.totals()
    drift = np.abs(t1 - t0) / t0[0]
    assert drift.max() <= tol, drift


def test_totals_match_oracle(orc):
    w = W.cloud_2d(scale=16, precision=0)
    g, _ = run_gpu(w, 50, rlb.FP64)
    s, _ = run_oracle(orc, w, 50)
    _, c, _, _, xi0 = orc.lattice()
    f = s.f.reshape(19, -1)
    h = s.h.reshape(19, -1)
    t = np.r_[xi0 * xi0 * f.sum(), xi0 * (c.T @ f.sum(1)), xi0 * h.sum()]
    assert np.allclose(g.totals(), t, rtol=1e-12, atol=1e-12 * abs(t[0]))


def test_full_size_cloud_3d_sampled_cells(orc):
    # the benchmark's workload and launch configuration, full size (FP32 form)
    w = W.cloud_3d()
    g = rlb.Grid.from_workload(w)
    g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
    g.step(2)
    fa, ha, _ = g.get_state()          # time level 2
    g.step(1)
    f0, h0, p0 = g.get_state()         # time level 3; p0 = raw moment sums of level 2
    g.step(1)
    f1, h1, p1 = g.get_state()         # time level 4; p1 = raw moment sums of level 3
    rng = np.random.default_rng(2024)
    nx, ny, nz = w.nx, w.ny, w.nz
    special = [x + nx * (y + ny * z) for x in (0, 1, 2, 63, 64, nx - 2, nx - 1)
               for y in (0, ny // 2, ny - 1) for z in (0, nz // 2, nz - 1)]
    cells = np.unique(np.r_[rng.integers(0, w.N, 3000), special]).astype(np.int64)
    # the oracle's previous level: its own moments and recovery of level 2
    prev = np.zeros((5, w.N), np.float32)
    for c in cells:
        mac, bad = orc.recover(orc.moments(fa[:, c].astype(np.float64), ha[:, c].astype(np.float64)))
        assert not bad
        prev[:, c] = mac
    fo, ho, mo, bad = orc.step_cells(oparams(orc, w), f0, h0, prev, cells)
    assert bad == 0
    # one FP32 step rounds each population about 50 times (streaming, moments,
    # recovery, coefficients, relaxation) on values up to ~3x the population's
    # scale; 64 units of float rounding (2^-24 each) of the plane's scale bound it
    tol = 64 * 2.0 ** -24
    for a, b in ((f1[:, cells], fo.T), (h1[:, cells], ho.T)):
        for k in range(19):
            err = np.abs(a[k] - b[k]).max() / np.abs(b[k]).max()
            assert err <= tol, (k, err)
    # the stored previous level is the raw sums of the step's own input
    # (c_a = 1, so the oracle's lattice vectors are the integer vectors c_i)
    _, c, _, _, _ = orc.lattice()
    f0c = f0[:, cells].astype(np.float64)
    sums = np.vstack([f0c.sum(0), c.T @ f0c, h0[:, cells].astype(np.float64).sum(0)])
    for k in range(5):
        scale = np.abs(sums[k]).max() if k in (0, 4) else np.abs(sums[1:4]).max() + 1e-300
        assert np.abs(p1[k, cells] - sums[k]).max() / scale <= 1e-6, k


def test_checkpoint_resume_is_bit_exact():
    w = W.cloud_2d(scale=16)
    for precision in (rlb.FP64, rlb.FP32_STORAGE):
        a = rlb.Grid.from_workload(w, precision=precision)
        a.init(*[torch.as_tensor(x, device="cuda") for x in w.fields()])
        a.step(30)
        snap = a.get_state()
        a.step(30)
        b = rlb.Grid.from_workload(w, precision=precision)
        b.set_state(*snap)
        b.step(30)
        for x, y in zip(a.get_state(), b.get_state()):
            assert np.array_equal(x, y)


def test_host_and_device_inputs_agree():
    w = W.tube_800()
    a = rlb.Grid.from_workload(w).init(*w.fields())
    b = rlb.Grid.from_workload(w).init(*[torch.as_tensor(x, device="cuda") for x in w.fields()])
    a.step(10)
    b.step(10)
    assert np.array_equal(a.macroscopic(device=False), b.macroscopic(device=True).cpu().numpy())


def test_runs_on_a_side_stream():
    w = W.cloud_2d(scale=16)
    ref = rlb.Grid.from_workload(w).init(*w.fields()).step(20).macroscopic(device=False)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g = rlb.Grid.from_workload(w).init(*w.fields()).step(20)
        out = g.macroscopic(device=False)
    assert np.array_equal(ref, out)


def test_superluminal_or_nan_initial_state_is_rejected():
    w = W.tube_800()
    n, T, ux, uy, uz = w.fields()
    for bad in ("u", "nan"):
        g = rlb.Grid.from_workload(w)
        n2, ux2 = n.copy(), ux.copy()
        if bad == "u":
            ux2[17] = 1.0
        else:
            n2[5] = math.nan
        with pytest.raises(rlb.RLBError) as e:
            g.init(n2, T, ux2, uy, uz)
        assert e.value.status == rlb.RLB_E_INVALID
        g.init(n, T, ux, uy, uz)          # the context stays usable
        g.step(2)


def test_non_physical_state_is_reported_and_cleared():
    w = W.tube_800()
    g = rlb.Grid.from_workload(w).init(*w.fields())
    f, h, p = g.get_state()
    f = f.copy()
    f[1, 400] += 50.0 * abs(f[0, 400])      # |M| > E at one cell
    f[0, 400] -= 50.0 * abs(f[0, 400])
    g.set_state(f, h, p)
    with pytest.raises(rlb.RLBError) as e:
        g.step(1)
    assert e.value.status == rlb.RLB_E_NONPHYSICAL
    g.init(*w.fields())
    g.step(3)                                # status was cleared
