"""The seeded input recipes (Sec. III sets their shapes), checked on the CPU
against what each recipe states:

* layout: n, T and u are float64 arrays of N = nx ny nz values, x fastest;
* states "at lambda = 1" have n = n_eq(T) = d_G T^3 / pi^2 with d_G = 16;
* the shock tubes' pressure ratios and temperatures, the clouds' pressure
  balance with the ambient gas and their slab state, the sphere's solid
  cells (the integer points of a ball of radius 10 and 5: 4169 and 515, the
  counts of points of norm <= r^2 in the cubic lattice);
* the batched tubes' draws (order, ranges, reproducibility), packed offsets,
  4 Nx steps, and the totals quoted for the 512-tube sweep;
* every velocity is below the speed of light, and a periodic box stays below
  its gamma bound.
"""
import math

import numpy as np
import pytest

from paper_1302_1125_gb300 import workloads as W


def grid(w, a):
    return a.reshape(w.nz, w.ny, w.nx)


def test_n_eq():
    assert W.n_eq(1.0) == pytest.approx(16.0 / math.pi ** 2, rel=1e-15)
    assert W.n_eq(2.0) == pytest.approx(8.0 * W.n_eq(1.0), rel=1e-15)


@pytest.mark.parametrize("make", [W.tube_800, lambda: W.tube_8192("a", nx=512),
                                  lambda: W.cloud_2d(scale=16), lambda: W.cloud_3d(scale=8),
                                  lambda: W.sphere_cloud("beta02", scale=4),
                                  lambda: W.periodic_box(12, 10, 6)])
def test_fields_layout_and_light_cone(make):
    w = make()
    fl = w.fields()
    assert len(fl) == 5
    for a in fl:
        assert a.dtype == np.float64 and a.shape == (w.N,) and a.flags.c_contiguous
    n, T, ux, uy, uz = fl
    assert np.all(n > 0) and np.all(T > 0)
    assert np.all(ux * ux + uy * uy + uz * uz < 1.0)
    if w.ny == 1:
        assert not uy.any()
    if w.nz == 1:
        assert not uz.any()
    again = w.fields()
    for a, b in zip(fl, again):
        assert np.array_equal(a, b)          # the recipe is deterministic
        assert a is not b


def test_tube_800():
    w = W.tube_800()
    assert (w.nx, w.ny, w.nz, w.steps) == (800, 1, 1, 2000)
    assert (w.dt_over_dx, w.eta_over_s, w.zeta_over_s) == (0.25, 0.1, 0.0)
    n, T, ux, uy, uz = w.fields()
    L, R = slice(0, 400), slice(400, 800)
    assert np.all(T[L] == 2.0) and np.all(T[R] == 1.0)
    assert np.all(n[R] == W.n_eq(1.0))
    assert n[0] * T[0] / (n[-1] * T[-1]) == pytest.approx(5.43 / 0.339, rel=1e-14)
    assert not ux.any()
    assert w.bc_lo[0] == W.BC_OUTFLOW and w.bc_hi[0] == W.BC_OUTFLOW


@pytest.mark.parametrize("variant,eta,zeta", [("a", 0.01, 0.0), ("b", 0.5, 0.05)])
def test_tube_8192(variant, eta, zeta):
    w = W.tube_8192(variant)
    assert (w.nx, w.steps, w.dt_over_dx, w.alpha_override) == (8192, 20000, 0.15, 0.2)
    assert (w.eta_over_s, w.zeta_over_s) == (eta, zeta)
    n, T, ux, _, _ = w.fields()
    # both sides at lambda = 1, pressure ratio 1000, at rest
    assert n == pytest.approx(W.n_eq(T), rel=1e-14)
    assert n[0] * T[0] / (n[-1] * T[-1]) == pytest.approx(1000.0, rel=1e-14)
    assert not ux.any()


@pytest.mark.parametrize("make,R,centre,slab", [
    (lambda: W.cloud_2d(), 96.0, (700.0, 512.0), 256),
    (lambda: W.cloud_2d(scale=16), 6.0, (43.75, 32.0), 16),
    (lambda: W.cloud_3d(scale=4), 12.0, (45.0, 32.0, 32.0), 16),
])
def test_cloud_recipe(make, R, centre, slab):
    w = make()
    n, T, ux, uy, uz = (grid(w, a) for a in w.fields())
    nA = W.n_eq(1.0)
    ambient = n[:, :, slab:]
    # pressure balance with the ambient gas outside the slab
    assert np.allclose(ambient * T[:, :, slab:], nA, rtol=1e-14)
    # the slab: at rest, lambda = 1, pressure ratio 10
    sn, sT = n[:, :, :slab], T[:, :, :slab]
    assert np.all(sn == sn.flat[0]) and np.all(sT == sT.flat[0])
    assert sn.flat[0] == pytest.approx(W.n_eq(sT.flat[0]), rel=1e-14)
    assert sn.flat[0] * sT.flat[0] / nA == pytest.approx(10.0, rel=1e-14)
    assert not (ux.any() or uy.any() or uz.any())
    # density between the ambient and 10x it, highest at the centre (10x when
    # the radius is many edge widths), ambient far away, half-way at r = R
    assert ambient.min() >= nA and ambient.max() <= 10.0 * nA
    c = [int(round(v)) for v in centre]
    idx = (c[2] if w.nz > 1 else 0, c[1], c[0])
    assert n[idx] == ambient.max()
    if R >= 40:
        assert n[idx] == pytest.approx(10.0 * nA, rel=1e-6)
    assert n[0, 0, -1] == pytest.approx(nA, rel=1e-6)
    edge = (idx[0], idx[1], int(round(centre[0] + R)))
    if abs(centre[0] + R - edge[2]) < 1e-9:
        assert n[edge] == pytest.approx(5.5 * nA, rel=1e-12)
    assert w.bc_lo[0] == W.BC_INLET and w.bc_hi[0] == W.BC_OUTFLOW
    assert w.inlet[0] == sn.flat[0] and w.inlet[1] == sT.flat[0]


def test_cloud_sizes():
    assert (W.cloud_2d().nx, W.cloud_2d().ny, W.cloud_2d().nz) == (2048, 1024, 1)
    w = W.cloud_3d()
    assert (w.nx, w.ny, w.nz, w.steps) == (512, 256, 256, 2000)
    assert (w.eta_over_s, w.zeta_over_s, w.alpha_override, w.dt_over_dx) == (0.05, 0.01, 0.2, 0.15)


@pytest.mark.parametrize("scale,count", [(1, 4169), (2, 515)])
def test_sphere_solid_cells(scale, count):
    w = W.sphere_cloud("beta09", scale=scale)
    m = w.solid_mask()
    assert m.dtype == np.uint8 and m.shape == (w.N,)
    assert int(m.sum()) == count
    cells = np.argwhere(grid(w, m))
    assert np.array_equal(cells.mean(axis=0), np.array([50, 50, 100]) / scale)


@pytest.mark.parametrize("case,T0,r", [("beta02", 2.71, 0.9), ("beta09", 54.77, 10.95)])
def test_sphere_states(case, T0, r):
    w = W.sphere_cloud(case, scale=4)
    n, T, _, _, _ = (grid(w, a) for a in w.fields())
    n1 = W.n_eq(1.0)
    slab = np.arange(w.nx) <= 65.0 / 4
    assert np.all(T[:, :, slab] == T0) and np.all(n[:, :, slab] == r * n1)
    assert np.all(T[:, :, ~slab] == 1.0) and np.all(n[:, :, ~slab] == n1)
    assert w.inlet[:2] == (r * n1, T0)
    assert w.solid[1:] == (n1, 1.0)
    assert w.euler_mode == 1 and W.sphere_cloud(case, viscous=True).tau_override == 1.0


def test_batch_tubes_draws():
    b = W.batch_tubes()
    rng = np.random.default_rng(1234)
    nx = np.exp(rng.uniform(math.log(256), math.log(8192), 512)).round()
    assert np.array_equal(b.nx, nx.astype(np.int32))
    assert np.array_equal(b.eta_over_s, rng.uniform(0.01, 0.5, 512))
    assert np.array_equal(b.zeta_over_s, rng.uniform(0.0, 0.1, 512))
    assert np.array_equal(b.ratio, np.exp(rng.uniform(math.log(2.0), math.log(40.0), 512)))
    assert np.array_equal(b.gamma_left, rng.uniform(1.0, 1.5, 512))
    assert b.B == 512 and b.nx.min() >= 256 and b.nx.max() <= 8192
    assert np.array_equal(b.steps, 4 * b.nx.astype(np.int64))
    assert b.offsets[0] == 0 and np.array_equal(np.diff(b.offsets), b.nx)
    # the totals of the 512-tube sweep
    assert int(b.offsets[-1]) == 1156618
    assert int((b.nx.astype(np.int64) * b.steps).sum()) == 19491919584


def test_batch_tubes_fields():
    b = W.batch_tubes(count=16, seed=5)
    n, T, ux = b.fields()
    assert n.shape == T.shape == ux.shape == (int(b.offsets[-1]),)
    nR = W.n_eq(1.0)
    for k in range(b.B):
        o, m = int(b.offsets[k]), int(b.nx[k])
        L, R = slice(o, o + m // 2), slice(o + m // 2, o + m)
        assert np.all(T[R] == 1.0) and np.all(n[R] == nR) and not ux[R].any()
        assert n[o] == pytest.approx(W.n_eq(T[o]), rel=1e-14)
        assert n[o] * T[o] / nR == pytest.approx(b.ratio[k], rel=1e-14)
        g = 1.0 / math.sqrt(1.0 - ux[o] ** 2)
        assert g == pytest.approx(b.gamma_left[k], rel=1e-12)
        assert np.all(ux[L] == ux[o]) and ux[o] < 1.0


def test_periodic_box_gamma_bound():
    for seed in range(5):
        w = W.periodic_box(16, 8, 4, seed=seed, gamma_max=3.0)
        n, T, ux, uy, uz = w.fields()
        gam = 1.0 / np.sqrt(1.0 - (ux * ux + uy * uy + uz * uz))
        assert gam.max() <= 3.0
        assert w.bc_lo == (W.BC_PERIODIC,) * 3 and w.bc_hi == (W.BC_PERIODIC,) * 3


@pytest.mark.parametrize("make,kw", [
    (W.tube_800, {}), (W.tube_800, {"symmetry_1d": 1}), (lambda: W.tube_8192("a"), {}),
    (lambda: W.tube_8192("b"), {}), (W.cloud_2d, {}), (W.cloud_2d, {"symmetry_2d": 1}),
    (W.cloud_3d, {}), (lambda: W.sphere_cloud("beta02", viscous=True), {}),
    (lambda: W.sphere_cloud("beta09"), {}), (lambda: W.periodic_box(16, 8, 4), {}),
    (W.cloud_3d, {"model": 1}), (W.tube_800, {"model": 1}),
])
@pytest.mark.parametrize("precision", [W.FP64, W.FP32_STORAGE])
def test_every_recipe_passes_host_validation(make, kw, precision):
    """each workload's grid, boundaries, dt/dx and alpha pass rlb_create's
    checks (stability bounds included): without a device the call gets as
    far as the device, RLB_E_CUDA"""
    from paper_1302_1125_gb300 import rlb
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(rlb.RLBError) as e:
        rlb.Grid.from_workload(make(), precision=precision, **kw)
    assert e.value.status == rlb.RLB_E_CUDA, str(e.value)


@pytest.mark.parametrize("gamma,direction,amp", [(10.0, (1.0, 0.0, 0.0), 1e-3), (20.0, (1.0, 1.0, 1.0), 0.0),
                                                 (5.0, (0.0, 2.0, 1.0), 1e-2)])
def test_boosted_box(gamma, direction, amp):
    w = W.boosted_box(16, 4, 2, gamma=gamma, direction=direction, amp=amp)
    assert w.bc_lo == w.bc_hi == (W.BC_PERIODIC,) * 3
    n, T, ux, uy, uz = (grid(w, a) for a in w.fields())
    v2 = ux ** 2 + uy ** 2 + uz ** 2
    assert np.allclose(1.0 / np.sqrt(1.0 - v2), gamma, rtol=1e-12)
    d = np.asarray(direction) / np.linalg.norm(direction)
    for a, c in zip((ux, uy, uz), d):
        assert np.allclose(a / np.sqrt(v2), c, atol=1e-15)
    # the ripple: relative size amp in T (amp / 2 in n) and along x only
    assert np.abs(T - 1.0).max() <= 1.5 * amp + 1e-15
    assert np.abs(n / W.n_eq(1.0) - 1.0).max() <= 0.5 * amp + 1e-15
    for a in (n, T):
        assert np.array_equal(a, np.broadcast_to(a[:1, :1, :], a.shape))
    if amp == 0.0:
        assert np.all(T == 1.0) and np.all(n == W.n_eq(1.0))


def test_smooth_gamma_box_spans_the_range():
    w = W.smooth_gamma_box(128, 8, 4, gamma_max=15.0)
    n, T, ux, uy, uz = (grid(w, a) for a in w.fields())
    gam = 1.0 / np.sqrt(1.0 - (ux ** 2 + uy ** 2 + uz ** 2))
    assert gam.min() == pytest.approx(1.0, abs=1e-12)
    assert gam.max() == pytest.approx(15.0, rel=2e-3)
    assert np.all(n > 0) and np.all(T > 0)
    # every field varies along x only (no gradient across the flow)
    for a in (n, T, ux, uy, uz, gam):
        assert np.array_equal(a, np.broadcast_to(a[:1, :1, :], a.shape))
