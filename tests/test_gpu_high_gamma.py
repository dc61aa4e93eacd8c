"""The FP32-storage form where the Landau-frame recovery is hardest: gamma 5,
10 and 20, against the FP64 oracle, with the recovery in double-float (the
default) and in FP64 (recovery_fp64 = 1).

In the Landau frame for eps = 3P (Sec. II), E = 4 P gamma^2 - P and
|M| = 4 P gamma^2 beta, so E - |M| is about E / (4 gamma^2): the rest-frame
energy density e = 3P and n = N^0 / gamma hang on a difference that is
4 gamma^2 times smaller than the lab-frame densities E, M.  Both recoveries
form that difference from the exact sums of the stored populations, so a
single step is exact to float roundings in either (the one-step and
recovery checks below).  What they cannot undo is the storage: every step
rounds the 19 populations of f (and of h) to float, which moves a cell's E
and M by about one float rounding of E each (2^-24 E) at random, and moves
e by 4 gamma^2 times as much relative to its size.  Over K steps these add
up like a random walk:

    L1(e) ~ 4 sqrt(2) gamma^2 2^-24 sqrt(K)     (n: about half of it)

which exceeds the FP32 bar of 1e-4 above gamma ~ 2.5 over 2000 steps
(3.8e-4 at gamma 5, 1.5e-3 at 10, 6.0e-3 at 20 for K = 2000).  Measured on
GB300: 0.04 to 1.0 times this model, for both recoveries alike (FP64
arithmetic does not store more bits).  The lab-frame fields, which do not
suffer the cancellation, meet the bar at every gamma: the velocity (u_x
and the velocity vector) and E = T^00 within 1e-4.  These tests assert
exactly that:

* one step, every cell, gamma 1 .. 15: 64 float roundings, as at low gamma;
* the macroscopic output of a stored state, gamma up to 20: 8 roundings;
* 2000 steps at gamma 5, 10, 20: u_x, u and T^00 within 1e-4; e and n
  within twice the storage model; conserved totals within the same walk,
  4 x 2^-24 sqrt(K) of T^00 (on these states every cell of a y-z plane
  carries the same roundings, so the totals do not average them out as
  they do on the irregular states of the 1e-6 conservation test).

States (paper_1302_1125_gb300/workloads.py): periodic boxes moving as a
whole at gamma along x or along a diagonal, uniform, or with a 0.1 % ripple
of T and n along x.  The method itself stays physical on these (the oracle
runs them).  A ripple across the direction of motion at gamma >= 2 in 2-D
or 3-D, and the gamma = 20 diagonal ripple, it does not carry (the second-
order equilibrium's populations across the motion turn negative for
|u'|^2 > 15/16 and the lattice's diagonal velocities are faster than
light), so none is used here.
"""
import math

import numpy as np
import pytest

from paper_1302_1125_gb300 import rlb
from paper_1302_1125_gb300 import workloads as W

from norms import l1_fields

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP32_L1_TOL = 1e-4
DRIFT_TOL = 1e-6
STEPS = 2000
U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1302_1125_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def oparams(orc, w):
    return orc.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt=w.dt_over_dx,
                      eta_over_s=w.eta_over_s, zeta_over_s=w.zeta_over_s, tau_override=w.tau_override,
                      alpha_override=w.alpha_override)


def storage_model(gamma, steps):
    """L1 error of e from the random walk of the FP32 roundings (module doc)"""
    return 4.0 * math.sqrt(2.0) * gamma ** 2 * U * math.sqrt(steps)


def lab_energy(m):
    """T^00 = (e + P) gamma^2 - P with P = e / 3, from the (6, N) output"""
    return m[1] / 3.0 * (4.0 * m[5] ** 2 - 1.0)


def run_both(orc, w, steps, recovery_fp64, mapping=rlb.MAPPING_TILES):
    g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, thread_mapping=mapping,
                               recovery_fp64=recovery_fp64)
    g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
    t0 = g.totals()
    g.step(steps)
    t1 = g.totals()
    mg = g.macroscopic(device=False)
    g.close()
    s = orc.init(oparams(orc, w), *w.fields())
    orc.step(s, steps)
    assert s.nonphysical == 0
    mo = orc.macroscopic(s)
    errs = l1_fields(mg, mo)
    errs["T00"] = float(np.abs(lab_energy(mg) - lab_energy(mo)).sum() / np.abs(lab_energy(mo)).sum())
    # T^00 sets the scale of every total (|T^0a| < T^00, N^0 of the same order)
    drift = np.abs(t1 - t0) / np.abs(t0[0])
    return errs, drift


def check_long_run(errs, drift, gamma, steps):
    model = storage_model(gamma, steps)
    for k in ("u_x", "u", "T00"):
        assert errs[k] <= FP32_L1_TOL, (k, errs)
    for k in ("e", "n"):
        assert errs[k] <= 2.0 * model, (k, errs, model)
    assert drift.max() <= 4.0 * U * math.sqrt(steps), drift


DIRS = {"x": (1.0, 0.0, 0.0), "diagonal": (1.0, 1.0, 1.0)}


@pytest.mark.parametrize("recovery_fp64", [0, 1])
@pytest.mark.parametrize("direction", sorted(DIRS))
@pytest.mark.parametrize("gamma", [5.0, 10.0, 20.0])
def test_uniform_boost_3d(orc, gamma, direction, recovery_fp64):
    """a uniform state moving at gamma stays that state (16 x 8 x 4 cells,
    the tiled 3-D kernel)"""
    w = W.boosted_box(16, 8, 4, gamma=gamma, direction=DIRS[direction], amp=0.0)
    errs, drift = run_both(orc, w, STEPS, recovery_fp64)
    print(f"gamma {gamma} {direction} rec64={recovery_fp64}: L1 {errs} drift {drift.max():.2e} "
          f"model {storage_model(gamma, STEPS):.2e}")
    check_long_run(errs, drift, gamma, STEPS)


RIPPLE_CASES = [(g, d, dims) for g in (5.0, 10.0, 20.0) for d in sorted(DIRS)
                for dims in ((64, 1, 1), (32, 8, 4))
                # the diagonal ripple at gamma = 20 grows in the method itself
                if not (g == 20.0 and d == "diagonal")]


@pytest.mark.parametrize("recovery_fp64", [0, 1])
@pytest.mark.parametrize("gamma,direction,dims", RIPPLE_CASES)
def test_boosted_ripple(orc, gamma, direction, dims, recovery_fp64):
    """a 0.1 % ripple of T and n along x carried at gamma (sound waves in the
    moving gas), 1-D form and tiled 3-D kernel"""
    w = W.boosted_box(*dims, gamma=gamma, direction=DIRS[direction], amp=1e-3)
    errs, drift = run_both(orc, w, STEPS, recovery_fp64)
    print(f"gamma {gamma} {direction} {dims} rec64={recovery_fp64}: L1 {errs} drift {drift.max():.2e} "
          f"model {storage_model(gamma, STEPS):.2e}")
    check_long_run(errs, drift, gamma, STEPS)


@pytest.mark.parametrize("gamma_max", [10.0, 20.0])
def test_macroscopic_recovers_the_stored_state_at_high_gamma(orc, gamma_max):
    """rlb_macroscopic of an off-equilibrium FP32 state equals the oracle's
    FP64 recovery of the same stored populations within a few float
    roundings, with gamma up to gamma_max"""
    w = W.smooth_gamma_box(128, 8, 4, gamma_max=gamma_max)
    g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE)
    g.init(*w.fields()).step(3)             # off equilibrium
    f, h, _ = g.get_state()
    m = g.macroscopic(device=False)
    g.close()
    ref = np.zeros((6, w.N))
    for i in range(w.N):
        mac, bad = orc.recover(orc.moments(f[:, i].astype(np.float64), h[:, i].astype(np.float64)))
        assert not bad
        P, u, nn = mac[0], mac[1:4], mac[4]
        gam = math.sqrt(1.0 + u @ u)
        ref[:, i] = [nn, 3 * P, u[0] / gam, u[1] / gam, u[2] / gam, gam]
    assert ref[5].max() > 0.8 * gamma_max     # the peak relaxes a little in 3 steps
    # per cell: n, e and gamma relative to their own value, u (|u| < 1)
    # absolutely; 8 float roundings, as at low gamma
    for k in range(6):
        scale = np.abs(ref[k]) if k in (0, 1, 5) else 1.0
        err = np.max(np.abs(m[k] - ref[k]) / scale)
        assert err <= 8 * U, (k, err)


@pytest.mark.parametrize("recovery_fp64", [0, 1])
def test_one_step_cells_spanning_gamma_1_to_15(orc, recovery_fp64):
    """one FP32 step, every cell recomputed by the oracle from the GPU's own
    input state, on a state whose Lorentz factor runs from 1 to 15"""
    w = W.smooth_gamma_box(128, 8, 4, gamma_max=15.0)
    g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, thread_mapping=rlb.MAPPING_TILES,
                               recovery_fp64=recovery_fp64)
    g.init(*w.fields())
    g.step(1)
    f0, h0, p0 = g.get_state()         # level 1; p0 = the stored raw moment sums of level 0
    g.step(1)
    f1, h1, _ = g.get_state()          # level 2
    g.close()
    cells = np.arange(w.N, dtype=np.int64)
    # the oracle's previous level (P, u', n): its FP64 recovery of the sums the
    # GPU stored for level 0 (sum f, sum c_a f, sum h; E = xi0^2 sum f,
    # M = xi0 sum c f, N^0 = xi0 sum h)
    xi0 = orc.lattice()[4]
    prev = np.zeros((5, w.N), np.float64)
    for c in cells:
        sums = p0[:, c].astype(np.float64)
        mac, bad = orc.recover(np.r_[xi0 * xi0 * sums[0], xi0 * sums[1:4], xi0 * sums[4]])
        assert not bad
        prev[:, c] = mac
    fo, ho, mo, bad = orc.step_cells(oparams(orc, w), f0.astype(np.float64), h0.astype(np.float64), prev,
                                     cells)
    assert bad == 0
    assert mo[:, 1:4].max() > 10.0          # u' reaches gamma ~ 15 cells
    # Each output population is relaxed towards equilibrium values whose terms
    # reach |u'|^2 ~ 225 times the pressure, far above the population itself.
    # Measure the error per cell against the size of that cell's largest
    # population (the equilibrium's scale there): 64 float roundings, the
    # bound the low-gamma full-size check uses per plane.
    tol = 64 * U
    for a, b in ((f1, fo.T), (h1, ho.T)):
        scale = np.abs(b).max(0)
        err = (np.abs(a - b) / scale).max()
        print(f"rec64={recovery_fp64}: max error / cell scale {err:.2e} ({err / U:.1f} roundings)")
        assert err <= tol, err
