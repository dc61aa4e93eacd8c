"""Pins of the oracle against the exact solution of the relativistic Riemann
problem (Sec. III validates the method's inviscid limit against it).

The exact solver (oracle/riemann.py) is itself checked against the
conservation laws: the Rankine-Hugoniot conditions at each shock, constant
Riemann invariants through each rarefaction fan, continuous P and v at the
contact.  The paper's printed prose values are a weak pin of the solver
(tests/golden/paper_riemann.txt).  The oracle is then run on shock tubes and
its L1 error against the exact solution must shrink as the grid is refined.
"""
import os

import numpy as np
import pytest

from oracle import riemann as R
from paper_1302_1125_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_riemann.txt")
CASES = [(2.445946, 0.0, 1.0, 0.0), (1000.0, 0.0, 1.0, 0.0), (20.0, 0.5, 1.0, 0.0),
         (3.0, -0.3, 1.0, 0.4), (1.0, 0.6, 1.0, -0.6), (0.2, 0.0, 1.0, 0.3)]


def _states(PL, vL, PR, vR):
    return R.solve(PL, vL, 1.3 * PL ** 0.75, PR, vR, PR ** 0.75)


@pytest.mark.parametrize("PL,vL,PR,vR", CASES)
def test_exact_solver_satisfies_jump_conditions(PL, vL, PR, vR):
    s = _states(PL, vL, PR, vR)
    # contact: P and v continuous by construction of the star state
    for kind, speeds, up, down in (
        (s.left_kind, s.left_speeds, (s.PL, s.vL, s.nL), (s.Pstar, s.vstar, s.nLstar)),
        (s.right_kind, s.right_speeds, (s.PR, s.vR, s.nR), (s.Pstar, s.vstar, s.nRstar)),
    ):
        if kind == "shock":
            sh = speeds[0]
            Ua, Fa = R.conserved_fluxes(*up)
            Ub, Fb = R.conserved_fluxes(*down)
            for k in range(3):
                # [F - s U] = 0 across a discontinuity moving at speed s
                jump = (Fb[k] - sh * Ub[k]) - (Fa[k] - sh * Ua[k])
                assert abs(jump) < 1e-9 * max(abs(Fa[k]), abs(Ua[k]), abs(Fb[k]), 1e-300)
        else:
            lo, hi = min(speeds), max(speeds)
            xi = np.linspace(lo, hi, 9)
            P, v, n = s.sample(xi)
            sign = 1.0 if s.left_kind == kind and speeds == s.left_speeds else -1.0
            J = np.arctanh(v) + sign * np.sqrt(3.0) / 4.0 * np.log(P)
            assert np.ptp(J) < 1e-9
            assert np.allclose(n / P ** 0.75, n[0] / P[0] ** 0.75, rtol=1e-9)
    # self-similar sampling reproduces the end states
    P, v, n = s.sample(np.array([-0.999999, 0.999999]))
    assert np.allclose([P[0], v[0], P[1], v[1]], [s.PL, s.vL, s.PR, s.vR])


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        ratio, qty, val, tol, status = line.split()[:5]
        rows.append((float(ratio), qty, float(val), float(tol), status))
    return rows


@pytest.mark.parametrize("ratio,qty,val,tol,status", _golden())
def test_paper_printed_riemann_values(ratio, qty, val, tol, status):
    s = R.solve(ratio, 0.0, 1.0, 1.0, 0.0, 1.0)
    exact = {"beta_plateau": s.vstar, "v_shock": s.right_speeds[0],
             "gamma_plateau": 1.0 / np.sqrt(1.0 - s.vstar ** 2)}[qty]
    if status == "pin":
        assert abs(exact - val) <= tol
    else:
        assert abs(exact - val) > tol     # recorded disagreement stays a disagreement


def _tube_error(orc, nx, ratio, euler, alpha, dt, eta=0.01, frac=0.3):
    w = W.riemann_tube(nx, ratio, 1.0, eta_over_s=eta, dt_over_dx=dt)
    n, T, ux, uy, uz = w.fields()
    p = orc.Params(nx=nx, dt=dt, eta_over_s=eta, euler_mode=euler, alpha_override=alpha)
    st = orc.init(p, n, T, ux, uy, uz)
    sol = R.solve(n[0] * T[0], 0.0, n[0], n[-1] * T[-1], 0.0, n[-1])
    vmax = max(abs(sol.left_speeds[0]), abs(sol.right_speeds[-1]))
    steps = int(round(frac * nx / vmax / dt))
    orc.step(st, steps)
    assert st.nonphysical == 0
    m = orc.macroscopic(st)
    P, v, nn = sol.sample((np.arange(nx) + 0.5 - nx / 2) / (steps * dt))
    l1 = lambda a, b: np.abs(a - b).sum() / np.abs(b).sum()
    return np.array([l1(m[1] / 3.0, P), l1(m[2], v), l1(m[0], nn)])


@pytest.mark.parametrize("euler", [1, 0])
def test_weakly_relativistic_tube_converges_to_exact_solution(orc, euler):
    # Sec. III first validation test: P0/P1 = 5.43/2.22, plateau beta ~ 0.2
    errs = [_tube_error(orc, nx, 5.43 / 2.22, euler, 0.0, 0.25) for nx in (200, 400, 800)]
    assert np.all(errs[1] < 0.8 * errs[0]) and np.all(errs[2] < 0.8 * errs[1]), errs
    assert np.all(errs[2] < [3e-3, 1e-2, 4e-3]), errs[2]


def test_highly_relativistic_tube_converges_to_exact_solution(orc):
    # Sec. III inviscid test: P0/P1 = 1e3 (plateau beta 0.91), Euler mode with
    # the bulk term alpha = 0.2 that the paper uses at high velocity
    errs = [_tube_error(orc, nx, 1000.0, 1, 0.2, 0.15) for nx in (200, 400, 800)]
    assert np.all(errs[1] < 0.8 * errs[0]) and np.all(errs[2] < 0.8 * errs[1]), errs
    assert np.all(errs[2] < [0.04, 0.2, 0.04]), errs[2]


@pytest.mark.parametrize("case,tol", [("beta02", 0.005), ("beta09", 0.025)])
def test_astrophysical_run_states_reach_the_printed_velocity(orc, case, tol):
    """The slab and ambient states of the paper's 3-D run (Sec. III), in its
    setting (Euler mode, alpha 0.2, dt/dx 0.15), on a 1-D tube: the gas
    behind the shock moves at the exact plateau velocity, which the golden
    file ties to the printed beta = 0.2 and 0.9."""
    w = W.sphere_cloud(case, scale=1)
    n0, T0 = w.inlet[0], w.inlet[1]
    n1, T1 = w.solid[1], w.solid[2]
    nx, steps, dt = 400, 800, 0.15
    x = np.arange(nx)
    slab = x < nx // 2
    z = np.zeros(nx)
    p = orc.Params(nx=nx, dt=dt, alpha_override=0.2, euler_mode=1)
    st = orc.init(p, np.where(slab, n0, n1), np.where(slab, T0, T1), z, z, z)
    orc.step(st, steps)
    assert st.nonphysical == 0
    m = orc.macroscopic(st)
    sol = R.solve(n0 * T0, 0.0, n0, n1 * T1, 0.0, n1)
    _, v, _ = sol.sample((x + 0.5 - nx // 2) / (steps * dt))
    plateau = np.abs(v - sol.vstar) < 1e-12
    assert plateau.sum() > 30
    assert abs(float(np.median(m[2][plateau])) - sol.vstar) < tol
    printed = {"beta02": 0.2, "beta09": 0.9}[case]
    assert abs(sol.vstar - printed) < 0.015


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_exact_solver_weak_shock_limit(eps):
    """As the pressure jump P_L/P_R = 1 + eps vanishes the solution becomes
    linear acoustics of the e = 3P gas: the plateau moves at
    u* = (P_L - P_R)/(2 w c_s) (impedance w c_s, w = e + P = 4P), the
    rarefaction head at -c_s, and the shock at the mean of the characteristic
    speeds ahead (c_s) and behind ((u* + c_s)/(1 + u* c_s)), i.e.
    c_s + u*/3 = c_s (1 + eps/8) to first order."""
    cs = 1.0 / np.sqrt(3.0)
    PL = 1.0 + eps
    s = R.solve(PL, 0.0, 1.0, 1.0, 0.0, 1.0)
    w = 4.0 * (1.0 + eps / 2.0)
    assert s.vstar == pytest.approx((PL - 1.0) / (2.0 * w * cs), rel=100 * eps ** 2)
    assert s.left_speeds[0] == pytest.approx(-cs, rel=1e-12)
    assert (s.right_speeds[0] / cs - 1.0) / eps == pytest.approx(1.0 / 8.0, rel=0.01)
