"""Pins of the oracle's basic model (Sec. II before the extension: the D3Q19
lattice with unit diagonals; readings R13 and R14).

* Constants from the printed formulas of the basic quadrature: with
  c_a = sqrt(19)/nu and nu = sqrt(19), the weights are the rationals
  -44/361, 99/722, 9/361 and (c_t/c_0)^2 = 27/19.
* The equilibrium reproduces the energy-momentum tensor of Eq. 36 on this
  lattice (brute-force 4x4 sums) and the rest-frame equation of state.
* The number distribution carries N^0 = n gamma and N^a = n gamma u^a.
* The step keeps a uniform boosted state uniform and conserves the totals on
  periodic grids; shock tubes converge in L1 to the exact Riemann solution.
* The paper's own comparison (Sec. III: P ratio 32, beta ~ 0.7, eta/s 0.01,
  dt/dx 0.25): the basic model fails where the extended model (alpha 0.15)
  follows the exact solution; at beta ~ 0.2 the basic model converges but
  overshoots the velocity at the shock, the extended model does not.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import riemann as R
from paper_1302_1125_gb300 import workloads as W

BASIC = 1
ETA = np.diag([1.0, -1.0, -1.0, -1.0])


def test_basic_lattice_constants_follow_the_printed_formulas(orc):
    e, c, w, wh, xi0 = orc.lattice(BASIC)
    assert abs(orc.nu(BASIC) - math.sqrt(19.0)) < 1e-15
    assert abs(xi0 * xi0 - 27.0 / 19.0) < 1e-15
    # weights of the basic quadrature with nu^2 = 19, c_a = 1, (c_t/c_0)^2 = 27/19
    r2, nu2, ca2 = Fraction(27, 19), Fraction(19), Fraction(1)
    w0 = 1 + 4 * r2 * nu2 / 361 - r2 / ca2
    w1 = r2 / (2166 * ca2) * (361 - 8 * ca2 * nu2)
    w2 = r2 * nu2 / 1083
    assert (w0, w1, w2) == (Fraction(-44, 361), Fraction(99, 722), Fraction(9, 361))
    assert np.allclose(w, [float(w0)] + [float(w1)] * 6 + [float(w2)] * 12, rtol=0, atol=1e-15)
    assert abs(w.sum() - 1.0) < 1e-15
    # unit diagonals: every component of every velocity is 0 or +-1
    assert set(np.unique(c)) == {-1.0, 0.0, 1.0}
    assert len({tuple(v) for v in e}) == 19
    assert np.all(np.abs(c).sum(1)[7:] == 2.0)
    assert np.allclose(wh, [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12, rtol=0, atol=1e-16)


def _tensor(orc, f):
    _, c, _, _, xi0 = orc.lattice(BASIC)
    p = np.column_stack([np.full(19, xi0), c])
    return np.einsum("ia,ib,i->ab", p, p, f)


def test_basic_feq_reproduces_energy_momentum_tensor(orc):
    rng = np.random.default_rng(19)
    worst = 0.0
    for _ in range(300):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        beta = rng.uniform(0.0, 0.995)
        g = 1.0 / math.sqrt(1.0 - beta * beta)
        P = rng.uniform(0.05, 5.0)
        up = g * beta * d
        T = _tensor(orc, orc.feq(P, up, BASIC))
        U = np.r_[g, up]
        Teq = 4.0 * P * np.outer(U, U) - P * ETA
        worst = max(worst, np.abs(T - Teq).max() / np.abs(Teq).max())
    assert worst < 1e-13
    # rest frame: e = 3P, isotropic pressure
    Tt = _tensor(orc, orc.feq(0.8, np.zeros(3), BASIC))
    assert np.allclose(np.diag(Tt), [2.4, 0.8, 0.8, 0.8], rtol=1e-13)


def test_basic_heq_particle_current(orc):
    _, c, _, _, xi0 = orc.lattice(BASIC)
    rng = np.random.default_rng(23)
    for _ in range(200):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        beta = rng.uniform(0.0, 0.99)
        g = 1.0 / math.sqrt(1.0 - beta * beta)
        n = rng.uniform(0.05, 5.0)
        h = orc.heq(n, g * beta * d, BASIC)
        assert abs(xi0 * h.sum() - n * g) < 1e-13 * n * g
        assert np.allclose(c.T @ h, n * g * beta * d, rtol=0, atol=1e-13 * n * g)
    mom = orc.moments(orc.feq(1.1, [0.3, -0.2, 0.1], BASIC), orc.heq(0.7, [0.3, -0.2, 0.1], BASIC), BASIC)
    mac, bad = orc.recover(mom, BASIC)
    assert not bad and np.allclose(mac, [1.1, 0.3, -0.2, 0.1, 0.7], rtol=1e-13, atol=1e-14)


def test_basic_uniform_boosted_state_stays_uniform(orc):
    N = 6 * 5 * 4
    p = orc.Params(nx=6, ny=5, nz=4, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=0.25, eta_over_s=0.1,
                   alpha_override=0.0, model=BASIC)
    d = np.array([0.6, -0.48, 0.64])
    s = orc.init(p, np.full(N, 0.7), np.full(N, 1.3), 0.5 * d[0], 0.5 * d[1], 0.5 * d[2])
    orc.step(s, 30)
    m = orc.macroscopic(s)
    assert s.nonphysical == 0
    assert np.allclose(m[0], 0.7, rtol=1e-12) and np.allclose(m[1], 3 * 0.7 * 1.3, rtol=1e-12)
    for a in range(3):
        assert np.allclose(m[2 + a], 0.5 * d[a], rtol=0, atol=1e-12)


@pytest.mark.parametrize("dims", [(24, 1, 1), (7, 6, 5)])
def test_basic_conservation_on_periodic_grid(orc, dims):
    w = W.periodic_box(*dims, seed=9, tau_override=0.7, alpha_override=0.0, gamma_max=1.5)
    p = orc.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt=0.25, tau_override=0.7,
                   alpha_override=0.0, model=BASIC)
    s = orc.init(p, *w.fields())
    _, c, _, _, xi0 = orc.lattice(BASIC)

    def tot():
        f = s.f.reshape(19, -1)
        return np.r_[xi0 * xi0 * f.sum(), xi0 * (c.T @ f.sum(1)), xi0 * s.h.sum()]
    t0 = tot()
    orc.step(s, 100)
    assert s.nonphysical == 0
    t1 = tot()
    assert np.all(np.abs(t1 - t0) <= 1e-13 * t0[0] + 1e-13 * np.abs(t0))


def _tube(orc, model, nx, ratio, alpha, dt=0.25, eta=0.01, frac=0.4):
    w = W.riemann_tube(nx, ratio, 2.0)
    n, T, ux, uy, uz = w.fields()
    p = orc.Params(nx=nx, dt=dt, eta_over_s=eta, alpha_override=alpha, model=model)
    st = orc.init(p, n, T, ux, uy, uz)
    sol = R.solve(n[0] * T[0], 0.0, n[0], n[-1] * T[-1], 0.0, n[-1])
    vmax = max(abs(sol.left_speeds[0]), abs(sol.right_speeds[-1]))
    steps = int(round(frac * nx / vmax / dt))
    done = 0
    while done < steps:
        k = min(50, steps - done)
        orc.step(st, k)
        done += k
        if st.nonphysical:
            return None
    m = orc.macroscopic(st)
    P, v, _ = sol.sample((np.arange(nx) + 0.5 - nx / 2) / (steps * dt))
    l1 = lambda a, b: np.abs(a - b).sum() / np.abs(b).sum()
    return l1(m[1] / 3.0, P), l1(m[2], v), (m[2].max() - v.max()) / v.max()


def test_basic_tube_converges_to_exact_solution(orc):
    errs = [_tube(orc, BASIC, nx, 5.43 / 2.22, 0.0)[:2] for nx in (200, 400, 800)]
    errs = np.array(errs)
    assert np.all(errs[1] < 0.85 * errs[0]) and np.all(errs[2] < 0.85 * errs[1]), errs


def test_paper_basic_versus_extended_comparison(orc):
    # P ratio 32 (5.43 / 0.1695 GeV/fm^3), beta ~ 0.7, eta/s 0.01, dt/dx 0.25;
    # alpha 0.15 for the extended model only, as in the paper
    assert _tube(orc, BASIC, 400, 32.0, 0.0) is None          # the basic model breaks down
    ext = _tube(orc, 0, 400, 32.0, 0.15)
    assert ext is not None and ext[0] < 0.05 and ext[1] < 0.06 and abs(ext[2]) < 0.02
    # at beta ~ 0.2 the basic model runs but overshoots the velocity at the shock
    basic = _tube(orc, BASIC, 400, 5.43 / 2.22, 0.0)
    ext = _tube(orc, 0, 400, 5.43 / 2.22, 0.0)
    assert basic[2] > 0.05 and abs(ext[2]) < 0.01
