"""Pins of the oracle's full time step (Eq. 57 with the h equation of Eq. 58).

Invariants and closed forms the paper fixes: a uniform boosted state stays
uniform; on a periodic grid with one relaxation time the totals of N^0 and
T^{0 mu} are conserved; the step commutes with rotations of the axes and with
mirror reflections of the lattice; a uniform non-equilibrium state relaxes
geometrically with the implicit factor 1/(1 + omega), omega = c0 nu dt /(c_t
tau); the bulk term adds (c0 nu dt / c_t) alpha dx Laplacian(f_i) / (1 + omega)
to every moving population and nothing to the rest population; tau follows
Eq. 41 with the entropy of Sec. III.
"""
import math

import numpy as np
import pytest

from paper_1302_1125_gb300 import workloads as W

NU = math.sqrt(13.0)
C0_CT = NU / math.sqrt(27.0)        # c_0/c_t (Eq. 46)


def params_from(orc, w):
    return orc.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi,
                      dt=w.dt_over_dx, eta_over_s=w.eta_over_s, zeta_over_s=w.zeta_over_s,
                      tau_override=w.tau_override, alpha_override=w.alpha_override,
                      inlet_n=w.inlet[0], inlet_T=w.inlet[1], inlet_u=tuple(w.inlet[2]),
                      euler_mode=w.euler_mode)


def totals(orc, s):
    _, c, _, _, xi0 = orc.lattice()
    N = s.p.N
    f = s.f.reshape(19, N)
    h = s.h.reshape(19, N)
    E = xi0 * xi0 * f.sum()
    M = xi0 * (c.T @ f.sum(1))
    return np.r_[E, M, xi0 * h.sum()]


@pytest.mark.parametrize("euler", [0, 1])
def test_uniform_boosted_state_stays_uniform(orc, euler):
    N = 6 * 5 * 4
    p = orc.Params(nx=6, ny=5, nz=4, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=0.15,
                   eta_over_s=0.1, zeta_over_s=0.02, euler_mode=euler)
    b = math.sqrt(0.99)                 # gamma = 10
    d = np.array([0.6, -0.48, 0.64])    # unit vector
    s = orc.init(p, np.full(N, 0.7), np.full(N, 1.3), b * d[0], b * d[1], b * d[2])
    orc.step(s, 40)
    m = orc.macroscopic(s)
    assert s.nonphysical == 0
    assert np.allclose(m[0], 0.7, rtol=1e-12)
    assert np.allclose(m[1], 3 * 0.7 * 1.3, rtol=1e-12)
    for a in range(3):
        assert np.allclose(m[2 + a], b * d[a], rtol=0, atol=1e-12)
    assert np.allclose(m[5], 10.0, rtol=1e-11)


@pytest.mark.parametrize("dims,euler", [((24, 1, 1), 0), ((10, 9, 1), 0), ((7, 6, 5), 0),
                                         ((10, 9, 1), 1)])
def test_conservation_on_periodic_grid(orc, dims, euler):
    w = W.periodic_box(*dims, seed=4, tau_override=0.7, alpha_override=0.15)
    p = params_from(orc, w)
    p.euler_mode = euler
    s = orc.init(p, *w.fields())
    t0 = totals(orc, s)
    orc.step(s, 120)
    assert s.nonphysical == 0
    t1 = totals(orc, s)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * t0[0] + 1e-13 * np.abs(t0))


def _perm_fields(fields, shape, perm):
    """permute axes of (n, T, ux, uy, uz) fields; perm maps new axis k <- old perm[k]"""
    nz, ny, nx = shape
    arrs = [a.reshape(nz, ny, nx) for a in fields]
    # array axes are (z, y, x) = lattice axes (2, 1, 0)
    ax = [2 - perm[2 - k] for k in range(3)]
    tr = [np.ascontiguousarray(np.transpose(a, ax)) for a in arrs]
    u = [tr[2], tr[3], tr[4]]
    return [tr[0], tr[1], u[perm[0]], u[perm[1]], u[perm[2]]]


def test_step_commutes_with_axis_rotation(orc):
    w = W.periodic_box(6, 7, 8, seed=5, tau_override=0.0, alpha_override=0.1)
    w.eta_over_s = 0.2
    fields = w.fields()
    p = params_from(orc, w)
    s = orc.init(p, *fields)
    orc.step(s, 6)
    m = orc.macroscopic(s).reshape(6, 8, 7, 6)
    perm = (1, 2, 0)                    # new x = old y, new y = old z, new z = old x
    pf = [a.reshape(-1) for a in _perm_fields(fields, (8, 7, 6), perm)]
    q = params_from(orc, w)
    q.nx, q.ny, q.nz = 7, 8, 6
    s2 = orc.init(q, *pf)
    orc.step(s2, 6)
    m2 = orc.macroscopic(s2)
    expect = [a.reshape(-1) for a in _perm_fields([m[0], m[1], m[2], m[3], m[4]], (8, 7, 6), perm)]
    for a, b in zip(expect, m2[:5]):
        assert np.allclose(a, b, rtol=0, atol=1e-12 * np.abs(a).max())


def test_step_commutes_with_mirror_reflection(orc):
    w = W.tube_800(steps=0)
    w.nx = 64
    w.make_fields = lambda: W._tube_fields(64, 1, 1, (3.0, 2.0, 0.3), (1.0, 1.0, -0.2), x0=40)
    p = params_from(orc, w)
    n, T, ux, uy, uz = w.fields()
    s = orc.init(p, n, T, ux, uy, uz)
    orc.step(s, 30)
    m = orc.macroscopic(s)
    s2 = orc.init(p, n[::-1].copy(), T[::-1].copy(), -ux[::-1], uy, uz)
    orc.step(s2, 30)
    m2 = orc.macroscopic(s2)
    assert np.allclose(m[0], m2[0][::-1], rtol=1e-12)
    assert np.allclose(m[2], -m2[2][::-1], rtol=0, atol=1e-12)


def test_implicit_relaxation_of_a_uniform_state(orc):
    # Uniform periodic state f = f^eq + delta with delta orthogonal to the
    # collision invariants: streaming and the Laplacian vanish, f^eq stays
    # fixed, and Eq. 57 gives delta_{t+1} = delta_t / (1 + omega).
    N = 4
    tau, dt = 0.9, 0.25
    p = orc.Params(nx=N, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, tau_override=tau,
                   alpha_override=0.2)
    _, c, _, _, xi0 = orc.lattice()
    s = orc.init(p, np.full(N, 1.0), np.full(N, 1.0), 0.3, 0.0, 0.0)
    f0 = s.f.reshape(19, N)[:, 0].copy()
    A = np.column_stack([np.ones(19), c])           # span of the invariants 1, c_a
    delta = np.random.default_rng(0).normal(size=19) * 1e-3
    delta -= A @ np.linalg.lstsq(A, delta, rcond=None)[0]
    s.f = (s.f.reshape(19, N) + delta[:, None]).reshape(-1).copy()
    omega = C0_CT * NU * dt / tau
    for k in range(1, 6):
        orc.step(s, 1)
        d = s.f.reshape(19, N)[:, 0] - f0
        assert np.allclose(d, delta / (1 + omega) ** k, rtol=1e-9, atol=1e-15)


def test_bulk_term_closed_form(orc):
    # Two runs that differ only in alpha: the difference after one step is
    # (c0 nu dt/c_t) alpha dx Lap(f_i) / (1 + omega) for i != 0 and zero for i = 0.
    N, dt, tau, alpha = 16, 0.2, 0.8, 0.3
    x = np.arange(N)
    mk = lambda a: orc.Params(nx=N, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, tau_override=tau,
                              alpha_override=a)
    sA, sB = (orc.init(mk(a), np.full(N, 1.0), np.full(N, 1.0), 0.2, 0, 0) for a in (alpha, 0.0))
    pert = 1e-3 * np.sin(2 * np.pi * 2 * x / N)
    for s in (sA, sB):
        f = s.f.reshape(19, N).copy()
        f[0] += pert
        f[7] += pert
        s.f = f.reshape(-1).copy()
    orc.step(sA, 1)
    orc.step(sB, 1)
    diff = (sA.f - sB.f).reshape(19, N)
    omega = C0_CT * NU * dt / tau
    lap = -4 * np.sin(np.pi * 2 / N) ** 2 * pert
    expect = C0_CT * NU * dt * alpha * lap / (1 + omega)
    assert np.allclose(diff[7], expect, rtol=1e-8, atol=1e-18)
    assert np.all(np.abs(np.delete(diff, 7, axis=0)) < 1e-17)


def test_extrapolated_equilibrium(orc):
    # a uniform equilibrium whose previous level differs: Eq. 57 gives
    # f(t+dt) = f^eq(t) + omega (f^eq(t) - f^eq(t - dt)) / (1 + omega)
    N, dt, tau = 3, 0.25, 0.7
    p = orc.Params(nx=N, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, tau_override=tau,
                   alpha_override=0.0)
    s = orc.init(p, np.full(N, 1.0), np.full(N, 2.0), 0.1, 0.0, 0.0)
    prev = s.prev.reshape(5, N)
    prev[0] = 1.5
    prev[1] = 0.4
    s.prev = prev.reshape(-1).copy()
    g = 1 / math.sqrt(1 - 0.01)
    fe = orc.feq(2.0, [g * 0.1, 0, 0])
    fp = orc.feq(1.5, [0.4, 0, 0])
    omega = C0_CT * NU * dt / tau
    orc.step(s, 1)
    assert np.allclose(s.f.reshape(19, N)[:, 1], fe + omega * (fe - fp) / (1 + omega),
                       rtol=1e-12, atol=1e-15)


def test_tau_from_eta_over_s(orc):
    # Eq. 41: eta = (e + P)(tau - 1/2)/nu^2 = 4 P (tau - 1/2)/13; eta = (eta/s) s,
    # s = n (4 - ln lambda), lambda = n / n_eq, n_eq = 16 T^3 / pi^2 (Sec. III)
    p = orc.Params(nx=1, eta_over_s=0.1)
    neq = lambda T: 16 * T ** 3 / math.pi ** 2
    assert abs(orc.tau(p, neq(1.0) * 1.0, neq(1.0)) - 1.8) < 1e-14          # T = 1, lambda = 1
    assert abs(orc.tau(p, neq(2.0) * 2.0, neq(2.0)) - 1.15) < 1e-14         # T = 2
    n = math.e * neq(1.0)                                                    # lambda = e
    assert abs(orc.tau(p, n * 1.0, n) - (0.5 + 13 * 0.1 * 3.0 / 4.0)) < 1e-14
    n = math.exp(5.0) * neq(1.0)                                             # R7 floor
    assert abs(orc.tau(p, n * 1.0, n) - (0.5 + 13 * 0.1 * 1e-3 / 4.0)) < 1e-14
    p.tau_override = 0.77
    assert orc.tau(p, 1.0, 1.0) == 0.77


def test_alpha_from_zeta_over_s(orc):
    # Eq. 56 at the reference state T = 1, lambda = 1: alpha = 27 (zeta/s) / nu^6
    assert abs(orc.alpha(orc.Params(nx=1, zeta_over_s=0.01)) - 0.27 / 13 ** 3) < 1e-17
    assert orc.alpha(orc.Params(nx=1, zeta_over_s=0.0)) == 0.0
    assert orc.alpha(orc.Params(nx=1, zeta_over_s=0.3, alpha_override=0.15)) == 0.15


def test_non_physical_cells_are_counted(orc):
    N = 8
    p = orc.Params(nx=N, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0))
    s = orc.init(p, np.full(N, 1.0), np.full(N, 1.0), 0.0, 0.0, 0.0)
    f = s.f.reshape(19, N).copy()
    f[1, 3] += 50.0       # E < |M| at cell 3
    f[0, 3] -= 50.0
    s.f = f.reshape(-1).copy()
    orc.step(s, 1)
    assert s.nonphysical >= 1


def test_step_cells_matches_the_full_step(orc):
    w = W.shock_cloud(24, 16, 8, 3.0, (8.0, 8.0, 4.0), zeta_over_s=0.01, precision=0)
    p = params_from(orc, w)
    s = orc.init(p, *w.fields())
    orc.step(s, 2)
    f0, h0, pv0 = s.f.copy(), s.h.copy(), s.prev.copy()
    orc.step(s, 1)
    cells = np.array([0, 1, 23, 24 * 16 - 1, 5 + 24 * (3 + 16 * 7), p.N - 1])
    fo, ho, mo, bad = orc.step_cells(p, f0, h0, pv0, cells)
    assert bad == 0
    assert np.array_equal(fo, s.f.reshape(19, -1)[:, cells].T)
    assert np.array_equal(ho, s.h.reshape(19, -1)[:, cells].T)
    assert np.array_equal(mo, s.prev.reshape(5, -1)[:, cells].T)
    # float32 input path reads the same values
    fo32, _, _, _ = orc.step_cells(p, f0.astype(np.float32), h0.astype(np.float32),
                                   pv0.astype(np.float32), cells)
    assert np.allclose(fo32, fo, rtol=1e-5, atol=1e-6 * np.abs(fo).max())
