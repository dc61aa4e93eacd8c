"""Pins of the oracle's step by the hydrodynamics it must reproduce and by
statements of Sec. II.B and Sec. III, not by its own formulas:

* Linear acoustics of the e = 3P gas: a small pressure pulse splits into two
  halves that move at the speed of sound c_s = 1/sqrt(3) (c_s^2 = dP/de), and
  in each half the flow velocity is u = +-c_s de / (e + P) =
  +-(sqrt(3)/4) dP / P0 (the acoustic impedance).  Euler mode and a
  low-viscosity run.
* The number distribution h follows Eq. 57 without the lambda_i (bulk)
  term (Sec. II.B): after one viscous step h does not depend on alpha,
  while f does.
* An inlet face holding the gas's own state (Sec. III) is invisible: a
  uniform moving state next to it stays uniform.
* Shear viscosity: the Chapman-Enskog expansion of the continuum limit of
  Eq. 57, df_i/dt + (c0/c_t) c_i . grad f_i = -(c0 nu/(c_t tau)) (f_i - f^eq_i),
  gives for a transverse shear wave the momentum flux
  -(c0/c_t)^2 tau_R xi0 sum_i c_x^2 c_y df^eq_i/dx with tau_R = c_t tau/(c0 nu),
  so with the first-order coefficient 4 P gamma/(xi0 sigma2) of f^eq the shear
  viscosity is eta = (c0/c_t) tau 4 P m22 / (nu sigma2), sigma2 = sum w c_x^2,
  m22 = sum w c_x^2 c_y^2: 0.2369 P tau on the extended lattice, 0.1621 P tau
  on the basic one, with no dependence on dt.  A shear wave's decay rate
  eta k^2/(e + P) matches it on both lattices.
* The lambda_i term of Eq. 55 diffuses every moving population with the
  same coefficient per unit time, D = (c0/c_t) nu alpha dx, and the rest
  population not at all; momentum lives on the moving populations only, so
  it diffuses with D and a shear wave decays at (eta/(e + P) + D) k^2.
* Particle diffusion: a density wave at uniform pressure and rest leaves f
  uniform, and the same expansion for h (first-order part
  -tau_R (c0/c_t) c_i . grad h^eq_i, h^eq_i = w'_i n c0/c_t at rest, and
  N^x = sum c_x h with xi0 c0/c_t = 1) gives the diffusion coefficient
  tau_R (c0/c_t)^2 sum w' c_x^2 = tau/(3 sqrt(27)) on both lattices, with
  no lambda_i term (Sec. II.B): the result does not depend on alpha.
* Anisotropy: sum_i w_i c_a c_b c_c c_d is cubic, not isotropic, on these
  lattices (m4 != 3 m22), so the shear viscosity depends on direction: a
  shear wave with k along (1, 1, 0) and u along (1, -1, 0) sees
  eta (1 + (m4 - 3 m22)/(2 m22)), 1.875 eta on both lattices.  Particle
  diffusion needs only sum w' c_a c_b = delta_ab/3 and is isotropic: a
  density wave along (1, 1, 0) diffuses at the rate of one along x.
* Euler mode (Sec. III: f and h set to the equilibria of the streamed state
  every step) carries no viscosity of its own: a shear wave decays only
  through the limiter's numerical viscosity, which does not depend on dt,
  halves when the resolution doubles and is far below the viscous mode's.
* Sound attenuation: the longitudinal stress of the same expansion,
  -tau_R (d/dt sum c_x^2 f^eq + (c0/c_t) d/dx sum c_x^3 f^eq), with
  dP/dt = -(e + P) du/dx / 3, gives eta_L = tau_R 4 P ((c0/c_t)^2 m4/sigma2 - 1/3),
  m4 = sum w c_x^4 (for massless particles in the continuum this is
  4 eta/3; on these lattices 1.875 times that).  A standing sound wave decays at
  eta_L k^2 / (2 (e + P)) in the limit dt -> 0; the time scheme takes away
  damping as dt grows.
"""
import math

import numpy as np
import pytest

CS = 1.0 / math.sqrt(3.0)
D_G = 16.0


def n_eq(T):
    return D_G * np.asarray(T) ** 3 / math.pi ** 2


@pytest.mark.parametrize("euler,eta,tol", [(1, 0.0, 0.1), (0, 0.01, 0.5)])
def test_sound_pulse(orc, euler, eta, tol):
    nx, x0, sig, amp, dt, steps = 600, 300.0, 8.0, 1e-3, 0.25, 480
    x = np.arange(nx)
    T = (1.0 + amp * np.exp(-(x - x0) ** 2 / (2 * sig ** 2))) ** 0.25   # P = n_eq(T) T: dP/P0 = amp
    z = np.zeros(nx)
    p = orc.Params(nx=nx, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, eta_over_s=eta,
                   alpha_override=0.0, euler_mode=euler)
    s = orc.init(p, n_eq(T), T, z, z, z)
    P0 = float(n_eq(1.0))
    orc.step(s, steps)
    assert s.nonphysical == 0
    m = orc.macroscopic(s)
    dP = m[1] / 3.0 - P0
    u = m[2]
    t = steps * dt
    for side, sign in ((x > x0, 1.0), (x < x0, -1.0)):
        centroid = (x[side] * dP[side]).sum() / dP[side].sum()
        assert abs(centroid - (x0 + sign * CS * t)) < tol, (centroid, x0 + sign * CS * t)
        ratio = (u[side] * dP[side]).sum() / (dP[side] ** 2).sum()
        assert ratio == pytest.approx(sign * math.sqrt(3.0) / (4.0 * P0), rel=5e-3)
    # each half carries half the pulse and the peak has split
    assert dP[x > x0].sum() == pytest.approx(dP[x < x0].sum(), rel=1e-9)
    assert dP.max() < 0.55 * amp * P0


def test_number_distribution_has_no_bulk_term(orc):
    from paper_1302_1125_gb300 import workloads as W
    w = W.periodic_box(7, 6, 5, seed=11, amp=0.3)
    out = {}
    for alpha in (0.0, 0.3):
        p = orc.Params(nx=w.nx, ny=w.ny, nz=w.nz, bc_lo=w.bc_lo, bc_hi=w.bc_hi, dt=0.2,
                       tau_override=0.8, alpha_override=alpha)
        s = orc.init(p, *w.fields())
        orc.step(s, 1)
        out[alpha] = (s.f.copy(), s.h.copy())
    assert np.array_equal(out[0.0][1], out[0.3][1])
    df = np.abs(out[0.0][0] - out[0.3][0]).reshape(19, -1)
    assert np.all(df[0] == 0.0)             # lambda_0 = 0
    assert df[1:].max() > 1e-4 * np.abs(out[0.0][0]).max()


@pytest.mark.parametrize("dims,u", [((40, 1, 1), (0.4, 0.0, 0.0)), ((24, 6, 1), (0.35, 0.2, 0.0)),
                                    ((40, 1, 1), (-0.3, 0.0, 0.0))])
def test_inlet_at_the_gas_state_is_invisible(orc, dims, u):
    nx, ny, nz = dims
    N = nx * ny * nz
    n, T = 0.8, 1.7
    p = orc.Params(nx=nx, ny=ny, nz=nz, bc_lo=(2, 0, 0), bc_hi=(1, 0, 0), dt=0.15, eta_over_s=0.05,
                   alpha_override=0.2, inlet_n=n, inlet_T=T, inlet_u=u)
    s = orc.init(p, np.full(N, n), np.full(N, T), np.full(N, u[0]), np.full(N, u[1]), np.full(N, u[2]))
    f0, h0 = s.f.copy(), s.h.copy()
    orc.step(s, 30)
    assert np.allclose(s.f, f0, rtol=0, atol=1e-13 * np.abs(f0).max())
    assert np.allclose(s.h, h0, rtol=0, atol=1e-13 * np.abs(h0).max())
    # a different inlet state does reach the gas
    p.inlet_T = 1.0
    s = orc.init(p, np.full(N, n), np.full(N, T), np.full(N, u[0]), np.full(N, u[1]), np.full(N, u[2]))
    orc.step(s, 5)
    assert np.abs(s.f - f0).max() > 1e-3 * np.abs(f0).max()


@pytest.mark.parametrize("model,tol", [(0, 0.01), (1, 0.025)])
@pytest.mark.parametrize("tau", [1.0, 3.0])
def test_shear_wave_decays_at_the_chapman_enskog_viscosity(orc, model, tol, tau):
    e, c, w, wh, xi0 = orc.lattice(model)
    sigma2 = float((w * c[:, 0] ** 2).sum())
    m22 = float((w * c[:, 0] ** 2 * c[:, 1] ** 2).sum())
    nu = orc.nu(model)
    c0_ct = nu / math.sqrt(27.0)                  # Eq. 46 (c_t/c_0 = sqrt(27)/nu)
    eta_per_Ptau = c0_ct * 4.0 * m22 / (nu * sigma2)
    assert eta_per_Ptau == pytest.approx({0: 0.23686, 1: 0.16206}[model], abs=1e-5)
    nx, A = 256, 1e-4
    x = np.arange(nx)
    k = 2 * math.pi / nx
    mode = np.sin(k * (x + 0.5))
    T = np.ones(nx)
    n = n_eq(T)
    P0 = float(n[0])
    z = np.zeros(nx)
    etas = []
    for dt in (0.25, 0.1):
        p = orc.Params(nx=nx, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, tau_override=tau,
                       alpha_override=0.0, model=model)
        s = orc.init(p, n, T, z, A * mode, z)
        steps = int(round(nx / (dt * tau)))        # about 1 % decay
        amp = []
        # the first quarter lets the viscous stress build up (over ~tau_R)
        for k_steps in (steps // 4, steps - steps // 4):
            orc.step(s, k_steps)
            m = orc.macroscopic(s)
            amp.append(2.0 / nx * float((m[3] * mode).sum()))
        rate = math.log(amp[0] / amp[1]) / ((steps - steps // 4) * dt)
        eta = rate * 4.0 * P0 / k ** 2              # e + P = 4 P
        assert eta / (P0 * tau) == pytest.approx(eta_per_Ptau, rel=tol), (dt, eta / (P0 * tau))
        assert np.abs(m[2]).max() < 1e-3 * A and np.abs(m[4]).max() == 0.0
        etas.append(eta)
    assert etas[0] == pytest.approx(etas[1], rel=1e-3)     # no dependence on dt


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("tau,alpha", [(1.0, 0.2), (2.0, 0.05)])
def test_bulk_term_diffuses_momentum(orc, model, tau, alpha):
    e, c, w, wh, xi0 = orc.lattice(model)
    sigma2 = float((w * c[:, 0] ** 2).sum())
    m22 = float((w * c[:, 0] ** 2 * c[:, 1] ** 2).sum())
    nu = orc.nu(model)
    c0_ct = nu / math.sqrt(27.0)
    eta_over_w = c0_ct * 4.0 * m22 / (nu * sigma2) * tau / 4.0     # eta/(e + P), e + P = 4 P
    D = c0_ct * nu * alpha                                          # dx = 1
    nx, A, dt = 256, 1e-4, 0.25
    x = np.arange(nx)
    k = 2 * math.pi / nx
    mode = np.sin(k * (x + 0.5))
    T = np.ones(nx)
    z = np.zeros(nx)
    p = orc.Params(nx=nx, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, tau_override=tau,
                   alpha_override=alpha, model=model)
    s = orc.init(p, n_eq(T), T, z, A * mode, z)
    steps = int(round(0.01 / ((eta_over_w + D) * k * k * dt)))      # about 1 % decay
    amp = []
    for k_steps in (steps // 4, steps - steps // 4):
        orc.step(s, k_steps)
        amp.append(2.0 / nx * float((orc.macroscopic(s)[3] * mode).sum()))
    rate = math.log(amp[0] / amp[1]) / ((steps - steps // 4) * dt)
    assert rate == pytest.approx((eta_over_w + D) * k * k, rel=5e-3)
    assert D / (eta_over_w + D) > 0.5          # the lambda term dominates here


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("tau", [1.0, 2.0])
def test_density_wave_diffuses_at_the_chapman_enskog_rate(orc, model, tau):
    e, c, w, wh, xi0 = orc.lattice(model)
    nu = orc.nu(model)
    c0_ct = nu / math.sqrt(27.0)
    assert xi0 * c0_ct == pytest.approx(1.0, rel=1e-14)
    tau_R = tau / (c0_ct * nu)
    kappa = tau_R * c0_ct ** 2 * float((wh * c[:, 0] ** 2).sum())
    assert kappa == pytest.approx(tau / (3.0 * math.sqrt(27.0)), rel=1e-12)
    nx, A, dt = 256, 1e-3, 0.25
    x = np.arange(nx)
    k = 2 * math.pi / nx
    mode = np.sin(k * (x + 0.5))
    n0 = float(n_eq(1.0))
    n = n0 * (1.0 + A * mode)
    T = n0 / n                                   # P = n T uniform
    z = np.zeros(nx)
    steps = int(round(0.01 / (kappa * k * k * dt)))
    dens = {}
    for alpha in (0.0, 0.2):
        p = orc.Params(nx=nx, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, tau_override=tau,
                       alpha_override=alpha, model=model)
        s = orc.init(p, n, T, z, z, z)
        amp = []
        for k_steps in (steps // 4, steps - steps // 4):
            orc.step(s, k_steps)
            m = orc.macroscopic(s)
            amp.append(2.0 / nx * float(((m[0] / n0 - 1.0) * mode).sum()))
        dens[alpha] = m[0].copy()
        rate = math.log(amp[0] / amp[1]) / ((steps - steps // 4) * dt)
        assert rate == pytest.approx(kappa * k * k, rel=0.03)
        assert np.abs(m[2]).max() < 1e-12            # the gas stays at rest
    # f is uniform up to the rounding of n T, so alpha reaches n only at that level
    assert np.abs(dens[0.0] - dens[0.2]).max() < 1e-12 * n0


def _sound_decay(orc, model, tau, nx, dt, periods=6, alpha=0.0):
    """fitted (decay rate, angular frequency) of a standing sound wave"""
    from scipy.optimize import curve_fit
    P0 = float(n_eq(1.0))
    A = 1e-4
    x = np.arange(nx)
    k = 2 * math.pi / nx
    mode = np.sin(k * (x + 0.5))
    T = (1.0 + A * mode) ** 0.25
    z = np.zeros(nx)
    p = orc.Params(nx=nx, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, tau_override=tau,
                   alpha_override=alpha, model=model)
    s = orc.init(p, n_eq(T), T, z, z, z)
    om = CS * k
    total = int(periods * 2 * math.pi / om / dt)
    blk = max(total // 150, 1)
    ts, amp = [], []
    for i in range(total // blk):
        orc.step(s, blk)
        m = orc.macroscopic(s)
        ts.append((i + 1) * blk * dt)
        amp.append(2.0 / nx * float(((m[1] - 3.0 * P0) * mode).sum()) / (3.0 * P0 * A))
    f = lambda t, a, g, o, ph: a * np.exp(-g * t) * np.cos(o * t + ph)
    (a, g, o, ph), _ = curve_fit(f, np.array(ts), np.array(amp), p0=(1.0, 1e-3, om, 0.0))
    return g, o


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("tau,tol", [(1.0, 0.06), (2.0, 0.04)])
def test_sound_wave_decays_at_the_longitudinal_viscosity(orc, model, tau, tol):
    pytest.importorskip("scipy")
    e, c, w, wh, xi0 = orc.lattice(model)
    sigma2 = float((w * c[:, 0] ** 2).sum())
    m4 = float((w * c[:, 0] ** 4).sum())
    m22 = float((w * c[:, 0] ** 2 * c[:, 1] ** 2).sum())
    nu = orc.nu(model)
    c0_ct = nu / math.sqrt(27.0)
    tau_R = tau / (c0_ct * nu)
    P0 = float(n_eq(1.0))
    eta_L = tau_R * 4.0 * P0 * (c0_ct ** 2 * m4 / sigma2 - 1.0 / 3.0)
    eta = tau_R * 4.0 * P0 * c0_ct ** 2 * m22 / sigma2
    assert eta_L / (4.0 * eta / 3.0) == pytest.approx(1.875, rel=1e-12)
    nx = 64
    k = 2 * math.pi / nx
    g, om = _sound_decay(orc, model, tau, nx, 0.05)
    assert g == pytest.approx(eta_L * k * k / (2.0 * 4.0 * P0), rel=tol)
    assert om == pytest.approx(CS * k, rel=3e-3)
    # the time scheme takes damping away as dt grows
    g25, _ = _sound_decay(orc, model, tau, nx, 0.25)
    assert g25 < 0.75 * g


def _shear_rate_2d(orc, model, L, diagonal, tau=1.0, frac=0.05, guess=1.0):
    """fitted decay rate of a 2-D shear wave along x or along (1, 1)"""
    yy, xx = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    A = 1e-4
    if diagonal:
        ph = 2 * math.pi * (xx + yy + 1.0) / L
        k2 = 2 * (2 * math.pi / L) ** 2
        ux = A * np.sin(ph) / math.sqrt(2.0)
        uy = -ux
    else:
        ph = 2 * math.pi * (xx + 0.5) / L
        k2 = (2 * math.pi / L) ** 2
        ux = np.zeros((L, L))
        uy = A * np.sin(ph)
    N = L * L
    T = np.ones(N)
    p = orc.Params(nx=L, ny=L, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=0.25, tau_override=tau,
                   alpha_override=0.0, model=model)
    s = orc.init(p, n_eq(T), T, ux.reshape(-1), uy.reshape(-1), np.zeros(N))
    steps = int(round(frac / (guess * k2 * 0.25)))
    skip = max(steps // 4, 16)                   # the viscous stress builds up over ~tau_R
    amp = []
    for k_steps in (skip, steps):
        orc.step(s, k_steps)
        m = orc.macroscopic(s)
        v = (m[2] - m[3]) / math.sqrt(2.0) if diagonal else m[3]
        amp.append(2.0 / N * float((v.reshape(L, L) * np.sin(ph)).sum()))
    return math.log(amp[0] / amp[1]) / (steps * 0.25)


@pytest.mark.parametrize("model,L,tol", [(0, 64, 0.06), (1, 64, 0.06)])
def test_shear_viscosity_is_anisotropic(orc, model, L, tol):
    e, c, w, wh, xi0 = orc.lattice(model)
    m4 = float((w * c[:, 0] ** 4).sum())
    m22 = float((w * c[:, 0] ** 2 * c[:, 1] ** 2).sum())
    factor = 1.0 + (m4 - 3.0 * m22) / (2.0 * m22)
    assert factor == pytest.approx(1.875, rel=1e-12)
    g_axis = _shear_rate_2d(orc, model, L, False, guess=0.06)
    g_diag = _shear_rate_2d(orc, model, L, True, guess=0.11)
    # both waves have |k| chosen so that the ratio of rates is the ratio of viscosities x 2
    assert g_diag / (2.0 * g_axis) == pytest.approx(factor, rel=tol)


@pytest.mark.parametrize("model", [0, 1])
def test_euler_mode_is_inviscid_up_to_the_limiter(orc, model):
    A = 1e-4
    etas = {}
    for nx, dt in ((128, 0.25), (256, 0.25), (128, 0.1)):
        x = np.arange(nx)
        k = 2 * math.pi / nx
        mode = np.sin(k * (x + 0.5))
        T = np.ones(nx)
        z = np.zeros(nx)
        p = orc.Params(nx=nx, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, alpha_override=0.0,
                       euler_mode=1, model=model)
        s = orc.init(p, n_eq(T), T, z, A * mode, z)
        steps = int(round(0.5 * nx * nx / (dt * 256)))
        amp = []
        for k_steps in (16, steps):
            orc.step(s, k_steps)
            amp.append(2.0 / nx * float((orc.macroscopic(s)[3] * mode).sum()))
        rate = math.log(amp[0] / amp[1]) / (steps * dt)
        etas[nx, dt] = rate * 4.0 * float(n_eq(1.0)) / k ** 2
    P0 = float(n_eq(1.0))
    viscous = 0.2369 * P0 * 1.0 if model == 0 else 0.1621 * P0 * 1.0     # tau = 1
    assert 0.0 < etas[256, 0.25] < 0.03 * viscous
    assert 0.4 < etas[256, 0.25] / etas[128, 0.25] < 0.6                 # first order in dx
    assert etas[128, 0.1] == pytest.approx(etas[128, 0.25], rel=0.05)    # no dependence on dt


def _density_rate_2d(orc, model, L, diagonal, tau=1.0, dt=0.25):
    """fitted decay rate of a 2-D density wave at uniform pressure, along x or (1, 1)"""
    yy, xx = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    ph = 2 * math.pi * ((xx + yy + 1.0) if diagonal else (xx + 0.5)) / L
    k2 = (2 if diagonal else 1) * (2 * math.pi / L) ** 2
    n0 = float(n_eq(1.0))
    n = n0 * (1.0 + 1e-3 * np.sin(ph)).reshape(-1)
    N = L * L
    z = np.zeros(N)
    p = orc.Params(nx=L, ny=L, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0), dt=dt, tau_override=tau,
                   alpha_override=0.0, model=model)
    s = orc.init(p, n, n0 / n, z, z, z)
    steps = int(round(0.03 / (tau / (3 * math.sqrt(27.0)) * k2 * dt)))
    amp = []
    for k_steps in (max(steps // 4, 16), steps):
        orc.step(s, k_steps)
        m = orc.macroscopic(s)
        amp.append(2.0 / N * float(((m[0] / n0 - 1.0).reshape(L, L) * np.sin(ph)).sum()))
    return math.log(amp[0] / amp[1]) / (steps * dt) / k2


@pytest.mark.parametrize("model", [0, 1])
def test_particle_diffusion_is_isotropic(orc, model):
    axis = _density_rate_2d(orc, model, 64, False)
    diag = _density_rate_2d(orc, model, 64, True)
    assert diag == pytest.approx(axis, rel=0.01)
    assert axis == pytest.approx(1.0 / (3 * math.sqrt(27.0)), rel=0.1)     # tau = 1


@pytest.mark.parametrize("alpha", [0.05, 0.2])
def test_bulk_term_is_not_the_bulk_viscosity_of_eq56(orc, alpha):
    """The lambda_i term (Eqs. 54-55) adds sound damping in proportion to
    alpha, whatever dt, but about 12 times less than the bulk viscosity
    Eq. 56 assigns to it, eta_b = 4 P alpha nu^6 / 27, would (a standing
    sound wave decays at (4 eta / 3 + zeta) k^2 / (2 (e + P)), e + P = 4 P):
    Eq. 56 does not describe the lattice term, so the map zeta/s -> alpha
    built on it (R4) gives alpha ~ 1e-3 for zeta/s ~ 0.1, which does
    nothing the measurements can see; the workloads give alpha directly, as
    the paper's runs do."""
    pytest.importorskip("scipy")
    nx = 64
    k = 2 * math.pi / nx
    nu = orc.nu(0)
    added = []
    for dt in (0.05, 0.1):
        g0, _ = _sound_decay(orc, 0, 1.0, nx, dt)
        g1, _ = _sound_decay(orc, 0, 1.0, nx, dt, alpha=alpha)
        added.append(g1 - g0)
    assert added[0] == pytest.approx(added[1], rel=0.01)          # independent of dt
    eq56 = (4.0 * alpha * nu ** 6 / 27.0) * k * k / (2.0 * 4.0)    # per unit P
    assert 10.0 < eq56 / added[0] < 14.0, eq56 / added[0]
    # in units of the term's momentum diffusivity D = (c0/c_t) nu alpha dx
    D = nu * alpha / orc.lattice(0)[4]
    assert 2.6 < added[0] / (D * k * k / 2.0) < 2.95
