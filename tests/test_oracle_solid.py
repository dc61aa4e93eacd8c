"""Pins of the oracle's solid cells (Sec. III, the astrophysical run: a fixed
cloud whose cells are held at the equilibrium of a constant state n1, T1,
u = 0; reading R11: every cell inside the sphere is reset after every step).

* Read-back: after steps of a shock driven into the cloud, the moments of
  every solid cell, recovered through the Landau frame, give back exactly
  n1, e = 3 n1 T1 and u = 0 (the recovery and Eq. 36 are pinned elsewhere),
  while cells next to the cloud have moved away from that state.
* Invisibility: a gas at rest in the cloud's own state stays uniform to
  round-off with the cloud in it (a uniform state at rest is a fixed point of
  the step, and the cloud does not perturb it).
* Geometry: a cloud centred in a y-z periodic box with a shock along x keeps
  the solution mirror symmetric about the cloud's centre planes.
"""
import numpy as np
import pytest

from paper_1302_1125_gb300 import workloads as W


def params(orc, nx, ny, nz, **kw):
    p = orc.Params(nx=nx, ny=ny, nz=nz, bc_lo=(1, 0, 0), bc_hi=(1, 0, 0), dt=0.15, eta_over_s=0.0,
                   zeta_over_s=0.0, tau_override=1.0, alpha_override=0.2)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def sphere_mask(nx, ny, nz, c, R):
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return ((xx - c[0]) ** 2 + (yy - c[1]) ** 2 + (zz - c[2]) ** 2 <= R * R).reshape(-1)


def shocked(nx, ny, nz, x0, nL, TL, nR, TR):
    x = np.broadcast_to(np.arange(nx), (nz, ny, nx)).reshape(-1)
    n = np.where(x < x0, nL, nR).astype(float)
    T = np.where(x < x0, TL, TR).astype(float)
    z = np.zeros_like(n)
    return n, T, z, z.copy(), z.copy()


def test_solid_cells_read_back_their_state(orc):
    nx, ny, nz = 20, 12, 12
    p = params(orc, nx, ny, nz)
    n1, T1 = 0.7 * float(W.n_eq(0.8)), 0.8          # cloud state differs from the gas around it
    nR, TR = float(W.n_eq(1.0)), 1.0
    s = orc.init(p, *shocked(nx, ny, nz, 6, 3.0 * nR, 1.5, nR, TR))
    mask = sphere_mask(nx, ny, nz, (13, 6, 6), 3.0)
    orc.set_solid(s, mask, n1, T1)
    orc.step(s, 40)
    assert s.nonphysical == 0
    m = orc.macroscopic(s)
    sol = mask.nonzero()[0]
    assert sol.size == 123
    assert np.allclose(m[0, sol], n1, rtol=1e-12, atol=0)
    assert np.allclose(m[1, sol], 3.0 * n1 * T1, rtol=1e-12, atol=0)
    assert np.all(np.abs(m[2:5, sol]) < 1e-13)
    # the gas touching the cloud is not in the cloud's state
    grown = sphere_mask(nx, ny, nz, (13, 6, 6), 4.0) & ~mask
    assert np.max(np.abs(m[0, grown] - n1)) > 1e-3 * n1


def test_cloud_in_its_own_state_is_invisible(orc):
    nx, ny, nz = 14, 10, 10
    p = params(orc, nx, ny, nz, bc_lo=(0, 0, 0), bc_hi=(0, 0, 0))
    n1, T1 = float(W.n_eq(1.0)), 1.0
    N = nx * ny * nz
    s = orc.init(p, np.full(N, n1), np.full(N, T1), np.zeros(N), np.zeros(N), np.zeros(N))
    f0 = s.f.copy()
    orc.set_solid(s, sphere_mask(nx, ny, nz, (7, 5, 5), 2.5), n1, T1)
    orc.step(s, 20)
    assert np.max(np.abs(s.f - f0)) <= 1e-14 * np.max(np.abs(f0))


def mirror(a, ny, nz, nx, axis, c):
    """value of field a at the mirror image about the plane through c (cells)"""
    a = a.reshape(nz, ny, nx)
    n = a.shape[axis]
    idx = (2 * c - np.arange(n)) % n
    return np.take(a, idx, axis=axis).reshape(-1)


def test_cloud_keeps_mirror_symmetry(orc):
    nx, ny, nz = 24, 12, 12
    p = params(orc, nx, ny, nz)
    nR = float(W.n_eq(1.0))
    s = orc.init(p, *shocked(nx, ny, nz, 8, 4.0 * nR, 1.6, nR, 1.0))
    orc.set_solid(s, sphere_mask(nx, ny, nz, (15, 6, 6), 3.2), nR, 1.0)
    orc.step(s, 60)
    assert s.nonphysical == 0
    m = orc.macroscopic(s)
    for axis, comp in ((1, 3), (0, 4)):      # y mirror flips u_y, z mirror flips u_z
        for k in range(6):
            sign = -1.0 if k == comp else 1.0
            got = sign * mirror(m[k], ny, nz, nx, axis, 6)
            assert np.allclose(got, m[k], rtol=1e-12, atol=1e-12 * np.max(np.abs(m[k])) + 1e-300), (axis, k)
    # and the cloud did perturb the flow (the test is not vacuous)
    assert np.max(np.abs(m[3])) > 1e-4
