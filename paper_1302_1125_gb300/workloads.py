"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds initial fields (n, T, u) and run parameters.  It holds
none of the method's arithmetic, imports neither the CUDA library nor the
oracle, and is shared by both sides: the oracle and the CUDA path each turn
these fields into populations on their own.

Units are lattice units: delta x = 1, c = k_B = 1 and the reference
temperature of each workload is T = 1.  Temperatures quoted in MeV
are divided by the reference temperature; pressures are used only through
their ratios.  Equilibrium density at temperature T is
n_eq = d_G T^3 / pi^2 with d_G = 16 (Sec. III), so a state "at lambda = 1"
has n = n_eq(T).

Workloads (Sec. III of the paper sets the shapes).  Every one of them runs
without a non-physical cell in the oracle; where a literal reading of the
benchmark description does not (see the notes), the paper's own setting is
used instead:
  tube_800      1-D viscous QGP shock tube, 800 cells, P ratio 5.43/0.339,
                T 400/200 MeV, eta/s 0.1, zeta/s 0, dt/dx 0.25, 2000 steps.
                (CFL 0.5, i.e. dt/dx 0.36, leaves the method unstable at
                zeta/s = 0; 0.25 is the paper's dt/dx for its 1-D runs.)
  tube_8192     1-D highly relativistic tube, 8192 cells, the paper's
                inviscid-test pressure ratio 1000 from rest (plateau beta 0.91,
                gamma up to 2.5), lambda = 1 on both sides; variant "a" eta/s
                0.01, variant "b" eta/s 0.5 (zeta/s 0.05); alpha 0.2 and dt/dx
                0.15 as in the paper's high-velocity runs; 20000 steps.
                (A slab already moving at gamma = 10 into gas at rest puts
                the second-order equilibrium at |u'| ~ 10, where it has
                populations of +-300 P/9; the first step is non-physical.)
  cloud_2d      2048 x 1024 shock-cloud: ambient T = 1 at rest; the shock is
                driven, as in the paper's 3-D run, by a slab at rest
                (x < nx/8) at pressure ratio 10 and lambda = 1, with the inlet
                at x = 0 holding that slab state; pressure-balanced cloud of
                radius 96 at (700, 512), density x10, tanh edge 4 cells;
                eta/s 0.05, alpha 0.2, dt/dx 0.15; 10000 steps.
  cloud_3d      512 x 256 x 256 version, slab x < 64, cloud radius 48 at
                (180, 128, 128), eta/s 0.05 (zeta/s 0.01), alpha 0.2,
                dt/dx 0.15, 2000 steps.
  batch_tubes   512 tubes from numpy.random.default_rng(1234); draws, in this
                order, 512 values each: Nx log-uniform [256, 8192], eta/s
                U[0.01, 0.5], zeta/s U[0, 0.1], P ratio log-uniform [2, 40],
                left gamma U[1, 1.5]; T_R = 1, left T = ratio^(1/4) (lambda = 1),
                membrane at Nx/2, alpha 0.2, dt/dx 0.15, 4 Nx steps each.
                (Left slabs moving faster than gamma ~ 1.5 into gas at rest
                are non-physical after one step, as for tube_8192.)
  sphere_cloud  the paper's 3-D astrophysical run: 200 x 100 x 100 cells, a
                slab x <= 65 at (n0, T0) and ambient (n1, T1) = (n_eq(1), 1) at
                rest, a solid sphere of radius 10 at (100, 50, 50) held at
                (n1, T1, u = 0), the inlet at x = 0 holding (n0, T0), open
                faces elsewhere; case "beta02": T0 = 2.71 T1, n0 = 0.9 n1;
                case "beta09": T0 = 54.77 T1, n0 = 10.95 n1; inviscid (Euler
                mode) or viscous with tau = 1; alpha 0.2, dt/dx 0.15, 1000
                steps.  (The printed setup puts (n1, T1) on the slab side but
                fixes the inlet there at (n0, T0) and the cloud, held at
                (n1, T1), on the other side: read as slab = (n0, T0).)
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BC_PERIODIC, BC_OUTFLOW, BC_INLET = 0, 1, 2
FP64, FP32_STORAGE = 0, 1
D_G = 16.0


def n_eq(T):
    """equilibrium gluon density at temperature T (Sec. III)"""
    return D_G * np.asarray(T, np.float64) ** 3 / math.pi ** 2


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    bc_lo: tuple
    bc_hi: tuple
    dt_over_dx: float
    eta_over_s: float
    zeta_over_s: float
    steps: int
    precision: int
    inlet: tuple = (1.0, 1.0, (0.0, 0.0, 0.0))   # (n, T, u)
    tau_override: float = 0.0
    alpha_override: float = -1.0
    euler_mode: int = 0
    make_fields: object = field(default=None, repr=False)
    solid: tuple = None     # (make_mask -> uint8[N], n, T): cells held at equilibrium (n, T, u = 0)

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def fields(self):
        """(n, T, ux, uy, uz), float64 arrays of N values, x fastest."""
        return self.make_fields()

    def solid_mask(self):
        """uint8[N] mask of the solid cells (None without solid cells)."""
        return None if self.solid is None else self.solid[0]()


def _tube_fields(nx, ny, nz, left, right, x0=None):
    """left/right = (n, T, ux); membrane between x0-1 and x0"""
    x0 = nx // 2 if x0 is None else x0
    x = np.arange(nx)
    sel = (x < x0)
    def col(a, b):
        v = np.where(sel, a, b).astype(np.float64)
        return np.array(np.broadcast_to(v, (nz, ny, nx)).reshape(-1))   # a writable copy
    n = col(left[0], right[0])
    T = col(left[1], right[1])
    ux = col(left[2], right[2])
    z = np.zeros_like(n)
    return n, T, ux, z, z.copy()


def riemann_tube(nx, P_ratio, T_left, v_left=0.0, T_right=1.0, v_right=0.0, *,
                 dt_over_dx=0.25, eta_over_s=0.01, zeta_over_s=0.0, steps=100,
                 precision=FP64, ny=1, nz=1, name="riemann_tube", **kw) -> Workload:
    """Shock tube: right state n = n_eq(T_right), P_R = n_R T_right; left
    P_L = P_ratio P_R at temperature T_left, n_L = P_L / T_left."""
    nR = float(n_eq(T_right))
    PR = nR * T_right
    PL = P_ratio * PR
    nL = PL / T_left
    make = lambda: _tube_fields(nx, ny, nz, (nL, T_left, v_left), (nR, T_right, v_right))
    return Workload(name, nx, ny, nz, (BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC),
                    (BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC), dt_over_dx, eta_over_s,
                    zeta_over_s, steps, precision, make_fields=make, **kw)


def tube_800(steps=2000, precision=FP64) -> Workload:
    return riemann_tube(800, 5.43 / 0.339, 2.0, dt_over_dx=0.25, eta_over_s=0.1,
                        zeta_over_s=0.0, steps=steps, precision=precision, name="tube_800")


def tube_8192(variant="a", steps=20000, precision=FP64, nx=8192) -> Workload:
    ratio = 1000.0
    eta, zeta = (0.01, 0.0) if variant == "a" else (0.5, 0.05)
    return riemann_tube(nx, ratio, ratio ** 0.25, 0.0, dt_over_dx=0.15, eta_over_s=eta,
                        zeta_over_s=zeta, alpha_override=0.2, steps=steps,
                        precision=precision, name=f"tube_{nx}_{variant}")


def _cloud_fields(nx, ny, nz, R, centre, slab_x, slab_n, slab_T, contrast=10.0, width=4.0):
    nA = float(n_eq(1.0))
    PA = nA * 1.0
    zz, yy, xx = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                             np.arange(nx, dtype=np.float64), indexing="ij")
    r2 = (xx - centre[0]) ** 2 + (yy - centre[1]) ** 2
    if nz > 1:
        r2 += (zz - centre[2]) ** 2
    r = np.sqrt(r2)
    n = nA * (1.0 + (contrast - 1.0) * 0.5 * (1.0 - np.tanh((r - R) / width)))
    T = PA / n                      # pressure balance with the ambient gas
    slab = xx < slab_x
    n = np.where(slab, slab_n, n)
    T = np.where(slab, slab_T, T)
    n = np.ascontiguousarray(n.reshape(-1))
    T = np.ascontiguousarray(T.reshape(-1))
    z = np.zeros_like(n)
    return n, T, z, z.copy(), z.copy()


def shock_cloud(nx, ny, nz, R, centre, *, slab_x=None, ratio=10.0, eta_over_s=0.05,
                zeta_over_s=0.0, alpha_override=0.2, steps=100, precision=FP32_STORAGE,
                dt_over_dx=0.15, name="shock_cloud", **kw) -> Workload:
    """Ambient T = 1, n = n_eq(1) at rest; a slab x < slab_x at rest with
    pressure ratio `ratio` at lambda = 1 drives the shock; the inlet at x = 0
    holds the slab state; outflow at x = nx - 1; periodic in y and z; the
    cloud is in pressure balance with the ambient gas."""
    slab_x = nx // 8 if slab_x is None else slab_x
    nA = float(n_eq(1.0))
    T_s = ratio ** 0.25
    n_s = ratio * nA / T_s
    make = lambda: _cloud_fields(nx, ny, nz, R, centre, slab_x, n_s, T_s)
    return Workload(name, nx, ny, nz, (BC_INLET, BC_PERIODIC, BC_PERIODIC),
                    (BC_OUTFLOW, BC_PERIODIC, BC_PERIODIC), dt_over_dx, eta_over_s,
                    zeta_over_s, steps, precision, inlet=(n_s, T_s, (0.0, 0.0, 0.0)),
                    alpha_override=alpha_override, make_fields=make, **kw)


def cloud_2d(steps=10000, precision=FP32_STORAGE, scale=1) -> Workload:
    """scale = k shrinks the grid and the cloud by k (parity-size cases)"""
    return shock_cloud(2048 // scale, 1024 // scale, 1, 96.0 / scale,
                       (700.0 / scale, 512.0 / scale, 0.0), eta_over_s=0.05, zeta_over_s=0.0,
                       steps=steps, precision=precision, name=f"cloud_2d_s{scale}")


def cloud_3d(steps=2000, precision=FP32_STORAGE, scale=1) -> Workload:
    return shock_cloud(512 // scale, 256 // scale, 256 // scale, 48.0 / scale,
                       (180.0 / scale, 128.0 / scale, 128.0 / scale), slab_x=64 // scale,
                       eta_over_s=0.05,
                       zeta_over_s=0.01, steps=steps, precision=precision,
                       name=f"cloud_3d_s{scale}")


@dataclass
class BatchSpec:
    nx: np.ndarray          # int32 [B]
    eta_over_s: np.ndarray  # [B]
    zeta_over_s: np.ndarray
    ratio: np.ndarray
    gamma_left: np.ndarray
    steps: np.ndarray       # int64 [B] = 4 nx
    offsets: np.ndarray     # int64 [B+1], packed cell offsets
    dt_over_dx: float = 0.15
    alpha: float = 0.2

    @property
    def B(self) -> int:
        return int(self.nx.size)

    def fields(self):
        """packed (n, T, ux) over all tubes, float64 arrays of offsets[-1] values"""
        tot = int(self.offsets[-1])
        n = np.empty(tot)
        T = np.empty(tot)
        ux = np.empty(tot)
        nR = float(n_eq(1.0))
        for b in range(self.B):
            o, m = int(self.offsets[b]), int(self.nx[b])
            TL = float(self.ratio[b]) ** 0.25
            nL = self.ratio[b] * nR / TL
            vL = math.sqrt(1.0 - 1.0 / float(self.gamma_left[b]) ** 2)
            x = np.arange(m)
            left = x < m // 2
            n[o:o + m] = np.where(left, nL, nR)
            T[o:o + m] = np.where(left, TL, 1.0)
            ux[o:o + m] = np.where(left, vL, 0.0)
        return n, T, ux


def batch_tubes(count=512, seed=1234, nx_min=256, nx_max=8192) -> BatchSpec:
    rng = np.random.default_rng(seed)
    nx = np.exp(rng.uniform(math.log(nx_min), math.log(nx_max), count)).round().astype(np.int32)
    eta = rng.uniform(0.01, 0.5, count)
    zeta = rng.uniform(0.0, 0.1, count)
    ratio = np.exp(rng.uniform(math.log(2.0), math.log(40.0), count))
    gam = rng.uniform(1.0, 1.5, count)
    off = np.zeros(count + 1, np.int64)
    off[1:] = np.cumsum(nx)
    return BatchSpec(nx, eta, zeta, ratio, gam, 4 * nx.astype(np.int64), off)


def periodic_box(nx, ny=1, nz=1, *, seed=7, amp=0.2, gamma_max=3.0, dt_over_dx=0.25,
                 tau_override=0.8, alpha_override=0.1, precision=FP64, steps=50,
                 name="periodic_box") -> Workload:
    """Smooth random periodic state (for conservation and parity tests):
    n, T and u are low-order Fourier sums with a seeded rng."""
    rng = np.random.default_rng(seed)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    def smooth():
        acc = np.zeros((nz, ny, nx))
        for _ in range(4):
            k = rng.integers(-2, 3, 3)
            ph = rng.uniform(0, 2 * math.pi)
            acc += rng.normal() * np.cos(2 * math.pi * (k[0] * xx / nx + k[1] * yy / max(ny, 1)
                                                        + k[2] * zz / max(nz, 1)) + ph)
        return acc / 4.0
    T = 1.0 + amp * smooth()
    n = n_eq(T) * (1.0 + amp * smooth())
    bmax = math.sqrt(1.0 - 1.0 / gamma_max ** 2)
    u = [np.clip(0.5 * bmax * smooth(), -0.57 * bmax, 0.57 * bmax) for _ in range(3)]
    if ny == 1:
        u[1][:] = 0.0
    if nz == 1:
        u[2][:] = 0.0
    fl = [np.ascontiguousarray(a.reshape(-1), np.float64) for a in (n, T, *u)]
    per = (BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    return Workload(name, nx, ny, nz, per, per, dt_over_dx, 0.1, 0.0, steps, precision,
                    tau_override=tau_override, alpha_override=alpha_override,
                    make_fields=lambda: tuple(a.copy() for a in fl))


def boosted_box(nx, ny=1, nz=1, *, gamma=10.0, direction=(1.0, 0.0, 0.0), amp=1e-3, dt_over_dx=0.15,
                tau_override=1.0, alpha_override=0.2, precision=FP32_STORAGE, steps=2000,
                name="boosted_box") -> Workload:
    """Periodic box of gas at T = 1, n = n_eq(1) moving as a whole at Lorentz
    factor `gamma` along `direction` (normalised here), with a small
    temperature and density ripple of relative size `amp` that varies along
    x only (amp = 0: a uniform boosted state).  The states of the
    high-gamma precision checks: the regime, gamma ~ 10, where the
    Landau-frame recovery meets the 1 - beta^2 cancellation."""
    d = np.asarray(direction, np.float64)
    d = d / np.linalg.norm(d)
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    x = np.arange(nx, dtype=np.float64)
    ripple = np.cos(2 * math.pi * x / nx + 0.3) + 0.5 * np.sin(4 * math.pi * x / nx + 1.1)
    T1 = 1.0 + amp * ripple
    n1 = float(n_eq(1.0)) * (1.0 + 0.5 * amp * np.cos(2 * math.pi * x / nx + 2.0))

    def col(v):
        return np.array(np.broadcast_to(v, (nz, ny, nx)).reshape(-1), np.float64)   # a writable copy
    fl = [col(n1), col(T1)] + [col(np.full(nx, beta * d[a])) for a in range(3)]
    per = (BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    return Workload(name, nx, ny, nz, per, per, dt_over_dx, 0.05, 0.0, steps, precision,
                    tau_override=tau_override, alpha_override=alpha_override,
                    make_fields=lambda: tuple(a.copy() for a in fl))


def smooth_gamma_box(nx, ny, nz, *, gamma_max=15.0, seed=11, ripple=0.0, dt_over_dx=0.15, tau_override=1.0,
                     alpha_override=0.2, precision=FP32_STORAGE, name="smooth_gamma_box") -> Workload:
    """Periodic box whose Lorentz factor rises smoothly along x from 1 to
    gamma_max and back (a raised cosine), moving in a direction that turns
    slowly along x, with seeded ripples of relative size `ripple` in T and n
    across y and z: a state spanning gamma 1 .. gamma_max for cell-by-cell
    checks of single steps."""
    rng = np.random.default_rng(seed)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    g = 1.0 + (gamma_max - 1.0) * 0.5 * (1.0 - np.cos(2 * math.pi * xx / nx))
    beta = np.sqrt(1.0 - 1.0 / g ** 2)
    ph = rng.uniform(0, 2 * math.pi, 4)
    th = 0.5 * np.sin(2 * math.pi * xx / nx + ph[0])
    ps = 0.3 * np.cos(2 * math.pi * xx / nx + ph[1])
    d = [np.cos(th) * np.cos(ps), np.sin(th) * np.cos(ps), np.sin(ps)]
    T = 1.0 + ripple * np.cos(2 * math.pi * (yy / max(ny, 1) + zz / max(nz, 1)) + ph[2])
    n = n_eq(T) * (1.0 + ripple * np.sin(2 * math.pi * (zz / max(nz, 1) - yy / max(ny, 1)) + ph[3]))
    fl = [np.ascontiguousarray(a.reshape(-1), np.float64) for a in (n, T, *(beta * c for c in d))]
    per = (BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)
    return Workload(name, nx, ny, nz, per, per, dt_over_dx, 0.05, 0.0, 1, precision,
                    tau_override=tau_override, alpha_override=alpha_override,
                    make_fields=lambda: tuple(a.copy() for a in fl))


def sphere_cloud(case="beta09", scale=1, *, viscous=False, precision=FP32_STORAGE, steps=None) -> Workload:
    """The paper's 3-D shock-cloud run with a solid sphere (Sec. III), every
    length divided by `scale` (steps too, so the same physical time)."""
    T0, r = {"beta02": (2.71, 0.9), "beta09": (54.77, 10.95)}[case]
    nx, ny, nz = 200 // scale, 100 // scale, 100 // scale
    T1 = 1.0
    n1 = float(n_eq(T1))
    n0 = r * n1
    xs = 65.0 / scale
    cx, cy, cz, R = 100.0 / scale, 50.0 / scale, 50.0 / scale, 10.0 / scale

    def make():
        x = np.arange(nx, dtype=np.float64)
        slab = np.broadcast_to(x <= xs, (nz, ny, nx)).reshape(-1)
        n = np.where(slab, n0, n1).astype(np.float64)
        T = np.where(slab, T0, T1).astype(np.float64)
        z = np.zeros_like(n)
        return n, T, z, z.copy(), z.copy()

    def mask():
        zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        d2 = (xx - cx) ** 2 + (yy - cy) ** 2 + (zz - cz) ** 2
        return np.ascontiguousarray((d2 <= R * R).reshape(-1), np.uint8)

    out = (BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW)
    return Workload(f"sphere_cloud_{case}" + ("_viscous" if viscous else "") + (f"_s{scale}" if scale > 1 else ""),
                    nx, ny, nz, (BC_INLET, BC_OUTFLOW, BC_OUTFLOW), out, 0.15, 0.0, 0.0,
                    steps if steps is not None else 1000 // scale, precision,
                    inlet=(n0, T0, (0.0, 0.0, 0.0)), tau_override=1.0 if viscous else 0.0,
                    alpha_override=0.2, euler_mode=0 if viscous else 1, make_fields=make,
                    solid=(mask, n1, T1))
