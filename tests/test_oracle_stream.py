"""Pins of the oracle's minmod streaming (Sec. II.A, Eqs. 47-53) and of the
central Laplacian of the bulk term (Eq. 54).

The operator is exercised on a single scalar plane q moving with a given
velocity p, with increment -k sum_a [h^a(x) - h^a(x - e_a)].  Closed forms:
linear data is differentiated exactly; first-order upwind (limiter off) is the
textbook scheme; the limited scheme is total-variation diminishing, mirror
symmetric, conservative and second order in L1 on smooth data; the Laplacian
is exact on quadratics and has the discrete eigenvalue -4 sin^2(k/2) on
Fourier modes.
"""
import numpy as np
import pytest


def P1(orc, nx, ny=1, nz=1, bc=None, limiter=0):
    bc = bc if bc is not None else (0, 0, 0)
    return orc.Params(nx=nx, ny=ny, nz=nz, bc_lo=bc, bc_hi=bc, limiter=limiter)


def test_minmod_definition(orc):
    rng = np.random.default_rng(0)
    for X, Y in rng.normal(size=(200, 2)):
        m = orc.minmod(X, Y)
        assert m == orc.minmod(Y, X)
        assert orc.minmod(-X, -Y) == -m
        if X * Y <= 0:
            assert m == 0.0
        else:
            assert m == np.sign(X) * min(abs(X), abs(Y))
    assert orc.minmod(0.0, 3.0) == 0.0


@pytest.mark.parametrize("v", [0.7, -1.3])
def test_linear_data_is_differentiated_exactly(orc, v):
    nx = 32
    x = np.arange(nx, dtype=float)
    q = 2.0 + 0.25 * x
    p = P1(orc, nx, bc=(1, 0, 0))
    out = orc.stream(p, q, [v, 0, 0], 0.1)
    assert np.allclose(out[2:-2], -0.1 * v * 0.25, rtol=1e-13, atol=0)


@pytest.mark.parametrize("v", [0.9, -0.6])
def test_limiter_off_is_first_order_upwind(orc, v):
    rng = np.random.default_rng(1)
    nx = 40
    q = rng.normal(size=nx)
    out = orc.stream(P1(orc, nx, limiter=1), q, [v, 0, 0], 0.3)
    up = (q - np.roll(q, 1)) if v > 0 else (np.roll(q, -1) - q)
    assert np.allclose(out, -0.3 * v * up, rtol=0, atol=1e-14)


def _tv(q):
    return np.abs(np.diff(np.r_[q, q[0]])).sum()


@pytest.mark.parametrize("v", [1.0, -1.0])
def test_tvd_and_no_new_extrema(orc, v):
    nx = 100
    q = np.where((np.arange(nx) > 30) & (np.arange(nx) < 60), 1.0, 0.0)
    p = P1(orc, nx)
    tv = _tv(q)
    for _ in range(150):
        q = q + orc.stream(p, q, [v, 0, 0], 0.4)      # Courant number 0.4
        assert _tv(q) <= tv + 1e-12
        tv = _tv(q)
        assert q.min() >= -1e-14 and q.max() <= 1 + 1e-14


def test_conservative_and_centroid_moves_with_the_velocity(orc):
    nx = 400
    x = np.arange(nx, dtype=float)
    q = np.exp(-((x - 150.0) / 12.0) ** 2)
    v, k, steps = 0.8, 0.25, 200
    for lim, tol in ((1, 1e-9), (0, 5e-3)):
        p = P1(orc, nx, limiter=lim)
        qq = q.copy()
        for _ in range(steps):
            qq = qq + orc.stream(p, qq, [v, 0, 0], k)
        assert abs(qq.sum() - q.sum()) < 1e-12 * q.sum()
        shift = (x * qq).sum() / qq.sum() - (x * q).sum() / q.sum()
        assert abs(shift - v * k * steps) < tol * v * k * steps


def test_mirror_symmetry(orc):
    # reading R2: with Delta f^{a-} in f^{aR} the scheme for p < 0 is the exact
    # mirror image of the scheme for p > 0
    rng = np.random.default_rng(2)
    for bc in (0, 1):
        nx = 37
        q = np.cumsum(rng.normal(size=nx))
        p = P1(orc, nx, bc=(bc, 0, 0))
        a = orc.stream(p, q, [1.1, 0, 0], 0.2)
        b = orc.stream(p, q[::-1].copy(), [-1.1, 0, 0], 0.2)
        assert np.allclose(a, b[::-1], rtol=0, atol=1e-15 * np.abs(q).max())


def test_second_order_on_smooth_data(orc):
    errs = []
    for nx in (64, 128, 256, 512):
        x = (np.arange(nx) + 0.5) / nx
        q = np.sin(2 * np.pi * x) + 0.3 * np.cos(4 * np.pi * x)
        dq = 2 * np.pi * np.cos(2 * np.pi * x) - 1.2 * np.pi * np.sin(4 * np.pi * x)
        out = orc.stream(P1(orc, nx), q, [1.0, 0, 0], 1.0)   # = -dq/dx * dx
        errs.append(np.abs(-out * nx - dq).mean())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 1.7), orders


def test_multidimensional_flux_sums_over_axes(orc):
    # a diagonal velocity on a 2-D linear field: increment = -k (p_x b_x + p_y b_y)
    nx, ny = 12, 10
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    q = (1.0 + 0.3 * xx - 0.2 * yy).reshape(-1)
    p = P1(orc, nx, ny, bc=(1, 1, 0))
    out = orc.stream(p, q, [0.5, -0.7, 0], 0.2).reshape(ny, nx)
    assert np.allclose(out[2:-2, 2:-2], -0.2 * (0.5 * 0.3 + (-0.7) * (-0.2)), rtol=1e-13)


def test_boundaries(orc):
    nx = 16
    # zero-gradient ends: a constant field streams to nothing
    p = P1(orc, nx, bc=(1, 0, 0))
    assert np.all(orc.stream(p, np.full(nx, 3.0), [1.0, 0, 0], 0.3) == 0.0)
    assert np.all(orc.laplacian(p, np.full(nx, 3.0)) == 0.0)
    # inlet ghost: the ghost value enters through the upwind face
    p = orc.Params(nx=nx, bc_lo=(2, 0, 0), bc_hi=(1, 0, 0), limiter=1)
    out = orc.stream(p, np.zeros(nx), [1.0, 0, 0], 0.5, ghost=2.0)
    assert out[0] == -0.5 * (0.0 - 2.0) and np.all(out[1:] == 0.0)
    # periodic wrap: a shifted copy gives a shifted result
    q = np.random.default_rng(3).normal(size=nx)
    p = P1(orc, nx)
    assert np.allclose(np.roll(orc.stream(p, q, [0.9, 0, 0], 0.2), 3),
                       orc.stream(p, np.roll(q, 3), [0.9, 0, 0], 0.2), atol=1e-15)


@pytest.mark.parametrize("limiter", [0, 1])
def test_outflow_ghosts_copy_the_edge_cell(orc, limiter):
    """Zero-gradient open ends (Sec. III): both ghost cells past an end hold
    the edge cell's value.  So the upstream edge cell receives its own value
    through the open face and its increment is zero whatever the data, and
    the Laplacian there is the one-sided difference q[1] - q[0]."""
    nx = 12
    q = np.random.default_rng(8).normal(size=nx)
    p = P1(orc, nx, bc=(1, 0, 0), limiter=limiter)
    up = orc.stream(p, q, [0.8, 0, 0], 0.3)      # moving right: x = 0 is upstream
    down = orc.stream(p, q, [-0.8, 0, 0], 0.3)   # moving left: x = nx - 1 is upstream
    assert up[0] == 0.0 and down[-1] == 0.0
    assert up[-1] != 0.0 and down[0] != 0.0
    lap = orc.laplacian(p, q)
    assert lap[0] == pytest.approx(q[1] - q[0], abs=1e-15)
    assert lap[-1] == pytest.approx(q[-2] - q[-1], abs=1e-15)


def test_laplacian_closed_forms(orc):
    nx, ny, nz = 9, 8, 7
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    q = (xx ** 2 + 2.0 * yy ** 2 - 0.5 * zz ** 2).reshape(-1).astype(float)
    out = orc.laplacian(orc.Params(nx=nx, ny=ny, nz=nz, bc_lo=(1, 1, 1), bc_hi=(1, 1, 1)),
                        q).reshape(nz, ny, nx)
    assert np.allclose(out[1:-1, 1:-1, 1:-1], 2.0 + 4.0 - 1.0, rtol=1e-13)
    m = 32
    x = np.arange(m)
    q = np.sin(2 * np.pi * 3 * x / m)
    out = orc.laplacian(P1(orc, m), q)
    assert np.allclose(out, -4 * np.sin(np.pi * 3 / m) ** 2 * q, atol=1e-14)
