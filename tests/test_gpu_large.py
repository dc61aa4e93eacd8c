"""Large grids: the index arithmetic past 2^31 elements.

A 512 x 512 x 2P periodic grid whose fields repeat with period P in z sees,
at every cell, the same stencil values as the 512 x 512 x P grid with the
first period of those fields; the step computes each cell from its stencil
alone, so after a few steps the two macroscopic states agree bit for bit (a
wrong plane, row or z offset anywhere in the larger grid breaks it).
Fields are generated on the device (smooth seeded Fourier modes), so
nothing of the size crosses the host.  In both precisions the larger grid's
population planes hold more than 2^31 elements in all (19 planes of N
cells: FP32 storage at 512 x 512 x 768, 2.0 x 10^8 cells; FP64 at
512 x 512 x 448, 1.17 x 10^8 cells), so the plane offsets cross the 32-bit
range.  Each case needs about 90 GB of device memory at its peak.
"""
import math

import numpy as np
import pytest

from paper_1302_1125_gb300 import rlb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1302_1125_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def fields(nx, ny, nz, period, seed):
    """n, T, u (x-fastest, on the device): sums of seeded Fourier modes with
    periods nx, ny and `period` in z"""
    g = torch.Generator().manual_seed(seed)
    # z reduced modulo the period first: the fields then repeat bit for bit
    z = torch.remainder(torch.arange(nz, device="cuda", dtype=torch.float64), period).view(nz, 1, 1)
    y = torch.arange(ny, device="cuda", dtype=torch.float64).view(1, ny, 1)
    x = torch.arange(nx, device="cuda", dtype=torch.float64).view(1, 1, nx)

    def smooth():
        acc = torch.zeros(nz, ny, nx, device="cuda", dtype=torch.float64)
        for _ in range(3):
            k = torch.randint(-2, 3, (3,), generator=g).tolist()
            ph = float(torch.rand(1, generator=g)) * 2 * math.pi
            acc += float(torch.randn(1, generator=g)) * torch.cos(
                2 * math.pi * (k[0] * x / nx + k[1] * y / ny + k[2] * z / period) + ph)
        return acc / 3.0

    T = 1.0 + 0.2 * smooth()
    n = (16.0 / math.pi ** 2) * T ** 3 * (1.0 + 0.2 * smooth())
    u = [0.15 * smooth() for _ in range(3)]
    return [a.reshape(-1).contiguous() for a in (n, T, *u)]


def run(nx, ny, nz, period, steps, precision):
    per = (rlb.BC_PERIODIC,) * 3
    g = rlb.Grid(nx, ny, nz, bc_lo=per, bc_hi=per, dt_over_dx=0.15, eta_over_s=0.1, alpha_override=0.2,
                 precision=precision)
    f = fields(nx, ny, nz, period, 77)
    g.init(*f)
    del f
    g.step(steps)
    out = torch.empty(6 * g.N, dtype=torch.float64, device="cuda")
    rlb.rlb_macroscopic(g.ctx, out, 1)
    g.close()
    return out.view(6, nz, ny, nx)


@pytest.mark.parametrize("precision,period", [(rlb.FP32_STORAGE, 384), (rlb.FP64, 224)])
def test_two_periods_equal_one_bit_for_bit(precision, period):
    nx, ny = 512, 512
    assert 19 * nx * ny * 2 * period > 2 ** 31
    # memory that earlier tests left in torch's cache goes back to the device
    import gc
    gc.collect()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 110e9:
        pytest.skip("needs ~110 GB of free device memory")
    small = run(nx, ny, period, period, 3, precision)
    big = run(nx, ny, 2 * period, period, 3, precision)
    assert big.shape[1] * ny * nx == 2 * period * ny * nx
    assert torch.equal(big[:, :period], small)
    assert torch.equal(big[:, period:], small)
    assert bool(torch.isfinite(small).all())
