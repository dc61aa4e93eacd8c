"""The order in which the blocks of the FP32 3-D tiled step start
(rlb_options.slab_rows; csrc/rlb_step_f32.cuh, the block remap of
step_f32_kernel).

Each block computes the same 64 x 8 cells whatever its place in the order,
and a step reads only the previous buffers, so every slab height gives the
state of the plain x, y, z order bit for bit: full slabs, a ragged last slab
(block rows not a multiple of the slab height), one-row slabs, the automatic
height on a grid wide enough to use it, the FP64-recovery variant of the
kernel and the bulk-staged kernel (thread_mapping 3), which takes the same
order.  The oracle parity of the step is tests/test_gpu_parity.py's.
"""
import numpy as np
import pytest

from paper_1302_1125_gb300 import rlb
from paper_1302_1125_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1302_1125_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "the gpu tests need a CUDA device"


def _box(nx, ny, nz, seed, lo, hi):
    w = W.periodic_box(nx, ny, nz, seed=seed, tau_override=0.0, alpha_override=0.1)
    w.bc_lo, w.bc_hi = lo, hi
    return w


def _state(w, slab_rows, steps, **kw):
    g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, thread_mapping=rlb.MAPPING_TILES,
                               slab_rows=slab_rows, **kw)
    g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
    kernel = g.step_kernel
    g.step(steps)
    s = g.get_state()
    g.close()
    return kernel, s


# (grid, faces): 6 block rows of 8 cells
CASES = {
    "periodic": ((128, 48, 10), (0, 0, 0), (0, 0, 0)),
    "inlet_open": ((192, 48, 7), (2, 1, 1), (1, 1, 1)),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("slab_rows", [1, 2, 4, 5])
def test_slab_orders_equal_the_plain_order(name, slab_rows):
    dims, lo, hi = CASES[name]
    w = _box(*dims, seed=21, lo=lo, hi=hi)
    k0, plain = _state(w, 1000, 25)
    k1, slab = _state(w, slab_rows, 25)
    assert k0 == k1 == "fp32_tiles"
    for a, b in zip(plain, slab):
        assert np.array_equal(a, b)


def test_automatic_slab_height_on_a_wide_grid():
    # nx = 1024: the automatic height is 8 block rows (a 10 MB slab plane)
    # of the 12 here, so the last slab is ragged
    w = _box(1024, 96, 6, seed=22, lo=(1, 0, 0), hi=(1, 0, 0))
    _, plain = _state(w, 1000, 6)
    _, auto = _state(w, 0, 6)
    for a, b in zip(plain, auto):
        assert np.array_equal(a, b)


def test_slab_order_of_the_fp64_recovery_variant():
    w = _box(128, 48, 6, seed=23, lo=(1, 0, 0), hi=(1, 0, 0))
    k0, plain = _state(w, 1000, 10, recovery_fp64=1)
    k1, slab = _state(w, 2, 10, recovery_fp64=1)
    assert k0 == k1 == "fp32_rec64"
    for a, b in zip(plain, slab):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("slab_rows", [1, 4])
def test_slab_order_of_the_bulk_staged_kernel(slab_rows):
    # thread_mapping 3: the block-wide bulk-copy kernel takes the same order
    w = _box(192, 48, 7, seed=24, lo=(2, 1, 1), hi=(1, 1, 1))
    _, plain = _state(w, 1000, 12)
    g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, thread_mapping=rlb.MAPPING_BULK_TILES,
                               slab_rows=slab_rows)
    g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
    assert g.step_kernel == "fp32_bulk_tiles"
    g.step(12)
    bulk = g.get_state()
    g.close()
    for a, b in zip(plain, bulk):
        assert np.array_equal(a, b)
