"""The FP32-storage step with its stencil tiles staged by block-wide bulk
copies (csrc/rlb_bulk.cuh, csrc/rlb_step_f32_bulk.cu; rlb_options
thread_mapping = 3 on the grids that allow it).

It runs the same per-cell arithmetic as the per-thread staged kernel and only
moves the data differently, so on every grid it takes, the states of the
two after the same steps are equal bit for bit.  The grids below cover its
boundary handling: the inlet and the open end on the x faces (halo columns
not copied, replaced by the edge threads' fix-ups), periodic and open y and
z faces (source rows picked through the boundary map), nz = 2 (z +- 2 wraps
onto the cell's own plane), one and several tiles along x.  The oracle
parity of the path is the FP32 parity of tests/test_gpu_parity.py, whose
3-D shock-cloud cases it runs.
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


def _box(nx, ny, nz, seed, lo, hi, **kw):
    w = W.periodic_box(nx, ny, nz, seed=seed, tau_override=0.0, alpha_override=0.1, **kw)
    w.bc_lo, w.bc_hi = lo, hi
    w.precision = rlb.FP32_STORAGE
    return w


CASES = {
    "cloud_3d_s4": lambda: W.cloud_3d(scale=4),                                   # inlet x, periodic y z
    "open_faces": lambda: _box(64, 16, 8, 3, (1, 1, 1), (1, 1, 1)),               # one tile along x
    "mixed_faces": lambda: _box(192, 8, 6, 4, (2, 0, 1), (1, 0, 1)),             # inlet, periodic y, open z
    "two_planes": lambda: _box(128, 16, 2, 5, (1, 0, 0), (1, 0, 0)),             # z +- 2 wraps to z
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_bulk_tiles_equal_per_thread_staging(name):
    w = CASES[name]()
    states, kernels = [], []
    for mapping in (rlb.MAPPING_BULK_TILES, rlb.MAPPING_TILES, rlb.MAPPING_AUTO):
        g = rlb.Grid.from_workload(w, precision=rlb.FP32_STORAGE, thread_mapping=mapping)
        g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
        kernels.append(g.step_kernel)
        g.step(30)
        states.append(g.get_state())
        g.close()
    assert kernels == ["fp32_bulk_tiles", "fp32_tiles", "fp32_tiles"], kernels
    for other in states[1:]:
        for a, b in zip(states[0], other):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("dims,lo,hi,euler,expect", [
    ((64, 8, 4), (1, 0, 0), (1, 0, 0), 0, "fp32_bulk_tiles"),
    ((190, 8, 4), (1, 0, 0), (1, 0, 0), 0, "fp32_tiles"),           # nx not a multiple of 64
    ((64, 12, 4), (1, 0, 0), (1, 0, 0), 0, "fp32_tiles"),           # ny not a multiple of 8
    ((64, 8, 4), (0, 0, 0), (0, 0, 0), 0, "fp32_tiles"),     # periodic x faces
    ((64, 8, 4), (1, 0, 0), (1, 0, 0), 1, "fp32_tiles"),     # Euler mode
    ((64, 8, 1), (1, 0, 0), (1, 0, 0), 0, "fp32_tiles"),     # 2-D
])
def test_which_grids_take_the_bulk_path(dims, lo, hi, euler, expect):
    g = rlb.Grid(*dims, bc_lo=lo, bc_hi=hi, precision=rlb.FP32_STORAGE, euler_mode=euler, dt_over_dx=0.15,
                 alpha_override=0.1, thread_mapping=rlb.MAPPING_BULK_TILES)
    assert g.step_kernel == expect
    g.close()


def test_step_kernel_names_of_the_other_forms():
    g = rlb.Grid(512, 256, 4, precision=rlb.FP64, dt_over_dx=0.15, alpha_override=0.1)
    assert g.step_kernel == "fp64_tiles"
    g.close()
    g = rlb.Grid(800, precision=rlb.FP64)
    assert g.step_kernel == "fp64_small"
    g.close()
    g = rlb.Grid(64, 8, 4, precision=rlb.FP32_STORAGE, recovery_fp64=1, dt_over_dx=0.15, alpha_override=0.1)
    assert g.step_kernel == "fp32_rec64"
    g.close()
