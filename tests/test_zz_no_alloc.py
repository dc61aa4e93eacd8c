"""rlb_conserved_totals_noalloc: the grid totals for callers that cannot
allocate device memory (an application whose own allocator or pool holds all
device memory, or a loop that cannot afford the synchronisation of
cudaMalloc/cudaFree).  The entry point reads the caller's buffers, writes a
caller-owned 5-double device buffer and keeps its reduction scratch in a
fixed array inside the library.

Checked through the C ABI against the allocating entry point
rlb_conserved_totals, within the tolerance the other totals test uses, on
two calls in a row, with a large grid (every scratch slot used) followed by a
small one (stale slots must not leak into the result).  This file is
collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_1302_1125_gb300 import rlb
from paper_1302_1125_gb300 import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _state_on_device(w, precision, steps):
    g = rlb.Grid.from_workload(w, precision=precision)
    g.init(*[torch.as_tensor(a, device="cuda") for a in w.fields()])
    g.step(steps)
    dtype = torch.float32 if precision == rlb.FP32_STORAGE else torch.float64
    buf = torch.empty(43 * w.N, dtype=dtype, device="cuda")   # caller-owned, compact planes
    rlb.rlb_get_state(g.ctx, buf, 1)
    return g, buf


@pytest.mark.parametrize("precision", [rlb.FP64, rlb.FP32_STORAGE])
def test_noalloc_totals_match_allocating_entry_point(precision):
    from paper_1302_1125_gb300 import build
    build.build()
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for w, steps in ((W.cloud_3d(scale=4), 3), (W.cloud_2d(scale=16), 7)):
        g, buf = _state_on_device(w, precision, steps)
        ref = g.totals()
        esize = buf.element_size()
        for _ in range(2):
            out.fill_(float("nan"))
            rlb.rlb_conserved_totals_noalloc(buf.data_ptr(), buf.data_ptr() + 19 * w.N * esize, w.N,
                                             w.N, precision, out.data_ptr(), stream)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-12 * abs(ref[0])), (got, ref)
        g.close()


def test_noalloc_rejects_bad_arguments():
    out = torch.empty(5, dtype=torch.float64, device="cuda")
    buf = torch.zeros(43 * 8, dtype=torch.float64, device="cuda")
    L = rlb.lib()
    p = buf.data_ptr()
    assert L.rlb_conserved_totals_noalloc(p, p, 0, 8, rlb.FP64, out.data_ptr(), None) == rlb.RLB_E_INVALID
    assert L.rlb_conserved_totals_noalloc(p, p, 2146959361, 2146959361, rlb.FP64, out.data_ptr(),
                                          None) == rlb.RLB_E_INVALID
    assert "RLB_NOALLOC_MAX_CELLS" in rlb.last_error()
    assert L.rlb_conserved_totals_noalloc(p, p, 8, 7, rlb.FP64, out.data_ptr(), None) == rlb.RLB_E_INVALID
    assert L.rlb_conserved_totals_noalloc(None, p, 8, 8, rlb.FP64, out.data_ptr(), None) == rlb.RLB_E_INVALID
    assert L.rlb_conserved_totals_noalloc(p, p, 8, 8, 5, out.data_ptr(), None) == rlb.RLB_E_INVALID
