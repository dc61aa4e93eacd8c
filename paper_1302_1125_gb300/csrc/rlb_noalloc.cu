// rlb_noalloc.cu -- rlb_conserved_totals_noalloc: the grid-total reduction
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// entirely reserved up front by its own allocator or memory pool, or a loop
// that cannot afford the implicit device-wide synchronisation cudaMalloc and
// cudaFree bring.  This entry point takes the caller's population planes and
// a caller-owned 5-double output buffer and allocates nothing: the per-block
// partial sums of the reduction live in the file-scope array below, which
// every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/rlb.h"
#include "rlb_internal.h"

namespace {

// one partial sum of (T^00, T^0x, T^0y, T^0z, N^0) per block of the
// reduction; the reduction never uses more than RLB_NOALLOC_MAX_BLOCKS blocks
constexpr int kMaxBlocks = RLB_NOALLOC_MAX_BLOCKS;
static __device__ __align__(256) double g_partial[5 * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_partial_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device and kept for the life of the process (the header states that a
// cudaDeviceReset invalidates it).  The name g_partial is only a host-side
// stand-in in host code.
cudaError_t scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_partial_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partial);
        if (e != cudaSuccess) return e;
        g_partial_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_partial_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" rlb_status rlb_conserved_totals_noalloc(const void *f, const void *h, int N,
                                                   long long plane_stride, int precision,
                                                   double *out_device, void *cuda_stream)
{
    auto invalid = [](const char *msg) {
        rlb::set_thread_error(msg);
        return RLB_E_INVALID;
    };
    if (!f || !h || !out_device) return invalid("rlb_conserved_totals_noalloc: a pointer is NULL");
    if (N < 1 || N > RLB_NOALLOC_MAX_CELLS)
        return invalid("rlb_conserved_totals_noalloc: N must be in [1, RLB_NOALLOC_MAX_CELLS]");
    if (plane_stride < N) return invalid("rlb_conserved_totals_noalloc: plane_stride < N");
    if (precision != RLB_FP64 && precision != RLB_FP32_STORAGE)
        return invalid("rlb_conserved_totals_noalloc: unknown precision");
    if (rlb::totals_blocks(N) > kMaxBlocks)
        return invalid("rlb_conserved_totals_noalloc: reduction exceeds the scratch array");
    double *partial = nullptr;
    if (scratch_for_current_device(&partial) != cudaSuccess) {
        rlb::set_thread_error("rlb_conserved_totals_noalloc: cudaGetSymbolAddress failed");
        return RLB_E_CUDA;
    }
    // every partial slot the finishing kernel reads is written earlier in the
    // same call, so nothing has to be cleared between calls
    const cudaError_t e = rlb::launch_totals(precision == RLB_FP32_STORAGE, N, plane_stride, f, h,
                                             partial, out_device, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        rlb::set_thread_error(cudaGetErrorString(e));
        return RLB_E_CUDA;
    }
    return RLB_OK;
}
