// rlb_batch.cuh -- the batched form of the FP32-storage step: B independent
// 1-D tubes (zero-gradient ends, Sec. III), each with its own length, eta/s
// and bulk coefficient, advanced by one persistent launch.
//
// Work division.  A cluster of C blocks (C = 1: one block) takes a job, one
// tube or a few consecutive tubes of similar length, and runs all of the
// job's steps; its C x blockDim threads split the job's cell pairs and meet
// at a barrier after each step (the block barrier for C = 1, the hardware
// cluster barrier otherwise).  No block ever waits on a block outside its
// own cluster, so there is no grid-wide barrier and no software spin.  Jobs
// are assigned to clusters on the host, longest first, each to the least
// loaded cluster; the grid holds exactly as many clusters as fit on the GPU
// at once.
#pragma once

#include "rlb_step_f32.cuh"

namespace rlb {
namespace batch {

__device__ __forceinline__ unsigned cluster_rank()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_index()
{
    unsigned r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}

// hardware barrier over every thread of the cluster; release/acquire order
// each thread's earlier global stores before the other blocks' later loads
__device__ __forceinline__ void cluster_barrier()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// geometry of the pair (x0, x0 + 1) of a tube of nx cells stored at `off`
// (zero-gradient at both ends; an odd tube's last pair holds one pad cell)
__device__ __forceinline__ f32::Geo tube_geo(int off, int nx, int x0)
{
    f32::Geo g;
    g.x0 = x0;
    g.idx0 = off + x0;
    g.has1 = x0 + 1 < nx;
    g.idx1 = g.has1 ? g.idx0 + 1 : g.idx0;
    g.oa = -2;
    g.oc = 2;
    g.xfix = 0u;
    if (x0 == 0) {
        g.oa = 0;
        g.xfix |= f32::XF_LO_CLAMP;
    }
    if (x0 + 2 >= nx) {
        g.oc = 0;
        g.xfix |= g.has1 ? f32::XF_HI_CLAMP : f32::XF_HI_ODD1;
    } else if (x0 + 3 == nx) {
        g.xfix |= f32::XF_HI_ODD3;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) g.yoff[k] = g.zoff[k] = 0;
    return g;
}

// LD = f32::LD_CA for C = 1 (only this block writes the job's tubes),
// f32::LD_CG for C > 1 (the other blocks of the cluster write them too).
// The stencils are staged through shared memory by cp.async (see
// update_pair).
// MAXT = launch bound: 512 caps the kernel at 128 registers (some spill),
// 384 at 168, 256 leaves it unconstrained; the autotuner picks.
template <int LD, int MAXT, int NP>
__global__ void __launch_bounds__(MAXT, 1) tubes_kernel(const Args a)
{
    __shared__ int s_off[kMaxJobTubes], s_nx[kMaxJobTubes], s_steps[kMaxJobTubes], s_par[kMaxJobTubes];
    __shared__ int s_tube[kMaxJobTubes], s_p0[kMaxJobTubes + 1];
    __shared__ float s_eos[kMaxJobTubes], s_kb[kMaxJobTubes];
    extern __shared__ f2 s_dyn[];   // parked coefficients and staged stencils (see update_pair)

    const int C = a.cluster;
    const unsigned rank = C > 1 ? cluster_rank() : 0u;
    const int cid = C > 1 ? int(cluster_index()) : int(blockIdx.x);
    if (cid >= a.nclusters) return;   // uniform over the cluster
    const int stride = C * int(blockDim.x);
    const int base = int(rank) * int(blockDim.x) + int(threadIdx.x);

    for (int j = a.cl_start[cid]; j < a.cl_start[cid + 1]; ++j) {
        const Job J = a.jobs[j];
        __syncthreads();   // the previous job's readers of the tables are done
        if (int(threadIdx.x) < J.count) {
            const int t = a.order[J.first + threadIdx.x];
            const Tube T = a.tubes[t];
            s_tube[threadIdx.x] = t;
            s_off[threadIdx.x] = T.off;
            s_nx[threadIdx.x] = T.nx;
            s_eos[threadIdx.x] = T.eos;
            s_kb[threadIdx.x] = T.kb;
            s_steps[threadIdx.x] = a.steps[t];
            s_par[threadIdx.x] = a.par[t];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int i = 0; i < J.count; ++i) {
                s_p0[i] = acc;
                acc += (s_nx[i] + 1) >> 1;
            }
            s_p0[J.count] = acc;
        }
        __syncthreads();

        for (int s = 0; s < J.steps; ++s) {
            for (int q = base; q < J.pairs; q += stride) {
                int i = 0;
                while (i + 1 < J.count && q >= s_p0[i + 1]) ++i;
                if (s < s_steps[i]) {
                    const f32::Geo g = tube_geo(s_off[i], s_nx[i], 2 * (q - s_p0[i]));
                    const bool odd = ((s_par[i] + s) & 1) != 0;
                    const float *f = odd ? a.f1 : a.f0, *h = odd ? a.h1 : a.h0;
                    float *fo = odd ? a.f0 : a.f1, *ho = odd ? a.h0 : a.h1;
                    // the slots of the shared-memory arrays are MAXT apart (the
                    // launch bound, a compile-time constant: fixed offsets
                    // from one base address), whatever blockDim.x <= MAXT is
                    f32::update_pair<1, false, true, LD, f32::kParkOn, f32::kStageOn, NP>(
                        a.p, g, s_eos[i], s_kb[i], f, h, fo, ho, a.prev, a.ps, s_dyn + threadIdx.x, MAXT,
                        s_dyn + (f32::kParkOn ? f32::kParkSlots * MAXT : 0) + threadIdx.x, MAXT);
                }
            }
            if (C > 1) cluster_barrier();
            else __syncthreads();
        }
        if (rank == 0 && int(threadIdx.x) < J.count)
            a.par[s_tube[threadIdx.x]] = (s_par[threadIdx.x] + s_steps[threadIdx.x]) & 1;
    }
}

template <int LD, int MAXT, int NP>
cudaError_t launch_variant(const Args &a, int threads, int cluster, cudaStream_t s, int *nclusters_out)
{
    auto kern = tubes_kernel<LD, MAXT, NP>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nclusters_out ? unsigned(cluster) : unsigned(a.nclusters * cluster), 1, 1);
    cfg.blockDim = dim3(unsigned(threads), 1, 1);
    const size_t smem = f32::step_smem_bytes(MAXT, f32::kStageOn, 1);   // slots MAXT apart
    cfg.dynamicSmemBytes = smem;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
    }
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    if (cluster > 1) {
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = unsigned(cluster);
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
    }
    if (nclusters_out) {
        if (cluster > 1) return cudaOccupancyMaxActiveClusters(nclusters_out, kern, &cfg);
        int per_sm = 0, dev = 0, sms = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        *nclusters_out = per_sm * sms;
        return e;
    }
    return cudaLaunchKernelEx(&cfg, kern, a);
}

template <int LD>
cudaError_t launch_ld(const Args &a, int threads, int bound, int cluster, cudaStream_t s, int *nclusters_out)
{
    if (threads < 32 || threads > bound || threads % 32 != 0) return cudaErrorInvalidValue;
    if (a.np == 7) {
        if (bound == 256) return launch_variant<LD, 256, 7>(a, threads, cluster, s, nclusters_out);
        if (bound == 384) return launch_variant<LD, 384, 7>(a, threads, cluster, s, nclusters_out);
        if (bound == 512) return launch_variant<LD, 512, 7>(a, threads, cluster, s, nclusters_out);
        return cudaErrorInvalidValue;
    }
    if (bound == 256) return launch_variant<LD, 256, 19>(a, threads, cluster, s, nclusters_out);
    if (bound == 384) return launch_variant<LD, 384, 19>(a, threads, cluster, s, nclusters_out);
    if (bound == 512) return launch_variant<LD, 512, 19>(a, threads, cluster, s, nclusters_out);
    return cudaErrorInvalidValue;
}

}  // namespace batch
}  // namespace rlb
