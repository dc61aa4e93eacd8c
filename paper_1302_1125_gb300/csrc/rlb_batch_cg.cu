// Batched tube kernel, one cluster of blocks per job (loads cached in L2
// only; see rlb_batch.cuh).
#include "rlb_batch.cuh"

namespace rlb {
namespace batch {

cudaError_t launch_tubes_cg(const Args &a, int threads, int bound, int cluster, cudaStream_t s,
                            int *nclusters_out)
{
    return launch_ld<f32::LD_CG>(a, threads, bound, cluster, s, nclusters_out);
}

}  // namespace batch
}  // namespace rlb
