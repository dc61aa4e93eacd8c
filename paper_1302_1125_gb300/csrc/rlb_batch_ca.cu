// Batched tube kernel, one block per job (loads cached in L1; see rlb_batch.cuh).
#include "rlb_batch.cuh"

namespace rlb {
namespace batch {

cudaError_t launch_tubes_ca(const Args &a, int threads, int bound, cudaStream_t s, int *nclusters_out)
{
    return launch_ld<f32::LD_CA>(a, threads, bound, 1, s, nclusters_out);
}

}  // namespace batch
}  // namespace rlb
