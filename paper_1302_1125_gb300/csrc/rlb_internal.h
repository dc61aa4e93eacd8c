// rlb_internal.h -- host/device interface between the C ABI (rlb_api.cu) and
// the kernel translation units.  Not part of the public ABI.
#pragma once

#include <cuda.h>   // CUtensorMap (the type only; the encoder is fetched from the driver at run time)
#include <cuda_runtime.h>

namespace rlb {

// Parameters of one step launch (passed by value to the kernel).
struct StepParams {
    int nx, ny, nz;
    long long ps;            // plane stride in elements (>= N, 64-aligned)
    int bc_lo[3], bc_hi[3];
    double half_lim;         // 0.5 for the minmod limiter, 0 for first-order upwind
    double k1, k2;           // (c0/ct) dt |c_ia| for |c_ia| = 1 and 2: streaming prefactors
    double kw;               // (c0/ct) nu dt: omega = kw / tau (Eq. 57)
    double kbulk;            // (c0/ct) nu dt alpha dx: bulk prefactor (Eqs. 55, 57)
    double eta_over_s;
    double tau_override;     // > 0: fixed tau
    double ghost_f[19], ghost_h[19];   // inlet equilibria
    unsigned *status;        // device status word (bit 0: non-physical cell)
    int lat;                 // lattice: 0 extended (Sec. II.A), 1 basic (Sec. II)
    int mapping;             // grids: 0 automatic, 1 tiles, 2 linear, 3 tiles staged by block-wide bulk
                             // copies where eligible (rlb_options.thread_mapping)
    int sym;                 // grids: exact symmetry reduction, 1 on 1-D grids (7 planes per
                             // distribution), 2 on 2-D grids (14 planes: mirror images in z), 0 none
    int slab_by;             // FP32 3-D tiles: blocks are taken in slabs of this many block rows,
                             // z-planes in order within a slab (>= the block rows: x, y, z order)
    // float copies for the FP32-storage kernel (no FP64 conversion on device)
    float f_k1, f_k2, f_half_lim, f_kw, f_kbulk, f_eta_over_s, f_tau_override;
    float f_ghost_f[19], f_ghost_h[19];
};

// Tensor maps of one buffer of f and h planes (x, y, z, population), with
// boxes of a tile's centre rows (72 x 12) and of one z-neighbour plane
// (64 x 8), for the bulk-staged FP32 step
struct TileMaps {
    CUtensorMap fc, fz, hc, hz;
};

// launchers (kernel translation units); dim = 1, 2 or 3, euler = 0/1; the
// step kernels take the lattice from p.lat, the others from lat (0 extended,
// 1 basic)
cudaError_t launch_step_f64(const StepParams &p, int dim, int euler, const double *f, const double *h,
                            double *fo, double *ho, double *prev, cudaStream_t s);
cudaError_t launch_step_f32(const StepParams &p, int dim, int euler, const float *f, const float *h,
                            float *fo, float *ho, float *prev, cudaStream_t s, const TileMaps *maps = nullptr);
// the FP32-storage step on eligible 3-D grids with its stencil tiles staged by
// bulk copies (rlb_step_f32_bulk.cu); it needs the tensor maps of the buffers
// it reads (launch_step_f32 runs the per-thread staged kernel without them)
bool f32_bulk_eligible(const StepParams &p, int dim, int euler);
// encode the maps of the planes at f and h (cudaSuccess, or the failure)
cudaError_t make_tile_maps(const StepParams &p, const float *f, const float *h, TileMaps *out);
cudaError_t launch_step_f32_bulk(const StepParams &p, const float *f, const float *h, float *fo, float *ho,
                                 float *prev, const TileMaps *maps, cudaStream_t s);
// block rows per slab of the FP32 3-D tiled step (StepParams::slab_by)
int f32_slab_rows(int nx, int ny);
// name of the step kernel launch_step_f64 / launch_step_f32 picks for p (see rlb_step_kernel)
const char *f64_step_kernel_name(const StepParams &p, int dim);
const char *f32_step_kernel_name(const StepParams &p, int dim, int euler, bool have_maps);
// the FP32-storage step with the FP64 recovery (rlb_options.recovery_fp64)
cudaError_t launch_step_f32_rec64(const StepParams &p, int dim, const float *f, const float *h, float *fo,
                                  float *ho, float *prev, cudaStream_t s);

cudaError_t launch_init(int fp32, int N, long long ps, const double *n, const double *T,
                        const double *ux, const double *uy, const double *uz, void *f, void *h,
                        void *prev, unsigned *status, cudaStream_t s, int lat = 0, int sym = 0);
// symmetry reductions of grids (sym = 1: 1-D, 2: 2-D; float or double
// planes per fp32): expand = 1 copies each class representative's plane into
// its members' and zeroes the previous level's entries that vanish (the y and
// z, or the z, components); expand = 0 sets ST_ASYMMETRIC in *status where a
// member differs from its representative
cudaError_t launch_sym(int fp32, int expand, int sym, int N, long long ps, void *f, void *h, void *prev,
                       unsigned *status, cudaStream_t s);
cudaError_t launch_macro(int fp32, int N, long long ps, const void *f, const void *h, double *out,
                         unsigned *status, cudaStream_t s, int lat = 0);
// partial holds 5 * totals_blocks(N) doubles; out 5 doubles (device)
int totals_blocks(int N);
cudaError_t launch_totals(int fp32, int N, long long ps, const void *f, const void *h,
                          double *partial, double *out, cudaStream_t s, int lat = 0);

// solid cells: the M cells idx[0..M) are set to the equilibrium of the
// state st = {n, T, 0} (device doubles) in f, h and the previous level
cudaError_t launch_solid_reset(int fp32, int M, const int *idx, long long ps, const double *st, void *f,
                               void *h, void *prev, unsigned *status, cudaStream_t s, int lat = 0);

// set the text rlb_last_error(NULL) returns on this thread
void set_thread_error(const char *msg);

// ---------------------------------------------------------------------------
// Batched tubes (rlb_batch.cuh): tables the host builds for the persistent
// launch.
// ---------------------------------------------------------------------------
namespace batch {

constexpr int kMaxJobTubes = 32;   // tubes per job
constexpr int kAlignCells = 32;    // tube storage offsets are multiples of this (128 B)

struct Tube {
    int off;     // storage offset of cell 0 in every plane (multiple of kAlignCells)
    int nx;      // cells
    float eos;   // eta/s
    float kb;    // bulk prefactor (c0/ct) nu dt alpha (Eq. 57)
};

struct Job {
    int first;   // position in the tube order of the job's first tube
    int count;   // tubes in the job (1 .. kMaxJobTubes)
    int steps;   // steps the job runs: the largest step count of its tubes
    int pairs;   // sum over its tubes of ceil(nx / 2)
};

struct Args {
    StepParams p;           // constants shared by all tubes, status word
    const Tube *tubes;      // [B]
    const int *order;       // [B] tube ids, the order jobs refer to
    const int *steps;       // [B] steps of each tube in this launch
    int *par;               // [B] buffer (0 or 1) holding each tube's current level
    const Job *jobs;        // jobs of cluster c: [cl_start[c], cl_start[c + 1])
    const int *cl_start;    // [nclusters + 1]
    int nclusters;
    int cluster;            // blocks per cluster
    int np;                 // planes updated per distribution: 19, or 7 under the 1-D symmetry reduction
    float *f0, *h0, *f1, *h1, *prev;
    long long ps;
};

// launch the persistent tube kernel (grid = a.nclusters x cluster blocks of
// `threads`), or, when nclusters_out is non-NULL, store the number of clusters
// that fit on the device at once instead of launching.  bound = the kernel
// variant's launch bound (256, 384 or 512 threads; threads <= bound).
cudaError_t launch_tubes(const Args &a, int threads, int bound, int cluster, cudaStream_t s,
                         int *nclusters_out);
cudaError_t launch_tubes_ca(const Args &a, int threads, int bound, cudaStream_t s, int *nclusters_out);
cudaError_t launch_tubes_cg(const Args &a, int threads, int bound, int cluster, cudaStream_t s,
                            int *nclusters_out);

// packed fields <-> tube storage; pack[b] = first packed index of tube b
cudaError_t launch_tubes_init(int B, int max_nx, const Tube *tubes, const long long *pack, long long ps,
                              const double *n, const double *T, const double *ux, float *f, float *h,
                              float *prev, unsigned *status, cudaStream_t s);
cudaError_t launch_tubes_macro(int B, int max_nx, const Tube *tubes, const long long *pack, const int *par,
                               long long ps, long long total, const float *f0, const float *h0,
                               const float *f1, const float *h1, double *out, unsigned *status,
                               cudaStream_t s);
// 1-D symmetry reduction: copy every class representative's plane into the
// planes of the other populations of its class, in each tube's current
// buffer, so that the full 19-population state is consistent again
cudaError_t launch_tubes_expand(int B, int max_nx, const Tube *tubes, const int *par, long long ps, float *f0,
                                float *h0, float *f1, float *h1, cudaStream_t s);
// per-tube totals of T^00, T^0x, T^0y, T^0z, N^0: out[5 b + k]
cudaError_t launch_tubes_totals(int B, const Tube *tubes, const int *par, long long ps, const float *f0,
                                const float *h0, const float *f1, const float *h1, double *out,
                                cudaStream_t s);

}  // namespace batch

}  // namespace rlb
