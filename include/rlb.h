/*
 * rlb.h -- C ABI of librlb, a GB300 (sm_103a) implementation of the fused
 * time step of the ultra-relativistic lattice Boltzmann (RLB) method of
 * Mohseni, Mendoza, Succi and Herrmann, "Lattice Boltzmann model for
 * ultra-relativistic flows" (arXiv:1302.1125).
 *
 * One time step (Sec. II.A, Eq. 57, with the number distribution of Eq. 58)
 * runs as one kernel per cell update: minmod flux-limited upwind streaming of
 * the 19 populations of f and of h (Eqs. 47-53), the bulk-viscosity Laplacian
 * on f (Eqs. 54-55), the moment sums T^{0 mu} and N^0 (Eq. 36), the
 * Landau-frame recovery of n, e, u (eps = 3P, Eq. 38), the second-order
 * equilibria f^eq (matched to Eq. 36) and h^eq (Eq. 58), and the implicit
 * (Mei-Shyy) BGK/Marle update with the extrapolated equilibrium
 * 2 f^eq(t) - f^eq(t - dt).
 *
 * Units and lattice.  Lattice units: delta x = 1, c = k_B = 1, temperatures
 * in units of a reference temperature.  The global lattice constant is
 * nu = sqrt(13), so c_a = sqrt(13)/nu = 1 and c_t/c_0 = sqrt(27/13) (Eq. 46);
 * the weights are those of Eqs. 43-45 and 59-60.  Population order:
 *   0        rest
 *   1..6     c_a (+x, -x, +y, -y, +z, -z)
 *   7..10    2 c_a (x, y) with signs (+,+) (+,-) (-,+) (-,-)
 *   11..14   2 c_a (x, z) with signs (+,+) (+,-) (-,+) (-,-)
 *   15..18   2 c_a (y, z) with signs (+,+) (+,-) (-,+) (-,-)
 *
 * Layout.  Cell index idx = x + nx * (y + ny * z) (x fastest).  Every field
 * passed through this ABI is structure-of-arrays: component k of cell idx is
 * at [k * N + idx] with N = nx * ny * nz.
 *
 * Ownership.  The context owns all device memory it allocates (populations,
 * previous-level macroscopic fields, status word, reduction scratch); the
 * caller owns every buffer it passes in and keeps ownership after the call.
 * Pointers flagged on_device = 1 are device pointers in the current CUDA
 * context; on_device = 0 means host memory (pageable or pinned).
 *
 * Errors.  No function throws or aborts.  Each returns an rlb_status; the
 * text of the last error of a context is available from rlb_last_error.
 * Device-side problems (a non-physical state, E <= |M| or non-finite; under
 * a symmetry reduction, a state that is not symmetric) are recorded in a
 * device status word and reported by the next call that synchronises
 * (rlb_init, rlb_step, rlb_macroscopic, rlb_set_state).
 *
 * Streams.  All work of a context is issued on the CUDA stream given in
 * rlb_options.cuda_stream (NULL = the legacy default stream).
 */
#ifndef RLB_H
#define RLB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RLB_Q 19

#if defined(__GNUC__)
#define RLB_API __attribute__((visibility("default")))
#else
#define RLB_API
#endif

typedef struct rlb_ctx rlb_ctx;

typedef enum {
    RLB_OK = 0,
    RLB_E_INVALID = -1,      /* bad argument: Q != 19, bad dims, null pointer, bad enum */
    RLB_E_NOMEM = -2,        /* device allocation failed */
    RLB_E_CUDA = -3,         /* a CUDA call failed (message in rlb_last_error) */
    RLB_E_UNSTABLE = -4,     /* dt/dx or alpha outside the explicit stability bounds */
    RLB_E_NONPHYSICAL = -5,  /* a cell had E <= |M| or a non-finite value */
    RLB_E_TIMEOUT = -6       /* a bounded device-side wait gave up */
} rlb_status;

enum { RLB_LIMITER_MINMOD = 0, RLB_LIMITER_NONE = 1 };  /* NONE: first-order upwind */
enum { RLB_BC_PERIODIC = 0, RLB_BC_OUTFLOW = 1, RLB_BC_INLET = 2 };
enum { RLB_FP64 = 0, RLB_FP32_STORAGE = 1 };

/* Grid and boundaries (Sec. III).  bc_lo/bc_hi per axis x, y, z:
 * PERIODIC wraps; OUTFLOW is the paper's open end (zero gradient: the ghost
 * cells repeat the edge cell); INLET (x faces only) holds the ghost cells at
 * the equilibrium of the state (inlet_n, inlet_T, inlet_u), as the paper's
 * inlet of Sec. III does. */
typedef struct {
    int nx, ny, nz;
    int bc_lo[3], bc_hi[3];
    double inlet_n, inlet_T, inlet_u[3];
} rlb_grid;

typedef struct {
    double dt_over_dx;       /* delta t / delta x (default 0.25) */
    double tau_override;     /* > 0: one relaxation time tau everywhere */
    double alpha_override;   /* >= 0: bulk coefficient alpha of Eq. 55 directly */
    int euler_mode;          /* 1: f <- f^eq, h <- h^eq of the streamed state (Sec. III) */
    int precision;           /* RLB_FP64 or RLB_FP32_STORAGE */
    void *cuda_stream;       /* cudaStream_t, NULL = legacy default stream */
    int symmetry_1d;         /* 1: exact 1-D symmetry reduction, for batched tubes and for
                              * grids with ny = nz = 1 (either precision, viscous step).  With
                              * u_y = u_z = 0 and fields uniform in y and z, populations with
                              * the same weight and the same c_x stay equal, leaving 7 classes
                              * per distribution (rest, +x, -x, the y/z axis populations, the
                              * diagonals with c_x = +2, with c_x = -2, the y-z diagonals); the
                              * step updates one plane per class (14 population planes and 3
                              * previous-level planes instead of 38 and 5).  On a grid
                              * rlb_init rejects u_y or u_z != 0 and rlb_set_state a state
                              * whose class members differ; rlb_macroscopic,
                              * rlb_conserved_totals and rlb_get_state see all 19 planes.
                              * Results equal the 19-population step up to the rounding order
                              * of the moment sums. */
    int model;               /* lattice: 0 the extended D3Q19 configuration (Sec. II.A, diagonals
                              * 2 c_a, nu = sqrt(13)); 1 the basic D3Q19 lattice of Sec. II
                              * (diagonals c_a, nu = sqrt(19) so c_a = 1, weights -44/361, 99/722,
                              * 9/361, number weights 1/3, 1/18, 1/36).  The step is the same
                              * (Eq. 57) on either; grids only (batched tubes: model 0). */
    int thread_mapping;      /* grids of 2 or 3 dimensions: how threads cover the grid.  0:
                              * automatic (tiles when they fill at least 97 % of their lanes,
                              * else the linear order); 1: tiles (FP32 storage: 32 x 8 threads
                              * of two x-adjacent cells each, 64 x 8 cells; FP64: 32 x 4 cells),
                              * the better reuse of y-neighbours in L1; 2: linear, one block per
                              * run of consecutive cells (pairs) of the x-fastest order, no idle
                              * lanes whatever nx and ny; 3: tiles, and in the FP32-storage form
                              * on grids that allow it (3-D, viscous, extended lattice, nx a
                              * multiple of 64, ny of 8, x faces not periodic) the block stages
                              * each population's stencil tile into shared memory by tensor-map
                              * bulk copies instead of each thread staging its own, when the
                              * driver provides the tensor-map encoder (see rlb_step_kernel).
                              * The results are the same bit for bit. */
    int symmetry_2d;         /* 1 (grids with nz = 1 < ny, either precision, viscous step): exact 2-D
                              * symmetry reduction.  With u_z = 0 in every cell (and at the
                              * inlet) the state is its own mirror image in z, so mirror-image
                              * populations stay equal: 14 classes per distribution (rest, +x,
                              * -x, +y, -y, {+z, -z}, the four x-y diagonals, (+x, +-z),
                              * (-x, +-z), (+y, +-z), (-y, +-z)); the step updates one plane per
                              * class (28 population planes and 4 previous-level planes instead
                              * of 38 and 5).  rlb_init rejects a state with u_z != 0 and
                              * rlb_set_state one whose mirror-image populations differ;
                              * rlb_macroscopic, rlb_conserved_totals and rlb_get_state see
                              * all 19 planes.  Results equal the 19-population step up to the
                              * rounding order of the moment sums. */
    int recovery_fp64;       /* RLB_FP32_STORAGE only.  1: the Landau-frame recovery of Sec. II (Eq. 38 with
                              * eps = 3P) of both time levels runs in FP64 arithmetic, from the exact double
                              * values of the double-float moment sums.  0 (default): E^2 - |M|^2 is formed in
                              * double-float and the rest of the recovery, well conditioned once E^2 - |M|^2 is
                              * known, in float.  Both reach the accuracy that the rounding of the stored FP32
                              * populations allows (relative error of P up to about gamma^2 x 2.6e-7 for
                              * either); the FP64 form costs FP64 instructions, which GB300 issues at 1/64 of
                              * the float rate.  Supported with the extended lattice, the viscous step, even nx
                              * and no symmetry reduction; the threads always take tiles (1-D grids: the 1-D
                              * form).  rlb_create rejects other combinations with RLB_E_INVALID. */
    int slab_rows;           /* RLB_FP32_STORAGE, 3-D grids, tiles: the order in which the blocks of
                              * 64 x 8 cells start.  They take the grid in slabs of slab_rows block
                              * rows (8 slab_rows cell rows), every z-plane of one slab before the
                              * next slab, so that the z-neighbour planes the resident blocks read
                              * stay in L2 for the blocks of the next planes.  0 (default): the
                              * slab height whose one z-plane holds about 10 MB of f and h
                              * (16 block rows at nx = 512); a value >= the grid's block rows:
                              * the plain x, y, z order.  The results are the same bit for bit
                              * whatever the order.  Must be >= 0; batched tubes: must be 0. */
} rlb_options;

/* Fill *opts with the defaults: dt/dx 0.25, no overrides, viscous mode, FP64,
 * default stream, no symmetry reduction, the extended lattice, automatic
 * thread mapping, double-float recovery (recovery_fp64 = 0), automatic slab
 * height (slab_rows = 0). */
RLB_API void rlb_default_options(rlb_options *opts);

/* Validate a configuration on the host without touching the GPU.  Same
 * arguments and checks as rlb_create.  Rules: Q must be 19 (the extended
 * lattice of Sec. II.A, Eq. 42); nx, ny, nz >= 1 and N < 2^31 (N < 2^30 in
 * the FP32-storage form, which needs about 330 GB at 2^30); eta_over_s,
 * zeta_over_s >= 0; INLET only on x faces with n > 0, T > 0, |u| < 1;
 * RLB_E_UNSTABLE if dt/dx times the largest sum over moving axes of
 * |c_ia| c_0/c_t of the chosen lattice exceeds 1, or if 2 d (c_0 nu / c_t) dt alpha exceeds 1
 * (d = number of axes with more than one cell, at least 1).  These bounds are
 * necessary, not sufficient: the time scheme takes damping away from sound
 * waves as dt/dx grows, so with little viscosity and alpha = 0 they can grow
 * inside the bounds: long sound waves stay damped only below about
 * dt/dx = 0.21 tau.  The alpha term restores the damping. */
RLB_API rlb_status rlb_check_config(const rlb_grid *grid, int Q, double eta_over_s,
                            double zeta_over_s, int limiter, const rlb_options *opts);

/* Create a context for one grid.  eta_over_s sets tau per cell through
 * Eq. 41 with the entropy s = n (4 - ln lambda) of Sec. III (the factor
 * 4 - ln lambda floored at 1e-3); zeta_over_s sets alpha through Eq. 56 at the
 * reference state T = 1, lambda = 1 (alpha = 27 (zeta/s) / nu^6, 0.0123 zeta/s
 * on the extended lattice) unless opts->alpha_override >= 0.
 * The step itself (limited-flux streaming, implicit collision) realises a
 * shear viscosity proportional to tau with no -1/2 shift: 0.2369 P tau
 * (extended lattice) or 0.1621 P tau (basic), larger along face diagonals;
 * and the alpha term diffuses momentum with 2.50 alpha (extended) per unit
 * time, adding a viscosity 2.50 alpha (e + P).  Eq. 56 does not describe
 * that term: the sound damping it adds is about 12 times less than the bulk
 * viscosity 4 P alpha nu^6 / 27 would give.  So zeta/s acts only through
 * this small alpha: at zeta/s <= 0.1, alpha <= 1.2e-3, far below the
 * alpha = 0.15 .. 0.2 the paper's runs use for stability.  To set the term
 * that keeps fast flows physical, give alpha_override. 
 * opts may be NULL (defaults).  Allocates 2 x 38 population planes, 5
 * previous-level planes and scratch on the device; *out receives the handle
 * (NULL on failure).  Errors: RLB_E_INVALID, RLB_E_UNSTABLE, RLB_E_NOMEM,
 * RLB_E_CUDA. */
RLB_API rlb_status rlb_create(const rlb_grid *grid, int Q, double eta_over_s, double zeta_over_s,
                      int limiter, const rlb_options *opts, rlb_ctx **out);

/* Initialise the populations to equilibrium: f = f^eq(P = n T, u) (Eq. 36 with
 * Eq. 38), h = h^eq(n, u) (Eq. 58), and the previous level to the same state
 * (so the first step uses f^eq(-dt) = f^eq(0)).  n, T, ux, uy, uz: N doubles
 * each (three-velocity components, |u| < 1), host or device memory per
 * on_device.  The FP64 form evaluates the equilibria in double; the
 * FP32-storage form in float from n T, n, u and 1 - |u|^2 rounded to float
 * (each population within a few float roundings of its double value), so it
 * also rejects states whose n, n T or 1 - |u|^2 fall outside the float range.
 * RLB_E_INVALID (the context stays usable) if a cell has n <= 0, T <= 0,
 * |u| >= 1 or a non-finite value, or, under symmetry_2d, u_z != 0.
 * Synchronous. */
RLB_API rlb_status rlb_init(rlb_ctx *ctx, const double *n, const double *T, const double *ux,
                    const double *uy, const double *uz, int on_device);

/* Advance nsteps time steps of Eq. 57 (nsteps >= 0): one step-kernel launch
 * per step (plus one solid-cell reset launch per step when rlb_set_solid
 * holds cells).  Kernels are queued on the context's stream; the call then
 * waits for them and returns
 * RLB_E_NONPHYSICAL if any cell of any step was non-physical (the status word
 * is then cleared). */
RLB_API rlb_status rlb_step(rlb_ctx *ctx, long long nsteps);

/* Solid cells (Sec. III, the astrophysical run: a fixed cloud whose cells
 * evolve to the equilibrium of the constant state n1, T1, u = 0).  Every
 * cell with mask[idx] != 0 (mask: N bytes, host or device memory per
 * on_device) is set to f^eq(P = n T, u = 0), h^eq(n, u = 0) and the previous
 * level of that state, now and after every later step, in a separate kernel
 * over the solid cells' index list (the step kernel itself is unchanged).
 * A call replaces the previous set; mask = NULL removes it.  RLB_E_INVALID
 * for n <= 0 or T <= 0; RLB_E_NOMEM if the index list cannot be allocated.
 * Synchronous. */
RLB_API rlb_status rlb_set_solid(rlb_ctx *ctx, const unsigned char *mask, double n, double T,
                                 int on_device);

/* Macroscopic fields of the current populations (Sec. II: moments and the
 * Landau-frame recovery): out holds 6 N doubles, planes n, e, u_x, u_y, u_z,
 * gamma.  Synchronous.  Under a symmetry reduction this call, like
 * rlb_conserved_totals and rlb_get_state, first refreshes the planes the
 * step leaves to the class representatives (one launch, once after steps). */
RLB_API rlb_status rlb_macroscopic(rlb_ctx *ctx, double *out, int on_device);

/* Grid totals of T^00, T^0x, T^0y, T^0z and N^0 (sums over cells of the
 * moments of Eq. 36), in FP64, deterministic order.  out: 5 host doubles.
 * Uses the context's device reduction scratch.  Synchronous. */
RLB_API rlb_status rlb_conserved_totals(rlb_ctx *ctx, double *out);

/* Size in bytes of a checkpoint: 19 N f values, 19 N h values and 5 N
 * previous-level values, each 8 bytes (RLB_FP64) or 4 bytes
 * (RLB_FP32_STORAGE), in that order, compact planes of N.  The previous
 * level is the macroscopic state of the last step, (P, u'_x, u'_y, u'_z, n)
 * with u' = gamma u, for RLB_FP64, and its raw moment sums (sum_i f_i,
 * sum_i c_ix f_i, sum_i c_iy f_i, sum_i c_iz f_i, sum_i h_i; c_i the integer
 * lattice vectors) for RLB_FP32_STORAGE, which keeps the extrapolated
 * equilibrium's moments exact in float. */
RLB_API size_t rlb_state_bytes(const rlb_ctx *ctx);

/* Copy the full state out / in (checkpoint and resume).  bytes must equal
 * rlb_state_bytes.  A resumed run continues bit for bit.  Synchronous.
 * Under a symmetry reduction rlb_set_state returns RLB_E_INVALID when a
 * population differs from its class representative (the state must be
 * symmetric; it is copied in all the same). */
RLB_API rlb_status rlb_get_state(rlb_ctx *ctx, void *buf, size_t bytes, int on_device);
RLB_API rlb_status rlb_set_state(rlb_ctx *ctx, const void *buf, size_t bytes, int on_device);

/* Change the stream later calls use (cudaStream_t, NULL = legacy default). */
RLB_API rlb_status rlb_set_stream(rlb_ctx *ctx, void *cuda_stream);

/* Number of kernels this context has launched since creation. */
RLB_API long long rlb_launch_count(const rlb_ctx *ctx);

/* Release every device buffer of the context.  NULL is a no-op. */
RLB_API void rlb_destroy(rlb_ctx *ctx);

/* Text of the last error of ctx (or of the calling thread when ctx is NULL,
 * e.g. after a failed rlb_create).  Never NULL. */
RLB_API const char *rlb_last_error(const rlb_ctx *ctx);

/* Name of a status code. */
RLB_API const char *rlb_status_string(int status);

/* Name of the step kernel rlb_step launches for this context (a
 * diagnostic; the paper has no counterpart): "fp32_bulk_tiles" (FP32
 * storage on 3-D grids whose stencil tiles are staged by block-wide bulk
 * copies: thread_mapping 3, viscous step, extended lattice, nx a multiple
 * of 64, ny of 8, x faces not periodic, tensor maps made at rlb_create),
 * "fp32_tiles" (tiles of
 * 64 x 8 cells, each thread loading its own stencil, staged by asynchronous
 * copies in the viscous step), "fp32_linear", "fp32_1d", "fp32_rec64" (recovery_fp64),
 * "fp64_tiles", "fp64_linear", "fp64_small" (blocks of one to four warps
 * on grids with fewer cells than one block per SM), "fp64_1d".  The
 * results are the same whichever kernel runs.  NULL ctx: "none". */
RLB_API const char *rlb_step_kernel(const rlb_ctx *ctx);

/* Grid totals without any allocation.  The paper has no counterpart: this
 * serves callers that cannot call cudaMalloc, for example an application
 * whose allocator or memory pool reserves all device memory up front, or a
 * loop that cannot afford the device-wide synchronisation that cudaMalloc
 * and cudaFree imply.  It computes the same sums as rlb_conserved_totals
 * (T^00, T^0x, T^0y, T^0z, N^0 over all cells, FP64, same order) from the
 * caller's buffers: f and h are device pointers to 19 planes each of N
 * values (float for RLB_FP32_STORAGE, double for RLB_FP64), consecutive
 * planes plane_stride elements apart (plane_stride >= N, e.g. the compact
 * layout of rlb_get_state has plane_stride = N); out_device is a
 * caller-owned device buffer of 5 doubles, written asynchronously on
 * cuda_stream (NULL = legacy default stream).
 * The sums take p_i = (xi0, c_i) of the extended lattice (model 0).
 * The reduction's per-block partial sums live in a fixed device array of
 * 5 x RLB_NOALLOC_MAX_BLOCKS doubles (47.5 KiB) inside the library, which
 * every GPU that loads the library holds until the process exits.  The
 * first call on a device looks up that array's address on the current
 * device (cudaGetSymbolAddress) and keeps it for the life of the process;
 * make that first call before any stream capture.  Do not use this entry
 * point on a device after cudaDeviceReset in the same process: the reset
 * unloads the library's device code, the array may come back at another
 * address, and the kept address would then be stale.  All calls on a device
 * share the array: calls whose kernels
 * overlap on the GPU (different streams, no ordering between them) race and
 * give wrong totals.  Nothing in the array needs clearing between calls;
 * every slot a call reads it has written first.  Calls no cudaMalloc,
 * cudaFree or other allocating routine.
 * Errors: RLB_E_INVALID for a NULL pointer, N < 1, N > RLB_NOALLOC_MAX_CELLS,
 * plane_stride < N or an unknown precision (message in rlb_last_error(NULL));
 * RLB_E_CUDA if the address lookup or the launch fails. */
#define RLB_NOALLOC_MAX_BLOCKS 1216
#define RLB_NOALLOC_MAX_CELLS 2146959360
RLB_API rlb_status rlb_conserved_totals_noalloc(const void *f, const void *h, int N,
                                                long long plane_stride, int precision,
                                                double *out_device, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Batched tubes.
 *
 * B independent one-dimensional tubes (grid nx_b x 1 x 1 each, zero-gradient
 * outflow at both ends: the paper's open ends, Sec. III), each with its own
 * length, eta/s and zeta/s, advanced by the step of Eq. 57 in the
 * FP32-storage form (the same per-cell arithmetic as rlb_step with
 * RLB_FP32_STORAGE).  One persistent kernel runs every tube for its own
 * number of steps; a CUDA graph replays that launch.
 *
 * Work division: tubes are grouped into jobs (one tube, or up to 32
 * consecutive tubes of similar length and step count) and each job is run,
 * all of its steps, by one cluster of `cluster` thread blocks that meet at
 * the hardware cluster barrier (the block barrier for cluster = 1) after
 * every step.  Jobs are assigned to the clusters that fit on the GPU at once,
 * longest first, each to the least loaded cluster (rlb_batch_plan).
 *
 * Packed layout of every field passed through this part of the ABI: tube b
 * holds cells [o_b, o_b + nx_b) with o_0 = 0, o_{b+1} = o_b + nx_b; total =
 * o_B cells.  Ownership, streams and errors as above; rlb_batch_last_error
 * gives the text of the last error of a batch (of the thread for NULL).
 * ------------------------------------------------------------------------ */
typedef struct rlb_batch rlb_batch;

/* Launch shape of the persistent tube kernel. */
typedef struct {
    int threads;           /* threads per block: a multiple of 32, <= bound */
    int bound;             /* kernel variant by launch bound: 512 (128 registers per thread),
                            * 384 (168) or 256 (unconstrained) threads */
    int cluster;           /* blocks per cluster sharing one job: 1, 2, 4 or 8 */
    int pairs_per_thread;  /* job capacity: consecutive tubes are grouped while their cell pairs
                            * fit in cluster x threads x pairs_per_thread (a longer tube is a job
                            * of its own); each thread updates two adjacent cells per pass */
    double ms;             /* rlb_batch_autotune: measured time of the trial in ms, -1 = did not run */
} rlb_batch_tuning;

/* Create a batch of B tubes (1 <= B <= 65535): nx[b] >= 1 cells,
 * eta_over_s[b] and zeta_over_s[b] >= 0 (tau through Eq. 41 and alpha
 * through Eq. 56 per tube, as in rlb_create; opts->alpha_override >= 0 sets
 * one alpha for all tubes).  opts may be NULL: defaults of
 * rlb_default_options with precision RLB_FP32_STORAGE.  Requirements:
 * precision RLB_FP32_STORAGE, euler_mode 0, model 0, recovery_fp64 0, symmetry_1d 0 or 1 (the
 * tubes are 1-D with u_y = u_z = 0, so the reduction is exact; thread_mapping
 * and symmetry_2d do not apply to tubes and are ignored), at most 2^30 stored cells
 * (each tube stored from a 128-byte boundary).  RLB_E_UNSTABLE if
 * 2 (c_0/c_t) dt/dx > 1 or 2 (c_0 nu / c_t) dt alpha_b > 1 for a tube.
 * Allocates 81 population and previous-level planes over the stored cells
 * plus staging and tables (about 324 B per cell + 48 B per cell of
 * staging).  *out receives the handle (NULL on failure; message in
 * rlb_batch_last_error(NULL)). */
RLB_API rlb_status rlb_batch_create(int B, const int *nx, const double *eta_over_s,
                                    const double *zeta_over_s, int limiter, const rlb_options *opts,
                                    rlb_batch **out);

/* Initialise every tube to equilibrium (as rlb_init): n, T, ux are packed
 * arrays of `total` doubles (three-velocity along the tube, |u| < 1).
 * RLB_E_INVALID if a cell has n <= 0, T <= 0 or |u| >= 1.  Synchronous. */
RLB_API rlb_status rlb_batch_init(rlb_batch *b, const double *n, const double *T, const double *ux,
                                  int on_device);

/* Advance tube b by nsteps[b] steps of Eq. 57 (host array of B counts in
 * [0, 2^31 - 1]; 0 leaves a tube unchanged) in one launch of the persistent
 * kernel, replayed from a CUDA graph.  The job plan is rebuilt when the step
 * counts or the tuning change.  Waits for the launch and returns
 * RLB_E_NONPHYSICAL if any cell of any step was non-physical. */
RLB_API rlb_status rlb_batch_step(rlb_batch *b, const long long *nsteps);

/* Macroscopic fields of every tube (as rlb_macroscopic): out holds 6 x total
 * doubles, planes n, e, u_x, u_y, u_z, gamma, each packed.  Synchronous. */
RLB_API rlb_status rlb_batch_macroscopic(rlb_batch *b, double *out, int on_device);

/* Per-tube totals of T^00, T^0x, T^0y, T^0z and N^0 (Eq. 36 summed over the
 * tube's cells, FP64, deterministic order): out[5 b + k], 5 B host doubles.
 * Synchronous. */
RLB_API rlb_status rlb_batch_totals(rlb_batch *b, double *out);

/* The job plan of a launch, computed on the host without a GPU (the plan
 * rlb_batch_step uploads).  Tubes with nsteps > 0 are ordered by step count,
 * then length, both descending (ties by index); consecutive tubes are
 * grouped into jobs while a job has fewer than 32 tubes and its cell pairs
 * (ceil(nx / 2) per tube) fit in t->cluster x t->threads x
 * t->pairs_per_thread; a job's cost is its largest step count x
 * ceil(pairs / (cluster x threads)) passes; jobs are taken in decreasing
 * cost and each is given to the cluster with the least cost so far (lowest
 * index on ties).  Outputs: order[B] (tube ids; tubes with no steps last),
 * jobs[4 x njobs] as (first position in order, tube count, steps, pairs),
 * grouped by cluster with cluster c owning jobs cl_start[c] ..
 * cl_start[c + 1] - 1 (cl_start has nclusters + 1 entries), *critical = the
 * largest per-cluster cost (NULL to skip).  jobs must hold 4 B ints.
 * RLB_E_INVALID for bad arguments (message in rlb_batch_last_error(NULL)). */
RLB_API rlb_status rlb_batch_plan(int B, const int *nx, const long long *nsteps,
                                  const rlb_batch_tuning *t, int nclusters, int *order, int *jobs,
                                  int *njobs, int *cl_start, long long *critical);

/* Autotuner: time the launch shapes on this batch and keep the fastest.
 * Each trial restores the state, runs ceil(nsteps[b] / divisor) steps per
 * tube in one launch and is timed with CUDA events; the candidates are every
 * (bound, threads <= bound) of {512, 384, 256} x {128, 256, 384, 512} with
 * clusters 1, 2, 4, 8 and pairs_per_thread 1, then pairs_per_thread 2 and 4
 * for the best of those.  The state is restored at the end (the tuning run
 * does not advance the batch).  trials (max_trials entries, may be NULL
 * when max_trials = 0) receives the trials in order with their times,
 * *n_trials their number; *best the one kept.  Needs a temporary device
 * buffer the size of the state (RLB_E_NOMEM if it cannot be had). */
RLB_API rlb_status rlb_batch_autotune(rlb_batch *b, const long long *nsteps, int divisor,
                                      rlb_batch_tuning *trials, int max_trials, int *n_trials,
                                      rlb_batch_tuning *best);

/* Set or read the launch shape (RLB_E_INVALID if it is malformed or does not
 * fit on the device).  *resident_clusters (may be NULL) receives how many
 * clusters of that shape the device holds at once: the persistent grid. */
RLB_API rlb_status rlb_batch_set_tuning(rlb_batch *b, const rlb_batch_tuning *t);
RLB_API rlb_status rlb_batch_get_tuning(const rlb_batch *b, rlb_batch_tuning *t,
                                        int *resident_clusters);

/* Change the stream later calls use (cudaStream_t, NULL = legacy default). */
RLB_API rlb_status rlb_batch_set_stream(rlb_batch *b, void *cuda_stream);

/* total = sum of nx_b (0 for NULL). */
RLB_API long long rlb_batch_total_cells(const rlb_batch *b);

/* Kernels this batch has launched (a graph replay counts as one). */
RLB_API long long rlb_batch_launch_count(const rlb_batch *b);

/* Release the batch's device and pinned memory.  NULL is a no-op. */
RLB_API void rlb_batch_destroy(rlb_batch *b);

/* Text of the last error of b (of the calling thread for NULL).  Never NULL. */
RLB_API const char *rlb_batch_last_error(const rlb_batch *b);

#ifdef __cplusplus
}
#endif
#endif /* RLB_H */
