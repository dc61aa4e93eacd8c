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
 * Device-side problems (a non-physical state, E <= |M| or non-finite) are
 * recorded in a device status word and reported by the next call that
 * synchronises (rlb_step, rlb_macroscopic).
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
} rlb_options;

/* Fill *opts with the defaults: dt/dx 0.25, no overrides, viscous mode, FP64,
 * default stream. */
RLB_API void rlb_default_options(rlb_options *opts);

/* Validate a configuration on the host without touching the GPU.  Same
 * arguments and checks as rlb_create.  Rules: Q must be 19 (the extended
 * lattice of Sec. II.A, Eq. 42); nx, ny, nz >= 1 and N < 2^31; eta_over_s,
 * zeta_over_s >= 0; INLET only on x faces with n > 0, T > 0, |u| < 1;
 * RLB_E_UNSTABLE if dt/dx times the largest sum over moving axes of
 * |c_ia| c_0/c_t exceeds 1, or if 2 d (c_0 nu / c_t) dt alpha exceeds 1
 * (d = number of axes with more than one cell). */
RLB_API rlb_status rlb_check_config(const rlb_grid *grid, int Q, double eta_over_s,
                            double zeta_over_s, int limiter, const rlb_options *opts);

/* Create a context for one grid.  eta_over_s sets tau per cell through
 * Eq. 41 with the entropy s = n (4 - ln lambda) of Sec. III (the factor
 * 4 - ln lambda floored at 1e-3); zeta_over_s sets alpha through Eq. 56 at the
 * reference state T = 1, lambda = 1 unless opts->alpha_override >= 0.
 * opts may be NULL (defaults).  Allocates 2 x 38 population planes, 5
 * previous-level planes and scratch on the device; *out receives the handle
 * (NULL on failure).  Errors: RLB_E_INVALID, RLB_E_UNSTABLE, RLB_E_NOMEM,
 * RLB_E_CUDA. */
RLB_API rlb_status rlb_create(const rlb_grid *grid, int Q, double eta_over_s, double zeta_over_s,
                      int limiter, const rlb_options *opts, rlb_ctx **out);

/* Initialise the populations to equilibrium: f = f^eq(P = n T, u) (Eq. 36 with
 * Eq. 38), h = h^eq(n, u) (Eq. 58), and the previous level to the same state
 * (so the first step uses f^eq(-dt) = f^eq(0)).  n, T, ux, uy, uz: N doubles
 * each (three-velocity components, |u| < 1).  Synchronous. */
RLB_API rlb_status rlb_init(rlb_ctx *ctx, const double *n, const double *T, const double *ux,
                    const double *uy, const double *uz, int on_device);

/* Advance nsteps time steps of Eq. 57 (nsteps >= 0).  Kernels are queued on
 * the context's stream; the call then waits for them and returns
 * RLB_E_NONPHYSICAL if any cell of any step was non-physical (the status word
 * is then cleared). */
RLB_API rlb_status rlb_step(rlb_ctx *ctx, long long nsteps);

/* Macroscopic fields of the current populations (Sec. II: moments and the
 * Landau-frame recovery): out holds 6 N doubles, planes n, e, u_x, u_y, u_z,
 * gamma.  Synchronous. */
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
 * rlb_state_bytes.  A resumed run continues bit for bit.  Synchronous. */
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
 * The reduction's per-block partial sums live in a fixed device array of
 * 5 x RLB_NOALLOC_MAX_BLOCKS doubles (47.5 KiB) inside the library, which
 * every GPU that loads the library holds until the process exits.  The
 * first call on a device looks up that array's address on the current
 * device (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls on a device share the array: calls whose kernels
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

#ifdef __cplusplus
}
#endif
#endif /* RLB_H */
