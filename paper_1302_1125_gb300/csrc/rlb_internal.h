// rlb_internal.h -- host/device interface between the C ABI (rlb_api.cu) and
// the kernel translation units.  Not part of the public ABI.
#pragma once

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
    // float copies for the FP32-storage kernel (no FP64 conversion on device)
    float f_k1, f_k2, f_half_lim, f_kw, f_kbulk, f_eta_over_s, f_tau_override;
    float f_ghost_f[19], f_ghost_h[19];
};

// launchers (kernel translation units); dim = 1, 2 or 3, euler = 0/1
cudaError_t launch_step_f64(const StepParams &p, int dim, int euler, const double *f, const double *h,
                            double *fo, double *ho, double *prev, cudaStream_t s);
cudaError_t launch_step_f32(const StepParams &p, int dim, int euler, const float *f, const float *h,
                            float *fo, float *ho, float *prev, cudaStream_t s);

cudaError_t launch_init(int fp32, int N, long long ps, const double *n, const double *T,
                        const double *ux, const double *uy, const double *uz, void *f, void *h,
                        void *prev, unsigned *status, cudaStream_t s);
cudaError_t launch_macro(int fp32, int N, long long ps, const void *f, const void *h, double *out,
                         unsigned *status, cudaStream_t s);
// partial holds 5 * totals_blocks(N) doubles; out 5 doubles (device)
int totals_blocks(int N);
cudaError_t launch_totals(int fp32, int N, long long ps, const void *f, const void *h,
                          double *partial, double *out, cudaStream_t s);

// set the text rlb_last_error(NULL) returns on this thread
void set_thread_error(const char *msg);

}  // namespace rlb
