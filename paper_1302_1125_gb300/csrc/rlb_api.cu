// rlb_api.cu -- the C ABI of librlb (declared in include/rlb.h): argument
// validation, device memory of a context, and the host side of every call.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/rlb.h"
#include "rlb_device.cuh"
#include "rlb_internal.h"

using rlb::StepParams;

struct rlb_ctx {
    rlb_grid grid;
    double eta_over_s, zeta_over_s, alpha;
    int limiter;
    rlb_options opt;
    int device;
    int N;
    long long ps;      // plane stride (elements)
    int dim;           // 1, 2 or 3: number of leading axes that are streamed
    int fp32;
    size_t esize;
    void *block;       // the single device allocation
    void *fbuf[2], *hbuf[2], *prev;
    unsigned *d_status;
    double *d_partial, *d_tot;
    unsigned *h_status;   // pinned
    double *h_tot;        // pinned
    int cur;
    int nsolid;           // solid cells (rlb_set_solid)
    void *solid;          // device: 3 doubles {n, T, 0}, then nsolid cell indices
    cudaStream_t stream;
    long long launches;
    StepParams sp;
    rlb::TileMaps tmaps[2];   // tensor maps of the population buffers (bulk-staged FP32 tiles)
    bool have_tmaps = false;
    bool sym_stale = false;   // symmetry reduction: the non-representative class planes are not yet refreshed
    std::string err;
};

namespace {

thread_local std::string g_err = "no error";

rlb_status fail(rlb_ctx *ctx, rlb_status st, const std::string &msg)
{
    if (ctx)
        ctx->err = msg;
    else
        g_err = msg;
    return st;
}

rlb_status cuda_fail(rlb_ctx *ctx, cudaError_t e, const char *where)
{
    return fail(ctx, RLB_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RLB_CUDA(ctx, call)                                        \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// alpha of Eq. 55 from zeta/s through Eq. 56 at the reference state
// T = 1, lambda = 1 (s = 4n, P = n): alpha = 27 (zeta/s) s / (4 P nu^6)
double alpha_from(double zeta_over_s, const rlb_options &o)
{
    if (o.alpha_override >= 0.0) return o.alpha_override;
    return rlb::alpha_of_zeta(zeta_over_s, o.model);
}

// c_0/c_t, (c_0/c_t) nu and |c_ia| of a diagonal population of a lattice
double lat_c0ct(int lat) { return lat == 1 ? rlb::Lat<1>::c0ct : rlb::Lat<0>::c0ct; }
double lat_omegaC(int lat) { return lat == 1 ? rlb::Lat<1>::omegaC : rlb::Lat<0>::omegaC; }
int lat_dmag(int lat) { return lat == 1 ? rlb::Lat<1>::dmag : rlb::Lat<0>::dmag; }

int active_axes(const rlb_grid &g)
{
    return (g.nx > 1) + (g.ny > 1) + (g.nz > 1);
}

rlb_status validate(const rlb_grid *grid, int Q, double eta_over_s, double zeta_over_s,
                    int limiter, const rlb_options &o, rlb_ctx *ctx)
{
    if (!grid) return fail(ctx, RLB_E_INVALID, "grid is NULL");
    if (Q != RLB_Q) return fail(ctx, RLB_E_INVALID, "Q must be 19 (the extended D3Q19 lattice)");
    const rlb_grid &g = *grid;
    if (g.nx < 1 || g.ny < 1 || g.nz < 1) return fail(ctx, RLB_E_INVALID, "grid dimensions must be >= 1");
    if ((long long)g.nx * g.ny * g.nz > (long long)INT_MAX)
        return fail(ctx, RLB_E_INVALID, "grid has more than 2^31 - 1 cells");
    bool inlet = false;
    for (int a = 0; a < 3; ++a) {
        for (int b : {g.bc_lo[a], g.bc_hi[a]}) {
            if (b != RLB_BC_PERIODIC && b != RLB_BC_OUTFLOW && b != RLB_BC_INLET)
                return fail(ctx, RLB_E_INVALID, "unknown boundary type");
            if (b == RLB_BC_INLET) {
                if (a != 0) return fail(ctx, RLB_E_INVALID, "inlet boundaries are supported on x faces only");
                inlet = true;
            }
        }
    }
    if (inlet) {
        const double u2 = g.inlet_u[0] * g.inlet_u[0] + g.inlet_u[1] * g.inlet_u[1] +
                          g.inlet_u[2] * g.inlet_u[2];
        if (!(g.inlet_n > 0.0) || !(g.inlet_T > 0.0) || !(u2 < 1.0) || !std::isfinite(g.inlet_n * g.inlet_T))
            return fail(ctx, RLB_E_INVALID, "inlet state must have n > 0, T > 0, |u| < 1");
    }
    if (!(eta_over_s >= 0.0) || !std::isfinite(eta_over_s))
        return fail(ctx, RLB_E_INVALID, "eta_over_s must be finite and >= 0");
    if (!(zeta_over_s >= 0.0) || !std::isfinite(zeta_over_s))
        return fail(ctx, RLB_E_INVALID, "zeta_over_s must be finite and >= 0");
    if (limiter != RLB_LIMITER_MINMOD && limiter != RLB_LIMITER_NONE)
        return fail(ctx, RLB_E_INVALID, "unknown limiter");
    if (!(o.dt_over_dx > 0.0) || !std::isfinite(o.dt_over_dx))
        return fail(ctx, RLB_E_INVALID, "dt_over_dx must be finite and > 0");
    if (o.precision != RLB_FP64 && o.precision != RLB_FP32_STORAGE)
        return fail(ctx, RLB_E_INVALID, "unknown precision");
    // the FP32 step addresses a population plane with 32-bit byte offsets
    if (o.precision == RLB_FP32_STORAGE && (long long)g.nx * g.ny * g.nz >= (1LL << 30))
        return fail(ctx, RLB_E_INVALID, "FP32-storage grids must have fewer than 2^30 cells");
    if (o.euler_mode != 0 && o.euler_mode != 1) return fail(ctx, RLB_E_INVALID, "euler_mode must be 0 or 1");
    if (o.symmetry_1d != 0 && o.symmetry_1d != 1) return fail(ctx, RLB_E_INVALID, "symmetry_1d must be 0 or 1");
    if (o.symmetry_1d) {
        if (o.euler_mode != 0) return fail(ctx, RLB_E_INVALID, "symmetry_1d needs the viscous step");
        if (g.ny != 1 || g.nz != 1)
            return fail(ctx, RLB_E_INVALID, "symmetry_1d on a grid needs a 1-D grid (ny = nz = 1)");
        if ((g.bc_lo[0] == RLB_BC_INLET || g.bc_hi[0] == RLB_BC_INLET) && (g.inlet_u[1] != 0.0 || g.inlet_u[2] != 0.0))
            return fail(ctx, RLB_E_INVALID, "symmetry_1d needs inlet_u[1] = inlet_u[2] = 0");
    }
    if (o.model != 0 && o.model != 1) return fail(ctx, RLB_E_INVALID, "model must be 0 (extended) or 1 (basic)");
    if (o.thread_mapping < 0 || o.thread_mapping > 3)
        return fail(ctx, RLB_E_INVALID,
                    "thread_mapping must be 0 (automatic), 1 (tiles), 2 (linear) or 3 (tiles, bulk-staged)");
    if (o.symmetry_2d != 0 && o.symmetry_2d != 1) return fail(ctx, RLB_E_INVALID, "symmetry_2d must be 0 or 1");
    if (o.symmetry_1d && o.symmetry_2d) return fail(ctx, RLB_E_INVALID, "symmetry_1d and symmetry_2d exclude each other");
    if (o.symmetry_2d) {
        if (o.euler_mode != 0) return fail(ctx, RLB_E_INVALID, "symmetry_2d needs the viscous step");
        if (g.nz != 1 || g.ny < 2)
            return fail(ctx, RLB_E_INVALID, "symmetry_2d needs a 2-D grid (nz = 1 < ny)");
        if ((g.bc_lo[0] == RLB_BC_INLET || g.bc_hi[0] == RLB_BC_INLET) && g.inlet_u[2] != 0.0)
            return fail(ctx, RLB_E_INVALID, "symmetry_2d needs inlet_u[2] = 0");
    }
    if (o.recovery_fp64 != 0 && o.recovery_fp64 != 1) return fail(ctx, RLB_E_INVALID, "recovery_fp64 must be 0 or 1");
    if (o.slab_rows < 0) return fail(ctx, RLB_E_INVALID, "slab_rows must be >= 0");
    if (o.recovery_fp64) {
        if (o.precision != RLB_FP32_STORAGE)
            return fail(ctx, RLB_E_INVALID, "recovery_fp64 is an option of the FP32-storage form");
        if (o.euler_mode != 0 || o.model != 0 || o.symmetry_1d || o.symmetry_2d || o.thread_mapping == 2 ||
            g.nx % 2 != 0)
            return fail(ctx, RLB_E_INVALID,
                        "recovery_fp64 needs the extended lattice, the viscous step, even nx, no symmetry "
                        "reduction and tiles");
    }
    if (!std::isfinite(o.tau_override) || !std::isfinite(o.alpha_override))
        return fail(ctx, RLB_E_INVALID, "overrides must be finite");
    // explicit stability bounds
    const int d = active_axes(g) > 0 ? active_axes(g) : 1;
    // largest sum over the streamed axes of |c_ia| c0/ct
    const double cmax = (d >= 2 ? 2.0 : 1.0) * lat_dmag(o.model) * lat_c0ct(o.model);
    if (o.dt_over_dx * cmax > 1.0)
        return fail(ctx, RLB_E_UNSTABLE, "dt/dx exceeds the Courant bound of the lattice");
    const double kb = lat_omegaC(o.model) * o.dt_over_dx * alpha_from(zeta_over_s, o);
    if (2.0 * d * kb > 1.0)
        return fail(ctx, RLB_E_UNSTABLE, "alpha dt exceeds the explicit diffusion bound");
    return RLB_OK;
}

// inlet ghost values: f^eq and h^eq of the inlet state
template <int LAT>
void inlet_ghosts(const rlb_grid &g, StepParams &sp)
{
    const double u2 = g.inlet_u[0] * g.inlet_u[0] + g.inlet_u[1] * g.inlet_u[1] +
                      g.inlet_u[2] * g.inlet_u[2];
    const double gam = 1.0 / std::sqrt(1.0 - (u2 < 1.0 ? u2 : 0.0));
    rlb::Macro m;
    m.P = g.inlet_n * g.inlet_T;
    m.ux = gam * g.inlet_u[0];
    m.uy = gam * g.inlet_u[1];
    m.uz = gam * g.inlet_u[2];
    m.n = g.inlet_n;
    rlb::Coef<double> cf, ch;
    rlb::coef_f<LAT>(m, cf);
    rlb::coef_h<LAT>(m, ch);
    const rlb::EqW<double> kf = rlb::weigh_f<double, LAT>(cf), kh = rlb::weigh_h<double, LAT>(ch);
    double *gf = sp.ghost_f, *gh = sp.ghost_h;
    [&]<int... I>(std::integer_sequence<int, I...>) {
        ((gf[I] = rlb::eq_pop<I>(kf)), ...);
        ((gh[I] = rlb::eq_pop<I>(kh)), ...);
    }(std::make_integer_sequence<int, 19>{});
}

rlb_status check_device_status(rlb_ctx *ctx, rlb_status if_bad)
{
    RLB_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    RLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const unsigned st = *ctx->h_status;
    if (st != 0u) {
        RLB_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(unsigned), ctx->stream));
        RLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (st & rlb::ST_TIMEOUT)
            return fail(ctx, RLB_E_TIMEOUT,
                        "a bounded wait of the step kernel gave up (a bulk copy of the stencil tiles did not "
                        "complete); the results of that step are not valid");
        if (st & rlb::ST_ASYMMETRIC)
            return fail(ctx, RLB_E_INVALID,
                        "symmetry reduction: the state is not its own mirror image (u_y or u_z != 0, or unequal "
                        "populations in a class)");
        return fail(ctx, if_bad, "a cell was non-physical (E <= |M|, n <= 0, |u| >= 1 or non-finite)");
    }
    return RLB_OK;
}

// symmetry reductions: the step updates the class representatives only;
// before the current level is read as 19 planes, the other members of each
// class are refreshed (one launch, skipped when nothing stepped since the
// last one)
rlb_status refresh_mirrors(rlb_ctx *ctx)
{
    if (!ctx->sp.sym || !ctx->sym_stale) return RLB_OK;
    RLB_CUDA(ctx, rlb::launch_sym(ctx->fp32, 1, ctx->sp.sym, ctx->N, ctx->ps, ctx->fbuf[ctx->cur],
                                  ctx->hbuf[ctx->cur], ctx->prev, ctx->d_status, ctx->stream));
    ctx->launches += 1;
    ctx->sym_stale = false;
    return RLB_OK;
}

}  // namespace

void rlb::set_thread_error(const char *msg)
{
    g_err = msg;
}

extern "C" {

void rlb_default_options(rlb_options *o)
{
    if (!o) return;
    o->dt_over_dx = 0.25;
    o->tau_override = 0.0;
    o->alpha_override = -1.0;
    o->euler_mode = 0;
    o->precision = RLB_FP64;
    o->cuda_stream = nullptr;
    o->symmetry_1d = 0;
    o->model = 0;
    o->thread_mapping = 0;
    o->symmetry_2d = 0;
    o->recovery_fp64 = 0;
    o->slab_rows = 0;
}

rlb_status rlb_check_config(const rlb_grid *grid, int Q, double eta_over_s, double zeta_over_s,
                            int limiter, const rlb_options *opts)
{
    rlb_options o;
    rlb_default_options(&o);
    if (opts) o = *opts;
    return validate(grid, Q, eta_over_s, zeta_over_s, limiter, o, nullptr);
}

rlb_status rlb_create(const rlb_grid *grid, int Q, double eta_over_s, double zeta_over_s,
                      int limiter, const rlb_options *opts, rlb_ctx **out)
{
    if (!out) return fail(nullptr, RLB_E_INVALID, "out is NULL");
    *out = nullptr;
    rlb_options o;
    rlb_default_options(&o);
    if (opts) o = *opts;
    rlb_status st = validate(grid, Q, eta_over_s, zeta_over_s, limiter, o, nullptr);
    if (st != RLB_OK) return st;

    rlb_ctx *ctx = new (std::nothrow) rlb_ctx();
    if (!ctx) return fail(nullptr, RLB_E_NOMEM, "host allocation failed");
    ctx->grid = *grid;
    ctx->eta_over_s = eta_over_s;
    ctx->zeta_over_s = zeta_over_s;
    ctx->limiter = limiter;
    ctx->opt = o;
    ctx->alpha = alpha_from(zeta_over_s, o);
    ctx->N = grid->nx * grid->ny * grid->nz;
    ctx->ps = (long long)align_up((size_t)ctx->N, 64);
    ctx->dim = grid->nz > 1 ? 3 : (grid->ny > 1 ? 2 : 1);
    ctx->fp32 = o.precision == RLB_FP32_STORAGE;
    ctx->esize = ctx->fp32 ? 4 : 8;
    ctx->stream = (cudaStream_t)o.cuda_stream;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) {
        delete ctx;
        return cuda_fail(nullptr, e, "cudaGetDevice");
    }

    const size_t plane = (size_t)ctx->ps * ctx->esize;
    const int nb = rlb::totals_blocks(ctx->N);
    size_t off = 0;
    size_t offs[8];
    offs[0] = off; off += align_up(19 * plane, 256);   // f0
    offs[1] = off; off += align_up(19 * plane, 256);   // h0
    offs[2] = off; off += align_up(19 * plane, 256);   // f1
    offs[3] = off; off += align_up(19 * plane, 256);   // h1
    offs[4] = off; off += align_up(5 * plane, 256);    // prev
    offs[5] = off; off += 256;                          // status
    offs[6] = off; off += align_up(5 * sizeof(double) * nb, 256);   // partial sums
    offs[7] = off; off += 256;                          // totals
    e = cudaMalloc(&ctx->block, off);
    if (e != cudaSuccess) {
        delete ctx;
        return fail(nullptr, RLB_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    char *b = (char *)ctx->block;
    ctx->fbuf[0] = b + offs[0];
    ctx->hbuf[0] = b + offs[1];
    ctx->fbuf[1] = b + offs[2];
    ctx->hbuf[1] = b + offs[3];
    ctx->prev = b + offs[4];
    ctx->d_status = (unsigned *)(b + offs[5]);
    ctx->d_partial = (double *)(b + offs[6]);
    ctx->d_tot = (double *)(b + offs[7]);
    e = cudaMallocHost(&ctx->h_status, sizeof(unsigned) + 8 * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(ctx->block);
        delete ctx;
        return fail(nullptr, RLB_E_NOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    }
    ctx->h_tot = (double *)((char *)ctx->h_status + 8);
    e = cudaMemsetAsync(ctx->block, 0, off, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        rlb_destroy(ctx);
        return cuda_fail(nullptr, e, "cudaMemset");
    }

    StepParams &sp = ctx->sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.nx = grid->nx;
    sp.ny = grid->ny;
    sp.nz = grid->nz;
    sp.ps = ctx->ps;
    for (int a = 0; a < 3; ++a) {
        sp.bc_lo[a] = grid->bc_lo[a];
        sp.bc_hi[a] = grid->bc_hi[a];
    }
    sp.half_lim = limiter == RLB_LIMITER_MINMOD ? 0.5 : 0.0;
    sp.lat = o.model;
    sp.mapping = o.thread_mapping;
    sp.slab_by = o.slab_rows > 0 ? o.slab_rows : rlb::f32_slab_rows(grid->nx, grid->ny);
    sp.sym = o.symmetry_1d ? 1 : (o.symmetry_2d ? 2 : 0);
    sp.k1 = lat_c0ct(o.model) * o.dt_over_dx;
    sp.k2 = double(lat_dmag(o.model)) * lat_c0ct(o.model) * o.dt_over_dx;
    sp.kw = lat_omegaC(o.model) * o.dt_over_dx;
    sp.kbulk = lat_omegaC(o.model) * o.dt_over_dx * ctx->alpha;
    sp.eta_over_s = eta_over_s;
    sp.tau_override = o.tau_override;
    sp.status = ctx->d_status;
    if (o.model == 1) inlet_ghosts<1>(*grid, sp);
    else inlet_ghosts<0>(*grid, sp);
    sp.f_k1 = float(sp.k1);
    sp.f_k2 = float(sp.k2);
    sp.f_half_lim = float(sp.half_lim);
    sp.f_kw = float(sp.kw);
    sp.f_kbulk = float(sp.kbulk);
    sp.f_eta_over_s = float(sp.eta_over_s);
    sp.f_tau_override = float(sp.tau_override);
    for (int i = 0; i < 19; ++i) {
        sp.f_ghost_f[i] = float(sp.ghost_f[i]);
        sp.f_ghost_h[i] = float(sp.ghost_h[i]);
    }
    // the bulk-staged FP32 tiles copy the centre rows and z-neighbour planes
    // as tensor-map boxes; without the maps the per-thread staged kernel runs
    if (ctx->fp32 && !o.recovery_fp64 && rlb::f32_bulk_eligible(sp, ctx->dim, o.euler_mode)) {
        ctx->have_tmaps = rlb::make_tile_maps(sp, (const float *)ctx->fbuf[0], (const float *)ctx->hbuf[0],
                                              &ctx->tmaps[0]) == cudaSuccess &&
                          rlb::make_tile_maps(sp, (const float *)ctx->fbuf[1], (const float *)ctx->hbuf[1],
                                              &ctx->tmaps[1]) == cudaSuccess;
    }
    ctx->cur = 0;
    ctx->err = "no error";
    *out = ctx;
    return RLB_OK;
}

rlb_status rlb_init(rlb_ctx *ctx, const double *n, const double *T, const double *ux,
                    const double *uy, const double *uz, int on_device)
{
    if (!ctx) return fail(nullptr, RLB_E_INVALID, "ctx is NULL");
    if (!n || !T || !ux || !uy || !uz) return fail(ctx, RLB_E_INVALID, "a field pointer is NULL");
    RLB_CUDA(ctx, cudaSetDevice(ctx->device));
    const size_t bytes = sizeof(double) * (size_t)ctx->N;
    const double *src[5] = {n, T, ux, uy, uz};
    const double *dev[5];
    if (on_device) {
        for (int k = 0; k < 5; ++k) dev[k] = src[k];
    } else {
        // stage through the idle population buffer (38 ps esize >= 40 N bytes)
        double *stage = (double *)ctx->fbuf[1 - ctx->cur];
        for (int k = 0; k < 5; ++k) {
            RLB_CUDA(ctx, cudaMemcpyAsync(stage + (size_t)k * ctx->N, src[k], bytes, cudaMemcpyHostToDevice,
                                          ctx->stream));
            dev[k] = stage + (size_t)k * ctx->N;
        }
    }
    RLB_CUDA(ctx, rlb::launch_init(ctx->fp32, ctx->N, ctx->ps, dev[0], dev[1], dev[2], dev[3], dev[4],
                                   ctx->fbuf[ctx->cur], ctx->hbuf[ctx->cur], ctx->prev, ctx->d_status,
                                   ctx->stream, ctx->sp.lat, ctx->sp.sym));
    ctx->launches += 1;
    ctx->sym_stale = false;
    return check_device_status(ctx, RLB_E_INVALID);
}

rlb_status rlb_step(rlb_ctx *ctx, long long nsteps)
{
    if (!ctx) return fail(nullptr, RLB_E_INVALID, "ctx is NULL");
    if (nsteps < 0) return fail(ctx, RLB_E_INVALID, "nsteps must be >= 0");
    RLB_CUDA(ctx, cudaSetDevice(ctx->device));
    if (nsteps > 0 && ctx->sp.sym) ctx->sym_stale = true;   // set first: a failed launch may follow steps that ran
    for (long long k = 0; k < nsteps; ++k) {
        const int c = ctx->cur, o = 1 - c;
        cudaError_t e;
        if (ctx->fp32 && ctx->opt.recovery_fp64)
            e = rlb::launch_step_f32_rec64(ctx->sp, ctx->dim, (const float *)ctx->fbuf[c],
                                           (const float *)ctx->hbuf[c], (float *)ctx->fbuf[o],
                                           (float *)ctx->hbuf[o], (float *)ctx->prev, ctx->stream);
        else if (ctx->fp32)
            e = rlb::launch_step_f32(ctx->sp, ctx->dim, ctx->opt.euler_mode, (const float *)ctx->fbuf[c],
                                     (const float *)ctx->hbuf[c], (float *)ctx->fbuf[o], (float *)ctx->hbuf[o],
                                     (float *)ctx->prev, ctx->stream, ctx->have_tmaps ? &ctx->tmaps[c] : nullptr);
        else
            e = rlb::launch_step_f64(ctx->sp, ctx->dim, ctx->opt.euler_mode, (const double *)ctx->fbuf[c],
                                     (const double *)ctx->hbuf[c], (double *)ctx->fbuf[o],
                                     (double *)ctx->hbuf[o], (double *)ctx->prev, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "step kernel launch");
        ctx->launches += 1;
        ctx->cur = o;
        if (ctx->nsolid > 0) {
            RLB_CUDA(ctx, rlb::launch_solid_reset(ctx->fp32, ctx->nsolid, (const int *)((double *)ctx->solid + 3),
                                                  ctx->ps, (const double *)ctx->solid, ctx->fbuf[o], ctx->hbuf[o],
                                                  ctx->prev, ctx->d_status, ctx->stream, ctx->sp.lat));
            ctx->launches += 1;
        }
    }
    return check_device_status(ctx, RLB_E_NONPHYSICAL);
}

rlb_status rlb_set_solid(rlb_ctx *ctx, const unsigned char *mask, double n, double T, int on_device)
{
    if (!ctx) return fail(nullptr, RLB_E_INVALID, "ctx is NULL");
    RLB_CUDA(ctx, cudaSetDevice(ctx->device));
    RLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->solid) cudaFree(ctx->solid);
    ctx->solid = nullptr;
    ctx->nsolid = 0;
    if (!mask) return RLB_OK;
    if (!(n > 0.0) || !(T > 0.0) || !std::isfinite(n * T))
        return fail(ctx, RLB_E_INVALID, "the solid state needs n > 0 and T > 0");
    std::vector<unsigned char> hm;
    const unsigned char *m = mask;
    if (on_device) {
        hm.resize((size_t)ctx->N);
        RLB_CUDA(ctx, cudaMemcpy(hm.data(), mask, (size_t)ctx->N, cudaMemcpyDeviceToHost));
        m = hm.data();
    }
    std::vector<int> idx;
    for (int i = 0; i < ctx->N; ++i)
        if (m[i]) idx.push_back(i);
    if (idx.empty()) return RLB_OK;
    const size_t bytes = 3 * sizeof(double) + sizeof(int) * idx.size();
    cudaError_t e = cudaMalloc(&ctx->solid, bytes);
    if (e != cudaSuccess) {
        ctx->solid = nullptr;
        return fail(ctx, RLB_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    const double st[3] = {n, T, 0.0};
    RLB_CUDA(ctx, cudaMemcpy(ctx->solid, st, sizeof(st), cudaMemcpyHostToDevice));
    RLB_CUDA(ctx, cudaMemcpy((double *)ctx->solid + 3, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice));
    ctx->nsolid = int(idx.size());
    const int c = ctx->cur;
    RLB_CUDA(ctx, rlb::launch_solid_reset(ctx->fp32, ctx->nsolid, (const int *)((double *)ctx->solid + 3), ctx->ps,
                                          (const double *)ctx->solid, ctx->fbuf[c], ctx->hbuf[c], ctx->prev,
                                          ctx->d_status, ctx->stream, ctx->sp.lat));
    ctx->launches += 1;
    return check_device_status(ctx, RLB_E_INVALID);
}

rlb_status rlb_macroscopic(rlb_ctx *ctx, double *out, int on_device)
{
    if (!ctx) return fail(nullptr, RLB_E_INVALID, "ctx is NULL");
    if (!out) return fail(ctx, RLB_E_INVALID, "out is NULL");
    RLB_CUDA(ctx, cudaSetDevice(ctx->device));
    if (rlb_status st = refresh_mirrors(ctx); st != RLB_OK) return st;
    double *dst = on_device ? out : (double *)ctx->fbuf[1 - ctx->cur];   // 48 N bytes of staging
    RLB_CUDA(ctx, rlb::launch_macro(ctx->fp32, ctx->N, ctx->ps, ctx->fbuf[ctx->cur], ctx->hbuf[ctx->cur],
                                    dst, ctx->d_status, ctx->stream, ctx->sp.lat));
    ctx->launches += 1;
    if (!on_device)
        RLB_CUDA(ctx, cudaMemcpyAsync(out, dst, 6 * sizeof(double) * (size_t)ctx->N, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    return check_device_status(ctx, RLB_E_NONPHYSICAL);
}

rlb_status rlb_conserved_totals(rlb_ctx *ctx, double *out)
{
    if (!ctx) return fail(nullptr, RLB_E_INVALID, "ctx is NULL");
    if (!out) return fail(ctx, RLB_E_INVALID, "out is NULL");
    RLB_CUDA(ctx, cudaSetDevice(ctx->device));
    if (rlb_status st = refresh_mirrors(ctx); st != RLB_OK) return st;
    RLB_CUDA(ctx, rlb::launch_totals(ctx->fp32, ctx->N, ctx->ps, ctx->fbuf[ctx->cur], ctx->hbuf[ctx->cur],
                                     ctx->d_partial, ctx->d_tot, ctx->stream, ctx->sp.lat));
    ctx->launches += 2;
    RLB_CUDA(ctx, cudaMemcpyAsync(ctx->h_tot, ctx->d_tot, 5 * sizeof(double), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    RLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < 5; ++k) out[k] = ctx->h_tot[k];
    return RLB_OK;
}

size_t rlb_state_bytes(const rlb_ctx *ctx)
{
    return ctx ? (size_t)43 * ctx->N * ctx->esize : 0;
}

static rlb_status copy_state(rlb_ctx *ctx, void *buf, size_t bytes, bool out)
{
    if (!ctx) return fail(nullptr, RLB_E_INVALID, "ctx is NULL");
    if (!buf) return fail(ctx, RLB_E_INVALID, "buffer is NULL");
    if (bytes != rlb_state_bytes(ctx)) return fail(ctx, RLB_E_INVALID, "buffer size must equal rlb_state_bytes");
    RLB_CUDA(ctx, cudaSetDevice(ctx->device));
    if (out) {
        if (rlb_status st = refresh_mirrors(ctx); st != RLB_OK) return st;
    }
    const size_t w = (size_t)ctx->N * ctx->esize, pitch = (size_t)ctx->ps * ctx->esize;
    char *host = (char *)buf;
    void *dev[3] = {ctx->fbuf[ctx->cur], ctx->hbuf[ctx->cur], ctx->prev};
    const int rows[3] = {19, 19, 5};
    size_t hoff = 0;
    for (int k = 0; k < 3; ++k) {
        if (out)
            RLB_CUDA(ctx, cudaMemcpy2DAsync(host + hoff, w, dev[k], pitch, w, rows[k], cudaMemcpyDefault,
                                            ctx->stream));
        else
            RLB_CUDA(ctx, cudaMemcpy2DAsync(dev[k], pitch, host + hoff, w, w, rows[k], cudaMemcpyDefault,
                                            ctx->stream));
        hoff += w * rows[k];
    }
    RLB_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (!out && ctx->sp.sym) {
        // a reduction steps the class representatives only: every member of
        // a class must equal its representative
        ctx->sym_stale = false;
        RLB_CUDA(ctx, rlb::launch_sym(ctx->fp32, 0, ctx->sp.sym, ctx->N, ctx->ps, ctx->fbuf[ctx->cur],
                                      ctx->hbuf[ctx->cur], ctx->prev, ctx->d_status, ctx->stream));
        ctx->launches += 1;
        return check_device_status(ctx, RLB_E_INVALID);
    }
    return RLB_OK;
}

rlb_status rlb_get_state(rlb_ctx *ctx, void *buf, size_t bytes, int on_device)
{
    (void)on_device;   // cudaMemcpyDefault resolves host and device pointers (UVA)
    return copy_state(ctx, buf, bytes, true);
}

rlb_status rlb_set_state(rlb_ctx *ctx, const void *buf, size_t bytes, int on_device)
{
    (void)on_device;
    return copy_state(ctx, const_cast<void *>(buf), bytes, false);
}

rlb_status rlb_set_stream(rlb_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return fail(nullptr, RLB_E_INVALID, "ctx is NULL");
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->opt.cuda_stream = cuda_stream;
    return RLB_OK;
}

long long rlb_launch_count(const rlb_ctx *ctx)
{
    return ctx ? ctx->launches : 0;
}

void rlb_destroy(rlb_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    if (ctx->block) cudaFree(ctx->block);
    if (ctx->solid) cudaFree(ctx->solid);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    delete ctx;
}

const char *rlb_last_error(const rlb_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_err.c_str();
}

const char *rlb_step_kernel(const rlb_ctx *ctx)
{
    if (!ctx) return "none";
    if (ctx->fp32) {
        if (ctx->opt.recovery_fp64) return "fp32_rec64";
        return rlb::f32_step_kernel_name(ctx->sp, ctx->dim, ctx->opt.euler_mode, ctx->have_tmaps);
    }
    return rlb::f64_step_kernel_name(ctx->sp, ctx->dim);
}

const char *rlb_status_string(int status)
{
    switch (status) {
    case RLB_OK: return "RLB_OK";
    case RLB_E_INVALID: return "RLB_E_INVALID";
    case RLB_E_NOMEM: return "RLB_E_NOMEM";
    case RLB_E_CUDA: return "RLB_E_CUDA";
    case RLB_E_UNSTABLE: return "RLB_E_UNSTABLE";
    case RLB_E_NONPHYSICAL: return "RLB_E_NONPHYSICAL";
    case RLB_E_TIMEOUT: return "RLB_E_TIMEOUT";
    default: return "RLB_E_UNKNOWN";
    }
}

}  // extern "C"
