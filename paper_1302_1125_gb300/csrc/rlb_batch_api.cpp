// rlb_batch_api.cpp -- host side of the batched-tube ABI (include/rlb.h):
// validation, tube storage, the job plan of the persistent launch, the CUDA
// graph that replays it, and the autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <queue>
#include <string>
#include <vector>

#include "../../include/rlb.h"
#include "rlb_consts.h"
#include "rlb_internal.h"

using rlb::StepParams;
using rlb::batch::Job;
using rlb::batch::Tube;

struct rlb_batch {
    int B = 0;
    int limiter = 0;
    rlb_options opt{};
    int device = 0;
    int sms = 0;
    std::vector<int> nx;
    std::vector<long long> pack;     // B + 1 packed offsets
    std::vector<Tube> tubes;
    long long total = 0;             // sum of nx
    long long ps = 0;                // plane stride (elements)
    int max_nx = 0;
    int max_clusters = 0;            // capacity of the cluster table
    void *block = nullptr;
    float *f0 = nullptr, *h0 = nullptr, *f1 = nullptr, *h1 = nullptr, *prev = nullptr;
    size_t state_bytes = 0;          // f0 .. prev, contiguous from f0
    double *stage = nullptr;         // 6 x total doubles
    Tube *d_tubes = nullptr;
    long long *d_pack = nullptr;
    int *d_par = nullptr, *d_steps = nullptr, *d_order = nullptr, *d_cl = nullptr;
    Job *d_jobs = nullptr;
    unsigned *d_status = nullptr;
    double *d_tot = nullptr;
    void *host = nullptr;            // pinned staging
    unsigned *h_status = nullptr;
    int *h_steps = nullptr, *h_order = nullptr, *h_cl = nullptr;
    Job *h_jobs = nullptr;
    double *h_tot = nullptr;
    rlb_batch_tuning tune{};
    int nclusters = 0;               // clusters resident at once for `tune`
    bool plan_ok = false;
    std::vector<long long> plan_steps;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    long long launches = 0;
    StepParams sp{};
    std::string err = "no error";
};

namespace {

thread_local std::string g_berr = "no error";

rlb_status bfail(rlb_batch *b, rlb_status st, const std::string &msg)
{
    if (b) b->err = msg;
    else {
        g_berr = msg;
        rlb::set_thread_error(msg.c_str());
    }
    return st;
}

rlb_status bcuda(rlb_batch *b, cudaError_t e, const char *where)
{
    return bfail(b, RLB_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define RLB_BCUDA(b, call)                                      \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return bcuda((b), e_, #call);    \
    } while (0)

size_t aup(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool valid_tuning(const rlb_batch_tuning &t, std::string &why)
{
    if (t.bound != 256 && t.bound != 384 && t.bound != 512) {
        why = "tuning.bound must be 256, 384 or 512";
        return false;
    }
    if (t.threads < 32 || t.threads > t.bound || t.threads % 32 != 0) {
        why = "tuning.threads must be a multiple of 32 in [32, bound]";
        return false;
    }
    if (t.cluster != 1 && t.cluster != 2 && t.cluster != 4 && t.cluster != 8) {
        why = "tuning.cluster must be 1, 2, 4 or 8";
        return false;
    }
    if (t.pairs_per_thread < 1 || t.pairs_per_thread > 64) {
        why = "tuning.pairs_per_thread must be in [1, 64]";
        return false;
    }
    return true;
}

// the job plan (see rlb_batch_plan in rlb.h)
struct Plan {
    std::vector<int> order;
    std::vector<Job> jobs;       // grouped by cluster
    std::vector<int> cl_start;   // nclusters + 1
    long long critical = 0;
};

rlb_status make_plan(int B, const int *nx, const long long *steps, const rlb_batch_tuning &t, int nclusters,
                     Plan &pl, std::string &why)
{
    if (B < 1 || !nx || !steps) {
        why = "B < 1 or a NULL array";
        return RLB_E_INVALID;
    }
    if (!valid_tuning(t, why)) return RLB_E_INVALID;
    if (nclusters < 1) {
        why = "nclusters must be >= 1";
        return RLB_E_INVALID;
    }
    for (int i = 0; i < B; ++i) {
        if (nx[i] < 1) {
            why = "every tube needs nx >= 1";
            return RLB_E_INVALID;
        }
        if (steps[i] < 0 || steps[i] > INT_MAX) {
            why = "step counts must be in [0, 2^31 - 1]";
            return RLB_E_INVALID;
        }
    }
    // longest-running first: steps, then length, then id
    std::vector<int> ids(B);
    for (int i = 0; i < B; ++i) ids[i] = i;
    std::stable_sort(ids.begin(), ids.end(), [&](int a, int b) {
        if (steps[a] != steps[b]) return steps[a] > steps[b];
        return nx[a] > nx[b];
    });
    pl.order = ids;
    // group consecutive tubes into jobs of at most cap pairs
    const long long per_pass = (long long)t.cluster * t.threads;
    const long long cap = per_pass * t.pairs_per_thread;
    std::vector<Job> jobs;
    for (int k = 0; k < B; ++k) {
        const int id = ids[k];
        if (steps[id] == 0) break;
        const int pairs = (nx[id] + 1) / 2;
        if (!jobs.empty()) {
            Job &J = jobs.back();
            if (J.count < rlb::batch::kMaxJobTubes && (long long)J.pairs + pairs <= cap) {
                J.count += 1;
                J.pairs += pairs;
                continue;
            }
        }
        jobs.push_back(Job{k, 1, int(steps[id]), pairs});
    }
    // longest processing time first, each job to the least loaded cluster
    auto cost = [&](const Job &J) { return (long long)J.steps * ((J.pairs + per_pass - 1) / per_pass); };
    std::vector<int> jorder(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i) jorder[i] = int(i);
    std::stable_sort(jorder.begin(), jorder.end(), [&](int a, int b) { return cost(jobs[a]) > cost(jobs[b]); });
    using Slot = std::pair<long long, int>;   // (load, cluster)
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int c = 0; c < nclusters; ++c) heap.push({0, c});
    std::vector<int> owner(jobs.size());
    std::vector<long long> load(nclusters, 0);
    for (int j : jorder) {
        Slot s = heap.top();
        heap.pop();
        owner[j] = s.second;
        s.first += cost(jobs[j]);
        load[s.second] = s.first;
        heap.push(s);
    }
    pl.cl_start.assign(nclusters + 1, 0);
    for (size_t j = 0; j < jobs.size(); ++j) pl.cl_start[owner[j] + 1] += 1;
    for (int c = 0; c < nclusters; ++c) pl.cl_start[c + 1] += pl.cl_start[c];
    std::vector<int> fill(pl.cl_start.begin(), pl.cl_start.end() - 1);
    pl.jobs.assign(jobs.size(), Job{});
    for (int j : jorder) pl.jobs[fill[owner[j]]++] = jobs[j];
    pl.critical = 0;
    for (long long v : load) pl.critical = std::max(pl.critical, v);
    return RLB_OK;
}

rlb_status check_status(rlb_batch *b)
{
    RLB_BCUDA(b, cudaMemcpyAsync(b->h_status, b->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    RLB_BCUDA(b, cudaStreamSynchronize(b->stream));
    if (*b->h_status != 0u) {
        RLB_BCUDA(b, cudaMemsetAsync(b->d_status, 0, sizeof(unsigned), b->stream));
        RLB_BCUDA(b, cudaStreamSynchronize(b->stream));
        return bfail(b, RLB_E_NONPHYSICAL, "a cell was non-physical (E <= |M|, n <= 0, |u| >= 1 or non-finite)");
    }
    return RLB_OK;
}

rlb::batch::Args make_args(rlb_batch *b)
{
    rlb::batch::Args a;
    a.p = b->sp;
    a.tubes = b->d_tubes;
    a.order = b->d_order;
    a.steps = b->d_steps;
    a.par = b->d_par;
    a.jobs = b->d_jobs;
    a.cl_start = b->d_cl;
    a.nclusters = b->nclusters;
    a.cluster = b->tune.cluster;
    a.np = b->opt.symmetry_1d ? 7 : 19;
    a.f0 = b->f0;
    a.h0 = b->h0;
    a.f1 = b->f1;
    a.h1 = b->h1;
    a.prev = b->prev;
    a.ps = b->ps;
    return a;
}

// clusters of tuning t resident at once (0: does not fit)
rlb_status resident_clusters(rlb_batch *b, const rlb_batch_tuning &t, int &n)
{
    rlb::batch::Args a = make_args(b);
    a.cluster = t.cluster;
    n = 0;
    cudaError_t e = rlb::batch::launch_tubes(a, t.threads, t.bound, t.cluster, b->stream, &n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    if (n > b->max_clusters) n = b->max_clusters;
    return RLB_OK;
}

rlb_status upload_plan(rlb_batch *b, const long long *steps, const Plan &pl)
{
    for (int i = 0; i < b->B; ++i) b->h_steps[i] = int(steps[i]);
    std::memcpy(b->h_order, pl.order.data(), sizeof(int) * b->B);
    if (!pl.jobs.empty()) std::memcpy(b->h_jobs, pl.jobs.data(), sizeof(Job) * pl.jobs.size());
    std::memcpy(b->h_cl, pl.cl_start.data(), sizeof(int) * pl.cl_start.size());
    RLB_BCUDA(b, cudaMemcpyAsync(b->d_steps, b->h_steps, sizeof(int) * b->B, cudaMemcpyHostToDevice, b->stream));
    RLB_BCUDA(b, cudaMemcpyAsync(b->d_order, b->h_order, sizeof(int) * b->B, cudaMemcpyHostToDevice, b->stream));
    if (!pl.jobs.empty())
        RLB_BCUDA(b, cudaMemcpyAsync(b->d_jobs, b->h_jobs, sizeof(Job) * pl.jobs.size(), cudaMemcpyHostToDevice,
                                     b->stream));
    RLB_BCUDA(b, cudaMemcpyAsync(b->d_cl, b->h_cl, sizeof(int) * pl.cl_start.size(), cudaMemcpyHostToDevice,
                                 b->stream));
    return RLB_OK;
}

// plan for `steps` under the current tuning, uploaded (the host staging is
// reused only after the previous call synchronised)
rlb_status prepare(rlb_batch *b, const long long *steps)
{
    if (b->plan_ok && std::equal(b->plan_steps.begin(), b->plan_steps.end(), steps)) return RLB_OK;
    Plan pl;
    std::string why;
    rlb_status st = make_plan(b->B, b->nx.data(), steps, b->tune, b->nclusters, pl, why);
    if (st != RLB_OK) return bfail(b, st, why);
    st = upload_plan(b, steps, pl);
    if (st != RLB_OK) return st;
    b->plan_steps.assign(steps, steps + b->B);
    b->plan_ok = true;
    return RLB_OK;
}

void drop_graph(rlb_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

rlb_status apply_tuning(rlb_batch *b, const rlb_batch_tuning &t)
{
    std::string why;
    if (!valid_tuning(t, why)) return bfail(b, RLB_E_INVALID, why);
    int n = 0;
    rlb_status st = resident_clusters(b, t, n);
    if (st != RLB_OK) return st;
    if (n < 1) return bfail(b, RLB_E_INVALID, "this tuning does not fit on the device");
    b->tune = t;
    b->tune.ms = 0.0;
    b->nclusters = n;
    b->plan_ok = false;
    drop_graph(b);
    return RLB_OK;
}

rlb_status ensure_graph(rlb_batch *b)
{
    if (b->graph) return RLB_OK;
    const rlb::batch::Args a = make_args(b);
    RLB_BCUDA(b, cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = rlb::batch::launch_tubes(a, b->tune.threads, b->tune.bound, b->tune.cluster, b->cap_stream,
                                             nullptr);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(b, e != cudaSuccess ? e : e2, "capture of the tube kernel");
    }
    e = cudaGraphInstantiate(&b->graph, g, 0ULL);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bcuda(b, e, "cudaGraphInstantiate");
    }
    return RLB_OK;
}

rlb_status check_steps(rlb_batch *b, const long long *nsteps)
{
    if (!nsteps) return bfail(b, RLB_E_INVALID, "nsteps is NULL");
    for (int i = 0; i < b->B; ++i)
        if (nsteps[i] < 0 || nsteps[i] > INT_MAX)
            return bfail(b, RLB_E_INVALID, "step counts must be in [0, 2^31 - 1]");
    return RLB_OK;
}

// under the 1-D symmetry reduction only the class representatives' planes
// are current: copy them to the other populations of their classes
rlb_status expand(rlb_batch *b)
{
    if (!b->opt.symmetry_1d) return RLB_OK;
    RLB_BCUDA(b, rlb::batch::launch_tubes_expand(b->B, b->max_nx, b->d_tubes, b->d_par, b->ps, b->f0, b->h0, b->f1,
                                                 b->h1, b->stream));
    b->launches += 1;
    return RLB_OK;
}

}  // namespace

extern "C" {

rlb_status rlb_batch_plan(int B, const int *nx, const long long *nsteps, const rlb_batch_tuning *t,
                          int nclusters, int *order, int *jobs, int *njobs, int *cl_start, long long *critical)
{
    if (!t || !order || !jobs || !njobs || !cl_start) return bfail(nullptr, RLB_E_INVALID, "a NULL argument");
    Plan pl;
    std::string why;
    const rlb_status st = make_plan(B, nx, nsteps, *t, nclusters, pl, why);
    if (st != RLB_OK) return bfail(nullptr, st, why);
    std::memcpy(order, pl.order.data(), sizeof(int) * B);
    for (size_t j = 0; j < pl.jobs.size(); ++j) {
        jobs[4 * j + 0] = pl.jobs[j].first;
        jobs[4 * j + 1] = pl.jobs[j].count;
        jobs[4 * j + 2] = pl.jobs[j].steps;
        jobs[4 * j + 3] = pl.jobs[j].pairs;
    }
    *njobs = int(pl.jobs.size());
    std::memcpy(cl_start, pl.cl_start.data(), sizeof(int) * pl.cl_start.size());
    if (critical) *critical = pl.critical;
    return RLB_OK;
}

rlb_status rlb_batch_create(int B, const int *nx, const double *eta_over_s, const double *zeta_over_s,
                            int limiter, const rlb_options *opts, rlb_batch **out)
{
    if (!out) return bfail(nullptr, RLB_E_INVALID, "out is NULL");
    *out = nullptr;
    if (B < 1 || B > 65535) return bfail(nullptr, RLB_E_INVALID, "B must be in [1, 65535]");
    if (!nx || !eta_over_s || !zeta_over_s) return bfail(nullptr, RLB_E_INVALID, "a per-tube array is NULL");
    rlb_options o;
    rlb_default_options(&o);
    o.precision = RLB_FP32_STORAGE;
    if (opts) o = *opts;
    if (o.precision != RLB_FP32_STORAGE)
        return bfail(nullptr, RLB_E_INVALID, "the batched path stores populations in FP32 (RLB_FP32_STORAGE)");
    if (o.euler_mode != 0) return bfail(nullptr, RLB_E_INVALID, "the batched path runs the viscous step only");
    if (o.symmetry_1d != 0 && o.symmetry_1d != 1) return bfail(nullptr, RLB_E_INVALID, "symmetry_1d must be 0 or 1");
    if (o.model != 0) return bfail(nullptr, RLB_E_INVALID, "the batched path runs the extended lattice (model 0)");
    if (o.recovery_fp64 != 0)
        return bfail(nullptr, RLB_E_INVALID, "the batched path runs the double-float recovery (recovery_fp64 = 0)");
    if (o.slab_rows != 0) return bfail(nullptr, RLB_E_INVALID, "slab_rows is an option of grids (0 for batches)");
    if (limiter != RLB_LIMITER_MINMOD && limiter != RLB_LIMITER_NONE)
        return bfail(nullptr, RLB_E_INVALID, "unknown limiter");
    if (!(o.dt_over_dx > 0.0) || !std::isfinite(o.dt_over_dx))
        return bfail(nullptr, RLB_E_INVALID, "dt_over_dx must be finite and > 0");
    if (!std::isfinite(o.tau_override) || !std::isfinite(o.alpha_override))
        return bfail(nullptr, RLB_E_INVALID, "overrides must be finite");
    if (o.dt_over_dx * 2.0 * rlb::kC0Ct > 1.0)
        return bfail(nullptr, RLB_E_UNSTABLE, "dt/dx exceeds the Courant bound of the extended lattice");
    long long cells = 0, stored = 0;
    int max_nx = 0;
    for (int i = 0; i < B; ++i) {
        if (nx[i] < 1) return bfail(nullptr, RLB_E_INVALID, "every tube needs nx >= 1");
        if (!(eta_over_s[i] >= 0.0) || !std::isfinite(eta_over_s[i]) || !(zeta_over_s[i] >= 0.0) ||
            !std::isfinite(zeta_over_s[i]))
            return bfail(nullptr, RLB_E_INVALID, "eta_over_s and zeta_over_s must be finite and >= 0");
        const double alpha = o.alpha_override >= 0.0 ? o.alpha_override : rlb::alpha_of_zeta(zeta_over_s[i]);
        if (2.0 * rlb::kOmegaC * o.dt_over_dx * alpha > 1.0)
            return bfail(nullptr, RLB_E_UNSTABLE, "alpha dt exceeds the explicit diffusion bound");
        cells += nx[i];
        stored += (long long)aup(size_t(nx[i]), rlb::batch::kAlignCells);
        max_nx = std::max(max_nx, nx[i]);
    }
    if (stored > (1LL << 30)) return bfail(nullptr, RLB_E_INVALID, "more than 2^30 cells in the batch");

    rlb_batch *b = new (std::nothrow) rlb_batch();
    if (!b) return bfail(nullptr, RLB_E_NOMEM, "host allocation failed");
    b->B = B;
    b->limiter = limiter;
    b->opt = o;
    b->nx.assign(nx, nx + B);
    b->total = cells;
    b->max_nx = max_nx;
    b->stream = (cudaStream_t)o.cuda_stream;
    b->pack.assign(B + 1, 0);
    b->tubes.resize(B);
    long long off = 0;
    for (int i = 0; i < B; ++i) {
        b->pack[i + 1] = b->pack[i] + nx[i];
        const double alpha = o.alpha_override >= 0.0 ? o.alpha_override : rlb::alpha_of_zeta(zeta_over_s[i]);
        b->tubes[i] = Tube{int(off), nx[i], float(eta_over_s[i]), float(rlb::kOmegaC * o.dt_over_dx * alpha)};
        off += (long long)aup(size_t(nx[i]), rlb::batch::kAlignCells);
    }
    b->ps = (long long)aup(size_t(off), 64);
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess) {
        delete b;
        return bcuda(nullptr, e, "cudaGetDevice");
    }
    b->max_clusters = b->sms * 32;

    const size_t plane = size_t(b->ps) * sizeof(float);
    size_t offs[14], o2 = 0;
    offs[0] = o2; o2 += 19 * plane;                                   // f0
    offs[1] = o2; o2 += 19 * plane;                                   // h0
    offs[2] = o2; o2 += 19 * plane;                                   // f1
    offs[3] = o2; o2 += 19 * plane;                                   // h1
    offs[4] = o2; o2 += 5 * plane;                                    // prev
    b->state_bytes = o2;
    o2 = aup(o2, 256);
    offs[5] = o2; o2 = aup(o2 + sizeof(int) * B, 256);                // par (kept with the state)
    offs[6] = o2; o2 = aup(o2 + 6 * sizeof(double) * size_t(cells), 256);   // stage
    offs[7] = o2; o2 = aup(o2 + sizeof(Tube) * B, 256);
    offs[8] = o2; o2 = aup(o2 + sizeof(long long) * (B + 1), 256);
    offs[9] = o2; o2 = aup(o2 + sizeof(int) * B, 256);                // steps
    offs[10] = o2; o2 = aup(o2 + sizeof(int) * B, 256);               // order
    offs[11] = o2; o2 = aup(o2 + sizeof(Job) * B, 256);               // jobs
    offs[12] = o2; o2 = aup(o2 + sizeof(int) * (b->max_clusters + 1), 256);   // cluster table
    offs[13] = o2; o2 = aup(o2 + 256 + 5 * sizeof(double) * B, 256);  // status, totals
    e = cudaMalloc(&b->block, o2);
    if (e != cudaSuccess) {
        delete b;
        return bfail(nullptr, RLB_E_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    char *base = (char *)b->block;
    b->f0 = (float *)(base + offs[0]);
    b->h0 = (float *)(base + offs[1]);
    b->f1 = (float *)(base + offs[2]);
    b->h1 = (float *)(base + offs[3]);
    b->prev = (float *)(base + offs[4]);
    b->d_par = (int *)(base + offs[5]);
    b->stage = (double *)(base + offs[6]);
    b->d_tubes = (Tube *)(base + offs[7]);
    b->d_pack = (long long *)(base + offs[8]);
    b->d_steps = (int *)(base + offs[9]);
    b->d_order = (int *)(base + offs[10]);
    b->d_jobs = (Job *)(base + offs[11]);
    b->d_cl = (int *)(base + offs[12]);
    b->d_status = (unsigned *)(base + offs[13]);
    b->d_tot = (double *)(base + offs[13] + 256);

    const size_t hbytes = 256 + sizeof(int) * 2 * B + sizeof(Job) * B + sizeof(int) * (b->max_clusters + 1) +
                          5 * sizeof(double) * B + 64;
    e = cudaMallocHost(&b->host, hbytes);
    if (e != cudaSuccess) {
        cudaFree(b->block);
        delete b;
        return bfail(nullptr, RLB_E_NOMEM, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    }
    char *hp = (char *)b->host;
    b->h_status = (unsigned *)hp;
    b->h_tot = (double *)(hp + 64);
    b->h_jobs = (Job *)(hp + 64 + 5 * sizeof(double) * B);
    b->h_steps = (int *)((char *)b->h_jobs + sizeof(Job) * B);
    b->h_order = b->h_steps + B;
    b->h_cl = b->h_order + B;

    e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->block, 0, o2, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_tubes, b->tubes.data(), sizeof(Tube) * B, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_pack, b->pack.data(), sizeof(long long) * (B + 1), cudaMemcpyHostToDevice,
                            b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        rlb_batch_destroy(b);
        return bcuda(nullptr, e, "batch setup");
    }

    StepParams &sp = b->sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.nx = max_nx;
    sp.ny = sp.nz = 1;
    sp.ps = b->ps;
    for (int a = 0; a < 3; ++a) sp.bc_lo[a] = sp.bc_hi[a] = RLB_BC_OUTFLOW;
    sp.half_lim = limiter == RLB_LIMITER_MINMOD ? 0.5 : 0.0;
    sp.k1 = rlb::kC0Ct * o.dt_over_dx;
    sp.k2 = 2.0 * rlb::kC0Ct * o.dt_over_dx;
    sp.kw = rlb::kOmegaC * o.dt_over_dx;
    sp.tau_override = o.tau_override;
    sp.status = b->d_status;
    sp.f_k1 = float(sp.k1);
    sp.f_k2 = float(sp.k2);
    sp.f_half_lim = float(sp.half_lim);
    sp.f_kw = float(sp.kw);
    sp.f_tau_override = float(sp.tau_override);

    // a default that fits every GB300 configuration; rlb_batch_autotune
    // measures the alternatives
    rlb_batch_tuning t{256, 256, 1, 1, 0.0};
    const rlb_status st = apply_tuning(b, t);
    if (st != RLB_OK) {
        const std::string msg = b->err;
        rlb_batch_destroy(b);
        return bfail(nullptr, st, msg);
    }
    *out = b;
    return RLB_OK;
}

rlb_status rlb_batch_init(rlb_batch *b, const double *n, const double *T, const double *ux, int on_device)
{
    if (!b) return bfail(nullptr, RLB_E_INVALID, "batch is NULL");
    if (!n || !T || !ux) return bfail(b, RLB_E_INVALID, "a field pointer is NULL");
    RLB_BCUDA(b, cudaSetDevice(b->device));
    const double *dev[3] = {n, T, ux};
    if (!on_device) {
        const size_t bytes = sizeof(double) * size_t(b->total);
        for (int k = 0; k < 3; ++k) {
            RLB_BCUDA(b, cudaMemcpyAsync(b->stage + size_t(k) * b->total, dev[k], bytes, cudaMemcpyHostToDevice,
                                         b->stream));
            dev[k] = b->stage + size_t(k) * b->total;
        }
    }
    RLB_BCUDA(b, cudaMemsetAsync(b->d_par, 0, sizeof(int) * b->B, b->stream));
    RLB_BCUDA(b, rlb::batch::launch_tubes_init(b->B, b->max_nx, b->d_tubes, b->d_pack, b->ps, dev[0], dev[1], dev[2],
                                               b->f0, b->h0, b->prev, b->d_status, b->stream));
    b->launches += 1;
    const rlb_status st = check_status(b);
    return st == RLB_E_NONPHYSICAL ? bfail(b, RLB_E_INVALID, "initial state has n <= 0, T <= 0 or |u| >= 1") : st;
}

rlb_status rlb_batch_step(rlb_batch *b, const long long *nsteps)
{
    if (!b) return bfail(nullptr, RLB_E_INVALID, "batch is NULL");
    rlb_status st = check_steps(b, nsteps);
    if (st != RLB_OK) return st;
    bool any = false;
    for (int i = 0; i < b->B; ++i) any = any || nsteps[i] > 0;
    if (!any) return RLB_OK;
    RLB_BCUDA(b, cudaSetDevice(b->device));
    if ((st = prepare(b, nsteps)) != RLB_OK) return st;
    if ((st = ensure_graph(b)) != RLB_OK) return st;
    RLB_BCUDA(b, cudaGraphLaunch(b->graph, b->stream));
    b->launches += 1;
    return check_status(b);
}

rlb_status rlb_batch_macroscopic(rlb_batch *b, double *out, int on_device)
{
    if (!b) return bfail(nullptr, RLB_E_INVALID, "batch is NULL");
    if (!out) return bfail(b, RLB_E_INVALID, "out is NULL");
    RLB_BCUDA(b, cudaSetDevice(b->device));
    if (rlb_status st = expand(b); st != RLB_OK) return st;
    double *dst = on_device ? out : b->stage;
    RLB_BCUDA(b, rlb::batch::launch_tubes_macro(b->B, b->max_nx, b->d_tubes, b->d_pack, b->d_par, b->ps, b->total,
                                                b->f0, b->h0, b->f1, b->h1, dst, b->d_status, b->stream));
    b->launches += 1;
    if (!on_device)
        RLB_BCUDA(b, cudaMemcpyAsync(out, b->stage, 6 * sizeof(double) * size_t(b->total), cudaMemcpyDeviceToHost,
                                     b->stream));
    return check_status(b);
}

rlb_status rlb_batch_totals(rlb_batch *b, double *out)
{
    if (!b) return bfail(nullptr, RLB_E_INVALID, "batch is NULL");
    if (!out) return bfail(b, RLB_E_INVALID, "out is NULL");
    RLB_BCUDA(b, cudaSetDevice(b->device));
    if (rlb_status st = expand(b); st != RLB_OK) return st;
    RLB_BCUDA(b, rlb::batch::launch_tubes_totals(b->B, b->d_tubes, b->d_par, b->ps, b->f0, b->h0, b->f1, b->h1,
                                                 b->d_tot, b->stream));
    b->launches += 1;
    RLB_BCUDA(b, cudaMemcpyAsync(b->h_tot, b->d_tot, 5 * sizeof(double) * b->B, cudaMemcpyDeviceToHost, b->stream));
    RLB_BCUDA(b, cudaStreamSynchronize(b->stream));
    std::memcpy(out, b->h_tot, 5 * sizeof(double) * b->B);
    return RLB_OK;
}

rlb_status rlb_batch_set_tuning(rlb_batch *b, const rlb_batch_tuning *t)
{
    if (!b) return bfail(nullptr, RLB_E_INVALID, "batch is NULL");
    if (!t) return bfail(b, RLB_E_INVALID, "tuning is NULL");
    RLB_BCUDA(b, cudaSetDevice(b->device));
    return apply_tuning(b, *t);
}

rlb_status rlb_batch_get_tuning(const rlb_batch *b, rlb_batch_tuning *t, int *resident_clusters)
{
    if (!b || !t) return bfail(nullptr, RLB_E_INVALID, "a NULL argument");
    *t = b->tune;
    if (resident_clusters) *resident_clusters = b->nclusters;
    return RLB_OK;
}

rlb_status rlb_batch_autotune(rlb_batch *b, const long long *nsteps, int divisor, rlb_batch_tuning *trials,
                              int max_trials, int *n_trials, rlb_batch_tuning *best)
{
    if (!b) return bfail(nullptr, RLB_E_INVALID, "batch is NULL");
    rlb_status st = check_steps(b, nsteps);
    if (st != RLB_OK) return st;
    if (divisor < 1) return bfail(b, RLB_E_INVALID, "divisor must be >= 1");
    if (max_trials > 0 && !trials) return bfail(b, RLB_E_INVALID, "trials is NULL");
    RLB_BCUDA(b, cudaSetDevice(b->device));
    std::vector<long long> ts(b->B);
    for (int i = 0; i < b->B; ++i) ts[i] = (nsteps[i] + divisor - 1) / divisor;

    // snapshot of the state (populations, previous level, buffer parities)
    const size_t snap_bytes = (size_t)((char *)b->d_par - (char *)b->f0) + sizeof(int) * b->B;
    void *snap = nullptr;
    cudaError_t e = cudaMalloc(&snap, snap_bytes);
    if (e != cudaSuccess) return bfail(b, RLB_E_NOMEM, std::string("autotune snapshot: ") + cudaGetErrorString(e));
    RLB_BCUDA(b, cudaMemcpyAsync(snap, b->f0, snap_bytes, cudaMemcpyDeviceToDevice, b->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);

    const rlb_batch_tuning saved = b->tune;
    std::vector<rlb_batch_tuning> done;
    rlb_status fail_st = RLB_OK;
    std::string fail_msg;
    auto run = [&](rlb_batch_tuning t) {
        if (fail_st != RLB_OK) return;
        t.ms = -1.0;
        if (apply_tuning(b, t) == RLB_OK) {
            cudaMemcpyAsync(b->f0, snap, snap_bytes, cudaMemcpyDeviceToDevice, b->stream);
            if (prepare(b, ts.data()) == RLB_OK) {
                const rlb::batch::Args a = make_args(b);
                cudaEventRecord(e0, b->stream);
                cudaError_t le = rlb::batch::launch_tubes(a, t.threads, t.bound, t.cluster, b->stream, nullptr);
                cudaEventRecord(e1, b->stream);
                cudaError_t se = cudaStreamSynchronize(b->stream);
                if (le == cudaSuccess && se == cudaSuccess) {
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    t.ms = ms;
                } else if (se != cudaSuccess) {
                    fail_st = RLB_E_CUDA;
                    fail_msg = std::string("autotune trial: ") + cudaGetErrorString(se);
                } else {
                    cudaGetLastError();
                }
                b->launches += 1;
                if (check_status(b) != RLB_OK) t.ms = -1.0;
            }
        }
        done.push_back(t);
    };
    for (int bound : {512, 384, 256})
        for (int threads : {128, 256, 384, 512})
            if (threads <= bound)
                for (int cluster : {1, 2, 4, 8}) run(rlb_batch_tuning{threads, bound, cluster, 1, 0.0});
    auto pick = [&]() {
        int k = -1;
        for (size_t i = 0; i < done.size(); ++i)
            if (done[i].ms > 0.0 && (k < 0 || done[i].ms < done[k].ms)) k = int(i);
        return k;
    };
    int k = pick();
    if (k >= 0) {
        const rlb_batch_tuning t1 = done[k];
        for (int ppt : {2, 4}) run(rlb_batch_tuning{t1.threads, t1.bound, t1.cluster, ppt, 0.0});
        k = pick();
    }
    cudaMemcpyAsync(b->f0, snap, snap_bytes, cudaMemcpyDeviceToDevice, b->stream);
    cudaStreamSynchronize(b->stream);
    cudaFree(snap);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (fail_st != RLB_OK) return bfail(b, fail_st, fail_msg);
    if (k < 0) {
        apply_tuning(b, saved);
        return bfail(b, RLB_E_CUDA, "no tuning candidate ran");
    }
    const rlb_batch_tuning chosen = done[k];
    st = apply_tuning(b, chosen);
    if (st != RLB_OK) return st;
    b->tune.ms = chosen.ms;
    if (n_trials) *n_trials = int(done.size());
    for (int i = 0; i < max_trials && i < int(done.size()); ++i) trials[i] = done[i];
    if (best) *best = chosen;
    return RLB_OK;
}

rlb_status rlb_batch_set_stream(rlb_batch *b, void *cuda_stream)
{
    if (!b) return bfail(nullptr, RLB_E_INVALID, "batch is NULL");
    b->stream = (cudaStream_t)cuda_stream;
    return RLB_OK;
}

long long rlb_batch_total_cells(const rlb_batch *b) { return b ? b->total : 0; }

long long rlb_batch_launch_count(const rlb_batch *b) { return b ? b->launches : 0; }

void rlb_batch_destroy(rlb_batch *b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->host) cudaFreeHost(b->host);
    if (b->block) cudaFree(b->block);
    delete b;
}

const char *rlb_batch_last_error(const rlb_batch *b) { return b ? b->err.c_str() : g_berr.c_str(); }

}  // extern "C"
