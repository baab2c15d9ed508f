// md_api.cu -- the C ABI of include/md.h: context lifetime, device memory, host/device
// I/O, the force evaluation sequence and the velocity-Verlet step loop replayed from
// captured CUDA graphs (no host involvement between steps).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "md.h"
#include "md_plan.cuh"

using namespace mdk;

namespace {

constexpr int kStepsPerGraph = 8;

struct Timing {
    cudaEvent_t ev[2];
};

}  // namespace

struct md_ctx {
    int device = 0;
    Plan p;
    int io = MD_IO_HOST;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0, allocated = 0;
    std::vector<void *> allocs;
    int64_t series_cap = 0;
    bool pos_set = false, forces_valid = false, have_wj = false;
    int64_t steps_done = 0;
    int kernels_per_step = 0;
    int kernels_per_rebuild = 0;
    // graph cache: an 8-step and a 1-step graph of the velocity-Verlet step
    cudaGraphExec_t gexec = nullptr, gexec1 = nullptr;
    double g_dt = 0.0;
    double *g_series = nullptr;
    bool g_prof = false;
    cudaStream_t side = nullptr;   // stream used to capture conditional bodies
    bool use_graphs = true;        // false: eager launches, rebuild decided on the host
    // profiling
    bool profiling = false;
    std::vector<Timing> ev;        // [steps_per_graph * KC_COUNT]
    double kt_ms[KC_COUNT] = {0, 0, 0, 0, 0};
    int64_t kt_n[KC_COUNT] = {0, 0, 0, 0, 0};
    std::string err;
};

namespace {

md_status fail(md_ctx *c, md_status s, const std::string &msg)
{
    if (c) c->err = msg;
    return s;
}

md_status cuda_fail(md_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, MD_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

md_status dalloc(md_ctx *ctx, void **ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    if (ctx->budget && ctx->allocated + bytes > ctx->budget)
        return fail(ctx, MD_ERR_OOM, "allocation exceeds hbm_budget");
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, MD_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ctx->allocs.push_back(*ptr);
    ctx->allocated += bytes;
    return MD_OK;
}

template <typename P>
md_status dalloc_t(md_ctx *ctx, P **ptr, size_t count)
{
    void *v = nullptr;
    md_status s = dalloc(ctx, &v, count * sizeof(P));
    *ptr = static_cast<P *>(v);
    return s;
}

void destroy_graph(md_ctx *ctx)
{
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->gexec1) cudaGraphExecDestroy(ctx->gexec1);
    ctx->gexec = nullptr;
    ctx->gexec1 = nullptr;
}

// copy a 3-vector SoA field given as three pointers into dst[3N]
md_status upload3(md_ctx *ctx, double *dst, const double *a, const double *b, const double *c)
{
    const int64_t N = ctx->p.N;
    const cudaMemcpyKind k = ctx->io == MD_IO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const double *src[3] = {a, b, c};
    for (int d = 0; d < 3; ++d)
        CK(cudaMemcpyAsync(dst + d * N, src[d], sizeof(double) * N, k, ctx->stream));
    return MD_OK;
}

md_status download(md_ctx *ctx, double *dst, const double *src, size_t count)
{
    if (!dst || count == 0) return MD_OK;
    const cudaMemcpyKind k = ctx->io == MD_IO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(dst, src, sizeof(double) * count, k, ctx->stream));
    return MD_OK;
}

md_status set_flag_rebuild(md_ctx *ctx)
{
    static const int one = 1;
    CK(cudaMemcpyAsync(&ctx->p.flags->rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    return MD_OK;
}

// Reset the per-call error words (the rebuild request and counters persist).
md_status clear_error_flags(md_ctx *ctx)
{
    const int zeros[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(&ctx->p.flags->list_overflow, zeros, 4 * sizeof(int), cudaMemcpyHostToDevice,
                       ctx->stream));
    return MD_OK;
}

md_status check_flags(md_ctx *ctx)
{
    Flags f;
    CK(cudaMemcpyAsync(&f, ctx->p.flags, sizeof(Flags), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (f.list_overflow || f.active_overflow || f.asym || f.nonfinite) {
        // results of this call are invalid; rebuild from scratch on the next one
        ctx->forces_valid = false;
        md_status s = set_flag_rebuild(ctx);
        if (s != MD_OK) return s;
    }
    if (f.list_overflow)
        return fail(ctx, MD_ERR_NEIGH_OVERFLOW, "neighbour list longer than max_neigh (" +
                                                    std::to_string(f.max_nn) + " > " +
                                                    std::to_string(ctx->p.cap) + ")");
    if (f.active_overflow)
        return fail(ctx, MD_ERR_NEIGH_OVERFLOW, "more in-cutoff neighbours than max_active");
    if (f.asym) return fail(ctx, MD_ERR_CUDA, "internal: asymmetric neighbour list");
    if (f.nonfinite) return fail(ctx, MD_ERR_NAN, "non-finite force");
    return MD_OK;
}

// half-kick factors dt/2 * acc / m per type (same expression order as the oracle)
void half_kick(const md_ctx *ctx, double dt, double *hk)
{
    for (int t = 0; t < kMaxTypes; ++t)
        hk[t] = ctx->p.mass[t] > 0 ? 0.5 * dt * kAccUnit / ctx->p.mass[t] : 0.0;
}

struct Recorder {
    md_ctx *ctx;
    int step;         // index of the step inside the graph (profiling events)
    bool capturing;   // enqueued under stream capture
    // Under capture the records must be "external" to become event-record nodes of the
    // graph (a plain record only marks a capture dependency); outside capture the flag
    // is not allowed, so a plain record is used there.
    void rec(cudaEvent_t e) const
    {
        if (capturing) cudaEventRecordWithFlags(e, ctx->stream, cudaEventRecordExternal);
        else cudaEventRecord(e, ctx->stream);
    }
    void begin(int kc) const
    {
        if (ctx->profiling) rec(ctx->ev[step * KC_COUNT + kc].ev[0]);
    }
    void end(int kc) const
    {
        if (ctx->profiling) rec(ctx->ev[step * KC_COUNT + kc].ev[1]);
    }
};

// Inside a capture on ctx->stream: a conditional IF node whose body is the list
// rebuild, taken when the handle's value is non-zero.  The body is captured on the
// side stream.  Returns the number of kernels in the body.
md_status add_conditional_rebuild(md_ctx *ctx, cudaGraphConditionalHandle h)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &g, &deps, &edges, &nd));
    if (cs != cudaStreamCaptureStatusActive) return fail(ctx, MD_ERR_CUDA, "stream is not capturing");
    // the parameter union has no usable default constructor: zero a raw buffer instead
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    std::memset(raw, 0, sizeof(raw));
    cudaGraphNodeParams &np = *reinterpret_cast<cudaGraphNodeParams *>(raw);
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    CK(cudaGraphAddNode(&node, g, deps, edges, nd, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    CK(cudaStreamUpdateCaptureDependencies(ctx->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    CK(cudaStreamBeginCaptureToGraph(ctx->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ctx->kernels_per_rebuild = launch_rebuild(ctx->p, ctx->side);
    cudaGraph_t out = nullptr;
    CK(cudaStreamEndCapture(ctx->side, &out));
    return MD_OK;
}

// One velocity-Verlet step inside a capture:
//   kick/drift -> [step begin: series row, rebuild condition] -> IF(rebuild) ->
//   pair pass -> gather (+ half-kick) -> reduce (series row)
md_status enqueue_step(md_ctx *ctx, const Recorder &rec, const double *hk, double dt, int *n_kernels)
{
    rec.begin(KC_KICK_DRIFT);
    launch_kick_drift(ctx->p, ctx->stream, hk, dt);
    rec.end(KC_KICK_DRIFT);
    rec.begin(KC_REBUILD);
    if (ctx->p.N > 0) {
        cudaGraphConditionalHandle h;
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        CK(cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr));
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        launch_step_begin(ctx->p, ctx->stream, &h);
        md_status s = add_conditional_rebuild(ctx, h);
        if (s != MD_OK) return s;
    } else {
        launch_step_begin(ctx->p, ctx->stream, nullptr);   // no atoms: nothing to rebuild
    }
    rec.end(KC_REBUILD);
    rec.begin(KC_PAIR);
    launch_pair(ctx->p, ctx->stream);
    rec.end(KC_PAIR);
    rec.begin(KC_GATHER);
    launch_gather(ctx->p, ctx->stream, hk, false);
    rec.end(KC_GATHER);
    rec.begin(KC_REDUCE);
    launch_reduce(ctx->p, ctx->stream, false, true);
    rec.end(KC_REDUCE);
    // kernels launched every step; a taken rebuild adds the body's kernels
    *n_kernels = ctx->p.N > 0 ? 5 : 2;
    return MD_OK;
}

// The same step with eager launches: the rebuild decision is read back to the host
// (one small copy and a synchronisation per step).  Kernels and arguments are those of
// the graph path; this mode exists so that profilers can see every kernel.
md_status eager_step(md_ctx *ctx, const double *hk, double dt)
{
    Recorder rec{ctx, 0, false};
    rec.begin(KC_KICK_DRIFT);
    launch_kick_drift(ctx->p, ctx->stream, hk, dt);
    rec.end(KC_KICK_DRIFT);
    launch_step_begin(ctx->p, ctx->stream, nullptr);
    int rebuild = 0;
    CK(cudaMemcpyAsync(&rebuild, &ctx->p.flags->rebuild, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    rec.begin(KC_REBUILD);
    if (rebuild) launch_rebuild(ctx->p, ctx->stream);
    rec.end(KC_REBUILD);
    rec.begin(KC_PAIR);
    launch_pair(ctx->p, ctx->stream);
    rec.end(KC_PAIR);
    rec.begin(KC_GATHER);
    launch_gather(ctx->p, ctx->stream, hk, false);
    rec.end(KC_GATHER);
    rec.begin(KC_REDUCE);
    launch_reduce(ctx->p, ctx->stream, false, true);
    rec.end(KC_REDUCE);
    CK(cudaGetLastError());
    return MD_OK;
}

md_status ensure_events(md_ctx *ctx)
{
    if (!ctx->ev.empty()) return MD_OK;
    ctx->ev.resize(kStepsPerGraph * KC_COUNT);
    for (auto &t : ctx->ev)
        for (auto &e : t.ev) CK(cudaEventCreate(&e));
    return MD_OK;
}

md_status accumulate_times(md_ctx *ctx, int steps)
{
    CK(cudaStreamSynchronize(ctx->stream));
    for (int s = 0; s < steps; ++s)
        for (int k = 0; k < KC_COUNT; ++k) {
            float ms = 0.f;
            cudaError_t e = cudaEventElapsedTime(&ms, ctx->ev[s * KC_COUNT + k].ev[0], ctx->ev[s * KC_COUNT + k].ev[1]);
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            ctx->kt_ms[k] += ms;
            ctx->kt_n[k] += 1;
        }
    return MD_OK;
}

md_status ensure_series(md_ctx *ctx, int64_t rows)
{
    if (rows <= ctx->series_cap) return MD_OK;
    if (ctx->p.series) {
        cudaFree(ctx->p.series);
        for (auto &a : ctx->allocs)
            if (a == ctx->p.series) a = nullptr;
        ctx->allocated -= sizeof(double) * 5 * ctx->series_cap;
        ctx->p.series = nullptr;
    }
    int64_t cap = rows < 1024 ? 1024 : rows;
    md_status s = dalloc_t(ctx, &ctx->p.series, (size_t)cap * 5);
    if (s != MD_OK) return s;
    ctx->series_cap = cap;
    destroy_graph(ctx);
    return MD_OK;
}

md_status ensure_wj(md_ctx *ctx)
{
    if (ctx->have_wj) return MD_OK;
    md_status s = dalloc_t(ctx, &ctx->p.w, (size_t)9 * (ctx->p.N > 0 ? ctx->p.N : 1));
    if (s != MD_OK) return s;
    s = dalloc_t(ctx, &ctx->p.j, (size_t)3 * (ctx->p.N > 0 ? ctx->p.N : 1));
    if (s != MD_OK) return s;
    ctx->have_wj = true;
    return MD_OK;
}

// One force evaluation (not a time step): rebuild the list if any atom moved more than
// skin/2 (checked on the host here; md_run decides on the device), then the pair pass,
// the full gather (F, W, J per atom) and the totals.
md_status force_eval(md_ctx *ctx, bool full)
{
    if (full) {
        md_status s = ensure_wj(ctx);
        if (s != MD_OK) return s;
    }
    md_status s0 = clear_error_flags(ctx);
    if (s0 != MD_OK) return s0;
    launch_displacement_check(ctx->p, ctx->stream);
    int rebuild = 0;
    CK(cudaMemcpyAsync(&rebuild, &ctx->p.flags->rebuild, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (rebuild) launch_rebuild(ctx->p, ctx->stream);
    launch_pair(ctx->p, ctx->stream);
    launch_gather(ctx->p, ctx->stream, nullptr, full);
    launch_reduce(ctx->p, ctx->stream, full, false);
    CK(cudaGetLastError());
    md_status s = check_flags(ctx);
    if (s != MD_OK) return s;
    ctx->forces_valid = true;
    return MD_OK;
}

md_status capture_one(md_ctx *ctx, const double *hk, double dt, int steps, cudaGraphExec_t *out)
{
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int per_step = 0;
    for (int st = 0; st < steps; ++st) {
        md_status s = enqueue_step(ctx, Recorder{ctx, st, true}, hk, dt, &per_step);
        if (s != MD_OK) {
            cudaStreamEndCapture(ctx->stream, &g);
            if (g) cudaGraphDestroy(g);
            return s;
        }
    }
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    ctx->kernels_per_step = per_step;
    return MD_OK;
}

md_status capture_graph(md_ctx *ctx, const double *hk, double dt)
{
    destroy_graph(ctx);
    md_status s = capture_one(ctx, hk, dt, kStepsPerGraph, &ctx->gexec);
    if (s != MD_OK) return s;
    s = capture_one(ctx, hk, dt, 1, &ctx->gexec1);
    if (s != MD_OK) return s;
    ctx->g_dt = dt;
    ctx->g_series = ctx->p.series;
    ctx->g_prof = ctx->profiling;
    return MD_OK;
}

}  // namespace

extern "C" {

md_status md_default_options(md_options *opt)
{
    if (!opt) return MD_ERR_ARG;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = MD_FP64;
    opt->skin = 0.0;
    opt->max_neigh = 32;
    opt->max_active = 0;
    opt->io = MD_IO_HOST;
    opt->cuda_stream = nullptr;
    opt->hbm_budget = 0;
    opt->device = 0;
    return MD_OK;
}

md_status md_create(md_ctx **out, const double box[3], const int pbc[3], int64_t n_atoms,
                    const int32_t *types, const double *masses_by_type, const md_params *params,
                    const md_options *opt_in)
{
    if (!out) return MD_ERR_ARG;
    *out = nullptr;
    if (!box || !pbc || n_atoms < 0 || (n_atoms > 0 && !types) || !masses_by_type || !params || !params->p)
        return MD_ERR_ARG;
    if (n_atoms > kMaxAtoms) return MD_ERR_ARG;   // list entries hold 26-bit atom indices
    md_options opt;
    if (opt_in) opt = *opt_in; else md_default_options(&opt);
    if (params->kind != MD_TERSOFF && params->kind != MD_SW) return MD_ERR_ARG;
    if (params->n_types != 1) return MD_ERR_ARG;
    if (opt.precision != MD_FP64 && opt.precision != MD_MIXED) return MD_ERR_ARG;
    if (opt.max_neigh < 1 || opt.max_neigh > kMaxListCap) return MD_ERR_ARG;
    if (opt.max_active < 0 || opt.max_active > 16) return MD_ERR_ARG;
    if (opt.skin < 0) return MD_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!(box[a] > 0) || !std::isfinite(box[a])) return MD_ERR_ARG;
    if (!(masses_by_type[0] > 0)) return MD_ERR_ARG;
    for (int64_t i = 0; i < n_atoms; ++i)
        if (types[i] != 0) return MD_ERR_ARG;   // single element

    md_ctx *ctx = new md_ctx();
    Plan &p = ctx->p;
    ctx->device = opt.device;
    ctx->io = opt.io;
    ctx->budget = opt.hbm_budget;
    p.N = n_atoms;
    p.kind = params->kind;
    p.precision = opt.precision;
    p.cap = opt.max_neigh;
    const int want_active = opt.max_active > 0 ? opt.max_active : (params->kind == MD_SW ? 16 : 8);
    p.maxa = want_active <= 8 ? 8 : 16;
    p.ntypes = params->n_types;
    p.mass[0] = masses_by_type[0];
    p.inv_mass[0] = 1.0 / masses_by_type[0];
    const double *q = params->p;
    if (p.kind == MD_TERSOFF) {
        TersoffP &t = p.tp;
        t.A = q[0]; t.B = q[1]; t.lam = q[2]; t.mu = q[3]; t.beta = q[4]; t.n = q[5];
        t.c = q[6]; t.d = q[7]; t.h = q[8]; t.R = q[9]; t.S = q[10];
        if (!(t.S > t.R) || !(t.R > 0) || !(t.n > 0) || t.beta < 0 || !(t.d != 0)) {
            delete ctx;
            return MD_ERR_ARG;
        }
        t.c2 = t.c * t.c;
        t.d2 = t.d * t.d;
        t.c2d2 = t.c2 / t.d2;
        t.pi_SR = M_PI / (t.S - t.R);
        t.beta_zero = t.beta == 0.0;
        t.ln_beta = t.beta > 0 ? std::log(t.beta) : 0.0;
        t.inv2n = 1.0 / (2.0 * t.n);
        p.rc = t.S;
    } else {
        SWP &s = p.sp;
        s.eps = q[0]; s.sig = q[1]; s.a = q[2]; s.lam = q[3]; s.gam = q[4]; s.A = q[5]; s.B = q[6];
        s.p = q[7]; s.q = q[8];
        if (!(s.sig > 0) || !(s.a > 0)) {
            delete ctx;
            return MD_ERR_ARG;
        }
        s.rc = s.a * s.sig;
        s.Aeps = s.A * s.eps;
        s.lameps = s.lam * s.eps;
        s.gamsig = s.gam * s.sig;
        s.p_int = (s.p == std::floor(s.p) && s.p >= 0 && s.p <= 16) ? (int)s.p : -1;
        s.q_int = (s.q == std::floor(s.q) && s.q >= 0 && s.q <= 16) ? (int)s.q : -1;
        p.rc = s.rc;
    }
    p.skin = opt.skin > 0 ? opt.skin : 0.15 * p.rc;
    p.rl = p.rc + p.skin;
    for (int a = 0; a < 3; ++a) {
        p.box.L[a] = box[a];
        p.box.invL[a] = 1.0 / box[a];
        p.box.pbc[a] = pbc[a] ? 1 : 0;
        if (p.box.pbc[a] && box[a] < 2.0 * p.rl + 0.01) {
            delete ctx;
            return MD_ERR_BOX;
        }
        int n = (int)std::floor(box[a] / p.rl);
        p.nc[a] = n < 1 ? 1 : n;
    }
    p.ncell = (int64_t)p.nc[0] * p.nc[1] * p.nc[2];

    md_status st = MD_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return MD_ERR_CUDA;
    }
    if (opt.cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(opt.cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete ctx;
            return MD_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
        delete ctx;
        return MD_ERR_CUDA;
    }
    configure_kernels(p);

    const size_t N1 = (size_t)(p.N > 0 ? p.N : 1);
    const size_t esz = p.precision == MD_FP64 ? sizeof(double) : sizeof(float);
#define AL(ptr, count)                                      \
    do {                                                    \
        st = dalloc_t(ctx, &(ptr), (size_t)(count));        \
        if (st != MD_OK) { md_destroy(ctx); return st; }    \
    } while (0)
    AL(p.pos, 3 * N1);
    AL(p.vel, 3 * N1);
    AL(p.force, 3 * N1);
    AL(p.pos_build, 3 * N1);
    AL(p.u, N1);
    AL(p.posf, 3 * N1);
    AL(p.stage, 3 * N1);
    AL(p.type, N1);
    AL(p.nn, N1);
    AL(p.nl, (size_t)p.cap * N1);
    AL(p.rev, (size_t)p.cap * N1);
    AL(p.mask, N1);
    {
        void *v = nullptr;
        st = dalloc(ctx, &v, 3 * (size_t)p.maxa * N1 * esz);
        if (st != MD_OK) { md_destroy(ctx); return st; }
        p.pd = v;
        st = dalloc(ctx, &v, 3 * (size_t)p.maxa * N1 * esz);
        if (st != MD_OK) { md_destroy(ctx); return st; }
        p.pr = v;
    }
    AL(p.cell_count, p.ncell);
    AL(p.cell_start, p.ncell);
    AL(p.cell_atoms, N1);
    AL(p.atom_cell, N1);
    AL(p.atom_rank, N1);
    p.nscanb = (p.ncell + scan_block_elems() - 1) / scan_block_elems();
    AL(p.scan_blocks, p.nscanb + 1);
    p.nb_gather = gather_blocks(p.N);
    AL(p.partials, (size_t)p.nb_gather * kNumPartials);
    AL(p.totals, kNumPartials);
    AL(p.flags, 1);
#undef AL
    st = ensure_series(ctx, 1024);
    if (st != MD_OK) { md_destroy(ctx); return st; }

    // zero state; types from the host
    cudaMemsetAsync(p.pos, 0, sizeof(double) * 3 * N1, ctx->stream);
    cudaMemsetAsync(p.vel, 0, sizeof(double) * 3 * N1, ctx->stream);
    cudaMemsetAsync(p.force, 0, sizeof(double) * 3 * N1, ctx->stream);
    cudaMemsetAsync(p.flags, 0, sizeof(Flags), ctx->stream);
    cudaMemsetAsync(p.nn, 0, sizeof(int) * N1, ctx->stream);
    if (p.N > 0) cudaMemcpyAsync(p.type, types, sizeof(int32_t) * p.N, cudaMemcpyHostToDevice, ctx->stream);
    e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        md_destroy(ctx);
        return MD_ERR_CUDA;
    }
    *out = ctx;
    return MD_OK;
}

md_status md_set_positions(md_ctx *ctx, const double *x, const double *y, const double *z)
{
    if (!ctx) return MD_ERR_ARG;
    if (ctx->p.N > 0 && (!x || !y || !z)) return fail(ctx, MD_ERR_ARG, "NULL position array");
    if (ctx->p.N > 0) {
        md_status s = upload3(ctx, ctx->p.pos, x, y, z);
        if (s != MD_OK) return s;
    }
    md_status s = set_flag_rebuild(ctx);
    if (s != MD_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->pos_set = true;
    ctx->forces_valid = false;
    return MD_OK;
}

md_status md_set_velocities(md_ctx *ctx, const double *vx, const double *vy, const double *vz)
{
    if (!ctx) return MD_ERR_ARG;
    if (ctx->p.N > 0 && (!vx || !vy || !vz)) return fail(ctx, MD_ERR_ARG, "NULL velocity array");
    if (ctx->p.N > 0) {
        md_status s = upload3(ctx, ctx->p.vel, vx, vy, vz);
        if (s != MD_OK) return s;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return MD_OK;
}

md_status md_compute(md_ctx *ctx, double *f, double *u, double *w, double *j, double *totals)
{
    if (!ctx) return MD_ERR_ARG;
    if (!ctx->pos_set && ctx->p.N > 0) return fail(ctx, MD_ERR_STATE, "positions not set");
    md_status s = force_eval(ctx, true);
    if (s != MD_OK) return s;
    const int64_t N = ctx->p.N;
    if ((s = download(ctx, f, ctx->p.force, 3 * N)) != MD_OK) return s;
    if ((s = download(ctx, u, ctx->p.u, N)) != MD_OK) return s;
    if ((s = download(ctx, w, ctx->p.w, 9 * N)) != MD_OK) return s;
    if ((s = download(ctx, j, ctx->p.j, 3 * N)) != MD_OK) return s;
    double t[kNumPartials];
    CK(cudaMemcpyAsync(t, ctx->p.totals, sizeof(t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (totals) {
        totals[0] = t[0];                                  // U
        for (int c = 0; c < 9; ++c) totals[1 + c] = t[5 + c];   // W
        for (int c = 0; c < 3; ++c) totals[10 + c] = t[2 + c];  // J
    }
    return MD_OK;
}

md_status md_run(md_ctx *ctx, int64_t n_steps, double dt_fs, double *series)
{
    if (!ctx) return MD_ERR_ARG;
    if (n_steps < 0 || !std::isfinite(dt_fs)) return fail(ctx, MD_ERR_ARG, "bad n_steps or dt");
    if (!ctx->pos_set && ctx->p.N > 0) return fail(ctx, MD_ERR_STATE, "positions not set");
    if (n_steps == 0) return MD_OK;
    md_status s = ensure_series(ctx, n_steps);
    if (s != MD_OK) return s;
    if (!ctx->forces_valid) {
        s = force_eval(ctx, false);
        if (s != MD_OK) return s;
    }
    if (ctx->profiling) {
        s = ensure_events(ctx);
        if (s != MD_OK) return s;
    }
    s = clear_error_flags(ctx);
    if (s != MD_OK) return s;
    double hk[kMaxTypes];
    half_kick(ctx, dt_fs, hk);
    {
        const long long zero = 0;
        CK(cudaMemcpyAsync(&ctx->p.flags->step, &zero, sizeof(zero), cudaMemcpyHostToDevice, ctx->stream));
    }
    if (!ctx->use_graphs) {
        for (int64_t done = 0; done < n_steps; ++done) {
            s = eager_step(ctx, hk, dt_fs);
            if (s != MD_OK) return s;
            if (ctx->profiling) {
                s = accumulate_times(ctx, 1);
                if (s != MD_OK) return s;
            }
        }
    } else {
        if (!ctx->gexec || !ctx->gexec1 || ctx->g_dt != dt_fs || ctx->g_series != ctx->p.series ||
            ctx->g_prof != ctx->profiling) {
            s = capture_graph(ctx, hk, dt_fs);
            if (s != MD_OK) return s;
        }
        int64_t done = 0;
        while (n_steps - done >= kStepsPerGraph) {
            CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
            if (ctx->profiling) {
                s = accumulate_times(ctx, kStepsPerGraph);
                if (s != MD_OK) return s;
            }
            done += kStepsPerGraph;
        }
        for (; done < n_steps; ++done) {
            CK(cudaGraphLaunch(ctx->gexec1, ctx->stream));
            if (ctx->profiling) {
                s = accumulate_times(ctx, 1);
                if (s != MD_OK) return s;
            }
        }
    }
    if (series) {
        const cudaMemcpyKind k = ctx->io == MD_IO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CK(cudaMemcpyAsync(series, ctx->p.series, sizeof(double) * 5 * n_steps, k, ctx->stream));
    }
    s = check_flags(ctx);
    ctx->steps_done += n_steps;
    if (s != MD_OK) {
        ctx->forces_valid = false;
        return s;
    }
    return MD_OK;
}

md_status md_get_state(md_ctx *ctx, double *x, double *v)
{
    if (!ctx) return MD_ERR_ARG;
    md_status s;
    if (x && ctx->p.N > 0) {
        // positions move unwrapped between list builds; report them wrapped into the box
        launch_wrap_copy(ctx->p, ctx->stream, ctx->p.stage);
        if ((s = download(ctx, x, ctx->p.stage, 3 * ctx->p.N)) != MD_OK) return s;
    }
    if ((s = download(ctx, v, ctx->p.vel, 3 * ctx->p.N)) != MD_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return MD_OK;
}

md_status md_get_stats(md_ctx *ctx, md_stats *out)
{
    if (!ctx || !out) return MD_ERR_ARG;
    Flags f;
    CK(cudaMemcpyAsync(&f, ctx->p.flags, sizeof(Flags), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    out->n_atoms = ctx->p.N;
    out->steps_done = ctx->steps_done;
    out->n_rebuilds = f.n_rebuilds;
    out->max_neigh_seen = f.max_nn;
    out->kernel_launches_per_step = ctx->kernels_per_step;
    out->kernel_launches_per_rebuild = ctx->kernels_per_rebuild;
    out->device_bytes = ctx->allocated;
    return MD_OK;
}

md_status md_set_graph_mode(md_ctx *ctx, int use_graphs)
{
    if (!ctx) return MD_ERR_ARG;
    ctx->use_graphs = use_graphs != 0;
    return MD_OK;
}

md_status md_set_profiling(md_ctx *ctx, int enable)
{
    if (!ctx) return MD_ERR_ARG;
    ctx->profiling = enable != 0;
    for (int k = 0; k < KC_COUNT; ++k) {
        ctx->kt_ms[k] = 0;
        ctx->kt_n[k] = 0;
    }
    return MD_OK;
}

md_status md_kernel_times(md_ctx *ctx, int max_k, const char **names, int64_t *launches,
                          double *total_ms, int *n_out)
{
    if (!ctx || max_k < 0) return MD_ERR_ARG;
    int n = max_k < KC_COUNT ? max_k : KC_COUNT;
    for (int k = 0; k < n; ++k) {
        if (names) names[k] = kKernelClassNames[k];
        if (launches) launches[k] = ctx->kt_n[k];
        if (total_ms) total_ms[k] = ctx->kt_ms[k];
    }
    if (n_out) *n_out = n;
    return MD_OK;
}

const char *md_last_error(const md_ctx *ctx)
{
    if (!ctx) return "";
    return ctx->err.c_str();
}

void md_destroy(md_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    destroy_graph(ctx);
    for (auto &t : ctx->ev)
        for (auto &e : t.ev) cudaEventDestroy(e);
    for (void *a : ctx->allocs)
        if (a) cudaFree(a);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    delete ctx;
}

}  // extern "C"
