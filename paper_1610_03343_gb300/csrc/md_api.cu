// md_api.cu -- the C ABI of include/md.h: context lifetime, device memory, host/device
// I/O, the force evaluation sequence and the velocity-Verlet step loop replayed from
// captured CUDA graphs (no host involvement between steps).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
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

// First-fit allocator of [start, start + len) ranges over [0, capacity).
struct RangeAlloc {
    std::map<int64_t, int64_t> free_;   // start -> length
    void init(int64_t capacity)
    {
        free_.clear();
        if (capacity > 0) free_[0] = capacity;
    }
    int64_t alloc(int64_t len)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                const int64_t start = it->first, rest = it->second - len;
                free_.erase(it);
                if (rest > 0) free_[start + len] = rest;
                return start;
            }
        }
        return -1;
    }
    void release(int64_t start, int64_t len)
    {
        if (len <= 0) return;
        auto it = free_.emplace(start, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
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
    int kernels_g8 = 0, kernels_g1 = 0;   // kernels of one replay of each step graph
    int64_t kernels_launched = 0;         // by md_run steps (rebuild bodies not counted)
    // graph cache: an 8-step and a 1-step graph of the velocity-Verlet step
    cudaGraphExec_t gexec = nullptr, gexec1 = nullptr;
    double g_dt = 0.0;
    double *g_series = nullptr;
    bool g_prof = false;
    cudaStream_t side = nullptr;   // stream used to capture conditional bodies
    cudaStream_t side2 = nullptr;  // pools: second branch of the step graph (rebuild)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    cudaEvent_t ev_red = nullptr;  // single systems: a step's reduction, on the side branch
    bool use_graphs = true;        // false: eager launches, rebuild decided on the host
    // profiling
    bool profiling = false;
    std::vector<Timing> ev;        // [steps_per_graph * KC_COUNT]
    double kt_ms[KC_COUNT] = {0, 0, 0, 0, 0};
    int64_t kt_n[KC_COUNT] = {0, 0, 0, 0, 0};
    // pools
    bool is_pool = false;
    std::vector<SysDev> sys_host;   // n_sys + 1 (the last: inactive sentinel for free atoms)
    std::vector<char> sys_used;
    RangeAlloc atoms_free, cells_free;
    int64_t cell_capacity = 0;
    int64_t min_atoms = 1;
    double skin_option = 0.0;
    int nc_full[3] = {1, 1, 1};    // single system: the cell grid from the box alone
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
    static const int zeros[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(&ctx->p.flags->list_overflow, zeros, 4 * sizeof(int), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemcpyAsync(&ctx->p.flags->box_error, zeros, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
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
    if (f.nonfinite) return fail(ctx, MD_ERR_NAN, "non-finite force, position or velocity");
    if (f.box_error) {
        ctx->forces_valid = false;
        return fail(ctx, MD_ERR_BOX, "NPT: a periodic box edge shrank below 2 (cutoff + skin)");
    }
    return MD_OK;
}

// Unpack one packed parameter set into set `idx` of the plan; returns its cutoff in rc.
md_status parse_params(const md_params *params, Plan &p, int idx, double *rc)
{
    if (!params || !params->p) return MD_ERR_ARG;
    const double *q = params->p;
    if (params->kind == MD_TERSOFF) {
        TersoffP &t = p.tp[idx];
        t.A = q[0]; t.B = q[1]; t.lam = q[2]; t.mu = q[3]; t.beta = q[4]; t.n = q[5];
        t.c = q[6]; t.d = q[7]; t.h = q[8]; t.R = q[9]; t.S = q[10];
        if (!(t.S > t.R) || !(t.R > 0) || !(t.n > 0) || t.beta < 0 || !(t.d != 0)) return MD_ERR_ARG;
        t.c2 = t.c * t.c;
        t.d2 = t.d * t.d;
        t.c2d2 = t.c2 / t.d2;
        t.pi_SR = M_PI / (t.S - t.R);
        t.beta_zero = t.beta == 0.0;
        t.ln_beta = t.beta > 0 ? std::log(t.beta) : 0.0;
        t.inv2n = 1.0 / (2.0 * t.n);
        *rc = t.S;
    } else if (params->kind == MD_SW) {
        SWP &w = p.sp[idx];
        w.eps = q[0]; w.sig = q[1]; w.a = q[2]; w.lam = q[3]; w.gam = q[4]; w.A = q[5]; w.B = q[6];
        w.p = q[7]; w.q = q[8];
        if (!(w.sig > 0) || !(w.a > 0)) return MD_ERR_ARG;
        w.rc = w.a * w.sig;
        w.Aeps = w.A * w.eps;
        w.lameps = w.lam * w.eps;
        w.gamsig = w.gam * w.sig;
        w.p_int = (w.p == std::floor(w.p) && w.p >= 0 && w.p <= 16) ? (int)w.p : -1;
        w.q_int = (w.q == std::floor(w.q) && w.q >= 0 && w.q <= 16) ? (int)w.q : -1;
        *rc = w.rc;
    } else {
        return MD_ERR_ARG;
    }
    return MD_OK;
}

// Multi-element Tersoff (Tersoff 1989 multicomponent form): n_types element rows of 11
// parameters followed by the n_types x n_types factors chi.  Element a goes to p.tp[a];
// every ordered pair (a, b) gets the constants of a bond from an atom of element a to one
// of element b: A, B, R, S mixed geometrically and lambda, mu arithmetically, B scaled by
// chi_ab (b_ij = chi_ab b~_ij enters U_i only as b~_ij (chi_ab f_A)), and element a's
// beta, n, c, d, h.  rc receives the largest mixed cutoff.
md_status parse_multi(const md_params *params, Plan &p, double *rc)
{
    const int nt = params->n_types;
    for (int a = 0; a < nt; ++a) {
        md_params e{MD_TERSOFF, 1, params->p + 11 * a};
        double rca = 0;
        if (parse_params(&e, p, a, &rca) != MD_OK) return MD_ERR_ARG;
    }
    const double *chi = params->p + 11 * nt;
    *rc = 0.0;
    for (int a = 0; a < nt; ++a)
        for (int b = 0; b < nt; ++b) {
            const double x = chi[a * nt + b];
            if (!(x > 0) || !std::isfinite(x)) return MD_ERR_ARG;
            const TersoffP &ea = p.tp[a], &eb = p.tp[b];
            TersoffP m = ea;
            m.A = std::sqrt(ea.A * eb.A);
            m.B = std::sqrt(ea.B * eb.B) * x;
            m.lam = 0.5 * (ea.lam + eb.lam);
            m.mu = 0.5 * (ea.mu + eb.mu);
            m.R = std::sqrt(ea.R * eb.R);
            m.S = std::sqrt(ea.S * eb.S);
            m.pi_SR = M_PI / (m.S - m.R);
            p.tpair[a][b] = m;
            *rc = std::max(*rc, m.S);
        }
    p.multi = true;
    p.n_elem = nt;
    return MD_OK;
}

// Box and cell grid of one system: periodic edges must exceed 2 (rl + margin); cells
// have edge >= rl + margin; a grid larger than `max_cells` is coarsened (coarser cells
// are still correct, only slower).
md_status system_box(const Plan &p, double rl, const double box[3], const int pbc[3], int64_t max_cells, Box *out,
                     int nc[3])
{
    const double edge = rl + p.list_margin;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0) || !std::isfinite(box[a])) return MD_ERR_ARG;
        out->L[a] = box[a];
        out->invL[a] = 1.0 / box[a];
        out->pbc[a] = pbc[a] ? 1 : 0;
        if (out->pbc[a] && box[a] < 2.0 * edge + 0.01) return MD_ERR_BOX;
        const int n = (int)std::floor(box[a] / edge);
        nc[a] = n < 1 ? 1 : n;
    }
    while ((int64_t)nc[0] * nc[1] * nc[2] > max_cells) {
        int a = 0;
        if (nc[1] > nc[a]) a = 1;
        if (nc[2] > nc[a]) a = 2;
        if (nc[a] == 1) break;
        nc[a] = (nc[a] + 1) / 2;
    }
    return MD_OK;
}

// Merge into one cell every cell axis that the atoms barely occupy -- at most a quarter of
// its cells hold an atom (a sheet with vacuum along a periodic axis, a slab).  Any grid
// whose cells are at least the list radius wide yields the same (index-sorted) lists, so
// this changes no result; it only removes empty cells from every rebuild's clear and scan.
void coarsen_sparse_axes(const double *const xyz[3], int64_t n, const Box &box, int nc[3])
{
    for (int a = 0; a < 3; ++a) {
        if (nc[a] < 4 || n <= 0) continue;
        std::vector<char> occ((size_t)nc[a], 0);
        int used = 0;
        for (int64_t i = 0; i < n && 4 * used <= nc[a]; ++i) {
            double x = xyz[a][i];
            if (box.pbc[a]) x -= box.L[a] * std::floor(x * box.invL[a]);
            int c = (int)std::floor(x * box.invL[a] * (double)nc[a]);
            c = c < 0 ? 0 : (c >= nc[a] ? nc[a] - 1 : c);
            if (!occ[(size_t)c]) {
                occ[(size_t)c] = 1;
                ++used;
            }
        }
        if (4 * used <= nc[a]) nc[a] = 1;
    }
}

// coarsen_sparse_axes for a single system's positions on the device (host or device IO):
// one pass over the atoms flags the occupied cells of each axis (launch_axis_occupancy) and
// the host counts them.
md_status coarsen_sparse_axes_dev(md_ctx *ctx, int nc[3])
{
    Plan &p = ctx->p;
    if (!p.occ || p.N <= 0) return MD_OK;
    const int n0 = nc[0], n1 = nc[1], n2 = nc[2], tot = n0 + n1 + n2;
    CK(cudaMemsetAsync(p.occ, 0, (size_t)tot, ctx->stream));
    launch_axis_occupancy(p, ctx->stream, p.box, nc, p.occ);
    CK(cudaGetLastError());
    std::vector<uint8_t> h((size_t)tot);
    CK(cudaMemcpyAsync(h.data(), p.occ, (size_t)tot, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int off[3] = {0, n0, n0 + n1}, len[3] = {n0, n1, n2};
    for (int a = 0; a < 3; ++a) {
        if (len[a] < 4) continue;
        int used = 0;
        for (int c = 0; c < len[a]; ++c) used += h[(size_t)(off[a] + c)] != 0;
        if (4 * used <= len[a]) nc[a] = 1;
    }
    return MD_OK;
}

// fp64 single-element Tersoff: the common-case stagings without f_C send every atom with a
// bond in the switching region R <= r < S to the full-capacity pass, which suits crystals
// (none at room temperature) but not liquids or hot amorphous states.  When the last pair
// pass of a call deferred more than 1/16 of the atoms, later calls use the 4-bond staging
// that keeps f_C.  Every staging computes each atom the same way, so results do not change.
md_status adapt_staging(md_ctx *ctx)
{
    Plan &p = ctx->p;
    if (p.kind != 1 || p.precision != MD_FP64 || p.multi || p.pair_fc || p.N <= 0) return MD_OK;
    int deferred = 0;
    CK(cudaMemcpyAsync(&deferred, p.ovf_count, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const int64_t n = p.n_owned >= 0 ? p.n_owned : p.N;
    if ((int64_t)deferred * 16 > n) {
        p.pair_fc = true;
        destroy_graph(ctx);
    }
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
    void rec(cudaEvent_t e, cudaStream_t st) const
    {
        if (capturing) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else cudaEventRecord(e, st);
    }
    void begin(int kc, cudaStream_t st = nullptr) const
    {
        if (ctx->profiling) rec(ctx->ev[step * KC_COUNT + kc].ev[0], st ? st : ctx->stream);
    }
    void end(int kc, cudaStream_t st = nullptr) const
    {
        if (ctx->profiling) rec(ctx->ev[step * KC_COUNT + kc].ev[1], st ? st : ctx->stream);
    }
};

// Inside a capture on stream `on`: a conditional IF node whose body is the list rebuild
// (pools, `with_pair`: followed by the pair pass of the rebuilt systems), taken when the
// handle's value is non-zero.  The body is captured on the side stream.
md_status add_conditional_rebuild(md_ctx *ctx, cudaGraphConditionalHandle h, cudaStream_t on, bool with_pair)
{
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t nd = 0;
    CK(cudaStreamGetCaptureInfo(on, &cs, nullptr, &g, &deps, &edges, &nd));
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
    CK(cudaStreamUpdateCaptureDependencies(on, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    CK(cudaStreamBeginCaptureToGraph(ctx->side, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    ctx->kernels_per_rebuild = launch_rebuild(ctx->p, ctx->side);
    if (with_pair) ctx->kernels_per_rebuild += launch_pair(ctx->p, ctx->side, PAIR_REBUILT, PAIR_FAST);
    cudaGraph_t out = nullptr;
    CK(cudaStreamEndCapture(ctx->side, &out));
    return MD_OK;
}

// Pools, the rest of a step after the kick: the pair pass of the systems that keep their
// lists runs while the others are rebuilt, on two branches of the graph:
//   step begin -> stable plan -+-> pair(stable) -------------------------------+
//                              +-> rebuild chain (flagged systems), pair(rebuilt) +
//   -> deferred atoms' pair pass -> gather (+ half-kick) -> reduce (series row)
// Each atom's work is the same as on a single branch, so results do not change.  Some
// system of a pool rebuilds on most steps, so the chain is launched every step (each of
// its kernels works on the flagged systems only, and on none when none is flagged) rather
// than behind a conditional node, whose body's launch cost exceeded the chain's work.
md_status enqueue_pool_tail(md_ctx *ctx, const Recorder &rec, const double *hk, double dt, int *n_kernels,
                            bool fuse_prev, bool fuse_next)
{
    launch_step_begin(ctx->p, ctx->stream, nullptr);
    launch_stable_plan(ctx->p, ctx->stream, nullptr);
    CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->side2, ctx->ev_fork, 0));
    rec.begin(KC_REBUILD, ctx->side2);
    const int n_rebuild = launch_rebuild(ctx->p, ctx->side2) + launch_pair(ctx->p, ctx->side2, PAIR_REBUILT, PAIR_FAST);
    ctx->kernels_per_rebuild = 0;   // launched every step, counted below
    rec.end(KC_REBUILD, ctx->side2);
    rec.begin(KC_PAIR);
    launch_pair(ctx->p, ctx->stream, PAIR_STABLE, PAIR_FAST);
    CK(cudaEventRecord(ctx->ev_join, ctx->side2));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_join, 0));
    launch_pair(ctx->p, ctx->stream, PAIR_ALL, PAIR_DEFERRED);
    rec.end(KC_PAIR);
    rec.begin(KC_GATHER);
    launch_gather(ctx->p, ctx->stream, hk, dt, false, fuse_next);
    rec.end(KC_GATHER);
    rec.begin(KC_REDUCE);
    launch_reduce(ctx->p, ctx->stream, false, true);
    launch_npt_couple(ctx->p, ctx->stream, dt);
    rec.end(KC_REDUCE);
    // active plan, kick (unless fused into the previous gather), step begin, stable plan,
    // 2 pair, gather, reduce (+ NPT apply, couple), the rebuild chain
    *n_kernels = 8 + (ctx->p.npt ? 2 : 0) - (fuse_prev ? 1 : 0) + n_rebuild;
    return MD_OK;
}

// One velocity-Verlet step inside a capture:
//   kick/drift -> [step begin: series row, rebuild condition] -> IF(rebuild) ->
//   pair pass -> gather (+ half-kick) -> reduce (series row)
// fuse_prev: the previous step's gather already took this step's kick and drift;
// fuse_next: this step's gather takes the next step's (see launch_gather).
// Single systems: when another step follows in the graph (and not under NPT, whose coupling
// needs the totals before the next kick), the step's reduction runs on a side branch beside
// the next step's step-begin, rebuild and pair pass; *reduce_pending tells the next step to
// join it before its gather, which overwrites the block partials.  The reduction takes its
// series row from flags->row_reduce, which the gather sets, so the next step-begin may move on.
md_status enqueue_step(md_ctx *ctx, const Recorder &rec, const double *hk, double dt, int *n_kernels,
                       bool fuse_prev = false, bool fuse_next = false, bool *reduce_pending = nullptr)
{
    launch_active_plan(ctx->p, ctx->stream);
    rec.begin(KC_KICK_DRIFT);
    if (!fuse_prev) launch_kick_drift(ctx->p, ctx->stream, hk, dt);
    launch_npt_apply(ctx->p, ctx->stream);
    rec.end(KC_KICK_DRIFT);
    if (ctx->p.batch && ctx->p.N > 0) return enqueue_pool_tail(ctx, rec, hk, dt, n_kernels, fuse_prev, fuse_next);
    rec.begin(KC_REBUILD);
    if (ctx->p.N > 0) {
        cudaGraphConditionalHandle h;
        cudaStreamCaptureStatus cs;
        cudaGraph_t g = nullptr;
        CK(cudaStreamGetCaptureInfo(ctx->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr));
        CK(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
        launch_step_begin(ctx->p, ctx->stream, &h);
        md_status s = add_conditional_rebuild(ctx, h, ctx->stream, false);
        if (s != MD_OK) return s;
    } else {
        launch_step_begin(ctx->p, ctx->stream, nullptr);   // no atoms: nothing to rebuild
    }
    rec.end(KC_REBUILD);
    rec.begin(KC_PAIR);
    launch_pair(ctx->p, ctx->stream);
    rec.end(KC_PAIR);
    if (reduce_pending && *reduce_pending) {
        CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_red, 0));
        *reduce_pending = false;
    }
    rec.begin(KC_GATHER);
    launch_gather(ctx->p, ctx->stream, hk, dt, false, fuse_next);
    rec.end(KC_GATHER);
    if (reduce_pending && fuse_next && !ctx->p.npt && ctx->p.N > 0) {
        CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
        CK(cudaStreamWaitEvent(ctx->side2, ctx->ev_fork, 0));
        rec.begin(KC_REDUCE, ctx->side2);
        launch_reduce(ctx->p, ctx->side2, false, true);
        rec.end(KC_REDUCE, ctx->side2);
        CK(cudaEventRecord(ctx->ev_red, ctx->side2));
        *reduce_pending = true;
    } else {
        rec.begin(KC_REDUCE);
        launch_reduce(ctx->p, ctx->stream, false, true);
        launch_npt_couple(ctx->p, ctx->stream, dt);
        rec.end(KC_REDUCE);
    }
    // kernels launched every step; a taken rebuild adds the body's kernels
    *n_kernels = (ctx->p.N > 0 ? 6 : 2) + (ctx->p.batch ? 1 : 0) + (ctx->p.npt && ctx->p.N > 0 ? 2 : 0) -
                 (fuse_prev && ctx->p.N > 0 ? 1 : 0);
    return MD_OK;
}

// The same step with eager launches: the rebuild decision is read back to the host
// (one small copy and a synchronisation per step).  Kernels and arguments are those of
// the graph path; this mode exists so that profilers can see every kernel.
md_status eager_step(md_ctx *ctx, const double *hk, double dt)
{
    Recorder rec{ctx, 0, false};
    launch_active_plan(ctx->p, ctx->stream);
    rec.begin(KC_KICK_DRIFT);
    launch_kick_drift(ctx->p, ctx->stream, hk, dt);
    launch_npt_apply(ctx->p, ctx->stream);
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
    launch_gather(ctx->p, ctx->stream, hk, dt, false);
    rec.end(KC_GATHER);
    rec.begin(KC_REDUCE);
    launch_reduce(ctx->p, ctx->stream, false, true);
    launch_npt_couple(ctx->p, ctx->stream, dt);
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
    rows *= ctx->p.n_sys;
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
md_status force_eval(md_ctx *ctx, bool full, bool fresh_only = false)
{
    if (full) {
        md_status s = ensure_wj(ctx);
        if (s != MD_OK) return s;
    }
    md_status s0 = clear_error_flags(ctx);
    if (s0 != MD_OK) return s0;
    if (fresh_only) {
        static const int one = 1;
        CK(cudaMemcpyAsync(&ctx->p.flags->fresh_only, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    }
    launch_displacement_check(ctx->p, ctx->stream);
    int rebuild = 0;
    CK(cudaMemcpyAsync(&rebuild, &ctx->p.flags->rebuild, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (rebuild) launch_rebuild(ctx->p, ctx->stream);
    launch_pair_reset(ctx->p, ctx->stream);
    launch_active_plan(ctx->p, ctx->stream);
    launch_pair(ctx->p, ctx->stream);
    launch_gather(ctx->p, ctx->stream, nullptr, 0.0, full);
    launch_reduce(ctx->p, ctx->stream, full, false);
    if (ctx->is_pool) launch_clear_fresh(ctx->p, ctx->stream);
    CK(cudaGetLastError());
    md_status s = check_flags(ctx);
    if (s != MD_OK) return s;
    ctx->forces_valid = true;
    return MD_OK;
}

// A graph of `steps` consecutive steps.  Inside it each step's first half-kick and drift
// run in the previous step's gather (not under NPT, whose scaling comes between them); the
// graph's first step launches its own kick, so every replay starts and ends on a state with
// x, v at the same time.  *kernels: kernels of one replay (rebuild bodies not counted).
md_status capture_one(md_ctx *ctx, const double *hk, double dt, int steps, cudaGraphExec_t *out, int *kernels)
{
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int per_step = 0;
    *kernels = 0;
    const bool fusable = !ctx->p.npt && ctx->p.N > 0;
    bool reduce_pending = false;
    for (int st = 0; st < steps; ++st) {
        md_status s = enqueue_step(ctx, Recorder{ctx, st, true}, hk, dt, &per_step, fusable && st > 0,
                                   fusable && st + 1 < steps, ctx->p.batch ? nullptr : &reduce_pending);
        *kernels += per_step;
        if (s != MD_OK) {
            cudaStreamEndCapture(ctx->stream, &g);
            if (g) cudaGraphDestroy(g);
            return s;
        }
    }
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    // honour the node priorities captured from the streams (the rebuild branch of a pool step
    // runs on a high-priority stream so that its short kernels go ahead of the pair pass)
    e = cudaGraphInstantiateWithFlags(out, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    ctx->kernels_per_step = per_step;
    return MD_OK;
}

md_status capture_graph(md_ctx *ctx, const double *hk, double dt)
{
    destroy_graph(ctx);
    md_status s = capture_one(ctx, hk, dt, kStepsPerGraph, &ctx->gexec, &ctx->kernels_g8);
    if (s != MD_OK) return s;
    s = capture_one(ctx, hk, dt, 1, &ctx->gexec1, &ctx->kernels_g1);
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

}  // extern "C"

namespace {

// Options common to single systems and pools; device, streams, kernel attributes.
md_status ctx_init(md_ctx *ctx, const md_options &opt)
{
    ctx->device = opt.device;
    ctx->io = opt.io;
    ctx->budget = opt.hbm_budget;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MD_ERR_CUDA;
    }
    if (opt.cuda_stream) {
        ctx->stream = static_cast<cudaStream_t>(opt.cuda_stream);
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return MD_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    // the rebuild branch of a pool step is a chain of short kernels beside a pair pass that
    // fills the GPU: its streams get the highest priority so that its blocks go first
    int prio_least = 0, prio_greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest) != cudaSuccess) {
        cudaGetLastError();
        prio_greatest = 0;
    }
    e = cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, prio_greatest);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&ctx->side2, cudaStreamNonBlocking, prio_greatest);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_red, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return MD_ERR_CUDA;
    }
    int n_sm = 0;
    if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess && n_sm > 0)
        ctx->p.n_sm = n_sm;
    cudaGetLastError();
    if (!configure_kernels(ctx->p)) return MD_ERR_CUDA;
    return MD_OK;
}

md_status check_options(const md_options &opt)
{
    if (opt.precision != MD_FP64 && opt.precision != MD_MIXED) return MD_ERR_ARG;
    if (opt.max_neigh < 1 || opt.max_neigh > kMaxListCap) return MD_ERR_ARG;
    if (opt.max_active < 0 || opt.max_active > 16) return MD_ERR_ARG;
    if (opt.skin < 0) return MD_ERR_ARG;
    return MD_OK;
}

void apply_options(Plan &p, const md_options &opt, int kind, double rc)
{
    p.kind = kind;
    p.precision = opt.precision;
    p.cap = opt.max_neigh;
    // SW: diamond Si's second shell sits 0.07 A outside the cutoff; several Tersoff elements:
    // zincblende SiC's second Si-Si shell (3.06 A) sits 0.06 A outside the Si-Si cutoff
    const int want_active = opt.max_active > 0 ? opt.max_active : ((kind == MD_SW || p.multi) ? 16 : 8);
    p.maxa = want_active <= 8 ? 8 : 16;
    p.rc = rc;
    p.skin = opt.skin > 0 ? opt.skin : 0.15 * rc;
    p.rl = p.rc + p.skin;
}

// Device arrays for p.N atoms, p.ncell cells, p.n_sys systems.
md_status ctx_alloc(md_ctx *ctx)
{
    Plan &p = ctx->p;
    md_status st = MD_OK;
    const size_t N1 = (size_t)(p.N > 0 ? p.N : 1);
    const size_t esz = p.precision == MD_FP64 ? sizeof(double) : sizeof(float);
#define AL(ptr, count)                                      \
    do {                                                    \
        st = dalloc_t(ctx, &(ptr), (size_t)(count));        \
        if (st != MD_OK) return st;                         \
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
    AL(p.ovf_count, 1);
    AL(p.ovf_list, N1);
    AL(p.sys_of, p.batch ? N1 : 1);
    AL(p.sys, (size_t)p.n_sys + 1);
    {
        void *v = nullptr;   // dU_i/dr_ij: one 4-word vector per compact row
        st = dalloc(ctx, &v, 4 * (size_t)p.maxa * N1 * esz);
        if (st != MD_OK) return st;
        p.pd = v;
        st = dalloc(ctx, &v, 3 * (size_t)p.maxa * N1 * esz);
        if (st != MD_OK) return st;
        p.pr = v;
    }
    if (!p.batch) AL(p.occ, (size_t)ctx->nc_full[0] + ctx->nc_full[1] + ctx->nc_full[2]);
    AL(p.cell_count, p.ncell);
    AL(p.cell_start, p.ncell);
    AL(p.cell_atoms, N1);
    AL(p.atom_cell, N1);
    AL(p.atom_rank, N1);
    p.nscanb = (p.ncell + scan_block_elems() - 1) / scan_block_elems();
    AL(p.scan_blocks, p.nscanb + 1);
    AL(p.rb_plan, 2);
    AL(p.rb_sys, (size_t)p.n_sys + 1);
    AL(p.rb_chunks, N1 / 128 + 1);
    AL(p.act_plan, 2);
    AL(p.act_chunks, N1 / 128 + 1);
    AL(p.stable_plan, 2);
    AL(p.stable_chunks, N1 / 128 + 1);
    p.nb_gather = gather_blocks(p.N);
    p.seg_max = 1;
    AL(p.partials, (size_t)p.nb_gather * kNumPartials);
    AL(p.totals, (size_t)p.n_sys * kNumPartials);
    AL(p.npt_totals, (size_t)p.n_sys * kNptExtra);
    AL(p.flags, 1);
#undef AL
    st = ensure_series(ctx, 1024);
    if (st != MD_OK) return st;
    cudaMemsetAsync(p.pos, 0, sizeof(double) * 3 * N1, ctx->stream);
    cudaMemsetAsync(p.vel, 0, sizeof(double) * 3 * N1, ctx->stream);
    cudaMemsetAsync(p.force, 0, sizeof(double) * 3 * N1, ctx->stream);
    cudaMemsetAsync(p.pos_build, 0, sizeof(double) * 3 * N1, ctx->stream);
    cudaMemsetAsync(p.flags, 0, sizeof(Flags), ctx->stream);
    cudaMemsetAsync(p.nn, 0, sizeof(int) * N1, ctx->stream);
    cudaMemsetAsync(p.mask, 0, sizeof(uint32_t) * N1, ctx->stream);
    cudaMemsetAsync(p.type, 0, sizeof(int) * N1, ctx->stream);
    cudaMemsetAsync(p.totals, 0, sizeof(double) * p.n_sys * kNumPartials, ctx->stream);
    cudaMemsetAsync(p.npt_totals, 0, sizeof(double) * p.n_sys * kNptExtra, ctx->stream);
    cudaMemsetAsync(p.act_plan, 0, sizeof(int) * 2, ctx->stream);
    cudaMemsetAsync(p.stable_plan, 0, sizeof(int) * 2, ctx->stream);
    cudaMemsetAsync(p.rb_plan, 0, sizeof(int) * 2, ctx->stream);
    return MD_OK;
}

md_status upload_sys_table(md_ctx *ctx)
{
    CK(cudaMemcpyAsync(ctx->p.sys, ctx->sys_host.data(), sizeof(SysDev) * ctx->sys_host.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    return MD_OK;
}

// Refresh the host copy of the system table (active flags, step budgets, rebuilds).
md_status download_sys_table(md_ctx *ctx)
{
    CK(cudaMemcpyAsync(ctx->sys_host.data(), ctx->p.sys, sizeof(SysDev) * ctx->sys_host.size(),
                       cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MD_OK;
}

}  // namespace

extern "C" {

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
    if (check_options(opt) != MD_OK) return MD_ERR_ARG;
    const int nt = params->n_types;   // several elements: Tersoff only
    if (nt < 1 || nt > kMaxTypes || (nt > 1 && params->kind != MD_TERSOFF)) return MD_ERR_ARG;
    for (int t = 0; t < nt; ++t)
        if (!(masses_by_type[t] > 0)) return MD_ERR_ARG;
    for (int64_t i = 0; i < n_atoms; ++i)
        if (types[i] < 0 || types[i] >= nt) return MD_ERR_ARG;

    md_ctx *ctx = new md_ctx();
    Plan &p = ctx->p;
    double rc = 0;
    if ((nt == 1 ? parse_params(params, p, 0, &rc) : parse_multi(params, p, &rc)) != MD_OK) {
        delete ctx;
        return MD_ERR_ARG;
    }
    apply_options(p, opt, params->kind, rc);
    p.N = n_atoms;
    p.ntypes = nt;
    p.n_sets = 1;
    for (int t = 0; t < nt; ++t) {
        p.mass[t] = masses_by_type[t];
        p.inv_mass[t] = 1.0 / masses_by_type[t];
    }
    double lmax = std::max(box[0], std::max(box[1], box[2]));
    p.list_margin = list_margin_for(lmax, p.rl);
    md_status st = system_box(p, p.rl, box, pbc, INT64_MAX, &p.box, p.nc);
    if (st != MD_OK) {
        delete ctx;
        return st;
    }
    p.ncell = (int64_t)p.nc[0] * p.nc[1] * p.nc[2];
    for (int a = 0; a < 3; ++a) ctx->nc_full[a] = p.nc[a];
    p.batch = false;
    p.n_sys = 1;
    if ((st = ctx_init(ctx, opt)) != MD_OK || (st = ctx_alloc(ctx)) != MD_OK) {
        md_destroy(ctx);
        return st;
    }
    // the one system, for the per-system reduce
    SysDev sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.box = p.box;
    sd.nc[0] = p.nc[0]; sd.nc[1] = p.nc[1]; sd.nc[2] = p.nc[2];
    sd.n_atoms = p.N;
    sd.steps_left = -1;
    sd.active = 1;
    sd.rc = p.rc;
    sd.rl = p.rl;
    sd.cell_edge = p.rl + p.list_margin;
    sd.half_skin2 = (float)(0.25 * p.skin * p.skin);
    sd.npt.mu_cum[0] = sd.npt.mu_cum[1] = sd.npt.mu_cum[2] = 1.0;
    ctx->sys_host.assign(2, SysDev{});
    ctx->sys_host[0] = sd;
    if ((st = upload_sys_table(ctx)) != MD_OK) {
        md_destroy(ctx);
        return st;
    }
    if (p.N > 0) cudaMemcpyAsync(p.type, types, sizeof(int32_t) * p.N, cudaMemcpyHostToDevice, ctx->stream);
    if (p.multi) {   // pair constants of every element pair, in the pair pass's precision
        std::vector<unsigned char> tab(tersoff_table_bytes(p));
        fill_tersoff_table(p, tab.data());
        if ((st = dalloc(ctx, &p.ttab, tab.size())) != MD_OK) {
            md_destroy(ctx);
            return st;
        }
        cudaMemcpyAsync(p.ttab, tab.data(), tab.size(), cudaMemcpyHostToDevice, ctx->stream);
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        md_destroy(ctx);
        return MD_ERR_CUDA;
    }
    *out = ctx;
    return MD_OK;
}

md_status md_batch_create(md_ctx **out, int64_t atom_capacity, int max_systems, int n_sets,
                          const md_params *param_sets, int n_types, const double *masses_by_type,
                          const md_batch_options *bopt, const md_options *opt_in)
{
    if (!out) return MD_ERR_ARG;
    *out = nullptr;
    if (atom_capacity < 1 || max_systems < 1 || n_sets < 1 || n_sets > kMaxSets || !param_sets ||
        n_types < 1 || n_types > kMaxTypes || !masses_by_type)
        return MD_ERR_ARG;
    md_options opt;
    if (opt_in) opt = *opt_in; else md_default_options(&opt);
    if (check_options(opt) != MD_OK) return MD_ERR_ARG;
    for (int t = 0; t < n_types; ++t)
        if (!(masses_by_type[t] > 0)) return MD_ERR_ARG;
    const int block = gather_block();
    const int64_t cap_atoms = (atom_capacity + block - 1) / block * block;
    if (cap_atoms > kMaxAtoms) return MD_ERR_ARG;

    md_ctx *ctx = new md_ctx();
    Plan &p = ctx->p;
    double rcmax = 0;
    for (int k = 0; k < n_sets; ++k) {
        double rc = 0;
        if (param_sets[k].kind != param_sets[0].kind || param_sets[k].n_types != 1 ||
            parse_params(&param_sets[k], p, k, &rc) != MD_OK) {
            delete ctx;
            return MD_ERR_ARG;
        }
        rcmax = std::max(rcmax, rc);
    }
    apply_options(p, opt, param_sets[0].kind, rcmax);
    ctx->skin_option = opt.skin;
    p.n_sets = n_sets;
    p.ntypes = n_types;
    for (int t = 0; t < n_types; ++t) {
        p.mass[t] = masses_by_type[t];
        p.inv_mass[t] = 1.0 / masses_by_type[t];
    }
    const double max_box = bopt && bopt->max_box > 0 ? bopt->max_box : 4096.0;
    p.list_margin = list_margin_for(max_box, p.rl);
    p.N = cap_atoms;
    p.batch = true;
    p.n_sys = max_systems;
    ctx->is_pool = true;
    ctx->min_atoms = 1;
    ctx->cell_capacity = bopt && bopt->cell_capacity > 0 ? bopt->cell_capacity : 4 * cap_atoms + 64;
    p.ncell = ctx->cell_capacity;
    md_status st;
    if ((st = ctx_init(ctx, opt)) != MD_OK || (st = ctx_alloc(ctx)) != MD_OK) {
        md_destroy(ctx);
        return st;
    }
    ctx->sys_host.assign((size_t)max_systems + 1, SysDev{});
    for (auto &sd : ctx->sys_host) {
        std::memset(&sd, 0, sizeof(sd));
        sd.steps_left = -1;
        for (int a = 0; a < 3; ++a) {
            sd.box.L[a] = 1.0;
            sd.box.invL[a] = 1.0;
            sd.nc[a] = 1;
        }
    }
    ctx->sys_used.assign((size_t)max_systems, 0);
    // cell counts start at zero; every rebuild zeroes the counts it used
    cudaMemsetAsync(p.cell_count, 0, sizeof(int) * (size_t)p.ncell, ctx->stream);
    ctx->atoms_free.init(cap_atoms);
    ctx->cells_free.init(ctx->cell_capacity);
    // every atom starts free: it belongs to the inactive sentinel system max_systems
    std::vector<int> sentinel((size_t)cap_atoms, max_systems);
    cudaMemcpyAsync(p.sys_of, sentinel.data(), sizeof(int) * cap_atoms, cudaMemcpyHostToDevice, ctx->stream);
    if ((st = upload_sys_table(ctx)) != MD_OK) {
        md_destroy(ctx);
        return st;
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        md_destroy(ctx);
        return MD_ERR_CUDA;
    }
    ctx->pos_set = true;
    ctx->forces_valid = true;
    *out = ctx;
    return MD_OK;
}

md_status md_batch_add(md_ctx *ctx, const md_system *sysd, int *id_out)
{
    if (!ctx || !sysd || !id_out) return MD_ERR_ARG;
    if (!ctx->is_pool) return fail(ctx, MD_ERR_STATE, "not a pool");
    Plan &p = ctx->p;
    const int64_t n = sysd->n_atoms;
    if (n < 1 || !sysd->types || !sysd->x || !sysd->y || !sysd->z) return fail(ctx, MD_ERR_ARG, "bad system");
    if (sysd->param_set < 0 || sysd->param_set >= p.n_sets) return fail(ctx, MD_ERR_ARG, "bad parameter set");
    if (!(sysd->damp >= 0)) return fail(ctx, MD_ERR_ARG, "bad damping");
    for (int64_t i = 0; i < n; ++i)
        if (sysd->types[i] < 0 || sysd->types[i] >= p.ntypes) return fail(ctx, MD_ERR_ARG, "bad type");
    if (ctx->io == MD_IO_HOST) {   // device inputs are checked by the first force evaluation
        const double *in[6] = {sysd->x, sysd->y, sysd->z, sysd->vx, sysd->vy, sysd->vz};
        for (int c = 0; c < 6; ++c)
            if (in[c])
                for (int64_t i = 0; i < n; ++i)
                    if (!std::isfinite(in[c][i])) return fail(ctx, MD_ERR_NAN, "non-finite position or velocity");
    }
    SysDev sd;
    std::memset(&sd, 0, sizeof(sd));
    // cutoff, skin and list radius of this system's parameter set
    const double rc = p.kind == MD_TERSOFF ? p.tp[sysd->param_set].S : p.sp[sysd->param_set].rc;
    const double skin = ctx->skin_option > 0 ? ctx->skin_option : 0.15 * rc;
    const double rl = rc + skin;
    sd.rlm2 = (float)((rl + p.list_margin) * (rl + p.list_margin));
    sd.half_skin2 = (float)(0.25 * skin * skin);
    sd.rc = rc;
    sd.rl = rl;
    sd.cell_edge = rl + p.list_margin;
    sd.npt.mu_cum[0] = sd.npt.mu_cum[1] = sd.npt.mu_cum[2] = 1.0;
    const int64_t max_cells = std::max<int64_t>(64, 4 * n);
    md_status st = system_box(p, rl, sysd->box, sysd->pbc, max_cells, &sd.box, sd.nc);
    if (st != MD_OK) return fail(ctx, st, "box too small for the cutoff");
    if (ctx->io == MD_IO_HOST) {
        const double *xyz[3] = {sysd->x, sysd->y, sysd->z};
        coarsen_sparse_axes(xyz, n, sd.box, sd.nc);
    }
    int id = -1;
    for (int k = 0; k < p.n_sys; ++k)
        if (!ctx->sys_used[k]) { id = k; break; }
    if (id < 0) return fail(ctx, MD_ERR_OOM, "no free system slot");
    const int block = gather_block();
    const int64_t len = (n + block - 1) / block * block;   // block-aligned: one system per gather block
    const int64_t a0 = ctx->atoms_free.alloc(len);
    if (a0 < 0) return fail(ctx, MD_ERR_OOM, "no room for the atoms");
    const int64_t ncell = (int64_t)sd.nc[0] * sd.nc[1] * sd.nc[2];
    const int64_t c0 = ctx->cells_free.alloc(ncell);
    if (c0 < 0) {
        ctx->atoms_free.release(a0, len);
        return fail(ctx, MD_ERR_OOM, "no room for the cell grid");
    }
    sd.pset = sysd->param_set;
    sd.cell_off = c0;
    sd.atom_start = a0;
    sd.n_atoms = n;
    sd.steps_left = sysd->n_steps < 0 ? -1 : sysd->n_steps;
    sd.damp = sysd->damp;
    sd.active = sysd->n_steps == 0 ? 0 : 1;
    sd.rebuild = 1;
    sd.fresh = 1;
    ctx->sys_host[id] = sd;
    ctx->sys_used[id] = 1;
    const cudaMemcpyKind k = ctx->io == MD_IO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const int64_t N = p.N;
    const double *src[6] = {sysd->x, sysd->y, sysd->z, sysd->vx, sysd->vy, sysd->vz};
    for (int c = 0; c < 3; ++c) {
        CK(cudaMemcpyAsync(p.pos + c * N + a0, src[c], sizeof(double) * n, k, ctx->stream));
        if (src[3 + c]) CK(cudaMemcpyAsync(p.vel + c * N + a0, src[3 + c], sizeof(double) * n, k, ctx->stream));
        else CK(cudaMemsetAsync(p.vel + c * N + a0, 0, sizeof(double) * n, ctx->stream));
        CK(cudaMemsetAsync(p.force + c * N + a0, 0, sizeof(double) * len, ctx->stream));
    }
    CK(cudaMemcpyAsync(p.type + a0, sysd->types, sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
    std::vector<int> ids((size_t)n, id);
    CK(cudaMemcpyAsync(p.sys_of + a0, ids.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(&p.sys[id], &ctx->sys_host[id], sizeof(SysDev), cudaMemcpyHostToDevice, ctx->stream));
    static const int one = 1;
    CK(cudaMemcpyAsync(&p.flags->rebuild, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->forces_valid = false;   // the new system needs forces before its first kick
    *id_out = id;
    return MD_OK;
}

md_status md_batch_remove(md_ctx *ctx, int id)
{
    if (!ctx) return MD_ERR_ARG;
    if (!ctx->is_pool || id < 0 || id >= ctx->p.n_sys || !ctx->sys_used[id])
        return fail(ctx, MD_ERR_ARG, "no such system");
    Plan &p = ctx->p;
    const SysDev sd = ctx->sys_host[id];
    const int block = gather_block();
    const int64_t len = (sd.n_atoms + block - 1) / block * block;
    std::vector<int> ids((size_t)sd.n_atoms, p.n_sys);
    CK(cudaMemcpyAsync(p.sys_of + sd.atom_start, ids.data(), sizeof(int) * sd.n_atoms, cudaMemcpyHostToDevice,
                       ctx->stream));
    SysDev off;
    std::memset(&off, 0, sizeof(off));
    off.steps_left = -1;
    for (int a = 0; a < 3; ++a) {
        off.box.L[a] = 1.0;
        off.box.invL[a] = 1.0;
        off.nc[a] = 1;
    }
    ctx->sys_host[id] = off;
    CK(cudaMemcpyAsync(&p.sys[id], &ctx->sys_host[id], sizeof(SysDev), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->atoms_free.release(sd.atom_start, len);
    ctx->cells_free.release(sd.cell_off, (int64_t)sd.nc[0] * sd.nc[1] * sd.nc[2]);
    ctx->sys_used[id] = 0;
    return MD_OK;
}

md_status md_batch_status(md_ctx *ctx, int *active, int64_t *steps_left, double *totals, double *kinetic)
{
    if (!ctx) return MD_ERR_ARG;
    if (!ctx->is_pool) return fail(ctx, MD_ERR_STATE, "not a pool");
    md_status s = download_sys_table(ctx);
    if (s != MD_OK) return s;
    const int n = ctx->p.n_sys;
    std::vector<double> t((size_t)n * kNumPartials);
    CK(cudaMemcpy(t.data(), ctx->p.totals, sizeof(double) * t.size(), cudaMemcpyDeviceToHost));
    for (int k = 0; k < n; ++k) {
        const bool used = ctx->sys_used[k] != 0;
        if (active) active[k] = used ? (ctx->sys_host[k].active ? 1 : 0) : -1;
        if (steps_left) steps_left[k] = used ? ctx->sys_host[k].steps_left : 0;
        if (kinetic) kinetic[k] = t[(size_t)k * kNumPartials + 1];
        if (totals) {
            double *o = totals + (size_t)k * 13;
            const double *q = t.data() + (size_t)k * kNumPartials;
            o[0] = q[0];
            for (int c = 0; c < 9; ++c) o[1 + c] = q[5 + c];
            for (int c = 0; c < 3; ++c) o[10 + c] = q[2 + c];
        }
    }
    return MD_OK;
}

md_status md_batch_errors(md_ctx *ctx, int *status)
{
    if (!ctx || !status) return MD_ERR_ARG;
    if (!ctx->is_pool) return fail(ctx, MD_ERR_STATE, "not a pool");
    md_status s = download_sys_table(ctx);
    if (s != MD_OK) return s;
    for (int k = 0; k < ctx->p.n_sys; ++k) status[k] = ctx->sys_used[k] ? ctx->sys_host[k].error : 0;
    return MD_OK;
}

md_status md_batch_get_state(md_ctx *ctx, int id, double *x, double *v)
{
    if (!ctx) return MD_ERR_ARG;
    if (!ctx->is_pool || id < 0 || id >= ctx->p.n_sys || !ctx->sys_used[id])
        return fail(ctx, MD_ERR_ARG, "no such system");
    const Plan &p = ctx->p;
    const SysDev &sd = ctx->sys_host[id];
    const cudaMemcpyKind k = ctx->io == MD_IO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (x) {
        launch_wrap_copy(p, ctx->stream, p.stage, sd.atom_start, sd.n_atoms);
        for (int c = 0; c < 3; ++c)
            CK(cudaMemcpyAsync(x + c * sd.n_atoms, p.stage + c * p.N + sd.atom_start, sizeof(double) * sd.n_atoms, k,
                               ctx->stream));
    }
    if (v)
        for (int c = 0; c < 3; ++c)
            CK(cudaMemcpyAsync(v + c * sd.n_atoms, p.vel + c * p.N + sd.atom_start, sizeof(double) * sd.n_atoms, k,
                               ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MD_OK;
}

md_status md_set_positions(md_ctx *ctx, const double *x, const double *y, const double *z)
{
    if (!ctx) return MD_ERR_ARG;
    if (ctx->is_pool) return fail(ctx, MD_ERR_STATE, "pools take positions through md_batch_add");
    if (ctx->p.N > 0 && (!x || !y || !z)) return fail(ctx, MD_ERR_ARG, "NULL position array");
    if (ctx->p.N > 0) {
        md_status s = upload3(ctx, ctx->p.pos, x, y, z);
        if (s != MD_OK) return s;
        if (ctx->p.npt) {   // the barostat may have scaled the box: take the device's
            if ((s = download_sys_table(ctx)) != MD_OK) return s;
            ctx->p.box = ctx->sys_host[0].box;
        }
        // cell grid for this box and configuration (within the allocated cells)
        int nc[3] = {ctx->nc_full[0], ctx->nc_full[1], ctx->nc_full[2]};
        if (ctx->p.npt)
            for (int a = 0; a < 3; ++a) {
                const int fit = (int)std::floor(ctx->p.box.L[a] / ctx->sys_host[0].cell_edge);
                nc[a] = std::max(1, std::min(nc[a], fit));
            }
        if ((s = coarsen_sparse_axes_dev(ctx, nc)) != MD_OK) return s;
        if (nc[0] != ctx->p.nc[0] || nc[1] != ctx->p.nc[1] || nc[2] != ctx->p.nc[2]) {
            for (int a = 0; a < 3; ++a) ctx->p.nc[a] = nc[a];
            ctx->p.ncell = (int64_t)nc[0] * nc[1] * nc[2];
            destroy_graph(ctx);   // the graphs carry the grid in their arguments
        }
        // the system entry: same grid; new positions drop a pending Berendsen scaling
        for (int a = 0; a < 3; ++a) ctx->sys_host[0].nc[a] = nc[a];
        ctx->sys_host[0].npt.pending = 0;
        CK(cudaMemcpyAsync(&ctx->p.sys[0], &ctx->sys_host[0], sizeof(SysDev), cudaMemcpyHostToDevice, ctx->stream));
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
    if (ctx->is_pool) return fail(ctx, MD_ERR_STATE, "pools take velocities through md_batch_add");
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
    std::vector<double> all((size_t)ctx->p.n_sys * kNumPartials);
    CK(cudaMemcpyAsync(all.data(), ctx->p.totals, sizeof(double) * all.size(), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (totals) {
        double t[kNumPartials] = {0};
        for (int k = 0; k < ctx->p.n_sys; ++k)   // systems in index order
            if (!ctx->is_pool || ctx->sys_used[k])
                for (int c = 0; c < kNumPartials; ++c) t[c] += all[(size_t)k * kNumPartials + c];
        totals[0] = t[0];                                       // U
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
    if (!ctx->forces_valid) {   // pools: forces for the systems admitted since the last call
        s = force_eval(ctx, false, ctx->is_pool);
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
            ctx->kernels_launched += (ctx->p.N > 0 ? 6 : 2) + (ctx->p.batch ? 1 : 0) +
                                     (ctx->p.npt && ctx->p.N > 0 ? 2 : 0);
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
            ctx->kernels_launched += ctx->kernels_g8;
            if (ctx->profiling) {
                s = accumulate_times(ctx, kStepsPerGraph);
                if (s != MD_OK) return s;
            }
            done += kStepsPerGraph;
        }
        for (; done < n_steps; ++done) {
            CK(cudaGraphLaunch(ctx->gexec1, ctx->stream));
            ctx->kernels_launched += ctx->kernels_g1;
            if (ctx->profiling) {
                s = accumulate_times(ctx, 1);
                if (s != MD_OK) return s;
            }
        }
    }
    if (series) {
        const cudaMemcpyKind k = ctx->io == MD_IO_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CK(cudaMemcpyAsync(series, ctx->p.series, sizeof(double) * 5 * n_steps * ctx->p.n_sys, k, ctx->stream));
    }
    s = check_flags(ctx);
    ctx->steps_done += n_steps;
    if (s != MD_OK) {
        ctx->forces_valid = false;
        return s;
    }
    return adapt_staging(ctx);
}

md_status md_set_npt(md_ctx *ctx, int system, const md_npt *npt)
{
    if (!ctx) return MD_ERR_ARG;
    const bool pool = ctx->is_pool;
    if (system < 0 || system >= ctx->p.n_sys || (pool && !ctx->sys_used[system]))
        return fail(ctx, MD_ERR_ARG, "no such system");
    if (npt) {
        const bool ok = std::isfinite(npt->T0) && npt->T0 >= 0 && std::isfinite(npt->P0) &&
                        std::isfinite(npt->tau_T) && std::isfinite(npt->tau_P) && std::isfinite(npt->beta) &&
                        npt->beta >= 0;
        if (!ok) return fail(ctx, MD_ERR_ARG, "bad NPT coupling parameters");
        for (int a = 0; a < 3; ++a)
            if (npt->couple[a] != 0 && npt->couple[a] != 1) return fail(ctx, MD_ERR_ARG, "couple[] must be 0 or 1");
    }
    md_status s = download_sys_table(ctx);   // current device state: box, budgets, scaling
    if (s != MD_OK) return s;
    SysDev &sd = ctx->sys_host[system];
    const bool was_on = sd.npt.on != 0;
    if (npt) {
        sd.npt.on = 1;
        sd.npt.T0 = npt->T0;
        sd.npt.P0 = npt->P0;
        sd.npt.tau_T = npt->tau_T;
        sd.npt.tau_P = npt->tau_P;
        sd.npt.beta = npt->beta;
        for (int a = 0; a < 3; ++a) sd.npt.couple[a] = npt->couple[a];
        if (!was_on) {
            sd.npt.pending = 0;
            sd.npt.lam = 1.0;
            sd.npt.mu[0] = sd.npt.mu[1] = sd.npt.mu[2] = 1.0;
        }
    } else {
        // back to NVE: drop a pending scaling; the plain skin test is exact only for a
        // list built in the current box, so rebuild
        sd.npt.on = 0;
        sd.npt.pending = 0;
        if (was_on) sd.rebuild = 1;
    }
    CK(cudaMemcpyAsync(&ctx->p.sys[system], &sd, sizeof(SysDev), cudaMemcpyHostToDevice, ctx->stream));
    if (!npt && was_on) {
        s = set_flag_rebuild(ctx);
        if (s != MD_OK) return s;
    }
    bool any = false;
    for (int k = 0; k < ctx->p.n_sys; ++k)
        if ((!pool || ctx->sys_used[k]) && ctx->sys_host[k].npt.on) any = true;
    // pools keep the NPT step once a system was coupled (uncoupled systems are unaffected);
    // a single system returns to the by-value box and grid of the NVE step
    const bool want = pool ? (ctx->p.npt || any) : any;
    if (want != ctx->p.npt) {
        if (!pool && !want) {
            ctx->p.box = ctx->sys_host[0].box;
            for (int a = 0; a < 3; ++a) ctx->p.nc[a] = ctx->sys_host[0].nc[a];
            ctx->p.ncell = (int64_t)ctx->p.nc[0] * ctx->p.nc[1] * ctx->p.nc[2];
        }
        ctx->p.npt = want;
        destroy_graph(ctx);
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return MD_OK;
}

md_status md_get_box(md_ctx *ctx, int system, double box[3])
{
    if (!ctx || !box) return MD_ERR_ARG;
    if (system < 0 || system >= ctx->p.n_sys || (ctx->is_pool && !ctx->sys_used[system]))
        return fail(ctx, MD_ERR_ARG, "no such system");
    SysDev sd;
    CK(cudaMemcpyAsync(&sd, &ctx->p.sys[system], sizeof(SysDev), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int a = 0; a < 3; ++a) box[a] = sd.box.L[a];
    return MD_OK;
}

md_status md_get_state(md_ctx *ctx, double *x, double *v)
{
    if (!ctx) return MD_ERR_ARG;
    md_status s;
    if (x && ctx->p.N > 0) {
        // positions move unwrapped between list builds; report them wrapped into the box
        launch_wrap_copy(ctx->p, ctx->stream, ctx->p.stage, 0, ctx->p.N);
        if ((s = download(ctx, x, ctx->p.stage, 3 * ctx->p.N)) != MD_OK) return s;
    }
    if ((s = download(ctx, v, ctx->p.vel, 3 * ctx->p.N)) != MD_OK) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    return MD_OK;
}

}  // extern "C"

namespace {

// Checkpoint image of a single-system context: a header, then the device state that the
// next step reads, in this order: positions (as stored: unwrapped since the last list
// build), velocities, forces, build positions (3N doubles each), fp32 positions (3N
// floats), list lengths (N ints), list entries (cap N ints), reverse slots (cap N bytes).
constexpr uint64_t kCheckpointMagic = 0x3130315444504b43ull;   // "CKPDT101"
struct CheckpointHeader {
    uint64_t magic;
    int64_t n_atoms;
    int32_t kind, precision, cap, maxa, ntypes, n_elem;
    int32_t pos_set, forces_valid, npt, pad;
    int64_t steps_done;
    double mass[kMaxTypes];
    double skin;
    TersoffP tp;       // parameter set 0 (a restored context must use the same potential)
    SWP sp;
    SysDev sys;        // box, cell grid, Berendsen state
    Flags flags;       // pending rebuild request, counters
};

size_t checkpoint_bytes(const Plan &p)
{
    const size_t N = (size_t)p.N;
    return sizeof(CheckpointHeader) + 4 * 3 * N * sizeof(double) + 3 * N * sizeof(float) + N * sizeof(int) +
           (size_t)p.cap * N * (sizeof(int) + sizeof(uint8_t));
}

struct Section {
    void *dev;
    size_t bytes;
};

std::vector<Section> checkpoint_sections(const Plan &p)
{
    const size_t N = (size_t)p.N;
    return {{p.pos, 3 * N * sizeof(double)},       {p.vel, 3 * N * sizeof(double)},
            {p.force, 3 * N * sizeof(double)},     {p.pos_build, 3 * N * sizeof(double)},
            {p.posf, 3 * N * sizeof(float)},       {p.nn, N * sizeof(int)},
            {p.nl, (size_t)p.cap * N * sizeof(int)}, {p.rev, (size_t)p.cap * N * sizeof(uint8_t)}};
}

}  // namespace

extern "C" {

md_status md_checkpoint_size(md_ctx *ctx, size_t *bytes)
{
    if (!ctx || !bytes) return MD_ERR_ARG;
    if (ctx->is_pool) return fail(ctx, MD_ERR_STATE, "checkpoints cover single-system contexts");
    *bytes = checkpoint_bytes(ctx->p);
    return MD_OK;
}

md_status md_checkpoint_save(md_ctx *ctx, void *buf, size_t bytes)
{
    if (!ctx || !buf) return MD_ERR_ARG;
    if (ctx->is_pool) return fail(ctx, MD_ERR_STATE, "checkpoints cover single-system contexts");
    const Plan &p = ctx->p;
    if (bytes < checkpoint_bytes(p)) return fail(ctx, MD_ERR_ARG, "checkpoint buffer too small");
    CheckpointHeader h;
    std::memset(&h, 0, sizeof(h));
    h.magic = kCheckpointMagic;
    h.n_atoms = p.N;
    h.kind = p.kind;
    h.precision = p.precision;
    h.cap = p.cap;
    h.maxa = p.maxa;
    h.ntypes = p.ntypes;
    h.n_elem = p.n_elem;
    h.pos_set = ctx->pos_set ? 1 : 0;
    h.forces_valid = ctx->forces_valid ? 1 : 0;
    h.npt = p.npt ? 1 : 0;
    h.steps_done = ctx->steps_done;
    for (int t = 0; t < kMaxTypes; ++t) h.mass[t] = p.mass[t];
    h.skin = p.skin;
    h.tp = p.tp[0];
    h.sp = p.sp[0];
    CK(cudaMemcpyAsync(&h.sys, p.sys, sizeof(SysDev), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&h.flags, p.flags, sizeof(Flags), cudaMemcpyDeviceToHost, ctx->stream));
    unsigned char *o = static_cast<unsigned char *>(buf) + sizeof(CheckpointHeader);
    for (const Section &sec : checkpoint_sections(p)) {
        if (sec.bytes) CK(cudaMemcpyAsync(o, sec.dev, sec.bytes, cudaMemcpyDeviceToHost, ctx->stream));
        o += sec.bytes;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    std::memcpy(buf, &h, sizeof(h));
    return MD_OK;
}

md_status md_checkpoint_load(md_ctx *ctx, const void *buf, size_t bytes)
{
    if (!ctx || !buf) return MD_ERR_ARG;
    if (ctx->is_pool) return fail(ctx, MD_ERR_STATE, "checkpoints cover single-system contexts");
    Plan &p = ctx->p;
    if (bytes < sizeof(CheckpointHeader)) return fail(ctx, MD_ERR_ARG, "not a checkpoint");
    CheckpointHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kCheckpointMagic) return fail(ctx, MD_ERR_ARG, "not a checkpoint");
    const bool same = h.n_atoms == p.N && h.kind == p.kind && h.precision == p.precision && h.cap == p.cap &&
                      h.maxa == p.maxa && h.ntypes == p.ntypes && h.n_elem == p.n_elem && h.skin == p.skin &&
                      std::memcmp(h.mass, p.mass, sizeof(h.mass)) == 0 &&
                      std::memcmp(&h.tp, &p.tp[0], sizeof(TersoffP)) == 0 &&
                      std::memcmp(&h.sp, &p.sp[0], sizeof(SWP)) == 0;
    if (!same) return fail(ctx, MD_ERR_ARG, "checkpoint of a context with other atoms, potential or options");
    if (bytes < checkpoint_bytes(p)) return fail(ctx, MD_ERR_ARG, "checkpoint truncated");
    for (int a = 0; a < 3; ++a)
        if (h.sys.nc[a] < 1 || h.sys.nc[a] > ctx->nc_full[a] || h.sys.box.pbc[a] != p.box.pbc[a])
            return fail(ctx, MD_ERR_ARG, "checkpoint cell grid or periodicity does not fit this context");
    const unsigned char *o = static_cast<const unsigned char *>(buf) + sizeof(CheckpointHeader);
    for (const Section &sec : checkpoint_sections(p)) {
        if (sec.bytes) CK(cudaMemcpyAsync(sec.dev, o, sec.bytes, cudaMemcpyHostToDevice, ctx->stream));
        o += sec.bytes;
    }
    CK(cudaMemcpyAsync(p.sys, &h.sys, sizeof(SysDev), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(p.flags, &h.flags, sizeof(Flags), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->sys_host[0] = h.sys;
    p.box = h.sys.box;
    for (int a = 0; a < 3; ++a) p.nc[a] = h.sys.nc[a];
    p.ncell = (int64_t)p.nc[0] * p.nc[1] * p.nc[2];
    p.npt = h.npt != 0;
    ctx->pos_set = h.pos_set != 0;
    ctx->forces_valid = h.forces_valid != 0;
    ctx->steps_done = h.steps_done;
    destroy_graph(ctx);   // the graphs carry the box and grid in their arguments
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
    int deferred = 0;
    CK(cudaMemcpy(&deferred, ctx->p.ovf_count, sizeof(int), cudaMemcpyDeviceToHost));
    out->pair_deferred = deferred;
    out->device_bytes = ctx->allocated;
    out->atoms_rebuilt = f.atoms_rebuilt;
    out->kernels_launched = ctx->kernels_launched;
    return MD_OK;
}

md_status md_set_graph_mode(md_ctx *ctx, int use_graphs)
{
    if (!ctx) return MD_ERR_ARG;
    ctx->use_graphs = use_graphs != 0;
    return MD_OK;
}

}  // extern "C"

namespace {

// Mean time of `repeats` launch sequences (pair pass, and the gather without the
// half-kick when `with_gather`) on the context's stream, after one untimed sequence.
// The sequence recomputes the current forces from the current positions and list, so it
// changes no state.
md_status time_launches(md_ctx *ctx, int repeats, bool with_gather, double *ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CK(cudaEventCreate(&e0));
    cudaError_t e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(ctx, e, "cudaEventCreate");
    }
    auto seq = [&]() {
        launch_pair_reset(ctx->p, ctx->stream);
        launch_active_plan(ctx->p, ctx->stream);
        launch_pair(ctx->p, ctx->stream);
        if (with_gather) launch_gather(ctx->p, ctx->stream, nullptr, 0.0, false);
    };
    seq();
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < repeats; ++r) seq();
    cudaEventRecord(e1, ctx->stream);
    e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune timing");
    *ms = (double)t / repeats;
    return MD_OK;
}

void fill_tuning(const md_ctx *ctx, md_tuning *out)
{
    out->pair_block = effective_pair_block(ctx->p);
    out->pool_blocks_per_sm = ctx->p.pool_bps;
    out->pair_cap = effective_pair_cap(ctx->p);
}

}  // namespace

extern "C" {

md_status md_autotune(md_ctx *ctx, int repeats, md_tuning *out)
{
    if (!ctx) return MD_ERR_ARG;
    if (repeats < 0 || repeats > 10000) return fail(ctx, MD_ERR_ARG, "repeats out of range");
    if (repeats == 0) repeats = 10;
    if (!ctx->pos_set && ctx->p.N > 0) return fail(ctx, MD_ERR_STATE, "positions not set");
    md_tuning res;
    std::memset(&res, 0, sizeof(res));
    if (ctx->p.N > 0) {
        md_status s;
        if (!ctx->forces_valid) {   // lists (and forces) for the current positions
            s = force_eval(ctx, false, ctx->is_pool);
            if (s != MD_OK) return s;
        }
        s = clear_error_flags(ctx);
        if (s != MD_OK) return s;
        static const int blocks[] = {32, 64, 128, 256};
        double best = 0.0;
        int best_b = effective_pair_block(ctx->p), best_c = ctx->p.pair_cap;
        // bond slots of the common-case pass: 4, and 3 where that staging exists
        int caps[2] = {4, 3};
        ctx->p.pair_cap = 3;
        const int n_caps = effective_pair_cap(ctx->p) == 3 ? 2 : 1;
        for (int ci = 0; ci < n_caps; ++ci) {
            ctx->p.pair_cap = caps[ci];
            for (int b : blocks) {
                ctx->p.pair_block = b;
                double ms = 0.0;
                s = time_launches(ctx, repeats, false, &ms);
                if (s != MD_OK) return s;
                res.tried_pair_block[res.n_tried] = b;
                res.tried_blocks_per_sm[res.n_tried] = ctx->p.pool_bps;
                res.tried_pair_cap[res.n_tried] = effective_pair_cap(ctx->p);
                res.tried_ms[res.n_tried++] = ms;
                if (best == 0.0 || ms < best) {
                    best = ms;
                    best_b = b;
                    best_c = caps[ci];
                }
            }
        }
        ctx->p.pair_block = best_b;
        ctx->p.pair_cap = best_c;
        if (ctx->is_pool) {
            static const int bps[] = {4, 8, 16, 32, 64};
            best = 0.0;
            int best_g = ctx->p.pool_bps;
            for (int g : bps) {
                ctx->p.pool_bps = g;
                double ms = 0.0;
                s = time_launches(ctx, repeats, true, &ms);
                if (s != MD_OK) return s;
                res.tried_pair_block[res.n_tried] = best_b;
                res.tried_blocks_per_sm[res.n_tried] = g;
                res.tried_pair_cap[res.n_tried] = effective_pair_cap(ctx->p);
                res.tried_ms[res.n_tried++] = ms;
                if (best == 0.0 || ms < best) {
                    best = ms;
                    best_g = g;
                }
            }
            ctx->p.pool_bps = best_g;
        }
        s = check_flags(ctx);
        if (s != MD_OK) return s;
        destroy_graph(ctx);   // the next md_run captures with the chosen launches
    }
    fill_tuning(ctx, &res);
    if (out) *out = res;
    return MD_OK;
}

md_status md_set_tuning(md_ctx *ctx, const md_tuning *t)
{
    if (!ctx || !t) return MD_ERR_ARG;
    if (t->pair_block != 0 && !valid_pair_block(t->pair_block))
        return fail(ctx, MD_ERR_ARG, "pair_block must be 0, 32, 64, 128 or 256");
    if (t->pool_blocks_per_sm < 1 || t->pool_blocks_per_sm > 64)
        return fail(ctx, MD_ERR_ARG, "pool_blocks_per_sm must be in 1..64");
    if (t->pair_cap != 0 && t->pair_cap != 3 && t->pair_cap != 4)
        return fail(ctx, MD_ERR_ARG, "pair_cap must be 0, 3 or 4");
    ctx->p.pair_block = t->pair_block;
    ctx->p.pool_bps = t->pool_blocks_per_sm;
    ctx->p.pair_cap = t->pair_cap;
    destroy_graph(ctx);
    return MD_OK;
}

md_status md_get_tuning(md_ctx *ctx, md_tuning *out)
{
    if (!ctx || !out) return MD_ERR_ARG;
    std::memset(out, 0, sizeof(*out));
    fill_tuning(ctx, out);
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
    if (ctx->side2) cudaStreamDestroy(ctx->side2);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    if (ctx->ev_red) cudaEventDestroy(ctx->ev_red);
    delete ctx;
}

}  // extern "C"

namespace mdk {

// Parameter and option parsing shared with the spatial decomposition (md_domain.cu).
md_status plan_params(const md_params *params, Plan &p, int idx, double *rc)
{
    return parse_params(params, p, idx, rc);
}
md_status plan_options(Plan &p, const md_options &opt, int kind, double rc)
{
    if (check_options(opt) != MD_OK) return MD_ERR_ARG;
    apply_options(p, opt, kind, rc);
    return MD_OK;
}

}  // namespace mdk
