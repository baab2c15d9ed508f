// md_domain.cu -- spatial decomposition of one system over ranks: slabs along one periodic
// axis, each rank running the force path on its own atoms plus a ghost shell.
//
// The paper runs one system on one GPU and quotes LAMMPS's MPI runs only for comparison
// (Sec. 3).  Splitting one system needs a halo: dU_j/dr_ji of a neighbour j of an owned atom
// depends on j's own neighbours (Eqs. 14, 28), so a rank holds, besides the atoms of its slab
// [lo, hi), every atom within G = 2 (r_list + margin) of the slab -- the neighbours of its
// atoms and their neighbours.  The rank then computes dU_j/dr_ji of its first-shell ghosts
// itself, and one exchange per step (the ghosts' positions) suffices.
//
// Per step, with the transport between the calls supplied by the caller:
//   md_domain_kick_drift   v += F/m dt/2, x += v dt on the owned atoms; local skin test
//   (caller: OR of the skin tests over the ranks)
//   no rebuild:  pack/unpack MD_DOMAIN_POSITIONS   ghosts' new positions from their owners
//   rebuild:     pack/unpack MD_DOMAIN_MIGRATE     atoms that left the slab, to their new rank
//                pack/unpack MD_DOMAIN_GHOSTS      the new ghost sets, then a list build
//   md_domain_force        pair pass over owned + ghosts, gather + second half-kick over
//                          the owned atoms; the rank's totals (the caller sums them)
// Ghosts are not integrated, gathered or summed (Plan::n_owned).  Between rebuilds the
// ghost sets are fixed: a ghost is refreshed from the same owner atom every step.
//
// Frames.  Along the decomposition axis a rank stores local coordinates x - origin, origin =
// lo - G, and treats the axis as open (the local box lo - G .. hi + G never wraps; slabs are
// at least 2G wide).  A position sent to the left neighbour gets +L along the axis when the
// sender is rank 0 and one sent right gets -L when it is the last rank, so that ghosts lie
// next to the receiver's slab.  At every rebuild all positions are wrapped into [0, L) on
// periodic axes before ghosts are chosen, so a ghost's owner and its copies see the same
// coordinates until the next rebuild (the list's image shifts stay valid for both).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "md.h"
#include "md_plan.cuh"

using namespace mdk;

namespace {

struct MsgHeader {
    int64_t count;
    int64_t mode;
};
struct MigrantRec {   // an atom changing rank: its id, element, position (global), velocity
    int64_t id;
    int32_t type, pad;
    double x[3], v[3];
};
struct GhostRec {     // a ghost: its id, element, position (global, shifted for the receiver)
    int64_t id;
    int32_t type, pad;
    double x[3];
};

// out[3k + c] = position c of atom idx[k], plus `offset` along the decomposition axis
__global__ void k_domain_pack(int64_t n, const int *idx, const double *pos, int64_t N, int axis, double offset,
                              double *out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t i = idx[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * k + c] = pos[c * N + i] + (c == axis ? offset : 0.0);
}

// positions of atoms first .. first + n - 1 from in[3k + c], minus `offset` along the axis,
// and their fp32 copies (the SW and fp64 Tersoff pair passes prefilter bonds with them, as
// the kick keeps them for the owned atoms)
__global__ void k_domain_unpack(int64_t n, int64_t first, double *pos, float *posf, int64_t N, int axis,
                                double offset, const double *in)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double x = in[3 * k + c] - (c == axis ? offset : 0.0);
        pos[c * N + first + k] = x;
        posf[c * N + first + k] = d2f_trunc(x);
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

double wrap(double x, double L)
{
    x -= L * std::floor(x / L);
    if (x >= L) x -= L;
    if (x < 0.0) x += L;
    return x;
}

enum Phase { PH_EMPTY = 0, PH_NEED_GHOSTS = 1, PH_MIGRATING = 2, PH_READY = 3 };

}  // namespace

struct md_domain {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Plan p;
    int64_t capacity = 0;
    std::vector<void *> allocs;
    int axis = 0, n_ranks = 1, rank = 0;
    double L[3] = {0, 0, 0};
    int pbc[3] = {1, 1, 1};
    double lo = 0, hi = 0, G = 0, origin = 0;
    double shift_left = 0, shift_right = 0;   // added along the axis to positions sent left / right
    // host view of the local atoms: owned [0, n_owned), then ghosts from the left neighbour,
    // then ghosts from the right neighbour
    std::vector<int64_t> id;
    std::vector<int32_t> type;
    int64_t n_owned = 0, n_left = 0, n_right = 0;
    // owned atoms while their ghosts are pending (global frame, wrapped): x, v as 3 per atom
    std::vector<double> hx, hv;
    std::vector<int32_t> send_left, send_right;   // owned indices whose positions go left / right
    int phase = PH_EMPTY;
    bool need_build = false, forces_valid = false;
    int *d_idx = nullptr;       // send lists on the device: left, then right
    double *d_stage = nullptr;  // 3 x capacity positions in transit
    std::vector<double> h_stage;
    std::string err;
};

namespace {

md_status dfail(md_domain *d, md_status s, const std::string &m)
{
    if (d) d->err = m;
    return s;
}

#define DCK(call)                                                                   \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            cudaGetLastError();                                                     \
            return dfail(dom, MD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                           \
    } while (0)

template <typename P>
md_status dalloc(md_domain *dom, P **ptr, size_t count)
{
    void *v = nullptr;
    if (cudaMalloc(&v, std::max<size_t>(16, count * sizeof(P))) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return dfail(dom, MD_ERR_OOM, "device allocation failed");
    }
    dom->allocs.push_back(v);
    *ptr = static_cast<P *>(v);
    return MD_OK;
}

size_t bound_bytes(const md_domain *dom, int mode)
{
    const size_t n = (size_t)std::max<int64_t>(dom->n_owned, (int64_t)dom->hx.size() / 3);
    if (mode == MD_DOMAIN_POSITIONS) return sizeof(MsgHeader) + 3 * sizeof(double) * n;
    if (mode == MD_DOMAIN_MIGRATE) return sizeof(MsgHeader) + sizeof(MigrantRec) * n;
    return sizeof(MsgHeader) + sizeof(GhostRec) * n;
}

md_status check_device_flags(md_domain *dom)
{
    Flags f;
    DCK(cudaMemcpyAsync(&f, dom->p.flags, sizeof(Flags), cudaMemcpyDeviceToHost, dom->stream));
    DCK(cudaStreamSynchronize(dom->stream));
    if (f.list_overflow) return dfail(dom, MD_ERR_NEIGH_OVERFLOW, "neighbour list longer than max_neigh");
    if (f.active_overflow) return dfail(dom, MD_ERR_NEIGH_OVERFLOW, "more in-cutoff neighbours than max_active");
    if (f.asym) return dfail(dom, MD_ERR_CUDA, "internal: asymmetric neighbour list");
    if (f.nonfinite) return dfail(dom, MD_ERR_NAN, "non-finite force, position or velocity");
    return MD_OK;
}

md_status clear_flags(md_domain *dom)
{
    static const int zeros[5] = {0, 0, 0, 0, 0};   // rebuild, list/active overflow, nonfinite, asym
    DCK(cudaMemcpyAsync(&dom->p.flags->rebuild, zeros, sizeof(zeros), cudaMemcpyHostToDevice, dom->stream));
    return MD_OK;
}

// Upload the assembled local system (owned atoms from hx/hv, ghosts from the received
// records) and the send lists; the next force evaluation builds the list.
md_status assemble(md_domain *dom, const std::vector<GhostRec> &ghosts)
{
    Plan &p = dom->p;
    const int64_t no = dom->n_owned, N = no + (int64_t)ghosts.size();
    if (N > dom->capacity)
        return dfail(dom, MD_ERR_OOM, "owned atoms and ghosts (" + std::to_string(N) + ") exceed the capacity");
    std::vector<double> pos((size_t)3 * N), vel((size_t)3 * N, 0.0);
    std::vector<int32_t> ty((size_t)N);
    for (int64_t i = 0; i < no; ++i) {
        for (int c = 0; c < 3; ++c) {
            pos[(size_t)c * N + i] = dom->hx[3 * i + c] - (c == dom->axis ? dom->origin : 0.0);
            vel[(size_t)c * N + i] = dom->hv[3 * i + c];
        }
        ty[(size_t)i] = dom->type[(size_t)i];
    }
    dom->id.resize((size_t)no);
    dom->type.resize((size_t)no);
    for (size_t g = 0; g < ghosts.size(); ++g) {
        const int64_t i = no + (int64_t)g;
        for (int c = 0; c < 3; ++c)
            pos[(size_t)c * N + i] = ghosts[g].x[c] - (c == dom->axis ? dom->origin : 0.0);
        ty[(size_t)i] = ghosts[g].type;
        dom->id.push_back(ghosts[g].id);
        dom->type.push_back(ghosts[g].type);
    }
    p.N = N;
    p.n_owned = no;
    p.nb_gather = gather_blocks(N);
    if (N > 0) {
        DCK(cudaMemcpyAsync(p.pos, pos.data(), sizeof(double) * pos.size(), cudaMemcpyHostToDevice, dom->stream));
        DCK(cudaMemcpyAsync(p.vel, vel.data(), sizeof(double) * vel.size(), cudaMemcpyHostToDevice, dom->stream));
        DCK(cudaMemsetAsync(p.force, 0, sizeof(double) * 3 * N, dom->stream));
        DCK(cudaMemcpyAsync(p.type, ty.data(), sizeof(int32_t) * N, cudaMemcpyHostToDevice, dom->stream));
    }
    std::vector<int32_t> idx(dom->send_left);
    idx.insert(idx.end(), dom->send_right.begin(), dom->send_right.end());
    if (!idx.empty())
        DCK(cudaMemcpyAsync(dom->d_idx, idx.data(), sizeof(int32_t) * idx.size(), cudaMemcpyHostToDevice,
                            dom->stream));
    DCK(cudaStreamSynchronize(dom->stream));
    dom->hx.clear();
    dom->hv.clear();
    dom->need_build = true;
    dom->forces_valid = false;
    dom->phase = PH_READY;
    return MD_OK;
}

// Owned atoms to the host (global frame, wrapped on periodic axes): x, v as 3 per atom.
md_status download_owned(md_domain *dom, std::vector<double> &x, std::vector<double> &v)
{
    const Plan &p = dom->p;
    const int64_t no = dom->n_owned, N = p.N;
    std::vector<double> px((size_t)3 * N), pv((size_t)3 * N);
    if (N > 0) {
        DCK(cudaMemcpyAsync(px.data(), p.pos, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, dom->stream));
        DCK(cudaMemcpyAsync(pv.data(), p.vel, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, dom->stream));
        DCK(cudaStreamSynchronize(dom->stream));
    }
    x.assign((size_t)3 * no, 0.0);
    v.assign((size_t)3 * no, 0.0);
    for (int64_t i = 0; i < no; ++i)
        for (int c = 0; c < 3; ++c) {
            double g = px[(size_t)c * N + i] + (c == dom->axis ? dom->origin : 0.0);
            if (dom->pbc[c]) g = wrap(g, dom->L[c]);
            x[3 * i + c] = g;
            v[3 * i + c] = pv[(size_t)c * N + i];
        }
    return MD_OK;
}

// Owned atoms (host hx, hv, id, type) sorted by id: a local order that does not depend on
// the order in which migrants arrived.
void sort_owned(md_domain *dom)
{
    const size_t n = dom->id.size();
    std::vector<size_t> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return dom->id[a] < dom->id[b]; });
    std::vector<int64_t> id(n);
    std::vector<int32_t> ty(n);
    std::vector<double> x(3 * n), v(3 * n);
    for (size_t k = 0; k < n; ++k) {
        id[k] = dom->id[ord[k]];
        ty[k] = dom->type[ord[k]];
        for (int c = 0; c < 3; ++c) {
            x[3 * k + c] = dom->hx[3 * ord[k] + c];
            v[3 * k + c] = dom->hv[3 * ord[k] + c];
        }
    }
    dom->id.swap(id);
    dom->type.swap(ty);
    dom->hx.swap(x);
    dom->hv.swap(v);
    dom->n_owned = (int64_t)n;
}

int owner_of(const md_domain *dom, double x)
{
    const double w = dom->L[dom->axis] / dom->n_ranks;
    int r = (int)std::floor(x / w);
    return std::min(std::max(r, 0), dom->n_ranks - 1);
}

}  // namespace

extern "C" {

md_status md_domain_create(md_domain **out, const double box[3], const int pbc[3], int axis, int n_ranks, int rank,
                           int64_t capacity, const md_params *params, const double *masses_by_type,
                           const md_options *opt_in)
{
    if (!out) return MD_ERR_ARG;
    *out = nullptr;
    if (!box || !pbc || !params || !params->p || !masses_by_type || axis < 0 || axis > 2 || n_ranks < 2 ||
        rank < 0 || rank >= n_ranks || capacity < 1 || capacity > kMaxAtoms || params->n_types != 1 ||
        !pbc[axis])
        return MD_ERR_ARG;
    md_options opt;
    if (opt_in) opt = *opt_in; else md_default_options(&opt);
    if (!(masses_by_type[0] > 0)) return MD_ERR_ARG;
    md_domain *dom = new md_domain();
    Plan &p = dom->p;
    double rc = 0;
    if (plan_params(params, p, 0, &rc) != MD_OK || plan_options(p, opt, params->kind, rc) != MD_OK) {
        delete dom;
        return MD_ERR_ARG;
    }
    p.ntypes = 1;
    p.n_sets = 1;
    p.mass[0] = masses_by_type[0];
    p.inv_mass[0] = 1.0 / masses_by_type[0];
    dom->axis = axis;
    dom->n_ranks = n_ranks;
    dom->rank = rank;
    dom->capacity = capacity;
    dom->device = opt.device;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0) || !std::isfinite(box[a])) {
            delete dom;
            return MD_ERR_ARG;
        }
        dom->L[a] = box[a];
        dom->pbc[a] = pbc[a] ? 1 : 0;
    }
    const double w = box[axis] / n_ranks;
    dom->lo = rank * w;
    dom->hi = rank == n_ranks - 1 ? box[axis] : (rank + 1) * w;
    // local box: the slab and its ghost shells along the axis (open), the global box elsewhere
    double lbox[3] = {box[0], box[1], box[2]};
    p.list_margin = list_margin_for(std::max(box[0], std::max(box[1], box[2])) + 0.0, p.rl);
    dom->G = 2.0 * (p.rl + p.list_margin) + 0.01;
    if (w < 2.0 * dom->G) {   // ghosts must come from the two neighbouring slabs only
        delete dom;
        return MD_ERR_BOX;
    }
    dom->origin = dom->lo - dom->G;
    lbox[axis] = (dom->hi - dom->lo) + 2.0 * dom->G;
    dom->shift_left = rank == 0 ? box[axis] : 0.0;
    dom->shift_right = rank == n_ranks - 1 ? -box[axis] : 0.0;
    const double edge = p.rl + p.list_margin;
    for (int a = 0; a < 3; ++a) {
        p.box.L[a] = lbox[a];
        p.box.invL[a] = 1.0 / lbox[a];
        p.box.pbc[a] = a == axis ? 0 : dom->pbc[a];
        if (p.box.pbc[a] && lbox[a] < 2.0 * edge + 0.01) {
            delete dom;
            return MD_ERR_BOX;
        }
        p.nc[a] = std::max(1, (int)std::floor(lbox[a] / edge));
    }
    while ((int64_t)p.nc[0] * p.nc[1] * p.nc[2] > 4 * capacity + 64) {   // coarser cells are still exact
        int a = 0;
        if (p.nc[1] > p.nc[a]) a = 1;
        if (p.nc[2] > p.nc[a]) a = 2;
        if (p.nc[a] == 1) break;
        p.nc[a] = (p.nc[a] + 1) / 2;
    }
    p.ncell = (int64_t)p.nc[0] * p.nc[1] * p.nc[2];
    p.batch = false;
    p.n_sys = 1;
    p.seg_max = 1;
    p.N = 0;
    p.n_owned = 0;

    cudaError_t e = cudaSetDevice(dom->device);
    if (e == cudaSuccess && opt.cuda_stream) {
        dom->stream = static_cast<cudaStream_t>(opt.cuda_stream);
    } else if (e == cudaSuccess) {
        e = cudaStreamCreateWithFlags(&dom->stream, cudaStreamNonBlocking);
        dom->own_stream = e == cudaSuccess;
    }
    if (e != cudaSuccess || !configure_kernels(p)) {
        cudaGetLastError();
        md_domain_destroy(dom);
        return MD_ERR_CUDA;
    }
    const size_t C = (size_t)capacity, esz = p.precision == MD_FP64 ? sizeof(double) : sizeof(float);
    md_status st = MD_OK;
#define DAL(ptr, count)                                    \
    do {                                                   \
        if ((st = dalloc(dom, &(ptr), (count))) != MD_OK) { \
            md_domain_destroy(dom);                        \
            return st;                                     \
        }                                                  \
    } while (0)
    DAL(p.pos, 3 * C);
    DAL(p.vel, 3 * C);
    DAL(p.force, 3 * C);
    DAL(p.pos_build, 3 * C);
    DAL(p.u, C);
    DAL(p.w, 9 * C);
    DAL(p.j, 3 * C);
    DAL(p.posf, 3 * C);
    DAL(p.type, C);
    DAL(p.nn, C);
    DAL(p.nl, (size_t)p.cap * C);
    DAL(p.rev, (size_t)p.cap * C);
    DAL(p.mask, C);
    DAL(p.ovf_count, 1);
    DAL(p.ovf_list, C);
    DAL(p.sys_of, 1);
    DAL(p.sys, 2);
    {
        unsigned char *v = nullptr;
        DAL(v, 4 * (size_t)p.maxa * C * esz);
        p.pd = v;
        DAL(v, 3 * (size_t)p.maxa * C * esz);
        p.pr = v;
    }
    DAL(p.cell_count, (size_t)p.ncell);
    DAL(p.cell_start, (size_t)p.ncell);
    DAL(p.cell_atoms, C);
    DAL(p.atom_cell, C);
    DAL(p.atom_rank, C);
    p.nscanb = (p.ncell + scan_block_elems() - 1) / scan_block_elems();
    DAL(p.scan_blocks, (size_t)p.nscanb + 1);
    DAL(p.partials, (size_t)gather_blocks(capacity) * kNumPartials);
    DAL(p.totals, (size_t)kNumPartials);
    DAL(p.flags, 1);
    DAL(dom->d_idx, C);
    DAL(dom->d_stage, 3 * C);
#undef DAL
    p.series = nullptr;
    p.npt_totals = nullptr;
    SysDev sd;
    std::memset(&sd, 0, sizeof(sd));
    sd.box = p.box;
    for (int a = 0; a < 3; ++a) sd.nc[a] = p.nc[a];
    sd.steps_left = -1;
    sd.active = 1;
    sd.rc = p.rc;
    sd.rl = p.rl;
    sd.cell_edge = edge;
    sd.half_skin2 = (float)(0.25 * p.skin * p.skin);
    sd.npt.mu_cum[0] = sd.npt.mu_cum[1] = sd.npt.mu_cum[2] = 1.0;
    SysDev both[2] = {sd, sd};
    if (cudaMemcpyAsync(p.sys, both, sizeof(both), cudaMemcpyHostToDevice, dom->stream) != cudaSuccess ||
        cudaMemsetAsync(p.flags, 0, sizeof(Flags), dom->stream) != cudaSuccess ||
        cudaStreamSynchronize(dom->stream) != cudaSuccess) {
        cudaGetLastError();
        md_domain_destroy(dom);
        return MD_ERR_CUDA;
    }
    dom->h_stage.resize(3 * C);
    *out = dom;
    return MD_OK;
}

md_status md_domain_set_atoms(md_domain *dom, int64_t n, const int64_t *ids, const int32_t *types, const double *x,
                              const double *y, const double *z, const double *vx, const double *vy, const double *vz)
{
    if (!dom) return MD_ERR_ARG;
    if (n < 0 || (n > 0 && (!ids || !types || !x || !y || !z))) return dfail(dom, MD_ERR_ARG, "bad atom arrays");
    dom->id.clear();
    dom->type.clear();
    dom->hx.clear();
    dom->hv.clear();
    const double *in[3] = {x, y, z}, *vin[3] = {vx, vy, vz};
    for (int64_t i = 0; i < n; ++i) {
        if (types[i] != 0) return dfail(dom, MD_ERR_ARG, "one element only");
        double g[3];
        for (int c = 0; c < 3; ++c) {
            g[c] = in[c][i];
            if (!std::isfinite(g[c]) || (vin[c] && !std::isfinite(vin[c][i])))
                return dfail(dom, MD_ERR_NAN, "non-finite position or velocity");
            if (dom->pbc[c]) g[c] = wrap(g[c], dom->L[c]);
        }
        if (owner_of(dom, g[dom->axis]) != dom->rank) continue;
        dom->id.push_back(ids[i]);
        dom->type.push_back(types[i]);
        for (int c = 0; c < 3; ++c) {
            dom->hx.push_back(g[c]);
            dom->hv.push_back(vin[c] ? vin[c][i] : 0.0);
        }
    }
    sort_owned(dom);
    if (dom->n_owned > dom->capacity) return dfail(dom, MD_ERR_OOM, "more owned atoms than the capacity");
    dom->phase = PH_NEED_GHOSTS;
    dom->forces_valid = false;
    return MD_OK;
}

md_status md_domain_message_bound(md_domain *dom, int mode, size_t *bytes)
{
    if (!dom || !bytes || mode < MD_DOMAIN_POSITIONS || mode > MD_DOMAIN_GHOSTS) return MD_ERR_ARG;
    *bytes = bound_bytes(dom, mode);
    return MD_OK;
}

md_status md_domain_pack(md_domain *dom, int mode, void *to_left, void *to_right, size_t cap, size_t *n_left,
                         size_t *n_right)
{
    if (!dom || !to_left || !to_right || !n_left || !n_right) return MD_ERR_ARG;
    if (cap < bound_bytes(dom, mode)) return dfail(dom, MD_ERR_ARG, "message buffers smaller than the bound");
    unsigned char *ol = static_cast<unsigned char *>(to_left), *orr = static_cast<unsigned char *>(to_right);
    if (mode == MD_DOMAIN_POSITIONS) {
        if (dom->phase != PH_READY) return dfail(dom, MD_ERR_STATE, "no ghost sets yet");
        const Plan &p = dom->p;
        const int64_t nl = (int64_t)dom->send_left.size(), nr = (int64_t)dom->send_right.size();
        if (nl > 0)
            k_domain_pack<<<blocks_for(nl, 256), 256, 0, dom->stream>>>(nl, dom->d_idx, p.pos, p.N, dom->axis,
                                                                        dom->origin + dom->shift_left, dom->d_stage);
        if (nr > 0)
            k_domain_pack<<<blocks_for(nr, 256), 256, 0, dom->stream>>>(nr, dom->d_idx + nl, p.pos, p.N, dom->axis,
                                                                        dom->origin + dom->shift_right,
                                                                        dom->d_stage + 3 * nl);
        const MsgHeader hl{nl, mode}, hr{nr, mode};
        std::memcpy(ol, &hl, sizeof(hl));
        std::memcpy(orr, &hr, sizeof(hr));
        if (nl + nr > 0) {
            DCK(cudaMemcpyAsync(dom->h_stage.data(), dom->d_stage, sizeof(double) * 3 * (nl + nr),
                                cudaMemcpyDeviceToHost, dom->stream));
            DCK(cudaStreamSynchronize(dom->stream));
        }
        std::memcpy(ol + sizeof(hl), dom->h_stage.data(), sizeof(double) * 3 * nl);
        std::memcpy(orr + sizeof(hr), dom->h_stage.data() + 3 * nl, sizeof(double) * 3 * nr);
        *n_left = sizeof(hl) + sizeof(double) * 3 * nl;
        *n_right = sizeof(hr) + sizeof(double) * 3 * nr;
        return MD_OK;
    }
    if (mode == MD_DOMAIN_MIGRATE) {
        if (dom->phase != PH_READY) return dfail(dom, MD_ERR_STATE, "migration needs a running domain");
        std::vector<double> x, v;
        md_status s = download_owned(dom, x, v);
        if (s != MD_OK) return s;
        std::vector<MigrantRec> left, right;
        std::vector<int64_t> kid;
        std::vector<int32_t> kty;
        std::vector<double> kx, kv;
        const int lr = (dom->rank + dom->n_ranks - 1) % dom->n_ranks, rr = (dom->rank + 1) % dom->n_ranks;
        for (int64_t i = 0; i < dom->n_owned; ++i) {
            const int o = owner_of(dom, x[3 * i + dom->axis]);
            if (o == dom->rank) {
                kid.push_back(dom->id[(size_t)i]);
                kty.push_back(dom->type[(size_t)i]);
                for (int c = 0; c < 3; ++c) {
                    kx.push_back(x[3 * i + c]);
                    kv.push_back(v[3 * i + c]);
                }
                continue;
            }
            if (o != lr && o != rr)
                return dfail(dom, MD_ERR_STATE, "an atom crossed more than one slab between rebuilds");
            MigrantRec m;
            std::memset(&m, 0, sizeof(m));
            m.id = dom->id[(size_t)i];
            m.type = dom->type[(size_t)i];
            for (int c = 0; c < 3; ++c) {
                m.x[c] = x[3 * i + c];
                m.v[c] = v[3 * i + c];
            }
            (o == rr ? right : left).push_back(m);
        }
        const MsgHeader hl{(int64_t)left.size(), mode}, hr{(int64_t)right.size(), mode};
        std::memcpy(ol, &hl, sizeof(hl));
        std::memcpy(orr, &hr, sizeof(hr));
        if (!left.empty()) std::memcpy(ol + sizeof(hl), left.data(), sizeof(MigrantRec) * left.size());
        if (!right.empty()) std::memcpy(orr + sizeof(hr), right.data(), sizeof(MigrantRec) * right.size());
        *n_left = sizeof(hl) + sizeof(MigrantRec) * left.size();
        *n_right = sizeof(hr) + sizeof(MigrantRec) * right.size();
        dom->id.swap(kid);
        dom->type.swap(kty);
        dom->hx.swap(kx);
        dom->hv.swap(kv);
        dom->n_owned = (int64_t)dom->id.size();
        dom->phase = PH_MIGRATING;
        return MD_OK;
    }
    if (mode == MD_DOMAIN_GHOSTS) {
        if (dom->phase != PH_NEED_GHOSTS) return dfail(dom, MD_ERR_STATE, "ghost sets follow a migration");
        std::vector<GhostRec> left, right;
        dom->send_left.clear();
        dom->send_right.clear();
        for (int64_t i = 0; i < dom->n_owned; ++i) {
            const double xa = dom->hx[3 * i + dom->axis];
            GhostRec g;
            std::memset(&g, 0, sizeof(g));
            g.id = dom->id[(size_t)i];
            g.type = dom->type[(size_t)i];
            for (int c = 0; c < 3; ++c) g.x[c] = dom->hx[3 * i + c];
            if (xa - dom->lo < dom->G) {
                GhostRec q = g;
                q.x[dom->axis] += dom->shift_left;
                left.push_back(q);
                dom->send_left.push_back((int32_t)i);
            }
            if (dom->hi - xa < dom->G) {
                GhostRec q = g;
                q.x[dom->axis] += dom->shift_right;
                right.push_back(q);
                dom->send_right.push_back((int32_t)i);
            }
        }
        const MsgHeader hl{(int64_t)left.size(), mode}, hr{(int64_t)right.size(), mode};
        std::memcpy(ol, &hl, sizeof(hl));
        std::memcpy(orr, &hr, sizeof(hr));
        if (!left.empty()) std::memcpy(ol + sizeof(hl), left.data(), sizeof(GhostRec) * left.size());
        if (!right.empty()) std::memcpy(orr + sizeof(hr), right.data(), sizeof(GhostRec) * right.size());
        *n_left = sizeof(hl) + sizeof(GhostRec) * left.size();
        *n_right = sizeof(hr) + sizeof(GhostRec) * right.size();
        return MD_OK;
    }
    return MD_ERR_ARG;
}

md_status md_domain_unpack(md_domain *dom, int mode, const void *from_left, size_t n_left, const void *from_right,
                           size_t n_right)
{
    if (!dom || !from_left || !from_right) return MD_ERR_ARG;
    if (n_left < sizeof(MsgHeader) || n_right < sizeof(MsgHeader)) return dfail(dom, MD_ERR_ARG, "short message");
    MsgHeader hl, hr;
    std::memcpy(&hl, from_left, sizeof(hl));
    std::memcpy(&hr, from_right, sizeof(hr));
    if (hl.mode != mode || hr.mode != mode || hl.count < 0 || hr.count < 0)
        return dfail(dom, MD_ERR_ARG, "message of another kind");
    const unsigned char *il = static_cast<const unsigned char *>(from_left) + sizeof(MsgHeader);
    const unsigned char *ir = static_cast<const unsigned char *>(from_right) + sizeof(MsgHeader);
    auto fits = [&](size_t rec) {
        return n_left >= sizeof(MsgHeader) + rec * (size_t)hl.count && n_right >= sizeof(MsgHeader) + rec * (size_t)hr.count;
    };
    if (mode == MD_DOMAIN_POSITIONS) {
        if (dom->phase != PH_READY) return dfail(dom, MD_ERR_STATE, "no ghost sets yet");
        if (hl.count != dom->n_left || hr.count != dom->n_right || !fits(3 * sizeof(double)))
            return dfail(dom, MD_ERR_ARG, "ghost position message does not match the ghost sets");
        const Plan &p = dom->p;
        const int64_t n = hl.count + hr.count;
        if (n == 0) return MD_OK;
        std::memcpy(dom->h_stage.data(), il, sizeof(double) * 3 * hl.count);
        std::memcpy(dom->h_stage.data() + 3 * hl.count, ir, sizeof(double) * 3 * hr.count);
        DCK(cudaMemcpyAsync(dom->d_stage, dom->h_stage.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice,
                            dom->stream));
        k_domain_unpack<<<blocks_for(n, 256), 256, 0, dom->stream>>>(n, dom->n_owned, p.pos, p.posf, p.N,
                                                                     dom->axis, dom->origin, dom->d_stage);
        DCK(cudaGetLastError());
        DCK(cudaStreamSynchronize(dom->stream));   // the host stage is reused by the next call
        return MD_OK;
    }
    if (mode == MD_DOMAIN_MIGRATE) {
        if (dom->phase != PH_MIGRATING) return dfail(dom, MD_ERR_STATE, "unpack of migrants without a pack");
        if (!fits(sizeof(MigrantRec))) return dfail(dom, MD_ERR_ARG, "truncated migrant message");
        for (int side = 0; side < 2; ++side) {
            const int64_t cnt = side == 0 ? hl.count : hr.count;
            const unsigned char *src = side == 0 ? il : ir;
            for (int64_t k = 0; k < cnt; ++k) {
                MigrantRec m;
                std::memcpy(&m, src + sizeof(MigrantRec) * k, sizeof(m));
                if (owner_of(dom, m.x[dom->axis]) != dom->rank)
                    return dfail(dom, MD_ERR_STATE, "a migrant does not belong to this slab");
                dom->id.push_back(m.id);
                dom->type.push_back(m.type);
                for (int c = 0; c < 3; ++c) {
                    dom->hx.push_back(m.x[c]);
                    dom->hv.push_back(m.v[c]);
                }
            }
        }
        sort_owned(dom);
        dom->phase = PH_NEED_GHOSTS;
        return MD_OK;
    }
    if (mode == MD_DOMAIN_GHOSTS) {
        if (dom->phase != PH_NEED_GHOSTS) return dfail(dom, MD_ERR_STATE, "ghost sets follow a migration");
        if (!fits(sizeof(GhostRec))) return dfail(dom, MD_ERR_ARG, "truncated ghost message");
        std::vector<GhostRec> ghosts((size_t)(hl.count + hr.count));
        if (hl.count) std::memcpy(ghosts.data(), il, sizeof(GhostRec) * hl.count);
        if (hr.count) std::memcpy(ghosts.data() + hl.count, ir, sizeof(GhostRec) * hr.count);
        for (const GhostRec &g : ghosts) {   // every ghost lies within the shell next to the slab
            const double xa = g.x[dom->axis];
            if (!(xa >= dom->lo - dom->G && xa < dom->hi + dom->G) || (xa >= dom->lo && xa < dom->hi))
                return dfail(dom, MD_ERR_STATE, "a ghost outside this rank's shell");
        }
        dom->n_left = hl.count;
        dom->n_right = hr.count;
        return assemble(dom, ghosts);
    }
    return MD_ERR_ARG;
}

md_status md_domain_kick_drift(md_domain *dom, double dt, int *rebuild)
{
    if (!dom || !rebuild || !std::isfinite(dt)) return MD_ERR_ARG;
    if (dom->phase != PH_READY || !dom->forces_valid) return dfail(dom, MD_ERR_STATE, "forces not computed yet");
    Plan &p = dom->p;
    double hk[kMaxTypes] = {0, 0, 0, 0};
    hk[0] = 0.5 * dt * kAccUnit / p.mass[0];
    md_status s = clear_flags(dom);
    if (s != MD_OK) return s;
    launch_kick_drift(p, dom->stream, hk, dt);
    DCK(cudaGetLastError());
    int r = 0;
    DCK(cudaMemcpyAsync(&r, &p.flags->rebuild, sizeof(int), cudaMemcpyDeviceToHost, dom->stream));
    DCK(cudaStreamSynchronize(dom->stream));
    *rebuild = r != 0;
    dom->forces_valid = false;
    return MD_OK;
}

md_status md_domain_force(md_domain *dom, double dt, double totals[5])
{
    if (!dom || !std::isfinite(dt)) return MD_ERR_ARG;
    if (dom->phase != PH_READY) return dfail(dom, MD_ERR_STATE, "no ghost sets yet");
    Plan &p = dom->p;
    md_status s = clear_flags(dom);
    if (s != MD_OK) return s;
    if (dom->need_build) {   // only after a migration: the ghost sets changed
        launch_rebuild(p, dom->stream);
        dom->need_build = false;
    }
    double hk[kMaxTypes] = {0, 0, 0, 0};
    hk[0] = 0.5 * dt * kAccUnit / p.mass[0];
    launch_pair_reset(p, dom->stream);
    launch_pair(p, dom->stream);
    launch_gather(p, dom->stream, dt != 0.0 ? hk : nullptr, dt, false);
    launch_reduce(p, dom->stream, false, false);
    DCK(cudaGetLastError());
    double t[kNumPartials];
    DCK(cudaMemcpyAsync(t, p.totals, sizeof(t), cudaMemcpyDeviceToHost, dom->stream));
    if ((s = check_device_flags(dom)) != MD_OK) return s;
    if (totals)
        for (int c = 0; c < kStepPartials; ++c) totals[c] = t[c];   // U, K, Jx, Jy, Jz of the owned atoms
    dom->forces_valid = true;
    return MD_OK;
}

md_status md_domain_compute(md_domain *dom, double *f, double *u, double *w, double *j, double totals[13])
{
    if (!dom) return MD_ERR_ARG;
    if (dom->phase != PH_READY) return dfail(dom, MD_ERR_STATE, "no ghost sets yet");
    Plan &p = dom->p;
    md_status s = clear_flags(dom);
    if (s != MD_OK) return s;
    if (dom->need_build) {
        launch_rebuild(p, dom->stream);
        dom->need_build = false;
    }
    launch_pair_reset(p, dom->stream);
    launch_pair(p, dom->stream);
    launch_gather(p, dom->stream, nullptr, 0.0, true);
    launch_reduce(p, dom->stream, true, false);
    DCK(cudaGetLastError());
    double t[kNumPartials];
    DCK(cudaMemcpyAsync(t, p.totals, sizeof(t), cudaMemcpyDeviceToHost, dom->stream));
    const int64_t no = dom->n_owned, N = p.N;
    struct Out {
        double *dst;
        const double *src;
        int comps;
    } outs[4] = {{f, p.force, 3}, {u, p.u, 1}, {w, p.w, 9}, {j, p.j, 3}};
    for (const Out &o : outs)
        if (o.dst && no > 0)
            for (int c = 0; c < o.comps; ++c)
                DCK(cudaMemcpyAsync(o.dst + c * no, o.src + c * N, sizeof(double) * no, cudaMemcpyDeviceToHost,
                                    dom->stream));
    if ((s = check_device_flags(dom)) != MD_OK) return s;
    if (totals) {
        totals[0] = t[0];
        for (int c = 0; c < 9; ++c) totals[1 + c] = t[5 + c];
        for (int c = 0; c < 3; ++c) totals[10 + c] = t[2 + c];
    }
    dom->forces_valid = true;
    return MD_OK;
}

md_status md_domain_owned(md_domain *dom, int64_t *n, int64_t *ids, double *x, double *v)
{
    if (!dom || !n) return MD_ERR_ARG;
    *n = dom->n_owned;
    if (ids)
        for (int64_t i = 0; i < dom->n_owned; ++i) ids[i] = dom->id[(size_t)i];
    if (!x && !v) return MD_OK;
    std::vector<double> hx, hv;
    if (dom->phase == PH_READY) {
        md_status s = download_owned(dom, hx, hv);
        if (s != MD_OK) return s;
    } else {
        hx = dom->hx;
        hv = dom->hv;
    }
    const int64_t no = dom->n_owned;
    for (int64_t i = 0; i < no; ++i)
        for (int c = 0; c < 3; ++c) {
            if (x) x[c * no + i] = hx[3 * i + c];
            if (v) v[c * no + i] = hv[3 * i + c];
        }
    return MD_OK;
}

const char *md_domain_last_error(const md_domain *dom) { return dom ? dom->err.c_str() : ""; }

void md_domain_destroy(md_domain *dom)
{
    if (!dom) return;
    cudaSetDevice(dom->device);
    if (dom->stream) cudaStreamSynchronize(dom->stream);
    for (void *a : dom->allocs) cudaFree(a);
    if (dom->own_stream) cudaStreamDestroy(dom->stream);
    delete dom;
}

}  // extern "C"
