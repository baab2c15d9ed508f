// md_static.cu -- md_compute_static: one force evaluation that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need forces: code
// running inside another runtime's memory pool or allocator callback, plugins whose host
// forbids allocation after start-up, or a host that pre-plans its whole device footprint.
// This entry point serves them: it runs the same kernel chain as md_compute (cell list,
// Verlet list, pair pass, gather, reduction) with every scratch buffer carved out of one
// file-scope device array, `g_scratch`, of fixed size.  The caller passes device inputs
// and outputs; nothing is created or freed.
//
// The array is resolved to a device address once per device (cudaGetSymbolAddress, with
// that device current) on the first call made there, so that first call should come
// before any stream capture.  Every call shares the array and it keeps the last call's
// contents: each call clears what must start at zero, and calls that overlap on the GPU
// (concurrent streams, threads) race on it.
#include <cmath>
#include <cstring>
#include <mutex>

#include "md.h"
#include "md_plan.cuh"

using namespace mdk;

namespace {

__device__ __align__(256) unsigned char g_scratch[MD_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {nullptr};

struct Carver {
    unsigned char *base;
    size_t used = 0, cap;
    template <typename P>
    P *take(size_t count)
    {
        used = (used + 255) / 256 * 256;
        P *p = reinterpret_cast<P *>(base + used);
        used += count * sizeof(P);
        return p;
    }
};

// Cell grid of the single system (same rule as md_create, coarsened to <= 4n + 64 cells).
md_status grid(Plan &p, const double box[3], const int pbc[3], int64_t n)
{
    const double edge = p.rl + p.list_margin;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0) || !std::isfinite(box[a])) return MD_ERR_ARG;
        p.box.L[a] = box[a];
        p.box.invL[a] = 1.0 / box[a];
        p.box.pbc[a] = pbc[a] ? 1 : 0;
        if (p.box.pbc[a] && box[a] < 2.0 * edge + 0.01) return MD_ERR_BOX;
        const int k = (int)std::floor(box[a] / edge);
        p.nc[a] = k < 1 ? 1 : k;
    }
    while ((int64_t)p.nc[0] * p.nc[1] * p.nc[2] > 4 * n + 64) {
        int a = 0;
        if (p.nc[1] > p.nc[a]) a = 1;
        if (p.nc[2] > p.nc[a]) a = 2;
        if (p.nc[a] == 1) break;
        p.nc[a] = (p.nc[a] + 1) / 2;
    }
    p.ncell = (int64_t)p.nc[0] * p.nc[1] * p.nc[2];
    return MD_OK;
}

}  // namespace

extern "C" md_status md_compute_static(int kind, const double *params, int precision, const double box[3],
                                       const int pbc[3], int64_t n_atoms, const double *x, const double *y,
                                       const double *z, const double *vx, const double *vy, const double *vz,
                                       double mass, double *f, double *u, double *w, double *j, double *totals,
                                       void *cuda_stream)
{
    if (!params || !box || !pbc || n_atoms < 1 || !x || !y || !z || !(mass > 0)) return MD_ERR_ARG;
    if (precision != MD_FP64 && precision != MD_MIXED) return MD_ERR_ARG;
    if (n_atoms > MD_STATIC_MAX_ATOMS) return MD_ERR_OOM;
    if (kind != MD_TERSOFF && kind != MD_SW) return MD_ERR_ARG;
    const int64_t n = n_atoms;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaGetLastError();   // an earlier call's error must not be reported as this call's

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MD_ERR_CUDA;
    unsigned char *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess) {
                cudaGetLastError();
                return MD_ERR_CUDA;
            }
            g_addr[dev] = static_cast<unsigned char *>(ptr);
        }
        base = g_addr[dev];
    }

    // parameters and cutoffs, as md_create, with no skin (the list is built every call)
    Plan p;
    const double *q = params;
    double rc = 0;
    if (kind == MD_TERSOFF) {
        TersoffP &t = p.tp[0];
        t.A = q[0]; t.B = q[1]; t.lam = q[2]; t.mu = q[3]; t.beta = q[4]; t.n = q[5];
        t.c = q[6]; t.d = q[7]; t.h = q[8]; t.R = q[9]; t.S = q[10];
        if (!(t.S > t.R) || !(t.R > 0) || !(t.n > 0) || t.beta < 0 || !(t.d != 0)) return MD_ERR_ARG;
        t.c2 = t.c * t.c; t.d2 = t.d * t.d; t.c2d2 = t.c2 / t.d2;
        t.pi_SR = M_PI / (t.S - t.R);
        t.beta_zero = t.beta == 0.0;
        t.ln_beta = t.beta > 0 ? std::log(t.beta) : 0.0;
        t.inv2n = 1.0 / (2.0 * t.n);
        rc = t.S;
    } else {
        SWP &sw = p.sp[0];
        sw.eps = q[0]; sw.sig = q[1]; sw.a = q[2]; sw.lam = q[3]; sw.gam = q[4]; sw.A = q[5]; sw.B = q[6];
        sw.p = q[7]; sw.q = q[8];
        if (!(sw.sig > 0) || !(sw.a > 0)) return MD_ERR_ARG;
        sw.rc = sw.a * sw.sig;
        sw.Aeps = sw.A * sw.eps; sw.lameps = sw.lam * sw.eps; sw.gamsig = sw.gam * sw.sig;
        sw.p_int = (sw.p == std::floor(sw.p) && sw.p >= 0 && sw.p <= 16) ? (int)sw.p : -1;
        sw.q_int = (sw.q == std::floor(sw.q) && sw.q >= 0 && sw.q <= 16) ? (int)sw.q : -1;
        rc = sw.rc;
    }
    p.kind = kind;
    p.precision = precision;
    p.cap = 32;
    p.maxa = kind == MD_SW ? 16 : 8;
    p.rc = rc;
    p.skin = 0.0;
    p.rl = rc;
    p.list_margin = list_margin_for(std::max(box[0], std::max(box[1], box[2])), p.rl);
    p.N = n;
    p.n_sets = 1;
    p.ntypes = 1;
    p.mass[0] = mass;
    p.inv_mass[0] = 1.0 / mass;
    p.batch = false;
    p.n_sys = 1;
    p.seg_max = 1;
    md_status st = grid(p, box, pbc, n);
    if (st != MD_OK) return st;

    // carve the scratch array
    Carver c{base, 0, (size_t)MD_STATIC_SCRATCH_BYTES};
    const size_t esz = precision == MD_FP64 ? sizeof(double) : sizeof(float);
    p.pos = c.take<double>(3 * n);
    p.vel = c.take<double>(3 * n);
    p.force = f ? f : c.take<double>(3 * n);
    p.pos_build = c.take<double>(3 * n);
    p.u = u ? u : c.take<double>(n);
    p.w = w;
    p.j = j;
    p.posf = c.take<float>(3 * n);
    p.type = c.take<int>(n);
    p.nn = c.take<int>(n);
    p.nl = c.take<int>((size_t)p.cap * n);
    p.rev = c.take<uint8_t>((size_t)p.cap * n);
    p.mask = c.take<uint32_t>(n);
    p.ovf_count = c.take<int>(1);
    p.ovf_list = c.take<int>(n);
    p.sys_of = c.take<int>(1);
    p.sys = c.take<SysDev>(2);
    p.pd = c.take<unsigned char>(4 * (size_t)p.maxa * n * esz);
    p.pr = c.take<unsigned char>(3 * (size_t)p.maxa * n * esz);
    p.cell_count = c.take<int>(p.ncell);
    p.cell_start = c.take<int>(p.ncell);
    p.cell_atoms = c.take<int>(n);
    p.atom_cell = c.take<int>(n);
    p.atom_rank = c.take<int>(n);
    p.nscanb = (p.ncell + scan_block_elems() - 1) / scan_block_elems();
    p.scan_blocks = c.take<int>(p.nscanb + 1);
    p.nb_gather = gather_blocks(n);
    p.partials = c.take<double>((size_t)p.nb_gather * kNumPartials);
    p.totals = c.take<double>(kNumPartials);
    p.series = nullptr;
    p.flags = c.take<Flags>(1);
    if (c.used > c.cap) return MD_ERR_OOM;   // the cell grid pushed the layout past the array

    if (!configure_kernels(p)) return MD_ERR_CUDA;
    // inputs in, zero-initialised state (the array keeps the previous call's contents);
    // every copy is checked before any kernel is launched
    const double *src[3] = {x, y, z};
    const double *vsrc[3] = {vx, vy, vz};
    for (int a = 0; a < 3; ++a) {
        if (cudaMemcpyAsync(p.pos + a * n, src[a], sizeof(double) * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return MD_ERR_CUDA;
        const cudaError_t e = vsrc[a] ? cudaMemcpyAsync(p.vel + a * n, vsrc[a], sizeof(double) * n,
                                                        cudaMemcpyDeviceToDevice, s)
                                      : cudaMemsetAsync(p.vel + a * n, 0, sizeof(double) * n, s);
        if (e != cudaSuccess) return MD_ERR_CUDA;
    }
    if (cudaMemsetAsync(p.type, 0, sizeof(int) * n, s) != cudaSuccess ||
        cudaMemsetAsync(p.flags, 0, sizeof(Flags), s) != cudaSuccess ||
        cudaMemsetAsync(p.sys, 0, sizeof(SysDev) * 2, s) != cudaSuccess)
        return MD_ERR_CUDA;
    launch_rebuild(p, s);
    launch_pair_reset(p, s);
    launch_pair(p, s);
    launch_gather(p, s, nullptr, 0.0, true);
    launch_reduce(p, s, true, false);
    if (cudaGetLastError() != cudaSuccess) return MD_ERR_CUDA;   // a launch failed
    Flags fl;
    double t[kNumPartials];
    if (cudaMemcpyAsync(&fl, p.flags, sizeof(Flags), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(t, p.totals, sizeof(t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return MD_ERR_CUDA;
    if (fl.list_overflow || fl.active_overflow) return MD_ERR_NEIGH_OVERFLOW;
    if (fl.asym) return MD_ERR_CUDA;
    if (fl.nonfinite) return MD_ERR_NAN;
    if (totals) {
        totals[0] = t[0];
        for (int k = 0; k < 9; ++k) totals[1 + k] = t[5 + k];
        for (int k = 0; k < 3; ++k) totals[10 + k] = t[2 + k];
    }
    return MD_OK;
}
