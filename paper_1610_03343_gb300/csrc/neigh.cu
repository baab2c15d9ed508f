// neigh.cu -- cell-list neighbour build (the paper's Sec. 2.1: a Verlet neighbour list
// built with the standard cell-list method for a uniform cutoff), the reverse-slot
// index the atomic-free gather needs, and the skin/2 displacement check.
//
// Pipeline (all on the device, one thread per atom or per cell):
//   clear counts -> bin atoms (cell id + rank in cell via atomicAdd) -> exclusive scan
//   of cell counts -> scatter atoms into cell order -> per-atom list search over the
//   distinct neighbouring cells, kept sorted by atom index -> reverse slot of i in j's
//   list -> done (clear the rebuild flag).
// The order of atoms inside a cell depends on atomic timing, but every list is sorted
// by index, so the lists are deterministic.
#include "md_plan.cuh"

namespace mdk {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 4;
constexpr int kScanElems = kScanThreads * kScanPerThread;  // per block

__device__ __forceinline__ bool skip(const Flags *f, bool conditional)
{
    return conditional && (*(volatile const int *)&f->rebuild) == 0;
}

__device__ __forceinline__ int cell_coord(double x, int nc, double invL)
{
    int c = (int)floor(x * invL * (double)nc);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_cell_clear(int64_t ncell, int *count, Flags *flags, bool cond)
{
    if (skip(flags, cond)) return;
    int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c == 0) flags->max_nn = 0;
    if (c < ncell) count[c] = 0;
}

__global__ void k_cell_count(int64_t N, const double *pos, Box box, int nc0, int nc1, int nc2,
                             int *atom_cell, int *atom_rank, int *count, Flags *flags, bool cond)
{
    if (skip(flags, cond)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int cx = cell_coord(pos[i], nc0, box.invL[0]);
    int cy = cell_coord(pos[N + i], nc1, box.invL[1]);
    int cz = cell_coord(pos[2 * N + i], nc2, box.invL[2]);
    int c = (cx * nc1 + cy) * nc2 + cz;
    atom_cell[i] = c;
    atom_rank[i] = atomicAdd(&count[c], 1);
}

// Exclusive scan, pass 1: scan each block's kScanElems counts, store block totals.
__global__ void __launch_bounds__(kScanThreads)
k_scan_blocks(int64_t n, const int *in, int *out, int *block_sums, Flags *flags, bool cond)
{
    if (skip(flags, cond)) return;
    __shared__ int warp_tot[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanElems + (int64_t)threadIdx.x * kScanPerThread;
    int v[kScanPerThread];
    int t = 0;
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        v[q] = (base + q < n) ? in[base + q] : 0;
        t += v[q];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
        int wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;   // exclusive warp offsets
        if (lane == kScanThreads / 32 - 1) block_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    int run = warp_tot[wid] + incl - t;
#pragma unroll
    for (int q = 0; q < kScanPerThread; ++q) {
        if (base + q < n) out[base + q] = run;
        run += v[q];
    }
}

// Pass 2: exclusive scan of the block totals by one block, in chunks, with a carry.
__global__ void __launch_bounds__(kScanThreads)
k_scan_sums(int64_t nb, int *block_sums, Flags *flags, bool cond)
{
    if (skip(flags, cond)) return;
    __shared__ int warp_tot[kScanThreads / 32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        int64_t idx = b0 + threadIdx.x;
        int v = idx < nb ? block_sums[idx] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int w = (lane < kScanThreads / 32) ? warp_tot[lane] : 0;
            int wi = w;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < kScanThreads / 32) warp_tot[lane] = wi - w;
        }
        __syncthreads();
        int excl = carry + warp_tot[wid] + incl - v;
        if (idx < nb) block_sums[idx] = excl;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) carry = excl + v;
        __syncthreads();
    }
}

// Pass 3: add each block's offset.
__global__ void k_scan_add(int64_t n, int *out, const int *block_sums, Flags *flags, bool cond)
{
    if (skip(flags, cond)) return;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] += block_sums[idx / kScanElems];
}

__global__ void k_cell_fill(int64_t N, const int *atom_cell, const int *atom_rank,
                            const int *cell_start, int *cell_atoms, Flags *flags, bool cond)
{
    if (skip(flags, cond)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    cell_atoms[cell_start[atom_cell[i]] + atom_rank[i]] = (int)i;
}

// distinct cell indices adjacent to c along one axis (periodic wrap or open clip)
__device__ __forceinline__ int stencil_axis(int c, int nc, int periodic, int *out)
{
    int n = 0;
#pragma unroll
    for (int t = -1; t <= 1; ++t) {
        int k = c + t;
        if (periodic) {
            k = (k + nc) % nc;
        } else if (k < 0 || k >= nc) {
            continue;
        }
        bool dup = false;
        for (int u = 0; u < n; ++u) dup |= (out[u] == k);
        if (!dup) out[n++] = k;
    }
    return n;
}

// One thread per atom: search the distinct neighbouring cells, keep every j != i with
// |r_ij| < rl (minimum image) in ascending index order.  Also snapshots the build
// positions for the skin/2 test.
__global__ void k_build_list(int64_t N, const double *pos, Box box, int nc0, int nc1, int nc2,
                             const int *atom_cell, const int *cell_start, const int *cell_count,
                             const int *cell_atoms, double rl2, int cap, int *nn, int *nl,
                             double *pos_build, Flags *flags, bool cond)
{
    if (skip(flags, cond)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double xi = pos[i], yi = pos[N + i], zi = pos[2 * N + i];
    pos_build[i] = xi;
    pos_build[N + i] = yi;
    pos_build[2 * N + i] = zi;
    const int c = atom_cell[i];
    const int cz = c % nc2, cy = (c / nc2) % nc1, cx = c / (nc1 * nc2);
    int ox[3], oy[3], oz[3];
    const int nx = stencil_axis(cx, nc0, box.pbc[0], ox);
    const int ny = stencil_axis(cy, nc1, box.pbc[1], oy);
    const int nz = stencil_axis(cz, nc2, box.pbc[2], oz);
    int loc[kMaxListCap];
    int cnt = 0;
    for (int a = 0; a < nx; ++a)
        for (int b = 0; b < ny; ++b)
            for (int e = 0; e < nz; ++e) {
                const int cc = (ox[a] * nc1 + oy[b]) * nc2 + oz[e];
                const int s0 = cell_start[cc], s1 = s0 + cell_count[cc];
                for (int q = s0; q < s1; ++q) {
                    const int j = cell_atoms[q];
                    if (j == (int)i) continue;
                    const double dx = min_image(pos[j] - xi, box.L[0], box.invL[0], box.pbc[0]);
                    const double dy = min_image(pos[N + j] - yi, box.L[1], box.invL[1], box.pbc[1]);
                    const double dz = min_image(pos[2 * N + j] - zi, box.L[2], box.invL[2], box.pbc[2]);
                    if (dx * dx + dy * dy + dz * dz < rl2) {
                        if (cnt < cap) {       // insertion into the sorted prefix
                            int m = cnt;
                            while (m > 0 && loc[m - 1] > j) {
                                loc[m] = loc[m - 1];
                                --m;
                            }
                            loc[m] = j;
                        }
                        ++cnt;
                    }
                }
            }
    const int keep = cnt < cap ? cnt : cap;
    for (int m = 0; m < keep; ++m) nl[(int64_t)m * N + i] = loc[m];
    nn[i] = keep;
    if (cnt > cap) flags->list_overflow = 1;
    atomicMax(&flags->max_nn, cnt);
}

// rev[m N + i] = slot of i in the list of j = nl[m N + i] (lists are symmetric).
__global__ void k_build_rev(int64_t N, const int *nn, const int *nl, uint8_t *rev, Flags *flags,
                            bool cond)
{
    if (skip(flags, cond)) return;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = nn[i];
    for (int m = 0; m < n; ++m) {
        const int j = nl[(int64_t)m * N + i];
        const int nj = nn[j];
        int found = -1;
        for (int q = 0; q < nj; ++q)
            if (nl[(int64_t)q * N + j] == (int)i) { found = q; break; }
        if (found < 0) { flags->asym = 1; found = 0; }
        rev[(int64_t)m * N + i] = (uint8_t)found;
    }
}

__global__ void k_build_done(Flags *flags, bool cond)
{
    if (skip(flags, cond)) return;
    flags->rebuild = 0;
    flags->n_rebuilds += 1;
}

__global__ void k_displacement(int64_t N, const double *pos, const double *pos_build, Box box,
                               double half_skin2, Flags *flags)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double d2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double d = min_image(pos[a * N + i] - pos_build[a * N + i], box.L[a], box.invL[a], box.pbc[a]);
        d2 = fma(d, d, d2);
    }
    if (!(d2 <= half_skin2)) flags->rebuild = 1;
}

__global__ void k_wrap(int64_t N, double *pos, Box box)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (!box.pbc[a]) continue;
        double x = pos[a * N + i];
        x -= box.L[a] * floor(x * box.invL[a]);
        if (x >= box.L[a]) x -= box.L[a];
        if (x < 0.0) x += box.L[a];
        pos[a * N + i] = x;
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int scan_block_elems() { return kScanElems; }

int launch_rebuild(const Plan &p, cudaStream_t s, bool cond)
{
    if (p.N == 0) return 0;
    const int T = 256;
    k_cell_clear<<<blocks_for(p.ncell, T), T, 0, s>>>(p.ncell, p.cell_count, p.flags, cond);
    k_cell_count<<<blocks_for(p.N, T), T, 0, s>>>(p.N, p.pos, p.box, p.nc[0], p.nc[1], p.nc[2],
                                                 p.atom_cell, p.atom_rank, p.cell_count, p.flags, cond);
    const int64_t nb = (p.ncell + kScanElems - 1) / kScanElems;
    k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, s>>>(p.ncell, p.cell_count, p.cell_start,
                                                        p.scan_blocks, p.flags, cond);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(nb, p.scan_blocks, p.flags, cond);
    k_scan_add<<<blocks_for(p.ncell, T), T, 0, s>>>(p.ncell, p.cell_start, p.scan_blocks, p.flags, cond);
    k_cell_fill<<<blocks_for(p.N, T), T, 0, s>>>(p.N, p.atom_cell, p.atom_rank, p.cell_start,
                                                p.cell_atoms, p.flags, cond);
    const int TB = 128;
    k_build_list<<<blocks_for(p.N, TB), TB, 0, s>>>(p.N, p.pos, p.box, p.nc[0], p.nc[1], p.nc[2],
                                                   p.atom_cell, p.cell_start, p.cell_count, p.cell_atoms,
                                                   p.rl * p.rl, p.cap, p.nn, p.nl, p.pos_build, p.flags, cond);
    k_build_rev<<<blocks_for(p.N, T), T, 0, s>>>(p.N, p.nn, p.nl, p.rev, p.flags, cond);
    k_build_done<<<1, 1, 0, s>>>(p.flags, cond);
    return 9;
}

void launch_displacement_check(const Plan &p, cudaStream_t s)
{
    if (p.N == 0) return;
    const int T = 256;
    const double hs = 0.5 * p.skin;
    k_displacement<<<blocks_for(p.N, T), T, 0, s>>>(p.N, p.pos, p.pos_build, p.box, hs * hs, p.flags);
}

void launch_wrap(const Plan &p, cudaStream_t s)
{
    if (p.N == 0) return;
    const int T = 256;
    k_wrap<<<blocks_for(p.N, T), T, 0, s>>>(p.N, p.pos, p.box);
}

}  // namespace mdk
