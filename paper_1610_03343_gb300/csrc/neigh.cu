// neigh.cu -- cell-list neighbour build (the paper's Sec. 2.1: a Verlet neighbour list
// built with the standard cell-list method for a uniform cutoff), the reverse-slot
// index the atomic-free gather needs, and the skin/2 displacement check.
//
// Build pipeline (one thread per atom or per cell):
//   zero cell counts -> wrap positions into the box, fp32 copy, cell id and rank in
//   cell (atomicAdd) -> exclusive scan of cell counts -> scatter atoms into cell order
//   -> per-atom search over the distinct neighbouring cells -> reverse slots -> done.
// Positions are wrapped only here: between builds they move freely, so every listed
// pair keeps the periodic image it was found with.  Each list entry therefore carries
// that image shift (see md_internal.cuh, "list entries") and a step computes r_ij with
// three fp64 subtractions instead of a minimum-image reduction.
//
// The candidate test runs in fp32 with a margin that covers the fp32 rounding of the
// coordinates, so the list is a superset of the exact fp64 list at rl; the force passes
// apply the exact cutoff.  fp32 negation is exact, so the test is symmetric in i and j
// and the lists stay symmetric.  Atom order inside a cell depends on atomic timing, but
// each list is sorted by atom index, so the lists are deterministic.
#include <algorithm>

#include "md_plan.cuh"

namespace mdk {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 4;
constexpr int kScanElems = kScanThreads * kScanPerThread;  // per block

// Cell index along one axis from the fp32 coordinate (FMA pipe instead of GB300's 1/64-rate
// fp64 pipe).  A coordinate within rounding distance of a cell boundary may land in the
// neighbouring cell; the cells are at least the list radius plus the fp32 margin wide, which
// exceeds that distance, so the 27-cell search still covers every neighbour within rl.
__device__ __forceinline__ int cell_coord_f(float x, int nc, float nc_over_L)
{
    const float t = fminf(fmaxf(x * nc_over_L, 0.f), (float)(nc - 1));
    return (int)t;
}

// x wrapped into [0, L) (periodic axis), in fp64 only for the atoms outside it: for
// non-negative doubles the bit patterns order like the values, so the test is integer.
__device__ __forceinline__ double wrap_coord(double x, double L, double invL)
{
    const long long xb = __double_as_longlong(x);
    if (xb >= 0 && xb < __double_as_longlong(L)) return x;
    x -= L * floor(x * invL);
    if (x >= L) x -= L;
    if (x < 0.0) x += L;
    return x;
}

// Wrap coordinates on periodic axes into [0, L), keep an fp32 copy, bin into cells.
// Pools (BATCH): only atoms of systems with a rebuild request, each in its own grid.
template <bool BATCH>
__device__ __forceinline__ void cell_count_atom(int64_t i, int64_t N, double *pos, float *posf, Box box0, int nc0,
                                                int nc1, int nc2, const int *sys_of, const SysDev *sys,
                                                int *atom_cell, int *atom_rank, int *count)
{
    const Box *bp = &box0;
    int nc[3] = {nc0, nc1, nc2};
    long long off = 0;
    if (BATCH) {
        const SysDev &sd = sys[sys_of[i]];
        if (!sd.rebuild) return;
        bp = &sd.box;
        nc[0] = sd.nc[0]; nc[1] = sd.nc[1]; nc[2] = sd.nc[2];
        off = sd.cell_off;
    } else if (sys) {   // single system under NPT: the box and grid of sys[0]
        bp = &sys[0].box;
        nc[0] = sys[0].nc[0]; nc[1] = sys[0].nc[1]; nc[2] = sys[0].nc[2];
    }
    const Box &box = *bp;
    int cc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = pos[a * N + i];
        if (box.pbc[a]) {
            const double xw = wrap_coord(x, box.L[a], box.invL[a]);
            if (__double_as_longlong(xw) != __double_as_longlong(x)) pos[a * N + i] = xw;
            x = xw;
        }
        const float xf = d2f_trunc(x);
        posf[a * N + i] = xf;
        cc[a] = cell_coord_f(xf, nc[a], (float)nc[a] * d2f_trunc(box.invL[a]));
    }
    const long long c = off + (cc[0] * nc[1] + cc[1]) * nc[2] + cc[2];
    atom_cell[i] = (int)c;
    atom_rank[i] = atomicAdd(&count[c], 1);
}

// Exclusive scan, pass 1: scan each block's kScanElems counts, store block totals.
__global__ void __launch_bounds__(kScanThreads)
k_scan_blocks(int64_t n, const int *in, int *out, int *block_sums)
{
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
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int64_t nb, int *block_sums)
{
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
__global__ void k_scan_add(int64_t n, int *out, const int *block_sums)
{
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n) out[idx] += block_sums[idx / kScanElems];
}

template <bool BATCH>
__device__ __forceinline__ void cell_fill_atom(int64_t i, const int *atom_cell, const int *atom_rank,
                                               const int *cell_start, int *cell_atoms, const int *sys_of,
                                               const SysDev *sys)
{
    if (BATCH && !sys[sys_of[i]].rebuild) return;
    cell_atoms[cell_start[atom_cell[i]] + atom_rank[i]] = (int)i;
}

// The stencil along one axis: the distinct cells c-1, c, c+1 (periodic: wrapped; open:
// clipped) as at most two runs of consecutive indices [lo0, hi0], [lo1, hi1]; `full` when
// they are every cell of the axis.  No integer division (the grid is not a power of two).
struct AxisRuns {
    int lo0, hi0, lo1, hi1, n;
    bool full;
};
__device__ __forceinline__ AxisRuns axis_runs(int c, int nc, int periodic)
{
    AxisRuns r{0, nc - 1, 0, 0, 1, true};
    if (periodic) {
        if (nc <= 3) return r;
        r.full = false;
        if (c == 0) { r.hi0 = 1; r.lo1 = r.hi1 = nc - 1; r.n = 2; }
        else if (c == nc - 1) { r.lo0 = nc - 2; r.lo1 = r.hi1 = 0; r.n = 2; }
        else { r.lo0 = c - 1; r.hi0 = c + 1; }
    } else {
        r.lo0 = c > 0 ? c - 1 : 0;
        r.hi0 = c + 1 < nc ? c + 1 : nc - 1;
        r.full = r.lo0 == 0 && r.hi0 == nc - 1;
    }
    return r;
}
// Item k of an axis: one of its runs (whole runs: the axes inside it are full, so the run's
// cells are one contiguous block of cell indices) or one of its cells.
__device__ __forceinline__ int axis_items(const AxisRuns &r, bool whole)
{
    return whole ? r.n : (r.hi0 - r.lo0 + 1) + (r.n == 2 ? r.hi1 - r.lo1 + 1 : 0);
}
__device__ __forceinline__ void axis_item(const AxisRuns &r, bool whole, int k, int &lo, int &hi)
{
    if (whole) {
        lo = k == 0 ? r.lo0 : r.lo1;
        hi = k == 0 ? r.hi0 : r.hi1;
    } else {
        const int n0 = r.hi0 - r.lo0 + 1;
        lo = hi = k < n0 ? r.lo0 + k : r.lo1 + (k - n0);
    }
}

// fp32 candidate test of the list build for atom i (coordinates xi, yi, zi, largest
// magnitude mag_i) and atom j: minimum-image separation below rl0 widened by the rounding
// of the larger coordinate of the two (the same test for (i, j) and (j, i)).  On success
// *entry is j with the image shift it was found at.
struct ListFrame {
    float xi, yi, zi, mag_i, rl0, L0, L1, L2, iL0, iL1, iL2;
    int p0, p1, p2;
};
__device__ __forceinline__ bool list_candidate(const ListFrame &f, float xj, float yj, float zj, int j, int *entry)
{
    float dx = xj - f.xi, dy = yj - f.yi, dz = zj - f.zi;
    // image shift s in {-1, 0, 1}: r_ij = x_j - x_i + s L
    const float sx = f.p0 ? -rintf(dx * f.iL0) : 0.f;
    const float sy = f.p1 ? -rintf(dy * f.iL1) : 0.f;
    const float sz = f.p2 ? -rintf(dz * f.iL2) : 0.f;
    dx = fmaf(sx, f.L0, dx);
    dy = fmaf(sy, f.L1, dy);
    dz = fmaf(sz, f.L2, dz);
    const float mag = fmaxf(f.mag_i, fmaxf(fabsf(xj), fmaxf(fabsf(yj), fabsf(zj))));
    const float lim = f.rl0 + 32.f * mag * 1.1920929e-7f;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    *entry = list_entry(j, (int)sx, (int)sy, (int)sz);
    return r2 < lim * lim;
}

__device__ __forceinline__ ListFrame list_frame(const float *posf, int64_t N, int64_t i, const Box &box, float rlm2)
{
    ListFrame f;
    f.xi = posf[i];
    f.yi = posf[N + i];
    f.zi = posf[2 * N + i];
    f.mag_i = fmaxf(fabsf(f.xi), fmaxf(fabsf(f.yi), fabsf(f.zi)));
    f.rl0 = sqrtf(rlm2);
    f.L0 = (float)box.L[0]; f.L1 = (float)box.L[1]; f.L2 = (float)box.L[2];
    f.iL0 = (float)box.invL[0]; f.iL1 = (float)box.invL[1]; f.iL2 = (float)box.invL[2];
    f.p0 = box.pbc[0]; f.p1 = box.pbc[1]; f.p2 = box.pbc[2];
    return f;
}

// One thread per atom: search the distinct neighbouring cells and keep every j != i
// with |r_ij| < rl + margin (fp32, minimum image), in ascending index order, each with
// the image shift it was found at.  Snapshots the build positions for the skin test.
// Returns the number of atoms found (0 for an atom of a system that is not rebuilt).
template <bool BATCH>
__device__ __forceinline__ int build_list_atom(int64_t i, int64_t N, const double *pos, const float *posf,
                                                Box box0, int nc0, int nc1, int nc2, const int *sys_of,
                                                SysDev *sys, const int *atom_cell, const int *cell_start,
                                                const int *cell_count, const int *cell_atoms, float rlm2, int cap,
                                                int *nn, int *nl, double *pos_build, Flags *flags)
{
    const Box *bp = &box0;
    int nc[3] = {nc0, nc1, nc2};
    long long off = 0;
    if (BATCH) {
        const SysDev &sd = sys[sys_of[i]];
        if (!sd.rebuild) return 0;
        bp = &sd.box;
        nc[0] = sd.nc[0]; nc[1] = sd.nc[1]; nc[2] = sd.nc[2];
        off = sd.cell_off;
        rlm2 = sd.rlm2;
    } else if (sys) {   // single system under NPT: the box and grid of sys[0]
        bp = &sys[0].box;
        nc[0] = sys[0].nc[0]; nc[1] = sys[0].nc[1]; nc[2] = sys[0].nc[2];
    }
    const Box &box = *bp;
    const double b0 = pos[i], b1 = pos[N + i], b2 = pos[2 * N + i];
    const ListFrame fr = list_frame(posf, N, i, box, rlm2);
    // the atom's cell from its fp32 coordinates, as the count pass computed it
    const int cx = cell_coord_f(fr.xi, nc[0], (float)nc[0] * d2f_trunc(box.invL[0]));
    const int cy = cell_coord_f(fr.yi, nc[1], (float)nc[1] * d2f_trunc(box.invL[1]));
    const int cz = cell_coord_f(fr.zi, nc[2], (float)nc[2] * d2f_trunc(box.invL[2]));
    // The stencil as ranges of cell indices (cell = (x nc1 + y) nc2 + z): z in runs; y in
    // runs when z is full, else cell by cell; x likewise when y and z are full.  A range's
    // atoms are one contiguous block of cell_atoms.  On the sheet (one cell along z) the 9
    // cells are 3 ranges.
    const AxisRuns rx = axis_runs(cx, nc[0], box.pbc[0]);
    const AxisRuns ry = axis_runs(cy, nc[1], box.pbc[1]);
    const AxisRuns rz = axis_runs(cz, nc[2], box.pbc[2]);
    const bool wy = rz.full, wx = rz.full && ry.full;
    const int nX = axis_items(rx, wx), nY = axis_items(ry, wy), nZ = rz.n;
    auto range_at = [&](int ix, int iy, int iz, int &q0, int &q1) {
        int xl, xh, yl, yh, zl, zh;
        axis_item(rx, wx, ix, xl, xh);
        axis_item(ry, wy, iy, yl, yh);
        axis_item(rz, true, iz, zl, zh);
        const long long clo = off + ((long long)xl * nc[1] + yl) * nc[2] + zl;
        const long long chi = off + ((long long)xh * nc[1] + yh) * nc[2] + zh;
        q0 = cell_start[clo];
        q1 = cell_start[chi] + cell_count[chi];
    };
    // odometer over the ranges; the next range's bounds are loaded one range ahead
    auto step = [&](int &ix, int &iy, int &iz) {
        if (++iz == nZ) {
            iz = 0;
            if (++iy == nY) {
                iy = 0;
                ++ix;
            }
        }
        return ix < nX;
    };
    int q, qe, q2 = 0, qe2 = 0;
    range_at(0, 0, 0, q, qe);
    int jx = 0, jy = 0, jz = 0;
    bool more = step(jx, jy, jz);
    if (more) range_at(jx, jy, jz, q2, qe2);
    int loc[kMaxListCap];
    int cnt = 0;
    // the candidates as one sequence taken four at a time, so that four candidates' loads
    // are in flight together
    while (true) {
        int jj[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            while (q >= qe && more) {
                q = q2;
                qe = qe2;
                more = step(jx, jy, jz);
                if (more) range_at(jx, jy, jz, q2, qe2);
            }
            jj[u] = q < qe ? cell_atoms[q++] : -1;
        }
        if (jj[0] < 0) break;
        float xs[4], ys[4], zs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = jj[u] < 0 ? (int)i : jj[u];
            xs[u] = posf[j];
            ys[u] = posf[N + j];
            zs[u] = posf[2 * N + j];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = jj[u];
            if (j < 0 || j == (int)i) continue;
            int e_;
            if (list_candidate(fr, xs[u], ys[u], zs[u], j, &e_)) {
                if (cnt < cap) {       // insertion into the index-sorted prefix
                    int m = cnt;
                    while (m > 0 && list_atom(loc[m - 1]) > j) {
                        loc[m] = loc[m - 1];
                        --m;
                    }
                    loc[m] = e_;
                }
                ++cnt;
            }
        }
    }
    pos_build[i] = b0;
    pos_build[N + i] = b1;
    pos_build[2 * N + i] = b2;
    const int keep = cnt < cap ? cnt : cap;
    for (int m = 0; m < keep; ++m) nl[(int64_t)m * N + i] = loc[m];
    nn[i] = keep;
    if (cnt > cap) {
        if (BATCH) fail_system(sys[sys_of[i]], MD_ERR_NEIGH_OVERFLOW);   // this system only
        else flags->list_overflow = 1;
    }
    return cnt;
}

// flags->max_nn = max(flags->max_nn, the warp's largest cnt): one atomic per warp.  Every
// lane of the warp calls it (0 for an atom it did not build).
__device__ __forceinline__ void warp_max_nn(int cnt, Flags *flags)
{
    const int wmax = __reduce_max_sync(0xffffffffu, cnt);
    if ((threadIdx.x & 31) == 0 && wmax > 0) atomicMax(&flags->max_nn, wmax);
}

// rev[m N + i] = slot of i in the list of j = atom of nl[m N + i] (lists are symmetric).
template <bool BATCH>
__device__ __forceinline__ void build_rev_atom(int64_t i, int64_t N, const int *nn, const int *nl, uint8_t *rev,
                                               const int *sys_of, const SysDev *sys, Flags *flags)
{
    if (BATCH && !sys[sys_of[i]].rebuild) return;
    const int n = nn[i];
    for (int m = 0; m < n; ++m) {
        const int j = list_atom(nl[(int64_t)m * N + i]);
        const int nj = nn[j];
        int found = -1;
        for (int q = 0; q < nj; ++q)
            if (list_atom(nl[(int64_t)q * N + j]) == (int)i) { found = q; break; }
        if (found < 0) { flags->asym = 1; found = 0; }
        rev[(int64_t)m * N + i] = (uint8_t)found;
    }
}

// Single system: one thread per atom.
// sys1: null, or (NPT) the system whose device box and grid replace box and nc.
__global__ void k_cell_count(int64_t N, double *pos, float *posf, Box box, int nc0, int nc1, int nc2,
                             const SysDev *sys1, int *atom_cell, int *atom_rank, int *count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) cell_count_atom<false>(i, N, pos, posf, box, nc0, nc1, nc2, nullptr, sys1, atom_cell, atom_rank, count);
}
__global__ void k_cell_fill(int64_t N, const int *atom_cell, const int *atom_rank, const int *cell_start,
                            int *cell_atoms)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) cell_fill_atom<false>(i, atom_cell, atom_rank, cell_start, cell_atoms, nullptr, nullptr);
}
__global__ void k_build_list(int64_t N, const double *pos, const float *posf, Box box, int nc0, int nc1, int nc2,
                             SysDev *sys1, const int *atom_cell, const int *cell_start,
                             const int *cell_count, const int *cell_atoms, float rlm2, int cap, int *nn, int *nl,
                             double *pos_build, Flags *flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int cnt = 0;
    if (i < N)
        cnt = build_list_atom<false>(i, N, pos, posf, box, nc0, nc1, nc2, nullptr, sys1, atom_cell, cell_start,
                                     cell_count, cell_atoms, rlm2, cap, nn, nl, pos_build, flags);
    warp_max_nn(cnt, flags);
}
__global__ void k_build_rev(int64_t N, const int *nn, const int *nl, uint8_t *rev, Flags *flags)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) build_rev_atom<false>(i, N, nn, nl, rev, nullptr, nullptr, flags);
}

// Pools: a rebuild touches only the systems that requested one.  The plan kernel lists
// them and their 128-atom chunks (every system starts on a chunk boundary); the other
// kernels loop over those lists with a bounded grid, so a rebuild costs in proportion
// to the systems rebuilt, not to the pool's capacity.
//   plan[0] = number of chunks, plan[1] = number of systems;
//   chunks[k] = first atom of chunk k; rsys[k] = k-th system to rebuild.
constexpr int kChunk = 128;
__global__ void __launch_bounds__(1024) k_rebuild_plan(int n_sys, const SysDev *sys, int *plan, int *rsys,
                                                       int *chunks, Flags *flags)
{
    __shared__ int warp_a[32], warp_b[32];
    __shared__ int carry_a, carry_b;
    if (threadIdx.x == 0) { carry_a = 0; carry_b = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int s0 = 0; s0 < n_sys; s0 += blockDim.x) {
        const int s = s0 + threadIdx.x;
        const bool f = s < n_sys && sys[s].rebuild;
        const int nch = f ? (int)((sys[s].n_atoms + kChunk - 1) / kChunk) : 0;
        int a = f ? 1 : 0, b = nch;          // inclusive scans of flags and chunk counts
        for (int o = 1; o < 32; o <<= 1) {
            const int ya = __shfl_up_sync(0xffffffffu, a, o), yb = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) { a += ya; b += yb; }
        }
        if (lane == 31) { warp_a[wid] = a; warp_b[wid] = b; }
        __syncthreads();
        if (wid == 0) {
            int wa = lane < (int)(blockDim.x >> 5) ? warp_a[lane] : 0, wb = lane < (int)(blockDim.x >> 5) ? warp_b[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int ya = __shfl_up_sync(0xffffffffu, wa, o), yb = __shfl_up_sync(0xffffffffu, wb, o);
                if (lane >= o) { wa += ya; wb += yb; }
            }
            warp_a[lane] = wa;
            warp_b[lane] = wb;
        }
        __syncthreads();
        const int pa = carry_a + (wid ? warp_a[wid - 1] : 0) + a - (f ? 1 : 0);
        const int pb = carry_b + (wid ? warp_b[wid - 1] : 0) + b - nch;
        if (f) {
            rsys[pa] = s;
            const long long a0 = sys[s].atom_start;
            for (int k = 0; k < nch; ++k) chunks[pb + k] = (int)(a0 + (long long)k * kChunk);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            carry_a += warp_a[(blockDim.x >> 5) - 1];
            carry_b += warp_b[(blockDim.x >> 5) - 1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        plan[0] = carry_b;
        plan[1] = carry_a;
        flags->rebuild = 0;                   // the requests are taken by this plan
        if (carry_a > 0) {
            flags->max_nn = 0;                // the longest list of this build
            flags->n_rebuilds += 1;
        }
    }
}

// Exclusive scan of each rebuilt system's cell counts, offset by its first atom (its
// atoms fill cell_atoms[atom_start, atom_start + n_atoms) in cell order).  One block per
// system: 1024 threads x 8 cells per pass.
constexpr int kPoolScanThreads = 1024;
constexpr int kPoolScanPer = 8;
__global__ void __launch_bounds__(kPoolScanThreads) k_cells_scan_pool(const int *plan, const int *rsys,
                                                                      const SysDev *sys, const int *count,
                                                                      int *start)
{
    __shared__ int warp_tot[32];
    __shared__ int carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int k = blockIdx.x; k < plan[1]; k += gridDim.x) {
        const SysDev &sd = sys[rsys[k]];
        const long long nc = (long long)sd.nc[0] * sd.nc[1] * sd.nc[2];
        if (threadIdx.x == 0) carry = (int)sd.atom_start;
        __syncthreads();
        for (long long c0 = 0; c0 < nc; c0 += (long long)kPoolScanThreads * kPoolScanPer) {
            const long long cb = c0 + (long long)threadIdx.x * kPoolScanPer;
            int v[kPoolScanPer];
            int t = 0;
#pragma unroll
            for (int q = 0; q < kPoolScanPer; ++q) {
                v[q] = cb + q < nc ? count[sd.cell_off + cb + q] : 0;
                t += v[q];
            }
            int incl = t;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) warp_tot[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                int w = warp_tot[lane];
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, w, o);
                    if (lane >= o) w += y;
                }
                warp_tot[lane] = w;
            }
            __syncthreads();
            int run = carry + (wid ? warp_tot[wid - 1] : 0) + incl - t;
#pragma unroll
            for (int q = 0; q < kPoolScanPer; ++q) {
                if (cb + q < nc) start[sd.cell_off + cb + q] = run;
                run += v[q];
            }
            __syncthreads();
            if (threadIdx.x == 0) carry += warp_tot[31];
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kChunk) k_cell_count_pool(const int *plan, const int *chunks, int64_t N,
                                                            double *pos, float *posf, const int *sys_of,
                                                            const SysDev *sys, int *atom_cell, int *atom_rank,
                                                            int *count)
{
    for (int k = blockIdx.x; k < plan[0]; k += gridDim.x)
        cell_count_atom<true>(chunks[k] + threadIdx.x, N, pos, posf, Box{}, 1, 1, 1, sys_of, sys, atom_cell,
                              atom_rank, count);
}
__global__ void __launch_bounds__(kChunk) k_cell_fill_pool(const int *plan, const int *chunks, const int *atom_cell,
                                                           const int *atom_rank, const int *cell_start,
                                                           int *cell_atoms, const int *sys_of, const SysDev *sys)
{
    for (int k = blockIdx.x; k < plan[0]; k += gridDim.x)
        cell_fill_atom<true>(chunks[k] + threadIdx.x, atom_cell, atom_rank, cell_start, cell_atoms, sys_of, sys);
}
__global__ void __launch_bounds__(kChunk) k_build_list_pool(const int *plan, const int *chunks, int64_t N,
                                                            const double *pos, const float *posf,
                                                            const int *sys_of, SysDev *sys,
                                                            const int *atom_cell, const int *cell_start,
                                                            const int *cell_count, const int *cell_atoms, int cap,
                                                            int *nn, int *nl, double *pos_build, Flags *flags)
{
    for (int k = blockIdx.x; k < plan[0]; k += gridDim.x) {
        const int cnt = build_list_atom<true>(chunks[k] + threadIdx.x, N, pos, posf, Box{}, 1, 1, 1, sys_of, sys,
                                              atom_cell, cell_start, cell_count, cell_atoms, 0.f, cap, nn, nl,
                                              pos_build, flags);
        warp_max_nn(cnt, flags);
    }
}
// Reverse slots of the rebuilt systems' atoms (their chunks only; padding atoms belong to the
// inactive sentinel, which has no atoms), then the rest of the build: every atom zeroes its
// cell's count (so the next build needs no clearing pass; every other cell is already zero)
// and the first atom of each system clears its request and marks it built.
__global__ void __launch_bounds__(kChunk) k_build_rev_pool(const int *plan, const int *chunks, int64_t N,
                                                           const int *nn, const int *nl, uint8_t *rev,
                                                           const int *sys_of, SysDev *sys, const int *atom_cell,
                                                           int *count, Flags *flags)
{
    for (int k = blockIdx.x; k < plan[0]; k += gridDim.x) {
        const int64_t i = chunks[k] + threadIdx.x;
        SysDev &sd = sys[sys_of[i]];
        if (i - sd.atom_start >= sd.n_atoms) continue;
        // a system whose list overflowed has truncated, asymmetric lists: it has failed
        // and stopped, and its reverse slots are not needed
        if (sd.error == 0) build_rev_atom<false>(i, N, nn, nl, rev, nullptr, nullptr, flags);
        count[atom_cell[i]] = 0;
        if (i == sd.atom_start) {
            sd.rebuild = 0;
            sd.built = 1;
            sd.npt.mu_cum[0] = sd.npt.mu_cum[1] = sd.npt.mu_cum[2] = 1.0;
            atomicAdd(reinterpret_cast<unsigned long long *>(&flags->atoms_rebuilt), (unsigned long long)sd.n_atoms);
        }
    }
}

// skin/2 test.  Positions are not wrapped between builds, so x - x_build is the true
// displacement; the difference is taken in fp64 and squared in fp32.  NPT systems use the
// bound that accounts for the box scaling since the build.
template <bool BATCH>
__global__ void k_displacement(int64_t N, const double *pos, const double *pos_build, float half_skin2,
                               const int *sys_of, SysDev *sys, int npt, Flags *flags)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (BATCH && !sys[sys_of[i]].active) return;
    if (BATCH) half_skin2 = sys[sys_of[i]].half_skin2;
    if (npt) {
        const SysDev &sd = BATCH ? sys[sys_of[i]] : sys[0];
        if (sd.npt.on) half_skin2 = npt_half_skin2(sd, false);
    }
    float d2 = 0.f;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float d = d2f_trunc(pos[a * N + i] - pos_build[a * N + i]);
        d2 = fmaf(d, d, d2);
    }
    if (!(d2 <= half_skin2)) {
        flags->rebuild = 1;
        if (BATCH) sys[sys_of[i]].rebuild = 1;
    }
}

// Per-axis cell occupancy (see launch_axis_occupancy): each atom flags the cell it falls in
// along each axis (the same coordinate as the count pass: wrapped on periodic axes).
__global__ void k_axis_occupancy(int64_t N, const double *pos, Box box, int nc0, int nc1, int nc2, uint8_t *occ)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int nc[3] = {nc0, nc1, nc2};
    int off = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = pos[a * N + i];
        if (box.pbc[a]) x = wrap_coord(x, box.L[a], box.invL[a]);
        const float xf = d2f_trunc(x);
        occ[off + cell_coord_f(xf, nc[a], (float)nc[a] * d2f_trunc(box.invL[a]))] = 1;
        off += nc[a];
    }
}

// Wrapped copy of the positions (for output): dst[3N] = pos wrapped into [0, L).
template <bool BATCH>
__global__ void k_wrap_copy(int64_t N, int64_t a0, int64_t n, const double *pos, double *dst, Box box0,
                            const int *sys_of, const SysDev *sys, int dev_box)
{
    const int64_t i = a0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a0 + n) return;
    const Box &box = BATCH ? sys[sys_of[i]].box : (dev_box ? sys[0].box : box0);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double x = pos[a * N + i];
        if (box.pbc[a]) {
            x -= box.L[a] * floor(x * box.invL[a]);
            if (x >= box.L[a]) x -= box.L[a];
            if (x < 0.0) x += box.L[a];
        }
        dst[a * N + i] = x;
    }
}

// Single system: clear the rebuild request and count the build.  The build positions are
// now the wrapped positions: no box scaling since the build (NPT).
__global__ void k_build_done(int64_t n_atoms, SysDev *sys, Flags *flags)
{
    flags->atoms_rebuilt += n_atoms;
    sys[0].npt.mu_cum[0] = sys[0].npt.mu_cum[1] = sys[0].npt.mu_cum[2] = 1.0;
    flags->rebuild = 0;
    flags->n_rebuilds += 1;
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int scan_block_elems() { return kScanElems; }

float list_margin_for(double lmax, double rl)
{
    // Bound on the fp32 error of a listed separation: coordinates below 2^e carry an
    // absolute rounding error of at most 2^(e-24); a difference, a shift by L and the
    // squared norm stay within a few of those units per component.
    if (lmax < 1.0) lmax = 1.0;
    const double ulp = std::ldexp(1.0, std::ilogb(lmax) + 1 - 24);
    return (float)(16.0 * ulp + 1e-6 * rl);
}

int rebuild_single(const Plan &p, cudaStream_t s)
{
    const int T = 256;
    cudaMemsetAsync(p.cell_count, 0, sizeof(int) * p.ncell, s);
    cudaMemsetAsync(&p.flags->max_nn, 0, sizeof(int), s);
    SysDev *sys1 = p.npt ? p.sys : nullptr;
    k_cell_count<<<blocks_for(p.N, T), T, 0, s>>>(p.N, p.pos, p.posf, p.box, p.nc[0], p.nc[1], p.nc[2], sys1,
                                                 p.atom_cell, p.atom_rank, p.cell_count);
    const int64_t nb = (p.ncell + kScanElems - 1) / kScanElems;
    k_scan_blocks<<<(unsigned)nb, kScanThreads, 0, s>>>(p.ncell, p.cell_count, p.cell_start, p.scan_blocks);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(nb, p.scan_blocks);
    k_scan_add<<<blocks_for(p.ncell, T), T, 0, s>>>(p.ncell, p.cell_start, p.scan_blocks);
    k_cell_fill<<<blocks_for(p.N, T), T, 0, s>>>(p.N, p.atom_cell, p.atom_rank, p.cell_start, p.cell_atoms);
    const int TB = 128;
    const float rlm = (float)p.rl + p.list_margin;
    k_build_list<<<blocks_for(p.N, TB), TB, 0, s>>>(p.N, p.pos, p.posf, p.box, p.nc[0], p.nc[1], p.nc[2], sys1,
                                                   p.atom_cell, p.cell_start, p.cell_count, p.cell_atoms,
                                                   rlm * rlm, p.cap, p.nn, p.nl, p.pos_build, p.flags);
    k_build_rev<<<blocks_for(p.N, T), T, 0, s>>>(p.N, p.nn, p.nl, p.rev, p.flags);
    k_build_done<<<1, 1, 0, s>>>(p.N, p.sys, p.flags);
    return 8;
}

int rebuild_pool(const Plan &p, cudaStream_t s)
{
    // grids bounded by the work a rebuild can have: loop over the listed chunks/systems
    const unsigned gc = (unsigned)std::min<int64_t>((p.N + kChunk - 1) / kChunk, 8 * 152);
    const unsigned gs = (unsigned)std::min<int64_t>(p.n_sys, 4 * 152);
    k_rebuild_plan<<<1, 1024, 0, s>>>(p.n_sys, p.sys, p.rb_plan, p.rb_sys, p.rb_chunks, p.flags);
    k_cell_count_pool<<<gc, kChunk, 0, s>>>(p.rb_plan, p.rb_chunks, p.N, p.pos, p.posf, p.sys_of, p.sys,
                                            p.atom_cell, p.atom_rank, p.cell_count);
    k_cells_scan_pool<<<gs, kPoolScanThreads, 0, s>>>(p.rb_plan, p.rb_sys, p.sys, p.cell_count, p.cell_start);
    k_cell_fill_pool<<<gc, kChunk, 0, s>>>(p.rb_plan, p.rb_chunks, p.atom_cell, p.atom_rank, p.cell_start,
                                           p.cell_atoms, p.sys_of, p.sys);
    k_build_list_pool<<<gc, kChunk, 0, s>>>(p.rb_plan, p.rb_chunks, p.N, p.pos, p.posf, p.sys_of, p.sys,
                                            p.atom_cell, p.cell_start, p.cell_count, p.cell_atoms, p.cap, p.nn,
                                            p.nl, p.pos_build, p.flags);
    k_build_rev_pool<<<gc, kChunk, 0, s>>>(p.rb_plan, p.rb_chunks, p.N, p.nn, p.nl, p.rev, p.sys_of, p.sys,
                                           p.atom_cell, p.cell_count, p.flags);
    return 6;
}

int launch_rebuild(const Plan &p, cudaStream_t s)
{
    if (p.N == 0) return 0;
    return p.batch ? rebuild_pool(p, s) : rebuild_single(p, s);
}

void launch_displacement_check(const Plan &p, cudaStream_t s)
{
    if (p.N == 0) return;
    const int T = 256;
    const double hs = 0.5 * p.skin;
    if (p.batch)
        k_displacement<true><<<blocks_for(p.N, T), T, 0, s>>>(p.N, p.pos, p.pos_build, (float)(hs * hs),
                                                             p.sys_of, p.sys, p.npt ? 1 : 0, p.flags);
    else
        k_displacement<false><<<blocks_for(p.N, T), T, 0, s>>>(p.N, p.pos, p.pos_build, (float)(hs * hs),
                                                              p.sys_of, p.sys, p.npt ? 1 : 0, p.flags);
}

void launch_axis_occupancy(const Plan &p, cudaStream_t s, const Box &box, const int nc[3], uint8_t *occ)
{
    if (p.N <= 0) return;
    k_axis_occupancy<<<blocks_for(p.N, 256), 256, 0, s>>>(p.N, p.pos, box, nc[0], nc[1], nc[2], occ);
}

void launch_wrap_copy(const Plan &p, cudaStream_t s, double *dst, int64_t a0, int64_t n)
{
    if (n <= 0) return;
    const int T = 256;
    if (p.batch)
        k_wrap_copy<true><<<blocks_for(n, T), T, 0, s>>>(p.N, a0, n, p.pos, dst, p.box, p.sys_of, p.sys, 0);
    else
        k_wrap_copy<false><<<blocks_for(n, T), T, 0, s>>>(p.N, a0, n, p.pos, dst, p.box, p.sys_of, p.sys,
                                                           p.npt ? 1 : 0);
}

}  // namespace mdk
