// md_internal.cuh -- device-side structures and helpers shared by the CUDA translation
// units of libmd (neighbour build, force passes, integrator, C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "md.h"

namespace mdk {

// eV/(A amu) -> A/fs^2 (exact elementary charge, CODATA-2018 atomic mass constant)
constexpr double kAccUnit = 9.648533215665328e-3;
constexpr int kMaxTypes = 4;
constexpr int kMaxListCap = 32;   // list slots per atom (active mask is 32 bits)

// List entries.  A neighbour-list entry packs the neighbour's index (low 26 bits, so a
// context holds at most 2^26 atoms) with the periodic image it was found at when the
// list was built: code = (sx+1) + 3 (sy+1) + 9 (sz+1) in bits 26..30, s in {-1, 0, 1},
// and r_ij = r_j - r_i + (sx Lx, sy Ly, sz Lz).  Code 13 means no shift.
constexpr int kAtomBits = 26;
constexpr int kAtomMask = (1 << kAtomBits) - 1;
constexpr int kNoShift = 13;
constexpr int64_t kMaxAtoms = (int64_t)1 << kAtomBits;

__host__ __device__ __forceinline__ int list_entry(int j, int sx, int sy, int sz)
{
    return j | (((sx + 1) + 3 * (sy + 1) + 9 * (sz + 1)) << kAtomBits);
}
__host__ __device__ __forceinline__ int list_atom(int e) { return e & kAtomMask; }
__host__ __device__ __forceinline__ int list_code(int e) { return (int)((unsigned)e >> kAtomBits); }

// Orthorhombic box with per-axis periodicity.
struct Box {
    double L[3];
    double invL[3];
    int pbc[3];
};

// Systems of a pool.  A context holds up to max_systems independent systems over one
// flattened atom index; each owns the contiguous atom range [atom_start, atom_start +
// n_atoms), its own box, cell grid (cells [cell_off, cell_off + nc0 nc1 nc2)) and
// parameter set.  The table lives in device memory; the host edits it between calls.
constexpr int kMaxSets = 4;

// Berendsen weak coupling of one system to a heat bath and a pressure bath (NPT;
// Berendsen et al., J. Chem. Phys. 81, 3684 (1984)), the ensemble of the paper's
// benchmarks (Sec. 3: 300 K, 0 Pa).  At the end of a step, from that step's totals,
//   lambda = sqrt(1 + dt/tau_T (T0/T - 1)),              T = 2K / (k_B (3N - 3)),
//   mu_a   = cbrt(1 - beta dt/tau_P (P0 - P_aa)),        P_aa = (2 K_aa + W_aa) / V,
// with W the total virial (the sum of Eq. 29); the next step starts by multiplying the
// velocities by lambda and every coordinate and box edge along a by mu_a.
struct NptDev {
    int on;               // 1: couple this system; 0: NVE (or damped)
    int couple[3];        // the barostat scales this axis (periodic axes only)
    double T0, P0;        // K, GPa
    double tau_T, tau_P;  // fs (<= 0: that half is off)
    double beta;          // isothermal compressibility, 1/GPa
    double lam;           // pending velocity scale ...
    double mu[3];         // ... and coordinate / edge scales
    int pending;          // 1: lam, mu computed at the end of the last step, not yet applied
    int pad;
    double mu_cum[3];     // product of the edge scales applied since the last list build
};

struct SysDev {
    Box box;
    int nc[3];
    int pset;                 // parameter set index
    long long cell_off;       // first cell of this system's grid
    long long atom_start;     // first atom
    long long n_atoms;
    long long steps_left;     // steps still to run (< 0: unlimited); 0 stops the system
    double damp;              // velocity damping gamma (1/fs) after each step; 0 = NVE
    float rlm2;               // (list cutoff + fp32 margin)^2 of this system's parameter set
    float half_skin2;         // (skin/2)^2
    int active;               // 1 while the system is stepped
    int rebuild;              // 1: rebuild this system's lists at the next rebuild
    int built;                // 1 once its lists exist
    int fresh;                // 1 until its first force evaluation (just admitted)
    int error;                // pools: md_status of the failure that stopped this system
                              // (0 = none); the rest of the pool keeps running
    double rc;                // potential cutoff of this system's parameter set
    double rl;                // list radius rc + skin
    double cell_edge;         // smallest cell edge the 27-cell stencil allows (rl + fp32 margin)
    NptDev npt;
};

// Device status words written by kernels and read by the host after a call.
struct Flags {
    int rebuild;          // 1: list must be rebuilt before the next force pass
    int list_overflow;    // an atom found more than max_neigh neighbours
    int active_overflow;  // an atom had more than max_active neighbours inside the cutoff
    int nonfinite;        // a non-finite force appeared
    int asym;             // a pair was missing from the partner's list
    int max_nn;           // longest list at the last build
    int n_rebuilds;       // builds since creation
    int box_error;        // NPT: a periodic edge shrank below 2 (list radius + margin)
    long long step;       // index of the next series row
    long long row;        // series row of the step in flight
    int fresh_only;       // pools: the force evaluation in flight covers admitted systems only
    int pad2;
    long long atoms_rebuilt;   // atoms whose list was built, summed over builds
    long long row_reduce;      // series row of the last gather's partials (the reduction of a
                               // step may run beside the next step's first kernels)
};

// Pools: a failure that concerns one system only (a non-finite force, position or
// velocity, an overlong neighbour list, a box shrunk below the cutoff) is recorded in that
// system's entry -- the first status stays -- and stops it; the other systems of the pool
// are not affected (their atoms never list its atoms).
__device__ __forceinline__ void fail_system(SysDev &sd, int status)
{
    atomicCAS(&sd.error, 0, status);
    sd.active = 0;
}

// Pools: does atom work of system `sd` run now?  Stopped systems never; during the
// force evaluation that follows admissions, only the newly admitted systems.
__device__ __forceinline__ bool system_live(const SysDev &sd, const Flags *f)
{
    return sd.active != 0 && (f->fresh_only == 0 || sd.fresh != 0);
}

// Tersoff (single element).  Eqs. 2-6 with Tersoff-1989 f_R, f_A, f_C.
struct TersoffP {
    double A, B, lam, mu, beta, n, c, d, h, R, S;
    double c2, d2, c2d2;        // c^2, d^2, c^2/d^2
    double pi_SR;               // pi / (S - R)
    double ln_beta;             // log(beta)   (beta > 0), used in (beta zeta)^n
    double inv2n;               // 1 / (2 n)
    int beta_zero;              // beta == 0: b = 1 (pair limit)
};

// Stillinger-Weber (single element), U_i = 1/2 sum_j phi2 + sum_{j<k} phi3 (vertex i).
struct SWP {
    double eps, sig, a, lam, gam, A, B, p, q;
    double rc;                  // a * sigma
    double Aeps, lameps, gamsig;
    int p_int, q_int;           // exponents as integers when they are (4 and 0 in SW 1985)
};

// dU_i/dr_ij of one bond as a 16- (fp32) or 32-byte (fp64) vector: x, y, z and an unused
// fourth word, so that the gather reads a partner's value with one vector load (one memory
// sector) instead of three loads from three component planes.
template <typename T>
struct alignas(4 * sizeof(T)) Vec4 {
    T x, y, z, w;
};

// Arguments of the per-atom pair pass (one thread per atom i; computes U_i and
// dU_i/dr_ij for every in-cutoff neighbour j of i, Eqs. 14 / 28-30's building block).
template <typename T>
struct PairArgs {
    int64_t N;
    Box box;
    const double *pos;      // 3N SoA
    const int *nn;          // N list lengths
    const int *nl;          // cap x N, column-major: nl[m N + i]
    int cap;                // list capacity
    T rc2;                  // cutoff^2 in T
    // outputs, "compact active" layout: row k = k-th in-cutoff neighbour of i, with a row
    // stride of S = allocated rows (the staging capacity of a kernel may be smaller)
    int stride;             // S
    Vec4<T> *d;             // S x N : d[k N + i] = dU_i/dr_ij
    T *r;                   // 3 x S x N : r[(c S + k) N + i] = r_ij (component c)
    const int *sys_of;      // N: system of each atom (pools)
    SysDev *sys;            // system table (pools; a single system: its one entry)
    int dev_box;            // single system: read the box from sys[0] (it changes under NPT)
    const int *type;        // N: element of each atom (multi-element Tersoff)
    const void *ttab;       // multi-element Tersoff: kMaxTypes x kMaxTypes constants per
                            // ordered element pair, in T (see force.cu, TersoffC)
    int *ovf_count;         // atoms deferred by the small-capacity pass ...
    int *ovf_list;          // ... and their indices (capacity N)
    const int *act_count;   // pools: number of live 128-atom chunks ...
    const int *act_chunks;  // ... and their first atoms
    const float *posf;      // fp32 positions of this step (prefilter of list entries)
    float margin;           // fp32 rounding margin of that prefilter
    uint32_t *mask;         // N : bit m set <=> list slot m is inside the cutoff
    double *u;              // N : U_i
    Flags *flags;
    int batch;              // pools: failures go to the atom's system entry (fail_system)
};

// Arguments of the per-atom gather (one thread per atom i; Eqs. 28-30 + half-kick).
template <typename T>
struct GatherArgs {
    int64_t N;
    int64_t n_live;         // atoms gathered, kicked and summed: [0, n_live) (ghosts beyond)
    const int *nl;
    const uint8_t *rev;     // cap x N: slot of i in j's list
    const uint32_t *mask;
    const Vec4<T> *d;       // MAXA x N (see PairArgs)
    const T *r;
    const double *u;
    const int *type;
    double mass[kMaxTypes];
    T hm[kMaxTypes];        // m / (2 acc) per type in T (kinetic energy m v^2 / 2)
    double hk[kMaxTypes];   // half-kick factor dt/2 * acc / m per type
    int kick;               // apply the half-kick v += hk F
    double *vel;            // 3N, updated in place when kicking
    double *force;          // 3N, written
    double *w_out;          // 9N or nullptr
    double *j_out;          // 3N or nullptr
    double *partials;       // per (block, system segment): partials[(b seg_max + seg) NC + c]
    int seg_max;            // system segments a block may hold
    const int *sys_of;      // N: system of each atom (pools)
    SysDev *sys;            // system table (pools)
    double dt;              // time step (damping, fused kick)
    const int *act_count;   // pools: live chunks (see PairArgs)
    const int *act_chunks;
    Flags *flags;
    // fused first half of the next step (graph-replayed steps that are followed by another
    // in the same graph): after the second half-kick, v += hk F, x += v dt and the skin test,
    // exactly as k_kick_drift would do at the start of the next step
    int fuse_kick;
    double *pos;
    const double *pos_build;
    float *posf;            // fp32 positions to refresh (pair-pass prefilter), or null
    float half_skin2;       // single system: (skin/2)^2
};

// per-block partial sums: U, K, J(3), W(9); a velocity-Verlet step needs the first 5,
// a step under Berendsen coupling (NPT) those 5 and K_aa(3), W_aa(3) (totals of the last
// 6 go to a separate n_sys x 6 array)
constexpr int kNumPartials = 14;
constexpr int kStepPartials = 5;
constexpr int kNptPartials = 11;
constexpr int kNptExtra = kNptPartials - kStepPartials;

// Skin test of a system under box scaling.  Positions and build positions are scaled
// together, so x - x_build is the displacement that scaling does not explain.  A pair
// left out of the list at the build (|r| > rl) now has |r| >= mu_min rl - 2 max|x - x_build|,
// mu_min the smallest per-axis scale since the build; it stays outside the cutoff rc
// while every displacement is below (mu_min rl - rc) / 2.  Returns that bound squared,
// or -1 (rebuild now) when it is not positive.
__host__ __device__ __forceinline__ float npt_half_skin2(const SysDev &sd, bool with_pending)
{
    double mmin = 1e300;
    for (int a = 0; a < 3; ++a) {
        const double m = sd.npt.mu_cum[a] * (with_pending && sd.npt.pending ? sd.npt.mu[a] : 1.0);
        mmin = m < mmin ? m : mmin;
    }
    const double h = 0.5 * (mmin * sd.rl - sd.rc);
    return h > 0.0 ? (float)(h * h) : -1.0f;
}

// Conversions between fp32 and fp64 with integer instructions.  GB300 executes
// F2F conversions on its fp64 pipe (1/64 of the fp32 rate); the mixed path needs a few per
// atom, and integer shifts and adds cost nothing next to that.
//   f2d_int: exact for zero and normal floats; subnormal floats become a signed zero (the
//            values converted -- forces, per-atom sums, bond vectors -- are never subnormal
//            in magnitude that matters); inf/NaN become large finite doubles (non-finite
//            forces are flagged before conversion).
//   d2f_trunc: rounds toward zero (at most 1 float ulp); magnitudes below the float normal
//            range become a signed zero; the argument must stay below 3.4e38.
__device__ __forceinline__ double f2d_int(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned a = u & 0x7fffffffu, s = u & 0x80000000u;
    const bool nrm = a >= 0x00800000u;
    const unsigned hi = nrm ? (s | ((a >> 3) + 0x38000000u)) : s;   // exponent bias 127 -> 1023
    const unsigned lo = nrm ? (a << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float d2f_trunc(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned a = hi & 0x7fffffffu, s = hi & 0x80000000u;
    const unsigned f = a >= 0x38100000u ? (((a - 0x38000000u) << 3) | (lo >> 29)) : 0u;
    return __uint_as_float(s | f);
}
// x is finite (exponent field not all ones), tested on the integer pipe
__device__ __forceinline__ bool finite_bits(double x)
{
    return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}
__device__ __forceinline__ bool finite_bits(float x)
{
    return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u;
}
// x in the pair pass's type T, and back to fp64 (identities for T = double)
template <typename T> __device__ __forceinline__ T to_t(double x);
template <> __device__ __forceinline__ double to_t<double>(double x) { return x; }
template <> __device__ __forceinline__ float to_t<float>(double x) { return d2f_trunc(x); }
__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return f2d_int(x); }

// r_ij from positions and a list entry's image code (three fp64 subtractions, plus
// one addition per shifted axis).
__device__ __forceinline__ void bond_vector(const double *pos, int64_t N, int64_t i, int e, const Box &box,
                                            double xi, double yi, double zi, double &dx, double &dy,
                                            double &dz)
{
    const int j = list_atom(e);
    dx = pos[j] - xi;
    dy = pos[N + j] - yi;
    dz = pos[2 * N + j] - zi;
    const int code = list_code(e);
    if (code != kNoShift) {
        const int sx = code % 3 - 1, sy = (code / 3) % 3 - 1, sz = code / 9 - 1;
        if (sx) dx += sx > 0 ? box.L[0] : -box.L[0];
        if (sy) dy += sy > 0 ? box.L[1] : -box.L[1];
        if (sz) dz += sz > 0 ? box.L[2] : -box.L[2];
    }
    (void)i;
}

}  // namespace mdk
