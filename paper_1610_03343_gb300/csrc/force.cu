// force.cu -- the force hot path in the paper's explicit pairwise-force form.
//
// Pass A, "pair pass" (one thread per atom i; Algorithm 3 and the dU_i/dr_ij part of
// Algorithm 2 fused): for every list neighbour j the fp64 bond r_ij (the list entry
// carries the periodic image, so this is three subtractions); the in-cutoff bonds are
// staged in shared memory (SoA across the block's threads), then
//   Tersoff: zeta_ij (Eq. 4) for every bond, b_ij and db/dzeta (Eq. 3), U_i (Eq. 2) and
//            dU_i/dr_ij, whose chain rule runs through b_ij and every b_ik (k != j);
//   SW:      the two-body and vertex three-body sums in one pass (no precompute, as
//            the paper notes for SW in Sec. 2.3).
// Every bond order is computed once per bond: the paper's force kernel recomputes
// dU_j/dr_ji inside atom i's thread (Algorithm 2, the loop over j's neighbours); here
// each atom writes its own dU_i/dr_ij once and the gather reads the partner's value.
//
// Pass B, "gather" (one thread per atom i, Eqs. 28-30): F_i = sum_j (d_ij - d_ji),
// W_i = -1/2 sum_j r_ij (x) (d_ij - d_ji), J_i = (sum_j r_ij (x) d_ji) . v_i, where
// d_ji is found through the reverse-slot index.  Each atom's sums live in one thread:
// no atomics, fixed summation order, bitwise-reproducible results.  The gather also
// applies the second velocity-Verlet half-kick and writes per-block fp64 partial sums
// of U, K, J (and W for a force evaluation); a small kernel adds them in fixed order.
//
// Precision: T = double (fp64 path) or float (mixed path: per-pair arithmetic and
// per-atom sums in fp32; bond vectors from fp64 positions; velocities, positions and
// the block / system totals in fp64).
#include <algorithm>
#include <mutex>

#include "fastmath.cuh"
#include "md_plan.cuh"

namespace mdk {

#if !defined(MD_FORCE_PART) || MD_FORCE_PART == 0
const char *kKernelClassNames[KC_COUNT] = {"kick_drift", "rebuild", "pair", "gather", "reduce"};
#endif

namespace {

constexpr int kPoolChunk = 128;   // pools place systems on 128-atom chunk boundaries

// ---------------------------------------------------------------- precision
template <typename T> struct M;
// texp_, tlog_, tlog1p_: the Tersoff pair pass's exponentials and logarithms, whose
// arguments stay inside the table-driven routines' domain (fastmath.cuh); tlog1p_ needs
// only absolute accuracy (it enters b = exp(-log(1 + x)/(2n))).
template <> struct M<double> {
    static __device__ __forceinline__ double rsqrt_(double x) { return rsqrt_ff(x); }
    static __device__ __forceinline__ double exp_(double x) { return exp(x); }
    static __device__ __forceinline__ double log_(double x) { return log(x); }
    static __device__ __forceinline__ double log1p_(double x) { return log1p(x); }
    static __device__ __forceinline__ double texp_(double x) { return exp_ff(x); }
    static __device__ __forceinline__ double tlog_(double x) { return log_ff(x); }
    static __device__ __forceinline__ double tlog1p_(double x) { return log_ff(1.0 + x); }
    // SW: exp(sigma/(r - a sigma)) and exp(gamma sigma/(r - a sigma)) go to -infinity at the
    // cutoff; below -700 the factor is < 1e-304 and is taken as e^-700
    static __device__ __forceinline__ double sexp_(double x) { return exp_ff(clamp_neg700(x)); }
    static __device__ __forceinline__ double rcp_(double x) { return rcp_ff(x); }
    static __device__ __forceinline__ void sincos_(double x, double *s, double *c) { sincos(x, s, c); }
    static __device__ __forceinline__ double pow_(double x, double y) { return pow(x, y); }
};
template <> struct M<float> {
    static __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float exp_(float x) { return expf(x); }
    static __device__ __forceinline__ float log_(float x) { return logf(x); }
    static __device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
    static __device__ __forceinline__ float texp_(float x) { return expf(x); }
    static __device__ __forceinline__ float tlog_(float x) { return logf(x); }
    static __device__ __forceinline__ float tlog1p_(float x) { return log1pf(x); }
    static __device__ __forceinline__ float sexp_(float x) { return expf(x); }
    static __device__ __forceinline__ float rcp_(float x) { return 1.0f / x; }
    static __device__ __forceinline__ void sincos_(float x, float *s, float *c) { sincosf(x, s, c); }
    static __device__ __forceinline__ float pow_(float x, float y) { return powf(x, y); }
};

template <typename T>
__device__ __forceinline__ T ipow(T x, int n)
{
    T r = T(1);
    for (int k = 0; k < n; ++k) r *= x;
    return r;
}

// Shared-memory staging of atom i's in-cutoff neighbours: field f of neighbour k of
// thread t lives at s[(f CAP + k) BLOCK + t] (consecutive threads, consecutive words).
template <typename T, int CAP, int BLOCK>
struct Stage {
    T *s;
    int t;
    __device__ __forceinline__ T &operator()(int f, int k) const { return s[(f * CAP + k) * BLOCK + t]; }
    __device__ __forceinline__ void set(int f, int k, T v) const { s[(f * CAP + k) * BLOCK + t] = v; }
};

// Potential constants in the pair pass's arithmetic type (no conversions in the loops).
template <typename T>
struct TersoffC {
    // hA = A/2, hB = B/2: the pair pass forms f_R/2 and f_A/2, which is what U_i (Eq. 2's
    // 1/2 f_C (f_R - b f_A)), the radial term and P take (exact: halving is a scaling by 2^-1)
    T hA, hB, lam, mu, n, c2, d2, c2d2, h, R, pi_SR, n_ln_beta, inv2n;   // n_ln_beta = n log(beta)
    T beta;
    T rc2;   // S^2
    int beta_zero;
};
template <typename T>
TersoffC<T> tersoff_const(const TersoffP &p)
{
    TersoffC<T> c;
    c.hA = T(0.5 * p.A); c.hB = T(0.5 * p.B); c.lam = T(p.lam); c.mu = T(p.mu); c.n = T(p.n);
    c.c2 = T(p.c2); c.d2 = T(p.d2); c.c2d2 = T(p.c2d2); c.h = T(p.h); c.R = T(p.R);
    c.pi_SR = T(p.pi_SR); c.n_ln_beta = T(p.n * p.ln_beta); c.inv2n = T(p.inv2n); c.beta = T(p.beta);
    c.rc2 = T(p.S * p.S);
    c.beta_zero = p.beta_zero;
    return c;
}
template <typename T>
struct SWC {
    T Aeps, B, p, q, sig, rc, gamsig, lameps;
    T rc2;   // (a sigma)^2
    int p_int, q_int;
};
template <typename T>
SWC<T> sw_const(const SWP &p)
{
    SWC<T> c;
    c.Aeps = T(p.Aeps); c.B = T(p.B); c.p = T(p.p); c.q = T(p.q); c.sig = T(p.sig);
    c.rc = T(p.rc); c.gamsig = T(p.gamsig); c.lameps = T(p.lameps);
    c.rc2 = T(p.rc * p.rc);
    c.p_int = p.p_int; c.q_int = p.q_int;
    return c;
}

// |r|^2 of a bond vector in the pass's type.  Every pass that decides whether a bond is
// inside the cutoff uses this one expression, so that atom i's pass and atom j's pass
// (which may be different kernels) reach the same decision from negated vectors.
template <typename T>
__device__ __forceinline__ T bond_r2(T x, T y, T z)
{
    return fma(z, z, fma(y, y, x * x));
}

// fp64 bond vector r_j - r_i of list entry e (image shift from the entry), in type T
template <typename T>
__device__ __forceinline__ void bond_vector_t(const double *pos, int64_t N, int64_t i, int e, double xi, double yi,
                                              double zi, const Box &box, T &tx, T &ty, T &tz)
{
    double dx, dy, dz;
    bond_vector(pos, N, i, e, box, xi, yi, zi, dx, dy, dz);
    tx = to_t<T>(dx); ty = to_t<T>(dy); tz = to_t<T>(dz);
}

// A failure found by the pair pass for atom i: its system's entry in a pool (the rest of
// the pool carries on), the context's status words otherwise.
template <typename T>
__device__ __noinline__ void pair_fail(const PairArgs<T> &a, int64_t i, int status)
{
    if (a.batch) fail_system(a.sys[a.sys_of[i]], status);
    else if (status == MD_ERR_NAN) a.flags->nonfinite = 1;
    else a.flags->active_overflow = 1;
}

// ------------------------------------------------------- neighbour staging
// For each list slot, the fp64 bond r_ij (image shift from the entry); keeps the slots
// with |r_ij|^2 < rc^2, writes their bond vectors (compact row k) to global memory and
// stages (x, y, z, r^2) in the shared fields fx, fy, fz, fr2.  Without a prefilter, slots
// are fetched four at a time so that their index and position loads are in flight together;
// with one (SW), an fp32 pass first marks the slots that may be bonds and the fp64 work
// then runs over those only.  Returns the
// in-cutoff count (and mask), or -1 when the count exceeds CAP in the small-capacity
// pass: the atom is then appended to the deferred list and left to the full pass.
// The cutoff decision is symmetric in i and j: the two fp64 differences are exact
// negatives of each other, and so are their conversions.
// MULTI (multi-element Tersoff): the cutoff is that of the element pair, row[t_j].rc2
// (row: atom i's row of the pair table; rc2, the prefilter's radius, its largest entry),
// and the neighbour's element is staged in field ftype.
template <typename T, int CAP, int BLOCK, bool FULL_CAP, bool PREFILTER, bool MULTI = false, typename ST>
__device__ __forceinline__ int collect_bonds(const PairArgs<T> &a, int64_t i, const Box &box, T rc2,
                                             uint32_t &mask, ST &S, int fx, int fy, int fz, int fr2,
                                             const TersoffC<T> *row = nullptr, int ftype = 0)
{
    const int64_t N = a.N;
    const int S_ = a.stride;
    const double xi = a.pos[i], yi = a.pos[N + i], zi = a.pos[2 * N + i];
    // a non-finite position has no bond inside the cutoff (its distances are NaN): report
    // it, as its force would otherwise be a silent zero
    if (!(finite_bits(xi) && finite_bits(yi) && finite_bits(zi))) pair_fail(a, i, MD_ERR_NAN);
    float fxi = 0.f, fyi = 0.f, fzi = 0.f, lim2 = 0.f, fL0 = 0.f, fL1 = 0.f, fL2 = 0.f;
    if (PREFILTER) {
        fxi = a.posf[i]; fyi = a.posf[N + i]; fzi = a.posf[2 * N + i];
        // box edges in fp32 once per atom, with integer instructions (within the margin)
        fL0 = d2f_trunc(box.L[0]); fL1 = d2f_trunc(box.L[1]); fL2 = d2f_trunc(box.L[2]);
        // margin: the box-based bound plus the rounding of this atom's own coordinates,
        // which on an open axis may lie far outside the box
        const float mag = fmaxf(fabsf(fxi), fmaxf(fabsf(fyi), fabsf(fzi)));
        const float lim = sqrtf((float)rc2) + a.margin + 32.f * mag * 1.1920929e-7f;
        lim2 = lim * lim;
    }
    const int nn = a.nn[i];
    int na = 0;
    mask = 0u;
    // one bond: the fp64 vector r_ij of list slot m (entry e, neighbour position p), the exact
    // cutoff test and the staging
    auto bond = [&](int m, int e, double px, double py, double pz) {
        double dx = px - xi, dy = py - yi, dz = pz - zi;
        const int code = list_code(e);
        if (code != kNoShift) {
            const int sx = code % 3 - 1, sy = (code / 3) % 3 - 1, sz = code / 9 - 1;
            if (sx) dx += sx > 0 ? box.L[0] : -box.L[0];
            if (sy) dy += sy > 0 ? box.L[1] : -box.L[1];
            if (sz) dz += sz > 0 ? box.L[2] : -box.L[2];
        }
        const T tx = to_t<T>(dx), ty = to_t<T>(dy), tz = to_t<T>(dz);
        const T r2 = bond_r2(tx, ty, tz);
        int tj = 0;
        T cut2 = rc2;
        if (MULTI) {
            tj = a.type[list_atom(e)];
            cut2 = row[tj].rc2;
        }
        if (lt_nonneg(r2, cut2)) {
            if (na < CAP) {
                S.set(fx, na, tx); S.set(fy, na, ty); S.set(fz, na, tz); S.set(fr2, na, r2);
                if (MULTI) S.set(ftype, na, T(tj));
                a.r[(int64_t)(0 * S_ + na) * N + i] = bond_out(tx);
                a.r[(int64_t)(1 * S_ + na) * N + i] = bond_out(ty);
                a.r[(int64_t)(2 * S_ + na) * N + i] = bond_out(tz);
            }
            mask |= 1u << m;
            ++na;
        }
    };
    if (PREFILTER) {
        // pass 1, fp32 and integer pipes: the list slots whose fp32 distance (from the step's
        // fp32 positions) is within the cutoff plus the fp32 rounding margin (exact: the fp64
        // test would reject every other slot; symmetric: fp32 negation is exact)
        uint32_t cand = 0u;
        for (int m0 = 0; m0 < nn; m0 += 4) {
            int e[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) e[q] = (m0 + q < nn) ? a.nl[(int64_t)(m0 + q) * N + i] : 0;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (m0 + q >= nn) break;
                const int j = list_atom(e[q]);
                float dx = a.posf[j] - fxi, dy = a.posf[N + j] - fyi, dz = a.posf[2 * N + j] - fzi;
                const int code = list_code(e[q]);
                if (code != kNoShift) {
                    const int sx = code % 3 - 1, sy = (code / 3) % 3 - 1, sz = code / 9 - 1;
                    dx = fmaf((float)sx, fL0, dx);
                    dy = fmaf((float)sy, fL1, dy);
                    dz = fmaf((float)sz, fL2, dz);
                }
                if (dx * dx + dy * dy + dz * dz < lim2) cand |= 1u << (m0 + q);
            }
        }
        // pass 2, fp64: only the candidates, in list order, so that every lane of a warp does
        // fp64 work for each iteration it takes (the list holds about three times as many
        // slots as bonds: SW silicon's second shell lies inside the list radius)
        while (cand != 0u) {
            const int m = __ffs(cand) - 1;
            cand &= cand - 1u;
            const int e = a.nl[(int64_t)m * N + i];
            const int j = list_atom(e);
            bond(m, e, a.pos[j], a.pos[N + j], a.pos[2 * N + j]);
        }
    } else {
        // slots fetched four at a time, so that their index and position loads are in flight
        // together
        for (int m0 = 0; m0 < nn; m0 += 4) {
            int e[4];
            double px[4], py[4], pz[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                e[q] = (m0 + q < nn) ? a.nl[(int64_t)(m0 + q) * N + i] : 0;
                const int j = list_atom(e[q]);
                if (m0 + q < nn) {
                    px[q] = a.pos[j];
                    py[q] = a.pos[N + j];
                    pz[q] = a.pos[2 * N + j];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (m0 + q >= nn) break;
                bond(m0 + q, e[q], px[q], py[q], pz[q]);
            }
        }
    }
    if (na > CAP) {
        if (!FULL_CAP) {
            a.ovf_list[atomicAdd(a.ovf_count, 1)] = (int)i;
            return -1;
        }
        pair_fail(a, i, MD_ERR_NEIGH_OVERFLOW);
        na = CAP;
    }
    return na;
}

// ------------------------------------------------------------------ Tersoff
enum { TF_UX, TF_UY, TF_UZ, TF_IR, TF_FC, TF_DFC, TF_FR, TF_Z, TF_FA, TF_DX, TF_DY, TF_DZ, TF_NF };

// g(cos) of Eq. 5 written as 1 + (c^2/d^2) (h-cos)^2 / (d^2 + (h-cos)^2): the same
// function as printed, without the cancellation of c^2/d^2 - c^2/(d^2+(h-cos)^2)
// (about 4e7 - 4e7 for silicon), so that it stays accurate in fp32.  inv = 1/den is
// kept so the derivative loop can reuse it; dg = dg/dcos.
template <typename T>
__device__ __forceinline__ T tersoff_inv_den(const TersoffC<T> &p, T cs)
{
    const T hc = p.h - cs;
    return M<T>::rcp_(p.d2 + hc * hc);
}
template <typename T>
__device__ __forceinline__ void tersoff_g(const TersoffC<T> &p, T cs, T inv, T &g, T &dg)
{
    const T hc = p.h - cs;
    const T t = hc * inv;                                // (h - cos)/den
    g = fma(p.c2d2 * hc, t, T(1));
    dg = T(-2) * p.c2 * t * inv;
}

// f_C' is +0 exactly for a bond below R (f_C = 1 there) and <= -0 inside the switching
// region: the bit pattern tells them apart on the integer pipe
template <typename T>
__device__ __forceinline__ bool no_switch(T dfc)
{
    if constexpr (sizeof(T) == 8) return __double_as_longlong(dfc) == 0;
    else return __float_as_int(dfc) == 0;
}

// b = (1 + (beta zeta)^n)^(-1/(2n)) (Eq. 3) and db/dzeta = -1/2 b x / (zeta (1 + x)),
// x = (beta zeta)^n.  b = 1, db = 0 at zeta = 0 (every dzeta/dr it multiplies is 0).
template <typename T>
__device__ __forceinline__ void tersoff_b(const TersoffC<T> &p, T zeta, T &b, T &db)
{
    if (!positive_nonneg(zeta) || p.beta_zero) {
        b = T(1);
        db = T(0);
        return;
    }
    const T x = M<T>::texp_(fma(p.n, M<T>::tlog_(zeta), p.n_ln_beta));   // (beta zeta)^n
    b = M<T>::texp_(-p.inv2n * M<T>::tlog1p_(x));
    db = T(-0.5) * b * x * M<T>::rcp_(zeta * (T(1) + x));
}

// fp64 pass: b as above and P = -1/2 f_C f_A db/dzeta = cfa b x / (zeta (1 + x))
// (cfa = f_C f_A / 4).  zeta arrives as a float pair from the float-pair zeta loop (relative
// error about 2^-47, which alone puts a relative error of x/(2(1 + x)) 2^-47 < 2^-50 on b),
// so x = (beta zeta)^n = exp(n log(beta zeta)) and log(1 + x) are formed as float pairs on
// the fp32 pipe (exp_f2, log_f2: each adds an error of the same order to b); the last step,
// b = exp(-log(1 + x)/(2n)), takes the fp64-assisted exp, since b multiplies f_A in the
// radial term 1/2 ((f_C f_R)' - b (f_C f_A)'), whose two parts nearly cancel at equilibrium.
// P only scales the angular terms, which the float-pair angular loop forms to 2^-47 anyway.
// beta zeta below the float normal range (zeta < 1e-31: a bond within about 1e-18 A of the
// cutoff) counts as zeta = 0.
__device__ __forceinline__ double tersoff_b_ff(const TersoffC<double> &p, F2 zf, F2 cfa, F2 &P)
{
    const F2 bz = ff_mul(split_d(p.beta), zf);
    if (p.beta_zero || !(bz.h >= 1.17549435e-38f)) {
        P = F2{0.f, 0.f};
        return 1.0;
    }
    const F2 x = exp_f2(ff_mul(split_d(p.n), log_f2(bz)));   // (beta zeta)^n
    const F2 opx = ff_add(F2{1.f, 0.f}, x);
    const double b = exp_ff(ff_to_d(ff_mul(split_d(-p.inv2n), log_f2(opx))));
    P = ff_mul(ff_mul(ff_mul(cfa, split_d(b)), x), ff_rcp(ff_mul(zf, opx)));
    return b;
}

// index of the unordered bond pair (j, k), j < k
__device__ __forceinline__ int tri(int j, int k) { return k * (k - 1) / 2 + j; }

// Shared-memory words per bond and per unordered bond pair.  fp32 pass: the twelve bond
// fields (the element code of MULTI in TF_DX until the angular loop), and per pair
// 1/(d^2 + (h - cos)^2) (it recomputes cos, g and g' in the angular loop: it is bound by
// instruction issue and occupancy).  fp64 pass: eight bond fields -- TF_FR holds r until the
// bond-order loop, which forms f_R and f_A itself, and its angular loop sums each bond's
// terms itself and scatters nothing, so it needs neither TF_FA nor TF_DX..TF_DZ -- plus the
// element code of MULTI in TF_FA, and per pair h - cos and g' as float pairs from the zeta
// loop (g is recomputed for the rare bonds in the switching region).
template <typename T, bool MULTI>
constexpr int kTersoffBondFields = sizeof(T) == 8 ? TF_FA + (MULTI ? 1 : 0) : TF_NF;
template <typename T>
constexpr int kTersoffTypeField = sizeof(T) == 8 ? TF_FA : TF_DX;
// The fp64 common-case staging of 3 or 4 bonds (single element) keeps no f_C and f_C'
// fields: an atom with a bond in the switching region R <= r < S goes to the full-capacity
// pass, like an atom with more bonds than the staging holds, and the common pass's bonds all
// have f_C = 1, f_C' = 0.  Its r (then the radial term) and zeta (then P) take the slots of
// f_C and f_C': six fields a bond -- 24 shared words a thread with 3 bonds (32 warps per SM
// at 256 threads), 36 with 4 (22 warps at 64 threads instead of 18).
// FC: the 4-bond staging that keeps f_C after all (a context switches to it where many atoms
// have bonds in the switching region, which the stagings without f_C would all defer).
template <typename T, int CAP, bool MULTI, bool FC = false>
constexpr bool kTersoffNoSwitch = sizeof(T) == 8 && CAP <= 4 && !MULTI && !FC;
template <bool NOSW>
constexpr int kTfFR = NOSW ? TF_FC : TF_FR;
template <bool NOSW>
constexpr int kTfZ = NOSW ? TF_DFC : TF_Z;
template <typename T, int CAP, bool MULTI = false, bool FC = false>
constexpr int tersoff_smem_fields()
{
    return (kTersoffNoSwitch<T, CAP, MULTI, FC> ? TF_FC + 2 : kTersoffBondFields<T, MULTI>) * CAP +
           (sizeof(T) == 8 ? 2 : 1) * (CAP * (CAP - 1) / 2);
}

// Constants of bond k of the atom: its element pair's (MULTI: the row entry of the element
// staged in field kTersoffTypeField), else the single set's.
template <bool MULTI, typename T>
__device__ __forceinline__ const TersoffC<T> &bond_const(const TersoffC<T> &p, const TersoffC<T> *row, T tcode)
{
    if constexpr (MULTI) return row[(int)tcode];
    else return p;
}

// The two bond-pair loops of the fp64 pass in float-pair arithmetic (fastmath.cuh): every
// result carries an absolute error of about 2^-47 of the magnitudes it is formed from -- the
// same order as rounding dU_i/dr_ij to a 47-bit mantissa.  The one exception is cos theta:
// g' is proportional to h - cos theta, which is small (0.07 in graphene, where cos = -1/2
// and h = -0.5706), so an absolute error e in cos is a relative error e/|h - cos| in g';
// cos theta and h - cos theta are therefore formed in fp64 from the fp64 unit vectors (four
// fp64 instructions per pair) and only then split.  The pair cache holds, per unordered
// bond pair q = tri(j, k), h - cos theta and dg/dcos in slots q and NP + q.
template <int CAP, int BLOCK, bool NOSW = false>
__device__ __forceinline__ void tersoff_zeta_ff(const TersoffC<double> &p, const Stage<double, CAP, BLOCK> &S,
                                                double *spair, int na)
{
    constexpr int NP = CAP * (CAP - 1) / 2;
    constexpr int ZF = kTfZ<NOSW>;
    double *pc = spair + threadIdx.x;
    const F2 d2 = split_d(p.d2), c2d2 = split_d(p.c2d2), m2c2 = split_d(-2.0 * p.c2);
    const F2 one{1.f, 0.f};
    // f_C as staged: the float pair of 1.0 is (1, 0)
    auto fc_of = [&](int k) -> F2 { return NOSW ? one : ff_unpack(S(TF_FC, k)); };
    for (int j = 0; j < na; ++j) {
        const double ujx = S(TF_UX, j), ujy = S(TF_UY, j), ujz = S(TF_UZ, j);
        const F2 fcj = fc_of(j);
        F2 zj = ff_unpack(S(ZF, j));
        for (int k = j + 1; k < na; ++k) {
            const double csd = ujx * S(TF_UX, k) + ujy * S(TF_UY, k) + ujz * S(TF_UZ, k);
            // g = 1 + (c^2/d^2) (h - cos)^2 / (d^2 + (h - cos)^2), g' = -2 c^2 (h - cos) / den^2
            const F2 hc = split_d(p.h - csd);
            const F2 inv = ff_rcp(ff_fma(hc, hc, d2));
            const F2 t = ff_mul(hc, inv);
            const F2 g = ff_fma(ff_mul(c2d2, hc), t, one);
            const F2 dg = ff_mul(ff_mul(m2c2, t), inv);
            const int q = tri(j, k);
            pc[q * BLOCK] = ff_pack(hc);
            pc[(NP + q) * BLOCK] = ff_pack(dg);
            zj = ff_fma(fc_of(k), g, zj);
            S(ZF, k) = ff_pack(ff_fma(fcj, g, ff_unpack(S(ZF, k))));
        }
        S(ZF, j) = ff_pack(zj);
    }
}

// The angular loop, each bond j on its own: A_j and V_j take the terms of every pair (j, k),
// k != j, so nothing is scattered into bond k's fields; the factor (P_j + P_k) g' of a pair
// is formed once from each side, from the same values, so both sides see the same number.
template <int CAP, int BLOCK, bool NOSW = false>
__device__ __forceinline__ void tersoff_angular_ff(const PairArgs<double> &a, const TersoffC<double> &p,
                                                   const Stage<double, CAP, BLOCK> &S, const double *spair,
                                                   int na, int64_t i)
{
    constexpr int NP = CAP * (CAP - 1) / 2;
    constexpr int ZF = kTfZ<NOSW>, FRF = kTfFR<NOSW>;
    const double *pc = spair + threadIdx.x;
    const F2 h = split_d(p.h);
    for (int j = 0; j < na; ++j) {
        const F2 irj = ff_unpack(S(TF_IR, j)), Pj = ff_unpack(S(ZF, j));
        const bool swj = NOSW || no_switch(S(TF_DFC, j));
        F2 Aj = ff_unpack(S(FRF, j));
        F2 vx{0.f, 0.f}, vy{0.f, 0.f}, vz{0.f, 0.f};
        for (int k = 0; k < na; ++k) {
            if (k == j) continue;
            const int q = k > j ? tri(j, k) : tri(k, j);
            const F2 hc = ff_unpack(pc[q * BLOCK]), dg = ff_unpack(pc[(NP + q) * BLOCK]);
            const F2 cs = ff_add(h, ff_neg(hc));
            const F2 Pk = ff_unpack(S(ZF, k));
            F2 qj;
            if (NOSW || (swj && no_switch(S(TF_DFC, k)))) {
                // both below R: f_C = 1, f_C' = 0
                qj = ff_mul(ff_mul(ff_add(Pj, Pk), dg), irj);
                Aj = ff_fma(ff_neg(qj), cs, Aj);
            } else {
                const F2 inv = ff_rcp(ff_fma(hc, hc, split_d(p.d2)));
                const F2 g = ff_fma(ff_mul(split_d(p.c2d2), hc), ff_mul(hc, inv), F2{1.f, 0.f});
                const F2 fcj = ff_unpack(S(TF_FC, j)), dfcj = ff_unpack(S(TF_DFC, j));
                const F2 fck = ff_unpack(S(TF_FC, k));
                qj = ff_mul(ff_mul(ff_fma(Pj, fck, ff_mul(Pk, fcj)), dg), irj);
                Aj = ff_add(Aj, ff_fma(ff_neg(qj), cs, ff_mul(ff_mul(Pk, dfcj), g)));
            }
            vx = ff_fma(qj, ff_unpack(S(TF_UX, k)), vx);
            vy = ff_fma(qj, ff_unpack(S(TF_UY, k)), vy);
            vz = ff_fma(qj, ff_unpack(S(TF_UZ, k)), vz);
        }
        const F2 ujx = ff_unpack(S(TF_UX, j)), ujy = ff_unpack(S(TF_UY, j)), ujz = ff_unpack(S(TF_UZ, j));
        a.d[(int64_t)j * a.N + i] = Vec4<double>{ff_pack(ff_fma(Aj, ujx, vx)), ff_pack(ff_fma(Aj, ujy, vy)),
                                                 ff_pack(ff_fma(Aj, ujz, vz)), 0.0};   // float pairs, as bond_out
    }
}

// Pair pass for one atom (Tersoff).  MULTI: p holds atom i's element constants (angular
// and bond-order) and row its pair-constant row; each bond's radial functions and cutoff
// take the pair's constants (chi folded into B).
template <typename T, int CAP, int BLOCK, bool FULL_CAP, bool MULTI = false, bool FC = false>
__device__ __forceinline__ void tersoff_atom(const PairArgs<T> &a, const TersoffC<T> &p, const Box &box, T *base,
                                             int64_t i, const TersoffC<T> *row = nullptr)
{
    const int64_t N = a.N;
    Stage<T, CAP, BLOCK> S{base, (int)threadIdx.x};
    constexpr bool NOSW = kTersoffNoSwitch<T, CAP, MULTI, FC>;
    static_assert(!(NOSW && FULL_CAP), "the full-capacity pass stages f_C");
    constexpr int FRF = kTfFR<NOSW>, ZF = kTfZ<NOSW>;
    // per unordered bond pair q: fp64, h - cos theta and dg/dcos from the zeta loop (float
    // pairs, two slots); fp32, 1/(d^2 + (h - cos)^2) (one slot)
    T *spair = base + (NOSW ? TF_FC + 2 : kTersoffBondFields<T, MULTI>) * CAP * BLOCK;
    auto PCS = [&](int q) -> T & { return spair[q * BLOCK + threadIdx.x]; };

    uint32_t mask;
    // fp64: the list slots outside the cutoff are dropped by an fp32 test first, so that only
    // bonds take the fp64 bond vector and |r|^2 (the fp64 pipe bounds this pass); MULTI tests
    // against the largest cutoff of atom i's row
    T rc2 = p.rc2;
    if constexpr (MULTI) {
#pragma unroll
        for (int t = 0; t < kMaxTypes; ++t) rc2 = row[t].rc2 > rc2 ? row[t].rc2 : rc2;
    }
    const int na = collect_bonds<T, CAP, BLOCK, FULL_CAP, sizeof(T) == 8, MULTI>(
        a, i, box, rc2, mask, S, TF_UX, TF_UY, TF_UZ, TF_IR, row, kTersoffTypeField<T>);
    if (na < 0) return;   // deferred to the full-capacity pass

    // fp64: after the radial loop f_C, and after the bond-order loop every value the angular
    // loop reads, are staged as float pairs (ff_pack); the two bond-pair loops then run on
    // the fp32 pipe but for cos theta (see tersoff_zeta_ff, tersoff_angular_ff)
    constexpr bool FF = sizeof(T) == 8;
    auto put = [&](int f, int k, T v) {
        if constexpr (FF) S(f, k) = ff_pack(split_d(v));
        else S(f, k) = v;
    };
    auto get = [&](int f, int k) -> T {
        if constexpr (FF) return ff_to_d(ff_unpack(S(f, k)));
        else return S(f, k);
    };

    // per-bond radial functions (the staged vectors become unit vectors, r^2 -> 1/r)
    for (int k = 0; k < na; ++k) {
        const TersoffC<T> &pk = bond_const<MULTI>(p, row, MULTI ? S(kTersoffTypeField<T>, k) : T(0));
        const T r2 = S(TF_IR, k);
        // the float-pair staging turns inf and NaN into finite values: a bond shorter than
        // 1e-15 A (coincident atoms, 1/r = +inf) is reported here instead of through F
        if constexpr (FF) {
            if (!(r2 >= T(1e-30))) pair_fail(a, i, MD_ERR_NAN);
        }
        const T ir = M<T>::rsqrt_(r2);
        const T r = r2 * ir;
        S(TF_UX, k) *= ir;
        S(TF_UY, k) *= ir;
        S(TF_UZ, k) *= ir;
        S(TF_IR, k) = ir;
        // f_C = 1/2 + 1/2 cos(x) = cos^2(x/2), f_C' = -(pi/(S-R)) sin(x/2) cos(x/2),
        // x = pi (r-R)/(S-R): the half-angle form has no cancellation as f_C -> 0 near S
        T fc = T(1), dfc = T(0);
        if (!lt_nonneg(r, pk.R)) {
            if constexpr (NOSW) {   // a bond in the switching region: the full-capacity pass
                a.ovf_list[atomicAdd(a.ovf_count, 1)] = (int)i;
                return;
            }
            T sn, cn;
            M<T>::sincos_(T(0.5) * pk.pi_SR * (r - pk.R), &sn, &cn);
            fc = cn * cn;
            dfc = -pk.pi_SR * sn * cn;
        }
        if constexpr (!NOSW) {
            put(TF_FC, k, fc);
            S(TF_DFC, k) = dfc;
        }
        if constexpr (FF) {
            S(FRF, k) = r;
        } else {
            S(TF_FR, k) = pk.hA * M<T>::texp_(-pk.lam * r);   // f_R / 2
            S(TF_FA, k) = pk.hB * M<T>::texp_(-pk.mu * r);    // f_A / 2
        }
        S(ZF, k) = T(0);   // also the float pair (0, 0)
    }
    // zeta_ij = sum_{k != j} f_C(r_ik) g(theta_ijk), each unordered pair once
    if constexpr (FF) {
        tersoff_zeta_ff<CAP, BLOCK, NOSW>(p, S, spair, na);
    } else {
        for (int j = 0; j < na; ++j) {
            const T ujx = S(TF_UX, j), ujy = S(TF_UY, j), ujz = S(TF_UZ, j), fcj = S(TF_FC, j);
            T zj = S(TF_Z, j);
            for (int k = j + 1; k < na; ++k) {
                const T cs = ujx * S(TF_UX, k) + ujy * S(TF_UY, k) + ujz * S(TF_UZ, k);
                const T inv = tersoff_inv_den(p, cs);
                T g, dg;
                tersoff_g(p, cs, inv, g, dg);
                PCS(tri(j, k)) = inv;
                zj += S(TF_FC, k) * g;
                S(TF_Z, k) += fcj * g;
            }
            S(TF_Z, j) = zj;
        }
    }
    // bond orders, U_i, radial part of dU_i/dr_ij; P_k = -1/2 f_C f_A b'_k kept in TF_Z.
    // dU_i/dr_ij is assembled as A_j u_j + V_j: the scalar A_j (radial part plus the
    // angular terms along u_j) in TF_FR, the vector V_j (angular terms along the other
    // bonds) in TF_DX..TF_DZ.
    T ui = T(0);
    for (int k = 0; k < na; ++k) {
        const TersoffC<T> &pk = bond_const<MULTI>(p, row, MULTI ? S(kTersoffTypeField<T>, k) : T(0));
        const T dfc = NOSW ? T(0) : S(TF_DFC, k);
        T fr, fa;   // f_R / 2, f_A / 2
        if constexpr (FF) {
            const T r = S(FRF, k);
            fr = pk.hA * M<T>::texp_(-pk.lam * r);
            fa = pk.hB * M<T>::texp_(-pk.mu * r);
        } else {
            fr = S(TF_FR, k);
            fa = S(TF_FA, k);
        }
        // f_C = 1, f_C' = 0 below R: the same arithmetic without the unit factors and zero terms
        const bool sw = !NOSW && !no_switch(dfc);
        T b;
        if constexpr (FF) {
            F2 cfa = split_d(fa);   // f_C f_A / 4
            cfa = F2{0.5f * cfa.h, 0.5f * cfa.l};
            if (sw) cfa = ff_mul(cfa, ff_unpack(S(TF_FC, k)));
            F2 P;
            b = tersoff_b_ff(p, ff_unpack(S(ZF, k)), cfa, P);
            S(ZF, k) = ff_pack(P);
        } else {
            T db;
            tersoff_b(p, S(TF_Z, k), b, db);
            S(TF_Z, k) = sw ? -(S(TF_FC, k) * fa * db) : -(fa * db);   // -1/2 f_C f_A b'
        }
        T radial;
        if (!sw) {
            ui += fr - b * fa;
            radial = -pk.lam * fr + b * (pk.mu * fa);
        } else {
            const T fc = get(TF_FC, k);
            ui += fc * (fr - b * fa);
            const T dR = dfc * fr - pk.lam * fc * fr;   // (f_C f_R)' / 2
            const T dA = dfc * fa - pk.mu * fc * fa;    // (f_C f_A)' / 2
            radial = dR - b * dA;
        }
        put(FRF, k, radial);
        if constexpr (FF) {
            S(TF_UX, k) = ff_pack(split_d(S(TF_UX, k)));
            S(TF_UY, k) = ff_pack(split_d(S(TF_UY, k)));
            S(TF_UZ, k) = ff_pack(split_d(S(TF_UZ, k)));
            S(TF_IR, k) = ff_pack(split_d(S(TF_IR, k)));
            if constexpr (!NOSW) S(TF_DFC, k) = ff_pack(split_d(dfc));   // +0 stays the all-zero pattern
        } else {
            S(TF_DX, k) = T(0);
            S(TF_DY, k) = T(0);
            S(TF_DZ, k) = T(0);
        }
    }
    // angular part: for each unordered pair (j,k), with dcos_j = (u_k - cos u_j)/r_ij,
    //   d_j += (P_j fc_k + P_k fc_j) g' dcos_j + P_k fc'_j g u_j   (and j <-> k),
    // i.e. V_j += q_j u_k and A_j += c_j - q_j cos, q_j = (P_j fc_k + P_k fc_j) g'/r_ij
    if constexpr (FF) {
        tersoff_angular_ff<CAP, BLOCK, NOSW>(a, p, S, spair, na, i);
    } else {
        for (int j = 0; j < na; ++j) {
            const T ujx = S(TF_UX, j), ujy = S(TF_UY, j), ujz = S(TF_UZ, j);
            const T irj = S(TF_IR, j), fcj = S(TF_FC, j), dfcj = S(TF_DFC, j), Pj = S(TF_Z, j);
            T Aj = S(TF_FR, j);
            T vjx = S(TF_DX, j), vjy = S(TF_DY, j), vjz = S(TF_DZ, j);
            for (int k = j + 1; k < na; ++k) {
                const T ukx = S(TF_UX, k), uky = S(TF_UY, k), ukz = S(TF_UZ, k);
                const T irk = S(TF_IR, k), fck = S(TF_FC, k), dfck = S(TF_DFC, k), Pk = S(TF_Z, k);
                const T cs = ujx * ukx + ujy * uky + ujz * ukz;
                T g, dg;
                tersoff_g(p, cs, PCS(tri(j, k)), g, dg);
                T qj, qk;
                if (no_switch(dfcj) && no_switch(dfck)) {
                    // both below R: f_C = 1, f_C' = 0
                    const T Q = (Pj + Pk) * dg;
                    qj = Q * irj; qk = Q * irk;
                    Aj = fma(-qj, cs, Aj);
                    S(TF_FR, k) = fma(-qk, cs, S(TF_FR, k));
                } else {
                    const T Q = (Pj * fck + Pk * fcj) * dg;
                    const T cj = Pk * dfcj * g, ck = Pj * dfck * g;
                    qj = Q * irj; qk = Q * irk;
                    Aj += cj - qj * cs;
                    S(TF_FR, k) += ck - qk * cs;
                }
                vjx = fma(qj, ukx, vjx);
                vjy = fma(qj, uky, vjy);
                vjz = fma(qj, ukz, vjz);
                S(TF_DX, k) = fma(qk, ujx, S(TF_DX, k));
                S(TF_DY, k) = fma(qk, ujy, S(TF_DY, k));
                S(TF_DZ, k) = fma(qk, ujz, S(TF_DZ, k));
            }
            a.d[(int64_t)j * N + i] = Vec4<T>{fma(Aj, ujx, vjx), fma(Aj, ujy, vjy), fma(Aj, ujz, vjz), T(0)};
        }
    }
    a.mask[i] = mask;
    a.u[i] = to_d(ui);
}

// ---------------------------------------------------------- Stillinger-Weber
enum { SW_UX, SW_UY, SW_UZ, SW_IR, SW_E, SW_DE, SW_DX, SW_DY, SW_DZ, SW_NF };

// Shared-memory words per bond: the fp32 pass stages u, 1/r, E, dE/dr and the dU/dr
// accumulators that the three-body loop scatters into (9); the fp64 pass's three-body loop
// sums each bond's terms itself, starting from the two-body part it left in the output row,
// so it stages the first six only (4 blocks of 128 resident instead of 3).
template <typename T, int CAP>
constexpr int sw_smem_fields() { return (sizeof(T) == 8 ? SW_DX : SW_NF) * CAP; }

// Per-bond SW terms from r^2 and the bond vector: the unit vector u, 1/r, E = exp(gamma
// sigma/(r - a sigma)) and dE/dr of the three-body factor, this bond's two-body share of U_i
// (half of phi2) and of dU_i/dr_ij (half of dphi2/dr along u).
template <typename T>
struct SWBond {
    T ux, uy, uz, ir, E, dE, u2, dx, dy, dz;
};
template <typename T>
__device__ __forceinline__ SWBond<T> sw_bond(const SWC<T> &p, T r2, T tx, T ty, T tz)
{
    SWBond<T> b;
    const T ir = M<T>::rsqrt_(r2);
    const T r = r2 * ir;
    b.ux = tx * ir; b.uy = ty * ir; b.uz = tz * ir; b.ir = ir;
    const T irc = M<T>::rcp_(r - p.rc);              // 1/(r - a sigma) < 0
    const T e2 = M<T>::sexp_(p.sig * irc);
    b.E = M<T>::sexp_(p.gamsig * irc);
    b.dE = -p.gamsig * irc * irc * b.E;
    // phi2 = A eps [B (sigma/r)^p - (sigma/r)^q] exp(sigma/(r - a sigma))
    const T sr = p.sig * ir;
    T sp, sq;
    if (p.p_int >= 0) sp = ipow(sr, p.p_int); else sp = M<T>::pow_(sr, p.p);
    if (p.q_int >= 0) sq = ipow(sr, p.q_int); else sq = M<T>::pow_(sr, p.q);
    const T poly = p.B * sp - sq;
    const T dpoly = (-p.p * p.B * sp + p.q * sq) * ir;
    b.u2 = T(0.5) * p.Aeps * poly * e2;
    const T dphi = p.Aeps * (dpoly * e2 - poly * p.sig * irc * irc * e2);
    b.dx = T(0.5) * dphi * b.ux;
    b.dy = T(0.5) * dphi * b.uy;
    b.dz = T(0.5) * dphi * b.uz;
    return b;
}

// fp64 pass, per-bond SW terms: phi2 and its derivative in fp64 (their two terms cancel at
// the equilibrium bond length), everything the float-pair three-body loop reads -- u, E and
// dE/dr -- and the two-body dU/dr = 1/2 phi2' u as float pairs.
struct SWBondFF {
    F2 ux, uy, uz, ir, E, dE, dx, dy, dz;
    double u2;
};
__device__ __forceinline__ SWBondFF sw_bond_ff(const SWC<double> &p, double r2, double tx, double ty, double tz)
{
    SWBondFF b;
    const double ir = M<double>::rsqrt_(r2);
    const double r = r2 * ir;
    b.ir = split_d(ir);
    b.ux = ff_mul(split_d(tx), b.ir);
    b.uy = ff_mul(split_d(ty), b.ir);
    b.uz = ff_mul(split_d(tz), b.ir);
    const double irc = M<double>::rcp_(r - p.rc);   // 1/(r - a sigma) < 0
    const double e2 = M<double>::sexp_(p.sig * irc);
    b.E = split_d(M<double>::sexp_(p.gamsig * irc));
    const F2 ircf = split_d(irc);
    b.dE = ff_mul(ff_mul(split_d(-p.gamsig), ff_mul(ircf, ircf)), b.E);
    // phi2 = A eps [B (sigma/r)^p - (sigma/r)^q] exp(sigma/(r - a sigma))
    const double sr = p.sig * ir;
    double sp, sq;
    if (p.p_int >= 0) sp = ipow(sr, p.p_int); else sp = M<double>::pow_(sr, p.p);
    if (p.q_int >= 0) sq = ipow(sr, p.q_int); else sq = M<double>::pow_(sr, p.q);
    const double poly = p.B * sp - sq;
    const double dpoly = (-p.p * p.B * sp + p.q * sq) * ir;
    b.u2 = 0.5 * p.Aeps * poly * e2;
    const double dphi = p.Aeps * (dpoly * e2 - poly * p.sig * irc * irc * e2);
    F2 h = split_d(dphi);
    h = F2{0.5f * h.h, 0.5f * h.l};
    b.dx = ff_mul(h, b.ux);
    b.dy = ff_mul(h, b.uy);
    b.dz = ff_mul(h, b.uz);
    return b;
}

// fp64 pass, three-body part in float-pair arithmetic: every term of phi3 and of its
// derivative carries the factor t = cos + 1/3 (which vanishes at the tetrahedral angle) or
// t^2, so an absolute error e in cos is an absolute error of about 2 lambda eps E E' e /r in
// dU_i/dr_ij -- no cancellation amplifies it -- while the two-body part, whose two terms
// cancel at the equilibrium bond length, stays fp64.  Each bond j sums the terms of its
// pairs (j, k), k != j, itself, onto the two-body part that the per-bond loop stored in its
// output row, so nothing is scattered into bond k's staging: per pair (j, k) the terms of
// phi3's derivative along r_ij are
//   2 lambda eps t E_j E_k dcos/dr_ij + lambda eps t^2 E_j' E_k u_j,
// with dcos/dr_ij = (u_k - cos u_j)/r_ij; phi3 itself is added once per unordered pair.
// dU_i/dr_ij is stored as float pairs (bond_out).
template <int CAP, int BLOCK>
__device__ __forceinline__ void sw_three_body_ff(const PairArgs<double> &a, const SWC<double> &p,
                                                 const Stage<double, CAP, BLOCK> &S, int na, int64_t i,
                                                 double &ui)
{
    const F2 third = split_d(1.0 / 3.0), lameps = split_d(p.lameps);
    F2 u3{0.f, 0.f};
    for (int j = 0; j < na; ++j) {
        const F2 ujx = ff_unpack(S(SW_UX, j)), ujy = ff_unpack(S(SW_UY, j)), ujz = ff_unpack(S(SW_UZ, j));
        const F2 irj = ff_unpack(S(SW_IR, j)), Ej = ff_unpack(S(SW_E, j)), dEj = ff_unpack(S(SW_DE, j));
        const Vec4<double> d2 = a.d[(int64_t)j * a.N + i];   // the two-body part
        F2 djx = ff_unpack(d2.x), djy = ff_unpack(d2.y), djz = ff_unpack(d2.z);
        for (int k = 0; k < na; ++k) {
            if (k == j) continue;
            const F2 ukx = ff_unpack(S(SW_UX, k)), uky = ff_unpack(S(SW_UY, k)), ukz = ff_unpack(S(SW_UZ, k));
            const F2 Ek = ff_unpack(S(SW_E, k));
            F2 cs = ff_mul(ujx, ukx);
            cs = ff_fma(ujy, uky, cs);
            cs = ff_fma(ujz, ukz, cs);
            const F2 t = ff_add(cs, third);
            const F2 EE = ff_mul(Ej, Ek);
            const F2 lt = ff_mul(lameps, t), lt2 = ff_mul(lt, t);
            if (k > j) u3 = ff_fma(lt2, EE, u3);
            F2 c1 = ff_mul(lt, EE);
            c1 = F2{2.f * c1.h, 2.f * c1.l};
            const F2 cj = ff_mul(ff_mul(lt2, dEj), Ek);
            const F2 qj = ff_mul(c1, irj);
            // d_j += qj (u_k - cos u_j) + cj u_j, written as qj u_k + (cj - qj cos) u_j
            const F2 aj = ff_fma(ff_neg(qj), cs, cj);
            djx = ff_fma(qj, ukx, ff_fma(aj, ujx, djx));
            djy = ff_fma(qj, uky, ff_fma(aj, ujy, djy));
            djz = ff_fma(qj, ukz, ff_fma(aj, ujz, djz));
        }
        a.d[(int64_t)j * a.N + i] = Vec4<double>{ff_pack(djx), ff_pack(djy), ff_pack(djz), 0.0};
    }
    ui += ff_to_d(u3);
}

// SW terms of atom i from its na bonds staged in shared-memory slot `slot` (by
// collect_bonds): two-body and vertex three-body terms, dU_i/dr_ij per bond, U_i.
template <typename T, int CAP, int BLOCK>
__device__ __forceinline__ void sw_terms(const PairArgs<T> &a, const SWC<T> &p, T *base, int64_t i, int slot, int na,
                                         uint32_t mask)
{
    const int64_t N = a.N;
    Stage<T, CAP, BLOCK> S{base, slot};
    T ui = T(0);
    for (int k = 0; k < na; ++k) {
        if constexpr (sizeof(T) == 8) {
            // the float-pair staging turns inf and NaN into finite values: a bond shorter
            // than 1e-15 A (coincident atoms, 1/r = +inf) is reported here instead of through F
            if (!(S(SW_IR, k) >= T(1e-30))) pair_fail(a, i, MD_ERR_NAN);
        }
        if constexpr (sizeof(T) == 8) {
            const SWBondFF b = sw_bond_ff(p, S(SW_IR, k), S(SW_UX, k), S(SW_UY, k), S(SW_UZ, k));
            S(SW_UX, k) = ff_pack(b.ux); S(SW_UY, k) = ff_pack(b.uy); S(SW_UZ, k) = ff_pack(b.uz);
            S(SW_IR, k) = ff_pack(b.ir);
            S(SW_E, k) = ff_pack(b.E);
            S(SW_DE, k) = ff_pack(b.dE);
            ui += b.u2;
            // the two-body part, in the output row until the three-body loop adds to it
            a.d[(int64_t)k * N + i] = Vec4<double>{ff_pack(b.dx), ff_pack(b.dy), ff_pack(b.dz), 0.0};
        } else {
            const SWBond<T> b = sw_bond(p, S(SW_IR, k), S(SW_UX, k), S(SW_UY, k), S(SW_UZ, k));
            S(SW_UX, k) = b.ux; S(SW_UY, k) = b.uy; S(SW_UZ, k) = b.uz; S(SW_IR, k) = b.ir;
            S(SW_E, k) = b.E;
            S(SW_DE, k) = b.dE;
            ui += b.u2;
            S(SW_DX, k) = b.dx;
            S(SW_DY, k) = b.dy;
            S(SW_DZ, k) = b.dz;
        }
    }
    if constexpr (sizeof(T) == 8) {
        sw_three_body_ff<CAP, BLOCK>(a, p, S, na, i, ui);
    } else {
        // phi3 = lambda eps (cos + 1/3)^2 E(r_ij) E(r_ik), vertex i, each unordered pair once
        for (int j = 0; j < na; ++j) {
            const T ujx = S(SW_UX, j), ujy = S(SW_UY, j), ujz = S(SW_UZ, j);
            const T irj = S(SW_IR, j), Ej = S(SW_E, j), dEj = S(SW_DE, j);
            T djx = S(SW_DX, j), djy = S(SW_DY, j), djz = S(SW_DZ, j);
            for (int k = j + 1; k < na; ++k) {
                const T ukx = S(SW_UX, k), uky = S(SW_UY, k), ukz = S(SW_UZ, k);
                const T irk = S(SW_IR, k), Ek = S(SW_E, k), dEk = S(SW_DE, k);
                const T cs = ujx * ukx + ujy * uky + ujz * ukz;
                const T t = cs + T(1.0 / 3.0);
                const T EE = Ej * Ek;
                ui += p.lameps * t * t * EE;
                const T c1 = T(2) * p.lameps * t * EE;
                const T cj = p.lameps * t * t * dEj * Ek, ck = p.lameps * t * t * Ej * dEk;
                const T qj = c1 * irj, qk = c1 * irk;
                // d_j += qj (u_k - cos u_j) + cj u_j, written as qj u_k + (cj - qj cos) u_j
                const T aj = fma(-qj, cs, cj), ak = fma(-qk, cs, ck);
                djx = fma(qj, ukx, fma(aj, ujx, djx));
                djy = fma(qj, uky, fma(aj, ujy, djy));
                djz = fma(qj, ukz, fma(aj, ujz, djz));
                S(SW_DX, k) = fma(qk, ujx, fma(ak, ukx, S(SW_DX, k)));
                S(SW_DY, k) = fma(qk, ujy, fma(ak, uky, S(SW_DY, k)));
                S(SW_DZ, k) = fma(qk, ujz, fma(ak, ukz, S(SW_DZ, k)));
            }
            a.d[(int64_t)j * N + i] = Vec4<T>{djx, djy, djz, T(0)};
        }
    }
    a.mask[i] = mask;
    a.u[i] = to_d(ui);
}

template <typename T, int CAP, int BLOCK, bool FULL_CAP>
__device__ __forceinline__ void sw_atom(const PairArgs<T> &a, const SWC<T> &p, const Box &box, T *base, int64_t i)
{
    Stage<T, CAP, BLOCK> S{base, (int)threadIdx.x};
    uint32_t mask;
    const int na = collect_bonds<T, CAP, BLOCK, FULL_CAP, true>(a, i, box, p.rc2, mask, S, SW_UX, SW_UY, SW_UZ, SW_IR);
    if (na < 0) return;   // deferred to the full-capacity pass
    sw_terms<T, CAP, BLOCK>(a, p, base, i, (int)threadIdx.x, na, mask);
}

// Position of this thread's key among the block's keys (0 <= key < NK) in the stable
// order by key: the number of threads with a smaller key plus those with the same key
// and a lower thread index.  Deterministic; every thread of the block must call it.
template <int BLOCK, int NK>
__device__ __forceinline__ int block_rank(int key)
{
    constexpr int NW = BLOCK / 32;
    __shared__ int cnt[NW][NK];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int below = 0;
#pragma unroll
    for (int v = 0; v < NK; ++v) {
        const unsigned b = __ballot_sync(0xffffffffu, key == v);
        if (lane == 0) cnt[w][v] = __popc(b);
        if (key == v) below = __popc(b & ((1u << lane) - 1u));
    }
    __syncthreads();
    // the bucket's start, then the same key in lower warps
    int r = below;
    for (int v = 0; v < key; ++v)
#pragma unroll
        for (int q = 0; q < NW; ++q) r += cnt[q][v];
    for (int q = 0; q < w; ++q) r += cnt[q][key];
    return r;
}

// Single systems, common case (SW): the block's atoms are processed in the order of their
// bond count.  Each thread stages its own atom's bonds; the block then ranks the atoms by
// that count and thread t takes the atom of rank t, so the atoms of one warp have (nearly)
// the same number of bonds and bond pairs and the warp's loops do not wait for its
// heaviest atom (at room temperature SW silicon's atoms have 4 to 8 bonds, since its second
// shell lies just outside the cutoff).  Each atom's arithmetic is the same whichever
// thread runs it: results do not depend on the order.
template <typename T, int CAP, int BLOCK>
__device__ __forceinline__ void sw_block_sorted(const PairArgs<T> &a, const SWC<T> &p, const Box &box, T *base)
{
    __shared__ short perm[BLOCK];
    __shared__ signed char nas[BLOCK];
    __shared__ uint32_t masks[BLOCK];
    const int t = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * BLOCK;
    int na = -1;
    uint32_t mask = 0u;
    if (i0 + t < a.N) {
        Stage<T, CAP, BLOCK> S{base, t};
        na = collect_bonds<T, CAP, BLOCK, false, true>(a, i0 + t, box, p.rc2, mask, S, SW_UX, SW_UY, SW_UZ, SW_IR);
    }
    // deferred atoms and the tail past N go last and do nothing here
    const int r = block_rank<BLOCK, CAP + 2>(na < 0 ? CAP + 1 : na);
    perm[r] = (short)t;
    nas[t] = (signed char)na;
    masks[t] = mask;
    __syncthreads();
    const int slot = perm[t];
    const int n_s = nas[slot];
    if (n_s >= 0) sw_terms<T, CAP, BLOCK>(a, p, base, i0 + slot, slot, n_s, masks[slot]);
}

// Full-capacity pass for one deferred atom (SW), one warp per atom: lane m tests list slot m
// (lists hold at most 32), the in-cutoff slots are numbered in list order by a ballot, and
// lane k then owns bond k: its per-bond terms, and dU_i/dr_ik from the ordered pairs (k, m),
// m != k (the k side of each vertex three-body term; the m side is lane m's).  U_i is the
// warp's sum in a fixed order.  sh: this warp's staging of u and E, 4 x FULL values.
template <typename T, int FULL>
__device__ __forceinline__ void sw_atom_warp(const PairArgs<T> &a, const SWC<T> &p, const Box &box, T (*sh)[FULL],
                                             int64_t i, int lane)
{
    const int64_t N = a.N;
    const int S_ = a.stride;
    const int nn = a.nn[i];
    T tx = T(0), ty = T(0), tz = T(0), r2 = T(0);
    bool in = false;
    if (lane < nn) {
        bond_vector_t<T>(a.pos, N, i, a.nl[(int64_t)lane * N + i], a.pos[i], a.pos[N + i], a.pos[2 * N + i], box,
                         tx, ty, tz);
        r2 = bond_r2(tx, ty, tz);
        in = lt_nonneg(r2, p.rc2);
    }
    const uint32_t mask = __ballot_sync(0xffffffffu, in);
    const int k = __popc(mask & ((1u << lane) - 1u));
    int na = __popc(mask);
    if (na > FULL) {
        if (lane == 0) pair_fail(a, i, MD_ERR_NEIGH_OVERFLOW);
        na = FULL;
    }
    const bool mine = in && k < FULL;
    T ui = T(0), dx = T(0), dy = T(0), dz = T(0);
    SWBond<T> b{};
    if (mine) {
        a.r[(int64_t)(0 * S_ + k) * N + i] = bond_out(tx);
        a.r[(int64_t)(1 * S_ + k) * N + i] = bond_out(ty);
        a.r[(int64_t)(2 * S_ + k) * N + i] = bond_out(tz);
        b = sw_bond(p, r2, tx, ty, tz);
        sh[0][k] = b.ux; sh[1][k] = b.uy; sh[2][k] = b.uz; sh[3][k] = b.E;
        ui = b.u2;
        dx = b.dx; dy = b.dy; dz = b.dz;
    }
    __syncwarp();
    if (mine) {
        // phi3 = lambda eps (cos + 1/3)^2 E(r_ik) E(r_im); its energy is counted by the
        // lower of the two bonds
        for (int m = 0; m < na; ++m) {
            if (m == k) continue;
            const T umx = sh[0][m], umy = sh[1][m], umz = sh[2][m], Em = sh[3][m];
            const T cs = b.ux * umx + b.uy * umy + b.uz * umz;
            const T t = cs + T(1.0 / 3.0);
            const T EE = b.E * Em;
            if (m > k) ui += p.lameps * t * t * EE;
            const T q = T(2) * p.lameps * t * EE * b.ir;
            const T c = p.lameps * t * t * b.dE * Em;
            const T ac = fma(-q, cs, c);   // q (u_m - cos u_k) + c u_k = q u_m + (c - q cos) u_k
            dx = fma(q, umx, fma(ac, b.ux, dx));
            dy = fma(q, umy, fma(ac, b.uy, dy));
            dz = fma(q, umz, fma(ac, b.uz, dz));
        }
        if (sizeof(T) == 8 && !(finite_bits(dx) && finite_bits(dy) && finite_bits(dz))) pair_fail(a, i, MD_ERR_NAN);
        a.d[(int64_t)k * N + i] = Vec4<T>{bond_out(dx), bond_out(dy), bond_out(dz), T(0)};
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ui += __shfl_xor_sync(0xffffffffu, ui, o);
    if (lane == 0) {
        a.mask[i] = mask;
        a.u[i] = to_d(ui);
    }
    __syncwarp();   // the staging is reused by the warp's next atom
}

template <typename T>
struct TersoffSets {
    TersoffC<T> s[kMaxSets];
};
template <typename T>
struct SWSets {
    SWC<T> s[kMaxSets];
};

// Kernels: the small-capacity pass (one thread per atom, CAP = 4) and the full-capacity
// pass over the deferred atoms (grid-stride over the deferred list).  Pools (BATCH):
// each atom uses its system's box and parameter set; atoms of stopped systems are
// skipped.
template <typename T, int CAP, int BLOCK, bool FULL_CAP, bool BATCH, typename Sets, typename Fn>
__device__ __forceinline__ void pair_dispatch(const PairArgs<T> &a, const Sets &ps, T *base, Fn fn)
{
    auto one = [&](int64_t i) {
        if (BATCH) {
            const SysDev &sd = a.sys[a.sys_of[i]];
            if (!system_live(sd, a.flags)) return;
            fn(ps.s[sd.pset], sd.box, i);
        } else if (a.dev_box) {
            const Box bx = a.sys[0].box;
            fn(ps.s[0], bx, i);
        } else {
            fn(ps.s[0], a.box, i);
        }
    };
    if (!FULL_CAP && BATCH) {
        // pools: loop over the live systems' 128-atom chunks
        const int nch = *a.act_count;
        for (int k = blockIdx.x; k < nch; k += gridDim.x)
            for (int t = threadIdx.x; t < kPoolChunk; t += BLOCK) one((int64_t)a.act_chunks[k] + t);
    } else if (!FULL_CAP) {
        const int64_t i = (int64_t)blockIdx.x * BLOCK + threadIdx.x;
        if (i < a.N) one(i);
    } else {
        const int cnt = *a.ovf_count;
        for (int64_t q = (int64_t)blockIdx.x * BLOCK + threadIdx.x; q < cnt; q += (int64_t)gridDim.x * BLOCK)
            one(a.ovf_list[q]);
    }
}

template <typename T, int CAP, int BLOCK, bool FULL_CAP, bool BATCH, bool MULTI = false, bool FC = false>
__global__ void __launch_bounds__(BLOCK) k_pair_tersoff(PairArgs<T> a, TersoffSets<T> ps)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *base = reinterpret_cast<T *>(smem);
    pair_dispatch<T, CAP, BLOCK, FULL_CAP, BATCH>(a, ps, base, [&](const TersoffC<T> &p, const Box &box, int64_t i) {
        if constexpr (MULTI) {
            // atom i's row of the pair table; its own element's entry carries the angular
            // and bond-order constants (each bond's cutoff is its row entry's)
            const int ti = a.type[i];
            const TersoffC<T> *row = static_cast<const TersoffC<T> *>(a.ttab) + ti * kMaxTypes;
            const TersoffC<T> own = row[ti];
            tersoff_atom<T, CAP, BLOCK, FULL_CAP, true>(a, own, box, base, i, row);
        } else {
            tersoff_atom<T, CAP, BLOCK, FULL_CAP, false, FC>(a, p, box, base, i);
        }
    });
}

template <typename T, int CAP, int BLOCK, bool FULL_CAP, bool BATCH>
__global__ void __launch_bounds__(BLOCK) k_pair_sw(PairArgs<T> a, SWSets<T> ps)
{
    extern __shared__ __align__(16) unsigned char smem[];
    T *base = reinterpret_cast<T *>(smem);
    if constexpr (!FULL_CAP && !BATCH) {
        if (a.dev_box) {
            const Box bx = a.sys[0].box;
            sw_block_sorted<T, CAP, BLOCK>(a, ps.s[0], bx, base);
        } else {
            sw_block_sorted<T, CAP, BLOCK>(a, ps.s[0], a.box, base);
        }
    } else {
        pair_dispatch<T, CAP, BLOCK, FULL_CAP, BATCH>(a, ps, base, [&](const SWC<T> &p, const Box &box, int64_t i) {
            sw_atom<T, CAP, BLOCK, FULL_CAP>(a, p, box, base, i);
        });
    }
}

// Full-capacity pass (SW): WARPS warps per block, each taking deferred atoms in turn.
// Deferred atoms are few (a fraction of a percent at room temperature) and heavy: one
// thread per atom would leave them to a handful of warps on a few SMs.
template <typename T, int FULL, int WARPS, bool BATCH>
__global__ void __launch_bounds__(32 * WARPS) k_pair_sw_warp(PairArgs<T> a, SWSets<T> ps)
{
    __shared__ T sh[WARPS][4][FULL];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int cnt = *a.ovf_count;
    for (int q = blockIdx.x * WARPS + w; q < cnt; q += gridDim.x * WARPS) {
        const int64_t i = a.ovf_list[q];
        if (BATCH) {
            const SysDev &sd = a.sys[a.sys_of[i]];
            if (!system_live(sd, a.flags)) continue;
            sw_atom_warp<T, FULL>(a, ps.s[sd.pset], sd.box, sh[w], i, lane);
        } else if (a.dev_box) {
            const Box bx = a.sys[0].box;
            sw_atom_warp<T, FULL>(a, ps.s[0], bx, sh[w], i, lane);
        } else {
            sw_atom_warp<T, FULL>(a, ps.s[0], a.box, sh[w], i, lane);
        }
    }
}
constexpr int kSwFullWarps = 4;

__global__ void k_pair_reset(int *ovf_count) { *ovf_count = 0; }

// Pools: the 128-atom chunks of the systems that run now (stopped systems and free atom
// ranges are skipped).  plan[0] = number of chunks.  With skip_rebuilding, systems whose
// list is to be rebuilt this step are left out too, and the rebuild conditional (when
// has_cond) is set if any running system is to be rebuilt or a rebuild was requested.
__global__ void __launch_bounds__(1024) k_active_plan(int n_sys, const SysDev *sys, const Flags *flags, int *plan,
                                                      int *chunks, int skip_rebuilding, cudaGraphConditionalHandle h,
                                                      int has_cond)
{
    __shared__ int warp_b[32];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    int skipped_any = 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int s0 = 0; s0 < n_sys; s0 += blockDim.x) {
        const int s = s0 + threadIdx.x;
        const bool live = s < n_sys && system_live(sys[s], flags);
        const bool skip = live && skip_rebuilding && sys[s].rebuild;
        skipped_any |= __syncthreads_or(skip ? 1 : 0);
        const bool f = live && !skip;
        const int nch = f ? (int)((sys[s].n_atoms + kPoolChunk - 1) / kPoolChunk) : 0;
        int b = nch;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) b += y;
        }
        if (lane == 31) warp_b[wid] = b;
        __syncthreads();
        if (wid == 0) {
            int w = lane < (int)(blockDim.x >> 5) ? warp_b[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_b[lane] = w;
        }
        __syncthreads();
        const int pb = carry + (wid ? warp_b[wid - 1] : 0) + b - nch;
        const long long a0 = f ? sys[s].atom_start : 0;
        for (int k = 0; k < nch; ++k) chunks[pb + k] = (int)(a0 + (long long)k * kPoolChunk);
        __syncthreads();
        if (threadIdx.x == 0) carry += warp_b[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        plan[0] = carry;
        if (has_cond) cudaGraphSetConditional(h, (skipped_any || flags->rebuild) ? 1u : 0u);
    }
}

// End of the force evaluation that follows admissions: the new systems are no longer
// fresh, and later evaluations cover every running system again.
__global__ void k_clear_fresh(int n_sys, SysDev *sys, Flags *flags)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < n_sys) sys[s].fresh = 0;
    if (s == 0) flags->fresh_only = 0;
}

// ------------------------------------------------------------------ gather
// Block sums of NC per-thread fp64 values per system segment, in a fixed order:
// transpose through shared memory, then 8 threads per component add 16 values each and
// combine by shuffles.  A block of a pool can hold atoms of several systems (segment =
// system - system of the block's first atom); a single system has one segment.
template <int BLOCK, int NC>
__device__ __forceinline__ void block_partials(const double (&vals)[NC], int seg, int nseg, int seg_max,
                                               double *out, int64_t bidx)
{
    static_assert(BLOCK == 128, "block_partials assumes 128 threads");
    __shared__ double red[NC][BLOCK];
    __shared__ int sseg[BLOCK];
#pragma unroll
    for (int c = 0; c < NC; ++c) red[c][threadIdx.x] = vals[c];
    sseg[threadIdx.x] = seg;
    __syncthreads();
    const int t = threadIdx.x;
    if (t < NC * 8) {
        const int c = t >> 3, sub = t & 7;
        const unsigned grp = 0xffu << (t & 24);
        for (int g = 0; g < nseg; ++g) {
            double s = 0.0;
#pragma unroll
            for (int q = 0; q < BLOCK / 8; ++q) {
                const int k = sub + 8 * q;
                if (nseg == 1 || sseg[k] == g) s += red[c][k];
            }
            s += __shfl_xor_sync(grp, s, 4, 8);
            s += __shfl_xor_sync(grp, s, 2, 8);
            s += __shfl_xor_sync(grp, s, 1, 8);
            if (sub == 0) out[(bidx * seg_max + g) * NC + c] = s;
        }
    }
    __syncthreads();   // the shared buffers are reused by the next chunk
}

// FULL: a force evaluation (per-atom F, W, J stored; U, K, J, W partials) or a
// velocity-Verlet step (F and the kick only; U, K, J partials).  NPT (steps): also the
// diagonal kinetic and virial partials K_aa, W_aa that the barostat's pressure needs.
template <typename T, int MAXA, int BLOCK, bool FULL, bool BATCH, bool NPT>
__device__ __forceinline__ void gather_atom(const GatherArgs<T> &a, int64_t i, int64_t bidx)
{
    constexpr int NC = FULL ? kNumPartials : (NPT ? kNptPartials : kStepPartials);
    constexpr bool WDIAG = NPT && !FULL;
    // heat current: fp64 by a second walk over the bonds (fewer fp64 instructions, fewer
    // registers); fp32 from the 3x3 tensor of the first walk (one walk over memory)
    constexpr bool JPASS = sizeof(T) == 8;
    const int64_t N = a.N;
    double vals[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) vals[c] = 0.0;
    // Pools place every system on a block boundary, so a block holds one system plus
    // inactive padding atoms (which contribute zeros): one segment per block.
    const int seg = 0, nseg = 1;
    bool live = i < a.n_live;
    double damp = 0.0;
    bool fuse = a.fuse_kick != 0;
    float hs2 = a.half_skin2;
    int sid = 0;
    if (BATCH && live) {
        sid = a.sys_of[i];
        const SysDev &sd = a.sys[sid];
        live = system_live(sd, a.flags);
        damp = sd.damp;
        fuse = fuse && sd.steps_left != 1;   // a system's last budgeted step ends here
        hs2 = sd.half_skin2;
    }
    if (live) {
        uint32_t mask = a.mask[i];
        T f0 = 0, f1 = 0, f2 = 0;
        T w[9], mj[9];
        T wd0 = 0, wd1 = 0, wd2 = 0;
#pragma unroll
        for (int c = 0; c < 9; ++c) { w[c] = 0; mj[c] = 0; }
        // fp64: the stored d and r are float pairs (bond_out), summed as float pairs
        constexpr bool FFG = sizeof(T) == 8;
        F2 ff[3] = {}, fw[9] = {}, fwd[3] = {};
        int k = 0;
        // fp64 heat current (second walk): an atom with at most eight bonds keeps its two
        // groups' partners and their rows (j | row << kAtomBits), so the second walk needs no
        // list, mask or reverse-slot loads
        const bool kept = __popc(mask) <= 8;
        int jk0[4], jk1[4];
        int n0 = 0, n1 = 0;
        // bonds in groups of four: the group's list entries and reverse slots, then its
        // partners' masks, then the partners' rows, each a batch of independent loads (three
        // dependent round trips per group instead of two per bond)
        while (mask != 0u && k < MAXA) {
            int jg[4], mrg[4];
            uint32_t mjg[4];
            int ng = 0;
            const int grp = k >> 2;   // k is a multiple of 4 here
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (mask != 0u && k + u < MAXA) {
                    const int m = __ffs(mask) - 1;
                    mask &= mask - 1u;
                    jg[u] = list_atom(a.nl[(int64_t)m * N + i]);
                    mrg[u] = a.rev[(int64_t)m * N + i];
                    ng = u + 1;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < ng) mjg[u] = a.mask[jg[u]];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (u >= ng) break;
                const int j = jg[u];
                const int kr = __popc(mjg[u] & ((1u << mrg[u]) - 1u));
                if (JPASS && grp == 0) {
                    jk0[u] = j | (kr << kAtomBits);
                    n0 = u + 1;
                } else if (JPASS && grp == 1) {
                    jk1[u] = j | (kr << kAtomBits);
                    n1 = u + 1;
                }
                if (FFG && kr < MAXA) {
                    const Vec4<T> dv = a.d[(int64_t)k * N + i], ev = a.d[(int64_t)kr * N + j];
                    const F2 r[3] = {ff_unpack(a.r[(int64_t)(0 * MAXA + k) * N + i]),
                                     ff_unpack(a.r[(int64_t)(1 * MAXA + k) * N + i]),
                                     ff_unpack(a.r[(int64_t)(2 * MAXA + k) * N + i])};
                    const F2 g[3] = {ff_add(ff_unpack(dv.x), ff_neg(ff_unpack(ev.x))),
                                     ff_add(ff_unpack(dv.y), ff_neg(ff_unpack(ev.y))),
                                     ff_add(ff_unpack(dv.z), ff_neg(ff_unpack(ev.z)))};   // F_ij = d_ij - d_ji
#pragma unroll
                    for (int c = 0; c < 3; ++c) ff[c] = ff_add(ff[c], g[c]);
                    if (FULL) {
#pragma unroll
                        for (int c = 0; c < 9; ++c) fw[c] = ff_fma(r[c / 3], g[c % 3], fw[c]);
                    }
                    if (WDIAG) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) fwd[c] = ff_fma(r[c], g[c], fwd[c]);
                    }
                } else if (kr < MAXA) {
                    const Vec4<T> dv = a.d[(int64_t)k * N + i], ev = a.d[(int64_t)kr * N + j];
                    const T dx = dv.x, dy = dv.y, dz = dv.z, ex = ev.x, ey = ev.y, ez = ev.z;
                    const T rx = a.r[(int64_t)(0 * MAXA + k) * N + i], ry = a.r[(int64_t)(1 * MAXA + k) * N + i],
                            rz = a.r[(int64_t)(2 * MAXA + k) * N + i];
                    const T gx = dx - ex, gy = dy - ey, gz = dz - ez;   // F_ij = d_ij - d_ji
                    f0 += gx; f1 += gy; f2 += gz;
                    if (FULL) {
                        w[0] += rx * gx; w[1] += rx * gy; w[2] += rx * gz;
                        w[3] += ry * gx; w[4] += ry * gy; w[5] += ry * gz;
                        w[6] += rz * gx; w[7] += rz * gy; w[8] += rz * gz;
                    }
                    if (WDIAG) { wd0 += rx * gx; wd1 += ry * gy; wd2 += rz * gz; }
                    if (!JPASS) {   // M_i = sum_j r_ij (x) d_ji
                        mj[0] += rx * ex; mj[1] += rx * ey; mj[2] += rx * ez;
                        mj[3] += ry * ex; mj[4] += ry * ey; mj[5] += ry * ez;
                        mj[6] += rz * ex; mj[7] += rz * ey; mj[8] += rz * ez;
                    }
                }
                ++k;
            }
        }
        const double F[3] = {FFG ? ff_to_d(ff[0]) : to_d(f0), FFG ? ff_to_d(ff[1]) : to_d(f1),
                             FFG ? ff_to_d(ff[2]) : to_d(f2)};
        // finiteness of the sums, tested before a conversion to double (f2d_int gives inf and
        // NaN finite values)
        const bool f_fin = FFG ? finite_bits(ff[0].h) && finite_bits(ff[1].h) && finite_bits(ff[2].h)
                               : finite_bits(f0) && finite_bits(f1) && finite_bits(f2);
        // the epilogue's own loads, issued as one batch before any store: the pointers may
        // alias as far as the compiler knows, so a load placed after a store would wait for
        // a round trip of its own (one per component of the drift)
        const int t = a.type[i];
        double v[3] = {a.vel[i], a.vel[N + i], a.vel[2 * N + i]};
        const double u_i = a.u[i];
        const bool drift = a.kick && fuse;
        double x0[3] = {0.0, 0.0, 0.0}, xb[3] = {0.0, 0.0, 0.0};
        if (drift) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                x0[c] = a.pos[c * N + i];
                xb[c] = a.pos_build[c * N + i];
            }
        }
        // a step whose gather also takes the next step's kick keeps F in registers: only the
        // next step's k_kick_drift reads the stored forces, and the last step of every graph
        // and of every system's budget stores them (no fused drift there)
        if (!drift) {
            a.force[i] = F[0];
            a.force[N + i] = F[1];
            a.force[2 * N + i] = F[2];
        }
        if (a.kick) {
            const double h = a.hk[t];
            v[0] = fma(h, F[0], v[0]);
            v[1] = fma(h, F[1], v[1]);
            v[2] = fma(h, F[2], v[2]);
            if (BATCH && damp > 0.0) {   // damped-MD relaxation: v <- v (1 - gamma dt)
                const double f = 1.0 - damp * a.dt;
                v[0] *= f; v[1] *= f; v[2] *= f;
            }
            double vn[3] = {v[0], v[1], v[2]};
            if (drift) {   // the next step's half-kick and drift (k_kick_drift's arithmetic)
                float d2 = 0.f;
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    vn[c] = fma(h, F[c], v[c]);
                    const double x = fma(a.dt, vn[c], x0[c]);
                    a.pos[c * N + i] = x;
                    if (a.posf) a.posf[c * N + i] = d2f_trunc(x);
                    const float d = d2f_trunc(x - xb[c]);
                    d2 = fmaf(d, d, d2);
                }
                if (!(d2 <= hs2)) {
                    a.flags->rebuild = 1;
                    if (BATCH) a.sys[sid].rebuild = 1;
                }
            }
            a.vel[i] = vn[0];
            a.vel[N + i] = vn[1];
            a.vel[2 * N + i] = vn[2];
        }
        // a non-finite force or velocity (after the kick; without one, as given) stops the
        // system in a pool and fails the call for a single system
        if (!(f_fin && finite_bits(v[0]) && finite_bits(v[1]) && finite_bits(v[2]))) {
            if (BATCH) fail_system(a.sys[sid], MD_ERR_NAN);
            else a.flags->nonfinite = 1;
        }
        // J_i (Eq. 30) with v_i after the half-kick, and K_i = m v^2 / 2, in T (the fp32
        // per-atom value of the mixed path feeds an fp64 total).  fp64: a second walk over
        // the bonds, J_i = sum_j r_ij (d_ji . v_i), six float-pair FMAs per bond (its loads
        // hit the cache); fp32: J_i = M_i . v_i.
        const T vx = to_t<T>(v[0]), vy = to_t<T>(v[1]), vz = to_t<T>(v[2]);
        T J0 = T(0), J1 = T(0), J2 = T(0);
        F2 fj[3] = {};
        if (!JPASS) {
            J0 = mj[0] * vx + mj[1] * vy + mj[2] * vz;
            J1 = mj[3] * vx + mj[4] * vy + mj[5] * vz;
            J2 = mj[6] * vx + mj[7] * vy + mj[8] * vz;
        } else {
            // JPASS is the fp64 path: d and r are float pairs
            const F2 vf[3] = {split_d(v[0]), split_d(v[1]), split_d(v[2])};
            // the bonds in the first walk's order, the same sums
            auto jbond = [&](int kb, int jb, int kr) {
                const Vec4<T> ev = a.d[(int64_t)kr * N + jb];
                F2 dv = ff_mul(ff_unpack(ev.x), vf[0]);
                dv = ff_fma(ff_unpack(ev.y), vf[1], dv);
                dv = ff_fma(ff_unpack(ev.z), vf[2], dv);
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    fj[c] = ff_fma(ff_unpack(a.r[(int64_t)(c * MAXA + kb) * N + i]), dv, fj[c]);
            };
            uint32_t m2 = kept ? 0u : a.mask[i];
            if (kept) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int kr = (unsigned)jk0[u] >> kAtomBits;
                    if (u < n0 && kr < MAXA) jbond(u, jk0[u] & kAtomMask, kr);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int kr = (unsigned)jk1[u] >> kAtomBits;
                    if (u < n1 && kr < MAXA) jbond(4 + u, jk1[u] & kAtomMask, kr);
                }
            }
            int k2 = 0;
            while (m2 != 0u && k2 < MAXA) {   // grouped as in the first walk
                int jg[4], mrg[4];
                uint32_t mjg[4];
                int ng = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (m2 != 0u && k2 + u < MAXA) {
                        const int m = __ffs(m2) - 1;
                        m2 &= m2 - 1u;
                        jg[u] = list_atom(a.nl[(int64_t)m * N + i]);
                        mrg[u] = a.rev[(int64_t)m * N + i];
                        ng = u + 1;
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u < ng) mjg[u] = a.mask[jg[u]];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (u >= ng) break;
                    const int kr = __popc(mjg[u] & ((1u << mrg[u]) - 1u));
                    if (kr < MAXA) jbond(k2, jg[u], kr);
                    ++k2;
                }
            }
        }
        const T hm = a.hm[t];
        const T ke = hm * (vx * vx + vy * vy + vz * vz);
        // -1/2 of a float pair: both parts scaled exactly, one conversion
        auto half_neg = [](F2 x) { return ff_to_d(F2{-0.5f * x.h, -0.5f * x.l}); };
        vals[0] = u_i;
        vals[1] = to_d(ke);
        vals[2] = JPASS ? ff_to_d(fj[0]) : to_d(J0);
        vals[3] = JPASS ? ff_to_d(fj[1]) : to_d(J1);
        vals[4] = JPASS ? ff_to_d(fj[2]) : to_d(J2);
        if (WDIAG) {
            vals[5] = to_d(hm * vx * vx);
            vals[6] = to_d(hm * vy * vy);
            vals[7] = to_d(hm * vz * vz);
            vals[8] = FFG ? half_neg(fwd[0]) : -0.5 * to_d(wd0);
            vals[9] = FFG ? half_neg(fwd[1]) : -0.5 * to_d(wd1);
            vals[10] = FFG ? half_neg(fwd[2]) : -0.5 * to_d(wd2);
        }
        if (FULL) {
#pragma unroll
            for (int c = 0; c < 9; ++c) vals[5 + c] = FFG ? half_neg(fw[c]) : -0.5 * to_d(w[c]);
            if (a.w_out) {
#pragma unroll
                for (int c = 0; c < 9; ++c) a.w_out[c * N + i] = vals[5 + c];
            }
            if (a.j_out) {
                a.j_out[i] = vals[2];
                a.j_out[N + i] = vals[3];
                a.j_out[2 * N + i] = vals[4];
            }
        }
    }
    block_partials<BLOCK, NC>(vals, seg, nseg, a.seg_max, a.partials, bidx);
}

// Single system: one thread per atom.  Pools: loop over the live systems' chunks (a
// chunk is one gather block: every system starts on a chunk boundary).
template <typename T, int MAXA, int BLOCK, bool FULL, bool BATCH, bool NPT>
__global__ void __launch_bounds__(BLOCK) k_gather(GatherArgs<T> a)
{
    static_assert(BLOCK == kPoolChunk, "a gather block is one pool chunk");
    if (blockIdx.x == 0 && threadIdx.x == 0) a.flags->row_reduce = a.flags->row;
    if (BATCH) {
        const int nch = *a.act_count;
        for (int k = blockIdx.x; k < nch; k += gridDim.x) {
            const int64_t c0 = a.act_chunks[k];
            gather_atom<T, MAXA, BLOCK, FULL, BATCH, NPT>(a, c0 + threadIdx.x, c0 / BLOCK);
        }
    } else {
        gather_atom<T, MAXA, BLOCK, FULL, BATCH, NPT>(a, (int64_t)blockIdx.x * BLOCK + threadIdx.x, blockIdx.x);
    }
}



// One block per (system, component): that system's block partials of that component
// added in a fixed order; totals[s NC_ALL + c] (an NPT step's K_aa, W_aa components:
// npt_totals[s kNptExtra + c - 5]) and, when recording, series[(row n_sys + s) 5 + c].  Pools: a system that ran this step counts down its
// step budget (component-0 block) and stops at zero.
constexpr int kReduceThreads = 512;       // single system: thousands of blocks to add
constexpr int kReduceThreadsPool = 128;   // pools: one reduction per system
template <bool BATCH>
__global__ void __launch_bounds__(kReduceThreads)
k_reduce(const double *partials, int nc, int seg_max, int64_t N, int block, const int *sys_of, SysDev *sys,
         int n_sys, double *totals, double *npt_totals, double *series, Flags *flags, bool record)
{
    __shared__ double red[kReduceThreads / 32];
    const int s = blockIdx.x, c = blockIdx.y;
    int64_t a0 = 0, na = N;
    bool ran = true;
    if (BATCH) {
        a0 = sys[s].atom_start;
        na = sys[s].n_atoms;
        ran = system_live(sys[s], flags) && na > 0;
        if (!ran) return;
    }
    const int64_t b0 = na > 0 ? a0 / block : 0, b1 = na > 0 ? (a0 + na - 1) / block : -1;
    // each thread adds its blocks b0 + t, b0 + t + T, ... in that order; eight loads are
    // issued before their additions so that they are in flight together
    // (a missing block contributes +0.0, which leaves the sum unchanged)
    double acc = 0.0;
    const int64_t stride = blockDim.x;
    for (int64_t b = b0 + threadIdx.x; b <= b1; b += 8 * stride) {
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t bq = b + q * stride;
            v[q] = 0.0;
            if (bq <= b1) {
                const int seg = BATCH ? s - sys_of[bq * block] : 0;
                v[q] = partials[(bq * seg_max + seg) * nc + c];
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) acc += v[q];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        if (nc == kNptPartials && c >= kStepPartials) npt_totals[(int64_t)s * kNptExtra + c - kStepPartials] = t;
        else totals[(int64_t)s * kNumPartials + c] = t;
        if (record && c < kStepPartials) series[(flags->row_reduce * n_sys + s) * kStepPartials + c] = t;
        if (BATCH && record && c == 0 && sys[s].steps_left > 0) {
            sys[s].steps_left -= 1;
            if (sys[s].steps_left == 0) sys[s].active = 0;
        }
    }
}

// ------------------------------------------------------------------ integrator
struct KickDriftArgs {
    int64_t N;
    int64_t n_live;         // atoms integrated: [0, n_live) (ghosts beyond)
    float *posf;   // fp32 positions, refreshed every step only where the pair pass reads them
                   // between list builds (the SW and fp64 Tersoff prefilters); null otherwise (the list build
                   // writes its own copy)
    const int *act_count, *act_chunks;
    const int *sys_of;
    SysDev *sys;
    double *pos, *vel;
    const double *force;
    double *pos_build;      // scaled with the positions under NPT
    const int *type;
    double hk[kMaxTypes];   // dt/2 * acc / m per type
    double dt;
    float half_skin2;
    Flags *flags;
};

// v += F/m dt/2; x += v dt (no wrap: positions are wrapped when the list is rebuilt);
// request a rebuild when an atom has moved more than skin/2 since the last build.
// NPT: a pending Berendsen scaling is applied first (v *= lambda; x, x_build *= mu), and
// the skin test takes the box scaling since the build into account (npt_half_skin2).
template <bool BATCH, bool NPT>
__device__ __forceinline__ void kick_drift_atom(const KickDriftArgs &a, int64_t i)
{
    if (i >= a.n_live) return;
    if (BATCH && !a.sys[a.sys_of[i]].active) return;
    const int64_t N = a.N;
    const double h = a.hk[a.type[i]];
    const SysDev *sdp = NPT ? (BATCH ? &a.sys[a.sys_of[i]] : a.sys) : nullptr;
    const bool scale = NPT && sdp->npt.on && sdp->npt.pending;
    // every load before the first store (one round trip: the compiler must assume the
    // arrays may alias, so it cannot move a load above a store)
    double vv[3], xx[3], bb[3], ff[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        vv[c] = a.vel[c * N + i];
        xx[c] = a.pos[c * N + i];
        bb[c] = a.pos_build[c * N + i];
        ff[c] = a.force[c * N + i];
    }
    float d2 = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double v0 = vv[c], x0 = xx[c], xb = bb[c];
        if (scale) {
            v0 *= sdp->npt.lam;
            x0 *= sdp->npt.mu[c];
            xb *= sdp->npt.mu[c];
            a.pos_build[c * N + i] = xb;
        }
        const double v = fma(h, ff[c], v0);
        const double x = fma(a.dt, v, x0);
        a.vel[c * N + i] = v;
        a.pos[c * N + i] = x;
        if (a.posf) a.posf[c * N + i] = d2f_trunc(x);
        const float d = d2f_trunc(x - xb);
        d2 = fmaf(d, d, d2);
    }
    const float hs2 = (NPT && sdp->npt.on) ? npt_half_skin2(*sdp, true)
                                           : (BATCH ? a.sys[a.sys_of[i]].half_skin2 : a.half_skin2);
    if (!(d2 <= hs2)) {
        a.flags->rebuild = 1;
        if (BATCH) a.sys[a.sys_of[i]].rebuild = 1;
    }
}

template <bool BATCH, bool NPT>
__global__ void k_kick_drift(KickDriftArgs a)
{
    if (BATCH) {
        const int nch = *a.act_count;
        for (int k = blockIdx.x; k < nch; k += gridDim.x)
            for (int t = threadIdx.x; t < kPoolChunk; t += blockDim.x)
                kick_drift_atom<true, NPT>(a, (int64_t)a.act_chunks[k] + t);
    } else {
        kick_drift_atom<false, NPT>(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    }
}

// ------------------------------------------------------------------ Berendsen (NPT)
constexpr double kBoltzmann = 8.617333262e-5;        // eV / K (CODATA 2018, exact)
constexpr double kEvPerA3InGPa = 160.21766340;       // 1 eV / A^3 = 1.602176634e-19 J / 1e-30 m^3

// After the kick of a step: the kick scaled the velocities and coordinates of every
// running coupled system with a pending scaling; scale its box edges the same way,
// shrink its cell grid where a cell became narrower than the stencil needs, and clear the
// pending flag.  A periodic edge below 2 cell edges + 0.01 A sets flags->box_error (the
// minimum image would no longer be unique).  One thread per system.
__global__ void k_npt_apply(int n_sys, SysDev *sys, int batch, Flags *flags)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sys) return;
    SysDev &sd = sys[s];
    if (!sd.npt.on || !sd.npt.pending) return;
    if (batch && !sd.active) return;   // the kick skipped it too
    for (int a = 0; a < 3; ++a) {
        const double m = sd.npt.mu[a];
        sd.box.L[a] *= m;
        sd.box.invL[a] = 1.0 / sd.box.L[a];
        sd.npt.mu_cum[a] *= m;
        if (sd.box.pbc[a]) {
            if (!(sd.box.L[a] >= 2.0 * sd.cell_edge + 0.01)) {
                if (batch) fail_system(sd, MD_ERR_BOX);
                else flags->box_error = 1;
            }
            const int fit = (int)floor(sd.box.L[a] / sd.cell_edge);
            if (fit < sd.nc[a]) sd.nc[a] = fit < 1 ? 1 : fit;
        }
    }
    sd.npt.pending = 0;
}

// At the end of a step: lambda and mu of every coupled system from this step's totals
// (K, U in totals; K_aa, W_aa in npt_totals), left pending for the next step's kick.
__global__ void k_npt_couple(int n_sys, SysDev *sys, const double *totals, const double *npt_totals, double dt)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sys) return;
    SysDev &sd = sys[s];
    if (!sd.npt.on || sd.n_atoms < 1) return;
    const double K = totals[(int64_t)s * kNumPartials + 1];
    const double *e = npt_totals + (int64_t)s * kNptExtra;
    const double ndof = 3.0 * (double)sd.n_atoms - 3.0;
    const double T = ndof > 0.0 ? 2.0 * K / (kBoltzmann * ndof) : 0.0;
    double lam = 1.0;
    if (sd.npt.tau_T > 0.0 && T > 0.0) {
        const double l2 = 1.0 + dt / sd.npt.tau_T * (sd.npt.T0 / T - 1.0);
        lam = l2 > 0.0 ? sqrt(l2) : 0.0;
    }
    const double V = sd.box.L[0] * sd.box.L[1] * sd.box.L[2];
    for (int a = 0; a < 3; ++a) {
        double m = 1.0;
        if (sd.npt.tau_P > 0.0 && sd.box.pbc[a] && sd.npt.couple[a]) {
            const double P = (2.0 * e[a] + e[3 + a]) / V * kEvPerA3InGPa;
            m = cbrt(1.0 - sd.npt.beta * dt / sd.npt.tau_P * (sd.npt.P0 - P));
        }
        sd.npt.mu[a] = m;
    }
    sd.npt.lam = lam;
    sd.npt.pending = 1;
}

__global__ void k_step_begin(Flags *flags, int *ovf_count, cudaGraphConditionalHandle h, int has_cond)
{
    *ovf_count = 0;
    flags->row = flags->step;
    flags->step += 1;
    if (has_cond) cudaGraphSetConditional(h, flags->rebuild != 0 ? 1u : 0u);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// The pair passes that test list slots in fp32 first (SW; fp64 Tersoff) read the fp32
// positions every step, so the kick and drift keep them current; the others read them only
// in the list build, which writes its own copy.
inline bool pair_reads_posf(const Plan &p) { return p.kind == 2 || (p.kind == 1 && p.precision == 0); }

// Bounded grid of the pool kernels that loop over the chunk list (tuned: blocks per SM).
unsigned pool_grid(const Plan &p)
{
    const int64_t chunks = (p.N + kPoolChunk - 1) / kPoolChunk;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)p.pool_bps * p.n_sm));
}

constexpr int kPairCapSmall = 4;     // Tersoff: bonds staged per atom in the common-case pass
// single-system fp64 Tersoff: a 3-bond staging (44 -> 30 shared words a thread) for
// three-coordinated structures (the honeycomb sheet); a tuning choice (effective_pair_cap)
constexpr int kPairCapSmall3 = 3;
// SW: its second shell sits just outside the cutoff, and at room temperature many atoms have
// 5-6 bonds inside it (a 12-bond fp32 staging moved the rarer heavier atoms into the common
// pass but cost the pools' occupancy more than it saved: serving 2.94e9 -> 2.7e9 atom-steps/s)
template <typename T>
constexpr int kPairCapSmallSW = 8;
constexpr int kPairBlockFull = 32;   // full-capacity pass over the deferred atoms
constexpr int kGatherBlock = 128;

template <typename T, int CAP, int BLOCK, bool MULTI = false, bool FC = false>
size_t smem_for(int kind)
{
    const int nf = kind == 1 ? tersoff_smem_fields<T, CAP, MULTI, FC>() : sw_smem_fields<T, CAP>();
    return (size_t)nf * BLOCK * sizeof(T);
}

template <typename T, int CAP, int BLOCK, bool FULL_CAP, bool BATCH>
void set_smem()
{
    cudaFuncSetAttribute(k_pair_tersoff<T, CAP, BLOCK, FULL_CAP, BATCH>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_for<T, CAP, BLOCK>(1));
    if constexpr (!FULL_CAP)
        cudaFuncSetAttribute(k_pair_sw<T, CAP, BLOCK, FULL_CAP, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_for<T, CAP, BLOCK>(2));
    if constexpr (!BATCH)
        cudaFuncSetAttribute(k_pair_tersoff<T, CAP, BLOCK, FULL_CAP, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_for<T, CAP, BLOCK, true>(1));
    if constexpr (sizeof(T) == 8 && CAP == kPairCapSmall && !FULL_CAP)
        cudaFuncSetAttribute(k_pair_tersoff<T, CAP, BLOCK, false, BATCH, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_for<T, CAP, BLOCK, false, true>(1));
}

template <typename T, int B, bool BATCH>
void configure_block()
{
    set_smem<T, kPairCapSmall, B, false, BATCH>();
    set_smem<T, kPairCapSmallSW<T>, B, false, BATCH>();
    if constexpr (sizeof(T) == 8 && !BATCH)
        cudaFuncSetAttribute(k_pair_tersoff<T, kPairCapSmall3, B, false, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_for<T, kPairCapSmall3, B>(1));
}

template <typename T, bool BATCH>
void configure_type()
{
    configure_block<T, 32, BATCH>();
    configure_block<T, 64, BATCH>();
    configure_block<T, 128, BATCH>();
    configure_block<T, 256, BATCH>();
    set_smem<T, 8, kPairBlockFull, true, BATCH>();
    set_smem<T, 16, kPairBlockFull, true, BATCH>();
}

template <typename T, int FULL, bool BATCH, int B>
void pair_launch_b(const Plan &p, cudaStream_t s, int list, int parts)
{
    PairArgs<T> a;
    a.N = p.N;
    a.box = p.box;
    a.pos = p.pos;
    a.dev_box = (!BATCH && p.npt) ? 1 : 0;
    a.type = p.type;
    a.ttab = p.ttab;
    a.nn = p.nn;
    a.nl = p.nl;
    a.cap = p.cap;
    a.rc2 = T(p.rc * p.rc);
    a.stride = p.maxa;
    a.d = static_cast<Vec4<T> *>(p.pd);
    a.r = static_cast<T *>(p.pr);
    a.sys_of = p.sys_of;
    a.sys = p.sys;
    a.ovf_count = p.ovf_count;
    a.ovf_list = p.ovf_list;
    a.act_count = list == PAIR_STABLE ? p.stable_plan : (list == PAIR_REBUILT ? p.rb_plan : p.act_plan);
    a.act_chunks = list == PAIR_STABLE ? p.stable_chunks : (list == PAIR_REBUILT ? p.rb_chunks : p.act_chunks);
    a.posf = p.posf;
    a.margin = p.list_margin;
    a.mask = p.mask;
    a.u = p.u;
    a.flags = p.flags;
    a.batch = BATCH ? 1 : 0;
    const unsigned nb = BATCH ? pool_grid(p) : blocks_for(p.N, B);
    int64_t nbf = (p.N + kPairBlockFull - 1) / kPairBlockFull;
    if (nbf > 4 * (int64_t)p.n_sm) nbf = 4 * (int64_t)p.n_sm;
    if (p.kind == 1) {
        TersoffSets<T> c;
        for (int k = 0; k < kMaxSets; ++k) c.s[k] = tersoff_const<T>(p.tp[k < p.n_sets ? k : 0]);
        if constexpr (!BATCH) {
            if (p.multi) {   // several elements: per-pair constants from the device table
                if (parts & PAIR_FAST)
                    k_pair_tersoff<T, kPairCapSmall, B, false, false, true>
                        <<<nb, B, smem_for<T, kPairCapSmall, B, true>(1), s>>>(a, c);
                if (parts & PAIR_DEFERRED)
                    k_pair_tersoff<T, FULL, kPairBlockFull, true, false, true>
                        <<<(unsigned)nbf, kPairBlockFull, smem_for<T, FULL, kPairBlockFull, true>(1), s>>>(a, c);
                return;
            }
        }
        bool fast3 = false;
        if constexpr (sizeof(T) == 8 && !BATCH) fast3 = effective_pair_cap(p) == kPairCapSmall3;
        if (parts & PAIR_FAST) {
            if constexpr (sizeof(T) == 8 && !BATCH) {
                if (fast3)
                    k_pair_tersoff<T, kPairCapSmall3, B, false, false>
                        <<<nb, B, smem_for<T, kPairCapSmall3, B>(1), s>>>(a, c);
            }
            bool keep_fc = false;
            if constexpr (sizeof(T) == 8) {
                keep_fc = !fast3 && p.pair_fc;
                if (keep_fc)
                    k_pair_tersoff<T, kPairCapSmall, B, false, BATCH, false, true>
                        <<<nb, B, smem_for<T, kPairCapSmall, B, false, true>(1), s>>>(a, c);
            }
            if (!fast3 && !keep_fc)
                k_pair_tersoff<T, kPairCapSmall, B, false, BATCH><<<nb, B, smem_for<T, kPairCapSmall, B>(1), s>>>(a, c);
        }
        if (parts & PAIR_DEFERRED)
            k_pair_tersoff<T, FULL, kPairBlockFull, true, BATCH>
                <<<(unsigned)nbf, kPairBlockFull, smem_for<T, FULL, kPairBlockFull>(1), s>>>(a, c);
    } else {
        SWSets<T> c;
        for (int k = 0; k < kMaxSets; ++k) c.s[k] = sw_const<T>(p.sp[k < p.n_sets ? k : 0]);
        if (parts & PAIR_FAST)
            k_pair_sw<T, kPairCapSmallSW<T>, B, false, BATCH><<<nb, B, smem_for<T, kPairCapSmallSW<T>, B>(2), s>>>(a, c);
        if (parts & PAIR_DEFERRED)
            k_pair_sw_warp<T, FULL, kSwFullWarps, BATCH><<<(unsigned)nbf, 32 * kSwFullWarps, 0, s>>>(a, c);
    }
}

// The common-case pass's block size is a run-time choice (the autotuner's); every
// candidate computes each atom in one thread the same way, so results do not depend on it.
template <typename T, int FULL, bool BATCH>
void pair_launch(const Plan &p, cudaStream_t s, int list, int parts)
{
    switch (effective_pair_block(p)) {
    case 32: pair_launch_b<T, FULL, BATCH, 32>(p, s, list, parts); break;
    case 128: pair_launch_b<T, FULL, BATCH, 128>(p, s, list, parts); break;
    case 256: pair_launch_b<T, FULL, BATCH, 256>(p, s, list, parts); break;
    default: pair_launch_b<T, FULL, BATCH, 64>(p, s, list, parts); break;
    }
}

template <typename T, int MAXA, bool BATCH>
void gather_launch(const Plan &p, cudaStream_t s, const double *hk, double dt, bool full, bool fuse_next)
{
    GatherArgs<T> a;
    a.N = p.N;
    a.n_live = p.n_owned >= 0 ? p.n_owned : p.N;
    a.nl = p.nl;
    a.rev = p.rev;
    a.mask = p.mask;
    a.d = static_cast<const Vec4<T> *>(p.pd);
    a.r = static_cast<const T *>(p.pr);
    a.u = p.u;
    a.type = p.type;
    for (int t = 0; t < kMaxTypes; ++t) {
        a.mass[t] = p.mass[t];
        a.hm[t] = T(0.5 / kAccUnit) * T(p.mass[t]);
        a.hk[t] = hk ? hk[t] : 0.0;
    }
    a.kick = hk != nullptr;
    a.vel = p.vel;
    a.force = p.force;
    a.w_out = full ? p.w : nullptr;
    a.j_out = full ? p.j : nullptr;
    a.partials = p.partials;
    a.seg_max = p.seg_max;
    a.sys_of = p.sys_of;
    a.sys = p.sys;
    a.dt = dt;
    a.flags = p.flags;
    a.act_count = p.act_plan;
    a.act_chunks = p.act_chunks;
    a.fuse_kick = (fuse_next && hk && !full && !p.npt) ? 1 : 0;
    a.pos = p.pos;
    a.pos_build = p.pos_build;
    a.posf = pair_reads_posf(p) ? p.posf : nullptr;
    a.half_skin2 = (float)(0.25 * p.skin * p.skin);
    const unsigned nb = BATCH ? pool_grid(p) : blocks_for(p.N, kGatherBlock);
    if (full)
        k_gather<T, MAXA, kGatherBlock, true, BATCH, false><<<nb, kGatherBlock, 0, s>>>(a);
    else if (p.npt)
        k_gather<T, MAXA, kGatherBlock, false, BATCH, true><<<nb, kGatherBlock, 0, s>>>(a);
    else
        k_gather<T, MAXA, kGatherBlock, false, BATCH, false><<<nb, kGatherBlock, 0, s>>>(a);
}

template <typename T>
void fill_table(const Plan &p, void *host)
{
    TersoffC<T> *t = static_cast<TersoffC<T> *>(host);
    for (int a = 0; a < kMaxTypes; ++a)
        for (int b = 0; b < kMaxTypes; ++b)
            t[a * kMaxTypes + b] = tersoff_const<T>(p.tpair[a < p.n_elem ? a : 0][b < p.n_elem ? b : 0]);
}

}  // namespace

// The build compiles this file four times, so that its large sets of kernel instantiations
// compile in parallel: MD_FORCE_PART 1 emits the fp64 launch code and kernels of single
// systems, 3 those of pools, 2 the fp32 ones, 0 the rest (the entry points below, which call
// into the others).  Without MD_FORCE_PART the file holds every part.
void pair_dispatch_fp64(const Plan &p, cudaStream_t s, int list, int parts);
void pair_dispatch_fp64_pool(const Plan &p, cudaStream_t s, int list, int parts);
void pair_dispatch_fp32(const Plan &p, cudaStream_t s, int list, int parts);
void gather_dispatch_fp64(const Plan &p, cudaStream_t s, const double *hk, double dt, bool full, bool fuse);
void gather_dispatch_fp64_pool(const Plan &p, cudaStream_t s, const double *hk, double dt, bool full, bool fuse);
void gather_dispatch_fp32(const Plan &p, cudaStream_t s, const double *hk, double dt, bool full, bool fuse);
void configure_fp64();
void configure_fp64_pool();
void configure_fp32();

#if !defined(MD_FORCE_PART) || MD_FORCE_PART == 1
void pair_dispatch_fp64(const Plan &p, cudaStream_t s, int list, int parts)
{
    if (p.maxa <= 8) pair_launch<double, 8, false>(p, s, list, parts);
    else pair_launch<double, 16, false>(p, s, list, parts);
}
void gather_dispatch_fp64(const Plan &p, cudaStream_t s, const double *hk, double dt, bool full, bool fuse)
{
    if (p.maxa <= 8) gather_launch<double, 8, false>(p, s, hk, dt, full, fuse);
    else gather_launch<double, 16, false>(p, s, hk, dt, full, fuse);
}
void configure_fp64() { configure_type<double, false>(); }
#endif

#if !defined(MD_FORCE_PART) || MD_FORCE_PART == 3
void pair_dispatch_fp64_pool(const Plan &p, cudaStream_t s, int list, int parts)
{
    if (p.maxa <= 8) pair_launch<double, 8, true>(p, s, list, parts);
    else pair_launch<double, 16, true>(p, s, list, parts);
}
void gather_dispatch_fp64_pool(const Plan &p, cudaStream_t s, const double *hk, double dt, bool full, bool fuse)
{
    if (p.maxa <= 8) gather_launch<double, 8, true>(p, s, hk, dt, full, fuse);
    else gather_launch<double, 16, true>(p, s, hk, dt, full, fuse);
}
void configure_fp64_pool() { configure_type<double, true>(); }
#endif

#if !defined(MD_FORCE_PART) || MD_FORCE_PART == 2
void pair_dispatch_fp32(const Plan &p, cudaStream_t s, int list, int parts)
{
    if (p.batch) {
        if (p.maxa <= 8) pair_launch<float, 8, true>(p, s, list, parts);
        else pair_launch<float, 16, true>(p, s, list, parts);
    } else {
        if (p.maxa <= 8) pair_launch<float, 8, false>(p, s, list, parts);
        else pair_launch<float, 16, false>(p, s, list, parts);
    }
}
void gather_dispatch_fp32(const Plan &p, cudaStream_t s, const double *hk, double dt, bool full, bool fuse)
{
    if (p.batch) {
        if (p.maxa <= 8) gather_launch<float, 8, true>(p, s, hk, dt, full, fuse);
        else gather_launch<float, 16, true>(p, s, hk, dt, full, fuse);
    } else {
        if (p.maxa <= 8) gather_launch<float, 8, false>(p, s, hk, dt, full, fuse);
        else gather_launch<float, 16, false>(p, s, hk, dt, full, fuse);
    }
}
void configure_fp32()
{
    configure_type<float, false>();
    configure_type<float, true>();
}
#endif

#if !defined(MD_FORCE_PART) || MD_FORCE_PART == 0
namespace {
__global__ void k_fastmath_eval(int fn, int64_t n, const double *x, double *y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    switch (fn) {
    case 0: y[i] = exp_tab(x[i]); break;
    case 1: y[i] = log_tab(x[i]); break;
    case 2: y[i] = rcp_nr(x[i]); break;
    case 3: y[i] = rsqrt_nr(x[i]); break;
    case 4: y[i] = exp_ff(x[i]); break;
    case 5: y[i] = log_ff(x[i]); break;
    case 6: y[i] = rcp_ff(x[i]); break;
    case 7: y[i] = rsqrt_ff(x[i]); break;
    case 8: y[i] = ff_to_d(exp_f2(split_d(x[i]))); break;
    default: y[i] = ff_to_d(log_f2(split_d(x[i]))); break;
    }
}
}  // namespace

size_t tersoff_table_bytes(const Plan &p)
{
    return (size_t)kMaxTypes * kMaxTypes * (p.precision == 0 ? sizeof(TersoffC<double>) : sizeof(TersoffC<float>));
}

void fill_tersoff_table(const Plan &p, void *host)
{
    if (p.precision == 0) fill_table<double>(p, host);
    else fill_table<float>(p, host);
}

int effective_pair_block(const Plan &p)
{
    if (valid_pair_block(p.pair_block)) return p.pair_block;
    return p.precision == 0 ? 64 : 128;   // measured defaults (fp64: 64, fp32: 128)
}

bool valid_pair_block(int b) { return b == 32 || b == 64 || b == 128 || b == 256; }

// The 3-bond staging exists for the single-system fp64 Tersoff pass only (one element);
// everywhere else the common-case pass stages 4 (Tersoff) or 8 (SW) bonds.
int effective_pair_cap(const Plan &p)
{
    const bool can3 = p.kind == 1 && p.precision == 0 && !p.batch && !p.multi && !p.pair_fc;
    return (can3 && p.pair_cap == kPairCapSmall3) ? kPairCapSmall3 : kPairCapSmall;
}

// The shared-memory opt-in of the pair kernels is an attribute of the kernel in the
// current device's context: it is set once per device, under a lock (contexts, servers and
// the allocation-free entry point may be created from several threads and on several
// devices).  Returns false when the current device cannot be read or the opt-in failed.
bool configure_kernels(const Plan &)
{
    static std::mutex mu;
    static bool done[kMaxConfigDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxConfigDevices) {
        cudaGetLastError();
        return false;
    }
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return true;
    cudaGetLastError();   // a stale error of an earlier call must not count as this one's
    configure_fp64();
    configure_fp64_pool();
    configure_fp32();
    if (cudaGetLastError() != cudaSuccess) return false;
    done[dev] = true;
    return true;
}

void launch_kick_drift(const Plan &p, cudaStream_t s, const double *hk, double dt)
{
    if (p.N == 0) return;
    KickDriftArgs a;
    a.N = p.N;
    a.n_live = p.n_owned >= 0 ? p.n_owned : p.N;
    a.sys_of = p.sys_of;
    a.sys = p.sys;
    a.pos = p.pos;
    a.vel = p.vel;
    a.force = p.force;
    a.pos_build = p.pos_build;
    a.posf = pair_reads_posf(p) ? p.posf : nullptr;
    a.type = p.type;
    for (int t = 0; t < kMaxTypes; ++t) a.hk[t] = hk[t];
    a.dt = dt;
    const double hs = 0.5 * p.skin;
    a.half_skin2 = (float)(hs * hs);
    a.flags = p.flags;
    a.act_count = p.act_plan;
    a.act_chunks = p.act_chunks;
    if (p.batch) {
        if (p.npt) k_kick_drift<true, true><<<pool_grid(p), kPoolChunk, 0, s>>>(a);
        else k_kick_drift<true, false><<<pool_grid(p), kPoolChunk, 0, s>>>(a);
    } else {
        if (p.npt) k_kick_drift<false, true><<<blocks_for(p.N, 256), 256, 0, s>>>(a);
        else k_kick_drift<false, false><<<blocks_for(p.N, 256), 256, 0, s>>>(a);
    }
}

void launch_step_begin(const Plan &p, cudaStream_t s, const cudaGraphConditionalHandle *h)
{
    k_step_begin<<<1, 1, 0, s>>>(p.flags, p.ovf_count, h ? *h : cudaGraphConditionalHandle(0), h ? 1 : 0);
}

void launch_pair_reset(const Plan &p, cudaStream_t s) { k_pair_reset<<<1, 1, 0, s>>>(p.ovf_count); }

void launch_active_plan(const Plan &p, cudaStream_t s)
{
    if (!p.batch) return;
    k_active_plan<<<1, 1024, 0, s>>>(p.n_sys, p.sys, p.flags, p.act_plan, p.act_chunks, 0,
                                     cudaGraphConditionalHandle(0), 0);
}

void launch_stable_plan(const Plan &p, cudaStream_t s, const cudaGraphConditionalHandle *h)
{
    if (!p.batch) return;
    k_active_plan<<<1, 1024, 0, s>>>(p.n_sys, p.sys, p.flags, p.stable_plan, p.stable_chunks, 1,
                                     h ? *h : cudaGraphConditionalHandle(0), h ? 1 : 0);
}

void launch_clear_fresh(const Plan &p, cudaStream_t s)
{
    k_clear_fresh<<<(unsigned)((p.n_sys + 255) / 256), 256, 0, s>>>(p.n_sys, p.sys, p.flags);
}

int launch_pair(const Plan &p, cudaStream_t s, int list, int parts)
{
    if (p.N == 0) return 0;
    const int l = p.batch ? list : PAIR_ALL;
    if (p.precision != 0) pair_dispatch_fp32(p, s, l, parts);
    else if (p.batch) pair_dispatch_fp64_pool(p, s, l, parts);
    else pair_dispatch_fp64(p, s, l, parts);
    return (parts & PAIR_FAST ? 1 : 0) + (parts & PAIR_DEFERRED ? 1 : 0);
}

void launch_gather(const Plan &p, cudaStream_t s, const double *hk, double dt, bool full, bool fuse_next)
{
    if (p.N == 0) return;
    if (p.precision != 0) gather_dispatch_fp32(p, s, hk, dt, full, fuse_next);
    else if (p.batch) gather_dispatch_fp64_pool(p, s, hk, dt, full, fuse_next);
    else gather_dispatch_fp64(p, s, hk, dt, full, fuse_next);
}

void launch_reduce(const Plan &p, cudaStream_t s, bool full, bool record_series)
{
    const int nc = full ? kNumPartials : (p.npt ? kNptPartials : kStepPartials);
    const bool rec = record_series && p.series != nullptr;
    if (p.batch)
        k_reduce<true><<<dim3(p.n_sys, nc), kReduceThreadsPool, 0, s>>>(p.partials, nc, p.seg_max, p.N, kGatherBlock,
                                                                    p.sys_of, p.sys, p.n_sys, p.totals,
                                                                    p.npt_totals, p.series, p.flags, rec);
    else
        k_reduce<false><<<dim3(1, nc), kReduceThreads, 0, s>>>(p.partials, nc, p.seg_max, p.N, kGatherBlock,
                                                               p.sys_of, p.sys, 1, p.totals, p.npt_totals,
                                                               p.series, p.flags, rec);
}

void launch_npt_apply(const Plan &p, cudaStream_t s)
{
    if (!p.npt || p.N == 0) return;
    k_npt_apply<<<(unsigned)((p.n_sys + 127) / 128), 128, 0, s>>>(p.n_sys, p.sys, p.batch ? 1 : 0, p.flags);
}

void launch_npt_couple(const Plan &p, cudaStream_t s, double dt)
{
    if (!p.npt || p.N == 0) return;
    k_npt_couple<<<(unsigned)((p.n_sys + 127) / 128), 128, 0, s>>>(p.n_sys, p.sys, p.totals, p.npt_totals, dt);
}

int gather_block() { return kGatherBlock; }
int gather_blocks(int64_t N) { return N == 0 ? 1 : (int)blocks_for(N, kGatherBlock); }
#endif  // part 0

}  // namespace mdk

#if !defined(MD_FORCE_PART) || MD_FORCE_PART == 0

// Diagnostics: the pair passes' exp, log, reciprocal and reciprocal square root routines
// (fn 0..9, as k_fastmath_eval lists them) on n host values, on the current device
// (accuracy tests).  Returns 0, -1 for bad arguments, -5 on a CUDA error.
extern "C" int md_fastmath_eval(int fn, int64_t n, const double *x, double *y)
{
    if (fn < 0 || fn > 9 || n < 0 || (n > 0 && (!x || !y))) return -1;
    if (n == 0) return 0;
    double *d = nullptr;
    if (cudaMalloc(&d, sizeof(double) * 2 * (size_t)n) != cudaSuccess) {
        cudaGetLastError();
        return -5;
    }
    cudaError_t e = cudaMemcpy(d, x, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        mdk::k_fastmath_eval<<<(unsigned)((n + 255) / 256), 256>>>(fn, n, d, d + n);
        e = cudaMemcpy(y, d + n, sizeof(double) * n, cudaMemcpyDeviceToHost);
    }
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return -5;
    }
    return 0;
}
#endif  // part 0
