// fastmath.cuh -- table-driven fp64 exp and log for the Tersoff pair pass.
//
// GB300 issues fp64 at 1/64 of its fp32 rate, and the Tersoff pair pass spends most of its
// fp64 instructions in four exponentials and two logarithms per bond (f_R, f_A and the bond
// order b = (1 + (beta zeta)^n)^(-1/(2n))).  These follow the table-driven method of
// P. T. P. Tang (exp: ACM TOMS 15 (1989) 144-157; log: ACM TOMS 16 (1990) 378-400), written
// here from the mathematics with short Taylor polynomials:
//
//   exp: x = (256 m + j) ln2/256 + r, |r| <= ln2/512;  e^x = 2^m 2^(j/256) (1 + p(r)),
//        p(r) = r + r^2/2 + r^3/6 + r^4/24.  The integer k = 256 m + j is rounded in fp32
//        from x truncated to fp32 and becomes a double by integer instructions; it can be
//        one off the exact rounding near a half-integer, which widens |r| to at most
//        0.547 ln2/256 for |x| <= 708 (truncation then below 0.3 ulp).
//        Seven fp64 instructions; error within 2 ulp.  Domain |x| <= 708 (no clamping: the
//        pair pass's arguments are -lambda r with r < S, and n log(beta zeta) and
//        -log(1 + x)/(2n) with zeta >= f_C > 1e-32, all far inside).
//   log: x = 2^e m, m in [1, 2), c_j = 1 + (j + 1/2)/256 for the top eight bits j of m,
//        log x = e ln2 - log(RN(1/c_j)) + log(1 + r), r = m RN(1/c_j) - 1 (one fma),
//        |r| < 1/512, log(1 + r) by its Taylor series to r^5 (truncation 1e-17); e becomes a
//        double by integer and fp32 instructions.
//        Nine fp64 instructions; absolute error about 1e-16 (1 + |e|), which is what the
//        bond order needs (an absolute error d in log(1 + x) is a relative error d/(2n) in
//        b, and an absolute error in log zeta a relative error n d in (beta zeta)^n).
//        Domain: positive normal x.
// The tables are written by gen_fastmath_tables.py (decimal arithmetic at 50 digits).
#pragma once

#include "fastmath_tables.cuh"
#include "md_internal.cuh"

namespace mdk {

// 1.5 * 2^23: adding it to a float of magnitude below 2^22 rounds that float to an
// integer, held in the low mantissa bits
constexpr float kShiftF = 12582912.0f;
constexpr int kShiftBits = 0x4b400000;
constexpr float kInvLn2o256F = (float)kInvLn2o256;

// a small integer (|k| < 2^22) as a double, without the fp64 pipe
__device__ __forceinline__ double int_to_d(int k)
{
    return f2d_int(__int_as_float(kShiftBits + k) - kShiftF);
}

__device__ __forceinline__ double exp_tab(double x)
{
    const float tf = fmaf(d2f_trunc(x), kInvLn2o256F, kShiftF);
    const int k = __float_as_int(tf) - kShiftBits;       // ~round(x 256/ln2), two's complement
    const double kd = f2d_int(tf - kShiftF);            // k exactly
    double r = fma(kd, -kLn2o256Hi, x);
    r = fma(kd, -kLn2o256Lo, r);
    double q = fma(r, 1.0 / 24.0, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    const double p = fma(q, r * r, r);                   // e^r - 1
    const double tj = __ldg(&kExp2Tab[k & 255]);
    const double y = fma(tj, p, tj);                     // 2^(j/256) e^r, in [0.997, 2)
    return __hiloint2double(__double2hiint(y) + ((k >> 8) << 20), __double2loint(y));
}

__device__ __forceinline__ double log_tab(double x)
{
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int e = (hi >> 20) - 1023;
    const int j = (hi >> 12) & 255;
    const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);
    const double r = fma(m, __ldg(&kLogInvTab[j]), -1.0);
    double q = fma(r, 0.2, -0.25);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    const double p = fma(q, r * r, r);                   // log(1 + r)
    const double ed = int_to_d(e);
    return fma(ed, kLn2Hi, __ldg(&kLogTab[j]) + fma(ed, kLn2Lo, p));
}

// ---------------------------------------------------------------- float pairs
// GB300 issues fp64 at 1/64 of its fp32 rate.  The exponential and logarithm below keep in
// fp64 only what must be exact -- the range reduction and the final multiply-add with the
// table value -- and evaluate the small correction polynomial, whose result needs far fewer
// than 53 bits relative to itself, as a pair of floats (hi + lo, about 48 bits) on the fp32
// pipe, with the error-free transformations of Knuth (two-sum) and Dekker (two-product, via
// the fused multiply-add).  The _rn intrinsics keep the compiler from contracting them.
struct F2 {
    float h, l;
};
// s + e = a + b exactly, for |a| >= |b| (Dekker's fast two-sum)
__device__ __forceinline__ F2 fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// s + e = a + b exactly, any a, b (Knuth's two-sum)
__device__ __forceinline__ F2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// p + e = a b exactly (Dekker's two-product with a fused multiply-add)
__device__ __forceinline__ F2 two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
// the integer n (0 <= n <= 2^23) as a float, exactly, on the fp32 pipe
__device__ __forceinline__ float int23_to_f(unsigned n) { return __fsub_rn(__uint_as_float(0x4b000000u | n), 8388608.0f); }

// x = h + l + t: h = x truncated to a float (d2f_trunc), l = the next 23 bits of x rounded
// to nearest on the last 6 (l is at most 2^23 units of 2^(e-46), exact as a float),
// |t| <= 2^-47 |x|.  l is zero for |x| < 2^-79.
__device__ __forceinline__ F2 split_d(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int se = (int)((hi >> 20) & 0x7ffu) - 1023 - 46 + 127;   // float exponent of the lo part's unit
    float l = 0.f;
    if (se >= 1 && se <= 254) l = __fmul_rn(int23_to_f(((lo & 0x1fffffffu) + 32u) >> 6), __int_as_float(se << 23));
    if (hi & 0x80000000u) l = -l;
    return {d2f_trunc(x), l};
}

// e^x for |x| <= 700, within about 1 ulp: x = k ln2/256 + r (k = round(x 256/ln2), computed
// as in exp_tab), e^x = 2^(k >> 8) T_j (1 + p), p = e^r - 1, j = k & 255.  fp64: the exact
// first reduction step r1 = x - k ln2hi (ln2hi has 32 bits, so k ln2hi is exact for |k| <
// 2^21), p rounded once to a double, and T_j + T_j p.  On the fp32 pipe: r = r1 - k ln2lo
// (ln2lo as a float pair, k ln2lo by two-product) and p = r + r^2/2 + r^3/6 + r^4/24 + r^5/120
// as a float pair (|r| <= 0.55 ln2/256 < 2^-8.4: r^6/720 < 2^-63).  Three fp64 instructions.
__device__ __forceinline__ double exp_ff(double x)
{
    const float tf = fmaf(d2f_trunc(x), kInvLn2o256F, kShiftF);
    const int k = __float_as_int(tf) - kShiftBits;
    const float kf = __fsub_rn(tf, kShiftF);                 // k exactly
    const double r1 = fma(f2d_int(kf), -kLn2o256Hi, x);      // exact
    const F2 rs = split_d(r1);
    const F2 d = two_prod(kf, kLn2o256LoF[0]);               // k ln2lo, head exactly
    const float dl = __fmaf_rn(kf, kLn2o256LoF[1], d.l);
    // r = rs.h + m + ml, m = rs.l - k ln2lo (|m| < 2^-22 for |k| < 2^19: its square counts)
    const F2 mm = two_sum(rs.l, -d.h);
    const float m = mm.h, ml = __fsub_rn(mm.l, dl);
    const float rh = rs.h;
    // r^2 = rh^2 + 2 rh m + m^2, rh^2 = s.h + s.l exactly
    const F2 s = two_prod(rh, rh);
    const float sq_l = __fmaf_rn(m, m, __fmaf_rn(2.f * rh, m, s.l));
    // r^3 = rh^3 + 3 rh^2 m + 3 rh m^2: rh^3 = c.h + c.l + s.l rh;  r^3/6 = (c6.h, c6.l)
    const F2 c = two_prod(s.h, rh);
    const float c_l = __fmaf_rn(s.l, rh, __fmaf_rn(3.f * s.h, m, __fmaf_rn(3.f * rh * m, m, c.l)));
    const F2 c6 = two_prod(c.h, kSixthF[0]);
    const float c6l = __fmaf_rn(c.h, kSixthF[1], __fmaf_rn(c_l, kSixthF[0], c6.l));
    // r^4/24 + r^5/120 (below 2^-41: one float suffices)
    const float s2 = __fmul_rn(s.h, s.h);
    const float q45 = __fmul_rn(s2, __fmaf_rn(rh, 1.f / 120.f, 1.f / 24.f));
    // p = rh + s.h/2 + m + c6.h + (small terms)
    F2 P = fast_two_sum(rh, __fmul_rn(0.5f, s.h));
    const F2 P2 = two_sum(P.h, m);
    const F2 P3 = two_sum(P2.h, c6.h);
    const float pl = ((((P.l + P2.l) + P3.l) + ml) + __fmaf_rn(0.5f, sq_l, c6l)) + q45;
    const double p = f2d_int(P3.h) + f2d_int(pl);
    const double tj = __ldg(&kExp2Tab[k & 255]);
    const double y = fma(tj, p, tj);                          // 2^(j/256) e^r, in [0.997, 2)
    return __hiloint2double(__double2hiint(y) + ((k >> 8) << 20), __double2loint(y));
}

// log x for positive normal x, absolute error about 1e-16 (1 + |e|), e the binary exponent:
// x = 2^e m, m in [1, 2) split exactly into three floats (m1 + m2 + m3, integer
// instructions), i_j = RN_float(1/c_j), c_j = 1 + (j + 1/2)/256 for the top eight bits j of m;
// log x = e ln2 + (-log i_j) + log(1 + r), r = m i_j - 1 (|r| < 2^-8.9) formed exactly-enough
// as a float pair by two-products (m1 i_j is within 2^-9 of 1, so its difference from 1 is
// exact), log(1 + r) = r - r^2/2 + r^3/3 - r^4/4 + r^5/5 as a float pair together with e ln2lo,
// rounded once to a double and added to e ln2hi - log i_j (an exact product and one rounding).
// Three fp64 instructions.
__device__ __forceinline__ double log_ff(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)(hi >> 20) - 1023;
    const int j = (hi >> 12) & 255;
    const float m1 = __uint_as_float(0x3f800000u | ((hi & 0xfffffu) << 3) | (lo >> 29));
    const float m2 = __fmul_rn(int23_to_f((lo >> 6) & 0x7fffffu), 0x1p-46f);
    const float m3 = __fmul_rn(int23_to_f(lo & 63u), 0x1p-52f);
    const float inv = __ldg(&kLogInvTabF[j]);
    const F2 p1 = two_prod(m1, inv);
    const float r0 = __fsub_rn(p1.h, 1.f);                    // exact: p1.h is within 2^-8 of 1
    const F2 p2 = two_prod(m2, inv);
    const F2 t = two_sum(p1.l, p2.h);
    const F2 R = two_sum(r0, t.h);
    const float rl = __fmaf_rn(m3, inv, (R.l + t.l) + p2.l);
    const F2 rr = fast_two_sum(R.h, rl);                      // r = rr.h + rr.l
    const float rh = rr.h, m = rr.l;
    const F2 s = two_prod(rh, rh);
    const float sq_l = __fmaf_rn(2.f * rh, m, s.l);           // r^2 = s.h + sq_l
    const F2 c = two_prod(s.h, rh);
    const float c_l = __fmaf_rn(s.l, rh, __fmaf_rn(3.f * s.h, m, c.l));   // r^3 = c.h + c_l
    const F2 c3 = two_prod(c.h, kThirdF[0]);
    const float c3l = __fmaf_rn(c.h, kThirdF[1], __fmaf_rn(c_l, kThirdF[0], c3.l));
    const float s2 = __fmul_rn(s.h, s.h);
    const float q45 = __fmul_rn(s2, __fmaf_rn(rh, 0.2f, -0.25f));            // -r^4/4 + r^5/5
    // e ln2lo (|e| <= 1023: the head product exact by two-product)
    const float ef = __fsub_rn(__int_as_float(kShiftBits + e), kShiftF);   // e exactly
    const F2 el = two_prod(ef, kLn2LoF[0]);
    const float ell = __fmaf_rn(ef, kLn2LoF[1], el.l);
    // q = rh - s.h/2 + c3.h + e ln2lo + (small terms)
    const F2 Q = fast_two_sum(rh, __fmul_rn(-0.5f, s.h));
    const F2 Q2 = two_sum(Q.h, c3.h);
    const F2 Q3 = two_sum(Q2.h, el.h);
    const float ql = (((((Q.l + Q2.l) + Q3.l) + m) + ell) + __fmaf_rn(-0.5f, sq_l, c3l)) + q45;
    const double q = f2d_int(Q3.h) + f2d_int(ql);
    return fma(int_to_d(e), kLn2Hi, __ldg(&kLogTabF[j])) + q;
}

// ---- float-pair arithmetic (about 48 bits; absolute error about 2^-48 of the operands'
// magnitudes, which is what sums of force terms need).  A pair travels through an fp64
// shared-memory slot as the two floats' bit patterns (ff_pack / ff_unpack: integer moves).
__device__ __forceinline__ double ff_pack(F2 a) { return __hiloint2double(__float_as_int(a.h), __float_as_int(a.l)); }
__device__ __forceinline__ F2 ff_unpack(double d)
{
    return {__int_as_float(__double2hiint(d)), __int_as_float(__double2loint(d))};
}
// a pair as a double (one fp64 addition, exact: the two floats span at most 48 bits);
// split_d goes the other way
__device__ __forceinline__ double ff_to_d(F2 a) { return f2d_int(a.h) + f2d_int(a.l); }
__device__ __forceinline__ F2 ff_neg(F2 a) { return {-a.h, -a.l}; }
__device__ __forceinline__ F2 ff_add(F2 a, F2 b)
{
    const F2 s = two_sum(a.h, b.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ F2 ff_mul(F2 a, F2 b)
{
    const F2 p = two_prod(a.h, b.h);
    return fast_two_sum(p.h, __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l)));
}
// a b + c
__device__ __forceinline__ F2 ff_fma(F2 a, F2 b, F2 c)
{
    const F2 p = two_prod(a.h, b.h);
    const F2 s = two_sum(p.h, c.h);
    const float l = __fadd_rn(__fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, p.l)), __fadd_rn(c.l, s.l));
    return fast_two_sum(s.h, l);
}
// 1/a: the correctly rounded float reciprocal y of a.h, then y + y e, e = 1 - a y (y a.h is
// within 2^-23 of 1, so 1 minus its head is exact)
__device__ __forceinline__ F2 ff_rcp(F2 a)
{
    const float y = __frcp_rn(a.h);
    const F2 p = two_prod(a.h, y);
    const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.f, p.h), p.l), __fmul_rn(a.l, y));
    const F2 t = two_prod(y, e);
    return fast_two_sum(y, __fadd_rn(t.h, t.l));
}

// e^y of a float pair on the fp32 pipe alone, error about 2^-47 e^y plus, where the result's
// low float is subnormal, an absolute error below 2^-126 (y.h clamped to [-80, 80]): y = k ln2/256 + r with k = round(y.h 256/ln2)
// (as in exp_tab), r = y - k C1 - k C2 - k C3 (ln2/256 = C1 + C2 + C3: C1 has 9 bits, so
// k C1 is exact for |k| < 2^15; k C2 by two-product), |r| <= 0.55 ln2/256;
// e^r - 1 = r + r^2/2 (float pair) + r^3/6 + r^4/24 + r^5/120 (one float: below 2^-31);
// e^y = 2^(k >> 8) T_j (1 + p), T_j = 2^(j/256) from the fp64 table, split.
__device__ __forceinline__ F2 exp_f2(F2 y)
{
    const bool lo = y.h < -80.f, hi = y.h > 80.f;
    const float yh = lo ? -80.f : (hi ? 80.f : y.h), yl = (lo || hi) ? 0.f : y.l;
    const float tf = __fmaf_rn(yh, kInvLn2o256F, kShiftF);
    const int k = __float_as_int(tf) - kShiftBits;
    const float kf = __fsub_rn(tf, kShiftF);                          // k exactly
    const float a = __fsub_rn(yh, __fmul_rn(kf, kLn2o256F3[0]));     // exact (Sterbenz)
    const F2 p2 = two_prod(kf, kLn2o256F3[1]);
    // r = a + yl - k C2 - k C3: the two larger additions exact, the small rest in one float
    const F2 s1 = two_sum(a, yl);
    const F2 t = two_sum(s1.h, -p2.h);
    const float rl = __fsub_rn(__fsub_rn(__fadd_rn(t.l, s1.l), p2.l), __fmul_rn(kf, kLn2o256F3[2]));
    const F2 r = fast_two_sum(t.h, rl);
    F2 s = two_prod(r.h, r.h);                                         // r^2
    s.l = __fmaf_rn(2.f * r.h, r.l, s.l);
    const float c3 = __fmul_rn(__fmul_rn(s.h, r.h),
                               __fmaf_rn(r.h, __fmaf_rn(r.h, 1.f / 120.f, 1.f / 24.f), kSixthF[0]));
    F2 P = fast_two_sum(r.h, 0.5f * s.h);
    P = fast_two_sum(P.h, __fadd_rn(__fadd_rn(P.l, r.l), __fmaf_rn(0.5f, s.l, c3)));
    const F2 T = split_d(__ldg(&kExp2Tab[k & 255]));
    const F2 e = ff_fma(T, P, T);
    const float sc = __int_as_float((127 + (k >> 8)) << 23);          // 2^(k >> 8), |k >> 8| <= 116
    return F2{__fmul_rn(e.h, sc), __fmul_rn(e.l, sc)};
}

// log z of a positive float pair on the fp32 pipe alone, absolute error about
// 2^-47 (1 + |log z|), for z.h a normal float below 2^127 (with z.l normal or zero; below
// z ~ 2^-102 the low float is subnormal and z itself holds fewer bits): z = 2^e m, m in [1, 2) (both parts scaled
// exactly), j = the top eight bits of m's fraction, r = m i_j - 1 with i_j = RN_float(1/c_j)
// (|r| < 2^-8.9), log z = e ln2 - log(i_j) + log(1 + r),
// log(1 + r) = r - r^2/2 (float pair) + r^3/3 - r^4/4 + r^5/5 (one float: below 2^-27);
// e ln2 with ln2 = H1 + H2 + H3 (H1 has 16 bits: e H1 exact; e H2 by two-product).
__device__ __forceinline__ F2 log_f2(F2 z)
{
    const unsigned bits = __float_as_uint(z.h);
    const int e = (int)(bits >> 23) - 127;
    const int j = (int)((bits >> 15) & 255u);
    const float mh = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);
    const float ml = __fmul_rn(z.l, __uint_as_float((unsigned)(127 - e) << 23));
    const float ic = __ldg(&kLogInvTabF[j]);
    const F2 pr = two_prod(mh, ic);
    // r = (pr.h - 1) + pr.l + ml ic, pr.h - 1 exact: the larger additions exact
    const F2 q = two_prod(ml, ic);
    const F2 u = two_sum(pr.l, q.h);
    F2 r = two_sum(__fsub_rn(pr.h, 1.f), u.h);
    r = fast_two_sum(r.h, __fadd_rn(r.l, __fadd_rn(u.l, q.l)));
    F2 s = two_prod(r.h, r.h);
    s.l = __fmaf_rn(2.f * r.h, r.l, s.l);
    const float c3 = __fmul_rn(__fmul_rn(s.h, r.h), __fmaf_rn(r.h, __fmaf_rn(r.h, 0.2f, -0.25f), kThirdF[0]));
    F2 L = fast_two_sum(r.h, -0.5f * s.h);
    L = fast_two_sum(L.h, __fadd_rn(__fadd_rn(L.l, r.l), __fmaf_rn(-0.5f, s.l, c3)));
    const float ef = (float)e;
    const F2 e2 = two_prod(ef, kLn2F3[1]);
    const F2 b = two_sum(__fmul_rn(ef, kLn2F3[0]), e2.h);
    const F2 eln2 = fast_two_sum(b.h, __fadd_rn(b.l, __fmaf_rn(ef, kLn2F3[2], e2.l)));
    return ff_add(ff_add(eln2, split_d(__ldg(&kLogTabF[j]))), L);
}

// The per-bond outputs of the pair passes that the gather reads (dU_i/dr_ij and r_ij): the
// fp64 path stores them as float pairs (ff_pack of split_d, integer instructions) and its
// gather sums them in float-pair arithmetic; the fp32 path stores floats.  split_d turns inf
// and NaN into finite values, so an fp64 writer checks finiteness itself before storing.
__device__ __forceinline__ double bond_out(double x) { return ff_pack(split_d(x)); }
__device__ __forceinline__ float bond_out(float x) { return x; }

// x = x1 + x2 + x3 exactly, three floats (x1: 24 leading bits, x2: the next 23, x3: the last
// 6), for 2^-74 <= |x| < 2^128 (every part then a normal float or zero); the callers pass
// mantissas in [1, 4).
struct F3 {
    float a, b, c;
};
__device__ __forceinline__ F3 split3_d(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
    float b = __fmul_rn(int23_to_f((lo >> 6) & 0x7fffffu), __int_as_float((e - 46 + 127) << 23));
    float c = __fmul_rn(int23_to_f(lo & 63u), __int_as_float((e - 52 + 127) << 23));
    if (hi & 0x80000000u) {
        b = -b;
        c = -c;
    }
    return {d2f_trunc(x), b, c};
}

// 1/sqrt(x) for positive normal x within 1 ulp, two fp64 instructions.  x = m 2^(2h), m in
// [1, 4) (integer instructions), 1/sqrt(x) = 2^-h / sqrt(m).  For m: the fp32 seed y of
// rsqrt_nr (relative error below 2^-22), e = 1 - m y^2 formed exactly enough as a float pair
// (m split into three floats, y^2 and the products by two-product; m1 y^2 lies within 2^-21
// of 1, so its difference from 1 is exact), then m^(-1/2) = y (1 + e/2 + 3e^2/8) (the next
// term, 5e^3/16, is below 2^-64): y + y c, with y c by two-product, added in fp64 (the first
// addition exact, the second rounding once); 2^-h by integer instructions.  +inf below
// 2^-126, as rsqrt_nr.
__device__ __forceinline__ double rsqrt_ff(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
    const int odd = e & 1;
    const int h = (e - odd) / 2;
    const double md = __hiloint2double((int)((hi & 0x000fffffu) | ((unsigned)(0x3ff + odd) << 20)), (int)lo);
    const float mf = d2f_trunc(md);
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(mf));
    const F3 ms = split3_d(md);
    const F2 s = two_prod(y, y);                           // y^2 = s.h + s.l exactly
    const F2 p = two_prod(ms.a, s.h);                      // m1 y^2 head
    const F2 q1 = two_prod(ms.a, s.l);
    const F2 q2 = two_prod(ms.b, s.h);
    const F2 m1 = two_sum(q1.h, q2.h);
    const F2 m2 = two_sum(m1.h, p.l);
    const F2 E = two_sum(__fsub_rn(p.h, 1.f), m2.h);      // m y^2 - 1 = -e, head
    const float el = (((E.l + m1.l) + m2.l) + (q1.l + q2.l)) + __fmaf_rn(ms.b, s.l, __fmul_rn(ms.c, s.h));
    // c = e/2 + 3e^2/8 with e = -(E.h + el)
    const float ch = __fmul_rn(-0.5f, E.h);
    const float cl = __fmaf_rn(0.375f * E.h, E.h, __fmul_rn(-0.5f, el));
    const F2 t = two_prod(y, ch);
    // y + t.h is exact in fp64 (two floats 2^-21 apart in scale); the rest is rounded once
    const double v = (f2d_int(y) + f2d_int(t.h)) + f2d_int(__fmaf_rn(y, cl, t.l));
    const double r = __hiloint2double(__double2hiint(v) - (h << 20), __double2loint(v));
    return __double_as_longlong(x) < 0x3810000000000000ll ? __longlong_as_double(0x7ff0000000000000ll) : r;
}

// 1/x for normal x (|x| < 2^1022) within 1 ulp, two fp64 instructions: x = m 2^e, m in
// [1, 2) with x's sign, 1/x = 2^-e / m; for m the fp32 seed y of rcp_nr, e = 1 - m y as a
// float pair (m split into three floats; m1 y lies within 2^-21 of 1), then 1/m = y (1 + e +
// e^2) (the next term, e^3, is below 2^-63): y + y c added in fp64 as in rsqrt_ff; 2^-e by
// integer instructions.
__device__ __forceinline__ double rcp_ff(double x)
{
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023;
    const double md = __hiloint2double((int)((hi & 0x800fffffu) | 0x3ff00000u), (int)lo);
    const float mf = d2f_trunc(md);
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(mf));
    const F3 ms = split3_d(md);
    const F2 p = two_prod(ms.a, y);
    const F2 q = two_prod(ms.b, y);
    const F2 m = two_sum(q.h, p.l);
    const F2 E = two_sum(__fsub_rn(p.h, 1.f), m.h);       // m y - 1 = -e, head
    const float el = ((E.l + m.l) + q.l) + __fmul_rn(ms.c, y);
    // c = e + e^2 with e = -(E.h + el)
    const float ch = -E.h;
    const float cl = __fmaf_rn(E.h, E.h, -el);
    const F2 t = two_prod(y, ch);
    const double v = (f2d_int(y) + f2d_int(t.h)) + f2d_int(__fmaf_rn(y, cl, t.l));
    return __hiloint2double(__double2hiint(v) - (e << 20), __double2loint(v));
}

// 1/x for 1.2e-38 < |x| < 8.5e37 (x and 1/x normal in fp32): an fp32 seed y
// (rcp.approx on the value truncated to fp32 with integer instructions, relative error
// e = 1 - x y below 2^-21), then one third-order step y (1 + e + e^2), for which
// x y (1 + e + e^2) = 1 - e^3: relative error below 2^-63 before the final rounding.
// Three fp64 FMAs, within 1 ulp.  Used for the Tersoff
// angular denominator d^2 + (h - cos)^2, zeta (1 + (beta zeta)^n) and the SW 1/(r - a sigma)
// (whose magnitude is at least 1/(a sigma) and at most 1/(fp64 rounding of r - a sigma)).
__device__ __forceinline__ double rcp_nr(double x)
{
    const float xf = d2f_trunc(x);
    float yf;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
    const double y = f2d_int(yf);
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// 1/sqrt(x) for 1.2e-38 < x < 3.4e38 (x normal in fp32): an fp32 seed y (rsqrt.approx on
// x truncated to fp32 with integer instructions, relative error below 2^-22), then one
// step of the series x^(-1/2) = y (1 - e)^(-1/2) = y (1 + e/2 + 3e^2/8 + 5e^3/16 + ...),
// e = 1 - x y^2, cut after e^2: relative error 5e^3/16 < 2^-64 before the final rounding.
// y^2 is exact (y has 24 significant bits), so e carries a single rounding.  Five fp64
// instructions, within 1 ulp.  Used for 1/r of every bond (r^2 of a bond is far inside
// the domain).
__device__ __forceinline__ double rsqrt_nr(double x)
{
    const float xf = d2f_trunc(x);
    float yf;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(yf) : "f"(xf));
    const double y = f2d_int(yf);
    const double e = fma(-x, y * y, 1.0);
    const double r = fma(y, e * fma(e, 0.375, 0.5), y);
    // below the fp32 normal range (only a zero bond, i.e. coincident atoms, gets there) the
    // seed is not finite: return +inf, as 1/sqrt(+0) is, so that the forces turn non-finite
    // and the step reports it (integer compare: x's bit pattern below that of 2^-126)
    return __double_as_longlong(x) < 0x3810000000000000ll ? __longlong_as_double(0x7ff0000000000000ll) : r;
}

// a < b for a, b >= +0 (not NaN): non-negative doubles order like their bit patterns read
// as integers, so the comparison runs on the integer pipe
__device__ __forceinline__ bool lt_nonneg(double a, double b)
{
    return __double_as_longlong(a) < __double_as_longlong(b);
}
__device__ __forceinline__ bool lt_nonneg(float a, float b) { return a < b; }

// 0 < x <= +inf for x >= +0 or NaN (the bit pattern read as an integer), on the integer pipe
__device__ __forceinline__ bool positive_nonneg(double x)
{
    return (unsigned long long)__double_as_longlong(x) - 1ull < 0x7ff0000000000000ull;
}
__device__ __forceinline__ bool positive_nonneg(float x) { return x > 0.f; }

// max(x, -700) for x < 0: for negative doubles the larger magnitude has the larger bit
// pattern read as a signed integer.  (A positive x, which only r rounded up to the
// cutoff could give, also becomes -700.)
__device__ __forceinline__ double clamp_neg700(double x)
{
    constexpr long long kNeg700 = (long long)0xc085e00000000000ull;   // -700.0
    return __double_as_longlong(x) > kNeg700 ? -700.0 : x;
}

}  // namespace mdk
