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
