// Double-float ("f32x2") arithmetic: a value is an unevaluated sum hi + lo of
// two binary32 numbers with |lo| <= ulp(hi)/2, which carries about 48
// significant bits.  On GB300 the FP32 units issue 64 times as many
// operations per clock as the FP64 units, so the pointwise functional of the
// FP64 path runs in this representation (pointwise.cuh, pw_point_f2).
//
// Building blocks (error-free transformations):
//   two_sum       Knuth's TwoSum (TAOCP vol. 2, 4.2.2)
//   fast_two_sum  Dekker's Fast2Sum (Numer. Math. 18, 1971), |a| >= |b|
//   two_prod      exact product with one FMA
// Double-word sums and products follow Joldes, Muller, Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic"
// (ACM TOMS 44, 2017): add = AccurateDWPlusDW (relative error <= 3u^2),
// add(f2, float) = DWPlusFP, mul = DWTimesDW with FMA, mul(f2, float) =
// DWTimesFP with FMA; u = 2^-24.  Quotients and square roots take one
// correction step on the binary32 result (Karp and Markstein, ACM TOMS 23,
// 1997).  exp, expm1, log and n^(-1/3) are written below from their series
// and Newton iterations; each states its reduction.
//
// Every operation of an error-free transformation goes through fadd / fmul /
// ffma, which on the device are the round-to-nearest intrinsics that the
// compiler never contracts into an FMA.  Host builds must not contract either
// (the library is compiled with -ffp-contract=off on the host side).
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

namespace ofdft {
namespace ff {

#ifdef __CUDACC__
#define FF_HD __host__ __device__ __forceinline__
#define FF_CALL static __host__ __device__ __noinline__   // one copy of a long routine per kernel
#else
#define FF_HD inline
#define FF_CALL static inline
#endif

struct f2 {
    float hi, lo;
    f2() = default;
    FF_HD constexpr f2(float h, float l) : hi(h), lo(l) {}
    // nearest double-float to a binary64 (constants and host code)
    FF_HD constexpr explicit f2(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    FF_HD constexpr explicit f2(int i) : hi((float)i), lo(0.0f) {}   // exact for |i| < 2^24
};

// Complex double-float (the layout of a double2: 16 bytes).
struct cf2 {
    f2 x, y;
};

FF_HD float fadd(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
FF_HD float fsub(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
FF_HD float fmul(float a, float b)
{
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
FF_HD float ffma(float a, float b, float c)
{
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}

FF_HD f2 two_sum(float a, float b)
{
    float s = fadd(a, b);
    float bb = fsub(s, a);
    float e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
    return {s, e};
}

FF_HD f2 fast_two_sum(float a, float b)
{
    float s = fadd(a, b);
    float e = fsub(b, fsub(s, a));
    return {s, e};
}

FF_HD f2 two_prod(float a, float b)
{
    float p = fmul(a, b);
    return {p, ffma(a, b, -p)};
}

// binary32 -> binary64 by rebuilding the bit pattern (exact; zero and
// subnormal inputs give zero, inf and NaN stay so): integer operations only,
// where the conversion instruction would occupy the FP64 unit.
FF_HD double widen_bits(float f)
{
#ifdef __CUDA_ARCH__
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(u & 0x80000000u) << 32;
    if (e == 0u) return __longlong_as_double((long long)sign);
    const uint64_t de = e == 0xffu ? 0x7ffull : (uint64_t)(e + 896u);
    return __longlong_as_double((long long)(sign | (de << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
#else
    return (double)f;
#endif
}

// Conversions.  from_double rounds to the nearest double-float (error
// <= 2^-48 relative); to_double returns hi + lo rounded to binary64, with
// one binary64 addition.
FF_HD f2 from_double(double d)
{
    float h = (float)d;
    return {h, (float)(d - (double)h)};
}
FF_HD double to_double(f2 x) { return widen_bits(x.hi) + widen_bits(x.lo); }

// Compile-time constant split of a double: the constexpr local makes the
// compiler fold the split (a plain call of the constexpr constructor inside
// an expression may be evaluated at run time, by the FP64 units).
constexpr f2 cst_split(double d) { return f2(d); }
#define FFC(d) ([] { constexpr ::ofdft::ff::f2 k_ = ::ofdft::ff::cst_split(d); return k_; }())

FF_HD f2 neg(f2 x) { return {-x.hi, -x.lo}; }

FF_HD float int_bits_float(uint32_t b)
{
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, 4);
    return f;
#endif
}

// 2^k as a binary32 for -126 <= k <= 127.
FF_HD float pow2i(int k) { return int_bits_float((uint32_t)(k + 127) << 23); }

// AccurateDWPlusDW: relative error <= 3u^2 even under cancellation.
FF_HD f2 add(f2 x, f2 y)
{
    f2 s = two_sum(x.hi, y.hi);
    f2 t = two_sum(x.lo, y.lo);
    float c = fadd(s.lo, t.hi);
    f2 v = fast_two_sum(s.hi, c);
    float w = fadd(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}
FF_HD f2 sub(f2 x, f2 y) { return add(x, neg(y)); }

// DWPlusFP: relative error <= 2u^2.
FF_HD f2 add(f2 x, float b)
{
    f2 s = two_sum(x.hi, b);
    float v = fadd(x.lo, s.lo);
    return fast_two_sum(s.hi, v);
}

// DWTimesDW with FMA: relative error <= 5u^2.
FF_HD f2 mul(f2 x, f2 y)
{
    f2 c = two_prod(x.hi, y.hi);
    float t = fmul(x.lo, y.lo);
    t = ffma(x.hi, y.lo, t);
    t = ffma(x.lo, y.hi, t);
    return fast_two_sum(c.hi, fadd(c.lo, t));
}

// DWTimesFP with FMA: relative error <= 2u^2.
FF_HD f2 mul(f2 x, float b)
{
    f2 c = two_prod(x.hi, b);
    float t = ffma(x.lo, b, c.lo);
    return fast_two_sum(c.hi, t);
}

// Exact scaling by a power of two (no underflow or overflow in range).
FF_HD f2 scale(f2 x, float p2) { return {fmul(x.hi, p2), fmul(x.lo, p2)}; }

// SloppyDWPlusDW: absolute error a few u^2 (|x| + |y|) (no relative bound
// under cancellation) -- enough for sums whose error is judged against the
// size of the operands, as in FFT butterflies.
FF_HD f2 add_s(f2 x, f2 y)
{
    f2 s = two_sum(x.hi, y.hi);
    float t = fadd(x.lo, y.lo);
    return fast_two_sum(s.hi, fadd(s.lo, t));
}

// a b - c d as one double-float: both leading products exact (TwoProd),
// their difference by TwoSum, every lower-order product and error term
// gathered in one binary32 chain, one final Fast2Sum.  Absolute error a few
// u^2 (|a b| + |c d|), as a DD product and a DD sum would give, in about
// two thirds of their instructions.
FF_HD f2 dot2_sub(f2 a, f2 b, f2 c, f2 d)
{
    const f2 p = two_prod(a.hi, b.hi), q = two_prod(c.hi, d.hi);
    const f2 s = two_sum(p.hi, -q.hi);
    float t = fsub(p.lo, q.lo);
    t = ffma(a.hi, b.lo, t);
    t = ffma(a.lo, b.hi, t);
    t = ffma(-c.hi, d.lo, t);
    t = ffma(-c.lo, d.hi, t);
    return fast_two_sum(s.hi, fadd(s.lo, t));
}

// Complex double-float product (the FFT's twiddle multiply): each part one
// dot2_sub.
FF_HD cf2 cmul(cf2 a, cf2 b)
{
    cf2 r;
    r.x = dot2_sub(a.x, b.x, a.y, b.y);
    r.y = dot2_sub(a.x, b.y, neg(a.y), b.x);
    return r;
}

// Arithmetic operators for generic (FFT, G-space) code: sums use add_s.
FF_HD f2 operator+(f2 x, f2 y) { return add_s(x, y); }
FF_HD f2 operator-(f2 x, f2 y) { return add_s(x, neg(y)); }
FF_HD f2 operator-(f2 x) { return neg(x); }
FF_HD f2 operator*(f2 x, f2 y) { return mul(x, y); }
FF_HD f2 &operator+=(f2 &x, f2 y) { return x = add_s(x, y); }
FF_HD bool operator>(f2 x, f2 y) { return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo); }

// Binary64 -> double-float with integer operations only: hi takes the
// leading 24 significand bits (truncated), lo the next 23 (exact, built with
// the 2^23 trick); the 6 bits left are dropped (relative error < 2^-46).
// Magnitudes below 2^-126 (and zero) give zero; beyond the binary32 range
// inf of the same sign, NaN for NaN, with lo = 0.  The result is a
// valid double-float with |lo| < ulp(hi).
FF_HD f2 split_int(double d)
{
    uint64_t b;
#ifdef __CUDA_ARCH__
    b = (uint64_t)__double_as_longlong(d);
#else
    memcpy(&b, &d, 8);
#endif
    const uint32_t top = (uint32_t)(b >> 32);
    const int E = (int)((top >> 20) & 0x7ff) - 1023;
    const uint32_t sign = top & 0x80000000u;
    if (E < -126) return f2(0.0f, 0.0f);
    if (E > 127) {
        // beyond the binary32 range: inf of the sign, NaN for NaN (built from
        // bits: a conversion instruction would run on the FP64 units, and the
        // compiler may evaluate this branch for every element)
        const bool nan = E == 1024 && (b & 0xfffffffffffffull) != 0;
        return f2(int_bits_float(nan ? 0x7fc00000u : (sign | 0x7f800000u)), 0.0f);
    }
    const uint32_t hib = sign | ((uint32_t)(E + 127) << 23) | (uint32_t)((b >> 29) & 0x7fffffu);
    const uint32_t lint = (uint32_t)(b >> 6) & 0x7fffffu;    // significand bits 28..6
    float lo = fsub(int_bits_float(0x4b000000u | lint), 8388608.0f);   // exact integer < 2^23
    lo = fmul(fmul(lo, 1.4210854715202004e-14f), pow2i(E));              // * 2^-46 * 2^E
    return f2(int_bits_float(hib), sign ? -lo : lo);
}

// p u + c for a Horner step with a binary32 variable: absolute error a few
// u^2 (|p u| + |c|), which is what a polynomial evaluation needs.
FF_HD f2 fma_step(f2 p, float u, f2 c)
{
    f2 m = two_prod(p.hi, u);
    float ml = ffma(p.lo, u, m.lo);
    f2 s = two_sum(m.hi, c.hi);
    float w = fadd(s.lo, fadd(ml, c.lo));
    return fast_two_sum(s.hi, w);
}


// x / y: binary32 quotient q1, remainder r = x - q1 y in double-float, then
// q1 + r/y.  Relative error a few u^2.
FF_HD f2 div(f2 x, f2 y)
{
    float q1 = x.hi / y.hi;
    f2 r = sub(x, mul(y, q1));
    float q2 = r.hi / y.hi;
    return fast_two_sum(q1, q2);
}
FF_HD f2 recip(f2 y) { return div(f2{1.0f, 0.0f}, y); }
FF_HD f2 operator/(f2 x, f2 y) { return div(x, y); }

// sqrt(x), x > 0: s = binary32 root, then s + (x - s^2)/(2 s).
FF_HD f2 sqrt(f2 x)
{
    float s = sqrtf(x.hi);
    f2 r = sub(x, two_prod(s, s));
    return fast_two_sum(s, r.hi / (2.0f * s));
}

// e^r - 1 for |r| <= 0.35.  With s = r/8 (|s| <= 0.044) the Taylor series
// e^s - 1 = s (1 + s/2 + s^2/6 + s^3/24 + s^4 q(s)), q = 1/120 + s/720 +
// s^2/5040 + s^3/40320, truncation below 2e-18 relative; the s^4 q tail is
// below 3e-8 of the sum and is kept in binary32.  The low part of s enters
// through d/ds (e^s - 1) = 1 + (e^s - 1).  Three doublings
// E(2s) = E(s) (E(s) + 2) then give e^r - 1 without cancellation.
FF_HD f2 expm1_reduced(f2 r)
{
    const float sh = fmul(r.hi, 0.125f), sl = fmul(r.lo, 0.125f);
    const float q = ffma(ffma(ffma(sh, 1.0f / 40320.0f, 1.0f / 5040.0f), sh, 1.0f / 720.0f), sh,
                         1.0f / 120.0f);
    f2 p = {q, 0.0f};
    p = fma_step(p, sh, FFC(1.0 / 24.0));
    p = fma_step(p, sh, FFC(1.0 / 6.0));
    p = fma_step(p, sh, f2{0.5f, 0.0f});
    p = fma_step(p, sh, f2{1.0f, 0.0f});
    f2 E = mul(p, sh);
    E = add(E, sl * (1.0f + E.hi));
#pragma unroll
    for (int k = 0; k < 3; ++k) E = mul(E, add(E, 2.0f));
    return E;
}

// e^x.  x = k ln2 + r with |r| <= ln2/2; ln2 is split into three parts, the
// first with 16 significant bits so that k * part exactly fits a binary32
// for |k| <= 128.  Returns 0 below x = -87 (e^-87 < 2^-125) — callers use
// it only where such a term is negligible.
constexpr double kLn2 = 0.69314718055994530942;
constexpr float kLn2A = 0.693145751953125f;   // ln2 to 16 bits: 22713 / 2^15
constexpr double kLn2Rest = kLn2 - 0.693145751953125;
constexpr float kLn2B = (float)kLn2Rest;
constexpr float kLn2C = (float)(kLn2Rest - (double)(float)kLn2Rest);

FF_CALL f2 exp(f2 x)
{
    if (x.hi < -87.0f) return {0.0f, 0.0f};
    const float k = rintf(x.hi * 1.44269504088896341f);
    f2 r = two_sum(fsub(x.hi, fmul(k, kLn2A)), x.lo);    // x.hi - k A is exact (Sterbenz)
    r = sub(r, two_prod(k, kLn2B));
    r = add(r, -fmul(k, kLn2C));
    f2 E = expm1_reduced(r);
    return scale(add(E, 1.0f), pow2i((int)k));
}

// e^x - 1 for x <= 0 (the functional's only use): the reduced series while
// |x| <= ln2/2, else e^x - 1, where e^x <= 0.71 leaves no cancellation.
FF_HD f2 expm1_neg(f2 x)
{
    if (x.hi > -0.3465f) return expm1_reduced(x);
    return add(exp(x), -1.0f);
}

// ln x for x > 0 (normal binary32 range): binary32 seed y0, then one Newton
// step on e^y = x written as y = y0 + log1p(d), d = x e^(-y0) - 1, with
// log1p(d) = d - d^2/2 (|d| ~ 1e-7, the d^3 term is below 1e-21).
FF_HD f2 log(f2 x)
{
    const float y0 = logf(x.hi);
    f2 d = add(mul(x, exp(f2{-y0, 0.0f})), -1.0f);
    const float c = fadd(d.hi, d.lo - 0.5f * d.hi * d.hi);
    return two_sum(y0, c);
}

// n^(-1/3) for n > 0 (normal binary32 range): binary32 seed y0, then
// y = y0 (1 - r)^(-1/3) = y0 (1 + r/3 + 2 r^2/9 + ...) with r = 1 - n y0^3
// formed in double-float (|r| ~ 1e-7, so the series to r^2 is exact to
// double-float rounding).
FF_HD f2 rcbrt(f2 n)
{
#ifdef __CUDA_ARCH__
    const float y0 = rcbrtf(n.hi);
#else
    const float y0 = 1.0f / cbrtf(n.hi);
#endif
    f2 y3 = mul(two_prod(y0, y0), y0);
    f2 r = add(neg(mul(n, y3)), 1.0f);
    const float c = r.hi * (1.0f / 3.0f + r.hi * (2.0f / 9.0f)) + r.lo * (1.0f / 3.0f);
    return fast_two_sum(y0, y0 * c);
}

}  // namespace ff
}  // namespace ofdft
