// lbm_df64.cuh -- double-binary32 ("df64") arithmetic on the FP32 pipe, and
// the Peng-Robinson chemical potentials of Eqs. (9)-(12) with the interface
// term of Eq. (5) evaluated in it.
//
// GB300 executes binary64 at about 1/64 of the binary32 rate, so the
// thermodynamics that must keep binary64 accuracy (the mixture parameters of
// Eqs. (10)-(11), the logarithmic fugacity terms of Eq. (12) and the
// chemical-potential differences that make the force of Eq. (5)) are carried
// as unevaluated sums hi + lo of two binary32 numbers.  The building blocks
// are the classical error-free transformations:
//   TwoSum      s + e = a + b exactly              (Knuth, TAOCP 2, 4.2.2)
//   FastTwoSum  s + e = a + b exactly if |a| >= |b| (Dekker 1971)
//   TwoProd     p + e = a * b exactly, e = fma(a, b, -p)
// Sums of products use compensated dot products (Ogita, Rump and Oishi
// 2005, "Dot2"); a quotient is refined once by its remainder.  The relative
// error of every derived quantity is about 2^-44 (binary64: 2^-53, binary32:
// 2^-24); the tests compare ln f_i, mu_i and the force with the binary64
// oracle at that level.
//
// The logarithm is table-driven (Tang's method): x = 2^k m, m in [1, 2); the
// top 7 bits of m pick c_j = 1 + (j + 1/2)/128 and a binary32 v_j ~ 1/c_j;
// m v_j = P + P' exactly (TwoProd), r = P - 1 is exact (Sterbenz), so
//   ln x = k ln2 - ln v_j + log1p(r) + P'/P,
// with -ln v_j tabulated in df64 (from binary64 on the host) and log1p(r),
// |r| <= 2^-8, as its Taylor series to r^5 (truncation below 2^-50).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

namespace lbmfug {
namespace df {

struct F2 {
    float hi, lo;
};

// binary32 split of a binary64 constant (host or device, constant-folded)
__host__ __device__ constexpr float hi_of(double x) { return (float)x; }
__host__ __device__ constexpr float lo_of(double x) { return (float)(x - (double)(float)x); }

// The intrinsics below are never contracted into a fused multiply-add, which
// the error-free transformations rely on.
__device__ __forceinline__ F2 two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    return {s, e};
}

// TwoSum of two non-negative numbers: FastTwoSum of the larger and the
// smaller, which is exact, so (s, e) equals two_sum's.  The operands are
// ordered by their bit patterns, which order non-negative binary32 numbers as
// their values and put a NaN above every number, so a NaN propagates.  Three
// additions on the FMA pipe and two integer min/max on the ALU pipe, against
// six additions.
__device__ __forceinline__ F2 two_sum_pos(float a, float b)
{
    const int ia = __float_as_int(a), ib = __float_as_int(b);
    const float big = __int_as_float(max(ia, ib)), small = __int_as_float(min(ia, ib));
    const float s = __fadd_rn(big, small);
    return {s, __fsub_rn(small, __fsub_rn(s, big))};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b)  // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ F2 two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ F2 norm(F2 a) { return fast_two_sum(a.hi, a.lo); }

// a + b.  Absolute error about 2^-48 (|a| + |b|) (the "sloppy" double-word
// sum); the callers need absolute, not relative, accuracy of sums.
__device__ __forceinline__ F2 add(F2 a, F2 b)
{
    const F2 s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ F2 neg(F2 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ F2 sub(F2 a, F2 b) { return add(a, neg(b)); }

// a * b, relative error about 2^-46
__device__ __forceinline__ F2 mul(F2 a, F2 b)
{
    const F2 p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}

__device__ __forceinline__ F2 mulf(F2 a, float b)
{
    const F2 p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

// binary32 reciprocal to about 1 ulp (the hardware approximation); callers
// refine or scale it so that its error stays below 2^-44 of the result
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// a / b: binary32 quotient refined once by the df64 remainder a - q b
__device__ __forceinline__ F2 div(F2 a, F2 b)
{
    const float r = rcp_approx(b.hi);
    const float q1 = __fmul_rn(a.hi, r);
    const F2 qb = two_prod(q1, b.hi);
    // a - q1 b: the leading parts cancel to within |q1 b| 2^-23
    const float rem = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, qb.hi), qb.lo), fmaf(-q1, b.lo, a.lo));
    const float q2 = __fmul_rn(rem, r);
    return fast_two_sum(q1, q2);
}

// Compensated sum of products sum_j c_j x_j (c_j, x_j in df64).
struct Dot {
    float s, c;
    __device__ __forceinline__ void first(F2 cj, F2 xj)
    {
        const F2 p = two_prod(cj.hi, xj.hi);
        s = p.hi;
        c = fmaf(cj.hi, xj.lo, fmaf(cj.lo, xj.hi, p.lo));
    }
    __device__ __forceinline__ void add(F2 cj, F2 xj)
    {
        const F2 p = two_prod(cj.hi, xj.hi);
        const F2 t = two_sum(s, p.hi);
        s = t.hi;
        c = __fadd_rn(c, __fadd_rn(t.lo, fmaf(cj.hi, xj.lo, fmaf(cj.lo, xj.hi, p.lo))));
    }
    // the product term itself (unnormalised), for callers that keep it
    __device__ __forceinline__ static F2 term(F2 cj, F2 xj)
    {
        const F2 p = two_prod(cj.hi, xj.hi);
        return {p.hi, fmaf(cj.hi, xj.lo, fmaf(cj.lo, xj.hi, p.lo))};
    }
    __device__ __forceinline__ void add_term(F2 t)
    {
        const F2 u = two_sum(s, t.hi);
        s = u.hi;
        c = __fadd_rn(c, __fadd_rn(u.lo, t.lo));
    }
    __device__ __forceinline__ F2 value() const { return fast_two_sum(s, c); }
};

// Dot for sums whose products c_j.hi x_j.hi are all non-negative (the
// mixture sums of Eqs. 4, 10 and 11: positive parameters times positive
// densities): the same operations as Dot with two_sum_pos for the running
// sum, so the same result.
struct DotPos {
    float s, c;
    __device__ __forceinline__ void first(F2 cj, F2 xj)
    {
        const F2 p = two_prod(cj.hi, xj.hi);
        s = p.hi;
        c = fmaf(cj.hi, xj.lo, fmaf(cj.lo, xj.hi, p.lo));
    }
    __device__ __forceinline__ void add(F2 cj, F2 xj)
    {
        const F2 p = two_prod(cj.hi, xj.hi);
        const F2 t = two_sum_pos(s, p.hi);
        s = t.hi;
        c = __fadd_rn(c, __fadd_rn(t.lo, fmaf(cj.hi, xj.lo, fmaf(cj.lo, xj.hi, p.lo))));
    }
    __device__ __forceinline__ void add_term(F2 t)  // t.hi >= 0
    {
        const F2 u = two_sum_pos(s, t.hi);
        s = u.hi;
        c = __fadd_rn(c, __fadd_rn(u.lo, t.lo));
    }
    __device__ __forceinline__ F2 value() const { return fast_two_sum(s, c); }
};

// Log table entry j: {v_j, -ln v_j (hi), -ln v_j (lo), 0}.
constexpr int kLogTab = 128;

constexpr double kLn2 = 0.693147180559945309417232121458;

// Views of the table: its float4 entries, or the same values split into
// {v_j, -ln v_j hi} pairs and the lo words (1.5 KB of shared memory, not 2).
struct TabF4 {
    const float4 *__restrict__ p;
    __device__ __forceinline__ float3 operator[](int j) const
    {
        const float4 t = p[j];
        return make_float3(t.x, t.y, t.z);
    }
};
struct TabSplit {
    const float2 *__restrict__ vt;
    const float *__restrict__ tl;
    __device__ __forceinline__ float3 operator[](int j) const
    {
        const float2 a = vt[j];
        return make_float3(a.x, a.y, tl[j]);
    }
};

// ln(x.hi + x.lo) for x.hi a positive normal binary32 number (NaN otherwise),
// unnormalised result.  ln(hi + lo) = ln hi + lo/hi to 2^-49.
template <typename Tab>
__device__ __forceinline__ F2 log(F2 x, Tab tab)
{
    const int u = __float_as_int(x.hi);
    const int ex = u >> 23;  // biased exponent (x > 0)
    const float kf = __fsub_rn(__int_as_float(0x4b000000 + ex), 8388608.0f + 127.0f);
    const float m = __int_as_float((u & 0x007fffff) | 0x3f800000);
    const float3 t = tab[(u >> 16) & 0x7f];
    const F2 P = two_prod(m, t.x);
    const float r = __fsub_rn(P.hi, 1.0f);  // exact
    // first-order terms of the two small remainders: P.lo / P.hi and x.lo / x.hi
    const float corr = fmaf(P.lo, rcp_approx(P.hi), __fmul_rn(x.lo, rcp_approx(x.hi)));
    const F2 r2 = two_prod(r, r);
    const float r3 = __fmul_rn(r2.hi, r);
    const float tail = __fmul_rn(r3, fmaf(r, fmaf(r, 0.2f, -0.25f), 0.333333343f));
    const F2 h = fast_two_sum(r, __fmul_rn(-0.5f, r2.hi));  // r - r^2/2, |r| >= r^2/2
    const F2 kl = two_prod(kf, hi_of(kLn2));
    const F2 big = two_sum(kl.hi, t.y);
    const F2 s = two_sum(big.hi, h.hi);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(big.lo, s.lo), __fadd_rn(h.lo, t.z)),
                               __fadd_rn(fmaf(kf, lo_of(kLn2), kl.lo), fmaf(-0.5f, r2.lo, __fadd_rn(tail, corr))));
    // positive, normal and finite; NaN, infinity and non-positive densities give NaN
    const bool ok = x.hi >= 1.17549435e-38f && x.hi <= 3.40282347e38f;
    return {ok ? s.hi : __int_as_float(0x7fc00000), lo};
}

__device__ __forceinline__ F2 log(F2 x, const float4 *__restrict__ tab) { return log(x, TabF4{tab}); }

// ---- packed FP32x2 operations --------------------------------------------------
// One instruction does the binary32 operation on both lanes, each rounded as
// the scalar operation rounds it.  They are written in PTX with an explicit
// rounding mode, so that no compiler pass fuses a product into a following
// sum: the error-free transformations built on them need the same guarantee
// that __fmul_rn and __fadd_rn give the scalar routines.
__device__ __forceinline__ float2 vbc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return vadd(a, vneg(b)); }
__device__ __forceinline__ float2 vmul(float2 a, float2 b)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c)
{
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}

// Host: fill the log table (binary64 arithmetic; called once per problem).
inline void make_log_table(float *tab4)
{
    for (int j = 0; j < kLogTab; ++j) {
        const double c = 1.0 + (j + 0.5) / kLogTab;
        const float v = (float)(1.0 / c);
        const double T = -std::log((double)v);
        tab4[4 * j + 0] = v;
        tab4[4 * j + 1] = (float)T;
        tab4[4 * j + 2] = (float)(T - (double)(float)T);
        tab4[4 * j + 3] = 0.0f;
    }
}

}  // namespace df
}  // namespace lbmfug
