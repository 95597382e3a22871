// lbm_thermo_df.cuh -- the Peng-Robinson chemical potentials of one node in
// double-binary32 arithmetic (lbm_df64.cuh), for the binary32-storage kernels
// whose thermodynamics keep binary64 accuracy (LBM_FP32DEV).
//
// Paper: Soomro & Ayala, arXiv 2306.10652.
//   Sec. 2.1, Eq. (4)-(5)  interface term sum_j kappa_ij lap rho~_j with
//                          kappa_ij = sqrt(kappa_i kappa_j) = sqrt(kappa_i) lap psi,
//                          psi = sum_j sqrt(kappa_j) rho~_j
//   Sec. 2.2, Eq. (6)      kappa_i = kappa_ref a_i / a_ref
//   Sec. 2.3, Eqs. (9)-(12) PR mixture and fugacities
//
// Evaluated from the mass densities rho_j = h_j + l_j (the exact binary32
// pair of the state) with the molar masses folded into the constants
// (rho~_j = rho_j / M_j).  With B = b_m rho~ = sum_j (b_j / M_j) rho_j,
// T_i = rho~ S_i = sum_j (A_ij / M_j) rho_j and Q = rho~^2 (a alpha)_m =
// sum_i rho~_i T_i, the regrouped Eq. (12) (the printed form plus ln(x_i p),
// so that p cancels and it holds for p <= 0 too) reads
//   RT ln f_i = RT ln rho_i + RT (ln RT - ln M_i) - RT ln(1 - B)
//               + b_i RT C1 + T_i RT C2',
//   RT C1  = RT rho~ / (1 - B) + (Q / B) [Lr / (2 sqrt2 B) - 1 / (1 + 2B - B^2)],
//   RT C2' = -Lr / (sqrt2 B),  Lr = ln[(1 + (1 + sqrt2) B) / (1 + (1 - sqrt2) B)],
// and mu_i = RT ln f_i - sqrt(kappa_i) lap psi (Eq. 5 rewritten through
// Eq. 4).  Every step is a df64 operation; the result's absolute error is
// about 2^-44 of the largest term.
#pragma once

#include "lbm_core.cuh"
#include "lbm_df64.cuh"

namespace lbmfug {
namespace df {

__device__ __forceinline__ F2 f2(float2 v) { return {v.x, v.y}; }

// unnormalised product (for accumulation into a compensated sum)
__device__ __forceinline__ F2 mul_u(F2 a, F2 b)
{
    const F2 p = two_prod(a.hi, b.hi);
    return {p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo))};
}

// Two compensated dot products at once on the packed FP32x2 units: the
// lanes are rows 2r and 2r+1 of T_i = sum_j (A_ij / M_j) rho_j, with the
// same TwoProd / TwoSum steps as Dot, so each lane equals Dot's result.
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }

struct Dot2x {
    float2 s, c;
    __device__ __forceinline__ void first(float4 A, float xh, float xl)
    {
        const float2 X = make_float2(xh, xh), XL = make_float2(xl, xl);
        const float2 ch = make_float2(A.x, A.y), cl = make_float2(A.z, A.w);
        const float2 p = vmul(ch, X);
        const float2 pe = vfma(ch, X, pneg(p));
        s = p;
        c = vfma(ch, XL, vfma(cl, X, pe));
    }
    __device__ __forceinline__ void add(float4 A, float xh, float xl)
    {
        const float2 X = make_float2(xh, xh), XL = make_float2(xl, xl);
        const float2 ch = make_float2(A.x, A.y), cl = make_float2(A.z, A.w);
        const float2 p = vmul(ch, X);
        const float2 pe = vfma(ch, X, pneg(p));
        // TwoSum(s, p) lane by lane, as FastTwoSum of the larger and the
        // smaller (both non-negative: see two_sum_pos)
        const int sx = __float_as_int(s.x), sy = __float_as_int(s.y);
        const int px = __float_as_int(p.x), py = __float_as_int(p.y);
        const float2 big = make_float2(__int_as_float(max(sx, px)), __int_as_float(max(sy, py)));
        const float2 small = make_float2(__int_as_float(min(sx, px)), __int_as_float(min(sy, py)));
        const float2 t = vadd(big, small);
        const float2 e = vadd(small, pneg(vadd(t, pneg(big))));
        s = t;
        c = vadd(c, vadd(e, vfma(ch, XL, vfma(cl, X, pe))));
    }
};

// psi = sum_j sqrt(kappa_j) rho~_j at one node (Eq. 4)
template <int NC>
__device__ __forceinline__ F2 psi(const Params &P, const float (&h)[NC], const float (&l)[NC])
{
    DotPos d;
    d.first(f2(P.dPk[0]), {h[0], l[0]});
#pragma unroll
    for (int j = 1; j < NC; ++j) d.add(f2(P.dPk[j]), {h[j], l[j]});
    return d.value();
}

// D2Q9 lap X = (2/cs2) sum_a w_a (X(r + e_a) - X(r))
//            = (4 (faces) + (diagonals) - 20 X(r)) / 6
__device__ __forceinline__ F2 lap9(F2 c, F2 e, F2 w, F2 n, F2 s, F2 ne, F2 nw, F2 se, F2 sw)
{
    // the neighbours' psi are non-negative (Eq. 4): their running sum takes
    // two_sum_pos; the centre term, negative, the general TwoSum
    DotPos a;
    a.s = __fmul_rn(4.0f, e.hi);
    a.c = __fmul_rn(4.0f, e.lo);
    a.add_term({__fmul_rn(4.0f, w.hi), __fmul_rn(4.0f, w.lo)});
    a.add_term({__fmul_rn(4.0f, n.hi), __fmul_rn(4.0f, n.lo)});
    a.add_term({__fmul_rn(4.0f, s.hi), __fmul_rn(4.0f, s.lo)});
    a.add_term(ne);
    a.add_term(nw);
    a.add_term(se);
    a.add_term(sw);
    Dot b;
    b.s = a.s;
    b.c = a.c;
    const F2 c20 = two_prod(-20.0f, c.hi);
    b.add_term({c20.hi, fmaf(-20.0f, c.lo, c20.lo)});
    return mul(b.value(), {hi_of(1.0 / 6.0), lo_of(1.0 / 6.0)});
}

// mu_i = RT ln f_i - sqrt(kappa_i) lap psi for i < NC at one node
template <int NC>
__device__ __forceinline__ void mu(const Params &P, const float4 *__restrict__ tab, const float (&h)[NC],
                                   const float (&l)[NC], F2 lap, F2 (&out)[NC])
{
    constexpr double kS2 = 1.41421356237309504880168872421;
    // rho~_i and rho~ = sum_i rho~_i
    F2 y[NC];
    DotPos rt;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        y[i] = Dot::term(f2(P.dM[i]), {h[i], l[i]});
        if (i == 0) {
            rt.s = y[0].hi;
            rt.c = y[0].lo;
        } else {
            rt.add_term(y[i]);
        }
    }
    const F2 rho = rt.value();
    // Eq. (11) times rho~: B = b_m rho~
    DotPos bd;
    bd.first(f2(P.dB[0]), {h[0], l[0]});
#pragma unroll
    for (int j = 1; j < NC; ++j) bd.add(f2(P.dB[j]), {h[j], l[j]});
    const F2 B = bd.value();
    // Eq. (10): T_i = rho~ sum_j x_j (a alpha)_ij, Q = rho~^2 (a alpha)_m
    F2 T[NC];
#pragma unroll
    for (int r = 0; r < NC / 2; ++r) {  // rows 2r, 2r+1 on the two lanes
        Dot2x t;
        t.first(P.dAp[r * kMaxNc], h[0], l[0]);
#pragma unroll
        for (int j = 1; j < NC; ++j) t.add(P.dAp[r * kMaxNc + j], h[j], l[j]);
        T[2 * r] = fast_two_sum(t.s.x, t.c.x);
        T[2 * r + 1] = fast_two_sum(t.s.y, t.c.y);
    }
    if constexpr (NC % 2 == 1) {
        DotPos t;
        t.first(f2(P.dA[(NC - 1) * kMaxNc]), {h[0], l[0]});
#pragma unroll
        for (int j = 1; j < NC; ++j) t.add(f2(P.dA[(NC - 1) * kMaxNc + j]), {h[j], l[j]});
        T[NC - 1] = t.value();
    }
    DotPos qd;
    qd.first(y[0], T[0]);
#pragma unroll
    for (int i = 1; i < NC; ++i) qd.add(y[i], T[i]);
    const F2 Q = qd.value();
    // per-node terms of Eq. (12)
    const F2 one = {1.0f, 0.0f};
    const F2 omB = add(one, neg(B));
    const F2 den = add(one, mul(B, add({2.0f, 0.0f}, neg(B))));  // 1 + 2B - B^2
    const F2 N1 = add(one, mul(B, {hi_of(1.0 + kS2), lo_of(1.0 + kS2)}));
    const F2 N2 = add(one, mul(B, {hi_of(1.0 - kS2), lo_of(1.0 - kS2)}));
    const F2 Lr = norm(log(div(N1, N2), tab));
    const F2 lnomB = norm(log(omB, tab));
    const F2 u = div(one, B), v = div(one, omB), w = div(one, den);
    const F2 RT = f2(P.dRT);
    const F2 Lu = mul(Lr, u);
    const F2 RC1 = add(mul(mul(RT, rho), v),
                       mul(mul(Q, u), add(mul(Lu, {hi_of(0.5 / kS2), lo_of(0.5 / kS2)}), neg(w))));
    const F2 RC2 = mul(Lu, {hi_of(-1.0 / kS2), lo_of(-1.0 / kS2)});
    const F2 RG = mul(RT, lnomB);
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        Dot a;  // compensated sum of the terms of mu_i
        const F2 t0 = mul_u(RT, log({h[i], l[i]}, tab));
        a.s = t0.hi;
        a.c = t0.lo;
        a.add_term(f2(P.dRK[i]));
        a.add_term(neg(RG));
        a.add_term(mul_u(f2(P.db[i]), RC1));
        a.add_term(mul_u(T[i], RC2));
        a.add_term(neg(mul_u(f2(P.dsqk[i]), lap)));
        out[i] = a.value();
    }
}

// B = b_m rho~ = sum_j (b_j / M_j) rho_j at one node (Eq. 11), as mu() forms it
template <int NC>
__device__ __forceinline__ F2 mix_B(const Params &P, const float (&h)[NC], const float (&l)[NC])
{
    DotPos bd;
    bd.first(f2(P.dB[0]), {h[0], l[0]});
#pragma unroll
    for (int j = 1; j < NC; ++j) bd.add(f2(P.dB[j]), {h[j], l[j]});
    return bd.value();
}

// psi (Eq. 4) and B (Eq. 11) of one node in one packed sum: lane x is psi<NC>,
// lane y is mix_B<NC>, each with the operations of the scalar form.
template <int NC>
__device__ __forceinline__ void psi_and_B(const Params &P, const float (&h)[NC], const float (&l)[NC], F2 &psi,
                                          F2 &B)
{
    Dot2x t;
    t.first(P.dPBp[0], h[0], l[0]);
#pragma unroll
    for (int j = 1; j < NC; ++j) t.add(P.dPBp[j], h[j], l[j]);
    psi = fast_two_sum(t.s.x, t.c.x);
    B = fast_two_sum(t.s.y, t.c.y);
}


// mu of one node with rolled loops over the row pairs of T_i and over the
// components (the unrolled form above is a few thousand instructions of
// straight-line code at Nc = 10, more than the instruction cache holds).
// The same operations in the same order as mu(), so the result is bitwise
// that of mu().  B (Eq. 11, from mix_B or psi_and_B) comes in.  Per-thread
// scratch in shared memory with stride `pitch`: PH, PL [NC] floats (the
// density pair) and TS [NC] float2 (T_i as (hi, lo)); mu_i is written to
// out[i * ostride].  TS may be out itself (same stride): iteration i reads
// T_i before it stores mu_i.  Tab: a view of the log table (lbm_df64.cuh).
template <int NC, typename Tab>
__device__ __forceinline__ void mu_rolled(const Params &P, Tab tab, const float (&h)[NC], const float (&l)[NC],
                                          F2 B, F2 lap, float *PH, float *PL, float2 *TS, int pitch, float2 *out,
                                          int ostride)
{
    constexpr double kS2 = 1.41421356237309504880168872421;
    F2 y[NC];
    DotPos rt;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        PH[i * pitch] = h[i];
        PL[i * pitch] = l[i];
        y[i] = Dot::term(f2(P.dM[i]), {h[i], l[i]});
        if (i == 0) {
            rt.s = y[0].hi;
            rt.c = y[0].lo;
        } else {
            rt.add_term(y[i]);
        }
    }
    const F2 rho = rt.value();
#pragma unroll 1
    for (int r = 0; r < NC / 2; ++r) {
        Dot2x t;
        t.first(P.dAp[r * kMaxNc], h[0], l[0]);
#pragma unroll
        for (int j = 1; j < NC; ++j) t.add(P.dAp[r * kMaxNc + j], h[j], l[j]);
        const F2 a = fast_two_sum(t.s.x, t.c.x), b = fast_two_sum(t.s.y, t.c.y);
        TS[(2 * r) * pitch] = make_float2(a.hi, a.lo);
        TS[(2 * r + 1) * pitch] = make_float2(b.hi, b.lo);
    }
    if constexpr (NC % 2 == 1) {
        DotPos t;
        t.first(f2(P.dA[(NC - 1) * kMaxNc]), {h[0], l[0]});
#pragma unroll
        for (int j = 1; j < NC; ++j) t.add(f2(P.dA[(NC - 1) * kMaxNc + j]), {h[j], l[j]});
        const F2 v = t.value();
        TS[(NC - 1) * pitch] = make_float2(v.hi, v.lo);
    }
    auto Ti = [&](int i) -> F2 { return f2(TS[i * pitch]); };
    DotPos qd;
    qd.first(y[0], Ti(0));
#pragma unroll
    for (int i = 1; i < NC; ++i) qd.add(y[i], Ti(i));
    const F2 Q = qd.value();
    const F2 one = {1.0f, 0.0f};
    const F2 omB = add(one, neg(B));
    const F2 den = add(one, mul(B, add({2.0f, 0.0f}, neg(B))));  // 1 + 2B - B^2
    const F2 N1 = add(one, mul(B, {hi_of(1.0 + kS2), lo_of(1.0 + kS2)}));
    const F2 N2 = add(one, mul(B, {hi_of(1.0 - kS2), lo_of(1.0 - kS2)}));
    const F2 Lr = norm(log(div(N1, N2), tab));
    const F2 lnomB = norm(log(omB, tab));
    const F2 u = div(one, B), v = div(one, omB), w = div(one, den);
    const F2 RT = f2(P.dRT);
    const F2 Lu = mul(Lr, u);
    const F2 RC1 = add(mul(mul(RT, rho), v),
                       mul(mul(Q, u), add(mul(Lu, {hi_of(0.5 / kS2), lo_of(0.5 / kS2)}), neg(w))));
    const F2 RC2 = mul(Lu, {hi_of(-1.0 / kS2), lo_of(-1.0 / kS2)});
    const F2 RG = mul(RT, lnomB);
#pragma unroll 1
    for (int i = 0; i < NC; ++i) {
        Dot a;
        const F2 t0 = mul_u(RT, log({PH[i * pitch], PL[i * pitch]}, tab));
        a.s = t0.hi;
        a.c = t0.lo;
        a.add_term(f2(P.dRK[i]));
        a.add_term(neg(RG));
        a.add_term(mul_u(f2(P.db[i]), RC1));
        a.add_term(mul_u(Ti(i), RC2));
        a.add_term(neg(mul_u(f2(P.dsqk[i]), lap)));
        const F2 m = a.value();
        out[(long long)i * ostride] = make_float2(m.hi, m.lo);
    }
}

}  // namespace df
}  // namespace lbmfug
