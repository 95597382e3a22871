// lbm_core.cuh -- lattice traits, the per-problem parameter block and the
// Peng-Robinson thermodynamics shared by every kernel of the library.
//
// Paper: Soomro & Ayala, arXiv 2306.10652.
//   Sec. 2.3, Eq. (9)   PR mixture pressure
//   Sec. 2.3, Eqs. (10)-(11)  van der Waals mixing rules with delta_ij
//   Sec. 2.3, Eq. (12)  PR fugacity
//   Sec. 2.1, Eq. (1b), (1c)  well-balanced equilibrium and forcing
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbmfug {

constexpr int kMaxNc = 16;
constexpr double kCs2 = 1.0 / 3.0;

// ---------------------------------------------------------------------------
// Lattices.  Velocities are ordered rest first, then opposite pairs
// (2k-1, 2k) with e_{2k} = -e_{2k-1}; gradients are summed pair by pair.
// ---------------------------------------------------------------------------
template <int LAT> struct Lattice;

template <> struct Lattice<0> {  // D2Q9
    static constexpr int D = 2;
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int e(int a, int d)
    {
        constexpr int E[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                 {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
        return E[a][d];
    }
    __host__ __device__ static constexpr double w(int a)
    {
        return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

template <> struct Lattice<1> {  // D3Q19
    static constexpr int D = 3;
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int e(int a, int d)
    {
        constexpr int E[19][3] = {{0, 0, 0},   {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
                                  {0, 0, 1},   {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0},  {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},   {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
        return E[a][d];
    }
    __host__ __device__ static constexpr double w(int a)
    {
        return a == 0 ? 1.0 / 3.0 : (a < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

// ---------------------------------------------------------------------------
// Per-problem constants, computed once on the host (T is fixed per problem,
// so the temperature function alpha_i and every pair product are constant).
// ---------------------------------------------------------------------------
struct Params {
    int nx, ny, nz, nc;
    long long N;        // nodes
    double RT, lnRT;    // R T and ln(R T)
    double omega;       // 1 / tau
    double b[kMaxNc];       // co-volumes b_i
    double invM[kMaxNc];    // 1 / M_i
    double sqk[kMaxNc];     // sqrt(kappa_i), Eq. (4) and Eq. (6)
    double rhobar[kMaxNc];  // reference density of the deviation storage
    double A[kMaxNc * kMaxNc];  // sqrt((a alpha)_i (a alpha)_j) (1 - delta_ij), Eq. (10)
    // binary32 copies for kernels whose thermodynamics run in binary32
    float fRT, flnRT;
    float fb[kMaxNc], finvM[kMaxNc], fsqk[kMaxNc], frhobar[kMaxNc];
    float fA[kMaxNc * kMaxNc];
    // double-binary32 (hi, lo) constants of the df64 thermodynamics
    // (lbm_thermo_df.cuh), molar masses folded in
    float2 dM[kMaxNc];           // 1 / M_i
    float2 dB[kMaxNc];           // b_i / M_i
    float2 db[kMaxNc];           // b_i
    float2 dA[kMaxNc * kMaxNc];  // A_ij / M_j
    float4 dAp[kMaxNc / 2 * kMaxNc];  // rows 2r, 2r+1 side by side: (hi_2r, hi_2r+1, lo_2r, lo_2r+1) at column j
    float2 dRK[kMaxNc];          // RT (ln RT - ln M_i)
    float2 dsqk[kMaxNc];         // sqrt(kappa_i)
    float2 dPk[kMaxNc];          // sqrt(kappa_j) / M_j
    float2 dRT;                  // RT
    float4 dPBp[kMaxNc];         // (dPk_j hi, dB_j hi, dPk_j lo, dB_j lo): psi and B in one packed sum
    float4 logtab[128];          // df64 logarithm table (lbm_df64.cuh)
};

// Parameter access in the arithmetic type E of a kernel.
template <typename E> struct PV;
template <> struct PV<double> {
    __device__ static double A(const Params &P, int k) { return P.A[k]; }
    __device__ static double b(const Params &P, int i) { return P.b[i]; }
    __device__ static double RT(const Params &P) { return P.RT; }
    __device__ static double lnRT(const Params &P) { return P.lnRT; }
    __device__ static double sqk(const Params &P, int i) { return P.sqk[i]; }
    __device__ static double invM(const Params &P, int i) { return P.invM[i]; }
    __device__ static double rhobar(const Params &P, int i) { return P.rhobar[i]; }
};
template <> struct PV<float> {
    __device__ static float A(const Params &P, int k) { return P.fA[k]; }
    __device__ static float b(const Params &P, int i) { return P.fb[i]; }
    __device__ static float RT(const Params &P) { return P.fRT; }
    __device__ static float lnRT(const Params &P) { return P.flnRT; }
    __device__ static float sqk(const Params &P, int i) { return P.fsqk[i]; }
    __device__ static float invM(const Params &P, int i) { return P.finvM[i]; }
    __device__ static float rhobar(const Params &P, int i) { return P.frhobar[i]; }
};

// ---------------------------------------------------------------------------
// Eqs. (9)-(12) at one node from the molar densities rm[i] = rho~_i.
//
// With x_i = rho~_i / rho~, B = b_m rho~ and Z = p / (rho~ RT), Eq. (12)
// plus ln(x_i p) reads
//   ln f_i = ln rho~_i + [ln RT - ln(1 - B)] + b_i C1 + S_i C2,
//   C1 = (Z - 1)/b_m + (a alpha)_m Lr / (2 sqrt2 b_m^2 RT),
//   C2 = -Lr / (sqrt2 b_m RT),
//   Lr = ln[(1 + (1+sqrt2) B) / (1 + (1-sqrt2) B)],
//   S_i = sum_j x_j (a alpha)_ij,
// which is the printed equation regrouped (the two p's cancel, so it holds
// for p <= 0 too).  Every operation is in the arithmetic type E.
// ---------------------------------------------------------------------------
// Quotient and logarithm in the arithmetic type of a kernel: binary64 uses
// the correctly rounded operations; binary32 thermodynamics use the
// hardware approximations __fdividef (2 ulp) and __logf (absolute error
// 2^-21.41 on [0.5, 2], 3 ulp elsewhere).
__device__ __forceinline__ double tdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float tdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double tlog(double x) { return log(x); }
__device__ __forceinline__ float tlog(float x) { return __logf(x); }

// Constants of pr_lnf seen through a view: A(i, j) = (a alpha)_ij at the
// problem's temperature, b(i), RT() and lnRT().  ParamsView reads a single
// problem's block; the batched form supplies one per job (its own T).
template <typename E> struct ParamsView {
    const Params &P;
    __device__ E A(int i, int j) const { return PV<E>::A(P, i * kMaxNc + j); }
    __device__ E b(int i) const { return PV<E>::b(P, i); }
    __device__ E RT() const { return PV<E>::RT(P); }
    __device__ E lnRT() const { return PV<E>::lnRT(P); }
};

template <int NC, typename E, typename View>
__device__ __forceinline__ void pr_lnf_v(const View &V, const E (&rm)[NC], E (&lnf)[NC], E *p_out)
{
    const E kSqrt2 = (E)1.4142135623730951;
    E rho = 0;
#pragma unroll
    for (int i = 0; i < NC; ++i) rho += rm[i];
    const E inv = tdiv((E)1, rho);
    E x[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) x[i] = rm[i] * inv;
    E bm = 0;
#pragma unroll
    for (int i = 0; i < NC; ++i) bm = fma(x[i], V.b(i), bm);
    E S[NC];
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        E s = 0;
#pragma unroll
        for (int j = 0; j < NC; ++j) s = fma(V.A(i, j), x[j], s);
        S[i] = s;
    }
    E am = 0;
#pragma unroll
    for (int i = 0; i < NC; ++i) am = fma(x[i], S[i], am);
    const E RT = V.RT();
    const E B = bm * rho;
    const E omB = (E)1 - B;
    const E den = fma(B, (E)2 - B, (E)1);  // 1 + 2B - B^2
    const E amr = tdiv(am * rho, RT);
    const E Zm1 = tdiv(B, omB) - tdiv(amr, den);
    const E Lr = tlog(tdiv(fma((E)1 + kSqrt2, B, (E)1), fma((E)1 - kSqrt2, B, (E)1)));
    const E C0 = V.lnRT() - tlog(omB);
    const E invbm = tdiv((E)1, bm);
    const E C1 = Zm1 * invbm + tdiv(am * Lr * invbm * invbm, (E)2 * kSqrt2 * RT);
    const E C2 = tdiv(-Lr * invbm, kSqrt2 * RT);
#pragma unroll
    for (int i = 0; i < NC; ++i) lnf[i] = tlog(rm[i]) + C0 + fma(V.b(i), C1, S[i] * C2);
    if (p_out) *p_out = RT * rho / omB - am * rho * rho / den;
}

template <int NC, typename E = double>
__device__ __forceinline__ void pr_lnf(const Params &P, const E (&rm)[NC], E (&lnf)[NC], E *p_out)
{
    pr_lnf_v<NC, E>(ParamsView<E>{P}, rm, lnf, p_out);
}

// Error-free binary32 transformations (Knuth TwoSum, Dekker fast TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}
// compensated accumulation (s, c) += x
__device__ __forceinline__ void acc_add(float &s, float &c, float x)
{
    float e;
    two_sum(s, x, s, e);
    c += e;
}
// (hi, lo) + (s, c), renormalised
__device__ __forceinline__ void pair_add(float &hi, float &lo, float s, float c)
{
    float h, e;
    two_sum(hi, s, h, e);
    const float l = lo + (e + c);
    hi = h + l;
    lo = l - (hi - h);
}

// periodic neighbour index
__device__ __forceinline__ int wrap(int v, int n)
{
    v = v % n;
    return v < 0 ? v + n : v;
}

}  // namespace lbmfug
