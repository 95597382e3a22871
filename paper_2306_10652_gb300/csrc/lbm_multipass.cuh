// lbm_multipass.cuh -- the binary32 multi-pass step of LBM_FP32DEV on any
// lattice (D3Q19 has no single-pass kernel): double-binary32 thermodynamics,
// binary32 collision, exact density pairs.
//
// Paper: Soomro & Ayala, arXiv 2306.10652 -- Sec. 2.1, Eqs. (1a)-(1c), (3)-(5);
// Sec. 2.2, Eq. (6); Sec. 2.3, Eqs. (9)-(12).
//
// State: the Q-1 moving populations g[i][a-1][node] (binary32, post-streaming)
// and rho_i = hi + lo (exact binary32 pair), as in the other binary32 forms,
// plus psi = sum_j sqrt(kappa_j) rho~_j of the current state (df64, [N]).
// One step, three launches:
//   k_mp_mu      lap psi (isotropic stencil, df64) and mu_i = RT ln f_i -
//                sqrt(kappa_i) lap psi (lbm_thermo_df.cuh) -> mu [nc][N] (hi, lo)
//   k_mp_collide grad mu_i (differences of opposite neighbours taken on the
//                pairs and rounded once), F_i = -rho~_i grad mu_i, grad rho_i,
//                u = (sum e g + F/2)/rho, Eqs. (1a)-(1c) in binary32, push to
//                the neighbours; the compensated sum of what left each node
//   k_mp_update  rho(t+1) = rho(t) - (left) + (arrived) by compensated sums
//                into the pair, and psi of the new state for the next step
// k_mp_psi forms psi after an initialisation.
#pragma once

#include "lbm_internal.h"
#include "lbm_thermo_df.cuh"

namespace lbmfug {
namespace mp {

constexpr int kThreads = 256;

// Neighbour offsets r + e_a (periodic); the schedule requires N < 2^31.
template <int LAT>
__device__ __forceinline__ void neighbours(const Params &P, int r, int (&nb)[Lattice<LAT>::Q])
{
    using L = Lattice<LAT>;
    const int x = r % P.nx, t = r / P.nx;
    const int y = t % P.ny, z = t / P.ny;
#pragma unroll
    for (int a = 0; a < L::Q; ++a)
        nb[a] = wrap(x + L::e(a, 0), P.nx) + P.nx * (wrap(y + L::e(a, 1), P.ny) + P.ny * wrap(z + L::e(a, 2), P.nz));
}

// lap X = (2/cs2) sum_a w_a (X(r+e_a) - X(r)) in df64, with the weights scaled
// to small integers: D2Q9 (4 faces + diagonals - 20 X)/6, D3Q19
// (2 faces + edges - 24 X)/6.
template <int LAT>
__device__ __forceinline__ df::F2 lapQ(const float2 *__restrict__ X, const int (&nb)[Lattice<LAT>::Q])
{
    using L = Lattice<LAT>;
    constexpr float kFace = LAT == 0 ? 4.0f : 2.0f;
    constexpr float kCentre = LAT == 0 ? -20.0f : -24.0f;
    df::Dot d;
    const float2 c = X[nb[0]];
    const df::F2 cc = df::two_prod(kCentre, c.x);
    d.s = cc.hi;
    d.c = fmaf(kCentre, c.y, cc.lo);
#pragma unroll
    for (int a = 1; a < L::Q; ++a) {
        const float2 v = X[nb[a]];
        int e2 = 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) e2 += L::e(a, k) * L::e(a, k);
        const float s = e2 == 1 ? kFace : 1.0f;  // exact scalings by a power of two or one
        d.add_term({__fmul_rn(s, v.x), __fmul_rn(s, v.y)});
    }
    return df::mul(d.value(), {df::hi_of(1.0 / 6.0), df::lo_of(1.0 / 6.0)});
}

template <int NC>
__global__ void __launch_bounds__(kThreads) k_mp_psi(const Params P, StateBufs st, float2 *__restrict__ psi)
{
    const long long N = P.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        float h[NC], l[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            h[i] = st.rhi_f()[i * N + r];
            l[i] = st.rlo[i * N + r];
        }
        const df::F2 p = df::psi<NC>(P, h, l);
        psi[r] = make_float2(p.hi, p.lo);
    }
}

// per-thread scratch of mu_rolled: PH, PL [NC] floats and TS [NC] float2
template <int NC> constexpr size_t mp_mu_smem() { return (size_t)NC * kThreads * (2 * sizeof(float) + sizeof(float2)); }

template <int LAT, int NC>
__global__ void __launch_bounds__(kThreads)
    k_mp_mu(const Params P, StateBufs st, const float2 *__restrict__ psi, float2 *__restrict__ mu)
{
    using L = Lattice<LAT>;
    __shared__ float4 LT[df::kLogTab];
    extern __shared__ __align__(16) unsigned char scratch[];
    float2 *TS = (float2 *)scratch;
    float *PH = (float *)(TS + NC * kThreads);
    float *PL = PH + NC * kThreads;
    const int t = threadIdx.x;
    for (int j = t; j < df::kLogTab; j += blockDim.x) LT[j] = P.logtab[j];
    __syncthreads();
    const int N = (int)P.N;
    for (int r = blockIdx.x * blockDim.x + t; r < N; r += gridDim.x * blockDim.x) {
        int nb[L::Q];
        neighbours<LAT>(P, r, nb);
        float h[NC], l[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            h[i] = __ldg(st.rhi_f() + (long long)i * N + r);
            l[i] = __ldg(st.rlo + (long long)i * N + r);
        }
        df::mu_rolled<NC>(P, df::TabF4{LT}, h, l, df::mix_B<NC>(P, h, l), lapQ<LAT>(psi, nb), PH + t, PL + t, TS + t,
                          kThreads, mu + r, N);
    }
}

template <int LAT, int NC>
__global__ void __launch_bounds__(kThreads)
    k_mp_collide(const Params P, StateBufs in, StateBufs out, const float2 *__restrict__ mu,
                 float *__restrict__ osum, float *__restrict__ ocmp)
{
    using L = Lattice<LAT>;
    constexpr int D = L::D, Q = L::Q, NS = Q - 1;
    __shared__ float FS[NC * 3][kThreads];  // this thread's forces F_i
    const float *gin = (const float *)in.g;
    float *gout = (float *)out.g;
    const float *rh = in.rhi_f();
    const float *rl = in.rlo;
    const int N = (int)P.N;
    const int t = threadIdx.x;
    const float om = (float)P.omega, om1 = (float)(1.0 - P.omega), cF = (float)(1.0 - 0.5 * P.omega);
    for (int r = blockIdx.x * blockDim.x + t; r < N; r += gridDim.x * blockDim.x) {
        int nb[Q];
        neighbours<LAT>(P, r, nb);
        // momentum sum_i sum_a e_a g_a and the total density
        float j[3] = {0.0f, 0.0f, 0.0f}, rt = 0.0f;
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const float *gi = gin + (long long)i * NS * N;
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                const float v = __ldg(gi + (long long)(a - 1) * N + r);
#pragma unroll
                for (int d = 0; d < D; ++d)
                    if (L::e(a, d) > 0) j[d] += v;
                    else if (L::e(a, d) < 0) j[d] -= v;
            }
            rt += __ldg(rh + (long long)i * N + r) + __ldg(rl + (long long)i * N + r);
        }
        // Eq. (5): F_i = -rho~_i grad mu_i; grad X = 3 sum_pairs w e (X(r+e) - X(r-e)),
        // each difference on the (hi, lo) pairs rounded once
        float Fs[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll 2
        for (int i = 0; i < NC; ++i) {
            const float2 *mi = mu + (long long)i * N;
            float g[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int a = 1; a < Q; a += 2) {  // (a, a+1) opposite
                const float2 p = __ldg(mi + nb[a]), m = __ldg(mi + nb[a + 1]);
                const float dd = 3.0f * (float)L::w(a) * ((p.x - m.x) + (p.y - m.y));
#pragma unroll
                for (int d = 0; d < D; ++d) g[d] = fmaf((float)L::e(a, d), dd, g[d]);
            }
            const float ri = __ldg(rh + (long long)i * N + r) + __ldg(rl + (long long)i * N + r);
            const float rmi = ri * PV<float>::invM(P, i);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float f = -rmi * g[d];
                FS[i * 3 + d][t] = f;
                Fs[d] += f;
            }
        }
        const float irt = __fdividef(1.0f, rt);
        float u[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int d = 0; d < D; ++d) u[d] = fmaf(0.5f, Fs[d], j[d]) * irt;
        const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
#pragma unroll 1
        for (int i = 0; i < NC; ++i) {
            const float *rhi = rh + (long long)i * N, *rli = rl + (long long)i * N;
            // grad rho_i from the neighbours' pairs (binary32)
            float G[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int a = 1; a < Q; a += 2) {
                const float p = __ldg(rhi + nb[a]) + __ldg(rli + nb[a]);
                const float m = __ldg(rhi + nb[a + 1]) + __ldg(rli + nb[a + 1]);
                const float dd = 3.0f * (float)L::w(a) * (p - m);
#pragma unroll
                for (int d = 0; d < D; ++d) G[d] = fmaf((float)L::e(a, d), dd, G[d]);
            }
            const float ri = __ldg(rhi + r) + __ldg(rli + r);
            float F[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int d = 0; d < D; ++d) F[d] = FS[i * 3 + d][t];
            float Fu = 0.0f, Gu = 0.0f;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                Fu = fmaf(F[d], u[d], Fu);
                Gu = fmaf(G[d], u[d], Gu);
            }
            const float *gi = gin + (long long)i * NS * N;
            float *go = gout + (long long)i * NS * N;
            float os = 0.0f, oc = 0.0f;  // compensated sum of what leaves the node
#pragma unroll
            for (int a = 1; a < Q; ++a) {
                float ue = 0.0f, Fe = 0.0f, Ge = 0.0f;
                int e2 = 0;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const int ed = L::e(a, d);
                    e2 += ed * ed;
                    if (ed > 0) { ue += u[d]; Fe += F[d]; Ge += G[d]; }
                    if (ed < 0) { ue -= u[d]; Fe -= F[d]; Ge -= G[d]; }
                }
                const float w = (float)L::w(a);
                const float Bq = ue * fmaf(4.5f, ue, 3.0f) - 1.5f * u2;
                // Eq. (1c): F.[(e-u)/cs2 + (u.e)e/cs4] + grad rho.[-u + (u.e)e/cs2 + (e^2/cs2 - D)u/2]
                const float cW = (float)(0.5 * (3.0 * e2 - D) - 1.0);
                const float Fa = w * (Fe * fmaf(9.0f, ue, 3.0f) - 3.0f * Fu + 3.0f * ue * Ge + cW * Gu);
                // Eq. (1a) for a moving population: (1 - w) g + w g^eq + (1 - w/2) F_a
                const float gs = fmaf(om1, __ldg(gi + (long long)(a - 1) * N + r), fmaf(om * w * ri, Bq, cF * Fa));
                go[(long long)(a - 1) * N + nb[a]] = gs;
                acc_add(os, oc, gs);
            }
            osum[(long long)i * N + r] = os;
            ocmp[(long long)i * N + r] = oc;
        }
    }
}

template <int LAT, int NC>
__global__ void __launch_bounds__(kThreads)
    k_mp_update(const Params P, StateBufs in, StateBufs out, const float *__restrict__ osum,
                const float *__restrict__ ocmp, float2 *__restrict__ psi)
{
    using L = Lattice<LAT>;
    constexpr int NS = L::Q - 1;
    const float *g = (const float *)out.g;
    const long long N = P.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        float h[NC], l[NC];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            float s = -osum[i * N + r], c = -ocmp[i * N + r];
#pragma unroll
            for (int k = 0; k < NS; ++k) acc_add(s, c, __ldg(g + (i * NS + k) * N + r));
            float hi = in.rhi_f()[i * N + r], lo = in.rlo[i * N + r];
            pair_add(hi, lo, s, c);
            out.rhi_f()[i * N + r] = hi;
            out.rlo[i * N + r] = lo;
            h[i] = hi;
            l[i] = lo;
        }
        const df::F2 p = df::psi<NC>(P, h, l);
        psi[r] = make_float2(p.hi, p.lo);
    }
}

inline unsigned grid_for(long long n)
{
    long long b = (n + kThreads - 1) / kThreads;
    if (b > 152LL * 32) b = 152LL * 32;
    if (b < 1) b = 1;
    return (unsigned)b;
}

struct Ops {
    int (*psi)(const Params &, StateBufs, float2 *, cudaStream_t);
    int (*step)(const Params &, StateBufs, StateBufs, float2 *psi, float2 *mu, float *osum, float *ocmp,
                KernelTimer *, cudaStream_t);
};

template <int LAT, int NC> struct Impl {
    static int psi(const Params &P, StateBufs st, float2 *ps, cudaStream_t s)
    {
        k_mp_psi<NC><<<grid_for(P.N), kThreads, 0, s>>>(P, st, ps);
        return (int)cudaGetLastError();
    }
    static int step(const Params &P, StateBufs in, StateBufs out, float2 *ps, float2 *mu, float *osum,
                    float *ocmp, KernelTimer *kt, cudaStream_t s)
    {
        const unsigned G = grid_for(P.N);
        const size_t sm = mp_mu_smem<NC>();
        if (sm > 48 * 1024 &&
            cudaFuncSetAttribute(k_mp_mu<LAT, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
            return (int)cudaGetLastError();
        kt_begin(kt, kKtMpMu, s);
        k_mp_mu<LAT, NC><<<G, kThreads, sm, s>>>(P, in, ps, mu);
        kt_end(kt, s);
        kt_begin(kt, kKtMpCollide, s);
        k_mp_collide<LAT, NC><<<G, kThreads, 0, s>>>(P, in, out, mu, osum, ocmp);
        kt_end(kt, s);
        kt_begin(kt, kKtMpUpdate, s);
        k_mp_update<LAT, NC><<<G, kThreads, 0, s>>>(P, in, out, osum, ocmp, ps);
        kt_end(kt, s);
        return (int)cudaGetLastError();
    }
};

template <int LAT, int NC> const Ops *ops_of()
{
    static const Ops o = {&Impl<LAT, NC>::psi, &Impl<LAT, NC>::step};
    return &o;
}

template <int LAT, int LO, int HI> const Ops *ops_range(int nc)
{
    if constexpr (LO > HI) {
        return nullptr;
    } else {
        if (nc == LO) return ops_of<LAT, LO>();
        return ops_range<LAT, LO + 1, HI>(nc);
    }
}

}  // namespace mp
}  // namespace lbmfug

#define LBM_MP_TU(NAME, LAT, LO, HI)                                      \
    namespace lbmfug {                                                    \
    namespace mp {                                                        \
    const Ops *NAME(int nc) { return ops_range<LAT, LO, HI>(nc); }        \
    }                                                                     \
    }
