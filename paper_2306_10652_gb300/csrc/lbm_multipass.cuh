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

#include <algorithm>

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
        df::mu_rolled<NC>(P, df::TabF4{LT}, h, l, lapQ<LAT>(psi, nb), PH + t, PL + t, TS + t, kThreads, mu + r, N);
    }
}

// A CTA of k_mp_collide owns a block of TX x TY x TZ nodes (one per thread)
// and stages the mu_i of every component for the block and its one-node halo
// in shared memory (asynchronous copies, all in flight at once), then the
// density pairs in the same space, so each neighbour value is read from L2
// about once instead of once per neighbour.
template <int LAT> struct MpTile {
    static constexpr int TX = 32, TY = LAT == 0 ? 8 : 4, TZ = LAT == 0 ? 1 : 2;
    static constexpr int HX = TX + 2, HY = TY + 2, HZ = LAT == 0 ? 1 : TZ + 2;
    static constexpr int HN = HX * HY * HZ;
    static_assert(TX * TY * TZ == kThreads, "one node per thread");
};

template <int LAT, int NC> constexpr size_t mp_collide_smem()
{
    // forces, then one space for mu [NC][HN] (float2) or the pairs [2][NC][HN] (float)
    return (size_t)NC * 3 * kThreads * sizeof(float) + (size_t)NC * MpTile<LAT>::HN * sizeof(float2);
}

// cp.async of 4 or 8 bytes from global to shared memory (both aligned to the size)
__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(a), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void *sdst, const void *gsrc)
{
    const unsigned a = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ int wrap_any(int v, int n)
{
    if (v < 0) return v + n;  // v >= -1
    return v < n ? v : v % n;
}

template <int LAT, int NC>
__global__ void __launch_bounds__(kThreads)
    k_mp_collide(const Params P, StateBufs in, StateBufs out, const float2 *__restrict__ mu,
                 float *__restrict__ osum, float *__restrict__ ocmp)
{
    using L = Lattice<LAT>;
    using TL = MpTile<LAT>;
    constexpr int D = L::D, Q = L::Q, NS = Q - 1;
    extern __shared__ __align__(16) unsigned char smem[];
    float *FS = (float *)smem;                        // [NC * 3][kThreads] this thread's forces F_i
    float2 *MT = (float2 *)(FS + NC * 3 * kThreads);  // [NC][HN] mu_i of the block and halo
    float *RH = (float *)MT;                          // [NC][HN] rho_i hi (after the forces)
    float *RL = RH + NC * TL::HN;                     // [NC][HN] rho_i lo
    const float *gin = (const float *)in.g;
    float *gout = (float *)out.g;
    const float *rh = in.rhi_f();
    const float *rl = in.rlo;
    const int nx = P.nx, ny = P.ny, nz = P.nz;
    const int N = (int)P.N;
    const int t = threadIdx.x;
    const int tx = t % TL::TX, ty = (t / TL::TX) % TL::TY, tz = t / (TL::TX * TL::TY);
    const int nbx = (nx + TL::TX - 1) / TL::TX, nby = (ny + TL::TY - 1) / TL::TY, nbz = (nz + TL::TZ - 1) / TL::TZ;
    const int nblk = nbx * nby * nbz;
    // tile offset of each direction and of this thread's node
    int toff[Q];
#pragma unroll
    for (int a = 0; a < Q; ++a) toff[a] = L::e(a, 0) + TL::HX * (L::e(a, 1) + TL::HY * L::e(a, 2));
    const int ti = (tx + 1) + TL::HX * ((ty + 1) + TL::HY * (tz + (TL::HZ > 1 ? 1 : 0)));
    const float om = (float)P.omega, om1 = (float)(1.0 - P.omega), cF = (float)(1.0 - 0.5 * P.omega);
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int bx = blk % nbx, by = (blk / nbx) % nby, bz = blk / (nbx * nby);
        const int x0 = bx * TL::TX, y0 = by * TL::TY, z0 = bz * TL::TZ;
        const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
        const bool active = x < nx && y < ny && z < nz;
        const int r = active ? x + nx * (y + ny * z) : 0;
        // the tile's node index for tile entry k (periodic; any block size)
        auto gnode = [&](int k) {
            const int hx = k % TL::HX, hy = (k / TL::HX) % TL::HY, hz = k / (TL::HX * TL::HY);
            const int gx = wrap_any(x0 + hx - 1, nx), gy = wrap_any(y0 + hy - 1, ny);
            const int gz = TL::HZ > 1 ? wrap_any(z0 + hz - 1, nz) : z0;
            return gx + nx * (gy + ny * gz);
        };
        // the node of each tile entry this thread loads, once per block
        constexpr int KPT = (TL::HN + kThreads - 1) / kThreads;
        int gk[KPT];
#pragma unroll
        for (int q = 0; q < KPT; ++q) {
            const int k = t + q * kThreads;
            gk[q] = k < TL::HN ? gnode(k) : 0;
        }
        int nb[Q];
        neighbours<LAT>(P, r, nb);
        // momentum sum_i sum_a e_a g_a and the total density
        float j[3] = {0.0f, 0.0f, 0.0f}, rt = 0.0f;
        if (active) {
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
        }
        // Eq. (5): F_i = -rho~_i grad mu_i; grad X = 3 sum_pairs w e (X(r+e) - X(r-e)),
        // each difference on the (hi, lo) pairs rounded once
        float Fs[3] = {0.0f, 0.0f, 0.0f};
        __syncthreads();  // the previous block's readers of the tiles are done
#pragma unroll 1
        for (int i = 0; i < NC; ++i)
#pragma unroll
            for (int q = 0; q < KPT; ++q)
                if (t + q * kThreads < TL::HN) cp_async8(MT + i * TL::HN + t + q * kThreads, mu + (long long)i * N + gk[q]);
        cp_async_wait_all();
        __syncthreads();
        if (active) {
#pragma unroll 1
            for (int i = 0; i < NC; ++i) {
                const float2 *mt = MT + i * TL::HN;
                float g[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int a = 1; a < Q; a += 2) {  // (a, a+1) opposite
                    const float2 p = mt[ti + toff[a]], m = mt[ti + toff[a + 1]];
                    const float dd = 3.0f * (float)L::w(a) * ((p.x - m.x) + (p.y - m.y));
#pragma unroll
                    for (int d = 0; d < D; ++d) g[d] = fmaf((float)L::e(a, d), dd, g[d]);
                }
                const float ri = __ldg(rh + (long long)i * N + r) + __ldg(rl + (long long)i * N + r);
                const float rmi = ri * PV<float>::invM(P, i);
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const float f = -rmi * g[d];
                    FS[(i * 3 + d) * kThreads + t] = f;
                    Fs[d] += f;
                }
            }
        }
        const float irt = __fdividef(1.0f, rt);
        float u[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int d = 0; d < D; ++d) u[d] = fmaf(0.5f, Fs[d], j[d]) * irt;
        const float u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        __syncthreads();  // the mu tiles are read
#pragma unroll 1
        for (int i = 0; i < NC; ++i)
#pragma unroll
            for (int q = 0; q < KPT; ++q)
                if (t + q * kThreads < TL::HN) {
                    cp_async4(RH + i * TL::HN + t + q * kThreads, rh + (long long)i * N + gk[q]);
                    cp_async4(RL + i * TL::HN + t + q * kThreads, rl + (long long)i * N + gk[q]);
                }
        cp_async_wait_all();
        __syncthreads();
        if (!active) continue;
#pragma unroll 1
        for (int i = 0; i < NC; ++i) {
            const float *rhi = RH + i * TL::HN, *rli = RL + i * TL::HN;
            // grad rho_i from the neighbours' pairs (binary32)
            float G[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int a = 1; a < Q; a += 2) {
                const float p = rhi[ti + toff[a]] + rli[ti + toff[a]];
                const float m = rhi[ti + toff[a + 1]] + rli[ti + toff[a + 1]];
                const float dd = 3.0f * (float)L::w(a) * (p - m);
#pragma unroll
                for (int d = 0; d < D; ++d) G[d] = fmaf((float)L::e(a, d), dd, G[d]);
            }
            const float ri = rhi[ti] + rli[ti];
            float F[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
            for (int d = 0; d < D; ++d) F[d] = FS[(i * 3 + d) * kThreads + t];
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
        using TL = MpTile<LAT>;
        const long long nblk = (long long)((P.nx + TL::TX - 1) / TL::TX) * ((P.ny + TL::TY - 1) / TL::TY) *
                               ((P.nz + TL::TZ - 1) / TL::TZ);
        const unsigned GC = (unsigned)std::min<long long>(nblk, 152LL * 16);
        const size_t smc = mp_collide_smem<LAT, NC>();
        if (smc > 48 * 1024 &&
            cudaFuncSetAttribute(k_mp_collide<LAT, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc) !=
                cudaSuccess)
            return (int)cudaGetLastError();
        kt_begin(kt, kKtMpCollide, s);
        k_mp_collide<LAT, NC><<<GC, kThreads, smc, s>>>(P, in, out, mu, osum, ocmp);
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
