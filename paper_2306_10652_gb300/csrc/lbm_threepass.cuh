// lbm_threepass.cuh -- the three-pass time step (any lattice, any Nc <= 16).
//
// Pass 1 (k_macro):   rho_i, the momentum sum_i sum_a e_a g_{a,i}, ln f_i
//                     (Eqs. 9-12) and psi = sum_j sqrt(kappa_j) rho~_j.
// Pass 2 (k_lap):     lap psi with the isotropic lattice Laplacian.
// Pass 3 (k_collide): F_i = -rho~_i grad(RT ln f_i - sqrt(kappa_i) lap psi)
//                     (Eq. 5 with kappa_ij = sqrt(kappa_i kappa_j), Eq. 4, so
//                     sum_j kappa_ij lap rho~_j = sqrt(kappa_i) lap psi),
//                     u = (sum e g + F/2) / rho, the equilibrium (Eq. 1b) and
//                     forcing term (Eq. 1c), BGK (Eq. 1a) and push streaming
//                     g_{a,i}(r + e_a) <- g*_{a,i}(r).
//
// State formats (post-streaming populations, the convention of Eq. 1a):
//  * binary64 (S = double): all Q populations g[i][a][node].
//  * binary32 (S = float): the Q-1 moving populations g[i][a-1][node] (a >= 1)
//    and the density rho_i as an unevaluated binary32 sum hi + lo.  The rest
//    population is never needed: rho_i is the state, and the collision of
//    a >= 1 uses only rho_i, u, F_i and grad rho_i.  Pass 4 (k_rupdate) moves
//    the density by exactly the populations that left and arrived,
//    rho(t+1) = rho(t) - sum_{a>=1} g*_a(r) + sum_{a>=1} g_a(t+1)(r), with
//    compensated sums of the stored binary32 values, so the component mass
//    is conserved to the rounding of the pair.
#pragma once
#include "lbm_internal.h"

namespace lbmfug {

namespace tp {

constexpr int kThreads = 256;

__device__ __forceinline__ void node_xyz(long long r, const Params &P, int &x, int &y, int &z)
{
    x = (int)(r % P.nx);
    long long t = r / P.nx;
    y = (int)(t % P.ny);
    z = (int)(t / P.ny);
}

template <int LAT>
__device__ __forceinline__ void neighbours(const Params &P, int x, int y, int z,
                                           long long (&nb)[Lattice<LAT>::Q])
{
    using L = Lattice<LAT>;
#pragma unroll
    for (int a = 0; a < L::Q; ++a) {
        int xx = wrap(x + L::e(a, 0), P.nx);
        int yy = wrap(y + L::e(a, 1), P.ny);
        int zz = wrap(z + L::e(a, 2), P.nz);
        nb[a] = xx + (long long)P.nx * (yy + (long long)P.ny * zz);
    }
}

// grad X(r) = (1/cs2) sum_a w_a e_a X(r + e_a), summed over opposite pairs.
template <int LAT>
__device__ __forceinline__ void grad_pairs(const double *__restrict__ X,
                                           const long long (&nb)[Lattice<LAT>::Q], double (&G)[3])
{
    using L = Lattice<LAT>;
    G[0] = G[1] = G[2] = 0.0;
#pragma unroll
    for (int a = 1; a < L::Q; a += 2) {
        const double d = __ldg(X + nb[a]) - __ldg(X + nb[a + 1]);
#pragma unroll
        for (int k = 0; k < L::D; ++k)
            if (L::e(a, k) != 0) G[k] = fma(L::w(a) * L::e(a, k), d, G[k]);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) G[k] *= 3.0;
}

// population slot of direction a in the storage format of S (-1: not stored)
template <int LAT, typename S> __host__ __device__ constexpr int slot(int a)
{
    return sizeof(S) == 8 ? a : a - 1;
}
template <int LAT, typename S> __host__ __device__ constexpr int nslots()
{
    return sizeof(S) == 8 ? Lattice<LAT>::Q : Lattice<LAT>::Q - 1;
}

template <int LAT, int NC, typename S>
__global__ void __launch_bounds__(kThreads)
    k_init(const Params P, const double *__restrict__ rho, const double *__restrict__ u, StateBufs st)
{
    using L = Lattice<LAT>;
    constexpr int NS = nslots<LAT, S>();
    S *g = (S *)st.g;
    const long long N = P.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        double uu[3] = {0.0, 0.0, 0.0};
        if (u)
            for (int d = 0; d < L::D; ++d) uu[d] = u[d * N + r];
        const double u2 = uu[0] * uu[0] + uu[1] * uu[1] + uu[2] * uu[2];
#pragma unroll
        for (int a = 0; a < L::Q; ++a) {
            double ue = 0.0;
#pragma unroll
            for (int d = 0; d < L::D; ++d) ue += L::e(a, d) * uu[d];
            const double Bq = 3.0 * ue + 4.5 * ue * ue - 1.5 * u2;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const double ri = rho[i * N + r];
                const double geq = L::w(a) * ri * Bq + (a == 0 ? ri : 0.0);  // Eq. (1b), rho^c = 0
                if (slot<LAT, S>(a) >= 0) g[(i * NS + slot<LAT, S>(a)) * N + r] = (S)geq;
            }
        }
        if (sizeof(S) == 4) {
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const double ri = rho[i * N + r];
                const float hi = (float)ri;
                st.rhi_f()[i * N + r] = hi;
                st.rlo[i * N + r] = (float)(ri - (double)hi);
            }
        }
    }
}

// kRhoOnly: the densities alone (lbm_moments asked for nothing else), no EOS
template <int LAT, int NC, typename S, bool kRhoOnly = false>
__global__ void __launch_bounds__(kThreads)
    k_macro(const Params P, StateBufs st, double *__restrict__ rho, double *__restrict__ lnf,
            double *__restrict__ psi, double *__restrict__ jm, double *__restrict__ pout)
{
    using L = Lattice<LAT>;
    constexpr int NS = nslots<LAT, S>();
    const S *g = (const S *)st.g;
    const long long N = P.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        double rm[NC];
        double j[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            if constexpr (kRhoOnly && sizeof(S) == 4) {
                rho[i * N + r] = (double)st.rhi_f()[i * N + r] + (double)st.rlo[i * N + r];
                continue;
            }
            S s = 0, ji[3] = {0, 0, 0};
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                if (slot<LAT, S>(a) < 0) continue;
                const S v = __ldg(g + (i * NS + slot<LAT, S>(a)) * N + r);
                s += v;
#pragma unroll
                for (int d = 0; d < L::D; ++d)
                    if (L::e(a, d) > 0) ji[d] += v;
                    else if (L::e(a, d) < 0) ji[d] -= v;
            }
            const double ri = sizeof(S) == 8
                                  ? (double)s
                                  : (double)st.rhi_f()[i * N + r] + (double)st.rlo[i * N + r];
            rho[i * N + r] = ri;
            rm[i] = ri * P.invM[i];
#pragma unroll
            for (int d = 0; d < L::D; ++d) j[d] += (double)ji[d];
        }
        if constexpr (kRhoOnly) continue;
        double lf[NC], p;
        pr_lnf<NC>(P, rm, lf, &p);
        double ps = 0.0;
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            lnf[i * N + r] = lf[i];
            ps = fma(P.sqk[i], rm[i], ps);
        }
        psi[r] = ps;
#pragma unroll
        for (int d = 0; d < L::D; ++d) jm[d * N + r] = j[d];
        if (pout) pout[r] = p;
    }
}

template <int LAT>
__global__ void __launch_bounds__(kThreads)
    k_lap(const Params P, const double *__restrict__ psi, double *__restrict__ lap)
{
    using L = Lattice<LAT>;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < P.N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(r, P, x, y, z);
        long long nb[L::Q];
        neighbours<LAT>(P, x, y, z, nb);
        const double c = psi[r];
        double s = 0.0;
#pragma unroll
        for (int a = 1; a < L::Q; ++a) s = fma(L::w(a), __ldg(psi + nb[a]) - c, s);
        lap[r] = 6.0 * s;  // 2 / cs2
    }
}

template <int LAT, int NC, typename S, bool STEP>
__global__ void __launch_bounds__(kThreads)
    k_collide(const Params P, StateBufs in, StateBufs out, const double *__restrict__ rho,
              const double *__restrict__ lnf, const double *__restrict__ lap,
              const double *__restrict__ jm, double *__restrict__ uout, float *__restrict__ osum,
              float *__restrict__ ocmp)
{
    using L = Lattice<LAT>;
    constexpr int D = L::D;
    constexpr int NS = nslots<LAT, S>();
    const S *gin = (const S *)in.g;
    S *gout = (S *)out.g;
    const long long N = P.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        node_xyz(r, P, x, y, z);
        long long nb[L::Q];
        neighbours<LAT>(P, x, y, z, nb);
        double GL[3];
        grad_pairs<LAT>(lap, nb, GL);
        // Eq. (5): F_i = -rho~_i (RT grad ln f_i - sqrt(kappa_i) grad lap psi)
        double F[NC][D];
        double Fs[3] = {0.0, 0.0, 0.0}, rt = 0.0;
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            double Gl[3];
            grad_pairs<LAT>(lnf + i * N, nb, Gl);
            const double ri = rho[i * N + r];
            rt += ri;
            const double rmi = ri * P.invM[i];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                F[i][d] = -rmi * (P.RT * Gl[d] - P.sqk[i] * GL[d]);
                Fs[d] += F[i][d];
            }
        }
        double u[3] = {0.0, 0.0, 0.0};
        const double irt = 1.0 / rt;
#pragma unroll
        for (int d = 0; d < D; ++d) u[d] = fma(0.5, Fs[d], jm[d * N + r]) * irt;
        if (!STEP) {
#pragma unroll
            for (int d = 0; d < D; ++d) uout[d * N + r] = u[d];
            continue;
        }
        const double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double om = P.omega, cF = 1.0 - 0.5 * P.omega;
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            double Gr[3];
            grad_pairs<LAT>(rho + i * N, nb, Gr);
            const double ri = rho[i * N + r];
            double Fu = 0.0, Gu = 0.0;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                Fu = fma(F[i][d], u[d], Fu);
                Gu = fma(Gr[d], u[d], Gu);
            }
            float os = 0.0f, oc = 0.0f;  // binary32: compensated sum of what leaves the node
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                if (slot<LAT, S>(a) < 0) continue;
                double ue = 0.0, Fe = 0.0, Ge = 0.0;
                int e2 = 0;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const int ed = L::e(a, d);
                    e2 += ed * ed;
                    if (ed > 0) { ue += u[d]; Fe += F[i][d]; Ge += Gr[d]; }
                    if (ed < 0) { ue -= u[d]; Fe -= F[i][d]; Ge -= Gr[d]; }
                }
                const double w = L::w(a);
                const double Bq = ue * fma(4.5, ue, 3.0) - 1.5 * u2;
                // Eq. (1c): F.[(e-u)/cs2 + (u.e)e/cs4] + grad rho.[-u + (u.e)e/cs2 + (e^2/cs2 - D)u/2]
                const double cW = 0.5 * (3.0 * e2 - D) - 1.0;
                const double Fa = w * (Fe * fma(9.0, ue, 3.0) - 3.0 * Fu + 3.0 * ue * Ge + cW * Gu);
                const long long k = (i * NS + slot<LAT, S>(a)) * N;
                if (sizeof(S) == 8) {
                    const double geq = w * ri * Bq + (a == 0 ? ri : 0.0);
                    const double gv = (double)gin[k + r];
                    gout[k + nb[a]] = (S)(gv + om * (geq - gv) + cF * Fa);
                } else {
                    // Eq. (1a) for a moving population in binary32
                    const float hv = (float)gin[k + r];
                    const float geq = (float)(w * ri * Bq);
                    const float ho = fmaf((float)om, geq - hv, hv) + (float)cF * (float)Fa;
                    gout[k + nb[a]] = (S)ho;
                    acc_add(os, oc, ho);
                }
            }
            if (sizeof(S) == 4) {
                osum[i * N + r] = os;
                ocmp[i * N + r] = oc;
            }
        }
    }
}

// binary32 pass 4: rho(t+1) = rho(t) - (left) + (arrived), all compensated.
template <int LAT, int NC>
__global__ void __launch_bounds__(kThreads)
    k_rupdate(const Params P, StateBufs in, StateBufs out, const float *__restrict__ osum,
              const float *__restrict__ ocmp)
{
    using L = Lattice<LAT>;
    constexpr int NS = L::Q - 1;
    const float *g = (const float *)out.g;
    const long long N = P.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            float s = -osum[i * N + r], c = -ocmp[i * N + r];
#pragma unroll
            for (int k = 0; k < NS; ++k) acc_add(s, c, __ldg(g + (i * NS + k) * N + r));
            float hi = in.rhi_f()[i * N + r], lo = in.rlo[i * N + r];
            pair_add(hi, lo, s, c);
            out.rhi_f()[i * N + r] = hi;
            out.rlo[i * N + r] = lo;
        }
    }
}

template <int LAT, int NC, typename S>
__global__ void k_to_f64(const Params P, StateBufs st, double *__restrict__ out)
{
    using L = Lattice<LAT>;
    constexpr int NS = nslots<LAT, S>();
    const S *g = (const S *)st.g;
    const long long N = P.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            double moving = 0.0;
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                if (slot<LAT, S>(a) < 0) continue;
                const double v = (double)g[(i * NS + slot<LAT, S>(a)) * N + r];
                out[(i * L::Q + a) * N + r] = v;
                moving += a > 0 ? v : 0.0;
            }
            if (sizeof(S) == 4)
                out[(i * L::Q) * N + r] =
                    (double)st.rhi_f()[i * N + r] + (double)st.rlo[i * N + r] - moving;
        }
    }
}

template <int LAT, int NC, typename S>
__global__ void k_from_f64(const Params P, const double *__restrict__ in, StateBufs st)
{
    using L = Lattice<LAT>;
    constexpr int NS = nslots<LAT, S>();
    S *g = (S *)st.g;
    const long long N = P.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            double rho = 0.0;
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                const double v = in[(i * L::Q + a) * N + r];
                rho += v;
                if (slot<LAT, S>(a) >= 0) g[(i * NS + slot<LAT, S>(a)) * N + r] = (S)v;
            }
            if (sizeof(S) == 4) {
                const float hi = (float)rho;
                st.rhi_f()[i * N + r] = hi;
                st.rlo[i * N + r] = (float)(rho - (double)hi);
            }
        }
    }
}

inline unsigned grid_for(long long n)
{
    long long b = (n + kThreads - 1) / kThreads;
    if (b > 152LL * 64) b = 152LL * 64;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <int LAT, int NC, typename S> struct Impl {
    static int init(const Params &P, const double *rho, const double *u, StateBufs st, cudaStream_t s)
    {
        k_init<LAT, NC, S><<<grid_for(P.N), kThreads, 0, s>>>(P, rho, u, st);
        return (int)cudaGetLastError();
    }
    static int step(const Params &P, StateBufs in, StateBufs out, const ThreePassWork &w,
                    cudaStream_t s)
    {
        const unsigned G = grid_for(P.N);
        k_macro<LAT, NC, S><<<G, kThreads, 0, s>>>(P, in, w.rho, w.lnf, w.psi, w.jm, nullptr);
        k_lap<LAT><<<G, kThreads, 0, s>>>(P, w.psi, w.lap);
        k_collide<LAT, NC, S, true><<<G, kThreads, 0, s>>>(P, in, out, w.rho, w.lnf, w.lap, w.jm,
                                                           nullptr, w.osum, w.ocmp);
        if (sizeof(S) == 4)
            k_rupdate<LAT, NC><<<G, kThreads, 0, s>>>(P, in, out, w.osum, w.ocmp);
        return (int)cudaGetLastError();
    }
    static int fields(const Params &P, StateBufs st, const ThreePassWork &w, double *rho,
                      double *u, double *p, double *lnf, cudaStream_t s)
    {
        const unsigned G = grid_for(P.N);
        if (!u && !p && !lnf)
            k_macro<LAT, NC, S, true><<<G, kThreads, 0, s>>>(P, st, w.rho, nullptr, nullptr, nullptr, nullptr);
        else
            k_macro<LAT, NC, S><<<G, kThreads, 0, s>>>(P, st, w.rho, w.lnf, w.psi, w.jm, p);
        if (u) {
            k_lap<LAT><<<G, kThreads, 0, s>>>(P, w.psi, w.lap);
            k_collide<LAT, NC, S, false><<<G, kThreads, 0, s>>>(P, st, StateBufs{}, w.rho, w.lnf,
                                                                w.lap, w.jm, u, nullptr, nullptr);
        }
        const size_t fb = (size_t)NC * P.N * sizeof(double);
        if (rho && rho != w.rho) cudaMemcpyAsync(rho, w.rho, fb, cudaMemcpyDeviceToDevice, s);
        if (lnf && lnf != w.lnf) cudaMemcpyAsync(lnf, w.lnf, fb, cudaMemcpyDeviceToDevice, s);
        return (int)cudaGetLastError();
    }
    static int to_f64(const Params &P, StateBufs st, double *out, cudaStream_t s)
    {
        k_to_f64<LAT, NC, S><<<grid_for(P.N), kThreads, 0, s>>>(P, st, out);
        return (int)cudaGetLastError();
    }
    static int from_f64(const Params &P, const double *in, StateBufs st, cudaStream_t s)
    {
        k_from_f64<LAT, NC, S><<<grid_for(P.N), kThreads, 0, s>>>(P, in, st);
        return (int)cudaGetLastError();
    }
    static int launches_per_step() { return sizeof(S) == 4 ? 4 : 3; }
};

// Function table of one (lattice, storage, Nc) instantiation.
struct Ops {
    int (*init)(const Params &, const double *, const double *, StateBufs, cudaStream_t);
    int (*step)(const Params &, StateBufs, StateBufs, const ThreePassWork &, cudaStream_t);
    int (*fields)(const Params &, StateBufs, const ThreePassWork &, double *, double *, double *,
                  double *, cudaStream_t);
    int (*to_f64)(const Params &, StateBufs, double *, cudaStream_t);
    int (*from_f64)(const Params &, const double *, StateBufs, cudaStream_t);
    int (*launches_per_step)();
};

template <int LAT, int NC, typename S> const Ops *ops_of()
{
    static const Ops o = {&Impl<LAT, NC, S>::init,   &Impl<LAT, NC, S>::step,
                          &Impl<LAT, NC, S>::fields, &Impl<LAT, NC, S>::to_f64,
                          &Impl<LAT, NC, S>::from_f64, &Impl<LAT, NC, S>::launches_per_step};
    return &o;
}

// Table of one translation unit: lattice LAT, storage S, Nc in [LO, HI].
template <int LAT, typename S, int LO, int HI> const Ops *ops_range(int nc)
{
    if constexpr (LO > HI) {
        return nullptr;
    } else {
        if (nc == LO) return ops_of<LAT, LO, S>();
        return ops_range<LAT, S, LO + 1, HI>(nc);
    }
}

}  // namespace tp

#define LBM_TP_TU(NAME, LAT, S, LO, HI) \
    namespace lbmfug { namespace tp { \
    const Ops *NAME(int nc) { return ops_range<LAT, S, LO, HI>(nc); } \
    } }

}  // namespace lbmfug
