// lbm_fields.cuh -- chemical potentials mu_i and interaction forces F_i of a
// D2Q9 state, evaluated node by node with the same device routines as the
// fused step in each precision form (lbm_forces).
//
// Paper: Soomro & Ayala, arXiv 2306.10652.
//   Sec. 2.1, Eq. (5)  F_i = -rho~_i grad mu_i, mu_i = RT ln f_i - sqrt(kappa_i) lap psi
//                      (the printed force with kappa_ij = sqrt(kappa_i kappa_j), Eq. 4)
//   Sec. 2.3, Eqs. (9)-(12)
//
// Input: the mass densities rho[i][N] in binary64 (for binary32 storage the
// exact pair hi + lo, which binary64 holds exactly and splits back).
// E = double: binary64 (LBM_FP64); float: binary32 (LBM_FP32); DF64: double-
// binary32 (LBM_FP32DEV).  Three passes: psi, mu (with lap psi), force.
#pragma once

#include <type_traits>

#include "lbm_fused2d.cuh"

namespace lbmfug {
namespace fields {

using fz::DF64;

template <typename E> struct Store { using T = E; };
template <> struct Store<DF64> { using T = float2; };

__device__ __forceinline__ long long nb(long long r, int nx, int ny, int dx, int dy)
{
    const int x = (int)(r % nx), y = (int)(r / nx);
    return (long long)wrap(y + dy, ny) * nx + wrap(x + dx, nx);
}

__device__ __forceinline__ void split(double v, float &h, float &l)
{
    h = (float)v;
    l = (float)(v - (double)h);
}

template <int NC, typename E>
__global__ void k_psi(const Params P, const double *__restrict__ rho, typename Store<E>::T *__restrict__ psi)
{
    const long long N = P.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        if constexpr (std::is_same<E, DF64>::value) {
            float h[NC], l[NC];
#pragma unroll
            for (int i = 0; i < NC; ++i) split(rho[i * N + r], h[i], l[i]);
            const df::F2 v = df::psi<NC>(P, h, l);
            psi[r] = make_float2(v.hi, v.lo);
        } else {
            using V = PV<E>;
            E s = 0;
#pragma unroll
            for (int i = 0; i < NC; ++i) s = fma(V::sqk(P, i), (E)rho[i * N + r] * V::invM(P, i), s);
            psi[r] = s;
        }
    }
}

template <int NC, typename E>
__global__ void k_mu(const Params P, const double *__restrict__ rho, const typename Store<E>::T *__restrict__ psi,
                     typename Store<E>::T *__restrict__ mu)
{
    const long long N = P.N;
    const int nx = P.nx, ny = P.ny;
    __shared__ float4 LT[df::kLogTab];
    if constexpr (std::is_same<E, DF64>::value) {
        for (int j = threadIdx.x; j < df::kLogTab; j += blockDim.x) LT[j] = P.logtab[j];
        __syncthreads();
    }
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
        if constexpr (std::is_same<E, DF64>::value) {
            float h[NC], l[NC];
#pragma unroll
            for (int i = 0; i < NC; ++i) split(rho[i * N + r], h[i], l[i]);
            auto at = [&](int dx, int dy) { return df::f2(psi[nb(r, nx, ny, dx, dy)]); };
            const df::F2 lap = df::lap9(at(0, 0), at(1, 0), at(-1, 0), at(0, 1), at(0, -1), at(1, 1), at(-1, 1),
                                        at(1, -1), at(-1, -1));
            df::F2 m[NC];
            df::mu<NC>(P, LT, h, l, lap, m);
#pragma unroll
            for (int i = 0; i < NC; ++i) mu[i * N + r] = make_float2(m[i].hi, m[i].lo);
        } else {
            using V = PV<E>;
            E rm[NC], lf[NC];
#pragma unroll
            for (int i = 0; i < NC; ++i) rm[i] = (E)rho[i * N + r] * V::invM(P, i);
            pr_lnf<NC, E>(P, rm, lf, nullptr);
            auto at = [&](int dx, int dy) { return psi[nb(r, nx, ny, dx, dy)]; };
            const E c0 = at(0, 0);
            const E faces = (at(1, 0) - c0) + (at(-1, 0) - c0) + (at(0, 1) - c0) + (at(0, -1) - c0);
            const E diags = (at(1, 1) - c0) + (at(-1, -1) - c0) + (at(1, -1) - c0) + (at(-1, 1) - c0);
            const E lap = (E)6 * fma((E)(1.0 / 9.0), faces, (E)(1.0 / 36.0) * diags);
#pragma unroll
            for (int i = 0; i < NC; ++i) mu[i * N + r] = fma(V::RT(P), lf[i], -V::sqk(P, i) * lap);
        }
    }
}

template <int NC, typename E>
__global__ void k_force(const Params P, const double *__restrict__ rho, const typename Store<E>::T *__restrict__ mu,
                        double *__restrict__ F, double *__restrict__ muout)
{
    const long long N = P.N;
    const int nx = P.nx, ny = P.ny;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            const auto *m = mu + i * N;
            double mc;
            if constexpr (std::is_same<E, DF64>::value) {
                // the differences of the fused kernel: on the (hi, lo) pairs, rounded once
                auto d = [&](int ax, int ay, int bx, int by) {
                    const float2 a = m[nb(r, nx, ny, ax, ay)], b = m[nb(r, nx, ny, bx, by)];
                    return (a.x - b.x) + (a.y - b.y);
                };
                const float dE = d(1, 0, -1, 0), dN = d(0, 1, 0, -1), dNE = d(1, 1, -1, -1), dSE = d(1, -1, -1, 1);
                const float gx = 3.0f * fmaf(1.0f / 9.0f, dE, (1.0f / 36.0f) * (dNE + dSE));
                const float gy = 3.0f * fmaf(1.0f / 9.0f, dN, (1.0f / 36.0f) * (dNE - dSE));
                const float2 c = m[r];
                mc = (double)c.x + (double)c.y;
                float hf, lf;
                split(rho[i * N + r], hf, lf);
                const float rmi = (hf + lf) * PV<float>::invM(P, i);
                F[(i * 2 + 0) * N + r] = (double)(-rmi * gx);
                F[(i * 2 + 1) * N + r] = (double)(-rmi * gy);
            } else {
                using V = PV<E>;
                auto d = [&](int ax, int ay, int bx, int by) {
                    return m[nb(r, nx, ny, ax, ay)] - m[nb(r, nx, ny, bx, by)];
                };
                const E dE = d(1, 0, -1, 0), dN = d(0, 1, 0, -1), dNE = d(1, 1, -1, -1), dSE = d(1, -1, -1, 1);
                const E ex = (E)3 * fma((E)(1.0 / 9.0), dE, (E)(1.0 / 36.0) * (dNE + dSE));
                const E ey = (E)3 * fma((E)(1.0 / 9.0), dN, (E)(1.0 / 36.0) * (dNE - dSE));
                const E rmi = (E)rho[i * N + r] * V::invM(P, i);
                mc = m[r];
                F[(i * 2 + 0) * N + r] = (double)(-rmi * ex);
                F[(i * 2 + 1) * N + r] = (double)(-rmi * ey);
            }
            if (muout) muout[i * N + r] = mc;
        }
    }
}

// psi/mu scratch: (NC + 1) N values of Store<E>::T.
template <int NC, typename E>
int launch(const Params &P, const double *rho, void *scratch, double *F, double *mu, cudaStream_t s)
{
    using T = typename Store<E>::T;
    T *psi = (T *)scratch;
    T *m = psi + P.N;
    long long b = (P.N + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    k_psi<NC, E><<<(unsigned)b, 256, 0, s>>>(P, rho, psi);
    k_mu<NC, E><<<(unsigned)b, 256, 0, s>>>(P, rho, psi, m);
    k_force<NC, E><<<(unsigned)b, 256, 0, s>>>(P, rho, m, F, mu);
    return (int)cudaGetLastError();
}

template <typename E, int LO, int HI>
int launch_range(int nc, const Params &P, const double *rho, void *scratch, double *F, double *mu, cudaStream_t s)
{
    if constexpr (LO > HI) {
        return (int)cudaErrorInvalidValue;
    } else {
        if (nc == LO) return launch<LO, E>(P, rho, scratch, F, mu, s);
        return launch_range<E, LO + 1, HI>(nc, P, rho, scratch, F, mu, s);
    }
}

}  // namespace fields
}  // namespace lbmfug

#define LBM_FIELDS_TU(NAME, LO, HI)                                                                   \
    namespace lbmfug {                                                                                \
    int NAME(int prec, int nc, const Params &P, const double *rho, void *scratch, double *F, double *mu, \
             cudaStream_t s)                                                                          \
    {                                                                                                 \
        if (prec == 0) return fields::launch_range<double, LO, HI>(nc, P, rho, scratch, F, mu, s);   \
        if (prec == 1) return fields::launch_range<fz::DF64, LO, HI>(nc, P, rho, scratch, F, mu, s); \
        return fields::launch_range<float, LO, HI>(nc, P, rho, scratch, F, mu, s);                   \
    }                                                                                                 \
    }
