// lbm_fused2d.cuh -- single-pass D2Q9 time step.
//
// One launch per step.  The state is the post-streaming population set g(t)
// (Eq. 1a) plus the density state R(t) = sum_a g_{a,i}(t) per node and
// component, which the previous step produced on chip.  Each CTA owns a strip
// of W interior columns (one thread per column, plus one halo column on each
// side) and a segment of H rows, which it walks row by row:
//
//   row k   : load R(k) on columns [-3, W+3) -> psi(k) = sum_j sqrt(kappa_j) rho~_j
//   row k-1 : ln f_i (Eqs. 9-12) and mu_i = RT ln f_i - sqrt(kappa_i) lap psi
//             on columns [-2, W+2)   (Eq. 5 with Eq. 4: sum_j kappa_ij lap rho~_j
//             = sqrt(kappa_i) lap psi)
//   row k-2 : F_i = -rho~_i grad mu_i, grad rho_i, u = (sum e g + F/2)/rho,
//             equilibrium (Eq. 1b), forcing (Eq. 1c), BGK (Eq. 1a) on columns
//             [-1, W+1); push streaming of the interior columns to g(t+1);
//             the new densities R(t+1) of the interior are gathered from the
//             collided values of rows k-3..k-1 and columns -1..W in a fixed
//             order (no atomics), so R(t+1) needs no second pass over g.
//
// DRAM traffic per node-step: g read + g written (the algorithmic bytes) plus
// R read + R written (Nc values each); halo rows and columns come from L2.
// Storage S (double, or float deviation h = g - delta_a0 rhobar_i), EOS and
// force arithmetic E (double or float), collision arithmetic S.
#pragma once

#include <type_traits>

#include "lbm_internal.h"
#include "lbm_thermo_df.cuh"

namespace lbmfug {
namespace fz {

constexpr int kT = 128;     // threads per CTA: one column each
constexpr int kWmax = kT - 2;

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

template <int NC, typename S, typename E> struct Smem {
    static __host__ __device__ constexpr size_t rs(int W) { return align16((size_t)4 * NC * (W + 6) * sizeof(S)); }
    static __host__ __device__ constexpr size_t ps(int W) { return align16((size_t)3 * (W + 6) * sizeof(E)); }
    static __host__ __device__ constexpr size_t mu(int W) { return align16((size_t)3 * NC * (W + 4) * sizeof(E)); }
    static __host__ __device__ constexpr size_t xc() { return align16((size_t)6 * NC * kT * sizeof(S)); }
    static __host__ __device__ constexpr size_t red() { return align16((size_t)(kT / 32) * NC * sizeof(double)); }
    static __host__ __device__ constexpr size_t total(int W) { return rs(W) + ps(W) + mu(W) + xc() + red(); }
};

__device__ __forceinline__ int wrapc(int v, int n)
{
    if (v >= 0 && v < n) return v;
    v %= n;
    return v < 0 ? v + n : v;
}

template <int NC, typename S, typename E>
__global__ void __launch_bounds__(kT)
    k_fused(const Params P, const int W, const int H, const S *__restrict__ gin,
            S *__restrict__ gout, const S *__restrict__ rin, S *__restrict__ rout,
            double *__restrict__ mass_partials)
{
    using L = Lattice<0>;
    using V = PV<E>;
    using VS = PV<S>;
    constexpr bool kDev = sizeof(S) == 4;                 // deviation storage
    constexpr bool kKeep = 9 * NC * sizeof(S) <= 360;     // populations held in registers
    extern __shared__ __align__(16) unsigned char smem[];
    using SM = Smem<NC, S, E>;
    S *RS = (S *)smem;                                   // [4][NC][W+6]  R rows
    E *PS = (E *)(smem + SM::rs(W));                     // [3][W+6]      psi rows
    E *MU = (E *)(smem + SM::rs(W) + SM::ps(W));         // [3][NC][W+4]  mu rows
    S *XC = (S *)(smem + SM::rs(W) + SM::ps(W) + SM::mu(W));  // [6][NC][kT] exchange
    double *RED = (double *)(smem + SM::rs(W) + SM::ps(W) + SM::mu(W) + SM::xc());

    const int nx = P.nx, ny = P.ny;
    const long long N = P.N;
    const int CW = W + 6, CM = W + 4;
    const int x0 = blockIdx.x * W;
    const int w = min(W, nx - x0);
    const int y0 = blockIdx.y * H;
    const int h = min(H, ny - y0);
    const int t = threadIdx.x;
    const int col = t - 1;                 // collision column of this thread
    const bool active = t < w + 2;         // columns -1 .. w
    const bool interior = col >= 0 && col < w;
    const int xg = wrapc(x0 + col, nx);
    const int xd[3] = {wrapc(xg - 1, nx), xg, wrapc(xg + 1, nx)};  // destination columns, ex = -1, 0, 1
    // phase (A) columns of this thread: c = t - 3 and c = t - 3 + kT
    const int cA0 = t - 3, cA1 = t - 3 + kT;
    const bool hasA0 = cA0 < w + 3, hasA1 = cA1 < w + 3;
    const int xA0 = wrapc(x0 + cA0, nx), xA1 = hasA1 ? wrapc(x0 + cA1, nx) : 0;
    const E RT = V::RT(P);
    const S om = (S)P.omega, cF = (S)(1.0 - 0.5 * P.omega);

    S msum[NC], mcmp[NC];      // per-thread mass of the written rows (compensated)
    S accA[NC], accB[NC];
    S rp0[NC], rp1[NC];        // prefetched density state of the next row
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        msum[i] = 0;
        mcmp[i] = 0;
        accA[i] = 0;
        accB[i] = 0;
    }
    {
        const long long rowb = (long long)wrapc(y0 - 3, ny) * nx;
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            rp0[i] = hasA0 ? __ldg(rin + i * N + rowb + xA0) : (S)0;
            rp1[i] = hasA1 ? __ldg(rin + i * N + rowb + xA1) : (S)0;
        }
    }

    const int nrows = h + 6;  // rows y0-3 .. y0+h+2
    for (int kk = 0; kk < nrows; ++kk) {
        const int k = y0 - 3 + kk;
        // ---- (0) populations of the collision row k-2, in flight during (A), (B) ----
        const int crow = k - 2;
        const int yc = wrapc(crow, ny);
        const long long rc = (long long)yc * nx + xg;
        S hv[kKeep ? NC : 1][9];
        if (kKeep && kk >= 4 && active) {
#pragma unroll
            for (int i = 0; i < NC; ++i)
#pragma unroll
                for (int a = 0; a < 9; ++a) hv[kKeep ? i : 0][a] = __ldg(gin + (i * 9 + a) * N + rc);
        }
        // ---- (A) density state and psi of row k --------------------------------
        {
            const int s4 = kk & 3, s3 = kk % 3;
            if (hasA0) {
                E ps = 0;
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    RS[(s4 * NC + i) * CW + cA0 + 3] = rp0[i];
                    ps = fma(V::sqk(P, i), (V::rhobar(P, i) + (E)rp0[i]) * V::invM(P, i), ps);
                }
                PS[s3 * CW + cA0 + 3] = ps;
            }
            if (hasA1) {
                E ps = 0;
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    RS[(s4 * NC + i) * CW + cA1 + 3] = rp1[i];
                    ps = fma(V::sqk(P, i), (V::rhobar(P, i) + (E)rp1[i]) * V::invM(P, i), ps);
                }
                PS[s3 * CW + cA1 + 3] = ps;
            }
        }
        __syncthreads();
        // ---- (B) ln f and mu of row k-1 ------------------------------------------
        if (kk >= 2) {
            const int q = kk - 1;
            const int s4 = q & 3;
            const E *p0 = PS + ((q + 2) % 3) * CW;  // row q-1
            const E *p1 = PS + (q % 3) * CW;        // row q
            const E *p2 = PS + ((q + 1) % 3) * CW;  // row q+1
            for (int c = t - 2; c < w + 2; c += kT) {
                const int cc = c + 3;
                E rm[NC], lf[NC];
#pragma unroll
                for (int i = 0; i < NC; ++i)
                    rm[i] = (V::rhobar(P, i) + (E)RS[(s4 * NC + i) * CW + cc]) * V::invM(P, i);
                pr_lnf<NC, E>(P, rm, lf, nullptr);
                const E c0 = p1[cc];
                const E faces = (p1[cc + 1] - c0) + (p1[cc - 1] - c0) + (p2[cc] - c0) + (p0[cc] - c0);
                const E diags = (p2[cc + 1] - c0) + (p0[cc - 1] - c0) + (p0[cc + 1] - c0) + (p2[cc - 1] - c0);
                const E lap = (E)6 * fma((E)(1.0 / 9.0), faces, (E)(1.0 / 36.0) * diags);
#pragma unroll
                for (int i = 0; i < NC; ++i)
                    MU[((q % 3) * NC + i) * CM + c + 2] = fma(RT, lf[i], -V::sqk(P, i) * lap);
            }
        }
        __syncthreads();
        // ---- prefetch the density state of row k+1 (in flight during (C)) ---------
        if (kk + 1 < nrows) {
            const long long rowb = (long long)wrapc(k + 1, ny) * nx;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                if (hasA0) rp0[i] = __ldg(rin + i * N + rowb + xA0);
                if (hasA1) rp1[i] = __ldg(rin + i * N + rowb + xA1);
            }
        }
        if (kk < 4) continue;
        // ---- (C) collision of row k-2 --------------------------------------------
        const int q = kk - 2;
        const bool own_row = crow >= y0 && crow < y0 + h;
        S ownv[3][NC];  // collided values with dx = 0, by dy = -1, 0, +1
        if (active) {
            const long long yd[3] = {(long long)wrapc(yc - 1, ny) * nx, (long long)yc * nx,
                                     (long long)wrapc(yc + 1, ny) * nx};
            const int cc = col + 3, cm = col + 2;
            const S *R0 = RS + ((q + 3) & 3) * NC * CW;  // row q-1
            const S *R1 = RS + (q & 3) * NC * CW;        // row q
            const S *R2 = RS + ((q + 1) & 3) * NC * CW;  // row q+1
            const E *M0 = MU + ((q + 2) % 3) * NC * CM;
            const E *M1 = MU + (q % 3) * NC * CM;
            const E *M2 = MU + ((q + 1) % 3) * NC * CM;
            // momentum sum_i sum_a e_a g_{a,i}
            S jx = 0, jy = 0;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                S v[9];
#pragma unroll
                for (int a = 0; a < 9; ++a)
                    v[a] = kKeep ? hv[kKeep ? i : 0][a] : __ldg(gin + (i * 9 + a) * N + rc);
                jx += (v[1] - v[2]) + (v[5] - v[6]) + (v[7] - v[8]);
                jy += (v[3] - v[4]) + (v[5] - v[6]) + (v[8] - v[7]);
            }
            // Eq. (5): F_i = -rho~_i grad mu_i
            S Fx[NC], Fy[NC];
            E Fsx = 0, Fsy = 0, rt = 0;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const E *m0 = M0 + i * CM, *m1 = M1 + i * CM, *m2 = M2 + i * CM;
                // grad X = 3 sum_pairs w e (X(r+e) - X(r-e)): faces 1/9, diagonals 1/36
                const E dE = m1[cm + 1] - m1[cm - 1];
                const E dN = m2[cm] - m0[cm];
                const E dNE = m2[cm + 1] - m0[cm - 1];
                const E dSE = m0[cm + 1] - m2[cm - 1];
                const E gx = (E)3 * fma((E)(1.0 / 9.0), dE, (E)(1.0 / 36.0) * (dNE + dSE));
                const E gy = (E)3 * fma((E)(1.0 / 9.0), dN, (E)(1.0 / 36.0) * (dNE - dSE));
                const E ri = V::rhobar(P, i) + (E)R1[i * CW + cc];
                rt += ri;
                const E rmi = ri * V::invM(P, i);
                const E fx = -rmi * gx, fy = -rmi * gy;
                Fsx += fx;
                Fsy += fy;
                Fx[i] = (S)fx;
                Fy[i] = (S)fy;
            }
            const E irt = (E)1 / rt;
            const S ux = (S)(fma((E)0.5, Fsx, (E)jx) * irt);
            const S uy = (S)(fma((E)0.5, Fsy, (E)jy) * irt);
            const S u2 = ux * ux + uy * uy;
            // per-direction scalars (component independent)
            S ue[9], Bq[9], c9[9];
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                ue[a] = (S)L::e(a, 0) * ux + (S)L::e(a, 1) * uy;
                Bq[a] = ue[a] * fma((S)4.5, ue[a], (S)3) - (S)1.5 * u2;
                c9[a] = fma((S)9, ue[a], (S)3);
            }
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const S *r0 = R0 + i * CW, *r1 = R1 + i * CW, *r2 = R2 + i * CW;
                const S dE = r1[cc + 1] - r1[cc - 1];
                const S dN = r2[cc] - r0[cc];
                const S dNE = r2[cc + 1] - r0[cc - 1];
                const S dSE = r0[cc + 1] - r2[cc - 1];
                const S Gx = (S)3 * fma((S)(1.0 / 9.0), dE, (S)(1.0 / 36.0) * (dNE + dSE));
                const S Gy = (S)3 * fma((S)(1.0 / 9.0), dN, (S)(1.0 / 36.0) * (dNE - dSE));
                const S dri = r1[cc];                          // rho_i - rhobar_i
                const S ri = VS::rhobar(P, i) + dri;
                const S Fu3 = (S)3 * (Fx[i] * ux + Fy[i] * uy);
                const S Gu = Gx * ux + Gy * uy;
                S v[9];
#pragma unroll
                for (int a = 0; a < 9; ++a)
                    v[a] = kKeep ? hv[kKeep ? i : 0][a] : __ldg(gin + (i * 9 + a) * N + rc);
                S others = 0;  // sum of the moving populations of this node
                if (kDev)
#pragma unroll
                    for (int a = 1; a < 9; ++a) others += v[a];
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const int ex = L::e(a, 0), ey = L::e(a, 1);
                    const S wa = (S)L::w(a);
                    const S Fe = (S)ex * Fx[i] + (S)ey * Fy[i];
                    const S Ge = (S)ex * Gx + (S)ey * Gy;
                    const S cW = (S)(0.5 * (3.0 * (ex * ex + ey * ey) - 2.0) - 1.0);
                    // Eq. (1c): F.[(e-u)/cs2 + (u.e)e/cs4] + grad rho.[-u + (u.e)e/cs2 + (e^2/cs2 - D)u/2]
                    const S Fa = wa * (fma(Fe, c9[a], -Fu3) + fma((S)3 * ue[a], Ge, cW * Gu));
                    S gs;
                    if (kDev && a == 0) {
                        // Eq. (1a) at rest with Eq. (1b): h0 + w (sum_a h_a - h0 + w0 rho B0) + cF F0,
                        // the node's own populations carrying its mass exactly
                        gs = v[0] + fma(om, others + wa * ri * Bq[0], cF * Fa);
                    } else {
                        const S geq = wa * ri * Bq[a] + (a == 0 ? dri : (S)0);
                        gs = fma(om, geq - v[a], v[a]) + cF * Fa;
                    }
                    if (interior && own_row) gout[(i * 9 + a) * N + yd[ey + 1] + xd[ex + 1]] = gs;
                    if (ex == 0)
                        ownv[ey + 1][i] = gs;
                    else
                        XC[(((ey + 1) * 2 + (ex > 0 ? 0 : 1)) * NC + i) * kT + t] = gs;
                }
            }
        }
        __syncthreads();
        // ---- gather R(t+1) of the interior columns ---------------------------------
        if (interior) {
            const bool write_row = (crow - 1) >= y0 && (crow - 1) < y0 + h;
            const long long rw = (long long)wrapc(crow - 1, ny) * nx + xg;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                S Pd[3];
#pragma unroll
                for (int dy = 0; dy < 3; ++dy)
                    Pd[dy] = (XC[((dy * 2 + 0) * NC + i) * kT + t - 1] + ownv[dy][i]) +
                             XC[((dy * 2 + 1) * NC + i) * kT + t + 1];
                accA[i] += Pd[0];  // row crow-1 now complete
                if (write_row) {
                    rout[i * N + rw] = accA[i];
                    // compensated (Kahan) running sum of the written densities
                    const S yv = accA[i] - mcmp[i];
                    const S tv = msum[i] + yv;
                    mcmp[i] = (tv - msum[i]) - yv;
                    msum[i] = tv;
                }
                accA[i] = accB[i] + Pd[1];
                accB[i] = Pd[2];
            }
        }
    }
    if (mass_partials) {
        // deterministic block reduction of the mass of the rows written
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            double v = (double)msum[i] - (double)mcmp[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((t & 31) == 0) RED[(t >> 5) * NC + i] = v;
        }
        __syncthreads();
        if (t < NC) {
            double s = 0.0;
            for (int wv = 0; wv < kT / 32; ++wv) s += RED[wv * NC + t];
            s += P.rhobar[t] * (double)w * (double)h;
            mass_partials[((long long)blockIdx.y * gridDim.x + blockIdx.x) * NC + t] = s;
        }
    }
}

// Thermodynamics arithmetic of the binary32-state kernel: binary32 (LBM_FP32,
// evaluated inside the step kernel) or double-binary32 (LBM_FP32DEV: a
// separate pass, k_mu32, writes mu as (hi, lo) pairs, which the step kernel
// reads).  ET is the shared-memory type of mu: one binary32 value, or a pair.
struct DF64 {};
template <typename E> struct ThermoT { using ET = float; };
template <> struct ThermoT<DF64> { using ET = float2; };

// Shared rows of the binary32 kernel have a fixed pitch of kT entries (a strip
// needs at most W + 6 <= kT), so every row offset is a compile-time constant.
// The exchange XC holds the collided values that move to a neighbouring
// column (6 slots: row below, same row, row above; to the right or left).
template <int NC, typename E> struct Smem32 {
    using ET = typename ThermoT<E>::ET;
    static constexpr bool kDF = sizeof(ET) == 8;
    static __host__ __device__ constexpr size_t rs(int) { return align16((size_t)4 * NC * kT * sizeof(float)); }
    static __host__ __device__ constexpr size_t ps(int) { return kDF ? 0 : align16((size_t)3 * kT * sizeof(float)); }
    static __host__ __device__ constexpr size_t mu(int) { return kDF ? 0 : align16((size_t)3 * NC * kT * sizeof(ET)); }
    static __host__ __device__ constexpr size_t xc() { return align16((size_t)6 * NC * kT * sizeof(float)); }
    static __host__ __device__ constexpr size_t red() { return align16((size_t)(kT / 32) * NC * sizeof(double)); }
    static __host__ __device__ constexpr size_t ms() { return align16((size_t)2 * NC * kT * sizeof(float)); }
    static __host__ __device__ constexpr size_t total(int W)
    {
        return 2 * rs(W) + ps(W) + mu(W) + xc() + red() + ms();
    }
};
constexpr int kWmax32 = kT - 6;  // binary32 kernel: one density column per thread

// Double-binary32 chemical potentials and their gradients (LBM_FP32DEV), one
// pass before the step kernel.  Each CTA walks a segment of rows of a strip
// of W <= kT - 4 columns; for row k it forms
//   psi(k) (Eq. 4) on columns [-2, W + 1] from the state's exact density pairs,
//     with B(k) = b_m rho~ (Eq. 11) in the same packed sum,
//   mu(k-1) (Eqs. 5, 9-12 through lbm_thermo_df.cuh) on columns [-1, W] from
//     psi rows k-2..k and the pairs and B of row k-1 kept from the previous row,
//   grad mu(k-2) on the interior columns from mu rows k-3..k-1, every
//     difference mu(r + e) - mu(r - e) taken on the (hi, lo) pairs and
//     rounded once (so it carries the df64 accuracy of mu), written to
//     G[i][node] = (d mu_i / dx, d mu_i / dy) in binary32.
// The step kernel forms F_i = -rho~_i G_i.  psi and mu rows live in rings of
// three: a slot is rewritten only after the barrier that follows its last
// reader.  mu_rolled keeps T_i in the thread's own mu slots of the row it is
// writing (it reads T_i just before it writes mu_i there), and the log table
// is split into {v, -ln v hi} pairs and lo words, so that a CTA needs 44.5 KB
// of shared memory at Nc = 10 and five fit on an SM.
constexpr int kWmaxMu = kT - 4;

template <int NC> struct SmemMu {
    static __host__ __device__ constexpr size_t bytes()
    {
        // log table (pairs, lo words), psi ring, mu ring, density-pair scratch of mu_rolled
        return (size_t)df::kLogTab * (sizeof(float2) + sizeof(float)) + 3 * kT * sizeof(float2) +
               3 * NC * kT * sizeof(float2) + 2 * (size_t)NC * kT * sizeof(float);
    }
};

template <int NC, typename IDX>
__global__ void __launch_bounds__(kT) k_mu32(const Params P, const int W, const int H, StateBufs in,
                                             float2 *__restrict__ G)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *LV = (float2 *)smem;          // [128] {v_j, -ln v_j hi}
    float *LL = (float *)(LV + df::kLogTab);  // [128] -ln v_j lo
    float2 *PS = (float2 *)(LL + df::kLogTab);  // [3][kT]
    float2 *MU = PS + 3 * kT;             // [3][NC][kT]
    float *PHs = (float *)(MU + 3 * NC * kT);  // [NC][kT] pair hi
    float *PLs = PHs + NC * kT;           // [NC][kT] pair lo
    const int nx = P.nx, ny = P.ny;
    const IDX N = (IDX)P.N;
    const int x0 = blockIdx.x * W;
    const int w = min(W, nx - x0);
    const int y0 = blockIdx.y * H;
    const int h = min(H, ny - y0);
    const int t = threadIdx.x;
    const int c = t - 2;  // column of this thread, -2 .. w + 1
    const bool hasP = c <= w + 1;
    const bool hasM = c >= -1 && c <= w;
    const bool interior = c >= 0 && c < w;
    const int xg = wrapc(x0 + c, nx);
    const float *rhin = in.rhi_f();
    const float *rlin = in.rlo;
    for (int j = t; j < df::kLogTab; j += kT) {
        LV[j] = make_float2(P.logtab[j].x, P.logtab[j].y);
        LL[j] = P.logtab[j].z;
    }
    const df::TabSplit LT{LV, LL};
    float ph[NC], pl[NC];  // density pairs of row k-1 at this column
    df::F2 Bp = {0.0f, 0.0f};  // and its B (Eq. 11)
#pragma unroll
    for (int i = 0; i < NC; ++i) ph[i] = pl[i] = 0.0f;
    for (int kk = 0; kk < h + 4; ++kk) {
        const int k = y0 - 2 + kk;
        float hh[NC], ll[NC];
        df::F2 Bk = {0.0f, 0.0f};
        if (hasP) {
            const IDX rb = (IDX)wrapc(k, ny) * (IDX)nx + (IDX)xg;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                hh[i] = __ldg(rhin + i * N + rb);
                ll[i] = __ldg(rlin + i * N + rb);
            }
            df::F2 ps;
            df::psi_and_B<NC>(P, hh, ll, ps, Bk);
            PS[(kk % 3) * kT + t] = make_float2(ps.hi, ps.lo);
        }
        __syncthreads();
        if (kk >= 2 && kk < h + 4 && hasM) {
            const float2 *p0 = PS + ((kk - 2) % 3) * kT, *p1 = PS + ((kk - 1) % 3) * kT, *p2 = PS + (kk % 3) * kT;
            const df::F2 lap = df::lap9(df::f2(p1[t]), df::f2(p1[t + 1]), df::f2(p1[t - 1]), df::f2(p2[t]),
                                        df::f2(p0[t]), df::f2(p2[t + 1]), df::f2(p2[t - 1]), df::f2(p0[t + 1]),
                                        df::f2(p0[t - 1]));
            float2 *out = MU + ((kk - 1) % 3) * NC * kT + t;
            df::mu_rolled<NC>(P, LT, ph, pl, Bp, lap, PHs + t, PLs + t, out, kT, out, kT);
        }
        if (hasP) {
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                ph[i] = hh[i];
                pl[i] = ll[i];
            }
            Bp = Bk;
        }
        __syncthreads();
        if (kk >= 4 && interior) {
            // gradient of mu at row k-2: rows k-3 (south), k-2, k-1 (north)
            const float2 *S = MU + ((kk - 3) % 3) * NC * kT, *C = MU + ((kk - 2) % 3) * NC * kT,
                         *Nr = MU + ((kk - 1) % 3) * NC * kT;
            const IDX ob = (IDX)wrapc(k - 2, ny) * (IDX)nx + (IDX)xg;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const float2 *s0 = S + i * kT, *c0 = C + i * kT, *n0 = Nr + i * kT;
                const float2 e1 = c0[t + 1], w1 = c0[t - 1], n1 = n0[t], s1 = s0[t];
                const float2 ne = n0[t + 1], sw = s0[t - 1], se = s0[t + 1], nw = n0[t - 1];
                const float dE = (e1.x - w1.x) + (e1.y - w1.y);
                const float dN = (n1.x - s1.x) + (n1.y - s1.y);
                const float dNE = (ne.x - sw.x) + (ne.y - sw.y);
                const float dSE = (se.x - nw.x) + (se.y - nw.y);
                // grad X = 3 sum_pairs w e (X(r+e) - X(r-e)): faces 1/9, diagonals 1/36
                const float gx = 3.0f * fmaf(1.0f / 9.0f, dE, (1.0f / 36.0f) * (dNE + dSE));
                const float gy = 3.0f * fmaf(1.0f / 9.0f, dN, (1.0f / 36.0f) * (dNE - dSE));
                G[i * N + ob] = make_float2(gx, gy);
            }
        }
    }
}

// Binary32 state: the 8 moving populations g[i][a-1][node] (a = 1..8) and the
// density rho_i = hi + lo.  Collision arithmetic in binary32; thermodynamics
// and forces in E.  The new density of a node is its old density minus the
// populations that left it plus those that arrived: every stored binary32
// population is added once where it arrives and subtracted once where it
// left, each by an error-free Fast2Sum into the (hi, lo) pair of the node,
// so the component mass is conserved to the rounding of the pairs.
// Fast2Sum is exact when |hi| >= |term|, i.e. when no single moving
// population exceeds the density of the node it leaves or enters.
__device__ __forceinline__ void pair_acc(float &hi, float &lo, float x)
{
    const float s = hi + x;
    lo += x - (s - hi);
    hi = s;
}

template <int NC, typename E, typename IDX>
__global__ void __launch_bounds__(kT)
    k_fused32(const Params P, const int W, const int H, StateBufs in, StateBufs out,
              double *__restrict__ mass_partials, const float2 *__restrict__ mug /* grad mu, DF64 */)
{
    using L = Lattice<0>;
    using SM = Smem32<NC, E>;
    using ET = typename SM::ET;
    constexpr bool kDF = SM::kDF;
    using VF = PV<float>;
    extern __shared__ __align__(16) unsigned char smem[];
    float *RS = (float *)smem;                                   // [4][NC][kT] rho hi rows
    float *RL = (float *)(smem + SM::rs(W));                     // [4][NC][kT] rho lo rows
    float *PS = (float *)(smem + 2 * SM::rs(W));                 // [3][kT]     psi rows (binary32 only)
    ET *MU = (ET *)((unsigned char *)PS + SM::ps(W));            // [3][NC][kT] mu rows
    float *XC = (float *)((unsigned char *)MU + SM::mu(W));      // [6][NC][kT] exchange
    double *RED = (double *)((unsigned char *)XC + SM::xc());
    float *MS = (float *)((unsigned char *)RED + SM::red());     // [2][NC][kT] mass of rows written
    const float *gin = (const float *)in.g;
    float *gout = (float *)out.g;
    const float *rhin = in.rhi_f();
    const float *rlin = in.rlo;

    const int nx = P.nx, ny = P.ny;
    const IDX N = (IDX)P.N;
    constexpr int CW = kT, CM = kT;  // row pitch (columns used: W + 6 and W + 4)
    const int x0 = blockIdx.x * W;
    const int w = min(W, nx - x0);
    const int y0 = blockIdx.y * H;
    const int h = min(H, ny - y0);
    const int t = threadIdx.x;
    const int col = t - 1;
    const bool active = t < w + 2;
    const bool interior = col >= 0 && col < w;
    const int xg = wrapc(x0 + col, nx);
    const int xd[3] = {wrapc(xg - 1, nx), xg, wrapc(xg + 1, nx)};
    // phase (A): one density column per thread (strips are at most kT - 6 wide)
    const int cA0 = t - 3;
    const bool hasA0 = cA0 < w + 3;
    const int xA0 = wrapc(x0 + cA0, nx);
    const float om = (float)P.omega, om1 = (float)(1.0 - P.omega), cF = (float)(1.0 - 0.5 * P.omega);

#pragma unroll
    for (int i = 0; i < NC; ++i) {
        MS[(0 * NC + i) * kT + t] = 0.0f;
        MS[(1 * NC + i) * kT + t] = 0.0f;
    }
    float aH[NC], aL[NC], bH[NC], bL[NC];  // density pairs being updated: rows crow-1, crow
    float rh0[NC], rl0[NC];                // prefetched density pair of the next row
#pragma unroll
    for (int i = 0; i < NC; ++i) aH[i] = aL[i] = bH[i] = bL[i] = 0.0f;
    {
        const IDX rowb = (IDX)wrapc(y0 - 3, ny) * (IDX)nx;
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            rh0[i] = hasA0 ? __ldg(rhin + i * N + rowb + xA0) : 0.0f;
            rl0[i] = hasA0 ? __ldg(rlin + i * N + rowb + xA0) : 0.0f;
        }
    }

    const int nrows = h + 6;
    for (int kk = 0; kk < nrows; ++kk) {
        const int k = y0 - 3 + kk;
        const int crow = k - 2;
        // ---- (A) density pair (and binary32 psi) of row k --------------------------
        {
            const int s4 = kk & 3, s3 = kk % 3;
            if (hasA0) {
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    RS[(s4 * NC + i) * CW + cA0 + 3] = rh0[i];
                    RL[(s4 * NC + i) * CW + cA0 + 3] = rl0[i];
                }
                if constexpr (!kDF) {
                    float ps = 0.0f;
#pragma unroll
                    for (int i = 0; i < NC; ++i) ps = fmaf(VF::sqk(P, i), (rh0[i] + rl0[i]) * VF::invM(P, i), ps);
                    PS[s3 * CW + cA0 + 3] = ps;
                }
            }
        }
        __syncthreads();
        // ---- (B) binary32: ln f and mu of row k-1 ----------------------------------
        if constexpr (!kDF) {
            if (kk >= 2) {
                const int q = kk - 1;
                const int s4 = q & 3;
                const float *p0 = PS + ((q + 2) % 3) * CW;
                const float *p1 = PS + (q % 3) * CW;
                const float *p2 = PS + ((q + 1) % 3) * CW;
                for (int c = t - 2; c < w + 2; c += kT) {
                    const int cc = c + 3;
                    float rm[NC], lf[NC];
#pragma unroll
                    for (int i = 0; i < NC; ++i)
                        rm[i] = (RS[(s4 * NC + i) * CW + cc] + RL[(s4 * NC + i) * CW + cc]) * VF::invM(P, i);
                    pr_lnf<NC, float>(P, rm, lf, nullptr);
                    const float c0 = p1[cc];
                    const float faces = (p1[cc + 1] - c0) + (p1[cc - 1] - c0) + (p2[cc] - c0) + (p0[cc] - c0);
                    const float diags = (p2[cc + 1] - c0) + (p0[cc - 1] - c0) + (p0[cc + 1] - c0) + (p2[cc - 1] - c0);
                    const float lap = 6.0f * fmaf(1.0f / 9.0f, faces, (1.0f / 36.0f) * diags);
                    const float RT = VF::RT(P);
#pragma unroll
                    for (int i = 0; i < NC; ++i)
                        MU[((q % 3) * NC + i) * CM + c + 2] = fmaf(RT, lf[i], -VF::sqk(P, i) * lap);
                }
            }
            __syncthreads();
        }
        // density pair of row k+1 for phase (A) of the next row: issued here
        // before the first collision row, in the density update after it
        const IDX rowb1 = (IDX)wrapc(k + 1, ny) * (IDX)nx + (IDX)xA0;
        if (kk < 4) {
            if (kk + 1 < nrows && hasA0) {
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    rh0[i] = __ldg(rhin + i * N + rowb1);
                    rl0[i] = __ldg(rlin + i * N + rowb1);
                }
            }
            continue;
        }
        // ---- (C) collision of row k-2 (moving populations only) --------------------
        const int q = kk - 2;
        const bool own_row = crow >= y0 && crow < y0 + h;
        const int yc = wrapc(crow, ny);
        float own0[NC], own2[NC];  // dx = 0 moving values, dy = -1 and +1
        if (active) {
            const IDX yd[3] = {(IDX)wrapc(yc - 1, ny) * (IDX)nx, (IDX)yc * (IDX)nx,
                               (IDX)wrapc(yc + 1, ny) * (IDX)nx};
            IDX dst[9];
#pragma unroll
            for (int a = 1; a < 9; ++a) dst[a] = yd[L::e(a, 1) + 1] + (IDX)xd[L::e(a, 0) + 1];
            const int cc = col + 3, cm = col + 2;
            const float *R0 = RS + ((q + 3) & 3) * NC * CW;
            const float *R1 = RS + (q & 3) * NC * CW;
            const float *R2 = RS + ((q + 1) & 3) * NC * CW;
            const ET *M0 = MU + ((q + 2) % 3) * NC * CM;
            const ET *M1 = MU + (q % 3) * NC * CM;
            const ET *M2 = MU + ((q + 1) % 3) * NC * CM;
            const IDX rc = (IDX)yc * (IDX)nx + (IDX)xg;
            float hv[NC][8];
            float2 gm[kDF ? NC : 1];  // double-binary32: grad mu_i from k_mu32
#pragma unroll
            for (int i = 0; i < NC; ++i) {
#pragma unroll
                for (int a = 0; a < 8; ++a) hv[i][a] = __ldg(gin + (i * 8 + a) * N + rc);
                if constexpr (kDF) gm[i] = __ldg(mug + i * N + rc);
            }
            float jx = 0.0f, jy = 0.0f;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const float *v = hv[i];  // v[a - 1] = g_a, a = 1..8
                jx += (v[0] - v[1]) + (v[4] - v[5]) + (v[6] - v[7]);
                jy += (v[2] - v[3]) + (v[4] - v[5]) + (v[7] - v[6]);
            }
            // Eq. (5): F_i = -rho~_i grad mu_i, grad X = 3 sum_pairs w e (X(r+e) - X(r-e));
            // double-binary32: the gradient comes from k_mu32
            float Fx[NC], Fy[NC], rlo1[NC];
            float Fsx = 0.0f, Fsy = 0.0f, rt = 0.0f;
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                float gx, gy;
                if constexpr (kDF) {
                    gx = gm[i].x;
                    gy = gm[i].y;
                } else {
                    const ET *m0 = M0 + i * CM, *m1 = M1 + i * CM, *m2 = M2 + i * CM;
                    const float dE = m1[cm + 1] - m1[cm - 1];
                    const float dN = m2[cm] - m0[cm];
                    const float dNE = m2[cm + 1] - m0[cm - 1];
                    const float dSE = m0[cm + 1] - m2[cm - 1];
                    gx = 3.0f * fmaf(1.0f / 9.0f, dE, (1.0f / 36.0f) * (dNE + dSE));
                    gy = 3.0f * fmaf(1.0f / 9.0f, dN, (1.0f / 36.0f) * (dNE - dSE));
                }
                rlo1[i] = RL[((q & 3) * NC + i) * CW + cc];
                const float ri = R1[i * CW + cc] + rlo1[i];
                rt += ri;
                const float rmi = ri * VF::invM(P, i);
                Fx[i] = -rmi * gx;
                Fy[i] = -rmi * gy;
                Fsx += Fx[i];
                Fsy += Fy[i];
            }
            const float irt = __fdividef(1.0f, rt);
            const float ux = fmaf(0.5f, Fsx, jx) * irt;
            const float uy = fmaf(0.5f, Fsy, jy) * irt;
            const float u2 = ux * ux + uy * uy;
            // Eqs. (1a)-(1c) over the four pairs of opposite directions (a, a+1):
            //   g*_a = (1 - w) g_a + sym +- anti,
            //   sym  = rho_i WBs + cw [3ue (3Fe + Ge) + K],  anti = rho_i WBa + 3 cw Fe,
            // WBs = w w_a (4.5 ue^2 - 1.5 u^2), WBa = 3 w w_a ue, cw = (1 - w/2) w_a,
            // ue = e_a.u, Fe = e_a.F_i, Ge = e_a.grad rho_i, K the class term
            float WBs[4], WBa[4], U3[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const int a = 2 * p + 1;
                const float ue = (float)L::e(a, 0) * ux + (float)L::e(a, 1) * uy;
                const float ow = om * (float)L::w(a);
                WBs[p] = ow * fmaf(4.5f * ue, ue, -1.5f * u2);
                WBa[p] = (3.0f * ow) * ue;
                U3[p] = 3.0f * ue;
            }
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const float *r0 = R0 + i * CW, *r1 = R1 + i * CW, *r2 = R2 + i * CW;
                const float dE = r1[cc + 1] - r1[cc - 1];
                const float dN = r2[cc] - r0[cc];
                const float dNE = r2[cc + 1] - r0[cc - 1];
                const float dSE = r0[cc + 1] - r2[cc - 1];
                const float Gx = 3.0f * fmaf(1.0f / 9.0f, dE, (1.0f / 36.0f) * (dNE + dSE));
                const float Gy = 3.0f * fmaf(1.0f / 9.0f, dN, (1.0f / 36.0f) * (dNE - dSE));
                const float ri = r1[cc] + rlo1[i];
                const float Fu3 = 3.0f * (Fx[i] * ux + Fy[i] * uy);
                const float Gu = Gx * ux + Gy * uy;
                // class term: faces -Gu/2 - 3F.u, diagonals Gu - 3F.u
                const float Kf = fmaf(-0.5f, Gu, -Fu3), Kd = Gu - Fu3;
                const float *v = hv[i];  // v[a - 1] = g_a, a = 1..8
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const int a = 2 * p + 1;  // e_{a+1} = -e_a
                    const int ex = L::e(a, 0), ey = L::e(a, 1);
                    const float cw = cF * (float)L::w(a);
                    const float Fe = (float)ex * Fx[i] + (float)ey * Fy[i];
                    const float Ge = (float)ex * Gx + (float)ey * Gy;
                    const float S = fmaf(U3[p], fmaf(3.0f, Fe, Ge), (ex != 0 && ey != 0) ? Kd : Kf);
                    const float sym = fmaf(ri, WBs[p], cw * S);
                    const float anti = fmaf(ri, WBa[p], (3.0f * cw) * Fe);
                    const float gp = fmaf(om1, v[a - 1], sym + anti);
                    const float gm = fmaf(om1, v[a], sym - anti);
                    // each departure leaves the pair of row crow (bH, bL) by its own Fast2Sum
                    pair_acc(bH[i], bL[i], -gp);
                    pair_acc(bH[i], bL[i], -gm);
#pragma unroll
                    for (int sgn = 0; sgn < 2; ++sgn) {
                        const int b = a + sgn;
                        const float gs = sgn ? gm : gp;
                        const int bx = L::e(b, 0), by = L::e(b, 1);
                        if (interior && own_row) gout[(i * 8 + b - 1) * N + dst[b]] = gs;
                        if (bx == 0) {
                            if (by < 0) own0[i] = gs;
                            else own2[i] = gs;
                        } else {
                            XC[(((by + 1) * 2 + (bx > 0 ? 0 : 1)) * NC + i) * kT + t] = gs;
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (kk + 1 < nrows && hasA0) {
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                rh0[i] = __ldg(rhin + i * N + rowb1);
                rl0[i] = __ldg(rlin + i * N + rowb1);
            }
        }
        // ---- density update of the interior columns ---------------------------------
        if (interior) {
            const bool write_row = (crow - 1) >= y0 && (crow - 1) < y0 + h;
            const IDX rw = (IDX)wrapc(crow - 1, ny) * (IDX)nx + (IDX)xg;
            const int cc = col + 3;
            const float *Rh2 = RS + ((q + 1) & 3) * NC * CW;  // row crow+1
#pragma unroll
            for (int i = 0; i < NC; ++i) {
                const float *xc = XC + i * kT;  // slot s of component i at xc[s * NC * kT]
                // row crow-1: last arrivals complete its update
                pair_acc(aH[i], aL[i], xc[0 * NC * kT + t - 1]);
                pair_acc(aH[i], aL[i], own0[i]);
                pair_acc(aH[i], aL[i], xc[1 * NC * kT + t + 1]);
                if (write_row) {
                    const float hi = aH[i] + aL[i];
                    const float lo = aL[i] - (hi - aH[i]);
                    out.rhi_f()[i * N + rw] = hi;
                    out.rlo[i * N + rw] = lo;
                    float ms = MS[(0 * NC + i) * kT + t], mc = MS[(1 * NC + i) * kT + t];
                    acc_add(ms, mc, hi);
                    MS[(0 * NC + i) * kT + t] = ms;
                    MS[(1 * NC + i) * kT + t] = mc + lo;
                }
                // row crow (its departures left during the collision): arrivals along the row
                aH[i] = bH[i];
                aL[i] = bL[i];
                pair_acc(aH[i], aL[i], xc[2 * NC * kT + t - 1]);
                pair_acc(aH[i], aL[i], xc[3 * NC * kT + t + 1]);
                // row crow+1: its old density, then the first arrivals
                bH[i] = Rh2[i * CW + cc];
                bL[i] = RL[(((q + 1) & 3) * NC + i) * CW + cc];
                pair_acc(bH[i], bL[i], xc[4 * NC * kT + t - 1]);
                pair_acc(bH[i], bL[i], own2[i]);
                pair_acc(bH[i], bL[i], xc[5 * NC * kT + t + 1]);
            }
        }
    }
    if (mass_partials) {
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            double v = (double)MS[(0 * NC + i) * kT + t] + (double)MS[(1 * NC + i) * kT + t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((t & 31) == 0) RED[(t >> 5) * NC + i] = v;
        }
        __syncthreads();
        if (t < NC) {
            double s = 0.0;
            for (int wv = 0; wv < kT / 32; ++wv) s += RED[wv * NC + t];
            mass_partials[((long long)blockIdx.y * gridDim.x + blockIdx.x) * NC + t] = s;
        }
    }
}

// R(0) = sum_a g_{a,i} for every node (fixed order a = 0..8).
template <int NC, typename S>
__global__ void k_density(const Params P, const S *__restrict__ g, S *__restrict__ R)
{
    const long long N = P.N;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
         r += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            S s = 0;
#pragma unroll
            for (int a = 0; a < 9; ++a) s += g[(i * 9 + a) * N + r];
            R[i * N + r] = s;
        }
    }
}

struct Ops {
    int wmax;
    int (*density)(const Params &, StateBufs, cudaStream_t);
    // one step; mu: the gradient buffer of the double-binary32 chemical
    // potentials, [nc][N] (d/dx, d/dy) (LBM_FP32DEV), else unused.  Returns the launches made through *launches.
    int (*step)(const Params &, const FusedGeom &, StateBufs, StateBufs, double *, float2 *mu, int *launches,
                KernelTimer *, cudaStream_t);
    size_t (*smem)(int W);
    int (*occupancy)(size_t smem);
    int (*occupancy_mu)();  // CTAs per SM of the mu pass (0: the form has none)
};

// S = double: binary64 kernel (all populations, binary64 densities).
// S = float:  binary32 kernel with thermodynamics in E (DF64: a mu pass first).
template <int NC, typename S, typename E> struct Impl {
    static constexpr bool k64 = sizeof(S) == 8;
    static constexpr bool kDF = std::is_same<E, DF64>::value;
    static auto kernel()
    {
        if constexpr (k64) return k_fused<NC, double, double>;
        else return k_fused32<NC, E, long long>;
    }
    static constexpr int wmax() { return k64 ? kWmax : kWmax32; }
    static int density(const Params &P, StateBufs st, cudaStream_t s)
    {
        if constexpr (k64) {
            long long b = (P.N + 255) / 256;
            if (b > 152 * 32) b = 152 * 32;
            k_density<NC, double><<<(unsigned)b, 256, 0, s>>>(P, (const double *)st.g, st.rhi_d());
        }
        return (int)cudaGetLastError();
    }
    static size_t smem(int W)
    {
        if constexpr (k64) return Smem<NC, double, double>::total(W);
        else return Smem32<NC, E>::total(W);
    }
    static int occupancy(size_t bytes)
    {
        // the limit is the widest strip's need, so that problems of other
        // widths launched later keep fitting under it
        if (cudaFuncSetAttribute(kernel(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem(wmax())) != cudaSuccess)
            return 0;
        if constexpr (!k64)
            if (cudaFuncSetAttribute(k_fused32<NC, E, int>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem(wmax())) != cudaSuccess)
                return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel(), kT, bytes) != cudaSuccess)
            return 0;
        return n;
    }
    static int occupancy_mu()
    {
        if constexpr (kDF) {
            const size_t b = SmemMu<NC>::bytes();
            if (cudaFuncSetAttribute(k_mu32<NC, long long>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b) !=
                    cudaSuccess ||
                cudaFuncSetAttribute(k_mu32<NC, int>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b) !=
                    cudaSuccess)
                return 0;
            int n = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_mu32<NC, long long>, kT, b) != cudaSuccess)
                return 0;
            return n;
        } else {
            return 0;
        }
    }
    static int step(const Params &P, const FusedGeom &g, StateBufs in, StateBufs out, double *mp, float2 *mu,
                    int *launches, KernelTimer *kt, cudaStream_t s)
    {
        dim3 grid(g.nstrips, g.segs);
        const bool small = (long long)NC * 8 * P.N < (1LL << 31);
        *launches = 1;
        if constexpr (k64) {
            kt_begin(kt, kKtStep, s);
            k_fused<NC, double, double><<<grid, kT, g.smem, s>>>(
                P, g.strip, g.seg_h, (const double *)in.g, (double *)out.g, in.rhi_d(),
                out.rhi_d(), mp);
            kt_end(kt, s);
        } else {
            if constexpr (kDF) {
                if (!mu) return (int)cudaErrorInvalidValue;
                dim3 mgrid(g.mnstrips, g.msegs);
                const size_t b = SmemMu<NC>::bytes();
                kt_begin(kt, kKtMuPass, s);
                if (small)
                    k_mu32<NC, int><<<mgrid, kT, b, s>>>(P, g.mstrip, g.mseg_h, in, mu);
                else
                    k_mu32<NC, long long><<<mgrid, kT, b, s>>>(P, g.mstrip, g.mseg_h, in, mu);
                kt_end(kt, s);
                *launches = 2;
            }
            kt_begin(kt, kKtStep, s);
            if (small)
                k_fused32<NC, E, int><<<grid, kT, g.smem, s>>>(P, g.strip, g.seg_h, in, out, mp, mu);
            else
                k_fused32<NC, E, long long><<<grid, kT, g.smem, s>>>(P, g.strip, g.seg_h, in, out, mp, mu);
            kt_end(kt, s);
        }
        return (int)cudaGetLastError();
    }
};

template <int NC, typename S, typename E> const Ops *ops_of()
{
    static const Ops o = {Impl<NC, S, E>::wmax(),     &Impl<NC, S, E>::density,
                          &Impl<NC, S, E>::step,      &Impl<NC, S, E>::smem,
                          &Impl<NC, S, E>::occupancy, &Impl<NC, S, E>::occupancy_mu};
    return &o;
}

template <typename S, typename E, int LO, int HI> const Ops *ops_range(int nc)
{
    if constexpr (LO > HI) {
        return nullptr;
    } else {
        if (nc == LO) return ops_of<LO, S, E>();
        return ops_range<S, E, LO + 1, HI>(nc);
    }
}

}  // namespace fz
}  // namespace lbmfug

#define LBM_FZ_TU(NAME, S, E, LO, HI)                                                          \
    namespace lbmfug {                                                                         \
    namespace fz {                                                                             \
    const Ops *NAME(int nc) { return ops_range<S, E, LO, HI>(nc); }                            \
    }                                                                                          \
    }
