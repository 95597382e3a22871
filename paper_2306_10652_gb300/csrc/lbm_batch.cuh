// lbm_batch.cuh -- the batched form: many small independent D2Q9 problems
// (slabs, droplets) advanced by one persistent kernel.
//
// Each CTA takes jobs from a device work counter (largest jobs first) and
// runs one job for a whole round of `steps` time steps before taking the
// next; jobs already converged are skipped.  A job's densities (binary32
// (hi, lo) pairs), psi and mu live in shared memory for the round; its moving
// populations stay in global memory, which a round keeps resident in L2.
// One step of a job (Sec. 2.1, Eqs. 1a-1c, 5; Sec. 2.3, Eqs. 9-12):
//   P1  psi = sum_j sqrt(kappa_j) rho~_j at every node
//   P2  ln f_i and mu_i = RT ln f_i - sqrt(kappa_i) lap psi at every node
//   P3  F_i = -rho~_i grad mu_i, grad rho_i, u, equilibrium, forcing and BGK of
//       the moving populations, pushed to the other buffer; each departure
//       leaves the node's density pair by its own Fast2Sum (the hi part goes
//       to DEP, the lo part stays in RL, which no other node reads in P3)
//   P4  new densities: that pair plus the populations that arrived (read back
//       from the other buffer), by Fast2Sum
// State format is the binary32 one of the single-problem path (Q-1 moving
// populations and an exact density pair), so a job's result does not depend
// on the other jobs, on which CTA runs it, or on the CTA size.
// After each round the change of every density over the round is reduced
// (max, order-free) and compared with the tolerance: that is the paper's run
// "to equilibrium", checked every `steps` steps.
#pragma once

#include "lbm_internal.h"

namespace lbmfug {
namespace bt {

constexpr int kMaxNcBatch = 10;

struct Job {          // device job table, one entry per problem
    int nx, ny;
    long long N;
    long long g[2];   // float offsets of the two population buffers [nc][8][N] in the pool
    long long rh, rl; // float offsets of the density pair [nc][N]
    double RT, lnRT;  // per-job temperature
    double A[kMaxNcBatch * kMaxNcBatch];  // sqrt((a alpha)_i (a alpha)_j)(1 - delta_ij) at the job's T
};

struct Status {
    int converged;    // 0 running, 1 converged, 2 failed (non-finite densities)
    int cur;          // population buffer holding the current state
    long long steps;
    double last_drho; // max over the last round of |rho_i(end) - rho_i(start)|
};

struct Shared {       // batch-wide constants
    int nc;
    double omega;
    double b[kMaxNcBatch], invM[kMaxNcBatch], sqk[kMaxNcBatch];
};

template <int NC, typename E> struct SmemB {
    static __host__ __device__ size_t bytes(long long maxN)
    {
        return (size_t)maxN * (2 * NC * sizeof(float) + sizeof(E) + NC * sizeof(E) + NC * sizeof(float)) + 256;
    }
};

__device__ __forceinline__ int wrapb(int v, int n)
{
    if (v >= 0 && v < n) return v;
    v %= n;
    return v < 0 ? v + n : v;
}

// unit in the last place of a positive normal binary32 number
__device__ __forceinline__ double ulp32(float x)
{
    return ldexp(1.0, ((__float_as_int(x) >> 23) & 0xff) - 127 - 23);
}

__device__ __forceinline__ void pair_acc_b(float &hi, float &lo, float x)
{
    const float s = hi + x;
    lo += x - (s - hi);
    hi = s;
}

// Constants of Eqs. (9)-(12) for one job: the shared b_i and the job's own
// temperature (pr_lnf_v of lbm_core.cuh evaluates the equations).
template <typename E> struct JobView {
    const Shared &S;
    const Job &J;
    __device__ E A(int i, int j) const { return (E)J.A[i * kMaxNcBatch + j]; }
    __device__ E b(int i) const { return (E)S.b[i]; }
    __device__ E RT() const { return (E)J.RT; }
    __device__ E lnRT() const { return (E)J.lnRT; }
};

template <int NC, typename E>
__global__ void k_batch_round(const Shared S, const Job *__restrict__ jobs, Status *__restrict__ status,
                              const int *__restrict__ order, int njobs, int *__restrict__ work,
                              int steps, double tol, float *__restrict__ pool,
                              int *__restrict__ n_converged)
{
    using L = Lattice<0>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_job;
    __shared__ float s_red[32];
    __shared__ float s_rmax[32];
    const int t = threadIdx.x, T = blockDim.x;
    const float om = (float)S.omega, om1 = (float)(1.0 - S.omega), cF = (float)(1.0 - 0.5 * S.omega);
    for (;;) {
        if (t == 0) s_job = atomicAdd(work, 1);
        __syncthreads();
        const int slot = s_job;
        __syncthreads();
        if (slot >= njobs) break;
        const int jid = order[slot];
        if (status[jid].converged) continue;
        const Job &J = jobs[jid];
        const int nx = J.nx, ny = J.ny;
        const int N = (int)J.N;
        float *RH = (float *)smem;              // [NC][N]
        float *RL = RH + NC * N;                // [NC][N]
        E *PSI = (E *)(RL + NC * N);            // [N]
        E *MU = PSI + N;                        // [NC][N]
        float *DEP = (float *)(MU + NC * N);    // [NC][N]
        const float *rhg = pool + J.rh, *rlg = pool + J.rl;
        for (int k = t; k < NC * N; k += T) {
            RH[k] = rhg[k];
            RL[k] = rlg[k];
        }
        int cur = status[jid].cur;
        __syncthreads();
        for (int s = 0; s < steps; ++s) {
            const float *gin = pool + J.g[cur];
            float *gout = pool + J.g[cur ^ 1];
            // P1: psi
            for (int n = t; n < N; n += T) {
                E ps = 0;
#pragma unroll
                for (int i = 0; i < NC; ++i)
                    ps = fma((E)S.sqk[i], ((E)RH[i * N + n] + (E)RL[i * N + n]) * (E)S.invM[i], ps);
                PSI[n] = ps;
            }
            __syncthreads();
            // P2: ln f and mu
            for (int n = t; n < N; n += T) {
                const int x = n % nx, y = n / nx;
                const int xp = wrapb(x + 1, nx), xm = wrapb(x - 1, nx);
                const int yp = wrapb(y + 1, ny), ym = wrapb(y - 1, ny);
                E rm[NC], lf[NC];
#pragma unroll
                for (int i = 0; i < NC; ++i) rm[i] = ((E)RH[i * N + n] + (E)RL[i * N + n]) * (E)S.invM[i];
                pr_lnf_v<NC, E>(JobView<E>{S, J}, rm, lf, nullptr);
                const E c0 = PSI[n];
                const E faces = (PSI[y * nx + xp] - c0) + (PSI[y * nx + xm] - c0) + (PSI[yp * nx + x] - c0) +
                                (PSI[ym * nx + x] - c0);
                const E diags = (PSI[yp * nx + xp] - c0) + (PSI[ym * nx + xm] - c0) + (PSI[ym * nx + xp] - c0) +
                                (PSI[yp * nx + xm] - c0);
                const E lap = (E)6 * fma((E)(1.0 / 9.0), faces, (E)(1.0 / 36.0) * diags);
#pragma unroll
                for (int i = 0; i < NC; ++i) MU[i * N + n] = fma((E)J.RT, lf[i], -(E)S.sqk[i] * lap);
            }
            __syncthreads();
            // P3: forces, velocity, collision of the moving populations, push
            for (int n = t; n < N; n += T) {
                const int x = n % nx, y = n / nx;
                const int xp = wrapb(x + 1, nx), xm = wrapb(x - 1, nx);
                const int yp = wrapb(y + 1, ny), ym = wrapb(y - 1, ny);
                const int nE = y * nx + xp, nW = y * nx + xm, nN = yp * nx + x, nS = ym * nx + x;
                const int nNE = yp * nx + xp, nSW = ym * nx + xm, nSE = ym * nx + xp, nNW = yp * nx + xm;
                float hv[NC][8];
                float jx = 0.0f, jy = 0.0f;
#pragma unroll
                for (int i = 0; i < NC; ++i) {
#pragma unroll
                    for (int a = 0; a < 8; ++a) hv[i][a] = gin[(long long)(i * 8 + a) * N + n];
                    const float *v = hv[i];  // v[a - 1] = g_a, a = 1..8
                    jx += (v[0] - v[1]) + (v[4] - v[5]) + (v[6] - v[7]);
                    jy += (v[2] - v[3]) + (v[4] - v[5]) + (v[7] - v[6]);
                }
                float Fx[NC], Fy[NC], ri[NC];
                E Fsx = 0, Fsy = 0, rt = 0;
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    const E *m = MU + i * N;
                    const E gx = (E)3 * fma((E)(1.0 / 9.0), m[nE] - m[nW], (E)(1.0 / 36.0) * ((m[nNE] - m[nSW]) + (m[nSE] - m[nNW])));
                    const E gy = (E)3 * fma((E)(1.0 / 9.0), m[nN] - m[nS], (E)(1.0 / 36.0) * ((m[nNE] - m[nSW]) - (m[nSE] - m[nNW])));
                    const E r = (E)RH[i * N + n] + (E)RL[i * N + n];
                    ri[i] = (float)r;
                    rt += r;
                    const E rmi = r * (E)S.invM[i];
                    const E fx = -rmi * gx, fy = -rmi * gy;
                    Fsx += fx;
                    Fsy += fy;
                    Fx[i] = (float)fx;
                    Fy[i] = (float)fy;
                }
                const E irt = tdiv((E)1, rt);
                const float ux = (float)(fma((E)0.5, Fsx, (E)jx) * irt);
                const float uy = (float)(fma((E)0.5, Fsy, (E)jy) * irt);
                const float u2 = ux * ux + uy * uy;
                float WB[9], C9[9], U3[9];
#pragma unroll
                for (int a = 1; a < 9; ++a) {
                    const float ue = (float)L::e(a, 0) * ux + (float)L::e(a, 1) * uy;
                    WB[a] = om * (float)L::w(a) * (ue * fmaf(4.5f, ue, 3.0f) - 1.5f * u2);
                    C9[a] = fmaf(9.0f, ue, 3.0f);
                    U3[a] = 3.0f * ue;
                }
                int dst[9];
                dst[1] = nE; dst[2] = nW; dst[3] = nN; dst[4] = nS;
                dst[5] = nNE; dst[6] = nSW; dst[7] = nSE; dst[8] = nNW;
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    const float *r = RH + i * N;
                    const float Gx = 3.0f * fmaf(1.0f / 9.0f, r[nE] - r[nW], (1.0f / 36.0f) * ((r[nNE] - r[nSW]) + (r[nSE] - r[nNW])));
                    const float Gy = 3.0f * fmaf(1.0f / 9.0f, r[nN] - r[nS], (1.0f / 36.0f) * ((r[nNE] - r[nSW]) - (r[nSE] - r[nNW])));
                    const float Fu3 = 3.0f * (Fx[i] * ux + Fy[i] * uy);
                    const float Gu = Gx * ux + Gy * uy;
                    const float Kf = fmaf(-0.5f, Gu, -Fu3), Kd = Gu - Fu3;
                    float dh = RH[i * N + n], dl = RL[i * N + n];
#pragma unroll
                    for (int a = 1; a < 9; ++a) {
                        const int ex = L::e(a, 0), ey = L::e(a, 1);
                        const float cw = cF * (float)L::w(a);
                        const float Fe = (float)ex * Fx[i] + (float)ey * Fy[i];
                        const float Ge = (float)ex * Gx + (float)ey * Gy;
                        const float Fa = fmaf(Fe, C9[a], fmaf(U3[a], Ge, (ex != 0 && ey != 0) ? Kd : Kf));
                        const float gs = fmaf(om1, hv[i][a - 1], fmaf(ri[i], WB[a], cw * Fa));
                        gout[(long long)(i * 8 + a - 1) * N + dst[a]] = gs;
                        pair_acc_b(dh, dl, -gs);
                    }
                    DEP[i * N + n] = dh;
                    RL[i * N + n] = dl;
                }
            }
            __syncthreads();
            // P4: densities move by departures and arrivals
            for (int n = t; n < N; n += T) {
#pragma unroll
                for (int i = 0; i < NC; ++i) {
                    float hi = DEP[i * N + n], lo = RL[i * N + n];
#pragma unroll
                    for (int a = 0; a < 8; ++a) pair_acc_b(hi, lo, gout[(long long)(i * 8 + a) * N + n]);
                    const float h2 = hi + lo;
                    RL[i * N + n] = lo - (h2 - hi);
                    RH[i * N + n] = h2;
                }
            }
            cur ^= 1;
            __syncthreads();
        }
        // round end: change of the densities over the round, then store them
        float dmax = 0.0f, rmax = 0.0f;
        bool finite = true;
        for (int k = t; k < NC * N; k += T) {
            const double now = (double)RH[k] + (double)RL[k];
            const double was = (double)rhg[k] + (double)rlg[k];
            const float d = (float)fabs(now - was);
            finite = finite && isfinite(now);
            dmax = fmaxf(dmax, d);
        }
        for (int n = t; n < N; n += T) {  // largest total density of the job
            float tot = 0.0f;
#pragma unroll
            for (int i = 0; i < NC; ++i) tot += RH[i * N + n];
            rmax = fmaxf(rmax, tot);
        }
        if (!finite) dmax = INFINITY;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dmax = fmaxf(dmax, __shfl_down_sync(0xffffffffu, dmax, o));
            rmax = fmaxf(rmax, __shfl_down_sync(0xffffffffu, rmax, o));
        }
        if ((t & 31) == 0) {
            s_red[t >> 5] = dmax;
            s_rmax[t >> 5] = rmax;
        }
        __syncthreads();
        for (int k = t; k < NC * N; k += T) {
            pool[J.rh + k] = RH[k];
            pool[J.rl + k] = RL[k];
        }
        if (t == 0) {
            float m = 0.0f, r = 0.0f;
            for (int w = 0; w < (T + 31) / 32; ++w) {
                m = fmaxf(m, s_red[w]);
                r = fmaxf(r, s_rmax[w]);
            }
            // the stored populations are binary32: below 8 ulp of the largest
            // total density a change is their rounding jitter, not relaxation
            const double bar = tol > 0.0 ? fmax(tol, 8.0 * ulp32(r)) : 0.0;  // tol = 0: run to the step cap
            Status &st = status[jid];
            st.cur = cur;
            st.steps += steps;
            st.last_drho = m;
            if (!(m <= 3.0e38f)) {           // non-finite densities: the job failed, retire it
                st.converged = 2;
                atomicAdd(n_converged, 1);
            } else if (m < bar) {
                st.converged = 1;
                atomicAdd(n_converged, 1);
            }
        }
        __syncthreads();
    }
}

// Initial state of one job: moving populations at rest (zero) and the exact density pair.
static __global__ void k_batch_init(const double *__restrict__ rho, long long N, int nc, float *__restrict__ g,
                             float *__restrict__ rh, float *__restrict__ rl)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)nc * N;
         k += (long long)gridDim.x * blockDim.x) {
        const double r = rho[k];
        const float h = (float)r;
        rh[k] = h;
        rl[k] = (float)(r - (double)h);
    }
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)nc * 8 * N;
         k += (long long)gridDim.x * blockDim.x)
        g[k] = 0.0f;
}

struct Ops {
    size_t (*smem)(long long maxN);
    int (*launch)(const Shared &, const Job *, Status *, const int *, int, int *, int, double, float *,
                  int *, int ctas, int threads, size_t smem, cudaStream_t);
    int (*occupancy)(int threads, size_t smem);
};

template <int NC, typename E> struct Impl {
    static size_t smem(long long maxN) { return SmemB<NC, E>::bytes(maxN); }
    static int occupancy(int threads, size_t bytes)
    {
        if (cudaFuncSetAttribute(k_batch_round<NC, E>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)bytes) != cudaSuccess)
            return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_round<NC, E>, threads, bytes) !=
            cudaSuccess)
            return 0;
        return n;
    }
    static int launch(const Shared &S, const Job *jobs, Status *status, const int *order, int njobs,
                      int *work, int steps, double tol, float *pool, int *nconv, int ctas, int threads,
                      size_t smem, cudaStream_t s)
    {
        k_batch_round<NC, E><<<ctas, threads, smem, s>>>(S, jobs, status, order, njobs, work, steps, tol,
                                                         pool, nconv);
        return (int)cudaGetLastError();
    }
};

template <int NC, typename E> const Ops *ops_of()
{
    static const Ops o = {&Impl<NC, E>::smem, &Impl<NC, E>::launch, &Impl<NC, E>::occupancy};
    return &o;
}

template <typename E, int LO, int HI> const Ops *ops_range(int nc)
{
    if constexpr (LO > HI) {
        return nullptr;
    } else {
        if (nc == LO) return ops_of<LO, E>();
        return ops_range<E, LO + 1, HI>(nc);
    }
}

}  // namespace bt
}  // namespace lbmfug

#define LBM_BT_TU(NAME, E, LO, HI)                                                            \
    namespace lbmfug {                                                                         \
    namespace bt {                                                                             \
    const Ops *NAME(int nc) { return ops_range<E, LO, HI>(nc); }                               \
    }                                                                                          \
    }
