// lbm_reduce.cu -- deterministic per-component reductions over the lattice.
//
// Mass: M_i = sum_r rho_i(r).  Convergence: max_{i,r} |rho_i(r) - snap_i(r)|.
// Two launches: kReduceBlocks blocks each reduce a fixed contiguous chunk of
// nodes (per-thread strided sums, then a warp-shuffle tree and a shared-memory
// tree in a fixed order) into partials[block][i]; one block then sums the
// partials in block order.  The result is bitwise reproducible for a given
// lattice size.  A non-finite density sets *nonfinite.
#include "lbm_internal.h"

namespace lbmfug {
namespace {

template <bool MAXDIFF>
__global__ void __launch_bounds__(kReduceThreads)
    k_partials(int nc, long long N, const double *__restrict__ rho, const double *__restrict__ snap,
               double *__restrict__ partials, int *__restrict__ nonfinite)
{
    __shared__ double sh[kReduceThreads / 32];
    const long long chunk = (N + gridDim.x - 1) / gridDim.x;
    const long long lo = blockIdx.x * chunk;
    const long long hi = lo + chunk < N ? lo + chunk : N;
    for (int i = 0; i < nc; ++i) {
        double acc = 0.0;
        bool bad = false;
        for (long long r = lo + threadIdx.x; r < hi; r += blockDim.x) {
            const double v = rho[(long long)i * N + r];
            if (!isfinite(v)) bad = true;
            if (MAXDIFF) {
                const double d = fabs(v - snap[(long long)i * N + r]);
                acc = d > acc ? d : acc;
            } else {
                acc += v;
            }
        }
        if (bad) atomicExch(nonfinite, 1);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double t = __shfl_down_sync(0xffffffffu, acc, o);
            acc = MAXDIFF ? (t > acc ? t : acc) : acc + t;
        }
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = sh[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s = MAXDIFF ? (sh[w] > s ? sh[w] : s) : s + sh[w];
            partials[(long long)blockIdx.x * nc + i] = s;
        }
        __syncthreads();
    }
}

template <bool MAXDIFF>
__global__ void k_final(int nc, int nblocks, const double *__restrict__ partials,
                        double *__restrict__ out)
{
    const int i = threadIdx.x;
    if (i >= nc) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) {
        const double v = partials[(long long)b * nc + i];
        s = MAXDIFF ? (v > s ? v : s) : s + v;
    }
    out[i] = s;
}

}  // namespace

int launch_mass(int nc, long long N, const double *rho, double *partials, double *out,
                int *nonfinite, cudaStream_t s)
{
    k_partials<false><<<kReduceBlocks, kReduceThreads, 0, s>>>(nc, N, rho, nullptr, partials,
                                                               nonfinite);
    k_final<false><<<1, 32, 0, s>>>(nc, kReduceBlocks, partials, out);
    return (int)cudaGetLastError();
}

int launch_maxdiff(int nc, long long N, const double *rho, const double *snap, double *partials,
                   double *out, int *nonfinite, cudaStream_t s)
{
    k_partials<true><<<kReduceBlocks, kReduceThreads, 0, s>>>(nc, N, rho, snap, partials,
                                                              nonfinite);
    k_final<true><<<1, 32, 0, s>>>(nc, kReduceBlocks, partials, out);
    return (int)cudaGetLastError();
}

}  // namespace lbmfug
