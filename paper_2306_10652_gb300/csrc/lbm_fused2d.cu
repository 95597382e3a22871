// lbm_fused2d.cu -- dispatch, launch geometry and reductions of the fused
// single-pass D2Q9 schedule; the kernels are instantiated in lbm_fz_*.cu.
#include "lbm_fused2d.cuh"

namespace lbmfug {
namespace fz {
const Ops *f64_lo(int nc);
const Ops *f64_hi(int nc);
const Ops *f32d_lo(int nc);
const Ops *f32d_hi(int nc);
const Ops *f32f_lo(int nc);
const Ops *f32f_hi(int nc);
}  // namespace fz

namespace {

// prec: 0 = binary64 storage and arithmetic; 1 = binary32 deviation storage
// with binary64 thermodynamics and forces; 2 = binary32 throughout.
const fz::Ops *lookup(int prec, int nc)
{
    if (nc < 1 || nc > kMaxNc) return nullptr;
    const bool lo = nc <= 8;
    switch (prec) {
    case 0: return lo ? fz::f64_lo(nc) : fz::f64_hi(nc);
    case 1: return lo ? fz::f32d_lo(nc) : fz::f32d_hi(nc);
    case 2: return lo ? fz::f32f_lo(nc) : fz::f32f_hi(nc);
    default: return nullptr;
    }
}

size_t max_optin_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return 48 * 1024;
    return (size_t)v;
}

// One block per component: threads sum strided partials, then a fixed-order
// warp-shuffle and shared-memory tree (deterministic for a given geometry).
__global__ void __launch_bounds__(256) k_mass_final(int nc, int nblocks, const double *__restrict__ partials,
                                                    double *__restrict__ out, int *__restrict__ nonfinite)
{
    __shared__ double sh[8];
    const int i = blockIdx.x;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[(long long)b * nc + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        out[i] = t;
        if (!isfinite(t)) atomicExch(nonfinite, 1);
    }
}

}  // namespace

bool fused_supported(int lat, int prec, int nc)
{
    if (lat != 0) return false;
    const fz::Ops *o = lookup(prec, nc);
    return o && o->smem(o->wmax) <= max_optin_smem();
}

// Launch geometry: strips of at most wmax columns (extra_strips more than the
// fewest, balanced), segments filling seg_mult waves of the resident CTA
// slots; the mu pass of LBM_FP32DEV likewise with mseg_mult waves.
FusedGeom fused_geometry(int prec, int nc, const Params &P, int num_sms, int extra_strips, int seg_mult,
                         int mseg_mult)
{
    FusedGeom g{};
    const fz::Ops *o = lookup(prec, nc);
    if (!o) return g;
    g.threads = fz::kT;
    g.nstrips = (P.nx + o->wmax - 1) / o->wmax + (extra_strips > 0 ? extra_strips : 0);
    if (g.nstrips > P.nx) g.nstrips = P.nx;
    g.strip = (P.nx + g.nstrips - 1) / g.nstrips;   // balanced strip width <= wmax
    g.nstrips = (P.nx + g.strip - 1) / g.strip;
    g.smem = o->smem(g.strip);
    int per_sm = o->occupancy(g.smem);
    if (per_sm < 1) per_sm = 1;
    const long long slots = (long long)num_sms * per_sm * (seg_mult > 0 ? seg_mult : 1);
    long long segs = slots / g.nstrips;
    if (segs < 1) segs = 1;
    if (segs > P.ny) segs = P.ny;
    g.seg_h = (int)((P.ny + segs - 1) / segs);
    g.segs = (P.ny + g.seg_h - 1) / g.seg_h;
    const int mper_sm = o->occupancy_mu();
    if (mper_sm > 0) {
        // mu pass: strips of at most kT - 4 columns, segments filling the slots
        g.mnstrips = (P.nx + fz::kWmaxMu - 1) / fz::kWmaxMu;
        g.mstrip = (P.nx + g.mnstrips - 1) / g.mnstrips;
        long long ms = (long long)num_sms * mper_sm * (mseg_mult > 0 ? mseg_mult : 1) / g.mnstrips;
        if (ms < 1) ms = 1;
        if (ms > P.ny) ms = P.ny;
        g.mseg_h = (int)((P.ny + ms - 1) / ms);
        g.msegs = (P.ny + g.mseg_h - 1) / g.mseg_h;
    }
    return g;
}

// Caller-chosen strip width and segment height (0 = as fused_geometry).
FusedGeom fused_geometry_forced(int prec, int nc, const Params &P, int num_sms, int strip, int seg_h)
{
    FusedGeom g = fused_geometry(prec, nc, P, num_sms, 0, 1, 1);
    const fz::Ops *o = lookup(prec, nc);
    if (!o || g.nstrips < 1) return g;
    if (strip > 0) {
        g.strip = strip < o->wmax ? strip : o->wmax;
        if (g.strip > P.nx) g.strip = P.nx;
        g.nstrips = (P.nx + g.strip - 1) / g.strip;
        g.smem = o->smem(g.strip);
    }
    if (seg_h > 0) {
        g.seg_h = seg_h < P.ny ? seg_h : P.ny;
        g.segs = (P.ny + g.seg_h - 1) / g.seg_h;
    }
    return g;
}

int launch_fused_density(int prec, int nc, const Params &P, StateBufs st, cudaStream_t s)
{
    const fz::Ops *o = lookup(prec, nc);
    return o ? o->density(P, st, s) : (int)cudaErrorInvalidValue;
}

int launch_fused_step(int prec, int nc, const Params &P, const FusedGeom &geo, StateBufs in,
                      StateBufs out, double *mass_partials, float2 *mu, int *launches, KernelTimer *kt,
                      cudaStream_t s)
{
    const fz::Ops *o = lookup(prec, nc);
    return o ? o->step(P, geo, in, out, mass_partials, mu, launches, kt, s) : (int)cudaErrorInvalidValue;
}

int launch_fused_mass_final(int nc, const FusedGeom &geo, const double *partials, double *out,
                            int *nonfinite, cudaStream_t s)
{
    k_mass_final<<<nc, 256, 0, s>>>(nc, geo.nstrips * geo.segs, partials, out, nonfinite);
    return (int)cudaGetLastError();
}

}  // namespace lbmfug
