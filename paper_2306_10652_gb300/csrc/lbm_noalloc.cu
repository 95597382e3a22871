// lbm_noalloc.cu -- per-component field sums that allocate no device memory.
//
// Some callers cannot allocate device memory when they need a reduction:
// code running under another framework's memory pool that owns all device
// memory, a solver step driven from a host callback or a real-time loop
// where the implicit device synchronisation of cudaMalloc/cudaFree is not
// acceptable, or a serving loop whose memory was budgeted up front.  For
// them this entry point runs the library's deterministic two-level
// reduction with its per-block partial sums in a fixed scratch area that is
// part of the library image itself.
//
// The scratch is a file-scope __device__ array: every GPU that loads the
// library holds it (kNoAllocScratchBytes) until the process exits.  Host code
// cannot use the array's name as a device address, so the first call on
// each device looks the address up with cudaGetSymbolAddress (with that
// device current) and keeps it; that first call should therefore come before
// any stream capture.  All calls share the one scratch area, so calls that
// overlap on the GPU (different streams, no ordering) race on it.
#include <mutex>

#include "lbm_internal.h"
#include "lbmfug.h"

namespace {

// kReduceBlocks partial sums for each of at most LBM_MAX_NC components,
// plus a non-finite flag for callers that pass none: 1216 * 16 * 8 + 256 bytes.
constexpr int kNoAllocMaxNc = LBM_MAX_NC;
static __device__ __align__(256) double g_noalloc_partials[lbmfug::kReduceBlocks * kNoAllocMaxNc];
static __device__ __align__(256) int g_noalloc_flag[64];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double *g_partials_addr[kMaxDevices] = {};
int *g_flag_addr[kMaxDevices] = {};

// Device addresses of the scratch on the current device (looked up once).
int scratch_for_current_device(double **partials, int **flag)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
        void *p = nullptr, *f = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess) return LBM_ECUDA;
        if (cudaGetSymbolAddress(&f, g_noalloc_flag) != cudaSuccess) return LBM_ECUDA;
        g_partials_addr[dev] = (double *)p;
        g_flag_addr[dev] = (int *)f;
    }
    *partials = g_partials_addr[dev];
    *flag = g_flag_addr[dev];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_field_sums_noalloc(const double *d_field, int nc, long long n, double *d_out,
                                      int *d_nonfinite, void *stream)
{
    if (!d_field || !d_out || n < 1) return LBM_EINVAL;
    if (nc < 1 || nc > kNoAllocMaxNc) return LBM_EINVAL;  // beyond the fixed scratch capacity
    double *partials = nullptr;
    int *flag = nullptr;
    int st = scratch_for_current_device(&partials, &flag);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int *nf = d_nonfinite ? d_nonfinite : flag;
    // the flag is an output that starts at zero; every partial is overwritten
    if (cudaMemsetAsync(nf, 0, sizeof(int), s) != cudaSuccess) return LBM_ECUDA;
    if (lbmfug::launch_mass(nc, n, d_field, partials, d_out, nf, s)) return LBM_ECUDA;
    return LBM_OK;
}
