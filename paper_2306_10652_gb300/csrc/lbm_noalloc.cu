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
// any stream capture.  The kept address belongs to the device's current CUDA
// context: if that context is torn down and rebuilt (cudaDeviceReset, or the
// primary context released and retained again) the library image is loaded
// anew, possibly elsewhere, so the address is looked up again whenever the
// context's unique id differs from the one it was taken under.  All calls
// share the one scratch area, so calls that overlap on the GPU (different
// streams, no ordering) race on it.
#include <cuda.h>

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
unsigned long long g_ctx_id[kMaxDevices] = {};

// Unique id of the calling thread's current context, through the driver
// entry points the runtime hands out (no link-time dependency on libcuda).
typedef CUresult (*ctx_current_fn)(CUcontext *);
typedef CUresult (*ctx_id_fn)(CUcontext, unsigned long long *);

int current_context_id(unsigned long long *id)
{
    static ctx_current_fn get_current = nullptr;
    static ctx_id_fn get_id = nullptr;
    if (!get_current || !get_id) {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa, qb;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) !=
                cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) !=
                cudaSuccess ||
            qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess)
            return LBM_ECUDA;
        get_current = (ctx_current_fn)a;
        get_id = (ctx_id_fn)b;
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return LBM_ECUDA;
    return get_id(ctx, id) == CUDA_SUCCESS ? LBM_OK : LBM_ECUDA;
}

// Device addresses of the scratch in the current device's context (looked
// up on the first call, and again after the context was rebuilt).
int scratch_for_current_device(double **partials, int **flag)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ECUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    unsigned long long id = 0;
    // no current context yet (first runtime call of this thread): the lookup
    // below makes the device's primary context current
    const bool have_id = current_context_id(&id) == LBM_OK;
    if (!have_id || !g_partials_addr[dev] || g_ctx_id[dev] != id) {
        void *p = nullptr, *f = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess) return LBM_ECUDA;
        if (cudaGetSymbolAddress(&f, g_noalloc_flag) != cudaSuccess) return LBM_ECUDA;
        if (!have_id && current_context_id(&id)) return LBM_ECUDA;
        g_partials_addr[dev] = (double *)p;
        g_flag_addr[dev] = (int *)f;
        g_ctx_id[dev] = id;
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
