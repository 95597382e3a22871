// lbm_multipass.cu -- dispatch of the binary32 multi-pass step (LBM_FP32DEV
// on any lattice); the kernels are instantiated in lbm_mp_*.cu.
#include "lbm_multipass.cuh"

namespace lbmfug {
namespace mp {
const Ops *d2q9_lo(int nc);
const Ops *d2q9_hi(int nc);
const Ops *d3q19_lo(int nc);
const Ops *d3q19_hi(int nc);
}  // namespace mp

namespace {
const mp::Ops *lookup(int lat, int nc)
{
    if (nc < 1 || nc > kMaxNc) return nullptr;
    const bool lo = nc <= 8;
    if (lat == 0) return lo ? mp::d2q9_lo(nc) : mp::d2q9_hi(nc);
    if (lat == 1) return lo ? mp::d3q19_lo(nc) : mp::d3q19_hi(nc);
    return nullptr;
}
}  // namespace

// The multi-pass kernels index nodes in 32 bits.
bool multipass_supported(int lat, int prec, int nc, long long N)
{
    return prec == 1 && N < (1LL << 31) && lookup(lat, nc) != nullptr;
}

int launch_multipass_psi(int lat, int nc, const Params &P, StateBufs st, float2 *psi, cudaStream_t s)
{
    const mp::Ops *o = lookup(lat, nc);
    return o ? o->psi(P, st, psi, s) : (int)cudaErrorInvalidValue;
}

int launch_multipass_step(int lat, int nc, const Params &P, StateBufs in, StateBufs out, float2 *psi,
                          float2 *mu, float *osum, float *ocmp, KernelTimer *kt, cudaStream_t s)
{
    const mp::Ops *o = lookup(lat, nc);
    return o ? o->step(P, in, out, psi, mu, osum, ocmp, kt, s) : (int)cudaErrorInvalidValue;
}

}  // namespace lbmfug
