// lbm_fused2d.cu -- single-pass D2Q9 time step (not built yet: the library
// reports it unsupported and runs the three-pass schedule).
#include "lbm_internal.h"

namespace lbmfug {

bool fused_supported(int, int) { return false; }

FusedGeom fused_geometry(int, int, const Params &, int) { return FusedGeom{}; }

int launch_fused_density(int, int, const Params &, const void *, void *, cudaStream_t)
{
    return (int)cudaErrorNotSupported;
}

int launch_fused_step(int, int, const Params &, const FusedGeom &, const void *, void *,
                      const void *, void *, double *, cudaStream_t)
{
    return (int)cudaErrorNotSupported;
}

int launch_fused_mass_final(int, const FusedGeom &, const double *, double *, int *, cudaStream_t)
{
    return (int)cudaErrorNotSupported;
}

}  // namespace lbmfug
