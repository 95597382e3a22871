// lbm_threepass.cu -- dispatch of the three-pass schedule over
// (lattice, storage, Nc); the instantiations live in lbm_tp_*.cu so that
// they compile in parallel.
#include "lbm_internal.h"
#include "lbm_threepass.cuh"

namespace lbmfug {
namespace tp {
const Ops *d2q9_f64_lo(int nc);
const Ops *d2q9_f64_hi(int nc);
const Ops *d2q9_f32_lo(int nc);
const Ops *d2q9_f32_hi(int nc);
const Ops *d3q19_f64_lo(int nc);
const Ops *d3q19_f64_hi(int nc);
const Ops *d3q19_f32_lo(int nc);
const Ops *d3q19_f32_hi(int nc);
}  // namespace tp

namespace {
const tp::Ops *lookup(int lat, int prec, int nc)
{
    if (nc < 1 || nc > kMaxNc) return nullptr;
    const bool lo = nc <= 8;
    if (lat == 0 && prec == 0) return lo ? tp::d2q9_f64_lo(nc) : tp::d2q9_f64_hi(nc);
    if (lat == 0 && prec == 1) return lo ? tp::d2q9_f32_lo(nc) : tp::d2q9_f32_hi(nc);
    if (lat == 1 && prec == 0) return lo ? tp::d3q19_f64_lo(nc) : tp::d3q19_f64_hi(nc);
    if (lat == 1 && prec == 1) return lo ? tp::d3q19_f32_lo(nc) : tp::d3q19_f32_hi(nc);
    return nullptr;
}
constexpr int kBad = (int)cudaErrorInvalidValue;
}  // namespace

int launch_init_equilibrium(int lat, int prec, int nc, const Params &P, const double *rho,
                            const double *u, StateBufs st, cudaStream_t s)
{
    const tp::Ops *o = lookup(lat, prec, nc);
    return o ? o->init(P, rho, u, st, s) : kBad;
}

int launch_threepass_step(int lat, int prec, int nc, const Params &P, StateBufs in, StateBufs out,
                          const ThreePassWork &w, cudaStream_t s)
{
    const tp::Ops *o = lookup(lat, prec, nc);
    return o ? o->step(P, in, out, w, s) : kBad;
}

int threepass_launches_per_step(int lat, int prec, int nc)
{
    const tp::Ops *o = lookup(lat, prec, nc);
    return o ? o->launches_per_step() : 0;
}

int launch_fields(int lat, int prec, int nc, const Params &P, StateBufs st,
                  const ThreePassWork &w, double *rho, double *u, double *p, double *lnf,
                  cudaStream_t s)
{
    const tp::Ops *o = lookup(lat, prec, nc);
    return o ? o->fields(P, st, w, rho, u, p, lnf, s) : kBad;
}

int launch_state_to_f64(int lat, int prec, int nc, const Params &P, StateBufs st, double *out,
                        cudaStream_t s)
{
    const tp::Ops *o = lookup(lat, prec, nc);
    return o ? o->to_f64(P, st, out, s) : kBad;
}

int launch_state_from_f64(int lat, int prec, int nc, const Params &P, const double *in,
                          StateBufs st, cudaStream_t s)
{
    const tp::Ops *o = lookup(lat, prec, nc);
    return o ? o->from_f64(P, in, st, s) : kBad;
}

}  // namespace lbmfug
