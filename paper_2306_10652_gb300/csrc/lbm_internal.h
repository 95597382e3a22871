// lbm_internal.h -- host-side interface between the C ABI (lbm_api.cu) and
// the kernel translation units.  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "lbm_core.cuh"

namespace lbmfug {

// Optional CUDA-event timing of the kernels of a step (lbm_timing_enable /
// lbm_timing_read): a launch site records an event before and after its
// launch on the launching stream.  A null timer records nothing.
enum KtSlot : int {
    kKtMuPass = 0,   // k_mu32: double-binary32 chemical potentials and their gradients
    kKtStep,         // k_fused32 / k_fused: the fused step kernel
    kKtMass,         // k_mass_final: monitored mass of a fused step
    kKtMpPsi,        // k_mp_psi
    kKtMpMu,         // k_mp_mu
    kKtMpCollide,    // k_mp_collide
    kKtMpUpdate,     // k_mp_update
    kKtThreePass,    // the three-pass step (k_macro, k_lap, k_collide, k_rupdate)
    kKtMonitor,      // densities and mass of a monitored multi- or three-pass step
    kKtSlots
};
struct KernelTimer {
    struct Rec {
        int slot;
        cudaEvent_t a, b;
        bool a_shared;  // a is the previous record's b (recycled with that record)
    };
    std::vector<cudaEvent_t> pool;  // recycled events
    std::vector<Rec> pending;       // recorded, not yet read
    long long launches[kKtSlots] = {};
    double ms[kKtSlots] = {};
    int open = -1;  // slot between begin and end
    cudaEvent_t open_ev = nullptr;
    bool open_shared = false;
    // The end event of the last timed launch, while nothing else has been
    // enqueued after it: the next begin() takes it as its start event, so
    // back-to-back launches cost one event each.  lbm_step clears it on entry.
    cudaEvent_t last_end = nullptr;
    int err = 0;    // a CUDA error met while recording
    void begin(int slot, cudaStream_t s);
    void end(cudaStream_t s);
    // read every pending pair (their stream has completed) and recycle the events
    int collect();
    void release();
};
inline void kt_begin(KernelTimer *t, int slot, cudaStream_t s)
{
    if (t) t->begin(slot, s);
}
inline void kt_end(KernelTimer *t, cudaStream_t s)
{
    if (t) t->end(s);
}

// Device state of one time level.
//  binary64 storage: g = all Q populations [nc][Q][N] (double); the fused
//    schedule also keeps the densities rhi = [nc][N] (double).
//  binary32 storage: g = the Q-1 moving populations [nc][Q-1][N] (float) and
//    the densities as the pair rhi + rlo ([nc][N] float each).
struct StateBufs {
    void *g = nullptr;
    void *rhi = nullptr;
    float *rlo = nullptr;
    __host__ __device__ float *rhi_f() const { return (float *)rhi; }
    __host__ __device__ double *rhi_d() const { return (double *)rhi; }
};

// Scratch fields of the three-pass schedule (device).
struct ThreePassWork {
    double *rho;  // [nc][N] mass densities rho_i
    double *lnf;  // [nc][N] ln f_i
    double *psi;  // [N]     psi = sum_j sqrt(kappa_j) rho~_j
    double *lap;  // [N]     lap psi
    double *jm;   // [D][N]  sum_i sum_a e_a g_{a,i}
    float *osum;  // [nc][N] binary32 storage: compensated sum of the populations
    float *ocmp;  //         that left each node in the last collision
};

// Fused single-pass D2Q9 schedule: density state and launch geometry.
struct FusedGeom {
    int strip;    // interior columns per CTA
    int nstrips;  // CTAs along x
    int segs;     // CTAs along y
    int seg_h;    // rows per CTA
    int threads;  // threads per CTA
    size_t smem;  // dynamic shared memory bytes
    // the chemical-potential pass of LBM_FP32DEV (0 for the other forms)
    int mstrip, mnstrips, msegs, mseg_h;
};

// All launchers return a cudaError_t cast to int (0 = success).
// Three-pass prec: 0 = binary64 storage, 1 = binary32 deviation storage
// (thermodynamics in binary64).  Fused prec: 0 = binary64, 1 = binary32
// deviation storage with binary64 thermodynamics, 2 = binary32 throughout.
int launch_init_equilibrium(int lat, int prec, int nc, const Params &P, const double *rho,
                            const double *u, StateBufs st, cudaStream_t s);
int launch_threepass_step(int lat, int prec, int nc, const Params &P, StateBufs in, StateBufs out,
                          const ThreePassWork &w, cudaStream_t s);
int threepass_launches_per_step(int lat, int prec, int nc);
// Macroscopic outputs of state st into device buffers (any may be null).
int launch_fields(int lat, int prec, int nc, const Params &P, StateBufs st,
                  const ThreePassWork &w, double *rho, double *u, double *p, double *lnf,
                  cudaStream_t s);
// Populations <-> binary64 post-streaming layout [nc][Q][N].
int launch_state_to_f64(int lat, int prec, int nc, const Params &P, StateBufs st, double *out,
                        cudaStream_t s);
int launch_state_from_f64(int lat, int prec, int nc, const Params &P, const double *in,
                          StateBufs st, cudaStream_t s);

// Fused D2Q9 schedule (lbm_fused2d.cu).  prec as the options: 0 binary64,
// 1 binary32 storage with binary64 thermodynamics, 2 binary32 throughout.
bool fused_supported(int lat, int prec, int nc);
FusedGeom fused_geometry(int prec, int nc, const Params &P, int num_sms, int extra_strips = 0,
                         int seg_mult = 1, int mseg_mult = 1);
FusedGeom fused_geometry_forced(int prec, int nc, const Params &P, int num_sms, int strip, int seg_h);
// binary64 only: densities of the fused state from the populations
int launch_fused_density(int prec, int nc, const Params &P, StateBufs st, cudaStream_t s);
// mu: [nc][N] grad mu_i of LBM_FP32DEV (else unused); *launches receives the
// kernels launched.
int launch_fused_step(int prec, int nc, const Params &P, const FusedGeom &geo, StateBufs in,
                      StateBufs out, double *mass_partials, float2 *mu, int *launches, KernelTimer *kt,
                      cudaStream_t s);
// Sum the per-CTA mass partials of a monitored fused step into out[nc].
int launch_fused_mass_final(int nc, const FusedGeom &geo, const double *partials, double *out,
                            int *nonfinite, cudaStream_t s);

// Binary32 multi-pass schedule of LBM_FP32DEV on any lattice
// (lbm_multipass.cu): psi [N] (hi, lo) of the current state, mu [nc][N]
// (hi, lo) scratch, osum/ocmp [nc][N] departures.
bool multipass_supported(int lat, int prec, int nc, long long N);
int launch_multipass_psi(int lat, int nc, const Params &P, StateBufs st, float2 *psi, cudaStream_t s);
int launch_multipass_step(int lat, int nc, const Params &P, StateBufs in, StateBufs out, float2 *psi,
                          float2 *mu, float *osum, float *ocmp, KernelTimer *kt, cudaStream_t s);

// Chemical potentials and forces of a D2Q9 state from its binary64 densities
// (lbm_fields_*.cu).  prec: 0 binary64, 1 double-binary32, 2 binary32
// thermodynamics.  scratch: (nc + 1) * N * 8 bytes; F [nc][2][N], mu [nc][N]
// (mu may be null).
int launch_forces_lo(int prec, int nc, const Params &P, const double *rho, void *scratch, double *F,
                     double *mu, cudaStream_t s);
int launch_forces_hi(int prec, int nc, const Params &P, const double *rho, void *scratch, double *F,
                     double *mu, cudaStream_t s);

// Deterministic reductions (lbm_reduce.cu).  Partials: [blocks][nc].
constexpr int kReduceBlocks = 1216;  // 8 x 152 SMs
constexpr int kReduceThreads = 256;
int launch_mass(int nc, long long N, const double *rho, double *partials, double *out,
                int *nonfinite, cudaStream_t s);
int launch_maxdiff(int nc, long long N, const double *rho, const double *snap, double *partials,
                   double *out, int *nonfinite, cudaStream_t s);

}  // namespace lbmfug
