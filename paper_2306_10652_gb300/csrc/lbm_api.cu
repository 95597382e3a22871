// lbm_api.cu -- the C ABI declared in include/lbmfug.h.
//
// Owns the handle, validates arguments, turns the problem statement of the
// paper (Sec. 2.3: a_i, b_i, omega_i, delta_ij, T; Sec. 2.1: tau; Sec. 2.2:
// kappa_ref) into the per-problem constant block, manages device memory and
// dispatches to the kernels.  No exception or abort crosses the ABI.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <vector>

#include "lbm_df64.cuh"
#include "lbm_internal.h"
#include "lbmfug.h"

using namespace lbmfug;

struct lbm_problem {
    int lattice = 0, nx = 0, ny = 0, nz = 0, nc = 0, D = 0, Q = 0;
    long long N = 0;
    double a[kMaxNc] = {}, b[kMaxNc] = {}, omega[kMaxNc] = {}, kij[kMaxNc * kMaxNc] = {};
    double T = 0, tau = 1;
    double M[kMaxNc] = {};
    lbm_options opt{};
    Params P{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    bool allocated = false;
    bool initialized = false;
    long long steps = 0;
    int sticky = LBM_OK;
    bool fused = false;
    bool tuned = false;        // fused: the launch geometry is final
    int nsm = 152;
    bool multipass = false;
    bool psi_valid = false;    // multi-pass: psi2 holds psi of the current state
    float2 *psi2 = nullptr;    // multi-pass: psi [N] (hi, lo)
    FusedGeom geo{};
    StateBufs st[2];  // two time levels
    int cur = 0;
    ThreePassWork w{};
    double *snap = nullptr;
    bool have_snap = false;
    void *fscratch = nullptr;  // psi / mu scratch of lbm_forces
    float2 *mu = nullptr;      // [nc][N] grad mu_i of the LBM_FP32DEV step (the mu pass writes it)
    // lbm_step_graph: n steps captured once per starting buffer (cur = 0, 1)
    long long graph_n = 0;
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
    long long graph_launches = 0;  // kernels in one replay
    long long launches = 0;
    KernelTimer *timer = nullptr;  // lbm_timing_enable: per-kernel CUDA-event timing (null: off)
    long long monitor_step = -1;
    double *mon = nullptr;  // [nc] latest monitored mass
    double *partials = nullptr;
    double *res = nullptr;
    double *mass_partials = nullptr;
    int *flag = nullptr;
    std::vector<void *> blocks;
    std::vector<size_t> block_bytes;
};

namespace {

struct TuneCand {
    int extra, seg, mseg;  // extra strips, segment waves, mu-pass waves
};
std::vector<TuneCand> tune_candidates(const lbm_problem *p);

int cuda_status(cudaError_t e) { return e == cudaSuccess ? LBM_OK : LBM_ECUDA; }

const char *const kKtNames[kKtSlots] = {
    "k_mu32 (double-binary32 mu pass)", "k_fused32 / k_fused (fused step kernel)",
    "k_mass_final (monitored mass)",    "k_mp_psi",
    "k_mp_mu",                          "k_mp_collide",
    "k_mp_update",                      "three-pass step (k_macro, k_lap, k_collide, k_rupdate)",
    "monitor (densities and mass)"};

// Events recorded but not yet read, above which lbm_step synchronises the
// stream to recycle them.
constexpr size_t kKtMaxPending = 4096;

}  // namespace

namespace lbmfug {

void KernelTimer::begin(int slot, cudaStream_t s)
{
    if (err) return;
    if (last_end) {
        open = slot;
        open_ev = last_end;
        open_shared = true;
        last_end = nullptr;
        return;
    }
    cudaEvent_t e = nullptr;
    if (!pool.empty()) {
        e = pool.back();
        pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        err = 1;
        return;
    }
    if (cudaEventRecord(e, s) != cudaSuccess) {
        pool.push_back(e);
        err = 1;
        return;
    }
    open = slot;
    open_ev = e;
    open_shared = false;
}

void KernelTimer::end(cudaStream_t s)
{
    if (err || open < 0) return;
    cudaEvent_t e = nullptr;
    if (!pool.empty()) {
        e = pool.back();
        pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        err = 1;
        return;
    }
    if (cudaEventRecord(e, s) != cudaSuccess) {
        pool.push_back(e);
        err = 1;
        return;
    }
    pending.push_back({open, open_ev, e, open_shared});
    open = -1;
    open_ev = nullptr;
    last_end = e;
}

int KernelTimer::collect()
{
    for (const Rec &r : pending) {
        float t = 0.0f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) err = 1;
        ms[r.slot] += t;
        launches[r.slot] += 1;
        if (!r.a_shared) pool.push_back(r.a);
        pool.push_back(r.b);
    }
    pending.clear();
    last_end = nullptr;
    return err ? LBM_ECUDA : LBM_OK;
}

void KernelTimer::release()
{
    for (const Rec &r : pending) {
        if (!r.a_shared) cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    pending.clear();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    if (open_ev && !open_shared) cudaEventDestroy(open_ev);
    open_ev = nullptr;
    last_end = nullptr;
}

}  // namespace lbmfug

namespace {

int pstore_bytes(const lbm_problem *p) { return p->opt.precision == LBM_FP64 ? 8 : 4; }

// storage format of the three-pass kernels: 0 = binary64, 1 = binary32 deviation
int sprec(const lbm_problem *p) { return p->opt.precision == LBM_FP64 ? 0 : 1; }

void *dev_alloc(lbm_problem *p, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    void *ptr = nullptr;
    if (p->opt.alloc) {
        ptr = p->opt.alloc(bytes, p->opt.alloc_ctx);
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) {
        p->blocks.push_back(ptr);
        p->block_bytes.push_back(bytes);
    }
    return ptr;
}

void dev_free_all(lbm_problem *p)
{
    for (size_t k = 0; k < p->blocks.size(); ++k) {
        if (p->opt.alloc && p->opt.free)
            p->opt.free(p->blocks[k], p->block_bytes[k], p->opt.alloc_ctx);
        else if (!p->opt.alloc)
            cudaFree(p->blocks[k]);
    }
    p->blocks.clear();
    p->block_bytes.clear();
}

// Sec. 2.3: alpha_i(omega_i, T_r), with T_c,i implied by a_i and b_i.
double pr_alpha(double a, double b, double omega, double T, double R)
{
    const double Tc = (0.077796074 / 0.457235529) * a / (R * b);
    const double Tr = T / Tc;
    double m;
    if (omega <= 0.49)
        m = 0.374640 + 1.54226 * omega - 0.26992 * omega * omega;
    else
        m = 0.379642 + 1.48503 * omega - 0.164423 * omega * omega + 0.016666 * omega * omega * omega;
    const double s = 1.0 + m * (1.0 - std::sqrt(Tr));
    return s * s;
}

float2 split2(double x)
{
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
}

// binary64 constants -> the binary32 and double-binary32 copies
void refresh_float_params(Params &P)
{
    P.fRT = (float)P.RT;
    P.flnRT = (float)P.lnRT;
    for (int i = 0; i < kMaxNc; ++i) {
        P.fb[i] = (float)P.b[i];
        P.finvM[i] = (float)P.invM[i];
        P.fsqk[i] = (float)P.sqk[i];
        P.frhobar[i] = (float)P.rhobar[i];
    }
    for (int k = 0; k < kMaxNc * kMaxNc; ++k) P.fA[k] = (float)P.A[k];
    for (int i = 0; i < kMaxNc; ++i) {
        const double invM = P.invM[i] > 0.0 ? P.invM[i] : 1.0;
        P.dM[i] = split2(invM);
        P.dB[i] = split2(P.b[i] * invM);
        P.db[i] = split2(P.b[i]);
        P.dRK[i] = split2(P.RT * (P.lnRT + std::log(invM)));
        P.dsqk[i] = split2(P.sqk[i]);
        P.dPk[i] = split2(P.sqk[i] * invM);
        for (int j = 0; j < kMaxNc; ++j) {
            const double invMj = P.invM[j] > 0.0 ? P.invM[j] : 1.0;
            P.dA[i * kMaxNc + j] = split2(P.A[i * kMaxNc + j] * invMj);
        }
    }
    for (int r = 0; r < kMaxNc / 2; ++r)
        for (int j = 0; j < kMaxNc; ++j) {
            const float2 a = P.dA[(2 * r) * kMaxNc + j], b = P.dA[(2 * r + 1) * kMaxNc + j];
            P.dAp[r * kMaxNc + j] = make_float4(a.x, b.x, a.y, b.y);
        }
    P.dRT = split2(P.RT);
    for (int j = 0; j < kMaxNc; ++j) P.dPBp[j] = make_float4(P.dPk[j].x, P.dB[j].x, P.dPk[j].y, P.dB[j].y);
    df::make_log_table(&P.logtab[0].x);
}

void build_params(lbm_problem *p)
{
    Params &P = p->P;
    std::memset(&P, 0, sizeof(P));
    P.nx = p->nx;
    P.ny = p->ny;
    P.nz = p->nz;
    P.nc = p->nc;
    P.N = p->N;
    P.RT = p->opt.R * p->T;
    P.lnRT = std::log(P.RT);
    P.omega = 1.0 / p->tau;
    double aa[kMaxNc];
    const double aref = p->a[p->opt.kappa_ref_index];
    for (int i = 0; i < p->nc; ++i) {
        aa[i] = p->a[i] * pr_alpha(p->a[i], p->b[i], p->omega[i], p->T, p->opt.R);
        P.b[i] = p->b[i];
        P.invM[i] = 1.0 / p->M[i];
        P.sqk[i] = std::sqrt(p->opt.kappa_ref * p->a[i] / aref);  // Eq. (6), Eq. (4)
    }
    for (int i = 0; i < p->nc; ++i)
        for (int j = 0; j < p->nc; ++j)
            P.A[i * kMaxNc + j] = std::sqrt(aa[i] * aa[j]) * (1.0 - p->kij[i * kMaxNc + j]);
    refresh_float_params(P);
}

int ensure_allocated(lbm_problem *p)
{
    if (p->allocated) return LBM_OK;
    if (!p->stream) {
        if (p->opt.stream) {
            p->stream = (cudaStream_t)p->opt.stream;
        } else {
            if (cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking) != cudaSuccess)
                return LBM_ECUDA;
            p->own_stream = true;
        }
    }
    build_params(p);
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int sched = p->opt.schedule;
    const bool can_fuse = fused_supported(p->lattice, p->opt.precision, p->nc);
    const bool can_mp = multipass_supported(p->lattice, p->opt.precision, p->nc, p->N);
    if (sched == LBM_SCHED_FUSED && !can_fuse) return LBM_ENOTSUP;
    if (sched == LBM_SCHED_MULTIPASS && !can_mp) return LBM_ENOTSUP;
    p->fused = can_fuse && (sched == LBM_SCHED_FUSED || sched == LBM_SCHED_AUTO);
    p->multipass = can_mp && (sched == LBM_SCHED_MULTIPASS || (sched == LBM_SCHED_AUTO && !p->fused));
    const bool f32 = p->opt.precision != LBM_FP64;
    const size_t nf = (size_t)p->nc * p->N;  // one field per component
    for (int k = 0; k < 2; ++k) {
        if (f32) {
            p->st[k].g = dev_alloc(p, nf * (p->Q - 1) * sizeof(float));
            p->st[k].rhi = dev_alloc(p, nf * sizeof(float));
            p->st[k].rlo = (float *)dev_alloc(p, nf * sizeof(float));
            if (!p->st[k].g || !p->st[k].rhi || !p->st[k].rlo) return LBM_ENOMEM;
        } else {
            p->st[k].g = dev_alloc(p, nf * p->Q * sizeof(double));
            if (!p->st[k].g) return LBM_ENOMEM;
            if (p->fused) {
                p->st[k].rhi = dev_alloc(p, nf * sizeof(double));
                if (!p->st[k].rhi) return LBM_ENOMEM;
            }
        }
    }
    const size_t fb = nf * sizeof(double);
    p->w.rho = (double *)dev_alloc(p, fb);
    p->w.lnf = (double *)dev_alloc(p, fb);
    p->w.psi = (double *)dev_alloc(p, (size_t)p->N * sizeof(double));
    p->w.lap = (double *)dev_alloc(p, (size_t)p->N * sizeof(double));
    p->w.jm = (double *)dev_alloc(p, (size_t)p->D * p->N * sizeof(double));
    if (f32) {
        p->w.osum = (float *)dev_alloc(p, nf * sizeof(float));
        p->w.ocmp = (float *)dev_alloc(p, nf * sizeof(float));
        if (!p->w.osum || !p->w.ocmp) return LBM_ENOMEM;
    }
    p->partials = (double *)dev_alloc(p, (size_t)kReduceBlocks * p->nc * sizeof(double));
    p->res = (double *)dev_alloc(p, 64 * sizeof(double));
    p->flag = (int *)dev_alloc(p, 16);
    p->mon = (double *)dev_alloc(p, kMaxNc * sizeof(double));
    if (!p->mon || !p->w.rho || !p->w.lnf || !p->w.psi || !p->w.lap || !p->w.jm ||
        !p->partials || !p->res || !p->flag)
        return LBM_ENOMEM;
    if (p->fused) {
        p->nsm = nsm;
        size_t parts = 0;
        if (p->opt.strip > 0 || p->opt.seg_h > 0) {
            p->geo = fused_geometry_forced(p->opt.precision, p->nc, p->P, nsm, p->opt.strip, p->opt.seg_h);
            p->tuned = true;  // the caller chose the geometry
            parts = (size_t)p->geo.nstrips * p->geo.segs;
        } else {
            p->geo = fused_geometry(p->opt.precision, p->nc, p->P, nsm);
            p->tuned = !p->opt.tune;
            for (const TuneCand &c : tune_candidates(p)) {  // room for every candidate's partials
                const FusedGeom g = fused_geometry(p->opt.precision, p->nc, p->P, nsm, c.extra, c.seg, c.mseg);
                parts = std::max(parts, (size_t)g.nstrips * g.segs);
            }
        }
        p->mass_partials = (double *)dev_alloc(p, parts * p->nc * sizeof(double));
        if (!p->mass_partials || p->geo.nstrips < 1) return LBM_ENOMEM;
        if (p->opt.precision == LBM_FP32DEV) {
            p->mu = (float2 *)dev_alloc(p, nf * sizeof(float2));  // grad mu_i, written by the mu pass
            if (!p->mu || p->geo.mnstrips < 1) return LBM_ENOMEM;
        }
    }
    if (p->multipass) {
        p->mu = (float2 *)dev_alloc(p, nf * sizeof(float2));
        p->psi2 = (float2 *)dev_alloc(p, (size_t)p->N * sizeof(float2));
        if (!p->mu || !p->psi2) return LBM_ENOMEM;
    }
    if (cudaMemsetAsync(p->flag, 0, 16, p->stream) != cudaSuccess) return LBM_ECUDA;
    p->allocated = true;
    return LBM_OK;
}

// ---- launch-geometry tuner of the fused schedule -------------------------------
std::vector<TuneCand> tune_candidates(const lbm_problem *p)
{
    std::vector<TuneCand> c;
    const bool df = p->opt.precision == LBM_FP32DEV;
    for (int extra = 0; extra <= 1; ++extra)
        for (int seg = 1; seg <= 2; ++seg)
            for (int mseg = 1; mseg <= (df ? 2 : 1); ++mseg) c.push_back({extra, seg, mseg});
    return c;
}

struct TuneKey {
    int prec, nc, nx, ny;
    bool operator<(const TuneKey &o) const
    {
        return std::tie(prec, nc, nx, ny) < std::tie(o.prec, o.nc, o.nx, o.ny);
    }
};
std::mutex g_tune_mutex;
std::map<TuneKey, TuneCand> g_tune_cache;

// Time every candidate geometry on the problem's own state: each trial steps
// st[cur] -> st[cur ^ 1] without swapping, so the state is untouched.
int tune_geometry(lbm_problem *p)
{
    const TuneKey key{p->opt.precision, p->nc, p->nx, p->ny};
    TuneCand best{0, 1, 1};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess) return LBM_ECUDA;
        if (cudaEventCreate(&e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            return LBM_ECUDA;
        }
        float best_ms = 1e30f;
        int st = LBM_OK;
        for (const TuneCand &c : tune_candidates(p)) {
            const FusedGeom g = fused_geometry(p->opt.precision, p->nc, p->P, p->nsm, c.extra, c.seg, c.mseg);
            int nl = 0, e = 0;
            for (int k = 0; k < 4 && !e; ++k) {
                if (k == 1) e = (int)cudaEventRecord(e0, p->stream);
                if (!e)
                    e = launch_fused_step(p->opt.precision, p->nc, p->P, g, p->st[p->cur], p->st[p->cur ^ 1],
                                          nullptr, p->mu, &nl, nullptr, p->stream);
                p->launches += nl;
            }
            if (!e) e = (int)cudaEventRecord(e1, p->stream);
            if (!e) e = (int)cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (!e) e = (int)cudaEventElapsedTime(&ms, e0, e1);
            if (e) {
                st = LBM_ECUDA;
                break;
            }
            if (ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (st) return st;
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = best;
    }
    p->geo = fused_geometry(p->opt.precision, p->nc, p->P, p->nsm, best.extra, best.seg, best.mseg);
    p->tuned = true;
    return LBM_OK;
}

int finish_init(lbm_problem *p)
{
    p->cur = 0;
    p->steps = 0;
    p->have_snap = false;
    p->psi_valid = false;
    p->monitor_step = -1;
    if (cudaMemsetAsync(p->flag, 0, 16, p->stream) != cudaSuccess) return LBM_ECUDA;
    if (p->fused && p->opt.precision == LBM_FP64) {
        int e = launch_fused_density(p->opt.precision, p->nc, p->P, p->st[0], p->stream);
        if (e) return LBM_ECUDA;
        p->launches += 1;
    }
    p->initialized = true;
    p->sticky = LBM_OK;
    return cuda_status(cudaGetLastError());
}

// Host validation of the initial fields, branch-free within blocks of 4096
// values so that the compiler can vectorise it; large fields are split over
// up to eight host threads.
template <typename Pred> bool all_of_blocks(const double *x, size_t n, Pred ok)
{
    auto range = [&](size_t lo, size_t hi) {
        for (size_t b = lo; b < hi; b += 4096) {
            const size_t e = std::min(hi, b + 4096);
            int bad = 0;
            for (size_t k = b; k < e; ++k) bad |= !ok(x[k]);
            if (bad) return false;
        }
        return true;
    };
    const unsigned hw = std::thread::hardware_concurrency();
    const unsigned nt = n < ((size_t)1 << 22) ? 1u : std::max(1u, std::min(8u, hw));
    if (nt == 1) return range(0, n);
    std::vector<std::thread> th;
    std::vector<char> res(nt, 1);
    const size_t chunk = (n + nt - 1) / nt;
    for (unsigned t = 0; t < nt; ++t)
        th.emplace_back([&, t] { res[t] = range(std::min(n, t * chunk), std::min(n, (t + 1) * chunk)); });
    for (auto &x_ : th) x_.join();
    for (char r : res)
        if (!r) return false;
    return true;
}

bool all_positive_finite(const double *x, size_t n)
{
    return all_of_blocks(x, n, [](double v) { return v > 0.0 && v <= 1.7976931348623157e308; });
}

bool all_finite(const double *x, size_t n)
{
    return all_of_blocks(x, n, [](double v) { return v >= -1.7976931348623157e308 && v <= 1.7976931348623157e308; });
}

int check_flag(lbm_problem *p)
{
    int f = 0;
    if (cudaMemcpyAsync(&f, p->flag, sizeof(int), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
        return LBM_ECUDA;
    return f ? LBM_ENONFINITE : LBM_OK;
}

}  // namespace

extern "C" {

int lbm_options_default(lbm_options *opt)
{
    if (!opt) return LBM_EINVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->precision = LBM_FP64;
    opt->schedule = LBM_SCHED_AUTO;
    opt->kappa_ref = 0.02;
    opt->kappa_ref_index = 0;
    opt->M = nullptr;
    opt->R = 1.0;
    opt->tune = 1;
    return LBM_OK;
}

int lbm_create(lbm_problem **out, int lattice, int nx, int ny, int nz, int Nc, const double *a,
               const double *b, const double *omega, const double *kij, double T, double tau)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (lattice != LBM_D2Q9 && lattice != LBM_D3Q19) return LBM_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1 || (lattice == LBM_D2Q9 && nz != 1)) return LBM_EINVAL;
    if (Nc < 1 || Nc > LBM_MAX_NC || !a || !b || !omega) return LBM_EINVAL;
    if (!(T > 0.0) || !std::isfinite(T) || !(tau > 0.5) || !std::isfinite(tau)) return LBM_EINVAL;
    if ((double)nx * ny * nz > 4.0e9) return LBM_EINVAL;
    for (int i = 0; i < Nc; ++i) {
        if (!(a[i] > 0.0) || !(b[i] > 0.0) || !std::isfinite(a[i]) || !std::isfinite(b[i]) ||
            !std::isfinite(omega[i]))
            return LBM_EINVAL;
        if (kij) {
            if (kij[i * Nc + i] != 0.0) return LBM_EINVAL;
            for (int j = 0; j < Nc; ++j) {
                const double k = kij[i * Nc + j];
                if (!std::isfinite(k) || !(std::fabs(k) < 1.0) || k != kij[j * Nc + i]) return LBM_EINVAL;
            }
        }
    }
    lbm_problem *p = new (std::nothrow) lbm_problem();
    if (!p) return LBM_ENOMEM;
    p->lattice = lattice;
    p->nx = nx;
    p->ny = ny;
    p->nz = nz;
    p->nc = Nc;
    p->D = lattice == LBM_D2Q9 ? 2 : 3;
    p->Q = lattice == LBM_D2Q9 ? 9 : 19;
    p->N = (long long)nx * ny * nz;
    for (int i = 0; i < Nc; ++i) {
        p->a[i] = a[i];
        p->b[i] = b[i];
        p->omega[i] = omega[i];
        p->M[i] = 1.0;
        for (int j = 0; j < Nc; ++j) p->kij[i * kMaxNc + j] = kij ? kij[i * Nc + j] : 0.0;
    }
    p->T = T;
    p->tau = tau;
    lbm_options_default(&p->opt);
    *out = p;
    return LBM_OK;
}

int lbm_set_options(lbm_problem *p, const lbm_options *opt)
{
    if (!p || !opt) return LBM_EINVAL;
    if (p->allocated) return LBM_ESTATE;
    if (opt->precision != LBM_FP64 && opt->precision != LBM_FP32DEV && opt->precision != LBM_FP32)
        return LBM_EINVAL;
    if (opt->schedule < LBM_SCHED_AUTO || opt->schedule > LBM_SCHED_MULTIPASS) return LBM_EINVAL;
    if (!(opt->kappa_ref >= 0.0) || !std::isfinite(opt->kappa_ref)) return LBM_EINVAL;
    if (opt->kappa_ref_index < 0 || opt->kappa_ref_index >= p->nc) return LBM_EINVAL;
    if (!(opt->R > 0.0) || !std::isfinite(opt->R)) return LBM_EINVAL;
    if ((opt->alloc == nullptr) != (opt->free == nullptr)) return LBM_EINVAL;
    if (opt->strip < 0 || opt->seg_h < 0 || opt->tune < 0 || opt->tune > 1) return LBM_EINVAL;
    if (opt->M)
        for (int i = 0; i < p->nc; ++i)
            if (!(opt->M[i] > 0.0) || !std::isfinite(opt->M[i])) return LBM_EINVAL;
    p->opt = *opt;
    for (int i = 0; i < p->nc; ++i) p->M[i] = opt->M ? opt->M[i] : 1.0;
    p->opt.M = nullptr;
    return LBM_OK;
}

int lbm_init_fields_device(lbm_problem *p, const double *d_rho, const double *d_u)
{
    if (!p || !d_rho) return LBM_EINVAL;
    int st = ensure_allocated(p);
    if (st) return st;
    p->launches += 1;
    if (launch_init_equilibrium(p->lattice, sprec(p), p->nc, p->P, d_rho, d_u, p->st[0],
                                p->stream))
        return LBM_ECUDA;
    return finish_init(p);
}

int lbm_init_fields(lbm_problem *p, const double *rho, const double *u)
{
    if (!p || !rho) return LBM_EINVAL;
    const size_t nrho = (size_t)p->nc * p->N;
    if (!all_positive_finite(rho, nrho)) return LBM_EINVAL;
    if (u && !all_finite(u, (size_t)p->D * p->N)) return LBM_EINVAL;
    int st = ensure_allocated(p);
    if (st) return st;
    // stage through the three-pass scratch (rho: nc*N doubles; u: lnf buffer holds D*N <= nc*N? no)
    double *d_rho = p->w.rho;
    double *d_u = nullptr;
    if (cudaMemcpyAsync(d_rho, rho, nrho * sizeof(double), cudaMemcpyHostToDevice, p->stream) !=
        cudaSuccess)
        return LBM_ECUDA;
    if (u) {
        d_u = p->w.jm;  // D*N doubles
        if (cudaMemcpyAsync(d_u, u, (size_t)p->D * p->N * sizeof(double), cudaMemcpyHostToDevice,
                            p->stream) != cudaSuccess)
            return LBM_ECUDA;
    }
    return lbm_init_fields_device(p, d_rho, d_u);
}

int lbm_step(lbm_problem *p, long long n)
{
    if (!p || n < 0) return LBM_EINVAL;
    if (!p->initialized) return LBM_ESTATE;
    if (p->sticky) return p->sticky;
    const int every = p->opt.monitor_every;
    if (n > 0 && p->fused && !p->tuned) {
        const int st = tune_geometry(p);
        if (st) {
            p->sticky = st;
            return st;
        }
    }
    if (p->timer) p->timer->last_end = nullptr;  // other work may have been enqueued since
    for (long long s = 0; s < n; ++s) {
        const bool mon = every > 0 && ((p->steps + 1) % every == 0);
        int e = 0;
        KernelTimer *kt = p->timer;
        if (kt && kt->pending.size() >= kKtMaxPending) {
            if (cudaStreamSynchronize(p->stream) != cudaSuccess || kt->collect()) {
                p->sticky = LBM_ECUDA;
                return p->sticky;
            }
        }
        if (p->fused) {
            int nl = 0;
            e = launch_fused_step(p->opt.precision, p->nc, p->P, p->geo, p->st[p->cur],
                                  p->st[p->cur ^ 1], mon ? p->mass_partials : nullptr, p->mu, &nl,
                                  kt, p->stream);
            p->launches += nl;
            if (!e && mon) {
                kt_begin(kt, kKtMass, p->stream);
                e = launch_fused_mass_final(p->nc, p->geo, p->mass_partials, p->mon, p->flag, p->stream);
                kt_end(kt, p->stream);
                p->launches += 1;
            }
        } else if (p->multipass) {
            if (!p->psi_valid) {
                kt_begin(kt, kKtMpPsi, p->stream);
                e = launch_multipass_psi(p->lattice, p->nc, p->P, p->st[p->cur], p->psi2, p->stream);
                kt_end(kt, p->stream);
                p->launches += 1;
                p->psi_valid = true;
            }
            if (!e)
                e = launch_multipass_step(p->lattice, p->nc, p->P, p->st[p->cur], p->st[p->cur ^ 1], p->psi2,
                                          p->mu, p->w.osum, p->w.ocmp, kt, p->stream);
            p->launches += 3;
        } else {
            kt_begin(kt, kKtThreePass, p->stream);
            e = launch_threepass_step(p->lattice, sprec(p), p->nc, p->P, p->st[p->cur],
                                      p->st[p->cur ^ 1], p->w, p->stream);
            kt_end(kt, p->stream);
            p->launches += threepass_launches_per_step(p->lattice, sprec(p), p->nc);
        }
        if (e) {
            p->sticky = LBM_ECUDA;
            return p->sticky;
        }
        p->cur ^= 1;
        p->steps++;
        if (mon && !p->fused) {
            // (the multi-pass schedule's psi of the new state stays valid: moments do not touch it)
            // mass of the new state: densities by the first pass of the next step's kernels
            kt_begin(kt, kKtMonitor, p->stream);
            e = launch_fields(p->lattice, sprec(p), p->nc, p->P, p->st[p->cur], p->w, p->w.rho,
                              nullptr, nullptr, nullptr, p->stream);
            if (!e) e = launch_mass(p->nc, p->N, p->w.rho, p->partials, p->mon, p->flag, p->stream);
            kt_end(kt, p->stream);
            p->launches += 3;
            if (e) {
                p->sticky = LBM_ECUDA;
                return p->sticky;
            }
        }
        if (mon) p->monitor_step = p->steps;
    }
    return LBM_OK;
}

int lbm_step_graph(lbm_problem *p, long long n)
{
    if (!p || n < 1) return LBM_EINVAL;
    if (!p->initialized) return LBM_ESTATE;
    if (p->sticky) return p->sticky;
    if (p->opt.monitor_every > 0) return lbm_step(p, n);  // the monitor's host bookkeeping is per step
    if (p->timer) return lbm_step(p, n);                  // per-launch events are host bookkeeping too
    if (p->fused && !p->tuned) {                          // timing trials cannot run inside a capture
        const int st = tune_geometry(p);
        if (st) return p->sticky = st;
    }
    if (p->multipass && !p->psi_valid) {                   // psi of the initial state, before the capture
        if (launch_multipass_psi(p->lattice, p->nc, p->P, p->st[p->cur], p->psi2, p->stream))
            return p->sticky = LBM_ECUDA;
        p->launches += 1;
        p->psi_valid = true;
    }
    if (p->graph_n != n) {
        for (int k = 0; k < 2; ++k)
            if (p->graph_exec[k]) {
                cudaGraphExecDestroy(p->graph_exec[k]);
                p->graph_exec[k] = nullptr;
            }
        p->graph_n = n;
    }
    const int c = p->cur;
    if (!p->graph_exec[c]) {
        const long long steps0 = p->steps, launches0 = p->launches;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return lbm_step(p, n);  // the stream cannot be captured (for example, already capturing)
        }
        const int st = lbm_step(p, n);
        const cudaError_t ce = cudaStreamEndCapture(p->stream, &g);
        // the capture recorded the steps without running them: undo the bookkeeping
        p->cur = c;
        p->steps = steps0;
        p->graph_launches = p->launches - launches0;
        p->launches = launches0;
        if (st || ce != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            p->sticky = LBM_OK;
            return st ? st : LBM_ECUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&p->graph_exec[c], g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            p->graph_exec[c] = nullptr;
            return LBM_ECUDA;
        }
    }
    if (cudaGraphLaunch(p->graph_exec[c], p->stream) != cudaSuccess) return p->sticky = LBM_ECUDA;
    p->launches += p->graph_launches;
    p->steps += n;
    if (n % 2) p->cur ^= 1;
    return LBM_OK;
}

int lbm_moments_device(lbm_problem *p, double *d_rho, double *d_u, double *d_pressure, double *d_lnf)
{
    if (!p) return LBM_EINVAL;
    if (!p->initialized) return LBM_ESTATE;
    if (p->sticky) return p->sticky;
    if (launch_fields(p->lattice, sprec(p), p->nc, p->P, p->st[p->cur], p->w, d_rho, d_u,
                      d_pressure, d_lnf, p->stream))
        return LBM_ECUDA;
    return LBM_OK;
}

int lbm_moments(lbm_problem *p, double *rho, double *u, double *pressure, double *lnf)
{
    if (!p) return LBM_EINVAL;
    if (!p->initialized) return LBM_ESTATE;
    if (p->sticky) return p->sticky;
    // device staging: rho and lnf land in the scratch fields; u and p need their own
    double *d_u = nullptr, *d_p = nullptr;
    const size_t nb = (size_t)p->N * sizeof(double);
    if (u && cudaMalloc(&d_u, (size_t)p->D * nb) != cudaSuccess) return LBM_ENOMEM;
    if (pressure && cudaMalloc(&d_p, nb) != cudaSuccess) {
        cudaFree(d_u);
        return LBM_ENOMEM;
    }
    int st = lbm_moments_device(p, p->w.rho, d_u, d_p, lnf ? p->w.lnf : nullptr);
    const size_t fb = (size_t)p->nc * nb;
    if (!st && rho && cudaMemcpyAsync(rho, p->w.rho, fb, cudaMemcpyDeviceToHost, p->stream)) st = LBM_ECUDA;
    if (!st && lnf && cudaMemcpyAsync(lnf, p->w.lnf, fb, cudaMemcpyDeviceToHost, p->stream)) st = LBM_ECUDA;
    if (!st && u && cudaMemcpyAsync(u, d_u, (size_t)p->D * nb, cudaMemcpyDeviceToHost, p->stream)) st = LBM_ECUDA;
    if (!st && pressure && cudaMemcpyAsync(pressure, d_p, nb, cudaMemcpyDeviceToHost, p->stream)) st = LBM_ECUDA;
    if (!st && cudaStreamSynchronize(p->stream) != cudaSuccess) st = LBM_ECUDA;
    cudaFree(d_u);
    cudaFree(d_p);
    return st;
}

int lbm_forces(lbm_problem *p, double *F, double *mu)
{
    if (!p || (!F && !mu)) return LBM_EINVAL;
    if (!p->initialized) return LBM_ESTATE;
    if (p->sticky) return p->sticky;
    if (p->lattice != LBM_D2Q9) return LBM_ENOTSUP;
    // the arithmetic of the step: the fused schedule's thermodynamics form, or
    // binary64 for the three-pass schedule and for binary64 storage
    const int prec = (!p->fused || p->opt.precision == LBM_FP64) ? 0 : (p->opt.precision == LBM_FP32DEV ? 1 : 2);
    const size_t N = (size_t)p->N, nc = (size_t)p->nc;
    if (!p->fscratch) {
        p->fscratch = dev_alloc(p, (nc + 1) * N * sizeof(double));
        if (!p->fscratch) return LBM_ENOMEM;
    }
    double *dF = nullptr, *dmu = nullptr;
    if (cudaMalloc(&dF, nc * 2 * N * sizeof(double)) != cudaSuccess) return LBM_ENOMEM;
    if (mu && cudaMalloc(&dmu, nc * N * sizeof(double)) != cudaSuccess) {
        cudaFree(dF);
        return LBM_ENOMEM;
    }
    int st = LBM_OK;
    if (launch_fields(p->lattice, sprec(p), p->nc, p->P, p->st[p->cur], p->w, p->w.rho, nullptr, nullptr,
                      nullptr, p->stream))
        st = LBM_ECUDA;
    p->launches += 1;
    if (!st) {
        const int e = p->nc <= 8 ? launch_forces_lo(prec, p->nc, p->P, p->w.rho, p->fscratch, dF, dmu, p->stream)
                                 : launch_forces_hi(prec, p->nc, p->P, p->w.rho, p->fscratch, dF, dmu, p->stream);
        p->launches += 3;
        if (e) st = LBM_ECUDA;
    }
    if (!st && F && cudaMemcpyAsync(F, dF, nc * 2 * N * sizeof(double), cudaMemcpyDeviceToHost, p->stream))
        st = LBM_ECUDA;
    if (!st && mu && cudaMemcpyAsync(mu, dmu, nc * N * sizeof(double), cudaMemcpyDeviceToHost, p->stream))
        st = LBM_ECUDA;
    if (!st && cudaStreamSynchronize(p->stream) != cudaSuccess) st = LBM_ECUDA;
    cudaFree(dF);
    cudaFree(dmu);
    return st;
}

int lbm_schedule_info(const lbm_problem *p, int *fused, int *strip, int *nstrips, int *seg_h, int *segs)
{
    if (!p) return LBM_EINVAL;
    if (!p->allocated) return LBM_ESTATE;
    if (fused) *fused = p->fused ? 1 : 0;
    if (strip) *strip = p->fused ? p->geo.strip : 0;
    if (nstrips) *nstrips = p->fused ? p->geo.nstrips : 0;
    if (seg_h) *seg_h = p->fused ? p->geo.seg_h : 0;
    if (segs) *segs = p->fused ? p->geo.segs : 0;
    return LBM_OK;
}

int lbm_mass(lbm_problem *p, double *mass)
{
    if (!p || !mass) return LBM_EINVAL;
    if (!p->initialized) return LBM_ESTATE;
    if (p->sticky) return p->sticky;
    if (launch_fields(p->lattice, sprec(p), p->nc, p->P, p->st[p->cur], p->w, p->w.rho,
                      nullptr, nullptr, nullptr, p->stream))
        return LBM_ECUDA;
    if (cudaMemsetAsync(p->flag, 0, sizeof(int), p->stream) != cudaSuccess) return LBM_ECUDA;
    if (launch_mass(p->nc, p->N, p->w.rho, p->partials, p->res, p->flag, p->stream)) return LBM_ECUDA;
    if (cudaMemcpyAsync(mass, p->res, p->nc * sizeof(double), cudaMemcpyDeviceToHost, p->stream) !=
        cudaSuccess)
        return LBM_ECUDA;
    return check_flag(p);
}

int lbm_convergence(lbm_problem *p, double *max_abs_drho)
{
    if (!p || !max_abs_drho) return LBM_EINVAL;
    if (!p->initialized) return LBM_ESTATE;
    if (p->sticky) return p->sticky;
    const size_t fb = (size_t)p->nc * p->N * sizeof(double);
    if (!p->snap) {
        p->snap = (double *)dev_alloc(p, fb);
        if (!p->snap) return LBM_ENOMEM;
    }
    if (launch_fields(p->lattice, sprec(p), p->nc, p->P, p->st[p->cur], p->w, p->w.rho,
                      nullptr, nullptr, nullptr, p->stream))
        return LBM_ECUDA;
    if (cudaMemsetAsync(p->flag, 0, sizeof(int), p->stream) != cudaSuccess) return LBM_ECUDA;
    double vals[kMaxNc];
    if (p->have_snap) {
        if (launch_maxdiff(p->nc, p->N, p->w.rho, p->snap, p->partials, p->res, p->flag, p->stream))
            return LBM_ECUDA;
        if (cudaMemcpyAsync(vals, p->res, p->nc * sizeof(double), cudaMemcpyDeviceToHost,
                            p->stream) != cudaSuccess)
            return LBM_ECUDA;
    }
    if (cudaMemcpyAsync(p->snap, p->w.rho, fb, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess)
        return LBM_ECUDA;
    int st = check_flag(p);
    if (st) return st;
    double m = INFINITY;
    if (p->have_snap) {
        m = 0.0;
        for (int i = 0; i < p->nc; ++i) m = vals[i] > m ? vals[i] : m;
    }
    p->have_snap = true;
    *max_abs_drho = m;
    return LBM_OK;
}

int lbm_get_state(lbm_problem *p, double *buf, size_t *bytes)
{
    if (!p || !bytes) return LBM_EINVAL;
    const size_t need = (size_t)p->nc * p->Q * p->N * sizeof(double);
    if (!buf) {
        *bytes = need;
        return LBM_OK;
    }
    if (*bytes < need) {
        *bytes = need;
        return LBM_EINVAL;
    }
    if (!p->initialized) return LBM_ESTATE;
    if (p->sticky) return p->sticky;
    double *d = nullptr;
    if (cudaMalloc(&d, need) != cudaSuccess) return LBM_ENOMEM;
    int st = LBM_OK;
    if (launch_state_to_f64(p->lattice, sprec(p), p->nc, p->P, p->st[p->cur], d, p->stream))
        st = LBM_ECUDA;
    if (!st && cudaMemcpyAsync(buf, d, need, cudaMemcpyDeviceToHost, p->stream) != cudaSuccess) st = LBM_ECUDA;
    if (!st && cudaStreamSynchronize(p->stream) != cudaSuccess) st = LBM_ECUDA;
    cudaFree(d);
    *bytes = need;
    return st;
}

int lbm_set_state(lbm_problem *p, const double *buf, size_t bytes)
{
    if (!p || !buf) return LBM_EINVAL;
    const size_t need = (size_t)p->nc * p->Q * p->N * sizeof(double);
    if (bytes != need) return LBM_EINVAL;
    for (size_t k = 0; k < need / sizeof(double); ++k)
        if (!std::isfinite(buf[k])) return LBM_EINVAL;
    int st = ensure_allocated(p);
    if (st) return st;
    double *d = nullptr;
    if (cudaMalloc(&d, need) != cudaSuccess) return LBM_ENOMEM;
    if (cudaMemcpyAsync(d, buf, need, cudaMemcpyHostToDevice, p->stream) != cudaSuccess) st = LBM_ECUDA;
    if (!st && launch_state_from_f64(p->lattice, sprec(p), p->nc, p->P, d, p->st[0], p->stream))
        st = LBM_ECUDA;
    if (!st && cudaStreamSynchronize(p->stream) != cudaSuccess) st = LBM_ECUDA;
    cudaFree(d);
    if (st) return st;
    return finish_init(p);
}

int lbm_monitor(lbm_problem *p, double *mass, long long *at_step, int *nonfinite)
{
    if (!p) return LBM_EINVAL;
    if (!p->initialized) return LBM_ESTATE;
    int f = 0;
    if (mass && p->monitor_step >= 0 &&
        cudaMemcpyAsync(mass, p->mon, p->nc * sizeof(double), cudaMemcpyDeviceToHost, p->stream) !=
            cudaSuccess)
        return LBM_ECUDA;
    if (cudaMemcpyAsync(&f, p->flag, sizeof(int), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess)
        return LBM_ECUDA;
    if (at_step) *at_step = p->monitor_step;
    if (nonfinite) *nonfinite = f;
    return LBM_OK;
}

int lbm_timing_enable(lbm_problem *p, int on)
{
    if (!p || on < 0 || on > 1) return LBM_EINVAL;
    if (p->timer) {
        if (p->stream && cudaStreamSynchronize(p->stream) != cudaSuccess) return LBM_ECUDA;
        p->timer->release();
        delete p->timer;
        p->timer = nullptr;
    }
    if (on) {
        p->timer = new (std::nothrow) KernelTimer();
        if (!p->timer) return LBM_ENOMEM;
    }
    return LBM_OK;
}

int lbm_timing_read(lbm_problem *p, lbm_kernel_time *out, int max, int *n)
{
    if (!p || !n || max < 0 || (max > 0 && !out)) return LBM_EINVAL;
    *n = 0;
    if (!p->timer) return LBM_ESTATE;
    if (p->stream && cudaStreamSynchronize(p->stream) != cudaSuccess) return LBM_ECUDA;
    const int st = p->timer->collect();
    int k = 0;
    for (int s = 0; s < kKtSlots; ++s) {
        if (p->timer->launches[s] == 0) continue;
        if (k < max) {
            out[k].name = kKtNames[s];
            out[k].launches = p->timer->launches[s];
            out[k].total_ms = p->timer->ms[s];
        }
        ++k;
    }
    *n = k;
    return st;
}

int lbm_launch_count(const lbm_problem *p, long long *launches)
{
    if (!p || !launches) return LBM_EINVAL;
    *launches = p->launches;
    return LBM_OK;
}

int lbm_step_count(const lbm_problem *p, long long *steps)
{
    if (!p || !steps) return LBM_EINVAL;
    *steps = p->steps;
    return LBM_OK;
}

int lbm_synchronize(lbm_problem *p)
{
    if (!p) return LBM_EINVAL;
    if (!p->stream) return LBM_OK;
    if (cudaStreamSynchronize(p->stream) != cudaSuccess) {
        p->sticky = LBM_ECUDA;
        return LBM_ECUDA;
    }
    return p->sticky;
}

int lbm_destroy(lbm_problem *p)
{
    if (!p) return LBM_OK;
    if (p->stream) cudaStreamSynchronize(p->stream);
    for (int k = 0; k < 2; ++k)
        if (p->graph_exec[k]) cudaGraphExecDestroy(p->graph_exec[k]);
    if (p->timer) {
        p->timer->release();
        delete p->timer;
    }
    dev_free_all(p);
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
    delete p;
    return LBM_OK;
}

int lbm_lattice_velocities(int lattice, int *D, int *Q, int *e)
{
    if (!D || !Q) return LBM_EINVAL;
    if (lattice == LBM_D2Q9) {
        *D = 2;
        *Q = 9;
        if (e)
            for (int a = 0; a < 9; ++a)
                for (int d = 0; d < 3; ++d) e[a * 3 + d] = Lattice<0>::e(a, d);
    } else if (lattice == LBM_D3Q19) {
        *D = 3;
        *Q = 19;
        if (e)
            for (int a = 0; a < 19; ++a)
                for (int d = 0; d < 3; ++d) e[a * 3 + d] = Lattice<1>::e(a, d);
    } else {
        return LBM_EINVAL;
    }
    return LBM_OK;
}

const char *lbm_strerror(int status)
{
    switch (status) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_ECUDA: return "CUDA error";
    case LBM_ENONFINITE: return "non-finite density";
    case LBM_ETIMEOUT: return "device wait timed out";
    case LBM_ESTATE: return "invalid state for this call";
    case LBM_ENOTSUP: return "not supported";
    default: return "unknown status";
    }
}

}  // extern "C"
