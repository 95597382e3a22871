// lbm_batch.cu -- C ABI of the batched form (lbm_batch_*), its job table,
// the autotuner of the batched kernel and the captured CUDA graph of a round.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "lbm_batch.cuh"
#include "lbmfug.h"

using namespace lbmfug;

namespace lbmfug {
namespace bt {
const Ops *f32_lo(int nc);
const Ops *f32_hi(int nc);
const Ops *f64_lo(int nc);
const Ops *f64_hi(int nc);
}  // namespace bt
}  // namespace lbmfug

struct lbm_batch {
    int nc = 0, njobs = 0, precision = LBM_FP32;
    bt::Shared S{};
    std::vector<bt::Job> jobs;
    std::vector<int> order;  // largest jobs first
    bt::Job *d_jobs = nullptr;
    bt::Status *d_status = nullptr;
    int *d_order = nullptr, *d_work = nullptr, *d_nconv = nullptr;
    int *h_nconv = nullptr;  // pinned
    float *pool = nullptr;
    size_t pool_floats = 0;
    long long maxN = 0;
    const bt::Ops *ops = nullptr;
    int threads = 0, ctas = 0;
    size_t smem = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_steps = -1;
    double graph_tol = -1.0;
    long long launches = 0;
    long long rounds = 0;
};

namespace {

const bt::Ops *lookup(int prec, int nc)
{
    if (nc < 1 || nc > bt::kMaxNcBatch) return nullptr;
    const bool lo = nc <= 5;
    if (prec == LBM_FP32) return lo ? bt::f32_lo(nc) : bt::f32_hi(nc);
    if (prec == LBM_FP32DEV) return lo ? bt::f64_lo(nc) : bt::f64_hi(nc);
    return nullptr;
}

double alpha_of(double a, double b, double omega, double T, double R)
{
    const double Tc = (0.077796074 / 0.457235529) * a / (R * b);  // Sec. 2.3
    double m;
    if (omega <= 0.49)
        m = 0.374640 + 1.54226 * omega - 0.26992 * omega * omega;
    else
        m = 0.379642 + 1.48503 * omega - 0.164423 * omega * omega + 0.016666 * omega * omega * omega;
    const double s = 1.0 + m * (1.0 - std::sqrt(T / Tc));
    return s * s;
}

// autotuner cache: (precision, nc, max nodes) -> threads per CTA
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, long long>, int> g_tune_cache;

void release(lbm_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    cudaFree(b->d_jobs);
    cudaFree(b->d_status);
    cudaFree(b->d_order);
    cudaFree(b->d_work);
    cudaFree(b->d_nconv);
    cudaFree(b->pool);
    if (b->h_nconv) cudaFreeHost(b->h_nconv);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

int launch_round(lbm_batch *b, int steps, double tol)
{
    if (cudaMemsetAsync(b->d_work, 0, sizeof(int), b->stream) != cudaSuccess) return LBM_ECUDA;
    if (b->ops->launch(b->S, b->d_jobs, b->d_status, b->d_order, b->njobs, b->d_work, steps, tol, b->pool,
                       b->d_nconv, b->ctas, b->threads, b->smem, b->stream))
        return LBM_ECUDA;
    if (cudaMemcpyAsync(b->h_nconv, b->d_nconv, sizeof(int), cudaMemcpyDeviceToHost, b->stream) !=
        cudaSuccess)
        return LBM_ECUDA;
    return LBM_OK;
}

int configure(lbm_batch *b, int threads)
{
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = b->ops->smem(b->maxN);
    const int per_sm = b->ops->occupancy(threads, smem);
    if (per_sm < 1) return LBM_ENOTSUP;
    b->threads = threads;
    b->smem = smem;
    b->ctas = std::min((long long)nsm * per_sm, (long long)b->njobs);
    return LBM_OK;
}

// Time one short round per candidate on a copy of the state, keep the fastest.
int autotune(lbm_batch *b)
{
    const auto key = std::make_tuple(b->precision, b->nc, b->maxN);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return configure(b, it->second);
    }
    float *backup = nullptr;
    bt::Status *sbackup = nullptr;
    if (cudaMalloc(&backup, b->pool_floats * sizeof(float)) != cudaSuccess) return LBM_ENOMEM;
    if (cudaMalloc(&sbackup, b->njobs * sizeof(bt::Status)) != cudaSuccess) {
        cudaFree(backup);
        return LBM_ENOMEM;
    }
    cudaMemcpyAsync(backup, b->pool, b->pool_floats * sizeof(float), cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(sbackup, b->d_status, b->njobs * sizeof(bt::Status), cudaMemcpyDeviceToDevice, b->stream);
    const int candidates[] = {128, 256, 512};
    int best = 0;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int th : candidates) {
        if (configure(b, th) != LBM_OK) continue;
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {  // the first repetition warms up
            cudaEventRecord(e0, b->stream);
            if (launch_round(b, 20, -1.0) != LBM_OK) break;
            b->launches += 1;
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
        }
        if (ms > 0.0f && ms < best_ms) {
            best_ms = ms;
            best = th;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemcpyAsync(b->pool, backup, b->pool_floats * sizeof(float), cudaMemcpyDeviceToDevice, b->stream);
    cudaMemcpyAsync(b->d_status, sbackup, b->njobs * sizeof(bt::Status), cudaMemcpyDeviceToDevice, b->stream);
    cudaMemsetAsync(b->d_nconv, 0, sizeof(int), b->stream);
    cudaStreamSynchronize(b->stream);
    cudaFree(backup);
    cudaFree(sbackup);
    if (!best) return LBM_ENOTSUP;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = best;
    }
    return configure(b, best);
}

int capture(lbm_batch *b, int steps, double tol)
{
    if (b->exec && b->graph_steps == steps && b->graph_tol == tol) return LBM_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LBM_ECUDA;
    const int st = launch_round(b, steps, tol);
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(b->stream, &g) != cudaSuccess || st != LBM_OK) {
        if (g) cudaGraphDestroy(g);
        return LBM_ECUDA;
    }
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        return LBM_ECUDA;
    }
    b->graph = g;
    b->graph_steps = steps;
    b->graph_tol = tol;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_batch **out, int Nc, const double *a, const double *b, const double *omega,
                     const double *kij, double tau, const lbm_options *opt, const lbm_job *jobs, int njobs)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (Nc < 1 || Nc > bt::kMaxNcBatch || !a || !b || !omega || !jobs || njobs < 1) return LBM_EINVAL;
    if (!(tau > 0.5) || !std::isfinite(tau)) return LBM_EINVAL;
    lbm_options o;
    lbm_options_default(&o);
    if (opt) o = *opt;
    if (o.precision == LBM_FP64) o.precision = LBM_FP32DEV;  // the batched form stores binary32
    if (o.precision != LBM_FP32 && o.precision != LBM_FP32DEV) return LBM_EINVAL;
    if (!(o.R > 0.0) || o.kappa_ref_index < 0 || o.kappa_ref_index >= Nc || !(o.kappa_ref >= 0.0))
        return LBM_EINVAL;
    for (int i = 0; i < Nc; ++i) {
        if (!(a[i] > 0.0) || !(b[i] > 0.0) || !std::isfinite(omega[i])) return LBM_EINVAL;
        if (o.M && !(o.M[i] > 0.0)) return LBM_EINVAL;
        if (kij)
            for (int j = 0; j < Nc; ++j)
                if (!(std::fabs(kij[i * Nc + j]) < 1.0) || kij[i * Nc + j] != kij[j * Nc + i] ||
                    (i == j && kij[i * Nc + j] != 0.0))
                    return LBM_EINVAL;
    }
    long long total = 0;
    for (int k = 0; k < njobs; ++k) {
        const lbm_job &J = jobs[k];
        if (J.nx < 1 || J.ny < 1 || !(J.T > 0.0) || !J.rho) return LBM_EINVAL;
        if ((long long)J.nx * J.ny > (1LL << 20)) return LBM_EINVAL;
        for (long long r = 0; r < (long long)Nc * J.nx * J.ny; ++r)
            if (!(J.rho[r] > 0.0) || !std::isfinite(J.rho[r])) return LBM_EINVAL;
        total += (long long)J.nx * J.ny;
    }
    const bt::Ops *ops = lookup(o.precision, Nc);
    if (!ops) return LBM_ENOTSUP;

    lbm_batch *bt_ = new (std::nothrow) lbm_batch();
    if (!bt_) return LBM_ENOMEM;
    bt_->nc = Nc;
    bt_->njobs = njobs;
    bt_->precision = o.precision;
    bt_->ops = ops;
    bt_->S.nc = Nc;
    bt_->S.omega = 1.0 / tau;
    const double aref = a[o.kappa_ref_index];
    for (int i = 0; i < Nc; ++i) {
        bt_->S.b[i] = b[i];
        bt_->S.invM[i] = 1.0 / (o.M ? o.M[i] : 1.0);
        bt_->S.sqk[i] = std::sqrt(o.kappa_ref * a[i] / aref);  // Eqs. (4), (6)
    }
    // job table and pool: per job 2 x [nc][8][N] populations + [nc][N] hi + [nc][N] lo
    bt_->jobs.resize(njobs);
    size_t off = 0;
    for (int k = 0; k < njobs; ++k) {
        bt::Job &J = bt_->jobs[k];
        std::memset(&J, 0, sizeof(J));
        J.nx = jobs[k].nx;
        J.ny = jobs[k].ny;
        J.N = (long long)J.nx * J.ny;
        J.g[0] = off;
        off += (size_t)Nc * 8 * J.N;
        J.g[1] = off;
        off += (size_t)Nc * 8 * J.N;
        J.rh = off;
        off += (size_t)Nc * J.N;
        J.rl = off;
        off += (size_t)Nc * J.N;
        off = (off + 31) & ~(size_t)31;
        J.RT = o.R * jobs[k].T;
        J.lnRT = std::log(J.RT);
        double aa[bt::kMaxNcBatch];
        for (int i = 0; i < Nc; ++i) aa[i] = a[i] * alpha_of(a[i], b[i], omega[i], jobs[k].T, o.R);
        for (int i = 0; i < Nc; ++i)
            for (int j = 0; j < Nc; ++j)
                J.A[i * bt::kMaxNcBatch + j] = std::sqrt(aa[i] * aa[j]) * (1.0 - (kij ? kij[i * Nc + j] : 0.0));
        bt_->maxN = std::max(bt_->maxN, J.N);
    }
    bt_->pool_floats = off;
    bt_->order.resize(njobs);
    for (int k = 0; k < njobs; ++k) bt_->order[k] = k;
    std::stable_sort(bt_->order.begin(), bt_->order.end(),
                     [&](int x, int y) { return bt_->jobs[x].N > bt_->jobs[y].N; });
    int st = LBM_OK;
    if (o.stream) {
        bt_->stream = (cudaStream_t)o.stream;
    } else if (cudaStreamCreateWithFlags(&bt_->stream, cudaStreamNonBlocking) == cudaSuccess) {
        bt_->own_stream = true;
    } else {
        st = LBM_ECUDA;
    }
    if (!st && (cudaMalloc(&bt_->pool, off * sizeof(float)) != cudaSuccess ||
                cudaMalloc(&bt_->d_jobs, njobs * sizeof(bt::Job)) != cudaSuccess ||
                cudaMalloc(&bt_->d_status, njobs * sizeof(bt::Status)) != cudaSuccess ||
                cudaMalloc(&bt_->d_order, njobs * sizeof(int)) != cudaSuccess ||
                cudaMalloc(&bt_->d_work, sizeof(int)) != cudaSuccess ||
                cudaMalloc(&bt_->d_nconv, sizeof(int)) != cudaSuccess ||
                cudaHostAlloc(&bt_->h_nconv, sizeof(int), cudaHostAllocDefault) != cudaSuccess))
        st = LBM_ENOMEM;
    if (!st) {
        cudaMemcpyAsync(bt_->d_jobs, bt_->jobs.data(), njobs * sizeof(bt::Job), cudaMemcpyHostToDevice, bt_->stream);
        cudaMemcpyAsync(bt_->d_order, bt_->order.data(), njobs * sizeof(int), cudaMemcpyHostToDevice, bt_->stream);
        cudaMemsetAsync(bt_->d_status, 0, njobs * sizeof(bt::Status), bt_->stream);
        cudaMemsetAsync(bt_->d_nconv, 0, sizeof(int), bt_->stream);
        double *d_rho = nullptr;
        long long maxf = (long long)Nc * bt_->maxN;
        if (cudaMalloc(&d_rho, maxf * sizeof(double)) != cudaSuccess) st = LBM_ENOMEM;
        for (int k = 0; !st && k < njobs; ++k) {
            const bt::Job &J = bt_->jobs[k];
            if (cudaMemcpyAsync(d_rho, jobs[k].rho, (size_t)Nc * J.N * sizeof(double), cudaMemcpyHostToDevice,
                                bt_->stream) != cudaSuccess) {
                st = LBM_ECUDA;
                break;
            }
            bt::k_batch_init<<<(unsigned)std::min<long long>((Nc * 8 * J.N + 255) / 256, 4096), 256, 0,
                               bt_->stream>>>(d_rho, J.N, Nc, bt_->pool + J.g[0], bt_->pool + J.rh,
                                              bt_->pool + J.rl);
            bt_->launches += 1;
        }
        if (cudaStreamSynchronize(bt_->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) st = LBM_ECUDA;
        cudaFree(d_rho);
    }
    if (!st) st = autotune(bt_);
    if (st) {
        release(bt_);
        delete bt_;
        return st;
    }
    *out = bt_;
    return LBM_OK;
}

int lbm_batch_run(lbm_batch *b, long long max_steps, int check_every, double tol, int *n_converged)
{
    if (!b || check_every < 1 || max_steps < 0 || !(tol >= 0.0)) return LBM_EINVAL;
    int st = capture(b, check_every, tol);
    if (st) return st;
    long long done = 0;
    for (;;) {
        if (cudaStreamSynchronize(b->stream) != cudaSuccess) return LBM_ECUDA;
        const int nconv = *b->h_nconv;
        if (n_converged) *n_converged = nconv;
        if (nconv >= b->njobs || done + check_every > max_steps) break;
        if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return LBM_ECUDA;
        b->launches += 1;
        b->rounds += 1;
        done += check_every;
    }
    return LBM_OK;
}

int lbm_batch_job_state(lbm_batch *b, int job, double *rho, long long *steps, double *last_drho,
                        int *converged)
{
    if (!b || job < 0 || job >= b->njobs) return LBM_EINVAL;
    bt::Status s;
    if (cudaMemcpyAsync(&s, b->d_status + job, sizeof(s), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return LBM_ECUDA;
    if (steps) *steps = s.steps;
    if (last_drho) *last_drho = s.last_drho;
    if (converged) *converged = s.converged;
    if (rho) {
        const bt::Job &J = b->jobs[job];
        const size_t n = (size_t)b->nc * J.N;
        std::vector<float> hi(n), lo(n);
        if (cudaMemcpyAsync(hi.data(), b->pool + J.rh, n * sizeof(float), cudaMemcpyDeviceToHost, b->stream) !=
                cudaSuccess ||
            cudaMemcpyAsync(lo.data(), b->pool + J.rl, n * sizeof(float), cudaMemcpyDeviceToHost, b->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(b->stream) != cudaSuccess)
            return LBM_ECUDA;
        for (size_t k = 0; k < n; ++k) rho[k] = (double)hi[k] + (double)lo[k];
    }
    return LBM_OK;
}

int lbm_batch_info(const lbm_batch *b, int *threads, int *ctas, long long *rounds, long long *launches)
{
    if (!b) return LBM_EINVAL;
    if (threads) *threads = b->threads;
    if (ctas) *ctas = b->ctas;
    if (rounds) *rounds = b->rounds;
    if (launches) *launches = b->launches;
    return LBM_OK;
}

int lbm_batch_set_threads(lbm_batch *b, int threads)
{
    if (!b || (threads != 128 && threads != 256 && threads != 512)) return LBM_EINVAL;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_steps = -1;
    return configure(b, threads);
}

int lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return LBM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    release(b);
    delete b;
    return LBM_OK;
}

}  // extern "C"
