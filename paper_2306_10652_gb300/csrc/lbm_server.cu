// lbm_server.cu -- the served form: a request loop over phase-equilibrium
// jobs with admission by a device-memory budget and continuous batching.
//
// Requests arrive at any time (lbm_server_submit copies them and returns).  A
// worker thread admits queued requests in arrival order while the estimated
// device bytes of the running jobs plus the next one stay within the budget
// and a slot is free.  Every admitted job is its own lbm_problem on its own
// CUDA stream, so the kernels of all running jobs overlap on the GPU.  The
// worker runs rounds: it enqueues `check_every` steps for every running job,
// then checks each job's convergence (largest density change over the round,
// the criterion of the batched form); converged, failed (non-finite
// densities) or exhausted jobs are retired with their densities and their
// latency, which frees their memory for the queue.  Because every job is an
// independent handle with deterministic kernels, a job's result is the same
// alone and in the mix.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <cmath>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "lbmfug.h"

namespace {

using clock_type = std::chrono::steady_clock;

struct Request {
    long long id = 0;
    int lattice = 0, nx = 0, ny = 0, nz = 0, nc = 0, precision = LBM_FP32DEV, check_every = 1000;
    std::vector<double> a, b, omega, kij, M, rho;
    double T = 0, tau = 1, kappa_ref = 0.02, tol = 1e-10;
    double bar = 1e-10;  // the convergence bar in use: tol, or 8 binary32 ulp of the largest density
    long long max_steps = 0;
    size_t bytes = 0;
    int state = 0;  // 0 queued, 1 running, 2 converged, 3 failed, 4 exhausted (max_steps)
    bool mem_wait = false;  // waited at the head of the queue for memory while a slot was free
    int error = LBM_OK;
    long long steps = 0;
    double last_drho = 0.0;
    clock_type::time_point t_submit, t_start, t_end;
    lbm_problem *h = nullptr;
    std::vector<double> result;
};

size_t estimate_bytes(int lattice, long long N, int nc, int precision)
{
    const int Q = lattice == LBM_D2Q9 ? 9 : 19;
    const int D = lattice == LBM_D2Q9 ? 2 : 3;
    const size_t f = (size_t)nc * N;
    size_t b = (precision == LBM_FP64) ? 2 * f * Q * 8 + 2 * f * 8 : 2 * f * ((Q - 1) * 4 + 8) + 2 * f * 4;
    if (precision != LBM_FP64) b += f * 8 + (size_t)N * 8;  // grad mu (or mu) pairs, psi pairs
    b += 2 * f * 8 + (size_t)N * 8 * (2 + D);  // three-pass scratch fields
    b += f * 8;                                 // convergence snapshot
    // reductions and launch tables, plus the device allocator's rounding of
    // each of about twenty buffers to its 2 MiB granule
    return b + (48u << 20);
}

}  // namespace

struct lbm_server {
    double budget_bytes = 0;
    int max_active = 8;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<long long, std::shared_ptr<Request>> all;
    std::vector<std::shared_ptr<Request>> active;
    long long next_id = 1;
    bool stop = false;
    size_t active_bytes = 0, peak_bytes = 0;
    long long completed = 0, rounds = 0;
    int peak_active = 0;         // most jobs running at once
    long long memory_waits = 0;  // requests held back by the budget with a slot free
    std::thread worker;

    void finish(const std::shared_ptr<Request> &r, int state)
    {
        if (r->h) {
            if (state == 2 || state == 4) {
                r->result.resize((size_t)r->nc * r->nx * r->ny * r->nz);
                const int st = lbm_moments(r->h, r->result.data(), nullptr, nullptr, nullptr);
                if (st) {
                    state = 3;
                    r->error = st;
                }
            }
            lbm_destroy(r->h);
            r->h = nullptr;
        }
        std::lock_guard<std::mutex> lock(mu);
        r->state = state;
        r->t_end = clock_type::now();
        active_bytes -= r->bytes;
        completed += 1;
        cv.notify_all();
    }

    bool start(const std::shared_ptr<Request> &r)
    {
        lbm_problem *h = nullptr;
        int st = lbm_create(&h, r->lattice, r->nx, r->ny, r->nz, r->nc, r->a.data(), r->b.data(),
                            r->omega.data(), r->kij.empty() ? nullptr : r->kij.data(), r->T, r->tau);
        if (!st) {
            lbm_options o;
            lbm_options_default(&o);
            o.precision = r->precision;
            o.kappa_ref = r->kappa_ref;
            o.M = r->M.empty() ? nullptr : r->M.data();
            st = lbm_set_options(h, &o);
        }
        if (!st) st = lbm_init_fields(h, r->rho.data(), nullptr);
        double d = 0.0;
        if (!st) st = lbm_convergence(h, &d);  // first call: snapshot of the initial state
        r->t_start = clock_type::now();
        r->h = h;
        if (st) {
            r->error = st;
            finish(r, 3);
            return false;
        }
        // binary32 storage jitters at the rounding of its populations: changes
        // below 8 ulp of binary32 at the largest density count as converged
        r->bar = r->tol;
        if (r->precision != LBM_FP64 && r->tol > 0.0) {
            double rmax = 0.0;  // largest total density over the nodes
            const size_t nn = r->rho.size() / (size_t)r->nc;
            for (size_t k = 0; k < nn; ++k) {
                double tot = 0.0;
                for (int i = 0; i < r->nc; ++i) tot += r->rho[(size_t)i * nn + k];
                rmax = std::max(rmax, tot);
            }
            int e = 0;
            std::frexp(1.05 * rmax, &e);  // 1.05 rmax in [2^(e-1), 2^e)
            r->bar = std::max(r->tol, 8.0 * std::ldexp(1.0, e - 1 - 23));
        }
        r->rho.clear();
        r->rho.shrink_to_fit();
        return true;
    }

    void loop()
    {
        for (;;) {
            // admission in arrival order, within the budget and the slots
            std::vector<std::shared_ptr<Request>> admit;
            {
                std::unique_lock<std::mutex> lock(mu);
                cv.wait_for(lock, std::chrono::milliseconds(active.empty() ? 50 : 0),
                            [&] { return stop || !queue.empty() || !active.empty(); });
                if (stop && queue.empty() && active.empty()) return;
                while (!queue.empty() && (int)(active.size() + admit.size()) < max_active &&
                       (double)(active_bytes + queue.front()->bytes) <= budget_bytes) {
                    auto r = queue.front();
                    queue.pop_front();
                    r->state = 1;
                    active_bytes += r->bytes;
                    if (active_bytes > peak_bytes) peak_bytes = active_bytes;
                    admit.push_back(r);
                }
                const int running = (int)(active.size() + admit.size());
                if (running > peak_active) peak_active = running;
                if (!queue.empty() && running < max_active && !queue.front()->mem_wait) {
                    queue.front()->mem_wait = true;
                    memory_waits += 1;
                }
            }
            for (auto &r : admit)
                if (start(r)) active.push_back(r);
            if (active.empty()) continue;
            // one round: enqueue every job's steps first, so that they overlap
            for (auto &r : active) {
                const long long n = std::min<long long>(r->check_every, r->max_steps - r->steps);
                if (n > 0 && !r->error) {
                    const int st = lbm_step_graph(r->h, n);
                    if (st) r->error = st;
                    r->steps += n;
                }
            }
            rounds += 1;
            std::vector<std::shared_ptr<Request>> still;
            for (auto &r : active) {
                double d = 0.0;
                int st = r->error ? r->error : lbm_convergence(r->h, &d);
                r->last_drho = d;
                if (st) {
                    r->error = st;
                    finish(r, 3);
                } else if (d < r->bar) {
                    finish(r, 2);
                } else if (r->steps >= r->max_steps) {
                    finish(r, 4);
                } else {
                    still.push_back(r);
                }
            }
            active.swap(still);
        }
    }
};

extern "C" {

int lbm_server_estimate_bytes(int lattice, int nx, int ny, int nz, int Nc, int precision, size_t *bytes)
{
    if (!bytes || nx < 1 || ny < 1 || nz < 1 || Nc < 1 || Nc > LBM_MAX_NC) return LBM_EINVAL;
    *bytes = estimate_bytes(lattice, (long long)nx * ny * nz, Nc, precision);
    return LBM_OK;
}

int lbm_server_create(lbm_server **out, double hbm_budget_frac, int max_active)
{
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!(hbm_budget_frac > 0.0 && hbm_budget_frac <= 1.0) || max_active < 1) return LBM_EINVAL;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return LBM_ECUDA;
    lbm_server *s = new (std::nothrow) lbm_server();
    if (!s) return LBM_ENOMEM;
    s->budget_bytes = hbm_budget_frac * (double)total_b;
    s->max_active = max_active;
    int dev = 0;
    cudaGetDevice(&dev);
    s->worker = std::thread([s, dev] {
        cudaSetDevice(dev);
        s->loop();
    });
    *out = s;
    return LBM_OK;
}

int lbm_server_submit(lbm_server *s, const lbm_request *q, long long *id)
{
    if (!s || !q || !q->a || !q->b || !q->omega || !q->rho) return LBM_EINVAL;
    if (q->Nc < 1 || q->Nc > LBM_MAX_NC || q->nx < 1 || q->ny < 1 || q->nz < 1 || q->check_every < 1 ||
        q->max_steps < 1 || !(q->tol >= 0.0))
        return LBM_EINVAL;
    auto r = std::make_shared<Request>();
    r->lattice = q->lattice;
    r->nx = q->nx;
    r->ny = q->ny;
    r->nz = q->nz;
    r->nc = q->Nc;
    r->precision = q->precision;
    r->check_every = q->check_every;
    r->a.assign(q->a, q->a + q->Nc);
    r->b.assign(q->b, q->b + q->Nc);
    r->omega.assign(q->omega, q->omega + q->Nc);
    if (q->kij) r->kij.assign(q->kij, q->kij + q->Nc * q->Nc);
    if (q->M) r->M.assign(q->M, q->M + q->Nc);
    const size_t n = (size_t)q->Nc * q->nx * q->ny * q->nz;
    r->rho.assign(q->rho, q->rho + n);
    r->T = q->T;
    r->tau = q->tau;
    r->kappa_ref = q->kappa_ref > 0.0 ? q->kappa_ref : 0.02;
    r->tol = q->tol;
    r->max_steps = q->max_steps;
    r->bytes = estimate_bytes(q->lattice, (long long)q->nx * q->ny * q->nz, q->Nc, q->precision);
    std::lock_guard<std::mutex> lock(s->mu);
    if ((double)r->bytes > s->budget_bytes) return LBM_ENOMEM;  // can never be admitted
    r->id = s->next_id++;
    r->t_submit = clock_type::now();
    s->queue.push_back(r);
    s->all[r->id] = r;
    if (id) *id = r->id;
    s->cv.notify_all();
    return LBM_OK;
}

int lbm_server_poll(lbm_server *s, long long id, int *state, long long *steps, double *latency_s,
                    double *last_drho)
{
    if (!s) return LBM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return LBM_EINVAL;
    const Request &r = *it->second;
    if (state) *state = r.state;
    if (steps) *steps = r.steps;
    if (last_drho) *last_drho = r.last_drho;
    if (latency_s)
        *latency_s = r.state >= 2 ? std::chrono::duration<double>(r.t_end - r.t_submit).count() : -1.0;
    return r.state == 3 ? r.error : LBM_OK;
}

int lbm_server_result(lbm_server *s, long long id, double *rho)
{
    if (!s || !rho) return LBM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return LBM_EINVAL;
    const Request &r = *it->second;
    if (r.state != 2 && r.state != 4) return LBM_ESTATE;
    std::memcpy(rho, r.result.data(), r.result.size() * sizeof(double));
    return LBM_OK;
}

int lbm_server_wait_all(lbm_server *s)
{
    if (!s) return LBM_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    s->cv.wait(lock, [&] { return s->queue.empty() && s->completed == (long long)s->all.size(); });
    return LBM_OK;
}

int lbm_server_stats(lbm_server *s, long long *submitted, long long *completed, size_t *peak_bytes,
                     double *budget_bytes, long long *rounds)
{
    if (!s) return LBM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (submitted) *submitted = (long long)s->all.size();
    if (completed) *completed = s->completed;
    if (peak_bytes) *peak_bytes = s->peak_bytes;
    if (budget_bytes) *budget_bytes = s->budget_bytes;
    if (rounds) *rounds = s->rounds;
    return LBM_OK;
}

int lbm_server_admission(lbm_server *s, int *peak_active, long long *memory_waits)
{
    if (!s) return LBM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    if (peak_active) *peak_active = s->peak_active;
    if (memory_waits) *memory_waits = s->memory_waits;
    return LBM_OK;
}

int lbm_server_times(lbm_server *s, long long id, double *queued_s, double *run_s)
{
    if (!s) return LBM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return LBM_EINVAL;
    const Request &r = *it->second;
    if (r.state < 2) return LBM_ESTATE;
    if (queued_s) *queued_s = std::chrono::duration<double>(r.t_start - r.t_submit).count();
    if (run_s) *run_s = std::chrono::duration<double>(r.t_end - r.t_start).count();
    return LBM_OK;
}

int lbm_server_destroy(lbm_server *s)
{
    if (!s) return LBM_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    delete s;
    return LBM_OK;
}

}  // extern "C"
