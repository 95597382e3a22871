/*
 * lbmfug.h -- C ABI of the GB300-native fugacity-based multicomponent lattice
 * Boltzmann library (Soomro & Ayala, "Unrestricted component count in
 * multiphase lattice Boltzmann: a fugacity-based approach", arXiv 2306.10652).
 *
 * One time step updates, at every node of a periodic D2Q9 or D3Q19 lattice,
 * the populations of all Nc components:
 *   Eq. (1a)  g_{a,i}(r + e_a, t + 1) = g_{a,i} - (g_{a,i} - g^eq_{a,i})/tau
 *                                      + (1 - 1/(2 tau)) F_{a,i}
 *   Eq. (1b)  well-balanced equilibrium with rho_i^c = 0
 *   Eq. (1c)  well-balanced forcing term
 *   Eq. (5)   F_i = -rho~_i RT grad ln f_i + rho~_i sum_j grad(sqrt(k_i k_j) lap rho~_j)
 *   Eqs. (9)-(12)  Peng-Robinson mixture pressure and fugacities with the
 *             van der Waals mixing rules and binary parameters delta_ij
 *   Eq. (6)   kappa_i = kappa_ref a_i / a_ref
 * Readings of what the paper leaves open (shared velocity, discrete
 * gradient/Laplacian, initial populations) are those of the library's design
 * notes: u = (sum e g + F/2)/rho, isotropic lattice stencils, g = g^eq(rho, u).
 *
 * Conventions
 *  - Every call returns an int status (LBM_OK = 0 or a negative LBM_E*);
 *    nothing else crosses the ABI (no exceptions, no aborts).
 *  - Host arrays are owned by the caller and copied; device memory of a
 *    problem is owned by the library (or by the caller's allocator hooks).
 *  - Field layout: component-major, then z, y, x with x fastest:
 *    rho[i][z][y][x], u[d][z][y][x].  Populations (get/set_state) are
 *    g[i][a][z][y][x] in the post-streaming convention of Eq. (1a), with the
 *    velocity order of lbm_lattice_velocities().
 *  - A handle is not thread-safe; separate handles are independent.
 *  - Work is enqueued on the handle's CUDA stream; calls that return host
 *    data synchronise that stream.
 */
#ifndef LBMFUG_H
#define LBMFUG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_MAX_NC 16

enum lbm_lattice { LBM_D2Q9 = 0, LBM_D3Q19 = 1 };

/* Population storage and arithmetic.
 *  LBM_FP64:    all Q populations stored in binary64, every operation binary64
 *               (the plain path).
 *  LBM_FP32DEV: populations stored as their deviation from the rest
 *               equilibrium (rho_i, 0, ..., 0) of Eq. (1b): the Q-1 moving
 *               populations in binary32, with the density rho_i itself kept
 *               exactly as a binary32 pair (hi + lo) that each step moves by
 *               compensated sums of the populations that left and arrived
 *               (component mass conserved to the rounding of the pair);
 *               collision in binary32; Peng-Robinson mixture, fugacities,
 *               chemical-potential differences of the force and mass sums at
 *               binary64 accuracy: the fused schedule evaluates them in
 *               double-binary32 arithmetic (pairs hi + lo of binary32 values
 *               with error-free sums and products, relative error about
 *               2^-44) on the binary32 units, which GB300 runs at 64 times
 *               its binary64 rate; the three-pass schedule uses binary64.
 *  LBM_FP32:    the LBM_FP32DEV storage, with the thermodynamics and forces of
 *               the fused schedule in binary32 too (the three-pass schedule
 *               keeps them in binary64). */
enum lbm_precision { LBM_FP64 = 0, LBM_FP32DEV = 1, LBM_FP32 = 2 };

/* Kernel schedule.
 *  LBM_SCHED_FUSED:     D2Q9 only: one step kernel that walks rows with the
 *                       densities, psi and mu rows on chip (LBM_FP32DEV adds
 *                       a pass that forms the double-binary32 grad mu).
 *  LBM_SCHED_MULTIPASS: LBM_FP32DEV on any lattice: a mu pass (double-
 *                       binary32), a collision pass (binary32) and a density
 *                       update that also forms psi for the next step.
 *  LBM_SCHED_THREEPASS: any lattice and storage, thermodynamics and forces
 *                       in binary64.
 *  LBM_SCHED_AUTO:      fused on D2Q9; multi-pass for LBM_FP32DEV on D3Q19;
 *                       three-pass otherwise. */
enum lbm_schedule { LBM_SCHED_AUTO = 0, LBM_SCHED_THREEPASS = 1, LBM_SCHED_FUSED = 2, LBM_SCHED_MULTIPASS = 3 };

enum lbm_status {
    LBM_OK = 0,
    LBM_EINVAL = -1,     /* invalid argument or parameter */
    LBM_ENOMEM = -2,     /* device or host allocation failed */
    LBM_ECUDA = -3,      /* CUDA runtime error (launch, copy, device) */
    LBM_ENONFINITE = -4, /* a non-finite density was detected */
    LBM_ETIMEOUT = -5,   /* a bounded device wait ran out */
    LBM_ESTATE = -6,     /* call not valid in the handle's current state */
    LBM_ENOTSUP = -7     /* combination not supported by this build */
};

typedef struct lbm_problem lbm_problem;

/* Allocation hooks: alloc returns device memory of `bytes` bytes on the
 * current device, free releases it.  ctx is passed through unchanged. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbm_free_fn)(void *ptr, size_t bytes, void *ctx);

typedef struct lbm_options {
    int precision;        /* enum lbm_precision, default LBM_FP64 */
    int schedule;         /* enum lbm_schedule, default LBM_SCHED_AUTO */
    double kappa_ref;     /* interface parameter of the reference component, default 0.02 (Sec. 3) */
    int kappa_ref_index;  /* reference component for Eq. (6), default 0 */
    const double *M;      /* molar masses M_i (rho_i = M_i rho~_i); NULL = all 1 */
    double R;             /* gas constant in lattice units, default 1 (Sec. 3.1) */
    void *stream;         /* cudaStream_t to enqueue on; NULL = a stream the library creates */
    int monitor_every;    /* > 0: every that many steps lbm_step also reduces the
                             per-component mass of the new state on the device
                             (read with lbm_monitor); 0 = off (default) */
    lbm_alloc_fn alloc;   /* NULL = cudaMalloc */
    lbm_free_fn free;     /* must be set together with alloc */
    void *alloc_ctx;
    int tune;             /* fused schedule: 1 (default) = the first lbm_step times
                             candidate launch geometries (strips per row, segment
                             waves, mu-pass waves) on the problem itself and keeps
                             the fastest, cached for the process by (precision, Nc,
                             nx, ny); 0 = the built-in geometry.  The geometry does
                             not change any result (every node's arithmetic is the
                             same); the first lbm_step then synchronises once. */
    int strip;            /* > 0: interior columns per CTA of the fused kernel (forces
                             the geometry, no tuning); 0 = automatic */
    int seg_h;            /* > 0: rows per CTA of the fused kernel; 0 = automatic */
} lbm_options;

/* Fill *opt with the defaults listed above. */
int lbm_options_default(lbm_options *opt);

/*
 * Create a problem: lattice LBM_D2Q9 (nz must be 1) or LBM_D3Q19, a periodic
 * nx*ny*nz box, Nc in 1..LBM_MAX_NC components with PR attraction a_i > 0 and
 * co-volume b_i > 0 in lattice units (Sec. 2.3), acentric factors omega_i,
 * binary parameters kij (Nc*Nc row-major, symmetric, zero diagonal,
 * |k_ij| < 1; NULL = all zero), temperature T > 0 and relaxation time
 * tau > 0.5.  T_c,i is implied by a_i/b_i (Sec. 2.3).  Allocates nothing on
 * the device until lbm_init_fields.  *out is NULL on failure.
 */
int lbm_create(lbm_problem **out, int lattice, int nx, int ny, int nz, int Nc,
               const double *a, const double *b, const double *omega, const double *kij,
               double T, double tau);

/* Set options; valid only before the first lbm_init_fields / lbm_set_state.
 * opt->M is copied. */
int lbm_set_options(lbm_problem *p, const lbm_options *opt);

/*
 * Initialise the populations at the equilibrium of Eq. (1b) for the given
 * mass densities rho[i][z][y][x] (> 0, finite) and velocity u[d][z][y][x]
 * (NULL = fluid at rest).  Host pointers.  Resets the step counter.
 */
int lbm_init_fields(lbm_problem *p, const double *rho, const double *u);

/* Same with device pointers (binary64, same layouts), enqueued on the handle's stream. */
int lbm_init_fields_device(lbm_problem *p, const double *d_rho, const double *d_u);

/* Advance n >= 0 time steps (asynchronous on the handle's stream).  Returns a
 * launch error or a sticky earlier error. */
int lbm_step(lbm_problem *p, long long n);

/*
 * The same as lbm_step(p, n), replayed from a CUDA graph: the first call for
 * a given n (and each of the two state buffers it can start from) captures
 * the n steps on the handle's stream and instantiates them, later calls
 * launch the graph.  For loops that advance a problem by the same n again
 * and again (the served form's rounds), where launching n steps kernel by
 * kernel would cost more than running them.  The first call synchronises
 * once if the fused schedule's geometry is not tuned yet; it must not be
 * made while the handle's stream is being captured by the caller (it then
 * falls back to lbm_step).  With the mass monitor on it is lbm_step.
 */
int lbm_step_graph(lbm_problem *p, long long n);

/*
 * Macroscopic fields of the current state into caller-owned host buffers
 * (any may be NULL): rho[i][...] mass densities; u[d][...] the velocity of
 * the forced step, (sum e g + F/2)/rho; p[...] the PR pressure of Eq. (9) at
 * the local composition; lnf[i][...] ln f_i of Eq. (12).  Synchronises.
 */
int lbm_moments(lbm_problem *p, double *rho, double *u, double *pressure, double *lnf);

/* Same into device buffers, enqueued on the handle's stream. */
int lbm_moments_device(lbm_problem *p, double *d_rho, double *d_u, double *d_pressure,
                       double *d_lnf);

/*
 * Chemical potentials and interaction forces of the current state, D2Q9
 * only, into caller-owned host buffers (either may be NULL, not both):
 * F[i][d][y][x] = -rho~_i (grad mu_i)_d and mu[i][y][x] = RT ln f_i -
 * sqrt(kappa_i) lap psi, the force of Eq. (5) with kappa_ij =
 * sqrt(kappa_i kappa_j) (Eq. 4), psi = sum_j sqrt(kappa_j) rho~_j and the
 * isotropic lattice stencils for grad and lap.  They are evaluated with the
 * arithmetic the step uses: binary64 (LBM_FP64, or the three-pass
 * schedule), double-binary32 (LBM_FP32DEV fused: mu carried as a pair,
 * every difference of the gradient taken on the pairs and rounded once, F
 * in binary32) or binary32 (LBM_FP32 fused).  LBM_ENOTSUP for D3Q19.
 * Synchronises.
 */
int lbm_forces(lbm_problem *p, double *F, double *mu);

/*
 * Launch geometry of the handle's step (valid after lbm_init_fields):
 * *fused = 1 for the single-pass D2Q9 kernel, 0 for the three-pass
 * schedule; for the fused kernel, the interior columns per CTA (*strip),
 * CTAs along x (*nstrips), rows per CTA (*seg_h) and CTAs along y (*segs).
 * Any pointer may be NULL.
 */
int lbm_schedule_info(const lbm_problem *p, int *fused, int *strip, int *nstrips, int *seg_h,
                      int *segs);

/*
 * Per-component total mass sum_r rho_i(r) into mass[Nc] (host), summed in a
 * fixed order (bitwise reproducible).  Returns LBM_ENONFINITE if any density
 * is not finite.  Synchronises.
 */
int lbm_mass(lbm_problem *p, double *mass);

/*
 * Convergence monitor: max over nodes and components of
 * |rho_i(t) - rho_i(t_snap)|, where t_snap is the state at the previous call
 * (the first call only takes the snapshot and reports +inf).  Synchronises.
 */
int lbm_convergence(lbm_problem *p, double *max_abs_drho);

/* Latest on-device mass reduction of lbm_step's monitor (see
 * lbm_options.monitor_every) into mass[Nc] (host) and the step it was taken
 * at; *nonfinite = 1 if a non-finite density was seen since the last
 * lbm_init_fields.  Synchronises. */
int lbm_monitor(lbm_problem *p, double *mass, long long *at_step, int *nonfinite);

/* Number of kernels this handle has launched (every launch is counted). */
int lbm_launch_count(const lbm_problem *p, long long *launches);

/* Device time of each kernel of the steps, measured with two CUDA events
 * recorded on the handle's stream around every launch of lbm_step (the
 * launch-geometry trials of the first step are not recorded).  Off by
 * default.  lbm_timing_enable(p, 1) zeroes the counters and starts recording;
 * lbm_timing_enable(p, 0) stops and discards them (both synchronise the
 * stream when a timer exists).  While recording, lbm_step_graph runs as
 * lbm_step, and lbm_step synchronises the stream once per 4096 recorded
 * launches to read and recycle the events.  Returns LBM_EINVAL (null p, on
 * not 0 or 1), LBM_ENOMEM, LBM_ECUDA. */
int lbm_timing_enable(lbm_problem *p, int on);

typedef struct lbm_kernel_time {
    const char *name;   /* static string naming the kernel (owned by the library) */
    long long launches; /* launches timed since lbm_timing_enable(p, 1) */
    double total_ms;    /* sum of their event-to-event times, milliseconds */
} lbm_kernel_time;

/* Synchronises the handle's stream, then writes one entry per kernel that
 * has launched since timing was enabled (a fixed order) into out[0 ..
 * min(max, *n)) and the number of such kernels into *n.  The counters keep
 * accumulating.  Returns LBM_EINVAL (null p or n, max < 0, out null with
 * max > 0), LBM_ESTATE (timing not enabled), LBM_ECUDA. */
int lbm_timing_read(lbm_problem *p, lbm_kernel_time *out, int max, int *n);

/* Raw populations, binary64, layout g[i][a][z][y][x] (post-streaming).
 * *bytes in: capacity of buf; out: bytes needed.  buf NULL = size query. */
int lbm_get_state(lbm_problem *p, double *buf, size_t *bytes);
int lbm_set_state(lbm_problem *p, const double *buf, size_t bytes);

/* Steps taken since the last init/set_state. */
int lbm_step_count(const lbm_problem *p, long long *steps);

/* Wait for all work enqueued on the handle's stream. */
int lbm_synchronize(lbm_problem *p);

/* Release the handle and its device memory.  NULL-safe. */
int lbm_destroy(lbm_problem *p);

/*
 * Per-component sums out[i] = sum_{r < n} field[i * n + r] of a caller-owned
 * binary64 device array field[nc][n] (for example the densities written by
 * lbm_moments_device), into the caller's device array out[nc], enqueued on
 * `stream` (a cudaStream_t; NULL = the legacy default stream).  The paper
 * has no counterpart: this is a service for callers that cannot allocate
 * device memory at the point where they need the reduction (a foreign
 * memory pool owns the device, or a host callback or real-time loop cannot
 * take the synchronisation of cudaMalloc).  It allocates nothing: the
 * per-block partial sums live in a fixed scratch area inside the library
 * (1216 * LBM_MAX_NC doubles, about 152 KB, held on every device that loads
 * the library until the process exits).  The summation order is the same
 * fixed order as lbm_mass.  If d_nonfinite is not NULL it receives 1 when a
 * non-finite value was seen, else 0.  Returns LBM_EINVAL for NULL pointers,
 * n < 1, or nc outside 1..LBM_MAX_NC (the scratch capacity).  The first call
 * on a device looks up the scratch address and should come before any
 * stream capture; the address is looked up again after the device's context
 * was rebuilt (for example by cudaDeviceReset).  Calls share the scratch:
 * calls that can overlap on the GPU race.
 */
int lbm_field_sums_noalloc(const double *d_field, int nc, long long n, double *d_out,
                           int *d_nonfinite, void *stream);

/* ------------------------------------------------------------------------
 * Batched form: many small independent D2Q9 problems (for example the
 * points of a ternary-diagram sweep, each a flat-interface slab at its own
 * temperature, as in the paper's Sec. 3.3) sharing the components' PR
 * parameters.  One persistent kernel advances all of them, a round of
 * `check_every` steps per problem per launch, replayed from a captured CUDA
 * graph; every round each problem's densities are compared with those at
 * the start of the round and a problem whose largest change is below `tol`
 * is finished and skipped from then on.  Storage is the binary32 format of
 * LBM_FP32DEV/LBM_FP32 (opt->precision selects binary64 or binary32
 * thermodynamics; LBM_FP64 is taken as LBM_FP32DEV).  The CTA size is chosen
 * by timed trials on the first creation for a given (precision, Nc, largest
 * box) and cached for the process; results do not depend on it.
 * ------------------------------------------------------------------------ */
typedef struct lbm_job {
    int nx, ny;          /* periodic box, nx * ny <= 2^20 and fitting shared memory */
    double T;            /* temperature (lattice units) */
    const double *rho;   /* initial mass densities [Nc][ny][nx] (host, > 0) */
} lbm_job;

typedef struct lbm_batch lbm_batch;

/* Nc in 1..10; a, b, omega, kij (NULL = 0) and tau as lbm_create; opt may be
 * NULL (defaults; opt->M, R, kappa_ref, kappa_ref_index, stream are used). */
int lbm_batch_create(lbm_batch **out, int Nc, const double *a, const double *b, const double *omega,
                     const double *kij, double tau, const lbm_options *opt, const lbm_job *jobs,
                     int njobs);

/* Run rounds of check_every steps until every problem has finished or
 * max_steps steps have been taken.  A problem finishes when the largest
 * change of its densities over a round is below max(tol, 8 ulp) (converged),
 * ulp being the spacing of binary32 numbers at the problem's largest total
 * density sum_i rho_i (the stored populations are binary32, and below that their
 * rounding, not relaxation, moves the densities), or when a density is not
 * finite (failed; it is retired and the others go on).  tol = 0 runs every
 * problem to max_steps.
 * *n_converged receives the number of finished problems.  Synchronises. */
int lbm_batch_run(lbm_batch *b, long long max_steps, int check_every, double tol, int *n_converged);

/* State of problem `job`: densities rho[Nc][ny][nx] (host, may be NULL), steps
 * taken, the largest density change of its last round, and *converged =
 * 0 running, 1 converged, 2 failed. */
int lbm_batch_job_state(lbm_batch *b, int job, double *rho, long long *steps, double *last_drho,
                        int *converged);

/* Launch geometry chosen by the tuner, rounds run and kernels launched. */
int lbm_batch_info(const lbm_batch *b, int *threads, int *ctas, long long *rounds,
                   long long *launches);

/* Override the CTA size (128, 256 or 512 threads). */
int lbm_batch_set_threads(lbm_batch *b, int threads);

int lbm_batch_destroy(lbm_batch *b);

/* ------------------------------------------------------------------------
 * Served form: a request loop over phase-equilibrium jobs (a problem run
 * "to equilibrium" as in the paper's Sec. 3, Eqs. 1-12).  Requests of any
 * lattice, size, Nc and (T, composition) arrive at any time; a worker thread
 * admits them in arrival order while the estimated device bytes of the
 * running jobs stay within hbm_budget_frac of the device memory and fewer
 * than max_active jobs run; every running job is its own problem on its own
 * stream, advanced in rounds of check_every steps whose kernels overlap on
 * the GPU; a job finishes when the largest density change over a round is
 * below tol (converged; with binary32 storage and tol > 0 below max(tol,
 * 8 ulp of binary32 at 1.05 times its largest initial total density)), when a density is
 * not finite (failed) or after
 * max_steps steps (exhausted), and its memory goes to the next request.
 * ------------------------------------------------------------------------ */
typedef struct lbm_request {
    int lattice, nx, ny, nz, Nc;          /* as lbm_create */
    const double *a, *b, *omega, *kij;    /* kij may be NULL */
    const double *M;                      /* molar masses, NULL = 1 */
    double T, tau, kappa_ref;             /* kappa_ref <= 0 = 0.02 */
    const double *rho;                    /* initial densities [Nc][nz][ny][nx] (host; copied) */
    int precision;                        /* enum lbm_precision */
    int check_every;                      /* steps per round */
    long long max_steps;
    double tol;                           /* convergence: max |d rho| per round */
} lbm_request;

typedef struct lbm_server lbm_server;

/* Device bytes a request of this size would hold while running. */
int lbm_server_estimate_bytes(int lattice, int nx, int ny, int nz, int Nc, int precision, size_t *bytes);

/* Start the request loop on the current device.  hbm_budget_frac in (0, 1]
 * of the device's total memory (0.8 is the intended setting). */
int lbm_server_create(lbm_server **out, double hbm_budget_frac, int max_active);

/* Queue a request (inputs are copied; returns at once).  *id identifies it.
 * LBM_ENOMEM if the request alone exceeds the budget. */
int lbm_server_submit(lbm_server *s, const lbm_request *r, long long *id);

/* *state: 0 queued, 1 running, 2 converged, 3 failed, 4 max_steps reached;
 * latency (submit to finish, seconds; -1 while unfinished).  Returns the
 * job's error status if it failed. */
int lbm_server_poll(lbm_server *s, long long id, int *state, long long *steps, double *latency_s,
                    double *last_drho);

/* Final densities [Nc][nz][ny][nx] of a finished (state 2 or 4) request. */
int lbm_server_result(lbm_server *s, long long id, double *rho);

/* Block until every submitted request has finished. */
int lbm_server_wait_all(lbm_server *s);

int lbm_server_stats(lbm_server *s, long long *submitted, long long *completed, size_t *peak_bytes,
                     double *budget_bytes, long long *rounds);

/* Admission record: the most requests that ran at once, and the number of
 * requests that waited at the head of the queue because the memory budget
 * (not the max_active slots) held them back. */
int lbm_server_admission(lbm_server *s, int *peak_active, long long *memory_waits);

/* Seconds a finished request (state 2, 3 or 4) spent queued (submission to
 * start) and running (start to finish).  LBM_ESTATE while it is unfinished,
 * LBM_EINVAL for an unknown id. */
int lbm_server_times(lbm_server *s, long long id, double *queued_s, double *run_s);

/* Finish the queued and running requests, then stop the loop. */
int lbm_server_destroy(lbm_server *s);

/* Lattice description: D, Q and the velocities e[Q][3] used by get/set_state. */
int lbm_lattice_velocities(int lattice, int *D, int *Q, int *e);

/* Static text for a status code. */
const char *lbm_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* LBMFUG_H */
