/*
 * lbm_oracle.c -- plain, slow, FP64 CPU oracle for the fugacity-based
 * multicomponent lattice Boltzmann method (Soomro & Ayala, arXiv 2306.10652).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  It shares no code, header, table or constant
 * generator with the CUDA library; only tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.
 *
 * Every routine walks the equations of the paper in the paper's order and
 * notation, one lattice node at a time, with no blocking and no fusion:
 *   - Sec. 2.1, Eq. (1a)   lattice Boltzmann equation (BGK + forcing)
 *   - Sec. 2.1, Eq. (1b)   well-balanced equilibrium, rho^c = 0
 *   - Sec. 2.1, Eq. (1c)   well-balanced forcing term
 *   - Sec. 2.1, Eq. (5)    body force -rho~_i RT grad ln f_i
 *                           + rho~_i sum_j grad(sqrt(k_i k_j) lap rho~_j)
 *   - Sec. 2.2, Eq. (6)    kappa_i = kappa_ref a_i / a_ref
 *   - Sec. 2.3, Eq. (9)    Peng-Robinson pressure
 *   - Sec. 2.3, Eqs. (10)-(11) van der Waals mixing rules with delta_ij
 *   - Sec. 2.3, alpha_i(omega_i, T_r) below Eq. (11)
 *   - Sec. 2.3, Eq. (12)   Peng-Robinson fugacity
 * Readings where the paper is silent (macroscopic velocity, discrete
 * gradient and Laplacian, initial populations) are stated at the routine
 * that takes them.
 *
 * Population state convention: g[i][alpha][node] holds the post-streaming
 * (pre-collision) populations g_{alpha,i}(r, t) of Eq. (1a), node index
 * x + nx*(y + ny*z), x fastest.
 *
 * Loops over nodes whose iterations are independent carry OpenMP pragmas
 * (built with -fopenmp; orc_set_threads picks the thread count).  Every
 * value is computed by one thread with the same operations in the same
 * order as serially, so results do not depend on the thread count; the one
 * reduction (orc_mass) stays serial.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define ORC_MAXNC 16
#define ORC_PAR_MIN 4096 /* nodes below which the loops run on one thread */
#define ORC_MAXQ 19

/* ------------------------------------------------------------------ */
/* Lattices (standard D2Q9 / D3Q19 velocity sets and weights).          */
/* ------------------------------------------------------------------ */
typedef struct {
    int D, Q;
    int e[ORC_MAXQ][3];
    double w[ORC_MAXQ];
    double cs2;
} orc_lattice;

static void orc_make_lattice(int lattice, orc_lattice *L)
{
    memset(L, 0, sizeof(*L));
    L->cs2 = 1.0 / 3.0;
    if (lattice == 0) { /* D2Q9 */
        static const int e9[9][2] = {{0, 0},  {1, 0},  {0, 1},  {-1, 0}, {0, -1},
                                     {1, 1},  {-1, 1}, {-1, -1}, {1, -1}};
        L->D = 2;
        L->Q = 9;
        for (int a = 0; a < 9; ++a) {
            L->e[a][0] = e9[a][0];
            L->e[a][1] = e9[a][1];
            L->e[a][2] = 0;
            L->w[a] = (a == 0) ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
        }
    } else { /* D3Q19 */
        int a = 0;
        L->D = 3;
        L->Q = 19;
        L->e[a][0] = L->e[a][1] = L->e[a][2] = 0;
        L->w[a++] = 1.0 / 3.0;
        for (int d = 0; d < 3; ++d)
            for (int s = 1; s >= -1; s -= 2) {
                L->e[a][0] = L->e[a][1] = L->e[a][2] = 0;
                L->e[a][d] = s;
                L->w[a++] = 1.0 / 18.0;
            }
        for (int d1 = 0; d1 < 3; ++d1)
            for (int d2 = d1 + 1; d2 < 3; ++d2)
                for (int s1 = 1; s1 >= -1; s1 -= 2)
                    for (int s2 = 1; s2 >= -1; s2 -= 2) {
                        L->e[a][0] = L->e[a][1] = L->e[a][2] = 0;
                        L->e[a][d1] = s1;
                        L->e[a][d2] = s2;
                        L->w[a++] = 1.0 / 36.0;
                    }
    }
}

/* ------------------------------------------------------------------ */
/* Problem description (lattice units).                                 */
/* ------------------------------------------------------------------ */
typedef struct {
    int lattice;         /* 0 = D2Q9, 1 = D3Q19 */
    int nx, ny, nz;      /* periodic box; nz = 1 for D2Q9 */
    int nc;              /* number of components N */
    double a[ORC_MAXNC]; /* PR attraction a_i */
    double b[ORC_MAXNC]; /* PR co-volume b_i */
    double omega[ORC_MAXNC];
    double kij[ORC_MAXNC * ORC_MAXNC]; /* binary interaction delta_ij */
    double M[ORC_MAXNC];               /* molar masses, rho_i = M_i rho~_i */
    double T, tau, R;
    double kappa_ref;
    int kappa_ref_index;
} orc_problem;

int orc_problem_size(void) { return (int)sizeof(orc_problem); }

int orc_problem_set(orc_problem *P, int lattice, int nx, int ny, int nz, int nc,
                    const double *a, const double *b, const double *omega,
                    const double *kij, const double *M, double T, double tau,
                    double R, double kappa_ref, int kappa_ref_index)
{
    if (nc < 1 || nc > ORC_MAXNC || nx < 1 || ny < 1 || nz < 1) return -1;
    if (lattice == 0 && nz != 1) return -1;
    memset(P, 0, sizeof(*P));
    P->lattice = lattice;
    P->nx = nx;
    P->ny = ny;
    P->nz = nz;
    P->nc = nc;
    for (int i = 0; i < nc; ++i) {
        P->a[i] = a[i];
        P->b[i] = b[i];
        P->omega[i] = omega[i];
        P->M[i] = M ? M[i] : 1.0;
        for (int j = 0; j < nc; ++j) P->kij[i * ORC_MAXNC + j] = kij ? kij[i * nc + j] : 0.0;
    }
    P->T = T;
    P->tau = tau;
    P->R = R;
    P->kappa_ref = kappa_ref;
    P->kappa_ref_index = kappa_ref_index;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3: pure-component PR temperature function alpha_i.            */
/* a_i = 0.457235529 R^2 Tc^2 / pc and b_i = 0.077796074 R Tc / pc, so  */
/* the critical temperature follows from (a_i, b_i) alone:              */
/*   Tc_i = (0.077796074 / 0.457235529) a_i / (R b_i).                  */
/* ------------------------------------------------------------------ */
double orc_critical_temperature(double a, double b, double R)
{
    return (0.077796074 / 0.457235529) * a / (R * b);
}

double orc_alpha(double a, double b, double omega, double T, double R)
{
    double Tr = T / orc_critical_temperature(a, b, R);
    double m;
    if (omega <= 0.49)
        m = 0.374640 + 1.54226 * omega - 0.26992 * omega * omega;
    else
        m = 0.379642 + 1.48503 * omega - 0.164423 * omega * omega +
            0.016666 * omega * omega * omega;
    double s = 1.0 + m * (1.0 - sqrt(Tr));
    return s * s;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.3: mixture pressure (Eq. 9) and fugacities (Eq. 12) at one    */
/* state given by the molar densities rho~_i.                           */
/*                                                                      */
/* Eq. (12) as printed is ln(f_i/(x_i p)) = ... - ln((v-b_m) p / RT)    */
/* + ...; adding ln(x_i p) to both sides, the two p's cancel and        */
/* ln f_i = ln(x_i RT/(v - b_m)) + ...  The oracle uses that cancelled  */
/* form, which is Eq. (12) exactly when p > 0 and stays defined when    */
/* the PR pressure is not positive (inside the spinodal).               */
/* ------------------------------------------------------------------ */
int orc_eos(const orc_problem *P, const double *rho_molar, double *p_out, double *lnf_out)
{
    const int N = P->nc;
    const double R = P->R, T = P->T, RT = R * T;
    double rho = 0.0;
    for (int i = 0; i < N; ++i) rho += rho_molar[i];
    if (!(rho > 0.0)) return -1;
    double x[ORC_MAXNC], aal[ORC_MAXNC];
    for (int i = 0; i < N; ++i) {
        x[i] = rho_molar[i] / rho;
        aal[i] = P->a[i] * orc_alpha(P->a[i], P->b[i], P->omega[i], T, R);
    }
    /* Eq. (10): (a alpha)_m = sum_i sum_j x_i x_j sqrt((aa)_i (aa)_j)(1 - delta_ij) */
    double aam = 0.0;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            aam += x[i] * x[j] * sqrt(aal[i] * aal[j]) * (1.0 - P->kij[i * ORC_MAXNC + j]);
    /* Eq. (11): b_m = sum_i x_i b_i */
    double bm = 0.0;
    for (int i = 0; i < N; ++i) bm += x[i] * P->b[i];
    /* Eq. (9) with v = 1/rho~ */
    double v = 1.0 / rho;
    double p = RT / (v - bm) - aam / (v * v + 2.0 * bm * v - bm * bm);
    if (p_out) *p_out = p;
    if (lnf_out) {
        const double sq2 = sqrt(2.0);
        double logratio = log((v + (1.0 + sq2) * bm) / (v + (1.0 - sq2) * bm));
        for (int i = 0; i < N; ++i) {
            double sum_aij = 0.0; /* sum_j x_j (a alpha)_ij */
            for (int j = 0; j < N; ++j)
                sum_aij += x[j] * sqrt(aal[i] * aal[j]) * (1.0 - P->kij[i * ORC_MAXNC + j]);
            double t1 = (P->b[i] / bm) * (p * v / RT - 1.0);
            double t2 = log(x[i] * RT / (v - bm)); /* ln(x_i p) - ln((v-b_m) p/RT) */
            double t3 = aam / (2.0 * sq2 * bm * RT) * (P->b[i] / bm - 2.0 / aam * sum_aij) * logratio;
            lnf_out[i] = t1 + t2 + t3;
        }
    }
    return 0;
}

/* Eq. (6): kappa_i = kappa_ref a_i / a_ref (reference component index). */
static void orc_kappa(const orc_problem *P, double *kappa)
{
    double aref = P->a[P->kappa_ref_index];
    for (int i = 0; i < P->nc; ++i) kappa[i] = P->kappa_ref * P->a[i] / aref;
}

/* ------------------------------------------------------------------ */
/* Eq. (1b) with rho^c = 0 and Eq. (1c) at one node for one component.  */
/* ------------------------------------------------------------------ */
static void orc_feq_forcing_L(const orc_lattice *L, double rho_i, const double *u,
                              const double *F_i, const double *grad_rho_i,
                              double *geq, double *Fa)
{
    const double cs2 = L->cs2;
    const int D = L->D;
    double uu = 0.0;
    for (int d = 0; d < D; ++d) uu += u[d] * u[d];
    for (int a = 0; a < L->Q; ++a) {
        double ue = 0.0, e2 = 0.0;
        for (int d = 0; d < D; ++d) {
            ue += u[d] * L->e[a][d];
            e2 += (double)(L->e[a][d] * L->e[a][d]);
        }
        double bracket = ue / cs2 + ue * ue / (2.0 * cs2 * cs2) - uu / (2.0 * cs2);
        const double rho_c = 0.0; /* numerical constant rho_i^c, set to 0 */
        if (a == 0)
            geq[a] = rho_i - (1.0 - L->w[0]) * rho_c + L->w[0] * rho_i * bracket;
        else
            geq[a] = L->w[a] * rho_c + L->w[a] * rho_i * bracket;
        /* Eq. (1c) */
        double t1 = 0.0, t2 = 0.0;
        for (int d = 0; d < D; ++d) {
            double ed = (double)L->e[a][d];
            double vF = (ed - u[d]) / cs2 + ue * ed / (cs2 * cs2);
            double vG = -u[d] + ue * ed / cs2 + 0.5 * (e2 / cs2 - (double)D) * u[d];
            t1 += F_i[d] * vF;
            t2 += grad_rho_i[d] * vG;
        }
        Fa[a] = L->w[a] * t1 + L->w[a] * t2;
    }
}

int orc_feq_forcing(int lattice, double rho_i, const double *u, const double *F_i,
                    const double *grad_rho_i, double *geq, double *Fa)
{
    orc_lattice L;
    orc_make_lattice(lattice, &L);
    orc_feq_forcing_L(&L, rho_i, u, F_i, grad_rho_i, geq, Fa);
    return L.Q;
}

/* ------------------------------------------------------------------ */
/* Discrete differential operators (the paper does not state them; the  */
/* reading taken is the isotropic lattice stencils):                    */
/*   grad X(r) = (1/cs2) sum_a w_a e_a X(r + e_a)                       */
/*   lap  X(r) = (2/cs2) sum_a w_a [X(r + e_a) - X(r)]                  */
/* on the periodic box.                                                 */
/* ------------------------------------------------------------------ */
static long orc_neighbor(const orc_problem *P, int x, int y, int z, const int *e)
{
    int xx = ((x + e[0]) % P->nx + P->nx) % P->nx;
    int yy = ((y + e[1]) % P->ny + P->ny) % P->ny;
    int zz = ((z + e[2]) % P->nz + P->nz) % P->nz;
    return (long)xx + (long)P->nx * ((long)yy + (long)P->ny * zz);
}

static void orc_gradient_L(const orc_problem *P, const orc_lattice *L, const double *X,
                           double *G /*[D][N]*/)
{
    const long N = (long)P->nx * P->ny * P->nz;
#pragma omp parallel for collapse(2) schedule(static) if ((long)P->nx * P->ny * P->nz >= ORC_PAR_MIN)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long r = (long)x + (long)P->nx * ((long)y + (long)P->ny * z);
                for (int d = 0; d < L->D; ++d) {
                    double s = 0.0;
                    for (int a = 0; a < L->Q; ++a)
                        s += L->w[a] * L->e[a][d] * X[orc_neighbor(P, x, y, z, L->e[a])];
                    G[d * N + r] = s / L->cs2;
                }
            }
}

static void orc_laplacian_L(const orc_problem *P, const orc_lattice *L, const double *X,
                            double *Y)
{
#pragma omp parallel for collapse(2) schedule(static) if ((long)P->nx * P->ny * P->nz >= ORC_PAR_MIN)
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                long r = (long)x + (long)P->nx * ((long)y + (long)P->ny * z);
                double s = 0.0;
                for (int a = 0; a < L->Q; ++a)
                    s += L->w[a] * (X[orc_neighbor(P, x, y, z, L->e[a])] - X[r]);
                Y[r] = 2.0 * s / L->cs2;
            }
}

int orc_gradient(const orc_problem *P, const double *X, double *G)
{
    orc_lattice L;
    orc_make_lattice(P->lattice, &L);
    orc_gradient_L(P, &L, X, G);
    return 0;
}

int orc_laplacian(const orc_problem *P, const double *X, double *Y)
{
    orc_lattice L;
    orc_make_lattice(P->lattice, &L);
    orc_laplacian_L(P, &L, X, Y);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Macroscopic fields of one state g(t): densities, body forces         */
/* (Eq. 5), velocity, pressure (Eq. 9) and ln f_i (Eq. 12).             */
/*                                                                      */
/* Velocity reading (the paper names u but defers its definition):      */
/*   u = (sum_i sum_a e_a g_{a,i} + 1/2 sum_i F_i) / sum_i rho_i,       */
/* one barycentric velocity shared by all components.                   */
/* ------------------------------------------------------------------ */
typedef struct {
    double *rho;      /* [nc][N] mass density rho_i */
    double *rhom;     /* [nc][N] molar density rho~_i = rho_i / M_i */
    double *lnf;      /* [nc][N] */
    double *p;        /* [N] */
    double *F;        /* [nc][D][N] body force F_i */
    double *gradrho;  /* [nc][D][N] grad rho_i */
    double *u;        /* [D][N] */
    double *scratch;  /* work: lap rho~_j [nc][N], Phi_i [N], grad [D][N] */
} orc_fields;

static int orc_fields_alloc(const orc_problem *P, int D, orc_fields *f)
{
    const long N = (long)P->nx * P->ny * P->nz;
    const int nc = P->nc;
    f->rho = calloc((size_t)nc * N, sizeof(double));
    f->rhom = calloc((size_t)nc * N, sizeof(double));
    f->lnf = calloc((size_t)nc * N, sizeof(double));
    f->p = calloc((size_t)N, sizeof(double));
    f->F = calloc((size_t)nc * D * N, sizeof(double));
    f->gradrho = calloc((size_t)nc * D * N, sizeof(double));
    f->u = calloc((size_t)D * N, sizeof(double));
    f->scratch = calloc((size_t)(nc + 1 + D) * N, sizeof(double));
    if (!f->rho || !f->rhom || !f->lnf || !f->p || !f->F || !f->gradrho || !f->u || !f->scratch)
        return -1;
    return 0;
}

static void orc_fields_free(orc_fields *f)
{
    free(f->rho);
    free(f->rhom);
    free(f->lnf);
    free(f->p);
    free(f->F);
    free(f->gradrho);
    free(f->u);
    free(f->scratch);
}

static int orc_macroscopic(const orc_problem *P, const orc_lattice *L, const double *g,
                           orc_fields *f)
{
    const long N = (long)P->nx * P->ny * P->nz;
    const int nc = P->nc, Q = L->Q, D = L->D;
    const double RT = P->R * P->T;
    double kappa[ORC_MAXNC];
    orc_kappa(P, kappa);

    /* densities: rho_i = sum_a g_{a,i}; rho~_i = rho_i / M_i */
    for (int i = 0; i < nc; ++i)
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
        for (long r = 0; r < N; ++r) {
            double s = 0.0;
            for (int a = 0; a < Q; ++a) s += g[((long)i * Q + a) * N + r];
            f->rho[(long)i * N + r] = s;
            f->rhom[(long)i * N + r] = s / P->M[i];
        }
    /* Eq. (9), Eq. (12) node by node */
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad) if (N >= ORC_PAR_MIN)
    for (long r = 0; r < N; ++r) {
        double rm[ORC_MAXNC], lf[ORC_MAXNC], p;
        for (int i = 0; i < nc; ++i) rm[i] = f->rhom[(long)i * N + r];
        if (orc_eos(P, rm, &p, lf) != 0) {
            bad = 1;
            continue;
        }
        f->p[r] = p;
        for (int i = 0; i < nc; ++i) f->lnf[(long)i * N + r] = lf[i];
    }
    if (bad) return -2;
    /* Eq. (5): F_i = -rho~_i RT grad ln f_i + rho~_i sum_j grad(sqrt(k_i k_j) lap rho~_j) */
    double *lap = f->scratch;               /* [nc][N] lap rho~_j */
    double *Phi = f->scratch + (long)nc * N; /* [N] */
    double *G = Phi + N;                     /* [D][N] */
    for (int j = 0; j < nc; ++j) orc_laplacian_L(P, L, f->rhom + (long)j * N, lap + (long)j * N);
    for (int i = 0; i < nc; ++i) {
        /* interface part: Phi_i = sum_j sqrt(kappa_i kappa_j) lap rho~_j */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
        for (long r = 0; r < N; ++r) {
            double s = 0.0;
            for (int j = 0; j < nc; ++j) s += sqrt(kappa[i] * kappa[j]) * lap[(long)j * N + r];
            Phi[r] = s;
        }
        orc_gradient_L(P, L, Phi, G);
        for (int d = 0; d < D; ++d)
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
            for (long r = 0; r < N; ++r)
                f->F[((long)i * D + d) * N + r] = f->rhom[(long)i * N + r] * G[(long)d * N + r];
        /* bulk part: -rho~_i RT grad ln f_i */
        orc_gradient_L(P, L, f->lnf + (long)i * N, G);
        for (int d = 0; d < D; ++d)
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
            for (long r = 0; r < N; ++r)
                f->F[((long)i * D + d) * N + r] += -f->rhom[(long)i * N + r] * RT * G[(long)d * N + r];
        /* grad rho_i for the forcing term, Eq. (1c) */
        orc_gradient_L(P, L, f->rho + (long)i * N, f->gradrho + (long)i * D * N);
    }
    /* barycentric velocity with the half-force shift */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
    for (long r = 0; r < N; ++r) {
        double rho_tot = 0.0;
        for (int i = 0; i < nc; ++i) rho_tot += f->rho[(long)i * N + r];
        for (int d = 0; d < D; ++d) {
            double j = 0.0;
            for (int i = 0; i < nc; ++i) {
                for (int a = 0; a < Q; ++a) j += L->e[a][d] * g[((long)i * Q + a) * N + r];
                j += 0.5 * f->F[((long)i * D + d) * N + r];
            }
            f->u[(long)d * N + r] = j / rho_tot;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* One or more time steps of Eq. (1a): collide every node, then stream  */
/* g_{a,i}(r + e_a, t+1) = g*_{a,i}(r, t) with periodic wrap.           */
/* g_in and g_out may alias.                                            */
/* ------------------------------------------------------------------ */
int orc_step(const orc_problem *P, const double *g_in, double *g_out, long long nsteps)
{
    orc_lattice L;
    orc_make_lattice(P->lattice, &L);
    const long N = (long)P->nx * P->ny * P->nz;
    const int nc = P->nc, Q = L.Q, D = L.D;
    const long tot = (long)nc * Q * N;
    double *g = malloc((size_t)tot * sizeof(double));
    double *gs = malloc((size_t)tot * sizeof(double));
    orc_fields f;
    if (!g || !gs || orc_fields_alloc(P, D, &f) != 0) {
        free(g);
        free(gs);
        return -3;
    }
    memcpy(g, g_in, (size_t)tot * sizeof(double));
    int status = 0;
    for (long long s = 0; s < nsteps && status == 0; ++s) {
        status = orc_macroscopic(P, &L, g, &f);
        if (status) break;
        /* collision, Eq. (1a) right-hand side */
#pragma omp parallel for schedule(static) if (N >= ORC_PAR_MIN)
        for (long r = 0; r < N; ++r) {
            double u[3] = {0, 0, 0};
            for (int d = 0; d < D; ++d) u[d] = f.u[(long)d * N + r];
            for (int i = 0; i < nc; ++i) {
                double Fi[3] = {0, 0, 0}, gr[3] = {0, 0, 0};
                for (int d = 0; d < D; ++d) {
                    Fi[d] = f.F[((long)i * D + d) * N + r];
                    gr[d] = f.gradrho[((long)i * D + d) * N + r];
                }
                double geq[ORC_MAXQ], Fa[ORC_MAXQ];
                orc_feq_forcing_L(&L, f.rho[(long)i * N + r], u, Fi, gr, geq, Fa);
                for (int a = 0; a < Q; ++a) {
                    long k = ((long)i * Q + a) * N + r;
                    gs[k] = g[k] - (g[k] - geq[a]) / P->tau + (1.0 - 1.0 / (2.0 * P->tau)) * Fa[a];
                }
            }
        }
        /* streaming, Eq. (1a) left-hand side (a permutation: no two nodes write one place) */
#pragma omp parallel for collapse(2) schedule(static) if ((long)P->nx * P->ny * P->nz >= ORC_PAR_MIN)
        for (int z = 0; z < P->nz; ++z)
            for (int y = 0; y < P->ny; ++y)
                for (int x = 0; x < P->nx; ++x) {
                    long r = (long)x + (long)P->nx * ((long)y + (long)P->ny * z);
                    for (int a = 0; a < Q; ++a) {
                        long rn = orc_neighbor(P, x, y, z, L.e[a]);
                        for (int i = 0; i < nc; ++i)
                            g[((long)i * Q + a) * N + rn] = gs[((long)i * Q + a) * N + r];
                    }
                }
    }
    if (status == 0) memcpy(g_out, g, (size_t)tot * sizeof(double));
    orc_fields_free(&f);
    free(g);
    free(gs);
    return status;
}

/* Macroscopic outputs of a state; any output pointer may be NULL. */
int orc_moments(const orc_problem *P, const double *g, double *rho, double *u, double *p,
                double *lnf, double *F)
{
    orc_lattice L;
    orc_make_lattice(P->lattice, &L);
    const long N = (long)P->nx * P->ny * P->nz;
    const int nc = P->nc, D = L.D;
    orc_fields f;
    if (orc_fields_alloc(P, D, &f) != 0) return -3;
    int status = orc_macroscopic(P, &L, g, &f);
    if (status == 0) {
        if (rho) memcpy(rho, f.rho, (size_t)nc * N * sizeof(double));
        if (u) memcpy(u, f.u, (size_t)D * N * sizeof(double));
        if (p) memcpy(p, f.p, (size_t)N * sizeof(double));
        if (lnf) memcpy(lnf, f.lnf, (size_t)nc * N * sizeof(double));
        if (F) memcpy(F, f.F, (size_t)nc * D * N * sizeof(double));
    }
    orc_fields_free(&f);
    return status;
}

/* ------------------------------------------------------------------ */
/* Initial populations (the paper gives densities only; the reading is  */
/* the equilibrium of Eq. (1b) at the given densities and velocity,     */
/* which for u = 0 is g_0 = rho_i and g_{a != 0} = 0).                  */
/* ------------------------------------------------------------------ */
int orc_init_equilibrium(const orc_problem *P, const double *rho, const double *u, double *g)
{
    orc_lattice L;
    orc_make_lattice(P->lattice, &L);
    const long N = (long)P->nx * P->ny * P->nz;
    const int Q = L.Q, D = L.D;
    for (int i = 0; i < P->nc; ++i)
        for (long r = 0; r < N; ++r) {
            double uu[3] = {0, 0, 0}, zero[3] = {0, 0, 0};
            if (u)
                for (int d = 0; d < D; ++d) uu[d] = u[(long)d * N + r];
            double geq[ORC_MAXQ], Fa[ORC_MAXQ];
            orc_feq_forcing_L(&L, rho[(long)i * N + r], uu, zero, zero, geq, Fa);
            for (int a = 0; a < Q; ++a) g[((long)i * Q + a) * N + r] = geq[a];
        }
    return 0;
}

/* Threads of the OpenMP loops (n < 1: all the runtime offers); returns the
 * count in use, 1 without OpenMP. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n < 1 ? omp_get_num_procs() : n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Per-component total mass sum_r rho_i(r). */
int orc_mass(const orc_problem *P, const double *g, double *mass)
{
    orc_lattice L;
    orc_make_lattice(P->lattice, &L);
    const long N = (long)P->nx * P->ny * P->nz;
    for (int i = 0; i < P->nc; ++i) {
        double s = 0.0;
        for (int a = 0; a < L.Q; ++a)
            for (long r = 0; r < N; ++r) s += g[((long)i * L.Q + a) * N + r];
        mass[i] = s;
    }
    return 0;
}

/* Lattice tables for tests (velocities as doubles, weights). */
int orc_lattice_info(int lattice, int *D, int *Q, int *e /*[Q][3]*/, double *w)
{
    orc_lattice L;
    orc_make_lattice(lattice, &L);
    *D = L.D;
    *Q = L.Q;
    for (int a = 0; a < L.Q; ++a) {
        for (int d = 0; d < 3; ++d) e[a * 3 + d] = L.e[a][d];
        w[a] = L.w[a];
    }
    return 0;
}
