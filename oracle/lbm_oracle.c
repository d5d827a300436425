/*
 * lbm_oracle.c -- plain, slow FP64 CPU oracle of one time step of the coupled
 * three-lattice central-moment lattice Boltzmann method of arXiv 2210.07501
 * (Sec. 4.1 phase field, Sec. 4.2 two-fluid flow, Sec. 4.3 energy, App. B maps).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load this file.  It shares no code, header, table or constant
 * with the CUDA library: every table below is built here from its definition.
 *
 * Plainness over speed: the central moments are formed with dense 9x9 matrices
 * P (raw moments) and F(u) (binomial shift), the post-collision populations with
 * F(-u) and a numerically inverted P, exactly in the order of the paper's
 * algorithm lists (Sec. 4.1-4.3).  No blocking, fusion or reordering.
 *
 * Readings of the paper that this file fixes (each one is also shared by the
 * CUDA path, which is written independently):
 *   - D2Q9 velocity 8 is (+1,-1) (the printed e_x list has a typo; App. B's P
 *     matrix has +1).
 *   - Raw basis ordering 00,10,01,20,02,11,21,12,22 of the P matrix (App. B);
 *     the flow lattice forms the trace/deviator pair 2s/2d only inside the
 *     relaxation (Sec. 4.2).
 *   - F(u) is the binomial expansion the text states; the printed kappa_22 row
 *     lacks the factor 2 on the 10 and 01 columns, the expansion has it.
 *   - theta = 4 phi (1 - phi) / W with phi_A = 0 (bottom), phi_B = 1 (top), so
 *     that the equilibrium of the conservative Allen-Cahn equation is the tanh
 *     profile of width W (Sec. 3).
 *   - Properties are linear in phi and equal the phase values at phi_A, phi_B.
 *   - The CSF force uses the printed components times delta_s' factor 1.5 W.
 *   - Isotropic finite differences: d_i psi = (1/c^2) sum_a w_a e_ai psi(x+e_a)
 *     with the D2Q9 weights, for grad(phi), div(n), grad(sigma) and grad(p).
 *   - n = 0 where |grad phi|^2 <= 1e-24.
 *   - The pressure force uses the pressure stored by the previous step
 *     (F_p = -grad(p^{n-1} - rho^n c^2)), the only explicit reading of Sec. 4.2.
 *   - Walls at y = 0 and y = ny (halfway), nodes at y_j = j + 1/2, periodic x:
 *     g bounce-back, f specular reflection (free slip, no flux), h anti-bounce-
 *     back to the wall temperature at the crossing point of the link.  Ghost
 *     rows for the stencils: phi and p mirrored, T = 2 T_w - T_adjacent.
 *   - The pressure lattice is carried as the deviation g - w p0 (p0 = rho_A c^2),
 *     an exact affine change of variables; p is carried as p - p0.  The velocity
 *     is 1e-5 of p, so without it round-off alone would exceed the 1e-12 parity
 *     bar.  Its equilibrium central moments are the printed ones minus the
 *     central moments of w p0 (same algebra, no cancellation).
 *   - D2Q5 (not in the paper) for phi and T: velocities 0..4 of D2Q9, weights
 *     1/3, 1/6, c^2 = 1/3, basis 1, e_x, e_y, e_x^2, e_y^2, the same equilibria
 *     truncated to those moments.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define QMAX 9
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int32_t nx, ny;          /* nodes; walls at y = 0 and y = ny, periodic in x */
    int32_t heat_periods;    /* cosine periods of the bottom-wall heating along x */
    int32_t q_phi, q_T;      /* 5 or 9 */
    int32_t pad_;
    double b;                /* bottom-layer thickness: interface at y = b */
    double W;                /* interface width */
    double sigma0, sigma1, sigma2;   /* sigma(T) = s0 + s1 (T-Tref) + s2 (T-Tref)^2 */
    double T_ref, T_hot, T_cold, dT; /* bottom wall T_hot + dT cos(..), top T_cold */
    double tau_flow;         /* bottom fluid: nu_A = (tau - 1/2)/3 */
    double visc_ratio;       /* mu_B / mu_A (top over bottom) */
    double tau_T;            /* bottom fluid: alpha_A = (tau_T - 1/2)/3 */
    double cond_ratio;       /* k_B / k_A */
    double tau_phi;          /* mobility M = (tau_phi - 1/2)/3 */
    double rho_bottom, rho_top;
    double Fx_ext, Fy_ext;   /* uniform external body force */
} or_params;

/* ---- lattice (Sec. 4.1): D2Q9 velocities, the first five form the D2Q5 ---- */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int MX[9] = {0, 1, 0, 2, 0, 1, 2, 1, 2};
static const int MY[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};
static const double CS2 = 1.0 / 3.0;

static double weight(int Q, int a)
{
    if (Q == 9) return a == 0 ? 4.0 / 9.0 : (a < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    return a == 0 ? 1.0 / 3.0 : 1.0 / 6.0;
}

static int find_dir(int Q, int ex, int ey)
{
    for (int a = 0; a < Q; ++a)
        if (EX[a] == ex && EY[a] == ey) return a;
    return -1;
}

static double ipow(double x, int k)
{
    double r = 1.0;
    for (int i = 0; i < k; ++i) r *= x;
    return r;
}

static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

/* App. B: P maps populations to raw moments, P[k][a] = e_ax^m e_ay^n. */
static void build_P(int Q, double P[QMAX][QMAX])
{
    for (int k = 0; k < Q; ++k)
        for (int a = 0; a < Q; ++a)
            P[k][a] = ipow((double)EX[a], MX[k]) * ipow((double)EY[a], MY[k]);
}

/* App. B: F(u) maps raw to central moments by the binomial expansion of
 * (e_x - u_x)^m (e_y - u_y)^n; F(u)^{-1} = F(-u). */
static void build_F(int Q, double ux, double uy, double F[QMAX][QMAX])
{
    for (int k = 0; k < Q; ++k)
        for (int l = 0; l < Q; ++l) {
            int m = MX[k], n = MY[k], p = MX[l], q = MY[l];
            if (p <= m && q <= n)
                F[k][l] = binom(m, p) * binom(n, q) * ipow(-ux, m - p) * ipow(-uy, n - q);
            else
                F[k][l] = 0.0;
        }
}

/* Gauss-Jordan inverse with partial pivoting (a library-style primitive). */
static int invert(int Q, const double A_in[QMAX][QMAX], double Ainv[QMAX][QMAX])
{
    double A[QMAX][QMAX];
    memcpy(A, A_in, sizeof(A));
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) Ainv[i][j] = (i == j) ? 1.0 : 0.0;
    for (int c = 0; c < Q; ++c) {
        int piv = c;
        for (int r = c + 1; r < Q; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (fabs(A[piv][c]) < 1e-300) return -1;
        if (piv != c)
            for (int j = 0; j < Q; ++j) {
                double t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t;
                t = Ainv[c][j]; Ainv[c][j] = Ainv[piv][j]; Ainv[piv][j] = t;
            }
        double d = A[c][c];
        for (int j = 0; j < Q; ++j) { A[c][j] /= d; Ainv[c][j] /= d; }
        for (int r = 0; r < Q; ++r)
            if (r != c) {
                double s = A[r][c];
                if (s != 0.0)
                    for (int j = 0; j < Q; ++j) { A[r][j] -= s * A[c][j]; Ainv[r][j] -= s * Ainv[c][j]; }
            }
    }
    return 0;
}

static void matvec(int Q, const double M[QMAX][QMAX], const double *x, double *y)
{
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int j = 0; j < Q; ++j) s += M[i][j] * x[j];
        y[i] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* Site-level collisions.  Each takes pre-collision populations and returns   */
/* post-collision populations: P, F(u), relax, F(-u), P^{-1}.                */
/* ------------------------------------------------------------------------ */

typedef struct {
    int Q;
    double P[QMAX][QMAX], Pinv[QMAX][QMAX];
} basis_t;

static int basis_init(basis_t *B, int Q)
{
    B->Q = Q;
    build_P(Q, B->P);
    return invert(Q, B->P, B->Pinv);
}

static void to_central(const basis_t *B, double ux, double uy, const double *pop, double *cm)
{
    double raw[QMAX], F[QMAX][QMAX];
    matvec(B->Q, B->P, pop, raw);          /* kappa' = P f        */
    build_F(B->Q, ux, uy, F);
    matvec(B->Q, F, raw, cm);              /* kappa  = F kappa'   */
}

static void from_central(const basis_t *B, double ux, double uy, const double *cm, double *pop)
{
    double raw[QMAX], Finv[QMAX][QMAX];
    build_F(B->Q, -ux, -uy, Finv);
    matvec(B->Q, Finv, cm, raw);           /* kappa~' = F^{-1} kappa~ */
    matvec(B->Q, B->Pinv, raw, pop);       /* f~ = P^{-1} kappa~'     */
}

/* Sec. 4.1: conservative Allen-Cahn lattice.  Equilibria (phi, M theta n_x,
 * M theta n_y, c^2 phi, c^2 phi, 0, 0, 0, c^4 phi); first moments relax at
 * omega_phi, every other moment at 1. */
static void collide_phase(const basis_t *B, double *pop, double phi, double ux, double uy,
                          double Mtnx, double Mtny, double omega_phi)
{
    double k[QMAX], eq[QMAX] = {phi, Mtnx, Mtny, CS2 * phi, CS2 * phi, 0.0, 0.0, 0.0, CS2 * CS2 * phi};
    to_central(B, ux, uy, pop, k);
    for (int m = 0; m < B->Q; ++m) {
        double w = (m == 1 || m == 2) ? omega_phi : 1.0;
        k[m] = k[m] + w * (eq[m] - k[m]);
    }
    from_central(B, ux, uy, k, pop);
}

/* Sec. 4.3: energy lattice.  Equilibria (T, 0, 0, c^2 T, c^2 T, 0, 0, 0, c^4 T);
 * first moments relax at omega_T, every other moment at 1. */
static void collide_energy(const basis_t *B, double *pop, double T, double ux, double uy, double omega_T)
{
    double k[QMAX], eq[QMAX] = {T, 0.0, 0.0, CS2 * T, CS2 * T, 0.0, 0.0, 0.0, CS2 * CS2 * T};
    to_central(B, ux, uy, pop, k);
    for (int m = 0; m < B->Q; ++m) {
        double w = (m == 1 || m == 2) ? omega_T : 1.0;
        k[m] = k[m] + w * (eq[m] - k[m]);
    }
    from_central(B, ux, uy, k, pop);
}

/* Sec. 4.2 equilibrium central moments of g, minus the central moments of the
 * reference w_a p0 at the same velocity.  The printed equilibrium is
 *   eta^eq = rho c^2 (1,0,0,c^2,c^2,0,0,0,c^4) + phi_p Wc(u),
 *   Wc(u)  = (1, -ux, -uy, c^2+ux^2, c^2+uy^2, ux uy, -(c^2+ux^2) uy,
 *             -(c^2+uy^2) ux, (c^2+ux^2)(c^2+uy^2)),   phi_p = p - rho c^2,
 * and the reference contributes p0 Wc(u); with p = p0 + dp the difference is
 *   dp Wc(u) + rho c^2 [ (1,0,0,c^2,c^2,0,0,0,c^4) - Wc(u) ]. */
static void flow_equilibrium_dev(double rho, double dp, double ux, double uy, double *eq)
{
    double c2 = CS2, ax = c2 + ux * ux, ay = c2 + uy * uy;
    double Wc[9] = {1.0, -ux, -uy, ax, ay, ux * uy, -ax * uy, -ay * ux, ax * ay};
    double D[9] = {0.0, ux, uy, -ux * ux, -uy * uy, -ux * uy, ax * uy, ay * ux,
                   -(c2 * (ux * ux + uy * uy) + ux * ux * uy * uy)};
    for (int m = 0; m < 9; ++m) eq[m] = dp * Wc[m] + rho * c2 * D[m];
}

/* Sec. 4.2 central moments of the source, with Gamma = F_p . u. */
static void flow_source(double ux, double uy, double Fpx, double Fpy, double Ftx, double Fty, double *s)
{
    double c2 = CS2, G = Fpx * ux + Fpy * uy;
    s[0] = G;
    s[1] = c2 * Ftx - ux * G;
    s[2] = c2 * Fty - uy * G;
    s[3] = 2.0 * c2 * Fpx * ux + (ux * ux + c2) * G;
    s[4] = 2.0 * c2 * Fpy * uy + (uy * uy + c2) * G;
    s[5] = c2 * (Fpx * uy + Fpy * ux) + ux * uy * G;
    s[6] = 0.0;
    s[7] = 0.0;
    s[8] = 0.0;
}

/* Sec. 4.2 two-fluid collision on the deviation populations g - w p0.
 * eta~ = eta + w (eta^eq - eta) + (1 - w/2) sigma, with the second-order pair
 * combined to 2s = 20 + 02 (rate 1) and 2d = 20 - 02 (rate omega_nu), 11 at
 * omega_nu, all other rates 1, then split back. */
static void collide_flow(const basis_t *B, double *pop, double rho, double dp, double ux, double uy,
                         double Fpx, double Fpy, double Ftx, double Fty, double omega_nu)
{
    double e[QMAX], eq[QMAX], s[QMAX], out[QMAX];
    to_central(B, ux, uy, pop, e);
    flow_equilibrium_dev(rho, dp, ux, uy, eq);
    flow_source(ux, uy, Fpx, Fpy, Ftx, Fty, s);
    for (int m = 0; m < 9; ++m) {
        if (m == 3 || m == 4) continue;
        double w = (m == 5) ? omega_nu : 1.0;
        out[m] = e[m] + w * (eq[m] - e[m]) + (1.0 - 0.5 * w) * s[m];
    }
    double e2s = e[3] + e[4], e2d = e[3] - e[4];
    double q2s = eq[3] + eq[4], q2d = eq[3] - eq[4];
    double s2s = s[3] + s[4], s2d = s[3] - s[4];
    double w2s = 1.0, w2d = omega_nu;
    double t2s = e2s + w2s * (q2s - e2s) + (1.0 - 0.5 * w2s) * s2s;
    double t2d = e2d + w2d * (q2d - e2d) + (1.0 - 0.5 * w2d) * s2d;
    out[3] = 0.5 * (t2s + t2d);
    out[4] = 0.5 * (t2s - t2d);
    from_central(B, ux, uy, out, pop);
}

/* ------------------------------------------------------------------------ */
/* Whole-lattice state                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    or_params p;
    int nx, ny, Qf, Qh;
    basis_t B9, Bf, Bh;
    double *f, *g, *h;          /* post-collision state (f, g - w p0, h) [Q][ny][nx] */
    double *fpre, *gpre, *hpre; /* streamed, pre-collision               */
    double *dp_prev;            /* p^{n-1} - p0                           */
    double *phi, *ux, *uy, *T, *dp;   /* macros of the last step [ny][nx] */
    /* stencil work arrays on rows -2 .. ny+1 (extended) */
    double *phix, *nxs, *nys, *sig, *psi;
    double *gx, *gy, *fpx, *fpy, *ftx, *fty;   /* grad phi, F_p, F_t on [ny][nx] */
    double *dsx, *dsy;                         /* grad sigma on [ny][nx] */
    double p0, muA, muB, kA, kB, omega_phi, Mphi;
    long step;
} oracle_t;

#define IDX(q, j, i) (((size_t)(q) * (size_t)o->ny + (size_t)(j)) * (size_t)o->nx + (size_t)(i))
#define FLD(j, i) ((size_t)(j) * (size_t)o->nx + (size_t)(i))
/* extended rows: ext row r holds lattice row r - 2 */
#define EXT(j, i) ((size_t)((j) + 2) * (size_t)o->nx + (size_t)(i))

static int wrapx(const oracle_t *o, int i) { return ((i % o->nx) + o->nx) % o->nx; }

static double T_bottom(const oracle_t *o, double x)
{
    return o->p.T_hot + o->p.dT * cos(2.0 * M_PI * (double)o->p.heat_periods * x / (double)o->nx);
}

static double rho_of(const oracle_t *o, double phi) { return o->p.rho_bottom + phi * (o->p.rho_top - o->p.rho_bottom); }
static double mu_of(const oracle_t *o, double phi) { return o->muA + phi * (o->muB - o->muA); }
static double k_of(const oracle_t *o, double phi) { return o->kA + phi * (o->kB - o->kA); }
static double sigma_of(const oracle_t *o, double T)
{
    double d = T - o->p.T_ref;
    return o->p.sigma0 + o->p.sigma1 * d + o->p.sigma2 * d * d;
}

static double dsigma_of(const oracle_t *o, double T)   /* sigma(T) - sigma0 */
{
    double d = T - o->p.T_ref;
    return o->p.sigma1 * d + o->p.sigma2 * d * d;
}

void or_destroy(void *handle);

void *or_create(const or_params *prm)
{
    if (!prm || prm->nx < 3 || prm->ny < 3) return NULL;
    if ((prm->q_phi != 5 && prm->q_phi != 9) || (prm->q_T != 5 && prm->q_T != 9)) return NULL;
    if (!(prm->W > 0.0) || !(prm->tau_flow > 0.5) || !(prm->tau_T > 0.5) || !(prm->tau_phi > 0.5)) return NULL;
    oracle_t *o = (oracle_t *)calloc(1, sizeof(oracle_t));
    if (!o) return NULL;
    o->p = *prm;
    o->nx = prm->nx;
    o->ny = prm->ny;
    o->Qf = prm->q_phi;
    o->Qh = prm->q_T;
    if (basis_init(&o->B9, 9) || basis_init(&o->Bf, o->Qf) || basis_init(&o->Bh, o->Qh)) { free(o); return NULL; }
    size_t N = (size_t)o->nx * o->ny, NE = (size_t)o->nx * (o->ny + 4);
    o->f = calloc((size_t)o->Qf * N, sizeof(double));
    o->g = calloc(9 * N, sizeof(double));
    o->h = calloc((size_t)o->Qh * N, sizeof(double));
    o->fpre = calloc((size_t)o->Qf * N, sizeof(double));
    o->gpre = calloc(9 * N, sizeof(double));
    o->hpre = calloc((size_t)o->Qh * N, sizeof(double));
    o->dp_prev = calloc(N, sizeof(double));
    o->phi = calloc(N, sizeof(double));
    o->ux = calloc(N, sizeof(double));
    o->uy = calloc(N, sizeof(double));
    o->T = calloc(N, sizeof(double));
    o->dp = calloc(N, sizeof(double));
    o->phix = calloc(NE, sizeof(double));
    o->nxs = calloc(NE, sizeof(double));
    o->nys = calloc(NE, sizeof(double));
    o->sig = calloc(NE, sizeof(double));
    o->psi = calloc(NE, sizeof(double));
    o->gx = calloc(N, sizeof(double));
    o->gy = calloc(N, sizeof(double));
    o->fpx = calloc(N, sizeof(double));
    o->fpy = calloc(N, sizeof(double));
    o->ftx = calloc(N, sizeof(double));
    o->fty = calloc(N, sizeof(double));
    o->dsx = calloc(N, sizeof(double));
    o->dsy = calloc(N, sizeof(double));
    if (!o->f || !o->g || !o->h || !o->fpre || !o->gpre || !o->hpre || !o->dp_prev || !o->phi || !o->ux ||
        !o->uy || !o->T || !o->dp || !o->phix || !o->nxs || !o->nys || !o->sig || !o->psi || !o->gx ||
        !o->gy || !o->fpx || !o->fpy || !o->ftx || !o->fty || !o->dsx || !o->dsy) {
        or_destroy(o);
        return NULL;
    }
    o->p0 = prm->rho_bottom * CS2;
    double nuA = (prm->tau_flow - 0.5) * CS2;
    o->muA = prm->rho_bottom * nuA;
    o->muB = prm->visc_ratio * o->muA;
    double alphaA = (prm->tau_T - 0.5) * CS2;
    o->kA = prm->rho_bottom * alphaA;         /* rho c_p with c_p = 1 */
    o->kB = prm->cond_ratio * o->kA;
    o->omega_phi = 1.0 / prm->tau_phi;
    o->Mphi = CS2 * (1.0 / o->omega_phi - 0.5);
    return o;
}

void or_destroy(void *handle)
{
    oracle_t *o = (oracle_t *)handle;
    if (!o) return;
    double *arrs[] = {o->f, o->g, o->h, o->fpre, o->gpre, o->hpre, o->dp_prev, o->phi, o->ux, o->uy, o->T,
                      o->dp, o->phix, o->nxs, o->nys, o->sig, o->psi, o->gx, o->gy, o->fpx, o->fpy,
                      o->ftx, o->fty, o->dsx, o->dsy};
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); ++k) free(arrs[k]);
    free(o);
}

int or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Extended phi field (rows -2..ny+1): mirror ghost rows (zero normal gradient). */
static void fill_phi_ext(oracle_t *o, const double *phi)
{
    for (int j = -2; j < o->ny + 2; ++j) {
        int js = j < 0 ? -1 - j : (j >= o->ny ? 2 * o->ny - 1 - j : j);
        for (int i = 0; i < o->nx; ++i) o->phix[EXT(j, i)] = phi[FLD(js, i)];
    }
}

/* grad(phi) and the unit normal on rows -1..ny from the extended phi. */
static void normals(oracle_t *o)
{
    #pragma omp parallel for schedule(static)
    for (int j = -1; j < o->ny + 1; ++j)
        for (int i = 0; i < o->nx; ++i) {
            double gx = 0.0, gy = 0.0;
            for (int a = 0; a < 9; ++a) {
                double v = o->phix[EXT(j + EY[a], wrapx(o, i + EX[a]))];
                gx += weight(9, a) * EX[a] * v;
                gy += weight(9, a) * EY[a] * v;
            }
            gx /= CS2;
            gy /= CS2;
            double g2 = gx * gx + gy * gy, nx = 0.0, ny = 0.0;
            if (g2 > 1e-24) { double m = sqrt(g2); nx = gx / m; ny = gy / m; }
            o->nxs[EXT(j, i)] = nx;
            o->nys[EXT(j, i)] = ny;
            if (j >= 0 && j < o->ny) { o->gx[FLD(j, i)] = gx; o->gy[FLD(j, i)] = gy; }
        }
}

/* Isotropic gradient of an extended field at node (j, i). */
static void iso_grad(const oracle_t *o, const double *fe, int j, int i, double *dx, double *dy)
{
    double sx = 0.0, sy = 0.0;
    for (int a = 0; a < 9; ++a) {
        double v = fe[EXT(j + EY[a], wrapx(o, i + EX[a]))];
        sx += weight(9, a) * EX[a] * v;
        sy += weight(9, a) * EY[a] * v;
    }
    *dx = sx / CS2;
    *dy = sy / CS2;
}

/* Equilibrium initial state from macroscopic fields (phi, u, v, T, p - p0).
 * Defaults: tanh interface of width W at y = b, rest, T = T_ref and uniform pressure
 * p = p0 (a fluid at rest without gravity has uniform pressure; p = rho c^2 would put a
 * jump of c^2 (rho_B - rho_A) across the interface). */
int or_init(void *handle, const double *phi_in, const double *u_in, const double *v_in, const double *T_in,
            const double *dp_in)
{
    oracle_t *o = (oracle_t *)handle;
    if (!o) return -1;
    int nx = o->nx, ny = o->ny;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = FLD(j, i);
            double y = j + 0.5;
            o->phi[c] = phi_in ? phi_in[c] : 0.5 + 0.5 * tanh(2.0 * (y - o->p.b) / o->p.W);
            o->ux[c] = u_in ? u_in[c] : 0.0;
            o->uy[c] = v_in ? v_in[c] : 0.0;
            o->T[c] = T_in ? T_in[c] : o->p.T_ref;
            o->dp[c] = dp_in ? dp_in[c] : 0.0;      /* at rest: uniform pressure p0 */
        }
    fill_phi_ext(o, o->phi);
    normals(o);
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = FLD(j, i);
            double ph = o->phi[c], ux = o->ux[c], uy = o->uy[c];
            double theta = 4.0 * ph * (1.0 - ph) / o->p.W;
            double kf[QMAX] = {ph, o->Mphi * theta * o->nxs[EXT(j, i)], o->Mphi * theta * o->nys[EXT(j, i)],
                               CS2 * ph, CS2 * ph, 0.0, 0.0, 0.0, CS2 * CS2 * ph};
            double pop[QMAX];
            from_central(&o->Bf, ux, uy, kf, pop);
            for (int a = 0; a < o->Qf; ++a) o->f[IDX(a, j, i)] = pop[a];
            double eq[QMAX];
            flow_equilibrium_dev(rho_of(o, ph), o->dp[c], ux, uy, eq);
            from_central(&o->B9, ux, uy, eq, pop);
            for (int a = 0; a < 9; ++a) o->g[IDX(a, j, i)] = pop[a];
            double T = o->T[c];
            double kh[QMAX] = {T, 0.0, 0.0, CS2 * T, CS2 * T, 0.0, 0.0, 0.0, CS2 * CS2 * T};
            from_central(&o->Bh, ux, uy, kh, pop);
            for (int a = 0; a < o->Qh; ++a) o->h[IDX(a, j, i)] = pop[a];
            o->dp_prev[c] = o->dp[c];
        }
    o->step = 0;
    return 0;
}

/* Pull streaming with the wall rules; walls sit halfway below row 0 and above row ny-1. */
static void stream(oracle_t *o)
{
    int nx = o->nx, ny = o->ny;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            for (int a = 0; a < 9; ++a) {
                int js = j - EY[a], is = wrapx(o, i - EX[a]);
                int in = (js >= 0 && js < ny);
                /* flow: halfway bounce-back */
                int ob = find_dir(9, -EX[a], -EY[a]);
                o->gpre[IDX(a, j, i)] = in ? o->g[IDX(a, js, is)] : o->g[IDX(ob, j, i)];
                /* phase field: specular reflection of the mirrored velocity */
                if (a < o->Qf) {
                    int am = find_dir(o->Qf, EX[a], -EY[a]);
                    o->fpre[IDX(a, j, i)] = in ? o->f[IDX(a, js, is)] : o->f[IDX(am, j, is)];
                }
                /* energy: anti-bounce-back to the wall temperature at the link's crossing */
                if (a < o->Qh) {
                    if (in) {
                        o->hpre[IDX(a, j, i)] = o->h[IDX(a, js, is)];
                    } else {
                        int oh = find_dir(o->Qh, -EX[a], -EY[a]);
                        double xc = (double)i - 0.5 * (double)EX[a];
                        double Tw = (js < 0) ? T_bottom(o, xc) : o->p.T_cold;
                        o->hpre[IDX(a, j, i)] = -o->h[IDX(oh, j, i)] + 2.0 * weight(o->Qh, a) * Tw;
                    }
                }
            }
        }
}

static void collide_all(oracle_t *o)
{
    int nx = o->nx, ny = o->ny;
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = FLD(j, i);
            double ph = o->phi[c], ux = o->ux[c], uy = o->uy[c], T = o->T[c];
            double rho = rho_of(o, ph);
            double nu = mu_of(o, ph) / rho;
            double omega_nu = 1.0 / (nu / CS2 + 0.5);
            double alpha = k_of(o, ph) / rho;          /* c_p = 1 */
            double omega_T = 1.0 / (alpha / CS2 + 0.5);
            double theta = 4.0 * ph * (1.0 - ph) / o->p.W;
            double pop[QMAX];
            for (int a = 0; a < o->Qf; ++a) pop[a] = o->fpre[IDX(a, j, i)];
            collide_phase(&o->Bf, pop, ph, ux, uy, o->Mphi * theta * o->nxs[EXT(j, i)],
                          o->Mphi * theta * o->nys[EXT(j, i)], o->omega_phi);
            for (int a = 0; a < o->Qf; ++a) o->f[IDX(a, j, i)] = pop[a];
            for (int a = 0; a < 9; ++a) pop[a] = o->gpre[IDX(a, j, i)];
            collide_flow(&o->B9, pop, rho, o->dp[c], ux, uy, o->fpx[c], o->fpy[c], o->ftx[c], o->fty[c],
                         omega_nu);
            for (int a = 0; a < 9; ++a) o->g[IDX(a, j, i)] = pop[a];
            for (int a = 0; a < o->Qh; ++a) pop[a] = o->hpre[IDX(a, j, i)];
            collide_energy(&o->Bh, pop, T, ux, uy, omega_T);
            for (int a = 0; a < o->Qh; ++a) o->h[IDX(a, j, i)] = pop[a];
            o->dp_prev[c] = o->dp[c];
        }
}

/* One time step in the order: stream, local moments, stencil fields, forces and
 * macros, collisions, store.  Macros kept afterwards are those of this step. */
static void step_once(oracle_t *o)
{
    int nx = o->nx, ny = o->ny;
    stream(o);
    /* phi = sum f, T = sum h (Sec. 4.1, 4.3) */
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            double s = 0.0, t = 0.0;
            for (int a = 0; a < o->Qf; ++a) s += o->fpre[IDX(a, j, i)];
            for (int a = 0; a < o->Qh; ++a) t += o->hpre[IDX(a, j, i)];
            o->phi[FLD(j, i)] = s;
            o->T[FLD(j, i)] = t;
        }
    /* stencil fields */
    fill_phi_ext(o, o->phi);
    normals(o);
    #pragma omp parallel for schedule(static)
    for (int j = -1; j < ny + 1; ++j)
        for (int i = 0; i < nx; ++i) {
            double T;
            if (j < 0) T = 2.0 * T_bottom(o, (double)i) - o->T[FLD(0, i)];
            else if (j >= ny) T = 2.0 * o->p.T_cold - o->T[FLD(ny - 1, i)];
            else T = o->T[FLD(j, i)];
            /* grad(sigma) = grad(sigma - sigma0): the constant is left out of the
             * differences, where it would only add round-off. */
            o->sig[EXT(j, i)] = dsigma_of(o, T);
            int js = j < 0 ? 0 : (j >= ny ? ny - 1 : j);
            double ph = o->phix[EXT(j, i)];
            o->psi[EXT(j, i)] = o->dp_prev[FLD(js, i)] - rho_of(o, ph) * CS2;
        }
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = FLD(j, i);
            /* curvature term: div(n) */
            double dv = 0.0;
            for (int a = 0; a < 9; ++a) {
                size_t e = EXT(j + EY[a], wrapx(o, i + EX[a]));
                dv += weight(9, a) * (EX[a] * o->nxs[e] + EY[a] * o->nys[e]);
            }
            dv /= CS2;
            double dsx, dsy, dpx, dpy;
            iso_grad(o, o->sig, j, i, &dsx, &dsy);
            iso_grad(o, o->psi, j, i, &dpx, &dpy);
            double nxv = o->nxs[EXT(j, i)], nyv = o->nys[EXT(j, i)];
            double g2 = o->gx[c] * o->gx[c] + o->gy[c] * o->gy[c];
            double sg = sigma_of(o, o->T[c]);
            double ds = 1.5 * o->p.W;      /* delta_s = 1.5 W |grad phi|^2 */
            double Fsx = ds * (-sg * g2 * dv * nxv + g2 * ((1.0 - nxv * nxv) * dsx - nxv * nyv * dsy));
            double Fsy = ds * (-sg * g2 * dv * nyv + g2 * ((1.0 - nyv * nyv) * dsy - nxv * nyv * dsx));
            double Ftx = Fsx + o->p.Fx_ext, Fty = Fsy + o->p.Fy_ext;
            double Fpx = -dpx, Fpy = -dpy;
            /* macros (Sec. 4.2): rho c^2 u = sum g e + c^2 F_t / 2;  p = sum g + F_p.u / 2 */
            double s0 = 0.0, sx = 0.0, sy = 0.0;
            for (int a = 0; a < 9; ++a) {
                double v = o->gpre[IDX(a, j, i)];
                s0 += v;
                sx += v * EX[a];
                sy += v * EY[a];
            }
            double rho = rho_of(o, o->phi[c]);
            double ux = (sx + 0.5 * CS2 * Ftx) / (rho * CS2);
            double uy = (sy + 0.5 * CS2 * Fty) / (rho * CS2);
            o->ux[c] = ux;
            o->uy[c] = uy;
            o->dp[c] = s0 + 0.5 * (Fpx * ux + Fpy * uy);
            o->fpx[c] = Fpx;
            o->fpy[c] = Fpy;
            o->ftx[c] = Ftx;
            o->fty[c] = Fty;
            o->dsx[c] = dsx;
            o->dsy[c] = dsy;
        }
    collide_all(o);
    o->step += 1;
}

int or_step(void *handle, long nsteps)
{
    oracle_t *o = (oracle_t *)handle;
    if (!o || nsteps < 0) return -1;
    for (long s = 0; s < nsteps; ++s) step_once(o);
    return 0;
}

/* Macros (phi, u, v, T, p - p0) at the current time level. */
void or_fields(void *handle, double *phi, double *u, double *v, double *T, double *dp)
{
    oracle_t *o = (oracle_t *)handle;
    size_t N = (size_t)o->nx * o->ny;
    if (phi) memcpy(phi, o->phi, N * sizeof(double));
    if (u) memcpy(u, o->ux, N * sizeof(double));
    if (v) memcpy(v, o->uy, N * sizeof(double));
    if (T) memcpy(T, o->T, N * sizeof(double));
    if (dp) memcpy(dp, o->dp, N * sizeof(double));
}

/* Post-collision state: f [Qf][ny][nx], g - w p0 [9][ny][nx], h - w T_ref [Qh][ny][nx], p - p0 [ny][nx]. */
void or_get_state(void *handle, double *f, double *g, double *h, double *dp)
{
    oracle_t *o = (oracle_t *)handle;
    size_t N = (size_t)o->nx * o->ny;
    memcpy(f, o->f, (size_t)o->Qf * N * sizeof(double));
    memcpy(g, o->g, 9 * N * sizeof(double));
    for (int a = 0; a < o->Qh; ++a)
        for (size_t c = 0; c < N; ++c) h[a * N + c] = o->h[a * N + c] - weight(o->Qh, a) * o->p.T_ref;
    memcpy(dp, o->dp_prev, N * sizeof(double));
}

void or_set_state(void *handle, const double *f, const double *g, const double *h, const double *dp)
{
    oracle_t *o = (oracle_t *)handle;
    size_t N = (size_t)o->nx * o->ny;
    memcpy(o->f, f, (size_t)o->Qf * N * sizeof(double));
    memcpy(o->g, g, 9 * N * sizeof(double));
    for (int a = 0; a < o->Qh; ++a)
        for (size_t c = 0; c < N; ++c) o->h[a * N + c] = h[a * N + c] + weight(o->Qh, a) * o->p.T_ref;
    memcpy(o->dp_prev, dp, N * sizeof(double));
}

long or_step_count(void *handle) { return ((oracle_t *)handle)->step; }

/* Sum of phi over the lattice: phi = sum_a f_a of the current post-collision state. */
double or_mass(void *handle)
{
    oracle_t *o = (oracle_t *)handle;
    double s = 0.0;
    for (int j = 0; j < o->ny; ++j)
        for (int i = 0; i < o->nx; ++i)
            for (int a = 0; a < o->Qf; ++a) s += o->f[IDX(a, j, i)];
    return s;
}

/* ---- site-level entry points for the pins ---- */

/* Dense P, P^{-1}, F(u), F(-u) for Q = 5 or 9, row-major Q x Q. */
int or_matrices(int Q, double ux, double uy, double *P, double *Pinv, double *F, double *Finv)
{
    if (Q != 5 && Q != 9) return -1;
    basis_t B;
    if (basis_init(&B, Q)) return -1;
    double Fm[QMAX][QMAX], Fi[QMAX][QMAX];
    build_F(Q, ux, uy, Fm);
    build_F(Q, -ux, -uy, Fi);
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) {
            P[i * Q + j] = B.P[i][j];
            Pinv[i * Q + j] = B.Pinv[i][j];
            F[i * Q + j] = Fm[i][j];
            Finv[i * Q + j] = Fi[i][j];
        }
    return 0;
}

int or_collide_phase_site(int Q, double *pop, double phi, double ux, double uy, double Mtnx, double Mtny,
                          double omega_phi)
{
    basis_t B;
    if ((Q != 5 && Q != 9) || basis_init(&B, Q)) return -1;
    collide_phase(&B, pop, phi, ux, uy, Mtnx, Mtny, omega_phi);
    return 0;
}

int or_collide_energy_site(int Q, double *pop, double T, double ux, double uy, double omega_T)
{
    basis_t B;
    if ((Q != 5 && Q != 9) || basis_init(&B, Q)) return -1;
    collide_energy(&B, pop, T, ux, uy, omega_T);
    return 0;
}

int or_collide_flow_site(double *pop, double rho, double dp, double ux, double uy, double Fpx, double Fpy,
                         double Ftx, double Fty, double omega_nu)
{
    basis_t B;
    if (basis_init(&B, 9)) return -1;
    collide_flow(&B, pop, rho, dp, ux, uy, Fpx, Fpy, Ftx, Fty, omega_nu);
    return 0;
}

int or_sizeof_params(void) { return (int)sizeof(or_params); }

/* Stencil fields of the last step: grad sigma, F_t and F_p, each [ny][nx]. */
void or_debug_fields(void *handle, double *dsx, double *dsy, double *ftx, double *fty, double *fpx, double *fpy)
{
    oracle_t *o = (oracle_t *)handle;
    size_t N = (size_t)o->nx * o->ny;
    memcpy(dsx, o->dsx, N * sizeof(double));
    memcpy(dsy, o->dsy, N * sizeof(double));
    memcpy(ftx, o->ftx, N * sizeof(double));
    memcpy(fty, o->fty, N * sizeof(double));
    memcpy(fpx, o->fpx, N * sizeof(double));
    memcpy(fpy, o->fpy, N * sizeof(double));
}

/* Streaming alone, applied to the current post-collision state (which is left
 * unchanged): pre-collision f, g - w p0 and h - w T_ref, each [Q][ny][nx]. */
void or_streamed(void *handle, double *f, double *g, double *h)
{
    oracle_t *o = (oracle_t *)handle;
    size_t N = (size_t)o->nx * o->ny;
    stream(o);
    memcpy(f, o->fpre, (size_t)o->Qf * N * sizeof(double));
    memcpy(g, o->gpre, 9 * N * sizeof(double));
    for (int a = 0; a < o->Qh; ++a)
        for (size_t c = 0; c < N; ++c) h[a * N + c] = o->hpre[a * N + c] - weight(o->Qh, a) * o->p.T_ref;
}
