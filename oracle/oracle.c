/*
 * FP64 CPU oracle for the Bingham lattice Boltzmann step (PR and IR models).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference leg of bench.py use it.  It shares no code, header, table or
 * helper with the CUDA path.
 *
 * What it computes, step by step, in the order and notation of
 * Regulski, Leonardi & Szumbarski, "On the spatial convergence and transient
 * behaviour of lattice Boltzmann methods for modelling fluids with yield stress"
 * (arXiv:1610.01388):
 *
 *   - lattices D2Q9, D3Q15, D3Q19, D3Q27 with c_s^2 = 1/3 (Sec. 2, Sec. 4.1;
 *     the weights are the textbook ones, the paper does not print them);
 *   - streaming, eq. (8), in pull form with halfway bounce-back on cells
 *     flagged solid (Sec. 4.3, Sec. 4.5) and periodic wrap elsewhere;
 *   - moments, eq. (MomentsLBM); equilibrium, eq. (f_eq);
 *   - PR: strain rate from the non-equilibrium second moment with the
 *     previous step's tau, eq. (LBM_strain_rate); Papanastasiou apparent
 *     viscosity, eq. (Pap_reg_1), with the linear cut-off of eq.
 *     (PR_interpolation); tau from eq. (tau_visc); TRT with magic number
 *     Lambda (Sec. 2.1); exact difference method forcing, eq. (14);
 *   - IR: T = sum c c (f - f_eq), the closed-form Bingham solution of
 *     eq. (Vikh_main_short) given by eqs. (Vikh_sigmaS_formula) and
 *     (Vikh_sigmaS_tensor); post-collision populations eq. (Vikh_postCol)
 *     with f^sigma of eq. (Vikh_f_stress) and the force term of eq.
 *     (Vikh_force).
 *
 * Where the printed paper is garbled or silent, the reading taken is:
 *   R1  eq. (PR_interpolation): the first denominator is gdot_C (a linear
 *       interpolation between nu_0 at gdot = 0 and nu_app(gdot_C));
 *   R2  (1 - exp(-m gdot)) is evaluated as -expm1(-m gdot);
 *   R3  IR yield test: |T| >= sqrt(2) sigma_y (the value at which
 *       eq. (Vikh_sigmaS_formula)'s s vanishes, so both branches agree there);
 *   R4  eq. (Vikh_f_stress): f^sigma_i = w_i/(2 c_s^4) (c_i c_i - c_s^2 I):A,
 *       A = -sigma_bar + s/2, whose second moment is exactly A;
 *   R5  deviatoric part sigma_bar = sigma - (tr sigma / d) I, d = 2 or 3;
 *   R6  eq. (Vikh_force): Phi_i = w_i (c_i . F) / c_s^2 with F = rho g;
 *       "f_eq half a step back" is f_eq(rho, u) - Phi_i / 2 with
 *       u = (j + F/2) / rho;
 *   R7  eq. (LBM_strain_rate) as printed (no rho);
 *   R8  PR collision uses the tau computed in this step from the previous
 *       step's tau (explicit update of Sec. 3);
 *   R9  macroscopic fields are the moments of the streamed (pre-collision)
 *       populations, u_real = (j + F/2) / rho for both models (Sec. 2.4);
 *   R10 implicit PR (Sec. 3 names Newton iterations, no more): the unknown is
 *       the strain rate gdot; a fixed number of iterations starts from the
 *       explicit estimate; each iterate is clamped at gdot >= 0 and the
 *       derivative of H is floored at 1/2 (the constant part of tau), which
 *       only matters where the cut-off interpolation makes H non-monotone.
 *
 * Populations are full f (not offsets), layout f[i * N + cell],
 * cell = x + nx * (y + ny * z), in this file's own velocity order
 * (lexicographic over (c_z, c_y, c_x)).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXQ 27

enum { ORC_D2Q9 = 0, ORC_D3Q15 = 1, ORC_D3Q19 = 2, ORC_D3Q27 = 3 };
enum { ORC_PR = 0, ORC_IR = 1 };

typedef struct {
    int model;        /* ORC_PR or ORC_IR */
    double nu_p;      /* plastic kinematic viscosity, mu_p / rho_0 with rho_0 = 1 */
    double sigma_y;   /* yield stress */
    double m;         /* Papanastasiou regularisation parameter (PR) */
    double gdot_c;    /* PR zero-strain cut-off gdot^C */
    double g[3];      /* body acceleration; force density F = rho g */
    double magic;     /* TRT magic number Lambda (PR) */
    int burnett_x;    /* 1: Burnett-suppressed variant for flow along x (Secs. 4.2.1,
                         4.2.2): d_xx = 0 in the PR strain rate, T_xx = 0 in IR */
    int newton;       /* PR: Newton iterations making tau consistent with the strain
                         rate it implies (implicit update of Sec. 3); 0 = explicit */
} orc_params;

typedef struct {
    int Q, D;
    int c[ORC_MAXQ][3];
    double w[ORC_MAXQ];
} orc_lattice;

static const double CS2 = 1.0 / 3.0; /* c_s^2, Sec. 2 */

/* Velocity sets in lexicographic order of (c_z, c_y, c_x). */
static const orc_lattice LAT_D2Q9 = {
    9, 2,
    {{-1,-1,0}, {0,-1,0}, {1,-1,0}, {-1,0,0}, {0,0,0}, {1,0,0}, {-1,1,0}, {0,1,0}, {1,1,0}},
    {1.0/36.0, 1.0/9.0, 1.0/36.0, 1.0/9.0, 4.0/9.0, 1.0/9.0, 1.0/36.0, 1.0/9.0, 1.0/36.0}};

static const orc_lattice LAT_D3Q15 = {
    15, 3,
    {{-1,-1,-1}, {1,-1,-1}, {0,0,-1}, {-1,1,-1}, {1,1,-1}, {0,-1,0}, {-1,0,0}, {0,0,0},
     {1,0,0}, {0,1,0}, {-1,-1,1}, {1,-1,1}, {0,0,1}, {-1,1,1}, {1,1,1}},
    {1.0/72.0, 1.0/72.0, 1.0/9.0, 1.0/72.0, 1.0/72.0, 1.0/9.0, 1.0/9.0, 2.0/9.0,
     1.0/9.0, 1.0/9.0, 1.0/72.0, 1.0/72.0, 1.0/9.0, 1.0/72.0, 1.0/72.0}};

static const orc_lattice LAT_D3Q19 = {
    19, 3,
    {{0,-1,-1}, {-1,0,-1}, {0,0,-1}, {1,0,-1}, {0,1,-1}, {-1,-1,0}, {0,-1,0}, {1,-1,0},
     {-1,0,0}, {0,0,0}, {1,0,0}, {-1,1,0}, {0,1,0}, {1,1,0}, {0,-1,1}, {-1,0,1},
     {0,0,1}, {1,0,1}, {0,1,1}},
    {1.0/36.0, 1.0/36.0, 1.0/18.0, 1.0/36.0, 1.0/36.0, 1.0/36.0, 1.0/18.0, 1.0/36.0,
     1.0/18.0, 1.0/3.0, 1.0/18.0, 1.0/36.0, 1.0/18.0, 1.0/36.0, 1.0/36.0, 1.0/36.0,
     1.0/18.0, 1.0/36.0, 1.0/36.0}};

static const orc_lattice LAT_D3Q27 = {
    27, 3,
    {{-1,-1,-1}, {0,-1,-1}, {1,-1,-1}, {-1,0,-1}, {0,0,-1}, {1,0,-1}, {-1,1,-1}, {0,1,-1},
     {1,1,-1}, {-1,-1,0}, {0,-1,0}, {1,-1,0}, {-1,0,0}, {0,0,0}, {1,0,0}, {-1,1,0},
     {0,1,0}, {1,1,0}, {-1,-1,1}, {0,-1,1}, {1,-1,1}, {-1,0,1}, {0,0,1}, {1,0,1},
     {-1,1,1}, {0,1,1}, {1,1,1}},
    {1.0/216.0, 1.0/54.0, 1.0/216.0, 1.0/54.0, 2.0/27.0, 1.0/54.0, 1.0/216.0, 1.0/54.0,
     1.0/216.0, 1.0/54.0, 2.0/27.0, 1.0/54.0, 2.0/27.0, 8.0/27.0, 2.0/27.0, 1.0/54.0,
     2.0/27.0, 1.0/54.0, 1.0/216.0, 1.0/54.0, 1.0/216.0, 1.0/54.0, 2.0/27.0, 1.0/54.0,
     1.0/216.0, 1.0/54.0, 1.0/216.0}};

static const orc_lattice *get_lattice(int lat)
{
    switch (lat) {
    case ORC_D2Q9: return &LAT_D2Q9;
    case ORC_D3Q15: return &LAT_D3Q15;
    case ORC_D3Q19: return &LAT_D3Q19;
    case ORC_D3Q27: return &LAT_D3Q27;
    default: return NULL;
    }
}

/* Index of the velocity opposite to c_i, found by search. */
static int opposite(const orc_lattice *L, int i)
{
    for (int j = 0; j < L->Q; ++j)
        if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] && L->c[j][2] == -L->c[i][2])
            return j;
    return -1;
}

int orc_lattice_info(int lat, int *Q, int *D, int *c, double *w)
{
    const orc_lattice *L = get_lattice(lat);
    if (!L) return -1;
    if (Q) *Q = L->Q;
    if (D) *D = L->D;
    for (int i = 0; i < L->Q; ++i) {
        if (c) { c[3*i] = L->c[i][0]; c[3*i+1] = L->c[i][1]; c[3*i+2] = L->c[i][2]; }
        if (w) w[i] = L->w[i];
    }
    return 0;
}

int orc_opposite(int lat, int *opp)
{
    const orc_lattice *L = get_lattice(lat);
    if (!L) return -1;
    for (int i = 0; i < L->Q; ++i) opp[i] = opposite(L, i);
    return 0;
}

/* Second-order equilibrium, eq. (f_eq). */
static void equilibrium(const orc_lattice *L, double rho, const double u[3], double *feq)
{
    double uu = u[0]*u[0] + u[1]*u[1] + u[2]*u[2];
    for (int i = 0; i < L->Q; ++i) {
        double uc = u[0]*L->c[i][0] + u[1]*L->c[i][1] + u[2]*L->c[i][2];
        feq[i] = rho * L->w[i] * (1.0 + uc / CS2 + (uc*uc) / (2.0*CS2*CS2) - uu / (2.0*CS2));
    }
}

int orc_feq(int lat, double rho, const double *u, double *feq)
{
    const orc_lattice *L = get_lattice(lat);
    if (!L) return -1;
    equilibrium(L, rho, u, feq);
    return 0;
}

/* Papanastasiou apparent viscosity, eq. (Pap_reg_1), above the cut-off. */
static double nu_app_pap(const orc_params *p, double gdot, double rho)
{
    return p->nu_p + p->sigma_y / (rho * gdot) * (-expm1(-p->m * gdot));
}

/* eq. (Pap_reg_1) with the zero-strain interpolation of eq. (PR_interpolation),
 * reading R1: nu_0 at gdot = 0, linear up to nu_app(gdot_C). */
static double nu_app_pr(const orc_params *p, double gdot, double rho)
{
    double nu0 = p->nu_p + p->m * p->sigma_y / rho;
    if (gdot >= p->gdot_c)
        return nu_app_pap(p, gdot, rho);
    double gc = p->gdot_c;
    return (gc - gdot) / gc * nu0 + gdot / gc * nu_app_pap(p, gc, rho);
}

double orc_pr_nu_app(const orc_params *p, double gdot, double rho)
{
    return nu_app_pr(p, gdot, rho);
}

/* d nu_app / d gdot of nu_app_pr: the derivative of eq. (Pap_reg_1) above
 * the cut-off, the slope of the linear interpolation (reading R1) below it. */
static double nu_app_pr_slope(const orc_params *p, double gdot, double rho)
{
    if (gdot >= p->gdot_c) {
        double e = exp(-p->m * gdot);
        return p->sigma_y / rho * (p->m * e / gdot - (1.0 - e) / (gdot * gdot));
    }
    double nu0 = p->nu_p + p->m * p->sigma_y / rho;
    return (nu_app_pap(p, p->gdot_c, rho) - nu0) / p->gdot_c;
}

/* Implicit PR update (Sec. 3, second approach; reading R10).  The strain
 * rate of eq. (LBM_strain_rate) with the unknown tau is gdot(tau) = a / tau,
 * a = sqrt(2 T:T) / (2 c_s^2); tau itself follows from gdot through eqs.
 * (Pap_reg_1), (PR_interpolation) and (tau_visc).  Consistency is the root
 * of H(gdot) = gdot tau(gdot) - a.  Newton iterations on H start from the
 * explicit estimate gdot0 (previous step's tau). */
static double pr_newton_gdot(const orc_params *p, double a, double gdot0, double rho)
{
    double gdot = gdot0;
    for (int k = 0; k < p->newton; ++k) {
        double tau = nu_app_pr(p, gdot, rho) / CS2 + 0.5;
        double dtau = nu_app_pr_slope(p, gdot, rho) / CS2;
        double H = gdot * tau - a;
        double dH = tau + gdot * dtau;
        if (dH < 0.5) dH = 0.5;
        gdot = gdot - H / dH;
        if (gdot < 0.0) gdot = 0.0;
    }
    return gdot;
}

/* diag layout (optional output of orc_collide):
 *   [0] rho, [1..3] u (velocity used in f_eq), [4..12] T, [13..21] s,
 *   [22..30] sigma, [31..39] A, [40] gdot (PR), [41] nu_app (PR),
 *   [42] tau_new (PR), [43] yielded flag (IR)                              */
#define DIAG_N 44

/* One collision of one cell.  fin: the Q streamed populations; fout: the Q
 * post-collision populations.  tau_old / tau_new only matter for PR. */
static void collide(const orc_lattice *L, const orc_params *p, const double *fin,
                    double tau_old, double *fout, double *tau_new, double *diag)
{
    const int Q = L->Q;
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        rho += fin[i];
        for (int a = 0; a < 3; ++a) j[a] += L->c[i][a] * fin[i];
    }
    double F[3] = {rho * p->g[0], rho * p->g[1], rho * p->g[2]};
    double u[3], feq[ORC_MAXQ], T[3][3];
    double s[3][3] = {{0}}, sig[3][3] = {{0}}, A[3][3] = {{0}};
    double gdot = 0.0, nu = 0.0, tnew = tau_old;
    int yielded = 0;

    if (p->model == ORC_PR) {
        /* EDM: equilibrium at u = j / rho (eq. 14). */
        for (int a = 0; a < 3; ++a) u[a] = j[a] / rho;
    } else {
        /* IR: u = (j + F/2) / rho (reading R6). */
        for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / rho;
    }
    equilibrium(L, rho, u, feq);

    /* T = sum_i c_i c_i (f_i - f_i^eq), per population. */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double acc = 0.0;
            for (int i = 0; i < Q; ++i) acc += L->c[i][a] * L->c[i][b] * (fin[i] - feq[i]);
            T[a][b] = acc;
        }
    /* Burnett-suppressed variant: the xx component is dropped (for PR this is
     * d_xx = 0, since D is proportional to T). */
    if (p->burnett_x) T[0][0] = 0.0;

    if (p->model == ORC_PR) {
        /* eq. (LBM_strain_rate): D = -T / (2 tau_old c_s^2), previous step's tau. */
        double D[3][3], dd = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                D[a][b] = -T[a][b] / (2.0 * tau_old * CS2);
                dd += D[a][b] * D[a][b];
            }
        gdot = sqrt(2.0 * dd);                 /* eq. (strainInvariant) */
        if (p->newton > 0) {
            double tt = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) tt += T[a][b] * T[a][b];
            gdot = pr_newton_gdot(p, sqrt(2.0 * tt) / (2.0 * CS2), gdot, rho);
        }
        nu = nu_app_pr(p, gdot, rho);          /* eqs. (Pap_reg_1), (PR_interpolation) */
        tnew = nu / CS2 + 0.5;                 /* eq. (tau_visc) */
        double todd = 0.5 + p->magic / (tnew - 0.5); /* Lambda = (1/2 - tau_odd)(1/2 - tau_even) */
        double u2[3], feq2[ORC_MAXQ];
        for (int a = 0; a < 3; ++a) u2[a] = u[a] + F[a] / rho; /* u + du, du = F dt / rho */
        equilibrium(L, rho, u2, feq2);
        for (int i = 0; i < Q; ++i) {
            int k = opposite(L, i);
            double fp = 0.5 * (fin[i] + fin[k]), fm = 0.5 * (fin[i] - fin[k]);
            double ep = 0.5 * (feq[i] + feq[k]), em = 0.5 * (feq[i] - feq[k]);
            fout[i] = fin[i] - (fp - ep) / tnew - (fm - em) / todd + (feq2[i] - feq[i]);
        }
        if (tau_new) *tau_new = tnew;
    } else {
        /* eqs. (Vikh_sigmaS_formula), (Vikh_sigmaS_tensor) with reading R3. */
        double Tn = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Tn += T[a][b] * T[a][b];
        Tn = sqrt(Tn);
        double sy = sqrt(2.0) * p->sigma_y;
        if (Tn > 0.0 && Tn >= sy) {
            yielded = 1;
            double sc = -(Tn - sy) / (0.5 + 3.0 * p->nu_p);
            double gc = -(6.0 * p->nu_p * Tn + sy) / (1.0 + 6.0 * p->nu_p);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    s[a][b] = sc * T[a][b] / Tn;
                    sig[a][b] = gc * T[a][b] / Tn;
                }
        } else {
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    s[a][b] = 0.0;
                    sig[a][b] = -T[a][b];
                }
        }
        /* Deviatoric stress (reading R5) and A = -sigma_bar + s/2. */
        double tr = 0.0;
        for (int a = 0; a < L->D; ++a) tr += sig[a][a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double sbar = sig[a][b] - ((a == b && a < L->D) ? tr / L->D : 0.0);
                A[a][b] = -sbar + 0.5 * s[a][b];
            }
        /* eq. (Vikh_postCol) with f^sigma (reading R4) and force (reading R6). */
        for (int i = 0; i < Q; ++i) {
            double cA = 0.0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double h = L->c[i][a] * L->c[i][b] - ((a == b && a < L->D) ? CS2 : 0.0);
                    cA += h * A[a][b];
                }
            double fsig = L->w[i] / (2.0 * CS2 * CS2) * cA;
            double cF = L->c[i][0] * F[0] + L->c[i][1] * F[1] + L->c[i][2] * F[2];
            double phi = L->w[i] * cF / CS2;
            fout[i] = (feq[i] - 0.5 * phi) + fsig + phi;
        }
        if (tau_new) *tau_new = tau_old;
    }

    if (diag) {
        diag[0] = rho;
        for (int a = 0; a < 3; ++a) diag[1 + a] = u[a];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                diag[4 + 3*a + b] = T[a][b];
                diag[13 + 3*a + b] = s[a][b];
                diag[22 + 3*a + b] = sig[a][b];
                diag[31 + 3*a + b] = A[a][b];
            }
        diag[40] = gdot;
        diag[41] = nu;
        diag[42] = tnew;
        diag[43] = yielded;
    }
}

int orc_collide(int lat, const orc_params *p, const double *fin, double tau_old,
                double *fout, double *tau_new, double *diag)
{
    const orc_lattice *L = get_lattice(lat);
    if (!L || !p) return -1;
    collide(L, p, fin, tau_old, fout, tau_new, diag);
    return 0;
}

static int64_t wrap(int64_t a, int64_t n) { return ((a % n) + n) % n; }

/* Pull streaming with halfway bounce-back (eq. 8, Sec. 4.3): population i of
 * cell (x,y,z) comes from the cell at (x,y,z) - c_i; if that cell is solid the
 * population is the cell's own outgoing population in the opposite direction. */
static void gather(const orc_lattice *L, int nx, int ny, int nz, const uint8_t *mask,
                   const double *f, int x, int y, int z, double *fin)
{
    const int64_t N = (int64_t)nx * ny * nz;
    const int64_t self = x + (int64_t)nx * (y + (int64_t)ny * z);
    for (int i = 0; i < L->Q; ++i) {
        int64_t xs = wrap(x - L->c[i][0], nx);
        int64_t ys = wrap(y - L->c[i][1], ny);
        int64_t zs = wrap(z - L->c[i][2], nz);
        int64_t src = xs + (int64_t)nx * (ys + (int64_t)ny * zs);
        if (mask[src])
            fin[i] = f[(int64_t)opposite(L, i) * N + self];
        else
            fin[i] = f[(int64_t)i * N + src];
    }
}

static int check_dims(const orc_lattice *L, int nx, int ny, int nz)
{
    if (!L || nx < 1 || ny < 1 || nz < 1) return -1;
    if (L->D == 2 && nz != 1) return -1;
    return 0;
}

/* One time step: fdst <- collide(stream(fsrc)) on fluid cells; solid cells
 * copy through.  tau_src / tau_dst (may be NULL for IR) hold the PR per-cell
 * relaxation time. */
int orc_step(int lat, const orc_params *p, int nx, int ny, int nz, const uint8_t *mask,
             const double *fsrc, double *fdst, const double *tau_src, double *tau_dst,
             int nthreads)
{
    const orc_lattice *L = get_lattice(lat);
    if (check_dims(L, nx, ny, nz) || !p) return -1;
    if (p->model == ORC_PR && (!tau_src || !tau_dst)) return -1;
    const int64_t N = (int64_t)nx * ny * nz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    int64_t cell;
#pragma omp parallel for schedule(static)
    for (cell = 0; cell < N; ++cell) {
        int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((int64_t)nx * ny));
        if (mask[cell]) {
            for (int i = 0; i < L->Q; ++i) fdst[(int64_t)i * N + cell] = fsrc[(int64_t)i * N + cell];
            if (tau_dst && tau_src) tau_dst[cell] = tau_src[cell];
            continue;
        }
        double fin[ORC_MAXQ], fout[ORC_MAXQ], tnew = 0.0;
        gather(L, nx, ny, nz, mask, fsrc, x, y, z, fin);
        collide(L, p, fin, tau_src ? tau_src[cell] : 0.0, fout, &tnew, NULL);
        for (int i = 0; i < L->Q; ++i) fdst[(int64_t)i * N + cell] = fout[i];
        if (tau_dst) tau_dst[cell] = tnew;
    }
    return 0;
}

/* nsteps time steps in place on f (and tau for PR). */
int orc_run(int lat, const orc_params *p, int nx, int ny, int nz, const uint8_t *mask,
            double *f, double *tau, int64_t nsteps, int nthreads)
{
    const orc_lattice *L = get_lattice(lat);
    if (check_dims(L, nx, ny, nz) || !p || nsteps < 0) return -1;
    const int64_t N = (int64_t)nx * ny * nz;
    double *g = (double *)malloc(sizeof(double) * (size_t)(N * L->Q));
    double *t2 = (p->model == ORC_PR) ? (double *)malloc(sizeof(double) * (size_t)N) : NULL;
    if (!g || (p->model == ORC_PR && !t2)) { free(g); free(t2); return -2; }
    /* IR carries no relaxation-time field. */
    double *a = f, *b = g, *ta = (p->model == ORC_PR) ? tau : NULL, *tb = t2;
    for (int64_t s = 0; s < nsteps; ++s) {
        int rc = orc_step(lat, p, nx, ny, nz, mask, a, b, ta, tb, nthreads);
        if (rc) { free(g); free(t2); return rc; }
        double *t = a; a = b; b = t;
        t = ta; ta = tb; tb = t;
    }
    if (a != f) {
        memcpy(f, a, sizeof(double) * (size_t)(N * L->Q));
        if (p->model == ORC_PR) memcpy(tau, ta, sizeof(double) * (size_t)N);
    }
    free(g);
    free(t2);
    return 0;
}

/* Macroscopic fields of the state f (reading R9): rho and u_real of the
 * streamed populations; solid cells get rho = 0, u = 0.  u is [3][N]. */
int orc_fields(int lat, const orc_params *p, int nx, int ny, int nz, const uint8_t *mask,
               const double *f, double *rho, double *u)
{
    const orc_lattice *L = get_lattice(lat);
    if (check_dims(L, nx, ny, nz) || !p) return -1;
    const int64_t N = (int64_t)nx * ny * nz;
    int64_t cell;
#pragma omp parallel for schedule(static)
    for (cell = 0; cell < N; ++cell) {
        int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((int64_t)nx * ny));
        if (mask[cell]) {
            if (rho) rho[cell] = 0.0;
            if (u) { u[cell] = 0.0; u[N + cell] = 0.0; u[2*N + cell] = 0.0; }
            continue;
        }
        double fin[ORC_MAXQ], r = 0.0, j[3] = {0.0, 0.0, 0.0};
        gather(L, nx, ny, nz, mask, f, x, y, z, fin);
        for (int i = 0; i < L->Q; ++i) {
            r += fin[i];
            for (int a = 0; a < 3; ++a) j[a] += L->c[i][a] * fin[i];
        }
        if (rho) rho[cell] = r;
        if (u)
            for (int a = 0; a < 3; ++a) u[(int64_t)a * N + cell] = (j[a] + 0.5 * r * p->g[a]) / r;
    }
    return 0;
}

/* Post-collision populations of selected fluid cells only (for sampled checks
 * of very large domains).  fout is [ncells][Q], tau_out [ncells] (PR). */
int orc_step_cells(int lat, const orc_params *p, int nx, int ny, int nz, const uint8_t *mask,
                   const double *fsrc, const double *tau_src, int64_t ncells,
                   const int64_t *cells, double *fout, double *tau_out)
{
    const orc_lattice *L = get_lattice(lat);
    if (check_dims(L, nx, ny, nz) || !p) return -1;
    for (int64_t k = 0; k < ncells; ++k) {
        int64_t cell = cells[k];
        int x = (int)(cell % nx), y = (int)((cell / nx) % ny), z = (int)(cell / ((int64_t)nx * ny));
        double fin[ORC_MAXQ], tnew = 0.0;
        gather(L, nx, ny, nz, mask, fsrc, x, y, z, fin);
        collide(L, p, fin, tau_src ? tau_src[cell] : 0.0, fout + k * L->Q, &tnew, NULL);
        if (tau_out) tau_out[k] = tnew;
    }
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
