/*
 * dmrt_oracle.c -- plain FP64 CPU oracle of the double-MRT thermal lattice
 * Boltzmann method of "LBM Simulation of 3-D Natural Convection with Double
 * MRT Model" (arXiv:1511.04633).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference the
 * CUDA library is checked against.  Only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the library never does, and
 * this file shares no source, header, table or helper with the CUDA path.
 *
 * It follows the paper's statement of the method step by step, with DENSE
 * matrices (no use of their sparsity or orthogonality):
 *   D3Q19 flow  : Eqs. (11)-(26), Sec. 3.1
 *   D3Q7 energy : Eqs. (27)-(37), Sec. 3.2
 *   walls       : bounce-back for the flow (Sec. 3.1, closing paragraph);
 *                 thermal walls (Sec. 3.2, closing paragraph; rule below)
 *   lattice units, Nusselt numbers: Eqs. (38)-(41), Sec. 4
 *
 * One time step, for every cell x (Eqs. (14), (19), (29)):
 *   1. pull   f_i(x) <- f*_i(x - e_i),  g_i(x) <- g*_i(x - u_i)  (walls below)
 *   2. rho = sum f, rho V = sum e f, T = sum g                    Eqs. (20),(30)
 *   3. m = M f, n = N g                                           Eqs. (20),(30)
 *   4. m* = m - S (m - m_eq), n* = n - Q (n - n_eq)               Eqs. (19),(29)
 *   5. f* = M^-1 m* + F,  g* = N^-1 n*                            Eqs. (14),(15)
 * The stored state after a step is (f*, g*).  Reported fields are the
 * moments of the pulled (pre-collision) populations.
 *
 * Readings of garbled or silent passages (each is a named choice here):
 *   A1  Eq. (21) row 14 (p_xy) is printed (1,-1,1,-1) on columns 8..11, which
 *       makes M singular; it is e_x e_y = (1,-1,-1,1).  ORC_M_ROW14_FIX.
 *   A2  Eq. (20) "rho V = sum f_i" is read as rho V = sum e_i f_i.
 *   A3  Eq. (15) divides by "p"; read as c_s^2 = 1/3.  The force is added in
 *       velocity space after the collision, as Eq. (14) writes it.
 *   A4  Eq. (24) uses rho0 = 1 (the text below Eq. (25)); Eq. (15) uses the
 *       f_eq of Eq. (17) with the local rho.  orc_set_options() can make
 *       rho0 the local rho (a test-only switch for textbook identities).
 *   A6  T_l of Eqs. (4),(16) is the mean of T_h and T_c: theta_ref = 0 in the
 *       theta in [-1/2, 1/2] convention.  Switchable via orc_set_options().
 *   A7  H = ny lattice units (walls half-way between nodes), dT = 1, c = 1.
 *       Eq. (38): u_c = Ma c_s, Ra = g beta dT H^3 Pr / nu^2, Pr = nu/alpha.
 *   A8  Eq. (35) prints Q^-1; the rates are reciprocals.  Isotropic D = alpha I
 *       gives tau_xx = tau_yy = tau_zz = 1/2 + alpha/eps, eps = 1/4 (Eq. (36));
 *       tau_1 = tau_5 = tau_6 = tau_7 = 1 (text after Eq. (37)).
 *   A10 V in n_eq is the V of step 2 (same time level, no force shift).
 *   A11 Residual (paper silent): r = max(|th^n - th^{n-K}|/|th^n|,
 *       |V^n - V^{n-K}|/|V^n|) / K with 2-norms over all cells.
 *   A12 Thermal walls (rule not printed): Dirichlet walls (hot, cold, linear)
 *       by anti-bounce-back g_i(x) = -g*_opp(x) + 2 w_T,i T_w; adiabatic walls
 *       by bounce-back g_i(x) = g*_opp(x).  On a linear wall T_w is taken at
 *       the cell's own y.  Flow: half-way bounce-back f_i(x) = f*_opp(x) for
 *       every link that leaves the box (resting walls).
 *   A13 Nu (Eq. (39), discretisation not given): second-order one-sided
 *       difference d(theta)/dy = (-8 th_w + 9 th_1 - th_2) / 3 with th_1, th_2
 *       at 1/2 and 3/2 cells from the wall; Nu = -H d(theta)/dy.  Nu_3D: mean
 *       over the wall cells (Eq. (40)); Nu_2D: mean over z at X = 1/2, the two
 *       centre columns for even nx (Eq. (41)); Nu_max: maximum.
 *   A15 theta = (T - T_c)/dT - 1/2, so theta_h = +1/2, theta_c = -1/2.
 *
 * Layout of every population array: [q][z][y][x], x fastest.
 * Wall types: 0 = periodic (test-only, no walls), 1, 2, 3 = the paper's
 * Type 1 (Sec. 2, adiabatic sides), Type 2 (Eq. (9)), Type 3 (Eq. (10)).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q19 19
#define Q7 7

/* Eq. (12): the D3Q19 velocities, columns 1..19 in the printed order. */
static const int E19[Q19][3] = {
    {0, 0, 0},
    {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, 1, 0}, {1, -1, 0}, {-1, -1, 0},
    {1, 0, 1}, {-1, 0, 1}, {1, 0, -1}, {-1, 0, -1},
    {0, 1, 1}, {0, -1, 1}, {0, 1, -1}, {0, -1, -1},
};

/* Eq. (18): weights. */
static const double W19[Q19] = {
    1.0 / 3,
    1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
};

/* Eq. (13) with c = 1. */
static const double CS2 = 1.0 / 3.0;

/* Eq. (21), exactly as printed (row 14 included; see A1). */
static const double M_PRINTED[Q19][Q19] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {-30, -11, -11, -11, -11, -11, -11, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8, 8},
    {12, -4, -4, -4, -4, -4, -4, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, -4, 4, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, -4, 4, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, -4, 4, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1},
    {0, 2, 2, -1, -1, -1, -1, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, -4, -4, 2, 2, 2, 2, 1, 1, 1, 1, 1, 1, 1, 1, -2, -2, -2, -2},
    {0, 0, 0, 1, 1, -1, -1, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, -2, -2, 2, 2, 1, 1, 1, 1, -1, -1, -1, -1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1, 0, 0, 0, 0},
    {0, 0, 0, 0, 0, 0, 0, -1, -1, 1, 1, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1},
};

/* Reading A1: the corrected entries of row 14 (0-based row 13), columns 8..11. */
static const double ORC_M_ROW14_FIX[4] = {1, -1, -1, 1};

/* Eq. (28): D3Q7 velocities. */
static const int E7[Q7][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
};

/* Eq. (31): thermal weights. */
static const double W7[Q7] = {1.0 / 4, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8, 1.0 / 8};

/* Eq. (32). */
static const double N_MAT[Q7][Q7] = {
    {1, 1, 1, 1, 1, 1, 1},
    {0, 1, -1, 0, 0, 0, 0},
    {0, 0, 0, 1, -1, 0, 0},
    {0, 0, 0, 0, 0, 1, -1},
    {6, -1, -1, -1, -1, -1, -1},
    {0, 2, 2, -1, -1, -1, -1},
    {0, 0, 0, 1, 1, -1, -1},
};

/* Eq. (34): a = 7 w_T,1 - 1. */
static const double A_EQ34 = 7.0 * (1.0 / 4) - 1.0;

/* Eq. (36): epsilon for three dimensions. */
static const double EPS_EQ36 = 0.25;

/* Eq. (26): the fixed rates; the shear rates (10,12,14,15,16) depend on nu. */
static const double S_FIXED[Q19] = {
    1.0, 1.19, 1.4, 1.0, 1.2, 1.0, 1.2, 1.0, 1.2,
    -1 /* s10: nu */, 1.4, -1 /* s12: nu */, 1.4,
    -1 /* s14 */, -1 /* s15 */, -1 /* s16 */, 1.98, 1.98, 1.98,
};

typedef struct orc {
    int nx, ny, nz, wall;
    double nu, alpha, gbeta;
    double theta_ref; /* A6 */
    int rho0_local;   /* A4 test switch */
    double s[Q19], q[Q7];
    /* Eq. (35): the full relaxation matrix Q (inverse of the printed Q^-1);
     * diagonal (q) unless a diffusion tensor was set */
    double Qm[Q7][Q7];
    double M[Q19][Q19], Minv[Q19][Q19];
    double N[Q7][Q7], Ninv[Q7][Q7];
    int opp19[Q19], opp7[Q7];
    long cells;
    double *f, *g;   /* post-collision state */
    double *f2, *g2; /* scratch for the next state */
    long steps;
} orc_t;

/* ------------------------------------------------------------------ */
/* dense linear algebra                                                */

/* General inverse by Gauss-Jordan elimination with partial pivoting.
 * Returns 0 on success, -1 if the matrix is singular. */
int orc_invert(const double *A, int n, double *Ainv)
{
    double *w = (double *)malloc(sizeof(double) * n * 2 * n);
    if (!w) return -2;
    for (int r = 0; r < n; ++r) {
        for (int c = 0; c < n; ++c) {
            w[r * 2 * n + c] = A[r * n + c];
            w[r * 2 * n + n + c] = (r == c) ? 1.0 : 0.0;
        }
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = fabs(w[col * 2 * n + col]);
        for (int r = col + 1; r < n; ++r) {
            double v = fabs(w[r * 2 * n + col]);
            if (v > best) { best = v; piv = r; }
        }
        if (best < 1e-12) { free(w); return -1; }
        if (piv != col) {
            for (int c = 0; c < 2 * n; ++c) {
                double t = w[col * 2 * n + c];
                w[col * 2 * n + c] = w[piv * 2 * n + c];
                w[piv * 2 * n + c] = t;
            }
        }
        double d = w[col * 2 * n + col];
        for (int c = 0; c < 2 * n; ++c) w[col * 2 * n + c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double fct = w[r * 2 * n + col];
            if (fct == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) w[r * 2 * n + c] -= fct * w[col * 2 * n + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = w[r * 2 * n + n + c];
    free(w);
    return 0;
}

static void matvec(const double *A, const double *x, double *y, int n)
{
    for (int r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int c = 0; c < n; ++c) acc += A[r * n + c] * x[c];
        y[r] = acc;
    }
}

/* ------------------------------------------------------------------ */
/* the paper's matrices, equilibria and force                          */

/* Eq. (21).  printed != 0 returns the matrix exactly as printed. */
void orc_matrix_M(double *out, int printed)
{
    for (int r = 0; r < Q19; ++r)
        for (int c = 0; c < Q19; ++c) out[r * Q19 + c] = M_PRINTED[r][c];
    if (!printed)
        for (int c = 0; c < 4; ++c) out[13 * Q19 + 7 + c] = ORC_M_ROW14_FIX[c];
}

/* Eq. (32). */
void orc_matrix_N(double *out)
{
    for (int r = 0; r < Q7; ++r)
        for (int c = 0; c < Q7; ++c) out[r * Q7 + c] = N_MAT[r][c];
}

void orc_velocities19(int *out) { memcpy(out, E19, sizeof(E19)); }
void orc_weights19(double *out) { memcpy(out, W19, sizeof(W19)); }
void orc_velocities7(int *out) { memcpy(out, E7, sizeof(E7)); }
void orc_weights7(double *out) { memcpy(out, W7, sizeof(W7)); }

/* Eq. (17): f_i^eq(rho, V). */
void orc_feq(double rho, const double V[3], double *feq)
{
    double vv = V[0] * V[0] + V[1] * V[1] + V[2] * V[2];
    for (int i = 0; i < Q19; ++i) {
        double ev = E19[i][0] * V[0] + E19[i][1] * V[1] + E19[i][2] * V[2];
        feq[i] = rho * W19[i] *
                 (1.0 + ev / CS2 + (ev * ev) / (2.0 * CS2 * CS2) - vv / (2.0 * CS2));
    }
}

/* Eq. (24) with j from Eq. (25); rho0 as given (A4). */
void orc_meq(double rho, const double j[3], double rho0, double *meq)
{
    double jx = j[0], jy = j[1], jz = j[2];
    double jj = jx * jx + jy * jy + jz * jz;
    meq[0] = rho;
    meq[1] = -11.0 * rho + 19.0 * jj / rho0;
    meq[2] = 3.0 * rho - 5.5 * jj / rho0;
    meq[3] = jx;
    meq[4] = -2.0 / 3.0 * jx;
    meq[5] = jy;
    meq[6] = -2.0 / 3.0 * jy;
    meq[7] = jz;
    meq[8] = -2.0 / 3.0 * jz;
    meq[9] = (2.0 * jx * jx - (jy * jy + jz * jz)) / rho0;
    meq[10] = -0.5 * (2.0 * jx * jx - (jy * jy + jz * jz)) / rho0;
    meq[11] = (jy * jy - jz * jz) / rho0;
    meq[12] = -0.5 * (jy * jy - jz * jz) / rho0;
    meq[13] = jx * jy / rho0;
    meq[14] = jy * jz / rho0;
    meq[15] = jx * jz / rho0;
    meq[16] = 0.0;
    meq[17] = 0.0;
    meq[18] = 0.0;
}

/* Eq. (33) with a from Eq. (34). */
void orc_neq(double T, const double V[3], double *neq)
{
    neq[0] = T;
    neq[1] = V[0] * T;
    neq[2] = V[1] * T;
    neq[3] = V[2] * T;
    neq[4] = A_EQ34 * T;
    neq[5] = 0.0;
    neq[6] = 0.0;
}

/* Eq. (15) with "p" read as c_s^2 (A3) and dt = 1. */
void orc_force(double rho, const double V[3], const double G[3], double *F)
{
    double feq[Q19];
    orc_feq(rho, V, feq);
    for (int i = 0; i < Q19; ++i) {
        double gdot = 0.0;
        for (int a = 0; a < 3; ++a) gdot += G[a] * (E19[i][a] - V[a]);
        F[i] = gdot / CS2 * feq[i];
    }
}

/* Eq. (38), reading A7: lattice nu, alpha, g*beta for hot-to-cold distance H. */
void orc_lattice_from_physics(int H, double Ra, double Pr, double Ma, double out[3])
{
    double cs = sqrt(CS2);
    double uc = Ma * cs;                  /* Ma = u_c / c_s */
    double gbeta = uc * uc / (double)H;   /* u_c^2 = g beta dT H, dT = 1 */
    double nu = uc * (double)H * sqrt(Pr / Ra); /* Ra = g beta dT H^3 Pr / nu^2 */
    out[0] = nu;
    out[1] = nu / Pr;                     /* Pr = nu / alpha */
    out[2] = gbeta;
}

/* ------------------------------------------------------------------ */
/* state                                                               */

static long cell_index(const orc_t *o, int x, int y, int z)
{
    return ((long)z * o->ny + y) * o->nx + x;
}

static void q_from_rates(orc_t *o)
{
    for (int r = 0; r < Q7; ++r)
        for (int c = 0; c < Q7; ++c) o->Qm[r][c] = (r == c) ? o->q[r] : 0.0;
}

static void set_default_rates(orc_t *o)
{
    double s_nu = 1.0 / (3.0 * o->nu + 0.5); /* Eq. (26) */
    for (int k = 0; k < Q19; ++k) o->s[k] = (S_FIXED[k] < 0) ? s_nu : S_FIXED[k];
    double tau_a = 0.5 + o->alpha / EPS_EQ36; /* Eq. (36), dt = dx = 1 */
    o->q[0] = 1.0;
    o->q[1] = o->q[2] = o->q[3] = 1.0 / tau_a;
    o->q[4] = o->q[5] = o->q[6] = 1.0;
    q_from_rates(o);
}

orc_t *orc_create(int nx, int ny, int nz, int wall, double nu, double alpha, double gbeta)
{
    if (nx < 1 || ny < 1 || nz < 1 || wall < 0 || wall > 3) return NULL;
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    if (!o) return NULL;
    o->nx = nx; o->ny = ny; o->nz = nz; o->wall = wall;
    o->nu = nu; o->alpha = alpha; o->gbeta = gbeta;
    o->theta_ref = 0.0;
    o->rho0_local = 0;
    o->cells = (long)nx * ny * nz;
    orc_matrix_M(&o->M[0][0], 0);
    orc_matrix_N(&o->N[0][0]);
    if (orc_invert(&o->M[0][0], Q19, &o->Minv[0][0]) != 0 ||
        orc_invert(&o->N[0][0], Q7, &o->Ninv[0][0]) != 0) {
        free(o);
        return NULL;
    }
    for (int i = 0; i < Q19; ++i)
        for (int k = 0; k < Q19; ++k)
            if (E19[k][0] == -E19[i][0] && E19[k][1] == -E19[i][1] && E19[k][2] == -E19[i][2])
                o->opp19[i] = k;
    for (int i = 0; i < Q7; ++i)
        for (int k = 0; k < Q7; ++k)
            if (E7[k][0] == -E7[i][0] && E7[k][1] == -E7[i][1] && E7[k][2] == -E7[i][2])
                o->opp7[i] = k;
    set_default_rates(o);
    o->f = (double *)malloc(sizeof(double) * Q19 * o->cells);
    o->g = (double *)malloc(sizeof(double) * Q7 * o->cells);
    o->f2 = (double *)malloc(sizeof(double) * Q19 * o->cells);
    o->g2 = (double *)malloc(sizeof(double) * Q7 * o->cells);
    if (!o->f || !o->g || !o->f2 || !o->g2) {
        free(o->f); free(o->g); free(o->f2); free(o->g2); free(o);
        return NULL;
    }
    /* Initial state (from rest): f = f_eq(rho = 1, V = 0) = w, g = 0 (theta = 0). */
    for (int i = 0; i < Q19; ++i)
        for (long c = 0; c < o->cells; ++c) o->f[i * o->cells + c] = W19[i];
    memset(o->g, 0, sizeof(double) * Q7 * o->cells);
    o->steps = 0;
    return o;
}

void orc_destroy(orc_t *o)
{
    if (!o) return;
    free(o->f); free(o->g); free(o->f2); free(o->g2);
    free(o);
}

void orc_set_options(orc_t *o, double theta_ref, int rho0_local)
{
    o->theta_ref = theta_ref;
    o->rho0_local = rho0_local;
}

void orc_set_rates(orc_t *o, const double *s, const double *q)
{
    memcpy(o->s, s, sizeof(o->s));
    memcpy(o->q, q, sizeof(o->q));
    q_from_rates(o);
}

/* Eqs. (35)-(37) with a general diffusion tensor D (row-major 3x3, lattice
 * units, dt = dx = 1): Q^-1 = diag(tau_1, [tau_bar_ij], tau_5, tau_6, tau_7)
 * with tau_bar_ij = delta_ij / 2 + D_ij / eps, eps = 1/4, and
 * tau_1 = tau_5 = tau_6 = tau_7 = 1; Q is its inverse.  Returns 0, or -1 if
 * the matrix is singular. */
int orc_set_diffusion(orc_t *o, const double *D)
{
    double Qi[Q7][Q7];
    for (int r = 0; r < Q7; ++r)
        for (int c = 0; c < Q7; ++c) Qi[r][c] = (r == c) ? 1.0 : 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Qi[1 + i][1 + j] = (i == j ? 0.5 : 0.0) + D[3 * i + j] / EPS_EQ36;
    return orc_invert(&Qi[0][0], Q7, &o->Qm[0][0]);
}

void orc_get_rates(const orc_t *o, double *s, double *q)
{
    memcpy(s, o->s, sizeof(o->s));
    memcpy(q, o->q, sizeof(o->q));
}

long orc_steps(const orc_t *o) { return o->steps; }

void orc_set_populations(orc_t *o, const double *f, const double *g)
{
    memcpy(o->f, f, sizeof(double) * Q19 * o->cells);
    memcpy(o->g, g, sizeof(double) * Q7 * o->cells);
}

void orc_get_populations(const orc_t *o, double *f, double *g)
{
    memcpy(f, o->f, sizeof(double) * Q19 * o->cells);
    memcpy(g, o->g, sizeof(double) * Q7 * o->cells);
}

/* Equilibrium state from macroscopic fields: f = f_eq(rho, V) (Eq. (17)),
 * g = N^-1 n_eq(T, V) (Eq. (33)).  u is [3][cells]. */
void orc_init_fields(orc_t *o, const double *rho, const double *u, const double *T)
{
    for (long c = 0; c < o->cells; ++c) {
        double V[3] = {u[c], u[o->cells + c], u[2 * o->cells + c]};
        double feq[Q19], neq[Q7], geq[Q7];
        orc_feq(rho[c], V, feq);
        orc_neq(T[c], V, neq);
        matvec(&o->Ninv[0][0], neq, geq, Q7);
        for (int i = 0; i < Q19; ++i) o->f[i * o->cells + c] = feq[i];
        for (int i = 0; i < Q7; ++i) o->g[i * o->cells + c] = geq[i];
    }
}

/* ------------------------------------------------------------------ */
/* collision of one cell                                               */

/* Steps 2-5 above for one cell: pulled (fin, gin) -> stored (fout, gout). */
static void collide(const orc_t *o, const double *fin, const double *gin,
                    double *fout, double *gout)
{
    /* Eq. (20) with reading A2 */
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q19; ++i) {
        rho += fin[i];
        for (int a = 0; a < 3; ++a) j[a] += E19[i][a] * fin[i];
    }
    double V[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    /* Eq. (30) */
    double T = 0.0;
    for (int i = 0; i < Q7; ++i) T += gin[i];

    /* flow: Eq. (20) m = M f; Eq. (24) m_eq; Eq. (19) relax; back by M^-1 */
    double m[Q19], meq[Q19], ms[Q19];
    matvec(&o->M[0][0], fin, m, Q19);
    orc_meq(rho, j, o->rho0_local ? rho : 1.0, meq);
    for (int k = 0; k < Q19; ++k) ms[k] = m[k] - o->s[k] * (m[k] - meq[k]);
    matvec(&o->Minv[0][0], ms, fout, Q19);

    /* Eqs. (14)-(16): buoyancy along +z for gravity along -z, reading A6 */
    double G[3] = {0.0, 0.0, o->gbeta * (T - o->theta_ref)};
    double F[Q19];
    orc_force(rho, V, G, F);
    for (int i = 0; i < Q19; ++i) fout[i] += F[i];

    /* energy: Eq. (30) n = N g; Eq. (33) n_eq; Eq. (29) relax; back by N^-1 */
    double n[Q7], neq[Q7], ns[Q7];
    matvec(&o->N[0][0], gin, n, Q7);
    orc_neq(T, V, neq);
    /* Eq. (29): n* = n - Q (n - n_eq), Q the full matrix of Eq. (35) */
    for (int k = 0; k < Q7; ++k) {
        double acc = 0.0;
        for (int l = 0; l < Q7; ++l) acc += o->Qm[k][l] * (n[l] - neq[l]);
        ns[k] = n[k] - acc;
    }
    matvec(&o->Ninv[0][0], ns, gout, Q7);
}

/* One-cell collision, exported for the unit tests. */
void orc_collide(const orc_t *o, const double *fin, const double *gin, double *fout, double *gout)
{
    collide(o, fin, gin, fout, gout);
}

/* ------------------------------------------------------------------ */
/* streaming with walls                                                */

static int wrap(int a, int n) { return ((a % n) + n) % n; }

/* Temperature of a Dirichlet wall crossed by a link leaving the cell at
 * height y through a face on axis `axis` (0 = x, 1 = y, 2 = z), side `hi`.
 * Returns 1 and sets *Tw for a Dirichlet wall, 0 for an adiabatic one. */
static int thermal_wall(const orc_t *o, int axis, int hi, int y, double *Tw)
{
    double linear = 0.5 - ((double)y + 0.5) / (double)o->ny; /* Eq. (9), theta form */
    if (axis == 1) { /* Eqs. (6),(7): hot y = 0, cold y = H */
        *Tw = hi ? -0.5 : 0.5;
        return 1;
    }
    if (o->wall == 1) return 0; /* Type 1: the other four walls adiabatic */
    if (o->wall == 2) { *Tw = linear; return 1; } /* Type 2: Eq. (9) */
    /* Type 3, Eq. (10): x walls linear, z walls adiabatic */
    if (axis == 0) { *Tw = linear; return 1; }
    return 0;
}

/* Step 1 for one cell: the populations arriving at (x,y,z) from state (f,g). */
static void pull(const orc_t *o, const double *f, const double *g, int x, int y, int z,
                 double *fin, double *gin)
{
    long self = cell_index(o, x, y, z);
    for (int i = 0; i < Q19; ++i) {
        int sx = x - E19[i][0], sy = y - E19[i][1], sz = z - E19[i][2];
        if (o->wall == 0) {
            fin[i] = f[i * o->cells + cell_index(o, wrap(sx, o->nx), wrap(sy, o->ny), wrap(sz, o->nz))];
        } else if (sx >= 0 && sx < o->nx && sy >= 0 && sy < o->ny && sz >= 0 && sz < o->nz) {
            fin[i] = f[i * o->cells + cell_index(o, sx, sy, sz)];
        } else {
            fin[i] = f[o->opp19[i] * o->cells + self]; /* half-way bounce-back */
        }
    }
    for (int i = 0; i < Q7; ++i) {
        int sx = x - E7[i][0], sy = y - E7[i][1], sz = z - E7[i][2];
        if (o->wall == 0) {
            gin[i] = g[i * o->cells + cell_index(o, wrap(sx, o->nx), wrap(sy, o->ny), wrap(sz, o->nz))];
            continue;
        }
        if (sx >= 0 && sx < o->nx && sy >= 0 && sy < o->ny && sz >= 0 && sz < o->nz) {
            gin[i] = g[i * o->cells + cell_index(o, sx, sy, sz)];
            continue;
        }
        int axis = (sx < 0 || sx >= o->nx) ? 0 : (sy < 0 || sy >= o->ny) ? 1 : 2;
        int hi = (axis == 0) ? (sx >= o->nx) : (axis == 1) ? (sy >= o->ny) : (sz >= o->nz);
        double back = g[o->opp7[i] * o->cells + self];
        double Tw;
        if (thermal_wall(o, axis, hi, y, &Tw))
            gin[i] = -back + 2.0 * W7[i] * Tw; /* anti-bounce-back, A12 */
        else
            gin[i] = back; /* bounce-back, A12 */
    }
}

void orc_step(orc_t *o, long nsteps)
{
    for (long s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < o->nz; ++z) {
            double fin[Q19], gin[Q7], fout[Q19], gout[Q7];
            for (int y = 0; y < o->ny; ++y)
                for (int x = 0; x < o->nx; ++x) {
                    pull(o, o->f, o->g, x, y, z, fin, gin);
                    collide(o, fin, gin, fout, gout);
                    long c = cell_index(o, x, y, z);
                    for (int i = 0; i < Q19; ++i) o->f2[i * o->cells + c] = fout[i];
                    for (int i = 0; i < Q7; ++i) o->g2[i * o->cells + c] = gout[i];
                }
        }
        double *t = o->f; o->f = o->f2; o->f2 = t;
        t = o->g; o->g = o->g2; o->g2 = t;
        o->steps++;
    }
}

/* Reported fields: moments of the pulled populations (rho, V, T).
 * Any output pointer may be NULL.  u is [3][cells]. */
void orc_fields(const orc_t *o, double *rho, double *u, double *T)
{
#pragma omp parallel for schedule(static)
    for (int z = 0; z < o->nz; ++z) {
        double fin[Q19], gin[Q7];
        for (int y = 0; y < o->ny; ++y)
            for (int x = 0; x < o->nx; ++x) {
                pull(o, o->f, o->g, x, y, z, fin, gin);
                double r = 0.0, j[3] = {0.0, 0.0, 0.0}, t = 0.0;
                for (int i = 0; i < Q19; ++i) {
                    r += fin[i];
                    for (int a = 0; a < 3; ++a) j[a] += E19[i][a] * fin[i];
                }
                for (int i = 0; i < Q7; ++i) t += gin[i];
                long c = cell_index(o, x, y, z);
                if (rho) rho[c] = r;
                if (u)
                    for (int a = 0; a < 3; ++a) u[a * o->cells + c] = j[a] / r;
                if (T) T[c] = t;
            }
    }
}

/* ------------------------------------------------------------------ */
/* Nusselt numbers and residual                                        */

/* Eqs. (39)-(41) with reading A13 on a theta field [z][y][x].
 * wall 0: hot wall y = 0 (theta_w = +1/2); wall 1: cold wall y = H
 * (theta_w = -1/2).  out = (Nu_3D, Nu_2D, Nu_max); local (nullable) receives
 * the local Nu as [z][x].  Returns 0, or -1 if ny < 2. */
int orc_nusselt_from_theta(const double *theta, int nx, int ny, int nz, int wall,
                           double out[3], double *local)
{
    if (ny < 2 || nx < 1 || nz < 1) return -1;
    double H = (double)ny;
    double th_w = (wall == 0) ? 0.5 : -0.5;
    int y1 = (wall == 0) ? 0 : ny - 1;
    int y2 = (wall == 0) ? 1 : ny - 2;
    double sum = 0.0, mid = 0.0, mx = -INFINITY;
    int c_lo = (nx % 2 == 0) ? nx / 2 - 1 : (nx - 1) / 2;
    int c_hi = (nx % 2 == 0) ? nx / 2 : (nx - 1) / 2;
    for (int z = 0; z < nz; ++z)
        for (int x = 0; x < nx; ++x) {
            double t1 = theta[((long)z * ny + y1) * nx + x];
            double t2 = theta[((long)z * ny + y2) * nx + x];
            /* derivative along the inward normal s, at the wall */
            double dth_ds = (-8.0 * th_w + 9.0 * t1 - t2) / 3.0;
            /* Eq. (39): Nu = -d(theta)/dY; dY = dy / H; y = s on the hot wall,
             * y = H - s on the cold wall */
            double nu_loc = (wall == 0) ? -H * dth_ds : H * dth_ds;
            if (local) local[(long)z * nx + x] = nu_loc;
            sum += nu_loc;
            if (nu_loc > mx) mx = nu_loc;
            if (x == c_lo || x == c_hi) mid += nu_loc;
        }
    out[0] = sum / ((double)nx * nz);
    out[1] = mid / ((double)nz * (c_lo == c_hi ? 1 : 2));
    out[2] = mx;
    return 0;
}

int orc_nusselt(const orc_t *o, int wall, double out[3], double *local)
{
    double *T = (double *)malloc(sizeof(double) * o->cells);
    if (!T) return -2;
    orc_fields(o, NULL, NULL, T);
    int rc = orc_nusselt_from_theta(T, o->nx, o->ny, o->nz, wall, out, local);
    free(T);
    return rc;
}

/* Conservative cross-check of Eq. (39): the heat carried across the wall
 * links in one step, from the stored populations.  At the hot wall the
 * population g*_(-y) of a first-layer cell leaves through the wall and the
 * anti-bounce-back population -g*_(-y) + 2 w_T theta_w enters, so the net
 * flux in +y per unit area is 2 w_T theta_w - 2 g*_(-y); at the cold wall
 * it is 2 g*_(+y) - 2 w_T theta_w.  Nu = H q / (alpha dT), dT = 1.
 * Same averages as orc_nusselt_from_theta. */
int orc_nusselt_flux(const orc_t *o, int wall, double out[3], double *local)
{
    if (o->wall == 0 || o->ny < 1) return -1;
    const int ym = (wall == 0) ? 4 : 3; /* D3Q7 index of -y / +y */
    const int y = (wall == 0) ? 0 : o->ny - 1;
    const double th_w = (wall == 0) ? 0.5 : -0.5;
    const double H = (double)o->ny;
    const int nx = o->nx, nz = o->nz;
    double sum = 0.0, mid = 0.0, mx = -INFINITY;
    int c_lo = (nx % 2 == 0) ? nx / 2 - 1 : (nx - 1) / 2;
    int c_hi = (nx % 2 == 0) ? nx / 2 : (nx - 1) / 2;
    for (int z = 0; z < nz; ++z)
        for (int x = 0; x < nx; ++x) {
            double gl = o->g[ym * o->cells + cell_index(o, x, y, z)];
            double q = (wall == 0) ? 2.0 * W7[3] * th_w - 2.0 * gl : 2.0 * gl - 2.0 * W7[4] * th_w;
            double nu_loc = H * q / o->alpha;
            if (local) local[(long)z * nx + x] = nu_loc;
            sum += nu_loc;
            if (nu_loc > mx) mx = nu_loc;
            if (x == c_lo || x == c_hi) mid += nu_loc;
        }
    out[0] = sum / ((double)nx * nz);
    out[1] = mid / ((double)nz * (c_lo == c_hi ? 1 : 2));
    out[2] = mx;
    return 0;
}

/* Reading A11, from two snapshots taken K steps apart.  u is [3][cells]. */
static double rel_change(double num2, double den2)
{
    if (den2 == 0.0) return (num2 == 0.0) ? 0.0 : INFINITY;
    return sqrt(num2) / sqrt(den2);
}

double orc_residual(const double *th_now, const double *u_now, const double *th_prev,
                    const double *u_prev, long cells, int K)
{
    double dth = 0.0, th = 0.0, du = 0.0, uu = 0.0;
    for (long c = 0; c < cells; ++c) {
        double d = th_now[c] - th_prev[c];
        dth += d * d;
        th += th_now[c] * th_now[c];
        for (int a = 0; a < 3; ++a) {
            double e = u_now[a * cells + c] - u_prev[a * cells + c];
            du += e * e;
            uu += u_now[a * cells + c] * u_now[a * cells + c];
        }
    }
    double r1 = rel_change(dth, th), r2 = rel_change(du, uu);
    return (r1 > r2 ? r1 : r2) / (double)K;
}
