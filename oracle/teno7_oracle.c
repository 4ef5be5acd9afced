/*
 * teno7_oracle.c -- plain, slow, FP64 oracle for the extended seventh-order
 * TENO scheme ("TENO7-ext") of F. Zhang, J. Liu, H. Zhang, C. Xu,
 * "An extending strategy based on TENO framework for hyperbolic conservation
 * laws", arXiv:1808.00037.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path loads this library:
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg do.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * It runs the method step by step, in the paper's order:
 *   pass 1 -- every face's five-point smoothness measure and cutoff bits
 *             (Eqs. smooth_expl, tau5, TENO1, norm, seclect; epsilon = dx^3,
 *             Sec. "The parameter epsilon"), stored for the whole field
 *             (Sec. "The stencil-selection procedure": measure first, then
 *             reconstruct);
 *   pass 2 -- the binary vector Delta_i (Eq. vec) from this face's and the two
 *             neighbouring faces' bits, the selection of Table co3, and the
 *             polynomial of Table co2;
 * inside the conservative finite-difference form (Eq. app), characteristic-wise
 * with Roe-averaged eigenvectors and global Lax-Friedrichs splitting
 * (Remark 3; Sec. "One dimensional Euler equations"), and the third-order SSP
 * Runge-Kutta method (Sec. "The fundamental of the spatial solution").
 * A scheme switch (or_set_scheme) replaces pass 2 by the fifth-order TENO
 * baseline the paper compares with: each face's own three bits select a
 * Table co1 polynomial (epsilon 1e-40 as given with Eq. TENO1).
 * An alpha switch (or_set_alpha_mode; 1D systems) replaces the one global
 * Lax-Friedrichs alpha by one per characteristic field, alpha_k = max_i
 * |lambda_k(U_i)|, each field's split flux formed from the projections of
 * the flux and the state, q+-_k = (L_k F +- alpha_k L_k U) / 2.
 * The 2D form (or_rhs_2d, or_run_2d) applies the same face procedure
 * dimension by dimension, each direction in its own characteristic frame.
 *
 * Build with -O2 -ffp-contract=off and without fast-math, so that each
 * expression is evaluated exactly as written, one IEEE operation at a time.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENONPHYSICAL (-3)
#define OR_ENONFINITE (-4)

#define SYS_ADVECTION 0
#define SYS_EULER1D 1
#define SYS_EULER2D 2
#define SYS_BURGERS 3

#define BC_PERIODIC 0
#define BC_ZERO_GRADIENT 1

#define NG 4 /* ghost cells per side */

/* ------------------------------------------------------------------------ */
/* Table co2: coefficients a_{m,l} of the 13 candidate polynomials on        */
/* f_{i-3} .. f_{i+3}, rows exactly as printed.                              */
/* ------------------------------------------------------------------------ */
static const double COEF[13][7] = {
    {-1.0 / 140.0, 5.0 / 84.0, -101.0 / 420.0, 319.0 / 420.0, 107.0 / 210.0, -19.0 / 210.0, 1.0 / 105.0},
    {0.0, 1.0 / 60.0, -2.0 / 15.0, 37.0 / 60.0, 37.0 / 60.0, -2.0 / 15.0, 1.0 / 60.0},
    {-1.0 / 60.0, 7.0 / 60.0, -23.0 / 60.0, 19.0 / 20.0, 11.0 / 30.0, -1.0 / 30.0, 0.0},
    {0.0, 0.0, -1.0 / 20.0, 9.0 / 20.0, 47.0 / 60.0, -13.0 / 60.0, 1.0 / 30.0},
    {0.0, 1.0 / 30.0, -13.0 / 60.0, 47.0 / 60.0, 9.0 / 20.0, -1.0 / 20.0, 0.0},
    {-1.0 / 20.0, 17.0 / 60.0, -43.0 / 60.0, 77.0 / 60.0, 1.0 / 5.0, 0.0, 0.0},
    {0.0, 0.0, 0.0, 1.0 / 4.0, 13.0 / 12.0, -5.0 / 12.0, 1.0 / 12.0},
    {0.0, 0.0, -1.0 / 12.0, 7.0 / 12.0, 7.0 / 12.0, -1.0 / 12.0, 0.0},
    {0.0, 1.0 / 12.0, -5.0 / 12.0, 13.0 / 12.0, 1.0 / 4.0, 0.0, 0.0},
    {-1.0 / 4.0, 13.0 / 12.0, -23.0 / 12.0, 25.0 / 12.0, 0.0, 0.0, 0.0},
    {0.0, 0.0, 0.0, 1.0 / 3.0, 5.0 / 6.0, -1.0 / 6.0, 0.0},
    {0.0, 0.0, -1.0 / 6.0, 5.0 / 6.0, 1.0 / 3.0, 0.0, 0.0},
    {0.0, 1.0 / 3.0, -7.0 / 6.0, 11.0 / 6.0, 0.0, 0.0, 0.0},
};

/* Table co3: the binary vector Delta_i = (d_{i-1,0}, d_{i,0}, d_{i,1},
 * d_{i,2}, d_{i+1,2}) selects polynomial m; '*' matches 0 or 1.  The pattern
 * (*,0,0,0,*) is marked "no exist" in the table and has no row here. */
static const char *PATTERN[13] = {
    "11111", /* f0 */
    "01111", /* f1 */
    "11110", /* f2 */
    "*0111", /* f3 */
    "01110", /* f4 */
    "1110*", /* f5 */
    "**011", /* f6 */
    "*0110", /* f7 */
    "0110*", /* f8 */
    "1100*", /* f9 */
    "**010", /* f10 */
    "*010*", /* f11 */
    "0100*", /* f12 */
};

/* Table co1: the fifth-order TENO scheme (TENO5) written as single
 * polynomials on f_{i-2} .. f_{i+2}, selected by its own cutoff bits
 * (delta_0, delta_1, delta_2), rows as printed; (0,0,0) cannot occur. */
static const char *CO1_KEY[7] = {"111", "011", "110", "001", "010", "100", "101"};
static const double CO1[7][5] = {
    {1.0 / 30.0, -13.0 / 60.0, 47.0 / 60.0, 9.0 / 20.0, -1.0 / 20.0},
    {0.0, -1.0 / 9.0, 2.0 / 3.0, 1.0 / 2.0, -1.0 / 18.0},
    {1.0 / 21.0, -13.0 / 42.0, 41.0 / 42.0, 2.0 / 7.0, 0.0},
    {0.0, 0.0, 1.0 / 3.0, 5.0 / 6.0, -1.0 / 6.0},
    {0.0, -1.0 / 6.0, 5.0 / 6.0, 1.0 / 3.0, 0.0},
    {1.0 / 3.0, -7.0 / 6.0, 11.0 / 6.0, 0.0, 0.0},
    {1.0 / 12.0, -7.0 / 24.0, 17.0 / 24.0, 5.0 / 8.0, -1.0 / 8.0},
};

/* Scheme switch of the whole oracle: 0 = TENO7-ext (the paper's method),
 * 1 = TENO5 (the baseline it is compared with). */
#define SCHEME_TENO7EXT 0
#define SCHEME_TENO5 1
static int g_scheme = SCHEME_TENO7EXT;
void or_set_scheme(int scheme) { g_scheme = scheme; }
int or_get_scheme(void) { return g_scheme; }

/* Alpha switch (1D systems): 0 = one global Lax-Friedrichs alpha (Sec. "One
 * dimensional Euler equations"), 1 = one alpha per characteristic field. */
static int g_alpha_mode = 0;
void or_set_alpha_mode(int mode) { g_alpha_mode = mode; }
int or_get_alpha_mode(void) { return g_alpha_mode; }

/* Table co1 row for the three cutoff bits d0 | d1<<1 | d2<<2, -1 if none. */
int or_select5(int bits) {
    for (int r = 0; r < 7; r++) {
        int key = (CO1_KEY[r][0] - '0') | ((CO1_KEY[r][1] - '0') << 1) | ((CO1_KEY[r][2] - '0') << 2);
        if (key == bits) return r;
    }
    return -1;
}

void or_coeffs5(double *out /* 7*5 */) {
    for (int r = 0; r < 7; r++)
        for (int t = 0; t < 5; t++) out[r * 5 + t] = CO1[r][t];
}

static double poly5(int r, const double *v) {
    double s = 0.0;
    for (int t = 0; t < 5; t++) s = s + CO1[r][t] * v[t];
    return s;
}

void or_coeffs(double *out /* 13*7 */) {
    for (int m = 0; m < 13; m++)
        for (int t = 0; t < 7; t++) out[m * 7 + t] = COEF[m][t];
}

/* Delta packed as an integer: bit 4 = first component d_{i-1,0}, ...,
 * bit 0 = last component d_{i+1,2}.  Returns m, or -1 for "no exist". */
int or_select(int Delta) {
    int d[5];
    for (int c = 0; c < 5; c++) d[c] = (Delta >> (4 - c)) & 1;
    for (int m = 0; m < 13; m++) {
        int match = 1;
        for (int c = 0; c < 5; c++) {
            char p = PATTERN[m][c];
            if (p != '*' && (p - '0') != d[c]) match = 0;
        }
        if (match) return m;
    }
    return -1;
}

/* Five-point smoothness measure of one window w0..w4 = f_{i-2}..f_{i+2}
 * (upwind order), Eqs. smooth_expl, tau5, TENO1 (C = 1, q = 6), norm and
 * seclect.  Returns bits d0 | d1<<1 | d2<<2, delta_k = 0 iff chi_k < CT.
 * beta_out (nullable) receives beta_0..2. */
int or_face_bits(const double *w, double eps, double CT, double *beta_out) {
    double s0a = w[0] - 4.0 * w[1] + 3.0 * w[2];
    double s0b = w[0] - 2.0 * w[1] + w[2];
    double s1a = w[1] - w[3];
    double s1b = w[1] - 2.0 * w[2] + w[3];
    double s2a = 3.0 * w[2] - 4.0 * w[3] + w[4];
    double s2b = w[2] - 2.0 * w[3] + w[4];
    double beta[3];
    beta[0] = 0.25 * (s0a * s0a) + (13.0 / 12.0) * (s0b * s0b);
    beta[1] = 0.25 * (s1a * s1a) + (13.0 / 12.0) * (s1b * s1b);
    beta[2] = 0.25 * (s2a * s2a) + (13.0 / 12.0) * (s2b * s2b);
    double tau = fabs(beta[0] - beta[2]);
    double gam[3];
    for (int k = 0; k < 3; k++) {
        double g = 1.0 + tau / (beta[k] + eps);
        double g2 = g * g;
        gam[k] = (g2 * g2) * g2; /* (C + tau/(beta+eps))^6 */
    }
    double S = (gam[0] + gam[1]) + gam[2];
    int bits = 0;
    for (int k = 0; k < 3; k++) {
        double chi = gam[k] / S;
        int delta = (chi < CT) ? 0 : 1;
        bits |= delta << k;
    }
    if (beta_out) {
        beta_out[0] = beta[0];
        beta_out[1] = beta[1];
        beta_out[2] = beta[2];
    }
    return bits;
}

/* Delta_i for the '+' (left-biased) split at face i+1/2 from the stored
 * three-bit codes of faces i-1/2 (dm), i+1/2 (d0), i+3/2 (dp) (Eq. vec); the
 * '-' split is its mirror image, with the roles of dm and dp exchanged by the
 * caller. */
static int pack_delta(int dm, int d0, int dp) {
    int v0 = dm & 1, v1 = d0 & 1, v2 = (d0 >> 1) & 1, v3 = (d0 >> 2) & 1, v4 = (dp >> 2) & 1;
    return (v0 << 4) | (v1 << 3) | (v2 << 2) | (v3 << 1) | v4;
}

static double poly(int m, const double *v) {
    double s = 0.0;
    for (int t = 0; t < 7; t++) s = s + COEF[m][t] * v[t];
    return s;
}

/* ------------------------------------------------------------------------ */
/* Scalar reconstruction of one sequence of point values.                    */
/*   v[0 .. n+7]  values at cells -4 .. n+3 (caller-padded)                  */
/*   sign = +1: upwind from the left; sign = -1: the mirror image            */
/*   fhat[0 .. n]  face values at i+1/2, i = -1 .. n-1                       */
/*   d3[0 .. n+2]  (nullable) three-bit codes of faces -2 .. n               */
/*   D5[0 .. n]    (nullable) five-bit Delta of faces -1 .. n-1              */
/* ------------------------------------------------------------------------ */
int or_teno7_reconstruct(const double *v, int n, int sign, double eps, double CT, double *fhat, uint8_t *d3,
                         uint8_t *D5) {
    if (n < 1 || (sign != 1 && sign != -1)) return OR_EINVAL;
    int nf = n + 3;
    int *bits = (int *)malloc(sizeof(int) * nf);
    const double *c = v + NG; /* c[l] = value at cell l */
    int status = OR_OK;
    for (int j = -2; j <= n; j++) {
        double w[5];
        for (int t = 0; t < 5; t++) w[t] = (sign > 0) ? c[j - 2 + t] : c[j + 3 - t];
        bits[j + 2] = or_face_bits(w, eps, CT, NULL);
        if (d3) d3[j + 2] = (uint8_t)bits[j + 2];
    }
    for (int i = -1; i <= n - 1; i++) {
        if (g_scheme == SCHEME_TENO5) {
            int r = or_select5(bits[i + 2]);
            if (r < 0) {
                r = 0;
                status = OR_ENONFINITE;
            }
            double vv[5];
            for (int t = 0; t < 5; t++) vv[t] = (sign > 0) ? c[i - 2 + t] : c[i + 3 - t];
            fhat[i + 1] = poly5(r, vv);
            if (D5) D5[i + 1] = (uint8_t)bits[i + 2];
            continue;
        }
        int D = (sign > 0) ? pack_delta(bits[i + 1], bits[i + 2], bits[i + 3])
                           : pack_delta(bits[i + 3], bits[i + 2], bits[i + 1]);
        int m = or_select(D);
        if (m < 0) {
            m = 11;
            status = OR_ENONFINITE;
        }
        double vv[7];
        for (int t = 0; t < 7; t++) vv[t] = (sign > 0) ? c[i - 3 + t] : c[i + 4 - t];
        fhat[i + 1] = poly(m, vv);
        if (D5) D5[i + 1] = (uint8_t)D;
    }
    free(bits);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Physical systems.                                                         */
/* ------------------------------------------------------------------------ */
typedef struct {
    int sys;
    int m;
    double gamma;
    double a; /* advection speed */
} sysdef;

static int nvars_of(int sys) { return sys == SYS_EULER1D ? 3 : (sys == SYS_EULER2D ? 4 : 1); }

/* Physical flux along the sweep direction; for 2D Euler, dir 0 = x, 1 = y. */
static void flux(const sysdef *S, int dir, const double *U, double *F) {
    if (S->sys == SYS_ADVECTION) {
        F[0] = S->a * U[0];
    } else if (S->sys == SYS_BURGERS) {
        F[0] = 0.5 * U[0] * U[0];
    } else if (S->sys == SYS_EULER1D) {
        double u = U[1] / U[0];
        double p = (S->gamma - 1.0) * (U[2] - 0.5 * U[1] * u);
        F[0] = U[1];
        F[1] = U[1] * u + p;
        F[2] = u * (U[2] + p);
    } else {
        double u = U[1] / U[0];
        double v = U[2] / U[0];
        double p = (S->gamma - 1.0) * (U[3] - 0.5 * (U[1] * u + U[2] * v));
        if (dir == 0) {
            F[0] = U[1];
            F[1] = U[1] * u + p;
            F[2] = U[2] * u;
            F[3] = u * (U[3] + p);
        } else {
            F[0] = U[2];
            F[1] = U[1] * v;
            F[2] = U[2] * v + p;
            F[3] = v * (U[3] + p);
        }
    }
}

/* Largest characteristic speed of one cell along dir; sets *bad on a
 * non-physical or non-finite state. */
static double wavespeed(const sysdef *S, int dir, const double *U, int *bad) {
    if (S->sys == SYS_ADVECTION) return fabs(S->a);
    if (S->sys == SYS_BURGERS) {
        if (!isfinite(U[0])) *bad |= 2;
        return fabs(U[0]);
    }
    if (S->sys == SYS_EULER1D) {
        double u = U[1] / U[0];
        double p = (S->gamma - 1.0) * (U[2] - 0.5 * U[1] * u);
        double c = sqrt(S->gamma * p / U[0]);
        if (!(U[0] > 0.0) || !(p > 0.0)) *bad |= 1;
        if (!isfinite(U[0]) || !isfinite(U[1]) || !isfinite(U[2])) *bad |= 2;
        return fabs(u) + c;
    }
    double u = U[1] / U[0];
    double v = U[2] / U[0];
    double p = (S->gamma - 1.0) * (U[3] - 0.5 * (U[1] * u + U[2] * v));
    double c = sqrt(S->gamma * p / U[0]);
    if (!(U[0] > 0.0) || !(p > 0.0)) *bad |= 1;
    if (!isfinite(U[0]) || !isfinite(U[1]) || !isfinite(U[2]) || !isfinite(U[3])) *bad |= 2;
    return (dir == 0 ? fabs(u) : fabs(v)) + c;
}

/* Roe-averaged left (L, rows) and right (R, columns) eigenvectors of the flux
 * Jacobian at the face between states UL and UR (Remark 3).  Field order:
 * 1D Euler (u-c, u, u+c); 2D Euler along dir (un-c, un, shear, un+c).
 * Scalar systems: L = R = 1.  Returns nonzero if the Roe state has c^2 <= 0. */
static int frame(const sysdef *S, int dir, const double *UL, const double *UR, double L[4][4], double R[4][4]) {
    if (S->m == 1) {
        L[0][0] = 1.0;
        R[0][0] = 1.0;
        return 0;
    }
    double g = S->gamma;
    if (S->sys == SYS_EULER1D) {
        double rl = UL[0], rr = UR[0];
        double ul = UL[1] / rl, ur = UR[1] / rr;
        double pl = (g - 1.0) * (UL[2] - 0.5 * UL[1] * ul);
        double pr = (g - 1.0) * (UR[2] - 0.5 * UR[1] * ur);
        double Hl = (UL[2] + pl) / rl, Hr = (UR[2] + pr) / rr;
        double sl = sqrt(rl), sr = sqrt(rr);
        double ut = (sl * ul + sr * ur) / (sl + sr);
        double Ht = (sl * Hl + sr * Hr) / (sl + sr);
        double c2 = (g - 1.0) * (Ht - 0.5 * ut * ut);
        double c = sqrt(c2);
        double b1 = (g - 1.0) / c2;
        double b2 = 0.5 * ut * ut * b1;
        R[0][0] = 1.0;            R[0][1] = 1.0;           R[0][2] = 1.0;
        R[1][0] = ut - c;         R[1][1] = ut;            R[1][2] = ut + c;
        R[2][0] = Ht - ut * c;    R[2][1] = 0.5 * ut * ut; R[2][2] = Ht + ut * c;
        L[0][0] = 0.5 * (b2 + ut / c); L[0][1] = -0.5 * (b1 * ut + 1.0 / c); L[0][2] = 0.5 * b1;
        L[1][0] = 1.0 - b2;            L[1][1] = b1 * ut;                   L[1][2] = -b1;
        L[2][0] = 0.5 * (b2 - ut / c); L[2][1] = -0.5 * (b1 * ut - 1.0 / c); L[2][2] = 0.5 * b1;
        return !(c2 > 0.0);
    }
    /* 2D Euler: work in rotated order (rho, rho*un, rho*ut, E), then map back
     * to the physical order (rho, rho*u, rho*v, E). */
    int in = (dir == 0) ? 1 : 2, it = (dir == 0) ? 2 : 1;
    double rl = UL[0], rr = UR[0];
    double unl = UL[in] / rl, unr = UR[in] / rr;
    double utl = UL[it] / rl, utr = UR[it] / rr;
    double pl = (g - 1.0) * (UL[3] - 0.5 * (UL[1] * (UL[1] / rl) + UL[2] * (UL[2] / rl)));
    double pr = (g - 1.0) * (UR[3] - 0.5 * (UR[1] * (UR[1] / rr) + UR[2] * (UR[2] / rr)));
    double Hl = (UL[3] + pl) / rl, Hr = (UR[3] + pr) / rr;
    double sl = sqrt(rl), sr = sqrt(rr);
    double un = (sl * unl + sr * unr) / (sl + sr);
    double vt = (sl * utl + sr * utr) / (sl + sr);
    double Ht = (sl * Hl + sr * Hr) / (sl + sr);
    double q2 = 0.5 * (un * un + vt * vt);
    double c2 = (g - 1.0) * (Ht - q2);
    double c = sqrt(c2);
    double b1 = (g - 1.0) / c2;
    double b2 = q2 * b1;
    double Rr[4][4] = {
        {1.0, 1.0, 0.0, 1.0},
        {un - c, un, 0.0, un + c},
        {vt, vt, 1.0, vt},
        {Ht - un * c, q2, vt, Ht + un * c},
    };
    double Lr[4][4] = {
        {0.5 * (b2 + un / c), -0.5 * (b1 * un + 1.0 / c), -0.5 * (b1 * vt), 0.5 * b1},
        {1.0 - b2, b1 * un, b1 * vt, -b1},
        {-vt, 0.0, 1.0, 0.0},
        {0.5 * (b2 - un / c), -0.5 * (b1 * un - 1.0 / c), -0.5 * (b1 * vt), 0.5 * b1},
    };
    int perm[4] = {0, in, it, 3}; /* rotated index r <-> physical index perm[r] */
    for (int k = 0; k < 4; k++)
        for (int r = 0; r < 4; r++) {
            L[k][perm[r]] = Lr[k][r];
            R[perm[r]][k] = Rr[r][k];
        }
    return !(c2 > 0.0);
}

/* ------------------------------------------------------------------------ */
/* One directional sweep over a line of n cells with stride 1 in a padded    */
/* buffer P (m variables, each n + 2*NG long, cell l at P[c][l+NG]).          */
/* Writes the face fluxes Fh[c][i+1], i = -1..n-1 (face i+1/2) and, if masks  */
/* is non-null, the Delta codes masks[(s*m + k)*(n+1) + i+1].                 */
/* ------------------------------------------------------------------------ */
/* Characteristic split values of field k at padded cell l, split sign
 * (0: '+', 1: '-').  One alpha (alf == NULL): L_k G+- with the split fluxes
 * G+- = (F +- alpha U)/2 of the cell; per field (alf[k]): (L_k F +- alf[k]
 * L_k U)/2 with the cell's flux F and state U (arrays FF and UU). */
typedef struct {
    const double *Gp, *Gm, *FF, *UU, *alf;
    int m, np;
} splitdef;

static double split_value(const splitdef *D, const double L[4][4], int k, int l, int sign) {
    if (!D->alf) {
        const double *G = sign ? D->Gm : D->Gp;
        double s = L[k][0] * G[l];
        for (int c = 1; c < D->m; c++) s = s + L[k][c] * G[c * D->np + l];
        return s;
    }
    double lf = L[k][0] * D->FF[l], lu = L[k][0] * D->UU[l];
    for (int c = 1; c < D->m; c++) {
        lf = lf + L[k][c] * D->FF[c * D->np + l];
        lu = lu + L[k][c] * D->UU[c * D->np + l];
    }
    return sign ? 0.5 * (lf - D->alf[k] * lu) : 0.5 * (lf + D->alf[k] * lu);
}

/* alf (nullable): per-field alphas (the alpha switch); NULL: one global alpha */
static int sweep(const sysdef *S, int dir, double **P, int n, double alpha, const double *alf, double eps, double CT,
                 double **Fh, uint8_t *masks) {
    int m = S->m, np = n + 2 * NG;
    int status = OR_OK;
    /* global Lax-Friedrichs split fluxes G+- = (F +- alpha U)/2 per cell, or
     * (per-field alphas) the cell's flux and state */
    double *Gp = (double *)malloc(sizeof(double) * m * np);
    double *Gm = (double *)malloc(sizeof(double) * m * np);
    for (int l = 0; l < np; l++) {
        double U[4], F[4];
        for (int c = 0; c < m; c++) U[c] = P[c][l];
        flux(S, dir, U, F);
        for (int c = 0; c < m; c++) {
            if (alf) {
                Gp[c * np + l] = F[c];
                Gm[c * np + l] = U[c];
            } else {
                Gp[c * np + l] = 0.5 * (F[c] + alpha * U[c]);
                Gm[c * np + l] = 0.5 * (F[c] - alpha * U[c]);
            }
        }
    }
    splitdef D = {Gp, Gm, Gp, Gm, alf, m, np};
    /* pass 1: every face's bits in its own characteristic frame */
    int nf = n + 3;
    int *bits = (int *)malloc(sizeof(int) * 2 * m * nf); /* [s][k][face] */
    for (int j = -2; j <= n; j++) {
        double L[4][4], R[4][4], UL[4], UR[4];
        for (int c = 0; c < m; c++) {
            UL[c] = P[c][j + NG];
            UR[c] = P[c][j + 1 + NG];
        }
        if (frame(S, dir, UL, UR, L, R)) status = OR_ENONPHYSICAL;
        for (int k = 0; k < m; k++) {
            double wp[5], wm[5];
            for (int t = 0; t < 5; t++) {
                int lp = j - 2 + t + NG, lm = j + 3 - t + NG;
                wp[t] = split_value(&D, L, k, lp, 0);
                wm[t] = split_value(&D, L, k, lm, 1);
            }
            bits[(0 * m + k) * nf + j + 2] = or_face_bits(wp, eps, CT, NULL);
            bits[(1 * m + k) * nf + j + 2] = or_face_bits(wm, eps, CT, NULL);
        }
    }
    /* pass 2: selection and polynomial at faces -1 .. n-1 */
    for (int i = -1; i <= n - 1; i++) {
        double L[4][4], R[4][4], UL[4], UR[4], f[4];
        for (int c = 0; c < m; c++) {
            UL[c] = P[c][i + NG];
            UR[c] = P[c][i + 1 + NG];
        }
        frame(S, dir, UL, UR, L, R);
        for (int k = 0; k < m; k++) {
            const int *bp = bits + (0 * m + k) * nf, *bm = bits + (1 * m + k) * nf;
            if (g_scheme == SCHEME_TENO5) {
                /* TENO5: the face's own bits select a Table co1 row (no
                 * neighbour faces); masks report the three-bit code */
                int rp = or_select5(bp[i + 2]), rm = or_select5(bm[i + 2]);
                if (rp < 0 || rm < 0) {
                    status = OR_ENONFINITE;
                    if (rp < 0) rp = 0;
                    if (rm < 0) rm = 0;
                }
                double vp[5], vm[5];
                for (int t = 0; t < 5; t++) {
                    int lp = i - 2 + t + NG, lm = i + 3 - t + NG;
                    vp[t] = split_value(&D, L, k, lp, 0);
                    vm[t] = split_value(&D, L, k, lm, 1);
                }
                f[k] = poly5(rp, vp) + poly5(rm, vm);
                if (masks) {
                    masks[(0 * m + k) * (n + 1) + i + 1] = (uint8_t)bp[i + 2];
                    masks[(1 * m + k) * (n + 1) + i + 1] = (uint8_t)bm[i + 2];
                }
                continue;
            }
            int Dp = pack_delta(bp[i + 1], bp[i + 2], bp[i + 3]);
            int Dm = pack_delta(bm[i + 3], bm[i + 2], bm[i + 1]);
            int mp = or_select(Dp), mm = or_select(Dm);
            if (mp < 0) {
                mp = 11;
                status = OR_ENONFINITE;
            }
            if (mm < 0) {
                mm = 11;
                status = OR_ENONFINITE;
            }
            double vp[7], vm[7];
            for (int t = 0; t < 7; t++) {
                int lp = i - 3 + t + NG, lm = i + 4 - t + NG;
                vp[t] = split_value(&D, L, k, lp, 0);
                vm[t] = split_value(&D, L, k, lm, 1);
            }
            f[k] = poly(mp, vp) + poly(mm, vm);
            if (masks) {
                masks[(0 * m + k) * (n + 1) + i + 1] = (uint8_t)Dp;
                masks[(1 * m + k) * (n + 1) + i + 1] = (uint8_t)Dm;
            }
        }
        for (int c = 0; c < m; c++) {
            double s = R[c][0] * f[0];
            for (int k = 1; k < m; k++) s = s + R[c][k] * f[k];
            Fh[c][i + 1] = s;
        }
    }
    free(bits);
    free(Gp);
    free(Gm);
    return status;
}

/* Ghost cells: periodic U_l = U_(l mod n) (U_{-k} = U_{n-k} when n >= 4);
 * zero-gradient copies the nearest interior cell. */
static int ghost_index(int l, int n, int bc_lo, int bc_hi) {
    if (l < 0) return bc_lo == BC_PERIODIC ? ((l % n) + n) % n : 0;
    if (l >= n) return bc_hi == BC_PERIODIC ? l % n : n - 1;
    return l;
}

static int check_sys(int sys, int bc_lo, int bc_hi) {
    if (sys != SYS_ADVECTION && sys != SYS_EULER1D && sys != SYS_BURGERS) return 0;
    if (bc_lo != BC_PERIODIC && bc_lo != BC_ZERO_GRADIENT) return 0;
    if (bc_hi != BC_PERIODIC && bc_hi != BC_ZERO_GRADIENT) return 0;
    return 1;
}

/* Global Lax-Friedrichs alpha of a 1D state U[m][n]: max_i of the largest
 * characteristic speed over interior cells. */
static double alpha_1d(const sysdef *S, const double *U, int n, int *bad) {
    double a = 0.0;
    for (int i = 0; i < n; i++) {
        double Uc[4];
        for (int c = 0; c < S->m; c++) Uc[c] = U[c * n + i];
        double s = wavespeed(S, 0, Uc, bad);
        if (s > a || s != s) a = s;
    }
    return a;
}

/* Per-field alphas of a 1D state: alf[k] = max_i |lambda_k(U_i)| over interior
 * cells, lambda = (u - c, u, u + c) for Euler, the one wave speed for the
 * scalar laws.  max_k alf[k] equals the global alpha bit for bit (|u| + c is
 * the larger of |u - c| and |u + c|, rounded alike). */
static void alpha_fields_1d(const sysdef *S, const double *U, int n, int *bad, double *alf) {
    for (int k = 0; k < S->m; k++) alf[k] = 0.0;
    for (int i = 0; i < n; i++) {
        double Uc[4];
        for (int c = 0; c < S->m; c++) Uc[c] = U[c * n + i];
        if (S->sys != SYS_EULER1D) {
            double s = wavespeed(S, 0, Uc, bad);
            if (s > alf[0] || s != s) alf[0] = s;
            continue;
        }
        double u = Uc[1] / Uc[0];
        double p = (S->gamma - 1.0) * (Uc[2] - 0.5 * Uc[1] * u);
        double c = sqrt(S->gamma * p / Uc[0]);
        if (!(Uc[0] > 0.0) || !(p > 0.0)) *bad |= 1;
        if (!isfinite(Uc[0]) || !isfinite(Uc[1]) || !isfinite(Uc[2])) *bad |= 2;
        double lam[3] = {fabs(u - c), fabs(u), fabs(u + c)};
        for (int k = 0; k < 3; k++)
            if (lam[k] > alf[k] || lam[k] != lam[k]) alf[k] = lam[k];
    }
}

int or_alpha_fields_1d(int sys, const double *U, int n, double gamma, double a, double *alf) {
    if (n < 1 || !check_sys(sys, BC_PERIODIC, BC_PERIODIC)) return OR_EINVAL;
    sysdef S = {sys, nvars_of(sys), gamma, a};
    int bad = 0;
    alpha_fields_1d(&S, U, n, &bad, alf);
    if (bad & 2) return OR_ENONFINITE;
    if (bad & 1) return OR_ENONPHYSICAL;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* 1D right-hand side L(U) = -(F_{i+1/2} - F_{i-1/2})/dx (Eq. app).           */
/*   U, dUdt: [m][n] row-major (variable-major).  alpha_in < 0: computed from */
/*   U; otherwise used as given.  masks (nullable): [2][m][n+1] Delta codes.  */
/*   alpha_out (nullable) receives the alpha used.  Alpha switch = 1: the     */
/*   per-field alphas of U (alpha_in >= 0: that value for every field), and   */
/*   alpha_out receives their maximum.                                        */
/* ------------------------------------------------------------------------ */
int or_rhs_1d(int sys, const double *U, int n, double dx, double gamma, double a, double CT, double eps_in,
              int bc_lo, int bc_hi, double alpha_in, double *dUdt, uint8_t *masks, double *alpha_out) {
    if (n < 1 || !check_sys(sys, bc_lo, bc_hi) || !(dx > 0.0)) return OR_EINVAL;
    sysdef S = {sys, nvars_of(sys), gamma, a};
    int m = S.m, np = n + 2 * NG;
    int bad = 0;
    /* default epsilon: dx^3 for TENO7-ext (Sec. "The parameter epsilon"),
     * 1e-40 for TENO5 (as given with Eq. TENO1) */
    double eps = (eps_in < 0.0) ? (g_scheme == SCHEME_TENO5 ? 1e-40 : dx * dx * dx) : eps_in;
    double alpha = (alpha_in < 0.0) ? alpha_1d(&S, U, n, &bad) : alpha_in;
    double alf[4] = {alpha, alpha, alpha, alpha};
    if (g_alpha_mode && alpha_in < 0.0) alpha_fields_1d(&S, U, n, &bad, alf);
    if (alpha_out) *alpha_out = alpha;
    double *P[4], *Fh[4];
    for (int c = 0; c < m; c++) {
        P[c] = (double *)malloc(sizeof(double) * np);
        Fh[c] = (double *)malloc(sizeof(double) * (n + 1));
        for (int l = -NG; l < n + NG; l++) P[c][l + NG] = U[c * n + ghost_index(l, n, bc_lo, bc_hi)];
    }
    int status = sweep(&S, 0, P, n, alpha, g_alpha_mode ? alf : NULL, eps, CT, Fh, masks);
    for (int c = 0; c < m; c++)
        for (int i = 0; i < n; i++) dUdt[c * n + i] = (Fh[c][i] - Fh[c][i + 1]) / dx;
    for (int c = 0; c < m; c++) {
        free(P[c]);
        free(Fh[c]);
    }
    if (bad & 2) return OR_ENONFINITE;
    if (bad & 1) return OR_ENONPHYSICAL;
    return status;
}

/* The characteristic split values of face i+1/2 (i = -1 .. n-1) of a 1D
 * state, as the sweep forms them: Pp[k*7 + t] = '+' value of field k at cell
 * i-3+t, Pm[k*7 + t] = '-' value at cell i+4-t, in the face's Roe frame, with
 * the alphas of or_rhs_1d (alpha_in < 0: from U; the alpha switch applies). */
int or_face_split_1d(int sys, const double *U, int n, double gamma, double a, int bc_lo, int bc_hi, double alpha_in,
                     int i, double *Pp, double *Pm) {
    if (n < 1 || i < -1 || i > n - 1 || !check_sys(sys, bc_lo, bc_hi)) return OR_EINVAL;
    sysdef S = {sys, nvars_of(sys), gamma, a};
    int m = S.m, np = n + 2 * NG, bad = 0;
    double alpha = (alpha_in < 0.0) ? alpha_1d(&S, U, n, &bad) : alpha_in;
    double alf[4] = {alpha, alpha, alpha, alpha};
    if (g_alpha_mode && alpha_in < 0.0) alpha_fields_1d(&S, U, n, &bad, alf);
    double *G[2];
    for (int h = 0; h < 2; h++) G[h] = (double *)malloc(sizeof(double) * m * np);
    for (int l = 0; l < np; l++) {
        double Uc[4], F[4];
        for (int c = 0; c < m; c++) Uc[c] = U[c * n + ghost_index(l - NG, n, bc_lo, bc_hi)];
        flux(&S, 0, Uc, F);
        for (int c = 0; c < m; c++) {
            G[0][c * np + l] = g_alpha_mode ? F[c] : 0.5 * (F[c] + alpha * Uc[c]);
            G[1][c * np + l] = g_alpha_mode ? Uc[c] : 0.5 * (F[c] - alpha * Uc[c]);
        }
    }
    splitdef D = {G[0], G[1], G[0], G[1], g_alpha_mode ? alf : NULL, m, np};
    double L[4][4], R[4][4], UL[4], UR[4];
    for (int c = 0; c < m; c++) {
        UL[c] = U[c * n + ghost_index(i, n, bc_lo, bc_hi)];
        UR[c] = U[c * n + ghost_index(i + 1, n, bc_lo, bc_hi)];
    }
    if (frame(&S, 0, UL, UR, L, R)) bad |= 1;
    for (int k = 0; k < m; k++)
        for (int t = 0; t < 7; t++) {
            Pp[k * 7 + t] = split_value(&D, L, k, i - 3 + t + NG, 0);
            Pm[k * 7 + t] = split_value(&D, L, k, i + 4 - t + NG, 1);
        }
    for (int h = 0; h < 2; h++) free(G[h]);
    if (bad & 2) return OR_ENONFINITE;
    if (bad & 1) return OR_ENONPHYSICAL;
    return OR_OK;
}

/* Third-order SSP Runge-Kutta step (Shu-Osher form), in place on U[m][n]. */
int or_rk3_step_1d(int sys, double *U, int n, double dx, double gamma, double a, double CT, double eps, int bc_lo,
                   int bc_hi, double dt) {
    int m = nvars_of(sys), N = m * n, st, status = OR_OK;
    double *U0 = (double *)malloc(sizeof(double) * N);
    double *U1 = (double *)malloc(sizeof(double) * N);
    double *r = (double *)malloc(sizeof(double) * N);
    memcpy(U0, U, sizeof(double) * N);
    st = or_rhs_1d(sys, U0, n, dx, gamma, a, CT, eps, bc_lo, bc_hi, -1.0, r, NULL, NULL);
    if (st) status = st;
    for (int q = 0; q < N; q++) U1[q] = U0[q] + dt * r[q];
    st = or_rhs_1d(sys, U1, n, dx, gamma, a, CT, eps, bc_lo, bc_hi, -1.0, r, NULL, NULL);
    if (st) status = st;
    for (int q = 0; q < N; q++) U1[q] = 0.75 * U0[q] + 0.25 * (U1[q] + dt * r[q]);
    st = or_rhs_1d(sys, U1, n, dx, gamma, a, CT, eps, bc_lo, bc_hi, -1.0, r, NULL, NULL);
    if (st) status = st;
    for (int q = 0; q < N; q++) U[q] = (1.0 / 3.0) * U0[q] + (2.0 / 3.0) * (U1[q] + dt * r[q]);
    free(U0);
    free(U1);
    free(r);
    return status;
}

/* CFL time step dt = CFL dx / alpha(U). */
int or_cfl_dt_1d(int sys, const double *U, int n, double dx, double gamma, double a, double cfl, double *dt_out) {
    sysdef S = {sys, nvars_of(sys), gamma, a};
    int bad = 0;
    double alpha = alpha_1d(&S, U, n, &bad);
    *dt_out = (cfl * dx) / alpha;
    if (bad & 2) return OR_ENONFINITE;
    if (bad & 1) return OR_ENONPHYSICAL;
    return OR_OK;
}

/* March U to t_end (last step clipped to land on it) or for max_steps steps.
 * dt_fixed > 0 uses that step; otherwise dt = CFL dx / alpha(U^n) each step. */
int or_run_1d(int sys, double *U, int n, double dx, double gamma, double a, double CT, double eps, int bc_lo,
              int bc_hi, double cfl, double dt_fixed, double t_end, int max_steps, int *steps_out, double *t_out) {
    double t = 0.0;
    int steps = 0, status = OR_OK;
    while (steps < max_steps && t < t_end) {
        double dt;
        if (dt_fixed > 0.0) {
            dt = dt_fixed;
        } else {
            int st = or_cfl_dt_1d(sys, U, n, dx, gamma, a, cfl, &dt);
            if (st) {
                status = st;
                break;
            }
        }
        if (t + dt > t_end) dt = t_end - t;
        int st = or_rk3_step_1d(sys, U, n, dx, gamma, a, CT, eps, bc_lo, bc_hi, dt);
        t = t + dt;
        steps++;
        if (st) {
            status = st;
            break;
        }
    }
    if (steps_out) *steps_out = steps;
    if (t_out) *t_out = t;
    return status;
}

/* ------------------------------------------------------------------------ */
/* 2D Euler, dimension by dimension: L(U) = Lx(U) + Ly(U).  U, dUdt are      */
/* [4][ny][nx] (x fastest).  bc[4] = {x_lo, x_hi, y_lo, y_hi}.               */
/* alpha_in[2] (nullable) overrides the (x, y) global Lax-Friedrichs alphas. */
/* masks (nullable): x faces [2][4][ny][nx+1] followed by y faces            */
/* [2][4][nx][ny+1] (column-major for y, one column per x index).           */
/* ------------------------------------------------------------------------ */
static void alpha_2d(const sysdef *S, const double *U, int nx, int ny, double *ax, double *ay, int *bad) {
    int N = nx * ny;
    double a0 = 0.0, a1 = 0.0;
    for (int q = 0; q < N; q++) {
        double Uc[4] = {U[q], U[N + q], U[2 * N + q], U[3 * N + q]};
        double sx = wavespeed(S, 0, Uc, bad), sy = wavespeed(S, 1, Uc, bad);
        if (sx > a0 || sx != sx) a0 = sx;
        if (sy > a1 || sy != sy) a1 = sy;
    }
    *ax = a0;
    *ay = a1;
}

int or_rhs_2d(const double *U, int nx, int ny, double dx, double dy, double gamma, double CT, double eps_x_in,
              double eps_y_in, const int *bc, const double *alpha_in, double *dUdt, uint8_t *masks,
              double *alpha_out) {
    if (nx < 1 || ny < 1 || g_alpha_mode) return OR_EINVAL;  /* the alpha switch is 1D only */
    sysdef S = {SYS_EULER2D, 4, gamma, 0.0};
    int N = nx * ny, bad = 0, status = OR_OK;
    double ax, ay;
    if (alpha_in) {
        ax = alpha_in[0];
        ay = alpha_in[1];
    } else {
        alpha_2d(&S, U, nx, ny, &ax, &ay, &bad);
    }
    if (alpha_out) {
        alpha_out[0] = ax;
        alpha_out[1] = ay;
    }
    double epsx = (eps_x_in < 0.0) ? (g_scheme == SCHEME_TENO5 ? 1e-40 : dx * dx * dx) : eps_x_in;
    double epsy = (eps_y_in < 0.0) ? (g_scheme == SCHEME_TENO5 ? 1e-40 : dy * dy * dy) : eps_y_in;
    double *P[4], *Fh[4];
    int nmax = nx > ny ? nx : ny;
    for (int c = 0; c < 4; c++) {
        P[c] = (double *)malloc(sizeof(double) * (nmax + 2 * NG));
        Fh[c] = (double *)malloc(sizeof(double) * (nmax + 1));
    }
    /* x sweeps */
    for (int y = 0; y < ny; y++) {
        for (int c = 0; c < 4; c++)
            for (int l = -NG; l < nx + NG; l++) P[c][l + NG] = U[c * N + y * nx + ghost_index(l, nx, bc[0], bc[1])];
        uint8_t *mk = masks ? masks + (size_t)y * (nx + 1) : NULL;
        /* per-row masks are scattered below, so sweep into a temporary */
        uint8_t *tmp = masks ? (uint8_t *)malloc(2 * 4 * (nx + 1)) : NULL;
        int st = sweep(&S, 0, P, nx, ax, NULL, epsx, CT, Fh, tmp);
        if (st) status = st;
        for (int c = 0; c < 4; c++)
            for (int i = 0; i < nx; i++) dUdt[c * N + y * nx + i] = (Fh[c][i] - Fh[c][i + 1]) / dx;
        if (masks) {
            for (int sk = 0; sk < 8; sk++) memcpy(mk + (size_t)sk * ny * (nx + 1), tmp + sk * (nx + 1), nx + 1);
            free(tmp);
        }
    }
    /* y sweeps, added to the x part */
    uint8_t *ymasks = masks ? masks + (size_t)8 * ny * (nx + 1) : NULL;
    for (int x = 0; x < nx; x++) {
        for (int c = 0; c < 4; c++)
            for (int l = -NG; l < ny + NG; l++) P[c][l + NG] = U[c * N + ghost_index(l, ny, bc[2], bc[3]) * nx + x];
        uint8_t *tmp = masks ? (uint8_t *)malloc(2 * 4 * (ny + 1)) : NULL;
        int st = sweep(&S, 1, P, ny, ay, NULL, epsy, CT, Fh, tmp);
        if (st) status = st;
        for (int c = 0; c < 4; c++)
            for (int j = 0; j < ny; j++) {
                double ry = (Fh[c][j] - Fh[c][j + 1]) / dy;
                dUdt[c * N + j * nx + x] = dUdt[c * N + j * nx + x] + ry;
            }
        if (masks) {
            for (int sk = 0; sk < 8; sk++)
                memcpy(ymasks + (size_t)sk * nx * (ny + 1) + (size_t)x * (ny + 1), tmp + sk * (ny + 1), ny + 1);
            free(tmp);
        }
    }
    for (int c = 0; c < 4; c++) {
        free(P[c]);
        free(Fh[c]);
    }
    if (bad & 2) return OR_ENONFINITE;
    if (bad & 1) return OR_ENONPHYSICAL;
    return status;
}

int or_cfl_dt_2d(const double *U, int nx, int ny, double dx, double dy, double gamma, double cfl, double *dt_out) {
    sysdef S = {SYS_EULER2D, 4, gamma, 0.0};
    int bad = 0;
    double ax, ay;
    alpha_2d(&S, U, nx, ny, &ax, &ay, &bad);
    *dt_out = cfl / (ax / dx + ay / dy);
    if (bad & 2) return OR_ENONFINITE;
    if (bad & 1) return OR_ENONPHYSICAL;
    return OR_OK;
}

int or_rk3_step_2d(double *U, int nx, int ny, double dx, double dy, double gamma, double CT, double epsx,
                   double epsy, const int *bc, double dt) {
    int N = 4 * nx * ny, st, status = OR_OK;
    double *U0 = (double *)malloc(sizeof(double) * N);
    double *U1 = (double *)malloc(sizeof(double) * N);
    double *r = (double *)malloc(sizeof(double) * N);
    memcpy(U0, U, sizeof(double) * N);
    st = or_rhs_2d(U0, nx, ny, dx, dy, gamma, CT, epsx, epsy, bc, NULL, r, NULL, NULL);
    if (st) status = st;
    for (int q = 0; q < N; q++) U1[q] = U0[q] + dt * r[q];
    st = or_rhs_2d(U1, nx, ny, dx, dy, gamma, CT, epsx, epsy, bc, NULL, r, NULL, NULL);
    if (st) status = st;
    for (int q = 0; q < N; q++) U1[q] = 0.75 * U0[q] + 0.25 * (U1[q] + dt * r[q]);
    st = or_rhs_2d(U1, nx, ny, dx, dy, gamma, CT, epsx, epsy, bc, NULL, r, NULL, NULL);
    if (st) status = st;
    for (int q = 0; q < N; q++) U[q] = (1.0 / 3.0) * U0[q] + (2.0 / 3.0) * (U1[q] + dt * r[q]);
    free(U0);
    free(U1);
    free(r);
    return status;
}

int or_run_2d(double *U, int nx, int ny, double dx, double dy, double gamma, double CT, double epsx, double epsy,
              const int *bc, double cfl, double dt_fixed, double t_end, int max_steps, int *steps_out,
              double *t_out) {
    double t = 0.0;
    int steps = 0, status = OR_OK;
    while (steps < max_steps && t < t_end) {
        double dt;
        if (dt_fixed > 0.0) {
            dt = dt_fixed;
        } else {
            int st = or_cfl_dt_2d(U, nx, ny, dx, dy, gamma, cfl, &dt);
            if (st) {
                status = st;
                break;
            }
        }
        if (t + dt > t_end) dt = t_end - t;
        int st = or_rk3_step_2d(U, nx, ny, dx, dy, gamma, CT, epsx, epsy, bc, dt);
        t = t + dt;
        steps++;
        if (st) {
            status = st;
            break;
        }
    }
    if (steps_out) *steps_out = steps;
    if (t_out) *t_out = t;
    return status;
}

/* Euler-1D characteristic frame, exported for the tests' eigen checks. */
int or_frame_1d(const double *UL, const double *UR, double gamma, double *L9, double *R9) {
    sysdef S = {SYS_EULER1D, 3, gamma, 0.0};
    double L[4][4], R[4][4];
    int st = frame(&S, 0, UL, UR, L, R);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            L9[a * 3 + b] = L[a][b];
            R9[a * 3 + b] = R[a][b];
        }
    return st;
}

int or_frame_2d(const double *UL, const double *UR, double gamma, int dir, double *L16, double *R16) {
    sysdef S = {SYS_EULER2D, 4, gamma, 0.0};
    double L[4][4], R[4][4];
    int st = frame(&S, dir, UL, UR, L, R);
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            L16[a * 4 + b] = L[a][b];
            R16[a * 4 + b] = R[a][b];
        }
    return st;
}

/* Global Lax-Friedrichs alpha of a 1D state (exported for sampled checks). */
int or_alpha_1d(int sys, const double *U, int n, double gamma, double a, double *alpha_out) {
    sysdef S = {sys, nvars_of(sys), gamma, a};
    int bad = 0;
    *alpha_out = alpha_1d(&S, U, n, &bad);
    if (bad & 2) return OR_ENONFINITE;
    if (bad & 1) return OR_ENONPHYSICAL;
    return OR_OK;
}

/* Global Lax-Friedrichs alphas (x, y) of a 2D state (exported for sampled checks). */
int or_alpha_2d(const double *U, int nx, int ny, double gamma, double *alpha_out) {
    sysdef S = {SYS_EULER2D, 4, gamma, 0.0};
    int bad = 0;
    alpha_2d(&S, U, nx, ny, &alpha_out[0], &alpha_out[1], &bad);
    if (bad & 2) return OR_ENONFINITE;
    if (bad & 1) return OR_ENONPHYSICAL;
    return OR_OK;
}

/* ======================================================================== */
/* Tangent-linear (forward-mode) 1D right-hand side and SSP-RK3 step.        */
/*                                                                          */
/* The discrete adjoint of the scheme differentiates it with the stencil    */
/* selection (every Delta of both splits and all fields) and the global      */
/* Lax-Friedrichs alpha held at their values for the state: with those       */
/* frozen, L is a smooth function of U (Eq. app through the Roe frame of     */
/* Remark 3, the split fluxes and the fixed Table co2 polynomials).  This    */
/* section evaluates the directional derivative dL = (dL/dU) dU exactly, by  */
/* carrying every quantity as a dual number (value, derivative) through the  */
/* same operations, in the same order, as the primal code above; the value   */
/* parts therefore equal the primal results.  It is the reference the        */
/* hand-written GPU adjoint is checked against by the dot-product identity   */
/* <v, J u> = <J^T v, u>.  TENO7-ext, 1D systems.                            */
/* ======================================================================== */
typedef struct {
    double v, d;
} dual;

static dual dcst(double v) { return (dual){v, 0.0}; }
static dual dadd(dual a, dual b) { return (dual){a.v + b.v, a.d + b.d}; }
static dual dsub(dual a, dual b) { return (dual){a.v - b.v, a.d - b.d}; }
static dual dmul(dual a, dual b) { return (dual){a.v * b.v, a.d * b.v + a.v * b.d}; }
static dual dscale(double c, dual a) { return (dual){c * a.v, c * a.d}; }
static dual ddiv(dual a, dual b) {
    double q = a.v / b.v;
    return (dual){q, (a.d - q * b.d) / b.v};
}
static dual dsqrt(dual a) {
    double s = sqrt(a.v);
    return (dual){s, a.d / (2.0 * s)};
}

static void flux_tl(const sysdef *S, const dual *U, dual *F) {
    if (S->sys == SYS_ADVECTION) {
        F[0] = dscale(S->a, U[0]);
    } else if (S->sys == SYS_BURGERS) {
        F[0] = dmul(dscale(0.5, U[0]), U[0]);
    } else {
        dual u = ddiv(U[1], U[0]);
        dual p = dscale(S->gamma - 1.0, dsub(U[2], dmul(dscale(0.5, U[1]), u)));
        F[0] = U[1];
        F[1] = dadd(dmul(U[1], u), p);
        F[2] = dmul(u, dadd(U[2], p));
    }
}

/* Roe frame of the 1D Euler system (as frame() above) in dual numbers. */
static void frame_tl(const sysdef *S, const dual *UL, const dual *UR, dual L[3][3], dual R[3][3]) {
    if (S->m == 1) {
        L[0][0] = dcst(1.0);
        R[0][0] = dcst(1.0);
        return;
    }
    double gm = S->gamma - 1.0;
    dual rl = UL[0], rr = UR[0];
    dual ul = ddiv(UL[1], rl), ur = ddiv(UR[1], rr);
    dual pl = dscale(gm, dsub(UL[2], dmul(dscale(0.5, UL[1]), ul)));
    dual pr = dscale(gm, dsub(UR[2], dmul(dscale(0.5, UR[1]), ur)));
    dual Hl = ddiv(dadd(UL[2], pl), rl), Hr = ddiv(dadd(UR[2], pr), rr);
    dual sl = dsqrt(rl), sr = dsqrt(rr);
    dual ut = ddiv(dadd(dmul(sl, ul), dmul(sr, ur)), dadd(sl, sr));
    dual Ht = ddiv(dadd(dmul(sl, Hl), dmul(sr, Hr)), dadd(sl, sr));
    dual c2 = dscale(gm, dsub(Ht, dmul(dscale(0.5, ut), ut)));
    dual c = dsqrt(c2);
    dual b1 = ddiv(dcst(gm), c2);
    dual b2 = dmul(dmul(dscale(0.5, ut), ut), b1);
    dual uc = ddiv(ut, c), rc = ddiv(dcst(1.0), c);
    R[0][0] = dcst(1.0);
    R[0][1] = dcst(1.0);
    R[0][2] = dcst(1.0);
    R[1][0] = dsub(ut, c);
    R[1][1] = ut;
    R[1][2] = dadd(ut, c);
    R[2][0] = dsub(Ht, dmul(ut, c));
    R[2][1] = dmul(dscale(0.5, ut), ut);
    R[2][2] = dadd(Ht, dmul(ut, c));
    L[0][0] = dscale(0.5, dadd(b2, uc));
    L[0][1] = dscale(-0.5, dadd(dmul(b1, ut), rc));
    L[0][2] = dscale(0.5, b1);
    L[1][0] = dsub(dcst(1.0), b2);
    L[1][1] = dmul(b1, ut);
    L[1][2] = dscale(-1.0, b1);
    L[2][0] = dscale(0.5, dsub(b2, uc));
    L[2][1] = dscale(-0.5, dsub(dmul(b1, ut), rc));
    L[2][2] = dscale(0.5, b1);
}

static dual poly_tl(int m, const dual *v) {
    dual s = dcst(0.0);
    for (int t = 0; t < 7; t++) s = dadd(s, dscale(COEF[m][t], v[t]));
    return s;
}

/* One x sweep (as sweep() above) with the selection taken from masks
 * ([2][m][n+1] Delta codes of faces -1 .. n-1) instead of the cutoff. */
static void sweep_tl(const sysdef *S, dual **P, int n, double alpha, const uint8_t *masks, dual **Fh) {
    int m = S->m, np = n + 2 * NG;
    dual *Gp = (dual *)malloc(sizeof(dual) * m * np);
    dual *Gm = (dual *)malloc(sizeof(dual) * m * np);
    for (int l = 0; l < np; l++) {
        dual U[3], F[3];
        for (int c = 0; c < m; c++) U[c] = P[c][l];
        flux_tl(S, U, F);
        for (int c = 0; c < m; c++) {
            Gp[c * np + l] = dscale(0.5, dadd(F[c], dscale(alpha, U[c])));
            Gm[c * np + l] = dscale(0.5, dsub(F[c], dscale(alpha, U[c])));
        }
    }
    for (int i = -1; i <= n - 1; i++) {
        dual L[3][3], R[3][3], UL[3], UR[3], f[3];
        for (int c = 0; c < m; c++) {
            UL[c] = P[c][i + NG];
            UR[c] = P[c][i + 1 + NG];
        }
        frame_tl(S, UL, UR, L, R);
        for (int k = 0; k < m; k++) {
            int mp = or_select(masks[(0 * m + k) * (n + 1) + i + 1]);
            int mm = or_select(masks[(1 * m + k) * (n + 1) + i + 1]);
            if (mp < 0) mp = 11;
            if (mm < 0) mm = 11;
            dual vp[7], vm[7];
            for (int t = 0; t < 7; t++) {
                int lp = i - 3 + t + NG, lm = i + 4 - t + NG;
                dual sp = dmul(L[k][0], Gp[lp]), sm = dmul(L[k][0], Gm[lm]);
                for (int c = 1; c < m; c++) {
                    sp = dadd(sp, dmul(L[k][c], Gp[c * np + lp]));
                    sm = dadd(sm, dmul(L[k][c], Gm[c * np + lm]));
                }
                vp[t] = sp;
                vm[t] = sm;
            }
            f[k] = dadd(poly_tl(mp, vp), poly_tl(mm, vm));
        }
        for (int c = 0; c < m; c++) {
            dual s = dmul(R[c][0], f[0]);
            for (int k = 1; k < m; k++) s = dadd(s, dmul(R[c][k], f[k]));
            Fh[c][i + 1] = s;
        }
    }
    free(Gp);
    free(Gm);
}

/* L(U) and dL = (dL/dU) dU with alpha and the selection (masks, as returned
 * by or_rhs_1d for U) frozen.  U, dU, L, dL: [m][n]. */
int or_rhs_1d_tl(int sys, const double *U, const double *dU, int n, double dx, double gamma, double a, int bc_lo,
                 int bc_hi, double alpha, const uint8_t *masks, double *L, double *dL) {
    if (n < 1 || !check_sys(sys, bc_lo, bc_hi) || !(dx > 0.0) || !masks || g_scheme != SCHEME_TENO7EXT ||
        g_alpha_mode)
        return OR_EINVAL;
    sysdef S = {sys, nvars_of(sys), gamma, a};
    int m = S.m, np = n + 2 * NG;
    dual *P[3], *Fh[3];
    for (int c = 0; c < m; c++) {
        P[c] = (dual *)malloc(sizeof(dual) * np);
        Fh[c] = (dual *)malloc(sizeof(dual) * (n + 1));
        for (int l = -NG; l < n + NG; l++) {
            int q = c * n + ghost_index(l, n, bc_lo, bc_hi);
            P[c][l + NG] = (dual){U[q], dU[q]};
        }
    }
    sweep_tl(&S, P, n, alpha, masks, Fh);
    for (int c = 0; c < m; c++)
        for (int i = 0; i < n; i++) {
            dual r = ddiv(dsub(Fh[c][i], Fh[c][i + 1]), dcst(dx));
            L[c * n + i] = r.v;
            dL[c * n + i] = r.d;
        }
    for (int c = 0; c < m; c++) {
        free(P[c]);
        free(Fh[c]);
    }
    return OR_OK;
}

/* One SSP-RK3 step of fixed dt (as or_rk3_step_1d) with its tangent: U and
 * dU advance in place; each stage's alpha and selection are those of the
 * primal stage state (computed by or_rhs_1d) and are not differentiated. */
int or_rk3_step_1d_tl(int sys, double *U, double *dU, int n, double dx, double gamma, double a, double CT,
                      double eps, int bc_lo, int bc_hi, double dt) {
    if (n < 1 || !check_sys(sys, bc_lo, bc_hi) || g_scheme != SCHEME_TENO7EXT) return OR_EINVAL;
    int m = nvars_of(sys), N = m * n, status = OR_OK;
    double *X[2], *dX[2], *r = (double *)malloc(sizeof(double) * N), *dr = (double *)malloc(sizeof(double) * N);
    uint8_t *masks = (uint8_t *)malloc(2 * m * (n + 1));
    for (int k = 0; k < 2; k++) {
        X[k] = (double *)malloc(sizeof(double) * N);
        dX[k] = (double *)malloc(sizeof(double) * N);
    }
    const double *stage_in[3] = {U, X[0], X[1]}, *dstage_in[3] = {dU, dX[0], dX[1]};
    for (int s = 0; s < 3; s++) {
        double alpha = 0.0;
        int st = or_rhs_1d(sys, stage_in[s], n, dx, gamma, a, CT, eps, bc_lo, bc_hi, -1.0, r, masks, &alpha);
        if (st) status = st;
        or_rhs_1d_tl(sys, stage_in[s], dstage_in[s], n, dx, gamma, a, bc_lo, bc_hi, alpha, masks, r, dr);
        for (int q = 0; q < N; q++) {
            /* the Shu-Osher stages, in the primal's expression order */
            dual u = {stage_in[s][q], dstage_in[s][q]}, u0 = {U[q], dU[q]}, rr = {r[q], dr[q]}, o;
            if (s == 0)
                o = dadd(u, dscale(dt, rr));
            else if (s == 1)
                o = dadd(dscale(0.75, u0), dscale(0.25, dadd(u, dscale(dt, rr))));
            else
                o = dadd(dscale(1.0 / 3.0, u0), dscale(2.0 / 3.0, dadd(u, dscale(dt, rr))));
            if (s < 2) {
                X[s][q] = o.v;
                dX[s][q] = o.d;
            } else {
                r[q] = o.v; /* U is still read by later q as u0: keep the result aside */
                dr[q] = o.d;
            }
        }
        if (s == 2) {
            memcpy(U, r, sizeof(double) * N);
            memcpy(dU, dr, sizeof(double) * N);
        }
    }
    for (int k = 0; k < 2; k++) {
        free(X[k]);
        free(dX[k]);
    }
    free(r);
    free(dr);
    free(masks);
    return status;
}

/* nsteps tangent-linear RK3 steps of fixed dt (U, dU in place). */
int or_run_1d_tl(int sys, double *U, double *dU, int n, double dx, double gamma, double a, double CT, double eps,
                 int bc_lo, int bc_hi, double dt, int nsteps) {
    int status = OR_OK;
    for (int s = 0; s < nsteps; s++) {
        int st = or_rk3_step_1d_tl(sys, U, dU, n, dx, gamma, a, CT, eps, bc_lo, bc_hi, dt);
        if (st) {
            status = st;
            break;
        }
    }
    return status;
}
