/*
 * goc_oracle.c -- plain FP64 CPU oracle of the GOC-LBM (test infrastructure).
 *
 * This file is TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and
 * the cpu_baseline / reference leg of bench.py may load it.  It shares no code,
 * header, table or constant with the CUDA library; the library never calls it.
 *
 * What it computes (one time step, Appendix E "Summary of the Algorithmic
 * Steps of the Central Moment GOC-LBM", plus Appendix G for the magnetic
 * induction equation), in the paper's order:
 *   Step 7 of the previous step (update hydrodynamic fields) is done first:
 *     rho = sum f / (h1 h2); U1 = (sum f e1 + F1/2)/(rho h2);
 *     U2 = (sum f e2 + F2/2)/(rho h1), with F the effective force stored by
 *     the previous step (F = 0 before the first step).
 *   App. G Step 5: h1 h2 B = sum g - Y/2 (Eq. 13_C, a 2x2 solve when Y != 0).
 *   Step 1: raw moments m = P f (Eq. Q-momentbasis, by the definition
 *     k'_mn = sum f e1^m e2^n).
 *   Step 2: central moments m^c = F(U) m (Eq. Fmatrix).
 *   Step 3: collision -- second-order finite differences of U1, U2, rho
 *     (normal derivatives only), normal stresses (Eq. viscousstress_OCC_
 *     modified3, Eq. tauc), local shear stress (Eq. shearlocallocalcomputation),
 *     effective force (Eq. bodyforce1/2; the external part includes the
 *     Lorentz force of Eq. Lorentzforce-GOC), central-moment sources
 *     (Eq. cmsourcesGOC), equilibria (Eq. cmequilibriaGOC) with corrections
 *     (Eq. cmeqcorrections, Eqs. 82-85), relaxation, split of k2s/k2d.
 *   Step 4: m~ = F(-U) m~^c.   Step 5: f~ = P^-1 m~.
 *   Step 6: streaming with boundary conditions (half-way bounce-back,
 *     momentum-augmented moving wall, Eq. 101/103; MIE anti-bounce-back).
 *   Alternative Steps 1-5 (Appendix D, orc_set_collision 2): the raw-moment
 *     MRT -- relaxation of m = P f in the combined basis towards Eq.
 *     GOCmomentequilibria with the same corrections, sources of Eq.
 *     GOCmomentsources, f~ = P^-1 m~ through the printed expansion.
 *   Alternative Steps 1-5 (Appendix F, orc_set_collision 1): the SRT collision in
 *     velocity space, f~ = f + (f^eq - f)/tau + (1 - 1/(2 tau)) S with f^eq and S
 *     from the raw moments of Eq. 14D / Eq. 14D-source through the printed
 *     expansions of Q^-1 (Eq. feqGOCLBE, Eq. SGOCLBE); stresses and force as
 *     above with zeta = nu.
 *   App. G Steps 1-3: local dB (Eqs. gradB1/gradB2), equilibria
 *     (Eq. EDF-MIE-base + Eq. 42_C), SRT collision (Eq. 12_C) with source
 *     S = -W Y (Eq. 8a_C); current density (Eq. currentdensity-GOC).
 *
 * Readings where the paper is silent, garbled or inconsistent (each is fixed
 * the same way in the CUDA path):
 *   - F in the velocity update is the force of the previous step (lagged);
 *     the first step uses F = 0.
 *   - q21, q12 take the sign of the binomial transform of the raw equilibria
 *     (q21 = (1-h2)(h1-1)^2/h1, q12 = (1-h1)(h2-1)^2/h2); the printed
 *     coefficients have the opposite sign.  Flag q3_printed selects the
 *     printed ones.
 *   - C4's theta21 bracket uses h2/h1 and its theta12 bracket h1/h2 (as in
 *     E4, Eq. 66b, and the SRT copy, Appendix F); the printed C4 swaps them.
 *   - The inverse frame map is m = F(-U) m^c (the printed Step 4 swaps primes).
 *   - Finite differences: central in the interior and across periodic
 *     boundaries; one-sided second order at the first/last fluid node of a
 *     wall axis.
 *   - Moving wall: rho_w is the density of the fluid node at the time of the
 *     outgoing population; the wall term applies to every link that crosses
 *     a moving wall (corner diagonals included).
 *
 * Weakest pins: the terms proportional to U1 theta21 and U2 theta12 vanish
 * in every flow with a closed-form answer available here (Taylor-Couette
 * flow and its transpose have no radial velocity and theta12 = 0, resp.
 * theta21 = 0).  tau^c (Eq. tauc, one function for the stresses and the
 * corrections) is pinned against the curvature part of the strain-rate
 * tensor the paper defines with its NSE in GOC; the other such terms of C3,
 * C4 (Eqs. 83/85) only against the paper's other printed forms of the
 * corrections (Eq. 79 with Eqs. 63b/66b; at zeta = nu, the SRT coefficients
 * of Appendix F), and their index placement by the spiral-grid reflection
 * pin.
 *
 * Layout: node n = j*nx + i (i along xi1, j along xi2); populations f[a*N+n];
 * vector populations g[(c*5+a)*N+n] for component c = 0 (B1), 1 (B2).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- lattices (Eq. 1a/1b for D2Q9, Eq. D2Q5a/b for D2Q5) ---------------- */
static const int E1[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int E2[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const int G1[5] = {0, 1, 0, -1, 0};
static const int G2[5] = {0, 0, 1, 0, -1};
static const int GOPP[5] = {0, 3, 4, 1, 2};
/* exponents (m, n) of the bare moment vector (k00,k10,k01,k20,k02,k11,k21,k12,k22) */
static const int MX[9] = {0, 1, 0, 2, 0, 1, 2, 1, 2};
static const int MY[9] = {0, 0, 1, 0, 2, 1, 1, 2, 2};

enum { W_WALL = 0, E_WALL = 1, S_WALL = 2, N_WALL = 3 };

typedef struct {
    int nx, ny, N;
    /* metric per node */
    double *h1, *h2, *t11, *t12, *t21, *t22;
    /* wall metric: for W/E arrays over j, for S/N arrays over i: (h1, h2) */
    double *wh1[4], *wh2[4];
    int wall[4];          /* 0 periodic, 1 wall */
    double uwall[4];      /* tangential wall velocity (S/N: along xi1, W/E: along xi2) */
    double bwall[4][2];   /* MIE wall field (B1, B2) */
    /* parameters */
    double cs2, nu, zeta, om[9], fext1, fext2;
    int gi;               /* 1: full corrections of Eqs. 83/85; 0: cubic GI terms dropped */
    int q3_printed;       /* 1: use the printed q21/q12 signs */
    int mhd;
    int srt;              /* 1: the SRT collision in velocity space (Appendix F) */
    int raw;              /* 1: the raw-moment MRT collision (Appendix D) */
    double csm2, taum, eta, mum;
    /* state */
    double *f, *ft;       /* populations (post-streaming) and post-collision */
    double *F1, *F2;      /* effective force of the previous step */
    double *g, *gt;       /* vector populations (post-streaming), post-collision */
    /* macroscopic fields of the current step */
    double *rho, *U1, *U2, *B1, *B2;
    double *dU1, *dU2, *dr1, *dr2;   /* normal derivatives */
    double *FL1, *FL2, *J3;
    double *dB;           /* [4][N] dB1/dxi1, dB2/dxi1, dB1/dxi2, dB2/dxi2 of the last step (diagnostic) */
    /* P and P^-1 */
    double P[9][9], Pinv[9][9];
    int nthreads;
} orc_t;

/* ---- small linear algebra ---------------------------------------------- */
static void matvec9(double A[9][9], const double *x, double *y) {
    for (int r = 0; r < 9; r++) {
        double s = 0.0;
        for (int c = 0; c < 9; c++) s += A[r][c] * x[c];
        y[r] = s;
    }
}

/* Gauss-Jordan inverse with partial pivoting; returns 0 on success. */
static int invert9(double A[9][9], double Ai[9][9]) {
    double M[9][18];
    for (int r = 0; r < 9; r++)
        for (int c = 0; c < 18; c++) M[r][c] = c < 9 ? A[r][c] : (c - 9 == r ? 1.0 : 0.0);
    for (int c = 0; c < 9; c++) {
        int p = c;
        for (int r = c + 1; r < 9; r++)
            if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
        if (fabs(M[p][c]) < 1e-300) return -1;
        if (p != c)
            for (int k = 0; k < 18; k++) { double t = M[p][k]; M[p][k] = M[c][k]; M[c][k] = t; }
        double d = M[c][c];
        for (int k = 0; k < 18; k++) M[c][k] /= d;
        for (int r = 0; r < 9; r++) {
            if (r == c) continue;
            double s = M[r][c];
            if (s != 0.0)
                for (int k = 0; k < 18; k++) M[r][k] -= s * M[c][k];
        }
    }
    for (int r = 0; r < 9; r++)
        for (int c = 0; c < 9; c++) Ai[r][c] = M[r][c + 9];
    return 0;
}

static double ipow(int e, int p) {
    double r = 1.0;
    for (int k = 0; k < p; k++) r *= (double)e;
    return r;
}

/* Frame transformation matrix F(U1, U2) as printed (Eq. Fmatrix); rows and
 * columns in the bare order (k00,k10,k01,k20,k02,k11,k21,k12,k22).  The
 * printed matrix is in the combined (2s, 2d) rows/columns for indices 3, 4;
 * here it is converted to the bare order: F_bare = B^-1 F_printed B. */
static void frame_matrix(double u, double v, double Fb[9][9]) {
    double Fp[9][9];
    memset(Fp, 0, sizeof Fp);
    Fp[0][0] = 1;
    Fp[1][0] = -u; Fp[1][1] = 1;
    Fp[2][0] = -v; Fp[2][2] = 1;
    Fp[3][0] = u * u + v * v; Fp[3][1] = -2 * u; Fp[3][2] = -2 * v; Fp[3][3] = 1;
    Fp[4][0] = u * u - v * v; Fp[4][1] = -2 * u; Fp[4][2] = 2 * v; Fp[4][4] = 1;
    Fp[5][0] = u * v; Fp[5][1] = -v; Fp[5][2] = -u; Fp[5][5] = 1;
    Fp[6][0] = -u * u * v; Fp[6][1] = 2 * u * v; Fp[6][2] = u * u;
    Fp[6][3] = -0.5 * v; Fp[6][4] = -0.5 * v; Fp[6][5] = -2 * u; Fp[6][6] = 1;
    Fp[7][0] = -u * v * v; Fp[7][1] = v * v; Fp[7][2] = 2 * u * v;
    Fp[7][3] = -0.5 * u; Fp[7][4] = 0.5 * u; Fp[7][5] = -2 * v; Fp[7][7] = 1;
    Fp[8][0] = u * u * v * v; Fp[8][1] = -2 * u * v * v; Fp[8][2] = -2 * u * u * v;
    Fp[8][3] = 0.5 * (u * u + v * v); Fp[8][4] = 0.5 * (v * v - u * u);
    Fp[8][5] = 4 * u * v; Fp[8][6] = -2 * v; Fp[8][7] = -2 * u; Fp[8][8] = 1;
    /* B: combined = B bare (rows 3,4: k2s = k20+k02, k2d = k20-k02) */
    double B[9][9], Bi[9][9], T[9][9];
    memset(B, 0, sizeof B);
    memset(Bi, 0, sizeof Bi);
    for (int k = 0; k < 9; k++) { B[k][k] = 1; Bi[k][k] = 1; }
    B[3][3] = 1; B[3][4] = 1; B[4][3] = 1; B[4][4] = -1;
    Bi[3][3] = 0.5; Bi[3][4] = 0.5; Bi[4][3] = 0.5; Bi[4][4] = -0.5;
    for (int r = 0; r < 9; r++)
        for (int c = 0; c < 9; c++) {
            double s = 0;
            for (int k = 0; k < 9; k++) s += Fp[r][k] * B[k][c];
            T[r][c] = s;
        }
    for (int r = 0; r < 9; r++)
        for (int c = 0; c < 9; c++) {
            double s = 0;
            for (int k = 0; k < 9; k++) s += Bi[r][k] * T[k][c];
            Fb[r][c] = s;
        }
}

/* ---- construction ------------------------------------------------------- */
static double *dup(const double *src, int n) {
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    if (src) memcpy(p, src, sizeof(double) * (size_t)n);
    else memset(p, 0, sizeof(double) * (size_t)n);
    return p;
}

orc_t *orc_create(int nx, int ny,
                  const double *h1, const double *h2, const double *t11,
                  const double *t12, const double *t21, const double *t22,
                  const int *wall, const double *uwall,
                  const double *wall_h1, const double *wall_h2,
                  double cs2, double nu, double zeta, const double *om,
                  double fext1, double fext2, int gi, int q3_printed,
                  int mhd, double csm2, double taum, double mum,
                  const double *bwall, int nthreads) {
    /* wall_h1, wall_h2: concatenation W(ny), E(ny), S(nx), N(nx) */
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    int N = nx * ny;
    o->nx = nx; o->ny = ny; o->N = N;
    o->h1 = dup(h1, N); o->h2 = dup(h2, N);
    o->t11 = dup(t11, N); o->t12 = dup(t12, N);
    o->t21 = dup(t21, N); o->t22 = dup(t22, N);
    int off = 0;
    for (int w = 0; w < 4; w++) {
        int len = (w < 2) ? ny : nx;
        o->wh1[w] = dup(wall_h1 + off, len);
        o->wh2[w] = dup(wall_h2 + off, len);
        off += len;
        o->wall[w] = wall[w];
        o->uwall[w] = uwall[w];
        o->bwall[w][0] = bwall[2 * w];
        o->bwall[w][1] = bwall[2 * w + 1];
    }
    o->cs2 = cs2; o->nu = nu; o->zeta = zeta;
    for (int k = 0; k < 9; k++) o->om[k] = om[k];
    o->fext1 = fext1; o->fext2 = fext2;
    o->gi = gi; o->q3_printed = q3_printed;
    o->mhd = mhd; o->csm2 = csm2; o->taum = taum; o->mum = mum;
    o->eta = csm2 * (taum - 0.5);   /* Eq. magneticresistivity */
    o->f = dup(NULL, 9 * N); o->ft = dup(NULL, 9 * N);
    o->F1 = dup(NULL, N); o->F2 = dup(NULL, N);
    o->g = dup(NULL, 10 * N); o->gt = dup(NULL, 10 * N);
    o->rho = dup(NULL, N); o->U1 = dup(NULL, N); o->U2 = dup(NULL, N);
    o->B1 = dup(NULL, N); o->B2 = dup(NULL, N);
    o->dU1 = dup(NULL, N); o->dU2 = dup(NULL, N);
    o->dr1 = dup(NULL, N); o->dr2 = dup(NULL, N);
    o->FL1 = dup(NULL, N); o->FL2 = dup(NULL, N); o->J3 = dup(NULL, N);
    o->dB = dup(NULL, 4 * N);
    /* P from its definition: row k is the monomial e1^MX e2^MY (Eq. Q-momentbasis) */
    for (int k = 0; k < 9; k++)
        for (int a = 0; a < 9; a++) o->P[k][a] = ipow(E1[a], MX[k]) * ipow(E2[a], MY[k]);
    invert9(o->P, o->Pinv);
    o->nthreads = nthreads > 0 ? nthreads : 1;
    return o;
}

void orc_destroy(orc_t *o) {
    if (!o) return;
    double *ptrs[] = {o->h1, o->h2, o->t11, o->t12, o->t21, o->t22, o->f, o->ft,
                      o->F1, o->F2, o->g, o->gt, o->rho, o->U1, o->U2, o->B1, o->B2,
                      o->dU1, o->dU2, o->dr1, o->dr2, o->FL1, o->FL2, o->J3, o->dB};
    for (size_t k = 0; k < sizeof ptrs / sizeof ptrs[0]; k++) free(ptrs[k]);
    for (int w = 0; w < 4; w++) { free(o->wh1[w]); free(o->wh2[w]); }
    free(o);
}

/* ---- finite differences (second order; central or one-sided at walls) -- */
static double d_xi1(const orc_t *o, const double *phi, int i, int j) {
    int nx = o->nx;
    const double *row = phi + (size_t)j * nx;
    int per = (o->wall[W_WALL] == 0);
    if (per) return 0.5 * (row[(i + 1) % nx] - row[(i - 1 + nx) % nx]);
    if (i == 0) return 0.5 * (-3.0 * row[0] + 4.0 * row[1] - row[2]);
    if (i == nx - 1) return 0.5 * (3.0 * row[nx - 1] - 4.0 * row[nx - 2] + row[nx - 3]);
    return 0.5 * (row[i + 1] - row[i - 1]);
}

static double d_xi2(const orc_t *o, const double *phi, int i, int j) {
    int nx = o->nx, ny = o->ny;
#define AT(jj) phi[(size_t)(jj) * nx + i]
    int per = (o->wall[S_WALL] == 0);
    if (per) return 0.5 * (AT((j + 1) % ny) - AT((j - 1 + ny) % ny));
    if (j == 0) return 0.5 * (-3.0 * AT(0) + 4.0 * AT(1) - AT(2));
    if (j == ny - 1) return 0.5 * (3.0 * AT(ny - 1) - 4.0 * AT(ny - 2) + AT(ny - 3));
    return 0.5 * (AT(j + 1) - AT(j - 1));
#undef AT
}

/* ---- equilibria --------------------------------------------------------- */

/* tau^c (Eq. tauc): the curvature part of the normal stresses. */
static void tau_c(double rho, double ze, double nu, double U1, double U2, double t12, double t21,
                  double *tc11, double *tc22) {
    *tc11 = rho * (ze + nu) * U2 * t12 + rho * (ze - nu) * U1 * t21;
    *tc22 = rho * (ze + nu) * U1 * t21 + rho * (ze - nu) * U2 * t12;
}

/* Normal-gradient corrections n3^eq(1), n4^eq(1) (Eqs. 82-85, Delta t = 1). */
static void corrections(const orc_t *o, double rho, double U1, double U2,
                        double h1, double h2, double t11, double t12, double t21, double t22,
                        double dU1, double dU2, double dr1, double dr2,
                        double *n3, double *n4) {
    double cs2 = o->cs2, nu = o->nu, ze = o->zeta;
    double gi = o->gi ? 1.0 : 0.0;
    double a1 = gi * U1 * U1 / cs2, a2 = gi * U2 * U2 / cs2;
    double tc11, tc22;
    tau_c(rho, ze, nu, U1, U2, t12, t21, &tc11, &tc22);
    double D31 = rho * (2 * ze - (ze + nu) * h2 / (h1 * h1) - (ze - nu) / h2
                        - ze * (2 - h2 / cs2 + (3 * a1 + 1) * h2 / (h1 * h1)));
    double D32 = rho * (2 * ze - (ze + nu) * h1 / (h2 * h2) - (ze - nu) / h1
                        - ze * (2 - h1 / cs2 + (3 * a2 + 1) * h1 / (h2 * h2)));
    double D33 = -ze * ((3 - a1) * h2 / (h1 * h1) - h2 / cs2 - a2 / h2) * U1;
    double D34 = -ze * ((3 - a2) * h1 / (h2 * h2) - h1 / cs2 - a1 / h1) * U2;
    double C3 = -(h2 / h1 * tc11 + h1 / h2 * tc22)
                - rho * ze * (-2 * U1 * (a1 + 1) * h2 / h1 * t11
                              - 2 * U2 * (a2 + 1) * h1 / h2 * t22
                              + U1 * ((3 + a1) * h2 / h1 + 2 * h1 / h2 - h1 * h2 / cs2) * t21
                              + U2 * ((3 + a2) * h1 / h2 + 2 * h2 / h1 - h1 * h2 / cs2) * t12);
    double D41 = rho * (2 * nu - (ze + nu) * h2 / (h1 * h1) + (ze - nu) / h2
                        - nu * (2 - h2 / cs2 + (3 * a1 + 1) * h2 / (h1 * h1)));
    double D42 = rho * (-2 * nu + (ze + nu) * h1 / (h2 * h2) - (ze - nu) / h1
                        - nu * (-2 + h1 / cs2 - (3 * a2 + 1) * h1 / (h2 * h2)));
    double D43 = -nu * ((3 - a1) * h2 / (h1 * h1) - h2 / cs2 + a2 / h2) * U1;
    double D44 = -nu * (-(3 - a2) * h1 / (h2 * h2) + h1 / cs2 - a1 / h1) * U2;
    double C4 = -(h2 / h1 * tc11 - h1 / h2 * tc22)
                - rho * nu * (-2 * U1 * (a1 + 1) * h2 / h1 * t11
                              + 2 * U2 * (a2 + 1) * h1 / h2 * t22
                              + U1 * ((3 + a1) * h2 / h1 - 2 * h1 / h2 - h1 * h2 / cs2) * t21
                              + U2 * (-(3 + a2) * h1 / h2 + 2 * h2 / h1 + h1 * h2 / cs2) * t12);
    *n3 = D31 * dU1 + D32 * dU2 + D33 * dr1 + D34 * dr2 + C3;
    *n4 = D41 * dU1 + D42 * dU2 + D43 * dr1 + D44 * dr2 + C4;
}

/* Central-moment equilibria (Eq. cmequilibriaGOC) in the bare order, with the
 * corrections added to k2s, k2d (Eq. cmeqcorrections). */
static void central_equilibria(const orc_t *o, double rho, double U1, double U2,
                               double h1, double h2, double n3, double n4, double *keq) {
    double cs2 = o->cs2;
    double q20 = h2 / h1 * (h1 - 1) * (h1 - 1);
    double q02 = h1 / h2 * (h2 - 1) * (h2 - 1);
    double q11 = (h1 - 1) * (h2 - 1);
    double q21 = (1 - h2) * (h1 - 1) * (h1 - 1) / h1;
    double q12 = (1 - h1) * (h2 - 1) * (h2 - 1) / h2;
    if (o->q3_printed) { q21 = -q21; q12 = -q12; }
    double k2s = q20 * rho * U1 * U1 + q02 * rho * U2 * U2 + (h2 / h1 + h1 / h2) * rho * cs2 + n3;
    double k2d = q20 * rho * U1 * U1 - q02 * rho * U2 * U2 + (h2 / h1 - h1 / h2) * rho * cs2 + n4;
    keq[0] = h1 * h2 * rho;
    keq[1] = (1 - h1) * h2 * rho * U1;
    keq[2] = (1 - h2) * h1 * rho * U2;
    keq[3] = 0.5 * (k2s + k2d);
    keq[4] = 0.5 * (k2s - k2d);
    keq[5] = q11 * rho * U1 * U2;
    keq[6] = q21 * rho * U1 * U1 * U2 + (1 - h2) * rho * cs2 * U2 / h1;
    keq[7] = q12 * rho * U1 * U2 * U2 + (1 - h1) * rho * cs2 * U1 / h2;
    keq[8] = cs2 * cs2 * rho;
}

/* Raw-moment equilibria with corrections (Eq. GOCmomentequilibria + n^eq(1)),
 * bare order; used for the initial state (Appendix C.1) and wall terms. */
static void raw_equilibria(const orc_t *o, double rho, double U1, double U2,
                           double h1, double h2, double n3, double n4, double *m) {
    double cs2 = o->cs2, P = rho * cs2;
    double k2s = h2 / h1 * rho * U1 * U1 + h1 / h2 * rho * U2 * U2 + (h2 / h1 + h1 / h2) * P + n3;
    double k2d = h2 / h1 * rho * U1 * U1 - h1 / h2 * rho * U2 * U2 + (h2 / h1 - h1 / h2) * P + n4;
    m[0] = h1 * h2 * rho;
    m[1] = h2 * rho * U1;
    m[2] = h1 * rho * U2;
    m[3] = 0.5 * (k2s + k2d);
    m[4] = 0.5 * (k2s - k2d);
    m[5] = rho * U1 * U2;
    m[6] = rho * (cs2 + U1 * U1) * U2 / h1;
    m[7] = rho * (cs2 + U2 * U2) * U1 / h2;
    m[8] = rho * cs2 * cs2 + rho * cs2 * (U1 * U1 + U2 * U2) + rho * U1 * U1 * U2 * U2;
}

/* ---- SRT GOC-LBM (Appendix F, "GOC-LBM Based on Collisions in Velocity
 * Space and SRT") ---------------------------------------------------------- */

/* Raw-moment equilibria of Eq. 14D in the bare order: the base equilibria
 * with the bare second-moment corrections G_j (Eq. 5D) and H_j (Eq. 6D),
 * written for zeta = nu.  Readings: H_2 carries h1/h2^2 (the printed h1/h1^2
 * is garbled: H_2 = (D_32 - D_42)/2); the density-gradient coefficients are
 * taken from the appendix's definition G_j = (D_3j + D_4j)/2, H_j = (D_3j -
 * D_4j)/2, which keeps the U^2/c_s^2 parts of D_33, D_43, D_34, D_44: G_3 =
 * -nu[(3 - U1^2/cs2) h2/h1^2 - h2/cs2] U1, G_4 = nu (U1^2/cs2) U2/h1, H_3 =
 * nu (U2^2/cs2) U1/h2, H_4 = -nu[(3 - U2^2/cs2) h1/h2^2 - h1/cs2] U2 (its
 * simplified forms drop these cubic parts and print G_4 = H_3 = 0).  gi = 0
 * drops the U^2/c_s^2 terms as everywhere else. */
static void srt_equilibria(const orc_t *o, double rho, double U1, double U2,
                           double h1, double h2, double t11, double t12, double t21, double t22,
                           double dU1, double dU2, double dr1, double dr2, double *m) {
    double cs2 = o->cs2, nu = o->nu;
    double gi = o->gi ? 1.0 : 0.0;
    double a1 = gi * U1 * U1 / cs2, a2 = gi * U2 * U2 / cs2;
    double tc11 = 2 * rho * nu * U2 * t12, tc22 = 2 * rho * nu * U1 * t21;
    double G1 = rho * nu * (h2 / cs2 - 3 * (1 + a1) * h2 / (h1 * h1));
    double G3 = -nu * ((3 - a1) * h2 / (h1 * h1) - h2 / cs2) * U1;
    double G4 = nu * a1 * U2 / h1;
    double G5 = -h2 / h1 * tc11
                - rho * nu * (-2 * U1 * (a1 + 1) * h2 / h1 * t11
                              + U1 * ((3 + a1) * h2 / h1 - h1 * h2 / cs2) * t21
                              + 2 * U2 * h2 / h1 * t12);
    double H2 = rho * nu * (h1 / cs2 - 3 * (1 + a2) * h1 / (h2 * h2));
    double H3 = nu * a2 * U1 / h2;
    double H4 = -nu * ((3 - a2) * h1 / (h2 * h2) - h1 / cs2) * U2;
    double H5 = -h1 / h2 * tc22
                - rho * nu * (-2 * U2 * (a2 + 1) * h1 / h2 * t22
                              + U2 * ((3 + a2) * h1 / h2 - h1 * h2 / cs2) * t12
                              + 2 * U1 * h1 / h2 * t21);
    m[0] = rho * h1 * h2;
    m[1] = rho * U1 * h2;
    m[2] = rho * U2 * h1;
    m[3] = h2 / h1 * rho * (U1 * U1 + cs2) + G1 * dU1 + G3 * dr1 + G4 * dr2 + G5;   /* G2 = 0 */
    m[4] = h1 / h2 * rho * (U2 * U2 + cs2) + H2 * dU2 + H3 * dr1 + H4 * dr2 + H5;   /* H1 = 0 */
    m[5] = rho * U1 * U2;
    m[6] = rho * U2 / h1 * (cs2 + U1 * U1);
    m[7] = rho * U1 / h2 * (cs2 + U2 * U2);
    m[8] = rho * cs2 * cs2 + rho * cs2 * (U1 * U1 + U2 * U2) + rho * U1 * U1 * U2 * U2;
}

/* Raw moments (bare order k00, k10, k01, k20, k02, k11, k21, k12, k22) to
 * populations: the expansions of Q^-1 printed as Eq. feqGOCLBE / Eq. SGOCLBE. */
static void srt_to_populations(const double *k, double *f) {
    f[0] = k[0] - k[3] - k[4] + k[8];
    f[1] = 0.5 * (k[1] + k[3] - k[7] - k[8]);
    f[2] = 0.5 * (k[2] + k[4] - k[6] - k[8]);
    f[3] = 0.5 * (-k[1] + k[3] + k[7] - k[8]);
    f[4] = 0.5 * (-k[2] + k[4] + k[6] - k[8]);
    f[5] = 0.25 * (k[5] + k[6] + k[7] + k[8]);
    f[6] = 0.25 * (-k[5] + k[6] - k[7] + k[8]);
    f[7] = 0.25 * (k[5] - k[6] - k[7] + k[8]);
    f[8] = 0.25 * (-k[5] - k[6] + k[7] + k[8]);
}

/* ---- macroscopic fields ------------------------------------------------- */
static void update_fields(orc_t *o) {
    int N = o->N;
#pragma omp parallel for num_threads(o->nthreads) schedule(static)
    for (int n = 0; n < N; n++) {
        double k00 = 0, k10 = 0, k01 = 0;
        for (int a = 0; a < 9; a++) {
            double fa = o->f[(size_t)a * N + n];
            k00 += fa; k10 += fa * E1[a]; k01 += fa * E2[a];
        }
        double h1 = o->h1[n], h2 = o->h2[n];
        double rho = k00 / (h1 * h2);
        o->rho[n] = rho;
        o->U1[n] = (k10 + 0.5 * o->F1[n]) / (rho * h2);
        o->U2[n] = (k01 + 0.5 * o->F2[n]) / (rho * h1);
        if (o->mhd) {
            /* h1 h2 B_i = sum g_i - Y_i/2 with Y_1 = H (U2 B1 - B2 U1) t12,
             * Y_2 = H (U1 B2 - B1 U2) t21 (Eq. 6ab_C, Eq. 13_C): a 2x2 solve. */
            double G[2] = {0, 0};
            for (int c = 0; c < 2; c++)
                for (int a = 0; a < 5; a++) G[c] += o->g[((size_t)c * 5 + a) * N + n];
            double H = h1 * h2, u = o->U1[n], v = o->U2[n];
            double a11 = H * (1 + 0.5 * o->t12[n] * v), a12 = -0.5 * H * o->t12[n] * u;
            double a21 = -0.5 * H * o->t21[n] * v, a22 = H * (1 + 0.5 * o->t21[n] * u);
            double det = a11 * a22 - a12 * a21;
            o->B1[n] = (G[0] * a22 - a12 * G[1]) / det;
            o->B2[n] = (a11 * G[1] - a21 * G[0]) / det;
        }
    }
}

static void update_gradients(orc_t *o) {
    int nx = o->nx, ny = o->ny;
#pragma omp parallel for num_threads(o->nthreads) schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int n = j * nx + i;
            o->dU1[n] = d_xi1(o, o->U1, i, j);
            o->dr1[n] = d_xi1(o, o->rho, i, j);
            o->dU2[n] = d_xi2(o, o->U2, i, j);
            o->dr2[n] = d_xi2(o, o->rho, i, j);
        }
}

/* ---- MIE at one node (App. G Steps 1-3 and Step 5-6 quantities) -------- */
static double mie_W(const orc_t *o, int a) { return a == 0 ? 1.0 - 2.0 * o->csm2 : 0.5 * o->csm2; }

static void mie_node(orc_t *o, int n) {
    int N = o->N;
    double h1 = o->h1[n], h2 = o->h2[n], H = h1 * h2;
    double t11 = o->t11[n], t12 = o->t12[n], t21 = o->t21[n], t22 = o->t22[n];
    double U[2] = {o->U1[n], o->U2[n]}, B[2] = {o->B1[n], o->B2[n]};
    double csm2 = o->csm2, taum = o->taum, eta = o->eta;
    double dB1[2], dB2[2];   /* dB_i/dxi1, dB_i/dxi2 */
    double geq0[2][5];
    for (int c = 0; c < 2; c++) {
        /* A_ij = U_j B_i - B_j U_i (Eq. 2_C) */
        double Ai1 = U[0] * B[c] - B[0] * U[c];
        double Ai2 = U[1] * B[c] - B[1] * U[c];
        double L1 = 0, L2 = 0;
        for (int a = 0; a < 5; a++) {
            double W = mie_W(o, a);
            geq0[c][a] = W * (H * B[c] + G1[a] / csm2 * (h2 * Ai1) + G2[a] / csm2 * (h1 * Ai2));
            double gn = o->g[((size_t)c * 5 + a) * N + n] - geq0[c][a];
            L1 += G1[a] * gn;
            L2 += G2[a] * gn;
        }
        /* Eqs. gradB1 / gradB2 */
        dB1[c] = -(L1 + 0.5 * csm2 * h1 * h1 * h2 * (t11 + t21) * B[c])
                 / (csm2 * (0.5 * H + (taum - 0.5) * h2 / h1));
        dB2[c] = -(L2 + 0.5 * csm2 * h1 * h2 * h2 * (t22 + t12) * B[c])
                 / (csm2 * (0.5 * H + (taum - 0.5) * h1 / h2));
    }
    for (int c = 0; c < 2; c++) {   /* kept for the diagnostic accessor only */
        o->dB[(size_t)c * N + n] = dB1[c];
        o->dB[(size_t)(2 + c) * N + n] = dB2[c];
    }
    /* current density (Eq. currentdensity-GOC) and Lorentz force (Eq. Lorentzforce-GOC) */
    double J3 = (1.0 / o->mum) / H * (h2 * dB1[1] - h1 * dB2[0] + H * (B[1] * t21 - B[0] * t12));
    o->J3[n] = J3;
    o->FL1[n] = -J3 * B[1];
    o->FL2[n] = J3 * B[0];
    /* collision (Eq. 12_C) with g^eq = g^eq(0) + g^corr (Eq. 42_C), S = -W Y (Eq. 8a_C) */
    double Y[2];
    Y[0] = H * ((U[1] * B[0] - B[1] * U[0]) * t12);
    Y[1] = H * ((U[0] * B[1] - B[0] * U[1]) * t21);
    for (int c = 0; c < 2; c++) {
        double lc1 = eta * (H - h2 / h1) * dB1[c] + eta * h1 * h1 * h2 * (t11 + t21) * B[c];
        double lc2 = eta * (H - h1 / h2) * dB2[c] + eta * h1 * h2 * h2 * (t22 + t12) * B[c];
        for (int a = 0; a < 5; a++) {
            double W = mie_W(o, a);
            double geq = geq0[c][a] + W * (G1[a] / csm2 * lc1 + G2[a] / csm2 * lc2);
            double S = -W * Y[c];
            double gb = o->g[((size_t)c * 5 + a) * N + n];
            o->gt[((size_t)c * 5 + a) * N + n] = gb - (gb - geq) / taum + (1.0 - 0.5 / taum) * S;
        }
    }
}

/* ---- NSE collision at one node (App. E Steps 1-5) ----------------------- */
static void nse_node(orc_t *o, int n) {
    int N = o->N;
    double h1 = o->h1[n], h2 = o->h2[n];
    double t11 = o->t11[n], t12 = o->t12[n], t21 = o->t21[n], t22 = o->t22[n];
    double rho = o->rho[n], U1 = o->U1[n], U2 = o->U2[n];
    double dU1 = o->dU1[n], dU2 = o->dU2[n], dr1 = o->dr1[n], dr2 = o->dr2[n];
    double cs2 = o->cs2, nu = o->nu, ze = o->zeta, *om = o->om;
    double f[9], m[9], mc[9];
    for (int a = 0; a < 9; a++) f[a] = o->f[(size_t)a * N + n];
    /* Step 1: raw moments by definition */
    matvec9(o->P, f, m);
    /* Step 2: central moments */
    double Fm[9][9], Fi[9][9];
    frame_matrix(U1, U2, Fm);
    matvec9(Fm, m, mc);
    /* Step 3a-d: stresses and effective force */
    double P = rho * cs2;
    double tc11, tc22;
    tau_c(rho, ze, nu, U1, U2, t12, t21, &tc11, &tc22);
    double tau11 = rho * (ze + nu) / h1 * dU1 + rho * (ze - nu) / h2 * dU2 + tc11;
    double tau22 = rho * (ze + nu) / h2 * dU2 + rho * (ze - nu) / h1 * dU1 + tc22;
    double fx1 = o->fext1 + (o->mhd ? o->FL1[n] : 0.0);
    double fx2 = o->fext2 + (o->mhd ? o->FL2[n] : 0.0);
    double Ft1 = h2 * (fx1 + (t21 - t11) * P + t11 * (tau11 - rho * U1 * U1)
                       - 2 * t12 * rho * U1 * U2 - t21 * (tau22 - rho * U2 * U2));
    double Ft2 = h1 * (fx2 + (t12 - t22) * P + t22 * (tau22 - rho * U2 * U2)
                       - 2 * t21 * rho * U1 * U2 - t12 * (tau11 - rho * U1 * U1));
    double c5 = 1.0 - 0.5 * om[5];
    double tau12 = -c5 * (m[5] + 0.5 * (Ft1 * U2 / h2 + Ft2 * U1 / h1) - rho * U1 * U2)
                   / (1.0 + c5 * (t12 * U2 + t21 * U1));
    double F1 = Ft1 + 2 * h2 * t12 * tau12;
    double F2 = Ft2 + 2 * h1 * t21 * tau12;
    if (o->raw) {
        /* Appendix D Step 2e-h: raw sources (Eq. GOCmomentsources), base
         * equilibria (Eq. GOCmomentequilibria) with n3, n4 (Eqs. 82-85) on the
         * combined k2s, k2d, relaxation of the nine moments in the combined
         * basis, split back; Step 3: f~ = P^-1 m~ (its printed expansion) */
        double n3, n4, meq[9], sg[9] = {0};
        corrections(o, rho, U1, U2, h1, h2, t11, t12, t21, t22, dU1, dU2, dr1, dr2, &n3, &n4);
        raw_equilibria(o, rho, U1, U2, h1, h2, n3, n4, meq);
        sg[1] = F1;
        sg[2] = F2;
        sg[3] = 2 * F1 * U1 / h1;
        sg[4] = 2 * F2 * U2 / h2;
        sg[5] = F1 * U2 / h2 + F2 * U1 / h1;
        double nb[9], nq[9], ns[9], nt[9], mt[9], ft[9];
        for (int k = 0; k < 9; k++) { nb[k] = m[k]; nq[k] = meq[k]; ns[k] = sg[k]; }
        nb[3] = m[3] + m[4]; nb[4] = m[3] - m[4];
        nq[3] = meq[3] + meq[4]; nq[4] = meq[3] - meq[4];
        ns[3] = sg[3] + sg[4]; ns[4] = sg[3] - sg[4];
        for (int k = 0; k < 9; k++) nt[k] = nb[k] + om[k] * (nq[k] - nb[k]) + (1 - 0.5 * om[k]) * ns[k];
        for (int k = 0; k < 9; k++) mt[k] = nt[k];
        mt[3] = 0.5 * (nt[3] + nt[4]); mt[4] = 0.5 * (nt[3] - nt[4]);
        srt_to_populations(mt, ft);
        for (int a = 0; a < 9; a++) o->ft[(size_t)a * N + n] = ft[a];
        o->F1[n] = F1;
        o->F2[n] = F2;
        return;
    }
    if (o->srt) {
        /* Appendix F Step 1: f~ = f + (f^eq - f)/tau + (1 - 1/(2 tau)) S with
         * f^eq = Q^-1 m^eq (Eq. 14D) and S = Q^-1 Psi (Eq. 14D-source; sigma11
         * read as F1 U2/h2 + F2 U1/h1, the value of Eq. GOCmomentsources, the
         * printed factor 2 on F1 U2/h2 being garbled) */
        double meq[9], psi[9] = {0}, fe[9], sv[9];
        srt_equilibria(o, rho, U1, U2, h1, h2, t11, t12, t21, t22, dU1, dU2, dr1, dr2, meq);
        psi[1] = F1;
        psi[2] = F2;
        psi[3] = 2 * F1 * U1 / h1;
        psi[4] = 2 * F2 * U2 / h2;
        psi[5] = F1 * U2 / h2 + F2 * U1 / h1;
        srt_to_populations(meq, fe);
        srt_to_populations(psi, sv);
        double w = om[4];
        for (int a = 0; a < 9; a++)
            o->ft[(size_t)a * N + n] = f[a] + w * (fe[a] - f[a]) + (1 - 0.5 * w) * sv[a];
        o->F1[n] = F1;
        o->F2[n] = F2;
        return;
    }
    /* Step 3e: central-moment sources (Eq. cmsourcesGOC), bare order */
    double sig[9] = {0};
    sig[1] = F1; sig[2] = F2;
    double s2s = 2 * (1 / h1 - 1) * F1 * U1 + 2 * (1 / h2 - 1) * F2 * U2;
    double s2d = 2 * (1 / h1 - 1) * F1 * U1 - 2 * (1 / h2 - 1) * F2 * U2;
    sig[3] = 0.5 * (s2s + s2d); sig[4] = 0.5 * (s2s - s2d);
    sig[5] = (1 / h2 - 1) * F1 * U2 + (1 / h1 - 1) * F2 * U1;
    /* Step 3f: equilibria with corrections */
    double n3, n4, keq[9];
    corrections(o, rho, U1, U2, h1, h2, t11, t12, t21, t22, dU1, dU2, dr1, dr2, &n3, &n4);
    central_equilibria(o, rho, U1, U2, h1, h2, n3, n4, keq);
    /* Steps 3g-3i: relax in the combined basis (B), split back (B^-1) */
    double nc[9], neq[9], ns[9], nt[9];
    for (int k = 0; k < 9; k++) { nc[k] = mc[k]; neq[k] = keq[k]; ns[k] = sig[k]; }
    nc[3] = mc[3] + mc[4]; nc[4] = mc[3] - mc[4];
    neq[3] = keq[3] + keq[4]; neq[4] = keq[3] - keq[4];
    ns[3] = sig[3] + sig[4]; ns[4] = sig[3] - sig[4];
    for (int k = 0; k < 9; k++) nt[k] = nc[k] + om[k] * (neq[k] - nc[k]) + (1 - 0.5 * om[k]) * ns[k];
    double mct[9];
    for (int k = 0; k < 9; k++) mct[k] = nt[k];
    mct[3] = 0.5 * (nt[3] + nt[4]); mct[4] = 0.5 * (nt[3] - nt[4]);
    /* Step 4: back to raw moments with F(-U); Step 5: to populations with P^-1 */
    double mt[9], ft[9];
    frame_matrix(-U1, -U2, Fi);
    matvec9(Fi, mct, mt);
    matvec9(o->Pinv, mt, ft);
    for (int a = 0; a < 9; a++) o->ft[(size_t)a * N + n] = ft[a];
    o->F1[n] = F1;
    o->F2[n] = F2;
}

/* ---- streaming with boundary conditions (Step 6) ------------------------ */

/* f_b^eq(w) - f_bbar^eq(w) for an incoming direction b through a wall moving
 * tangentially with (u1, u2); only the odd raw moments contribute (Eq. 101). */
static double wall_term(const orc_t *o, int b, double rho, double u1, double u2,
                        double h1, double h2) {
    double m[9];
    raw_equilibria(o, rho, u1, u2, h1, h2, 0.0, 0.0, m);
    double fe[9];
    matvec9(((orc_t *)o)->Pinv, m, fe);
    return fe[b] - fe[OPP[b]];
}

static void stream(orc_t *o) {
    int nx = o->nx, ny = o->ny, N = o->N;
    double *fn = o->f;
    /* fn is rebuilt completely: every (node, direction) receives exactly one value */
#pragma omp parallel for num_threads(o->nthreads) schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int n = j * nx + i;
            for (int a = 0; a < 9; a++) {
                int ti = i + E1[a], tj = j + E2[a];
                int outx = (ti < 0 || ti >= nx), outy = (tj < 0 || tj >= ny);
                double val = o->ft[(size_t)a * N + n];
                if (outx && o->wall[W_WALL] == 0) { ti = (ti + nx) % nx; outx = 0; }
                if (outy && o->wall[S_WALL] == 0) { tj = (tj + ny) % ny; outy = 0; }
                if (!outx && !outy) {
                    fn[(size_t)a * N + (size_t)tj * nx + ti] = val;
                    continue;
                }
                /* half-way bounce-back into the opposite direction at this node */
                int b = OPP[a];
                double add = 0.0;
                if (outy) {
                    int w = (E2[a] < 0) ? S_WALL : N_WALL;
                    if (o->uwall[w] != 0.0)
                        add += wall_term(o, b, o->rho[n], o->uwall[w], 0.0,
                                         o->wh1[w][i], o->wh2[w][i]);
                }
                if (outx) {
                    int w = (E1[a] < 0) ? W_WALL : E_WALL;
                    if (o->uwall[w] != 0.0)
                        add += wall_term(o, b, o->rho[n], 0.0, o->uwall[w],
                                         o->wh1[w][j], o->wh2[w][j]);
                }
                fn[(size_t)b * N + n] = val + add;
            }
        }
    if (!o->mhd) return;
    double *gn = o->g;
#pragma omp parallel for num_threads(o->nthreads) schedule(static)
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int n = j * nx + i;
            for (int c = 0; c < 2; c++)
                for (int a = 0; a < 5; a++) {
                    int ti = i + G1[a], tj = j + G2[a];
                    int outx = (ti < 0 || ti >= nx), outy = (tj < 0 || tj >= ny);
                    double val = o->gt[((size_t)c * 5 + a) * N + n];
                    if (outx && o->wall[W_WALL] == 0) { ti = (ti + nx) % nx; outx = 0; }
                    if (outy && o->wall[S_WALL] == 0) { tj = (tj + ny) % ny; outy = 0; }
                    if (!outx && !outy) {
                        gn[((size_t)c * 5 + a) * N + (size_t)tj * nx + ti] = val;
                        continue;
                    }
                    /* anti-bounce-back with the imposed wall field (App. G.5) */
                    int w = outy ? ((G2[a] < 0) ? S_WALL : N_WALL) : ((G1[a] < 0) ? W_WALL : E_WALL);
                    int b = GOPP[a];
                    int k = (w < 2) ? j : i;
                    double hw = o->wh1[w][k] * o->wh2[w][k];
                    gn[((size_t)c * 5 + b) * N + n] = -val + 2.0 * mie_W(o, b) * hw * o->bwall[w][c];
                }
        }
}

/* ---- public entry points ------------------------------------------------ */

/* Initial state (Appendix C.1): f = P^-1 m^eq,eff(rho0, U0) with gradients by
 * the same finite differences; g = g^eq(0) + g^corr with dB by finite
 * differences of B0; stored force F = 0. */
void orc_init(orc_t *o, const double *rho0, const double *u10, const double *u20,
              const double *b10, const double *b20) {
    int N = o->N;
    memcpy(o->rho, rho0, sizeof(double) * N);
    memcpy(o->U1, u10, sizeof(double) * N);
    memcpy(o->U2, u20, sizeof(double) * N);
    if (o->mhd) {
        memcpy(o->B1, b10, sizeof(double) * N);
        memcpy(o->B2, b20, sizeof(double) * N);
    }
    update_gradients(o);
    for (int n = 0; n < N; n++) {
        double n3, n4, m[9], fe[9];
        corrections(o, o->rho[n], o->U1[n], o->U2[n], o->h1[n], o->h2[n], o->t11[n], o->t12[n],
                    o->t21[n], o->t22[n], o->dU1[n], o->dU2[n], o->dr1[n], o->dr2[n], &n3, &n4);
        raw_equilibria(o, o->rho[n], o->U1[n], o->U2[n], o->h1[n], o->h2[n], n3, n4, m);
        matvec9(o->Pinv, m, fe);
        for (int a = 0; a < 9; a++) o->f[(size_t)a * N + n] = fe[a];
        o->F1[n] = 0.0;
        o->F2[n] = 0.0;
    }
    if (!o->mhd) return;
    int nx = o->nx, ny = o->ny;
    for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
            int n = j * nx + i;
            double h1 = o->h1[n], h2 = o->h2[n], H = h1 * h2;
            double U[2] = {o->U1[n], o->U2[n]}, B[2] = {o->B1[n], o->B2[n]};
            const double *Bc[2] = {o->B1, o->B2};
            for (int c = 0; c < 2; c++) {
                double d1 = d_xi1(o, Bc[c], i, j), d2 = d_xi2(o, Bc[c], i, j);
                double Ai1 = U[0] * B[c] - B[0] * U[c], Ai2 = U[1] * B[c] - B[1] * U[c];
                double lc1 = o->eta * (H - h2 / h1) * d1 + o->eta * h1 * h1 * h2 * (o->t11[n] + o->t21[n]) * B[c];
                double lc2 = o->eta * (H - h1 / h2) * d2 + o->eta * h1 * h2 * h2 * (o->t22[n] + o->t12[n]) * B[c];
                for (int a = 0; a < 5; a++) {
                    double W = mie_W(o, a);
                    o->g[((size_t)c * 5 + a) * N + n] =
                        W * (H * B[c] + G1[a] / o->csm2 * (h2 * Ai1 + lc1) + G2[a] / o->csm2 * (h1 * Ai2 + lc2));
                }
            }
        }
}

/* Advance nsteps time steps. */
void orc_step(orc_t *o, int nsteps) {
    for (int s = 0; s < nsteps; s++) {
        update_fields(o);
        update_gradients(o);
        int N = o->N;
        if (o->mhd) {
#pragma omp parallel for num_threads(o->nthreads) schedule(static)
            for (int n = 0; n < N; n++) mie_node(o, n);
        }
#pragma omp parallel for num_threads(o->nthreads) schedule(static)
        for (int n = 0; n < N; n++) nse_node(o, n);
        stream(o);
    }
}

/* Macroscopic fields of the current state (rho, U with the stored force, B,
 * and, after orc_fields_full, the normal derivatives and the current density). */
void orc_fields(orc_t *o, double *rho, double *u1, double *u2, double *b1, double *b2) {
    update_fields(o);
    int N = o->N;
    if (rho) memcpy(rho, o->rho, sizeof(double) * N);
    if (u1) memcpy(u1, o->U1, sizeof(double) * N);
    if (u2) memcpy(u2, o->U2, sizeof(double) * N);
    if (o->mhd) {
        if (b1) memcpy(b1, o->B1, sizeof(double) * N);
        if (b2) memcpy(b2, o->B2, sizeof(double) * N);
    }
}

/* Raw state access for tests: populations, stored force, vector populations. */
void orc_get_state(const orc_t *o, double *f, double *F1, double *F2, double *g) {
    int N = o->N;
    if (f) memcpy(f, o->f, sizeof(double) * 9 * N);
    if (F1) memcpy(F1, o->F1, sizeof(double) * N);
    if (F2) memcpy(F2, o->F2, sizeof(double) * N);
    if (g && o->mhd) memcpy(g, o->g, sizeof(double) * 10 * N);
}

void orc_set_state(orc_t *o, const double *f, const double *F1, const double *F2, const double *g) {
    int N = o->N;
    if (f) memcpy(o->f, f, sizeof(double) * 9 * N);
    if (F1) memcpy(o->F1, F1, sizeof(double) * N);
    if (F2) memcpy(o->F2, F2, sizeof(double) * N);
    if (g && o->mhd) memcpy(o->g, g, sizeof(double) * 10 * N);
}

/* ---- single-node helpers exposed for the pin tests ---------------------- */
void orc_frame_matrix(double u, double v, double *out81) {
    double Fb[9][9];
    frame_matrix(u, v, Fb);
    memcpy(out81, Fb, sizeof Fb);
}

void orc_p_matrix(const orc_t *o, double *P81, double *Pinv81) {
    memcpy(P81, o->P, sizeof o->P);
    memcpy(Pinv81, o->Pinv, sizeof o->Pinv);
}

void orc_central_equilibria(const orc_t *o, double rho, double U1, double U2,
                            double h1, double h2, double n3, double n4, double *keq) {
    central_equilibria(o, rho, U1, U2, h1, h2, n3, n4, keq);
}

void orc_raw_equilibria(const orc_t *o, double rho, double U1, double U2,
                        double h1, double h2, double n3, double n4, double *m) {
    raw_equilibria(o, rho, U1, U2, h1, h2, n3, n4, m);
}

void orc_corrections(const orc_t *o, double rho, double U1, double U2, double h1, double h2,
                     double t11, double t12, double t21, double t22,
                     double dU1, double dU2, double dr1, double dr2, double *n34) {
    corrections(o, rho, U1, U2, h1, h2, t11, t12, t21, t22, dU1, dU2, dr1, dr2, &n34[0], &n34[1]);
}

/* Collision: 0 central-moment MRT (Appendix E), 1 SRT (Appendix F; the caller
 * passes zeta = nu and all rates 1/tau at creation), 2 raw-moment MRT
 * (Appendix D). */
void orc_set_collision(orc_t *o, int kind) {
    o->srt = kind == 1;
    o->raw = kind == 2;
}

void orc_srt_equilibria(const orc_t *o, double rho, double U1, double U2, double h1, double h2,
                        double t11, double t12, double t21, double t22,
                        double dU1, double dU2, double dr1, double dr2, double *m) {
    srt_equilibria(o, rho, U1, U2, h1, h2, t11, t12, t21, t22, dU1, dU2, dr1, dr2, m);
}

void orc_srt_to_populations(const double *k, double *f) { srt_to_populations(k, f); }

/* Per-node diagnostics of the last orc_step's MIE part (J3, Lorentz force). */
void orc_mie_diag(const orc_t *o, double *J3, double *FL1, double *FL2) {
    int N = o->N;
    if (J3) memcpy(J3, o->J3, sizeof(double) * N);
    if (FL1) memcpy(FL1, o->FL1, sizeof(double) * N);
    if (FL2) memcpy(FL2, o->FL2, sizeof(double) * N);
}

/* The local gradients of B (Eqs. gradB1 / gradB2) the last orc_step used:
 * [4][ny][nx] dB1/dxi1, dB2/dxi1, dB1/dxi2, dB2/dxi2. */
void orc_mie_grad(const orc_t *o, double *dB) {
    if (dB && o->mhd) memcpy(dB, o->dB, sizeof(double) * 4 * o->N);
}

int orc_threads(const orc_t *o) { return o->nthreads; }
