/*
 * olb_oracle.c -- plain FP64 CPU oracle for one time step of the
 * two-dimensional off-lattice Boltzmann model for van der Waals fluids
 * with variable temperature (Busuioc, Ambrus, Biciusca, Sofonea,
 * arXiv:1702.01690).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. It shares no code,
 * header, table or constant generator with the CUDA path: every constant
 * below is derived here from the closed forms that the paper prints.
 *
 * The code is deliberately naive: unblocked loops over nodes, one quantity
 * at a time, in the order in which the paper states the method:
 *
 *   per stage of the TVD RK-3 integrator (Sec. 3.1, Eq. rk3):
 *     moments n, u, T (Sec. 2.2; T from the trace of Eq. sigmaq_def)
 *     Delta p = n T - p^w (Eq. vdw, Sec. 3.3)
 *     49-point gradient and gradient-of-Laplacian (Eqs. stencil_grad,
 *       stencil_glap) with the field reflection rule (Sec. 3.4.3)
 *     force F (Eq. F_def)
 *     diffuse-wall density n_w (Eqs. diffuse_flux, nw; Sec. 3.4.2)
 *     ghost populations of specular sides (Sec. 3.4.1) and diffuse walls
 *     WENO-5 fluxes (Eqs. weno5_flux, weno5_omega, weno5_delta,
 *       weno5_sigma, Table tab:weno)
 *     momentum-space derivative (Eq. derf), equilibrium (Eqs. feq, g_alpha)
 *     L[f] (Eq. ecast) and the Shu-Osher combination.
 *
 * Readings of points the paper leaves open:
 *   R1  gradient-of-Laplacian coefficients c1, c4 are misprinted; this file
 *       uses c1 = -17/2160, c4 = -59/540, the unique values that make the
 *       stencil 4th-order exact and reproduce the paper's 1-D reduction
 *       (-1/8, 1, -13/8) of Sec. 4.  Column 0 of the printed matrix is the
 *       offset l = +3 (fixed by that reduction).
 *   R3  WENO weights: if any indicator vanishes, Table tab:weno; otherwise
 *       w~_q = delta_q (s/sigma_q)^2 with s = min sigma_q, which is
 *       delta_q/sigma_q^2 times the common factor s^2 and cannot overflow.
 *   R4  negative velocities use the mirror-image stencil.
 *   R5  the left wall is the mirror image of the right wall of Sec. 3.4.2.
 *   R6  the numerator of Eq. nw is the WENO flux at the wall face built
 *       with the extrapolated ghosts; the flux includes the factor p/m.
 *   R7  field reflection is even about the wall or specular face (a double
 *       reflection at corners); periodic sides wrap modulo the grid size
 *       (which may be smaller than the stencil).
 *   R13 specular reflection, written for the bottom and left sides only,
 *       applies to the top and right sides as their mirror image; x and y
 *       sides are specular or periodic independently, and a specular x = 0
 *       side may face a diffuse wall at x = nx ds (the paper's half channel).
 *   R8  T = (sum |p|^2 f / n - |u|^2) / 2 (D = 2, m = 1).
 *
 * Units: m = 1 (Sec. 2.1).  Node (i, j), 0-based, sits at
 * x = (i + 1/2) ds, y = (j + 1/2) ds (Sec. 3.4).  Populations are indexed
 * kappa = 5*k1 + k2, k1 the x-index and k2 the y-index of the velocity,
 * 0..4 in ascending order of the root.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 5
#define K 25

/* ------------------------------------------------------------------ */
/* Quadrature (Table trots, Sec. 2.2)                                  */
/* ------------------------------------------------------------------ */

static double g_R[Q];  /* roots of He_5, ascending */
static double g_W[Q];  /* Gauss-Hermite weights */
static int g_init = 0;

/* Probabilists' Hermite polynomial He_l(x) by the three-term recurrence
 * He_{l+1} = x He_l - l He_{l-1} (orthogonal under exp(-x^2/2)/sqrt(2 pi),
 * Eq. eweight). */
double orc_hermite(int l, double x)
{
    double hm1 = 1.0, h = x;
    if (l == 0) return 1.0;
    for (int k = 1; k < l; ++k) {
        double hp = x * h - (double)k * hm1;
        hm1 = h;
        h = hp;
    }
    return h;
}

static void init_constants(void)
{
    if (g_init) return;
    double s10 = sqrt(10.0);
    /* Table trots: roots -sqrt(5+sqrt10), -sqrt(5-sqrt10), 0, ... */
    g_R[0] = -sqrt(5.0 + s10);
    g_R[1] = -sqrt(5.0 - s10);
    g_R[2] = 0.0;
    g_R[3] = sqrt(5.0 - s10);
    g_R[4] = sqrt(5.0 + s10);
    /* and weights (7 -+ 2 sqrt10)/60, 8/15 */
    g_W[0] = (7.0 - 2.0 * s10) / 60.0;
    g_W[1] = (7.0 + 2.0 * s10) / 60.0;
    g_W[2] = 8.0 / 15.0;
    g_W[3] = g_W[1];
    g_W[4] = g_W[0];
    g_init = 1;
}

void orc_quadrature(double *R, double *W)
{
    init_constants();
    for (int k = 0; k < Q; ++k) { R[k] = g_R[k]; W[k] = g_W[k]; }
}

/* ------------------------------------------------------------------ */
/* Equilibrium (Eqs. feq, g_alpha), N = 4, m = 1                       */
/* ------------------------------------------------------------------ */

static double factorial(int n)
{
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r *= (double)k;
    return r;
}

/* g_k(u, T) = w_k sum_{l=0}^{4} He_l(p_k) sum_{s=0}^{l/2}
 *             (T-1)^s u^(l-2s) / (2^s s! (l-2s)!) */
double orc_g(int k, double u, double T)
{
    init_constants();
    double acc = 0.0;
    for (int l = 0; l <= 4; ++l) {
        double inner = 0.0;
        for (int s = 0; s <= l / 2; ++s) {
            inner += pow(T - 1.0, (double)s) * pow(u, (double)(l - 2 * s))
                     / (pow(2.0, (double)s) * factorial(s) * factorial(l - 2 * s));
        }
        acc += orc_hermite(l, g_R[k]) * inner;
    }
    return g_W[k] * acc;
}

/* f^eq_kappa = n g_{k1}(ux, T) g_{k2}(uy, T) */
void orc_feq(double n, double ux, double uy, double T, double *out25)
{
    double gx[Q], gy[Q];
    for (int k = 0; k < Q; ++k) { gx[k] = orc_g(k, ux, T); gy[k] = orc_g(k, uy, T); }
    for (int k1 = 0; k1 < Q; ++k1)
        for (int k2 = 0; k2 < Q; ++k2)
            out25[Q * k1 + k2] = n * gx[k1] * gy[k2];
}

/* ------------------------------------------------------------------ */
/* Momentum-space derivative along one axis (Eq. derf)                 */
/* ------------------------------------------------------------------ */

/* line[k], k = 0..4: f at the five velocities of one axis with the other
 * velocity index held fixed.  F_l = sum_k f_k He_l(p_k);
 * out_k = -w_k sum_{l=0}^{N-1} F_l He_{l+1}(p_k) / l!. */
void orc_dp_line(const double *line, double *out)
{
    init_constants();
    double F[4];
    for (int l = 0; l < 4; ++l) {
        F[l] = 0.0;
        for (int k = 0; k < Q; ++k) F[l] += line[k] * orc_hermite(l, g_R[k]);
    }
    for (int k = 0; k < Q; ++k) {
        double acc = 0.0;
        for (int l = 0; l < 4; ++l) acc += F[l] * orc_hermite(l + 1, g_R[k]) / factorial(l);
        out[k] = -g_W[k] * acc;
    }
}

/* ------------------------------------------------------------------ */
/* Moments (Sec. 2.2) and pressures (Eq. vdw)                          */
/* ------------------------------------------------------------------ */

/* out4 = n, ux, uy, T from 25 populations. */
void orc_moments_node(const double *f25, double *out4)
{
    init_constants();
    double n = 0.0, jx = 0.0, jy = 0.0, e = 0.0;
    for (int k1 = 0; k1 < Q; ++k1)
        for (int k2 = 0; k2 < Q; ++k2) {
            double f = f25[Q * k1 + k2];
            n += f;
            jx += g_R[k1] * f;
            jy += g_R[k2] * f;
            e += (g_R[k1] * g_R[k1] + g_R[k2] * g_R[k2]) * f;
        }
    double ux = jx / n, uy = jy / n;
    out4[0] = n;
    out4[1] = ux;
    out4[2] = uy;
    out4[3] = 0.5 * (e / n - ux * ux - uy * uy);
}

/* van der Waals pressure in the a/b form; a = 9/8, b = 1/3 is Eq. vdw. */
double orc_pw(double n, double T, double a, double b)
{
    return n * T / (1.0 - b * n) - a * n * n;
}

/* ------------------------------------------------------------------ */
/* 49-point stencils (Eqs. stencil_grad, stencil_glap)                 */
/* ------------------------------------------------------------------ */

/* Coefficient of v_{i+l, j+m} in d/dx, as cx[(m+3)*7 + (l+3)], to be
 * divided by ds.  w^{|l|,|m|} symmetric; zero where the paper says so. */
void orc_grad_stencil(double *cx)
{
    double w[4][4];
    memset(w, 0, sizeof w);
    w[1][0] = w[0][1] = 31.0 / 70.0;
    w[1][1] = 27.0 / 140.0;
    w[2][1] = w[1][2] = -3.0 / 70.0;
    w[2][2] = 3.0 / 560.0;
    w[3][0] = w[0][3] = -1.0 / 630.0;
    w[3][1] = w[1][3] = 1.0 / 280.0;
    for (int m = -3; m <= 3; ++m)
        for (int l = -3; l <= 3; ++l)
            cx[(m + 3) * 7 + (l + 3)] = (double)l * w[abs(l)][abs(m)];
}

/* Coefficient of n_{i+l, j+m} in d/dx (Laplacian n), as cx[(m+3)*7+(l+3)],
 * to be divided by ds^3.  Rows of the printed matrix are |m| = 3,2,1,0
 * (symmetric); its column 0 is l = +3 and column 6 is l = -3 (reading R1). */
void orc_glap_stencil(double *cx)
{
    double c[13];
    memset(c, 0, sizeof c);
    c[1] = -17.0 / 2160.0;  /* printed -17/260: reading R1 */
    c[4] = -59.0 / 540.0;   /* printed -59/240: reading R1 */
    c[6] = 13.0 / 120.0;
    c[7] = -7.0 / 30.0;
    c[8] = 5.0 / 4.0;
    c[10] = -7.0 / 60.0;
    c[11] = 187.0 / 240.0;
    c[12] = -59.0 / 20.0;
    /* row |m| -> coefficient index for columns |l| = 3, 2, 1 */
    int idx[4][4];  /* idx[|m|][|l|] */
    memset(idx, 0, sizeof idx);
    idx[3][3] = 1; idx[3][2] = 5; idx[3][1] = 9;
    idx[2][3] = 2; idx[2][2] = 6; idx[2][1] = 10;
    idx[1][3] = 3; idx[1][2] = 7; idx[1][1] = 11;
    idx[0][3] = 4; idx[0][2] = 8; idx[0][1] = 12;
    for (int m = -3; m <= 3; ++m)
        for (int l = -3; l <= 3; ++l) {
            double v = 0.0;
            if (l != 0) {
                v = c[idx[abs(m)][abs(l)]];
                if (l < 0) v = -v;
            }
            cx[(m + 3) * 7 + (l + 3)] = v;
        }
}

/* ------------------------------------------------------------------ */
/* WENO-5 (Eqs. weno5_flux .. weno5_sigma, Table tab:weno)             */
/* ------------------------------------------------------------------ */

/* v[0..4] = f_{i-2}, f_{i-1}, f_i, f_{i+1}, f_{i+2} in the upwind
 * orientation (for p > 0 as printed; for p < 0 the caller passes the
 * mirror image, reading R4).  Returns sum_q wbar_q Fhat^q, the WENO value
 * at i+1/2 without the factor p/m.  wout (optional) receives wbar. */
double orc_weno5(const double *v, double *wout)
{
    double sg1 = 13.0 / 12.0 * (v[0] - 2.0 * v[1] + v[2]) * (v[0] - 2.0 * v[1] + v[2])
               + 0.25 * (v[0] - 4.0 * v[1] + 3.0 * v[2]) * (v[0] - 4.0 * v[1] + 3.0 * v[2]);
    double sg2 = 13.0 / 12.0 * (v[1] - 2.0 * v[2] + v[3]) * (v[1] - 2.0 * v[2] + v[3])
               + 0.25 * (v[1] - v[3]) * (v[1] - v[3]);
    double sg3 = 13.0 / 12.0 * (v[2] - 2.0 * v[3] + v[4]) * (v[2] - 2.0 * v[3] + v[4])
               + 0.25 * (3.0 * v[2] - 4.0 * v[3] + v[4]) * (3.0 * v[2] - 4.0 * v[3] + v[4]);
    double F1 = v[0] / 3.0 - 7.0 / 6.0 * v[1] + 11.0 / 6.0 * v[2];
    double F2 = -v[1] / 6.0 + 5.0 / 6.0 * v[2] + v[3] / 3.0;
    double F3 = v[2] / 3.0 + 5.0 / 6.0 * v[3] - v[4] / 6.0;
    const double d1 = 0.1, d2 = 0.6, d3 = 0.3;
    double w1, w2, w3;
    int z1 = (sg1 == 0.0), z2 = (sg2 == 0.0), z3 = (sg3 == 0.0);
    if (z1 || z2 || z3) {
        /* Table tab:weno */
        if (z1 && z2 && z3) { w1 = 0.1; w2 = 0.6; w3 = 0.3; }
        else if (z2 && z3) { w1 = 0.0; w2 = 2.0 / 3.0; w3 = 1.0 / 3.0; }
        else if (z3 && z1) { w1 = 0.25; w2 = 0.0; w3 = 0.75; }
        else if (z1 && z2) { w1 = 1.0 / 7.0; w2 = 6.0 / 7.0; w3 = 0.0; }
        else if (z1) { w1 = 1.0; w2 = 0.0; w3 = 0.0; }
        else if (z2) { w1 = 0.0; w2 = 1.0; w3 = 0.0; }
        else { w1 = 0.0; w2 = 0.0; w3 = 1.0; }
    } else {
        double s = sg1;
        if (sg2 < s) s = sg2;
        if (sg3 < s) s = sg3;
        double t1 = d1 * (s / sg1) * (s / sg1);
        double t2 = d2 * (s / sg2) * (s / sg2);
        double t3 = d3 * (s / sg3) * (s / sg3);
        double sum = t1 + t2 + t3;
        w1 = t1 / sum;
        w2 = t2 / sum;
        w3 = t3 / sum;
    }
    if (wout) { wout[0] = w1; wout[1] = w2; wout[2] = w3; }
    return w1 * F1 + w2 * F2 + w3 * F3;
}

/* Learned weights (the network described in oracle/mlp.py): the same
 * interface value with the three weights produced by a 5-32-32-3 MLP
 * (tanh, tanh, softmax) from the normalised stencil (v - mean)/(max - min).
 * Where any indicator vanishes, Table tab:weno applies as in orc_weno5, so
 * constant ghost layers keep their exact fluxes; where the stencil is smooth
 * (min sigma >= 0.9 max sigma) the Jiang-Shu weights apply.  theta: 1347
 * parameters, W1 [32][5], b1 [32], W2 [32][32], b2 [32], W3 [3][32], b3 [3]. */
#define MLP_H 32
double orc_weno5_learned(const double *theta, const double *v, double *wout)
{
    double sg[3];
    sg[0] = 13.0 / 12.0 * (v[0] - 2.0 * v[1] + v[2]) * (v[0] - 2.0 * v[1] + v[2])
          + 0.25 * (v[0] - 4.0 * v[1] + 3.0 * v[2]) * (v[0] - 4.0 * v[1] + 3.0 * v[2]);
    sg[1] = 13.0 / 12.0 * (v[1] - 2.0 * v[2] + v[3]) * (v[1] - 2.0 * v[2] + v[3])
          + 0.25 * (v[1] - v[3]) * (v[1] - v[3]);
    sg[2] = 13.0 / 12.0 * (v[2] - 2.0 * v[3] + v[4]) * (v[2] - 2.0 * v[3] + v[4])
          + 0.25 * (3.0 * v[2] - 4.0 * v[3] + v[4]) * (3.0 * v[2] - 4.0 * v[3] + v[4]);
    if (sg[0] == 0.0 || sg[1] == 0.0 || sg[2] == 0.0) return orc_weno5(v, wout);
    double smin = sg[0], smax = sg[0];
    for (int q = 1; q < 3; ++q) {
        if (sg[q] < smin) smin = sg[q];
        if (sg[q] > smax) smax = sg[q];
    }
    if (smin >= 0.9 * smax) return orc_weno5(v, wout);
    const double *W1 = theta, *b1 = theta + 160, *W2 = theta + 192, *b2 = theta + 1216;
    const double *W3 = theta + 1248, *b3 = theta + 1344;
    double mean = 0.0, mx = v[0], mn = v[0];
    for (int q = 0; q < 5; ++q) {
        mean += v[q];
        if (v[q] > mx) mx = v[q];
        if (v[q] < mn) mn = v[q];
    }
    mean /= 5.0;
    double x[5];
    for (int q = 0; q < 5; ++q) x[q] = (v[q] - mean) / (mx - mn);
    double h1[MLP_H], h2[MLP_H], z[3];
    for (int j = 0; j < MLP_H; ++j) {
        double a = b1[j];
        for (int q = 0; q < 5; ++q) a += W1[j * 5 + q] * x[q];
        h1[j] = tanh(a);
    }
    for (int j = 0; j < MLP_H; ++j) {
        double a = b2[j];
        for (int k = 0; k < MLP_H; ++k) a += W2[j * MLP_H + k] * h1[k];
        h2[j] = tanh(a);
    }
    double zmax = -1e300;
    for (int q = 0; q < 3; ++q) {
        double a = b3[q];
        for (int j = 0; j < MLP_H; ++j) a += W3[q * MLP_H + j] * h2[j];
        z[q] = a;
        if (a > zmax) zmax = a;
    }
    double w[3], sum = 0.0;
    for (int q = 0; q < 3; ++q) {
        w[q] = exp(z[q] - zmax);
        sum += w[q];
    }
    for (int q = 0; q < 3; ++q) w[q] /= sum;
    double F1 = v[0] / 3.0 - 7.0 / 6.0 * v[1] + 11.0 / 6.0 * v[2];
    double F2 = -v[1] / 6.0 + 5.0 / 6.0 * v[2] + v[3] / 3.0;
    double F3 = v[2] / 3.0 + 5.0 / 6.0 * v[3] - v[4] / 6.0;
    if (wout) { wout[0] = w[0]; wout[1] = w[1]; wout[2] = w[2]; }
    return w[0] * F1 + w[1] * F2 + w[2] * F3;
}

/* ------------------------------------------------------------------ */
/* Solver context                                                      */
/* ------------------------------------------------------------------ */

typedef struct orc_params {
    int nx, ny;
    double ds, dt, tau;
    double a, b, sigma;
    double Tw[2], uw[2];   /* [0] left wall (x = 0), [1] right wall (x = 1) */
    int side_x;            /* 0 periodic, 1 diffuse walls on both x sides,
                              2 specular on both x sides, 3 specular at
                              x = 0 and a diffuse wall at x = nx ds */
    int side_y;            /* 0 periodic, 2 specular on both y sides */
} orc_params;

/* Kind of one side: 0 periodic, 1 diffuse wall, 2 specular reflection. */
enum { SIDE_PERIODIC = 0, SIDE_DIFFUSE = 1, SIDE_SPECULAR = 2 };

static int side_lo_x(const orc_params *p) { return p->side_x == 3 ? SIDE_SPECULAR : p->side_x; }
static int side_hi_x(const orc_params *p) { return p->side_x == 3 ? SIDE_DIFFUSE : p->side_x; }

typedef struct orc_ctx {
    orc_params p;
    size_t N;
    double *f, *f1, *f2, *L;           /* [node][25] */
    double *n, *ux, *uy, *T, *dp;      /* [node] */
    double *Fx, *Fy;                   /* [node] */
    double *nw;                        /* [2][ny] */
    double geqw[2][K];                 /* g_{k1}(0,Tw) g_{k2}(uw,Tw) per wall */
    double denw[2];                    /* denominator of Eq. nw per wall */
    double cgrad[49], cglap[49];
    int learned;                       /* 1: learned weights (orc_set_mlp) */
    double mlp[1347];
} orc_ctx;

static int wrap(int i, int n)
{
    int r = i % n;
    return r < 0 ? r + n : r;
}

void orc_destroy(orc_ctx *c)
{
    if (!c) return;
    free(c->f); free(c->f1); free(c->f2); free(c->L);
    free(c->n); free(c->ux); free(c->uy); free(c->T); free(c->dp);
    free(c->Fx); free(c->Fy); free(c->nw);
    free(c);
}

orc_ctx *orc_create(const orc_params *p)
{
    init_constants();
    if (p->nx < 1 || p->ny < 1) return NULL;
    if (p->side_x < 0 || p->side_x > 3 || (p->side_y != 0 && p->side_y != 2)) return NULL;
    if (p->side_x != 0 && p->nx < 3) return NULL;
    if (p->side_y != 0 && p->ny < 3) return NULL;
    orc_ctx *c = (orc_ctx *)calloc(1, sizeof(orc_ctx));
    c->p = *p;
    c->N = (size_t)p->nx * (size_t)p->ny;
    size_t N = c->N;
    c->f = (double *)calloc(N * K, sizeof(double));
    c->f1 = (double *)calloc(N * K, sizeof(double));
    c->f2 = (double *)calloc(N * K, sizeof(double));
    c->L = (double *)calloc(N * K, sizeof(double));
    c->n = (double *)calloc(N, sizeof(double));
    c->ux = (double *)calloc(N, sizeof(double));
    c->uy = (double *)calloc(N, sizeof(double));
    c->T = (double *)calloc(N, sizeof(double));
    c->dp = (double *)calloc(N, sizeof(double));
    c->Fx = (double *)calloc(N, sizeof(double));
    c->Fy = (double *)calloc(N, sizeof(double));
    c->nw = (double *)calloc(2 * (size_t)p->ny, sizeof(double));
    orc_grad_stencil(c->cgrad);
    orc_glap_stencil(c->cglap);
    for (int s = 0; s < 2; ++s) {
        double den = 0.0;
        for (int k1 = 0; k1 < Q; ++k1)
            for (int k2 = 0; k2 < Q; ++k2) {
                double g = orc_g(k1, 0.0, p->Tw[s]) * orc_g(k2, p->uw[s], p->Tw[s]);
                c->geqw[s][Q * k1 + k2] = g;
                /* incoming velocities: p_x > 0 at the left wall, < 0 at the right */
                int incoming = (s == 0) ? (g_R[k1] > 0.0) : (g_R[k1] < 0.0);
                if (incoming) den += g * g_R[k1];
            }
        c->denw[s] = den;
    }
    return c;
}

/* Population kappa at x-index i and row j (either possibly a ghost) of
 * array fs.  Periodic sides wrap.  Specular sides (Sec. 3.4.1): the ghost at
 * distance m from the side takes the population of the velocity with the
 * normal component reversed at the m-th node inside (k1 -> 4 - k1 across an
 * x side, k2 -> 4 - k2 across a y side).  Diffuse walls (Sec. 3.4.2):
 * outgoing velocities take the quadratic extrapolation, incoming ones
 * f^eq_w = n_w g g.  Values no flux ever reads are NaN so that an accidental
 * use shows up. */
static double fval(const orc_ctx *c, const double *fs, int kap, int i, int j)
{
    int nx = c->p.nx, ny = c->p.ny;
    if (j < 0 || j >= ny) {
        if (c->p.side_y == SIDE_SPECULAR) {
            int m = j < 0 ? -1 - j : j - ny;
            if (m > 2) return NAN;
            j = j < 0 ? -1 - j : 2 * ny - 1 - j;
            kap = Q * (kap / Q) + (Q - 1 - kap % Q);
        } else {
            j = wrap(j, ny);
        }
    }
    if (i >= 0 && i < nx) return fs[((size_t)j * nx + i) * K + kap];
    int side = i < 0 ? side_lo_x(&c->p) : side_hi_x(&c->p);
    int m = i < 0 ? -1 - i : i - nx;  /* ghost layer 0, 1, 2 */
    if (side == SIDE_PERIODIC) return fs[((size_t)j * nx + wrap(i, nx)) * K + kap];
    if (side == SIDE_SPECULAR) {
        if (m > 2) return NAN;
        int im = i < 0 ? -1 - i : 2 * nx - 1 - i;
        return fs[((size_t)j * nx + im) * K + Q * (Q - 1 - kap / Q) + kap % Q];
    }
    int k1 = kap / Q;
    double px = g_R[k1];
    if (i >= nx) {  /* right wall */
        if (px > 0.0) {
            double a0 = fs[((size_t)j * nx + nx - 1) * K + kap];
            double a1 = fs[((size_t)j * nx + nx - 2) * K + kap];
            double a2 = fs[((size_t)j * nx + nx - 3) * K + kap];
            if (m == 0) return 3.0 * a0 - 3.0 * a1 + a2;
            if (m == 1) return 6.0 * a0 - 8.0 * a1 + 3.0 * a2;
            return NAN;
        }
        if (px < 0.0) return c->nw[1 * ny + j] * c->geqw[1][kap];
        return NAN;
    } else {        /* left wall, ghost layer m at i = -1 - m */
        if (px < 0.0) {
            double a0 = fs[((size_t)j * nx + 0) * K + kap];
            double a1 = fs[((size_t)j * nx + 1) * K + kap];
            double a2 = fs[((size_t)j * nx + 2) * K + kap];
            if (m == 0) return 3.0 * a0 - 3.0 * a1 + a2;
            if (m == 1) return 6.0 * a0 - 8.0 * a1 + 3.0 * a2;
            return NAN;
        }
        if (px > 0.0) return c->nw[0 * ny + j] * c->geqw[0][kap];
        return NAN;
    }
}

/* x-flux F_kappa at the face x = i ds between nodes i-1 and i (including
 * the factor p/m); faces 0 and nx are the wall faces when walls are on. */
static double flux_x(const orc_ctx *c, const double *fs, int kap, int i, int j)
{
    double px = g_R[kap / Q];
    double v[5];
    if (px > 0.0) {
        for (int q = 0; q < 5; ++q) v[q] = fval(c, fs, kap, i - 3 + q, j);
    } else if (px < 0.0) {
        for (int q = 0; q < 5; ++q) v[q] = fval(c, fs, kap, i + 2 - q, j);
    } else {
        return 0.0;
    }
    return px * (c->learned ? orc_weno5_learned(c->mlp, v, NULL) : orc_weno5(v, NULL));
}

/* y-flux at the face y = j ds between rows j-1 and j. */
static double flux_y(const orc_ctx *c, const double *fs, int kap, int i, int j)
{
    double py = g_R[kap % Q];
    double v[5];
    if (py > 0.0) {
        for (int q = 0; q < 5; ++q) v[q] = fval(c, fs, kap, i, j - 3 + q);
    } else if (py < 0.0) {
        for (int q = 0; q < 5; ++q) v[q] = fval(c, fs, kap, i, j + 2 - q);
    } else {
        return 0.0;
    }
    return py * (c->learned ? orc_weno5_learned(c->mlp, v, NULL) : orc_weno5(v, NULL));
}

/* Field value with the boundary rule of Sec. 3.4.3: even reflection about
 * a wall or specular side (a double reflection at corners), periodic wrap
 * otherwise. */
static double field_at(const orc_ctx *c, const double *fld, int i, int j)
{
    int nx = c->p.nx, ny = c->p.ny;
    if (i < 0) i = side_lo_x(&c->p) == SIDE_PERIODIC ? wrap(i, nx) : -1 - i;
    else if (i >= nx) i = side_hi_x(&c->p) == SIDE_PERIODIC ? wrap(i, nx) : 2 * nx - 1 - i;
    if (j < 0) j = c->p.side_y == SIDE_SPECULAR ? -1 - j : wrap(j, ny);
    else if (j >= ny) j = c->p.side_y == SIDE_SPECULAR ? 2 * ny - 1 - j : wrap(j, ny);
    return fld[(size_t)j * nx + i];
}

/* Moments, Delta p, force and wall densities of populations fs. */
static void stage_fields(orc_ctx *c, const double *fs)
{
    const orc_params *p = &c->p;
    int nx = p->nx, ny = p->ny;
    long N = (long)c->N;
#pragma omp parallel for schedule(static)
    for (long q = 0; q < N; ++q) {
        double m4[4];
        orc_moments_node(fs + (size_t)q * K, m4);
        c->n[q] = m4[0];
        c->ux[q] = m4[1];
        c->uy[q] = m4[2];
        c->T[q] = m4[3];
        c->dp[q] = m4[0] * m4[3] - orc_pw(m4[0], m4[3], p->a, p->b);
    }
#pragma omp parallel for schedule(static)
    for (long q = 0; q < N; ++q) {
        int i = (int)(q % nx), j = (int)(q / nx);
        double gx = 0.0, gy = 0.0, lx = 0.0, ly = 0.0;
        for (int m = -3; m <= 3; ++m)
            for (int l = -3; l <= 3; ++l) {
                /* x-derivative: coefficient of v_{i+l, j+m};
                 * y-derivative: the transposed stencil */
                double cgx = c->cgrad[(m + 3) * 7 + (l + 3)];
                double cgy = c->cgrad[(l + 3) * 7 + (m + 3)];
                double clx = c->cglap[(m + 3) * 7 + (l + 3)];
                double cly = c->cglap[(l + 3) * 7 + (m + 3)];
                double dpv = field_at(c, c->dp, i + l, j + m);
                double nv = field_at(c, c->n, i + l, j + m);
                gx += cgx * dpv;
                gy += cgy * dpv;
                lx += clx * nv;
                ly += cly * nv;
            }
        double ds = p->ds;
        double ds3 = ds * ds * ds;
        c->Fx[q] = (gx / ds) / c->n[q] + p->sigma * (lx / ds3);
        c->Fy[q] = (gy / ds) / c->n[q] + p->sigma * (ly / ds3);
    }
    for (int j = 0; j < ny; ++j) {
        if (side_hi_x(p) == SIDE_DIFFUSE) {
            /* right wall: outgoing p_x > 0, face x = nx ds */
            double num = 0.0;
            for (int kap = 0; kap < K; ++kap)
                if (g_R[kap / Q] > 0.0) num += flux_x(c, fs, kap, nx, j);
            c->nw[1 * ny + j] = -num / c->denw[1];
        }
        if (side_lo_x(p) == SIDE_DIFFUSE) {
            /* left wall: outgoing p_x < 0, face x = 0 */
            double num = 0.0;
            for (int kap = 0; kap < K; ++kap)
                if (g_R[kap / Q] < 0.0) num += flux_x(c, fs, kap, 0, j);
            c->nw[0 * ny + j] = -num / c->denw[0];
        }
    }
}

/* L[f] of Eq. ecast for populations fs, into c->L. */
static void eval_L(orc_ctx *c, const double *fs)
{
    stage_fields(c, fs);
    const orc_params *p = &c->p;
    int nx = p->nx;
    long N = (long)c->N;
#pragma omp parallel for schedule(static)
    for (long q = 0; q < N; ++q) {
        int i = (int)(q % nx), j = (int)(q / nx);
        const double *fq = fs + (size_t)q * K;
        double feq[K];
        orc_feq(c->n[q], c->ux[q], c->uy[q], c->T[q], feq);
        double dpx[K], dpy[K];
        for (int k2 = 0; k2 < Q; ++k2) {  /* d/dp_x along k1 at fixed k2 */
            double line[Q], out[Q];
            for (int k1 = 0; k1 < Q; ++k1) line[k1] = fq[Q * k1 + k2];
            orc_dp_line(line, out);
            for (int k1 = 0; k1 < Q; ++k1) dpx[Q * k1 + k2] = out[k1];
        }
        for (int k1 = 0; k1 < Q; ++k1) {  /* d/dp_y along k2 at fixed k1 */
            double line[Q], out[Q];
            for (int k2 = 0; k2 < Q; ++k2) line[k2] = fq[Q * k1 + k2];
            orc_dp_line(line, out);
            for (int k2 = 0; k2 < Q; ++k2) dpy[Q * k1 + k2] = out[k2];
        }
        for (int kap = 0; kap < K; ++kap) {
            double advx = (flux_x(c, fs, kap, i + 1, j) - flux_x(c, fs, kap, i, j)) / p->ds;
            double advy = (flux_y(c, fs, kap, i, j + 1) - flux_y(c, fs, kap, i, j)) / p->ds;
            double force = c->Fx[q] * dpx[kap] + c->Fy[q] * dpy[kap];
            double coll = (fq[kap] - feq[kap]) / p->tau;
            c->L[(size_t)q * K + kap] = -advx - advy - force - coll;
        }
    }
}

/* One TVD RK-3 step (Eq. rk3). */
static void rk3_step(orc_ctx *c)
{
    size_t M = c->N * K;
    double dt = c->p.dt;
    eval_L(c, c->f);
    for (size_t q = 0; q < M; ++q) c->f1[q] = c->f[q] + dt * c->L[q];
    eval_L(c, c->f1);
    for (size_t q = 0; q < M; ++q)
        c->f2[q] = 0.75 * c->f[q] + 0.25 * c->f1[q] + 0.25 * dt * c->L[q];
    eval_L(c, c->f2);
    for (size_t q = 0; q < M; ++q)
        c->f[q] = c->f[q] / 3.0 + 2.0 / 3.0 * c->f2[q] + 2.0 / 3.0 * dt * c->L[q];
}

/* ------------------------------------------------------------------ */
/* Exported driver calls                                               */
/* ------------------------------------------------------------------ */

/* Switch the context to learned WENO weights with parameters theta
 * (1347 values), or back to Jiang-Shu weights when theta is NULL. */
void orc_set_mlp(orc_ctx *c, const double *theta)
{
    if (!theta) { c->learned = 0; return; }
    memcpy(c->mlp, theta, sizeof c->mlp);
    c->learned = 1;
}

void orc_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* f = f^eq(n, ux, uy, T) at every node; fields are [ny][nx]. */
void orc_init(orc_ctx *c, const double *n, const double *ux, const double *uy, const double *T)
{
    for (size_t q = 0; q < c->N; ++q) orc_feq(n[q], ux[q], uy[q], T[q], c->f + q * K);
}

void orc_step(orc_ctx *c, int nsteps)
{
    for (int s = 0; s < nsteps; ++s) rk3_step(c);
}

/* Populations in the library's exchange layout [25][ny][nx]. */
void orc_get_f(const orc_ctx *c, double *out)
{
    for (size_t q = 0; q < c->N; ++q)
        for (int kap = 0; kap < K; ++kap) out[(size_t)kap * c->N + q] = c->f[q * K + kap];
}

void orc_set_f(orc_ctx *c, const double *in)
{
    for (size_t q = 0; q < c->N; ++q)
        for (int kap = 0; kap < K; ++kap) c->f[q * K + kap] = in[(size_t)kap * c->N + q];
}

/* n, ux, uy, T of the current populations, [ny][nx] each. */
void orc_get_moments(const orc_ctx *c, double *n, double *ux, double *uy, double *T)
{
    for (size_t q = 0; q < c->N; ++q) {
        double m4[4];
        orc_moments_node(c->f + q * K, m4);
        n[q] = m4[0]; ux[q] = m4[1]; uy[q] = m4[2]; T[q] = m4[3];
    }
}

/* L[f] of the current populations ([25][ny][nx]) and the stage fields
 * behind it: out7 = n, ux, uy, T, dp, Fx, Fy ([7][ny][nx]); nw = [2][ny]. */
void orc_eval(orc_ctx *c, double *Lout, double *out7, double *nw)
{
    eval_L(c, c->f);
    size_t N = c->N;
    if (Lout)
        for (size_t q = 0; q < N; ++q)
            for (int kap = 0; kap < K; ++kap) Lout[(size_t)kap * N + q] = c->L[q * K + kap];
    if (out7) {
        memcpy(out7 + 0 * N, c->n, N * sizeof(double));
        memcpy(out7 + 1 * N, c->ux, N * sizeof(double));
        memcpy(out7 + 2 * N, c->uy, N * sizeof(double));
        memcpy(out7 + 3 * N, c->T, N * sizeof(double));
        memcpy(out7 + 4 * N, c->dp, N * sizeof(double));
        memcpy(out7 + 5 * N, c->Fx, N * sizeof(double));
        memcpy(out7 + 6 * N, c->Fy, N * sizeof(double));
    }
    if (nw) memcpy(nw, c->nw, 2 * (size_t)c->p.ny * sizeof(double));
}
