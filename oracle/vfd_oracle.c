/*
 * vfd_oracle.c -- plain, slow, FP64 CPU oracle for the finite element
 * discretisation of the variable-order fractional diffusion operator of
 * Lei, Turkiyyah & Knio, "Finite element discretizations for variable-order
 * fractional diffusion problems" (arXiv 2302.02863).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is called by the tests, by the smoke
 * check and by the CPU-baseline leg of the benchmark; the product (the CUDA
 * library) never links, loads or calls it, and it shares no code, header or
 * table with the product.
 *
 * What it computes (no hierarchical-matrix or fast-multipole approximation):
 *   - the stiffness matrix by definition (route 1): the sum over ordered
 *     element pairs of A_{tau,tau'}(psi_j, psi_i) (Sec. 2.3, eq. e:l-stiff),
 *     touching pairs by the singular rules of Sec. 4, separated pairs by the
 *     product of the element rules;
 *   - the same matrix through the paper's split A = B + K + M (Sec. 3,
 *     eqs. e:decomp, e:b, e:k, e:m): B from the singular rules, K = -2 <gamma_T>
 *     densely, rho by the direct point sum e:tgt-sum (Sec. 6.1) plus the
 *     exterior tail rho_B of Sec. 7.1.1 (eq. e:rho), M the weighted mass matrix;
 *   - a dense Cholesky solve A U = F with F the P1 load M0 f.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   R1  separated/ touching (int, ext) pairs count in both orders (factor 2),
 *       as the paper itself does for M^ext (Sec. 3.2.2).
 *   R1' every touching unordered pair {tau,tau'} is integrated once, in a
 *       canonical orientation (interior cell first, else lower cell index
 *       first), and the result serves both orders (A_{tau,tau'} = A_{tau',tau}).
 *   R3  element rule: symmetric 3-point triangle rule (barycentric 2/3,1/6,1/6,
 *       weights |tau|/3) / 3-point Gauss on intervals; singular rules use
 *       n_s Gauss-Legendre points per direction.
 *   R13 identical case: region 2 is x=(xi, xi*eta1*(1-eta2+eta2*eta3)) (the
 *       printed map lost the factor eta1) and the scaled difference of
 *       region 3 is (-eta3, 1-eta3) (the printed d_I^(3) lost a sign); both
 *       follow from the map and the listed Psi functions.
 *   R14 1D singular rules (the paper gives 2D only): identical cell with
 *       relative coordinate z = zeta^(1/(2-2 sbar)); adjacent cells with
 *       (xi, xi*eta) / (xi*eta, xi) and xi = zeta^(1/(3-2 sbar)), the same
 *       construction as the 2D vertex case (exponent of zeta >= 0).
 *   R20 3D (tetrahedra): the element rule is the symmetric 4-point degree-2
 *       rule (barycentric (a,b,b,b) and permutations, a = (5+3 sqrt 5)/20,
 *       b = (5-sqrt 5)/20, weights |tau|/4); the paper gives no singular
 *       rules for tetrahedron pairs, so in 3D only the separated parts K, rho
 *       and M are assembled (B = 0; single-row applies give rows of K + M;
 *       route 1, the tail and the gradient refuse d = 3).
 *
 * Reference triangle: (0,0),(1,0),(1,1) with basis phi0 = 1-x1,
 * phi1 = x1-x2, phi2 = x2 (Sec. 4).  Reference interval [0,1] with
 * phi0 = 1-x, phi1 = x.
 *
 * Kernel: gamma(x,y) = a(x,y) |x-y|^{-(d+s(x)+s(y))}, a = sqrt(kappa(x)kappa(y))
 * (Sec. 2, L_Omega).  Fields are given by descriptors (see field_eval).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [0,1] (Newton iteration on P_n)                    */
/* ------------------------------------------------------------------------ */
void oracle_gauss01(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[n - 1 - i] = 0.5 * (1.0 + z) ;
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);   /* 2/((1-z^2)P'^2) scaled by 1/2 */
    }
}

/* ------------------------------------------------------------------------ */
/* fields                                                                    */
/* ------------------------------------------------------------------------ */
/* descriptor: [c0, nF, nG, nT, squash, lo, hi, rows...]; rows of 5 doubles:
 *   Fourier (k1,k2,k3, amp, phase): amp cos(pi k.x + phase)
 *   Gauss   (x0,y0,z0, amp, c):     amp exp(-c |x-x0|^2)
 *   tensor bump (x0,y0,z0, amp, ell): amp prod_i exp(-1/(1-r_i^2)), r_i = 2(x_i-x0_i)/ell
 * squash 1: lo + (hi-lo)/(1+exp(-v)).  When `nodal` is non-NULL the field
 * is the P1 interpolant of the vertex values and the descriptor is unused. */
typedef struct { const double *desc; const double *nodal; } ofield;

static double field_analytic(const double *F, int d, const double *x)
{
    double v = F[0];
    int nF = (int)F[1], nG = (int)F[2], nT = (int)F[3];
    const double *r = F + 7;
    for (int t = 0; t < nF; ++t, r += 5) {
        double kx = 0.0;
        for (int i = 0; i < d; ++i) kx += r[i] * x[i];
        v += r[3] * cos(M_PI * kx + r[4]);
    }
    for (int t = 0; t < nG; ++t, r += 5) {
        double q = 0.0;
        for (int i = 0; i < d; ++i) q += (x[i] - r[i]) * (x[i] - r[i]);
        v += r[3] * exp(-r[4] * q);
    }
    for (int t = 0; t < nT; ++t, r += 5) {
        double p = r[3];
        for (int i = 0; i < d; ++i) {
            double rr = 2.0 * (x[i] - r[i]) / r[4];
            p *= (fabs(rr) < 1.0) ? exp(-1.0 / (1.0 - rr * rr)) : 0.0;
        }
        v += p;
    }
    if ((int)F[4] == 1) v = F[5] + (F[6] - F[5]) / (1.0 + exp(-v));
    return v;
}

/* value at point x lying in the cell with (reordered) vertex ids vid and
 * barycentric coordinates bary (bary[a] belongs to vid[a]) */
static double field_eval(const ofield *F, int d, const double *x, const int *vid, const double *bary)
{
    if (F->nodal) {
        double v = 0.0;
        for (int a = 0; a <= d; ++a) v += bary[a] * F->nodal[vid[a]];
        return v;
    }
    return field_analytic(F->desc, d, x);
}

/* gamma(x,y) = sqrt(kappa(x) kappa(y)) / |x-y|^(d+s(x)+s(y)), with the fields
 * already evaluated: sx, sy, lkx = log kappa(x), lky = log kappa(y). */
static double kernel_gamma(int d, double r, double sx, double sy, double lkx, double lky)
{
    double a = sqrt(exp(lkx) * exp(lky));
    return a / pow(r, d + sx + sy);
}

/* ------------------------------------------------------------------------ */
/* mesh helpers                                                              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int d, M, C;
    const double *X;          /* M*d */
    const int *T;             /* C*(d+1) */
    const unsigned char *in;  /* C */
} omesh;

/* interior DoFs: vertices of no exterior cell that lie in some cell (Sec. 2.3:
 * U vanishes on Omega_e).  Numbered in increasing vertex order.  Returns N. */
int oracle_dofs(int d, int M, int C, const int *T, const unsigned char *in, int *dof)
{
    int nv = d + 1;
    char *used = calloc(M, 1), *ext = calloc(M, 1);
    for (int c = 0; c < C; ++c)
        for (int a = 0; a < nv; ++a) {
            used[T[c * nv + a]] = 1;
            if (!in[c]) ext[T[c * nv + a]] = 1;
        }
    int N = 0;
    for (int v = 0; v < M; ++v) dof[v] = (used[v] && !ext[v]) ? N++ : -1;
    free(used); free(ext);
    return N;
}

static int shared_count(const omesh *m, int c1, int c2)
{
    int nv = m->d + 1, n = 0;
    for (int a = 0; a < nv; ++a)
        for (int b = 0; b < nv; ++b)
            if (m->T[c1 * nv + a] == m->T[c2 * nv + b]) ++n;
    return n;
}

/* barycentric coordinates are stored with stride NB (entries beyond d are 0) */
#define NB 4

static double cell_measure(const omesh *m, int c)
{
    int nv = m->d + 1;
    const int *t = m->T + c * nv;
    if (m->d == 1) return fabs(m->X[t[1]] - m->X[t[0]]);
    if (m->d == 3) {
        /* |det(p1 - p0, p2 - p0, p3 - p0)| / 6 */
        const double *p0 = m->X + 3 * t[0], *p1 = m->X + 3 * t[1], *p2 = m->X + 3 * t[2], *p3 = m->X + 3 * t[3];
        double a[3], b[3], e[3];
        for (int i = 0; i < 3; ++i) { a[i] = p1[i] - p0[i]; b[i] = p2[i] - p0[i]; e[i] = p3[i] - p0[i]; }
        double det = a[0] * (b[1] * e[2] - b[2] * e[1]) - a[1] * (b[0] * e[2] - b[2] * e[0]) + a[2] * (b[0] * e[1] - b[1] * e[0]);
        return fabs(det) / 6.0;
    }
    const double *p0 = m->X + 2 * t[0], *p1 = m->X + 2 * t[1], *p2 = m->X + 2 * t[2];
    return 0.5 * fabs((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0]));
}

/* element rule (R3): nq points per cell, barycentric coordinates bq[q][a]
 * w.r.t. the cell's stored vertex order, weights relative to the measure. */
static int elem_rule(int d, double bq[][NB], double *wq)
{
    memset(bq, 0, sizeof(double) * NB * NB);
    if (d == 3) {
        /* R20: the symmetric 4-point rule, exact for quadratics on a tetrahedron */
        const double a = (5.0 + 3.0 * sqrt(5.0)) / 20.0, b = (5.0 - sqrt(5.0)) / 20.0;
        for (int q = 0; q < 4; ++q) {
            for (int k = 0; k < 4; ++k) bq[q][k] = (k == q) ? a : b;
            wq[q] = 0.25;
        }
        return 4;
    }
    if (d == 2) {
        for (int q = 0; q < 3; ++q) {
            for (int a = 0; a < 3; ++a) bq[q][a] = (a == q) ? 2.0 / 3.0 : 1.0 / 6.0;
            wq[q] = 1.0 / 3.0;
        }
        return 3;
    }
    double g = 0.5 * sqrt(0.6);
    double t[3] = {0.5 - g, 0.5, 0.5 + g}, w[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
    for (int q = 0; q < 3; ++q) { bq[q][0] = 1.0 - t[q]; bq[q][1] = t[q]; bq[q][2] = 0.0; wq[q] = w[q]; }
    return 3;
}

/* ------------------------------------------------------------------------ */
/* singular rules for touching pairs (Sec. 4)                                */
/* ------------------------------------------------------------------------ */
/* A touching pair after canonical reordering.
 * 2D: P[0..2] vertices of tau, Q[0..2] of tau' (coords), pv/qv vertex ids,
 *     vertex case: P[0]=Q[0] shared; edge case: P[0]=Q[0], P[1]=Q[1];
 *     identical: Q == P.
 * local DoF order: vertex [P0,P1,P2,Q1,Q2]; edge [P0,P1,P2,Q2]; identical [P0,P1,P2].
 * 1D: adjacent: P[0]=Q[0] shared, local [P0,P1,Q1]; identical: [P0,P1]. */
typedef struct {
    int d, type;               /* type: 1 vertex (1D: adjacent), 2 edge, 3 identical */
    double P[3][2], Q[3][2];
    int pv[3], qv[3];
    double measP, measQ;
} opair;

static void ref_to_phys2(const double P[3][2], const double *xh, double *x)
{
    /* chi(xh) = P0 + J xh, J = [P1-P0 | P2-P1] */
    for (int i = 0; i < 2; ++i)
        x[i] = P[0][i] + (P[1][i] - P[0][i]) * xh[0] + (P[2][i] - P[1][i]) * xh[1];
}

static void J_apply2(const double P[3][2], const double *v, double *out)
{
    for (int i = 0; i < 2; ++i)
        out[i] = (P[1][i] - P[0][i]) * v[0] + (P[2][i] - P[1][i]) * v[1];
}

static void bary2(const double *xh, double *b)
{
    b[0] = 1.0 - xh[0]; b[1] = xh[0] - xh[1]; b[2] = xh[1];
}

/* evaluate the integrand pieces at mapped points; returns a(x,y), S=s(x)+s(y) */
static void pair_fields(const opair *pp, const ofield *fs, const ofield *fk,
                        const double *xh, const double *yh, double *S, double *a)
{
    double x[2], y[2], bx[3], by[3];
    if (pp->d == 2) {
        ref_to_phys2(pp->P, xh, x); ref_to_phys2(pp->Q, yh, y);
        bary2(xh, bx); bary2(yh, by);
    } else {
        x[0] = pp->P[0][0] + (pp->P[1][0] - pp->P[0][0]) * xh[0];
        y[0] = pp->Q[0][0] + (pp->Q[1][0] - pp->Q[0][0]) * yh[0];
        bx[0] = 1.0 - xh[0]; bx[1] = xh[0]; by[0] = 1.0 - yh[0]; by[1] = yh[0];
    }
    double sx = field_eval(fs, pp->d, x, pp->pv, bx), sy = field_eval(fs, pp->d, y, pp->qv, by);
    double kx = field_eval(fk, pp->d, x, pp->pv, bx), ky = field_eval(fk, pp->d, y, pp->qv, by);
    *S = sx + sy;
    *a = sqrt(exp(kx) * exp(ky));
}

/* 2D vertex- and edge-sharing regions: given (eta1,eta2,eta3) return the
 * scaled reference points a = xhat/xi, b = yhat/xi, the listed difference
 * functions Phi (Sec. 4.1) / Psi (Sec. 4.2) and the Jacobian factor. */
static int region_vertex(int k, const double *e, double *a, double *b, double *phi, double *jac)
{
    double e1 = e[0], e2 = e[1], e3 = e[2];
    if (k == 0) {
        a[0] = 1.0; a[1] = e1; b[0] = e2; b[1] = e2 * e3;
        phi[0] = e2 - 1.0; phi[1] = 1.0 - e1; phi[2] = e1; phi[3] = e2 * e3 - e2; phi[4] = -e2 * e3;
    } else {
        a[0] = e2; a[1] = e2 * e3; b[0] = 1.0; b[1] = e1;
        phi[0] = 1.0 - e2; phi[1] = e2 - e2 * e3; phi[2] = e2 * e3; phi[3] = e1 - 1.0; phi[4] = -e1;
    }
    *jac = e2;
    return 5;
}

static int region_edge(int k, const double *e, double *a, double *b, double *psi, double *jac)
{
    double e1 = e[0], e2 = e[1], e3 = e[2];
    switch (k) {
    case 0:
        a[0] = 1.0; a[1] = e1 * e3; b[0] = 1.0 - e1 * e2; b[1] = e1 * (1.0 - e2);
        psi[0] = -e1 * e2; psi[1] = e1 * (1.0 - e3); psi[2] = e1 * e3; psi[3] = -e1 * (1.0 - e2);
        *jac = e1 * e1; break;
    case 1:
        a[0] = 1.0; a[1] = e1; b[0] = 1.0 - e1 * e2 * e3; b[1] = e1 * e2 * (1.0 - e3);
        psi[0] = -e1 * e2 * e3; psi[1] = -e1 * (1.0 - e2); psi[2] = e1; psi[3] = -e1 * e2 * (1.0 - e3);
        *jac = e1 * e1 * e2; break;
    case 2:
        a[0] = 1.0 - e1 * e2; a[1] = e1 * (1.0 - e2); b[0] = 1.0; b[1] = e1 * e2 * e3;
        psi[0] = e1 * e2; psi[1] = -e1 * (1.0 - e2 * e3); psi[2] = e1 * (1.0 - e2); psi[3] = -e1 * e2 * e3;
        *jac = e1 * e1 * e2; break;
    case 3:
        a[0] = 1.0 - e1 * e2 * e3; a[1] = e1 * e2 * (1.0 - e3); b[0] = 1.0; b[1] = e1;
        psi[0] = e1 * e2 * e3; psi[1] = e1 * (1.0 - e2); psi[2] = e1 * e2 * (1.0 - e3); psi[3] = -e1;
        *jac = e1 * e1 * e2; break;
    default:
        a[0] = 1.0 - e1 * e2 * e3; a[1] = e1 * (1.0 - e2 * e3); b[0] = 1.0; b[1] = e1 * e2;
        psi[0] = e1 * e2 * e3; psi[1] = -e1 * (1.0 - e2); psi[2] = e1 * (1.0 - e2 * e3); psi[3] = -e1 * e2;
        *jac = e1 * e1 * e2; break;
    }
    return 4;
}

/* 2D identical regions k=0,1,2 (the paper's 1,2,3): xhat, yhat divided by xi,
 * the scaled difference dref = (xhat - yhat)/(xi eta1 eta2) and Psi. */
static void region_identical(int k, double e1, double e2, double e3,
                             double *a, double *b, double *dref, double *psi)
{
    switch (k) {
    case 0:
        a[0] = 1.0; a[1] = 1.0 - e1 + e1 * e2; b[0] = 1.0 - e1 * e2 * e3; b[1] = 1.0 - e1;
        dref[0] = e3; dref[1] = 1.0;
        psi[0] = -e3; psi[1] = e3 - 1.0; psi[2] = 1.0; break;
    case 1:
        a[0] = 1.0; a[1] = e1 * (1.0 - e2 + e2 * e3); b[0] = 1.0 - e1 * e2; b[1] = e1 * (1.0 - e2);
        dref[0] = 1.0; dref[1] = e3;
        psi[0] = -1.0; psi[1] = 1.0 - e3; psi[2] = e3; break;
    default:
        a[0] = 1.0 - e1 * e2 * e3; a[1] = e1 * (1.0 - e2 * e3); b[0] = 1.0; b[1] = e1 * (1.0 - e2);
        dref[0] = -e3; dref[1] = 1.0 - e3;
        psi[0] = e3; psi[1] = -1.0; psi[2] = 1.0 - e3; break;
    }
}

/* Local matrix L (nl x nl, row-major) of A_{tau,tau'}(psi_j, psi_i) for a
 * touching pair by the tensor Gauss rules of Sec. 4 (eqs. e:int-v-2, e:int-e,
 * e:int-i-2; 1D analogue R14).  Returns nl. */
static int pair_singular(const opair *pp, const ofield *fs, const ofield *fk, double sbar,
                         int ns, const double *gx, const double *gw, double *L)
{
    int d = pp->d, nl;
    double phi[5], a[2], b[2];
    if (d == 2 && pp->type == 3) nl = 3;
    else if (d == 2 && pp->type == 2) nl = 4;
    else if (d == 2) nl = 5;
    else if (pp->type == 3) nl = 2;
    else nl = 3;
    memset(L, 0, sizeof(double) * nl * nl);

    if (d == 2 && (pp->type == 1 || pp->type == 2)) {
        double c = 4.0 - 2.0 * sbar;
        double pre = (2.0 * pp->measP) * (2.0 * pp->measQ) / c;   /* |J_tau||J_tau'| / (4-2 sbar) */
        int nreg = pp->type == 1 ? 2 : 5;
        for (int k = 0; k < nreg; ++k)
            for (int iz = 0; iz < ns; ++iz)
                for (int i1 = 0; i1 < ns; ++i1)
                    for (int i2 = 0; i2 < ns; ++i2)
                        for (int i3 = 0; i3 < ns; ++i3) {
                            double eta[3] = {gx[i1], gx[i2], gx[i3]}, jac;
                            if (pp->type == 1) region_vertex(k, eta, a, b, phi, &jac);
                            else region_edge(k, eta, a, b, phi, &jac);
                            double zeta = gx[iz], xi = pow(zeta, 1.0 / c);
                            double xh[2] = {xi * a[0], xi * a[1]}, yh[2] = {xi * b[0], xi * b[1]};
                            double S, aa;
                            pair_fields(pp, fs, fk, xh, yh, &S, &aa);
                            double ja[2], jb[2];
                            J_apply2(pp->P, a, ja); J_apply2(pp->Q, b, jb);
                            double D = hypot(ja[0] - jb[0], ja[1] - jb[1]);
                            double w = gw[iz] * gw[i1] * gw[i2] * gw[i3] * pre
                                     * pow(zeta, (2.0 * sbar - S) / c) * jac * aa / pow(D, 2.0 + S);
                            for (int i = 0; i < nl; ++i)
                                for (int j = 0; j < nl; ++j) L[i * nl + j] += w * phi[i] * phi[j];
                        }
    } else if (d == 2) {
        double c = 4.0 - 2.0 * sbar, c2 = 2.0 - 2.0 * sbar;
        double J2 = (2.0 * pp->measP) * (2.0 * pp->measP);
        double pre = 2.0 * J2 / (c * c2);   /* |J|^2 / ((2 - sbar)(2 - 2 sbar)) */
        double dref[2];
        for (int k = 0; k < 3; ++k)
            for (int iz = 0; iz < ns; ++iz)
                for (int i1 = 0; i1 < ns; ++i1)
                    for (int it = 0; it < ns; ++it)
                        for (int i3 = 0; i3 < ns; ++i3) {
                            double zeta = gx[iz], t = gx[it];
                            double xi = pow(zeta, 1.0 / c), e1 = gx[i1], e2 = pow(t, 1.0 / c2), e3 = gx[i3];
                            region_identical(k, e1, e2, e3, a, b, dref, phi);
                            double xh[2] = {xi * a[0], xi * a[1]}, yh[2] = {xi * b[0], xi * b[1]};
                            double S, aa;
                            pair_fields(pp, fs, fk, xh, yh, &S, &aa);
                            double jd[2];
                            J_apply2(pp->P, dref, jd);
                            double D = hypot(jd[0], jd[1]);
                            double w = gw[iz] * gw[i1] * gw[it] * gw[i3] * pre
                                     * pow(zeta, (2.0 * sbar - S) / c) * pow(e1, 2.0 - S)
                                     * pow(t, (2.0 * sbar - S) / c2) * aa / pow(D, 2.0 + S);
                            for (int i = 0; i < 3; ++i)
                                for (int j = 0; j < 3; ++j) L[i * 3 + j] += w * phi[i] * phi[j];
                        }
    } else if (pp->type == 3) {
        /* 1D identical: region xhat > yhat (times 2 for the mirror region),
         * z = xhat - yhat = zeta^(1/c), yhat = (1-z) t, c = 2 - 2 sbar */
        double c = 2.0 - 2.0 * sbar, h = pp->measP;
        double pre = 2.0 * h * h / c;
        for (int iz = 0; iz < ns; ++iz)
            for (int it = 0; it < ns; ++it) {
                double zeta = gx[iz], t = gx[it], z = pow(zeta, 1.0 / c);
                double yh = (1.0 - z) * t, xh = yh + z;
                double S, aa;
                pair_fields(pp, fs, fk, &xh, &yh, &S, &aa);
                double psi[2] = {-1.0, 1.0};
                double w = gw[iz] * gw[it] * pre * pow(zeta, (2.0 * sbar - S) / c) * (1.0 - z) * aa / pow(h, 1.0 + S);
                for (int i = 0; i < 2; ++i)
                    for (int j = 0; j < 2; ++j) L[i * 2 + j] += w * psi[i] * psi[j];
            }
    } else {
        /* 1D adjacent cells sharing P0=Q0: regions (xi, xi eta) and (xi eta, xi),
         * xi = zeta^(1/c), c = 3 - 2 sbar */
        double c = 3.0 - 2.0 * sbar;
        double pre = pp->measP * pp->measQ / c;
        double JP = pp->P[1][0] - pp->P[0][0], JQ = pp->Q[1][0] - pp->Q[0][0];
        for (int k = 0; k < 2; ++k)
            for (int iz = 0; iz < ns; ++iz)
                for (int ie = 0; ie < ns; ++ie) {
                    double zeta = gx[iz], eta = gx[ie], xi = pow(zeta, 1.0 / c);
                    double av = k == 0 ? 1.0 : eta, bv = k == 0 ? eta : 1.0;
                    double xh = xi * av, yh = xi * bv;
                    double S, aa;
                    pair_fields(pp, fs, fk, &xh, &yh, &S, &aa);
                    double D = fabs(JP * av - JQ * bv);
                    double f[3] = {bv - av, av, -bv};
                    double w = gw[iz] * gw[ie] * pre * pow(zeta, (2.0 * sbar - S) / c) * aa / pow(D, 1.0 + S);
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) L[i * 3 + j] += w * f[i] * f[j];
                }
    }
    return nl;
}

/* canonical orientation and reordering of a touching pair (R1').  Fills pp
 * and loc[] (global vertex ids of the local DoFs).  Returns nl. */
static int make_pair(const omesh *m, int c1, int c2, opair *pp, int *loc)
{
    int d = m->d, nv = d + 1;
    int first = c1, second = c2;
    if (c1 != c2) {
        if (m->in[c1] != m->in[c2]) { first = m->in[c1] ? c1 : c2; second = m->in[c1] ? c2 : c1; }
        else { first = c1 < c2 ? c1 : c2; second = c1 < c2 ? c2 : c1; }
    }
    const int *t = m->T + first * nv, *u = m->T + second * nv;
    int ns = shared_count(m, first, second);
    int tp[3], up[3];
    pp->d = d;
    if (first == second) {
        pp->type = 3;
        for (int a = 0; a < nv; ++a) tp[a] = up[a] = t[a];
    } else if (ns == 1) {
        pp->type = 1;
        int sv = -1;
        for (int a = 0; a < nv; ++a) for (int b = 0; b < nv; ++b) if (t[a] == u[b]) sv = t[a];
        int k = 1; tp[0] = sv; for (int a = 0; a < nv; ++a) if (t[a] != sv) tp[k++] = t[a];
        k = 1; up[0] = sv; for (int a = 0; a < nv; ++a) if (u[a] != sv) up[k++] = u[a];
    } else { /* 2D edge */
        pp->type = 2;
        int k = 0, apex = -1, apex2 = -1;
        for (int a = 0; a < 3; ++a) {
            int in2 = 0;
            for (int b = 0; b < 3; ++b) if (t[a] == u[b]) in2 = 1;
            if (in2) tp[k++] = t[a]; else apex = t[a];
        }
        tp[2] = apex;
        for (int b = 0; b < 3; ++b) if (u[b] != tp[0] && u[b] != tp[1]) apex2 = u[b];
        up[0] = tp[0]; up[1] = tp[1]; up[2] = apex2;
    }
    for (int a = 0; a < nv; ++a) {
        pp->pv[a] = tp[a]; pp->qv[a] = up[a];
        for (int i = 0; i < d; ++i) { pp->P[a][i] = m->X[tp[a] * d + i]; pp->Q[a][i] = m->X[up[a] * d + i]; }
    }
    pp->measP = cell_measure(m, first);
    pp->measQ = cell_measure(m, second);
    int nl;
    if (d == 2) {
        if (pp->type == 3) { nl = 3; for (int a = 0; a < 3; ++a) loc[a] = tp[a]; }
        else if (pp->type == 2) { nl = 4; loc[0] = tp[0]; loc[1] = tp[1]; loc[2] = tp[2]; loc[3] = up[2]; }
        else { nl = 5; loc[0] = tp[0]; loc[1] = tp[1]; loc[2] = tp[2]; loc[3] = up[1]; loc[4] = up[2]; }
    } else {
        if (pp->type == 3) { nl = 2; loc[0] = tp[0]; loc[1] = tp[1]; }
        else { nl = 3; loc[0] = tp[0]; loc[1] = tp[1]; loc[2] = up[1]; }
    }
    return nl;
}

/* Local matrix of a single touching pair given by explicit reordered vertex
 * coordinates (used by the quadrature pins).  type: 1 vertex/adjacent,
 * 2 edge, 3 identical.  P, Q: (d+1)*d coordinates; pv, qv vertex ids for
 * nodal fields (may be NULL for analytic fields).  Returns nl. */
int oracle_pair_local(int d, int type, const double *P, const double *Q, const int *pv, const int *qv,
                      const double *sdesc, const double *snodal, const double *kdesc, const double *knodal,
                      double sbar, int ns, double *L)
{
    opair pp;
    pp.d = d; pp.type = type;
    for (int a = 0; a <= d; ++a) {
        pp.pv[a] = pv ? pv[a] : 0; pp.qv[a] = qv ? qv[a] : 0;
        for (int i = 0; i < d; ++i) { pp.P[a][i] = P[a * d + i]; pp.Q[a][i] = Q[a * d + i]; }
    }
    if (d == 2) {
        pp.measP = 0.5 * fabs((pp.P[1][0] - pp.P[0][0]) * (pp.P[2][1] - pp.P[0][1]) - (pp.P[1][1] - pp.P[0][1]) * (pp.P[2][0] - pp.P[0][0]));
        pp.measQ = 0.5 * fabs((pp.Q[1][0] - pp.Q[0][0]) * (pp.Q[2][1] - pp.Q[0][1]) - (pp.Q[1][1] - pp.Q[0][1]) * (pp.Q[2][0] - pp.Q[0][0]));
    } else {
        pp.measP = fabs(pp.P[1][0] - pp.P[0][0]);
        pp.measQ = fabs(pp.Q[1][0] - pp.Q[0][0]);
    }
    ofield fs = {sdesc, snodal}, fk = {kdesc, knodal};
    double gx[64], gw[64];
    if (ns > 64) return -1;
    oracle_gauss01(ns, gx, gw);
    return pair_singular(&pp, &fs, &fk, sbar, ns, gx, gw, L);
}

/* ------------------------------------------------------------------------ */
/* quadrature point cloud                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;                 /* points */
    double *x;             /* n*d */
    double *w;             /* n, weight incl. measure */
    double *s, *lk;        /* field values */
    int *cell;             /* n */
    double *bary;          /* n*NB barycentric w.r.t. stored cell vertex order */
} oquad;

static void build_quad(const omesh *m, const ofield *fs, const ofield *fk, oquad *Q)
{
    int d = m->d, nv = d + 1;
    double bq[NB][NB], wq[NB];
    int nq = elem_rule(d, bq, wq);
    Q->n = m->C * nq;
    Q->x = malloc(sizeof(double) * Q->n * d);
    Q->w = malloc(sizeof(double) * Q->n);
    Q->s = malloc(sizeof(double) * Q->n);
    Q->lk = malloc(sizeof(double) * Q->n);
    Q->cell = malloc(sizeof(int) * Q->n);
    Q->bary = malloc(sizeof(double) * Q->n * NB);
    for (int c = 0; c < m->C; ++c) {
        double meas = cell_measure(m, c);
        const int *t = m->T + c * nv;
        for (int q = 0; q < nq; ++q) {
            int id = c * nq + q;
            for (int i = 0; i < d; ++i) {
                double v = 0.0;
                for (int a = 0; a < nv; ++a) v += bq[q][a] * m->X[t[a] * d + i];
                Q->x[id * d + i] = v;
            }
            Q->w[id] = wq[q] * meas;
            Q->cell[id] = c;
            for (int a = 0; a < NB; ++a) Q->bary[id * NB + a] = bq[q][a];
            Q->s[id] = field_eval(fs, d, Q->x + id * d, t, bq[q]);
            Q->lk[id] = field_eval(fk, d, Q->x + id * d, t, bq[q]);
        }
    }
}

static void free_quad(oquad *Q)
{
    free(Q->x); free(Q->w); free(Q->s); free(Q->lk); free(Q->cell); free(Q->bary);
}

static double qdist(int d, const double *a, const double *b)
{
    double r2 = 0.0;
    for (int i = 0; i < d; ++i) r2 += (a[i] - b[i]) * (a[i] - b[i]);
    return sqrt(r2);
}

/* ------------------------------------------------------------------------ */
/* exterior tail rho_B (Sec. 7.1.1, eq. e:rho); needs constant s and kappa   */
/* ------------------------------------------------------------------------ */
double oracle_tail(int d, const double *x, double s, double a, double R)
{
    if (d == 1) return a * (pow(R - x[0], -2.0 * s) + pow(R + x[0], -2.0 * s)) / (2.0 * s);
    /* rho_B(x) = a/(2s) int_0^{2 pi} t(theta,x)^{-2s} dtheta, 9-point Gauss */
    double gx[9], gw[9], acc = 0.0, r2 = x[0] * x[0] + x[1] * x[1];
    oracle_gauss01(9, gx, gw);
    for (int k = 0; k < 9; ++k) {
        double th = 2.0 * M_PI * gx[k];
        double mu = x[0] * cos(th) + x[1] * sin(th);
        double t = sqrt(mu * mu + R * R - r2) - mu;
        acc += 2.0 * M_PI * gw[k] * pow(t, -2.0 * s);
    }
    return a * acc / (2.0 * s);
}

/* ------------------------------------------------------------------------ */
/* assembly                                                                  */
/* ------------------------------------------------------------------------ */
/* params: [s_bar, n_sing, tail_mode, tail_R]
 * outputs (each may be NULL):
 *   B, K, Mw : N x N row-major, DoFs in increasing vertex order (oracle_dofs)
 *   rho      : values at the interior quadrature points, ordered by interior
 *              cell (increasing cell id) then element-rule point
 *   Afull    : M x M, route 1 over all vertices (pairs with >=1 interior cell)
 * returns N, or -1 on bad input. */
int oracle_assemble(int d, int M, int C, const double *X, const int *T, const unsigned char *in,
                    const double *sdesc, const double *snodal, const double *kdesc, const double *knodal,
                    const double *params, double *B, double *K, double *Mw, double *rho, double *Afull)
{
    omesh m = {d, M, C, X, T, in};
    ofield fs = {sdesc, snodal}, fk = {kdesc, knodal};
    double sbar = params[0];
    int ns = (int)params[1], tail = (int)params[2];
    double R = params[3];
    int nv = d + 1;
    int *dof = malloc(sizeof(int) * M);
    int N = oracle_dofs(d, M, C, T, in, dof);
    double gx[64], gw[64];
    if (ns < 1 || ns > 64) { free(dof); return -1; }
    if (d == 3 && (Afull || tail)) { free(dof); return -1; }   /* R20: no singular rules, no 3D tail */
    oracle_gauss01(ns, gx, gw);
    if (B) memset(B, 0, sizeof(double) * N * N);
    if (K) memset(K, 0, sizeof(double) * N * N);
    if (Mw) memset(Mw, 0, sizeof(double) * N * N);
    if (Afull) memset(Afull, 0, sizeof(double) * M * M);

    oquad Q;
    build_quad(&m, &fs, &fk, &Q);
    int nq = Q.n / C;

    /* cell adjacency by shared vertices (touching = at least one shared vertex) */
    /* vertex -> cells */
    int *vdeg = calloc(M + 1, sizeof(int));
    for (int c = 0; c < C; ++c) for (int a = 0; a < nv; ++a) vdeg[T[c * nv + a] + 1]++;
    for (int v = 0; v < M; ++v) vdeg[v + 1] += vdeg[v];
    int *vcell = malloc(sizeof(int) * vdeg[M]);
    int *fill = calloc(M, sizeof(int));
    for (int c = 0; c < C; ++c) for (int a = 0; a < nv; ++a) { int v = T[c * nv + a]; vcell[vdeg[v] + fill[v]++] = c; }
    free(fill);

    /* ---- touching pairs: B (route 2) and the touching part of route 1 ---- */
#pragma omp parallel
    {
        char *mark = calloc(C, 1);
        int *list = malloc(sizeof(int) * C);
#pragma omp for schedule(dynamic, 16)
        for (int c = 0; c < C; ++c) {
            int nl_ = 0;
            for (int a = 0; a < nv; ++a) {
                int v = T[c * nv + a];
                for (int k = vdeg[v]; k < vdeg[v + 1]; ++k) {
                    int c2 = vcell[k];
                    if (!mark[c2]) { mark[c2] = 1; list[nl_++] = c2; }
                }
            }
            for (int k = 0; k < nl_; ++k) {
                int c2 = list[k];
                mark[c2] = 0;
                if (c2 < c) continue;                     /* unordered pairs once */
                if (d == 3) continue;                     /* R20: B is not assembled in 3D */
                if (!in[c] && !in[c2]) continue;          /* U,V vanish on ext x ext */
                opair pp; int loc[5]; double L[25];
                int nl = make_pair(&m, c, c2, &pp, loc);
                pair_singular(&pp, &fs, &fk, sbar, ns, gx, gw, L);
                double wgt = (c == c2) ? 1.0 : 2.0;       /* both orders (R1, R1') */
#pragma omp critical
                {
                    for (int i = 0; i < nl; ++i)
                        for (int j = 0; j < nl; ++j) {
                            if (B && dof[loc[i]] >= 0 && dof[loc[j]] >= 0)
                                B[(size_t)dof[loc[i]] * N + dof[loc[j]]] += wgt * L[i * nl + j];
                            if (Afull) Afull[(size_t)loc[i] * M + loc[j]] += wgt * L[i * nl + j];
                        }
                }
            }
        }
        free(mark); free(list);
    }

    /* ---- separated pairs ---- */
    /* touching lookup per cell via marks */
    int nqi = 0;
    for (int c = 0; c < C; ++c) if (in[c]) nqi += nq;
    double *rho_all = calloc(Q.n, sizeof(double));
#pragma omp parallel
    {
        char *touch = calloc(C, 1);
#pragma omp for schedule(dynamic, 4)
        for (int c = 0; c < C; ++c) {
            if (!in[c]) continue;
            const int *t = T + c * nv;
            for (int a = 0; a < nv; ++a) {
                int v = t[a];
                for (int k = vdeg[v]; k < vdeg[v + 1]; ++k) touch[vcell[k]] = 1;
            }
            /* density rho at the points of c: direct sum e:tgt-sum over all
             * source points of cells not touching c */
            for (int q = 0; q < nq; ++q) {
                int iq = c * nq + q;
                double acc = 0.0;
                for (int c2 = 0; c2 < C; ++c2) {
                    if (touch[c2]) continue;
                    for (int q2 = 0; q2 < nq; ++q2) {
                        int jq = c2 * nq + q2;
                        double r = qdist(d, Q.x + iq * d, Q.x + jq * d);
                        acc += kernel_gamma(d, r, Q.s[iq], Q.s[jq], Q.lk[iq], Q.lk[jq]) * Q.w[jq];
                    }
                }
                if (tail) acc += oracle_tail(d, Q.x + iq * d, Q.s[iq], exp(Q.lk[iq]), R);
                rho_all[iq] = acc;
            }
            /* K (e:k) over interior separated pairs, and route 1 over all
             * separated pairs (c, c2) with c interior, both orders */
            for (int c2 = 0; c2 < C; ++c2) {
                if (touch[c2]) continue;
                const int *u = T + c2 * nv;
                double G[NB][NB];
                for (int q = 0; q < nq; ++q)
                    for (int q2 = 0; q2 < nq; ++q2) {
                        int iq = c * nq + q, jq = c2 * nq + q2;
                        double r = qdist(d, Q.x + iq * d, Q.x + jq * d);
                        G[q][q2] = kernel_gamma(d, r, Q.s[iq], Q.s[jq], Q.lk[iq], Q.lk[jq]) * Q.w[iq] * Q.w[jq];
                    }
                if (K && in[c2]) {
                    /* K_ij += -2 sum_q sum_q' w w' psi_i(q) psi_j(q') gamma */
                    double loc[NB][NB];
                    for (int a = 0; a < nv; ++a)
                        for (int b = 0; b < nv; ++b) {
                            double acc = 0.0;
                            for (int q = 0; q < nq; ++q)
                                for (int q2 = 0; q2 < nq; ++q2)
                                    acc += Q.bary[(c * nq + q) * NB + a] * Q.bary[(c2 * nq + q2) * NB + b] * G[q][q2];
                            loc[a][b] = -2.0 * acc;
                        }
#pragma omp critical
                    for (int a = 0; a < nv; ++a)
                        for (int b = 0; b < nv; ++b) {
                            int i = dof[t[a]], j = dof[u[b]];
                            if (i >= 0 && j >= 0) K[(size_t)i * N + j] += loc[a][b];
                        }
                }
                if (Afull) {
                    /* A_{c,c2} + A_{c2,c} by the product rule over all vertices
                     * of c and c2 (when c2 is interior the reverse order is
                     * visited from c2 itself, so count once there) */
                    double wgt = in[c2] ? 1.0 : 2.0;
                    int vids[2 * NB];
                    for (int a = 0; a < nv; ++a) { vids[a] = t[a]; vids[nv + a] = u[a]; }
                    double loc[2 * NB][2 * NB];
                    memset(loc, 0, sizeof(loc));
                    for (int q = 0; q < nq; ++q)
                        for (int q2 = 0; q2 < nq; ++q2) {
                            double diff[2 * NB];
                            for (int a = 0; a < nv; ++a) {
                                diff[a] = Q.bary[(c * nq + q) * NB + a];
                                diff[nv + a] = -Q.bary[(c2 * nq + q2) * NB + a];
                            }
                            for (int i = 0; i < 2 * nv; ++i)
                                for (int j = 0; j < 2 * nv; ++j) loc[i][j] += G[q][q2] * diff[i] * diff[j];
                        }
#pragma omp critical
                    for (int i = 0; i < 2 * nv; ++i)
                        for (int j = 0; j < 2 * nv; ++j) Afull[(size_t)vids[i] * M + vids[j]] += wgt * loc[i][j];
                }
            }
            for (int a = 0; a < nv; ++a) {
                int v = t[a];
                for (int k = vdeg[v]; k < vdeg[v + 1]; ++k) touch[vcell[k]] = 0;
            }
        }
        free(touch);
    }

    /* ---- weighted mass M (e:m, e:tau-quad): 2 sum_q w psi_i psi_j rho ---- */
    if (Mw) {
        for (int c = 0; c < C; ++c) {
            if (!in[c]) continue;
            const int *t = T + c * nv;
            for (int a = 0; a < nv; ++a)
                for (int b = 0; b < nv; ++b) {
                    int i = dof[t[a]], j = dof[t[b]];
                    if (i < 0 || j < 0) continue;
                    double acc = 0.0;
                    for (int q = 0; q < nq; ++q) {
                        int iq = c * nq + q;
                        acc += Q.w[iq] * Q.bary[iq * NB + a] * Q.bary[iq * NB + b] * rho_all[iq];
                    }
                    Mw[(size_t)i * N + j] += 2.0 * acc;
                }
        }
    }
    if (rho) {
        int k = 0;
        for (int c = 0; c < C; ++c)
            if (in[c]) for (int q = 0; q < nq; ++q) rho[k++] = rho_all[c * nq + q];
    }
    free(rho_all);
    free(vdeg); free(vcell); free(dof);
    free_quad(&Q);
    return N;
}

/* ------------------------------------------------------------------------ */
/* gradient of J = Lam^T U(theta) through the adjoint: g = -Lam^T (dA/dtheta) U */
/* ------------------------------------------------------------------------ */
/* The paper has no gradients; this is the derivative of the discrete matrix
 * A = B + K + M assembled above (same quadrature, s_bar and rules held
 * fixed) with respect to the nodal values of s and of log kappa (P1 fields).
 * Every quadrature term carries gamma(x,y) = a(x,y) |x-y|^-(d+s(x)+s(y)), so
 *   d gamma / d s_k      = -ln|x-y| (psi_k(x) + psi_k(y)) gamma,
 *   d gamma / d logk_k   = 1/2      (psi_k(x) + psi_k(y)) gamma,
 * and each term of B, K and M is differentiated where it is formed. */

/* pair_fields plus the barycentric coordinates of the mapped points (in the
 * pv / qv order of the pair) */
static void pair_fields_b(const opair *pp, const ofield *fs, const ofield *fk, const double *xh, const double *yh,
                          double *S, double *a, double *bx, double *by)
{
    double x[2], y[2];
    if (pp->d == 2) {
        ref_to_phys2(pp->P, xh, x); ref_to_phys2(pp->Q, yh, y);
        bary2(xh, bx); bary2(yh, by);
    } else {
        x[0] = pp->P[0][0] + (pp->P[1][0] - pp->P[0][0]) * xh[0];
        y[0] = pp->Q[0][0] + (pp->Q[1][0] - pp->Q[0][0]) * yh[0];
        bx[0] = 1.0 - xh[0]; bx[1] = xh[0]; bx[2] = 0.0;
        by[0] = 1.0 - yh[0]; by[1] = yh[0]; by[2] = 0.0;
    }
    double sx = field_eval(fs, pp->d, x, pp->pv, bx), sy = field_eval(fs, pp->d, y, pp->qv, by);
    double kx = field_eval(fk, pp->d, x, pp->pv, bx), ky = field_eval(fk, pp->d, y, pp->qv, by);
    *S = sx + sy;
    *a = sqrt(exp(kx) * exp(ky));
}

/* one rule point of a touching pair: weight w (as in pair_singular), the
 * local basis differences f[0..nl), dlw = d(log w)/dS (= -ln|x-y|, read off
 * the factors of w that depend on S), barycentrics bx, by.  Accumulates
 *   gs[a] (a < 3: vertex pv[a]; a >= 3: qv[a-3]) -= c dlw (bx | by),
 *   gk[a] -= c/2 (bx | by),  c = w sum_r (U_r . f)(Lam_r . f). */
static void grad_point(int nl, int nrhs, const double *Ul, const double *Ll, double w, const double *f, double dlw,
                       const double *bx, const double *by, double *gs, double *gk)
{
    double ul = 0.0;
    for (int r = 0; r < nrhs; ++r) {
        double u = 0.0, l = 0.0;
        for (int i = 0; i < nl; ++i) { u += Ul[r * nl + i] * f[i]; l += Ll[r * nl + i] * f[i]; }
        ul += u * l;
    }
    double c = w * ul;
    for (int a = 0; a < 3; ++a) {
        gs[a] -= c * dlw * bx[a]; gs[3 + a] -= c * dlw * by[a];
        gk[a] -= 0.5 * c * bx[a]; gk[3 + a] -= 0.5 * c * by[a];
    }
}

/* gradient contributions of one touching pair (the loops of pair_singular) */
static void pair_singular_grad(const opair *pp, const ofield *fs, const ofield *fk, double sbar, int ns,
                               const double *gx, const double *gw, int nl, int nrhs, const double *Ul,
                               const double *Ll, double *gs, double *gk)
{
    int d = pp->d;
    double phi[5], a[2], b[2], bx[3], by[3];
    if (d == 2 && (pp->type == 1 || pp->type == 2)) {
        double c = 4.0 - 2.0 * sbar;
        double pre = (2.0 * pp->measP) * (2.0 * pp->measQ) / c;
        int nreg = pp->type == 1 ? 2 : 5;
        for (int k = 0; k < nreg; ++k)
            for (int iz = 0; iz < ns; ++iz)
                for (int i1 = 0; i1 < ns; ++i1)
                    for (int i2 = 0; i2 < ns; ++i2)
                        for (int i3 = 0; i3 < ns; ++i3) {
                            double eta[3] = {gx[i1], gx[i2], gx[i3]}, jac;
                            if (pp->type == 1) region_vertex(k, eta, a, b, phi, &jac);
                            else region_edge(k, eta, a, b, phi, &jac);
                            double zeta = gx[iz], xi = pow(zeta, 1.0 / c);
                            double xh[2] = {xi * a[0], xi * a[1]}, yh[2] = {xi * b[0], xi * b[1]};
                            double S, aa;
                            pair_fields_b(pp, fs, fk, xh, yh, &S, &aa, bx, by);
                            double ja[2], jb[2];
                            J_apply2(pp->P, a, ja); J_apply2(pp->Q, b, jb);
                            double D = hypot(ja[0] - jb[0], ja[1] - jb[1]);
                            double w = gw[iz] * gw[i1] * gw[i2] * gw[i3] * pre
                                     * pow(zeta, (2.0 * sbar - S) / c) * jac * aa / pow(D, 2.0 + S);
                            double dlw = -log(zeta) / c - log(D);
                            grad_point(nl, nrhs, Ul, Ll, w, phi, dlw, bx, by, gs, gk);
                        }
    } else if (d == 2) {
        double c = 4.0 - 2.0 * sbar, c2 = 2.0 - 2.0 * sbar;
        double J2 = (2.0 * pp->measP) * (2.0 * pp->measP);
        double pre = 2.0 * J2 / (c * c2);
        double dref[2];
        for (int k = 0; k < 3; ++k)
            for (int iz = 0; iz < ns; ++iz)
                for (int i1 = 0; i1 < ns; ++i1)
                    for (int it = 0; it < ns; ++it)
                        for (int i3 = 0; i3 < ns; ++i3) {
                            double zeta = gx[iz], t = gx[it];
                            double xi = pow(zeta, 1.0 / c), e1 = gx[i1], e2 = pow(t, 1.0 / c2), e3 = gx[i3];
                            region_identical(k, e1, e2, e3, a, b, dref, phi);
                            double xh[2] = {xi * a[0], xi * a[1]}, yh[2] = {xi * b[0], xi * b[1]};
                            double S, aa;
                            pair_fields_b(pp, fs, fk, xh, yh, &S, &aa, bx, by);
                            double jd[2];
                            J_apply2(pp->P, dref, jd);
                            double D = hypot(jd[0], jd[1]);
                            double w = gw[iz] * gw[i1] * gw[it] * gw[i3] * pre
                                     * pow(zeta, (2.0 * sbar - S) / c) * pow(e1, 2.0 - S)
                                     * pow(t, (2.0 * sbar - S) / c2) * aa / pow(D, 2.0 + S);
                            double dlw = -log(zeta) / c - log(e1) - log(t) / c2 - log(D);
                            grad_point(nl, nrhs, Ul, Ll, w, phi, dlw, bx, by, gs, gk);
                        }
    } else if (pp->type == 3) {
        double c = 2.0 - 2.0 * sbar, h = pp->measP;
        double pre = 2.0 * h * h / c;
        for (int iz = 0; iz < ns; ++iz)
            for (int it = 0; it < ns; ++it) {
                double zeta = gx[iz], t = gx[it], z = pow(zeta, 1.0 / c);
                double yh = (1.0 - z) * t, xh = yh + z;
                double S, aa;
                pair_fields_b(pp, fs, fk, &xh, &yh, &S, &aa, bx, by);
                double psi[2] = {-1.0, 1.0};
                double w = gw[iz] * gw[it] * pre * pow(zeta, (2.0 * sbar - S) / c) * (1.0 - z) * aa / pow(h, 1.0 + S);
                double dlw = -log(zeta) / c - log(h);
                grad_point(nl, nrhs, Ul, Ll, w, psi, dlw, bx, by, gs, gk);
            }
    } else {
        double c = 3.0 - 2.0 * sbar;
        double pre = pp->measP * pp->measQ / c;
        double JP = pp->P[1][0] - pp->P[0][0], JQ = pp->Q[1][0] - pp->Q[0][0];
        for (int k = 0; k < 2; ++k)
            for (int iz = 0; iz < ns; ++iz)
                for (int ie = 0; ie < ns; ++ie) {
                    double zeta = gx[iz], eta = gx[ie], xi = pow(zeta, 1.0 / c);
                    double av = k == 0 ? 1.0 : eta, bv = k == 0 ? eta : 1.0;
                    double xh = xi * av, yh = xi * bv;
                    double S, aa;
                    pair_fields_b(pp, fs, fk, &xh, &yh, &S, &aa, bx, by);
                    double D = fabs(JP * av - JQ * bv);
                    double f[3] = {bv - av, av, -bv};
                    double w = gw[iz] * gw[ie] * pre * pow(zeta, (2.0 * sbar - S) / c) * aa / pow(D, 1.0 + S);
                    double dlw = -log(zeta) / c - log(D);
                    grad_point(nl, nrhs, Ul, Ll, w, f, dlw, bx, by, gs, gk);
                }
    }
}

/* g_s[k] = -sum_r Lam_r^T (dA/ds_k) U_r and g_lk[k] likewise for log kappa,
 * for P1 (nodal) s and log kappa given at all M vertices; A = B + K + M as in
 * oracle_assemble (route 2; bounded exterior only: tail_mode must be 0).
 * U, Lam: nrhs x N (row r contiguous, DoF order of oracle_dofs).  g_s, g_lk:
 * M entries each, overwritten.  Returns N, or -1 on bad input. */
int oracle_grad(int d, int M, int C, const double *X, const int *T, const unsigned char *in,
                const double *snodal, const double *knodal, const double *params, int nrhs,
                const double *U, const double *Lam, double *g_s, double *g_lk)
{
    omesh m = {d, M, C, X, T, in};
    ofield fs = {NULL, snodal}, fk = {NULL, knodal};
    double sbar = params[0];
    int ns = (int)params[1], tail = (int)params[2];
    int nv = d + 1;
    if (!snodal || !knodal || tail != 0 || ns < 1 || ns > 64 || nrhs < 1 || d == 3) return -1;
    int *dof = malloc(sizeof(int) * M);
    int N = oracle_dofs(d, M, C, T, in, dof);
    double gx[64], gw[64];
    oracle_gauss01(ns, gx, gw);
    oquad Q;
    build_quad(&m, &fs, &fk, &Q);
    int nq = Q.n / C;

    /* U and Lam at the quadrature points (zero on exterior cells) */
    double *Uq = calloc((size_t)nrhs * Q.n, sizeof(double)), *Lq = calloc((size_t)nrhs * Q.n, sizeof(double));
    for (int r = 0; r < nrhs; ++r)
        for (int iq = 0; iq < Q.n; ++iq) {
            const int *t = T + Q.cell[iq] * nv;
            double u = 0.0, l = 0.0;
            for (int a = 0; a < nv; ++a) {
                int i = dof[t[a]];
                if (i >= 0) { u += Q.bary[iq * NB + a] * U[(size_t)r * N + i]; l += Q.bary[iq * NB + a] * Lam[(size_t)r * N + i]; }
            }
            Uq[(size_t)r * Q.n + iq] = u;
            Lq[(size_t)r * Q.n + iq] = l;
        }

    int *vdeg = calloc(M + 1, sizeof(int));
    for (int c = 0; c < C; ++c) for (int a = 0; a < nv; ++a) vdeg[T[c * nv + a] + 1]++;
    for (int v = 0; v < M; ++v) vdeg[v + 1] += vdeg[v];
    int *vcell = malloc(sizeof(int) * vdeg[M]);
    int *fill = calloc(M, sizeof(int));
    for (int c = 0; c < C; ++c) for (int a = 0; a < nv; ++a) { int v = T[c * nv + a]; vcell[vdeg[v] + fill[v]++] = c; }
    free(fill);

    int nth = 1;
#ifdef _OPENMP
    nth = omp_get_max_threads();
#endif
    double *acc = calloc((size_t)nth * 2 * M, sizeof(double));   /* per thread: g_s, g_lk */

#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *gS = acc + (size_t)tid * 2 * M, *gK = gS + M;
        char *mark = calloc(C, 1);
        int *list = malloc(sizeof(int) * C);
        double *Ul = malloc(sizeof(double) * nrhs * 5), *Ll = malloc(sizeof(double) * nrhs * 5);

        /* ---- B: touching pairs (Sec. 4 rules), both orders by R1 / R1' ---- */
#pragma omp for schedule(static)
        for (int c = 0; c < C; ++c) {
            int nl_ = 0;
            for (int a = 0; a < nv; ++a) {
                int v = T[c * nv + a];
                for (int k = vdeg[v]; k < vdeg[v + 1]; ++k) {
                    int c2 = vcell[k];
                    if (!mark[c2]) { mark[c2] = 1; list[nl_++] = c2; }
                }
            }
            for (int k = 0; k < nl_; ++k) {
                int c2 = list[k];
                mark[c2] = 0;
                if (c2 < c) continue;
                if (!in[c] && !in[c2]) continue;
                opair pp; int loc[5];
                int nl = make_pair(&m, c, c2, &pp, loc);
                for (int r = 0; r < nrhs; ++r)
                    for (int i = 0; i < nl; ++i) {
                        int j = dof[loc[i]];
                        Ul[r * nl + i] = j >= 0 ? U[(size_t)r * N + j] : 0.0;
                        Ll[r * nl + i] = j >= 0 ? Lam[(size_t)r * N + j] : 0.0;
                    }
                double gs[6] = {0, 0, 0, 0, 0, 0}, gk[6] = {0, 0, 0, 0, 0, 0};
                pair_singular_grad(&pp, &fs, &fk, sbar, ns, gx, gw, nl, nrhs, Ul, Ll, gs, gk);
                double wgt = (c == c2) ? 1.0 : 2.0;
                for (int a = 0; a < nv; ++a) {
                    gS[pp.pv[a]] += wgt * gs[a]; gS[pp.qv[a]] += wgt * gs[3 + a];
                    gK[pp.pv[a]] += wgt * gk[a]; gK[pp.qv[a]] += wgt * gk[3 + a];
                }
            }
        }

        /* ---- K (e:k, interior separated pairs) and M (e:m with rho of
         * e:tgt-sum over all separated source points) ----
         * per point pair (q in interior c, q' in c2 not touching c):
         *   K: -2 w w' gamma Lam(q) U(q')   (c2 interior)
         *   M:  2 w w' gamma Lam(q) U(q)    (the rho(q) sum)
         * differentiated in gamma and contracted with -1. */
#pragma omp for schedule(static)
        for (int c = 0; c < C; ++c) {
            if (!in[c]) continue;
            const int *t = T + c * nv;
            for (int a = 0; a < nv; ++a) {
                int v = t[a];
                for (int k = vdeg[v]; k < vdeg[v + 1]; ++k) mark[vcell[k]] = 1;
            }
            for (int c2 = 0; c2 < C; ++c2) {
                if (mark[c2]) continue;
                const int *u = T + c2 * nv;
                for (int q = 0; q < nq; ++q)
                    for (int q2 = 0; q2 < nq; ++q2) {
                        int iq = c * nq + q, jq = c2 * nq + q2;
                        double r = qdist(d, Q.x + iq * d, Q.x + jq * d);
                        double G = kernel_gamma(d, r, Q.s[iq], Q.s[jq], Q.lk[iq], Q.lk[jq]) * Q.w[iq] * Q.w[jq];
                        double lu = 0.0, mu = 0.0;
                        for (int rr = 0; rr < nrhs; ++rr) {
                            mu += Lq[(size_t)rr * Q.n + iq] * Uq[(size_t)rr * Q.n + iq];
                            if (in[c2]) lu += Lq[(size_t)rr * Q.n + iq] * Uq[(size_t)rr * Q.n + jq];
                        }
                        /* g = -(dK + dM) contracted: dgamma_s = -ln r (...) gamma, dgamma_lk = (...) gamma / 2 */
                        double ts = 2.0 * G * log(r) * (mu - lu);
                        double tk = G * (lu - mu);
                        for (int a = 0; a < nv; ++a) {
                            double bq = Q.bary[iq * NB + a], bq2 = Q.bary[jq * NB + a];
                            gS[t[a]] += ts * bq; gS[u[a]] += ts * bq2;
                            gK[t[a]] += tk * bq; gK[u[a]] += tk * bq2;
                        }
                    }
            }
            for (int a = 0; a < nv; ++a) {
                int v = t[a];
                for (int k = vdeg[v]; k < vdeg[v + 1]; ++k) mark[vcell[k]] = 0;
            }
        }
        free(mark); free(list); free(Ul); free(Ll);
    }
    for (int v = 0; v < M; ++v) {
        double a1 = 0.0, a2 = 0.0;
        for (int th = 0; th < nth; ++th) { a1 += acc[(size_t)th * 2 * M + v]; a2 += acc[(size_t)th * 2 * M + M + v]; }
        g_s[v] = a1;
        g_lk[v] = a2;
    }
    free(acc); free(Uq); free(Lq); free(vdeg); free(vcell); free(dof);
    free_quad(&Q);
    return N;
}

/* ------------------------------------------------------------------------ */
/* single rows of A x (route 2, no approximation), for sampled parity checks  */
/* ------------------------------------------------------------------------ */
/* y[r] = (A x)_{rows[r]} with A = B + K + M exactly as oracle_assemble forms
 * them (Sec. 3 split; B by the Sec. 4 rules over the touching pairs whose
 * local DoFs contain the row's vertex; K and M through the point sums of
 * e:k and e:tgt-sum over all separated points; the tail when tail_mode = 1).
 * Cost O(|supp| x |Q|) per row.  x: N entries (DoF order of oracle_dofs);
 * rows: DoF indices.  Returns N, or -1 on bad input. */
int oracle_apply_rows(int d, int M, int C, const double *X, const int *T, const unsigned char *in,
                      const double *sdesc, const double *snodal, const double *kdesc, const double *knodal,
                      const double *params, const double *x, int nrows, const int *rows, double *y)
{
    omesh m = {d, M, C, X, T, in};
    ofield fs = {sdesc, snodal}, fk = {kdesc, knodal};
    double sbar = params[0];
    int ns = (int)params[1], tail = (int)params[2];
    double R = params[3];
    int nv = d + 1;
    if (ns < 1 || ns > 64 || (d == 3 && tail)) return -1;
    int *dof = malloc(sizeof(int) * M);
    int N = oracle_dofs(d, M, C, T, in, dof);
    int *vert = malloc(sizeof(int) * (N > 0 ? N : 1));
    for (int v = 0; v < M; ++v) if (dof[v] >= 0) vert[dof[v]] = v;
    double gx[64], gw[64];
    oracle_gauss01(ns, gx, gw);
    oquad Q;
    build_quad(&m, &fs, &fk, &Q);
    int nq = Q.n / C;
    double *xq = malloc(sizeof(double) * Q.n);
    for (int iq = 0; iq < Q.n; ++iq) {
        const int *t = T + Q.cell[iq] * nv;
        double v = 0.0;
        for (int a = 0; a < nv; ++a) if (dof[t[a]] >= 0) v += Q.bary[iq * NB + a] * x[dof[t[a]]];
        xq[iq] = v;
    }
    int *vdeg = calloc(M + 1, sizeof(int));
    for (int c = 0; c < C; ++c) for (int a = 0; a < nv; ++a) vdeg[T[c * nv + a] + 1]++;
    for (int v = 0; v < M; ++v) vdeg[v + 1] += vdeg[v];
    int *vcell = malloc(sizeof(int) * vdeg[M]);
    int *fill = calloc(M, sizeof(int));
    for (int c = 0; c < C; ++c) for (int a = 0; a < nv; ++a) { int v = T[c * nv + a]; vcell[vdeg[v] + fill[v]++] = c; }
    free(fill);
#pragma omp parallel
    {
        char *touch = calloc(C, 1);
        int *pairs = malloc(sizeof(int) * 2 * C);
#pragma omp for schedule(dynamic, 1)
        for (int r = 0; r < nrows; ++r) {
            const int vi = vert[rows[r]];
            double acc = 0.0;
            /* ---- B: the unordered touching pairs {c, c2} with vi a local DoF
             * (none in 3D: R20) ---- */
            int np = 0;
            for (int k = vdeg[vi]; k < vdeg[vi + 1] && d != 3; ++k) {
                int c = vcell[k];
                const int *t = T + c * nv;
                for (int a = 0; a < nv; ++a)
                    for (int k2 = vdeg[t[a]]; k2 < vdeg[t[a] + 1]; ++k2) {
                        int c2 = vcell[k2], lo = c < c2 ? c : c2, hi = c < c2 ? c2 : c, dup = 0;
                        for (int q = 0; q < np && !dup; ++q) dup = pairs[2 * q] == lo && pairs[2 * q + 1] == hi;
                        if (!dup) { pairs[2 * np] = lo; pairs[2 * np + 1] = hi; ++np; }
                    }
            }
            for (int q = 0; q < np; ++q) {
                int c = pairs[2 * q], c2 = pairs[2 * q + 1];
                if (!in[c] && !in[c2]) continue;
                opair pp; int loc[5]; double L[25];
                int nl = make_pair(&m, c, c2, &pp, loc);
                int li = -1;
                for (int a = 0; a < nl; ++a) if (loc[a] == vi) li = a;
                if (li < 0) continue;
                pair_singular(&pp, &fs, &fk, sbar, ns, gx, gw, L);
                double wgt = (c == c2) ? 1.0 : 2.0, s = 0.0;
                for (int j = 0; j < nl; ++j) if (dof[loc[j]] >= 0) s += L[li * nl + j] * x[dof[loc[j]]];
                acc += wgt * s;
            }
            /* ---- K and M at the points of the interior cells containing vi ---- */
            for (int k = vdeg[vi]; k < vdeg[vi + 1]; ++k) {
                int c = vcell[k];
                if (!in[c]) continue;
                const int *t = T + c * nv;
                int ai = -1;
                for (int a = 0; a < nv; ++a) if (t[a] == vi) ai = a;
                for (int a = 0; a < nv; ++a)
                    for (int k2 = vdeg[t[a]]; k2 < vdeg[t[a] + 1]; ++k2) touch[vcell[k2]] = 1;
                for (int q = 0; q < nq; ++q) {
                    int iq = c * nq + q;
                    double sk = 0.0, rho = 0.0;
                    for (int c2 = 0; c2 < C; ++c2) {
                        if (touch[c2]) continue;
                        for (int q2 = 0; q2 < nq; ++q2) {
                            int jq = c2 * nq + q2;
                            double g = kernel_gamma(d, qdist(d, Q.x + iq * d, Q.x + jq * d), Q.s[iq], Q.s[jq],
                                                    Q.lk[iq], Q.lk[jq]) * Q.w[jq];
                            rho += g;
                            if (in[c2]) sk += g * xq[jq];
                        }
                    }
                    if (tail) rho += oracle_tail(d, Q.x + iq * d, Q.s[iq], exp(Q.lk[iq]), R);
                    double wpsi = Q.w[iq] * Q.bary[iq * NB + ai];
                    acc += -2.0 * wpsi * sk + 2.0 * wpsi * xq[iq] * rho;
                }
                for (int a = 0; a < nv; ++a)
                    for (int k2 = vdeg[t[a]]; k2 < vdeg[t[a] + 1]; ++k2) touch[vcell[k2]] = 0;
            }
            y[r] = acc;
        }
        free(touch); free(pairs);
    }
    free(xq); free(vdeg); free(vcell); free(dof); free(vert);
    free_quad(&Q);
    return N;
}

/* P1 load vector F_i = int f_h psi_i over interior cells (exact P1 mass
 * matrix times nodal f), DoF order of oracle_dofs. */
int oracle_load(int d, int M, int C, const double *X, const int *T, const unsigned char *in,
                const double *fnodal, double *F)
{
    omesh m = {d, M, C, X, T, in};
    int nv = d + 1;
    int *dof = malloc(sizeof(int) * M);
    int N = oracle_dofs(d, M, C, T, in, dof);
    memset(F, 0, sizeof(double) * N);
    for (int c = 0; c < C; ++c) {
        if (!in[c]) continue;
        double meas = cell_measure(&m, c);
        const int *t = T + c * nv;
        for (int a = 0; a < nv; ++a) {
            int i = dof[t[a]];
            if (i < 0) continue;
            for (int b = 0; b < nv; ++b) {
                /* int_tau lambda_a lambda_b = |tau| (1+delta_ab) d! / (d+2)! */
                double mab = meas * (a == b ? 2.0 : 1.0) / (d == 3 ? 20.0 : d == 2 ? 12.0 : 6.0);
                F[i] += mab * fnodal[t[b]];
            }
        }
    }
    free(dof);
    return N;
}

/* dense Cholesky solve of A U = F (A SPD, N x N row-major, overwritten by
 * its factor).  Returns 0 on success, k+1 if the k-th pivot is not positive. */
int oracle_cholesky_solve(int N, double *A, const double *F, double *U)
{
    for (int j = 0; j < N; ++j) {
        double djj = A[(size_t)j * N + j];
        for (int k = 0; k < j; ++k) djj -= A[(size_t)j * N + k] * A[(size_t)j * N + k];
        if (!(djj > 0.0)) return j + 1;
        djj = sqrt(djj);
        A[(size_t)j * N + j] = djj;
#pragma omp parallel for schedule(static)
        for (int i = j + 1; i < N; ++i) {
            double v = A[(size_t)i * N + j];
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * N + k] * A[(size_t)j * N + k];
            A[(size_t)i * N + j] = v / djj;
        }
    }
    for (int i = 0; i < N; ++i) {
        double v = F[i];
        for (int k = 0; k < i; ++k) v -= A[(size_t)i * N + k] * U[k];
        U[i] = v / A[(size_t)i * N + i];
    }
    for (int i = N - 1; i >= 0; --i) {
        double v = U[i];
        for (int k = i + 1; k < N; ++k) v -= A[(size_t)k * N + i] * U[k];
        U[i] = v / A[(size_t)i * N + i];
    }
    return 0;
}

/* the kernel and the field evaluation, exported for the pins */
double oracle_field(int d, const double *desc, const double *x) { return field_analytic(desc, d, x); }
double oracle_gamma(int d, double r, double sx, double sy, double lkx, double lky)
{
    return kernel_gamma(d, r, sx, sy, lkx, lky);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the following calls (timing baselines only) */
void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* plain conjugate gradients on the dense matrix (the paper's solver, Sec. 7),
 * for the CPU timing baseline: A U = F from U = 0 until ||F - A U|| <= rtol ||F||.
 * Returns the number of iterations (matrix-vector products). */
int oracle_cg(int N, const double *A, const double *F, double *U, double rtol, int max_it)
{
    double *r = malloc(sizeof(double) * N), *p = malloc(sizeof(double) * N), *q = malloc(sizeof(double) * N);
    double bb = 0.0, rr = 0.0;
    for (int i = 0; i < N; ++i) { U[i] = 0.0; r[i] = F[i]; p[i] = F[i]; bb += F[i] * F[i]; }
    rr = bb;
    int it = 0;
    while (it < max_it && rr > rtol * rtol * bb) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < N; ++i) {
            double v = 0.0;
            for (int j = 0; j < N; ++j) v += A[(size_t)i * N + j] * p[j];
            q[i] = v;
        }
        double pq = 0.0;
        for (int i = 0; i < N; ++i) pq += p[i] * q[i];
        double alpha = rr / pq, rn = 0.0;
        for (int i = 0; i < N; ++i) { U[i] += alpha * p[i]; r[i] -= alpha * q[i]; rn += r[i] * r[i]; }
        double beta = rn / rr;
        rr = rn;
        for (int i = 0; i < N; ++i) p[i] = r[i] + beta * p[i];
        ++it;
    }
    free(r); free(p); free(q);
    return it;
}
