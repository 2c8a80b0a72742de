// Device helpers shared by the kernels: field evaluation and the kernel gamma.
#pragma once

#include "vfd_internal.h"

namespace vfd {

// gamma(x,y) = sqrt(kappa(x) kappa(y)) |x-y|^-(d + s(x) + s(y))   (Sec. 2),
// from r^2 and the field values at both points.
__device__ __forceinline__ double gamma_r2(int d, double r2, double sx, double sy, double lkx, double lky)
{
    return exp(0.5 * (lkx + lky) - 0.5 * (d + sx + sy) * log(r2));
}

__device__ __forceinline__ float gamma_r2f(int d, float r2, float sx, float sy, float lkx, float lky)
{
    return __expf(0.5f * (lkx + lky) - 0.5f * (d + sx + sy) * __logf(r2));
}

// Fourier rows on the device are stored as (k1, k2, k3, amp cos(phase), amp sin(phase)).
struct TrigTable {
    double c[3][5], s[3][5];
};

__device__ __forceinline__ void sincospi_tab(const double *__restrict__ mt, double x, double &s, double &c);

// e^{i pi m x_j}, m = 0..kmax; with the math tables mt, sin/cos of pi x_j by
// the table-driven scheme, else by sincospi
__device__ __forceinline__ void trig_table(int d, int kmax, const double *x, TrigTable &t,
                                           const double *mt = nullptr)
{
    for (int j = 0; j < d; ++j) {
        double sj, cj;
        if (mt) sincospi_tab(mt, x[j], sj, cj);
        else sincospi(x[j], &sj, &cj);
        t.c[j][0] = 1.0;
        t.s[j][0] = 0.0;
        t.c[j][1] = cj;
        t.s[j][1] = sj;
        for (int m = 2; m <= kmax; ++m) {
            t.c[j][m] = t.c[j][m - 1] * cj - t.s[j][m - 1] * sj;
            t.s[j][m] = t.s[j][m - 1] * cj + t.c[j][m - 1] * sj;
        }
    }
}

// A Fourier row (k, A = amp e^{i phase}) contributes Re(A e^{i pi k.x}).  With
// the trig table the rows are summed in groups of equal k_1:
// Re(e^{i pi k_1 x_1} sum_group A e^{i pi (k_2 x_2 + k_3 x_3)}).  2D rows with
// integer |k| <= 4 use the grouping prepared on the host (integer indices, the
// signs folded into four coefficients per row: four FMAs per row); other rows
// (sorted by k_1 on the host) are grouped on the fly.
__device__ __forceinline__ double field_terms(const DField &F, int d, const double *x, const TrigTable *tab)
{
    double v = F.c0;
    const double *r = F.rows;
    if (tab && F.ngrp > 0 && d == 2) {
        const int *mk = F.gint + 2 * F.ngrp;
        const double *a = F.gcoef;
        for (int g = 0; g < F.ngrp; ++g) {
            const int k1 = F.gint[2 * g], nm = F.gint[2 * g + 1];
            double gr = 0.0, gq = 0.0;
            for (int q = 0; q < nm; ++q, ++mk, a += 4) {
                const double c = tab->c[1][*mk], s = tab->s[1][*mk];
                gr = fma(a[0], c, fma(a[1], s, gr));
                gq = fma(a[2], s, fma(a[3], c, gq));
            }
            v = fma(tab->c[0][k1], gr, fma(tab->s[0][k1], gq, v));
        }
        r += 5 * F.nF;
    } else if (tab) {
        int t = 0;
        while (t < F.nF) {
            const int k1 = (int)r[5 * t];
            double gr = 0.0, gi = 0.0;
            for (; t < F.nF && (int)r[5 * t] == k1; ++t) {
                const double *q = r + 5 * t;
                double er = q[3], ei = q[4];
                for (int j = 1; j < d; ++j) {
                    const int kj = (int)q[j], ak = kj < 0 ? -kj : kj;
                    const double cr = tab->c[j][ak], ci = kj < 0 ? -tab->s[j][ak] : tab->s[j][ak];
                    const double nr = fma(er, cr, -ei * ci), ni = fma(er, ci, ei * cr);
                    er = nr;
                    ei = ni;
                }
                gr += er;
                gi += ei;
            }
            const int a1 = k1 < 0 ? -k1 : k1;
            const double ur = tab->c[0][a1], ui = k1 < 0 ? -tab->s[0][a1] : tab->s[0][a1];
            v = fma(ur, gr, fma(-ui, gi, v));
        }
        r += 5 * F.nF;
    } else {
        for (int t = 0; t < F.nF; ++t, r += 5) {
            double er, ei;   // e^{i pi k.x}
            double kx = 0.0;
            for (int j = 0; j < d; ++j) kx += r[j] * x[j];
            sincospi(kx, &ei, &er);
            v += r[3] * er - r[4] * ei;  // amp cos(pi k.x + phase)
        }
    }
    for (int t = 0; t < F.nG; ++t, r += 5) {
        double q = 0.0;
        for (int j = 0; j < d; ++j) q += (x[j] - r[j]) * (x[j] - r[j]);
        v += r[3] * exp(-r[4] * q);
    }
    for (int t = 0; t < F.nT; ++t, r += 5) {
        double pr = r[3];
        for (int j = 0; j < d; ++j) {
            double rr = 2.0 * (x[j] - r[j]) / r[4];
            pr *= (fabs(rr) < 1.0) ? exp(-1.0 / (1.0 - rr * rr)) : 0.0;
        }
        v += pr;
    }
    if (F.squash) v = F.lo + (F.hi - F.lo) / (1.0 + exp(-v));
    return v;
}

// s and log kappa at a point.  For P1 fields the point must lie in a cell
// with vertex ids vid[0..d] and barycentric coordinates bary.
__device__ __forceinline__ void fields2(const DField &Fs, const DField &Fk, int d, const double *x, const int *vid,
                                        const double *bary, double &s, double &lk, const double *mt = nullptr)
{
    TrigTable tab;
    bool need = (!Fs.nodal && Fs.nF > 0 && Fs.kmax <= 4) || (!Fk.nodal && Fk.nF > 0 && Fk.kmax <= 4);
    int km = max(Fs.nodal ? 0 : Fs.kmax, Fk.nodal ? 0 : Fk.kmax);
    if (need) trig_table(d, km < 1 ? 1 : (km > 4 ? 4 : km), x, tab, mt);
    if (Fs.nodal) {
        s = 0.0;
        for (int a = 0; a <= d; ++a) s += bary[a] * Fs.vals[vid[a]];
    } else {
        s = field_terms(Fs, d, x, (Fs.nF > 0 && Fs.kmax <= 4) ? &tab : nullptr);
    }
    if (Fk.nodal) {
        lk = 0.0;
        for (int a = 0; a <= d; ++a) lk += bary[a] * Fk.vals[vid[a]];
    } else {
        lk = field_terms(Fk, d, x, (Fk.nF > 0 && Fk.kmax <= 4) ? &tab : nullptr);
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace vfd

namespace vfd {

// ---------------------------------------------------------------------------
// Table-driven FP64 logarithm and exponential (P. T. P. Tang, "Table-driven
// implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16(4) 1990, and "Table-driven implementation of the
// exponential function in IEEE floating-point arithmetic", ACM TOMS 15(2)
// 1989), used for the kernel evaluations gamma on GB300, whose FP64 pipe is
// 1/58 of FP32.  Table layout (built on the host by make_math_tables):
//   [0..128]   c_j = 1/F_j, F_j = 1 + j/128
//   [129..257] log F_j
//   [258..321] 2^(j/64)
//   [322..325] ln2_hi, ln2_lo, ln2/64 hi, ln2/64 lo   (Cody-Waite splits)
//   [326..453] cos(pi j/64), [454..581] sin(pi j/64), j = 0..127
// Valid for normal positive x (log) and |y| < 700 (exp); relative error of a
// few ulp (tests/test_gpu_math.py).
// ---------------------------------------------------------------------------
constexpr int MT_C = 0, MT_LOGF = 129, MT_EXP2 = 258, MT_CONST = 322, MT_COSPI = 326, MT_SINPI = 454,
              MT_SIZE = 582;

__device__ __forceinline__ double fast_log(const double *__restrict__ mt, double x)
{
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7ff) - 1023;
    const double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    const int j = (int)(((bits >> 44) & 0xff) + 1) >> 1;   // nearest j/128 to m - 1
    const double r = fma(m, __ldg(mt + MT_C + j), -1.0);   // |r| <= 2^-8
    // log(1 + r) = r q(r) through r^6 (the next term, r^7 / 7, is below 2^-58)
    double q = -1.0 / 6.0;
    q = fma(q, r, 1.0 / 5.0);
    q = fma(q, r, -0.25);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    q = fma(q, r, 1.0);
    const double ed = (double)e;
    return fma(ed, __ldg(mt + MT_CONST), __ldg(mt + MT_LOGF + j) + fma(ed, __ldg(mt + MT_CONST + 1), q * r));
}

__device__ __forceinline__ double fast_exp(const double *__restrict__ mt, double y)
{
    y = fmin(fmax(y, -700.0), 700.0);
    // k = nearest integer to y 64/ln2: adding 1.5 2^52 leaves it in the low bits
    const double big = 6755399441055744.0;
    const double tk = fma(y, 92.33248261689366, big);   // 64 / ln 2
    const double kf = tk - big;
    const long long ki = (long long)(int)__double2loint(tk);
    double r = fma(-kf, __ldg(mt + MT_CONST + 2), y);
    r = fma(-kf, __ldg(mt + MT_CONST + 3), r);        // |r| <= ln2/128 (+ rounding)
    // exp(r) = 1 + r q(r) through r^5 (the next term, r^6 / 720, is below 4e-17)
    double q = 1.0 / 120.0;
    q = fma(q, r, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    q = fma(q, r, 1.0);
    const double s = __ldg(mt + MT_EXP2 + (int)(ki & 63));
    const double v = fma(s, q * r, s);
    return __longlong_as_double(__double_as_longlong(v) + ((ki >> 6) << 52));
}

// sin and cos of pi x by the same table-driven scheme: x = j/64 + f with j the
// nearest integer to 64 x and |f| <= 1/128, the table's values at pi j/64
// combined with the Taylor series of cos and sin at theta = pi f (|theta| <=
// pi/128; cos through theta^6, sin through theta^7, truncation below 4e-18)
__device__ __forceinline__ void sincospi_tab(const double *__restrict__ mt, double x, double &s, double &c)
{
    const double big = 6755399441055744.0;   // 1.5 2^52
    const double tj = fma(x, 64.0, big);
    const double jf = tj - big;
    const int j = (int)__double2loint(tj) & 127;
    const double th = 3.141592653589793 * fma(jf, -1.0 / 64.0, x), u = th * th;
    const double ct = fma(fma(fma(u, -1.0 / 720.0, 1.0 / 24.0), u, -0.5), u, 1.0);
    const double st = th * fma(fma(fma(u, -1.0 / 5040.0, 1.0 / 120.0), u, -1.0 / 6.0), u, 1.0);
    const double cj = __ldg(mt + MT_COSPI + j), sj = __ldg(mt + MT_SINPI + j);
    c = fma(cj, ct, -sj * st);
    s = fma(sj, ct, cj * st);
}

// gamma from r^2 and per-point exponent terms a = log(kappa)/2 (plus any log
// weight folded in) and b = s/2 + d/4: exp(a_x + a_y - (b_x + b_y) log r^2)
__device__ __forceinline__ double gamma_ab(const double *__restrict__ mt, double r2, double ax, double ay, double bx,
                                           double by)
{
    return fast_exp(mt, (ax + ay) - (bx + by) * fast_log(mt, r2));
}

// gamma from r^2 with the table-driven log/exp
__device__ __forceinline__ double gamma_r2t(const double *__restrict__ mt, int d, double r2, double sx, double sy,
                                            double lkx, double lky)
{
    return fast_exp(mt, 0.5 * (lkx + lky) - 0.5 * (d + sx + sy) * fast_log(mt, r2));
}

}  // namespace vfd
