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

__device__ __forceinline__ void trig_table(int d, int kmax, const double *x, TrigTable &t)
{
    for (int j = 0; j < d; ++j) {
        double sj, cj;
        sincospi(x[j], &sj, &cj);
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

__device__ __forceinline__ double field_terms(const DField &F, int d, const double *x, const TrigTable *tab)
{
    double v = F.c0;
    const double *r = F.rows;
    for (int t = 0; t < F.nF; ++t, r += 5) {
        double er = 1.0, ei = 0.0;  // e^{i pi k.x}
        if (tab) {
            for (int j = 0; j < d; ++j) {
                int kj = (int)r[j];
                int ak = kj < 0 ? -kj : kj;
                double cr = tab->c[j][ak], ci = kj < 0 ? -tab->s[j][ak] : tab->s[j][ak];
                double nr = er * cr - ei * ci, ni = er * ci + ei * cr;
                er = nr;
                ei = ni;
            }
        } else {
            double kx = 0.0;
            for (int j = 0; j < d; ++j) kx += r[j] * x[j];
            sincospi(kx, &ei, &er);
        }
        v += r[3] * er - r[4] * ei;  // amp cos(pi k.x + phase)
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
                                        const double *bary, double &s, double &lk)
{
    TrigTable tab;
    bool need = (!Fs.nodal && Fs.nF > 0 && Fs.kmax <= 4) || (!Fk.nodal && Fk.nF > 0 && Fk.kmax <= 4);
    int km = max(Fs.nodal ? 0 : Fs.kmax, Fk.nodal ? 0 : Fk.kmax);
    if (need) trig_table(d, km < 1 ? 1 : (km > 4 ? 4 : km), x, tab);
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
