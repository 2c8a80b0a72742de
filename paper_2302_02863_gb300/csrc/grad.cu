// Adjoint gradient of the discrete operator with respect to the nodal values
// of s and of log kappa (P1 fields):
//
//   g_s[k]  = -sum_r Lam_r^T (dA/ds_k) U_r,   g_lk[k] = -sum_r Lam_r^T (dA/dlogk_k) U_r.
//
// The paper has no gradients; A is the operator the solves use (Sec. 3,
// A = B + K + M, with K's admissible blocks and the density's far part in
// their interpolated H^2 forms of Sec. 5.3 and 6.2), every quadrature rule held
// fixed.  Every term carries the kernel
// gamma(x,y) = sqrt(kappa(x) kappa(y)) |x-y|^-(d+s(x)+s(y)), so
//   d gamma / d s(x) = -ln|x-y| gamma,   d gamma / d logk(x) = gamma / 2,
// where x is an element-rule point, a singular-rule point or, inside an
// interpolated block, a Chebyshev node whose field value is the P1
// interpolant at the node's nearest mesh point.  The contributions, each an
// "s-sensitivity" -d(Lam^T A U)/d s(x) at one point x, pushed to the vertices
// through the barycentric coordinates of x:
//
//   B (touching pairs)   the singular rules of Sec. 4 point by point, with
//                        d(log w)/dS read off the factors of the rule weight
//                        that depend on S (k_grad_sing);
//   K near blocks        D_ab = -2 sum_{q in P_a, q' in P_b} gamma_T(q,q')
//                        c_a(q) c_b(q'), c_a(q) = w_q sum_{i in a} psi_i(q) x_i:
//                        per row leaf a and point q of P_a the sum over the
//                        leaf's blocks of gamma_T (c_a^Lam(q) c_b^U(q') +
//                        c_a^U(q) c_b^Lam(q')) (k_gh_knear);
//   K admissible blocks  Lam^T U_a S_ab U_b^T U, S_ab = -2 gamma(xi, eta): per
//                        node and Chebyshev node xi the same contraction with
//                        the moments Uhat_b, Lamhat_b of the upsweep and S
//                        recomputed on the fly (k_gh_kfar);
//   M (density)          Lam^T M U = sum_q c_q rho(q), c_q = 2 w_q Lam(q) U(q):
//                        near sources by direct sums on the target side and,
//                        over the transposed lists, on the source side
//                        (k_gh_rho_near_t / _s); far sources through the target
//                        moments chat_t = sum_q c_q l^t(q) and the source
//                        moments (k_gh_rho_moments, k_gh_rho_far_t / _s).
//
// With lambda = rho_lambda = 0 every block is near and the density a direct
// sum: the same kernels then give the gradient of the exact-mode operator.
// All sums run in a fixed order (per-point and per-node results gathered per
// vertex through precomputed lists), so the result is deterministic.
#include <algorithm>
#include <cmath>

#include "device_common.cuh"

namespace vfd {

namespace {

// U and Lam at the element-rule points: Uq[r][q] = sum_a bary_a U[dof(v_a)]
__global__ void k_grad_vals(int nQ, int d, int nrhs, int64_t ld, const int *__restrict__ qcell,
                            const double *__restrict__ qbary, const int *__restrict__ cells,
                            const int *__restrict__ vdof, const double *__restrict__ U, const double *__restrict__ Lam,
                            double *__restrict__ Uq, double *__restrict__ Lq)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nQ) return;
    const int nv = d + 1, c = qcell[q];
    for (int r = 0; r < nrhs; ++r) {
        double u = 0.0, l = 0.0;
        for (int a = 0; a < nv; ++a) {
            const int i = vdof[cells[(size_t)c * nv + a]];
            if (i >= 0) {
                u += qbary[(size_t)q * QB + a] * U[(size_t)r * ld + i];
                l += qbary[(size_t)q * QB + a] * Lam[(size_t)r * ld + i];
            }
        }
        Uq[(size_t)r * nQ + q] = u;
        Lq[(size_t)r * nQ + q] = l;
    }
}


constexpr int GT = 128;     // points per CTA and per staged tile
constexpr int GNR = 8;      // right-hand sides per pass of the K kernels

// c_q = 2 w_q sum_r Lam_r(q) U_r(q) at the interior points (0 elsewhere)
__global__ void k_gh_cq(int nQ, int nQint, int nrhs, const double *__restrict__ qw, const double *__restrict__ Uq,
                        const double *__restrict__ Lq, double *__restrict__ cq)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nQ) return;
    double v = 0.0;
    if (q < nQint)
        for (int r = 0; r < nrhs; ++r) v = fma(Uq[(size_t)r * nQ + q], Lq[(size_t)r * nQ + q], v);
    cq[q] = 2.0 * qw[q] * v;
}

struct GKN {
    int nQ, fl, nr, accumulate;
    int64_t ld;
    const double *U, *Lam;   // first column of this pass
    const int *kt_begin, *kt_end, *lp_ptr, *lp_pts, *near_ptr, *near_col;
    const double *qx, *qw, *qs, *qlk, *qbary;
    const int *qcell, *cells, *vdof;
    const double *mt;
    double *hs, *hk;   // per leaf-point entry
};

// c_a(q) for the columns of this pass: w_q sum over the cell's vertices whose
// DoF lies in [r0, r1) of the barycentric coordinate times x
template <int NV>
__device__ __forceinline__ void leaf_coef(const GKN &P, int q, int r0, int r1, double *cl, double *cu)
{
    const int cell = P.qcell[q];
    const double w = P.qw[q];
#pragma unroll
    for (int r = 0; r < GNR; ++r) cl[r] = cu[r] = 0.0;
    for (int k = 0; k < NV; ++k) {
        const int i = P.vdof[P.cells[(size_t)cell * NV + k]];
        if (i >= r0 && i < r1) {
            const double c = w * P.qbary[(size_t)q * QB + k];
#pragma unroll
            for (int r = 0; r < GNR; ++r)
                if (r < P.nr) {
                    cl[r] = fma(c, P.Lam[(size_t)r * P.ld + i], cl[r]);
                    cu[r] = fma(c, P.U[(size_t)r * P.ld + i], cu[r]);
                }
        }
    }
}

// K near blocks, row side: CTA (row leaf a, slice of GT points of P_a); the
// column points of every block (a, b) staged in tiles
template <int D>
__global__ void __launch_bounds__(GT) k_gh_knear(GKN P)
{
    constexpr int NV = D + 1;
    __shared__ double sx[D][GT], sa[GT], sb[GT], sl[GNR][GT], su[GNR][GT];
    __shared__ int sv[NV][GT];
    const int a = blockIdx.x;
    const int pa0 = P.lp_ptr[a], npa = P.lp_ptr[a + 1] - pa0;
    if ((int)blockIdx.y * GT >= npa) return;   // the whole CTA
    const int t = blockIdx.y * GT + threadIdx.x;
    const bool live = t < npa;
    const int q = P.lp_pts[pa0 + (live ? t : 0)];
    double x[D];
    for (int c = 0; c < D; ++c) x[c] = P.qx[(size_t)c * P.nQ + q];
    const double aq = 0.5 * P.qlk[q], bq = fma(0.5, P.qs[q], 0.25 * D);
    int v[NV];
    for (int k = 0; k < NV; ++k) v[k] = P.cells[(size_t)P.qcell[q] * NV + k];
    double cl[GNR], cu[GNR];
    leaf_coef<NV>(P, q, P.kt_begin[P.fl + a], P.kt_end[P.fl + a], cl, cu);
    double accs = 0.0, acc1 = 0.0;
    for (int e = P.near_ptr[a]; e < P.near_ptr[a + 1]; ++e) {
        const int b = P.near_col[e];
        const int pb0 = P.lp_ptr[b], npb = P.lp_ptr[b + 1] - pb0;
        const int rb0 = P.kt_begin[P.fl + b], rb1 = P.kt_end[P.fl + b];
        for (int j0 = 0; j0 < npb; j0 += GT) {
            const int nt = min(GT, npb - j0);
            __syncthreads();
            if ((int)threadIdx.x < nt) {
                const int id = P.lp_pts[pb0 + j0 + threadIdx.x];
                for (int c = 0; c < D; ++c) sx[c][threadIdx.x] = P.qx[(size_t)c * P.nQ + id];
                sa[threadIdx.x] = 0.5 * P.qlk[id];
                sb[threadIdx.x] = fma(0.5, P.qs[id], 0.25 * D);
                for (int k = 0; k < NV; ++k) sv[k][threadIdx.x] = P.cells[(size_t)P.qcell[id] * NV + k];
                double ml[GNR], mu[GNR];
                leaf_coef<NV>(P, id, rb0, rb1, ml, mu);
#pragma unroll
                for (int r = 0; r < GNR; ++r) {
                    sl[r][threadIdx.x] = ml[r];
                    su[r][threadIdx.x] = mu[r];
                }
            }
            __syncthreads();
            if (live)
                for (int jj = 0; jj < nt; ++jj) {
                    bool touch = false;
#pragma unroll
                    for (int i = 0; i < NV; ++i)
#pragma unroll
                        for (int k = 0; k < NV; ++k) touch |= (v[i] == sv[k][jj]);
                    if (touch) continue;   // touching cells belong to B
                    double r2 = 0.0;
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        const double dd = x[c] - sx[c][jj];
                        r2 = fma(dd, dd, r2);
                    }
                    const double lr2 = fast_log(P.mt, r2);
                    const double g = fast_exp(P.mt, aq + sa[jj] - (bq + sb[jj]) * lr2);
                    double X = 0.0;
#pragma unroll
                    for (int r = 0; r < GNR; ++r)
                        if (r < P.nr) X = fma(cl[r], su[r][jj], fma(cu[r], sl[r][jj], X));
                    const double tX = g * X;
                    acc1 += tX;
                    accs = fma(tX, lr2, accs);
                }
        }
    }
    if (live) {
        // -d/ds(q) of -2 gamma X = -ln(r^2) gamma X; -d/dlogk(q) = gamma X
        const size_t o = (size_t)pa0 + t;
        P.hs[o] = P.accumulate ? P.hs[o] - accs : -accs;
        P.hk[o] = P.accumulate ? P.hk[o] + acc1 : acc1;
    }
}

// K far moments of U and Lam for the nodes with admissible blocks:
// xU[r][n][alpha] = sum_{i in n} Ul^(level n)[i][alpha] U_r[i]
__global__ void __launch_bounds__(128)
k_gh_moments(int nr, int k, int N, int lmin, int nnode, const int *__restrict__ fptr, const int *__restrict__ kb,
             const int *__restrict__ ke, const double *__restrict__ Ul, const double *__restrict__ U,
             const double *__restrict__ Lam, int64_t ld, double *__restrict__ xU, double *__restrict__ xL)
{
    __shared__ double ru[128], rl[128];
    const int n = blockIdx.x;
    if (fptr[n + 1] == fptr[n]) return;
    int l = 0;
    while ((2 << l) - 1 <= n) ++l;
    const int lv = l - lmin;
    const int b = kb[n], e = ke[n];
    const int kk = min(k, (int)blockDim.x), parts = blockDim.x / kk;
    const int al = threadIdx.x % kk, pt = threadIdx.x / kk;
    const double *u = Ul + (size_t)lv * N * k;
    for (int r = 0; r < nr; ++r)
        for (int a0 = 0; a0 < k; a0 += kk) {
            double au = 0.0, aL = 0.0;
            if (pt < parts)
                for (int i = b + pt; i < e; i += parts) {
                    const double w = u[(size_t)i * k + a0 + al];
                    au = fma(w, U[(size_t)r * ld + i], au);
                    aL = fma(w, Lam[(size_t)r * ld + i], aL);
                }
            ru[threadIdx.x] = au;
            rl[threadIdx.x] = aL;
            __syncthreads();
            if ((int)threadIdx.x < kk) {
                double su = 0.0, sl = 0.0;
                for (int q = 0; q < parts; ++q) {
                    su += ru[q * kk + threadIdx.x];
                    sl += rl[q * kk + threadIdx.x];
                }
                xU[((size_t)r * nnode + n) * k + a0 + threadIdx.x] = su;
                xL[((size_t)r * nnode + n) * k + a0 + threadIdx.x] = sl;
            }
            __syncthreads();
        }
}

// K admissible blocks: per row node a and node alpha, over the blocks e of
// the row (threads (alpha, block slot)), S_e recomputed:
//   Gs[a][alpha] += sum_e sum_beta ln(r^2)/2 S (Lhat_a Uhat_b + Uhat_a Lhat_b),
//   Gk[a][alpha] -= sum_e sum_beta S/2 (Lhat_a Uhat_b + Uhat_a Lhat_b)
__global__ void __launch_bounds__(256)
k_gh_kfar(int d, int k, int nnode, int nr, const int *__restrict__ fptr, const int *__restrict__ fcol,
          const double *__restrict__ ch, const double *__restrict__ cs, const double *__restrict__ clk,
          const double *__restrict__ xU, const double *__restrict__ xL, const double *__restrict__ mt,
          double *__restrict__ Gs, double *__restrict__ Gk)
{
    __shared__ double rs[256], rk[256];
    const int a = blockIdx.x;
    const int e0 = fptr[a], ne = fptr[a + 1] - e0;
    if (ne == 0) return;
    const int al = threadIdx.x % k, g = threadIdx.x / k, per = blockDim.x / k;
    const int ia = a * k + al;
    double xa[3];
    for (int c = 0; c < d; ++c) xa[c] = ch[(size_t)ia * d + c];
    const double sa = cs[ia], la = clk[ia];
    double Ua[GNR], La[GNR];
#pragma unroll
    for (int r = 0; r < GNR; ++r) {
        Ua[r] = r < nr ? xU[((size_t)r * nnode + a) * k + al] : 0.0;
        La[r] = r < nr ? xL[((size_t)r * nnode + a) * k + al] : 0.0;
    }
    double gs = 0.0, gk = 0.0;
    if (g < per)
        for (int e = g; e < ne; e += per) {
            const int b = fcol[e0 + e];
            double yU[GNR], yL[GNR], zU[GNR], zL[GNR];
#pragma unroll
            for (int r = 0; r < GNR; ++r) yU[r] = yL[r] = zU[r] = zL[r] = 0.0;
            for (int be = 0; be < k; ++be) {
                const int jb = b * k + be;
                double r2 = 0.0;
                for (int c = 0; c < d; ++c) {
                    const double dd = xa[c] - ch[(size_t)jb * d + c];
                    r2 = fma(dd, dd, r2);
                }
                const double lr2 = fast_log(mt, r2);
                const double S = -2.0 * fast_exp(mt, 0.5 * (la + clk[jb]) - 0.5 * (d + sa + cs[jb]) * lr2);
                const double hS = 0.5 * lr2 * S;
#pragma unroll
                for (int r = 0; r < GNR; ++r)
                    if (r < nr) {
                        const double ub = xU[((size_t)r * nnode + b) * k + be], lb = xL[((size_t)r * nnode + b) * k + be];
                        yU[r] = fma(hS, ub, yU[r]);
                        yL[r] = fma(hS, lb, yL[r]);
                        zU[r] = fma(S, ub, zU[r]);
                        zL[r] = fma(S, lb, zL[r]);
                    }
            }
#pragma unroll
            for (int r = 0; r < GNR; ++r) {
                gs += La[r] * yU[r] + Ua[r] * yL[r];
                gk -= 0.5 * (La[r] * zU[r] + Ua[r] * zL[r]);
            }
        }
    rs[threadIdx.x] = gs;
    rk[threadIdx.x] = gk;
    __syncthreads();
    if (g == 0) {
        double ts = 0.0, tk = 0.0;
        for (int q = 0; q < per; ++q) {
            ts += rs[q * k + al];
            tk += rk[q * k + al];
        }
        Gs[ia] += ts;
        Gk[ia] += tk;
    }
}

struct GRho {
    int d, nv, nQ, k, p;
    int tfl, sfl;   // first leaf of the target / source tree
    const int *tt_begin, *tt_end, *tt_perm, *st_begin, *st_end, *st_perm;
    const int *rnear_ptr, *rnear_col, *rnearT_ptr, *rnearT_col;
    const double *qx, *qw, *qs, *qlk, *cq;
    const int *qcell, *cells;
    const double *mt;
    double *hs, *hk;   // per point
};

constexpr int RCH = 128;   // staged points per tile of the density kernels

// density near part, target side: per interior point q
//   hs[q] = c_q/2 sum_{q'} w' gamma ln(r^2),  hk[q] = -c_q/2 sum_{q'} w' gamma
__global__ void __launch_bounds__(RCH) k_gh_rho_near_t(GRho P)
{
    __shared__ double sx[3][RCH], ss[RCH], sl[RCH];
    __shared__ int sv[4][RCH];
    const int d = P.d, leaf = blockIdx.x, node = P.tfl + leaf;
    const int b = P.tt_begin[node], e = P.tt_end[node];
    for (int i0 = b; i0 < e; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const bool act = i < e;
        const int id = act ? P.tt_perm[i] : P.tt_perm[b];
        double x[3] = {0, 0, 0};
        for (int c = 0; c < d; ++c) x[c] = P.qx[(size_t)c * P.nQ + id];
        const double a_ = 0.5 * P.qlk[id], b_ = fma(0.5, P.qs[id], 0.25 * d);
        int cv[4] = {-1, -1, -1, -1};
        for (int a = 0; a < P.nv; ++a) cv[a] = P.cells[(size_t)P.qcell[id] * P.nv + a];
        double accs = 0.0, acc1 = 0.0;
        for (int ne = P.rnear_ptr[leaf]; ne < P.rnear_ptr[leaf + 1]; ++ne) {
            const int sn = P.rnear_col[ne];
            const int sb = P.st_begin[sn], se = P.st_end[sn];
            for (int j0 = sb; j0 < se; j0 += RCH) {
                const int nj = min(RCH, se - j0);
                __syncthreads();
                if ((int)threadIdx.x < nj) {
                    const int jd = P.st_perm[j0 + threadIdx.x];
                    for (int c = 0; c < d; ++c) sx[c][threadIdx.x] = P.qx[(size_t)c * P.nQ + jd];
                    ss[threadIdx.x] = fma(0.5, P.qs[jd], 0.25 * d);
                    sl[threadIdx.x] = fma(0.5, P.qlk[jd], fast_log(P.mt, P.qw[jd]));
                    for (int a = 0; a < 4; ++a)
                        sv[a][threadIdx.x] = a < P.nv ? P.cells[(size_t)P.qcell[jd] * P.nv + a] : -2;
                }
                __syncthreads();
                if (act)
                    for (int t = 0; t < nj; ++t) {
                        bool touch = false;
                        for (int a = 0; a < P.nv; ++a)
                            for (int bb = 0; bb < P.nv; ++bb) touch |= (cv[a] == sv[bb][t]);
                        if (touch) continue;
                        double r2 = 0.0;
                        for (int c = 0; c < d; ++c) {
                            const double dd = x[c] - sx[c][t];
                            r2 = fma(dd, dd, r2);
                        }
                        const double lr2 = fast_log(P.mt, r2);
                        const double g = fast_exp(P.mt, a_ + sl[t] - (b_ + ss[t]) * lr2);   // w' gamma
                        acc1 += g;
                        accs = fma(g, lr2, accs);
                    }
            }
        }
        if (act) {
            const double c = P.cq[id];
            P.hs[id] = 0.5 * c * accs;
            P.hk[id] = -0.5 * c * acc1;
        }
    }
}

// density near part, source side: per point q' of a source leaf, over the
// target leaves whose near list holds it
//   hs[q'] += w'/2 sum_q c_q gamma ln(r^2),  hk[q'] -= w'/2 sum_q c_q gamma
__global__ void __launch_bounds__(RCH) k_gh_rho_near_s(GRho P)
{
    __shared__ double sx[3][RCH], ss[RCH], sl[RCH], sc[RCH];
    __shared__ int sv[4][RCH];
    const int d = P.d, sleaf = blockIdx.x, node = P.sfl + sleaf;
    const int b = P.st_begin[node], e = P.st_end[node];
    for (int i0 = b; i0 < e; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const bool act = i < e;
        const int id = act ? P.st_perm[i] : P.st_perm[b];
        double x[3] = {0, 0, 0};
        for (int c = 0; c < d; ++c) x[c] = P.qx[(size_t)c * P.nQ + id];
        const double a_ = 0.5 * P.qlk[id], b_ = fma(0.5, P.qs[id], 0.25 * d);
        int cv[4] = {-1, -1, -1, -1};
        for (int a = 0; a < P.nv; ++a) cv[a] = P.cells[(size_t)P.qcell[id] * P.nv + a];
        double accs = 0.0, acc1 = 0.0;
        for (int ne = P.rnearT_ptr[sleaf]; ne < P.rnearT_ptr[sleaf + 1]; ++ne) {
            const int tn = P.tfl + P.rnearT_col[ne];
            const int tb = P.tt_begin[tn], te = P.tt_end[tn];
            for (int j0 = tb; j0 < te; j0 += RCH) {
                const int nj = min(RCH, te - j0);
                __syncthreads();
                if ((int)threadIdx.x < nj) {
                    const int jd = P.tt_perm[j0 + threadIdx.x];
                    for (int c = 0; c < d; ++c) sx[c][threadIdx.x] = P.qx[(size_t)c * P.nQ + jd];
                    ss[threadIdx.x] = fma(0.5, P.qs[jd], 0.25 * d);
                    sl[threadIdx.x] = 0.5 * P.qlk[jd];
                    sc[threadIdx.x] = P.cq[jd];
                    for (int a = 0; a < 4; ++a)
                        sv[a][threadIdx.x] = a < P.nv ? P.cells[(size_t)P.qcell[jd] * P.nv + a] : -2;
                }
                __syncthreads();
                if (act)
                    for (int t = 0; t < nj; ++t) {
                        bool touch = false;
                        for (int a = 0; a < P.nv; ++a)
                            for (int bb = 0; bb < P.nv; ++bb) touch |= (cv[a] == sv[bb][t]);
                        if (touch) continue;
                        double r2 = 0.0;
                        for (int c = 0; c < d; ++c) {
                            const double dd = x[c] - sx[c][t];
                            r2 = fma(dd, dd, r2);
                        }
                        const double lr2 = fast_log(P.mt, r2);
                        const double cg = sc[t] * fast_exp(P.mt, a_ + sl[t] - (b_ + ss[t]) * lr2);
                        acc1 += cg;
                        accs = fma(cg, lr2, accs);
                    }
            }
        }
        if (act) {
            const double w = P.qw[id];
            P.hs[id] += 0.5 * w * accs;
            P.hk[id] -= 0.5 * w * acc1;
        }
    }
}

// target moments chat[t][alpha] = sum_{q in t} c_q l^t_alpha(q) for the target
// nodes with admissible blocks (the transpose of the downsweep's evaluation)
constexpr int MCH = 64;
__global__ void __launch_bounds__(128)
k_gh_rho_moments(int d, int p, int k, int nQ, const int *__restrict__ fptr, const int *__restrict__ tb,
                 const int *__restrict__ te, const int *__restrict__ perm, const double *__restrict__ tch,
                 const double *__restrict__ qx, const double *__restrict__ cq, double *__restrict__ chat)
{
    __shared__ double l1[MCH][3][PMAX], sc[MCH];
    const int t = blockIdx.x;
    if (fptr[t + 1] == fptr[t]) return;
    const double *ch = tch + (size_t)t * k * d;
    const int b = tb[t], e = te[t];
    double acc = 0.0;
    for (int i0 = b; i0 < e; i0 += MCH) {
        const int n = min(MCH, e - i0);
        __syncthreads();
        for (int pt = threadIdx.x; pt < n; pt += blockDim.x) {
            const int id = perm[i0 + pt];
            int stride = 1;
            for (int c = 0; c < d; ++c) {
                const double x = qx[(size_t)c * nQ + id];
                for (int a = 0; a < p; ++a) {
                    const double na = ch[(size_t)(a * stride) * d + c];
                    double v = 1.0;
                    for (int bb = 0; bb < p; ++bb)
                        if (bb != a) {
                            const double nb = ch[(size_t)(bb * stride) * d + c];
                            v *= (x - nb) / (na - nb);
                        }
                    l1[pt][c][a] = v;
                }
                stride *= p;
            }
            sc[pt] = cq[id];
        }
        __syncthreads();
        if ((int)threadIdx.x < k)
            for (int pt = 0; pt < n; ++pt) {
                double v = sc[pt];
                int r = threadIdx.x;
                for (int c = 0; c < d; ++c) {
                    v *= l1[pt][c][r % p];
                    r /= p;
                }
                acc += v;
            }
    }
    if ((int)threadIdx.x < k) chat[(size_t)t * k + threadIdx.x] = acc;
}

// density far part, target nodes: thread per (t, alpha)
//   Gs = chat/2 sum gamma ln(r^2) xs,  Gk = -chat/2 sum gamma xs
__global__ void k_gh_rho_far_t(int d, int k, int nnode_t, const int *__restrict__ fptr, const int *__restrict__ fcol,
                               const double *__restrict__ tch, const double *__restrict__ ts,
                               const double *__restrict__ tlk, const double *__restrict__ sch,
                               const double *__restrict__ ss, const double *__restrict__ slk,
                               const double *__restrict__ xs, const double *__restrict__ chat,
                               const double *__restrict__ mt, double *__restrict__ Gs, double *__restrict__ Gk)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnode_t * k) return;
    const int t = i / k;
    double accs = 0.0, acc1 = 0.0;
    if (fptr[t + 1] > fptr[t]) {
        const double *xa = tch + (size_t)i * d;
        const double sa = ts[i], la = tlk[i];
        for (int e = fptr[t]; e < fptr[t + 1]; ++e) {
            const int s = fcol[e];
            for (int be = 0; be < k; ++be) {
                const int j = s * k + be;
                double r2 = 0.0;
                for (int c = 0; c < d; ++c) {
                    const double dd = xa[c] - sch[(size_t)j * d + c];
                    r2 = fma(dd, dd, r2);
                }
                const double lr2 = fast_log(mt, r2);
                const double g = fast_exp(mt, 0.5 * (la + slk[j]) - 0.5 * (d + sa + ss[j]) * lr2) * xs[j];
                acc1 += g;
                accs = fma(g, lr2, accs);
            }
        }
        accs *= 0.5 * chat[i];
        acc1 *= -0.5 * chat[i];
    }
    Gs[i] = accs;
    Gk[i] = acc1;
}

// density far part, source nodes: thread per (s, beta) over the target nodes
// whose admissible list holds s
__global__ void k_gh_rho_far_s(int d, int k, int nnode_s, const int *__restrict__ tptr, const int *__restrict__ tcol,
                               const double *__restrict__ tch, const double *__restrict__ ts,
                               const double *__restrict__ tlk, const double *__restrict__ sch,
                               const double *__restrict__ ss, const double *__restrict__ slk,
                               const double *__restrict__ xs, const double *__restrict__ chat,
                               const double *__restrict__ mt, double *__restrict__ Gs, double *__restrict__ Gk)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nnode_s * k) return;
    const int s = j / k;
    double accs = 0.0, acc1 = 0.0;
    if (tptr[s + 1] > tptr[s]) {
        const double *xb = sch + (size_t)j * d;
        const double sb = ss[j], lb = slk[j];
        for (int e = tptr[s]; e < tptr[s + 1]; ++e) {
            const int t = tcol[e];
            for (int al = 0; al < k; ++al) {
                const int i = t * k + al;
                double r2 = 0.0;
                for (int c = 0; c < d; ++c) {
                    const double dd = tch[(size_t)i * d + c] - xb[c];
                    r2 = fma(dd, dd, r2);
                }
                const double lr2 = fast_log(mt, r2);
                const double g = fast_exp(mt, 0.5 * (tlk[i] + lb) - 0.5 * (d + ts[i] + sb) * lr2) * chat[i];
                acc1 += g;
                accs = fma(g, lr2, accs);
            }
        }
        accs *= 0.5 * xs[j];
        acc1 *= -0.5 * xs[j];
    }
    Gs[j] = accs;
    Gk[j] = acc1;
}

// touching pairs: per pair the 12 partial gradients (s at pv[0..2], qv[0..2];
// log kappa likewise), warp per pair, lanes over the rule points (the rules
// of Sec. 4 as in the assembly of B; 1D: the analogue of the vertex case)
struct GradSing {
    int d, ns, npairs, M, nrhs;
    int64_t ld;
    double sbar;
    const int *pinfo, *vdof;
    const double *vx, *gx, *gw, *s, *lk, *U, *Lam;
};

__device__ __forceinline__ void gs_point(const GradSing &P, int nl, const int *loc, double w, const double *f,
                                         double dlw, const double *bx, const double *by, double *gs, double *gk)
{
    double ul = 0.0;
    for (int r = 0; r < P.nrhs; ++r) {
        double u = 0.0, l = 0.0;
        for (int i = 0; i < nl; ++i) {
            const int j = P.vdof[loc[i]];
            if (j >= 0) {
                u += P.U[(size_t)r * P.ld + j] * f[i];
                l += P.Lam[(size_t)r * P.ld + j] * f[i];
            }
        }
        ul += u * l;
    }
    const double c = w * ul;
    for (int a = 0; a < 3; ++a) {
        gs[a] -= c * dlw * bx[a];
        gs[3 + a] -= c * dlw * by[a];
        gk[a] -= 0.5 * c * bx[a];
        gk[3 + a] -= 0.5 * c * by[a];
    }
}

__device__ __forceinline__ void gs_fields(const GradSing &P, const int *vid, const double *bary, double &s, double &lk)
{
    s = 0.0;
    lk = 0.0;
    for (int a = 0; a <= P.d; ++a) {
        s += bary[a] * P.s[vid[a]];
        lk += bary[a] * P.lk[vid[a]];
    }
}

__global__ void __launch_bounds__(256) k_grad_sing(GradSing P, double *__restrict__ pg)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= P.npairs) return;
    const int *pi = P.pinfo + (size_t)warp * 8;
    const int type = pi[0];
    const double wgt = (double)pi[1];
    const int d = P.d, ns = P.ns;
    const int pv[3] = {pi[2], pi[3], pi[4]}, qv[3] = {pi[5], pi[6], pi[7]};
    double Pv[6], Qv[6];
    for (int a = 0; a <= d; ++a)
        for (int j = 0; j < d; ++j) {
            Pv[a * d + j] = P.vx[(size_t)j * P.M + pv[a]];
            Qv[a * d + j] = P.vx[(size_t)j * P.M + qv[a]];
        }
    double gs[6] = {0, 0, 0, 0, 0, 0}, gk[6] = {0, 0, 0, 0, 0, 0};
    const double sbar = P.sbar;
    double bx[3] = {0, 0, 0}, by[3] = {0, 0, 0};
    if (d == 2) {
        const double JP[4] = {Pv[2] - Pv[0], Pv[4] - Pv[2], Pv[3] - Pv[1], Pv[5] - Pv[3]};
        const double JQ[4] = {Qv[2] - Qv[0], Qv[4] - Qv[2], Qv[3] - Qv[1], Qv[5] - Qv[3]};
        const double detP = fabs(JP[0] * JP[3] - JP[1] * JP[2]), detQ = fabs(JQ[0] * JQ[3] - JQ[1] * JQ[2]);
        const double c = 4.0 - 2.0 * sbar;
        const int per = ns * ns * ns * ns;
        if (type == 1 || type == 2) {
            const int nl = (type == 1) ? 5 : 4, nreg = (type == 1) ? 2 : 5;
            const int loc[5] = {pv[0], pv[1], pv[2], type == 1 ? qv[1] : qv[2], qv[2]};
            const double pre = detP * detQ / c;
            for (int idx = lane; idx < nreg * per; idx += 32) {
                const int reg = idx / per, r = idx - reg * per;
                const int iz = r % ns, i1 = (r / ns) % ns, i2 = (r / (ns * ns)) % ns, i3 = r / (ns * ns * ns);
                const double zeta = P.gx[iz], e1 = P.gx[i1], e2 = P.gx[i2], e3 = P.gx[i3];
                const double wq = P.gw[iz] * P.gw[i1] * P.gw[i2] * P.gw[i3];
                double a[2], b[2], jac;
                if (type == 1) {
                    if (reg == 0) { a[0] = 1.0; a[1] = e1; b[0] = e2; b[1] = e2 * e3; }
                    else { a[0] = e2; a[1] = e2 * e3; b[0] = 1.0; b[1] = e1; }
                    jac = e2;
                } else {
                    switch (reg) {
                    case 0: a[0] = 1.0; a[1] = e1 * e3; b[0] = 1.0 - e1 * e2; b[1] = e1 * (1.0 - e2); jac = e1 * e1; break;
                    case 1: a[0] = 1.0; a[1] = e1; b[0] = 1.0 - e1 * e2 * e3; b[1] = e1 * e2 * (1.0 - e3); jac = e1 * e1 * e2; break;
                    case 2: a[0] = 1.0 - e1 * e2; a[1] = e1 * (1.0 - e2); b[0] = 1.0; b[1] = e1 * e2 * e3; jac = e1 * e1 * e2; break;
                    case 3: a[0] = 1.0 - e1 * e2 * e3; a[1] = e1 * e2 * (1.0 - e3); b[0] = 1.0; b[1] = e1; jac = e1 * e1 * e2; break;
                    default: a[0] = 1.0 - e1 * e2 * e3; a[1] = e1 * (1.0 - e2 * e3); b[0] = 1.0; b[1] = e1 * e2; jac = e1 * e1 * e2; break;
                    }
                }
                const double lz = log(zeta), xi = exp(lz / c);
                const double xh[2] = {xi * a[0], xi * a[1]}, yh[2] = {xi * b[0], xi * b[1]};
                bx[0] = 1.0 - xh[0]; bx[1] = xh[0] - xh[1]; bx[2] = xh[1];
                by[0] = 1.0 - yh[0]; by[1] = yh[0] - yh[1]; by[2] = yh[1];
                double sx, sy, kx, ky;
                gs_fields(P, pv, bx, sx, kx);
                gs_fields(P, qv, by, sy, ky);
                const double S = sx + sy;
                const double dx = JP[0] * a[0] + JP[1] * a[1] - JQ[0] * b[0] - JQ[1] * b[1];
                const double dy = JP[2] * a[0] + JP[3] * a[1] - JQ[2] * b[0] - JQ[3] * b[1];
                const double lD2 = log(dx * dx + dy * dy);
                const double w = wq * pre * jac * exp((2.0 * sbar - S) / c * lz + 0.5 * (kx + ky) - 0.5 * (2.0 + S) * lD2);
                double f[5];
                if (type == 1) {
                    f[0] = b[0] - a[0]; f[1] = a[0] - a[1]; f[2] = a[1]; f[3] = -(b[0] - b[1]); f[4] = -b[1];
                } else {
                    f[0] = b[0] - a[0]; f[1] = (a[0] - a[1]) - (b[0] - b[1]); f[2] = a[1]; f[3] = -b[1]; f[4] = 0.0;
                }
                gs_point(P, nl, loc, w, f, -lz / c - 0.5 * lD2, bx, by, gs, gk);
            }
        } else {
            const int loc[3] = {pv[0], pv[1], pv[2]};
            const double c2 = 2.0 - 2.0 * sbar;
            const double pre = 2.0 * detP * detP / (c * c2);   // the mirror regions double the sum
            for (int idx = lane; idx < 3 * per; idx += 32) {
                const int reg = idx / per, r = idx - reg * per;
                const int iz = r % ns, i1 = (r / ns) % ns, it = (r / (ns * ns)) % ns, i3 = r / (ns * ns * ns);
                const double zeta = P.gx[iz], e1 = P.gx[i1], tt = P.gx[it], e3 = P.gx[i3];
                const double wq = P.gw[iz] * P.gw[i1] * P.gw[it] * P.gw[i3];
                const double lz = log(zeta), lt = log(tt), xi = exp(lz / c), e2 = exp(lt / c2);
                double a[2], b[2], dr[2];
                if (reg == 0) {
                    a[0] = 1.0; a[1] = 1.0 - e1 + e1 * e2; b[0] = 1.0 - e1 * e2 * e3; b[1] = 1.0 - e1;
                    dr[0] = e3; dr[1] = 1.0;
                } else if (reg == 1) {
                    a[0] = 1.0; a[1] = e1 * (1.0 - e2 + e2 * e3); b[0] = 1.0 - e1 * e2; b[1] = e1 * (1.0 - e2);
                    dr[0] = 1.0; dr[1] = e3;
                } else {
                    a[0] = 1.0 - e1 * e2 * e3; a[1] = e1 * (1.0 - e2 * e3); b[0] = 1.0; b[1] = e1 * (1.0 - e2);
                    dr[0] = -e3; dr[1] = 1.0 - e3;
                }
                const double xh[2] = {xi * a[0], xi * a[1]}, yh[2] = {xi * b[0], xi * b[1]};
                bx[0] = 1.0 - xh[0]; bx[1] = xh[0] - xh[1]; bx[2] = xh[1];
                by[0] = 1.0 - yh[0]; by[1] = yh[0] - yh[1]; by[2] = yh[1];
                double sx, sy, kx, ky;
                gs_fields(P, pv, bx, sx, kx);
                gs_fields(P, pv, by, sy, ky);
                const double S = sx + sy;
                const double dx = JP[0] * dr[0] + JP[1] * dr[1], dy = JP[2] * dr[0] + JP[3] * dr[1];
                const double lD2 = log(dx * dx + dy * dy), le1 = log(e1);
                const double w = wq * pre *
                                 exp((2.0 * sbar - S) * (lz / c + lt / c2) + (2.0 - S) * le1 + 0.5 * (kx + ky) -
                                     0.5 * (2.0 + S) * lD2);
                const double f[3] = {-dr[0], dr[0] - dr[1], dr[1]};
                gs_point(P, 3, loc, w, f, -(lz / c + lt / c2) - le1 - 0.5 * lD2, bx, by, gs, gk);
            }
        }
    } else {
        const double hP = fabs(Pv[1] - Pv[0]), hQ = fabs(Qv[1] - Qv[0]);
        if (type == 3) {
            const int loc[2] = {pv[0], pv[1]};
            const double c = 2.0 - 2.0 * sbar, pre = 2.0 * hP * hP / c;
            for (int idx = lane; idx < ns * ns; idx += 32) {
                const int iz = idx % ns, it = idx / ns;
                const double zeta = P.gx[iz], tt = P.gx[it], lz = log(zeta), z = exp(lz / c);
                const double yh = (1.0 - z) * tt, xh = yh + z;
                bx[0] = 1.0 - xh; bx[1] = xh;
                by[0] = 1.0 - yh; by[1] = yh;
                double sx, sy, kx, ky;
                gs_fields(P, pv, bx, sx, kx);
                gs_fields(P, pv, by, sy, ky);
                const double S = sx + sy, lh = log(hP);
                const double w = P.gw[iz] * P.gw[it] * pre * (1.0 - z) *
                                 exp((2.0 * sbar - S) / c * lz + 0.5 * (kx + ky) - (1.0 + S) * lh);
                const double f[2] = {-1.0, 1.0};
                gs_point(P, 2, loc, w, f, -lz / c - lh, bx, by, gs, gk);
            }
        } else {
            const int loc[3] = {pv[0], pv[1], qv[1]};
            const double c = 3.0 - 2.0 * sbar, pre = hP * hQ / c;
            const double JP = Pv[1] - Pv[0], JQ = Qv[1] - Qv[0];
            for (int idx = lane; idx < 2 * ns * ns; idx += 32) {
                const int reg = idx / (ns * ns), r = idx % (ns * ns);
                const int iz = r % ns, ie = r / ns;
                const double zeta = P.gx[iz], eta = P.gx[ie], lz = log(zeta), xi = exp(lz / c);
                const double av = reg == 0 ? 1.0 : eta, bv = reg == 0 ? eta : 1.0;
                const double xh = xi * av, yh = xi * bv;
                bx[0] = 1.0 - xh; bx[1] = xh;
                by[0] = 1.0 - yh; by[1] = yh;
                double sx, sy, kx, ky;
                gs_fields(P, pv, bx, sx, kx);
                gs_fields(P, qv, by, sy, ky);
                const double S = sx + sy, lD = log(fabs(JP * av - JQ * bv));
                const double w = P.gw[iz] * P.gw[ie] * pre * exp((2.0 * sbar - S) / c * lz + 0.5 * (kx + ky) - (1.0 + S) * lD);
                const double f[3] = {bv - av, av, -bv};
                gs_point(P, 3, loc, w, f, -lz / c - lD, bx, by, gs, gk);
            }
        }
    }
    for (int i = 0; i < 6; ++i) {
        gs[i] = warp_sum(gs[i]);
        gk[i] = warp_sum(gk[i]);
    }
    if (lane == 0)
        for (int i = 0; i < 6; ++i) {
            pg[(size_t)warp * 12 + i] = wgt * gs[i];
            pg[(size_t)warp * 12 + 6 + i] = wgt * gk[i];
        }
}

// per vertex: the point sensitivities (density), the K-near leaf-point
// sensitivities, the node sensitivities (K, target, source nodes) and the
// touching pairs' slots, each times the barycentric coordinate of the vertex
__global__ void k_gh_gather(int M, const int *__restrict__ qptr, const int *__restrict__ qidx,
                            const double *__restrict__ qbary, const double *__restrict__ hPs,
                            const double *__restrict__ hPk, const int *__restrict__ lptr,
                            const int *__restrict__ lidx, const int *__restrict__ lp_pts,
                            const double *__restrict__ hKs, const double *__restrict__ hKk,
                            const int *__restrict__ nptr, const int *__restrict__ nidx,
                            const double *__restrict__ nbary, const double *__restrict__ Gs,
                            const double *__restrict__ Gk, const int *__restrict__ pptr,
                            const int *__restrict__ pidx, const double *__restrict__ pg, double *__restrict__ g_s,
                            double *__restrict__ g_lk)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= M) return;
    double a = 0.0, b = 0.0;
    for (int e = qptr[v]; e < qptr[v + 1]; ++e) {
        const int code = qidx[e], q = code / QB;
        const double w = qbary[(size_t)code];   // qbary[q * QB + slot]
        a = fma(w, hPs[q], a);
        b = fma(w, hPk[q], b);
    }
    for (int e = lptr[v]; e < lptr[v + 1]; ++e) {
        const int code = lidx[e], t = code / QB, slot = code - t * QB;
        const double w = qbary[(size_t)lp_pts[t] * QB + slot];
        a = fma(w, hKs[t], a);
        b = fma(w, hKk[t], b);
    }
    for (int e = nptr[v]; e < nptr[v + 1]; ++e) {
        const int code = nidx[e], n = code / QB;
        const double w = nbary[code];
        a = fma(w, Gs[n], a);
        b = fma(w, Gk[n], b);
    }
    for (int e = pptr[v]; e < pptr[v + 1]; ++e) {
        const int code = pidx[e], p = code / 6, slot = code - p * 6;
        a += pg[(size_t)p * 12 + slot];
        b += pg[(size_t)p * 12 + 6 + slot];
    }
    g_s[v] = a;
    g_lk[v] = b;
}

}  // namespace

// node entries of the gradient: the K tree's nodes (when it has admissible
// blocks), then the density target and source trees' nodes (when the density
// has admissible blocks)
static int64_t node_entries(const MeshData &m, int64_t *oT, int64_t *oS)
{
    const int64_t nK = m.nfar > 0 ? (int64_t)m.kt.nnode * m.k : 0;
    const int64_t nT = m.nrfar > 0 ? (int64_t)m.tt.nnode * m.k : 0;
    const int64_t nS = m.nrfar > 0 ? (int64_t)m.st.nnode * m.k : 0;
    *oT = nK;
    *oS = nK + nT;
    return nK + nT + nS;
}

// vertex -> (point, slot), (pair, slot), (leaf-point entry, slot) and
// (node entry, slot) lists, built once per mesh
static void ensure_grad_lists(MeshData &m)
{
    if (m.grad_lists) return;
    const int nv = m.d + 1;
    auto build = [&](int n_items, auto vert_of, std::vector<int> &ptr, std::vector<int> &idx) {
        ptr.assign(m.M + 1, 0);
        for (int it = 0; it < n_items; ++it)
            for (int a = 0; a < nv; ++a) ptr[vert_of(it, a) + 1]++;
        for (int v = 0; v < m.M; ++v) ptr[v + 1] += ptr[v];
        idx.assign(ptr[m.M], 0);
        std::vector<int> f(ptr.begin(), ptr.end() - 1);
        for (int it = 0; it < n_items; ++it)
            for (int a = 0; a < nv; ++a) idx[f[vert_of(it, a)]++] = it * QB + a;
    };
    std::vector<int> ptr, idx;
    build(m.nQ, [&](int q, int a) { return m.T[(size_t)m.qcell_host[q] * nv + a]; }, ptr, idx);
    m.gq_ptr.upload(ptr);
    m.gq_idx.upload(idx);
    // pairs: two vertex triples per pair, slots 0..2 and 3..5
    {
        std::vector<int> pc(m.M + 1, 0);
        for (int p = 0; p < m.npairs; ++p)
            for (int a = 0; a < nv; ++a) {
                pc[m.pair_info_h[(size_t)p * 8 + 2 + a] + 1]++;
                pc[m.pair_info_h[(size_t)p * 8 + 5 + a] + 1]++;
            }
        for (int v = 0; v < m.M; ++v) pc[v + 1] += pc[v];
        std::vector<int> pidx(pc[m.M]), pf(pc.begin(), pc.end() - 1);
        for (int p = 0; p < m.npairs; ++p)
            for (int a = 0; a < nv; ++a) {
                pidx[pf[m.pair_info_h[(size_t)p * 8 + 2 + a]]++] = p * 6 + a;
                pidx[pf[m.pair_info_h[(size_t)p * 8 + 5 + a]]++] = p * 6 + 3 + a;
            }
        m.gp_ptr.upload(pc);
        m.gp_idx.upload(pidx);
    }
    build((int)m.lp_pts_h.size(), [&](int t, int a) { return m.T[(size_t)m.qcell_host[m.lp_pts_h[t]] * nv + a]; },
          ptr, idx);
    m.gl_ptr.upload(ptr);
    m.gl_idx.upload(idx);
    // node entries with their located cells
    int64_t oT, oS;
    const int64_t nn = node_entries(m, &oT, &oS);
    VFD_REQUIRE(nn * QB < (int64_t)1 << 31, VFD_EUNSUPPORTED, "vfd_grad: too many Chebyshev nodes");
    std::vector<int> ncell(nn);
    std::vector<double> nb((size_t)nn * QB, 0.0);
    auto put = [&](const NodeLoc &loc, int64_t off, int64_t n) {
        VFD_REQUIRE(n == 0 || (loc.done && (int64_t)loc.cell_h.size() == n), VFD_ECUDA, "nodes not located");
        for (int64_t i = 0; i < n; ++i) {
            ncell[off + i] = loc.cell_h[i];
            for (int a = 0; a < QB; ++a) nb[(size_t)(off + i) * QB + a] = loc.bary_h[(size_t)i * QB + a];
        }
    };
    put(m.kt_loc, 0, oT);
    put(m.tt_loc, oT, oS - oT);
    put(m.st_loc, oS, nn - oS);
    build((int)nn, [&](int n, int a) { return m.T[(size_t)ncell[n] * nv + a]; }, ptr, idx);
    m.gn_ptr.upload(ptr);
    m.gn_idx.upload(idx);
    if (nn) m.gn_bary.upload(nb);
    else m.gn_bary.alloc(1);
    m.grad_lists = true;
}

void grad_adjoint(MeshData &m, OpData &op, const double *U, const double *Lam, int nrhs, int64_t ld, double *g_s,
                  double *g_lk, cudaStream_t st)
{
    VFD_REQUIRE(m.d <= 2, VFD_EUNSUPPORTED, "vfd_grad is built for d = 1, 2");
    VFD_REQUIRE((m.nfar == 0 && m.nrfar == 0) || m.nodes_located, VFD_ECUDA, "vfd_grad: nodes not located");
    ensure_grad_lists(m);
    const size_t nq = (size_t)m.nQ, nlp = m.lp_pts_h.size();
    const int k = m.k;
    int64_t oT, oS;
    const int64_t nn = node_entries(m, &oT, &oS);
    if (op.gr_uq.n < nq * nrhs) {
        op.gr_uq.alloc(nq * nrhs);
        op.gr_lq.alloc(nq * nrhs);
    }
    if (op.gr_hs.n < nq) {
        op.gr_hs.alloc(nq);
        op.gr_h1.alloc(nq);
        op.gr_cq.alloc(nq);
    }
    if (op.gr_hKs.n < std::max<size_t>(nlp, 1)) {
        op.gr_hKs.alloc(std::max<size_t>(nlp, 1));
        op.gr_hKk.alloc(std::max<size_t>(nlp, 1));
    }
    if (op.gr_Gs.n < (size_t)std::max<int64_t>(nn, 1)) {
        op.gr_Gs.alloc(std::max<int64_t>(nn, 1));
        op.gr_Gk.alloc(std::max<int64_t>(nn, 1));
    }
    if (op.gr_pg.n < (size_t)m.npairs * 12 + 1) op.gr_pg.alloc((size_t)m.npairs * 12 + 1);
    // U, Lam at the points; c_q
    k_grad_vals<<<cdiv(m.nQ, 256), 256, 0, st>>>(m.nQ, m.d, nrhs, ld, m.qcell.p, m.qbary.p, m.cells.p, m.vdof.p, U,
                                                 Lam, op.gr_uq.p, op.gr_lq.p);
    k_gh_cq<<<cdiv(m.nQ, 256), 256, 0, st>>>(m.nQ, m.nQint, nrhs, m.qw.p, op.gr_uq.p, op.gr_lq.p, op.gr_cq.p);
    VFD_CUDA(cudaGetLastError());
    VFD_CUDA(cudaMemsetAsync(op.gr_Gs.p, 0, sizeof(double) * std::max<int64_t>(nn, 1), st));
    VFD_CUDA(cudaMemsetAsync(op.gr_Gk.p, 0, sizeof(double) * std::max<int64_t>(nn, 1), st));
    // K: near blocks and admissible blocks, GNR columns per pass
    const int fl = m.kt.first_leaf();
    const size_t hsz = (size_t)m.kt.nnode * k;
    if (m.nfar > 0 && op.gr_xU.n < hsz * GNR) {
        op.gr_xU.alloc(hsz * GNR);
        op.gr_xL.alloc(hsz * GNR);
    }
    if (m.nnear == 0) {
        VFD_CUDA(cudaMemsetAsync(op.gr_hKs.p, 0, sizeof(double) * std::max<size_t>(nlp, 1), st));
        VFD_CUDA(cudaMemsetAsync(op.gr_hKk.p, 0, sizeof(double) * std::max<size_t>(nlp, 1), st));
    }
    for (int r0 = 0; r0 < nrhs; r0 += GNR) {
        const int nr = std::min(GNR, nrhs - r0);
        if (m.nnear > 0) {
            GKN P;
            P.nQ = m.nQ;
            P.fl = fl;
            P.nr = nr;
            P.accumulate = r0 > 0;
            P.ld = ld;
            P.U = U + (size_t)r0 * ld;
            P.Lam = Lam + (size_t)r0 * ld;
            P.kt_begin = m.kt_begin.p;
            P.kt_end = m.kt_end.p;
            P.lp_ptr = m.lp_ptr.p;
            P.lp_pts = m.lp_pts.p;
            P.near_ptr = m.near_ptr.p;
            P.near_col = m.near_col.p;
            P.qx = m.qx.p;
            P.qw = m.qw.p;
            P.qs = op.q_s.p;
            P.qlk = op.q_lk.p;
            P.qbary = m.qbary.p;
            P.qcell = m.qcell.p;
            P.cells = m.cells.p;
            P.vdof = m.vdof.p;
            P.mt = m.mtab.p;
            P.hs = op.gr_hKs.p;
            P.hk = op.gr_hKk.p;
            dim3 g(m.kt.nleaf, cdiv(m.max_leaf_pts, GT));
            if (m.d == 2) k_gh_knear<2><<<g, GT, 0, st>>>(P);
            else k_gh_knear<1><<<g, GT, 0, st>>>(P);
            VFD_CUDA(cudaGetLastError());
        }
        if (m.nfar > 0) {
            k_gh_moments<<<m.kt.nnode, 128, 0, st>>>(nr, k, m.N, m.far_lmin, m.kt.nnode, m.far_ptr.p, m.kt_begin.p,
                                                     m.kt_end.p, m.Ul64.p, U + (size_t)r0 * ld, Lam + (size_t)r0 * ld,
                                                     ld, op.gr_xU.p, op.gr_xL.p);
            k_gh_kfar<<<m.kt.nnode, 256, 0, st>>>(m.d, k, m.kt.nnode, nr, m.far_ptr.p, m.far_col.p, m.kt_cheb.p,
                                                  op.kc_s.p, op.kc_lk.p, op.gr_xU.p, op.gr_xL.p, m.mtab.p, op.gr_Gs.p,
                                                  op.gr_Gk.p);
            VFD_CUDA(cudaGetLastError());
        }
    }
    // density: near sources on both sides, then the admissible blocks
    {
        GRho P;
        P.d = m.d;
        P.nv = m.d + 1;
        P.nQ = m.nQ;
        P.k = k;
        P.p = m.p;
        P.tfl = m.tt.first_leaf();
        P.sfl = m.st.first_leaf();
        P.tt_begin = m.tt_begin.p;
        P.tt_end = m.tt_end.p;
        P.tt_perm = m.tt_perm.p;
        P.st_begin = m.st_begin.p;
        P.st_end = m.st_end.p;
        P.st_perm = m.st_perm.p;
        P.rnear_ptr = m.rnear_ptr.p;
        P.rnear_col = m.rnear_col.p;
        P.rnearT_ptr = m.rnearT_ptr.p;
        P.rnearT_col = m.rnearT_col.p;
        P.qx = m.qx.p;
        P.qw = m.qw.p;
        P.qs = op.q_s.p;
        P.qlk = op.q_lk.p;
        P.cq = op.gr_cq.p;
        P.qcell = m.qcell.p;
        P.cells = m.cells.p;
        P.mt = m.mtab.p;
        P.hs = op.gr_hs.p;
        P.hk = op.gr_h1.p;
        VFD_CUDA(cudaMemsetAsync(op.gr_hs.p, 0, sizeof(double) * nq, st));
        VFD_CUDA(cudaMemsetAsync(op.gr_h1.p, 0, sizeof(double) * nq, st));
        k_gh_rho_near_t<<<m.tt.nleaf, RCH, 0, st>>>(P);
        k_gh_rho_near_s<<<m.st.nleaf, RCH, 0, st>>>(P);
        VFD_CUDA(cudaGetLastError());
    }
    if (m.nrfar > 0) {
        const size_t nt = (size_t)m.tt.nnode * k;
        if (op.gr_ct.n < nt) op.gr_ct.alloc(nt);
        VFD_CUDA(cudaMemsetAsync(op.gr_ct.p, 0, sizeof(double) * nt, st));
        k_gh_rho_moments<<<m.tt.nnode, 128, 0, st>>>(m.d, m.p, k, m.nQ, m.rfar_ptr.p, m.tt_begin.p, m.tt_end.p,
                                                     m.tt_perm.p, m.tt_cheb.p, m.qx.p, op.gr_cq.p, op.gr_ct.p);
        k_gh_rho_far_t<<<cdiv((long long)m.tt.nnode * k, 128), 128, 0, st>>>(
            m.d, k, m.tt.nnode, m.rfar_ptr.p, m.rfar_col.p, m.tt_cheb.p, op.tc_s.p, op.tc_lk.p, m.st_cheb.p,
            op.sc_s.p, op.sc_lk.p, m.st_xhat.p, op.gr_ct.p, m.mtab.p, op.gr_Gs.p + oT, op.gr_Gk.p + oT);
        k_gh_rho_far_s<<<cdiv((long long)m.st.nnode * k, 128), 128, 0, st>>>(
            m.d, k, m.st.nnode, m.rfarT_ptr.p, m.rfarT_col.p, m.tt_cheb.p, op.tc_s.p, op.tc_lk.p, m.st_cheb.p,
            op.sc_s.p, op.sc_lk.p, m.st_xhat.p, op.gr_ct.p, m.mtab.p, op.gr_Gs.p + oS, op.gr_Gk.p + oS);
        VFD_CUDA(cudaGetLastError());
    }
    if (m.npairs > 0) {
        GradSing P;
        P.d = m.d;
        P.ns = m.opts.n_sing;
        P.npairs = m.npairs;
        P.M = m.M;
        P.nrhs = nrhs;
        P.ld = ld;
        P.sbar = op.s_bar;
        P.pinfo = m.pair_info.p;
        P.vdof = m.vdof.p;
        P.vx = m.vx.p;
        P.gx = m.gl_x.p;
        P.gw = m.gl_w.p;
        P.s = op.fs.vals;
        P.lk = op.fk.vals;
        P.U = U;
        P.Lam = Lam;
        k_grad_sing<<<cdiv((long long)m.npairs * 32, 256), 256, 0, st>>>(P, op.gr_pg.p);
        VFD_CUDA(cudaGetLastError());
    }
    k_gh_gather<<<cdiv(m.M, 256), 256, 0, st>>>(m.M, m.gq_ptr.p, m.gq_idx.p, m.qbary.p, op.gr_hs.p, op.gr_h1.p,
                                                m.gl_ptr.p, m.gl_idx.p, m.lp_pts.p, op.gr_hKs.p, op.gr_hKk.p,
                                                m.gn_ptr.p, m.gn_idx.p, m.gn_bary.p, op.gr_Gs.p, op.gr_Gk.p,
                                                m.gp_ptr.p, m.gp_idx.p, op.gr_pg.p, g_s, g_lk);
    VFD_CUDA(cudaGetLastError());
}

}  // namespace vfd
