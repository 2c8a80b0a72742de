// Adjoint gradient of the discrete operator with respect to the nodal values
// of s and of log kappa (P1 fields):
//
//   g_s[k]  = -sum_r Lam_r^T (dA/ds_k) U_r,   g_lk[k] = -sum_r Lam_r^T (dA/dlogk_k) U_r.
//
// The paper has no gradients; A is the operator of Sec. 3 (B + K + M) with
// every quadrature rule held fixed, and every term carries the kernel
// gamma(x,y) = sqrt(kappa(x) kappa(y)) |x-y|^-(d+s(x)+s(y)), so that
//   d gamma / d s_k    = -ln|x-y| (psi_k(x) + psi_k(y)) gamma,
//   d gamma / d logk_k =  1/2     (psi_k(x) + psi_k(y)) gamma.
//
// Separated point pairs (K and M together): the bilinear form over ordered
// pairs (q, q') of element-rule points in non-touching cells, not both
// exterior, is sum G(q,q') dU dLam with G = w w' gamma and dU = U(q) - U(q')
// (Sec. 3, the split of the form into K and M is an identity), so
//   g_s[k]  =  2 sum_q psi_k(q) h_s(q),  h_s(q) = sum_q' G ln|q-q'| sum_r dU_r dLam_r,
//   g_lk[k] = -  sum_q psi_k(q) h_1(q),  h_1(q) = sum_q' G sum_r dU_r dLam_r.
// Touching pairs (B): the singular rules of Sec. 4 point by point, with
// d(log w)/dS read off the factors of the rule weight that depend on S.
//
// Operators with P1 fields have no low-rank part (every block is near and
// the density is a direct sum), so the gradient is that of the operator the
// solves use.  All sums are in a fixed order (per-point and per-pair partial
// results gathered per vertex through precomputed lists).
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

constexpr int GT = 128;     // target points per CTA and source points per tile
constexpr int GNR = 8;      // right-hand sides per pass of the separated-pair kernel

// h_s(q), h_1(q) for every element-rule point q (targets), over all source
// points in tiles staged in shared memory.  Points q < nQint lie in interior
// cells.  accumulate: add to h (later passes over the right-hand sides).
template <int D>
__global__ void __launch_bounds__(GT)
k_grad_sep(int nQ, int nQint, int nr, int accumulate, const double *__restrict__ qx, const double *__restrict__ qw,
           const double *__restrict__ qs, const double *__restrict__ qlk, const int *__restrict__ qcell,
           const int *__restrict__ cells, const double *__restrict__ Uq, const double *__restrict__ Lq,
           const double *__restrict__ mt, double *__restrict__ hs, double *__restrict__ h1)
{
    constexpr int NV = D + 1;
    __shared__ double sx[D][GT], sw[GT], ss[GT], sa[GT];
    __shared__ double su[GNR][GT], sl[GNR][GT];
    __shared__ int sv[NV][GT];
    const int q = blockIdx.x * GT + threadIdx.x;
    const bool live = q < nQ;
    const int qq = live ? q : 0;
    double x[D], u[GNR], l[GNR];
    for (int i = 0; i < D; ++i) x[i] = qx[(size_t)i * nQ + qq];
    const double w = qw[qq], s = qs[qq], a = 0.5 * qlk[qq];
    const bool ext = qq >= nQint;
    int v[NV];
    for (int i = 0; i < NV; ++i) v[i] = cells[(size_t)qcell[qq] * NV + i];
#pragma unroll
    for (int r = 0; r < GNR; ++r) {
        u[r] = r < nr ? Uq[(size_t)r * nQ + qq] : 0.0;
        l[r] = r < nr ? Lq[(size_t)r * nQ + qq] : 0.0;
    }
    double acc_s = 0.0, acc_1 = 0.0;
    for (int t0 = 0; t0 < nQ; t0 += GT) {
        const int j = t0 + threadIdx.x;
        if (j < nQ) {
            for (int i = 0; i < D; ++i) sx[i][threadIdx.x] = qx[(size_t)i * nQ + j];
            sw[threadIdx.x] = qw[j];
            ss[threadIdx.x] = qs[j];
            sa[threadIdx.x] = 0.5 * qlk[j];
            for (int i = 0; i < NV; ++i) sv[i][threadIdx.x] = cells[(size_t)qcell[j] * NV + i];
            for (int r = 0; r < nr; ++r) {
                su[r][threadIdx.x] = Uq[(size_t)r * nQ + j];
                sl[r][threadIdx.x] = Lq[(size_t)r * nQ + j];
            }
        }
        __syncthreads();
        const int nt = min(GT, nQ - t0);
        if (live)
            for (int jj = 0; jj < nt; ++jj) {
                if (ext && t0 + jj >= nQint) continue;   // exterior x exterior: no term
                bool touch = false;
                for (int i = 0; i < NV; ++i)
                    for (int k = 0; k < NV; ++k) touch |= (v[i] == sv[k][jj]);
                if (touch) continue;                      // touching cells belong to B
                double r2 = 0.0;
                for (int i = 0; i < D; ++i) {
                    const double dd = x[i] - sx[i][jj];
                    r2 = fma(dd, dd, r2);
                }
                const double lr2 = fast_log(mt, r2);
                const double G = w * sw[jj] * fast_exp(mt, a + sa[jj] - 0.5 * (D + s + ss[jj]) * lr2);
                double ul = 0.0;
#pragma unroll
                for (int r = 0; r < GNR; ++r)
                    if (r < nr) ul = fma(u[r] - su[r][jj], l[r] - sl[r][jj], ul);
                const double t = G * ul;
                acc_1 += t;
                acc_s = fma(t, 0.5 * lr2, acc_s);
            }
        __syncthreads();
    }
    if (live) {
        hs[q] = accumulate ? hs[q] + acc_s : acc_s;
        h1[q] = accumulate ? h1[q] + acc_1 : acc_1;
    }
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

// per vertex: g_s = 2 sum bary h_s + sum of its pair slots, g_lk = -sum bary h_1 + ...
__global__ void k_grad_gather(int M, const int *__restrict__ qptr, const int *__restrict__ qidx,
                              const double *__restrict__ qbary, const double *__restrict__ hs,
                              const double *__restrict__ h1, const int *__restrict__ pptr,
                              const int *__restrict__ pidx, const double *__restrict__ pg, double *__restrict__ g_s,
                              double *__restrict__ g_lk)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= M) return;
    double a = 0.0, b = 0.0;
    for (int e = qptr[v]; e < qptr[v + 1]; ++e) {
        const int code = qidx[e], q = code / QB;
        const double w = qbary[(size_t)code];   // qbary[q * QB + slot]
        a += 2.0 * w * hs[q];
        b -= w * h1[q];
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

// vertex -> (point, slot) and vertex -> (pair, slot) lists, built once per mesh
static void ensure_grad_lists(MeshData &m)
{
    if (m.grad_lists) return;
    const int nv = m.d + 1;
    std::vector<int> qcnt(m.M + 1, 0), pcnt(m.M + 1, 0);
    for (int q = 0; q < m.nQ; ++q)
        for (int a = 0; a < nv; ++a) qcnt[m.T[(size_t)m.qcell_host[q] * nv + a] + 1]++;
    for (int p = 0; p < m.npairs; ++p)
        for (int a = 0; a < nv; ++a) {
            pcnt[m.pair_info_h[(size_t)p * 8 + 2 + a] + 1]++;
            pcnt[m.pair_info_h[(size_t)p * 8 + 5 + a] + 1]++;
        }
    for (int v = 0; v < m.M; ++v) {
        qcnt[v + 1] += qcnt[v];
        pcnt[v + 1] += pcnt[v];
    }
    std::vector<int> qidx(qcnt[m.M]), pidx(pcnt[m.M]), qf(qcnt.begin(), qcnt.end() - 1), pf(pcnt.begin(), pcnt.end() - 1);
    for (int q = 0; q < m.nQ; ++q)
        for (int a = 0; a < nv; ++a) {
            const int v = m.T[(size_t)m.qcell_host[q] * nv + a];
            qidx[qf[v]++] = q * QB + a;
        }
    for (int p = 0; p < m.npairs; ++p)
        for (int a = 0; a < nv; ++a) {
            const int v1 = m.pair_info_h[(size_t)p * 8 + 2 + a], v2 = m.pair_info_h[(size_t)p * 8 + 5 + a];
            pidx[pf[v1]++] = p * 6 + a;
            pidx[pf[v2]++] = p * 6 + 3 + a;
        }
    m.gq_ptr.upload(qcnt);
    m.gq_idx.upload(qidx);
    m.gp_ptr.upload(pcnt);
    m.gp_idx.upload(pidx);
    m.grad_lists = true;
}

void grad_exact(MeshData &m, OpData &op, const double *U, const double *Lam, int nrhs, int64_t ld, double *g_s,
                double *g_lk, cudaStream_t st)
{
    ensure_grad_lists(m);
    const size_t nq = (size_t)m.nQ;
    if (op.gr_uq.n < nq * nrhs) {
        op.gr_uq.alloc(nq * nrhs);
        op.gr_lq.alloc(nq * nrhs);
    }
    if (op.gr_hs.n < nq) {
        op.gr_hs.alloc(nq);
        op.gr_h1.alloc(nq);
    }
    if (op.gr_pg.n < (size_t)m.npairs * 12) op.gr_pg.alloc((size_t)m.npairs * 12 + 1);
    k_grad_vals<<<cdiv(m.nQ, 256), 256, 0, st>>>(m.nQ, m.d, nrhs, ld, m.qcell.p, m.qbary.p, m.cells.p, m.vdof.p, U,
                                                 Lam, op.gr_uq.p, op.gr_lq.p);
    VFD_CUDA(cudaGetLastError());
    for (int r0 = 0; r0 < nrhs; r0 += GNR) {
        const int nr = std::min(GNR, nrhs - r0);
        const double *uq = op.gr_uq.p + (size_t)r0 * nq, *lq = op.gr_lq.p + (size_t)r0 * nq;
        if (m.d == 2)
            k_grad_sep<2><<<cdiv(m.nQ, GT), GT, 0, st>>>(m.nQ, m.nQint, nr, r0 > 0, m.qx.p, m.qw.p, op.q_s.p,
                                                        op.q_lk.p, m.qcell.p, m.cells.p, uq, lq, m.mtab.p,
                                                        op.gr_hs.p, op.gr_h1.p);
        else
            k_grad_sep<1><<<cdiv(m.nQ, GT), GT, 0, st>>>(m.nQ, m.nQint, nr, r0 > 0, m.qx.p, m.qw.p, op.q_s.p,
                                                        op.q_lk.p, m.qcell.p, m.cells.p, uq, lq, m.mtab.p,
                                                        op.gr_hs.p, op.gr_h1.p);
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
    k_grad_gather<<<cdiv(m.M, 256), 256, 0, st>>>(m.M, m.gq_ptr.p, m.gq_idx.p, m.qbary.p, op.gr_hs.p, op.gr_h1.p,
                                                  m.gp_ptr.p, m.gp_idx.p, op.gr_pg.p, g_s, g_lk);
    VFD_CUDA(cudaGetLastError());
}

}  // namespace vfd
