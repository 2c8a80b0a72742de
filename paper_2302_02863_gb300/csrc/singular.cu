// Singular near field B in 2D (Sec. 4): the tensor Gauss rules of the vertex
// (eq. e:int-v-2), edge (eq. e:int-e) and identical (eq. e:int-i-2) cases,
// one warp per touching pair.
//
// Each region's map sends (zeta, eta1, eta2, eta3) to (xhat, yhat), and xhat
// (yhat) depends on a subset of the four Gauss indices only (e.g. the vertex
// region 1 has xhat = xi (1, eta1)).  The warp first evaluates s and log kappa
// once per distinct mapped point into shared memory, then sweeps the 4D
// points with table lookups, so a 4D point costs one log and one exp.  The
// per-index powers and logarithms of zeta, t and eta1 are tabulated per CTA.
#include "device_common.cuh"

namespace vfd {

void launch_singular_B_generic(const MeshData &m, OpData &op, DBuf<double> &Lbuf, cudaStream_t st);

namespace {

// index masks (bit 0: zeta, bit 1: eta1, bit 2: eta2 (t in the identical
// case), bit 3: eta3) of the point each region's xhat / yhat depends on
__constant__ unsigned char c_xmask[3][5] = {{0x3, 0xD, 0, 0, 0}, {0xB, 0x3, 0x7, 0xF, 0xF}, {0x7, 0xF, 0xF, 0, 0}};
__constant__ unsigned char c_ymask[3][5] = {{0xD, 0x3, 0, 0, 0}, {0x7, 0xF, 0xF, 0x3, 0x7}, {0xF, 0x7, 0x7, 0, 0}};

struct Tab {
    double lz[NSMAX], xi[NSMAX], lt[NSMAX], e2[NSMAX], le1[NSMAX];
};

__device__ __forceinline__ int ipow(int b, int e)
{
    int r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

// table index of (iz,i1,i2,i3) for a mask; the table spans ns^popc(mask)
__device__ __forceinline__ int tindex(unsigned mask, int ns, const int *ind)
{
    int idx = 0, mul = 1;
    for (int j = 0; j < 4; ++j)
        if (mask & (1u << j)) {
            idx += ind[j] * mul;
            mul *= ns;
        }
    return idx;
}

__device__ __forceinline__ void tdecode(unsigned mask, int ns, int t, int *ind)
{
    for (int j = 0; j < 4; ++j) {
        ind[j] = 0;
        if (mask & (1u << j)) {
            ind[j] = t % ns;
            t /= ns;
        }
    }
}

// region maps divided by xi: xhat = xi a, yhat = xi b (vertex: T_V^(1,2)
// eq. e:map-v; edge: T_E^(1..5) Sec. 4.2), with the eta-Jacobian factor
__device__ __forceinline__ void map_ve(int type, int reg, double e1, double e2, double e3, double *a, double *b,
                                       double &jac)
{
    if (type == 1) {
        if (reg == 0) { a[0] = 1.0; a[1] = e1; b[0] = e2; b[1] = e2 * e3; }
        else { a[0] = e2; a[1] = e2 * e3; b[0] = 1.0; b[1] = e1; }
        jac = e2;
        return;
    }
    switch (reg) {
    case 0: a[0] = 1.0; a[1] = e1 * e3; b[0] = 1.0 - e1 * e2; b[1] = e1 * (1.0 - e2); jac = e1 * e1; break;
    case 1: a[0] = 1.0; a[1] = e1; b[0] = 1.0 - e1 * e2 * e3; b[1] = e1 * e2 * (1.0 - e3); jac = e1 * e1 * e2; break;
    case 2: a[0] = 1.0 - e1 * e2; a[1] = e1 * (1.0 - e2); b[0] = 1.0; b[1] = e1 * e2 * e3; jac = e1 * e1 * e2; break;
    case 3: a[0] = 1.0 - e1 * e2 * e3; a[1] = e1 * e2 * (1.0 - e3); b[0] = 1.0; b[1] = e1; jac = e1 * e1 * e2; break;
    default: a[0] = 1.0 - e1 * e2 * e3; a[1] = e1 * (1.0 - e2 * e3); b[0] = 1.0; b[1] = e1 * e2; jac = e1 * e1 * e2; break;
    }
}

// identical maps T_I^(1..3) (Sec. 4.3; region 2 with the factor eta1 on
// xhat_2, region 3 scaled difference (-eta3, 1-eta3)); dr = (xhat - yhat)/(xi eta1 eta2)
__device__ __forceinline__ void map_id(int reg, double e1, double e2, double e3, double *a, double *b, double *dr)
{
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
}

__device__ __forceinline__ void phys(const double *V, const double *xh, double *x, double *bary)
{
    // chi(xh) = V0 + (V1 - V0) xh1 + (V2 - V1) xh2 ; barycentric (1-xh1, xh1-xh2, xh2)
    x[0] = V[0] + (V[2] - V[0]) * xh[0] + (V[4] - V[2]) * xh[1];
    x[1] = V[1] + (V[3] - V[1]) * xh[0] + (V[5] - V[3]) * xh[1];
    bary[0] = 1.0 - xh[0];
    bary[1] = xh[0] - xh[1];
    bary[2] = xh[1];
}

struct Sing2Params {
    int ns, npairs, cap;   // cap: field-table entries per warp
    double sbar;
    const int *pinfo;
    const double *vx;
    int M;
    const double *gx, *gw;
    const double *mt;
    DField Fs, Fk;
};

__global__ void __launch_bounds__(256) k_singular2d(Sing2Params P, double *__restrict__ Lbuf)
{
    extern __shared__ __align__(16) double shs[];
    __shared__ Tab tab;
    const int ns = P.ns;
    const double sbar = P.sbar, c = 4.0 - 2.0 * sbar, c2 = 2.0 - 2.0 * sbar;
    if (threadIdx.x < ns) {
        double g = P.gx[threadIdx.x], lg = log(g);
        tab.lz[threadIdx.x] = lg;
        tab.xi[threadIdx.x] = exp(lg / c);
        tab.lt[threadIdx.x] = lg;
        tab.e2[threadIdx.x] = exp(lg / c2);
        tab.le1[threadIdx.x] = lg;
    }
    __syncthreads();
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pair = blockIdx.x * (blockDim.x >> 5) + wib;
    if (pair >= P.npairs) return;
    double *fs = shs + (size_t)wib * 2 * P.cap, *fk = fs + P.cap;
    const int *pi = P.pinfo + (size_t)pair * 8;
    const int type = pi[0];
    const double wgt = (double)pi[1];
    int pv[3] = {pi[2], pi[3], pi[4]}, qv[3] = {pi[5], pi[6], pi[7]};
    double Pv[6], Qv[6];
    for (int a = 0; a < 3; ++a)
        for (int j = 0; j < 2; ++j) {
            Pv[a * 2 + j] = P.vx[(size_t)j * P.M + pv[a]];
            Qv[a * 2 + j] = P.vx[(size_t)j * P.M + qv[a]];
        }
    const double JP[4] = {Pv[2] - Pv[0], Pv[4] - Pv[2], Pv[3] - Pv[1], Pv[5] - Pv[3]};
    const double JQ[4] = {Qv[2] - Qv[0], Qv[4] - Qv[2], Qv[3] - Qv[1], Qv[5] - Qv[3]};
    const double detP = fabs(JP[0] * JP[3] - JP[1] * JP[2]), detQ = fabs(JQ[0] * JQ[3] - JQ[1] * JQ[2]);
    const int ti = type - 1;   // 0 vertex, 1 edge, 2 identical
    const int nreg = type == 1 ? 2 : (type == 2 ? 5 : 3);
    const double *Vy = (type == 3) ? Pv : Qv;
    const int *vy = (type == 3) ? pv : qv;
    // ---- phase 1: fields at the distinct mapped points
    int xo[5], yo[5];
    {
        int off = 0;
        for (int reg = 0; reg < nreg; ++reg) {
            xo[reg] = off;
            off += ipow(ns, __popc(c_xmask[ti][reg]));
            yo[reg] = off;
            off += ipow(ns, __popc(c_ymask[ti][reg]));
        }
    }
    for (int reg = 0; reg < nreg; ++reg)
        for (int side = 0; side < 2; ++side) {
            const unsigned mask = side == 0 ? c_xmask[ti][reg] : c_ymask[ti][reg];
            const int size = ipow(ns, __popc(mask)), off = side == 0 ? xo[reg] : yo[reg];
            for (int t = lane; t < size; t += 32) {
                int ind[4];
                tdecode(mask, ns, t, ind);
                const double xi = tab.xi[ind[0]], e1 = P.gx[ind[1]], e3 = P.gx[ind[3]];
                double a[2], b[2], aux[2], jac;
                if (type == 3) map_id(reg, e1, tab.e2[ind[2]], e3, a, b, aux);
                else map_ve(type, reg, e1, P.gx[ind[2]], e3, a, b, jac);
                double h[2], x[2], bary[3], sv, kv;
                if (side == 0) {
                    h[0] = xi * a[0]; h[1] = xi * a[1];
                    phys(Pv, h, x, bary);
                    fields2(P.Fs, P.Fk, 2, x, pv, bary, sv, kv, P.mt);
                } else {
                    h[0] = xi * b[0]; h[1] = xi * b[1];
                    phys(Vy, h, x, bary);
                    fields2(P.Fs, P.Fk, 2, x, vy, bary, sv, kv, P.mt);
                }
                fs[off + t] = sv;
                fk[off + t] = kv;
            }
        }
    __syncwarp();
    // ---- phase 2: the 4D tensor rule
    double acc[15];
    for (int i = 0; i < 15; ++i) acc[i] = 0.0;
    const int per = ns * ns * ns * ns, tot = nreg * per;
    if (type != 3) {
        const double pre = detP * detQ / c;
        for (int idx = lane; idx < tot; idx += 32) {
            int reg = idx / per, r = idx - reg * per;
            int ind[4] = {r % ns, (r / ns) % ns, (r / (ns * ns)) % ns, r / (ns * ns * ns)};
            const double e1 = P.gx[ind[1]], e2 = P.gx[ind[2]], e3 = P.gx[ind[3]];
            double a[2], b[2], jac;
            map_ve(type, reg, e1, e2, e3, a, b, jac);
            const int ix = xo[reg] + tindex(c_xmask[ti][reg], ns, ind), iy = yo[reg] + tindex(c_ymask[ti][reg], ns, ind);
            const double S = fs[ix] + fs[iy];
            double dx = JP[0] * a[0] + JP[1] * a[1] - JQ[0] * b[0] - JQ[1] * b[1];
            double dy = JP[2] * a[0] + JP[3] * a[1] - JQ[2] * b[0] - JQ[3] * b[1];
            double D2 = dx * dx + dy * dy;
            double w = P.gw[ind[0]] * P.gw[ind[1]] * P.gw[ind[2]] * P.gw[ind[3]] * pre * jac *
                       fast_exp(P.mt, (2.0 * sbar - S) / c * tab.lz[ind[0]] + 0.5 * (fk[ix] + fk[iy]) -
                                          0.5 * (2.0 + S) * fast_log(P.mt, D2));
            // basis differences (psi(x) - psi(y))/xi, reference basis 1-x1, x1-x2, x2
            double f[5];
            if (type == 1) {
                f[0] = b[0] - a[0]; f[1] = a[0] - a[1]; f[2] = a[1]; f[3] = -(b[0] - b[1]); f[4] = -b[1];
            } else {
                f[0] = b[0] - a[0]; f[1] = (a[0] - a[1]) - (b[0] - b[1]); f[2] = a[1]; f[3] = -b[1]; f[4] = 0.0;
            }
            int t = 0;
            for (int i = 0; i < 5; ++i)
                for (int j = i; j < 5; ++j) acc[t++] += w * f[i] * f[j];
        }
    } else {
        const double pre = 2.0 * detP * detP / (c * c2);   // the mirror regions T_I^(4..6) double the sum
        for (int idx = lane; idx < tot; idx += 32) {
            int reg = idx / per, r = idx - reg * per;
            int ind[4] = {r % ns, (r / ns) % ns, (r / (ns * ns)) % ns, r / (ns * ns * ns)};
            const double e1 = P.gx[ind[1]], e2 = tab.e2[ind[2]], e3 = P.gx[ind[3]];
            double a[2], b[2], dr[2];
            map_id(reg, e1, e2, e3, a, b, dr);
            const int ix = xo[reg] + tindex(c_xmask[2][reg], ns, ind), iy = yo[reg] + tindex(c_ymask[2][reg], ns, ind);
            const double S = fs[ix] + fs[iy];
            double dx = JP[0] * dr[0] + JP[1] * dr[1], dy = JP[2] * dr[0] + JP[3] * dr[1];
            double D2 = dx * dx + dy * dy;
            double w = P.gw[ind[0]] * P.gw[ind[1]] * P.gw[ind[2]] * P.gw[ind[3]] * pre *
                       fast_exp(P.mt, (2.0 * sbar - S) * (tab.lz[ind[0]] / c + tab.lt[ind[2]] / c2) +
                                          (2.0 - S) * tab.le1[ind[1]] + 0.5 * (fk[ix] + fk[iy]) -
                                          0.5 * (2.0 + S) * fast_log(P.mt, D2));
            double f[3] = {-dr[0], dr[0] - dr[1], dr[1]};
            int t = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = i; j < 5; ++j) acc[t++] += (j < 3) ? w * f[i] * f[j] : 0.0;
        }
    }
    const int nl = type == 1 ? 5 : (type == 2 ? 4 : 3);
    for (int i = 0; i < 15; ++i) acc[i] = warp_sum(acc[i]);
    if (lane == 0) {
        double *L = Lbuf + (size_t)pair * 25;
        int t = 0;
        for (int i = 0; i < 5; ++i)
            for (int j = i; j < 5; ++j, ++t) {
                double v = (i < nl && j < nl) ? wgt * acc[t] : 0.0;
                L[i * 5 + j] = v;
                L[j * 5 + i] = v;
            }
    }
}

}  // namespace

void launch_singular_B(const MeshData &m, OpData &op, DBuf<double> &Lbuf, cudaStream_t st)
{
    const int ns = m.opts.n_sing;
    // largest field table: the edge case, 4 ns^4 + 4 ns^3 + 2 ns^2 points
    const int cap = 4 * ns * ns * ns * ns + 4 * ns * ns * ns + 2 * ns * ns;
    const size_t per_warp = (size_t)cap * 2 * sizeof(double);
    int wpb = 8;
    while (wpb > 1 && per_warp * wpb > 200 * 1024) wpb /= 2;
    if (m.d != 2 || per_warp * wpb > 200 * 1024) {
        launch_singular_B_generic(m, op, Lbuf, st);
        return;
    }
    Lbuf.alloc((size_t)m.npairs * 25);
    if (!m.npairs) return;
    Sing2Params P;
    P.ns = ns;
    P.npairs = m.npairs;
    P.cap = cap;
    P.sbar = op.s_bar;
    P.pinfo = m.pair_info.p;
    P.vx = m.vx.p;
    P.M = m.M;
    P.gx = m.gl_x.p;
    P.gw = m.gl_w.p;
    P.mt = m.mtab.p;
    P.Fs = op.fs;
    P.Fk = op.fk;
    size_t shm = per_warp * wpb;
    VFD_CUDA(cudaFuncSetAttribute(k_singular2d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_singular2d<<<cdiv(m.npairs, wpb), 32 * wpb, shm, st>>>(P, Lbuf.p);
    VFD_CUDA(cudaGetLastError());
}

}  // namespace vfd
