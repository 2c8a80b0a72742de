// Assembly kernels (Algorithm 1 of the paper, all on the device):
//   field values -> coupling blocks S (Sec. 5.3) -> dense inadmissible leaf
//   blocks (Sec. 5.2) -> density rho by the H^2 sweep (Sec. 6.2) + tail
//   (Sec. 7.1.1) -> singular near field B (Sec. 4) -> weighted mass M (Sec. 6.1).
#include "device_common.cuh"

namespace vfd {

// ---------------------------------------------------------------------------
// field values at the element-rule points and at the Chebyshev nodes
// ---------------------------------------------------------------------------
__global__ void k_fields_points(int d, int nQ, const double *__restrict__ qx, const int *__restrict__ qcell,
                                const double *__restrict__ qbary, const int *__restrict__ cells, DField Fs, DField Fk,
                                double *__restrict__ out_s, double *__restrict__ out_lk, double smin, double smax,
                                int *err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nQ) return;
    double x[3];
    for (int j = 0; j < d; ++j) x[j] = qx[(size_t)j * nQ + i];
    const int *vid = cells + (size_t)qcell[i] * (d + 1);
    double s, lk;
    fields2(Fs, Fk, d, x, vid, qbary + (size_t)i * QB, s, lk);
    out_s[i] = s;
    out_lk[i] = lk;
    if (!(s >= smin && s <= smax)) atomicOr(err, 1);
}

// lcell, lbary (nodal fields): the node's closest cell and the barycentric
// coordinates of its closest point there (nearest-point rule outside the mesh)
__global__ void k_fields_nodes(int d, int n, const double *__restrict__ pts, DField Fs, DField Fk,
                               const int *__restrict__ lcell, const double *__restrict__ lbary,
                               const int *__restrict__ cells, double *__restrict__ out_s, double *__restrict__ out_lk,
                               double smin, double smax, int *err)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[3];
    for (int j = 0; j < d; ++j) x[j] = pts[(size_t)i * d + j];
    double s, lk;
    const int *vid = lcell ? cells + (size_t)lcell[i] * (d + 1) : nullptr;
    fields2(Fs, Fk, d, x, vid, lcell ? lbary + (size_t)i * QB : nullptr, s, lk);
    out_s[i] = s;
    out_lk[i] = lk;
    if (!(s >= smin && s <= smax)) atomicOr(err, 2);
}

void launch_field_points(const MeshData &m, OpData &op, cudaStream_t st)
{
    const int d = m.d, k = m.k;
    bool chk = op.check_fields;
    double smin = chk ? 0.0 : -1e300, smax = chk ? op.s_bar : 1e300;
    op.q_s.alloc(m.nQ);
    op.q_lk.alloc(m.nQ);
    k_fields_points<<<cdiv(m.nQ, 256), 256, 0, st>>>(d, m.nQ, m.qx.p, m.qcell.p, m.qbary.p, m.cells.p, op.fs, op.fk,
                                                     op.q_s.p, op.q_lk.p, smin, smax, op.errflag.p);
    VFD_CUDA(cudaGetLastError());
    const bool nodal = op.fs.nodal || op.fk.nodal;
    auto nodes = [&](const DBuf<double> &pts, int n, const NodeLoc &loc, DBuf<double> &os, DBuf<double> &ol) {
        os.alloc(n);
        ol.alloc(n);
        VFD_REQUIRE(!nodal || loc.done, VFD_ECUDA, "Chebyshev nodes not located for a nodal field");
        if (n)
            k_fields_nodes<<<cdiv(n, 256), 256, 0, st>>>(d, n, pts.p, op.fs, op.fk, nodal ? loc.cell.p : nullptr,
                                                          nodal ? loc.bary.p : nullptr, m.cells.p, os.p, ol.p, smin,
                                                          smax, op.errflag.p);
        VFD_CUDA(cudaGetLastError());
    };
    if (m.nfar) nodes(m.kt_cheb, m.kt.nnode * k, m.kt_loc, op.kc_s, op.kc_lk);
    // the inner operator's nodes (k_in per box)
    if (m.nfar && m.k_in && op.precision != VFD_FP64)
        nodes(m.kt_cheb_in, m.kt.nnode * m.k_in, m.kt_in_loc, op.kc_s_in, op.kc_lk_in);
    if (m.nrfar) {
        nodes(m.tt_cheb, m.tt.nnode * k, m.tt_loc, op.tc_s, op.tc_lk);
        nodes(m.st_cheb, m.st.nnode * k, m.st_loc, op.sc_s, op.sc_lk);
    }
}

// ---------------------------------------------------------------------------
// singular near field B: one warp per touching pair, tensor Gauss rules of
// Sec. 4 (vertex: e:int-v-2, edge: e:int-e, identical: e:int-i-2) and the 1D
// analogue.  Writes the weighted local matrix (<= 5x5) to Lbuf[pair*25].
// ---------------------------------------------------------------------------
struct SingParams {
    int d, ns, npairs;
    double sbar;
    const int *pinfo;
    const double *vx;
    int M;
    const double *gx, *gw;
    DField Fs, Fk;
};

__device__ __forceinline__ void sing_point_fields(const SingParams &P, const double *xh, const double *V /*3x2*/,
                                                  const int *vid, double *x, double &s, double &lk)
{
    double bary[3];
    if (P.d == 2) {
        // chi(xh) = V0 + (V1 - V0) xh1 + (V2 - V1) xh2 ; barycentric (1-xh1, xh1-xh2, xh2)
        x[0] = V[0] + (V[2] - V[0]) * xh[0] + (V[4] - V[2]) * xh[1];
        x[1] = V[1] + (V[3] - V[1]) * xh[0] + (V[5] - V[3]) * xh[1];
        bary[0] = 1.0 - xh[0];
        bary[1] = xh[0] - xh[1];
        bary[2] = xh[1];
    } else {
        x[0] = V[0] + (V[1] - V[0]) * xh[0];
        bary[0] = 1.0 - xh[0];
        bary[1] = xh[0];
    }
    fields2(P.Fs, P.Fk, P.d, x, vid, bary, s, lk);
}

__global__ void __launch_bounds__(256) k_singular(SingParams P, double *__restrict__ Lbuf)
{
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= P.npairs) return;
    const int *pi = P.pinfo + (size_t)warp * 8;
    const int type = pi[0];
    const double wgt = (double)pi[1];
    const int d = P.d, ns = P.ns;
    int pv[3] = {pi[2], pi[3], pi[4]}, qv[3] = {pi[5], pi[6], pi[7]};
    double Pv[6], Qv[6];
    for (int a = 0; a <= d; ++a)
        for (int j = 0; j < d; ++j) {
            Pv[a * d + j] = P.vx[(size_t)j * P.M + pv[a]];
            Qv[a * d + j] = P.vx[(size_t)j * P.M + qv[a]];
        }
    // local matrix, upper triangle (nl <= 5)
    double acc[15];
    for (int i = 0; i < 15; ++i) acc[i] = 0.0;
    const double sbar = P.sbar;
    int nl;
    if (d == 2) {
        // Jacobians J = [V1-V0 | V2-V1] (the reference triangle (0,0),(1,0),(1,1))
        double JP[4] = {Pv[2] - Pv[0], Pv[4] - Pv[2], Pv[3] - Pv[1], Pv[5] - Pv[3]};  // row-major 2x2
        double JQ[4] = {Qv[2] - Qv[0], Qv[4] - Qv[2], Qv[3] - Qv[1], Qv[5] - Qv[3]};
        double detP = fabs(JP[0] * JP[3] - JP[1] * JP[2]), detQ = fabs(JQ[0] * JQ[3] - JQ[1] * JQ[2]);
        const double c = 4.0 - 2.0 * sbar;
        if (type == 1 || type == 2) {
            nl = (type == 1) ? 5 : 4;
            const int nreg = (type == 1) ? 2 : 5;
            const double pre = detP * detQ / c;
            const int per = ns * ns * ns * ns, tot = nreg * per;
            for (int idx = lane; idx < tot; idx += 32) {
                int reg = idx / per, r = idx - reg * per;
                int iz = r % ns, i1 = (r / ns) % ns, i2 = (r / (ns * ns)) % ns, i3 = r / (ns * ns * ns);
                double zeta = P.gx[iz], e1 = P.gx[i1], e2 = P.gx[i2], e3 = P.gx[i3];
                double wq = P.gw[iz] * P.gw[i1] * P.gw[i2] * P.gw[i3];
                double a[2], b[2], jac;
                if (type == 1) {
                    // vertex-sharing maps T_V^(1), T_V^(2) (eq. e:map-v), divided by xi
                    if (reg == 0) { a[0] = 1.0; a[1] = e1; b[0] = e2; b[1] = e2 * e3; }
                    else { a[0] = e2; a[1] = e2 * e3; b[0] = 1.0; b[1] = e1; }
                    jac = e2;
                } else {
                    // edge-sharing maps T_E^(1..5) (Sec. 4.2), divided by xi
                    switch (reg) {
                    case 0: a[0] = 1.0; a[1] = e1 * e3; b[0] = 1.0 - e1 * e2; b[1] = e1 * (1.0 - e2); jac = e1 * e1; break;
                    case 1: a[0] = 1.0; a[1] = e1; b[0] = 1.0 - e1 * e2 * e3; b[1] = e1 * e2 * (1.0 - e3); jac = e1 * e1 * e2; break;
                    case 2: a[0] = 1.0 - e1 * e2; a[1] = e1 * (1.0 - e2); b[0] = 1.0; b[1] = e1 * e2 * e3; jac = e1 * e1 * e2; break;
                    case 3: a[0] = 1.0 - e1 * e2 * e3; a[1] = e1 * e2 * (1.0 - e3); b[0] = 1.0; b[1] = e1; jac = e1 * e1 * e2; break;
                    default: a[0] = 1.0 - e1 * e2 * e3; a[1] = e1 * (1.0 - e2 * e3); b[0] = 1.0; b[1] = e1 * e2; jac = e1 * e1 * e2; break;
                    }
                }
                double lz = log(zeta), xi = exp(lz / c);
                double xh[2] = {xi * a[0], xi * a[1]}, yh[2] = {xi * b[0], xi * b[1]};
                double x[2], y[2], sx, sy, kx, ky;
                sing_point_fields(P, xh, Pv, pv, x, sx, kx);
                sing_point_fields(P, yh, Qv, qv, y, sy, ky);
                double S = sx + sy;
                // scaled distance |J_P a - J_Q b| (x - y = xi (J_P a - J_Q b))
                double dx = JP[0] * a[0] + JP[1] * a[1] - JQ[0] * b[0] - JQ[1] * b[1];
                double dy = JP[2] * a[0] + JP[3] * a[1] - JQ[2] * b[0] - JQ[3] * b[1];
                double D2 = dx * dx + dy * dy;
                double w = wq * pre * jac *
                           exp((2.0 * sbar - S) / c * lz + 0.5 * (kx + ky) - 0.5 * (2.0 + S) * log(D2));
                // basis differences (psi(x) - psi(y))/xi from the reference basis
                // phi0 = 1 - x1, phi1 = x1 - x2, phi2 = x2
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
            nl = 3;
            const double c2 = 2.0 - 2.0 * sbar;
            const double pre = 2.0 * detP * detP / (c * c2);  // the mirror regions T_I^(4..6) double the sum
            const int per = ns * ns * ns * ns, tot = 3 * per;
            for (int idx = lane; idx < tot; idx += 32) {
                int reg = idx / per, r = idx - reg * per;
                int iz = r % ns, i1 = (r / ns) % ns, it = (r / (ns * ns)) % ns, i3 = r / (ns * ns * ns);
                double zeta = P.gx[iz], e1 = P.gx[i1], tt = P.gx[it], e3 = P.gx[i3];
                double wq = P.gw[iz] * P.gw[i1] * P.gw[it] * P.gw[i3];
                double lz = log(zeta), lt = log(tt), xi = exp(lz / c), e2 = exp(lt / c2);
                double a[2], b[2], dr[2];
                // identical maps T_I^(1..3) (Sec. 4.3; region 2 with the factor eta1
                // on xhat_2, region 3 scaled difference (-eta3, 1-eta3))
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
                double xh[2] = {xi * a[0], xi * a[1]}, yh[2] = {xi * b[0], xi * b[1]};
                double x[2], y[2], sx, sy, kx, ky;
                sing_point_fields(P, xh, Pv, pv, x, sx, kx);
                sing_point_fields(P, yh, Pv, pv, y, sy, ky);
                double S = sx + sy;
                double dx = JP[0] * dr[0] + JP[1] * dr[1], dy = JP[2] * dr[0] + JP[3] * dr[1];
                double D2 = dx * dx + dy * dy;
                double w = wq * pre *
                           exp((2.0 * sbar - S) * (lz / c + lt / c2) + (2.0 - S) * log(e1) + 0.5 * (kx + ky) -
                               0.5 * (2.0 + S) * log(D2));
                double f[3] = {-dr[0], dr[0] - dr[1], dr[1]};
                int t = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = i; j < 5; ++j) {
                        acc[t++] += (j < 3) ? w * f[i] * f[j] : 0.0;
                    }
            }
        }
    } else {
        const double hP = fabs(Pv[1] - Pv[0]), hQ = fabs(Qv[1] - Qv[0]);
        if (type == 3) {
            nl = 2;
            const double c = 2.0 - 2.0 * sbar, pre = 2.0 * hP * hP / c;
            for (int idx = lane; idx < ns * ns; idx += 32) {
                int iz = idx % ns, it = idx / ns;
                double zeta = P.gx[iz], tt = P.gx[it], lz = log(zeta), z = exp(lz / c);
                double yh = (1.0 - z) * tt, xh = yh + z;
                double x, y, sx, sy, kx, ky;
                sing_point_fields(P, &xh, Pv, pv, &x, sx, kx);
                sing_point_fields(P, &yh, Pv, pv, &y, sy, ky);
                double S = sx + sy;
                double w = P.gw[iz] * P.gw[it] * pre * (1.0 - z) *
                           exp((2.0 * sbar - S) / c * lz + 0.5 * (kx + ky) - (1.0 + S) * log(hP));
                // psi differences / z: (-1, +1)
                acc[0] += w;
                acc[1] -= w;
                acc[5] += w;
            }
        } else {
            nl = 3;
            const double c = 3.0 - 2.0 * sbar, pre = hP * hQ / c;
            const double JP = Pv[1] - Pv[0], JQ = Qv[1] - Qv[0];
            for (int idx = lane; idx < 2 * ns * ns; idx += 32) {
                int reg = idx / (ns * ns), r = idx % (ns * ns);
                int iz = r % ns, ie = r / ns;
                double zeta = P.gx[iz], eta = P.gx[ie], lz = log(zeta), xi = exp(lz / c);
                double av = reg == 0 ? 1.0 : eta, bv = reg == 0 ? eta : 1.0;
                double xh = xi * av, yh = xi * bv;
                double x, y, sx, sy, kx, ky;
                sing_point_fields(P, &xh, Pv, pv, &x, sx, kx);
                sing_point_fields(P, &yh, Qv, qv, &y, sy, ky);
                double S = sx + sy;
                double D = fabs(JP * av - JQ * bv);
                double w = P.gw[iz] * P.gw[ie] * pre * exp((2.0 * sbar - S) / c * lz + 0.5 * (kx + ky) - (1.0 + S) * log(D));
                double f[3] = {bv - av, av, -bv};
                int t = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = i; j < 5; ++j) acc[t++] += (j < 3) ? w * f[i] * f[j] : 0.0;
            }
        }
    }
    for (int i = 0; i < 15; ++i) acc[i] = warp_sum(acc[i]);
    if (lane == 0) {
        double *L = Lbuf + (size_t)warp * 25;
        int t = 0;
        for (int i = 0; i < 5; ++i)
            for (int j = i; j < 5; ++j, ++t) {
                double v = (i < nl && j < nl) ? wgt * acc[t] : 0.0;
                L[i * 5 + j] = v;
                L[j * 5 + i] = v;
            }
    }
}

void launch_singular_B_generic(const MeshData &m, OpData &op, DBuf<double> &Lbuf, cudaStream_t st)
{
    Lbuf.alloc((size_t)m.npairs * 25);
    if (!m.npairs) return;
    if (m.d == 3) {   // tetrahedra: no singular rules (B = 0, reading R20)
        Lbuf.zero(st);
        return;
    }
    SingParams P;
    P.d = m.d;
    P.ns = m.opts.n_sing;
    P.npairs = m.npairs;
    P.sbar = op.s_bar;
    P.pinfo = m.pair_info.p;
    P.vx = m.vx.p;
    P.M = m.M;
    P.gx = m.gl_x.p;
    P.gw = m.gl_w.p;
    P.Fs = op.fs;
    P.Fk = op.fk;
    k_singular<<<cdiv((long long)m.npairs * 32, 256), 256, 0, st>>>(P, Lbuf.p);
    VFD_CUDA(cudaGetLastError());
}

// deterministic gather of the local matrices into the CSR values of B
__global__ void k_gather_B(int nnz, const int *__restrict__ ptr, const int *__restrict__ idx,
                           const double *__restrict__ L, double *__restrict__ val)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    double v = 0.0;
    for (int c = ptr[e]; c < ptr[e + 1]; ++c) v += L[idx[c]];
    val[e] = v;
}

void launch_gather_B(const MeshData &m, OpData &op, const DBuf<double> &Lbuf, cudaStream_t st)
{
    op.valB.alloc(m.nnz);
    k_gather_B<<<cdiv(m.nnz, 256), 256, 0, st>>>(m.nnz, m.cB_ptr.p, m.cB_idx.p, Lbuf.p, op.valB.p);
    VFD_CUDA(cudaGetLastError());
}

// weighted mass: M_ij = sum 2 w_q lam_i lam_j rho(q) (eq. e:m, e:tau-quad)
__global__ void k_gather_M(int nnz, const int *__restrict__ ptr, const int *__restrict__ q,
                           const double *__restrict__ coef, const double *__restrict__ rho,
                           const double *__restrict__ valB, double *__restrict__ valM, double *__restrict__ valBM)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnz) return;
    double v = 0.0;
    for (int c = ptr[e]; c < ptr[e + 1]; ++c) v += coef[c] * rho[q[c]];
    valM[e] = v;
    valBM[e] = valB[e] + v;
}

void launch_gather_M(const MeshData &m, OpData &op, cudaStream_t st)
{
    op.valM.alloc(m.nnz);
    op.valBM.alloc(m.nnz);
    k_gather_M<<<cdiv(m.nnz, 256), 256, 0, st>>>(m.nnz, m.cM_ptr.p, m.cM_q.p, m.cM_coef.p, op.rho.p, op.valB.p,
                                                 op.valM.p, op.valBM.p);
    VFD_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// density rho (Sec. 6.2): far part by an H^2 product with the fixed source
// moments (the source vector is the quadrature weights w, eq. eq:matvec),
// near part by the direct masked sum e:tgt-sum, plus the tail rho_B.
// ---------------------------------------------------------------------------
__global__ void k_rho_coupling(int d, int k, int nnode_t, const int *__restrict__ fptr, const int *__restrict__ fcol,
                               const double *__restrict__ tch, const double *__restrict__ ts,
                               const double *__restrict__ tlk, const double *__restrict__ sch,
                               const double *__restrict__ ss, const double *__restrict__ slk,
                               const double *__restrict__ xs, const double *__restrict__ mt, double *__restrict__ yt)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnode_t * k) return;
    int t = i / k;
    const double *xa = tch + (size_t)i * d;
    double sa = ts[i], la = tlk[i], acc = 0.0;
    for (int e = fptr[t]; e < fptr[t + 1]; ++e) {
        int s = fcol[e];
        for (int be = 0; be < k; ++be) {
            int j = s * k + be;
            double r2 = 0.0;
            for (int c = 0; c < d; ++c) {
                double dd = xa[c] - sch[(size_t)j * d + c];
                r2 += dd * dd;
            }
            acc += gamma_r2t(mt, d, r2, sa, ss[j], la, slk[j]) * xs[j];
        }
    }
    yt[i] = acc;
}

struct RhoParams {
    int d, k, p, Lt, nQ, nQint, nv;
    const int *tt_begin, *tt_end, *tt_perm, *st_begin, *st_end, *st_perm;
    const double *tt_cheb, *yt;
    const double *tt_lo, *tt_hi;     // target boxes
    double tref[PMAX], wref[PMAX];   // first-kind Chebyshev points of [-1, 1] and their barycentric weights
    const int *rnear_ptr, *rnear_col;
    const double *qx, *qw, *qs, *qlk;
    const int *qcell, *cells;
    int tail;
    double R;
    const double *g9x, *g9w;
    const double *mt;
    double *rho;
};

__global__ void __launch_bounds__(128) k_rho_points(RhoParams P)
{
    extern __shared__ double sh[];
    const int d = P.d;
    const int leaf = blockIdx.x;
    const int node = (1 << P.Lt) - 1 + leaf;
    const int b = P.tt_begin[node], e = P.tt_end[node];
    const int CH = 128;
    double *sx = sh;                  // CH * d
    double *ss = sx + CH * d;         // CH: b = s/2 + d/4
    double *sl = ss + CH;             // CH: a = log(kappa)/2 + log w
    int *sv = (int *)(sl + CH);       // CH * 4 vertex ids of the source cell
    for (int i0 = b; i0 < e; i0 += blockDim.x) {
        int i = i0 + threadIdx.x;
        bool act = i < e;
        int id = act ? P.tt_perm[i] : 0;
        double x[3] = {0, 0, 0};
        int cv[4] = {-1, -1, -1, -1};
        double s_ = 0, l_ = 0, a_ = 0, b_ = 0;
        if (act) {
            for (int c = 0; c < d; ++c) x[c] = P.qx[(size_t)c * P.nQ + id];
            s_ = P.qs[id];
            l_ = P.qlk[id];
            a_ = 0.5 * l_;
            b_ = fma(0.5, s_, 0.25 * d);
            int cell = P.qcell[id];
            for (int a = 0; a < P.nv; ++a) cv[a] = P.cells[(size_t)cell * P.nv + a];
        }
        double acc = 0.0;
        // near sources: masked direct sum
        for (int ne = P.rnear_ptr[leaf]; ne < P.rnear_ptr[leaf + 1]; ++ne) {
            int sn = P.rnear_col[ne];
            int sb = P.st_begin[sn], se = P.st_end[sn];
            for (int j0 = sb; j0 < se; j0 += CH) {
                int nj = min(CH, se - j0);
                __syncthreads();
                for (int t = threadIdx.x; t < nj; t += blockDim.x) {
                    int jd = P.st_perm[j0 + t];
                    for (int c = 0; c < d; ++c) sx[t * d + c] = P.qx[(size_t)c * P.nQ + jd];
                    // exponent terms of the source, its weight folded in: w gamma = exp(log w + ...)
                    ss[t] = fma(0.5, P.qs[jd], 0.25 * d);
                    sl[t] = fma(0.5, P.qlk[jd], fast_log(P.mt, P.qw[jd]));
                    int cell = P.qcell[jd];
                    for (int a = 0; a < 4; ++a) sv[t * 4 + a] = a < P.nv ? P.cells[(size_t)cell * P.nv + a] : -2;
                }
                __syncthreads();
                if (act)
                    for (int t = 0; t < nj; ++t) {
                        bool touch = false;
                        for (int a = 0; a < P.nv; ++a)
                            for (int bb = 0; bb < P.nv; ++bb) touch |= (cv[a] == sv[t * 4 + bb]);
                        if (touch) continue;
                        double r2 = 0.0;
                        for (int c = 0; c < d; ++c) {
                            double dd = x[c] - sx[t * d + c];
                            r2 += dd * dd;
                        }
                        acc += gamma_ab(P.mt, r2, a_, sl[t], b_, ss[t]);
                    }
            }
        }
        if (act) {
            // far part: sum over the ancestors of the leaf of l^node(q) . yhat_node
            int nd = node;
            for (int lev = P.Lt; lev >= 0; --lev) {
                // 1D Lagrange values on the node's box from the reference points:
                // l_a(t) = w_a prod_{b != a} (t - t_b), t the point in [-1, 1] box
                // coordinates (prefix and suffix products, no divisions per a)
                double l1[3][PMAX];
                for (int c = 0; c < d; ++c) {
                    const double lo = P.tt_lo[(size_t)nd * d + c], hi = P.tt_hi[(size_t)nd * d + c];
                    const double t = (x[c] - 0.5 * (lo + hi)) / (0.5 * (hi - lo));
                    double df[PMAX], pre = 1.0;
                    for (int a = 0; a < P.p; ++a) df[a] = t - P.tref[a];
                    for (int a = 0; a < P.p; ++a) {
                        l1[c][a] = pre;
                        pre *= df[a];
                    }
                    double suf = 1.0;
                    for (int a = P.p - 1; a >= 0; --a) {
                        l1[c][a] *= suf * P.wref[a];
                        suf *= df[a];
                    }
                }
                // tensor basis alpha = a0 + p a1 (+ p^2 a2): nested loops, no index division
                const double *y = P.yt + (size_t)nd * P.k;
                const int pp = P.p;
                if (d == 1) {
                    for (int a0 = 0; a0 < pp; ++a0) acc += l1[0][a0] * y[a0];
                } else if (d == 2) {
                    for (int a1 = 0; a1 < pp; ++a1) {
                        double s1 = 0.0;
                        for (int a0 = 0; a0 < pp; ++a0) s1 += l1[0][a0] * y[a1 * pp + a0];
                        acc += l1[1][a1] * s1;
                    }
                } else {
                    for (int a2 = 0; a2 < pp; ++a2) {
                        double s2 = 0.0;
                        for (int a1 = 0; a1 < pp; ++a1) {
                            double s1 = 0.0;
                            for (int a0 = 0; a0 < pp; ++a0) s1 += l1[0][a0] * y[(a2 * pp + a1) * pp + a0];
                            s2 += l1[1][a1] * s1;
                        }
                        acc += l1[2][a2] * s2;
                    }
                }
                nd = (nd - 1) / 2;
            }
            if (P.tail) {
                // rho_B (Sec. 7.1.1, eq. e:rho), constant s and kappa
                double a = exp(l_), tl;
                if (d == 1) {
                    tl = (pow(P.R - x[0], -2.0 * s_) + pow(P.R + x[0], -2.0 * s_)) / (2.0 * s_);
                } else {
                    double r2 = x[0] * x[0] + x[1] * x[1], t9 = 0.0;
                    for (int q = 0; q < 9; ++q) {
                        double sth, cth;
                        sincospi(2.0 * P.g9x[q], &sth, &cth);
                        double mu = x[0] * cth + x[1] * sth;
                        double t = sqrt(mu * mu + P.R * P.R - r2) - mu;
                        t9 += P.g9w[q] * exp(-2.0 * s_ * log(t));
                    }
                    tl = 2.0 * M_PI * t9 / (2.0 * s_);
                }
                acc += a * tl;
            }
            P.rho[id] = acc;
        }
    }
}

void launch_density(const MeshData &m, OpData &op, cudaStream_t st)
{
    const int d = m.d, k = m.k;
    op.rho.alloc(m.nQint);
    DBuf<double> yt;
    yt.alloc((size_t)m.tt.nnode * k);
    yt.zero(st);
    if (m.nrfar) {
        int n = m.tt.nnode * k;
        k_rho_coupling<<<cdiv(n, 128), 128, 0, st>>>(d, k, m.tt.nnode, m.rfar_ptr.p, m.rfar_col.p, m.tt_cheb.p,
                                                      op.tc_s.p, op.tc_lk.p, m.st_cheb.p, op.sc_s.p, op.sc_lk.p,
                                                      m.st_xhat.p, m.mtab.p, yt.p);
        VFD_CUDA(cudaGetLastError());
    }
    RhoParams P;
    P.d = d;
    P.k = k;
    P.p = m.p;
    P.Lt = m.tt.L;
    P.nQ = m.nQ;
    P.nQint = m.nQint;
    P.nv = d + 1;
    P.tt_begin = m.tt_begin.p;
    P.tt_end = m.tt_end.p;
    P.tt_perm = m.tt_perm.p;
    P.st_begin = m.st_begin.p;
    P.st_end = m.st_end.p;
    P.st_perm = m.st_perm.p;
    P.tt_cheb = m.tt_cheb.p;
    P.yt = yt.p;
    P.tt_lo = m.tt_lo.p;
    P.tt_hi = m.tt_hi.p;
    for (int a = 0; a < PMAX; ++a) P.tref[a] = P.wref[a] = 0.0;
    for (int a = 0; a < m.p; ++a) P.tref[a] = std::cos((2.0 * a + 1.0) * M_PI / (2.0 * m.p));
    for (int a = 0; a < m.p; ++a) {
        double w = 1.0;
        for (int b = 0; b < m.p; ++b)
            if (b != a) w *= P.tref[a] - P.tref[b];
        P.wref[a] = 1.0 / w;
    }
    P.rnear_ptr = m.rnear_ptr.p;
    P.rnear_col = m.rnear_col.p;
    P.qx = m.qx.p;
    P.qw = m.qw.p;
    P.qs = op.q_s.p;
    P.qlk = op.q_lk.p;
    P.qcell = m.qcell.p;
    P.cells = m.cells.p;
    P.tail = m.opts.tail_mode;
    P.R = m.opts.tail_R;
    P.g9x = m.gl9_x.p;
    P.g9w = m.gl9_w.p;
    P.mt = m.mtab.p;
    P.rho = op.rho.p;
    size_t shm = 128 * (d + 2) * sizeof(double) + 128 * 4 * sizeof(int);
    k_rho_points<<<m.tt.nleaf, 128, shm, st>>>(P);
    VFD_CUDA(cudaGetLastError());
    VFD_CUDA(cudaStreamSynchronize(st));   // yt is released on return
}

// ---------------------------------------------------------------------------
// coupling blocks S_{sigma,sigma'}[a][b] = -2 gamma(xi_a, xi_b) (eq. eq:triple_product),
// xi_a the Chebyshev nodes of the row box, xi_b those of the column box
// ---------------------------------------------------------------------------
__global__ void k_coupling(int d, int k, int nnode, const int *__restrict__ fptr, const int *__restrict__ fcol,
                           const double *__restrict__ ch, const double *__restrict__ cs,
                           const double *__restrict__ clk, const double *__restrict__ mt, double *__restrict__ S)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long kk = (long long)k * k;
    int nfar = fptr[nnode];
    if (i >= (long long)nfar * kk) return;
    // stored transposed, S_e[b][a], so that the apply reads rows coalesced
    int e = (int)(i / kk), r = (int)(i % kk), be = r / k, al = r % k;
    // row node of block e: binary search in fptr
    int lo = 0, hi = nnode;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (fptr[mid] <= e) lo = mid; else hi = mid;
    }
    int a = lo, b = fcol[e];
    int ia = a * k + al, ib = b * k + be;
    double r2 = 0.0;
    for (int c = 0; c < d; ++c) {
        double dd = ch[(size_t)ia * d + c] - ch[(size_t)ib * d + c];
        r2 += dd * dd;
    }
    S[i] = -2.0 * gamma_r2t(mt, d, r2, cs[ia], cs[ib], clk[ia], clk[ib]);
}

void launch_coupling_build(const MeshData &m, OpData &op, cudaStream_t st)
{
    const long long n = (long long)m.nfar * m.k * m.k;
    op.S64.alloc(n);
    if (!n) return;
    k_coupling<<<cdiv(n, 256), 256, 0, st>>>(m.d, m.k, m.kt.nnode, m.far_ptr.p, m.far_col.p, m.kt_cheb.p, op.kc_s.p,
                                             op.kc_lk.p, m.mtab.p, op.S64.p);
    VFD_CUDA(cudaGetLastError());
    if (m.k_in && op.precision != VFD_FP64) {
        // the inner operator's coupling blocks at its lower interpolation order
        const long long ni = (long long)m.nfar * m.k_in * m.k_in;
        op.S64_in.alloc(ni);
        k_coupling<<<cdiv(ni, 256), 256, 0, st>>>(m.d, m.k_in, m.kt.nnode, m.far_ptr.p, m.far_col.p, m.kt_cheb_in.p,
                                                  op.kc_s_in.p, op.kc_lk_in.p, m.mtab.p, op.S64_in.p);
        VFD_CUDA(cudaGetLastError());
    }
}

// ---------------------------------------------------------------------------
// dense inadmissible leaf blocks (Sec. 5.2, eq. e:k-near):
//   D[i][j] = -2 sum_{q in supp i} sum_{q' in supp j} c_i(q) c_j(q') gamma_T(q, q')
// with c_i(q) = w_q psi_i(q) and gamma_T = 0 on touching cells.  One CTA per
// block (row leaf <= col leaf); the point-pair kernel matrix is generated in
// shared-memory tiles of TQ row points and contracted with the sparse
// supports, so every gamma_T(q, q') is evaluated once per block.
// ---------------------------------------------------------------------------
struct NearParams {
    int d, nv, nQ, fl, TQ, maxpts, maxleaf;
    const int *near_ptr, *near_col, *near_src, *prow;
    const int64_t *near_off;
    const int *panel_w;
    const int *kt_begin, *kt_end;
    const int *lp_ptr, *lp_pts, *supp_ptr, *supp_loc;
    const double *supp_coef;
    const double *qx, *qs, *qlk;
    const int *qcell, *cells;
    const double *mt;
    double *D;
};

__global__ void __launch_bounds__(256) k_near_build(NearParams P)
{
    extern __shared__ double sh[];
    const int e = blockIdx.x;
    if (P.near_src[e] >= 0) return;   // transposed copy, filled by k_near_transpose
    const int a = P.prow[e], b = P.near_col[e];
    const int d = P.d, nv = P.nv, TQ = P.TQ;
    const int ra = P.kt_begin[P.fl + a], na = P.kt_end[P.fl + a] - ra;
    const int rb = P.kt_begin[P.fl + b], nb = P.kt_end[P.fl + b] - rb;
    const int pa0 = P.lp_ptr[a], npa = P.lp_ptr[a + 1] - pa0;
    const int pb0 = P.lp_ptr[b], npb = P.lp_ptr[b + 1] - pb0;
    // shared layout
    double *G = sh;                                  // TQ * maxpts
    double *Tm = G + (size_t)TQ * P.maxpts;          // TQ * maxleaf
    double *Dacc = Tm + (size_t)TQ * P.maxleaf;      // maxleaf * maxleaf
    double *bx = Dacc + (size_t)P.maxleaf * P.maxleaf;  // maxpts * d
    double *bs = bx + (size_t)P.maxpts * d;           // b = s/2 + d/4 of the column points
    double *bl = bs + P.maxpts;                       // a = log(kappa)/2
    double *tx = bl + P.maxpts;                       // row tile: TQ * d coordinates, a, b
    double *ta = tx + (size_t)TQ * d;
    double *tb = ta + TQ;
    int *bv = (int *)(tb + TQ);                       // maxpts * 4 cell vertex ids
    int *tv = bv + (size_t)P.maxpts * 4;              // TQ * 4
    const double dq = 0.25 * d;
    for (int t = threadIdx.x; t < npb; t += blockDim.x) {
        int id = P.lp_pts[pb0 + t];
        for (int c = 0; c < d; ++c) bx[t * d + c] = P.qx[(size_t)c * P.nQ + id];
        bs[t] = fma(0.5, P.qs[id], dq);
        bl[t] = 0.5 * P.qlk[id];
        int cell = P.qcell[id];
        for (int q = 0; q < 4; ++q) bv[t * 4 + q] = q < nv ? P.cells[(size_t)cell * nv + q] : -2;
    }
    for (int t = threadIdx.x; t < na * nb; t += blockDim.x) Dacc[t] = 0.0;
    __syncthreads();
    for (int t0 = 0; t0 < npa; t0 += TQ) {
        const int nt = min(TQ, npa - t0);
        for (int tq = threadIdx.x; tq < nt; tq += blockDim.x) {
            const int id = P.lp_pts[pa0 + t0 + tq], cell = P.qcell[id];
            for (int c = 0; c < d; ++c) tx[tq * d + c] = P.qx[(size_t)c * P.nQ + id];
            ta[tq] = 0.5 * P.qlk[id];
            tb[tq] = fma(0.5, P.qs[id], dq);
            for (int u = 0; u < 4; ++u) tv[tq * 4 + u] = u < nv ? P.cells[(size_t)cell * nv + u] : -3;
        }
        __syncthreads();
        // kernel tile G[tq][l] = gamma_T(q_{t0+tq}, q_l)
        for (int idx = threadIdx.x; idx < nt * npb; idx += blockDim.x) {
            int tq = idx / npb, l = idx - tq * npb;
            bool touch = false;
            for (int u = 0; u < nv; ++u) {
                int va = tv[tq * 4 + u];
                for (int w = 0; w < nv; ++w) touch |= (va == bv[l * 4 + w]);
            }
            double g = 0.0;
            if (!touch) {
                double r2 = 0.0;
                for (int c = 0; c < d; ++c) {
                    double dd = tx[tq * d + c] - bx[l * d + c];
                    r2 += dd * dd;
                }
                g = gamma_ab(P.mt, r2, ta[tq], bl[l], tb[tq], bs[l]);
            }
            G[(size_t)tq * npb + l] = g;
        }
        __syncthreads();
        // T[tq][j] = sum_{(l,c) in supp(j)} G[tq][l] c
        for (int idx = threadIdx.x; idx < nt * nb; idx += blockDim.x) {
            int tq = idx / nb, j = idx - tq * nb;
            int dj = rb + j;
            double v = 0.0;
            for (int s = P.supp_ptr[dj]; s < P.supp_ptr[dj + 1]; ++s) v += G[(size_t)tq * npb + P.supp_loc[s]] * P.supp_coef[s];
            Tm[(size_t)tq * nb + j] = v;
        }
        __syncthreads();
        // Dacc[i][j] += sum_{(l,c) in supp(i), l in tile} c T[l - t0][j]
        for (int idx = threadIdx.x; idx < na * nb; idx += blockDim.x) {
            int i = idx / nb, j = idx - i * nb;
            int di = ra + i;
            double v = 0.0;
            for (int s = P.supp_ptr[di]; s < P.supp_ptr[di + 1]; ++s) {
                int l = P.supp_loc[s] - t0;
                if (l >= 0 && l < nt) v += P.supp_coef[s] * Tm[(size_t)l * nb + j];
            }
            Dacc[idx] += v;
        }
        __syncthreads();
    }
    // write into the row panel of leaf a (row stride panel_w[a])
    double *out = P.D + P.near_off[e];
    const int W = P.panel_w[a];
    for (int t = threadIdx.x; t < na * nb; t += blockDim.x) {
        int i = t / nb, j = t - i * nb;
        out[(size_t)i * W + j] = -2.0 * Dacc[t];
    }
}

// The same block, with the column points tiled as well (leaf point sets too
// large to stage whole, as with tetrahedra): for each tile of TQ row points,
// T[tq][j] accumulates over tiles of TC column points, then the row supports
// fold T into the block.  Every gamma_T(q, q') is still evaluated once per block.
constexpr int NB_TC = 128;   // column points per tile

__global__ void __launch_bounds__(256) k_near_build_tiled(NearParams P)
{
    extern __shared__ double sh[];
    const int e = blockIdx.x;
    if (P.near_src[e] >= 0) return;   // transposed copy, filled by k_near_transpose
    const int a = P.prow[e], b = P.near_col[e];
    const int d = P.d, nv = P.nv, TQ = P.TQ, TC = NB_TC;
    const int ra = P.kt_begin[P.fl + a], na = P.kt_end[P.fl + a] - ra;
    const int rb = P.kt_begin[P.fl + b], nb = P.kt_end[P.fl + b] - rb;
    const int pa0 = P.lp_ptr[a], npa = P.lp_ptr[a + 1] - pa0;
    const int pb0 = P.lp_ptr[b], npb = P.lp_ptr[b + 1] - pb0;
    double *G = sh;                                   // TQ * TC
    double *Tm = G + (size_t)TQ * TC;                 // TQ * maxleaf
    double *Dacc = Tm + (size_t)TQ * P.maxleaf;       // maxleaf * maxleaf
    double *cx = Dacc + (size_t)P.maxleaf * P.maxleaf;   // TC * d, then b, a of the column tile
    double *cb = cx + (size_t)TC * d;
    double *ca = cb + TC;
    double *tx = ca + TC;                             // TQ * d, a, b of the row tile
    double *ta = tx + (size_t)TQ * d;
    double *tb = ta + TQ;
    int *cv = (int *)(tb + TQ);                       // TC * 4 cell vertex ids
    int *tv = cv + (size_t)TC * 4;                    // TQ * 4
    const double dq = 0.25 * d;
    for (int t = threadIdx.x; t < na * nb; t += blockDim.x) Dacc[t] = 0.0;
    for (int t0 = 0; t0 < npa; t0 += TQ) {
        const int nt = min(TQ, npa - t0);
        __syncthreads();
        for (int tq = threadIdx.x; tq < nt; tq += blockDim.x) {
            const int id = P.lp_pts[pa0 + t0 + tq], cell = P.qcell[id];
            for (int c = 0; c < d; ++c) tx[tq * d + c] = P.qx[(size_t)c * P.nQ + id];
            ta[tq] = 0.5 * P.qlk[id];
            tb[tq] = fma(0.5, P.qs[id], dq);
            for (int u = 0; u < 4; ++u) tv[tq * 4 + u] = u < nv ? P.cells[(size_t)cell * nv + u] : -3;
        }
        for (int t = threadIdx.x; t < nt * nb; t += blockDim.x) Tm[t] = 0.0;
        for (int c0 = 0; c0 < npb; c0 += TC) {
            const int nc = min(TC, npb - c0);
            __syncthreads();   // previous G / column tile consumed
            for (int t = threadIdx.x; t < nc; t += blockDim.x) {
                const int id = P.lp_pts[pb0 + c0 + t], cell = P.qcell[id];
                for (int c = 0; c < d; ++c) cx[t * d + c] = P.qx[(size_t)c * P.nQ + id];
                cb[t] = fma(0.5, P.qs[id], dq);
                ca[t] = 0.5 * P.qlk[id];
                for (int q = 0; q < 4; ++q) cv[t * 4 + q] = q < nv ? P.cells[(size_t)cell * nv + q] : -2;
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < nt * nc; idx += blockDim.x) {
                const int tq = idx / nc, l = idx - tq * nc;
                bool touch = false;
                for (int u = 0; u < nv; ++u) {
                    const int va = tv[tq * 4 + u];
                    for (int w = 0; w < nv; ++w) touch |= (va == cv[l * 4 + w]);
                }
                double g = 0.0;
                if (!touch) {
                    double r2 = 0.0;
                    for (int c = 0; c < d; ++c) {
                        const double dd = tx[tq * d + c] - cx[l * d + c];
                        r2 += dd * dd;
                    }
                    g = gamma_ab(P.mt, r2, ta[tq], ca[l], tb[tq], cb[l]);
                }
                G[(size_t)tq * TC + l] = g;
            }
            __syncthreads();
            // T[tq][j] += sum_{(l,c) in supp(j), l in this column tile} G[tq][l - c0] c
            for (int idx = threadIdx.x; idx < nt * nb; idx += blockDim.x) {
                const int tq = idx / nb, j = idx - tq * nb, dj = rb + j;
                double v = 0.0;
                for (int s2 = P.supp_ptr[dj]; s2 < P.supp_ptr[dj + 1]; ++s2) {
                    const int l = P.supp_loc[s2] - c0;
                    if (l >= 0 && l < nc) v += G[(size_t)tq * TC + l] * P.supp_coef[s2];
                }
                Tm[idx] += v;
            }
        }
        __syncthreads();
        // Dacc[i][j] += sum_{(l,c) in supp(i), l in the row tile} c T[l - t0][j]
        for (int idx = threadIdx.x; idx < na * nb; idx += blockDim.x) {
            const int i = idx / nb, j = idx - i * nb, di = ra + i;
            double v = 0.0;
            for (int s2 = P.supp_ptr[di]; s2 < P.supp_ptr[di + 1]; ++s2) {
                const int l = P.supp_loc[s2] - t0;
                if (l >= 0 && l < nt) v += P.supp_coef[s2] * Tm[(size_t)l * nb + j];
            }
            Dacc[idx] += v;
        }
    }
    __syncthreads();
    double *out = P.D + P.near_off[e];
    const int W = P.panel_w[a];
    for (int t = threadIdx.x; t < na * nb; t += blockDim.x) {
        const int i = t / nb, j = t - i * nb;
        out[(size_t)i * W + j] = -2.0 * Dacc[t];
    }
}

__global__ void k_near_transpose(int nnear, const int *__restrict__ src, const int *__restrict__ prow,
                                 const int *__restrict__ ncol, const int *__restrict__ kb, const int *__restrict__ ke,
                                 int fl, const int64_t *__restrict__ off, const int *__restrict__ pw,
                                 double *__restrict__ D)
{
    int e = blockIdx.x;
    int s = src[e];
    if (s < 0) return;
    int a = prow[e], b = ncol[e];
    int na = ke[fl + a] - kb[fl + a], nb = ke[fl + b] - kb[fl + b];
    const int Wa = pw[a], Wb = pw[b];
    const double *in = D + off[s];   // block (b, a): nb rows, stride Wb
    double *out = D + off[e];        // block (a, b): na rows, stride Wa
    for (int t = threadIdx.x; t < na * nb; t += blockDim.x) {
        int i = t / nb, j = t % nb;
        out[(size_t)i * Wa + j] = in[(size_t)j * Wb + i];
    }
}

void launch_near_build(const MeshData &m, OpData &op, cudaStream_t st)
{
    op.D64.alloc(m.near_entries);
    if (!m.nnear) return;
    op.D64.zero(st);   // panel padding columns stay zero
    NearParams P;
    P.d = m.d;
    P.nv = m.d + 1;
    P.nQ = m.nQ;
    P.fl = m.kt.first_leaf();
    P.maxpts = m.max_leaf_pts;
    P.maxleaf = m.max_leaf_size;
    P.near_ptr = m.near_ptr.p;
    P.near_col = m.near_col.p;
    P.near_src = m.near_src.p;
    P.prow = m.near_pair_row.p;
    P.near_off = m.near_off.p;
    P.panel_w = m.panel_w.p;
    P.kt_begin = m.kt_begin.p;
    P.kt_end = m.kt_end.p;
    P.lp_ptr = m.lp_ptr.p;
    P.lp_pts = m.lp_pts.p;
    P.supp_ptr = m.supp_ptr.p;
    P.supp_loc = m.supp_loc.p;
    P.supp_coef = m.supp_coef.p;
    P.qx = m.qx.p;
    P.qs = op.q_s.p;
    P.qlk = op.q_lk.p;
    P.qcell = m.qcell.p;
    P.cells = m.cells.p;
    P.mt = m.mtab.p;
    P.D = op.D64.p;
    auto shm_for = [&](int TQ) {
        return (size_t)TQ * P.maxpts * 8 + (size_t)TQ * P.maxleaf * 8 + (size_t)P.maxleaf * P.maxleaf * 8 +
               (size_t)P.maxpts * (m.d + 2) * 8 + (size_t)TQ * (m.d + 2) * 8 + (size_t)P.maxpts * 4 * 4 +
               (size_t)TQ * 4 * 4;
    };
    int TQ = 32;
    while (TQ > 1 && shm_for(TQ) > 200 * 1024) TQ /= 2;
    size_t shm = shm_for(TQ);
    if (shm <= 200 * 1024 && TQ >= 8) {
        P.TQ = TQ;
        VFD_CUDA(cudaFuncSetAttribute(k_near_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        k_near_build<<<m.nnear, 256, shm, st>>>(P);
    } else {
        // the column points tiled too (large leaf point sets, e.g. tetrahedra)
        P.TQ = 32;
        const size_t tshm = (size_t)P.TQ * NB_TC * 8 + (size_t)P.TQ * P.maxleaf * 8 + (size_t)P.maxleaf * P.maxleaf * 8 +
                            (size_t)NB_TC * (m.d + 2) * 8 + (size_t)P.TQ * (m.d + 2) * 8 + (size_t)NB_TC * 4 * 4 +
                            (size_t)P.TQ * 4 * 4;
        VFD_REQUIRE(tshm <= 220 * 1024, VFD_EUNSUPPORTED, "leaves too large for the near-block kernel");
        VFD_CUDA(cudaFuncSetAttribute(k_near_build_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tshm));
        k_near_build_tiled<<<m.nnear, 256, tshm, st>>>(P);
    }
    VFD_CUDA(cudaGetLastError());
    k_near_transpose<<<m.nnear, 256, 0, st>>>(m.nnear, m.near_src.p, m.near_pair_row.p, m.near_col.p, m.kt_begin.p,
                                              m.kt_end.p, P.fl, m.near_off.p, m.panel_w.p, op.D64.p);
    VFD_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// FP32 copies of the K data (VFD_FP32 operators)
// ---------------------------------------------------------------------------
__global__ void k_to_f32(long long n, const double *__restrict__ a, float *__restrict__ b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

static void to32(const DBuf<double> &a, DBuf<float> &b, cudaStream_t st)
{
    b.alloc(a.n);
    if (a.n) k_to_f32<<<cdiv((long long)a.n, 256), 256, 0, st>>>((long long)a.n, a.p, b.p);
    VFD_CUDA(cudaGetLastError());
}

void launch_convert_fp32(const MeshData &m, OpData &op, cudaStream_t st)
{
    to32(op.S64, op.S32, st);
    to32(op.D64, op.D32, st);
    to32(m.Ul64, op.Ul32, st);
}

// ---------------------------------------------------------------------------
// P1 load vector F_i = sum_{tau ∋ i} sum_b (M0^tau)_{ab} f_b
// ---------------------------------------------------------------------------
__global__ void k_load(int N, int d, int M, const int *__restrict__ ptr, const int *__restrict__ idx,
                       const int *__restrict__ cells, const double *__restrict__ vx, const double *__restrict__ f,
                       double *__restrict__ F)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int nv = d + 1;
    double acc = 0.0;
    for (int c = ptr[i]; c < ptr[i + 1]; ++c) {
        int cell = idx[c] / nv, a = idx[c] % nv;
        const int *t = cells + (size_t)cell * nv;
        double meas;
        if (d == 1) {
            meas = fabs(vx[t[1]] - vx[t[0]]);
        } else if (d == 2) {
            double x0 = vx[t[0]], y0 = vx[M + t[0]], x1 = vx[t[1]], y1 = vx[M + t[1]], x2 = vx[t[2]], y2 = vx[M + t[2]];
            meas = 0.5 * fabs((x1 - x0) * (y2 - y0) - (y1 - y0) * (x2 - x0));
        } else {
            double e[3][3];
            for (int u = 0; u < 3; ++u)
                for (int c = 0; c < 3; ++c) e[u][c] = vx[(size_t)c * M + t[u + 1]] - vx[(size_t)c * M + t[0]];
            meas = fabs(e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                        e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0])) / 6.0;
        }
        double den = (d == 1) ? 6.0 : (d == 2) ? 12.0 : 20.0;   // int lam_a lam_b = |tau|(1+delta_ab) d!/(d+2)!
        for (int bb = 0; bb < nv; ++bb) acc += meas * (a == bb ? 2.0 : 1.0) / den * f[t[bb]];
    }
    F[i] = acc;
}

__global__ void k_selftest_math(int which, long long n, const double *__restrict__ mt, const double *__restrict__ x,
                                double *__restrict__ out)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (which <= 1) {
        out[i] = which == 0 ? fast_log(mt, x[i]) : fast_exp(mt, x[i]);
    } else {
        double s, c;
        sincospi_tab(mt, x[i], s, c);
        out[i] = which == 2 ? c : s;
    }
}

void launch_selftest_math(const MeshData &m, int which, long long n, const double *x, double *out, cudaStream_t st)
{
    if (n > 0) k_selftest_math<<<cdiv(n, 256), 256, 0, st>>>(which, n, m.mtab.p, x, out);
    VFD_CUDA(cudaGetLastError());
}

void launch_load(const MeshData &m, const double *f, double *F, cudaStream_t st)
{
    k_load<<<cdiv(m.N, 256), 256, 0, st>>>(m.N, m.d, m.M, m.ld_ptr.p, m.ld_idx.p, m.cells.p, m.vx.p, f, F);
    VFD_CUDA(cudaGetLastError());
}

}  // namespace vfd
