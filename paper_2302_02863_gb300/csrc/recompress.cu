// Algebraic recompression of the interpolation H^2 far field of K (the last
// paragraph of Sec. 5.3: the Chebyshev bases have more columns than the
// coupling needs).  For the FP64 operator, with the bases of every level
// flattened (V_s = Ul^(l) restricted to the rows of node s):
//
//   1. orthogonalise every node's basis (geometry only, once per mesh):
//      G_s = V_s^T V_s = W L W^T,  V_s = Q_s R_s with Q_s = V_s W L^-1/2
//      (orthonormal columns) and R_s = L^1/2 W^T, eigenvalues below 1e-16 of
//      the largest dropped;
//   2. per assembly, the couplings in those coordinates, Sh_e = R_s S_e R_t^T,
//      and per node the Gram matrix of its coupling row C_s = sum_e Sh_e Sh_e^T
//      = P D P^T; keep the directions with sqrt(d) > tol * (largest over all
//      nodes) -- the singular directions of the node's coupling row;
//   3. new bases V'_s = V_s W L^-1/2 P_s and couplings S'_e = P_s^T Sh_e P_t,
//      ranks padded to the largest of each level.
//
// V_s S_e V_t^T = Q_s Sh_e Q_t^T, and the truncation removes only directions
// whose coupling row (and, by the symmetry of the block list, column) is below
// the tolerance.  Every symmetric eigenproblem is solved on the device by
// cyclic Jacobi with a parallel (round-robin) ordering, one CTA per matrix.
#include <algorithm>
#include <cmath>
#include <vector>

#include "device_common.cuh"

namespace vfd {

namespace {

__device__ __forceinline__ int node_level(int n)
{
    int l = 0;
    while ((2 << l) - 1 <= n) ++l;
    return l;
}

// G[n] = sum over the rows i of node n of Ul^(l)[i]^T Ul^(l)[i] (nodes with
// admissible blocks); rows staged in shared memory in chunks of 32
__global__ void __launch_bounds__(256) k_rc_gram(int k, int N, int lmin, const int *__restrict__ fptr,
                                                 const int *__restrict__ kb, const int *__restrict__ ke,
                                                 const double *__restrict__ Ul, double *__restrict__ G)
{
    __shared__ double rs[32][KMAX];
    const int n = blockIdx.x;
    if (fptr[n + 1] == fptr[n]) return;
    const int l = node_level(n);
    const double *U = Ul + (size_t)(l - lmin) * N * k;
    const int b = kb[n], e = ke[n];
    double acc[16];
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int i0 = b; i0 < e; i0 += 32) {
        const int nr = min(32, e - i0);
        __syncthreads();
        for (int t = threadIdx.x; t < nr * k; t += blockDim.x) rs[t / k][t % k] = U[(size_t)(i0 + t / k) * k + t % k];
        __syncthreads();
        for (int q = 0; q < 16; ++q) {
            const int t = threadIdx.x + q * blockDim.x;
            if (t >= k * k) break;
            const int a = t / k, c = t % k;
            double s = acc[q];
            for (int r = 0; r < nr; ++r) s = fma(rs[r][a], rs[r][c], s);
            acc[q] = s;
        }
    }
    for (int q = 0; q < 16; ++q) {
        const int t = threadIdx.x + q * blockDim.x;
        if (t < k * k) G[(size_t)n * k * k + t] = acc[q];
    }
}

// symmetric eigendecomposition of the k x k matrices mats[m] (m in ids, or
// every m when ids is null) by cyclic Jacobi, round-robin pairs of a padded
// even order; evals[m][i], evecs[m][row][i] (column i the i-th eigenvector)
__global__ void __launch_bounds__(256) k_rc_jacobi(int k, const int *__restrict__ ids, const double *__restrict__ mats,
                                                   double *__restrict__ evals, double *__restrict__ evecs)
{
    extern __shared__ double js[];
    const int m = ids ? ids[blockIdx.x] : blockIdx.x;
    const int n = k + (k & 1);   // even order (a zero row and column padded when k is odd)
    double *A = js, *V = js + n * n;
    __shared__ double cs_c[KMAX / 2 + 1], cs_s[KMAX / 2 + 1], red[256];
    __shared__ int cs_p[KMAX / 2 + 1], cs_q[KMAX / 2 + 1];
    __shared__ int stop;
    const double *M = mats + (size_t)m * k * k;
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        A[t] = (i < k && j < k) ? M[i * k + j] : 0.0;
        V[t] = i == j ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int sweep = 0; sweep < 20; ++sweep) {
        double off = 0.0, dg = 0.0;
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = t / n, j = t % n;
            const double v = A[t] * A[t];
            if (i == j) dg += v;
            else off += v;
        }
        red[threadIdx.x] = off;
        __syncthreads();
        if (threadIdx.x == 0) {
            double so = 0.0;
            for (int q = 0; q < (int)blockDim.x; ++q) so += red[q];
            red[0] = so;
        }
        __syncthreads();
        const double offs = red[0];
        __syncthreads();
        red[threadIdx.x] = dg;
        __syncthreads();
        if (threadIdx.x == 0) {
            double sd = 0.0;
            for (int q = 0; q < (int)blockDim.x; ++q) sd += red[q];
            stop = !(offs > 1e-30 * (sd + offs));
        }
        __syncthreads();
        if (stop) break;
        for (int r = 0; r < n - 1; ++r) {
            if ((int)threadIdx.x < n / 2) {
                const int t = threadIdx.x;
                int p, q;
                if (t == 0) {
                    p = r % (n - 1);
                    q = n - 1;
                } else {
                    p = (r + t) % (n - 1);
                    q = (r - t + (n - 1)) % (n - 1);
                }
                if (p > q) {
                    const int w = p;
                    p = q;
                    q = w;
                }
                const double apq = A[p * n + q];
                double c = 1.0, s = 0.0;
                if (fabs(apq) > 1e-300) {
                    const double tau = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                    const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = 1.0 / sqrt(1.0 + tt * tt);
                    s = tt * c;
                }
                cs_c[t] = c;
                cs_s[t] = s;
                cs_p[t] = p;
                cs_q[t] = q;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < (n / 2) * n; e += blockDim.x) {   // rows p, q
                const int t = e / n, col = e % n, p = cs_p[t], q = cs_q[t];
                const double c = cs_c[t], s = cs_s[t], ap = A[p * n + col], aq = A[q * n + col];
                A[p * n + col] = c * ap - s * aq;
                A[q * n + col] = s * ap + c * aq;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < (n / 2) * n; e += blockDim.x) {   // columns p, q of A and V
                const int t = e / n, row = e % n, p = cs_p[t], q = cs_q[t];
                const double c = cs_c[t], s = cs_s[t];
                const double ap = A[row * n + p], aq = A[row * n + q];
                A[row * n + p] = c * ap - s * aq;
                A[row * n + q] = s * ap + c * aq;
                const double vp = V[row * n + p], vq = V[row * n + q];
                V[row * n + p] = c * vp - s * vq;
                V[row * n + q] = s * vp + c * vq;
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) evals[(size_t)m * k + i] = A[i * n + i];
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) evecs[(size_t)m * k * k + t] = V[(t / k) * n + t % k];
}

// per node: the kept eigen-directions of its basis Gram matrix (eigenvalue >
// 1e-16 of the largest), T1 = W L^-1/2 (k x k, kept columns first, zero after)
// and R = L^1/2 W^T (kept rows first, zero after)
__global__ void k_rc_factors(int k, const int *__restrict__ fptr, const double *__restrict__ ev,
                             const double *__restrict__ W, double *__restrict__ T1, double *__restrict__ R)
{
    const int n = blockIdx.x;
    if (fptr[n + 1] == fptr[n]) return;
    __shared__ int slot[KMAX];
    const double *e = ev + (size_t)n * k;
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int i = 0; i < k; ++i) mx = fmax(mx, e[i]);
        int r = 0;
        for (int i = 0; i < k; ++i) slot[i] = (e[i] > 1e-16 * mx && e[i] > 0.0) ? r++ : -1;
    }
    __syncthreads();
    double *t1 = T1 + (size_t)n * k * k, *rr = R + (size_t)n * k * k;
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        t1[t] = 0.0;
        rr[t] = 0.0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int a = t / k, i = t % k;   // W[a][i]: row a, eigenvector i
        const int sl = slot[i];
        if (sl < 0) continue;
        const double w = W[(size_t)n * k * k + t], lam = e[i];
        t1[a * k + sl] = w / sqrt(lam);
        rr[sl * k + a] = w * sqrt(lam);
    }
}

// Sh_e = R_s S_e R_t^T per admissible block (S stored [b][a]: S(a, b) = Se[b k + a]);
// CTA per block, the three k x k matrices in shared memory
__global__ void __launch_bounds__(256) k_rc_shat(int k, int nnode, int nfar, const int *__restrict__ fptr,
                                                 const int *__restrict__ fcol, const double *__restrict__ S,
                                                 const double *__restrict__ R, double *__restrict__ Sh)
{
    extern __shared__ double ss[];
    double *Ss = ss, *Ts = ss + k * k;   // Ss: S(a, b); Ts: T = S R_t^T
    const int e = blockIdx.x;
    int lo = 0, hi = nnode;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (fptr[mid] <= e) lo = mid; else hi = mid;
    }
    const int sg = lo, tau = fcol[e];
    const double *Se = S + (size_t)e * k * k, *Rs = R + (size_t)sg * k * k, *Rt = R + (size_t)tau * k * k;
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) Ss[(t % k) * k + t / k] = Se[t];   // Ss[a][b]
    __syncthreads();
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {   // T[a][j] = sum_b S(a, b) R_t[j][b]
        const int a = t / k, j = t % k;
        double v = 0.0;
        for (int b = 0; b < k; ++b) v = fma(Ss[a * k + b], Rt[(size_t)j * k + b], v);
        Ts[t] = v;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {   // Sh[i][j] = sum_a R_s[i][a] T[a][j]
        const int i = t / k, j = t % k;
        double v = 0.0;
        for (int a = 0; a < k; ++a) v = fma(Rs[(size_t)i * k + a], Ts[a * k + j], v);
        Sh[(size_t)e * k * k + t] = v;
    }
}

// C[n] = sum over the node's blocks of Sh_e Sh_e^T
__global__ void __launch_bounds__(256) k_rc_cgram(int k, const int *__restrict__ fptr, const double *__restrict__ Sh,
                                                  double *__restrict__ C)
{
    extern __shared__ double cs[];
    const int n = blockIdx.x;
    if (fptr[n + 1] == fptr[n]) return;
    double acc[16];
    for (int q = 0; q < 16; ++q) acc[q] = 0.0;
    for (int e = fptr[n]; e < fptr[n + 1]; ++e) {
        __syncthreads();
        for (int t = threadIdx.x; t < k * k; t += blockDim.x) cs[t] = Sh[(size_t)e * k * k + t];
        __syncthreads();
        for (int q = 0; q < 16; ++q) {
            const int t = threadIdx.x + q * blockDim.x;
            if (t >= k * k) break;
            const int i = t / k, j = t % k;
            double s = acc[q];
            for (int b = 0; b < k; ++b) s = fma(cs[i * k + b], cs[j * k + b], s);
            acc[q] = s;
        }
    }
    for (int q = 0; q < 16; ++q) {
        const int t = threadIdx.x + q * blockDim.x;
        if (t < k * k) C[(size_t)n * k * k + t] = acc[q];
    }
}

// S'_e = P_s^T Sh_e P_t (kept directions of the nodes, compacted; slot[n][i]
// = position of eigenvector i among node n's kept ones or -1), stored
// transposed [b'][a'] with the level's padded rank kl
__global__ void __launch_bounds__(256) k_rc_snew(int k, int nnode, const int *__restrict__ fptr,
                                                 const int *__restrict__ fcol, const double *__restrict__ Sh,
                                                 const double *__restrict__ P, const int *__restrict__ slot,
                                                 const int *__restrict__ bk, const long long *__restrict__ so,
                                                 double *__restrict__ Sc)
{
    extern __shared__ double ss[];
    double *Hs = ss, *Ts = ss + k * k;
    const int e = blockIdx.x;
    int lo = 0, hi = nnode;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (fptr[mid] <= e) lo = mid; else hi = mid;
    }
    const int sg = lo, tau = fcol[e], kl = bk[e];
    const double *Ps = P + (size_t)sg * k * k, *Pt = P + (size_t)tau * k * k;
    const int *ls = slot + (size_t)sg * k, *lt = slot + (size_t)tau * k;
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) Hs[t] = Sh[(size_t)e * k * k + t];
    __syncthreads();
    // T[i][jj] = sum_j Sh[i][j] Pt[j][jj] for the kept eigenvectors jj of tau (original index)
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int i = t / k, jj = t % k;
        double v = 0.0;
        if (lt[jj] >= 0)
            for (int j = 0; j < k; ++j) v = fma(Hs[i * k + j], Pt[(size_t)j * k + jj], v);
        Ts[t] = v;
    }
    __syncthreads();
    double *out = Sc + so[e];
    for (int t = threadIdx.x; t < kl * kl; t += blockDim.x) out[t] = 0.0;
    __syncthreads();
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int ii = t / k, jj = t % k;   // kept eigenvector ii of s, jj of tau
        const int a = ls[ii], b = lt[jj];
        if (a < 0 || b < 0) continue;
        double v = 0.0;
        for (int i = 0; i < k; ++i) v = fma(Ps[(size_t)i * k + ii], Ts[i * k + jj], v);
        out[b * kl + a] = v;
    }
}

// per node: Z = T1 P (k x kl: the kept eigenvectors of C in slot order)
__global__ void k_rc_z(int k, const int *__restrict__ fptr, const double *__restrict__ T1,
                       const double *__restrict__ P, const int *__restrict__ slot, const int *__restrict__ nkl,
                       double *__restrict__ Z)
{
    const int n = blockIdx.x;
    double *z = Z + (size_t)n * k * k;
    const int kl = nkl[n];
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) z[t] = 0.0;
    if (fptr[n + 1] == fptr[n]) return;
    __syncthreads();
    const double *t1 = T1 + (size_t)n * k * k, *p = P + (size_t)n * k * k;
    const int *sl = slot + (size_t)n * k;
    for (int t = threadIdx.x; t < k * k; t += blockDim.x) {
        const int a = t / k, jj = t % k;
        const int c = sl[jj];
        if (c < 0 || c >= kl) continue;
        double v = 0.0;
        for (int i = 0; i < k; ++i) v = fma(t1[a * k + i], p[(size_t)i * k + jj], v);
        z[a * kl + c] = v;
    }
}

// new flattened bases: Ulc[lv][i][c] = sum_a Ul^(l)[i][a] Z_anc[a][c], c < kl[lv]
__global__ void k_rc_bases(int k, int N, int lmin, int L, int nlev, int fl, const int *__restrict__ vleaf,
                           const double *__restrict__ Ul, const double *__restrict__ Z, const int *__restrict__ kl,
                           const long long *__restrict__ uo, double *__restrict__ Ulc)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * nlev) return;
    const int i = (int)(t % N), lv = (int)(t / N), l = lmin + lv;
    const int node = ((fl + vleaf[i] + 1) >> (L - l)) - 1;
    const double *u = Ul + ((size_t)lv * N + i) * k, *z = Z + (size_t)node * k * k;
    const int kk = kl[lv];
    double *o = Ulc + uo[lv] + (size_t)i * kk;
    for (int c = 0; c < kk; ++c) {
        double v = 0.0;
        for (int a = 0; a < k; ++a) v = fma(u[a], z[a * kk + c], v);
        o[c] = v;
    }
}

}  // namespace

void recompress_far(MeshData &m, OpData &op, double tol, cudaStream_t st)
{
    op.rc_on = false;
    if (m.nfar == 0 || !(tol > 0.0)) return;
    const int k = m.k, nnode = m.kt.nnode, lmin = m.far_lmin, L = m.kt.L, nlev = L - lmin + 1;
    const size_t kk = (size_t)k * k;
    const size_t jshm = 2 * (size_t)(k + (k & 1)) * (k + (k & 1)) * sizeof(double);
    VFD_CUDA(cudaFuncSetAttribute(k_rc_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jshm));
    VFD_CUDA(cudaFuncSetAttribute(k_rc_shat, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * kk * 8)));
    VFD_CUDA(cudaFuncSetAttribute(k_rc_snew, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * kk * 8)));
    VFD_CUDA(cudaFuncSetAttribute(k_rc_cgram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kk * 8)));
    std::vector<int> nodes;   // nodes with admissible blocks
    for (int n = 0; n < nnode; ++n)
        if (m.far_ptr_h[n + 1] > m.far_ptr_h[n]) nodes.push_back(n);
    DBuf<int> ids;
    ids.upload(nodes);
    // 1. orthogonal factors of the bases (geometry only, once per mesh)
    if (!m.rc_factors) {
        DBuf<double> G, ev, W;
        G.alloc(nnode * kk);
        ev.alloc((size_t)nnode * k);
        W.alloc(nnode * kk);
        k_rc_gram<<<nnode, 256, 0, st>>>(k, m.N, lmin, m.far_ptr.p, m.kt_begin.p, m.kt_end.p, m.Ul64.p, G.p);
        k_rc_jacobi<<<(int)nodes.size(), 256, jshm, st>>>(k, ids.p, G.p, ev.p, W.p);
        m.rc_T1.alloc(nnode * kk);
        m.rc_R.alloc(nnode * kk);
        k_rc_factors<<<nnode, 256, 0, st>>>(k, m.far_ptr.p, ev.p, W.p, m.rc_T1.p, m.rc_R.p);
        VFD_CUDA(cudaGetLastError());
        VFD_CUDA(cudaStreamSynchronize(st));
        m.rc_factors = true;
    }
    // 2. couplings in orthonormal coordinates and the Gram matrices of the coupling rows
    DBuf<double> Sh, C, ev, P;
    Sh.alloc((size_t)m.nfar * kk);
    C.alloc(nnode * kk);
    ev.alloc((size_t)nnode * k);
    P.alloc(nnode * kk);
    ev.zero(st);
    k_rc_shat<<<m.nfar, 256, 2 * kk * 8, st>>>(k, nnode, m.nfar, m.far_ptr.p, m.far_col.p, op.S64.p, m.rc_R.p, Sh.p);
    k_rc_cgram<<<nnode, 256, kk * 8, st>>>(k, m.far_ptr.p, Sh.p, C.p);
    k_rc_jacobi<<<(int)nodes.size(), 256, jshm, st>>>(k, ids.p, C.p, ev.p, P.p);
    VFD_CUDA(cudaGetLastError());
    std::vector<double> hev((size_t)nnode * k);
    VFD_CUDA(cudaMemcpyAsync(hev.data(), ev.p, sizeof(double) * hev.size(), cudaMemcpyDeviceToHost, st));
    VFD_CUDA(cudaStreamSynchronize(st));
    // 3. ranks: singular values of the coupling rows against the largest
    double smax = 0.0;
    for (int n : nodes)
        for (int i = 0; i < k; ++i) smax = std::max(smax, std::sqrt(std::max(hev[(size_t)n * k + i], 0.0)));
    const double thr = tol * smax;
    std::vector<int> slot((size_t)nnode * k, -1), nk(nnode, 0), kl(nlev, 1);
    for (int n : nodes) {
        // kept directions in descending order of their singular values
        std::vector<int> idx;
        for (int i = 0; i < k; ++i)
            if (std::sqrt(std::max(hev[(size_t)n * k + i], 0.0)) > thr) idx.push_back(i);
        std::sort(idx.begin(), idx.end(), [&](int a, int b) { return hev[(size_t)n * k + a] > hev[(size_t)n * k + b]; });
        for (size_t c = 0; c < idx.size(); ++c) slot[(size_t)n * k + idx[c]] = (int)c;
        nk[n] = (int)idx.size();
        int l = 0;
        while ((2 << l) - 1 <= n) ++l;
        kl[l - lmin] = std::max(kl[l - lmin], nk[n]);
    }
    std::vector<int> nkl(nnode, 1), bk(m.nfar);
    for (int n = 0; n < nnode; ++n) {
        int l = 0;
        while ((2 << l) - 1 <= n) ++l;
        nkl[n] = l >= lmin ? kl[l - lmin] : 1;
    }
    std::vector<long long> so(m.nfar + 1, 0), uo(nlev + 1, 0);
    for (int n = 0; n < nnode; ++n)
        for (int e = m.far_ptr_h[n]; e < m.far_ptr_h[n + 1]; ++e) bk[e] = nkl[n];
    for (int e = 0; e < m.nfar; ++e) so[e + 1] = so[e] + (long long)bk[e] * bk[e];
    for (int lv = 0; lv < nlev; ++lv) uo[lv + 1] = uo[lv] + (long long)m.N * kl[lv];
    // 4. new couplings and bases
    DBuf<int> slot_d, bk_d, nkl_d, kl_d;
    slot_d.upload(slot);
    bk_d.upload(bk);
    nkl_d.upload(nkl);
    kl_d.upload(kl);
    op.rc_so.upload(so);
    op.rc_bk.upload(bk);
    op.Sc64.alloc(so[m.nfar]);
    k_rc_snew<<<m.nfar, 256, 2 * kk * 8, st>>>(k, nnode, m.far_ptr.p, m.far_col.p, Sh.p, P.p, slot_d.p, bk_d.p,
                                                op.rc_so.p, op.Sc64.p);
    DBuf<double> Z;
    Z.alloc(nnode * kk);
    k_rc_z<<<nnode, 256, 0, st>>>(k, m.far_ptr.p, m.rc_T1.p, P.p, slot_d.p, nkl_d.p, Z.p);
    DBuf<long long> uo_d;
    uo_d.upload(uo);
    op.Ulc64.alloc(uo[nlev]);
    k_rc_bases<<<cdiv((long long)m.N * nlev, 128), 128, 0, st>>>(k, m.N, lmin, L, nlev, m.kt.first_leaf(), m.vleaf.p,
                                                                 m.Ul64.p, Z.p, kl_d.p, uo_d.p, op.Ulc64.p);
    VFD_CUDA(cudaGetLastError());
    VFD_CUDA(cudaStreamSynchronize(st));
    op.rc_kl = kl;
    op.rc_uo = uo;
    op.rc_on = true;
}

}  // namespace vfd
