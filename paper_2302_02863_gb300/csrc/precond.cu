// Two-level preconditioner for the CG solves of A U = F (Sec. 7 solves with
// plain CG; a multilevel preconditioner is the paper's stated next step,
// Sec. 8):
//
//   M^-1 r = sum_leaves P_a^T A_aa^-1 P_a r  +  R^T A_c^-1 R r,
//
// an additive combination of exact solves with the diagonal block A_aa of
// every leaf of the cluster tree (its DoFs, A's rows and columns of that
// leaf: near panel block (a, a) plus the B + M entries inside the leaf) and a
// coarse solve on the space of functions constant on the clusters of one tree
// level (R the cluster indicator restriction, A_c = R A R^T; the level is the
// deepest one with at most PREC_MAX_COARSE clusters, the leaves themselves on
// meshes of up to that many leaves).  Both parts are symmetric positive
// definite, so M is too and CG applies.  Kind VFD_PREC_BLOCK_JACOBI keeps the
// leaf blocks only.
//
// Setup (once per operator, vfd_precondition): the diagonal blocks are
// gathered and inverted on the device (one CTA per leaf: Cholesky and the
// triangular inverses in shared memory, FP64); A_c is summed from the
// operator's parts (near-block sums, B + M entries, and per admissible block
// the coupling contracted with the per-level basis sums of the clusters) and
// inverted on the host.  FP32 copies of both serve the batched mixed-precision solve.  Apply
// (every PCG iteration, FP64 solve): one kernel per leaf for the local solves
// and the leaf sums, one for the coarse product, one for the prolongation.
#include <cmath>
#include <thread>
#include <vector>

#include "device_common.cuh"

namespace vfd {

namespace {

constexpr int PREC_MAX_COARSE = 512;
constexpr int PREC_SMEM_BLK = 96;   // largest leaf whose block is inverted in shared memory

// dense diagonal block of leaf a (na x na, row stride mb) from the near panel
// block (a, a) and the B + M rows of the leaf's DoFs
__global__ void k_diag_blocks(int fl, int mb, const int *__restrict__ kb, const int *__restrict__ ke,
                              const int *__restrict__ nptr, const int *__restrict__ ncol,
                              const int64_t *__restrict__ noff, const int *__restrict__ pw,
                              const double *__restrict__ D, const int *__restrict__ rowptr,
                              const int *__restrict__ colidx, const double *__restrict__ val,
                              double *__restrict__ out)
{
    const int a = blockIdx.x;
    const int b0 = kb[fl + a], na = ke[fl + a] - b0, W = pw[a];
    double *B = out + (size_t)a * mb * mb;
    int e_self = -1;
    for (int e = nptr[a]; e < nptr[a + 1]; ++e)
        if (ncol[e] == a) e_self = e;
    for (int t = threadIdx.x; t < mb * mb; t += blockDim.x) {
        const int i = t / mb, j = t % mb;
        double v = (i == j) ? 1.0 : 0.0;   // identity on the padding
        if (i < na && j < na) v = e_self >= 0 ? D[noff[e_self] + (size_t)i * W + j] : 0.0;
        B[t] = v;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < na; i += blockDim.x)
        for (int c = rowptr[b0 + i]; c < rowptr[b0 + i + 1]; ++c) {
            const int j = colidx[c] - b0;
            if (j >= 0 && j < na) B[(size_t)i * mb + j] += val[c];
        }
}

// in-place inverse of every leaf's SPD block (mb x mb, symmetric) in shared
// memory: right-looking Cholesky A = L L^T, Li = L^-1 column by column, then
// A^-1 = Li^T Li; err set when a pivot is not positive.  Also writes the FP32 copy.
__global__ void __launch_bounds__(256) k_blk_inv(int mb, double *__restrict__ blk, float *__restrict__ blk32,
                                                 int *err)
{
    extern __shared__ double sm[];
    double *A = sm;                       // mb x mb: L in the lower triangle
    double *Li = sm + (size_t)mb * mb;    // mb x mb
    __shared__ int bad;
    double *g = blk + (size_t)blockIdx.x * mb * mb;
    for (int t = threadIdx.x; t < mb * mb; t += blockDim.x) {
        A[t] = g[t];
        Li[t] = 0.0;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < mb; ++j) {
        if (threadIdx.x == 0) {
            const double d = A[j * mb + j];
            if (!(d > 0.0)) bad = 1;
            A[j * mb + j] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        const double ljj = A[j * mb + j];
        for (int i = j + 1 + threadIdx.x; i < mb; i += blockDim.x) A[i * mb + j] /= ljj;
        __syncthreads();
        // trailing update of the lower triangle: A[i][k] -= L[i][j] L[k][j], j < k <= i
        const int n = mb - j - 1;
        for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
            const int i = j + 1 + t / n, k = j + 1 + t % n;
            if (k <= i) A[i * mb + k] -= A[i * mb + j] * A[k * mb + j];
        }
        __syncthreads();
    }
    // Li = L^-1: thread per column c, forward substitution
    for (int c = threadIdx.x; c < mb; c += blockDim.x) {
        Li[c * mb + c] = 1.0 / A[c * mb + c];
        for (int i = c + 1; i < mb; ++i) {
            double v = 0.0;
            for (int k = c; k < i; ++k) v -= A[i * mb + k] * Li[k * mb + c];
            Li[i * mb + c] = v / A[i * mb + i];
        }
    }
    __syncthreads();
    // A^-1[i][j] = sum_{k >= max(i,j)} Li[k][i] Li[k][j]
    for (int t = threadIdx.x; t < mb * mb; t += blockDim.x) {
        const int i = t / mb, j = t % mb;
        double v = 0.0;
        for (int k = max(i, j); k < mb; ++k) v += Li[k * mb + i] * Li[k * mb + j];
        g[t] = v;
        blk32[(size_t)blockIdx.x * mb * mb + t] = (float)v;
    }
    if (threadIdx.x == 0 && bad) atomicOr(err, 1);
}

// A_c = R A R^T from the operator's parts directly (no applies): the sum of
// every near block's entries, the B + M entries, and for every admissible
// block (sigma, tau) the sums u_A^T S u_B over the coarse units A, B under
// sigma and tau, u_A = sum_{i in A} Ul^(l)[i] (l the block's level).
// Sum of the entries of near block e (rows of its row leaf, columns of its
// column leaf) in the row panel
__global__ void k_near_blocksum(int fl, const int *__restrict__ prow, const int *__restrict__ ncol,
                                const int *__restrict__ kb, const int *__restrict__ ke,
                                const int64_t *__restrict__ noff, const int *__restrict__ pw,
                                const double *__restrict__ D, double *__restrict__ out)
{
    __shared__ double sh[256];
    const int e = blockIdx.x, a = prow[e], b = ncol[e];
    const int na = ke[fl + a] - kb[fl + a], nb = ke[fl + b] - kb[fl + b], W = pw[a];
    double v = 0.0;
    for (int t = threadIdx.x; t < na * nb; t += blockDim.x) v += D[noff[e] + (size_t)(t / nb) * W + t % nb];
    sh[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)blockDim.x; ++q) s += sh[q];
        out[e] = s;
    }
}

// unit moments u[l][unit][alpha] = sum over the unit's rows of Ul^(l)[i][alpha],
// the units of level l being the nodes of level max(l, lc); CTA per (unit, level)
__global__ void k_unit_moments(int k, int N, int lmin, int lc, int nu_max, const int *__restrict__ kb,
                               const int *__restrict__ ke, const double *__restrict__ Ul, double *__restrict__ u)
{
    const int lv = blockIdx.y, l = lmin + lv, lu = max(l, lc);
    const int unit = blockIdx.x;
    if (unit >= (1 << lu)) return;
    const int node = (1 << lu) - 1 + unit;
    const double *U = Ul + (size_t)lv * N * k;
    for (int a = threadIdx.x; a < k; a += blockDim.x) {
        double s = 0.0;
        for (int i = kb[node]; i < ke[node]; ++i) s += U[(size_t)i * k + a];
        u[((size_t)lv * nu_max + unit) * k + a] = s;
    }
}

// per admissible block e (row node sigma, column tau, level l) and unit pair
// (A under sigma, B under tau): u_A^T S_e u_B; the pairs of block e start at
// off[e] (nA x nA of them, A-major).  CTA per block: t_B = S_e u_B for a chunk
// of units B in shared memory (threads over the rows of S_e), then a thread
// per pair (A, B) of the chunk
constexpr int UP_CHUNK = 16;
__global__ void __launch_bounds__(128) k_far_unitpairs(int k, int lmin, int lc, int nu_max, int nnode, int nfar,
                                                       const int *__restrict__ fptr, const int *__restrict__ fcol,
                                                       const long long *__restrict__ off,
                                                       const double *__restrict__ S, const double *__restrict__ u,
                                                       double *__restrict__ out)
{
    __shared__ double tB[UP_CHUNK][KMAX];
    const int e = blockIdx.x;
    if (e >= nfar) return;
    int lo = 0, hi = nnode;   // row node of block e
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (fptr[mid] <= e) lo = mid; else hi = mid;
    }
    const int sg = lo, tau = fcol[e];
    int l = 0;
    while ((2 << l) - 1 <= sg) ++l;
    const int lu = max(l, lc), sh = lu - l, nA = 1 << sh;
    const int ua0 = ((sg + 1) << sh) - (1 << lu), ub0 = ((tau + 1) << sh) - (1 << lu);
    const double *Se = S + (size_t)e * k * k;   // stored [b][a]: S(a, b) = Se[b * k + a]
    const double *ul = u + (size_t)(l - lmin) * nu_max * k;
    for (int B0 = 0; B0 < nA; B0 += UP_CHUNK) {
        const int nb = min(UP_CHUNK, nA - B0);
        __syncthreads();
        for (int t = threadIdx.x; t < nb * k; t += blockDim.x) {
            const int jb = t / k, a = t % k;
            const double *uB = ul + (size_t)(ub0 + B0 + jb) * k;
            double w = 0.0;
            for (int b = 0; b < k; ++b) w = fma(Se[(size_t)b * k + a], uB[b], w);
            tB[jb][a] = w;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nA * nb; t += blockDim.x) {
            const int iA = t / nb, jb = t % nb;
            const double *uA = ul + (size_t)(ua0 + iA) * k;
            double v = 0.0;
            for (int a = 0; a < k; ++a) v = fma(uA[a], tB[jb][a], v);
            out[off[e] + (size_t)iA * nA + B0 + jb] = v;
        }
    }
}

// local solves z_a = Binv_a r_a and the leaf sums rl[a] = sum_{i in a} r_i
__global__ void __launch_bounds__(128) k_prec_local(int fl, int mb, const int *__restrict__ kb,
                                                    const int *__restrict__ ke, const double *__restrict__ Binv,
                                                    const double *__restrict__ r, double *__restrict__ z,
                                                    double *__restrict__ rl, const int *skip)
{
    extern __shared__ double rs[];
    __shared__ double red[128];
    if (skip && *skip) return;
    const int a = blockIdx.x, b0 = kb[fl + a], na = ke[fl + a] - b0;
    double acc = 0.0;
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
        rs[i] = r[b0 + i];
        acc += rs[i];
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)blockDim.x; ++q) s += red[q];
        rl[a] = s;
    }
    // Binv_a is symmetric: row i is read as column i, so a warp's loads of
    // one j are contiguous
    const double *B = Binv + (size_t)a * mb * mb;
    for (int i = threadIdx.x; i < na; i += blockDim.x) {
        double v = 0.0;
        for (int j = 0; j < na; ++j) v = fma(B[(size_t)j * mb + i], rs[j], v);
        z[b0 + i] = v;
    }
}

// zc = Cinv rc (warp per row), rc[c] = sum of the leaf sums of cluster c
// (span consecutive leaves), formed per block in shared memory
__global__ void k_prec_coarse(int nc, int span, const double *__restrict__ Cinv, const double *__restrict__ rl,
                              double *__restrict__ zc, const int *skip)
{
    extern __shared__ double rc[];
    if (skip && *skip) return;
    for (int c = threadIdx.x; c < nc; c += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < span; ++q) s += rl[(size_t)c * span + q];
        rc[c] = s;
    }
    __syncthreads();
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= nc) return;
    double v = 0.0;
    for (int b = lane; b < nc; b += 32) v = fma(Cinv[(size_t)row * nc + b], rc[b], v);
    v = warp_sum(v);
    if (lane == 0) zc[row] = v;
}

__global__ void k_prec_add(int N, const int *__restrict__ cidx, const double *__restrict__ zc, double *__restrict__ z,
                           const int *skip)
{
    if (skip && *skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) z[i] += zc[cidx[i]];
}

// in-place inverse of an SPD n x n matrix (row stride ld) by Cholesky:
// A = L L^T (row dot products, sequential), then the columns of A^-1 by a
// forward and a backward substitution each, split over host threads; false if
// a pivot is not positive
bool spd_inverse(double *A, int n, int ld)
{
    std::vector<double> L((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        const double *Li = &L[(size_t)i * n];
        for (int j = 0; j <= i; ++j) {
            const double *Lj = &L[(size_t)j * n];
            double v = A[(size_t)i * ld + j];
            for (int k = 0; k < j; ++k) v -= Li[k] * Lj[k];
            if (j == i) {
                if (!(v > 0.0)) return false;
                L[(size_t)i * n + i] = std::sqrt(v);
            } else {
                L[(size_t)i * n + j] = v / Lj[j];
            }
        }
    }
    std::vector<double> Lt((size_t)n * n);   // L^T row-major: the backward solve reads rows
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) Lt[(size_t)j * n + i] = L[(size_t)i * n + j];
    auto solve_cols = [&](int c0, int c1) {
        std::vector<double> y(n);
        for (int c = c0; c < c1; ++c) {
            for (int i = 0; i < n; ++i) {   // L y = e_c
                double v = i == c ? 1.0 : 0.0;
                const double *Li = &L[(size_t)i * n];
                for (int k = c; k < i; ++k) v -= Li[k] * y[k];
                y[i] = i < c ? 0.0 : v / Li[i];
            }
            for (int i = n - 1; i >= 0; --i) {   // L^T x = y, x overwrites y
                double v = y[i];
                const double *Ui = &Lt[(size_t)i * n];
                for (int k = i + 1; k < n; ++k) v -= Ui[k] * y[k];
                y[i] = v / Ui[i];
            }
            for (int i = 0; i < n; ++i) A[(size_t)i * ld + c] = y[i];
        }
    };
    const int nth = n >= 128 ? (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency())) : 1;
    if (nth == 1) {
        solve_cols(0, n);
    } else {
        std::vector<std::thread> th;
        for (int t = 0; t < nth; ++t)
            th.emplace_back(solve_cols, (int)((int64_t)n * t / nth), (int)((int64_t)n * (t + 1) / nth));
        for (auto &t : th) t.join();
    }
    for (int i = 0; i < n; ++i)   // symmetrise the rounding
        for (int j = 0; j < i; ++j) {
            const double v = 0.5 * (A[(size_t)i * ld + j] + A[(size_t)j * ld + i]);
            A[(size_t)i * ld + j] = A[(size_t)j * ld + i] = v;
        }
    return true;
}

}  // namespace

void precond_setup(const MeshData &m, OpData &op, int kind, cudaStream_t st)
{
    release_graphs(op);
    op.prec_kind = 0;
    if (kind == 0) return;
    VFD_REQUIRE(kind == 1 || kind == 2, VFD_EINVAL, "unknown preconditioner kind");
    const int nleaf = m.kt.nleaf, fl = m.kt.first_leaf(), N = m.N, L = m.kt.L;
    const int mb = m.max_leaf_size;
    // leaf diagonal blocks, inverted on the device (large leaves on the host)
    op.prec_blk.alloc((size_t)nleaf * mb * mb);
    op.prec_blk32.alloc((size_t)nleaf * mb * mb);
    k_diag_blocks<<<nleaf, 128, 0, st>>>(fl, mb, m.kt_begin.p, m.kt_end.p, m.near_ptr.p, m.near_col.p, m.near_off.p,
                                         m.panel_w.p, op.D64.p, m.rowptr.p, m.colidx.p, op.valBM.p, op.prec_blk.p);
    VFD_CUDA(cudaGetLastError());
    if (mb <= PREC_SMEM_BLK) {
        const size_t shm = 2 * (size_t)mb * mb * sizeof(double);
        VFD_CUDA(cudaFuncSetAttribute(k_blk_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        DBuf<int> err;
        err.alloc(1);
        err.zero(st);
        k_blk_inv<<<nleaf, 256, shm, st>>>(mb, op.prec_blk.p, op.prec_blk32.p, err.p);
        VFD_CUDA(cudaGetLastError());
        int herr = 0;
        VFD_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaStreamSynchronize(st));
        VFD_REQUIRE(herr == 0, VFD_EINVAL, "a leaf diagonal block is not positive definite");
    } else {
        std::vector<double> blk((size_t)nleaf * mb * mb);
        VFD_CUDA(cudaMemcpyAsync(blk.data(), op.prec_blk.p, blk.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaStreamSynchronize(st));
        for (int a = 0; a < nleaf; ++a)
            VFD_REQUIRE(spd_inverse(&blk[(size_t)a * mb * mb], mb, mb), VFD_EINVAL,
                        "a leaf diagonal block is not positive definite");
        std::vector<float> b32(blk.begin(), blk.end());
        VFD_CUDA(cudaMemcpyAsync(op.prec_blk.p, blk.data(), blk.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        VFD_CUDA(cudaMemcpyAsync(op.prec_blk32.p, b32.data(), b32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
        VFD_CUDA(cudaStreamSynchronize(st));
    }
    op.prec_mb = mb;
    op.prec_nc = 0;
    if (kind == 1) {
        // coarse level: the deepest with at most PREC_MAX_COARSE clusters
        int lc = L;
        while (lc > 0 && (1 << lc) > PREC_MAX_COARSE) --lc;
        const int nc = 1 << lc, span = 1 << (L - lc);
        std::vector<int> cidx(N), cb(nc + 1);
        for (int c = 0; c <= nc; ++c) cb[c] = c < nc ? m.kt.begin[fl + c * span] : N;
        for (int c = 0; c < nc; ++c)
            for (int i = cb[c]; i < cb[c + 1]; ++i) cidx[i] = c;
        op.prec_cidx.upload(cidx);
        // coarse matrix A_c = R A R^T from the operator's parts
        std::vector<double> ac((size_t)nc * nc, 0.0);
        auto clu_of_leaf = [&](int leaf) { return leaf / span; };
        {   // near blocks
            DBuf<double> bs;
            bs.alloc(std::max(m.nnear, 1));
            if (m.nnear > 0)
                k_near_blocksum<<<m.nnear, 256, 0, st>>>(fl, m.near_pair_row.p, m.near_col.p, m.kt_begin.p,
                                                          m.kt_end.p, m.near_off.p, m.panel_w.p, op.D64.p, bs.p);
            VFD_CUDA(cudaGetLastError());
            std::vector<double> hb(m.nnear);
            VFD_CUDA(cudaMemcpyAsync(hb.data(), bs.p, sizeof(double) * m.nnear, cudaMemcpyDeviceToHost, st));
            VFD_CUDA(cudaStreamSynchronize(st));
            for (int a = 0; a < nleaf; ++a)
                for (int e = m.near_ptr_h[a]; e < m.near_ptr_h[a + 1]; ++e)
                    ac[(size_t)clu_of_leaf(a) * nc + clu_of_leaf(m.near_col_h[e])] += hb[e];
        }
        {   // B + M
            std::vector<int> rp(N + 1), ci(m.nnz);
            std::vector<double> v(m.nnz);
            VFD_CUDA(cudaMemcpyAsync(rp.data(), m.rowptr.p, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost, st));
            VFD_CUDA(cudaMemcpyAsync(ci.data(), m.colidx.p, sizeof(int) * m.nnz, cudaMemcpyDeviceToHost, st));
            VFD_CUDA(cudaMemcpyAsync(v.data(), op.valBM.p, sizeof(double) * m.nnz, cudaMemcpyDeviceToHost, st));
            VFD_CUDA(cudaStreamSynchronize(st));
            for (int i = 0; i < N; ++i)
                for (int e = rp[i]; e < rp[i + 1]; ++e) ac[(size_t)cidx[i] * nc + cidx[ci[e]]] += v[e];
        }
        if (m.nfar > 0) {   // admissible blocks
            const int k = m.k, lmin = m.far_lmin, nlev = L - lmin + 1;
            const int nu_max = 1 << std::max(L, lc);
            DBuf<double> u;
            u.alloc((size_t)nlev * nu_max * k);
            dim3 gu(nu_max, nlev);
            k_unit_moments<<<gu, 64, 0, st>>>(k, N, lmin, lc, nu_max, m.kt_begin.p, m.kt_end.p, m.Ul64.p, u.p);
            std::vector<long long> off(m.nfar + 1, 0);
            std::vector<int> erow(m.nfar);
            for (int n = 0; n < m.kt.nnode; ++n)
                for (int e = m.far_ptr_h[n]; e < m.far_ptr_h[n + 1]; ++e) erow[e] = n;
            for (int e = 0; e < m.nfar; ++e) {
                int l = 0;
                while ((2 << l) - 1 <= erow[e]) ++l;
                const long long nA = 1LL << (std::max(l, lc) - l);
                off[e + 1] = off[e] + nA * nA;
            }
            DBuf<long long> offd;
            offd.upload(off);
            DBuf<double> pv;
            pv.alloc(off[m.nfar]);
            k_far_unitpairs<<<m.nfar, 128, 0, st>>>(k, lmin, lc, nu_max, m.kt.nnode, m.nfar, m.far_ptr.p,
                                                     m.far_col.p, offd.p, op.S64.p, u.p, pv.p);
            VFD_CUDA(cudaGetLastError());
            std::vector<double> hv(off[m.nfar]);
            VFD_CUDA(cudaMemcpyAsync(hv.data(), pv.p, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, st));
            VFD_CUDA(cudaStreamSynchronize(st));
            for (int e = 0; e < m.nfar; ++e) {
                const int sg = erow[e], tau = m.far_col_h[e];
                int l = 0;
                while ((2 << l) - 1 <= sg) ++l;
                const int lu = std::max(l, lc), sh = lu - l, nA = 1 << sh;
                const int ua0 = ((sg + 1) << sh) - (1 << lu), ub0 = ((tau + 1) << sh) - (1 << lu);
                for (int t = 0; t < nA * nA; ++t) {
                    const int A = (ua0 + t / nA) >> (lu - lc), B = (ub0 + t % nA) >> (lu - lc);
                    ac[(size_t)A * nc + B] += hv[off[e] + t];
                }
            }
        }
        for (int a = 0; a < nc; ++a)   // symmetrise the rounding
            for (int b = 0; b < a; ++b) {
                const double v = 0.5 * (ac[(size_t)a * nc + b] + ac[(size_t)b * nc + a]);
                ac[(size_t)a * nc + b] = ac[(size_t)b * nc + a] = v;
            }
        VFD_REQUIRE(spd_inverse(ac.data(), nc, nc), VFD_EINVAL, "the coarse matrix is not positive definite");
        op.prec_coarse.upload(ac);
        op.prec_coarse32.upload(std::vector<float>(ac.begin(), ac.end()));
        op.prec_nc = nc;
        op.prec_span = span;
        op.prec_zc.alloc(nc);
    }
    op.prec_rl.alloc(nleaf);
    VFD_CUDA(cudaStreamSynchronize(st));
    op.prec_kind = kind;
    ++op.prec_version;
}

void precond_apply(const MeshData &m, const OpData &op, const double *r, double *z, cudaStream_t st, const int *skip)
{
    const int nleaf = m.kt.nleaf, mb = op.prec_mb;
    k_prec_local<<<nleaf, 128, (size_t)mb * sizeof(double), st>>>(m.kt.first_leaf(), mb, m.kt_begin.p, m.kt_end.p,
                                                                 op.prec_blk.p, r, z, op.prec_rl.p, skip);
    if (op.prec_nc > 0) {
        k_prec_coarse<<<cdiv((long long)op.prec_nc * 32, 256), 256, (size_t)op.prec_nc * sizeof(double), st>>>(
            op.prec_nc, op.prec_span, op.prec_coarse.p, op.prec_rl.p, op.prec_zc.p, skip);
        k_prec_add<<<cdiv(m.N, 256), 256, 0, st>>>(m.N, op.prec_cidx.p, op.prec_zc.p, z, skip);
    }
    VFD_CUDA(cudaGetLastError());
}

}  // namespace vfd
