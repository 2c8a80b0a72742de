// Two-level preconditioner for the CG solve of A U = F (Sec. 7 solves with
// plain CG; a multilevel preconditioner is the paper's stated next step,
// Sec. 8):
//
//   M^-1 r = sum_leaves P_a^T A_aa^-1 P_a r  +  R^T A_c^-1 R r,
//
// an additive combination of exact solves with the diagonal block A_aa of
// every leaf of the cluster tree (its DoFs, A's rows and columns of that
// leaf: near panel block (a, a) plus the B + M entries inside the leaf) and a
// coarse solve on the space of leaf-wise constant functions (R the leaf
// indicator restriction, A_c = R A R^T, one row and column per leaf).  Both
// factors are symmetric positive definite, so M is too and CG applies.
//
// Setup (once per operator, vfd_precondition): the diagonal blocks are
// gathered on the device and inverted on the host (Cholesky, FP64); A_c is
// formed on the device by applying A to the leaf indicator vectors and
// summing rows per leaf, and inverted on the host.  Apply (every PCG
// iteration): one kernel per leaf for the local solves and the restriction,
// one for the coarse product, one for the prolongation.
#include <cmath>
#include <vector>

#include "device_common.cuh"

namespace vfd {

void apply_parts_ex(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                    bool lowp, cudaStream_t st, const int *skip);

namespace {

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

// leaf indicator columns: X[c][i] = 1 if DoF i lies in leaf c0 + c
__global__ void k_indicators(int N, int ncol, int c0, const int *__restrict__ vleaf, double *__restrict__ X)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * ncol) return;
    const int c = (int)(t / N), i = (int)(t % N);
    X[t] = vleaf[i] == c0 + c ? 1.0 : 0.0;
}

// Ac[a][c0 + c] = sum over the DoFs of leaf a of Y[c][i]
__global__ void k_leaf_sums(int N, int nleaf, int ncol, int c0, int fl, const int *__restrict__ kb,
                            const int *__restrict__ ke, const double *__restrict__ Y, double *__restrict__ Ac)
{
    const int a = blockIdx.x, c = blockIdx.y;
    __shared__ double sh[128];
    double v = 0.0;
    for (int i = kb[fl + a] + threadIdx.x; i < ke[fl + a]; i += blockDim.x) v += Y[(size_t)c * N + i];
    sh[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)blockDim.x; ++q) s += sh[q];
        Ac[(size_t)a * nleaf + c0 + c] = s;
    }
}

// local solves z_a = Binv_a r_a and the restriction rc[a] = sum_{i in a} r_i
__global__ void __launch_bounds__(128) k_prec_local(int fl, int mb, const int *__restrict__ kb,
                                                    const int *__restrict__ ke, const double *__restrict__ Binv,
                                                    const double *__restrict__ r, double *__restrict__ z,
                                                    double *__restrict__ rc, const int *skip)
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
        rc[a] = s;
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

// zc = Cinv rc (warp per row)
__global__ void k_prec_coarse(int nleaf, const double *__restrict__ Cinv, const double *__restrict__ rc,
                              double *__restrict__ zc, const int *skip)
{
    if (skip && *skip) return;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= nleaf) return;
    double v = 0.0;
    for (int b = lane; b < nleaf; b += 32) v = fma(Cinv[(size_t)row * nleaf + b], rc[b], v);
    v = warp_sum(v);
    if (lane == 0) zc[row] = v;
}

__global__ void k_prec_add(int N, const int *__restrict__ vleaf, const double *__restrict__ zc, double *__restrict__ z,
                           const int *skip)
{
    if (skip && *skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) z[i] += zc[vleaf[i]];
}

// in-place inverse of an SPD n x n matrix (row stride ld) by Cholesky:
// A = L L^T, A^-1 = L^-T L^-1; false if a pivot is not positive
bool spd_inverse(double *A, int n, int ld)
{
    std::vector<double> L((size_t)n * n, 0.0), Li((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * ld + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0)) return false;
        const double ljj = std::sqrt(d);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double v = A[(size_t)i * ld + j];
            for (int k = 0; k < j; ++k) v -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = v / ljj;
        }
    }
    // Li = L^-1 (lower triangular), column by column
    for (int c = 0; c < n; ++c) {
        Li[(size_t)c * n + c] = 1.0 / L[(size_t)c * n + c];
        for (int i = c + 1; i < n; ++i) {
            double v = 0.0;
            for (int k = c; k < i; ++k) v -= L[(size_t)i * n + k] * Li[(size_t)k * n + c];
            Li[(size_t)i * n + c] = v / L[(size_t)i * n + i];
        }
    }
    // A^-1 = Li^T Li
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = 0.0;
            for (int k = i; k < n; ++k) v += Li[(size_t)k * n + i] * Li[(size_t)k * n + j];
            A[(size_t)i * ld + j] = v;
            A[(size_t)j * ld + i] = v;
        }
    return true;
}

}  // namespace

void precond_setup(const MeshData &m, OpData &op, int kind, cudaStream_t st)
{
    release_graphs(op);
    op.prec_kind = 0;
    if (kind == 0) return;
    VFD_REQUIRE(kind == 1, VFD_EINVAL, "unknown preconditioner kind");
    VFD_REQUIRE(op.precision == VFD_FP64, VFD_EUNSUPPORTED, "the preconditioner is built for VFD_FP64 operators");
    const int nleaf = m.kt.nleaf, fl = m.kt.first_leaf(), N = m.N;
    VFD_REQUIRE(nleaf <= 2048, VFD_EUNSUPPORTED, "too many leaves for the dense coarse solve (at most 2048)");
    const int mb = m.max_leaf_size;
    // leaf diagonal blocks, inverted on the host
    op.prec_blk.alloc((size_t)nleaf * mb * mb);
    k_diag_blocks<<<nleaf, 128, 0, st>>>(fl, mb, m.kt_begin.p, m.kt_end.p, m.near_ptr.p, m.near_col.p, m.near_off.p,
                                         m.panel_w.p, op.D64.p, m.rowptr.p, m.colidx.p, op.valBM.p, op.prec_blk.p);
    VFD_CUDA(cudaGetLastError());
    std::vector<double> blk((size_t)nleaf * mb * mb);
    VFD_CUDA(cudaMemcpyAsync(blk.data(), op.prec_blk.p, blk.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    VFD_CUDA(cudaStreamSynchronize(st));
    for (int a = 0; a < nleaf; ++a)
        VFD_REQUIRE(spd_inverse(&blk[(size_t)a * mb * mb], mb, mb), VFD_EINVAL,
                    "a leaf diagonal block is not positive definite");
    VFD_CUDA(cudaMemcpyAsync(op.prec_blk.p, blk.data(), blk.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    // coarse matrix A_c = R A R^T by applying A to the leaf indicators (in column chunks)
    DBuf<double> X, Y, Ac;
    const int chunk = std::max(1, std::min(nleaf, (int)(((size_t)1 << 27) / std::max(N, 1))));
    X.alloc((size_t)N * chunk);
    Y.alloc((size_t)N * chunk);
    Ac.alloc((size_t)nleaf * nleaf);
    for (int c0 = 0; c0 < nleaf; c0 += chunk) {
        const int nc = std::min(chunk, nleaf - c0);
        k_indicators<<<cdiv((long long)N * nc, 256), 256, 0, st>>>(N, nc, c0, m.vleaf.p, X.p);
        apply_parts_ex(m, op, VFD_PART_ALL, X.p, Y.p, nc, N, false, st, nullptr);
        dim3 g(nleaf, nc);
        k_leaf_sums<<<g, 128, 0, st>>>(N, nleaf, nc, c0, fl, m.kt_begin.p, m.kt_end.p, Y.p, Ac.p);
        VFD_CUDA(cudaGetLastError());
    }
    std::vector<double> ac((size_t)nleaf * nleaf);
    VFD_CUDA(cudaMemcpyAsync(ac.data(), Ac.p, ac.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    VFD_CUDA(cudaStreamSynchronize(st));
    for (int a = 0; a < nleaf; ++a)   // symmetrise the rounding
        for (int b = 0; b < a; ++b) {
            const double v = 0.5 * (ac[(size_t)a * nleaf + b] + ac[(size_t)b * nleaf + a]);
            ac[(size_t)a * nleaf + b] = ac[(size_t)b * nleaf + a] = v;
        }
    VFD_REQUIRE(spd_inverse(ac.data(), nleaf, nleaf), VFD_EINVAL, "the coarse matrix is not positive definite");
    op.prec_coarse.upload(ac);
    op.prec_rc.alloc(nleaf);
    op.prec_zc.alloc(nleaf);
    VFD_CUDA(cudaStreamSynchronize(st));
    op.prec_kind = kind;
}

void precond_apply(const MeshData &m, const OpData &op, const double *r, double *z, cudaStream_t st, const int *skip)
{
    const int nleaf = m.kt.nleaf, mb = m.max_leaf_size;
    k_prec_local<<<nleaf, 128, (size_t)mb * sizeof(double), st>>>(m.kt.first_leaf(), mb, m.kt_begin.p, m.kt_end.p,
                                                                 op.prec_blk.p, r, z, op.prec_rc.p, skip);
    k_prec_coarse<<<cdiv((long long)nleaf * 32, 256), 256, 0, st>>>(nleaf, op.prec_coarse.p, op.prec_rc.p,
                                                                    op.prec_zc.p, skip);
    k_prec_add<<<cdiv(m.N, 256), 256, 0, st>>>(m.N, m.vleaf.p, op.prec_zc.p, z, skip);
    VFD_CUDA(cudaGetLastError());
}

}  // namespace vfd
