// Operator apply Y = A X = (B + M) X + K_near X + K_far X (Sec. 3, eq. e:decomp):
//   K_far by the H^2 product (Sec. 5.3, eq. eq:triple_product_factored with
//   nested bases): leaf upsweep xhat = U^T x, transfer upsweep, coupling
//   yhat = S xhat over the admissible list, transfer downsweep, leaf
//   expansion U yhat;  K_near by the dense inadmissible leaf blocks;  B + M by
//   CSR.  The last kernel fuses the leaf expansion, the near blocks and the
//   CSR rows, writing each output row once.
// Tree order is the DoF order, so every leaf's x and y are contiguous.
#include "device_common.cuh"

namespace vfd {

// xhat[r][leaf][a] = sum_i U[i][a] x[i]    (thread per (leaf, a))
template <class T, class A>
__global__ void k_up_leaf(int k, int nleaf, int fl, const int *__restrict__ kb, const int *__restrict__ ke,
                          const int *__restrict__ Uoff, const T *__restrict__ U, const double *__restrict__ X,
                          int64_t ld, A *__restrict__ xhat, int64_t hstride, const int *skip)
{
    if (skip && *skip) return;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nleaf * k) return;
    int lf = t / k, al = t - lf * k, r = blockIdx.y;
    int b = kb[fl + lf], e = ke[fl + lf];
    const T *u = U + Uoff[lf] + al;
    const double *x = X + (size_t)r * ld;
    A acc = 0;
    for (int i = b; i < e; ++i) acc += (A)u[(size_t)(i - b) * k] * (A)x[i];
    xhat[(size_t)r * hstride + (size_t)(fl + lf) * k + al] = acc;
}

// xhat[parent][a] = sum_children sum_b E_c[b][a] xhat[c][b]  (level l)
template <class T, class A>
__global__ void k_up_level(int k, int first, int count, const T *__restrict__ E, A *__restrict__ xhat,
                           int64_t hstride, const int *skip)
{
    if (skip && *skip) return;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * k) return;
    int n = first + t / k, al = t % k;
    A *xh = xhat + (size_t)blockIdx.y * hstride;
    A acc = 0;
    for (int c = 2 * n + 1; c <= 2 * n + 2; ++c) {
        const T *Ec = E + (size_t)c * k * k + al;
        const A *xc = xh + (size_t)c * k;
        for (int be = 0; be < k; ++be) acc += (A)Ec[(size_t)be * k] * xc[be];
    }
    xh[(size_t)n * k + al] = acc;
}

// yhat[n][a] = sum_{blocks e of row n} sum_b S_e[a][b] xhat[col e][b]; S stored [b][a]
template <class T, class A>
__global__ void k_couple(int k, int nnode, const int *__restrict__ fptr, const int *__restrict__ fcol,
                         const T *__restrict__ S, const A *__restrict__ xhat, A *__restrict__ yhat, int64_t hstride,
                         const int *skip)
{
    if (skip && *skip) return;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnode * k) return;
    int n = t / k, al = t % k;
    const A *xh = xhat + (size_t)blockIdx.y * hstride;
    A acc = 0;
    for (int e = fptr[n]; e < fptr[n + 1]; ++e) {
        const T *s = S + (size_t)e * k * k + al;
        const A *xc = xh + (size_t)fcol[e] * k;
        for (int be = 0; be < k; ++be) acc += (A)s[(size_t)be * k] * xc[be];
    }
    yhat[(size_t)blockIdx.y * hstride + (size_t)n * k + al] = acc;
}

// yhat[c][b] += sum_a E_c[b][a] yhat[parent][a]  (level l, parents already final)
template <class T, class A>
__global__ void k_down_level(int k, int first, int count, const T *__restrict__ E, A *__restrict__ yhat,
                             int64_t hstride, const int *skip)
{
    if (skip && *skip) return;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * k) return;
    int c = first + t / k, be = t % k;
    A *yh = yhat + (size_t)blockIdx.y * hstride;
    const T *Ec = E + ((size_t)c * k + be) * k;
    const A *yp = yh + (size_t)((c - 1) / 2) * k;
    A acc = 0;
    for (int al = 0; al < k; ++al) acc += (A)Ec[al] * yp[al];
    yh[(size_t)c * k + be] += acc;
}

// Y[i] = [U yhat]_i + sum_near D x + sum_csr val x ; block per leaf, warp per row
template <class T, class A>
__global__ void __launch_bounds__(256)
k_leaf_out(int k, int fl, const int *__restrict__ kb, const int *__restrict__ ke, const int *__restrict__ Uoff,
           const T *__restrict__ U, const A *__restrict__ yhat, int64_t hstride, int use_far,
           const int *__restrict__ nptr, const int *__restrict__ ncol, const int64_t *__restrict__ noff,
           const T *__restrict__ D, int use_near, const int *__restrict__ rowptr, const int *__restrict__ colidx,
           const double *__restrict__ val, const double *__restrict__ X, int64_t ld, double *__restrict__ Y,
           const int *skip)
{
    if (skip && *skip) return;
    const int lf = blockIdx.x, r = blockIdx.y;
    const int b = kb[fl + lf], e = ke[fl + lf];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const double *x = X + (size_t)r * ld;
    const A *yh = yhat + (size_t)r * hstride + (size_t)(fl + lf) * k;
    for (int i = b + warp; i < e; i += nw) {
        const int il = i - b;
        A kacc = 0;
        if (use_far) {
            const T *u = U + Uoff[lf] + (size_t)il * k;
            for (int al = lane; al < k; al += 32) kacc += (A)u[al] * yh[al];
        }
        if (use_near) {
            for (int ne = nptr[lf]; ne < nptr[lf + 1]; ++ne) {
                int c = ncol[ne];
                int cb = kb[fl + c], nb = ke[fl + c] - cb;
                const T *drow = D + noff[ne] + (size_t)il * nb;
                const double *xc = x + cb;
                for (int j = lane; j < nb; j += 32) kacc += (A)drow[j] * (A)xc[j];
            }
        }
        double acc = (double)kacc;
        if (val) {
            for (int c = rowptr[i] + lane; c < rowptr[i + 1]; c += 32) acc += val[c] * x[colidx[c]];
        }
        acc = warp_sum(acc);
        if (lane == 0) Y[(size_t)r * ld + i] = acc;
    }
}

template <class T, class A>
static void apply_impl(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                       const T *U, const T *E, const T *S, const T *D, A *xhat, A *yhat, cudaStream_t st,
                       const int *skip)
{
    const int k = m.k, fl = m.kt.first_leaf(), L = m.kt.L, nnode = m.kt.nnode;
    const int64_t hs = (int64_t)nnode * k;
    const bool far = (parts & VFD_PART_KFAR) && m.nfar > 0;
    const bool near = (parts & VFD_PART_KNEAR) && m.nnear > 0;
    const double *val = nullptr;
    if ((parts & VFD_PART_B) && (parts & VFD_PART_M)) val = op.valBM.p;
    else if (parts & VFD_PART_B) val = op.valB.p;
    else if (parts & VFD_PART_M) val = op.valM.p;
    const int TB = 128;
    if (far) {
        dim3 g(cdiv((long long)m.kt.nleaf * k, TB), nrhs);
        k_up_leaf<T, A><<<g, TB, 0, st>>>(k, m.kt.nleaf, fl, m.kt_begin.p, m.kt_end.p, m.kt_Uoff.p, U, X, ld, xhat, hs,
                                          skip);
        for (int l = L - 1; l >= 0; --l) {
            int first = (1 << l) - 1, count = 1 << l;
            dim3 gl(cdiv((long long)count * k, TB), nrhs);
            k_up_level<T, A><<<gl, TB, 0, st>>>(k, first, count, E, xhat, hs, skip);
        }
        dim3 gc(cdiv((long long)nnode * k, TB), nrhs);
        k_couple<T, A><<<gc, TB, 0, st>>>(k, nnode, m.far_ptr.p, m.far_col.p, S, xhat, yhat, hs, skip);
        for (int l = 1; l <= L; ++l) {
            int first = (1 << l) - 1, count = 1 << l;
            dim3 gl(cdiv((long long)count * k, TB), nrhs);
            k_down_level<T, A><<<gl, TB, 0, st>>>(k, first, count, E, yhat, hs, skip);
        }
    }
    dim3 go(m.kt.nleaf, nrhs);
    k_leaf_out<T, A><<<go, 256, 0, st>>>(k, fl, m.kt_begin.p, m.kt_end.p, m.kt_Uoff.p, U, yhat, hs, far ? 1 : 0,
                                         m.near_ptr.p, m.near_col.p, m.near_off.p, D, near ? 1 : 0, m.rowptr.p,
                                         m.colidx.p, val, X, ld, Y, skip);
    VFD_CUDA(cudaGetLastError());
}

// parts: VFD_PART_* mask; lowp: use the FP32 copies of K (VFD_FP32 operators)
void apply_parts_ex(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                    bool lowp, cudaStream_t st, const int *skip)
{
    const size_t need = (size_t)m.kt.nnode * m.k * nrhs;
    if (lowp) {
        if (op.xhat32.n < need) {
            op.xhat32.alloc(need);
            op.yhat32.alloc(need);
        }
        apply_impl<float, float>(m, op, parts, X, Y, nrhs, ld, op.U32.p, op.E32.p, op.S32.p, op.D32.p, op.xhat32.p,
                                 op.yhat32.p, st, skip);
    } else {
        if (op.xhat.n < need) {
            op.xhat.alloc(need);
            op.yhat.alloc(need);
        }
        apply_impl<double, double>(m, op, parts, X, Y, nrhs, ld, m.U64.p, m.E64.p, op.S64.p, op.D64.p, op.xhat.p,
                                   op.yhat.p, st, skip);
    }
}

void apply_parts(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                 cudaStream_t st)
{
    apply_parts_ex(m, op, parts, X, Y, nrhs, ld, op.precision == VFD_FP32, st, nullptr);
}

}  // namespace vfd
