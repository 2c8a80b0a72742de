// Operator apply Y = A X = (B + M) X + K_near X + K_far X (Sec. 3, eq. e:decomp).
//
// K_far is the H^2 product of Sec. 5.3 (eq. eq:triple_product_factored):
// y_sigma += U_sigma (sum_{sigma'} S_{sigma sigma'} U_{sigma'}^T x_sigma').  The
// bases of all levels are the nested ones (U E ... E); the apply uses them
// flattened per level (Ul^(l), precomputed at setup from U and the transfer
// matrices), which turns the level-by-level transfer chain into independent
// work:
//   1. k_far_proj:   per (leaf, level) the projection Ul^(l)_leaf^T x_leaf
//   2. k_far_sum:    per node, xhat = sum of its leaves' projections
//   3. k_far_couple: per admissible block e (a warp) S_e xhat[col e], then
//                    k_far_couple_sum: per node the sum over its blocks
//   4. k_near_csr:   per row, the near panel row and the B + M CSR row
//                    (concurrently with 1-3, which run on a high-priority
//                    side stream)
//   5. k_far_expand: after the join, Y[i] += sum_l Ul^(l)[i] . yhat[ancestor]
// Tree order is the DoF order, so every leaf's x and y are contiguous.
#include <algorithm>
#include <mutex>

#include "device_common.cuh"

namespace vfd {

template <class T>
struct Vec;
template <>
struct Vec<double> {
    using V = double2;
    static constexpr int W = 2;
};
template <>
struct Vec<float> {
    using V = float4;
    static constexpr int W = 4;
};

__device__ __forceinline__ void fma_v(const double2 a, const double2 x, double &s0, double &s1)
{
    s0 = fma(a.x, x.x, s0);
    s1 = fma(a.y, x.y, s1);
}
__device__ __forceinline__ void fma_v(const float4 a, const float4 x, float &s0, float &s1)
{
    s0 = fmaf(a.x, x.x, s0);
    s1 = fmaf(a.y, x.y, s1);
    s0 = fmaf(a.z, x.z, s0);
    s1 = fmaf(a.w, x.w, s1);
}

constexpr int FV_MAXLEV = 24;
struct FarView {
    int use;         // apply K_far
    int lmin, L, nlev, k, N;    // k: the node stride of xhat / yhat / the projections (largest rank)
    int kl[FV_MAXLEV];          // rank of each far level (k, or less after recompression)
    long long uo[FV_MAXLEV];    // offset of each level's flattened basis (row stride kl[lv])
    const long long *so;        // offset of each admissible block's coupling (kl x kl), or null: e k^2
    const int *bk;              // rank of each admissible block, or null: k
};

__device__ __forceinline__ int fv_level(int node)
{
    int l = 0;
    while ((2 << l) - 1 <= node) ++l;
    return l;
}

// ---------------------------------------------------------------------------
// 1. leaf-level projections  part[r][lv][leaf][a] = sum_{i in leaf} Ul^(lmin+lv)[i][a] x[i]
// ---------------------------------------------------------------------------
template <class T, class A>
__global__ void __launch_bounds__(128)
k_far_proj(FarView F, int fl, int nleaf, const int *__restrict__ kb, const int *__restrict__ ke,
           const T *__restrict__ Ul, const double *__restrict__ X, int64_t ld, A *__restrict__ part, const int *skip)
{
    __shared__ A red[128];
    if (skip && *skip) return;
    const int leaf = blockIdx.x, lv = blockIdx.y, r = blockIdx.z, k = F.kl[lv];
    const int b = kb[fl + leaf], e = ke[fl + leaf];
    const int kk = min(k, (int)blockDim.x);
    const int parts = blockDim.x / kk;
    const int al = threadIdx.x % kk, pt = threadIdx.x / kk;
    const T *u = Ul + F.uo[lv];
    const double *x = X + (size_t)r * ld;
    for (int a0 = 0; a0 < k; a0 += kk) {
        A acc = 0;
        if (pt < parts)
            for (int i = b + pt; i < e; i += parts) acc += (A)u[(size_t)i * k + a0 + al] * (A)x[i];
        red[threadIdx.x] = acc;
        __syncthreads();
        if (threadIdx.x < kk) {
            A s = 0;
            for (int q = 0; q < parts; ++q) s += red[q * kk + threadIdx.x];
            part[(((size_t)r * F.nlev + lv) * nleaf + leaf) * F.k + a0 + threadIdx.x] = s;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 2. node sums  xhat[r][node][a] = sum over the node's leaves of part  (levels
//    lmin..L); one CTA per node, threads (a, part) over the leaves, reduced
//    in shared memory
// ---------------------------------------------------------------------------
template <class A>
__global__ void __launch_bounds__(128)
k_far_sum(FarView F, int nleaf, const A *__restrict__ part, A *__restrict__ xhat, int64_t hs, const int *skip)
{
    __shared__ A red[128];
    if (skip && *skip) return;
    const int node = (1 << F.lmin) - 1 + blockIdx.x, r = blockIdx.y;
    const int l = fv_level(node);
    const int lv = l - F.lmin, span = 1 << (F.L - l), k = F.kl[lv], K = F.k;
    const int leaf0 = ((node + 1) << (F.L - l)) - 1 - ((1 << F.L) - 1);
    const int kk = min(k, (int)blockDim.x), parts = blockDim.x / kk;
    const int al = threadIdx.x % kk, pt = threadIdx.x / kk;
    const A *p = part + (((size_t)r * F.nlev + lv) * nleaf + leaf0) * K;
    for (int a0 = 0; a0 < k; a0 += kk) {
        A s = 0;
        if (pt < parts)
            for (int j = pt; j < span; j += parts) s += p[(size_t)j * K + a0 + al];
        red[threadIdx.x] = s;
        __syncthreads();
        if (threadIdx.x < kk) {
            A t = 0;
            for (int q = 0; q < parts; ++q) t += red[q * kk + threadIdx.x];
            xhat[(size_t)r * hs + (size_t)node * K + a0 + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// 3. coupling  yhat[node][a] = sum_{e in row node} sum_b S_e[b][a] xhat[col e][b]
//    (S stored [b][a]).  The partial of one block for one a (couple_part, the
//    same arithmetic in both kernels below) takes the even and the odd rows b
//    in two chains; the node sum adds the partials in list order from zero,
//    so both kernels give bit-identical yhat.
//    k_far_couple + k_far_couple_sum: a warp per admissible block (lanes over
//    a, a contiguous row of S_e per step) into ye[e][a], then per (node, a)
//    the sum over the node's blocks.  k_far_couple_node (the no-allocation
//    apply): a CTA per node, a warp per block of each pass of eight.
// ---------------------------------------------------------------------------
template <class T, class A>
__device__ __forceinline__ void couple_part(const T *__restrict__ sp, const A *__restrict__ xc, int k, int a1, int a2,
                                            A &r1, A &r2)
{
    // columns a1 and a2 (a2 may be >= k: unused) together, each in two chains
    A s1 = 0, t1 = 0, s2 = 0, t2 = 0;
    const bool two = a2 < k;
    int be = 0;
#pragma unroll 4
    for (; be + 1 < k; be += 2) {
        const A x0 = xc[be], x1 = xc[be + 1];
        s1 += (A)sp[(size_t)be * k + a1] * x0;
        t1 += (A)sp[(size_t)(be + 1) * k + a1] * x1;
        if (two) {
            s2 += (A)sp[(size_t)be * k + a2] * x0;
            t2 += (A)sp[(size_t)(be + 1) * k + a2] * x1;
        }
    }
    if (be < k) {
        s1 += (A)sp[(size_t)be * k + a1] * xc[be];
        if (two) s2 += (A)sp[(size_t)be * k + a2] * xc[be];
    }
    r1 = s1 + t1;
    r2 = s2 + t2;
}

template <class T, class A>
__global__ void __launch_bounds__(256)
k_far_couple(FarView F, int nfar, int nnode, const int *__restrict__ fptr, const int *__restrict__ fcol,
             const T *__restrict__ S, const A *__restrict__ xhat, A *__restrict__ ye, int64_t hs, const int *skip)
{
    if (skip && *skip) return;
    const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31, r = blockIdx.y;
    if (e >= nfar) return;
    const int k = F.bk ? F.bk[e] : F.k;
    const T *sp = S + (F.so ? (size_t)F.so[e] : (size_t)e * k * k);
    const A *xc = xhat + (size_t)r * hs + (size_t)fcol[e] * F.k;
    A *out = ye + ((size_t)r * nfar + e) * F.k;
    for (int a = lane; a < k; a += 64) {
        A r1, r2;
        couple_part(sp, xc, k, a, a + 32, r1, r2);
        out[a] = r1;
        if (a + 32 < k) out[a + 32] = r2;
    }
}

template <class A>
__global__ void k_far_couple_sum(FarView F, int nfar, int nnode, const int *__restrict__ fptr,
                                 const A *__restrict__ ye, A *__restrict__ yhat, int64_t hs, const int *skip)
{
    if (skip && *skip) return;
    const int k = F.k, r = blockIdx.y;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nnode * k) return;
    const int node = t / k, a = t % k;
    const int l = fv_level(node), kl = l >= F.lmin ? F.kl[l - F.lmin] : k;
    A s = 0;
    if (a < kl)
        for (int e = fptr[node]; e < fptr[node + 1]; ++e) s += ye[((size_t)r * nfar + e) * k + a];
    yhat[(size_t)r * hs + t] = s;
}

template <class T, class A>
__global__ void __launch_bounds__(256)
k_far_couple_node(FarView F, const int *__restrict__ fptr, const int *__restrict__ fcol, const T *__restrict__ S,
                  const A *__restrict__ xhat, A *__restrict__ yhat, int64_t hs, const int *skip)
{
    __shared__ A pt[8][KMAX];
    if (skip && *skip) return;
    const int node = blockIdx.x, r = blockIdx.y, K = F.k;
    const int l = fv_level(node), k = l >= F.lmin ? F.kl[l - F.lmin] : K;
    const int e0 = fptr[node], ne = fptr[node + 1] - e0;
    const A *xh = xhat + (size_t)r * hs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    A tot = 0;   // thread a < k: the node sum of column a
    for (int eb = 0; eb < ne; eb += 8) {
        const int e = eb + warp;
        if (e < ne) {
            const T *sp = S + (F.so ? (size_t)F.so[e0 + e] : (size_t)(e0 + e) * k * k);
            const A *xc = xh + (size_t)fcol[e0 + e] * K;
            for (int a = lane; a < k; a += 64) {
                A r1, r2;
                couple_part(sp, xc, k, a, a + 32, r1, r2);
                pt[warp][a] = r1;
                if (a + 32 < k) pt[warp][a + 32] = r2;
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < k)
            for (int w = 0; w < 8 && eb + w < ne; ++w) tot += pt[w][threadIdx.x];
        __syncthreads();
    }
    if ((int)threadIdx.x < K) yhat[(size_t)r * hs + (size_t)node * K + threadIdx.x] = (int)threadIdx.x < k ? tot : 0;
}

// ---------------------------------------------------------------------------
// 4. rows: one CTA per (leaf, slice of NR rows): the partners' x gathered in
//    shared memory, warp per row over the contiguous panel entries, the CSR
//    row, and the far expansion over the levels lmin..L
// ---------------------------------------------------------------------------
template <class T, class A>
__global__ void __launch_bounds__(128)
k_near_csr(int fl, int NR, const int *__restrict__ kb, const int *__restrict__ ke, const int *__restrict__ nptr,
           const int *__restrict__ ncol, const int64_t *__restrict__ noff, const int *__restrict__ pw,
           const int64_t *__restrict__ poff, const int *__restrict__ gcol, const int *__restrict__ goff,
           const T *__restrict__ D, int use_near, const int *__restrict__ rowptr,
           const int *__restrict__ colidx, const double *__restrict__ val, FarView F, const T *__restrict__ Ul,
           const A *__restrict__ yhat, int64_t hs, const double *__restrict__ X, int64_t ld, double *__restrict__ Y,
           const int *skip)
{
    using V = typename Vec<T>::V;
    constexpr int VW = Vec<T>::W;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *xg = (T *)smraw;
    if (skip && *skip) return;
    const int lf = blockIdx.x, r = blockIdx.z;
    const int b_leaf = kb[fl + lf];
    const int b = b_leaf + blockIdx.y * NR, e = min(ke[fl + lf], b + NR);
    if (b >= e) return;
    const double *x = X + (size_t)r * ld;
    const int W = use_near ? pw[lf] : 0;
    const int64_t P0 = use_near ? poff[lf] : 0;
    if (use_near) {
        const int *gc = gcol + goff[lf];
        for (int t = threadIdx.x; t < W; t += blockDim.x) {
            int j = gc[t];
            xg[t] = j >= 0 ? (T)x[j] : (T)0;
        }
        __syncthreads();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const A *yh = yhat + (size_t)r * hs;
    // a warp takes four rows (b + warp + q nw, q = 0..3) at a time: one
    // accumulator per row and lane (FP64 issue is slow enough on this part that
    // the dependency chain costs nothing), then one butterfly over the four
    // rows together (6 adds instead of 4 x 5 for separate warp sums)
    for (int g0 = b; g0 < e; g0 += 4 * nw) {
        double part[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = g0 + warp + q * nw;
            double acc = 0.0;
            if (i < e) {
                if (use_near) {
                    T s = 0;
                    const V *row = (const V *)(D + P0 + (size_t)(i - b_leaf) * W);
                    const V *xv = (const V *)xg;
                    // a warp-uniform trip count for the full 128-vector steps and no
                    // unrolled copies of the ragged loops: predicated-off copies would
                    // still take FP64 issue slots
                    const int nv = W / VW, nfull = nv >> 7;
                    int c = lane;
#pragma unroll 1
                    for (int it = 0; it < nfull; ++it, c += 128) {
                        V a0 = row[c], a1 = row[c + 32], a2 = row[c + 64], a3 = row[c + 96];
                        fma_v(a0, xv[c], s, s);
                        fma_v(a1, xv[c + 32], s, s);
                        fma_v(a2, xv[c + 64], s, s);
                        fma_v(a3, xv[c + 96], s, s);
                    }
#pragma unroll 1
                    for (; c < nv; c += 32) fma_v(row[c], xv[c], s, s);
                    acc = (double)s;
                }
                if (val) {
#pragma unroll 1
                    for (int c = rowptr[i] + lane; c < rowptr[i + 1]; c += 32) acc = fma(val[c], x[colidx[c]], acc);
                }
            }
            part[q] = acc;
        }
        // butterfly: after the xor-16 and xor-8 steps lane L holds row
        // 2 (L >> 4 & 1) + (L >> 3 & 1) summed over 4 lanes; xor 4, 2, 1 finish it
        const bool h16 = lane & 16, h8 = lane & 8;
        double k0 = h16 ? part[2] : part[0], k1 = h16 ? part[3] : part[1];
        const double o0 = h16 ? part[0] : part[2], o1 = h16 ? part[1] : part[3];
        k0 += __shfl_xor_sync(0xffffffffu, o0, 16);
        k1 += __shfl_xor_sync(0xffffffffu, o1, 16);
        double kq = h8 ? k1 : k0;
        kq += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
        kq += __shfl_xor_sync(0xffffffffu, kq, 4);
        kq += __shfl_xor_sync(0xffffffffu, kq, 2);
        kq += __shfl_xor_sync(0xffffffffu, kq, 1);
        if ((lane & 7) == 0) {
            const int i = g0 + warp + ((lane >> 4) * 2 + ((lane >> 3) & 1)) * nw;
            if (i < e) Y[(size_t)r * ld + i] = kq;
        }
    }
}

// ---------------------------------------------------------------------------
// 5. far expansion after the join: Y[i] += sum_l Ul^(l)[i] . yhat[ancestor_l(i)]
//    (a warp takes rows i0 + q nw, q = 0..3, of its block's 4 nw; lanes over
//    (level, alpha); the four rows are reduced together by one xor butterfly)
// ---------------------------------------------------------------------------
constexpr int EXPAND_ROWS_PER_BLOCK = 16;   // 4 warps x 4 rows

template <class T, class A>
__global__ void __launch_bounds__(128)
k_far_expand(FarView F, int fl, const int *__restrict__ leaf_of, const T *__restrict__ Ul, const A *__restrict__ yhat,
             int64_t hs, double *__restrict__ Y, int64_t ld, const int *skip)
{
    if (skip && *skip) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5, r = blockIdx.y;
    const int i0 = blockIdx.x * 4 * nw + warp;
    const A *yh = yhat + (size_t)r * hs;
    double part[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + q * nw;
        A fa = 0;
        if (i < F.N) {
            const int lf = leaf_of[i];
            for (int l = F.lmin; l <= F.L; ++l) {
                const int lv = l - F.lmin, kl = F.kl[lv];
                const int node = ((fl + lf + 1) >> (F.L - l)) - 1;
                const T *u = Ul + F.uo[lv] + (size_t)i * kl;
                const A *y = yh + (size_t)node * F.k;
                for (int al = lane; al < kl; al += 32) fa += (A)u[al] * y[al];
            }
        }
        part[q] = (double)fa;
    }
    const bool h16 = lane & 16, h8 = lane & 8;
    double k0 = h16 ? part[2] : part[0], k1 = h16 ? part[3] : part[1];
    const double o0 = h16 ? part[0] : part[2], o1 = h16 ? part[1] : part[3];
    k0 += __shfl_xor_sync(0xffffffffu, o0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, o1, 16);
    double kq = h8 ? k1 : k0;
    kq += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
    kq += __shfl_xor_sync(0xffffffffu, kq, 4);
    kq += __shfl_xor_sync(0xffffffffu, kq, 2);
    kq += __shfl_xor_sync(0xffffffffu, kq, 1);
    if ((lane & 7) == 0) {
        const int i = i0 + ((lane >> 4) * 2 + ((lane >> 3) & 1)) * nw;
        if (i < F.N) Y[(size_t)r * ld + i] += kq;
    }
}

// the row kernel stages a whole panel row of x in shared memory: allow more
// than the default 48 KB (panels of exact-mode operators are N wide)
template <class T, class A>
static void row_kernel_smem(size_t shm)
{
    VFD_REQUIRE(shm <= 227 * 1024, VFD_EUNSUPPORTED,
                "apply: a near panel is wider than shared memory holds (use a low-rank operator, lambda > 0)");
    if (shm > 48 * 1024)
        VFD_CUDA(cudaFuncSetAttribute(k_near_csr<T, A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
}

// ---------------------------------------------------------------------------
// the far-field view: uniform rank k over the levels, or the per-level ranks
// of the recompressed far field (rc)
static FarView make_far_view(const MeshData &m, const OpData &op, bool use, bool rc)
{
    FarView F;
    F.use = (use && m.nfar > 0) ? 1 : 0;
    F.lmin = m.far_lmin;
    F.L = m.kt.L;
    F.nlev = F.use ? m.kt.L - m.far_lmin + 1 : 0;
    F.k = m.k;
    F.N = m.N;
    VFD_REQUIRE(F.nlev <= FV_MAXLEV, VFD_EUNSUPPORTED, "apply: too many far levels");
    for (int lv = 0; lv < FV_MAXLEV; ++lv) {
        F.kl[lv] = m.k;
        F.uo[lv] = (long long)lv * m.N * m.k;
    }
    F.so = nullptr;
    F.bk = nullptr;
    if (rc && F.use) {
        for (int lv = 0; lv < F.nlev; ++lv) {
            F.kl[lv] = op.rc_kl[lv];
            F.uo[lv] = op.rc_uo[lv];
        }
        F.so = op.rc_so.p;
        F.bk = op.rc_bk.p;
    }
    return F;
}

template <class T, class A>
static void apply_impl(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                       const T *Ul, const T *S, const T *D, A *xhat, A *yhat, A *part, A *ye, bool rc, cudaStream_t st,
                       const int *skip)
{
    const int k = m.k, fl = m.kt.first_leaf(), nnode = m.kt.nnode;
    const int64_t hs = (int64_t)nnode * k;
    const FarView F = make_far_view(m, op, (parts & VFD_PART_KFAR) != 0, rc);
    const bool near = (parts & VFD_PART_KNEAR) && m.nnear > 0;
    const double *val = nullptr;
    if ((parts & VFD_PART_B) && (parts & VFD_PART_M)) val = op.valBM.p;
    else if (parts & VFD_PART_B) val = op.valB.p;
    else if (parts & VFD_PART_M) val = op.valM.p;
    FarView Fn = F;
    Fn.use = 0;   // the expansion runs after the join (k_far_expand)
    if (F.use) {
        // far chain on the high-priority side stream, concurrent with the rows
        VFD_CUDA(cudaEventRecord(op.ev_fork, st));
        VFD_CUDA(cudaStreamWaitEvent(op.side, op.ev_fork, 0));
        dim3 gp(m.kt.nleaf, F.nlev, nrhs);
        k_far_proj<T, A><<<gp, 128, 0, op.side>>>(F, fl, m.kt.nleaf, m.kt_begin.p, m.kt_end.p, Ul, X, ld, part, skip);
        const int nn = nnode - ((1 << F.lmin) - 1);
        dim3 gs(nn, nrhs);
        k_far_sum<A><<<gs, 128, 0, op.side>>>(F, m.kt.nleaf, part, xhat, hs, skip);
        dim3 gc(cdiv((long long)m.nfar * 32, 256), nrhs);
        k_far_couple<T, A><<<gc, 256, 0, op.side>>>(F, m.nfar, nnode, m.far_ptr.p, m.far_col.p, S, xhat, ye, hs, skip);
        dim3 gy(cdiv((long long)nnode * k, 256), nrhs);
        k_far_couple_sum<A><<<gy, 256, 0, op.side>>>(F, m.nfar, nnode, m.far_ptr.p, ye, yhat, hs, skip);
    }
    const int NR = 16;
    dim3 go(m.kt.nleaf, cdiv(m.max_leaf_size, NR), nrhs);
    size_t shm = near ? (size_t)m.max_panel_w * sizeof(T) : 0;
    row_kernel_smem<T, A>(shm);
    k_near_csr<T, A><<<go, 128, shm, st>>>(fl, NR, m.kt_begin.p, m.kt_end.p, m.near_ptr.p, m.near_col.p, m.near_off.p,
                                           m.panel_w.p, m.panel_off.p, m.gcol.p, m.gcol_off.p, D, near ? 1 : 0,
                                           m.rowptr.p, m.colidx.p, val, Fn, Ul, yhat, hs, X, ld, Y, skip);
    if (F.use) {
        VFD_CUDA(cudaEventRecord(op.ev_join, op.side));
        VFD_CUDA(cudaStreamWaitEvent(st, op.ev_join, 0));
        dim3 ge(cdiv(m.N, EXPAND_ROWS_PER_BLOCK), nrhs);
        k_far_expand<T, A><<<ge, 128, 0, st>>>(F, fl, m.vleaf.p, Ul, yhat, hs, Y, ld, skip);
    }
    VFD_CUDA(cudaGetLastError());
}

static void ensure_streams(OpData &op)
{
    if (!op.side) {
        // the far chain is a short sequence of small launches: give it priority
        // so its CTAs are not queued behind the row kernel
        int lo = 0, hi = 0;
        VFD_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        VFD_CUDA(cudaStreamCreateWithPriority(&op.side, cudaStreamNonBlocking, hi));
        VFD_CUDA(cudaEventCreateWithFlags(&op.ev_fork, cudaEventDisableTiming));
        VFD_CUDA(cudaEventCreateWithFlags(&op.ev_join, cudaEventDisableTiming));
    }
}

void release_streams(OpData &op)
{
    if (op.side) {
        cudaStreamSynchronize(op.side);
        cudaStreamDestroy(op.side);
        cudaEventDestroy(op.ev_fork);
        cudaEventDestroy(op.ev_join);
        op.side = nullptr;
    }
}

// parts: VFD_PART_* mask; lowp: use the FP32 copies of K (VFD_FP32 and VFD_BF16 operators)
void apply_parts_ex(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                    bool lowp, cudaStream_t st, const int *skip)
{
    ensure_streams(op);
    const int nlev = m.nfar > 0 ? m.kt.L - m.far_lmin + 1 : 0;
    const size_t need = (size_t)m.kt.nnode * m.k * nrhs;
    const size_t needp = (size_t)std::max(nlev, 1) * m.kt.nleaf * m.k * nrhs;
    const size_t needy = (size_t)std::max(m.nfar, 1) * m.k * nrhs;
    if (lowp) {
        if (op.xhat32.n < need || op.P32.n < needp || op.ye32.n < needy) {
            release_graphs(op);   // captured solves refer to the old workspace
            op.xhat32.alloc(need);
            op.yhat32.alloc(need);
            op.P32.alloc(needp);
            op.ye32.alloc(needy);
        }
        apply_impl<float, float>(m, op, parts, X, Y, nrhs, ld, op.Ul32.p, op.S32.p, op.D32.p, op.xhat32.p, op.yhat32.p,
                                 op.P32.p, op.ye32.p, false, st, skip);
    } else {
        if (op.xhat.n < need || op.P64.n < needp || op.ye64.n < needy) {
            release_graphs(op);
            op.xhat.alloc(need);
            op.yhat.alloc(need);
            op.P64.alloc(needp);
            op.ye64.alloc(needy);
        }
        const bool rc = op.rc_on;   // the recompressed far field of the FP64 operator
        apply_impl<double, double>(m, op, parts, X, Y, nrhs, ld, rc ? op.Ulc64.p : m.Ul64.p, rc ? op.Sc64.p : op.S64.p,
                                   op.D64.p, op.xhat.p, op.yhat.p, op.P64.p, op.ye64.p, rc, st, skip);
    }
}

void apply_parts(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                 cudaStream_t st)
{
    // VFD_FP32 and VFD_BF16 operators both keep FP32 copies of K for the
    // column-by-column low-precision apply (BF16 is used by the batched path only)
    apply_parts_ex(m, op, parts, X, Y, nrhs, ld, op.precision != VFD_FP64, st, nullptr);
}

// ---------------------------------------------------------------------------
// Apply without any allocation (vfd_apply_noalloc).  The far-field scratch
// (node sums xhat, node results yhat, per-level leaf projections) lives in a
// fixed file-scope device array instead of operator workspaces, and the whole
// sequence runs on the caller's stream (no side stream, no events).  Every
// word of the scratch that a kernel reads has been written earlier in the
// same call, so nothing in it has to start at zero.  Two calls in flight at
// once on one device share the array and race.
// ---------------------------------------------------------------------------
static_assert(VFD_APPLY_NOALLOC_SCRATCH_BYTES % 256 == 0, "scratch size");
static __device__ __align__(256) unsigned char g_noalloc_scratch[VFD_APPLY_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

// the scratch address on the current device, looked up once per device
void *noalloc_scratch()
{
    int dev = -1;
    VFD_CUDA(cudaGetDevice(&dev));
    VFD_REQUIRE(dev >= 0 && dev < NOALLOC_MAX_DEVICES, VFD_EUNSUPPORTED, "vfd_apply_noalloc: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        VFD_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        VFD_REQUIRE(p != nullptr, VFD_ECUDA, "vfd_apply_noalloc: no address for the static scratch");
        g_noalloc_ptr[dev] = p;
    }
    return g_noalloc_ptr[dev];
}

// the launches of apply_impl, in order, on one stream
template <class T, class A>
void apply_one_stream(const MeshData &m, const OpData &op, const double *X, double *Y, int nrhs, int64_t ld,
                      const T *Ul, const T *S, const T *D, A *xhat, A *yhat, A *part, bool rc, cudaStream_t st)
{
    const int k = m.k, fl = m.kt.first_leaf(), nnode = m.kt.nnode;
    const int64_t hs = (int64_t)nnode * k;
    const FarView F = make_far_view(m, op, true, rc);
    const bool near = m.nnear > 0;
    FarView Fn = F;
    Fn.use = 0;
    if (F.use) {
        dim3 gp(m.kt.nleaf, F.nlev, nrhs);
        k_far_proj<T, A><<<gp, 128, 0, st>>>(F, fl, m.kt.nleaf, m.kt_begin.p, m.kt_end.p, Ul, X, ld, part, nullptr);
        const int nn = nnode - ((1 << F.lmin) - 1);
        dim3 gs(nn, nrhs);
        k_far_sum<A><<<gs, 128, 0, st>>>(F, m.kt.nleaf, part, xhat, hs, nullptr);
        dim3 gc(nnode, nrhs);
        k_far_couple_node<T, A><<<gc, 256, 0, st>>>(F, m.far_ptr.p, m.far_col.p, S, xhat, yhat, hs, nullptr);
    }
    const int NR = 16;
    dim3 go(m.kt.nleaf, cdiv(m.max_leaf_size, NR), nrhs);
    size_t shm = near ? (size_t)m.max_panel_w * sizeof(T) : 0;
    row_kernel_smem<T, A>(shm);
    k_near_csr<T, A><<<go, 128, shm, st>>>(fl, NR, m.kt_begin.p, m.kt_end.p, m.near_ptr.p, m.near_col.p, m.near_off.p,
                                           m.panel_w.p, m.panel_off.p, m.gcol.p, m.gcol_off.p, D, near ? 1 : 0,
                                           m.rowptr.p, m.colidx.p, op.valBM.p, Fn, Ul, yhat, hs, X, ld, Y, nullptr);
    if (F.use) {
        dim3 ge(cdiv(m.N, EXPAND_ROWS_PER_BLOCK), nrhs);
        k_far_expand<T, A><<<ge, 128, 0, st>>>(F, fl, m.vleaf.p, Ul, yhat, hs, Y, ld, nullptr);
    }
    VFD_CUDA(cudaGetLastError());
}
}  // namespace

// Y = A X (all parts) as apply_parts computes it, scratch in g_noalloc_scratch
void apply_noalloc(const MeshData &m, const OpData &op, const double *X, double *Y, int nrhs, int64_t ld,
                   cudaStream_t st)
{
    const bool lowp = op.precision != VFD_FP64;   // K in FP32 for VFD_FP32 and VFD_BF16 operators
    const size_t es = lowp ? sizeof(float) : sizeof(double);
    const int nlev = m.nfar > 0 ? m.kt.L - m.far_lmin + 1 : 0;
    const size_t nh = (size_t)m.kt.nnode * m.k * nrhs;
    const size_t np = (size_t)std::max(nlev, 1) * m.kt.nleaf * m.k * nrhs;
    const size_t bh = round256(nh * es), need = 2 * bh + round256(np * es);
    if (need > (size_t)VFD_APPLY_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "vfd_apply_noalloc: this operator and nrhs = %d need %zu bytes of far-field scratch; the static "
                 "scratch holds %zu bytes (use vfd_apply, or fewer columns per call)",
                 nrhs, need, (size_t)VFD_APPLY_NOALLOC_SCRATCH_BYTES);
        throw Error{VFD_EINVAL, msg};
    }
    unsigned char *base = (unsigned char *)noalloc_scratch();
    if (lowp)
        apply_one_stream<float, float>(m, op, X, Y, nrhs, ld, op.Ul32.p, op.S32.p, op.D32.p, (float *)base,
                                       (float *)(base + bh), (float *)(base + 2 * bh), false, st);
    else
        apply_one_stream<double, double>(m, op, X, Y, nrhs, ld, op.rc_on ? op.Ulc64.p : m.Ul64.p,
                                         op.rc_on ? op.Sc64.p : op.S64.p, op.D64.p, (double *)base,
                                         (double *)(base + bh), (double *)(base + 2 * bh), op.rc_on, st);
}

}  // namespace vfd
