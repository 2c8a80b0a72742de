// Far field of the batched low-precision apply (the admissible blocks of K,
// Sec. 5.3) for 64-RHS tiles, with the nested bases of the interpolation H^2
// matrix (the transfer matrices of the last paragraph of Sec. 5.3):
//
//   K1 upsweep   (CTA per leaf):  xhat_leaf = U_leaf^T X_leaf; then up the
//                tree: the second child to finish computes
//                xhat_parent = E_c1^T xhat_c1 + E_c2^T xhat_c2 (a counter per
//                node picks the last arriver; the two children are always
//                added in the same order, so the result is deterministic),
//                up to the first level with admissible blocks;
//   K2 coupling  (CTA per node):  yc_node = sum_e S_e xhat_col(e)  (eq.
//                eq:triple_product_factored), blocks streamed through shared
//                memory;
//   K3 downsweep + expansion (CTA per leaf): t = yc at the leaf's ancestor on
//                the first far level, then t = E_node t + yc_node down the
//                leaf's path, and Y_leaf += U_leaf t.  Each leaf walks its own
//                path (the ancestors' transfers are recomputed per leaf: a few
//                small products that cost less than a level-by-level chain of
//                launches).
//
// Matrices are stored in the operator's low precision (BF16, or FP32 rounded
// to TF32) with the rank padded to kp = k rounded up to 8 (zero rows and
// columns), products run on the tensor cores (mma.sync m16n8k8 TF32, FP32
// accumulation), vectors are FP32 in the interleaved layout [row][R].
#include <cuda_bf16.h>

#include "batched.cuh"

namespace vfd {

namespace {

constexpr int FT = 128;          // threads per CTA (4 warps)
constexpr int LDB = RT + 8;      // row stride (floats) of [k][64] operand tiles: conflict-free B fragments
__host__ __device__ constexpr int lda_t(int kp) { return ((kp + 31) & ~31) + 8; }   // transposed A tiles
__host__ __device__ constexpr int lda_r(int kp) { return ((kp + 31) & ~31) + 4; }   // row-major A tiles

__device__ __forceinline__ uint32_t tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float *c, const uint32_t *a, const uint32_t *b)
{
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <class T>
__device__ __forceinline__ float ld1(const T *p);
template <>
__device__ __forceinline__ float ld1<float>(const float *p) { return *p; }
template <>
__device__ __forceinline__ float ld1<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// 16-byte piece of a row: 8 BF16 or 4 FP32 values, widened to FP32
__device__ __forceinline__ int piece(const __nv_bfloat16 *p, float *v)
{
    const uint4 u = *(const uint4 *)p;
    const __nv_bfloat162 *h = (const __nv_bfloat162 *)&u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(h[j]);
        v[2 * j] = f.x;
        v[2 * j + 1] = f.y;
    }
    return 8;
}
__device__ __forceinline__ int piece(const float *p, float *v)
{
    const float4 u = *(const float4 *)p;
    v[0] = u.x;
    v[1] = u.y;
    v[2] = u.z;
    v[3] = u.w;
    return 4;
}

// rows [0, nrow) of kp columns (kp a multiple of 8) of a row-major global
// matrix with row stride kp into shared memory (row stride lds, FP32), rows
// [nrow, npad) zero; 16-byte loads, eight threads per row
template <class T>
__device__ __forceinline__ void stage(float *dst, int lds, const T *src, int kp, int nrow, int npad)
{
    constexpr int E = 16 / (int)sizeof(T);
    const int cpr = kp / E, sub = threadIdx.x & 7;
    for (int r = threadIdx.x >> 3; r < npad; r += blockDim.x >> 3)
        for (int c = sub; c < cpr; c += 8) {
            float v[8];
            if (r < nrow) piece(src + (size_t)r * kp + c * E, v);
            else
#pragma unroll
                for (int j = 0; j < E; ++j) v[j] = 0.f;
            float *d = dst + r * lds + c * E;
#pragma unroll
            for (int j = 0; j < E; j += 4) *(float4 *)(d + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
}

// a 64-column FP32 tile [nrow][R-slice] from global (row stride R) into shared memory
__device__ __forceinline__ void stage_x(float *dst, const float *src, int R, int nrow, int npad)
{
    for (int e = threadIdx.x; e < npad * (RT / 4); e += blockDim.x) {
        const int r = e / (RT / 4), q = e - r * (RT / 4);
        const float4 v = r < nrow ? __ldcg((const float4 *)(src + (size_t)r * R) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        *(float4 *)(dst + r * LDB + 4 * q) = v;
    }
}

// Warp w accumulates rows 16w..16w+15 (of M <= 64) x the 64 columns:
// acc[j] = n8 tile j.  A(m, k) = TRANS ? As[k * lda + m] : As[m * lda + k];
// B(k, n) = Bs[k * LDB + n]; K a multiple of 8 (operands zero-padded).
template <bool TRANS>
__device__ __forceinline__ void cta_gemm(float (&acc)[8][4], const float *As, int lda, const float *Bs, int K)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int m0 = 16 * warp;
    for (int k0 = 0; k0 < K; k0 += 8) {
        uint32_t a[4];
        if (TRANS) {
            a[0] = tf32(As[(k0 + t) * lda + m0 + g]);
            a[1] = tf32(As[(k0 + t) * lda + m0 + g + 8]);
            a[2] = tf32(As[(k0 + t + 4) * lda + m0 + g]);
            a[3] = tf32(As[(k0 + t + 4) * lda + m0 + g + 8]);
        } else {
            a[0] = tf32(As[(m0 + g) * lda + k0 + t]);
            a[1] = tf32(As[(m0 + g + 8) * lda + k0 + t]);
            a[2] = tf32(As[(m0 + g) * lda + k0 + t + 4]);
            a[3] = tf32(As[(m0 + g + 8) * lda + k0 + t + 4]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t b[2] = {tf32(Bs[(k0 + t) * LDB + 8 * j + g]), tf32(Bs[(k0 + t + 4) * LDB + 8 * j + g])};
            mma_tf32(acc[j], a, b);
        }
    }
}

__device__ __forceinline__ void acc_zero(float (&acc)[8][4])
{
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
}

// the warp's rows of the accumulator to a [rows][R-slice] FP32 tile (global or shared, row stride ld); rows < M
__device__ __forceinline__ void acc_store(const float (&acc)[8][4], float *dst, size_t ld, int M, bool add)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int m = 16 * warp + g + 8 * h;
        if (m >= M) continue;
        float *row = dst + (size_t)m * ld;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float2 v = make_float2(acc[j][2 * h], acc[j][2 * h + 1]);
            float2 *p = (float2 *)(row + 8 * j + 2 * t);
            if (add) {
                const float2 o = *p;
                v.x += o.x;
                v.y += o.y;
            }
            *p = v;
        }
    }
}

// accumulator += a [rows][R-slice] FP32 tile (global, row stride ld); rows < M
__device__ __forceinline__ void acc_add(float (&acc)[8][4], const float *src, size_t ld, int M)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int m = 16 * warp + g + 8 * h;
        if (m >= M) continue;
        const float *row = src + (size_t)m * ld;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 v = __ldcg((const float2 *)(row + 8 * j + 2 * t));
            acc[j][2 * h] += v.x;
            acc[j][2 * h + 1] += v.y;
        }
    }
}

}  // namespace

// shared memory of the three kernels (floats)
static size_t fb_smem_up(int kp) { return 4 * ((size_t)64 * LDB + (size_t)64 * lda_t(kp) + 2 * (size_t)kp * LDB + 2 * (size_t)kp * lda_t(kp)); }
static size_t fb_smem_couple(int kp) { return 4 * ((size_t)kp * lda_t(kp) + (size_t)kp * LDB); }
static size_t fb_smem_down(int kp) { return 4 * ((size_t)kp * lda_r(kp) + (size_t)kp * LDB + (size_t)64 * lda_r(kp)); }

// ---------------------------------------------------------------------------
// K1: leaf projections and the transfer upsweep (last arriver per node)
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(FT)
k_fb_up(const MrMesh *__restrict__ ms, const int2 *__restrict__ items, int R, const float *__restrict__ Xall,
        const int *skip, const int *mdone)
{
    extern __shared__ __align__(16) float fsm[];
    __shared__ int last;
    if (skip && *skip) return;
    const int2 item = items[blockIdx.x];
    if (mdone && mdone[item.x]) return;
    const MrMesh &M = ms[item.x];
    const int kp = M.kp, rt = blockIdx.y * RT, fl = M.fl;
    const int LA = lda_t(kp);
    float *Xs = fsm;                 // [64][LDB]   x rows of the leaf
    float *Us = Xs + 64 * LDB;       // [64][LA]    U rows of the leaf (A transposed)
    float *Ho = Us + 64 * LA;        // [kp][LDB]   xhat of the CTA's current node
    float *Hb = Ho + kp * LDB;       // [kp][LDB]   xhat of its sibling
    float *E1 = Hb + kp * LDB;       // [kp][LA]    transfers of the two children (A transposed)
    float *E2 = E1 + kp * LA;
    const T *U = (const T *)M.Ul, *E = (const T *)M.E;
    float *xhat = M.xhat;
    const size_t hs = (size_t)kp * R;   // node stride of xhat
    int node = fl + item.y;
    const int b = M.kb[node], na = M.ke[node] - b;
    const int npad = (na + 7) & ~7;
    stage_x(Xs, Xall + (size_t)(M.xoff + b) * R + rt, R, na, npad);
    stage<T>(Us, LA, U + (size_t)b * kp, kp, na, npad);
    __syncthreads();
    float acc[8][4];
    acc_zero(acc);
    const bool mw = 16 * (threadIdx.x >> 5) < kp;   // this warp owns rows of the result
    if (mw) cta_gemm<true>(acc, Us, LA, Xs, npad);
    acc_store(acc, xhat + (size_t)node * hs + rt, R, kp, false);
    acc_store(acc, Ho, LDB, kp, false);
    int lev = M.L;
    while (lev > M.lmin) {
        const int par = (node - 1) / 2, c1 = 2 * par + 1, sib = node == c1 ? c1 + 1 : c1;
        // the transfers are fixed data: fetch them before waiting for the sibling
        stage<T>(E1, LA, E + (size_t)c1 * kp * kp, kp, kp, kp);
        stage<T>(E2, LA, E + (size_t)(c1 + 1) * kp * kp, kp, kp, kp);
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            const int prev = atomicAdd(M.cnt + (size_t)par * (R / RT) + blockIdx.y, 1);
            last = prev == 1;
            if (last) M.cnt[(size_t)par * (R / RT) + blockIdx.y] = 0;   // ready for the next launch
        }
        __syncthreads();
        if (!last) return;
        __threadfence();
        stage_x(Hb, xhat + (size_t)sib * hs + rt, R, kp, kp);
        __syncthreads();
        // always child 1 then child 2, whichever CTA arrived last
        const float *H1 = node == c1 ? Ho : Hb, *H2 = node == c1 ? Hb : Ho;
        acc_zero(acc);
        if (mw) {
            cta_gemm<true>(acc, E1, LA, H1, kp);
            cta_gemm<true>(acc, E2, LA, H2, kp);
        }
        __syncthreads();   // Ho read by every warp
        acc_store(acc, xhat + (size_t)par * hs + rt, R, kp, false);
        acc_store(acc, Ho, LDB, kp, false);
        node = par;
        --lev;
    }
}

// ---------------------------------------------------------------------------
// K2: coupling yc_node = sum_e S_e xhat_col(e)   (S_e stored transposed [b][a])
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(FT)
k_fb_couple(const MrMesh *__restrict__ ms, const int2 *__restrict__ items, int R, const int *skip, const int *mdone)
{
    extern __shared__ __align__(16) float fsm[];
    if (skip && *skip) return;
    const int2 item = items[blockIdx.x];
    if (mdone && mdone[item.x]) return;
    const MrMesh &M = ms[item.x];
    const int kp = M.kp, rt = blockIdx.y * RT, node = item.y;
    const int LA = lda_t(kp);
    float *Ss = fsm;              // [kp][LA]
    float *Hs = Ss + kp * LA;     // [kp][LDB]
    const T *S = (const T *)M.S;
    const size_t hs = (size_t)kp * R;
    float acc[8][4];
    acc_zero(acc);
    for (int e = M.fptr[node]; e < M.fptr[node + 1]; ++e) {
        stage<T>(Ss, LA, S + (size_t)e * kp * kp, kp, kp, kp);
        stage_x(Hs, M.xhat + (size_t)M.fcol[e] * hs + rt, R, kp, kp);
        __syncthreads();
        if (16 * (threadIdx.x >> 5) < kp) cta_gemm<true>(acc, Ss, LA, Hs, kp);
        __syncthreads();
    }
    acc_store(acc, M.yhat + (size_t)node * hs + rt, R, kp, false);
}

// ---------------------------------------------------------------------------
// K3: downsweep along the leaf's path and expansion Y_leaf += U_leaf t
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(FT)
k_fb_down(const MrMesh *__restrict__ ms, const int2 *__restrict__ items, int R, float *__restrict__ Yall,
          const int *skip, const int *mdone)
{
    extern __shared__ __align__(16) float fsm[];
    if (skip && *skip) return;
    const int2 item = items[blockIdx.x];
    if (mdone && mdone[item.x]) return;
    const MrMesh &M = ms[item.x];
    const int kp = M.kp, rt = blockIdx.y * RT, fl = M.fl, L = M.L, lmin = M.lmin;
    const int LA = lda_r(kp);
    float *Es = fsm;              // [kp][LA]  E_node (row-major A)
    float *Ts = Es + kp * LA;     // [kp][LDB] the running t
    float *Us = Ts + kp * LDB;    // [64][LA]  U rows of the leaf (row-major A)
    const T *U = (const T *)M.Ul, *E = (const T *)M.E;
    const size_t hs = (size_t)kp * R;
    const int leafnode = fl + item.y;
    const int b = M.kb[leafnode], na = M.ke[leafnode] - b;
    float acc[8][4];
    for (int l = lmin; l <= L; ++l) {
        const int node = ((leafnode + 1) >> (L - l)) - 1;
        acc_zero(acc);
        if (l > lmin) {
            stage<T>(Es, LA, E + (size_t)node * kp * kp, kp, kp, kp);
            __syncthreads();
            if (16 * (threadIdx.x >> 5) < kp) cta_gemm<false>(acc, Es, LA, Ts, kp);
        }
        if (M.fptr[node + 1] > M.fptr[node]) acc_add(acc, M.yhat + (size_t)node * hs + rt, R, kp);
        __syncthreads();   // Ts fully read
        acc_store(acc, Ts, LDB, kp, false);
        __syncthreads();
    }
    const int npad = (na + 15) & ~15;
    stage<T>(Us, LA, U + (size_t)b * kp, kp, na, npad);
    __syncthreads();
    acc_zero(acc);
    if (16 * (threadIdx.x >> 5) < npad) cta_gemm<false>(acc, Us, LA, Ts, kp);
    acc_store(acc, Yall + (size_t)(M.xoff + b) * R + rt, R, na, true);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t far_batched_smem(int kp) { return std::max(fb_smem_up(kp), std::max(fb_smem_couple(kp), fb_smem_down(kp))); }

template <class T>
static void far_attrs(int kp)
{
    VFD_CUDA(cudaFuncSetAttribute(k_fb_up<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_up(kp)));
    VFD_CUDA(cudaFuncSetAttribute(k_fb_couple<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_couple(kp)));
    VFD_CUDA(cudaFuncSetAttribute(k_fb_down<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_down(kp)));
}

// upsweep and coupling (K1, K2) on stream `side`
void launch_far_side(BatchData &b, int R, const float *X, cudaStream_t side, const int *skip, const int *mdone)
{
    const MrMesh *ms = (const MrMesh *)b.desc.p;
    const int kp = b.max_kp;
    dim3 gl(b.n_leaf_items, R / RT), gn(b.n_node_items, R / RT);
    if (b.precision == VFD_BF16) {
        far_attrs<__nv_bfloat16>(kp);
        k_fb_up<__nv_bfloat16><<<gl, FT, fb_smem_up(kp), side>>>(ms, (const int2 *)b.leaf_items.p, R, X, skip, mdone);
        if (b.n_node_items)
            k_fb_couple<__nv_bfloat16><<<gn, FT, fb_smem_couple(kp), side>>>(ms, (const int2 *)b.node_items.p, R, skip,
                                                                             mdone);
    } else {
        far_attrs<float>(kp);
        k_fb_up<float><<<gl, FT, fb_smem_up(kp), side>>>(ms, (const int2 *)b.leaf_items.p, R, X, skip, mdone);
        if (b.n_node_items)
            k_fb_couple<float><<<gn, FT, fb_smem_couple(kp), side>>>(ms, (const int2 *)b.node_items.p, R, skip, mdone);
    }
    VFD_CUDA(cudaGetLastError());
}

// downsweep and expansion (K3) on stream `st`, adding into Y
void launch_far_down(BatchData &b, int R, float *Y, cudaStream_t st, const int *skip, const int *mdone)
{
    const MrMesh *ms = (const MrMesh *)b.desc.p;
    const int kp = b.max_kp;
    dim3 gl(b.n_leaf_items, R / RT);
    if (b.precision == VFD_BF16)
        k_fb_down<__nv_bfloat16><<<gl, FT, fb_smem_down(kp), st>>>(ms, (const int2 *)b.leaf_items.p, R, Y, skip, mdone);
    else
        k_fb_down<float><<<gl, FT, fb_smem_down(kp), st>>>(ms, (const int2 *)b.leaf_items.p, R, Y, skip, mdone);
    VFD_CUDA(cudaGetLastError());
}

// padded low-precision copies: nmat row-major matrices srows x scols (FP64)
// into drows x dcols (zero padding), BF16 rounded to nearest or FP32
// rounded to TF32 -- the leaf bases U (N x k -> N x kp), the transfers E and
// the coupling blocks S (k x k -> kp x kp)
__global__ void k_pad_copy(long long nmat, int srows, int scols, int drows, int dcols, const double *__restrict__ src,
                           int bf, void *__restrict__ dst)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long per = (long long)drows * dcols;
    if (i >= nmat * per) return;
    const long long mtx = i / per;
    const int r = (int)((i % per) / dcols), c = (int)(i % dcols);
    const double v = (r < srows && c < scols) ? src[(mtx * srows + r) * (long long)scols + c] : 0.0;
    if (bf) ((__nv_bfloat16 *)dst)[i] = __double2bfloat16(v);
    else ((float *)dst)[i] = __uint_as_float(tf32(__double2float_rn(v)));
}

static void pad_copy(long long nmat, int srows, int scols, int drows, int dcols, const double *src, int bf,
                     DBuf<unsigned char> &dst, cudaStream_t st)
{
    const long long n = nmat * drows * (long long)dcols;
    dst.alloc((size_t)std::max<long long>(n, 1) * (bf ? 2 : 4));
    if (n > 0) k_pad_copy<<<cdiv(n, 256), 256, 0, st>>>(nmat, srows, scols, drows, dcols, src, bf, dst.p);
    VFD_CUDA(cudaGetLastError());
}

// the operator's padded low-precision U, E and S for the batched far field (first batched use)
void build_far_lowp(const MeshData &m, OpData &op, cudaStream_t st)
{
    if (op.far_kp || m.nfar == 0) return;
    // the inner operator's interpolation order if the mesh has one, else the operator's
    const int k = m.k_in ? m.k_in : m.k, kp = (k + 7) & ~7, bf = op.precision == VFD_BF16 ? 1 : 0;
    const int nlev = m.kt.L - m.far_lmin + 1;
    const double *U = m.k_in ? m.U_in64.p : m.Ul64.p + (size_t)(nlev - 1) * m.N * m.k;   // leaf bases
    pad_copy(1, m.N, k, m.N, kp, U, bf, op.Up_lp, st);
    pad_copy(m.kt.nnode, k, k, kp, kp, m.k_in ? m.E_in64.p : m.E64.p, bf, op.Ep_lp, st);
    pad_copy(m.nfar, k, k, kp, kp, m.k_in ? op.S64_in.p : op.S64.p, bf, op.Sp_lp, st);
    op.far_kp = kp;
}

}  // namespace vfd
