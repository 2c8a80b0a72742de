// Far field of the batched low-precision apply (the admissible blocks of K,
// Sec. 5.3) for 64-RHS tiles, with the bases of every level flattened
// (Ul^(l) = U E ... E, the nested bases of the last paragraph of Sec. 5.3
// multiplied out once per operator), so that no step waits on another level:
//
//   K1 projections (CTA per leaf): P_leaf = Ulf_leaf^T X_leaf, all levels at
//                once (Ulf row i = [Ul^(lmin)[i], ..., Ul^(L)[i]]);
//   K1b node sums  (CTA per node with admissible blocks): xhat_node = sum of
//                the node's leaves' level-slices of P, in leaf order;
//   K2 coupling    (CTA per node):  yc_node = sum_e S_e xhat_col(e)  (eq.
//                eq:triple_product_factored);
//   K3 expansion   (CTA per leaf):  Y_leaf += Ulf_leaf [yc of the leaf's
//                ancestors, stacked by level].
//
// Matrices are stored in the operator's low precision (BF16, or FP32 rounded
// to TF32) with the rank padded to kp = k rounded up to 8 (zero columns),
// products run on the tensor cores (mma.sync m16n8k8 TF32, FP32
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
// matrix with row stride sstride (default kp) into shared memory (row stride lds, FP32), rows
// [nrow, npad) zero; 16-byte loads, eight threads per row
template <class T>
__device__ __forceinline__ void stage(float *dst, int lds, const T *src, int kp, int nrow, int npad, int sstride = 0)
{
    constexpr int E = 16 / (int)sizeof(T);
    const int cpr = kp / E, sub = threadIdx.x & 7, ss = sstride ? sstride : kp;
    for (int r = threadIdx.x >> 3; r < npad; r += blockDim.x >> 3)
        for (int c = sub; c < cpr; c += 8) {
            float v[8];
            if (r < nrow) piece(src + (size_t)r * ss + c * E, v);
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

// shared memory of the kernels (bytes); mt = nlev * kp, the flattened row width
// the flattened width is processed in chunks of fb_mc(kp, mt) columns (whole levels)
__host__ __device__ constexpr int fb_mc(int kp, int mt) { return kp * (kp >= 128 ? 1 : 128 / kp) < mt ? kp * (kp >= 128 ? 1 : 128 / kp) : mt; }
// host: shared memory for column chunks of at most mcmax = min(128, largest mt) columns
static size_t fb_smem_proj(int mcmax) { return 4 * ((size_t)64 * LDB + (size_t)64 * lda_t(mcmax)); }
static size_t fb_smem_couple(int kp) { return 4 * ((size_t)kp * lda_t(kp) + (size_t)kp * LDB); }
static size_t fb_smem_expand(int mcmax) { return 4 * ((size_t)64 * lda_r(mcmax) + (size_t)mcmax * LDB); }

// ---------------------------------------------------------------------------
// K1: leaf projections of every level, part[leaf][m][R-slice], m < mt
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(FT)
k_fb_proj(const MrMesh *__restrict__ ms, const int2 *__restrict__ items, int R, const float *__restrict__ Xall,
          const int *skip, const int *mdone)
{
    extern __shared__ __align__(16) float fsm[];
    if (skip && *skip) return;
    const int2 item = items[blockIdx.x];
    if (mdone && mdone[item.x]) return;
    const MrMesh &M = ms[item.x];
    const int mt = M.mt, rt = blockIdx.y * RT, mc = fb_mc(M.kp, mt);
    const int LA = lda_t(mc);
    float *Xs = fsm;                 // [64][LDB]   x rows of the leaf
    float *Us = Xs + 64 * LDB;       // [64][LA]    a column chunk of the leaf's Ulf rows (A transposed)
    const int node = M.fl + item.y;
    const int b = M.kb[node], na = M.ke[node] - b;
    const int npad = (na + 7) & ~7;
    stage_x(Xs, Xall + (size_t)(M.xoff + b) * R + rt, R, na, npad);
    float *dst = M.part + (size_t)item.y * mt * R + rt;
    for (int c0 = 0; c0 < mt; c0 += mc) {
        const int nc = min(mc, mt - c0);
        __syncthreads();   // the previous chunk's products are done with Us
        stage<T>(Us, LA, (const T *)M.Ulf + (size_t)b * mt + c0, nc, na, npad, mt);
        __syncthreads();
        for (int m0 = 0; m0 < nc; m0 += 64) {
            float acc[8][4];
            acc_zero(acc);
            if (m0 + 16 * (threadIdx.x >> 5) < nc) cta_gemm<true>(acc, Us + m0, LA, Xs, npad);
            acc_store(acc, dst + (size_t)(c0 + m0) * R, R, min(64, nc - m0), false);
        }
    }
}

// ---------------------------------------------------------------------------
// K1b: node sums xhat[node][a][R-slice] = sum over the node's leaves of their
// level-(node) slice of part, in leaf order
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_fb_nsum(const MrMesh *__restrict__ ms, const int2 *__restrict__ items, int R, const int *skip, const int *mdone)
{
    if (skip && *skip) return;
    const int2 item = items[blockIdx.x];
    if (mdone && mdone[item.x]) return;
    const MrMesh &M = ms[item.x];
    const int kp = M.kp, mt = M.mt, rt = blockIdx.y * RT, node = item.y;
    int l = 0;
    while ((2 << l) - 1 <= node) ++l;
    const int span = 1 << (M.L - l), leaf0 = ((node + 1) << (M.L - l)) - 1 - M.fl;
    const size_t hs = (size_t)kp * R;
    const float *src = M.part + (size_t)leaf0 * mt * R + (size_t)(l - M.lmin) * kp * R + rt;
    for (int e = threadIdx.x; e < kp * (RT / 4); e += blockDim.x) {
        const int a = e / (RT / 4), q = e % (RT / 4);
        // four interleaved partial sums (leaves j = 4t + u), combined in a fixed order
        float4 p[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) p[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        const float *base = src + (size_t)a * R;
        int j = 0;
        for (; j + 4 <= span; j += 4)
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 w = __ldcg((const float4 *)(base + (size_t)(j + u) * mt * R) + q);
                p[u].x += w.x;
                p[u].y += w.y;
                p[u].z += w.z;
                p[u].w += w.w;
            }
        for (int u = 0; j < span; ++j, ++u) {
            const float4 w = __ldcg((const float4 *)(base + (size_t)j * mt * R) + q);
            p[u].x += w.x;
            p[u].y += w.y;
            p[u].z += w.z;
            p[u].w += w.w;
        }
        float4 v;
        v.x = (p[0].x + p[1].x) + (p[2].x + p[3].x);
        v.y = (p[0].y + p[1].y) + (p[2].y + p[3].y);
        v.z = (p[0].z + p[1].z) + (p[2].z + p[3].z);
        v.w = (p[0].w + p[1].w) + (p[2].w + p[3].w);
        *(float4 *)(M.xhat + (size_t)node * hs + (size_t)a * R + rt + 4 * q) = v;
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
// K3: expansion Y_leaf += Ulf_leaf [yc of the leaf's ancestors by level]
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(FT)
k_fb_expand(const MrMesh *__restrict__ ms, const int2 *__restrict__ items, int R, float *__restrict__ Yall,
            const int *skip, const int *mdone)
{
    extern __shared__ __align__(16) float fsm[];
    if (skip && *skip) return;
    const int2 item = items[blockIdx.x];
    if (mdone && mdone[item.x]) return;
    const MrMesh &M = ms[item.x];
    const int kp = M.kp, mt = M.mt, rt = blockIdx.y * RT, L = M.L, lmin = M.lmin, mc = fb_mc(kp, mt);
    const int LA = lda_r(mc);
    float *Us = fsm;               // [64][LA]  a column chunk of the leaf's Ulf rows (row-major A)
    float *Ys = Us + 64 * LA;      // [mc][LDB] the matching levels of the ancestors' yc
    const size_t hs = (size_t)kp * R;
    const int leafnode = M.fl + item.y;
    const int b = M.kb[leafnode], na = M.ke[leafnode] - b;
    const int npad = (na + 15) & ~15;
    float acc[8][4];
    acc_zero(acc);
    for (int c0 = 0; c0 < mt; c0 += mc) {
        const int nc = min(mc, mt - c0);
        __syncthreads();   // the previous chunk's products are done with Us, Ys
        for (int lc = 0; lc < nc / kp; ++lc) {
            const int l = lmin + c0 / kp + lc;
            const int node = ((leafnode + 1) >> (L - l)) - 1;
            float *dst = Ys + (size_t)lc * kp * LDB;
            if (M.fptr[node + 1] > M.fptr[node]) {
                stage_x(dst, M.yhat + (size_t)node * hs + rt, R, kp, kp);
            } else {
                for (int e = threadIdx.x; e < kp * (RT / 4); e += blockDim.x)
                    *(float4 *)(dst + (e / (RT / 4)) * LDB + 4 * (e % (RT / 4))) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        stage<T>(Us, LA, (const T *)M.Ulf + (size_t)b * mt + c0, nc, na, npad, mt);
        __syncthreads();
        if (16 * (threadIdx.x >> 5) < npad) cta_gemm<false>(acc, Us, LA, Ys, nc);
    }
    acc_store(acc, Yall + (size_t)(M.xoff + b) * R + rt, R, na, true);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// the largest shared memory of the far kernels for padded rank kp and mt = nlev * kp
size_t far_batched_smem(int kp, int mt)
{
    const int mc = std::min(128, mt);
    return std::max(fb_smem_proj(mc), std::max(fb_smem_couple(kp), fb_smem_expand(mc)));
}

template <class T>
static void far_attrs(int kp, int mt)
{
    VFD_CUDA(cudaFuncSetAttribute(k_fb_proj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_proj(std::min(128, mt))));
    VFD_CUDA(cudaFuncSetAttribute(k_fb_couple<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_couple(kp)));
    VFD_CUDA(cudaFuncSetAttribute(k_fb_expand<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_expand(std::min(128, mt))));
}

// projections, node sums and coupling (K1, K1b, K2) on stream `side`
void launch_far_side(BatchData &b, int R, const float *X, cudaStream_t side, const int *skip, const int *mdone)
{
    const MrMesh *ms = (const MrMesh *)b.desc.p;
    const int kp = b.max_kp, mt = b.max_mt;
    dim3 gl(b.n_leaf_items, R / RT), gn(b.n_node_items, R / RT);
    if (b.precision == VFD_BF16) {
        far_attrs<__nv_bfloat16>(kp, mt);
        k_fb_proj<__nv_bfloat16><<<gl, FT, fb_smem_proj(std::min(128, mt)), side>>>(ms, (const int2 *)b.leaf_items.p, R, X, skip,
                                                                     mdone);
    } else {
        far_attrs<float>(kp, mt);
        k_fb_proj<float><<<gl, FT, fb_smem_proj(std::min(128, mt)), side>>>(ms, (const int2 *)b.leaf_items.p, R, X, skip, mdone);
    }
    if (b.n_node_items) {
        k_fb_nsum<<<gn, 256, 0, side>>>(ms, (const int2 *)b.node_items.p, R, skip, mdone);
        if (b.precision == VFD_BF16)
            k_fb_couple<__nv_bfloat16><<<gn, FT, fb_smem_couple(kp), side>>>(ms, (const int2 *)b.node_items.p, R, skip,
                                                                             mdone);
        else
            k_fb_couple<float><<<gn, FT, fb_smem_couple(kp), side>>>(ms, (const int2 *)b.node_items.p, R, skip, mdone);
    }
    VFD_CUDA(cudaGetLastError());
}

// expansion (K3) on stream `st`, adding into Y
void launch_far_down(BatchData &b, int R, float *Y, cudaStream_t st, const int *skip, const int *mdone)
{
    const MrMesh *ms = (const MrMesh *)b.desc.p;
    const int mt = b.max_mt;
    dim3 gl(b.n_leaf_items, R / RT);
    if (b.precision == VFD_BF16)
        k_fb_expand<__nv_bfloat16><<<gl, FT, fb_smem_expand(std::min(128, mt)), st>>>(ms, (const int2 *)b.leaf_items.p, R, Y, skip,
                                                                       mdone);
    else
        k_fb_expand<float><<<gl, FT, fb_smem_expand(std::min(128, mt)), st>>>(ms, (const int2 *)b.leaf_items.p, R, Y, skip, mdone);
    VFD_CUDA(cudaGetLastError());
}

// flattened bases of every far level in the operator's low precision:
// out[i][lv * kp + a] = (U_i E_{c_L} ... E_{c_{l+1}})[a], l = lmin + lv, c_j the
// level-j ancestor of row i's leaf (zero for a >= k); thread per row
__global__ void k_flat_bases(int N, int k, int kp, int nlev, int lmin, int L, int fl, const int *__restrict__ vleaf,
                             const double *__restrict__ U, const double *__restrict__ E, int bf, void *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double t[KMAX], t2[KMAX];
    for (int a = 0; a < k; ++a) t[a] = U[(size_t)i * k + a];
    const int leafnode = fl + vleaf[i], mt = nlev * kp;
    for (int l = L; l >= lmin; --l) {
        if (l < L) {   // t = t E_c, c the level-(l+1) ancestor
            const int c = ((leafnode + 1) >> (L - (l + 1))) - 1;
            const double *Ec = E + (size_t)c * k * k;
            for (int a = 0; a < k; ++a) {
                double v = 0.0;
                for (int be = 0; be < k; ++be) v += t[be] * Ec[(size_t)be * k + a];
                t2[a] = v;
            }
            for (int a = 0; a < k; ++a) t[a] = t2[a];
        }
        const size_t o = (size_t)i * mt + (size_t)(l - lmin) * kp;
        for (int a = 0; a < kp; ++a) {
            const double v = a < k ? t[a] : 0.0;
            if (bf) ((__nv_bfloat16 *)out)[o + a] = __double2bfloat16(v);
            else ((float *)out)[o + a] = __uint_as_float(tf32(__double2float_rn(v)));
        }
    }
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
    const int mt = nlev * kp;
    op.Up_lp.alloc((size_t)m.N * mt * (bf ? 2 : 4));
    k_flat_bases<<<cdiv(m.N, 128), 128, 0, st>>>(m.N, k, kp, nlev, m.far_lmin, m.kt.L, m.kt.first_leaf(), m.vleaf.p, U,
                                                m.k_in ? m.E_in64.p : m.E64.p, bf, op.Up_lp.p);
    VFD_CUDA(cudaGetLastError());
    pad_copy(m.nfar, k, k, kp, kp, m.k_in ? op.S64_in.p : op.S64.p, bf, op.Sp_lp, st);
    op.far_kp = kp;
}

}  // namespace vfd
