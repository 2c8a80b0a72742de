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
// Operand tiles reach shared memory by cp.async (matrices in their stored
// precision, widened when the fragments are read), so every copy of a stage
// is in flight at once; the coupling double-buffers its blocks per warp group.
#include <cuda_bf16.h>

#include "batched.cuh"

namespace vfd {

namespace {

constexpr int FT = 128;          // threads per CTA (4 warps)
constexpr int LDB = RT + 8;      // row stride (floats) of [k][64] operand tiles: conflict-free B fragments

// row strides (elements of T) of the A tiles in shared memory, conflict-free
// fragment loads: transposed tiles A(m, k) = As[k * lda + m] (rows 8 words
// apart modulo 32 banks) and row-major tiles A(m, k) = As[m * lda + k] (rows 4
// words apart)
template <class T>
__host__ __device__ constexpr int lda_t(int m)
{
    return sizeof(T) == 2 ? ((m + 63) & ~63) + 16 : ((m + 31) & ~31) + 8;
}
template <class T>
__host__ __device__ constexpr int lda_r(int k)
{
    return sizeof(T) == 2 ? ((k + 63) & ~63) + 8 : ((k + 31) & ~31) + 4;
}

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

// a stored matrix entry as a TF32 operand: BF16 widens exactly, and FP32
// matrices are stored already rounded to TF32
__device__ __forceinline__ uint32_t a_op(float v) { return __float_as_uint(v); }
__device__ __forceinline__ uint32_t a_op(__nv_bfloat16 v) { return __float_as_uint(__bfloat162float(v)); }

// 16-byte cp.async into shared memory; !valid: the 16 bytes are zero-filled, nothing is read
__device__ __forceinline__ void cp16(void *smem, const void *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// rows [0, nrow) of ncol columns (ncol * sizeof(T) a multiple of 16 bytes) of a
// row-major global matrix (row stride ss elements) into shared memory (row
// stride lds elements), rows [nrow, npad) zero; 16-byte copies, issued by
// threads t0 .. t0 + nt - 1 (not committed)
template <class T>
__device__ __forceinline__ void stage_async(T *dst, int lds, const T *src, int ncol, int nrow, int npad, int ss,
                                            int t, int nt)
{
    constexpr int E = 16 / (int)sizeof(T);
    const int cpr = ncol / E;
    for (int c = t; c < npad * cpr; c += nt) {
        const int r = c / cpr, q = c - r * cpr;
        cp16(dst + r * lds + q * E, r < nrow ? (const void *)(src + (size_t)r * ss + q * E) : (const void *)src,
             r < nrow);
    }
}

// a 64-column FP32 tile [nrow][R-slice] from global (row stride R) into shared
// memory (row stride LDB), rows [nrow, npad) zero (not committed)
__device__ __forceinline__ void stage_x_async(float *dst, const float *src, int R, int nrow, int npad, int t, int nt)
{
    for (int e = t; e < npad * (RT / 4); e += nt) {
        const int r = e / (RT / 4), q = e - r * (RT / 4);
        cp16(dst + r * LDB + 4 * q, r < nrow ? (const void *)(src + (size_t)r * R + 4 * q) : (const void *)src,
             r < nrow);
    }
}

// One warp accumulates rows m0..m0+15 (of M) x the 64 columns: acc[j] = n8
// tile j.  A(m, k) = TRANS ? As[k * lda + m] : As[m * lda + k] (stored
// precision T, taken as TF32 exactly); B(k, n) = Bs[k * LDB + n] (FP32,
// rounded to TF32); K a multiple of 8 (operands zero-padded).
template <bool TRANS, class T>
__device__ __forceinline__ void warp_gemm(float (&acc)[8][4], const T *As, int lda, const float *Bs, int K, int m0)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int k0 = 0; k0 < K; k0 += 8) {
        uint32_t a[4];
        if (TRANS) {
            a[0] = a_op(As[(k0 + t) * lda + m0 + g]);
            a[1] = a_op(As[(k0 + t) * lda + m0 + g + 8]);
            a[2] = a_op(As[(k0 + t + 4) * lda + m0 + g]);
            a[3] = a_op(As[(k0 + t + 4) * lda + m0 + g + 8]);
        } else {
            a[0] = a_op(As[(m0 + g) * lda + k0 + t]);
            a[1] = a_op(As[(m0 + g + 8) * lda + k0 + t]);
            a[2] = a_op(As[(m0 + g) * lda + k0 + t + 4]);
            a[3] = a_op(As[(m0 + g + 8) * lda + k0 + t + 4]);
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

// rows m0 + (0..15) of the accumulator to a [rows][R-slice] FP32 tile
// (global or shared, row stride ld); rows < M
__device__ __forceinline__ void acc_store(const float (&acc)[8][4], float *dst, size_t ld, int M, bool add, int m0)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int m = m0 + g + 8 * h;
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

// named barrier over the nthreads threads (a multiple of 32) of one warp group
__device__ __forceinline__ void group_sync(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(nthreads) : "memory");
}

}  // namespace

// the flattened width is processed in chunks of fb_mc(kp, mt) columns (whole levels)
__host__ __device__ constexpr int fb_mc(int kp, int mt) { return kp * (kp >= 128 ? 1 : 128 / kp) < mt ? kp * (kp >= 128 ? 1 : 128 / kp) : mt; }
// shared memory (bytes) for column chunks of at most mcmax = min(128, largest mt) columns
template <class T>
static size_t fb_smem_proj(int mcmax) { return 4 * (size_t)64 * LDB + sizeof(T) * (size_t)64 * lda_t<T>(mcmax); }
// coupling: per warp group two buffers of S (kp x kp) and xhat (kp x 64), or the group sums
__host__ __device__ constexpr int fb_groups(int kp) { return 4 / ((kp + 15) / 16); }
template <class T>
static size_t fb_smem_couple1(int kp)
{
    const size_t buf = sizeof(T) * (size_t)kp * lda_t<T>(kp) + 4 * (size_t)kp * LDB;
    const size_t stg = (size_t)fb_groups(kp) * 2 * buf, red = (size_t)fb_groups(kp) * 4 * kp * LDB;
    return stg > red ? stg : red;
}
// the meshes of a batch may have different padded ranks (multiples of 8, at most kpmax)
template <class T>
static size_t fb_smem_couple(int kpmax)
{
    size_t m = 0;
    for (int kp = 8; kp <= kpmax; kp += 8) m = std::max(m, fb_smem_couple1<T>(kp));
    return m;
}
template <class T>
static size_t fb_smem_expand(int mcmax) { return sizeof(T) * (size_t)64 * lda_r<T>(mcmax) + 4 * (size_t)mcmax * LDB; }

// ---------------------------------------------------------------------------
// K1: leaf projections of every level, part[leaf][m][R-slice], m < mt
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(FT)
k_fb_proj(const MrMesh *__restrict__ ms, const int2 *__restrict__ items, int R, const float *__restrict__ Xall,
          const int *skip, const int *mdone)
{
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    if (skip && *skip) return;
    const int2 item = items[blockIdx.x];
    if (mdone && mdone[item.x]) return;
    const MrMesh &M = ms[item.x];
    const int mt = M.mt, rt = blockIdx.y * RT, mc = fb_mc(M.kp, mt);
    const int LA = lda_t<T>(mc);
    float *Xs = (float *)fsm_raw;                      // [64][LDB]  x rows of the leaf
    T *Us = (T *)(fsm_raw + 4 * 64 * LDB);             // [64][LA]   a column chunk of the leaf's Ulf rows (A transposed)
    const int node = M.fl + item.y;
    const int b = M.kb[node], na = M.ke[node] - b;
    const int npad = (na + 7) & ~7;
    const int warp = threadIdx.x >> 5;
    stage_x_async(Xs, Xall + (size_t)(M.xoff + b) * R + rt, R, na, npad, threadIdx.x, FT);
    float *dst = M.part + (size_t)item.y * mt * R + rt;
    for (int c0 = 0; c0 < mt; c0 += mc) {
        const int nc = min(mc, mt - c0);
        if (c0 > 0) __syncthreads();   // the previous chunk's products are done with Us
        stage_async<T>(Us, LA, (const T *)M.Ulf + (size_t)b * mt + c0, nc, na, npad, mt, threadIdx.x, FT);
        cp_commit();
        cp_wait<0>();
        __syncthreads();
        for (int m0 = 0; m0 < nc; m0 += 64) {
            float acc[8][4];
            acc_zero(acc);
            if (m0 + 16 * warp < nc) warp_gemm<true, T>(acc, Us + m0, LA, Xs, npad, 16 * warp);
            acc_store(acc, dst + (size_t)(c0 + m0) * R, R, min(64, nc - m0), false, 16 * warp);
        }
    }
}

// ---------------------------------------------------------------------------
// K1b: node sums xhat[node][a][R-slice] = sum over the node's leaves of their
// level-(node) slice of part, in leaf order (eight interleaved partial sums)
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
    constexpr int U = 8;
    for (int e = threadIdx.x; e < kp * (RT / 4); e += blockDim.x) {
        const int a = e / (RT / 4), q = e % (RT / 4);
        // partial sum u takes the leaves j = U t + u; combined in a fixed order
        float4 p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) p[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        const float *base = src + (size_t)a * R;
        int j = 0;
        for (; j + U <= span; j += U) {
            float4 w[U];
#pragma unroll
            for (int u = 0; u < U; ++u) w[u] = __ldcg((const float4 *)(base + (size_t)(j + u) * mt * R) + q);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                p[u].x += w[u].x;
                p[u].y += w[u].y;
                p[u].z += w[u].z;
                p[u].w += w[u].w;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (j + u < span) {
                const float4 w = __ldcg((const float4 *)(base + (size_t)(j + u) * mt * R) + q);
                p[u].x += w.x;
                p[u].y += w.y;
                p[u].z += w.z;
                p[u].w += w.w;
            }
#pragma unroll
        for (int h = U / 2; h >= 1; h /= 2)
#pragma unroll
            for (int u = 0; u < h; ++u) {
                p[u].x += p[u + h].x;
                p[u].y += p[u + h].y;
                p[u].z += p[u + h].z;
                p[u].w += p[u + h].w;
            }
        *(float4 *)(M.xhat + (size_t)node * hs + (size_t)a * R + rt + 4 * q) = p[0];
    }
}

// ---------------------------------------------------------------------------
// K2: coupling yc_node = sum_e S_e xhat_col(e)   (S_e stored transposed [b][a]).
// The node's blocks are dealt round-robin to warp groups (a group = the
// ceil(kp / 16) warps covering the kp rows); each group double-buffers its
// blocks through cp.async and keeps its own accumulator; the group sums are
// added in group order at the end (deterministic).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(FT)
k_fb_couple(const MrMesh *__restrict__ ms, const int2 *__restrict__ items, int R, const int *skip, const int *mdone)
{
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    if (skip && *skip) return;
    const int2 item = items[blockIdx.x];
    if (mdone && mdone[item.x]) return;
    const MrMesh &M = ms[item.x];
    const int kp = M.kp, rt = blockIdx.y * RT, node = item.y;
    const int LA = lda_t<T>(kp);
    const int mtl = (kp + 15) / 16, ng = 4 / mtl;
    const int warp = threadIdx.x >> 5, grp = warp / mtl, m0 = 16 * (warp % mtl);
    const bool in_group = grp < ng;
    const int gt = threadIdx.x - grp * 32 * mtl, gn = 32 * mtl;   // thread index and size of the group
    const size_t sbytes = sizeof(T) * (size_t)kp * LA, buf = sbytes + 4 * (size_t)kp * LDB;
    unsigned char *gbase = fsm_raw + (size_t)grp * 2 * buf;
    const T *S = (const T *)M.S;
    const size_t hs = (size_t)kp * R;
    const int e0 = M.fptr[node], ne = M.fptr[node + 1] - e0;
    const int nmine = in_group && grp < ne ? (ne - grp + ng - 1) / ng : 0;   // this group's blocks grp, grp + ng, ...
    float acc[8][4];
    acc_zero(acc);
    auto issue = [&](int i) {
        const int e = e0 + grp + i * ng;
        unsigned char *bb = gbase + (size_t)(i & 1) * buf;
        stage_async<T>((T *)bb, LA, S + (size_t)e * kp * kp, kp, kp, kp, kp, gt, gn);
        stage_x_async((float *)(bb + sbytes), M.xhat + (size_t)M.fcol[e] * hs + rt, R, kp, kp, gt, gn);
    };
    if (nmine > 0) {
        issue(0);
        cp_commit();
        for (int i = 0; i < nmine; ++i) {
            if (i + 1 < nmine) issue(i + 1);
            cp_commit();
            cp_wait<1>();               // this thread's copies of block i have landed
            group_sync(1 + grp, gn);    // ... and every thread's of the group
            const unsigned char *bb = gbase + (size_t)(i & 1) * buf;
            if (m0 < kp) warp_gemm<true, T>(acc, (const T *)bb, LA, (const float *)(bb + sbytes), kp, m0);
            group_sync(1 + grp, gn);    // buffer i & 1 is free for block i + 2
        }
    }
    cp_wait<0>();
    __syncthreads();
    // group sums in shared memory (over the staging buffers), then in group order to yhat
    float *red = (float *)fsm_raw;   // [ng][kp][LDB]
    if (in_group) acc_store(acc, red + (size_t)grp * kp * LDB, LDB, kp, false, m0);
    __syncthreads();
    for (int e = threadIdx.x; e < kp * (RT / 4); e += blockDim.x) {
        const int a = e / (RT / 4), q = e % (RT / 4);
        float4 v = *(const float4 *)(red + (size_t)a * LDB + 4 * q);
        for (int gg = 1; gg < ng; ++gg) {
            const float4 w = *(const float4 *)(red + ((size_t)gg * kp + a) * LDB + 4 * q);
            v.x += w.x;
            v.y += w.y;
            v.z += w.z;
            v.w += w.w;
        }
        *(float4 *)(M.yhat + (size_t)node * hs + (size_t)a * R + rt + 4 * q) = v;
    }
}

// ---------------------------------------------------------------------------
// K3: expansion Y_leaf += Ulf_leaf [yc of the leaf's ancestors by level]
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(FT)
k_fb_expand(const MrMesh *__restrict__ ms, const int2 *__restrict__ items, int R, float *__restrict__ Yall,
            int add, const int *skip, const int *mdone)
{
    extern __shared__ __align__(16) unsigned char fsm_raw[];
    if (skip && *skip) return;
    const int2 item = items[blockIdx.x];
    if (mdone && mdone[item.x]) return;
    const MrMesh &M = ms[item.x];
    const int kp = M.kp, mt = M.mt, rt = blockIdx.y * RT, L = M.L, lmin = M.lmin, mc = fb_mc(kp, mt);
    const int LA = lda_r<T>(mc);
    T *Us = (T *)fsm_raw;                                               // [64][LA]  a column chunk of the leaf's Ulf rows
    float *Ys = (float *)(fsm_raw + sizeof(T) * (size_t)64 * LA);       // [mc][LDB] the matching levels of the ancestors' yc
    const size_t hs = (size_t)kp * R;
    const int leafnode = M.fl + item.y;
    const int b = M.kb[leafnode], na = M.ke[leafnode] - b;
    const int npad = (na + 15) & ~15;
    const int warp = threadIdx.x >> 5;
    float acc[8][4];
    acc_zero(acc);
    for (int c0 = 0; c0 < mt; c0 += mc) {
        const int nc = min(mc, mt - c0);
        if (c0 > 0) __syncthreads();   // the previous chunk's products are done with Us, Ys
        for (int lc = 0; lc < nc / kp; ++lc) {
            const int l = lmin + c0 / kp + lc;
            const int node = ((leafnode + 1) >> (L - l)) - 1;
            float *dst = Ys + (size_t)lc * kp * LDB;
            if (M.fptr[node + 1] > M.fptr[node]) {
                stage_x_async(dst, M.yhat + (size_t)node * hs + rt, R, kp, kp, threadIdx.x, FT);
            } else {   // a node without admissible blocks has no yc (zero)
                for (int e = threadIdx.x; e < kp * (RT / 4); e += blockDim.x)
                    *(float4 *)(dst + (e / (RT / 4)) * LDB + 4 * (e % (RT / 4))) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        stage_async<T>(Us, LA, (const T *)M.Ulf + (size_t)b * mt + c0, nc, na, npad, mt, threadIdx.x, FT);
        cp_commit();
        cp_wait<0>();
        __syncthreads();
        if (16 * warp < npad) warp_gemm<false, T>(acc, Us, LA, Ys, nc, 16 * warp);
    }
    acc_store(acc, Yall + (size_t)(M.xoff + b) * R + rt, R, na, add != 0, 16 * warp);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// the largest shared memory of the far kernels for padded rank kp and mt = nlev * kp (FP32 tiles: the larger)
size_t far_batched_smem(int kp, int mt)
{
    const int mc = std::min(128, mt);
    return std::max(fb_smem_proj<float>(mc), std::max(fb_smem_couple<float>(kp), fb_smem_expand<float>(mc)));
}

template <class T>
static void far_attrs(int kp, int mt)
{
    const int mc = std::min(128, mt);
    VFD_CUDA(cudaFuncSetAttribute(k_fb_proj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_proj<T>(mc)));
    VFD_CUDA(cudaFuncSetAttribute(k_fb_couple<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_couple<T>(kp)));
    VFD_CUDA(cudaFuncSetAttribute(k_fb_expand<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fb_smem_expand<T>(mc)));
}

template <class T>
static void launch_far_side_t(BatchData &b, int R, const float *X, cudaStream_t side, const int *skip,
                              const int *mdone)
{
    const MrMesh *ms = (const MrMesh *)b.desc.p;
    const int kp = b.max_kp, mt = b.max_mt, mc = std::min(128, mt);
    dim3 gl(b.n_leaf_items, R / RT), gn(b.n_node_items, R / RT);
    far_attrs<T>(kp, mt);
    k_fb_proj<T><<<gl, FT, fb_smem_proj<T>(mc), side>>>(ms, (const int2 *)b.leaf_items.p, R, X, skip, mdone);
    if (b.n_node_items) {
        k_fb_nsum<<<gn, 256, 0, side>>>(ms, (const int2 *)b.node_items.p, R, skip, mdone);
        k_fb_couple<T><<<gn, FT, fb_smem_couple<T>(kp), side>>>(ms, (const int2 *)b.node_items.p, R, skip, mdone);
    }
    VFD_CUDA(cudaGetLastError());
}

// projections, node sums and coupling (K1, K1b, K2) on stream `side`
void launch_far_side(BatchData &b, int R, const float *X, cudaStream_t side, const int *skip, const int *mdone)
{
    if (b.precision == VFD_BF16) launch_far_side_t<__nv_bfloat16>(b, R, X, side, skip, mdone);
    else launch_far_side_t<float>(b, R, X, side, skip, mdone);
}

// expansion (K3) on stream `st`, adding into Y (add) or writing it
void launch_far_down(BatchData &b, int R, float *Y, cudaStream_t st, const int *skip, const int *mdone, bool add)
{
    const MrMesh *ms = (const MrMesh *)b.desc.p;
    const int mc = std::min(128, b.max_mt);
    dim3 gl(b.n_leaf_items, R / RT);
    if (b.precision == VFD_BF16)
        k_fb_expand<__nv_bfloat16><<<gl, FT, fb_smem_expand<__nv_bfloat16>(mc), st>>>(ms, (const int2 *)b.leaf_items.p, R,
                                                                                        Y, add ? 1 : 0, skip, mdone);
    else
        k_fb_expand<float><<<gl, FT, fb_smem_expand<float>(mc), st>>>(ms, (const int2 *)b.leaf_items.p, R, Y,
                                                                        add ? 1 : 0, skip, mdone);
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
