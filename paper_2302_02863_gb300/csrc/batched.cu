// Batched multi-RHS apply of the low-precision operator (the inner operator
// of iterative refinement) for R right-hand sides at once, R a multiple of 64.
// Vectors are FP32 in the interleaved layout X[i][r] (DoF-major, RHS
// contiguous), so every gather of one DoF's entries is one contiguous read.
//
//   near panels: per (leaf, 64-RHS tile) a dense product Y = D_panel Xg on the
//     tensor cores (mma.sync m16n8k16 BF16 or m16n8k8 TF32, FP32 accumulate):
//     M = the leaf's rows (<= 64, four m16 tiles, one per warp), N = 64 RHS,
//     K = the panel width, staged through shared memory in chunks;
//   B + M: CSR rows in FP32 (thread per (row, rhs));
//   far field: per-level projections, node sums, coupling, expansion, all on
//     FP32 CUDA cores (small GEMMs).
#include <cuda_bf16.h>

#include <algorithm>

#include "device_common.cuh"

namespace vfd {

namespace {

constexpr int RT = 64;   // RHS per tile

template <class T>
struct MmaTraits;

// BF16: m16n8k16, operands packed two per 32-bit register
template <>
struct MmaTraits<__nv_bfloat16> {
    static constexpr int KS = 16;
    __device__ static void mma(float *c, const uint32_t *a, const uint32_t *b)
    {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
};

// TF32: m16n8k8, one operand per 32-bit register (FP32 storage, rounded to TF32)
template <>
struct MmaTraits<float> {
    static constexpr int KS = 8;
    __device__ static void mma(float *c, const uint32_t *a, const uint32_t *b)
    {
        asm volatile(
            "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};\n"
            : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
};

__device__ __forceinline__ uint32_t f2tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

template <class T>
__device__ __forceinline__ T from_f(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ float from_f<float>(float v) { return __uint_as_float(f2tf32(v)); }

}  // namespace

// ---------------------------------------------------------------------------
// near panels on the tensor cores.  CTA = (leaf, 64-RHS tile), 8 warps; warp
// w owns rows 16 (w & 3) .. +15 of the leaf and RHS 32 (w >> 2) .. +31 (four
// n8 tiles).  The panel is consumed in chunks of NK columns through an
// NSTAGE-deep cp.async pipeline:
//   As[stage][64][LDA]  panel rows (T, as stored: FP32 or BF16), zero-filled
//                       beyond the leaf's rows and the panel width;
//   Bs[stage][NK][LDB]  gathered x rows X[gcol[k]][rt .. rt+63] (FP32),
//                       zero-filled for the padding columns (gcol = -1).
// The gather indices of the whole panel are staged in shared memory first.
// A fragments come from ldmatrix, B fragments from two shared loads; FP32
// values are rounded to TF32 (cvt.rna), B values packed to BF16x2 (cvt.rn).
// Rounding to nearest matters: truncation (what the tensor core does with raw
// FP32 bits) biases the low-precision operator, and the refinement then
// needed about twice the inner iterations.  The
// panel's chunks are split over KSPLIT CTAs (blockIdx.z); CTA z writes its
// partial product to Y (z = 0) or Y2 (z = 1), summed by the CSR kernel.
// ---------------------------------------------------------------------------
constexpr int NK = 32;       // panel columns per stage
constexpr int NSTAGE = 3;    // pipeline depth
constexpr int KSPLIT = 2;    // CTAs per (leaf, RHS tile), each a contiguous range of chunks
constexpr int NEAR_THREADS = 256;

template <class T>
struct NearTile {
    static constexpr int LDA = NK + (sizeof(T) == 2 ? 8 : 4);   // A row stride (elements): conflict-free fragments
    static constexpr int LDB = RT + (sizeof(T) == 2 ? 4 : 8);   // B row stride (floats)
    static constexpr int A_BYTES = 64 * LDA * (int)sizeof(T);
    static constexpr int B_BYTES = NK * LDB * 4;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int A_CHUNKS = 64 * NK * (int)sizeof(T) / 16;   // 16-byte copies per stage
    static constexpr int B_CHUNKS = NK * RT * 4 / 16;
    static_assert(A_BYTES % 16 == 0 && B_BYTES % 16 == 0 && (LDA * sizeof(T)) % 16 == 0 && (LDB * 4) % 16 == 0,
                  "16-byte aligned rows");
};

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;   // 0: the 16 bytes are zero-filled, nothing is read
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t *r, const void *smem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    uint32_t r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

template <class T>
__global__ void __launch_bounds__(NEAR_THREADS)
k_mr_near(int fl, int R, const int *__restrict__ kb, const int *__restrict__ ke, const int *__restrict__ pw,
          const int64_t *__restrict__ poff, const int *__restrict__ gcol, const int *__restrict__ goff,
          const T *__restrict__ D, const float *__restrict__ X, float *__restrict__ Y, float *__restrict__ Y2,
          const int *skip)
{
    using TT = NearTile<T>;
    extern __shared__ __align__(16) unsigned char smem[];
    if (skip && *skip) return;
    const int lf = blockIdx.x, rt = blockIdx.y * RT;
    const int b0 = kb[fl + lf], na = ke[fl + lf] - b0;
    const int W = pw[lf];   // multiple of 8
    const T *Dp = D + poff[lf];
    int *gs = (int *)(smem + NSTAGE * TT::STAGE_BYTES);
    for (int c = threadIdx.x; c < W; c += NEAR_THREADS) gs[c] = gcol[goff[lf] + c];
    __syncthreads();

    auto load_stage = [&](int slot, int chunk) {
        const int k0 = chunk * NK;
        T *As = (T *)(smem + slot * TT::STAGE_BYTES);
        float *Bs = (float *)(smem + slot * TT::STAGE_BYTES + TT::A_BYTES);
        constexpr int EPC = 16 / (int)sizeof(T);   // elements per 16-byte copy
        for (int c = threadIdx.x; c < TT::A_CHUNKS; c += NEAR_THREADS) {
            const int row = c / (NK / EPC), q = c - row * (NK / EPC), col = k0 + q * EPC;
            const bool ok = row < na && col < W;
            cp_async16(As + row * TT::LDA + q * EPC, ok ? (const void *)(Dp + (size_t)row * W + col) : (const void *)D,
                       ok);
        }
        for (int c = threadIdx.x; c < TT::B_CHUNKS; c += NEAR_THREADS) {
            const int kr = c / (RT / 4), q = c - kr * (RT / 4), col = k0 + kr;
            const int j = col < W ? gs[col] : -1;
            cp_async16(Bs + kr * TT::LDB + q * 4, j >= 0 ? (const void *)(X + (size_t)j * R + rt + q * 4) : (const void *)X,
                       j >= 0);
        }
    };

    const int nkt = (W + NK - 1) / NK;
    const int kc0 = (int)(((long long)nkt * blockIdx.z) / KSPLIT), nk = (int)(((long long)nkt * (blockIdx.z + 1)) / KSPLIT) - kc0;
    for (int s = 0; s < NSTAGE - 1; ++s) {
        if (s < nk) load_stage(s, kc0 + s);
        cp_async_commit();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
    const int r0 = (warp & 3) * 16, n0 = (warp >> 2) * 32;
    const bool active = r0 < na;
    float acc[4][4];
    for (int j = 0; j < 4; ++j)
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
    for (int kt = 0; kt < nk; ++kt) {
        cp_async_wait<NSTAGE - 2>();
        __syncthreads();   // stage kt landed for every thread; stage kt-1 fully consumed
        if (kt + NSTAGE - 1 < nk) load_stage((kt + NSTAGE - 1) % NSTAGE, kc0 + kt + NSTAGE - 1);
        cp_async_commit();
        if (!active) continue;
        const T *As = (const T *)(smem + (kt % NSTAGE) * TT::STAGE_BYTES);
        const float *Bs = (const float *)(smem + (kt % NSTAGE) * TT::STAGE_BYTES + TT::A_BYTES);
        constexpr int KS = MmaTraits<T>::KS;
#pragma unroll
        for (int ks = 0; ks < NK; ks += KS) {
            uint32_t a[4];
            {
                // lanes 8m..8m+7 address the rows of 8x16-byte matrix m: rows +8 for m odd, columns +16 bytes for m >= 2
                const int m = lane >> 3, rr = lane & 7;
                ldmatrix_x4(a, As + (r0 + rr + (m & 1) * 8) * TT::LDA + ks + (m >> 1) * (16 / (int)sizeof(T)));
                if constexpr (sizeof(T) == 4)
                    for (int q = 0; q < 4; ++q) a[q] = f2tf32(__uint_as_float(a[q]));
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = n0 + j * 8 + g;
                uint32_t bb[2];
                if constexpr (sizeof(T) == 2) {
                    const float *B0 = Bs + (ks + 2 * t4) * TT::LDB + n;
                    bb[0] = pack_bf16x2(B0[0], B0[TT::LDB]);
                    bb[1] = pack_bf16x2(B0[8 * TT::LDB], B0[9 * TT::LDB]);
                } else {
                    const float *B0 = Bs + (ks + t4) * TT::LDB + n;
                    bb[0] = f2tf32(B0[0]);
                    bb[1] = f2tf32(B0[4 * TT::LDB]);
                }
                MmaTraits<T>::mma(acc[j], a, bb);
            }
        }
    }
    cp_async_wait<0>();
    if (!active) return;
    float *Yo = blockIdx.z == 0 ? Y : Y2;
    for (int j = 0; j < 4; ++j) {
        const int col = rt + n0 + j * 8 + 2 * t4;
        const int ra = r0 + g, rb = r0 + g + 8;
        if (ra < na) *(float2 *)(Yo + (size_t)(b0 + ra) * R + col) = make_float2(acc[j][0], acc[j][1]);
        if (rb < na) *(float2 *)(Yo + (size_t)(b0 + rb) * R + col) = make_float2(acc[j][2], acc[j][3]);
    }
}

template <class T>
static size_t near_smem_bytes(const MeshData &m)
{
    return (size_t)NSTAGE * NearTile<T>::STAGE_BYTES + (size_t)m.max_panel_w * sizeof(int);
}

// Y[i][r..r+3] = (Y + Y2)[i][r..r+3] + sum_c val[c] X[col c][r..r+3]   (B + M
// in FP32 added to the two partial near products; thread per (row, 4 RHS);
// accumulate = 0: no near products)
__global__ void k_mr_csr(int N, int R, int accumulate, const int *__restrict__ rowptr, const int *__restrict__ colidx,
                         const float *__restrict__ val, const float *__restrict__ X, float *__restrict__ Y,
                         const float *__restrict__ Y2, const int *skip)
{
    if (skip && *skip) return;
    const int R4 = R >> 2;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * R4) return;
    const int i = (int)(t / R4), q = (int)(t % R4);
    const float4 *X4 = (const float4 *)X;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (accumulate) {
        const float4 a = ((const float4 *)Y)[t], b = ((const float4 *)Y2)[t];
        acc = make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
    }
    for (int c = rowptr[i]; c < rowptr[i + 1]; ++c) {
        const float v = val[c];
        const float4 x = X4[(size_t)colidx[c] * R4 + q];
        acc.x = fmaf(v, x.x, acc.x);
        acc.y = fmaf(v, x.y, acc.y);
        acc.z = fmaf(v, x.z, acc.z);
        acc.w = fmaf(v, x.w, acc.w);
    }
    ((float4 *)Y)[t] = acc;
}

__device__ __forceinline__ void fma4(float4 &acc, float u, const float4 x)
{
    acc.x = fmaf(u, x.x, acc.x);
    acc.y = fmaf(u, x.y, acc.y);
    acc.z = fmaf(u, x.z, acc.z);
    acc.w = fmaf(u, x.w, acc.w);
}

// far field, R RHS in tiles of 64 (FP32 accumulation; T the stored basis /
// coupling type).  Thread micro-tiles of 4 outputs x 4 RHS (float4 over RHS).
//
// projections: part[lv][leaf][a][r] = sum_{i in leaf} Ul[lv][i][a] X[i][r].
// CTA (256 threads) per (leaf, RHS tile): the leaf's x rows and its basis rows
// of every level (Us[i][lva], lva = lv*k + a) staged in shared memory; thread
// (r-quad = t % 16, g = t / 16) computes lva = c*64 + g + 16 q (q < 4), chunk
// by chunk.
template <class T>
__global__ void __launch_bounds__(256)
k_mr_far_proj(int fl, int k, int nlev, int N, int R, const int *__restrict__ kb, const int *__restrict__ ke,
              const T *__restrict__ Ul, const float *__restrict__ X, float *__restrict__ part, int nleaf,
              const int *skip)
{
    __shared__ float4 Xs[64][RT / 4];
    extern __shared__ float Us[];   // [n][nlev * k]
    if (skip && *skip) return;
    const int leaf = blockIdx.x, rt = blockIdx.y * RT;
    const int b = kb[fl + leaf], n = ke[fl + leaf] - b;
    const int R4 = R >> 2, NL = nlev * k;
    for (int e = threadIdx.x; e < n * (RT / 4); e += blockDim.x) {
        const int i = e / (RT / 4), q = e % (RT / 4);
        Xs[i][q] = ((const float4 *)X)[(size_t)(b + i) * R4 + (rt >> 2) + q];
    }
    for (int e = threadIdx.x; e < nlev * n * k; e += blockDim.x) {
        const int l = e / (n * k), r = e - l * n * k, i = r / k, al = r - i * k;
        Us[i * NL + l * k + al] = (float)Ul[((size_t)l * N + b) * k + r];
    }
    __syncthreads();
    const int rq = threadIdx.x & 15, g = threadIdx.x >> 4;
    for (int c0 = 0; c0 < NL; c0 += 64) {
        float4 acc[4];
        int lva[4];
        for (int q = 0; q < 4; ++q) {
            acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            lva[q] = min(c0 + g + 16 * q, NL - 1);
        }
#pragma unroll 4
        for (int i = 0; i < n; ++i) {
            const float4 x = Xs[i][rq];
#pragma unroll
            for (int q = 0; q < 4; ++q) fma4(acc[q], Us[i * NL + lva[q]], x);
        }
        for (int q = 0; q < 4; ++q) {
            const int v = c0 + g + 16 * q;
            if (v < NL) {
                const int l = v / k, al = v % k;
                ((float4 *)part)[((((size_t)l * nleaf + leaf) * k + al) * R + rt) / 4 + rq] = acc[q];
            }
        }
    }
}

// xhat[node][a][r] = sum over the node's leaves of part (levels lmin..L)
__global__ void k_mr_far_sum(int lmin, int L, int k, int R, int nleaf, const float *__restrict__ part,
                             float *__restrict__ xhat, const int *skip)
{
    if (skip && *skip) return;
    const int node = (1 << lmin) - 1 + blockIdx.x;
    const int t = blockIdx.y * blockDim.x + threadIdx.x;
    if (t >= k * R / 4) return;
    int l = 0;
    while ((2 << l) - 1 <= node) ++l;
    const int span = 1 << (L - l), leaf0 = ((node + 1) << (L - l)) - 1 - ((1 << L) - 1);
    const float4 *p = (const float4 *)part + (((size_t)(l - lmin) * nleaf + leaf0) * k * R) / 4 + t;
    // eight independent partial sums (loads in flight together), combined in a fixed order
    float4 s[8];
    for (int q = 0; q < 8; ++q) s[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    const size_t stride = (size_t)k * R / 4;
    for (int j0 = 0; j0 < span; j0 += 8) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (j0 + q < span) {
                const float4 v = p[(size_t)(j0 + q) * stride];
                s[q].x += v.x;
                s[q].y += v.y;
                s[q].z += v.z;
                s[q].w += v.w;
            }
    }
    for (int q = 1; q < 8; ++q) {
        s[0].x += s[q].x;
        s[0].y += s[q].y;
        s[0].z += s[q].z;
        s[0].w += s[q].w;
    }
    ((float4 *)xhat)[(size_t)node * k * R / 4 + t] = s[0];
}

// coupling: yhat[node][a][r] = sum_e sum_b S_e[b][a] xhat[col e][b][r].
// CTA (64 threads) per (node, RHS tile); groups of EPS blocks S_e with their
// column nodes' xhat rows pass through a two-stage cp.async pipeline in
// shared memory; thread (r-quad = t % 16, g = t / 16) computes a = c*16 + g +
// 4 q (q < 4), chunk by chunk.
constexpr int EPS = 4;   // coupling blocks per pipeline stage

template <class T>
__host__ __device__ constexpr int couple_sbytes(int k)
{
    return (k * k * (int)sizeof(T) + 15) & ~15;
}

template <class T>
__global__ void __launch_bounds__(64)
k_mr_far_couple(int k, int R, const int *__restrict__ fptr, const int *__restrict__ fcol, const T *__restrict__ S,
                const float *__restrict__ xhat, float *__restrict__ yhat, const int *skip)
{
    extern __shared__ __align__(16) unsigned char csm[];
    if (skip && *skip) return;
    const int node = blockIdx.x, rt = blockIdx.y * RT;
    const int rq = threadIdx.x & 15, g = threadIdx.x >> 4;
    const int R4 = R >> 2;
    const int sbytes = couple_sbytes<T>(k), xbytes = k * RT * 4, slot_bytes = EPS * (sbytes + xbytes);
    const int e0 = fptr[node], ne = fptr[node + 1] - e0, ng = (ne + EPS - 1) / EPS;
    auto stage = [&](int slot, int grp) {
        for (int j = 0; j < EPS && grp * EPS + j < ne; ++j) {
            const int e = e0 + grp * EPS + j;
            unsigned char *base = csm + slot * slot_bytes + j * (sbytes + xbytes);
            const unsigned char *sg = (const unsigned char *)(S + (size_t)e * k * k);
            const int sb = k * k * (int)sizeof(T);
            // S_e: 16-byte copies where the block is 16-byte aligned, else 4-byte words
            if ((((size_t)sg) & 15) == 0 && (sb & 15) == 0) {
                for (int c = threadIdx.x; c < sb / 16; c += blockDim.x) cp_async16(base + 16 * c, sg + 16 * c, true);
            } else {
                for (int c = threadIdx.x; c < sb / 4; c += blockDim.x) ((uint32_t *)base)[c] = ((const uint32_t *)sg)[c];
            }
            const float *xg = xhat + (size_t)fcol[e] * k * R + rt;
            for (int c = threadIdx.x; c < k * (RT / 4); c += blockDim.x) {
                const int be = c / (RT / 4), q = c - be * (RT / 4);
                cp_async16(base + sbytes + 16 * c, xg + (size_t)be * R + 4 * q, true);
            }
        }
    };
    for (int c0 = 0; c0 < k; c0 += 16) {
        float4 acc[4];
        for (int q = 0; q < 4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ng > 0) stage(0, 0);
        cp_async_commit();
        for (int gi = 0; gi < ng; ++gi) {
            if (gi + 1 < ng) stage((gi + 1) & 1, gi + 1);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            for (int j = 0; j < EPS && gi * EPS + j < ne; ++j) {
                const unsigned char *base = csm + (gi & 1) * slot_bytes + j * (sbytes + xbytes);
                const T *Ss = (const T *)base;
                const float4 *Xs = (const float4 *)(base + sbytes);
                for (int be = 0; be < k; ++be) {
                    const float4 x = Xs[be * (RT / 4) + rq];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int al = c0 + g + 4 * q;
                        if (al < k) fma4(acc[q], (float)Ss[be * k + al], x);
                    }
                }
            }
            __syncthreads();   // the slot is refilled two steps later
        }
        cp_async_wait<0>();
        for (int q = 0; q < 4; ++q) {
            const int al = c0 + g + 4 * q;
            if (al < k) ((float4 *)yhat)[((size_t)node * k + al) * R4 + (rt >> 2) + rq] = acc[q];
        }
    }
}

// expansion: Y[i][r] += sum_l sum_a Ul[l][i][a] yhat[ancestor_l(i)][a][r].
// CTA (256 threads) per (leaf, RHS tile): the ancestors' yhat rows (nlev*k
// rows of 64 floats) and the leaf's basis rows Us[lva][i] staged in shared
// memory; thread (r-quad = t % 16, g = t / 16) owns rows g + 16 q (q < 4).
template <class T>
__global__ void __launch_bounds__(256)
k_mr_far_expand(int fl, int lmin, int L, int k, int N, int R, const int *__restrict__ kb, const int *__restrict__ ke,
                const T *__restrict__ Ul, const float *__restrict__ yhat, float *__restrict__ Y, const int *skip)
{
    extern __shared__ float4 Ys[];   // [nlev * k][16], then Us[nlev * k][64] (floats)
    if (skip && *skip) return;
    const int leaf = blockIdx.x, rt = blockIdx.y * RT;
    const int b = kb[fl + leaf], n = ke[fl + leaf] - b;
    const int nlev = L - lmin + 1, NL = nlev * k, R4 = R >> 2;
    float *Us = (float *)(Ys + NL * 16);
    for (int e = threadIdx.x; e < NL * 16; e += blockDim.x) {
        const int row = e >> 4, q = e & 15, l = lmin + row / k, al = row % k;
        const int node = ((fl + leaf + 1) >> (L - l)) - 1;
        Ys[e] = ((const float4 *)yhat)[((size_t)node * k + al) * R4 + (rt >> 2) + q];
    }
    for (int e = threadIdx.x; e < nlev * n * k; e += blockDim.x) {
        const int l = e / (n * k), r = e - l * n * k, i = r / k, al = r - i * k;
        Us[(l * k + al) * 64 + i] = (float)Ul[((size_t)l * N + b) * k + r];
    }
    __syncthreads();
    const int rq = threadIdx.x & 15, g = threadIdx.x >> 4;
    float4 acc[4];
    for (int q = 0; q < 4; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int lva = 0; lva < NL; ++lva) {
        const float4 y = Ys[lva * 16 + rq];
        const float *u = Us + lva * 64 + g;
#pragma unroll
        for (int q = 0; q < 4; ++q) fma4(acc[q], u[16 * q], y);
    }
    for (int q = 0; q < 4; ++q) {
        const int i = g + 16 * q;
        if (i < n) {
            float4 *yp = (float4 *)Y + (size_t)(b + i) * R4 + (rt >> 2) + rq;
            float4 v = *yp;
            v.x += acc[q].x;
            v.y += acc[q].y;
            v.z += acc[q].z;
            v.w += acc[q].w;
            *yp = v;
        }
    }
}

// ---------------------------------------------------------------------------
void release_bgraph(OpData &op);

template <class T>
static void mr_apply_impl(const MeshData &m, OpData &op, const float *X, float *Y, int R, const T *D, const T *Ul,
                          const T *S, cudaStream_t st, const int *skip)
{
    const int fl = m.kt.first_leaf(), k = m.k, N = m.N;
    const bool far = m.nfar > 0;
    const int nlev = far ? m.kt.L - m.far_lmin + 1 : 0;
    if (m.nnear > 0) {
        if (op.mr_y2.n < (size_t)N * R) {
            release_bgraph(op);   // a captured solve refers to the old workspace
            op.mr_y2.alloc((size_t)N * R);
        }
        const size_t shm = near_smem_bytes<T>(m);
        VFD_CUDA(cudaFuncSetAttribute(k_mr_near<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        dim3 g(m.kt.nleaf, R / RT, KSPLIT);
        k_mr_near<T><<<g, NEAR_THREADS, shm, st>>>(fl, R, m.kt_begin.p, m.kt_end.p, m.panel_w.p, m.panel_off.p,
                                                   m.gcol.p, m.gcol_off.p, D, X, Y, op.mr_y2.p, skip);
    }
    k_mr_csr<<<cdiv((long long)N * (R / 4), 256), 256, 0, st>>>(N, R, m.nnear > 0 ? 1 : 0, m.rowptr.p, m.colidx.p,
                                                                 op.valBM32.p, X, Y, op.mr_y2.p, skip);
    if (far) {
        const size_t need_p = (size_t)nlev * m.kt.nleaf * k * R, need_h = (size_t)m.kt.nnode * k * R;
        if (op.mr_part.n < need_p || op.mr_xh.n < need_h) {
            release_bgraph(op);   // a captured solve refers to the old workspace
            op.mr_part.alloc(need_p);
            op.mr_xh.alloc(need_h);
            op.mr_yh.alloc(need_h);
        }
        dim3 gp(m.kt.nleaf, R / RT);
        const size_t pshm = (size_t)m.max_leaf_size * nlev * k * sizeof(float);
        VFD_CUDA(cudaFuncSetAttribute(k_mr_far_proj<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pshm));
        k_mr_far_proj<T><<<gp, 256, pshm, st>>>(fl, k, nlev, N, R, m.kt_begin.p, m.kt_end.p, Ul, X, op.mr_part.p,
                                                m.kt.nleaf, skip);
        const int nn = m.kt.nnode - ((1 << m.far_lmin) - 1);
        dim3 gs(nn, cdiv(k * R / 4, 128));
        k_mr_far_sum<<<gs, 128, 0, st>>>(m.far_lmin, m.kt.L, k, R, m.kt.nleaf, op.mr_part.p, op.mr_xh.p, skip);
        dim3 gc(m.kt.nnode, R / RT);
        const size_t cshm = 2 * EPS * ((size_t)couple_sbytes<T>(k) + (size_t)k * RT * sizeof(float));
        VFD_CUDA(cudaFuncSetAttribute(k_mr_far_couple<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cshm));
        k_mr_far_couple<T><<<gc, 64, cshm, st>>>(k, R, m.far_ptr.p, m.far_col.p, S, op.mr_xh.p, op.mr_yh.p, skip);
        const size_t eshm = (size_t)nlev * k * (RT + 64) * sizeof(float);
        VFD_CUDA(cudaFuncSetAttribute(k_mr_far_expand<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eshm));
        dim3 ge(m.kt.nleaf, R / RT);
        k_mr_far_expand<T><<<ge, 256, eshm, st>>>(fl, m.far_lmin, m.kt.L, k, N, R, m.kt_begin.p, m.kt_end.p, Ul,
                                                  op.mr_yh.p, Y, skip);
    }
    VFD_CUDA(cudaGetLastError());
}

// Y = A_low X for R (multiple of 64) interleaved FP32 columns
void mr_apply(const MeshData &m, OpData &op, const float *X, float *Y, int R, cudaStream_t st, const int *skip)
{
    VFD_REQUIRE(R % RT == 0, VFD_EINVAL, "batched apply needs a multiple of 64 columns");
    VFD_REQUIRE(m.max_leaf_size <= 64, VFD_EUNSUPPORTED, "batched apply needs leaves of at most 64 DoFs");
    VFD_REQUIRE(near_smem_bytes<float>(m) <= 227 * 1024, VFD_EUNSUPPORTED, "batched apply: near panel too wide");
    VFD_REQUIRE(2 * EPS * ((size_t)couple_sbytes<float>(m.k) + (size_t)m.k * RT * sizeof(float)) <= 227 * 1024,
                VFD_EUNSUPPORTED, "batched apply: rank too large for the coupling tile");
    VFD_REQUIRE(m.nfar == 0 || (size_t)(m.kt.L - m.far_lmin + 1) * m.k * (RT + 64) * sizeof(float) <= 227 * 1024,
                VFD_EUNSUPPORTED, "batched apply: too many far levels x rank for the expansion tile");
    VFD_REQUIRE(m.nfar == 0 || (size_t)m.max_leaf_size * (m.kt.L - m.far_lmin + 1) * m.k * sizeof(float) +
                                       64 * RT * sizeof(float) <= 227 * 1024,
                VFD_EUNSUPPORTED, "batched apply: too many far levels x rank for the projection tile");
    if (op.precision == VFD_BF16)
        mr_apply_impl<__nv_bfloat16>(m, op, X, Y, R, (const __nv_bfloat16 *)op.D16.p,
                                     (const __nv_bfloat16 *)op.Ul16.p, (const __nv_bfloat16 *)op.S16.p, st, skip);
    else
        mr_apply_impl<float>(m, op, X, Y, R, op.D32.p, op.Ul32.p, op.S32.p, st, skip);
}

// column-major FP64 <-> interleaved FP32
__global__ void k_cm_to_il(int N, int R, int64_t ld, const double *__restrict__ X, float *__restrict__ Xi)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * R) return;
    const int i = (int)(t / R), r = (int)(t % R);
    Xi[t] = (float)X[(size_t)r * ld + i];
}

__global__ void k_il_to_cm(int N, int R, int64_t ld, const float *__restrict__ Yi, double *__restrict__ Y)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * R) return;
    const int r = (int)(t / N), i = (int)(t % N);
    Y[(size_t)r * ld + i] = (double)Yi[(size_t)i * R + r];
}

// Y = A_low X for column-major FP64 blocks (nrhs a multiple of 64)
void mr_apply_colmajor(const MeshData &m, OpData &op, const double *X, double *Y, int nrhs, int64_t ld,
                       cudaStream_t st)
{
    const size_t n = (size_t)m.N * nrhs;
    if (op.mr_xi.n < n) {
        op.mr_xi.alloc(n);
        op.mr_yi.alloc(n);
    }
    k_cm_to_il<<<cdiv((long long)n, 256), 256, 0, st>>>(m.N, nrhs, ld, X, op.mr_xi.p);
    mr_apply(m, op, op.mr_xi.p, op.mr_yi.p, nrhs, st, nullptr);
    k_il_to_cm<<<cdiv((long long)n, 256), 256, 0, st>>>(m.N, nrhs, ld, op.mr_yi.p, Y);
    VFD_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// BF16 copies of the K data (VFD_BF16 operators)
// ---------------------------------------------------------------------------
__global__ void k_to_bf16(long long n, const double *__restrict__ a, __nv_bfloat16 *__restrict__ b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __double2bfloat16(a[i]);
}

static void to16(const DBuf<double> &a, DBuf<unsigned short> &b, cudaStream_t st)
{
    b.alloc(a.n);
    if (a.n) k_to_bf16<<<cdiv((long long)a.n, 256), 256, 0, st>>>((long long)a.n, a.p, (__nv_bfloat16 *)b.p);
    VFD_CUDA(cudaGetLastError());
}

__global__ void k_d2f(long long n, const double *__restrict__ a, float *__restrict__ b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

void launch_convert_bf16(const MeshData &m, OpData &op, cudaStream_t st)
{
    to16(op.S64, op.S16, st);
    to16(op.D64, op.D16, st);
    to16(m.Ul64, op.Ul16, st);
}

void launch_lowp_csr(const MeshData &m, OpData &op, cudaStream_t st)
{
    op.valBM32.alloc(m.nnz);
    if (m.nnz) k_d2f<<<cdiv(m.nnz, 256), 256, 0, st>>>(m.nnz, op.valBM.p, op.valBM32.p);
    VFD_CUDA(cudaGetLastError());
}

}  // namespace vfd
