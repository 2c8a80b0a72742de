// Batched multi-RHS apply of the low-precision operator (the inner operator
// of iterative refinement) for R right-hand sides at once, R a multiple of 64,
// over a batch of operators (meshes) in one launch per stage: every kernel
// walks a global queue of work items (mesh, leaf) or (mesh, node) and reads
// the mesh's pointers and sizes from a device table of descriptors.  A
// single operator is a batch of one.
// Vectors are FP32 in the interleaved layout X[i][r] (DoF-major, RHS
// contiguous; the meshes' rows one after another), so every gather of one
// DoF's entries is one contiguous read.
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
#include <cstring>

#include "batched.cuh"

namespace vfd {

namespace {

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


}  // namespace

// ---------------------------------------------------------------------------
// near panels on the tensor cores.  CTA = (leaf, 64-RHS tile), 8 warps; warp
// w owns rows 16 (w & 3) .. +15 of the leaf and RHS 32 (w >> 2) .. +31 (four
// n8 tiles).  The panel is consumed in chunks of NK columns through an
// NSTAGE-deep cp.async pipeline:
//   As[stage][64][LDA]  panel rows (T, as stored: FP32 or BF16), zero-filled
//                       beyond the leaf's rows and the panel width;
//   Bs[stage]           gathered x rows X[gcol[k]][rt .. rt+63], zero-filled
//                       for the padding columns (gcol = -1): FP32 for TF32
//                       panels, the BF16 hi and lo rows for BF16 panels.
// The gather indices of the whole panel are staged in shared memory first.
// A fragments come from ldmatrix (FP32 panels are stored pre-rounded to
// TF32 for this kernel); B fragments from two shared loads rounded to TF32
// (cvt.rna), or for BF16 from ldmatrix.trans of the hi and lo rows (rounded
// to nearest once per apply).  Rounding to nearest matters: truncation (what
// the tensor core does with raw FP32 bits) biases the low-precision
// operator, and the refinement then needed about twice the inner
// iterations.  x enters as two terms, hi = round(x) and lo = round(x - hi),
// each multiplied by the panel (twice the MMAs): the panel's own rounding is
// a fixed perturbation of the operator (its row sums are compensated), but
// rounding x anew in every apply adds noise of the unit roundoff relative to
// each entry of x, and for the smooth directions of the preconditioned
// iteration that noise is larger than A x itself (the inner iteration on
// one 21k-DoF mesh took 1253 BF16 steps instead of 39).  The panel's chunks
// are split over gridDim.z CTAs; CTA z writes its partial product to Y (z =
// 0) or to partial buffer z - 1 of Y2, summed by the CSR kernel.  The stage
// width NK, the depth NSTAGE and the split are picked per batch by timing
// the candidates (near_configs).
// ---------------------------------------------------------------------------
constexpr int KSPLIT_MAX = 4;

// B tiles: TF32 panels take x in FP32 ([NK][LDB] floats, split at fragment
// time); BF16 panels take the hi and lo BF16 blocks of x made once per apply
// ([2][NK][LDB] BF16, hi then lo), read with ldmatrix.trans
template <class T, int NK>
struct NearTile {
    static constexpr bool BF = sizeof(T) == 2;
    static constexpr int LDA = NK + (BF ? 8 : 4);      // A row stride (elements): conflict-free fragments
    static constexpr int LDB = RT + 8;                  // B row stride (elements: BF16 or floats)
    static constexpr int B_ELEM = BF ? 2 : 4;
    static constexpr int A_BYTES = 64 * LDA * (int)sizeof(T);
    static constexpr int B_BYTES = (BF ? 2 : 1) * NK * LDB * B_ELEM;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int A_CHUNKS = 64 * NK * (int)sizeof(T) / 16;   // 16-byte copies per stage
    static constexpr int B_CPR = RT * B_ELEM / 16;                   // 16-byte copies per x row
    static constexpr int B_CHUNKS = (BF ? 2 : 1) * NK * B_CPR;
    static_assert(A_BYTES % 16 == 0 && B_BYTES % 16 == 0 && (LDA * sizeof(T)) % 16 == 0 && (LDB * B_ELEM) % 16 == 0,
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

__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t *r, const void *smem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t *r, const void *smem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(s));
}


// WARPS = 8: warp tile 16 rows x 32 RHS; WARPS = 4: 32 rows x 32 RHS (two m16
// tiles share each B fragment).  NACC = 2: even and odd k-steps accumulate
// into separate registers (twice the independent mma chains), summed at the end.
template <class T, int NK, int NSTAGE, int WARPS, int NACC>
__global__ void __launch_bounds__(WARPS * 32)
k_mr_near(const NearItem *__restrict__ items, int R, const float *__restrict__ Xall,
          const __nv_bfloat16 *__restrict__ Xc, size_t xlo, float *__restrict__ Yall, float *__restrict__ Y2all,
          size_t pstride, const int *skip, const int *mdone)
{
    using TT = NearTile<T, NK>;
    constexpr int NEAR_THREADS = WARPS * 32, MT = 8 / WARPS, RW = 4 / MT;   // m16 tiles per warp, warps per row band
    extern __shared__ __align__(16) unsigned char smem[];
    if (skip && *skip) return;
    const NearItem it = items[blockIdx.x];
    if (mdone && mdone[it.mesh]) return;
    const int rt = blockIdx.y * RT;
    const float *__restrict__ X = Xall + (size_t)it.xoff * R;   // gather columns are mesh-local rows
    float *__restrict__ Y = Yall;
    float *__restrict__ Y2 = Y2all;
    const T *__restrict__ Dp = (const T *)it.D;
    const T *__restrict__ D = Dp;
    const int b0 = it.row0, na = it.na, W = it.W;
    int *gs = (int *)(smem + NSTAGE * TT::STAGE_BYTES);
    const int *gcol = it.gcol;
    for (int c = threadIdx.x; c < W; c += NEAR_THREADS) gs[c] = gcol[c];
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
        if constexpr (TT::BF) {
            // hi rows [0, NK), lo rows [NK, 2 NK) of the stage's x tile
            __nv_bfloat16 *B16 = (__nv_bfloat16 *)Bs;
            for (int c = threadIdx.x; c < TT::B_CHUNKS; c += NEAR_THREADS) {
                const int hr = c / TT::B_CPR, q = c - hr * TT::B_CPR, h = hr / NK, kr = hr - h * NK, col = k0 + kr;
                const int j = col < W ? gs[col] : -1;
                const __nv_bfloat16 *src = Xc + (size_t)h * xlo + ((size_t)(it.xoff + j) * R + rt + q * 8);
                cp_async16(B16 + hr * TT::LDB + q * 8, j >= 0 ? (const void *)src : (const void *)Xc, j >= 0);
            }
        } else {
            for (int c = threadIdx.x; c < TT::B_CHUNKS; c += NEAR_THREADS) {
                const int kr = c / TT::B_CPR, q = c - kr * TT::B_CPR, col = k0 + kr;
                const int j = col < W ? gs[col] : -1;
                cp_async16(Bs + kr * TT::LDB + q * 4,
                           j >= 0 ? (const void *)(X + (size_t)j * R + rt + q * 4) : (const void *)X, j >= 0);
            }
        }
    };

    const int nkt = (W + NK - 1) / NK, ks = gridDim.z;
    const int kc0 = (int)(((long long)nkt * blockIdx.z) / ks), nk = (int)(((long long)nkt * (blockIdx.z + 1)) / ks) - kc0;
    for (int s = 0; s < NSTAGE - 1; ++s) {
        if (s < nk) load_stage(s, kc0 + s);
        cp_async_commit();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
    const int r0 = (warp % RW) * 16 * MT, n0 = (warp / RW) * 32;
    const bool active = r0 < na;
    float acc[NACC][MT][4][4];
    for (int h = 0; h < NACC; ++h)
        for (int mt = 0; mt < MT; ++mt)
            for (int j = 0; j < 4; ++j)
                for (int q = 0; q < 4; ++q) acc[h][mt][j][q] = 0.f;
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
            uint32_t a[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                // lanes 8m..8m+7 address the rows of 8x16-byte matrix m: rows +8 for m odd, columns +16 bytes for m >= 2
                const int m = lane >> 3, rr = lane & 7;
                ldmatrix_x4(a[mt], As + (r0 + 16 * mt + rr + (m & 1) * 8) * TT::LDA + ks + (m >> 1) * (16 / (int)sizeof(T)));
            }
            if constexpr (TT::BF) {
                // x = hi + lo, both BF16: the product sees x to ~2^-16 (one BF16
                // rounding of x alone errs by up to 2^-8 relative in every entry,
                // which swamps A x for the smooth directions of the
                // preconditioned iteration).  ldmatrix.trans: matrices (k 0-7 |
                // 8-15) x (n 0-7 | 8-15) of two n8 tiles give b0, b1 of each
                const __nv_bfloat16 *Bh = (const __nv_bfloat16 *)Bs, *Bl = Bh + NK * TT::LDB;
                const int brow = ks + (lane & 7) + ((lane >> 3) & 1) * 8, bcol = n0 + ((lane >> 4) & 1) * 8;
#pragma unroll
                for (int jp = 0; jp < 2; ++jp) {
                    uint32_t bh[4], bl[4];
                    ldmatrix_x4_trans(bh, Bh + brow * TT::LDB + bcol + 16 * jp);
                    ldmatrix_x4_trans(bl, Bl + brow * TT::LDB + bcol + 16 * jp);
#pragma unroll
                    for (int jj = 0; jj < 2; ++jj) {
                        const int j = 2 * jp + jj;
                        const uint32_t hi[2] = {bh[2 * jj], bh[2 * jj + 1]}, lo[2] = {bl[2 * jj], bl[2 * jj + 1]};
#pragma unroll
                        for (int mt = 0; mt < MT; ++mt)
                            if (r0 + 16 * mt < na) MmaTraits<T>::mma(acc[(ks / KS + 1) % NACC][mt][j], a[mt], lo);
#pragma unroll
                        for (int mt = 0; mt < MT; ++mt)
                            if (r0 + 16 * mt < na) MmaTraits<T>::mma(acc[(ks / KS) % NACC][mt][j], a[mt], hi);
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // the same split in TF32: x = hi + lo, both rounded to TF32
                    const float *B0 = Bs + (ks + t4) * TT::LDB + n0 + j * 8 + g;
                    const float x0 = B0[0], x1 = B0[4 * TT::LDB];
                    const uint32_t bb[2] = {f2tf32(x0), f2tf32(x1)};
                    const uint32_t bl[2] = {f2tf32(x0 - __uint_as_float(bb[0])), f2tf32(x1 - __uint_as_float(bb[1]))};
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
                        if (r0 + 16 * mt < na) MmaTraits<T>::mma(acc[(ks / KS + 1) % NACC][mt][j], a[mt], bl);
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt)
                        if (r0 + 16 * mt < na) MmaTraits<T>::mma(acc[(ks / KS) % NACC][mt][j], a[mt], bb);
                }
            }
        }
    }
    cp_async_wait<0>();
    if (!active) return;
    if constexpr (NACC == 2)
        for (int mt = 0; mt < MT; ++mt)
            for (int j = 0; j < 4; ++j)
                for (int q = 0; q < 4; ++q) acc[0][mt][j][q] += acc[1][mt][j][q];
    float *Yo = blockIdx.z == 0 ? Y : Y2 + (size_t)(blockIdx.z - 1) * pstride;
    for (int mt = 0; mt < MT; ++mt)
        for (int j = 0; j < 4; ++j) {
            const int col = rt + n0 + j * 8 + 2 * t4;
            const int ra = r0 + 16 * mt + g, rb = ra + 8;
            if (ra < na) *(float2 *)(Yo + (size_t)(b0 + ra) * R + col) = make_float2(acc[0][mt][j][0], acc[0][mt][j][1]);
            if (rb < na) *(float2 *)(Yo + (size_t)(b0 + rb) * R + col) = make_float2(acc[0][mt][j][2], acc[0][mt][j][3]);
        }
}

// x for the BF16 near kernels as two BF16 terms: b[i] = hi = BF16(x),
// b[n + i] = lo = BF16(x - hi)
__global__ void k_x_to_bf16(long long n, const float *__restrict__ a, __nv_bfloat16 *__restrict__ b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = a[i];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    b[i] = h;
    b[n + i] = __float2bfloat16_rn(v - __bfloat162float(h));
}

template <class T, int NK, int NSTAGE>
static size_t near_smem_bytes(int max_panel_w)
{
    return (size_t)NSTAGE * NearTile<T, NK>::STAGE_BYTES + (size_t)max_panel_w * sizeof(int);
}

// candidate tile configurations of the near-panel kernel
struct NearCfg {
    int nk, nstage, ksplit, warps, nacc, tc;   // tc = 1: TMA-fed tcgen05 kernel (near_tc.cu; BF16, B + M fused)
};
static const NearCfg kNearCfgs[] = {{32, 3, 2, 8, 1, 0}, {32, 3, 3, 8, 1, 0}, {16, 4, 3, 8, 1, 0},
                                    {64, 2, 2, 8, 1, 0}, {32, 3, 3, 4, 1, 0}, {16, 4, 3, 4, 1, 0},
                                    {32, 3, 2, 8, 2, 0}, {16, 4, 3, 8, 2, 0}, {16, 4, 3, 4, 2, 0},
                                    {64, 4, 1, 4, 1, 1}, {64, 4, 2, 4, 1, 1}, {64, 6, 1, 4, 1, 1},
                                    {64, 6, 2, 4, 1, 1}, {64, 3, 2, 4, 1, 1}, {64, 3, 3, 4, 1, 1},
                                    {64, 2, 1, 4, 1, 1}, {64, 2, 2, 4, 1, 1}, {64, 2, 3, 4, 1, 1}};
constexpr int kNearCfgCount = (int)(sizeof(kNearCfgs) / sizeof(kNearCfgs[0]));

template <class T, int NK, int NS, int WARPS, int NACC>
static bool launch_near_cfg(int ksplit, int n_items, int max_panel_w, const NearItem *items, int R, const float *X,
                            const __nv_bfloat16 *Xc, size_t xlo, float *Y, float *Y2, size_t pstride, cudaStream_t st,
                            const int *skip, const int *mdone)
{
    const size_t shm = near_smem_bytes<T, NK, NS>(max_panel_w);
    if (shm > 227 * 1024) return false;
    VFD_CUDA(cudaFuncSetAttribute(k_mr_near<T, NK, NS, WARPS, NACC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)shm));
    dim3 g(n_items, R / RT, ksplit);
    k_mr_near<T, NK, NS, WARPS, NACC><<<g, WARPS * 32, shm, st>>>(items, R, X, Xc, xlo, Y, Y2, pstride, skip, mdone);
    return true;
}

// launch configuration c of the mma.sync kernel (near products only); false
// if it does not fit in shared memory or c is a tcgen05 candidate
template <class T>
static bool launch_near(int c, int n_items, int max_panel_w, const NearItem *items, int R, const float *X,
                        const __nv_bfloat16 *Xc, size_t xlo, float *Y, float *Y2, size_t pstride, cudaStream_t st,
                        const int *skip, const int *mdone)
{
    const NearCfg &f = kNearCfgs[c];
    if (f.tc) return false;
#define VFD_NEAR_CASE(NKV, NSV, WV, AV)                                                                          \
    if (f.nk == NKV && f.nstage == NSV && f.warps == WV && f.nacc == AV)                                         \
        return launch_near_cfg<T, NKV, NSV, WV, AV>(f.ksplit, n_items, max_panel_w, items, R, X, Xc, xlo, Y, Y2, \
                                                    pstride, st, skip, mdone);
    VFD_NEAR_CASE(32, 3, 8, 1)
    VFD_NEAR_CASE(16, 4, 8, 1)
    VFD_NEAR_CASE(64, 2, 8, 1)
    VFD_NEAR_CASE(32, 3, 4, 1)
    VFD_NEAR_CASE(16, 4, 4, 1)
    VFD_NEAR_CASE(32, 3, 8, 2)
    VFD_NEAR_CASE(16, 4, 8, 2)
    VFD_NEAR_CASE(64, 2, 8, 2)
    VFD_NEAR_CASE(32, 3, 4, 2)
    VFD_NEAR_CASE(16, 4, 4, 2)
#undef VFD_NEAR_CASE
    return false;
}

// Y[i][r..r+3] = (Y + sum_z Y2_z)[i][r..r+3] + the rest of row i of A times X:
// the partial products of a split panel plus, per mesh, either the B + M CSR
// row (FP32) or, where B + M off the diagonal is folded into the panels, the
// diagonal term diag_i X[i]; thread per (row, 4 RHS)
__global__ void k_mr_rows(const MrMesh *__restrict__ ms, const long long *__restrict__ row_off, int nmesh,
                          long long ntot, int R, const float *__restrict__ Xall, float *__restrict__ Yall,
                          const float *__restrict__ Y2all, int nparts, const int *skip, const int *mdone)
{
    if (skip && *skip) return;
    const int R4 = R >> 2;
    long long tg = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tg >= ntot * R4) return;
    const long long ig = tg / R4;
    int lo = 0, hi = nmesh - 1;   // the mesh holding row ig: row_off[mesh] <= ig < row_off[mesh + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= ig) lo = mid;
        else hi = mid - 1;
    }
    if (mdone && mdone[lo]) return;
    const MrMesh &Ms = ms[lo];
    const size_t pstride = (size_t)ntot * R / 4;   // float4 stride between partial buffers
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (Ms.has_near) {
        acc = ((const float4 *)Yall)[tg];
        for (int z = 0; z < nparts; ++z) {
            const float4 b = ((const float4 *)Y2all)[(size_t)z * pstride + tg];
            acc.x += b.x;
            acc.y += b.y;
            acc.z += b.z;
            acc.w += b.w;
        }
    }
    const int i = (int)(ig - Ms.xoff), q = (int)(tg % R4);
    const float4 *X4 = (const float4 *)(Xall + (size_t)Ms.xoff * R);
    if (Ms.diag) {
        const float dg = Ms.diag[i];
        const float4 x = X4[(size_t)i * R4 + q];
        acc.x = fmaf(dg, x.x, acc.x);
        acc.y = fmaf(dg, x.y, acc.y);
        acc.z = fmaf(dg, x.z, acc.z);
        acc.w = fmaf(dg, x.w, acc.w);
    } else {
#pragma unroll 4
        for (int c = Ms.rowptr[i]; c < Ms.rowptr[i + 1]; ++c) {
            const float v = Ms.val[c];
            const float4 x = X4[(size_t)Ms.colidx[c] * R4 + q];
            acc.x = fmaf(v, x.x, acc.x);
            acc.y = fmaf(v, x.y, acc.y);
            acc.z = fmaf(v, x.z, acc.z);
            acc.w = fmaf(v, x.w, acc.w);
        }
    }
    ((float4 *)Yall)[tg] = acc;
}

// the near phase of the apply for candidate c: Y = (near panels + B + M) X:
// the panel products (mma.sync or tcgen05 kernel; partial tiles of a split
// panel in Y2), then k_mr_rows adds the partials and the B + M rows (or the
// diagonal, where B + M is folded into the panels).  false: the candidate
// does not apply (shared memory, precision, meshes without panels).
template <class T>
static bool launch_near_phase(BatchData &b, int c, int R, const float *X, float *Y, cudaStream_t st,
                              const int *skip, const int *mdone)
{
    const NearCfg &f = kNearCfgs[c];
    if (f.tc) {
        if (sizeof(T) != 2 || b.n_tc_items != b.n_near_items) return false;
        if (b.n_tc_items > 0 && !launch_near_tma(b, f.nstage, f.ksplit, R, X, Y, st, skip, mdone)) return false;
    } else if (b.n_near_items > 0 &&
               !launch_near<T>(c, b.n_near_items, b.max_panel_w, (const NearItem *)b.near_items.p, R, X,
                               (const __nv_bfloat16 *)b.xc.p, (size_t)b.ntot * R, Y, b.y2.p, (size_t)b.ntot * R, st,
                               skip, mdone)) {
        return false;
    }
    const MrMesh *ms = (const MrMesh *)b.desc.p;
    k_mr_rows<<<cdiv((long long)b.ntot * (R / 4), 256), 256, 0, st>>>(ms, b.row_off.p, b.nmesh, (long long)b.ntot, R,
                                                                       X, Y, b.y2.p, f.ksplit - 1, skip, mdone);
    VFD_CUDA(cudaGetLastError());
    return true;
}

// ---------------------------------------------------------------------------
// host side: descriptors, work items, workspaces, launches
// ---------------------------------------------------------------------------
BatchData::~BatchData()
{
    release_bgraph(*this);
    if (side) {
        cudaStreamSynchronize(side);
        cudaStreamDestroy(side);
        cudaEventDestroy(ev_fork);
        cudaEventDestroy(ev_join);
    }
}

void release_bgraph(BatchData &b)
{
    if (b.exec) {
        cudaGraphExecDestroy(b.exec);
        b.exec = nullptr;
    }
}

BatchData *op_batch(OpData &op)
{
    if (!op.self) {
        BatchData *b = new BatchData();
        b->ops.push_back(&op);
        b->nmesh = 1;
        b->precision = op.precision;
        b->ntot = op.m->N;
        b->xoff = {0, (int64_t)op.m->N};
        op.self = b;
    }
    return op.self;
}

static void upload_items(DBuf<int> &buf, const std::vector<int> &v)
{
    buf.upload(v.empty() ? std::vector<int>{0, 0} : v);
}

__global__ void k_tf32_copy(long long n, const float *__restrict__ a, float *__restrict__ b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __uint_as_float(f2tf32(a[i]));
}

// time every candidate configuration of the near phase (panels + B + M) once
// on this batch (zero inputs, scratch outputs) and keep the fastest
template <class T>
static void tune_near(BatchData &b, int R, cudaStream_t st)
{
    const size_t n = (size_t)b.ntot * R;
    DBuf<float> tx, ty;
    tx.alloc(n);
    ty.alloc(n);
    tx.zero(st);
    if (b.xc.n) VFD_CUDA(cudaMemsetAsync(b.xc.p, 0, b.xc.n, st));
    cudaEvent_t e0, e1;
    VFD_CUDA(cudaEventCreate(&e0));
    VFD_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int bestc = 0;
    for (int c = 0; c < kNearCfgCount; ++c) {
        b.near_cfg_us[c] = 0.f;
        if (!launch_near_phase<T>(b, c, R, tx.p, ty.p, st, nullptr, nullptr)) continue;
        VFD_CUDA(cudaEventRecord(e0, st));
        for (int rep = 0; rep < 3; ++rep) launch_near_phase<T>(b, c, R, tx.p, ty.p, st, nullptr, nullptr);
        VFD_CUDA(cudaEventRecord(e1, st));
        VFD_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        VFD_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        b.near_cfg_us[c] = 1000.f * ms / 3;
        if (ms < best) {
            best = ms;
            bestc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    VFD_CUDA(cudaStreamSynchronize(st));
    int herr = 0;
    VFD_CUDA(cudaMemcpy(&herr, b.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr) VFD_CUDA(cudaMemset(b.tc_err.p, 0, sizeof(int)));
    VFD_REQUIRE(herr == 0, VFD_ETIMEOUT, "batched apply: a tensor-core pipeline wait expired while tuning");
    b.near_cfg = bestc;
}

// descriptors, item queues and workspaces for R columns (allocates and times
// the near-panel candidates: call outside stream capture; a captured solve is
// released when they change)
static void ensure_batch(BatchData &b, int R, cudaStream_t st)
{
    if (b.R == R) return;
    release_bgraph(b);
    if (!b.side) {
        // the far chain is a sequence of small launches: give it priority so its
        // CTAs are not queued behind the near-panel kernel
        int lo = 0, hi = 0;
        VFD_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        VFD_CUDA(cudaStreamCreateWithPriority(&b.side, cudaStreamNonBlocking, hi));
        VFD_CUDA(cudaEventCreateWithFlags(&b.ev_fork, cudaEventDisableTiming));
        VFD_CUDA(cudaEventCreateWithFlags(&b.ev_join, cudaEventDisableTiming));
    }
    const bool bf = b.precision == VFD_BF16;
    size_t nh = 0, nc = 0;
    b.max_panel_w = b.max_k = b.max_kp = b.max_leaf = b.max_mt = 0;
    b.any_far = false;
    for (OpData *op : b.ops) {
        const MeshData &m = *op->m;
        VFD_REQUIRE(op->precision == b.precision, VFD_EINVAL, "batched apply: operators of different precision");
        VFD_REQUIRE(op->precision != VFD_FP64, VFD_EINVAL, "batched apply needs VFD_FP32 or VFD_BF16 operators");
        VFD_REQUIRE(m.max_leaf_size <= 64, VFD_EUNSUPPORTED, "batched apply needs leaves of at most 64 DoFs");
        if (m.nfar > 0) {
            build_far_lowp(m, *op, st);
            const int kp = op->far_kp, mt = (m.kt.L - m.far_lmin + 1) * kp;
            nh += (size_t)m.kt.nnode * kp * R;
            nc += (size_t)m.kt.nleaf * mt * R;
            b.any_far = true;
            b.max_kp = std::max(b.max_kp, kp);
            b.max_mt = std::max(b.max_mt, mt);
        }
        b.max_panel_w = std::max(b.max_panel_w, m.max_panel_w);
        b.max_k = std::max(b.max_k, m.k);
        b.max_leaf = std::max(b.max_leaf, m.max_leaf_size);
    }
    VFD_REQUIRE((near_smem_bytes<float, 32, 3>(b.max_panel_w) <= 227 * 1024), VFD_EUNSUPPORTED,
                "batched apply: near panel too wide");
    VFD_REQUIRE(b.max_kp <= 64 && far_batched_smem(b.max_kp, b.max_mt) <= 227 * 1024, VFD_EUNSUPPORTED,
                "batched apply: rank too large for the far-field tiles");
    b.xhat.alloc(std::max<size_t>(nh, 1));
    b.yhat.alloc(std::max<size_t>(nh, 1));
    b.fpart.alloc(std::max<size_t>(nc, 1));
    b.y2.alloc((size_t)(KSPLIT_MAX - 1) * b.ntot * R);
    b.xc.alloc((size_t)b.ntot * R * 2 * 2);   // x as BF16 hi and lo blocks for the tcgen05 kernel
    if (!b.tc_err.p) {
        b.tc_err.alloc(1);
        VFD_CUDA(cudaMemset(b.tc_err.p, 0, sizeof(int)));
    }
    for (OpData *op : b.ops) build_batched_panels(*op->m, *op, st);
    b.n_tc_items = 0;
    if (bf) {
        build_tc_items(b);   // tcgen05 near kernel: items over the pre-tiled panels
    }
    std::vector<MrMesh> d(b.nmesh);
    std::vector<int> li, ni;
    std::vector<NearItem> nri;
    size_t ho = 0, co = 0;
    for (int i = 0; i < b.nmesh; ++i) {
        const OpData &op = *b.ops[i];
        const MeshData &m = *op.m;
        MrMesh &e = d[i];
        e.N = m.N;
        e.fl = m.kt.first_leaf();
        e.k = m.k;
        e.L = m.kt.L;
        e.lmin = m.far_lmin;
        e.nlev = m.nfar > 0 ? m.kt.L - m.far_lmin + 1 : 0;
        e.nleaf = m.kt.nleaf;
        e.nnode = m.kt.nnode;
        e.has_near = m.nnear > 0;
        e.has_far = m.nfar > 0;
        e.xoff = b.xoff[i];
        e.kb = m.kt_begin.p;
        e.ke = m.kt_end.p;
        e.pw = m.panel_w.p;
        e.gcol = m.gcol.p;
        e.goff = m.gcol_off.p;
        e.rowptr = m.rowptr.p;
        e.colidx = m.colidx.p;
        e.fptr = m.far_ptr.p;
        e.fcol = m.far_col.p;
        e.poff = m.panel_off.p;
        e.D = bf ? (const void *)op.D16.p : (const void *)op.D32t.p;
        e.kp = op.far_kp;
        e.Ulf = op.Up_lp.p;
        e.mt = m.nfar > 0 ? (m.kt.L - m.far_lmin + 1) * op.far_kp : 0;
        e.S = op.Sp_lp.p;
        e.val = op.valBM32.p;
        e.diag = op.precision == VFD_FP32 ? op.diag32.p : nullptr;   // folded B + M (TF32 panels only)
        e.xhat = b.xhat.p + ho;
        e.yhat = b.yhat.p + ho;
        e.part = b.fpart.p + co;
        if (m.nfar > 0) {
            ho += (size_t)m.kt.nnode * op.far_kp * R;
            co += (size_t)m.kt.nleaf * e.mt * R;
        }
        std::vector<int> kb_h, ke_h, pw_h, goff_h;
        std::vector<int64_t> poff_h;
        if (m.nnear > 0) {
            kb_h.assign(m.kt.begin.begin(), m.kt.begin.end());
            ke_h.assign(m.kt.end.begin(), m.kt.end.end());
            pw_h.resize(m.kt.nleaf);
            goff_h.resize(m.kt.nleaf + 1);
            poff_h.resize(m.kt.nleaf + 1);
            VFD_CUDA(cudaMemcpy(pw_h.data(), m.panel_w.p, sizeof(int) * pw_h.size(), cudaMemcpyDeviceToHost));
            VFD_CUDA(cudaMemcpy(goff_h.data(), m.gcol_off.p, sizeof(int) * goff_h.size(), cudaMemcpyDeviceToHost));
            VFD_CUDA(cudaMemcpy(poff_h.data(), m.panel_off.p, sizeof(int64_t) * poff_h.size(), cudaMemcpyDeviceToHost));
        }
        const size_t esz = bf ? 2 : 4;
        for (int lf = 0; lf < m.kt.nleaf; ++lf) {
            if (m.nnear > 0) {
                NearItem it{};
                it.D = (const unsigned char *)e.D + (size_t)poff_h[lf] * esz;
                it.gcol = m.gcol.p + goff_h[lf];
                it.row0 = (int)b.xoff[i] + kb_h[e.fl + lf];
                it.na = ke_h[e.fl + lf] - kb_h[e.fl + lf];
                it.W = pw_h[lf];
                it.xoff = (int)b.xoff[i];
                it.mesh = i;
                nri.push_back(it);
            }
            if (m.nfar > 0) {
                li.push_back(i);
                li.push_back(lf);
            }
        }
        if (m.nfar > 0)
            for (int nd = 0; nd < m.kt.nnode; ++nd)
                if (m.far_ptr_h[nd + 1] > m.far_ptr_h[nd]) {
                    ni.push_back(i);
                    ni.push_back(nd);
                }
    }
    std::vector<unsigned char> bytes(sizeof(MrMesh) * d.size());
    memcpy(bytes.data(), d.data(), bytes.size());
    b.desc.upload(bytes);
    upload_items(b.leaf_items, li);
    upload_items(b.node_items, ni);
    {
        std::vector<unsigned char> nb(sizeof(NearItem) * std::max<size_t>(nri.size(), 1), 0);
        if (!nri.empty()) memcpy(nb.data(), nri.data(), sizeof(NearItem) * nri.size());
        b.near_items.upload(nb);
    }
    b.n_leaf_items = (int)li.size() / 2;
    b.n_node_items = (int)ni.size() / 2;
    b.n_near_items = (int)nri.size();
    std::vector<long long> ro(b.xoff.begin(), b.xoff.end());
    b.row_off.upload(ro);
    b.R = R;
    if (b.n_near_items > 0 && b.forced_cfg < 0) {
        if (bf) tune_near<__nv_bfloat16>(b, R, st);
        else tune_near<float>(b, R, st);
    } else {
        b.near_cfg = b.forced_cfg < 0 ? 0 : b.forced_cfg;
    }
}

template <class T>
static void batch_apply_impl(BatchData &b, const float *X, float *Y, int R, cudaStream_t st, const int *skip,
                             const int *mdone, bool x_bf16_ready, float *Yfar)
{
    if (b.any_far) {
        // projections and coupling on the side stream, concurrent with the near
        // panels; with Yfar the expansion too (written there)
        VFD_CUDA(cudaEventRecord(b.ev_fork, st));
        VFD_CUDA(cudaStreamWaitEvent(b.side, b.ev_fork, 0));
        launch_far_side(b, R, X, b.side, skip, mdone);
        if (Yfar) launch_far_down(b, R, Yfar, b.side, skip, mdone, false);
        VFD_CUDA(cudaEventRecord(b.ev_join, b.side));
    }
    if (sizeof(T) == 2 && !x_bf16_ready) {   // x as BF16 hi and lo blocks for either near kernel
        const long long n = (long long)b.ntot * R;
        k_x_to_bf16<<<cdiv(n, 256), 256, 0, st>>>(n, X, (__nv_bfloat16 *)b.xc.p);
        VFD_CUDA(cudaGetLastError());
    }
    const bool launched = launch_near_phase<T>(b, b.near_cfg, R, X, Y, st, skip, mdone);
    VFD_REQUIRE(launched, VFD_EUNSUPPORTED, "batched apply: the pinned near-panel configuration does not apply");
    if (b.any_far) {
        VFD_CUDA(cudaStreamWaitEvent(st, b.ev_join, 0));
        if (!Yfar) launch_far_down(b, R, Y, st, skip, mdone, true);
    }
    VFD_CUDA(cudaGetLastError());
}

// pin the near-panel configuration (cfg >= 0) or go back to timing the candidates (-1)
int batch_set_config(BatchData &b, int cfg)
{
    VFD_REQUIRE(cfg >= -1 && cfg < kNearCfgCount, VFD_EINVAL, "near-panel configuration out of range");
    release_bgraph(b);
    b.forced_cfg = cfg;
    b.R = 0;   // rebuilt (and re-tuned or pinned) on the next apply
    return kNearCfgCount;
}

// a tcgen05 pipeline wait that expired (kernel error flag) becomes VFD_ETIMEOUT
void batch_check(BatchData &b, cudaStream_t st)
{
    if (!b.tc_err.p) return;
    int e = 0;
    VFD_CUDA(cudaMemcpyAsync(&e, b.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    VFD_CUDA(cudaStreamSynchronize(st));
    if (e) {   // reported once; later calls start clean
        VFD_CUDA(cudaMemset(b.tc_err.p, 0, sizeof(int)));
        if (b.gbar.p) VFD_CUDA(cudaMemset(b.gbar.p, 0, b.gbar.bytes()));
    }
    VFD_REQUIRE(e == 0, VFD_ETIMEOUT, "batched apply / solve: a bounded device wait expired");
}

// the near-panel tuning of a batch: chosen (stage width, depth, split, warps, accumulator sets)
// and the candidates' times
int batch_tuning(const BatchData &b, int *chosen, float *us, int n)
{
    if (chosen) {
        const NearCfg &f = kNearCfgs[b.near_cfg < 0 ? 0 : b.near_cfg];
        chosen[0] = b.near_cfg < 0 ? 0 : f.nk;
        chosen[1] = b.near_cfg < 0 ? 0 : f.nstage;
        chosen[2] = b.near_cfg < 0 ? 0 : f.ksplit;
        chosen[3] = b.near_cfg < 0 ? 0 : f.warps;
        chosen[4] = b.near_cfg < 0 ? 0 : f.nacc;
        chosen[5] = b.near_cfg < 0 ? 0 : f.tc;
    }
    for (int i = 0; i < n && i < kNearCfgCount; ++i) us[i] = b.near_cfg_us[i];
    return kNearCfgCount;
}

__global__ void k_fill1f(long long n, float *__restrict__ a)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 1.f;
}
__global__ void k_fill1d(long long n, double *__restrict__ a)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = 1.0;
}

// c_i = (A_64 1)_i - (A_low 1)_i (ylow: column 0 of an interleaved block of
// stride R), added to the FP32 diagonal of the batched operator: diag[i], or
// the diagonal entry of the FP32 B + M row where B + M is not folded
__global__ void k_comp_diag(int N, const double *__restrict__ y64, const float *__restrict__ ylow, int R,
                            float *__restrict__ diag, const int *__restrict__ rowptr, const int *__restrict__ colidx,
                            float *__restrict__ val)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double c = y64[i] - (double)ylow[(size_t)i * R];
    if (diag) {
        diag[i] = (float)((double)diag[i] + c);
        return;
    }
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e)
        if (colidx[e] == i) val[e] = (float)((double)val[e] + c);
}

// Diagonal compensation of the low-precision operators, once per operator, on
// its first batched use: rounding the near panels, bases, transfers and
// coupling matrices (and B + M, folded into the panels) to TF32 / BF16
// perturbs every entry by up to 2^-11 / 2^-8 of itself, and the perturbation's row sums shift the smallest eigenvalues
// of the (nearly zero-row-sum) operator by a fraction of the largest -- enough
// to stall the inner CG on fine meshes.  Adding the row sums of the
// perturbation, c = A_64 1 - A_low 1 (A_low 1 computed by the batched
// low-precision apply itself, before compensation), to the FP32 diagonal makes
// the rounded operator exact on constant vectors up to FP32 arithmetic: the
// remaining perturbation acts on differences u_j - u_i only and leaves the
// smooth low modes alone.  The outer FP64 residual is unaffected.
template <class T>
static void batch_apply_impl(BatchData &b, const float *X, float *Y, int R, cudaStream_t st, const int *skip,
                             const int *mdone, bool x_bf16_ready, float *Yfar);

template <class T>
static void compensate_diag(BatchData &b, cudaStream_t st)
{
    bool any = false;
    for (OpData *op : b.ops) any |= !op->comp_done && op->m->N > 0;
    if (!any) return;
    const int R = b.R;
    const long long n = (long long)b.ntot * R;
    DBuf<float> ones, ylow;
    ones.alloc(n);
    ylow.alloc(n);
    k_fill1f<<<cdiv(n, 256), 256, 0, st>>>(n, ones.p);
    batch_apply_impl<T>(b, ones.p, ylow.p, R, st, nullptr, nullptr, false, nullptr);
    batch_check(b, st);
    for (int i = 0; i < b.nmesh; ++i) {
        OpData &op = *b.ops[i];
        const MeshData &m = *op.m;
        if (op.comp_done || m.N == 0) continue;
        DBuf<double> one, y64;
        one.alloc(m.N);
        y64.alloc(m.N);
        k_fill1d<<<cdiv((long long)m.N, 256), 256, 0, st>>>(m.N, one.p);
        apply_parts_ex(m, op, VFD_PART_ALL, one.p, y64.p, 1, m.N, false, st, nullptr);
        k_comp_diag<<<cdiv((long long)m.N, 256), 256, 0, st>>>(
            m.N, y64.p, ylow.p + (size_t)b.xoff[i] * R, R, op.precision == VFD_FP32 ? op.diag32.p : nullptr,
            m.rowptr.p, m.colidx.p, op.valBM32.p);
        VFD_CUDA(cudaGetLastError());
        VFD_CUDA(cudaStreamSynchronize(st));
        op.comp_done = true;
    }
}

// Y = A_low X for R (multiple of 64) interleaved FP32 columns over all meshes;
// skip: device flag, nonzero = launch nothing; mdone: per-mesh device flags,
// nonzero = leave that mesh's rows of Y alone (both may be null)
void batch_apply(BatchData &b, const float *X, float *Y, int R, cudaStream_t st, const int *skip, const int *mdone,
                 bool x_bf16_ready, float *Yfar)
{
    VFD_REQUIRE(R % RT == 0 && R > 0, VFD_EINVAL, "batched apply needs a multiple of 64 columns");
    ensure_batch(b, R, st);
    if (b.precision == VFD_BF16) {
        compensate_diag<__nv_bfloat16>(b, st);
        batch_apply_impl<__nv_bfloat16>(b, X, Y, R, st, skip, mdone, x_bf16_ready, Yfar);
    } else {
        compensate_diag<float>(b, st);
        batch_apply_impl<float>(b, X, Y, R, st, skip, mdone, x_bf16_ready, Yfar);
    }
}

// p (interleaved FP32, R columns) into the BF16 hi / lo x blocks of the near kernels
void batch_x_to_bf16(BatchData &b, const float *X, int R, cudaStream_t st)
{
    const long long n = (long long)b.ntot * R;
    k_x_to_bf16<<<cdiv(n, 256), 256, 0, st>>>(n, X, (__nv_bfloat16 *)b.xc.p);
    VFD_CUDA(cudaGetLastError());
}

void *batch_x16(BatchData &b)
{
    return b.precision == VFD_BF16 ? (void *)b.xc.p : nullptr;
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

// Y_m = A_low,m X_m for every mesh m (column-major FP64 blocks, nrhs a multiple of 64)
void batch_apply_colmajor(BatchData &b, const double *const *X, double *const *Y, const int64_t *ld, int nrhs,
                          cudaStream_t st)
{
    const size_t n = (size_t)b.ntot * nrhs;
    if (b.xi.n < n) {
        b.xi.alloc(n);
        b.yi.alloc(n);
    }
    for (int i = 0; i < b.nmesh; ++i) {
        const int N = b.ops[i]->m->N;
        k_cm_to_il<<<cdiv((long long)N * nrhs, 256), 256, 0, st>>>(N, nrhs, ld[i], X[i],
                                                                   b.xi.p + (size_t)b.xoff[i] * nrhs);
    }
    batch_apply(b, b.xi.p, b.yi.p, nrhs, st, nullptr, nullptr);
    batch_check(b, st);
    for (int i = 0; i < b.nmesh; ++i) {
        const int N = b.ops[i]->m->N;
        k_il_to_cm<<<cdiv((long long)N * nrhs, 256), 256, 0, st>>>(N, nrhs, ld[i], b.yi.p + (size_t)b.xoff[i] * nrhs,
                                                                   Y[i]);
    }
    VFD_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// panels of the batched path: D + (B + M) off the diagonal, the diagonal of
// A kept apart in FP32 (first batched use of an operator)
// ---------------------------------------------------------------------------
__global__ void k_fold_bm(int N, const int *__restrict__ rowptr, const int *__restrict__ colidx,
                          const int64_t *__restrict__ pos, const double *__restrict__ val, double *__restrict__ Dp,
                          float *__restrict__ diag)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double dg = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int64_t p = pos[e];   // every entry has its own panel position
        if (colidx[e] == i) {
            dg = val[e] + Dp[p];
            Dp[p] = 0.0;
        } else {
            Dp[p] += val[e];
        }
    }
    diag[i] = (float)dg;
}

__global__ void k_to_bf16(long long n, const double *__restrict__ a, __nv_bfloat16 *__restrict__ b);

__global__ void k_to_tf32(long long n, const double *__restrict__ a, float *__restrict__ b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __uint_as_float(f2tf32((float)a[i]));
}

// TF32 (VFD_FP32): B + M off the diagonal folded into the panels, the
// diagonal in FP32 (diag32) -- the near phase reads no CSR rows.  BF16
// (VFD_BF16): plain D in BF16 (row panels and the tiled images of the
// tcgen05 kernel); B + M stays an FP32 CSR matrix, because BF16 rounding of
// the large singular entries perturbs the low modes of the operator enough
// to triple the inner iterations.
void build_batched_panels(const MeshData &m, OpData &op, cudaStream_t st)
{
    if (op.bm_folded) return;
    const long long n = (long long)op.D64.n;
    if (op.precision == VFD_BF16) {
        op.D16.alloc(op.D64.n);
        if (n) k_to_bf16<<<cdiv(n, 256), 256, 0, st>>>(n, op.D64.p, (__nv_bfloat16 *)op.D16.p);
        build_tiled_panels(m, op, op.D64.p, st);
    } else {
        VFD_REQUIRE(m.bm_in_panels, VFD_EUNSUPPORTED,
                    "batched apply: some B + M entries lie outside the near blocks (admissibility lambda >= 1)");
        DBuf<double> Dp;
        Dp.alloc(std::max<size_t>(op.D64.n, 1));
        if (n) VFD_CUDA(cudaMemcpyAsync(Dp.p, op.D64.p, op.D64.bytes(), cudaMemcpyDeviceToDevice, st));
        op.diag32.alloc(m.N);
        k_fold_bm<<<cdiv(m.N, 256), 256, 0, st>>>(m.N, m.rowptr.p, m.colidx.p, m.bm_pos.p, op.valBM.p, Dp.p,
                                                  op.diag32.p);
        op.D32t.alloc(op.D64.n);
        if (n) k_to_tf32<<<cdiv(n, 256), 256, 0, st>>>(n, Dp.p, op.D32t.p);
        VFD_CUDA(cudaStreamSynchronize(st));   // Dp is released on return
    }
    VFD_CUDA(cudaGetLastError());
    op.bm_folded = true;
}

// ---------------------------------------------------------------------------
// BF16 copies of the K data (VFD_BF16 operators)
// ---------------------------------------------------------------------------
__global__ void k_to_bf16(long long n, const double *__restrict__ a, __nv_bfloat16 *__restrict__ b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __double2bfloat16(a[i]);
}


__global__ void k_d2f(long long n, const double *__restrict__ a, float *__restrict__ b)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}



void launch_lowp_csr(const MeshData &m, OpData &op, cudaStream_t st)
{
    op.valBM32.alloc(m.nnz);
    if (m.nnz) k_d2f<<<cdiv(m.nnz, 256), 256, 0, st>>>(m.nnz, op.valBM.p, op.valBM32.p);
    VFD_CUDA(cudaGetLastError());
}

}  // namespace vfd
