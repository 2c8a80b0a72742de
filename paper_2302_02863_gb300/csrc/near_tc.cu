// Near panels of the batched BF16 apply on the 5th-generation tensor cores,
// the panel streamed by bulk (TMA-engine) copies:
// Y[leaf rows][rt .. rt+63] = D_panel Xg (the B + M rows and the sum of a
// split panel's partial tiles follow in k_mr_rows, as for the mma.sync kernel).
//
// This is the dense inadmissible-leaf product of Sec. 5.2 (eq. e:k-near) for
// 64 right-hand sides at a time, plus the sparse singular near field and the
// weighted mass matrix (Sec. 3, eq. e:decomp), in the low-precision inner
// operator of the mixed-precision solve.
//
// Work item = (mesh, leaf); CTA = (item, 64-RHS tile, panel part).  Warp
// roles inside the CTA (128 threads), per stage of 64 panel columns:
//   warp 0, lane 0 (A producer): one bulk copy (cp.async.bulk, completing on
//     the stage's "full A" mbarrier by transaction bytes) of the leaf's
//     pre-tiled panel stage: na rows x 128 B, already in the K-major
//     128-byte-swizzled layout the MMA reads, so the copy is one contiguous
//     block;
//   warps 2-3 (B producers): thread t gathers the x row of panel column t
//     with 16-byte cp.async into the MN-major core-matrix layout (zero fill
//     for padding columns), x as two BF16 terms hi + lo (64 RHS = 128 B
//     each, two B tiles); once its copies of a stage have landed it fences
//     them for the async proxy and arrives on the stage's "full B" barrier
//     (64 arrivals);
//   warp 1, lane 0 (MMA issuer): waits for both, issues eight tcgen05.mma
//     (kind::f16, M = 128, N = 64, K = 16, FP32 accumulator in tensor
//     memory; per K step the hi and the lo tile) and commits them to the
//     stage's "empty" barrier, which hands the buffers back to the producers;
//   warp 2 also allocates / frees the 64 tensor-memory columns.
// Rows na..127 of the M = 128 operand are whatever the shared memory holds;
// they only produce accumulator rows that are never read.
// Epilogue: warps 0 and 1 read the accumulator rows of the leaf (tensor
// memory lanes 0..63) into shared memory; all four warps write the tile to Y
// (part 0 of a split panel) or to partial buffer z - 1 of Y2 (part z > 0).
//
// Every mbarrier wait is bounded by the global timer (limit passed in); on
// expiry the CTA records the error, stops issuing, waits (bounded again) for
// the copies and MMAs it already issued, frees its tensor memory and leaves
// Y unwritten.
#include <cuda_bf16.h>

#include "batched.cuh"

namespace vfd {

namespace {

constexpr int TC_NK = 64;                     // panel columns per stage (one 128-byte BF16 row)
constexpr int TC_STAGE_BYTES = 3 * 8192;      // A (<= 64 rows x 128 B) + B hi, B lo (64 rows x 128 B each)
constexpr int TC_LDS = RT + 4;                // row stride (floats) of the epilogue tile
constexpr long long TC_DRAIN_NS = 1000000000LL;   // bound of the waits that drain work already issued

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// wait for the completion of the phase with the given parity, until the
// global timer passes `deadline` (ns); false on expiry
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity, uint64_t deadline)
{
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (gtimer() > deadline) return false;
    }
}

// smem matrix descriptor (tcgen05): start, leading / stride byte offsets,
// version 1, swizzle mode 2 = 128-byte swizzle
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// smem matrix descriptor without swizzle (canonical core-matrix layout)
__device__ __forceinline__ uint64_t desc_plain(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFF) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFF) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// 16-byte cp.async (zero fill when !valid: nothing is read)
__device__ __forceinline__ void tc_cp16(void *smem, const void *gmem, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s_addr(smem)), "l"(gmem), "r"(valid ? 16 : 0)
                 : "memory");
}

// instruction descriptor: FP32 accumulator, A and B BF16, A K-major, B
// MN-major, N = 64, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

}  // namespace

// one (mesh, leaf) item of the TMA-fed tensor-core kernel
struct TcItem {
    const unsigned char *A;   // the leaf's pre-tiled panel: nst stages x na rows x 128 B (BF16, swizzled)
    const int *gcol;          // panel column -> mesh-local DoF (-1: padding), W entries
    int row0, na, W, nst;     // first batch row, leaf rows, panel width, stages
    int xoff, mesh;           // first batch row of the mesh, mesh index
};

template <int NSTAGE>
__global__ void __launch_bounds__(128, 1)
k_near_tma(const TcItem *__restrict__ items, int R, const void *__restrict__ Xc, size_t xlo,
           float *__restrict__ Yall, float *__restrict__ Y2all, size_t pstride, long long wait_ns, int *err,
           const int *skip, const int *mdone)
{
    extern __shared__ unsigned char tsm_raw[];
    if (skip && *skip) return;
    const TcItem it = items[blockIdx.x];
    if (mdone && mdone[it.mesh]) return;
    // 1024-byte aligned stage buffers (the swizzle pattern follows address bits 4-9)
    unsigned char *tsm = (unsigned char *)(((uintptr_t)tsm_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bars = (uint64_t *)(tsm + NSTAGE * TC_STAGE_BYTES);   // fullA, fullB, empty [NSTAGE each], done
    uint32_t *tslot = (uint32_t *)(bars + 3 * NSTAGE + 1);
    volatile int *abort_f = (volatile int *)(tslot + 1);
    int *gs = (int *)(tslot + 4);   // gather columns of this CTA's stages
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rt = blockIdx.y * RT, ksplit = gridDim.z, z = blockIdx.z;
    const int s0 = (int)(((long long)it.nst * z) / ksplit), n = (int)(((long long)it.nst * (z + 1)) / ksplit) - s0;
    const uint64_t t0 = gtimer();
    const uint64_t deadline = t0 + (uint64_t)(wait_ns > 0 ? wait_ns : 0);
    const uint32_t bar0 = s_addr(bars);
    auto fullA_b = [&](int s) { return bar0 + 8u * s; };
    auto fullB_b = [&](int s) { return bar0 + 8u * (NSTAGE + s); };
    auto empty_b = [&](int s) { return bar0 + 8u * (2 * NSTAGE + s); };
    const uint32_t done_b = bar0 + 24u * NSTAGE;

    if (tid == 0) {
        for (int s = 0; s < 3 * NSTAGE + 1; ++s) {
            const int count = (s >= NSTAGE && s < 2 * NSTAGE) ? 64 : 1;   // fullB: one arrival per B producer
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar0 + 8u * s), "r"(count));
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
        *abort_f = 0;
    }
    for (int c = tid; c < n * TC_NK; c += 128) {
        const int col = s0 * TC_NK + c;
        gs[c] = col < it.W ? it.gcol[col] : -1;
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;\n" ::"r"(s_addr(tslot)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t taddr = *tslot;
    const uint32_t a_bytes = (uint32_t)it.na * 128u;

    const unsigned char *Xb = (const unsigned char *)Xc;   // x in BF16, [nrow][R]: hi, then lo at element xlo
    int issued = 0;   // A producer: stages whose bulk copies were issued
    if (warp == 0) {
        if (lane == 0)
            for (int i = 0; i < n; ++i) {
                const int s = i % NSTAGE;
                if ((i >= NSTAGE && !bar_wait(empty_b(s), ((i / NSTAGE) - 1) & 1, deadline)) || *abort_f) {
                    *abort_f = 1;
                    break;
                }
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fullA_b(s)), "r"(a_bytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                        s_addr(tsm + s * TC_STAGE_BYTES)),
                    "l"(it.A + (size_t)(s0 + i) * a_bytes), "r"(a_bytes), "r"(fullA_b(s))
                    : "memory");
                issued = i + 1;
            }
    } else if (warp == 1) {
        if (lane == 0) {
            int i = 0;
            for (; i < n; ++i) {
                const int s = i % NSTAGE, par = (i / NSTAGE) & 1;
                if (*abort_f || !bar_wait(fullA_b(s), par, deadline) || !bar_wait(fullB_b(s), par, deadline)) {
                    *abort_f = 1;
                    break;
                }
                // the x rows came through the generic proxy (cp.async): order them before the MMA's reads
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t sa = s_addr(tsm + s * TC_STAGE_BYTES), sb = sa + 8192u;
#pragma unroll
                for (int k = 0; k < TC_NK / 16; ++k) {
                    const uint64_t da = desc_sw128(sa + 32u * k, 16u, 1024u);   // K-major, 128-byte swizzle: +32 B per K step
                    const uint64_t db = desc_plain(sb + 2048u * k, 1024u, 128u);  // MN-major, no swizzle: +16 rows per K step
                    const uint64_t dl = desc_plain(sb + 8192u + 2048u * k, 1024u, 128u);   // the lo tile
                    const uint32_t acc = (i > 0 || k > 0) ? 1u : 0u;
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
                                 "l"(da), "l"(db), "r"(TC_IDESC), "r"(acc));
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
                                 "l"(da), "l"(dl), "r"(TC_IDESC), "r"(1u));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    empty_b(s)));
            }
            // completion of every MMA issued above (also on an early exit); a CTA
            // without stages issues nothing and commits nothing
            if (n > 0)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    done_b));
        }
    } else {
        // B producers (warps 2, 3): thread t copies x row k = t of every stage
        // (hi and lo: 2 x 128 bytes = 16 core-matrix pieces of 16 bytes) with
        // cp.async; it signals a stage once its own copies of that stage have landed
        constexpr int LAG = NSTAGE - 1;   // stages of copies a thread keeps in flight
        const int t = tid - 64;
        int posted = 0, arrived = 0;
        for (int i = 0; i < n; ++i) {
            const int s = i % NSTAGE;
            if ((i >= NSTAGE && !bar_wait(empty_b(s), ((i / NSTAGE) - 1) & 1, deadline)) || *abort_f) {
                *abort_f = 1;
                break;
            }
            const int g = gs[i * TC_NK + t];
            const unsigned char *src = g >= 0 ? Xb + ((size_t)(it.xoff + g) * R + rt) * 2 : Xb;
            const unsigned char *srl = g >= 0 ? src + xlo * 2 : Xb;
            unsigned char *dst = tsm + s * TC_STAGE_BYTES + 8192 + (t >> 3) * 1024 + (t & 7) * 16;
#pragma unroll
            for (int c = 0; c < 8; ++c) tc_cp16(dst + c * 128, src + c * 16, g >= 0);
#pragma unroll
            for (int c = 0; c < 8; ++c) tc_cp16(dst + 8192 + c * 128, srl + c * 16, g >= 0);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
            posted = i + 1;
            if (i >= LAG) {
                asm volatile("cp.async.wait_group %0;\n" ::"n"(LAG) : "memory");
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(fullB_b((i - LAG) % NSTAGE))
                             : "memory");
                arrived = i - LAG + 1;
            }
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // every copy of this thread has landed
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (!*abort_f)
            for (int i = arrived; i < posted; ++i)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(fullB_b(i % NSTAGE)) : "memory");
    }
    __syncwarp();
    // all MMAs done (bounded); on expiry or an earlier abort, drain what was issued
    const bool ok = n == 0 || bar_wait(done_b, 0, deadline);
    if (!ok) *abort_f = 1;
    __syncthreads();
    const bool aborted = *abort_f != 0;
    if (aborted) {
        const uint64_t dl = gtimer() + TC_DRAIN_NS;
        bool drained = n == 0 || bar_wait(done_b, 0, dl);
        if (warp == 0 && lane == 0)
            for (int i = (issued > NSTAGE ? issued - NSTAGE : 0); i < issued; ++i)
                drained &= bar_wait(fullA_b(i % NSTAGE), (i / NSTAGE) & 1, dl);
        if (tid == 0) atomicOr(err, drained ? 1 : 3);
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    float *acc_s = (float *)tsm;   // [64][TC_LDS], over the (now idle) stage buffers
    if (!aborted && warp < 2) {
        const int row = 32 * warp + lane;
        for (int c0 = 0; c0 < RT; c0 += 16) {
            uint32_t r[16];
            if (n > 0) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) r[q] = 0u;
            }
            float4 *dst = (float4 *)(acc_s + row * TC_LDS + c0);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                     __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 2) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;\n" ::"r"(taddr));

    // ---- epilogue: the tile (or this part's partial tile) to Y / Y2
    if (aborted) return;   // Y unwritten; the host reports the expired wait
    const int na = it.na;
    float *Yo = z == 0 ? Yall : Y2all + (size_t)(z - 1) * pstride;
    for (int e = tid; e < na * (RT / 4); e += 128) {
        const int row = e / (RT / 4), q = e % (RT / 4);
        *(float4 *)(Yo + (size_t)(it.row0 + row) * R + rt + 4 * q) = *(const float4 *)(acc_s + row * TC_LDS + 4 * q);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// pre-tiled BF16 panel images: leaf a's panel (na rows, row stride W, FP64)
// as nst = ceil(W / 64) stages of na rows x 64 columns, each row 128 bytes
// with its 16-byte chunks permuted as the 128-byte swizzle places them
// (chunk c of row r at position c ^ (r % 8)); columns beyond W are zero.
__global__ void k_tile_panels(const double *__restrict__ D, const int64_t *__restrict__ poff,
                              const int *__restrict__ pw, const int *__restrict__ kb, const int *__restrict__ ke,
                              int fl, const int64_t *__restrict__ toff, __nv_bfloat16 *__restrict__ out)
{
    const int a = blockIdx.x;
    const int na = ke[fl + a] - kb[fl + a], W = pw[a], nst = (W + TC_NK - 1) / TC_NK;
    const double *P = D + poff[a];
    __nv_bfloat16 *img = out + toff[a];
    const int chunks = nst * na * 8;
    for (int t = threadIdx.x; t < chunks; t += blockDim.x) {
        const int c = t & 7, r = (t >> 3) % na, s = (t >> 3) / na;
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int col = s * TC_NK + c * 8 + e;
            v[e] = __double2bfloat16(col < W ? P[(size_t)r * W + col] : 0.0);
        }
        *(uint4 *)(img + ((size_t)(s * na + r) * 64 + ((c ^ (r & 7)) * 8))) = *(const uint4 *)v;
    }
}

// element offsets of the leaves' tiled images (nleaf + 1 entries) and the images
void build_tiled_panels(const MeshData &m, OpData &op, const double *D, cudaStream_t st)
{
    if (m.nnear == 0) return;
    std::vector<int> pw(m.kt.nleaf);
    VFD_CUDA(cudaMemcpy(pw.data(), m.panel_w.p, sizeof(int) * pw.size(), cudaMemcpyDeviceToHost));
    const int fl = m.kt.first_leaf();
    std::vector<int64_t> off(m.kt.nleaf + 1, 0);
    for (int a = 0; a < m.kt.nleaf; ++a) {
        const int na = m.kt.end[fl + a] - m.kt.begin[fl + a], nst = (pw[a] + TC_NK - 1) / TC_NK;
        off[a + 1] = off[a] + (int64_t)nst * na * TC_NK;
    }
    op.Dtc_off = off;
    op.Dtc_doff.upload(off);
    op.Dtc.alloc(std::max<int64_t>(off.back(), 8));
    k_tile_panels<<<m.kt.nleaf, 256, 0, st>>>(D, m.panel_off.p, m.panel_w.p, m.kt_begin.p, m.kt_end.p, fl,
                                             op.Dtc_doff.p, (__nv_bfloat16 *)op.Dtc.p);
    VFD_CUDA(cudaGetLastError());
}

// the items of a batch (one per (mesh, leaf) with a near panel)
void build_tc_items(BatchData &b)
{
    std::vector<TcItem> v;
    for (int i = 0; i < b.nmesh; ++i) {
        const OpData &op = *b.ops[i];
        const MeshData &m = *op.m;
        if (m.nnear == 0) continue;
        std::vector<int> pw(m.kt.nleaf), goff(m.kt.nleaf + 1);
        VFD_CUDA(cudaMemcpy(pw.data(), m.panel_w.p, sizeof(int) * pw.size(), cudaMemcpyDeviceToHost));
        VFD_CUDA(cudaMemcpy(goff.data(), m.gcol_off.p, sizeof(int) * goff.size(), cudaMemcpyDeviceToHost));
        const int fl = m.kt.first_leaf();
        for (int a = 0; a < m.kt.nleaf; ++a) {
            TcItem t{};
            t.A = (const unsigned char *)op.Dtc.p + (size_t)op.Dtc_off[a] * 2;
            t.gcol = m.gcol.p + goff[a];
            t.row0 = (int)b.xoff[i] + m.kt.begin[fl + a];
            t.na = m.kt.end[fl + a] - m.kt.begin[fl + a];
            t.W = pw[a];
            t.nst = (pw[a] + TC_NK - 1) / TC_NK;
            t.xoff = (int)b.xoff[i];
            t.mesh = i;
            v.push_back(t);
        }
    }
    b.n_tc_items = (int)v.size();
    std::vector<unsigned char> bytes(sizeof(TcItem) * std::max<size_t>(v.size(), 1), 0);
    if (!v.empty()) memcpy(bytes.data(), v.data(), sizeof(TcItem) * v.size());
    b.tc_items.upload(bytes);
}

size_t near_tma_smem(int nstage, int max_panel_w)
{
    return (size_t)nstage * TC_STAGE_BYTES + (3 * nstage + 1) * 8 + 16 + (size_t)(max_panel_w + TC_NK) * 4 + 1024;
}

// launch with nstage pipeline stages and the panel split over ksplit CTAs
bool launch_near_tma(BatchData &b, int nstage, int ksplit, int R, const float *X, float *Y, cudaStream_t st,
                     const int *skip, const int *mdone)
{
    const size_t shm = near_tma_smem(nstage, b.max_panel_w);
    const size_t pstride = (size_t)b.ntot * R;   // partial tiles of parts 1.. in Y2 (k_mr_rows sums them)
    if (shm > 227 * 1024 || ksplit < 1 || ksplit > 4 || b.n_tc_items == 0) return false;
    if (ksplit > 1 && b.y2.n < (size_t)(ksplit - 1) * pstride) return false;
    dim3 g(b.n_tc_items, R / RT, ksplit);
    const TcItem *items = (const TcItem *)b.tc_items.p;
#define VFD_TMA_CASE(NS)                                                                                         \
    if (nstage == NS) {                                                                                          \
        VFD_CUDA(cudaFuncSetAttribute(k_near_tma<NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));    \
        k_near_tma<NS><<<g, 128, shm, st>>>(items, R, b.xc.p, (size_t)b.ntot * R, Y, b.y2.p, pstride, b.wait_ns, \
                                            b.tc_err.p, skip, mdone);                                             \
        VFD_CUDA(cudaGetLastError());                                                                            \
        return true;                                                                                             \
    }
    VFD_TMA_CASE(2)
    VFD_TMA_CASE(3)
    VFD_TMA_CASE(4)
    VFD_TMA_CASE(6)
#undef VFD_TMA_CASE
    return false;
}

}  // namespace vfd
