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
constexpr int KC = 64;   // K chunk (panel columns) per stage

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
// near panels on the tensor cores.  CTA = (leaf, RHS tile), 4 warps; warp w
// owns rows 16w..16w+15 of the leaf and all 8 n8 tiles of the RHS tile.
// Shared: As[64][KC+PAD] (panel rows), Bs[64 rhs][KC+PAD] (gathered x, k
// contiguous per rhs).
// ---------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(128)
k_mr_near(int fl, int R, const int *__restrict__ kb, const int *__restrict__ ke, const int *__restrict__ pw,
          const int64_t *__restrict__ poff, const int *__restrict__ gcol, const int *__restrict__ goff,
          const T *__restrict__ D, const float *__restrict__ X, float *__restrict__ Y, const int *skip)
{
    constexpr int PAD = (sizeof(T) == 2) ? 8 : 4;   // row padding (elements) against bank conflicts
    constexpr int LDS = KC + PAD;
    __shared__ __align__(16) T As[64 * LDS];
    __shared__ __align__(16) T Bs[RT * LDS];
    if (skip && *skip) return;
    const int lf = blockIdx.x, rt = blockIdx.y * RT;
    const int b0 = kb[fl + lf], na = ke[fl + lf] - b0;
    const int W = pw[lf];
    const T *Dp = D + poff[lf];
    const int *gc = gcol + goff[lf];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
    float acc[8][4];
    for (int j = 0; j < 8; ++j)
        for (int q = 0; q < 4; ++q) acc[j][q] = 0.f;
    for (int k0 = 0; k0 < W; k0 += KC) {
        const int kc = min(KC, W - k0);   // multiple of 4 (panel width padded to 4)
        // A chunk: rows 0..63 (zero beyond na), columns k0..k0+KC (zero beyond W)
        for (int idx = threadIdx.x; idx < 64 * KC; idx += blockDim.x) {
            int row = idx / KC, c = idx - row * KC;
            T v = (T)0.f;
            if (row < na && c < kc) v = Dp[(size_t)row * W + k0 + c];
            As[row * LDS + c] = v;
        }
        // B chunk: Bs[n][c] = x[gcol[k0+c]][rt+n]
        for (int idx = threadIdx.x; idx < KC * RT; idx += blockDim.x) {
            int c = idx / RT, nn = idx - c * RT;
            float v = 0.f;
            if (c < kc) {
                int j = gc[k0 + c];
                if (j >= 0) v = X[(size_t)j * R + rt + nn];
            }
            Bs[nn * LDS + c] = from_f<T>(v);
        }
        __syncthreads();
        const int r0 = warp * 16;
        if (r0 < na) {
            constexpr int KS = MmaTraits<T>::KS;
            for (int ks = 0; ks < KC; ks += KS) {
                uint32_t a[4];
                if constexpr (sizeof(T) == 2) {
                    const T *A0 = As + (r0 + g) * LDS + ks + 2 * t4;
                    const T *A8 = As + (r0 + g + 8) * LDS + ks + 2 * t4;
                    a[0] = *(const uint32_t *)A0;
                    a[1] = *(const uint32_t *)A8;
                    a[2] = *(const uint32_t *)(A0 + 8);
                    a[3] = *(const uint32_t *)(A8 + 8);
                } else {
                    const float *A0 = (const float *)As + (r0 + g) * LDS + ks + t4;
                    const float *A8 = (const float *)As + (r0 + g + 8) * LDS + ks + t4;
                    a[0] = f2tf32(A0[0]);
                    a[1] = f2tf32(A8[0]);
                    a[2] = f2tf32(A0[4]);
                    a[3] = f2tf32(A8[4]);
                }
                for (int j = 0; j < 8; ++j) {
                    uint32_t bb[2];
                    if constexpr (sizeof(T) == 2) {
                        const T *B0 = Bs + (j * 8 + g) * LDS + ks + 2 * t4;
                        bb[0] = *(const uint32_t *)B0;
                        bb[1] = *(const uint32_t *)(B0 + 8);
                    } else {
                        const float *B0 = (const float *)Bs + (j * 8 + g) * LDS + ks + t4;
                        bb[0] = __float_as_uint(B0[0]);
                        bb[1] = __float_as_uint(B0[4]);
                    }
                    MmaTraits<T>::mma(acc[j], a, bb);
                }
            }
        }
        __syncthreads();
    }
    const int r0 = warp * 16;
    for (int j = 0; j < 8; ++j) {
        const int col = rt + j * 8 + 2 * t4;
        const int ra = r0 + g, rb = r0 + g + 8;
        if (ra < na) {
            Y[(size_t)(b0 + ra) * R + col] = acc[j][0];
            Y[(size_t)(b0 + ra) * R + col + 1] = acc[j][1];
        }
        if (rb < na) {
            Y[(size_t)(b0 + rb) * R + col] = acc[j][2];
            Y[(size_t)(b0 + rb) * R + col + 1] = acc[j][3];
        }
    }
}

// Y[i][r] (+)= sum_c val[c] X[col c][r]   (B + M in FP32; thread per (row, r))
__global__ void k_mr_csr(int N, int R, int accumulate, const int *__restrict__ rowptr, const int *__restrict__ colidx,
                         const float *__restrict__ val, const float *__restrict__ X, float *__restrict__ Y,
                         const int *skip)
{
    if (skip && *skip) return;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * R) return;
    const int i = (int)(t / R), r = (int)(t % R);
    float acc = accumulate ? Y[t] : 0.f;
    for (int c = rowptr[i]; c < rowptr[i + 1]; ++c) acc = fmaf(val[c], X[(size_t)colidx[c] * R + r], acc);
    Y[t] = acc;
}

// far field, R RHS (FP32 accumulation; T the stored basis / coupling type)
// part[lv][leaf][a][r] = sum_{i in leaf} Ul[lv][i][a] X[i][r]; CTA per (leaf, lv, 128-wide (a, r) slice)
template <class T>
__global__ void k_mr_far_proj(int fl, int k, int N, int R, const int *__restrict__ kb, const int *__restrict__ ke,
                              const T *__restrict__ Ul, const float *__restrict__ X, float *__restrict__ part,
                              int nleaf, const int *skip)
{
    if (skip && *skip) return;
    const int leaf = blockIdx.x, lv = blockIdx.y;
    const int t = blockIdx.z * blockDim.x + threadIdx.x;
    if (t >= k * R) return;
    const int al = t / R, r = t % R;
    const int b = kb[fl + leaf], e = ke[fl + leaf];
    const T *u = Ul + ((size_t)lv * N) * k + al;
    float acc = 0.f;
    for (int i = b; i < e; ++i) acc = fmaf((float)u[(size_t)i * k], X[(size_t)i * R + r], acc);
    part[(((size_t)lv * nleaf + leaf) * k + al) * R + r] = acc;
}

// xhat[node][a][r] = sum over the node's leaves of part (levels lmin..L)
__global__ void k_mr_far_sum(int lmin, int L, int k, int R, int nleaf, const float *__restrict__ part,
                             float *__restrict__ xhat, const int *skip)
{
    if (skip && *skip) return;
    const int node = (1 << lmin) - 1 + blockIdx.x;
    const int t = blockIdx.y * blockDim.x + threadIdx.x;
    if (t >= k * R) return;
    int l = 0;
    while ((2 << l) - 1 <= node) ++l;
    const int span = 1 << (L - l), leaf0 = ((node + 1) << (L - l)) - 1 - ((1 << L) - 1);
    const float *p = part + (((size_t)(l - lmin) * nleaf + leaf0) * k) * R + t;
    float s = 0.f;
    for (int j = 0; j < span; ++j) s += p[(size_t)j * k * R];
    xhat[(size_t)node * k * R + t] = s;
}

// yhat[node][a][r] = sum_e sum_b S_e[b][a] xhat[col e][b][r]
template <class T>
__global__ void k_mr_far_couple(int k, int R, const int *__restrict__ fptr, const int *__restrict__ fcol,
                                const T *__restrict__ S, const float *__restrict__ xhat, float *__restrict__ yhat,
                                const int *skip)
{
    if (skip && *skip) return;
    const int node = blockIdx.x;
    const int t = blockIdx.y * blockDim.x + threadIdx.x;
    if (t >= k * R) return;
    const int al = t / R, r = t % R;
    float acc = 0.f;
    for (int e = fptr[node]; e < fptr[node + 1]; ++e) {
        const T *s = S + (size_t)e * k * k + al;
        const float *xc = xhat + (size_t)fcol[e] * k * R + r;
        for (int be = 0; be < k; ++be) acc = fmaf((float)s[(size_t)be * k], xc[(size_t)be * R], acc);
    }
    yhat[(size_t)node * k * R + t] = acc;
}

// Y[i][r] += sum_l sum_a Ul[l][i][a] yhat[ancestor_l(i)][a][r]
template <class T>
__global__ void k_mr_far_expand(int fl, int lmin, int L, int k, int N, int R, const int *__restrict__ leaf_of,
                                const T *__restrict__ Ul, const float *__restrict__ yhat, float *__restrict__ Y,
                                const int *skip)
{
    if (skip && *skip) return;
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * R) return;
    const int i = (int)(t / R), r = (int)(t % R);
    const int lf = leaf_of[i];
    float acc = 0.f;
    for (int l = lmin; l <= L; ++l) {
        const int node = ((fl + lf + 1) >> (L - l)) - 1;
        const T *u = Ul + ((size_t)(l - lmin) * N + i) * k;
        const float *y = yhat + (size_t)node * k * R + r;
        for (int al = 0; al < k; ++al) acc = fmaf((float)u[al], y[(size_t)al * R], acc);
    }
    Y[t] += acc;
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
        dim3 g(m.kt.nleaf, R / RT);
        k_mr_near<T><<<g, 128, 0, st>>>(fl, R, m.kt_begin.p, m.kt_end.p, m.panel_w.p, m.panel_off.p, m.gcol.p,
                                        m.gcol_off.p, D, X, Y, skip);
    }
    k_mr_csr<<<cdiv((long long)N * R, 256), 256, 0, st>>>(N, R, m.nnear > 0 ? 1 : 0, m.rowptr.p, m.colidx.p,
                                                           op.valBM32.p, X, Y, skip);
    if (far) {
        const size_t need_p = (size_t)nlev * m.kt.nleaf * k * R, need_h = (size_t)m.kt.nnode * k * R;
        if (op.mr_part.n < need_p || op.mr_xh.n < need_h) {
            release_bgraph(op);   // a captured solve refers to the old workspace
            op.mr_part.alloc(need_p);
            op.mr_xh.alloc(need_h);
            op.mr_yh.alloc(need_h);
        }
        dim3 gp(m.kt.nleaf, nlev, cdiv(k * R, 128));
        k_mr_far_proj<T><<<gp, 128, 0, st>>>(fl, k, N, R, m.kt_begin.p, m.kt_end.p, Ul, X, op.mr_part.p, m.kt.nleaf,
                                            skip);
        const int nn = m.kt.nnode - ((1 << m.far_lmin) - 1);
        dim3 gs(nn, cdiv(k * R, 128));
        k_mr_far_sum<<<gs, 128, 0, st>>>(m.far_lmin, m.kt.L, k, R, m.kt.nleaf, op.mr_part.p, op.mr_xh.p, skip);
        dim3 gc(m.kt.nnode, cdiv(k * R, 128));
        k_mr_far_couple<T><<<gc, 128, 0, st>>>(k, R, m.far_ptr.p, m.far_col.p, S, op.mr_xh.p, op.mr_yh.p, skip);
        k_mr_far_expand<T><<<cdiv((long long)N * R, 256), 256, 0, st>>>(fl, m.far_lmin, m.kt.L, k, N, R, m.vleaf.p, Ul,
                                                                       op.mr_yh.p, Y, skip);
    }
    VFD_CUDA(cudaGetLastError());
}

// Y = A_low X for R (multiple of 64) interleaved FP32 columns
void mr_apply(const MeshData &m, OpData &op, const float *X, float *Y, int R, cudaStream_t st, const int *skip)
{
    VFD_REQUIRE(R % RT == 0, VFD_EINVAL, "batched apply needs a multiple of 64 columns");
    VFD_REQUIRE(m.max_leaf_size <= 64, VFD_EUNSUPPORTED, "batched apply needs leaves of at most 64 DoFs");
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
