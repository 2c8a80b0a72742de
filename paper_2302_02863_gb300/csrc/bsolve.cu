// Batched mixed-precision solve of A U = F for R right-hand sides (the CG of
// the paper's Sec. 7 run on all columns at once): iterative refinement with
// an FP64 residual F - A U from the FP64 operator, and an inner batched CG on
// the low-precision operator (K in TF32 or BF16 on the tensor cores, B + M in
// FP32) in FP32 vectors of interleaved layout [N][Rp] (Rp = R rounded up to
// 64).  Per-column scalars; deterministic per-column reductions (block
// partials summed in a fixed order by the last block); a device flag ends a
// captured chunk of iterations once every column has converged.
#include <algorithm>
#include <cmath>

#include "device_common.cuh"

namespace vfd {

void mr_apply(const MeshData &m, OpData &op, const float *X, float *Y, int R, cudaStream_t st, const int *skip);

namespace {

constexpr int BCHUNK = 8;
constexpr int BT = 1024;   // threads of the reduction kernels (one block per SM)
// per-column scalars (float arrays of Rp): rr, pq, alpha, beta, tol2
enum { C_RR = 0, C_PQ = 1, C_AL = 2, C_BE = 3, C_TOL = 4, C_N = 5 };
// flags (int): [0] all done, [1] iterations, [2] max_it, [3] counter
enum { BF_DONE = 0, BF_IT = 1, BF_MAX = 2, BF_CNT = 3 };

// Per-column sums over the rows of f(i, c); block = BT threads = (BT / Rc)
// row lanes x Rc columns with Rc = min(Rp, BT).  f may also update the
// vectors at (i, c): each block visits the same (i, c) set in every kernel
// that uses this helper, and reads only what it wrote itself.  The last block
// reduces the block partials in fixed order and calls fin(c, total); returns
// true in that block.
template <class Elem, class Fin>
__device__ bool col_reduce(int N, int Rp, Elem f, float *part, unsigned *cnt, Fin fin)
{
    __shared__ bool am_last;
    __shared__ float sh[BT];
    const int Rc = min(Rp, (int)blockDim.x), lanes = blockDim.x / Rc;
    for (int c0 = 0; c0 < Rp; c0 += Rc) {
        const int cl = threadIdx.x % Rc, c = c0 + cl, rl = threadIdx.x / Rc;
        const bool ok = rl < lanes && c < Rp;
        float v = 0.f;
        if (ok)
#pragma unroll 4
            for (int i = blockIdx.x * lanes + rl; i < N; i += gridDim.x * lanes) v += f((size_t)i * Rp + c);
        // fixed-order reduction over the row lanes of this block
        sh[threadIdx.x] = v;
        __syncthreads();
        if (rl == 0 && c < Rp) {
            float s = 0.f;
            for (int q = 0; q < lanes; ++q) s += sh[q * Rc + cl];
            part[(size_t)blockIdx.x * Rp + c] = s;
        }
        __syncthreads();
    }
    __threadfence();
    if (threadIdx.x == 0) {
        unsigned v = atomicInc(cnt, gridDim.x - 1);
        am_last = (v == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    // fixed-order reduction of the block partials: lane l of column c sums the
    // blocks l, l + lanes, ... ; the lanes are then summed in order
    for (int c0 = 0; c0 < Rp; c0 += Rc) {
        const int cl = threadIdx.x % Rc, c = c0 + cl, rl = threadIdx.x / Rc;
        float s = 0.f;
        if (rl < lanes && c < Rp)
            for (int bI = rl; bI < (int)gridDim.x; bI += lanes) s += __ldcg(part + (size_t)bI * Rp + c);
        sh[threadIdx.x] = s;
        __syncthreads();
        if (rl == 0 && c < Rp) {
            float tot = 0.f;
            for (int q = 0; q < lanes; ++q) tot += sh[q * Rc + cl];
            fin(c, tot);
        }
        __syncthreads();
    }
    return true;
}

__global__ void __launch_bounds__(BT) k_b_init(int N, int Rp, const float *__restrict__ b, float *__restrict__ x,
                                                float *__restrict__ r, float *__restrict__ p, float *part,
                                                unsigned *cnt, float *sc, int *flag, float tol, int max_it)
{
    col_reduce(
        N, Rp,
        [&](size_t t) {
            const float v = b[t];
            x[t] = 0.f;
            r[t] = v;
            p[t] = v;
            return v * v;
        },
        part, cnt, [&](int c, float s) {
            sc[C_RR * Rp + c] = s;
            sc[C_TOL * Rp + c] = tol * tol * s;
            sc[C_AL * Rp + c] = 0.f;
            sc[C_BE * Rp + c] = 0.f;
        });
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        flag[BF_IT] = 0;
        flag[BF_MAX] = max_it;
        flag[BF_DONE] = max_it <= 0 ? 1 : 0;
    }
}

// pq = p.q per column; alpha = rr / pq (0 for converged columns)
__global__ void __launch_bounds__(BT) k_b_pq(int N, int Rp, const float *__restrict__ p, const float *__restrict__ q,
                                              float *part, unsigned *cnt, float *sc, const int *flag)
{
    if (flag[BF_DONE]) return;
    col_reduce(
        N, Rp, [&](size_t t) { return p[t] * q[t]; }, part, cnt,
        [&](int c, float s) {
            float rr = sc[C_RR * Rp + c];
            bool live = rr > sc[C_TOL * Rp + c] && s > 0.f;
            sc[C_PQ * Rp + c] = s;
            sc[C_AL * Rp + c] = live ? rr / s : 0.f;
        });
}

// x += alpha p; r -= alpha q; rr_new; beta; convergence of every column
__global__ void __launch_bounds__(BT) k_b_xr(int N, int Rp, float *__restrict__ x, float *__restrict__ r,
                                              const float *__restrict__ p, const float *__restrict__ q, float *part,
                                              unsigned *cnt, float *sc, int *flag)
{
    if (flag[BF_DONE]) return;
    __shared__ int live;
    if (threadIdx.x == 0) live = 0;
    __syncthreads();
    const bool last = col_reduce(
        N, Rp,
        [&](size_t t) {
            const float al = sc[C_AL * Rp + (int)(t % Rp)];
            x[t] = fmaf(al, p[t], x[t]);
            const float rn = fmaf(-al, q[t], r[t]);
            r[t] = rn;
            return rn * rn;
        },
        part, cnt, [&](int c, float s) {
            float rr = sc[C_RR * Rp + c];
            bool was_live = sc[C_AL * Rp + c] != 0.f;
            if (was_live) {
                sc[C_BE * Rp + c] = rr > 0.f ? s / rr : 0.f;
                sc[C_RR * Rp + c] = s;
                if (s > sc[C_TOL * Rp + c]) atomicAdd(&live, 1);
            } else {
                sc[C_BE * Rp + c] = 0.f;
            }
        });
    if (!last) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        int it = flag[BF_IT] + 1;
        flag[BF_IT] = it;
        if (live == 0 || it >= flag[BF_MAX]) flag[BF_DONE] = 1;
    }
}

__global__ void k_b_p(int N, int Rp, const float *__restrict__ r, float *__restrict__ p, const float *sc,
                      const int *flag)
{
    if (flag[BF_DONE]) return;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)N * Rp; t += gridDim.x * blockDim.x)
        p[t] = fmaf(sc[C_BE * Rp + (int)(t % Rp)], p[t], r[t]);
}

// residual scaling between the FP64 column-major and the FP32 interleaved layouts
__global__ void k_b_to_inner(int N, int R, int Rp, int64_t ld, const double *__restrict__ res,
                             const double *__restrict__ scale, float *__restrict__ b)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * Rp) return;
    const int i = (int)(t / Rp), c = (int)(t % Rp);
    b[t] = (c < R && scale[c] > 0.0) ? (float)(res[(size_t)c * ld + i] / scale[c]) : 0.f;
}

__global__ void k_b_from_inner(int N, int R, int Rp, int64_t ld, const float *__restrict__ z,
                               const double *__restrict__ scale, double *__restrict__ U)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * R) return;
    const int c = (int)(t / N), i = (int)(t % N);
    if (scale[c] > 0.0) U[(size_t)c * ld + i] += scale[c] * (double)z[(size_t)i * Rp + c];
}

// res = F - AU (column-major FP64), and per-column norms^2 (FP64, one block per column)
__global__ void k_b_resid(int N, int64_t ld, const double *__restrict__ F, const double *__restrict__ AU,
                          double *__restrict__ res, double *__restrict__ nrm2, double *__restrict__ fn2)
{
    __shared__ double sh[32];
    const int c = blockIdx.x;
    double v = 0.0, f = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double d = F[(size_t)c * ld + i] - AU[(size_t)c * ld + i];
        res[(size_t)c * ld + i] = d;
        v += d * d;
        f += F[(size_t)c * ld + i] * F[(size_t)c * ld + i];
    }
    v = warp_sum(v);
    f = warp_sum(f);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sh[q];
        nrm2[c] = s;
    }
    __syncthreads();
    if (l == 0) sh[w] = f;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) s += sh[q];
        fn2[c] = s;
    }
}


}  // namespace

void apply_parts_ex(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                    bool lowp, cudaStream_t st, const int *skip);

void release_bgraph(OpData &op);

// blocks of the column reductions: one per SM of the current device
static int nb_reduce()
{
    int dev = 0, nsm = 0;
    VFD_CUDA(cudaGetDevice(&dev));
    VFD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    return std::max(1, nsm);
}

// inner batched CG: z ~ A_low^-1 b on op.mb_b (interleaved [N][Rp]); returns iterations
static int run_bcg(const MeshData &m, OpData &op, int Rp, float tol, int max_it, cudaStream_t st)
{
    const int N = m.N;
    const int VB = std::max(1, std::min(cdiv((long long)N * Rp, 256), 2048));
    unsigned *cnt = (unsigned *)(op.mb_flag.p + BF_CNT);
    k_b_init<<<nb_reduce(), BT, 0, st>>>(N, Rp, op.mb_b.p, op.mb_x.p, op.mb_r.p, op.mb_p.p, op.mb_part.p, cnt, op.mb_sc.p,
                                  op.mb_flag.p, tol, max_it);
    VFD_CUDA(cudaGetLastError());
    // eager apply first: allocates the apply workspace outside the capture
    mr_apply(m, op, op.mb_p.p, op.mb_q.p, Rp, st, nullptr);
    if (!op.mb_exec || op.mb_key != (const void *)op.mb_p.p || op.mb_R != Rp) {
        if (op.mb_exec) cudaGraphExecDestroy(op.mb_exec);
        op.mb_exec = nullptr;
        cudaStream_t cs;
        VFD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph;
        VFD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            for (int it = 0; it < BCHUNK; ++it) {
                mr_apply(m, op, op.mb_p.p, op.mb_q.p, Rp, cs, op.mb_flag.p);
                k_b_pq<<<nb_reduce(), BT, 0, cs>>>(N, Rp, op.mb_p.p, op.mb_q.p, op.mb_part.p, cnt, op.mb_sc.p, op.mb_flag.p);
                k_b_xr<<<nb_reduce(), BT, 0, cs>>>(N, Rp, op.mb_x.p, op.mb_r.p, op.mb_p.p, op.mb_q.p, op.mb_part.p, cnt,
                                            op.mb_sc.p, op.mb_flag.p);
                k_b_p<<<VB, 256, 0, cs>>>(N, Rp, op.mb_r.p, op.mb_p.p, op.mb_sc.p, op.mb_flag.p);
            }
        } catch (...) {
            cudaStreamEndCapture(cs, &graph);
            cudaStreamDestroy(cs);
            throw;
        }
        VFD_CUDA(cudaStreamEndCapture(cs, &graph));
        cudaStreamDestroy(cs);
        cudaError_t ie = cudaGraphInstantiate(&op.mb_exec, graph, 0);
        cudaGraphDestroy(graph);
        VFD_CUDA(ie);
        op.mb_key = op.mb_p.p;
        op.mb_R = Rp;
    }
    int hf[3] = {0, 0, 0};
    while (true) {
        VFD_CUDA(cudaGraphLaunch(op.mb_exec, st));
        VFD_CUDA(cudaMemcpyAsync(hf, op.mb_flag.p, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaStreamSynchronize(st));
        if (hf[BF_DONE]) break;
    }
    return hf[BF_IT];
}

// R columns of F, U (FP64, column-major, leading dimension ld, device)
vfd_status batched_solve(const MeshData &m, OpData &op, const double *F, double *U, int R, int64_t ld, double rtol,
                         int max_it, int *iters, double *relres, cudaStream_t st)
{
    const int N = m.N, Rp = ((R + 63) / 64) * 64;
    const size_t nv = (size_t)N * Rp;
    if (op.mb_x.n != nv || op.mb_sc.n != (size_t)C_N * Rp) {
        release_bgraph(op);   // the captured chunk refers to these buffers
        op.mb_x.alloc(nv);
        op.mb_r.alloc(nv);
        op.mb_p.alloc(nv);
        op.mb_q.alloc(nv);
        op.mb_b.alloc(nv);
        op.mb_part.alloc((size_t)nb_reduce() * Rp);
        op.mb_sc.alloc((size_t)C_N * Rp);
    }
    if (op.mb_flag.n < 8) {
        op.mb_flag.alloc(8);
        VFD_CUDA(cudaMemsetAsync(op.mb_flag.p, 0, 8 * sizeof(int), st));
    }
    DBuf<double> AU, res, n2, f2, scale;
    AU.alloc((size_t)ld * R);
    res.alloc((size_t)ld * R);
    n2.alloc(R);
    f2.alloc(R);
    scale.alloc(R);
    std::vector<double> hn(R), hf(R);
    int total = 0;
    const float inner_tol = 1e-4f;
    vfd_status status = VFD_ENOCONV;   // until every column meets rtol
    for (int outer = 0; outer < 100; ++outer) {
        // FP64 residual with the FP64 operator
        apply_parts_ex(m, op, VFD_PART_ALL, U, AU.p, R, ld, false, st, nullptr);
        k_b_resid<<<R, 256, 0, st>>>(N, ld, F, AU.p, res.p, n2.p, f2.p);
        VFD_CUDA(cudaGetLastError());
        VFD_CUDA(cudaMemcpyAsync(hn.data(), n2.p, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaMemcpyAsync(hf.data(), f2.p, sizeof(double) * R, cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaStreamSynchronize(st));
        bool all = true;
        std::vector<double> sc(R);
        for (int c = 0; c < R; ++c) {
            double rel = hf[c] > 0.0 ? std::sqrt(hn[c] / hf[c]) : std::sqrt(hn[c]);
            if (relres) relres[c] = rel;
            // converged columns get scale 0: no correction, zero inner RHS
            sc[c] = (rel > rtol) ? std::sqrt(hn[c]) : 0.0;
            if (rel > rtol) all = false;
        }
        if (all) {
            status = VFD_OK;
            break;
        }
        if (total >= max_it) break;
        VFD_CUDA(cudaMemcpyAsync(scale.p, sc.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
        k_b_to_inner<<<cdiv((long long)N * Rp, 256), 256, 0, st>>>(N, R, Rp, ld, res.p, scale.p, op.mb_b.p);
        total += run_bcg(m, op, Rp, inner_tol, std::max(1, max_it - total), st);
        k_b_from_inner<<<cdiv((long long)N * R, 256), 256, 0, st>>>(N, R, Rp, ld, op.mb_x.p, scale.p, U);
        VFD_CUDA(cudaGetLastError());
    }
    VFD_CUDA(cudaStreamSynchronize(st));
    if (iters)
        for (int c = 0; c < R; ++c) iters[c] = total;
    return status;
}

void release_bgraph(OpData &op)
{
    if (op.mb_exec) {
        cudaGraphExecDestroy(op.mb_exec);
        op.mb_exec = nullptr;
    }
}

}  // namespace vfd
