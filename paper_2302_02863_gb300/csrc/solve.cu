// Conjugate gradients on the device (the paper solves with CG, Sec. 7), with
// deterministic reductions (block partials summed in a fixed order by the
// last block to finish; no float atomics, no spin-wait) and a device-side
// convergence flag that turns the remaining kernels of a captured chunk of
// iterations into no-ops.  The host replays one captured CUDA graph per
// chunk and reads the flag once per chunk.
//
// For VFD_FP32 and VFD_BF16 operators the single-column solve is iterative
// refinement: FP64 residual r = F - A U with the FP64 operator, inner CG on
// the operator whose K part is FP32, U += correction.
#include <algorithm>
#include <cmath>

#include "device_common.cuh"

namespace vfd {

void apply_parts_ex(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                    bool lowp, cudaStream_t st, const int *skip);

namespace {

constexpr int RB = 256;        // reduction block size
constexpr int CHUNK = 8;       // CG iterations per captured graph
enum { S_RR = 0, S_PQ = 1, S_BB = 2, S_TOL2 = 3, S_BETA = 4, S_TMP = 5 };   // 6, 7: PCG (r.z)
enum { F_DONE = 0, F_ITERS = 1, F_MAXIT = 2, F_CNT = 4 };  // F_CNT..F_CNT+3: block counters

int red_blocks(int n) { return std::max(1, std::min(cdiv(n, RB * 4), 264)); }

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;  // valid in thread 0
}

// returns true in the (single) last block; its thread 0 gets the ordered sum in *total
__device__ bool last_block_sum(double mine, double *part, unsigned *cnt, double *total, double *sh)
{
    __shared__ bool am_last;
    double b = block_sum(mine, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x] = b;
        __threadfence();
        unsigned v = atomicInc(cnt, gridDim.x - 1);
        am_last = (v == gridDim.x - 1);
    }
    __syncthreads();
    if (!am_last) return false;
    __threadfence();
    double t = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += ((volatile double *)part)[i];
    // fixed-order combination: thread i sums indices i, i+RB, ...; then block_sum
    double s = block_sum(t, sh);
    if (threadIdx.x == 0) *total = s;
    return true;
}

// scal[slot] = a . b
__global__ void __launch_bounds__(RB) k_dot(int n, const double *__restrict__ a, const double *__restrict__ b,
                                            double *part, unsigned *cnt, double *scal, int slot, const int *flag)
{
    __shared__ double sh[32];
    if (flag && flag[F_DONE]) return;
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v += a[i] * b[i];
    double tot;
    if (last_block_sum(v, part, cnt, &tot, sh) && threadIdx.x == 0) scal[slot] = tot;
}

// r = b - q; p = r
__global__ void k_init_rp(int n, const double *__restrict__ b, const double *__restrict__ q, double *__restrict__ r,
                          double *__restrict__ p)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double v = b[i] - q[i];
        r[i] = v;
        p[i] = v;
    }
}

__global__ void k_init_flag(int *flag, double *scal, double rtol, int max_it)
{
    double tol2 = rtol * rtol * scal[S_BB];
    scal[S_TOL2] = tol2;
    flag[F_DONE] = (scal[S_RR] <= tol2) ? 1 : 0;
    flag[F_ITERS] = 0;
    flag[F_MAXIT] = max_it;
    if (max_it <= 0) flag[F_DONE] = 1;
}

// alpha = rr / pq; x += alpha p; r -= alpha q; rr_new = r.r; convergence test
__global__ void __launch_bounds__(RB) k_cg_xr(int n, double *__restrict__ x, double *__restrict__ r,
                                              const double *__restrict__ p, const double *__restrict__ q,
                                              double *part, unsigned *cnt, double *scal, int *flag)
{
    __shared__ double sh[32];
    if (flag[F_DONE]) return;
    const double rr = scal[S_RR], pq = scal[S_PQ];
    const double alpha = (pq != 0.0) ? rr / pq : 0.0;
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        double ri = r[i] - alpha * q[i];
        r[i] = ri;
        v += ri * ri;
    }
    double rrn;
    if (last_block_sum(v, part, cnt, &rrn, sh) && threadIdx.x == 0) {
        int it = flag[F_ITERS] + 1;
        flag[F_ITERS] = it;
        scal[S_BETA] = (rr != 0.0) ? rrn / rr : 0.0;
        scal[S_RR] = rrn;
        if (rrn <= scal[S_TOL2] || it >= flag[F_MAXIT] || !(pq > 0.0)) flag[F_DONE] = 1;
    }
}

__global__ void k_cg_p(int n, const double *__restrict__ r, double *__restrict__ p, const double *scal,
                       const int *flag)
{
    if (flag[F_DONE]) return;
    const double beta = scal[S_BETA];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = r[i] + beta * p[i];
}

__global__ void k_axpy(int n, double a, const double *__restrict__ x, double *__restrict__ y)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) y[i] += a * x[i];
}

__global__ void k_sub(int n, const double *__restrict__ b, const double *__restrict__ q, double *__restrict__ r)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) r[i] = b[i] - q[i];
}

}  // namespace

void release_graphs(OpData &op)
{
    for (int i = 0; i < 2; ++i)
        if (op.cg_exec[i]) {
            cudaGraphExecDestroy(op.cg_exec[i]);
            op.cg_exec[i] = nullptr;
            op.cg_key[i] = nullptr;
        }
    if (op.pcg_exec) {
        cudaGraphExecDestroy(op.pcg_exec);
        op.pcg_exec = nullptr;
        op.pcg_key = nullptr;
    }
}

// CG on (lowp ? A32 : A64) z = b, b and z in op.cg_b / op.cg_x (device, n).
// Returns iterations; *rr_final = final recursive residual^2, *bb = b.b.
static int run_cg(const MeshData &m, OpData &op, bool lowp, double rtol, int max_it, cudaStream_t st, double *rr_out,
                  double *bb_out)
{
    const int n = m.N, NB = red_blocks(n), VB = std::max(1, std::min(cdiv(n, RB), 1024));
    double *part = op.cg_red.p;
    unsigned *cnt = (unsigned *)(op.cg_flag.p + F_CNT);
    int *flag = op.cg_flag.p;
    double *scal = op.cg_scal.p;
    // init: q = A x; r = b - q; p = r; bb, rr
    apply_parts_ex(m, op, VFD_PART_ALL, op.cg_x.p, op.cg_q.p, 1, n, lowp, st, nullptr);
    k_init_rp<<<VB, RB, 0, st>>>(n, op.cg_b.p, op.cg_q.p, op.cg_r.p, op.cg_p.p);
    k_dot<<<NB, RB, 0, st>>>(n, op.cg_b.p, op.cg_b.p, part, cnt, scal, S_BB, nullptr);
    k_dot<<<NB, RB, 0, st>>>(n, op.cg_r.p, op.cg_r.p, part, cnt, scal, S_RR, nullptr);
    k_init_flag<<<1, 1, 0, st>>>(flag, scal, rtol, max_it);
    VFD_CUDA(cudaGetLastError());
    cudaGraphExec_t &gexec = op.cg_exec[lowp ? 1 : 0];
    const void *&gkey = op.cg_key[lowp ? 1 : 0];
    if (!gexec || gkey != (const void *)op.cg_p.p) {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        cudaStream_t cs;
        VFD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph;
        VFD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            for (int it = 0; it < CHUNK; ++it) {
                apply_parts_ex(m, op, VFD_PART_ALL, op.cg_p.p, op.cg_q.p, 1, n, lowp, cs, flag);
                k_dot<<<NB, RB, 0, cs>>>(n, op.cg_p.p, op.cg_q.p, part, cnt, scal, S_PQ, flag);
                k_cg_xr<<<NB, RB, 0, cs>>>(n, op.cg_x.p, op.cg_r.p, op.cg_p.p, op.cg_q.p, part, cnt, scal, flag);
                k_cg_p<<<VB, RB, 0, cs>>>(n, op.cg_r.p, op.cg_p.p, scal, flag);
            }
        } catch (...) {
            cudaStreamEndCapture(cs, &graph);
            cudaStreamDestroy(cs);
            throw;
        }
        VFD_CUDA(cudaStreamEndCapture(cs, &graph));
        cudaStreamDestroy(cs);
        cudaError_t ie = cudaGraphInstantiate(&gexec, graph, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(graph);
        VFD_CUDA(ie);
        gkey = op.cg_p.p;
    }
    int hflag[3] = {0, 0, 0};
    while (true) {
        VFD_CUDA(cudaGraphLaunch(gexec, st));
        VFD_CUDA(cudaMemcpyAsync(hflag, flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaStreamSynchronize(st));
        if (hflag[F_DONE]) break;
    }
    double hs[3];
    VFD_CUDA(cudaMemcpy(hs, scal, 3 * sizeof(double), cudaMemcpyDeviceToHost));
    *rr_out = hs[S_RR];
    *bb_out = hs[S_BB];
    return hflag[F_ITERS];
}

static void ensure_ws(const MeshData &m, OpData &op)
{
    const int n = m.N;
    if (op.cg_r.n != (size_t)n) {
        op.cg_r.alloc(n);
        op.cg_p.alloc(n);
        op.cg_q.alloc(n);
        op.cg_x.alloc(n);
        op.cg_b.alloc(n);
        op.cg_z.alloc(n);
        op.cg_red.alloc(1024);
        op.cg_scal.alloc(8);
        op.cg_flag.alloc(8);
        VFD_CUDA(cudaMemset(op.cg_flag.p, 0, 8 * sizeof(int)));
    }
}

static double dev_dot(const MeshData &m, OpData &op, const double *a, const double *b, cudaStream_t st)
{
    const int n = m.N, NB = red_blocks(n);
    k_dot<<<NB, RB, 0, st>>>(n, a, b, op.cg_red.p, (unsigned *)(op.cg_flag.p + F_CNT), op.cg_scal.p, S_TMP, nullptr);
    VFD_CUDA(cudaGetLastError());
    double v;
    VFD_CUDA(cudaMemcpyAsync(&v, op.cg_scal.p + S_TMP, sizeof(double), cudaMemcpyDeviceToHost, st));
    VFD_CUDA(cudaStreamSynchronize(st));
    return v;
}

// ---------------------------------------------------------------------------
// preconditioned CG (two-level preconditioner of precond.cu):
//   z = M^-1 r = (block inverse of the leaf's diagonal block) r + R^T A_c^-1 R r
// with R the leaf-indicator restriction.  Scalars: S_RZ = r.z, S_RZN = the new
// r.z, S_RR = r.r (the stopping test is on the true recursive residual r).
// ---------------------------------------------------------------------------
namespace {
enum { S_RZ = 6, S_RZN = 7 };

// alpha = rz / pq; x += alpha p; r -= alpha q; rr = r.r; convergence test
__global__ void __launch_bounds__(RB) k_pcg_xr(int n, double *__restrict__ x, double *__restrict__ r,
                                               const double *__restrict__ p, const double *__restrict__ q,
                                               double *part, unsigned *cnt, double *scal, int *flag)
{
    __shared__ double sh[32];
    if (flag[F_DONE]) return;
    const double rz = scal[S_RZ], pq = scal[S_PQ];
    const double alpha = (pq != 0.0) ? rz / pq : 0.0;
    double v = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        r[i] = ri;
        v += ri * ri;
    }
    double rrn;
    if (last_block_sum(v, part, cnt, &rrn, sh) && threadIdx.x == 0) {
        const int it = flag[F_ITERS] + 1;
        flag[F_ITERS] = it;
        scal[S_RR] = rrn;
        if (rrn <= scal[S_TOL2] || it >= flag[F_MAXIT] || !(pq > 0.0)) flag[F_DONE] = 1;
    }
}

// p = z + (rz_new / rz) p; rz = rz_new
__global__ void k_pcg_p(int n, const double *__restrict__ z, double *__restrict__ p, double *scal, const int *flag)
{
    if (flag[F_DONE]) return;
    const double rzn = scal[S_RZN], rz = scal[S_RZ];
    const double beta = rz != 0.0 ? rzn / rz : 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = z[i] + beta * p[i];
}

__global__ void k_pcg_rz_commit(double *scal, const int *flag)
{
    if (flag && flag[F_DONE]) return;
    scal[S_RZ] = scal[S_RZN];
}
}  // namespace

// z = M^-1 r (precond.cu)
void precond_apply(const MeshData &m, const OpData &op, const double *r, double *z, cudaStream_t st, const int *skip);

static int run_pcg(const MeshData &m, OpData &op, double rtol, int max_it, cudaStream_t st, double *rr_out,
                   double *bb_out)
{
    const int n = m.N, NB = red_blocks(n), VB = std::max(1, std::min(cdiv(n, RB), 1024));
    double *part = op.cg_red.p;
    unsigned *cnt = (unsigned *)(op.cg_flag.p + F_CNT);
    int *flag = op.cg_flag.p;
    double *scal = op.cg_scal.p;
    // init: r = b - A x; z = M^-1 r; p = z; rz = r.z; bb; rr
    apply_parts_ex(m, op, VFD_PART_ALL, op.cg_x.p, op.cg_q.p, 1, n, false, st, nullptr);
    k_sub<<<VB, RB, 0, st>>>(n, op.cg_b.p, op.cg_q.p, op.cg_r.p);
    precond_apply(m, op, op.cg_r.p, op.cg_z.p, st, nullptr);
    VFD_CUDA(cudaMemcpyAsync(op.cg_p.p, op.cg_z.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
    k_dot<<<NB, RB, 0, st>>>(n, op.cg_b.p, op.cg_b.p, part, cnt, scal, S_BB, nullptr);
    k_dot<<<NB, RB, 0, st>>>(n, op.cg_r.p, op.cg_r.p, part, cnt, scal, S_RR, nullptr);
    k_dot<<<NB, RB, 0, st>>>(n, op.cg_r.p, op.cg_z.p, part, cnt, scal, S_RZ, nullptr);
    k_init_flag<<<1, 1, 0, st>>>(flag, scal, rtol, max_it);
    VFD_CUDA(cudaGetLastError());
    cudaGraphExec_t &gexec = op.pcg_exec;
    if (!gexec || op.pcg_key != (const void *)op.cg_p.p) {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        cudaStream_t cs;
        VFD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t graph;
        VFD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        try {
            for (int it = 0; it < CHUNK; ++it) {
                apply_parts_ex(m, op, VFD_PART_ALL, op.cg_p.p, op.cg_q.p, 1, n, false, cs, flag);
                k_dot<<<NB, RB, 0, cs>>>(n, op.cg_p.p, op.cg_q.p, part, cnt, scal, S_PQ, flag);
                k_pcg_xr<<<NB, RB, 0, cs>>>(n, op.cg_x.p, op.cg_r.p, op.cg_p.p, op.cg_q.p, part, cnt, scal, flag);
                precond_apply(m, op, op.cg_r.p, op.cg_z.p, cs, flag);
                k_dot<<<NB, RB, 0, cs>>>(n, op.cg_r.p, op.cg_z.p, part, cnt, scal, S_RZN, flag);
                k_pcg_p<<<VB, RB, 0, cs>>>(n, op.cg_z.p, op.cg_p.p, scal, flag);
                k_pcg_rz_commit<<<1, 1, 0, cs>>>(scal, flag);
            }
        } catch (...) {
            cudaStreamEndCapture(cs, &graph);
            cudaStreamDestroy(cs);
            throw;
        }
        VFD_CUDA(cudaStreamEndCapture(cs, &graph));
        cudaStreamDestroy(cs);
        cudaError_t ie = cudaGraphInstantiate(&gexec, graph, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(graph);
        VFD_CUDA(ie);
        op.pcg_key = op.cg_p.p;
    }
    int hflag[3] = {0, 0, 0};
    while (true) {
        VFD_CUDA(cudaGraphLaunch(gexec, st));
        VFD_CUDA(cudaMemcpyAsync(hflag, flag, 3 * sizeof(int), cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaStreamSynchronize(st));
        if (hflag[F_DONE]) break;
    }
    double hs[3];
    VFD_CUDA(cudaMemcpy(hs, scal, 3 * sizeof(double), cudaMemcpyDeviceToHost));
    *rr_out = hs[S_RR];
    *bb_out = hs[S_BB];
    return hflag[F_ITERS];
}

vfd_status cg_solve(const MeshData &m, OpData &op, const double *F, double *U, int nrhs, int64_t ld, double rtol,
                    int max_it, int *iters, double *relres, cudaStream_t st)
{
    ensure_ws(m, op);
    const int n = m.N, VB = std::max(1, std::min(cdiv(n, RB), 1024));
    vfd_status status = VFD_OK;
    for (int r = 0; r < nrhs; ++r) {
        const double *f = F + (size_t)r * ld;
        double *u = U + (size_t)r * ld;
        int total = 0;
        double rel = 0.0;
        if (op.precision == VFD_FP64) {
            VFD_CUDA(cudaMemcpyAsync(op.cg_b.p, f, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            VFD_CUDA(cudaMemcpyAsync(op.cg_x.p, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
            // CG; when the recursive residual has converged but the true
            // residual of the iterate has not, restart from the iterate
            // (residual replacement), at most a few times
            for (int restart = 0; restart < 4; ++restart) {
                double rr, bb;
                total += op.prec_kind ? run_pcg(m, op, rtol, max_it - total, st, &rr, &bb)
                                      : run_cg(m, op, false, rtol, max_it - total, st, &rr, &bb);
                apply_parts_ex(m, op, VFD_PART_ALL, op.cg_x.p, op.cg_q.p, 1, n, false, st, nullptr);
                k_sub<<<VB, RB, 0, st>>>(n, f, op.cg_q.p, op.cg_r.p);
                double res2 = dev_dot(m, op, op.cg_r.p, op.cg_r.p, st);
                rel = (bb > 0.0) ? std::sqrt(res2 / bb) : std::sqrt(res2);
                if (rel <= rtol || total >= max_it) break;
            }
            VFD_CUDA(cudaMemcpyAsync(u, op.cg_x.p, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
        } else {
            // iterative refinement: outer FP64 residual, inner CG with FP32 K
            double bb = dev_dot(m, op, f, f, st);
            const double inner_tol = 1e-5;
            int outer = 0;
            while (true) {
                apply_parts_ex(m, op, VFD_PART_ALL, u, op.cg_q.p, 1, n, false, st, nullptr);
                k_sub<<<VB, RB, 0, st>>>(n, f, op.cg_q.p, op.cg_b.p);
                double res2 = dev_dot(m, op, op.cg_b.p, op.cg_b.p, st);
                rel = (bb > 0.0) ? std::sqrt(res2 / bb) : std::sqrt(res2);
                if (rel <= rtol || total >= max_it || outer >= 50) break;
                VFD_CUDA(cudaMemsetAsync(op.cg_x.p, 0, sizeof(double) * n, st));
                double rr, bb2;
                total += run_cg(m, op, true, inner_tol, max_it - total, st, &rr, &bb2);
                k_axpy<<<VB, RB, 0, st>>>(n, 1.0, op.cg_x.p, u);
                VFD_CUDA(cudaGetLastError());
                ++outer;
            }
        }
        if (iters) iters[r] = total;
        if (relres) relres[r] = rel;
        if (!(rel <= rtol)) status = VFD_ENOCONV;
    }
    return status;
}

}  // namespace vfd
