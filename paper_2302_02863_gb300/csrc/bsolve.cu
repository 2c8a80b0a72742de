// Batched mixed-precision solve of A_m U_m = F_m for a batch of operators
// (meshes) m with R right-hand sides each (the CG of the paper's Sec. 7 run
// on all columns of all meshes at once): CG on the low-precision operators
// (K in TF32 or BF16 on the tensor cores, B + M in FP32) in FP32 vectors of
// interleaved layout [sum N_m][Rp] (Rp = R rounded up to 64), solving for the
// correction to the FP64 iterate U, with reliable updates per mesh: once every
// still-iterating column of a mesh has cut its recursive residual by RU_DROP
// since that mesh's last update (or the mesh's inner iteration has
// converged), the mesh's correction is added to U in FP64, its true residual
// F - A U is recomputed with the FP64 operator and replaces the recursive one,
// and the search direction continues as p = r_true + beta p_old with beta
// taken from the true residual norm -- the Krylov space is not restarted, so
// the iteration count stays close to that of FP64 CG (the first step after an
// update takes the exact line search r.p / p.Ap, which keeps the iteration a
// descent method whatever the kept direction).  A column restarts from
// p = r_true instead (an iterative-refinement step) when its inner iteration
// had converged, when its true and recursive residuals differ by more than a
// factor of two, or when its true residual grew since the last update.  Other
// meshes keep iterating untouched.  Scalars per (mesh, column); deterministic
// segmented reductions (every reduction block works inside one mesh; the last
// block of a mesh sums that mesh's block partials in a fixed order); a device
// flag ends a captured chunk of iterations once every column of every mesh
// has converged.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "device_common.cuh"

namespace vfd {

namespace {

constexpr int BCHUNK = 8;
constexpr int BT = 1024;   // threads of the reduction kernels
// per (mesh, column) scalars, arrays of nmesh * Rp floats: rr, pq, alpha, beta,
// tol2, and rp = r.p (equal to rr except right after a reliable update)
// and rz = r.z of the preconditioned iteration
enum { C_RR = 0, C_PQ = 1, C_AL = 2, C_BE = 3, C_TOL = 4, C_RP = 5, C_RZ = 6, C_N = 7 };
// flags (int): [0] all done, [1] iterations, [2] max_it, [3] mesh-finish counter,
// then per mesh: a block counter (FL_CNT + m), its live-column count
// (FL_CNT + nmesh + m) and its done flag (FL_CNT + 2 nmesh + m: every column
// converged; its blocks then skip all element work and the apply skips it)
enum { BF_DONE = 0, BF_IT = 1, BF_MAX = 2, BF_GCNT = 3, FL_CNT = 4 };

struct Seg {
    int nmesh, Rp;
    const int *items;        // per block: mesh, index of the block inside the mesh
    const int *mesh;         // per mesh: first block, blocks, rows, first row
    float *red;              // block partials, nred x Rp
    int *flag;
    float *sc;               // C_N x (nmesh * Rp)
    __device__ int *mdone() const { return flag + FL_CNT + 2 * nmesh; }
};

__device__ __forceinline__ float &scal(const Seg &S, int kind, int m, int c)
{
    return S.sc[(size_t)kind * S.nmesh * S.Rp + (size_t)m * S.Rp + c];
}

// Per-(mesh, column) sums over the mesh's rows of f(global element index).
// Block = BT threads = (BT / Rc) row lanes x Rc columns, Rc = min(Rp, BT); the
// blocks of a mesh stride over its rows.  f may also update the vectors at
// its element: every kernel using this helper visits the same elements in
// the same block, and a block reads only what it wrote itself.  The last
// block of the mesh reduces the mesh's partials in a fixed order and calls
// fin(mesh, c, total); returns the mesh in that block, else -1.  With
// check_done, a mesh whose done flag is set does no element work and no fin
// (its blocks still take part in the counting).
template <bool check_done, class Elem, class Fin>
__device__ int seg_reduce(const Seg &S, Elem f, Fin fin)
{
    __shared__ bool am_last;
    __shared__ float sh[BT];
    const int m = S.items[2 * blockIdx.x], j = S.items[2 * blockIdx.x + 1];
    const bool work = !check_done || !S.mdone()[m];
    const int b0 = S.mesh[4 * m], nb = S.mesh[4 * m + 1], N = S.mesh[4 * m + 2], r0 = S.mesh[4 * m + 3];
    const int Rp = S.Rp, Rc = min(Rp, (int)blockDim.x), lanes = blockDim.x / Rc;
    for (int c0 = 0; c0 < Rp; c0 += Rc) {
        const int cl = threadIdx.x % Rc, c = c0 + cl, rl = threadIdx.x / Rc;
        float v = 0.f;
        if (work && rl < lanes && c < Rp)
#pragma unroll 4
            for (int i = j * lanes + rl; i < N; i += nb * lanes) v += f((size_t)(r0 + i) * Rp + c, m, c);
        sh[threadIdx.x] = v;
        __syncthreads();
        if (rl == 0 && c < Rp) {
            float s = 0.f;
            for (int q = 0; q < lanes; ++q) s += sh[q * Rc + cl];
            S.red[(size_t)blockIdx.x * Rp + c] = s;
        }
        __syncthreads();
    }
    __threadfence();
    if (threadIdx.x == 0) {
        unsigned v = atomicInc((unsigned *)&S.flag[FL_CNT + m], nb - 1);
        am_last = (v == (unsigned)(nb - 1));
    }
    __syncthreads();
    if (!am_last) return -1;
    __threadfence();
    for (int c0 = 0; c0 < Rp; c0 += Rc) {
        const int cl = threadIdx.x % Rc, c = c0 + cl, rl = threadIdx.x / Rc;
        float s = 0.f;
        if (rl < lanes && c < Rp)
            for (int bI = rl; bI < nb; bI += lanes) s += __ldcg(S.red + (size_t)(b0 + bI) * Rp + c);
        sh[threadIdx.x] = s;
        __syncthreads();
        if (work && rl == 0 && c < Rp) {
            float tot = 0.f;
            for (int q = 0; q < lanes; ++q) tot += sh[q * Rc + cl];
            fin(m, c, tot);
        }
        __syncthreads();
    }
    return m;
}

// x = 0, r = p = b; per column the stopping threshold tol2 (on rr, scaled units)
__global__ void __launch_bounds__(BT) k_b_init(Seg S, const float *__restrict__ b, float *__restrict__ x,
                                               float *__restrict__ r, float *__restrict__ p,
                                               const float *__restrict__ tol2, int max_it)
{
    __shared__ int live;
    if (threadIdx.x == 0) live = 0;
    __syncthreads();
    const int m = seg_reduce<false>(
        S,
        [&](size_t t, int, int) {
            const float v = b[t];
            x[t] = 0.f;
            r[t] = v;
            p[t] = v;
            return v * v;
        },
        [&](int m, int c, float s) {
            scal(S, C_RR, m, c) = s;
            scal(S, C_RP, m, c) = s;
            scal(S, C_TOL, m, c) = tol2[m * S.Rp + c];
            scal(S, C_AL, m, c) = 0.f;
            scal(S, C_BE, m, c) = 0.f;
            if (s > tol2[m * S.Rp + c]) atomicAdd(&live, 1);
        });
    if (m >= 0) {
        __syncthreads();
        if (threadIdx.x == 0) S.mdone()[m] = live == 0 ? 1 : 0;   // a mesh with zero right-hand sides is done
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        S.flag[BF_IT] = 0;
        S.flag[BF_MAX] = max_it;
        S.flag[BF_DONE] = max_it <= 0 ? 1 : 0;
    }
}

// pq = p.q per (mesh, column); alpha = rp / pq, the exact line search along p
// (rp = rr in plain CG; it differs right after a reliable update, where the
// step rr / pq would overshoot and break r_new . p = 0 for good); alpha = 0
// for converged columns and for a direction that is not a descent direction
// (the next p update then restarts the column from p = r)
__global__ void __launch_bounds__(BT) k_b_pq(Seg S, const float *__restrict__ p, const float *__restrict__ q,
                                             const float *__restrict__ qf)
{
    if (S.flag[BF_DONE]) return;
    seg_reduce<true>(
        S, [&](size_t t, int, int) { return p[t] * (qf ? q[t] + qf[t] : q[t]); },
        [&](int m, int c, float s) {
            const float rr = scal(S, C_RR, m, c), rp = scal(S, C_RP, m, c);
            const bool live = rr > scal(S, C_TOL, m, c) && s > 0.f && rp > 0.f;
            scal(S, C_PQ, m, c) = s;
            scal(S, C_AL, m, c) = live ? rp / s : 0.f;
        });
}

// x += alpha p; r -= alpha q; rr_new; beta; convergence of every column
// (pcg: beta and r.p come from r.z after the preconditioner, k_bp_zr)
__global__ void __launch_bounds__(BT) k_b_xr(Seg S, float *__restrict__ x, float *__restrict__ r,
                                             const float *__restrict__ p, const float *__restrict__ q,
                                             const float *__restrict__ qf, int pcg)
{
    if (S.flag[BF_DONE]) return;
    __shared__ int live;
    __shared__ bool all_last;
    if (threadIdx.x == 0) live = 0;
    __syncthreads();
    const bool was_done = S.mdone()[S.items[2 * blockIdx.x]];
    const int m = seg_reduce<true>(
        S,
        [&](size_t t, int mm, int c) {
            const float al = scal(S, C_AL, mm, c);
            x[t] = fmaf(al, p[t], x[t]);
            const float rn = fmaf(-al, qf ? q[t] + qf[t] : q[t], r[t]);
            r[t] = rn;
            return rn * rn;
        },
        [&](int mm, int c, float s) {
            const float rr = scal(S, C_RR, mm, c);
            if (scal(S, C_AL, mm, c) != 0.f) {
                if (!pcg) {
                    scal(S, C_BE, mm, c) = rr > 0.f ? s / rr : 0.f;
                    scal(S, C_RP, mm, c) = s;   // r_new . p_old = 0, so r_new . p_new = rr_new
                }
                scal(S, C_RR, mm, c) = s;
                if (s > scal(S, C_TOL, mm, c)) atomicAdd(&live, 1);
            } else if (!pcg) {
                scal(S, C_BE, mm, c) = 0.f;   // p = r next
                scal(S, C_RP, mm, c) = rr;
            }
        });
    if (m < 0) return;
    __syncthreads();
    // the last mesh to finish decides for the whole batch
    if (threadIdx.x == 0) {
        S.flag[FL_CNT + S.nmesh + m] = live;
        if (!was_done && live == 0) S.mdone()[m] = 1;
        __threadfence();
        unsigned v = atomicInc((unsigned *)&S.flag[BF_GCNT], S.nmesh - 1);
        all_last = (v == (unsigned)(S.nmesh - 1));
    }
    __syncthreads();
    if (!all_last || threadIdx.x != 0) return;
    __threadfence();
    int tot = 0;
    for (int mm = 0; mm < S.nmesh; ++mm) tot += __ldcg(S.flag + FL_CNT + S.nmesh + mm);
    const int it = S.flag[BF_IT] + 1;
    S.flag[BF_IT] = it;
    if (tot == 0 || it >= S.flag[BF_MAX]) S.flag[BF_DONE] = 1;
}

// p = r + beta p (same block decomposition as the reductions); r is z in the
// preconditioned iteration; upd (non-null): only the meshes just updated;
// p16 (non-null): p also as BF16 hi (p16) and lo (p16 + p16lo) for the near kernels
__global__ void __launch_bounds__(BT) k_b_p(Seg S, const float *__restrict__ r, float *__restrict__ p,
                                            const int *__restrict__ upd, __nv_bfloat16 *__restrict__ p16,
                                            long long p16lo)
{
    if (S.flag[BF_DONE]) return;
    const int m = S.items[2 * blockIdx.x], j = S.items[2 * blockIdx.x + 1];
    if (upd ? !upd[m] : S.mdone()[m]) return;
    const int nb = S.mesh[4 * m + 1], N = S.mesh[4 * m + 2], r0 = S.mesh[4 * m + 3];
    const int Rp = S.Rp;
    const size_t base = (size_t)r0 * Rp, n = (size_t)N * Rp;
    for (size_t e = (size_t)j * blockDim.x + threadIdx.x; e < n; e += (size_t)nb * blockDim.x) {
        const int c = (int)(e % Rp);
        const float v = fmaf(scal(S, C_BE, m, c), p[base + e], r[base + e]);
        p[base + e] = v;
        if (p16) {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            p16[base + e] = h;
            p16[p16lo + base + e] = __float2bfloat16_rn(v - __bfloat162float(h));
        }
    }
}

// reliable update of the meshes with upd[m] != 0: the recursive residual is
// replaced by the (rescaled) true residual b, the accumulated correction x
// restarts at zero, and the direction becomes p = b + gamma (p - r) per column
// (p - r = beta_old p_old from the last direction update, gamma converting it
// to the new scale and to beta from the true residual norm), or p = b where
// gamma < 0 (restart); rr, the thresholds and the done flags are recomputed.
// Meshes with upd[m] == 0 are left exactly as they are.
// (pcg: p keeps beta_old p_old = p - z_old; the preconditioner and k_bp_zr then
// form the new direction)
__global__ void __launch_bounds__(BT) k_b_replace(Seg S, const float *__restrict__ b, float *__restrict__ x,
                                                  float *__restrict__ r, float *__restrict__ p,
                                                  const float *__restrict__ gamma, const float *__restrict__ tol2,
                                                  const int *__restrict__ upd, const float *__restrict__ z)
{
    __shared__ int live;
    if (threadIdx.x == 0) live = 0;
    __syncthreads();
    const int m = seg_reduce<false>(
        S,
        [&](size_t t, int mm, int c) {
            if (!upd[mm]) return 0.f;
            const float v = b[t], g = gamma[mm * S.Rp + c];
            p[t] = z ? p[t] - z[t] : g < 0.f ? v : fmaf(g, p[t] - r[t], v);
            x[t] = 0.f;
            r[t] = v;
            return v * v;
        },
        [&](int mm, int c, float s) {
            if (!upd[mm]) return;
            scal(S, C_RR, mm, c) = s;
            scal(S, C_TOL, mm, c) = tol2[mm * S.Rp + c];
            scal(S, C_AL, mm, c) = 0.f;
            scal(S, C_BE, mm, c) = 0.f;
            if (s > tol2[mm * S.Rp + c]) atomicAdd(&live, 1);
        });
    if (m >= 0 && upd[m]) {
        __syncthreads();
        if (threadIdx.x == 0) S.mdone()[m] = live == 0 ? 1 : 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) S.flag[BF_DONE] = 0;
}

// rp = r . p of the meshes just updated (the step length of their first step)
__global__ void __launch_bounds__(BT) k_b_rp(Seg S, const float *__restrict__ r, const float *__restrict__ p,
                                             const int *__restrict__ upd)
{
    seg_reduce<false>(
        S, [&](size_t t, int mm, int) { return upd[mm] ? r[t] * p[t] : 0.f; },
        [&](int mm, int c, float s) {
            if (upd[mm]) scal(S, C_RP, mm, c) = s;
        });
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

// any nonzero entry in the first N rows of R columns of U (flag |= 1)
__global__ void k_b_nonzero(int N, int R, int64_t ld, const double *__restrict__ U, int *flag)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)N * R) return;
    const int c = (int)(t / N), i = (int)(t % N);
    if (U[(size_t)c * ld + i] != 0.0) atomicOr(flag, 1);
}

// res = F - AU (column-major FP64; AU null: U = 0), and per-column norms^2 (FP64, one block per column)
__global__ void k_b_resid(int N, int64_t ld, const double *__restrict__ F, const double *__restrict__ AU,
                          double *__restrict__ res, double *__restrict__ nrm2, double *__restrict__ fn2)
{
    __shared__ double sh[32];
    const int c = blockIdx.x;
    double v = 0.0, f = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        double d = AU ? F[(size_t)c * ld + i] - AU[(size_t)c * ld + i] : F[(size_t)c * ld + i];
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

__device__ __forceinline__ uint64_t b_gtimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// grid-wide barrier of a cooperative launch (every block resident): arrival
// counter + generation, the wait bounded by the global timer; false (and
// *err set) if the other blocks did not arrive in time
__device__ bool grid_barrier(unsigned *cnt, unsigned *gen, unsigned nblocks, long long wait_ns, int *err)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok_s = 1;
        const unsigned g = atomicAdd(gen, 0u);
        __threadfence();
        if (atomicAdd(cnt, 1u) == nblocks - 1) {
            atomicExch(cnt, 0u);
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t deadline = b_gtimer() + (uint64_t)wait_ns;
            while (atomicAdd(gen, 0u) == g)
                if (b_gtimer() > deadline) {
                    ok_s = 0;
                    atomicOr(err, 1);
                    break;
                }
        }
        __threadfence();
    }
    __syncthreads();
    return ok_s != 0;
}

// the sums over the blocks of mesh m of the per-column partials red[block][c],
// by the whole block in the order of seg_reduce's last block (lane rl takes
// blocks rl, rl + lanes, ...; the lanes' sums are added in lane order), into
// out[c] in shared memory; every block of the mesh gets the same values
__device__ void mesh_sums(const Seg &S, const float *red, int m, float *sh, float *out)
{
    const int b0 = S.mesh[4 * m], nb = S.mesh[4 * m + 1];
    const int Rp = S.Rp, Rc = min(Rp, (int)blockDim.x), lanes = blockDim.x / Rc;
    for (int c0 = 0; c0 < Rp; c0 += Rc) {
        const int cl = threadIdx.x % Rc, c = c0 + cl, rl = threadIdx.x / Rc;
        float s = 0.f;
        if (rl < lanes && c < Rp)
            for (int bI = rl; bI < nb; bI += lanes) s += __ldcg(red + (size_t)(b0 + bI) * Rp + c);
        sh[threadIdx.x] = s;
        __syncthreads();
        if (rl == 0 && c < Rp) {
            float tot = 0.f;
            for (int q = 0; q < lanes; ++q) tot += sh[q * Rc + cl];
            out[c] = tot;
        }
        __syncthreads();
    }
}

// One CG iteration's vector work after q = A p, for every (mesh, column), in
// one cooperative launch with two grid barriers:
//   A: p.q (block partials) | alpha = r.p / p.q per column
//   B: x += alpha p, r -= alpha q, r.r (partials) | beta, convergence
//   C: p = r + beta p, and p as two BF16 terms for the BF16 near kernels
//      (p16: hi; p16 + p16lo: lo = the rounding error of hi)
// Same arithmetic and the same fixed summation orders as k_b_pq, k_b_xr and
// k_b_p.  red2 holds the second partials (the first are still being read).
__global__ void __launch_bounds__(BT) k_b_iter(Seg S, float *__restrict__ red2, float *__restrict__ x,
                                               float *__restrict__ r, float *__restrict__ p,
                                               const float *__restrict__ q, const float *__restrict__ qf,
                                               __nv_bfloat16 *__restrict__ p16, long long p16lo, unsigned *gbar,
                                               long long wait_ns, int *err)
{
    __shared__ float sh[BT];
    __shared__ float al_s[BT], be_s[BT], rr_s[BT], sum_s[BT];   // per column (Rp <= BT)
    __shared__ int live_s, done_s;
    if (S.flag[BF_DONE]) return;   // stable during this launch: only written after barrier 1
    const int m = S.items[2 * blockIdx.x], j = S.items[2 * blockIdx.x + 1];
    const bool work = !S.mdone()[m];   // likewise written only after barrier 1
    const int nb = S.mesh[4 * m + 1], N = S.mesh[4 * m + 2], r0 = S.mesh[4 * m + 3];
    const int Rp = S.Rp, Rc = min(Rp, (int)blockDim.x), lanes = blockDim.x / Rc;
    const int cl = threadIdx.x % Rc, rl = threadIdx.x / Rc;
    // A: partials of p.q
    for (int c0 = 0; c0 < Rp; c0 += Rc) {
        const int c = c0 + cl;
        float v = 0.f;
        if (work && rl < lanes && c < Rp)
#pragma unroll 4
            for (int i = j * lanes + rl; i < N; i += nb * lanes) {
                const size_t t = (size_t)(r0 + i) * Rp + c;
                v += p[t] * (qf ? q[t] + qf[t] : q[t]);
            }
        sh[threadIdx.x] = v;
        __syncthreads();
        if (rl == 0 && c < Rp) {
            float s = 0.f;
            for (int qq = 0; qq < lanes; ++qq) s += sh[qq * Rc + cl];
            S.red[(size_t)blockIdx.x * Rp + c] = s;
        }
        __syncthreads();
    }
    if (!grid_barrier(gbar, gbar + 1, gridDim.x, wait_ns, err)) return;
    // alpha per column (the exact line search r.p / p.q)
    mesh_sums(S, S.red, m, sh, sum_s);
    for (int c = threadIdx.x; c < Rp; c += blockDim.x) {
        const float pq = sum_s[c];
        const float rr = scal(S, C_RR, m, c), rp = scal(S, C_RP, m, c);
        const bool live = work && rr > scal(S, C_TOL, m, c) && pq > 0.f && rp > 0.f;
        al_s[c] = live ? rp / pq : 0.f;
        rr_s[c] = rr;   // read before block 0 of the mesh overwrites it after barrier 2
        if (j == 0 && work) {
            scal(S, C_PQ, m, c) = pq;
            scal(S, C_AL, m, c) = al_s[c];
        }
    }
    __syncthreads();
    // B: x += alpha p; r -= alpha q; partials of r.r
    for (int c0 = 0; c0 < Rp; c0 += Rc) {
        const int c = c0 + cl;
        float v = 0.f;
        if (work && rl < lanes && c < Rp) {
            const float al = al_s[c];
#pragma unroll 4
            for (int i = j * lanes + rl; i < N; i += nb * lanes) {
                const size_t t = (size_t)(r0 + i) * Rp + c;
                x[t] = fmaf(al, p[t], x[t]);
                const float rn = fmaf(-al, qf ? q[t] + qf[t] : q[t], r[t]);
                r[t] = rn;
                v += rn * rn;
            }
        }
        sh[threadIdx.x] = v;
        __syncthreads();
        if (rl == 0 && c < Rp) {
            float s = 0.f;
            for (int qq = 0; qq < lanes; ++qq) s += sh[qq * Rc + cl];
            red2[(size_t)blockIdx.x * Rp + c] = s;
        }
        __syncthreads();
    }
    if (!grid_barrier(gbar, gbar + 1, gridDim.x, wait_ns, err)) return;
    // beta and convergence per column; every block of a mesh reaches the same decision
    if (threadIdx.x == 0) live_s = 0;
    mesh_sums(S, red2, m, sh, sum_s);
    for (int c = threadIdx.x; c < Rp; c += blockDim.x) {
        float be = 0.f;
        if (work) {
            const float s = sum_s[c], rr = rr_s[c];
            const bool moved = al_s[c] != 0.f;
            if (moved) {
                be = rr > 0.f ? s / rr : 0.f;
                if (s > scal(S, C_TOL, m, c)) atomicAdd(&live_s, 1);
            }
            if (j == 0) {
                scal(S, C_BE, m, c) = be;
                if (moved) {
                    scal(S, C_RR, m, c) = s;
                    scal(S, C_RP, m, c) = s;   // r_new . p_old = 0, so r_new . p_new = rr_new
                } else {
                    scal(S, C_RP, m, c) = rr;  // p = r next
                }
            }
        }
        be_s[c] = be;
    }
    __syncthreads();
    if (threadIdx.x == 0) done_s = work && live_s == 0;
    __syncthreads();
    if (j == 0 && threadIdx.x == 0 && work) {
        S.flag[FL_CNT + S.nmesh + m] = live_s;
        if (done_s) S.mdone()[m] = 1;
    }
    // C: p = r + beta p (meshes still iterating), p16 = BF16(p) and its rounding error
    if (work && !done_s) {
        const size_t base = (size_t)r0 * Rp, n = (size_t)N * Rp;
        for (size_t e = (size_t)j * blockDim.x + threadIdx.x; e < n; e += (size_t)nb * blockDim.x) {
            const int c = (int)(e % Rp);
            const float v = fmaf(be_s[c], p[base + e], r[base + e]);
            p[base + e] = v;
            if (p16) {
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                p16[base + e] = h;
                p16[p16lo + base + e] = __float2bfloat16_rn(v - __bfloat162float(h));
            }
        }
    }
    if (!grid_barrier(gbar, gbar + 1, gridDim.x, wait_ns, err)) return;
    // the whole batch: iteration count, done when no column anywhere is live
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int tot = 0;
        for (int mm = 0; mm < S.nmesh; ++mm)
            if (!S.mdone()[mm]) tot += __ldcg(S.flag + FL_CNT + S.nmesh + mm);
        const int it = S.flag[BF_IT] + 1;
        S.flag[BF_IT] = it;
        if (tot == 0 || it >= S.flag[BF_MAX]) S.flag[BF_DONE] = 1;
    }
}


// ---------------------------------------------------------------------------
// preconditioner of the batched iteration (the two-level preconditioner of
// precond.cu in FP32 on the interleaved vectors): z = Binv_a r_a per leaf,
// leaf sums rl, zc = Cinv rc per mesh (rc = the sums over each coarse
// cluster's leaves), z += zc[cluster of the row]
// ---------------------------------------------------------------------------
constexpr int PC_TILE = 64;   // columns per pass of the preconditioner kernels
constexpr int PC_CROWS = 4;   // coarse rows per CTA (one per thread group: many CTAs)

// leaf item: mesh, first row (global), rows, block stride, global leaf index
__global__ void __launch_bounds__(256) k_bp_local(Seg S, const int *__restrict__ items,
                                                  const long long *__restrict__ boff, const float *__restrict__ blk,
                                                  const float *__restrict__ r, float *__restrict__ z,
                                                  float *__restrict__ rl, const int *__restrict__ upd)
{
    extern __shared__ float smf[];
    if (S.flag[BF_DONE]) return;
    const int *it = items + 5 * blockIdx.x;
    const int m = it[0], row0 = it[1], na = it[2], mb = it[3], gl = it[4];
    if (upd ? !upd[m] : S.mdone()[m]) return;
    const int Rp = S.Rp;
    float *B = smf, *Rs = smf + (size_t)mb * mb;
    const float *g = blk + boff[blockIdx.x];
    for (int t = threadIdx.x; t < na * na; t += blockDim.x) B[(t / na) * mb + t % na] = g[(t / na) * mb + t % na];
    const int c = threadIdx.x % PC_TILE, grp = threadIdx.x / PC_TILE, ngrp = blockDim.x / PC_TILE;
    for (int c0 = 0; c0 < Rp; c0 += PC_TILE) {
        __syncthreads();
        for (int t = threadIdx.x; t < na * PC_TILE; t += blockDim.x)
            Rs[t] = r[(size_t)(row0 + t / PC_TILE) * Rp + c0 + t % PC_TILE];
        __syncthreads();
        // rows grp, grp + ngrp, ... four at a time; Binv symmetric, B[i][j] the
        // same address across the warp (broadcast)
        for (int i0 = grp; i0 < na; i0 += 4 * ngrp) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            for (int j = 0; j < na; ++j) {
                const float rv = Rs[j * PC_TILE + c];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = i0 + k * ngrp;
                    if (i < na) acc[k] = fmaf(B[i * mb + j], rv, acc[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = i0 + k * ngrp;
                if (i < na) z[(size_t)(row0 + i) * Rp + c0 + c] = acc[k];
            }
        }
        if (grp == 0) {
            float sum = 0.f;
            for (int i = 0; i < na; ++i) sum += Rs[i * PC_TILE + c];
            rl[(size_t)gl * Rp + c0 + c] = sum;
        }
    }
}

// coarse tile: mesh, first coarse row (PC_CROWS rows); per mesh (pmesh):
// clusters nc, leaves per cluster span, global index of its first leaf and
// of its first cluster.  zc = Cinv rc as a tiled product: chunks of PC_CB
// columns of Cinv and rows of rc (the cluster sums of the leaf sums, formed
// while staging) in shared memory; thread (column c, row group) keeps
// PC_CROWS / 4 rows
constexpr int PC_CB = 32;
__global__ void __launch_bounds__(256) k_bp_coarse(Seg S, const int *__restrict__ tiles, const int *__restrict__ pmesh,
                                                   const long long *__restrict__ coff,
                                                   const float *__restrict__ Cinv, const float *__restrict__ rl,
                                                   float *__restrict__ zc, const int *__restrict__ upd)
{
    __shared__ float Cs[PC_CROWS][PC_CB + 1], Rs[PC_CB][PC_TILE];
    if (S.flag[BF_DONE]) return;
    const int m = tiles[2 * blockIdx.x], a0 = tiles[2 * blockIdx.x + 1];
    if (upd ? !upd[m] : S.mdone()[m]) return;
    const int nc = pmesh[4 * m], span = pmesh[4 * m + 1], gl0 = pmesh[4 * m + 2], gc0 = pmesh[4 * m + 3];
    const int Rp = S.Rp;
    const float *C = Cinv + coff[m];
    const int c = threadIdx.x % PC_TILE, grp = threadIdx.x / PC_TILE;   // 4 groups
    constexpr int K = PC_CROWS / 4;
    for (int c0 = 0; c0 < Rp; c0 += PC_TILE) {
        float acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0.f;
        for (int b0 = 0; b0 < nc; b0 += PC_CB) {
            const int nb = min(PC_CB, nc - b0);
            __syncthreads();
            for (int t = threadIdx.x; t < PC_CROWS * PC_CB; t += blockDim.x) {
                const int i = t / PC_CB, bb = t % PC_CB;
                Cs[i][bb] = (a0 + i < nc && bb < nb) ? C[(size_t)(a0 + i) * nc + b0 + bb] : 0.f;
            }
            for (int t = threadIdx.x; t < PC_CB * PC_TILE; t += blockDim.x) {
                const int bb = t / PC_TILE, cc = t % PC_TILE;
                float v = 0.f;
                if (bb < nb)
                    for (int q = 0; q < span; ++q) v += rl[(size_t)(gl0 + (b0 + bb) * span + q) * Rp + c0 + cc];
                Rs[bb][cc] = v;
            }
            __syncthreads();
#pragma unroll 8
            for (int bb = 0; bb < PC_CB; ++bb) {
                const float r = Rs[bb][c];
#pragma unroll
                for (int k = 0; k < K; ++k) acc[k] = fmaf(Cs[grp * K + k][bb], r, acc[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int a = a0 + grp * K + k;
            if (a < nc) zc[(size_t)(gc0 + a) * Rp + c0 + c] = acc[k];
        }
    }
}

// z += zc[cluster of the row] (rowclu -1: no coarse space), rz = r.z, and
// the CG scalars:
//   mode 0 (start):  rz, r.p = rz, beta = 0 (then p = z)
//   mode 1 (step):   beta = rz_new / rz (0 for a column that did not move), rz, r.p = rz
//   mode 2 (reliable update of the meshes with upd): beta = g0 rz_new / rz_old
//            (g0 <= 0: restart from p = z), rz; r.p follows from k_b_rp
__global__ void __launch_bounds__(BT) k_bp_zr(Seg S, const int *__restrict__ rowclu, const float *__restrict__ zc,
                                              const float *__restrict__ r, float *__restrict__ z, int mode,
                                              const float *__restrict__ g0, const int *__restrict__ upd)
{
    if (S.flag[BF_DONE]) return;
    seg_reduce<true>(
        S,
        [&](size_t t, int mm, int c) {
            if (upd && !upd[mm]) return 0.f;
            float zv = z[t];
            if (zc) {
                const int cl = rowclu[t / S.Rp];
                if (cl >= 0) zv += zc[(size_t)cl * S.Rp + c];
                z[t] = zv;
            }
            return r[t] * zv;
        },
        [&](int mm, int c, float s) {
            if (upd && !upd[mm]) return;
            const float rz = scal(S, C_RZ, mm, c);
            if (mode == 0) {
                scal(S, C_RP, mm, c) = s;
                scal(S, C_BE, mm, c) = 0.f;
            } else if (mode == 1) {
                const bool moved = scal(S, C_AL, mm, c) != 0.f;
                scal(S, C_BE, mm, c) = moved && rz > 0.f ? s / rz : 0.f;
                scal(S, C_RP, mm, c) = s;   // r_new . p_old = 0, so r_new . p_new = r_new . z_new
            } else {
                const float g = g0[(size_t)mm * S.Rp + c];
                scal(S, C_BE, mm, c) = g > 0.f && rz > 0.f ? g * s / rz : 0.f;
            }
            scal(S, C_RZ, mm, c) = s;
        });
}

}  // namespace

void apply_parts_ex(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                    bool lowp, cudaStream_t st, const int *skip);

// reduction blocks: per mesh a share of one block per SM proportional to its
// rows (at least one); vectors, partials, scalars and flags for Rp columns
static void ensure_solve(BatchData &b, int Rp)
{
    if (b.sR == Rp) return;
    release_bgraph(b);   // the captured chunk refers to these buffers
    int dev = 0, nsm = 0;
    VFD_CUDA(cudaGetDevice(&dev));
    VFD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int target = std::max(1, nsm);
    std::vector<int> items, mesh(4 * (size_t)b.nmesh);
    int nred = 0;
    for (int i = 0; i < b.nmesh; ++i) {
        const int N = b.ops[i]->m->N;
        int nb = (int)std::llround((double)target * N / (double)std::max<int64_t>(b.ntot, 1));
        nb = std::max(1, std::min(nb, std::max(1, N)));
        mesh[4 * i] = nred;
        mesh[4 * i + 1] = nb;
        mesh[4 * i + 2] = N;
        mesh[4 * i + 3] = (int)b.xoff[i];
        for (int j = 0; j < nb; ++j) {
            items.push_back(i);
            items.push_back(j);
        }
        nred += nb;
    }
    b.nred = nred;
    b.red_items.upload(items);
    b.red_mesh.upload(mesh);
    const size_t nv = (size_t)b.ntot * Rp;
    b.x.alloc(nv);
    b.r.alloc(nv);
    b.p.alloc(nv);
    b.q.alloc(nv);
    b.qf.alloc(nv);   // rows of meshes without a far field stay zero
    VFD_CUDA(cudaMemset(b.qf.p, 0, b.qf.bytes()));
    b.b.alloc(nv);
    b.red.alloc((size_t)nred * Rp);
    b.red2.alloc((size_t)nred * Rp);
    b.sc.alloc((size_t)C_N * b.nmesh * Rp);
    b.flag.alloc(FL_CNT + 3 * (size_t)b.nmesh);
    VFD_CUDA(cudaMemset(b.flag.p, 0, b.flag.bytes()));
    b.sR = Rp;
}

static Seg make_seg(BatchData &b, int Rp)
{
    Seg S;
    S.nmesh = b.nmesh;
    S.Rp = Rp;
    S.items = b.red_items.p;
    S.mesh = b.red_mesh.p;
    S.red = b.red.p;
    S.flag = b.flag.p;
    S.sc = b.sc.p;
    return S;
}

// preconditioner tables of the batch: built when every operator carries a
// preconditioner (vfd_precondition), rebuilt when one of them changed
static void ensure_bprec(BatchData &b, int Rp)
{
    int npre = 0;
    for (OpData *op : b.ops) npre += op->prec_kind != 0;
    VFD_REQUIRE(npre == 0 || npre == b.nmesh, VFD_EINVAL,
                "batched solve: precondition every operator of the batch or none");
    const bool want = npre == b.nmesh;
    std::vector<long long> key;
    if (want) {
        key.push_back(Rp);
        for (OpData *op : b.ops) key.push_back(op->prec_version);
    }
    if (want == b.pcg && (!want || key == b.pc_key)) return;
    release_bgraph(b);   // the captured chunk differs
    b.pcg = want;
    b.pc_key = key;
    if (!want) return;
    std::vector<int> items, pmesh(4 * (size_t)b.nmesh), tiles, rowclu((size_t)b.ntot, -1);
    std::vector<long long> boff, coff(b.nmesh);
    long long nblk = 0, ncoarse = 0;
    int gleaf = 0, gclu = 0, mbmax = 0, any_coarse = 0;
    for (int i = 0; i < b.nmesh; ++i) {
        const OpData &op = *b.ops[i];
        const MeshData &m = *op.m;
        const int nleaf = m.kt.nleaf, fl = m.kt.first_leaf(), mb = op.prec_mb, nc = op.prec_nc;
        VFD_REQUIRE(mb <= 128, VFD_EUNSUPPORTED, "batched preconditioned solve: leaves of at most 128 DoFs");
        mbmax = std::max(mbmax, mb);
        for (int a = 0; a < nleaf; ++a) {
            items.push_back(i);
            items.push_back((int)b.xoff[i] + m.kt.begin[fl + a]);
            items.push_back(m.kt.end[fl + a] - m.kt.begin[fl + a]);
            items.push_back(mb);
            items.push_back(gleaf + a);
            boff.push_back(nblk + (long long)a * mb * mb);
        }
        pmesh[4 * i] = nc;
        pmesh[4 * i + 1] = op.prec_span;
        pmesh[4 * i + 2] = gleaf;
        pmesh[4 * i + 3] = gclu;
        coff[i] = ncoarse;
        if (nc > 0) {
            any_coarse = 1;
            for (int a0 = 0; a0 < nc; a0 += PC_CROWS) {
                tiles.push_back(i);
                tiles.push_back(a0);
            }
            for (int c = 0; c < nc; ++c) {
                const int r0 = m.kt.begin[fl + c * op.prec_span];
                const int r1 = c + 1 < nc ? m.kt.begin[fl + (c + 1) * op.prec_span] : m.N;
                for (int row = r0; row < r1; ++row) rowclu[(size_t)b.xoff[i] + row] = gclu + c;
            }
        }
        nblk += (long long)nleaf * mb * mb;
        ncoarse += (long long)nc * nc;
        gleaf += nleaf;
        gclu += nc;
    }
    b.pc_blk.alloc(nblk);
    b.pc_coarse.alloc(std::max<long long>(ncoarse, 1));
    for (int i = 0; i < b.nmesh; ++i) {
        const OpData &op = *b.ops[i];
        long long off = 0;
        for (int j = 0; j < i; ++j) off += (long long)b.ops[j]->m->kt.nleaf * b.ops[j]->prec_mb * b.ops[j]->prec_mb;
        VFD_CUDA(cudaMemcpy(b.pc_blk.p + off, op.prec_blk32.p, op.prec_blk32.bytes(), cudaMemcpyDeviceToDevice));
        if (op.prec_nc > 0)
            VFD_CUDA(cudaMemcpy(b.pc_coarse.p + coff[i], op.prec_coarse32.p, op.prec_coarse32.bytes(),
                                cudaMemcpyDeviceToDevice));
    }
    b.pc_items.upload(items);
    b.pc_boff.upload(boff);
    b.pc_pmesh.upload(pmesh);
    b.pc_coff.upload(coff);
    b.pc_ctiles.upload(tiles.empty() ? std::vector<int>{0, 0} : tiles);
    b.pc_rowclu.upload(rowclu);
    b.n_pc_items = (int)(items.size() / 5);
    b.n_pc_ctiles = (int)(tiles.size() / 2);
    b.pc_mbmax = mbmax;
    b.pc_any_coarse = any_coarse;
    b.z.alloc((size_t)b.ntot * Rp);
    b.pc_rl.alloc((size_t)gleaf * Rp);
    b.pc_zc.alloc((size_t)std::max(gclu, 1) * Rp);
    const size_t shm = ((size_t)mbmax * mbmax + (size_t)mbmax * PC_TILE) * sizeof(float);
    VFD_CUDA(cudaFuncSetAttribute(k_bp_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
}

// z = M^-1 r (all meshes, or the meshes with upd), then the scalars of mode (k_bp_zr)
static void bprec_apply(BatchData &b, const Seg &S, int mode, const float *g0, const int *upd, cudaStream_t st)
{
    const size_t shm = ((size_t)b.pc_mbmax * b.pc_mbmax + (size_t)b.pc_mbmax * PC_TILE) * sizeof(float);
    k_bp_local<<<b.n_pc_items, 256, shm, st>>>(S, b.pc_items.p, b.pc_boff.p, b.pc_blk.p, b.r.p, b.z.p, b.pc_rl.p,
                                               upd);
    if (b.pc_any_coarse)
        k_bp_coarse<<<b.n_pc_ctiles, 256, 0, st>>>(S, b.pc_ctiles.p, b.pc_pmesh.p, b.pc_coff.p, b.pc_coarse.p,
                                                   b.pc_rl.p, b.pc_zc.p, upd);
    k_bp_zr<<<b.nred, BT, 0, st>>>(S, b.pc_rowclu.p, b.pc_any_coarse ? b.pc_zc.p : nullptr, b.r.p, b.z.p, mode, g0,
                                   upd);
    VFD_CUDA(cudaGetLastError());
}

// capture one chunk of BCHUNK low-precision CG iterations (apply, p.q, x/r
// update, p update) as a graph; the eager apply first builds the apply's
// descriptors and workspaces outside the capture
static void capture_bcg(BatchData &b, int Rp, cudaStream_t st)
{
    const Seg S = make_seg(b, Rp);
    batch_apply(b, b.p.p, b.q.p, Rp, st, nullptr, nullptr);
    if (b.exec) return;
    // the fused vector kernel needs every block resident (cooperative launch)
    // and at most BT columns; in a BF16 batch it also writes p as the BF16 hi
    // and lo blocks the near kernels read
    {
        int dev = 0, nsm = 0, per = 0, coop = 0;
        VFD_CUDA(cudaGetDevice(&dev));
        VFD_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        VFD_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
        VFD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_b_iter, BT, 0));
        b.fused = coop && Rp <= BT && b.nred <= per * nsm && !b.pcg;
        b.p16_target = batch_x16(b);
        if (b.fused && !b.gbar.p) {
            b.gbar.alloc(2);
            VFD_CUDA(cudaMemset(b.gbar.p, 0, 2 * sizeof(unsigned)));
        }
    }
    // the far field's expansion runs on the side stream into qf, concurrent with
    // the near panels; the vector kernels read q + qf
    float *qf = b.any_far ? b.qf.p : nullptr;
    cudaStream_t cs;
    VFD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph;
    VFD_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
        for (int it = 0; it < BCHUNK; ++it) {
            // p in BF16 hi / lo comes from the vector kernels (BF16 batches)
            batch_apply(b, b.p.p, b.q.p, Rp, cs, b.flag.p, b.flag.p + FL_CNT + 2 * b.nmesh, b.p16_target != nullptr,
                        qf);
            if (b.fused) {
                // one cooperative launch for the iteration's vector work; p also in
                // BF16 hi / lo for the next apply's near kernel
                Seg Sv = S;
                float *red2 = b.red2.p, *xv = b.x.p, *rv = b.r.p, *pv = b.p.p;
                const float *qv = b.q.p, *qfv = qf;
                __nv_bfloat16 *p16 = (__nv_bfloat16 *)b.p16_target;
                long long p16lo = (long long)b.ntot * Rp;
                unsigned *gb = b.gbar.p;
                long long wns = b.wait_ns;
                int *err = b.tc_err.p;
                void *args[] = {&Sv, &red2, &xv, &rv, &pv, &qv, &qfv, &p16, &p16lo, &gb, &wns, &err};
                VFD_CUDA(cudaLaunchCooperativeKernel((const void *)k_b_iter, b.nred, BT, args, 0, cs));
            } else if (b.pcg) {
                // preconditioned: p.q, x/r update, z = M^-1 r with r.z and beta, p = z + beta p
                k_b_pq<<<b.nred, BT, 0, cs>>>(S, b.p.p, b.q.p, qf);
                k_b_xr<<<b.nred, BT, 0, cs>>>(S, b.x.p, b.r.p, b.p.p, b.q.p, qf, 1);
                bprec_apply(b, S, 1, nullptr, nullptr, cs);
                k_b_p<<<b.nred, BT, 0, cs>>>(S, b.z.p, b.p.p, nullptr, (__nv_bfloat16 *)b.p16_target,
                                             (long long)b.ntot * Rp);
            } else {
                k_b_pq<<<b.nred, BT, 0, cs>>>(S, b.p.p, b.q.p, qf);
                k_b_xr<<<b.nred, BT, 0, cs>>>(S, b.x.p, b.r.p, b.p.p, b.q.p, qf, 0);
                k_b_p<<<b.nred, BT, 0, cs>>>(S, b.r.p, b.p.p, nullptr, (__nv_bfloat16 *)b.p16_target,
                                             (long long)b.ntot * Rp);
            }
        }
    } catch (...) {
        cudaStreamEndCapture(cs, &graph);
        cudaStreamDestroy(cs);
        throw;
    }
    VFD_CUDA(cudaStreamEndCapture(cs, &graph));
    cudaStreamDestroy(cs);
    cudaError_t ie = cudaGraphInstantiate(&b.exec, graph, 0);
    cudaGraphDestroy(graph);
    VFD_CUDA(ie);
}

// R columns per mesh of F_m, U_m (FP64, column-major, leading dimension ld_m,
// device); relres and iters: nmesh x R, mesh-major (may be null); iters holds
// the inner iterations run until the column's mesh met rtol
vfd_status batch_solve(BatchData &b, const double *const *F, double *const *U, const int64_t *ld, int R, double rtol,
                       int max_it, int *iters, double *relres, cudaStream_t st)
{
    const double RU_DROP = b.ru_drop;   // recursive-residual reduction between reliable updates
    const int Rp = ((R + 63) / 64) * 64, nm = b.nmesh;
    const size_t nc = (size_t)nm * Rp, nr = (size_t)nm * R;
    ensure_solve(b, Rp);
    ensure_bprec(b, Rp);
    std::vector<DBuf<double>> AU(nm), res(nm);
    DBuf<double> n2, f2, scale;
    DBuf<float> gamma_d, tol2_d;
    DBuf<int> upd_d;
    for (int i = 0; i < nm; ++i) {
        AU[i].alloc((size_t)ld[i] * R);
        res[i].alloc((size_t)ld[i] * R);
    }
    n2.alloc(nr);
    f2.alloc(nr);
    scale.alloc(nr);
    gamma_d.alloc(nc);
    tol2_d.alloc(nc);
    upd_d.alloc(nm);
    // host state: true residual norms^2 (hn, F norms^2 hf), the scale of each
    // column's inner problem (sc: 0 = converged, frozen), the last true relres
    std::vector<double> hn(nr, 0.0), hf(nr, 0.0), sc(nr, 0.0), rel_last(nr, HUGE_VAL);
    std::vector<float> gamma(nc, 0.f), tol2(nc, 0.f), rr(nc, 0.f), rr_last(nc, 0.f);
    std::vector<int> upd(nm, 1), conv(nm, 0), it_conv(nm, 0), hflag(FL_CNT + 3 * (size_t)nm, 0);
    const Seg S = make_seg(b, Rp);
    bool breakdown = false;   // a non-finite residual: the solve stops with VFD_ENOCONV

    // for the meshes with upd[i]: FP64 residuals res = F - A U, relres, the new
    // scales, thresholds and direction factors (gamma); sets conv[i]
    // the first call skips the FP64 apply for meshes whose initial U is zero
    std::vector<int> u_nonzero(nm, 1);
    {
        DBuf<int> nzf;
        nzf.alloc(nm);
        nzf.zero(st);
        for (int i = 0; i < nm; ++i)
            k_b_nonzero<<<cdiv((long long)b.ops[i]->m->N * R, 256), 256, 0, st>>>(b.ops[i]->m->N, R, ld[i], U[i],
                                                                                 nzf.p + i);
        VFD_CUDA(cudaGetLastError());
        VFD_CUDA(cudaMemcpyAsync(u_nonzero.data(), nzf.p, sizeof(int) * nm, cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaStreamSynchronize(st));
    }
    bool first_residual = true;
    auto true_residual = [&](int it_now) {
        const bool first = first_residual;
        first_residual = false;
        for (int i = 0; i < nm; ++i) {
            if (!upd[i]) continue;
            OpData &op = *b.ops[i];
            const bool zero_u = first && !u_nonzero[i];
            if (!zero_u) apply_parts_ex(*op.m, op, VFD_PART_ALL, U[i], AU[i].p, R, ld[i], false, st, nullptr);
            k_b_resid<<<R, 256, 0, st>>>(op.m->N, ld[i], F[i], zero_u ? nullptr : AU[i].p, res[i].p,
                                         n2.p + (size_t)i * R, f2.p + (size_t)i * R);
            VFD_CUDA(cudaGetLastError());
        }
        VFD_CUDA(cudaMemcpyAsync(hn.data(), n2.p, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaMemcpyAsync(hf.data(), f2.p, sizeof(double) * nr, cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < nm; ++i) {
            if (!upd[i]) continue;
            const bool mesh_was_done = hflag[FL_CNT + 2 * (size_t)nm + i] != 0;
            bool all = true;
            for (int c = 0; c < R; ++c) {
                const size_t h = (size_t)i * R + c, k = (size_t)i * Rp + c;
                const double rel = hf[h] > 0.0 ? std::sqrt(hn[h] / hf[h]) : std::sqrt(hn[h]);
                if (relres) relres[h] = rel;
                if (!std::isfinite(rel)) breakdown = true;
                if (!(rel <= rtol)) all = false;
                const double s_new = rel > rtol ? std::sqrt(hn[h]) : 0.0;
                // continue the direction only for a column still iterating whose recursive
                // residual (sqrt(rr) in the old scale) agrees with the true one to a factor
                // of two and whose true residual did not grow since the last update
                const double rec = std::sqrt((double)rr[k]) * sc[h];
                const bool iterating = !mesh_was_done && tol2[k] > 0.f && rr[k] > tol2[k];
                const bool keep = s_new > 0.0 && sc[h] > 0.0 && iterating && rec < 2.0 * s_new &&
                                  s_new < 2.0 * rec && rel <= rel_last[h];
                // p_new = r_true + (|r_true|^2 / |r_rec|^2) beta_old p_old, in the new scale;
                // preconditioned: p_new = z_true + (rz_true / rz_rec) beta_old p_old, the
                // factor s_new / s_old here and the r.z ratio on the device (k_bp_zr)
                gamma[k] = s_new <= 0.0 ? 0.f
                           : keep       ? (float)(b.pcg ? s_new / sc[h] : s_new / (sc[h] * (double)rr[k]))
                                        : -1.f;
                // inner target in the scaled units: half of rtol (room for the recursive residual's drift)
                const double tgt = s_new > 0.0 ? 0.5 * rtol * std::sqrt(hf[h]) / s_new : 0.0;
                tol2[k] = (float)(tgt * tgt);
                rr_last[k] = s_new > 0.0 ? 1.f : 0.f;   // |b|^2 after the update
                sc[h] = s_new;
                rel_last[h] = rel;
            }
            if (all && !conv[i]) {
                conv[i] = 1;
                it_conv[i] = it_now;
            }
        }
    };
    // the scaled true residuals of the meshes with upd[i] into the inner right-hand side b
    auto residual_to_inner = [&]() {
        VFD_CUDA(cudaMemcpyAsync(scale.p, sc.data(), sizeof(double) * nr, cudaMemcpyHostToDevice, st));
        VFD_CUDA(cudaMemcpyAsync(tol2_d.p, tol2.data(), sizeof(float) * nc, cudaMemcpyHostToDevice, st));
        VFD_CUDA(cudaMemcpyAsync(gamma_d.p, gamma.data(), sizeof(float) * nc, cudaMemcpyHostToDevice, st));
        VFD_CUDA(cudaMemcpyAsync(upd_d.p, upd.data(), sizeof(int) * nm, cudaMemcpyHostToDevice, st));
        for (int i = 0; i < nm; ++i) {
            if (!upd[i]) continue;
            const int N = b.ops[i]->m->N;
            k_b_to_inner<<<cdiv((long long)N * Rp, 256), 256, 0, st>>>(N, R, Rp, ld[i], res[i].p,
                                                                       scale.p + (size_t)i * R,
                                                                       b.b.p + (size_t)b.xoff[i] * Rp);
        }
        VFD_CUDA(cudaGetLastError());
    };
    // U += scale x for the meshes with upd[i] (their correction since the last update)
    auto add_correction = [&]() {
        for (int i = 0; i < nm; ++i) {
            if (!upd[i]) continue;
            const int N = b.ops[i]->m->N;
            k_b_from_inner<<<cdiv((long long)N * R, 256), 256, 0, st>>>(N, R, Rp, ld[i],
                                                                        b.x.p + (size_t)b.xoff[i] * Rp,
                                                                        scale.p + (size_t)i * R, U[i]);
        }
        VFD_CUDA(cudaGetLastError());
    };
    auto all_conv = [&]() { return std::all_of(conv.begin(), conv.end(), [](int v) { return v != 0; }); };

    vfd_status status = VFD_ENOCONV;   // until every column meets rtol
    true_residual(0);
    if (breakdown) return VFD_ENOCONV;
    if (all_conv()) {
        if (iters) std::fill(iters, iters + nr, 0);
        return VFD_OK;
    }
    residual_to_inner();
    k_b_init<<<b.nred, BT, 0, st>>>(S, b.b.p, b.x.p, b.r.p, b.p.p, tol2_d.p, std::max(1, max_it));
    VFD_CUDA(cudaGetLastError());
    if (b.pcg) {   // z = M^-1 r, r.p = r.z, p = z
        bprec_apply(b, S, 0, nullptr, nullptr, st);
        k_b_p<<<b.nred, BT, 0, st>>>(S, b.z.p, b.p.p, nullptr, nullptr, 0);
    }
    capture_bcg(b, Rp, st);
    // the captured apply reads p in BF16 hi / lo from the vector kernels: provide the first one
    if (b.p16_target) batch_x_to_bf16(b, b.p.p, Rp, st);
    const float drop2 = (float)(RU_DROP * RU_DROP);
    int it = 0;
    while (true) {
        VFD_CUDA(cudaGraphLaunch(b.exec, st));
        VFD_CUDA(cudaMemcpyAsync(hflag.data(), b.flag.p, sizeof(int) * hflag.size(), cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaMemcpyAsync(rr.data(), b.sc.p + (size_t)C_RR * nc, sizeof(float) * nc, cudaMemcpyDeviceToHost,
                                 st));
        VFD_CUDA(cudaStreamSynchronize(st));
        batch_check(b, st);
        it = hflag[BF_IT];
        const bool out_of_its = it >= max_it;
        // meshes due for a reliable update
        bool any = false;
        for (int i = 0; i < nm; ++i) {
            bool ready = !conv[i] && (out_of_its || hflag[FL_CNT + 2 * (size_t)nm + i] != 0);
            if (!conv[i] && !ready) {
                ready = true;
                for (int c = 0; c < R && ready; ++c) {
                    const size_t k = (size_t)i * Rp + c;
                    if (rr[k] > tol2[k] && rr[k] > drop2 * rr_last[k]) ready = false;
                }
            }
            upd[i] = ready ? 1 : 0;
            any |= ready;
        }
        if (!any) continue;
        add_correction();
        true_residual(it);
        if (all_conv()) {
            status = VFD_OK;
            break;
        }
        if (out_of_its || breakdown) break;
        residual_to_inner();
        k_b_replace<<<b.nred, BT, 0, st>>>(S, b.b.p, b.x.p, b.r.p, b.p.p, gamma_d.p, tol2_d.p, upd_d.p,
                                           b.pcg ? b.z.p : nullptr);
        if (b.pcg) {   // z = M^-1 r_true, beta from r.z, p = z + beta (beta_old p_old)
            bprec_apply(b, S, 2, gamma_d.p, upd_d.p, st);
            k_b_p<<<b.nred, BT, 0, st>>>(S, b.z.p, b.p.p, upd_d.p, nullptr, 0);
        }
        k_b_rp<<<b.nred, BT, 0, st>>>(S, b.r.p, b.p.p, upd_d.p);
        VFD_CUDA(cudaGetLastError());
        if (b.p16_target) batch_x_to_bf16(b, b.p.p, Rp, st);
    }
    VFD_CUDA(cudaStreamSynchronize(st));
    if (iters)
        for (int i = 0; i < nm; ++i)
            for (int c = 0; c < R; ++c) iters[(size_t)i * R + c] = conv[i] ? it_conv[i] : it;
    return status;
}

}  // namespace vfd
