/*
 * vfd.h -- C ABI of the GB300 (sm_103a) library for the linear-complexity
 * finite element operator of variable-order fractional diffusion
 * (Lei, Turkiyyah & Knio, arXiv 2302.02863).
 *
 * Problem (Sec. 2, eqs. e:strong, e:weak-d): on a simplicial mesh of
 * Omega = Omega_i U Omega_e, find the P1 function U, zero on Omega_e, with
 *     A(U, V) = int_{Omega_i} f V   for all P1 V zero on Omega_e,
 *     A(u, v) = int int (u(x)-u(y)) (v(x)-v(y)) gamma(x,y) dy dx,
 *     gamma(x,y) = sqrt(kappa(x) kappa(y)) / |x-y|^(d + s(x) + s(y)).
 * The stiffness matrix is assembled as A = B + K + M (Sec. 3, eq. e:decomp):
 * B the singular near field (Sec. 4), K the H^2 matrix of the separated
 * interior pairs (Sec. 5), M the weighted mass matrix whose density rho is
 * computed by an H^2 (fast-multipole type) sweep (Sec. 6), plus the exterior
 * tail of Sec. 7.1.1 when Omega_e is all of R^d outside the mesh.
 *
 * Conventions for every entry point:
 *  - No exception crosses the ABI; a failing call returns a status and sets
 *    a message readable with vfd_last_error() (thread-local).
 *  - The caller owns every data pointer.  Handles own their device memory
 *    until vfd_free_*.  "device" pointers are CUDA device (or managed)
 *    memory of the current device; entry points that say "host or device"
 *    accept either and copy host memory through the library.
 *  - Vectors indexed by DoF use the library's DoF numbering (cluster-tree
 *    order), available from vfd_mesh_dofs.  Multi-RHS blocks are
 *    column-major: entry (i, r) at ptr[i + r*ld], ld >= n_dof.
 *  - Work is enqueued on the given cudaStream_t (passed as void*; NULL is the
 *    legacy default stream) and is asynchronous unless the call returns
 *    host values (vfd_solve's iteration counts and residuals, vfd_assemble's
 *    field check).  One handle must not be used from two streams at once.
 *  - Nothing falls back to the CPU: without a CUDA device every call that
 *    computes returns VFD_ECUDA.
 */
#ifndef VFD_H
#define VFD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VFD_OK = 0,
    VFD_EINVAL = 1,        /* bad argument, bad mesh, field outside 0 <= s <= s_bar < 1 */
    VFD_ENOMEM = 2,        /* device or host allocation failed */
    VFD_ECUDA = 3,         /* CUDA runtime error, or no CUDA device */
    VFD_ENOCONV = 4,       /* solver hit max_it; the last iterate is returned */
    VFD_ETIMEOUT = 5,      /* a bounded device wait gave up */
    VFD_EUNSUPPORTED = 6   /* valid request this build does not implement */
} vfd_status;

typedef struct vfd_mesh_s *vfd_mesh_t;
typedef struct vfd_op_s *vfd_op_t;
typedef struct vfd_batch_s *vfd_batch_t;

/* Precision of the assembled operator (argument `precision`). */
enum {
    VFD_FP64 = 0,   /* every part in FP64 */
    VFD_FP32 = 1,   /* K (near blocks, coupling, bases) stored and applied in
                       FP32 (single RHS) or TF32 tensor-core products (batched
                       solves) with FP32 accumulation; B, M, the density rho
                       and the refinement residuals stay FP64 */
    VFD_BF16 = 2    /* as VFD_FP32 with K in BF16 for the batched solves */
};

/* Parts of the operator for vfd_apply_parts (bit mask). */
enum {
    VFD_PART_B = 1,       /* singular near field B (Sec. 4) */
    VFD_PART_M = 2,       /* weighted mass matrix M incl. exterior tail (Sec. 6, 7.1.1) */
    VFD_PART_KNEAR = 4,   /* dense inadmissible leaf blocks of K (Sec. 5.2) */
    VFD_PART_KFAR = 8,    /* low-rank admissible blocks of K (Sec. 5.3) */
    VFD_PART_ALL = 15
};

/* Flags of vfd_assemble. */
enum {
    VFD_ASSEMBLE_UNCHECKED = 1, /* skip the check 0 <= s <= s_bar < 1 (lets the
                                   tests use polynomial kernels, e.g. s = -2) */
    VFD_ASSEMBLE_TIMED = 2      /* record CUDA events around every assembly phase
                                   (read back with vfd_op_timings) */
};

/* Phases reported by vfd_op_timings (milliseconds of device time). */
enum {
    VFD_T_FIELDS = 0,    /* field values at element points and Chebyshev nodes */
    VFD_T_COUPLING = 1,  /* coupling blocks S of K (Sec. 5.3) */
    VFD_T_NEAR = 2,      /* dense inadmissible leaf blocks of K (Sec. 5.2) */
    VFD_T_DENSITY = 3,   /* density rho, H^2 sweep + tail (Sec. 6.2, 7.1.1) */
    VFD_T_SINGULAR = 4,  /* singular near field B, local matrices (Sec. 4) */
    VFD_T_GATHER = 5,    /* CSR gathers of B and M (and the FP32 copies) */
    VFD_T_TOTAL = 6,
    VFD_T_COUNT = 7
};

/* Mesh-level options (geometry only; fixed for the life of the mesh handle). */
typedef struct {
    int leaf_m;         /* max DoFs per leaf of the K cluster tree (Sec. 5.1, m); default 64 */
    int cheb_p;         /* Chebyshev nodes per dimension; rank k = p^d (Sec. 5.3); default 4 */
    double lambda;      /* admissibility lambda ||C-C'|| >= (D+D')/2 on the support-extended
                           boxes (Sec. 7, first paragraph); default 0.75; 0 = no low-rank block */
    int n_sing;         /* Gauss points per direction in the singular rules (Sec. 4, n); default 3 */
    int tail_mode;      /* 0: Omega_e is the meshed exterior; 1: Omega_e = R^d minus the mesh,
                           whose outer boundary is the sphere |x| = tail_R (Sec. 7.1.1) */
    double tail_R;      /* radius of that sphere; default 1.1 */
    int rho_leaf_m;     /* max points per leaf of the density cluster trees (Sec. 6.2); default 64 */
    double rho_lambda;  /* admissibility of the density sweep on plain point boxes, with the
                           extra condition dist > 2 h_max (Sec. 6.2); default 0.75; 0 = direct */
    int inner_p;        /* Chebyshev nodes per dimension of the far field of the low-precision
                           inner operator of the batched mixed-precision solves (VFD_FP32 /
                           VFD_BF16 operators, nrhs a multiple of 64); 0 = cheb_p.  That
                           operator only has to match the FP64 operator to its own rounding
                           level (2^-11 or 2^-8), so a lower order serves; the solves still
                           converge to the solution of the FP64 operator.  Default 0. */
    double recompress_tol;  /* algebraic recompression of the far field of K of VFD_FP64 operators
                           (Sec. 5.3, last paragraph), done by vfd_assemble: every node's basis
                           is orthogonalised and cut to the singular directions of its coupling
                           row above recompress_tol x the largest over all nodes; ranks padded
                           per level.  The apply, the solves and the batched solves' FP64
                           residuals use the recompressed far field; vfd_grad differentiates
                           the interpolation operator before recompression.  0 = off (default). */
} vfd_mesh_opts;

/* Scalar field on R^d: value = squash(c0 + sum of terms), or a P1 field.
 * fourier rows (k1,k2,k3 integers, amp, phase): amp cos(pi k.x + phase)
 * gauss rows   (x0,y0,z0, amp, c):              amp exp(-c |x-x0|^2)
 * tbump rows   (x0,y0,z0, amp, ell):            amp prod_i exp(-1/(1-r_i^2)), r_i = 2(x_i-x0_i)/ell, |r_i|<1
 * squash = 1: lo + (hi-lo)/(1+exp(-v)).
 * Row arrays are host memory, read during the call.  kind = VFD_FIELD_NODAL
 * takes `nodal`, values at the n_vert mesh vertices (host or device): the P1
 * interpolant at element and singular-rule points, and at a Chebyshev node
 * the interpolant at the node's nearest point of the mesh (located once per
 * mesh on the first such assembly). */
enum { VFD_FIELD_ANALYTIC = 0, VFD_FIELD_NODAL = 1 };
typedef struct {
    int kind;
    double c0;
    int n_fourier;
    const double *fourier;
    int n_gauss;
    const double *gauss;
    int n_tbump;
    const double *tbump;
    int squash;
    double lo, hi;
    const double *nodal;
} vfd_field;

/* Fill *opts with the defaults listed above. */
void vfd_default_mesh_opts(vfd_mesh_opts *opts);

/* Build the mesh handle: topology (interior DoFs are the vertices of no
 * exterior cell, Sec. 2.3), touching element pairs with their type
 * (identical / edge / vertex, Sec. 4), the element quadrature cloud Q
 * (3 points per triangle / interval, Sec. 6.1 and Sec. 7), the KD cluster tree
 * on the DoFs with support-extended boxes, the admissible and inadmissible
 * block lists, leaf bases and transfer matrices (Sec. 5), the point cluster
 * trees of the density sweep (Sec. 6.2), and uploads them to the device.
 *   d: 1 or 2.  coords: host, n_vert*d (row-major).  cells: host,
 *   n_cell*(d+1) vertex ids.  cell_is_interior: host, n_cell flags.
 *   opts: may be NULL for the defaults.
 * Errors: VFD_EINVAL (d, degenerate cells, no interior DoF, bad options),
 * VFD_ENOMEM, VFD_ECUDA. */
vfd_status vfd_mesh(int d, int64_t n_vert, const double *coords, int64_t n_cell, const int32_t *cells,
                    const uint8_t *cell_is_interior, const vfd_mesh_opts *opts, vfd_mesh_t *out);

/* dof_of_vertex: host, n_vert entries, the DoF index of each vertex or -1.
 * n_dof: host.  Either pointer may be NULL. */
vfd_status vfd_mesh_dofs(vfd_mesh_t mesh, int32_t *dof_of_vertex, int64_t *n_dof);

/* Structure counts (host int64 array of n_info entries, in this order):
 * [0] n_dof  [1] n_vert  [2] n_cell  [3] touching pairs  [4] nnz(B+M)
 * [5] tree levels  [6] tree nodes  [7] rank k  [8] admissible blocks of K
 * [9] inadmissible leaf blocks of K  [10] dense near entries of K
 * [11] quadrature points  [12] interior quadrature points
 * [13] admissible blocks of the density sweep  [14] near point pairs of the
 * density sweep  [15] stored near entries (row panels, padded to 4 columns)
 * [16] kernel evaluations of the near-block build (point pairs of the
 * computed leaf blocks)  [17] 4D points of the singular rules over all
 * touching pairs (2D; 0 in 1D)  [18] rank of the far field of the inner
 * operator of the batched mixed-precision solves. */
vfd_status vfd_mesh_info(vfd_mesh_t mesh, int64_t *info, int n_info);

/* Assemble the operator for the fields s and log kappa (Algorithm 1):
 * field values, coupling blocks S = -2 gamma(xi_a, xi_b) (Sec. 5.3, eq.
 * eq:triple_product), dense inadmissible blocks (Sec. 5.2), singular B
 * (Sec. 4), density rho (Sec. 6.2) plus tail, and M (eq. e:m).
 *   s_bar: quadrature parameter of the singular rules (Sec. 4), 0 <= s <= s_bar < 1
 *          must hold at every evaluation point unless VFD_ASSEMBLE_UNCHECKED.
 *   precision: VFD_FP64, VFD_FP32 or VFD_BF16.  stream: cudaStream_t.
 * Blocks the host once to read the field check.
 * Errors: VFD_EINVAL (field out of range, bad s_bar), VFD_EUNSUPPORTED
 * (nodal field with a low-rank part; tail with non-constant fields),
 * VFD_ENOMEM, VFD_ECUDA. */
vfd_status vfd_assemble(vfd_mesh_t mesh, const vfd_field *s, const vfd_field *log_kappa, double s_bar,
                        int precision, int flags, void *stream, vfd_op_t *out);

/* Y = A X for nrhs columns (X, Y: host or device, n_dof x nrhs, leading
 * dimension ld).  X and Y must not overlap.  VFD_FP64 operators apply the
 * FP64 operator.  VFD_FP32 / VFD_BF16 operators apply the low-precision
 * operator of the mixed-precision solve: with nrhs a multiple of 64 (and
 * leaves of at most 64 DoFs) the batched path -- near panels on the tensor
 * cores in TF32 (VFD_FP32) or BF16 (VFD_BF16) with x entering as two rounded
 * terms hi + lo, B + M and the far field in FP32, with the diagonal of B + M
 * compensated on the first batched use so that the rounded operator is exact
 * on constant vectors -- else column by column with K in FP32 and B + M in
 * FP64. */
vfd_status vfd_apply(vfd_op_t op, const double *X, double *Y, int64_t nrhs, int64_t ld, void *stream);

/* Y = (sum of the selected parts) X; parts is a mask of VFD_PART_*. */
vfd_status vfd_apply_parts(vfd_op_t op, int parts, const double *X, double *Y, int64_t nrhs, int64_t ld,
                           void *stream);

/* Size of the fixed device scratch used by vfd_apply_noalloc (8 MiB per device). */
#define VFD_APPLY_NOALLOC_SCRATCH_BYTES 8388608

/* Y = A X for nrhs columns, as vfd_apply computes it column by column, but
 * without allocating anything during the call.  The paper has no counterpart:
 * this is a library convenience.
 *
 * Who needs it: callers that must not allocate device memory while they run,
 * e.g. a solver loop whose device memory is reserved in advance by another
 * framework's memory pool (a cudaMalloc could fail or make the pool give back
 * cached blocks), or code on a latency-critical path where cudaFree would wait
 * for the whole device.  vfd_apply may allocate on its first call and whenever
 * nrhs grows (operator workspaces, a side stream for the far field), and it
 * copies host arguments through device buffers.
 *
 * What differs from vfd_apply:
 *  - X and Y must be device pointers (n_dof x nrhs, leading dimension ld);
 *    host pointers are rejected with VFD_EINVAL.
 *  - The far-field scratch lives in one file-scope device array of
 *    VFD_APPLY_NOALLOC_SCRATCH_BYTES bytes per device.  An operator and nrhs
 *    whose scratch, 8 bytes (VFD_FP64 operators) or 4 bytes (VFD_FP32 and
 *    VFD_BF16 operators) times
 *    nrhs x (2 x tree nodes x rank + far levels x leaves x rank), rounded up
 *    to 256-byte pieces, exceeds that size is rejected with VFD_EINVAL and a
 *    message that gives both sizes; nothing is launched then.
 *  - Nothing in the scratch has to start at zero: every entry read is written
 *    earlier in the same call.
 *  - All kernels run in order on `stream`; the far field is not overlapped
 *    with the near field (so it can be slower than vfd_apply).
 *  - Low-precision operators always take the column-by-column path (K in
 *    FP32, B + M in FP64), never the batched tensor-core path.
 *  - Setup: the first call on each device (with that device current) looks up
 *    the device address of the scratch array once (cudaGetSymbolAddress);
 *    make that first call before any stream capture begins.
 *  - Calls that overlap in time on the same device (other streams or host
 *    threads) share the one scratch array and race; order them, e.g. on one
 *    stream.  X and Y must not overlap.
 * Errors: VFD_EINVAL (null or host pointers, bad nrhs / ld, scratch too
 * small), VFD_EUNSUPPORTED (device ordinal >= 64), VFD_ECUDA. */
vfd_status vfd_apply_noalloc(vfd_op_t op, const double *X, double *Y, int64_t nrhs, int64_t ld, void *stream);

/* Solve A U = F by conjugate gradients (Sec. 7: "conjugate gradient
 * solver"), every iteration on the device, column by column for nrhs > 1.
 * F, U: host or device, n_dof x nrhs, leading dimension ld; U holds the
 * initial guess on entry.  Converged when ||F - A U|| <= rtol ||F||.
 * iters, relres: host arrays of nrhs entries (may be NULL).
 * VFD_FP64 operators: FP64 CG, column by column.  VFD_FP32 / VFD_BF16
 * operators: the residual F - A U in FP64 with the FP64 operator; with
 * nrhs = 1 iterative refinement around an inner CG with FP32 K; with nrhs > 1
 * all columns are solved together as in vfd_batch_solve (a batched CG in
 * FP32 vectors whose near-field products run on the tensor cores, TF32 or
 * BF16, with FP64 reliable updates) -- this needs leaves of at most 64 DoFs.
 * iters reports the inner CG iterations.
 * Returns VFD_ENOCONV when some column did not converge in max_it. */
vfd_status vfd_solve(vfd_op_t op, const double *F, double *U, int64_t nrhs, int64_t ld, double rtol,
                     int max_it, int *iters, double *relres, void *stream);

/* Preconditioner of the CG solves of vfd_solve (the paper solves with plain
 * CG, Sec. 7, and names a multilevel preconditioner as the next step,
 * Sec. 8).  kind VFD_PREC_TWO_LEVEL: additive two-level preconditioner,
 * M^-1 = sum over the leaves of the cluster tree of exact solves with the
 * leaf's diagonal block of A (near panel block plus the B + M entries inside
 * the leaf), plus a coarse solve on the functions constant on the clusters of
 * one tree level (the deepest with at most 512 clusters; A_c = R A R^T, R the
 * cluster indicators); VFD_PREC_BLOCK_JACOBI: the leaf blocks only.  Both
 * parts are SPD, so the solves run preconditioned CG (stopping test
 * unchanged: the residual of A).  Used by the FP64 CG of VFD_FP64 operators
 * and by the batched mixed-precision solve (nrhs > 1 on a VFD_FP32 or
 * VFD_BF16 operator, or vfd_batch_solve when every operator of the batch is
 * preconditioned: FP32 copies of the inverses); not by the one-column
 * refinement of low-precision operators.  Setup, FP64 from the operator's
 * FP64 parts: the leaf blocks inverted on the device (Cholesky in shared
 * memory; leaves above 96 DoFs on the host), A_c summed from the operator's
 * parts (near-block sums, B + M entries, admissible blocks contracted with the
 * clusters' per-level basis sums) and inverted on the host; blocks until done.
 * VFD_PREC_NONE switches back to plain CG.  The batched solve needs leaves of
 * at most 128 DoFs.  Errors: VFD_EINVAL (unknown kind, a block that is not
 * positive definite), VFD_ECUDA. */
enum { VFD_PREC_NONE = 0, VFD_PREC_TWO_LEVEL = 1, VFD_PREC_BLOCK_JACOBI = 2 };
vfd_status vfd_precondition(vfd_op_t op, int kind, void *stream);

/* P1 load F = M0 f (exact P1 mass matrix of the interior cells times the
 * nodal values f at all n_vert vertices).  f_nodal, F: host or device. */
vfd_status vfd_load(vfd_mesh_t mesh, const double *f_nodal, double *F, void *stream);

/* Batch of operators (meshes) for the batched low-precision path: one
 * launch per stage over a global queue of work items of all meshes, and one
 * batched mixed-precision solve with scalars per (mesh, column).  The paper solves
 * one mesh at a time; the batch is a throughput construction on top of the
 * per-mesh operators of Sec. 5-7.
 * ops: nops operators, all VFD_FP32 or all VFD_BF16, leaves of at most 64
 * DoFs; they must outlive the batch (not owned).  Errors: VFD_EINVAL,
 * VFD_EUNSUPPORTED, VFD_ENOMEM. */
vfd_status vfd_batch_create(const vfd_op_t *ops, int nops, vfd_batch_t *out);

/* Y_m = A_low,m X_m for every mesh m of the batch: the batched apply of
 * vfd_apply (near panels on the tensor cores in TF32 or BF16, B + M and the
 * far field in FP32) for all meshes at once.  X, Y: host arrays of nops
 * device pointers, block m n_dof(m) x nrhs, leading dimension ld[m];
 * nrhs a multiple of 64. */
vfd_status vfd_batch_apply(vfd_batch_t batch, const double *const *X, double *const *Y, const int64_t *ld,
                           int64_t nrhs, void *stream);

/* Solve A_m U_m = F_m for every mesh (nrhs columns each): one CG on the
 * low-precision operators of all meshes at once (FP32 vectors, per-(mesh,
 * column) scalars) for the correction to U, with reliable updates per mesh:
 * once every still-iterating column of a mesh has cut its recursive residual
 * 0.03-fold, the mesh's correction is added to U in FP64 and its residual is
 * replaced by the true F - A U computed with its FP64 operator, the search
 * direction continuing (or restarting where the two residuals disagree).
 * The low-precision operators are made exact on constant vectors by a
 * diagonal compensation computed on their first batched use.  Stops when
 * ||F - A U|| <= rtol ||F|| for every column of every mesh.  F, U: host
 * arrays of nops device pointers (U holds the initial guess).  iters,
 * relres: host, nops x nrhs (mesh-major), may be NULL; iters = the inner
 * iterations run until the column's mesh converged.  VFD_ENOCONV when max_it
 * inner iterations did not suffice or a residual became non-finite (U holds
 * the last iterate). */
vfd_status vfd_batch_solve(vfd_batch_t batch, const double *const *F, double *const *U, const int64_t *ld,
                           int64_t nrhs, double rtol, int max_it, int *iters, double *relres, void *stream);

/* The tile configuration the batch picked for its near-panel kernel by timing
 * every candidate once on its first apply (zero inputs): chosen[0..5] = panel
 * columns per pipeline stage, pipeline depth, CTAs per panel, warps per CTA,
 * accumulator register sets, and 1 for the tcgen05 (tensor-memory) kernel, 0
 * for the mma.sync kernel (all 0 before the first apply); us[i] = candidate
 * i's time in microseconds (0 = not run or does not fit), n entries at most;
 * *ncand = the number of candidates.  VFD_ETIMEOUT from an apply or solve
 * means a tcgen05 pipeline wait expired (the kernel gave up, outputs invalid). */
vfd_status vfd_batch_tuning(vfd_batch_t batch, int *chosen, float *us, int n, int *ncand);

/* Pin the near-panel configuration of the batch to candidate cfg (0 <= cfg <
 * *ncand; a candidate that does not fit in shared memory makes the next apply
 * fail with VFD_EUNSUPPORTED), or cfg = -1: time the candidates on the next
 * apply and keep the fastest (the default).  Takes effect on the next apply. */
vfd_status vfd_batch_set_config(vfd_batch_t batch, int cfg, int *ncand);

/* Bound of the device-side pipeline waits of the batch's tensor-core near
 * kernel (default 1 second; the paper has no counterpart).  A wait that runs
 * out makes every CTA of the kernel stop issuing work, wait (again bounded)
 * for the copies and products it already issued, free its tensor memory and
 * leave its outputs unwritten; the apply or solve then returns VFD_ETIMEOUT
 * without touching the caller's output blocks, and the next call starts
 * clean.  seconds >= 0; 0 makes every wait that is not already satisfied
 * give up at once (a way to exercise the failure path).  Errors:
 * VFD_EINVAL (negative or non-finite seconds). */
vfd_status vfd_batch_set_wait_limit(vfd_batch_t batch, double seconds);

/* The factor by which every still-iterating column of a mesh must cut its
 * recursive (inner, low-precision) residual before the batched solve replaces
 * it by the FP64 true residual F - A U (a reliable update; the mixed
 * precision is not in the paper, whose CG is FP64, Sec. 7).  Default 0.03.
 * A deeper drop (smaller factor) runs fewer FP64 applies but trusts the
 * low-precision recursion longer.  Takes effect on the next solve.  Errors:
 * VFD_EINVAL (drop not in (0, 1)). */
vfd_status vfd_batch_set_update_drop(vfd_batch_t batch, double drop);

void vfd_batch_free(vfd_batch_t batch);

/* Adjoint gradient (the paper has no gradients; derivative of the discrete
 * operator A = B + K + M of Sec. 3 with every quadrature rule and s_bar held
 * fixed):
 *   g_s[k]        = -sum_r Lam_r^T (dA/ds_k) U_r,
 *   g_logkappa[k] = -sum_r Lam_r^T (dA/dlogkappa_k) U_r,
 * for P1 (nodal) fields s and log kappa, k over all n_vert vertices.  With
 * A Lam = dJ/dU this is dJ/dtheta of any J(U(theta)).  The kernel
 * derivatives are -ln|x-y| gamma (psi_k(x) + psi_k(y)) and
 * gamma (psi_k(x) + psi_k(y)) / 2; touching pairs go through the singular
 * rules of Sec. 4, separated pairs through the element rules.
 * U, Lam: device, n_dof x nrhs, leading dimension ld.  g_s, g_logkappa:
 * device, n_vert doubles each, overwritten.  The operator's fields must be
 * VFD_FIELD_NODAL (such operators have no low-rank part) and the mesh must
 * have tail_mode 0.  The separated pairs are summed directly: O(n_q^2) work.
 * Errors: VFD_EINVAL (null or host pointers, bad nrhs / ld), VFD_EUNSUPPORTED
 * (analytic fields, exterior tail), VFD_ECUDA. */
vfd_status vfd_grad(vfd_op_t op, const double *U, const double *Lam, int64_t nrhs, int64_t ld, double *g_s,
                    double *g_logkappa, void *stream);

/* Density rho (incl. tail) at the interior quadrature points, ordered by
 * interior cell (increasing cell id) then element-rule point (triangle:
 * the point nearest to stored vertex 0, 1, 2; interval: Gauss points left
 * to right in the stored orientation).  rho: host or device, n_qint doubles. */
vfd_status vfd_op_rho(vfd_op_t op, double *rho, void *stream);

/* Rank of every far level of the operator's FP64 far field, coarsest first:
 * the interpolation rank p^d, or after recompression (recompress_tol > 0)
 * the padded rank of each level.  *nlev = number of far levels (0 without
 * admissible blocks); ranks (may be null) receives min(n, *nlev) entries. */
vfd_status vfd_op_far_ranks(vfd_op_t op, int *ranks, int n, int *nlev);

/* Device time per assembly phase (VFD_T_* order) of the vfd_assemble call
 * that created op, if it was given VFD_ASSEMBLE_TIMED; ms: host, n entries
 * (at most VFD_T_COUNT are written).  Returns VFD_EINVAL if not recorded. */
vfd_status vfd_op_timings(vfd_op_t op, double *ms, int n);

/* Self-test of the library's table-driven FP64 logarithm / exponential used
 * for the kernel evaluations (Tang's table-driven method): out[i] =
 * log(x[i]) (which = 0), exp(x[i]) (which = 1), cos(pi x[i]) (which = 2) or
 * sin(pi x[i]) (which = 3), computed on the device.
 * x, out: device pointers, n entries.  Needs a mesh handle for the tables.
 * Valid inputs: x > 0 normal (log), |x| < 700 (exp), |x| < 2^24 (cos, sin). */
vfd_status vfd_selftest_math(vfd_mesh_t mesh, int which, int64_t n, const double *x, double *out, void *stream);

void vfd_free_op(vfd_op_t op);
void vfd_free_mesh(vfd_mesh_t mesh);

/* Message of the last failing call on this thread ("" if none). */
const char *vfd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VFD_H */
