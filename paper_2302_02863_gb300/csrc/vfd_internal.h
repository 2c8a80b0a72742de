// Internal declarations of the vfd library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/vfd.h"

namespace vfd {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string &msg);

struct Error {
    vfd_status st;
    std::string msg;
};

#define VFD_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            throw ::vfd::Error{e_ == cudaErrorMemoryAllocation ? VFD_ENOMEM : VFD_ECUDA,        \
                               std::string(#call) + ": " + cudaGetErrorString(e_)};            \
    } while (0)

#define VFD_REQUIRE(cond, st, msg)                                                             \
    do {                                                                                       \
        if (!(cond)) throw ::vfd::Error{st, msg};                                              \
    } while (0)

// device buffer (RAII, cudaMalloc/cudaFree)
template <class T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) VFD_CUDA(cudaMalloc(&p, sizeof(T) * count));
    }
    void upload(const std::vector<T> &h) {
        alloc(h.size());
        if (!h.empty()) VFD_CUDA(cudaMemcpy(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice));
    }
    void zero(cudaStream_t st) {
        if (n) VFD_CUDA(cudaMemsetAsync(p, 0, sizeof(T) * n, st));
    }
    size_t bytes() const { return sizeof(T) * n; }
};

constexpr int KMAX = 64;       // max rank p^d handled by the kernels
constexpr int PMAX = 8;        // max Chebyshev nodes per dimension
constexpr int NSMAX = 16;      // max Gauss points per direction of the singular rules
constexpr int QB = 4;          // stride of the barycentric coordinates of a quadrature point (d + 1 <= 4)
constexpr int NQMAX = 4;       // element-rule points per cell: 3 (interval, triangle), 4 (tetrahedron)

// ---------------------------------------------------------------------------
// device view of a field descriptor
// ---------------------------------------------------------------------------
struct DField {
    int nodal;          // 1: P1 values at vertices (vals)
    int nF, nG, nT;     // term counts
    int squash;
    int kmax;           // max |k_i| of the Fourier rows (fast path when <= 4)
    double c0, lo, hi;
    const double *rows; // device, (nF + nG + nT) * 5
    const double *vals; // device, n_vert (nodal)
    // 2D Fourier rows with integer |k| <= 4 and k_3 = 0, grouped by k_1 (0 groups
    // otherwise): gint = per group (|k_1|, rows), then per row |k_2|; gcoef = per
    // row four coefficients with the signs of k_1, k_2 folded in
    int ngrp;
    const int *gint;
    const double *gcoef;
};

// ---------------------------------------------------------------------------
// cluster tree (complete binary, heap numbering: children of n are 2n+1, 2n+2)
// ---------------------------------------------------------------------------
struct Tree {
    int L = 0;                     // leaf level; levels 0..L
    int nnode = 0, nleaf = 0;
    std::vector<int> begin, end;   // index range in tree order, per node
    std::vector<int> perm;         // tree position -> original item
    std::vector<double> lo, hi;    // boxes, nnode * d
    int first_leaf() const { return (1 << L) - 1; }
    bool is_leaf(int n) const { return n >= first_leaf(); }
};

// closest cell and its barycentric coordinates (QB per point) for a set of
// points (the Chebyshev nodes of a tree): P1 field values there
struct NodeLoc {
    bool done = false;
    std::vector<int> cell_h;
    std::vector<double> bary_h;
    DBuf<int> cell;
    DBuf<double> bary;
};

// ---------------------------------------------------------------------------
// mesh handle: geometry-only data, built once per mesh
// ---------------------------------------------------------------------------
struct MeshData {
    int d = 2, M = 0, C = 0, N = 0;
    int nQ = 0, nQint = 0;
    int nqc = 3;                     // element-rule points per cell
    vfd_mesh_opts opts{};
    double h_max = 0.0;
    int k = 16, p = 4;

    std::vector<double> X;           // host coords M*d
    std::vector<int> T;              // host cells C*(d+1)
    std::vector<uint8_t> inter;      // host
    std::vector<int> dof_of_vertex;  // host
    std::vector<int> vertex_of_dof;  // host
    std::vector<int> qcell_host;     // host, point -> cell (interior cells first)

    // device geometry
    DBuf<double> vx;       // M*d, SoA: vx[i*M + v]
    DBuf<int> cells;       // C*(d+1)
    DBuf<int> vdof;        // M: dof of vertex or -1
    DBuf<double> qx;       // nQ*d SoA
    DBuf<double> qw;       // nQ
    DBuf<int> qcell;       // nQ
    DBuf<double> qbary;    // nQ*QB barycentric coordinates

    // touching pairs (unordered, canonical orientation)
    int npairs = 0;
    DBuf<int> pair_info;   // npairs * 8: type, w(1|2), pv0..2, qv0..2
    std::vector<int> pair_info_h;   // host copy
    // gradient gather lists (built on the first vfd_grad): vertex -> point * QB + slot, vertex -> pair * 6 + slot
    bool grad_lists = false;
    DBuf<int> gq_ptr, gq_idx, gp_ptr, gp_idx;
    // B/M sparsity (DoF CSR) and deterministic gather lists
    int nnz = 0;
    DBuf<int> rowptr, colidx;
    DBuf<int> cB_ptr, cB_idx;             // entry -> list of pair*25 + li*5 + lj
    DBuf<int> cM_ptr, cM_q;               // entry -> list of interior point ids
    DBuf<double> cM_coef;                 //   with coefficient 2 w lam_i lam_j
    int64_t ncontribB = 0, ncontribM = 0;

    // K tree (over DoFs; DoF index = tree position)
    Tree kt;
    DBuf<int> kt_begin, kt_end;
    DBuf<double> kt_cheb;      // nnode * k * d (node-major, point, dim)
    DBuf<int> kt_Uoff;         // nleaf
    int far_lmin = 0;          // first level with admissible blocks
    DBuf<double> Ul64;         // per-level bases, (L - far_lmin + 1) x N x k (the last slice is U)
    DBuf<double> E64;          // transfers E_c[beta][alpha] = l^parent_alpha(xi^c_beta), nnode x k x k
    int p_in = 0, k_in = 0;    // interpolation order / rank of the inner operator's far field (0: p, k)
    DBuf<double> kt_cheb_in, U_in64, E_in64;   // its Chebyshev nodes, leaf bases (N x k_in), transfers
    // admissible blocks (both orders), CSR by row node
    int nfar = 0;
    std::vector<int> far_ptr_h, far_col_h;
    DBuf<int> far_ptr, far_col;
    // inadmissible leaf pairs (both orders), CSR by row leaf
    int nnear = 0;
    int64_t near_entries = 0;
    std::vector<int> near_ptr_h, near_col_h;
    std::vector<int64_t> near_off_h;
    DBuf<int> near_ptr, near_col;
    DBuf<int64_t> near_off;    // offset of block e's (0,0) entry in its row leaf's panel
    DBuf<int> panel_w;         // per row leaf: panel row stride (padded to 8)
    DBuf<int64_t> panel_off;   // per row leaf: panel start (nleaf + 1)
    int64_t near_entries_alg = 0;   // sum |sigma||sigma'| over near blocks (no padding)
    int64_t near_point_pairs = 0;   // kernel evaluations of the near-block build (computed blocks)
    int64_t sing_points = 0;        // 4D points of the singular rules over all touching pairs (2D)
    DBuf<int> gcol, gcol_off;  // per panel column the DoF of its x entry (-1: padding)
    DBuf<int64_t> bm_pos;      // per B + M entry its flat position in the near panels (-1: none)
    bool bm_in_panels = false; // every B + M entry has a panel position
    DBuf<int> vleaf;           // leaf of every DoF
    int max_panel_w = 0;
    DBuf<int> near_src;        // per block: index of the computed block it is the transpose of, or -1
    DBuf<int> near_pair_row;   // per block: row leaf (for launch over blocks)
    // per-leaf point sets for the near-block build
    DBuf<int> lp_ptr, lp_pts;          // leaf -> element-rule points of the cells in its supports
    DBuf<int> supp_ptr, supp_loc;      // DoF -> (index into its leaf's point list, coefficient)
    DBuf<double> supp_coef;
    int max_leaf_pts = 0, max_leaf_size = 0, max_supp = 0;

    // density sweep: target tree (interior points) and source tree (all points)
    Tree tt, st;
    DBuf<int> tt_begin, tt_end, tt_perm, st_begin, st_end, st_perm;
    DBuf<double> tt_lo, tt_hi;          // target boxes (for the downsweep basis)
    DBuf<double> tt_cheb, st_cheb;      // nnode * k * d
    DBuf<double> st_xhat;               // source node moments sum_q l_b(q) w_q, nnode_s * k
    int nrfar = 0;
    DBuf<int> rfar_ptr, rfar_col;       // by target node
    int nrnear = 0;
    int64_t rnear_pairs = 0;
    DBuf<int> rnear_ptr, rnear_col;     // by target leaf
    DBuf<double> gl_x, gl_w;            // Gauss-Legendre on [0,1], n_sing points
    DBuf<double> gl9_x, gl9_w;          // 9-point rule for the tail
    DBuf<double> mtab;                  // tables of the table-driven FP64 log/exp

    DBuf<int> rfarT_ptr, rfarT_col;     // transposed: source node -> target nodes
    DBuf<int> rnearT_ptr, rnearT_col;   // transposed: source leaf index -> target leaf indices

    // load assembly (exact P1 mass)
    DBuf<int> ld_ptr, ld_idx;           // DoF -> list of cell*(d+1)+a contributions

    // orthogonal factors of the far-field bases (recompress.cu, first recompressing assembly)
    bool rc_factors = false;
    DBuf<double> rc_T1, rc_R;          // per node W L^-1/2 and L^1/2 W^T of the basis Gram matrix

    // host copies for the nearest-point location of the Chebyshev nodes
    std::vector<double> kt_cheb_h, kt_cheb_in_h, tt_cheb_h, st_cheb_h;
    std::vector<int> lp_ptr_h, lp_pts_h;
    bool nodes_located = false;
    NodeLoc kt_loc, kt_in_loc, tt_loc, st_loc;   // built by locate_nodes (first nodal-field assembly)
    // gradient lists through the K-near point sets and the Chebyshev nodes (built on the first vfd_grad)
    DBuf<int> gl_ptr, gl_idx;           // vertex -> leaf-point entry * QB + slot (K near point sets)
    DBuf<int> gn_ptr, gn_idx;           // vertex -> node entry * QB + slot (K, target, source nodes)
    DBuf<double> gn_bary;               // barycentric coordinates of every node entry (QB each)
};

// ---------------------------------------------------------------------------
// operator handle: per-field data
// ---------------------------------------------------------------------------
struct OpData {
    MeshData *m = nullptr;
    int precision = VFD_FP64;
    double s_bar = 0.9;
    bool check_fields = true;
    DField fs{}, fk{};
    DBuf<double> f_rows_s, f_rows_k, f_vals_s, f_vals_k;
    DBuf<int> f_gint_s, f_gint_k;
    DBuf<double> q_s, q_lk;            // at all quadrature points
    DBuf<double> kc_s, kc_lk;          // at K-tree Chebyshev nodes
    DBuf<double> kc_s_in, kc_lk_in;    // at the inner operator's Chebyshev nodes (low-precision operators)
    DBuf<double> S64_in;               // the inner operator's coupling blocks, nfar x k_in x k_in
    DBuf<double> tc_s, tc_lk, sc_s, sc_lk;  // density trees' Chebyshev nodes
    DBuf<double> valB, valM, valBM;    // CSR values
    DBuf<double> rho;                  // interior points, canonical order
    DBuf<double> S64;                  // nfar * k * k
    DBuf<double> D64;                  // near entries
    DBuf<float> S32, D32, Ul32;        // FP32 copies (VFD_FP32)
    DBuf<unsigned short> Dtc;          // BF16 near panels pre-tiled for the TMA-fed tcgen05 kernel (first batched use)
    std::vector<int64_t> Dtc_off;      //   element offset of each leaf's image (nleaf + 1)
    DBuf<int64_t> Dtc_doff;
    DBuf<float> D32t;                  // D32 rounded to TF32 (batched tensor-core path, built on first use)
    DBuf<unsigned short> D16;          // batched-path BF16 near panels (VFD_BF16, mma.sync candidates)
    DBuf<float> diag32;                // batched TF32 path: diagonal of A (FP32, compensated); B + M off the
                                       //   diagonal is folded into its panels D32t
    bool bm_folded = false;            // the batched panels (D16 + Dtc, or D32t + diag32) are built
    int far_kp = 0;                    // padded rank of the batched far-field copies (0: not built)
    DBuf<unsigned char> Up_lp, Sp_lp;   // flattened bases (N x nlev kp) and S in the operator's low precision (batched path)
    DBuf<float> valBM32;               // FP32 copy of B + M (inner operator of refinement)
    bool comp_done = false;            // valBM32's diagonal compensated (batched path, first use)
    // the batch of one used by the batched (multi-RHS) low-precision apply / solve
    struct BatchData *self = nullptr;
    // adjoint gradient workspaces
    DBuf<double> gr_uq, gr_lq, gr_hs, gr_h1, gr_pg;   // point values, point sensitivities, pair slots
    DBuf<double> gr_cq, gr_hKs, gr_hKk;                // c_q; K-near leaf-point sensitivities
    DBuf<double> gr_Gs, gr_Gk, gr_xU, gr_xL, gr_ct;    // node sensitivities; K far moments; target moments
    // apply workspace
    int ws_nrhs = 0;
    DBuf<double> xhat, yhat;           // nnode * k * ws_nrhs
    DBuf<float> xhat32, yhat32;
    DBuf<double> P64;                  // leaf-level projections nlev * nleaf * k * nrhs
    DBuf<double> ye64;                 // per admissible block coupling products nfar * k * nrhs
    // recompressed far field of the FP64 operator (recompress.cu): per-level ranks
    bool rc_on = false;
    std::vector<int> rc_kl;            // rank of each far level
    std::vector<long long> rc_uo;      // offset of each level's flattened basis in Ulc64
    DBuf<double> Ulc64, Sc64;          // flattened bases (N x kl per level), couplings (kl x kl per block)
    DBuf<long long> rc_so;             // offset of each block's coupling in Sc64
    DBuf<int> rc_bk;                   // rank of each block
    DBuf<float> ye32;
    DBuf<float> P32;
    cudaStream_t side = nullptr;       // far-field branch of the apply
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    DBuf<double> xin, yout;            // staging for host pointers
    // solver workspace
    DBuf<double> cg_r, cg_p, cg_q, cg_x, cg_b, cg_z;
    DBuf<double> cg_red;               // reduction partials
    DBuf<double> cg_scal;              // device scalars (8)
    DBuf<int> cg_flag;
    DBuf<int> errflag;
    double phase_ms[VFD_T_COUNT] = {0};
    bool timed = false;
    cudaGraphExec_t cg_exec[2] = {nullptr, nullptr};   // captured CG chunks (FP64 K, FP32 K)
    const void *cg_key[2] = {nullptr, nullptr};
    cudaGraphExec_t pcg_exec = nullptr;  // captured PCG chunk
    const void *pcg_key = nullptr;
    // two-level preconditioner (precond.cu): leaf-block inverses and the coarse inverse
    int prec_kind = 0;                 // 0 none, 1 two-level, 2 leaf blocks only
    long long prec_version = 0;        // incremented by every setup
    int prec_mb = 0, prec_nc = 0, prec_span = 1;   // block size; coarse clusters; leaves per cluster
    DBuf<double> prec_blk;             // nleaf x mb x mb (inverse of each leaf's diagonal block)
    DBuf<float> prec_blk32;            //   FP32 copy (batched solve)
    DBuf<double> prec_coarse;          // nc x nc (inverse of R A R^T)
    DBuf<float> prec_coarse32;         //   FP32 copy
    DBuf<int> prec_cidx;               // coarse cluster of every DoF
    DBuf<double> prec_rl, prec_zc;     // leaf sums of the residual (nleaf), coarse correction (nc)
};

// ---------------------------------------------------------------------------
// batch of low-precision operators (one mesh each) for the batched apply and
// the batched refinement solve: the kernels walk global work-item queues
// over all meshes (batched.cu, bsolve.cu)
// ---------------------------------------------------------------------------
struct BatchData {
    std::vector<OpData *> ops;          // not owned
    int nmesh = 0, precision = VFD_FP32;
    int64_t ntot = 0;                   // sum of the meshes' DoFs
    std::vector<int64_t> xoff;          // first row of each mesh (nmesh + 1)
    int R = 0;                          // columns the workspaces below are built for (0: not built)
    DBuf<unsigned char> desc;           // nmesh descriptors (MrMesh)
    DBuf<int> leaf_items, node_items;   // (mesh, leaf) / (mesh, node with admissible blocks) pairs
    DBuf<unsigned char> near_items;     // NearItem records
    int n_leaf_items = 0, n_node_items = 0, n_near_items = 0;
    DBuf<long long> row_off;            // xoff on the device
    int max_panel_w = 0, max_k = 0, max_kp = 0, max_leaf = 0;
    int near_cfg = -1;                  // tile configuration of the near-panel kernel (timed on first use)
    int forced_cfg = -1;                // >= 0: configuration pinned by the caller
    float near_cfg_us[32] = {0};        // the timings of the candidates (0: not run)
    bool any_far = false;
    DBuf<float> xhat, yhat, y2;         // far-field workspaces (all meshes), near partials of a split
    DBuf<float> fpart;                  // far-field leaf projections (all meshes)
    int max_mt = 0;                     // largest flattened basis width nlev * kp
    DBuf<float> xi, yi;                 // interleaved staging of the column-major apply
    DBuf<unsigned char> xc;             // x for the BF16 near kernels, BF16 hi then lo ([2][ntot][R])
    DBuf<int> tc_err;                   // set by the tcgen05 kernel when a pipeline wait expires
    DBuf<unsigned char> tc_items;       // TcItem records of the tcgen05 kernel (one per (mesh, leaf))
    int n_tc_items = 0;
    long long wait_ns = 1000000000LL;   // bound of the tcgen05 kernel's pipeline waits
    double ru_drop = 0.03;              // recursive-residual reduction between reliable updates
    // batched refinement solve
    DBuf<float> x, r, p, q, b, red, red2, sc;
    DBuf<float> qf;                     // far-field part of q in the captured iteration (added by the vector kernels)
    bool fused = false;                 // the captured iteration uses the cooperative vector kernel
    void *p16_target = nullptr;         // where that kernel writes p as BF16 hi / lo (the near kernels' x blocks), or null
    DBuf<unsigned> gbar;                // its grid-barrier counter and generation
    DBuf<int> flag, red_items, red_mesh;
    int nred = 0, sR = 0;
    // preconditioned batched solve (every operator of the batch preconditioned):
    // FP32 leaf-block and coarse inverses of all meshes, work items and maps
    bool pcg = false;                   // the captured chunk is the preconditioned one
    std::vector<long long> pc_key;      // preconditioner versions the tables below were built from
    DBuf<float> z, pc_blk, pc_coarse, pc_rl, pc_zc;
    DBuf<int> pc_items, pc_pmesh, pc_ctiles, pc_rowclu;
    DBuf<long long> pc_boff, pc_coff;
    int n_pc_items = 0, n_pc_ctiles = 0, pc_mbmax = 0, pc_any_coarse = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t side = nullptr;        // far-field branch of the batched apply
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~BatchData();
};

// ---------------------------------------------------------------------------
// host setup (mesh_setup.cpp)
// ---------------------------------------------------------------------------
MeshData *build_mesh(int d, int64_t n_vert, const double *coords, int64_t n_cell, const int32_t *cells,
                     const uint8_t *inter, const vfd_mesh_opts &opts);
void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w);
std::vector<double> make_math_tables();
void cheb_nodes_1d(int p, double lo, double hi, double *out);

// ---------------------------------------------------------------------------
// kernels (launch wrappers)
// ---------------------------------------------------------------------------
// assemble.cu
void launch_field_points(const MeshData &m, OpData &op, cudaStream_t st);
// nearest-point location of every tree's Chebyshev nodes (mesh_setup.cpp)
void locate_nodes(MeshData &m);
void launch_singular_B(const MeshData &m, OpData &op, DBuf<double> &Lbuf, cudaStream_t st);
void launch_gather_B(const MeshData &m, OpData &op, const DBuf<double> &Lbuf, cudaStream_t st);
void launch_density(const MeshData &m, OpData &op, cudaStream_t st);
void launch_gather_M(const MeshData &m, OpData &op, cudaStream_t st);
void launch_coupling_build(const MeshData &m, OpData &op, cudaStream_t st);
void launch_near_build(const MeshData &m, OpData &op, cudaStream_t st);
void launch_convert_fp32(const MeshData &m, OpData &op, cudaStream_t st);
void launch_load(const MeshData &m, const double *f, double *F, cudaStream_t st);
void launch_selftest_math(const MeshData &m, int which, long long n, const double *x, double *out, cudaStream_t st);
// apply.cu
void apply_parts_ex(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                    bool lowp, cudaStream_t st, const int *skip);
void apply_parts(const MeshData &m, OpData &op, int parts, const double *X, double *Y, int nrhs, int64_t ld,
                 cudaStream_t st);
void recompress_far(MeshData &m, OpData &op, double tol, cudaStream_t st);
void grad_adjoint(MeshData &m, OpData &op, const double *U, const double *Lam, int nrhs, int64_t ld, double *g_s,
                double *g_lk, cudaStream_t st);
void apply_noalloc(const MeshData &m, const OpData &op, const double *X, double *Y, int nrhs, int64_t ld,
                   cudaStream_t st);
// solve.cu
void release_graphs(OpData &op);
void release_streams(OpData &op);
void release_bgraph(BatchData &b);
BatchData *op_batch(OpData &op);   // the op's batch of one (created on first use)
int batch_tuning(const BatchData &b, int *chosen, float *us, int n);
void batch_check(BatchData &b, cudaStream_t st);
int batch_set_config(BatchData &b, int cfg);
// Yfar (non-null): the far field goes to Yfar (written, on the side stream)
// instead of being added into Y; the caller adds the two
void batch_apply(BatchData &b, const float *X, float *Y, int R, cudaStream_t st, const int *skip,
                 const int *mdone, bool x_bf16_ready = false, float *Yfar = nullptr);
void *batch_x16(BatchData &b);   // the BF16 hi / lo x blocks the near kernels read (BF16 batches), or null
void batch_x_to_bf16(BatchData &b, const float *X, int R, cudaStream_t st);
void batch_apply_colmajor(BatchData &b, const double *const *X, double *const *Y, const int64_t *ld, int nrhs,
                          cudaStream_t st);
vfd_status batch_solve(BatchData &b, const double *const *F, double *const *U, const int64_t *ld, int R, double rtol,
                       int max_it, int *iters, double *relres, cudaStream_t st);
void build_batched_panels(const MeshData &m, OpData &op, cudaStream_t st);
// near_tc.cu (tcgen05 near panels with bulk-copied panel stages, BF16)
void build_tiled_panels(const MeshData &m, OpData &op, const double *D, cudaStream_t st);
void build_tc_items(BatchData &b);
size_t near_tma_smem(int nstage, int max_panel_w);
bool launch_near_tma(BatchData &b, int nstage, int ksplit, int R, const float *X, float *Y, cudaStream_t st,
                     const int *skip, const int *mdone);
// far_batched.cu (nested H^2 far field of the batched apply)
void build_far_lowp(const MeshData &m, OpData &op, cudaStream_t st);
size_t far_batched_smem(int kp, int mt);
void launch_far_side(BatchData &b, int R, const float *X, cudaStream_t side, const int *skip, const int *mdone);
void launch_far_down(BatchData &b, int R, float *Y, cudaStream_t st, const int *skip, const int *mdone, bool add);
void launch_lowp_csr(const MeshData &m, OpData &op, cudaStream_t st);
vfd_status cg_solve(const MeshData &m, OpData &op, const double *F, double *U, int nrhs, int64_t ld, double rtol,
                    int max_it, int *iters, double *relres, cudaStream_t st);
// precond.cu
void precond_setup(const MeshData &m, OpData &op, int kind, cudaStream_t st);

}  // namespace vfd
