// C ABI of the vfd library (declared in include/vfd.h): argument checks,
// host/device staging, handle lifetimes and error reporting.  All
// computation happens in the CUDA kernels of assemble.cu / apply.cu / solve.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>

#include "vfd_internal.h"

struct vfd_mesh_s {
    vfd::MeshData *m;
};
struct vfd_op_s {
    vfd::OpData *op;
};
struct vfd_batch_s {
    vfd::BatchData *b;
};

namespace vfd {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

}  // namespace vfd

using namespace vfd;

#define VFD_API_BEGIN try {
#define VFD_API_END                                                                \
    }                                                                              \
    catch (const vfd::Error &e) {                                                  \
        vfd::set_error(e.msg);                                                     \
        return e.st;                                                               \
    }                                                                              \
    catch (const std::bad_alloc &) {                                               \
        vfd::set_error("host allocation failed");                                  \
        return VFD_ENOMEM;                                                         \
    }                                                                              \
    catch (const std::exception &e) {                                              \
        vfd::set_error(e.what());                                                  \
        return VFD_EINVAL;                                                         \
    }

namespace {

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void require_device()
{
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        throw vfd::Error{VFD_ECUDA, "no CUDA device available (this library has no CPU path)"};
    }
}

// upload a field descriptor; Fourier rows become (k, amp cos(phase), amp sin(phase))
void upload_field(const vfd_field *f, int n_vert, DBuf<double> &rows, DBuf<double> &vals, DBuf<int> &gint,
                  DField &out)
{
    VFD_REQUIRE(f, VFD_EINVAL, "null field");
    out = DField{};
    out.c0 = f->c0;
    out.squash = f->squash;
    out.lo = f->lo;
    out.hi = f->hi;
    if (f->kind == VFD_FIELD_NODAL) {
        VFD_REQUIRE(f->nodal, VFD_EINVAL, "nodal field without values");
        out.nodal = 1;
        vals.alloc(n_vert);
        VFD_CUDA(cudaMemcpy(vals.p, f->nodal, sizeof(double) * n_vert, cudaMemcpyDefault));
        out.vals = vals.p;
        rows.alloc(0);
        return;
    }
    VFD_REQUIRE(f->kind == VFD_FIELD_ANALYTIC, VFD_EINVAL, "unknown field kind");
    VFD_REQUIRE(f->n_fourier >= 0 && f->n_gauss >= 0 && f->n_tbump >= 0, VFD_EINVAL, "negative term count");
    VFD_REQUIRE((f->n_fourier == 0 || f->fourier) && (f->n_gauss == 0 || f->gauss) && (f->n_tbump == 0 || f->tbump),
                VFD_EINVAL, "missing field rows");
    std::vector<double> h;
    int kmax = 0;
    // Fourier rows sorted by k_1 (stable): the device sums rows of equal k_1 together
    std::vector<int> order(f->n_fourier);
    for (int t = 0; t < f->n_fourier; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return f->fourier[5 * a] < f->fourier[5 * b]; });
    for (int t : order) {
        const double *r = f->fourier + 5 * t;
        for (int j = 0; j < 3; ++j) {
            if (r[j] != std::floor(r[j])) kmax = 99;           // non-integer: general path
            kmax = std::max(kmax, (int)std::min(99.0, std::fabs(r[j])));
            h.push_back(r[j]);
        }
        h.push_back(r[3] * std::cos(r[4]));
        h.push_back(r[3] * std::sin(r[4]));
    }
    for (int t = 0; t < 5 * f->n_gauss; ++t) h.push_back(f->gauss[t]);
    for (int t = 0; t < 5 * f->n_tbump; ++t) h.push_back(f->tbump[t]);
    // grouped form of 2D rows (integer |k| <= 4, k_3 = 0): group k_1 (signed)
    // holds rows A = amp e^{i phase}; with t = cos(pi|k_2|x_2) + i sign(k_2) sin(..)
    // and e_1 likewise, Re(e_1 sum A t) = c_1 gr + s_1 gq, gr = a0 c_2 + a1 s_2,
    // gq = a2 s_2 + a3 c_2 (the signs folded into a0..a3)
    bool grouped = f->n_fourier > 0;
    for (int t = 0; t < f->n_fourier && grouped; ++t) {
        const double *r = f->fourier + 5 * t;
        for (int j = 0; j < 3; ++j)
            if (r[j] != std::floor(r[j]) || std::fabs(r[j]) > 4.0) grouped = false;
        if (r[2] != 0.0) grouped = false;
    }
    std::vector<int> gi;
    size_t coef_off = h.size();
    int ngrp = 0;
    if (grouped) {
        std::vector<int> mk;
        size_t t0 = 0;
        while (t0 < order.size()) {
            const double k1 = f->fourier[5 * order[t0]];
            size_t t1 = t0;
            while (t1 < order.size() && f->fourier[5 * order[t1]] == k1) ++t1;
            gi.push_back((int)std::fabs(k1));
            gi.push_back((int)(t1 - t0));
            const double s1 = k1 < 0 ? -1.0 : 1.0;
            for (size_t q = t0; q < t1; ++q) {
                const double *r = f->fourier + 5 * order[q];
                const double ar = r[3] * std::cos(r[4]), ai = r[3] * std::sin(r[4]), s2 = r[1] < 0 ? -1.0 : 1.0;
                mk.push_back((int)std::fabs(r[1]));
                h.push_back(ar);
                h.push_back(-ai * s2);
                h.push_back(-s1 * s2 * ar);
                h.push_back(-s1 * ai);
            }
            ++ngrp;
            t0 = t1;
        }
        gi.insert(gi.end(), mk.begin(), mk.end());
    }
    rows.upload(h);
    gint.upload(gi);
    out.nF = f->n_fourier;
    out.nG = f->n_gauss;
    out.nT = f->n_tbump;
    out.kmax = kmax;
    out.rows = rows.p;
    out.ngrp = ngrp;
    out.gint = ngrp ? gint.p : nullptr;
    out.gcoef = ngrp ? rows.p + coef_off : nullptr;
}

bool field_is_const(const vfd_field *f)
{
    return f->kind == VFD_FIELD_ANALYTIC && f->n_fourier == 0 && f->n_gauss == 0 && f->n_tbump == 0 && !f->squash;
}

// stage a possibly-host input block into device memory
const double *stage_in(const double *X, int64_t n, int64_t nrhs, int64_t ld, DBuf<double> &buf, cudaStream_t st)
{
    if (is_device_ptr(X)) return X;
    size_t need = (size_t)ld * nrhs;
    if (buf.n < need) buf.alloc(need);
    VFD_CUDA(cudaMemcpyAsync(buf.p, X, sizeof(double) * ((size_t)ld * (nrhs - 1) + n), cudaMemcpyHostToDevice, st));
    return buf.p;
}

}  // namespace

extern "C" {

void vfd_default_mesh_opts(vfd_mesh_opts *o)
{
    if (!o) return;
    o->leaf_m = 64;
    o->cheb_p = 4;
    o->lambda = 0.75;
    o->n_sing = 3;
    o->tail_mode = 0;
    o->tail_R = 1.1;
    o->rho_leaf_m = 64;
    o->rho_lambda = 0.75;
    o->inner_p = 0;
    o->recompress_tol = 0.0;
}

const char *vfd_last_error(void) { return vfd::g_err.c_str(); }

vfd_status vfd_mesh(int d, int64_t n_vert, const double *coords, int64_t n_cell, const int32_t *cells,
                    const uint8_t *cell_is_interior, const vfd_mesh_opts *opts, vfd_mesh_t *out)
{
    VFD_API_BEGIN
    VFD_REQUIRE(out && coords && cells && cell_is_interior, VFD_EINVAL, "null argument");
    *out = nullptr;
    require_device();
    vfd_mesh_opts o;
    vfd_default_mesh_opts(&o);
    if (opts) o = *opts;
    MeshData *m = build_mesh(d, n_vert, coords, n_cell, cells, cell_is_interior, o);
    *out = new vfd_mesh_s{m};
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_mesh_dofs(vfd_mesh_t mesh, int32_t *dof_of_vertex, int64_t *n_dof)
{
    VFD_API_BEGIN
    VFD_REQUIRE(mesh, VFD_EINVAL, "null mesh");
    if (dof_of_vertex) std::memcpy(dof_of_vertex, mesh->m->dof_of_vertex.data(), sizeof(int32_t) * mesh->m->M);
    if (n_dof) *n_dof = mesh->m->N;
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_mesh_info(vfd_mesh_t mesh, int64_t *info, int n_info)
{
    VFD_API_BEGIN
    VFD_REQUIRE(mesh && info && n_info >= 0, VFD_EINVAL, "bad argument");
    const MeshData &m = *mesh->m;
    int64_t v[19] = {m.N,    m.M,     m.C,      m.npairs, m.nnz,   m.kt.L,      m.kt.nnode,  m.k,
                     m.nfar, m.nnear, m.near_entries_alg, m.nQ, m.nQint, m.nrfar, m.rnear_pairs, m.near_entries,
                     m.near_point_pairs, m.sing_points, m.k_in ? m.k_in : m.k};
    for (int i = 0; i < n_info && i < 19; ++i) info[i] = v[i];
    for (int i = 19; i < n_info; ++i) info[i] = 0;
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_assemble(vfd_mesh_t mesh, const vfd_field *s, const vfd_field *log_kappa, double s_bar,
                        int precision, int flags, void *stream, vfd_op_t *out)
{
    OpData *op = nullptr;
    VFD_API_BEGIN
    VFD_REQUIRE(mesh && s && log_kappa && out, VFD_EINVAL, "null argument");
    *out = nullptr;
    require_device();
    MeshData &m = *mesh->m;
    cudaStream_t st = (cudaStream_t)stream;
    VFD_REQUIRE(precision == VFD_FP64 || precision == VFD_FP32 || precision == VFD_BF16, VFD_EINVAL,
                "unknown precision");
    VFD_REQUIRE(s_bar < 1.0 && ((flags & VFD_ASSEMBLE_UNCHECKED) || s_bar >= 0.0), VFD_EINVAL,
                "s_bar must satisfy 0 <= s_bar < 1");
    bool nodal = s->kind == VFD_FIELD_NODAL || log_kappa->kind == VFD_FIELD_NODAL;
    // P1 fields at Chebyshev nodes: the nearest-point rule (located once per mesh)
    if (nodal && (m.nfar > 0 || m.nrfar > 0)) locate_nodes(m);
    VFD_REQUIRE(m.opts.tail_mode == 0 || (field_is_const(s) && field_is_const(log_kappa)), VFD_EUNSUPPORTED,
                "the exterior tail needs constant s and kappa");
    op = new OpData();
    op->m = mesh->m;
    op->precision = precision;
    op->s_bar = s_bar;
    op->check_fields = !(flags & VFD_ASSEMBLE_UNCHECKED);
    upload_field(s, m.M, op->f_rows_s, op->f_vals_s, op->f_gint_s, op->fs);
    upload_field(log_kappa, m.M, op->f_rows_k, op->f_vals_k, op->f_gint_k, op->fk);
    op->errflag.alloc(2);
    op->errflag.zero(st);
    op->timed = (flags & VFD_ASSEMBLE_TIMED) != 0;
    cudaEvent_t ev[VFD_T_COUNT];
    int nev = 0;
    auto mark = [&]() {
        if (!op->timed) return;
        VFD_CUDA(cudaEventCreate(&ev[nev]));
        VFD_CUDA(cudaEventRecord(ev[nev], st));
        ++nev;
    };
    mark();
    // a2: field values; check 0 <= s <= s_bar at every evaluation point (Sec. 2, i:s)
    launch_field_points(m, *op, st);
    mark();
    int herr[2] = {0, 0};
    VFD_CUDA(cudaMemcpyAsync(herr, op->errflag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    VFD_CUDA(cudaStreamSynchronize(st));
    VFD_REQUIRE(herr[0] == 0, VFD_EINVAL, "s(x) outside [0, s_bar] at some evaluation point");
    // a3: coupling blocks (and their algebraic recompression, FP64 operators)
    launch_coupling_build(m, *op, st);
    if (m.opts.recompress_tol > 0.0) recompress_far(m, *op, m.opts.recompress_tol, st);
    mark();
    // a4: dense inadmissible leaves
    launch_near_build(m, *op, st);
    mark();
    // a6: density by the H^2 sweep + tail
    launch_density(m, *op, st);
    mark();
    // a5: singular near field
    {
        DBuf<double> Lbuf;
        launch_singular_B(m, *op, Lbuf, st);
        mark();
        launch_gather_B(m, *op, Lbuf, st);
        VFD_CUDA(cudaStreamSynchronize(st));
    }
    // a7: weighted mass (and B + M for the apply)
    launch_gather_M(m, *op, st);
    if (precision != VFD_FP64) {
        launch_convert_fp32(m, *op, st);
        launch_lowp_csr(m, *op, st);
    }
    mark();
    VFD_CUDA(cudaStreamSynchronize(st));
    if (op->timed) {
        // events: 0 start, 1 fields, 2 coupling, 3 near, 4 density, 5 singular, 6 gathers
        for (int i = 0; i + 1 < nev && i < 6; ++i) {
            float ms = 0.f;
            VFD_CUDA(cudaEventElapsedTime(&ms, ev[i], ev[i + 1]));
            op->phase_ms[i] = ms;
        }
        float tot = 0.f;
        VFD_CUDA(cudaEventElapsedTime(&tot, ev[0], ev[nev - 1]));
        op->phase_ms[VFD_T_TOTAL] = tot;
        for (int i = 0; i < nev; ++i) cudaEventDestroy(ev[i]);
    }
    *out = new vfd_op_s{op};
    return VFD_OK;
    }
    catch (const vfd::Error &e) {
        delete op;
        vfd::set_error(e.msg);
        return e.st;
    }
    catch (const std::bad_alloc &) {
        delete op;
        vfd::set_error("host allocation failed");
        return VFD_ENOMEM;
    }
}

static vfd_status apply_common(vfd_op_t h, int parts, const double *X, double *Y, int64_t nrhs, int64_t ld,
                               void *stream)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h && X && Y, VFD_EINVAL, "null argument");
    OpData &op = *h->op;
    const MeshData &m = *op.m;
    VFD_REQUIRE(nrhs >= 1 && nrhs <= 65535 && ld >= m.N, VFD_EINVAL, "bad nrhs or ld");
    VFD_REQUIRE((parts & ~VFD_PART_ALL) == 0, VFD_EINVAL, "bad parts mask");
    cudaStream_t st = (cudaStream_t)stream;
    const double *dx = stage_in(X, m.N, nrhs, ld, op.xin, st);
    bool ydev = is_device_ptr(Y);
    double *dy = Y;
    if (!ydev) {
        size_t need = (size_t)ld * nrhs;
        if (op.yout.n < need) op.yout.alloc(need);
        dy = op.yout.p;
    }
    if (parts == VFD_PART_ALL && op.precision != VFD_FP64 && nrhs % 64 == 0 && m.max_leaf_size <= 64)
        batch_apply_colmajor(*op_batch(op), &dx, &dy, &ld, (int)nrhs, st);   // batched tensor-core path
    else
        apply_parts(m, op, parts, dx, dy, (int)nrhs, ld, st);
    if (!ydev) {
        VFD_CUDA(cudaMemcpyAsync(Y, dy, sizeof(double) * ((size_t)ld * (nrhs - 1) + m.N), cudaMemcpyDeviceToHost, st));
        VFD_CUDA(cudaStreamSynchronize(st));
    }
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_apply(vfd_op_t op, const double *X, double *Y, int64_t nrhs, int64_t ld, void *stream)
{
    return apply_common(op, VFD_PART_ALL, X, Y, nrhs, ld, stream);
}

vfd_status vfd_apply_parts(vfd_op_t op, int parts, const double *X, double *Y, int64_t nrhs, int64_t ld,
                           void *stream)
{
    return apply_common(op, parts, X, Y, nrhs, ld, stream);
}

vfd_status vfd_apply_noalloc(vfd_op_t h, const double *X, double *Y, int64_t nrhs, int64_t ld, void *stream)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h && X && Y, VFD_EINVAL, "null argument");
    const OpData &op = *h->op;
    const MeshData &m = *op.m;
    VFD_REQUIRE(nrhs >= 1 && nrhs <= 65535 && ld >= m.N, VFD_EINVAL, "bad nrhs or ld");
    VFD_REQUIRE(is_device_ptr(X) && is_device_ptr(Y), VFD_EINVAL,
                "vfd_apply_noalloc: X and Y must be device pointers (host copies would need device buffers)");
    apply_noalloc(m, op, X, Y, (int)nrhs, ld, (cudaStream_t)stream);
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_solve(vfd_op_t h, const double *F, double *U, int64_t nrhs, int64_t ld, double rtol, int max_it,
                     int *iters, double *relres, void *stream)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h && F && U, VFD_EINVAL, "null argument");
    OpData &op = *h->op;
    const MeshData &m = *op.m;
    VFD_REQUIRE(nrhs >= 1 && ld >= m.N && rtol > 0.0 && max_it >= 0, VFD_EINVAL, "bad solver arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const double *df = stage_in(F, m.N, nrhs, ld, op.xin, st);
    bool udev = is_device_ptr(U);
    double *du = U;
    if (!udev) {
        size_t need = (size_t)ld * nrhs;
        if (op.yout.n < need) op.yout.alloc(need);
        du = op.yout.p;
        VFD_CUDA(cudaMemcpyAsync(du, U, sizeof(double) * ((size_t)ld * (nrhs - 1) + m.N), cudaMemcpyHostToDevice, st));
    }
    vfd_status rs = (nrhs > 1 && op.precision != VFD_FP64)
                        ? batch_solve(*op_batch(op), &df, &du, &ld, (int)nrhs, rtol, max_it, iters, relres, st)
                        : cg_solve(m, op, df, du, (int)nrhs, ld, rtol, max_it, iters, relres, st);
    if (!udev) {
        VFD_CUDA(cudaMemcpyAsync(U, du, sizeof(double) * ((size_t)ld * (nrhs - 1) + m.N), cudaMemcpyDeviceToHost, st));
    }
    VFD_CUDA(cudaStreamSynchronize(st));
    if (rs != VFD_OK) vfd::set_error("CG did not reach rtol within max_it");
    return rs;
    VFD_API_END
}

vfd_status vfd_precondition(vfd_op_t h, int kind, void *stream)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h, VFD_EINVAL, "null operator");
    require_device();
    precond_setup(*h->op->m, *h->op, kind, (cudaStream_t)stream);
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_load(vfd_mesh_t mesh, const double *f_nodal, double *F, void *stream)
{
    VFD_API_BEGIN
    VFD_REQUIRE(mesh && f_nodal && F, VFD_EINVAL, "null argument");
    require_device();
    const MeshData &m = *mesh->m;
    cudaStream_t st = (cudaStream_t)stream;
    DBuf<double> fin, fout;
    const double *df = f_nodal;
    if (!is_device_ptr(f_nodal)) {
        fin.alloc(m.M);
        VFD_CUDA(cudaMemcpyAsync(fin.p, f_nodal, sizeof(double) * m.M, cudaMemcpyHostToDevice, st));
        df = fin.p;
    }
    bool fdev = is_device_ptr(F);
    double *dF = F;
    if (!fdev) {
        fout.alloc(m.N);
        dF = fout.p;
    }
    launch_load(m, df, dF, st);
    if (!fdev) VFD_CUDA(cudaMemcpyAsync(F, dF, sizeof(double) * m.N, cudaMemcpyDeviceToHost, st));
    VFD_CUDA(cudaStreamSynchronize(st));
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_grad(vfd_op_t h, const double *U, const double *Lam, int64_t nrhs, int64_t ld, double *g_s,
                    double *g_logkappa, void *stream)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h && U && Lam && g_s && g_logkappa, VFD_EINVAL, "null argument");
    OpData &op = *h->op;
    MeshData &m = *op.m;
    VFD_REQUIRE(op.fs.nodal && op.fk.nodal, VFD_EUNSUPPORTED, "vfd_grad needs P1 (nodal) s and log kappa");
    VFD_REQUIRE(m.opts.tail_mode == 0, VFD_EUNSUPPORTED, "vfd_grad needs a bounded exterior (tail_mode 0)");
    VFD_REQUIRE(m.d <= 2, VFD_EUNSUPPORTED, "vfd_grad is built for d = 1, 2");
    VFD_REQUIRE(op.q_s.n == (size_t)m.nQ, VFD_EINVAL, "vfd_grad: operator without point fields");
    VFD_REQUIRE(nrhs >= 1 && ld >= m.N, VFD_EINVAL, "bad nrhs or ld");
    VFD_REQUIRE(is_device_ptr(U) && is_device_ptr(Lam) && is_device_ptr(g_s) && is_device_ptr(g_logkappa),
                VFD_EINVAL, "vfd_grad: U, Lam, g_s and g_logkappa must be device pointers");
    grad_adjoint(m, op, U, Lam, (int)nrhs, ld, g_s, g_logkappa, (cudaStream_t)stream);
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_op_rho(vfd_op_t h, double *rho, void *stream)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h && rho, VFD_EINVAL, "null argument");
    OpData &op = *h->op;
    cudaStream_t st = (cudaStream_t)stream;
    VFD_CUDA(cudaMemcpyAsync(rho, op.rho.p, sizeof(double) * op.m->nQint, cudaMemcpyDefault, st));
    VFD_CUDA(cudaStreamSynchronize(st));
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_selftest_math(vfd_mesh_t mesh, int which, int64_t n, const double *x, double *out, void *stream)
{
    VFD_API_BEGIN
    VFD_REQUIRE(mesh && x && out && n >= 0 && which >= 0 && which <= 3, VFD_EINVAL, "bad argument");
    VFD_REQUIRE(is_device_ptr(x) && is_device_ptr(out), VFD_EINVAL, "x and out must be device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    launch_selftest_math(*mesh->m, which, n, x, out, st);
    VFD_CUDA(cudaStreamSynchronize(st));
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_op_far_ranks(vfd_op_t h, int *ranks, int n, int *nlev)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h && nlev, VFD_EINVAL, "null argument");
    const OpData &op = *h->op;
    const MeshData &m = *op.m;
    const int nl = m.nfar > 0 ? m.kt.L - m.far_lmin + 1 : 0;
    *nlev = nl;
    for (int lv = 0; lv < nl && lv < n && ranks; ++lv) ranks[lv] = op.rc_on ? op.rc_kl[lv] : m.k;
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_op_timings(vfd_op_t h, double *ms, int n)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h && ms && n >= 0, VFD_EINVAL, "bad argument");
    VFD_REQUIRE(h->op->timed, VFD_EINVAL, "the operator was assembled without VFD_ASSEMBLE_TIMED");
    for (int i = 0; i < n && i < VFD_T_COUNT; ++i) ms[i] = h->op->phase_ms[i];
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_batch_create(const vfd_op_t *ops, int nops, vfd_batch_t *out)
{
    VFD_API_BEGIN
    VFD_REQUIRE(ops && out && nops >= 1, VFD_EINVAL, "null argument or empty batch");
    *out = nullptr;
    std::unique_ptr<BatchData> b(new BatchData());
    for (int i = 0; i < nops; ++i) {
        VFD_REQUIRE(ops[i], VFD_EINVAL, "null operator in the batch");
        OpData *op = ops[i]->op;
        VFD_REQUIRE(op->precision == VFD_FP32 || op->precision == VFD_BF16, VFD_EINVAL,
                    "a batch takes VFD_FP32 or VFD_BF16 operators");
        VFD_REQUIRE(op->precision == ops[0]->op->precision, VFD_EINVAL, "a batch takes operators of one precision");
        VFD_REQUIRE(op->m->max_leaf_size <= 64, VFD_EUNSUPPORTED, "a batch needs leaves of at most 64 DoFs");
        b->ops.push_back(op);
    }
    b->nmesh = nops;
    b->precision = ops[0]->op->precision;
    b->xoff.assign(1, 0);
    for (int i = 0; i < nops; ++i) b->xoff.push_back(b->xoff.back() + b->ops[i]->m->N);
    b->ntot = b->xoff.back();
    *out = new vfd_batch_s{b.release()};
    return VFD_OK;
    VFD_API_END
}

static void batch_args(vfd::BatchData &b, const double *const *X, double *const *Y, const int64_t *ld, int64_t nrhs)
{
    VFD_REQUIRE(X && Y && ld, VFD_EINVAL, "null argument");
    VFD_REQUIRE(nrhs >= 1 && nrhs <= 65535, VFD_EINVAL, "bad nrhs");
    for (int i = 0; i < b.nmesh; ++i) {
        VFD_REQUIRE(X[i] && Y[i] && ld[i] >= b.ops[i]->m->N, VFD_EINVAL, "bad block or leading dimension");
        VFD_REQUIRE(is_device_ptr(X[i]) && is_device_ptr(Y[i]), VFD_EINVAL, "batch blocks must be device pointers");
    }
}

vfd_status vfd_batch_apply(vfd_batch_t h, const double *const *X, double *const *Y, const int64_t *ld, int64_t nrhs,
                           void *stream)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h, VFD_EINVAL, "null batch");
    batch_args(*h->b, X, Y, ld, nrhs);
    VFD_REQUIRE(nrhs % 64 == 0, VFD_EINVAL, "vfd_batch_apply needs a multiple of 64 columns");
    batch_apply_colmajor(*h->b, X, Y, ld, (int)nrhs, (cudaStream_t)stream);
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_batch_solve(vfd_batch_t h, const double *const *F, double *const *U, const int64_t *ld, int64_t nrhs,
                           double rtol, int max_it, int *iters, double *relres, void *stream)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h, VFD_EINVAL, "null batch");
    batch_args(*h->b, F, U, ld, nrhs);
    VFD_REQUIRE(rtol > 0.0 && max_it >= 0, VFD_EINVAL, "bad solver arguments");
    vfd_status rs = batch_solve(*h->b, F, U, ld, (int)nrhs, rtol, max_it, iters, relres, (cudaStream_t)stream);
    if (rs != VFD_OK) vfd::set_error("batched refinement did not reach rtol within max_it");
    return rs;
    VFD_API_END
}

vfd_status vfd_batch_tuning(vfd_batch_t h, int *chosen, float *us, int n, int *ncand)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h && chosen && (us || n == 0), VFD_EINVAL, "null argument");
    const int c = batch_tuning(*h->b, chosen, us, n);
    if (ncand) *ncand = c;
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_batch_set_config(vfd_batch_t h, int cfg, int *ncand)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h, VFD_EINVAL, "null batch");
    const int n = batch_set_config(*h->b, cfg);
    if (ncand) *ncand = n;
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_batch_set_wait_limit(vfd_batch_t h, double seconds)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h, VFD_EINVAL, "null batch");
    VFD_REQUIRE(std::isfinite(seconds) && seconds >= 0.0 && seconds < 3600.0, VFD_EINVAL,
                "the wait limit must be in [0, 3600) seconds");
    h->b->wait_ns = (long long)(seconds * 1e9);
    return VFD_OK;
    VFD_API_END
}

vfd_status vfd_batch_set_update_drop(vfd_batch_t h, double drop)
{
    VFD_API_BEGIN
    VFD_REQUIRE(h, VFD_EINVAL, "null batch");
    VFD_REQUIRE(std::isfinite(drop) && drop > 0.0 && drop < 1.0, VFD_EINVAL, "the update drop must be in (0, 1)");
    h->b->ru_drop = drop;
    return VFD_OK;
    VFD_API_END
}

void vfd_batch_free(vfd_batch_t h)
{
    if (!h) return;
    delete h->b;
    delete h;
}

void vfd_free_op(vfd_op_t h)
{
    if (!h) return;
    release_graphs(*h->op);
    delete h->op->self;
    h->op->self = nullptr;
    release_streams(*h->op);
    delete h->op;
    delete h;
}

void vfd_free_mesh(vfd_mesh_t h)
{
    if (!h) return;
    delete h->m;
    delete h;
}

}  // extern "C"
