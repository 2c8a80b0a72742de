// Host-side, geometry-only setup of the mesh handle (built once per mesh):
// interior DoFs (Sec. 2.3), touching element pairs and their type (Sec. 4),
// the element quadrature cloud (Sec. 6.1), the B/M sparsity with
// deterministic gather lists, the KD cluster trees with support-extended
// boxes, the admissible / inadmissible block lists, leaf bases and transfer
// matrices of the interpolation H^2 matrix (Sec. 5), and the point trees,
// lists and source moments of the density sweep (Sec. 6.2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>
#include <vector>

#include "vfd_internal.h"

namespace vfd {

void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w)
{
    // Golub-Welsch form of the rule: the nodes on [-1,1] are the eigenvalues of
    // the symmetric tridiagonal Jacobi matrix of the Legendre recurrence (zero
    // diagonal, off-diagonal b_k = k / sqrt(4k^2 - 1)), found one by one by
    // bisection on the Sturm count (number of negative pivots of J - t I); the
    // weights are the Christoffel numbers 1 / sum_{k<n} q_k(t)^2 with q_k the
    // Legendre polynomials orthonormal on [-1,1].  Mapped to [0,1] at the end.
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    std::vector<double> b2(n, 0.0);
    for (int k = 1; k < n; ++k) b2[k] = (double)k * k / (4.0 * k * k - 1.0);
    auto below = [&](double t) {   // eigenvalues of J smaller than t
        int cnt = 0;
        double q = -t;
        for (int k = 0; k < n; ++k) {
            if (k > 0) q = -t - b2[k] / q;
            if (q == 0.0) q = -1e-300;   // a zero pivot counts as negative (t just above it)
            if (q < 0.0) ++cnt;
        }
        return cnt;
    };
    for (int i = 0; i < n; ++i) {
        double lo = -1.0, hi = 1.0;   // the spectrum lies inside (-1, 1)
        for (int it = 0; it < 200; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (below(mid) > i) hi = mid;
            else lo = mid;
        }
        const double t = 0.5 * (lo + hi);
        double qm = 0.0, q = std::sqrt(0.5), s = 0.5;
        for (int k = 0; k + 1 < n; ++k) {
            const double bk1 = std::sqrt(b2[k + 1]);
            const double qn = (t * q - (k > 0 ? std::sqrt(b2[k]) * qm : 0.0)) / bk1;
            qm = q;
            q = qn;
            s += q * q;
        }
        x[i] = 0.5 * (1.0 + t);
        w[i] = 0.5 / s;
    }
}

std::vector<double> make_math_tables()
{
    // tables of the table-driven log/exp (layout in device_common.cuh),
    // computed with the host C library in extended precision
    std::vector<double> t(582, 0.0);
    for (int j = 0; j <= 128; ++j) {
        double c = 1.0 / (1.0 + j / 128.0);
        t[j] = c;
        t[129 + j] = (double)(-std::log((long double)c));
    }
    for (int j = 0; j < 64; ++j) t[258 + j] = (double)std::exp2((long double)j / 64.0L);
    const long double ln2 = std::log(2.0L);
    double hi = (double)ln2;
    long long b;
    std::memcpy(&b, &hi, 8);
    b &= ~((1LL << 28) - 1);   // 25 significant bits: e*hi and k*hi/64 are exact
    std::memcpy(&hi, &b, 8);
    double lo = (double)(ln2 - (long double)hi);
    t[322] = hi;
    t[323] = lo;
    t[324] = hi / 64.0;
    t[325] = lo / 64.0;
    // cos and sin of pi j / 64, j = 0..127 (the table-driven sin/cos of pi x)
    const long double pi = std::acos(-1.0L);
    for (int j = 0; j < 128; ++j) {
        t[326 + j] = (double)std::cos(pi * j / 64.0L);
        t[454 + j] = (double)std::sin(pi * j / 64.0L);
    }
    return t;
}

void cheb_nodes_1d(int p, double lo, double hi, double *out)
{
    // first-kind Chebyshev points of [lo, hi] (Sec. 5.3; reading: Chebyshev,
    // not the Legendre basis named in Sec. 7)
    double c = 0.5 * (lo + hi), h = 0.5 * (hi - lo);
    for (int i = 0; i < p; ++i) out[i] = c + h * std::cos((2.0 * i + 1.0) * M_PI / (2.0 * p));
}

namespace {

// tensor Lagrange basis on a box: values l_alpha(x), alpha = a0 + p*a1 (+p^2 a2)
void lagrange_box(int d, int p, const double *lo, const double *hi, const double *x, double *out)
{
    double nodes[PMAX], l1[3][PMAX];
    for (int i = 0; i < d; ++i) {
        cheb_nodes_1d(p, lo[i], hi[i], nodes);
        for (int a = 0; a < p; ++a) {
            double v = 1.0;
            for (int b = 0; b < p; ++b)
                if (b != a) v *= (x[i] - nodes[b]) / (nodes[a] - nodes[b]);
            l1[i][a] = v;
        }
    }
    int k = 1;
    for (int i = 0; i < d; ++i) k *= p;
    for (int al = 0; al < k; ++al) {
        int r = al;
        double v = 1.0;
        for (int i = 0; i < d; ++i) {
            v *= l1[i][r % p];
            r /= p;
        }
        out[al] = v;
    }
}

void cheb_box(int d, int p, const double *lo, const double *hi, double *pts /* k*d */)
{
    double nodes[3][PMAX];
    for (int i = 0; i < d; ++i) cheb_nodes_1d(p, lo[i], hi[i], nodes[i]);
    int k = 1;
    for (int i = 0; i < d; ++i) k *= p;
    for (int al = 0; al < k; ++al) {
        int r = al;
        for (int i = 0; i < d; ++i) {
            pts[al * d + i] = nodes[i][r % p];
            r /= p;
        }
    }
}

// complete binary KD tree: median splits along the longest box side (Sec. 5.1)
Tree build_kdtree(int d, const std::vector<double> &P /* n*d */, int n, int leaf_m)
{
    Tree t;
    int L = 0;
    while (n > leaf_m * (1 << L)) ++L;
    t.L = L;
    t.nnode = (1 << (L + 1)) - 1;
    t.nleaf = 1 << L;
    t.begin.assign(t.nnode, 0);
    t.end.assign(t.nnode, 0);
    t.perm.resize(n);
    std::iota(t.perm.begin(), t.perm.end(), 0);
    t.lo.assign((size_t)t.nnode * d, 0.0);
    t.hi.assign((size_t)t.nnode * d, 0.0);
    t.begin[0] = 0;
    t.end[0] = n;
    for (int node = 0; node < t.nnode; ++node) {
        int b = t.begin[node], e = t.end[node];
        double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
        for (int i = b; i < e; ++i)
            for (int c = 0; c < d; ++c) {
                double v = P[(size_t)t.perm[i] * d + c];
                lo[c] = std::min(lo[c], v);
                hi[c] = std::max(hi[c], v);
            }
        for (int c = 0; c < d; ++c) {
            t.lo[(size_t)node * d + c] = (e > b) ? lo[c] : 0.0;
            t.hi[(size_t)node * d + c] = (e > b) ? hi[c] : 0.0;
        }
        if (t.is_leaf(node)) continue;
        int dim = 0;
        for (int c = 1; c < d; ++c)
            if (hi[c] - lo[c] > hi[dim] - lo[dim]) dim = c;
        std::sort(t.perm.begin() + b, t.perm.begin() + e, [&](int u, int v) {
            double a = P[(size_t)u * d + dim], bb = P[(size_t)v * d + dim];
            return a < bb || (a == bb && u < v);
        });
        int mid = b + (e - b) / 2;
        t.begin[2 * node + 1] = b;
        t.end[2 * node + 1] = mid;
        t.begin[2 * node + 2] = mid;
        t.end[2 * node + 2] = e;
    }
    return t;
}

double box_diam(int d, const double *lo, const double *hi)
{
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += (hi[i] - lo[i]) * (hi[i] - lo[i]);
    return std::sqrt(s);
}

double box_dist(int d, const double *alo, const double *ahi, const double *blo, const double *bhi)
{
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        double g = std::max(0.0, std::max(alo[i] - bhi[i], blo[i] - ahi[i]));
        s += g * g;
    }
    return std::sqrt(s);
}

// admissibility as used in the paper's experiments (Sec. 7):
// lambda ||C - C'|| >= (D + D')/2, with strictly separated boxes
bool admissible(int d, double lambda, const double *alo, const double *ahi, const double *blo, const double *bhi,
                double min_dist)
{
    if (lambda <= 0.0) return false;
    double cc = 0.0;
    for (int i = 0; i < d; ++i) {
        double c = 0.5 * (alo[i] + ahi[i]) - 0.5 * (blo[i] + bhi[i]);
        cc += c * c;
    }
    double D = box_diam(d, alo, ahi), Dp = box_diam(d, blo, bhi);
    if (lambda * std::sqrt(cc) < 0.5 * (D + Dp)) return false;
    return box_dist(d, alo, ahi, blo, bhi) > min_dist;
}

void pad_boxes(Tree &t, int d)
{
    // keep Chebyshev nodes distinct on (nearly) flat boxes
    const double root = box_diam(d, &t.lo[0], &t.hi[0]);
    for (int n = 0; n < t.nnode; ++n) {
        double diam = box_diam(d, &t.lo[(size_t)n * d], &t.hi[(size_t)n * d]);
        for (int i = 0; i < d; ++i) {
            double w = t.hi[(size_t)n * d + i] - t.lo[(size_t)n * d + i];
            double need = 1e-9 * std::max(diam, 1e-6 * root);
            if (w < need) {
                t.lo[(size_t)n * d + i] -= 0.5 * need;
                t.hi[(size_t)n * d + i] += 0.5 * need;
            }
        }
    }
}

template <class T>
void csr_from_lists(const std::vector<std::vector<T>> &lists, std::vector<int> &ptr, std::vector<T> &val)
{
    ptr.assign(lists.size() + 1, 0);
    for (size_t i = 0; i < lists.size(); ++i) ptr[i + 1] = ptr[i] + (int)lists[i].size();
    val.clear();
    val.reserve(ptr.back());
    for (auto &l : lists) val.insert(val.end(), l.begin(), l.end());
}

}  // namespace

MeshData *build_mesh(int d, int64_t n_vert, const double *coords, int64_t n_cell, const int32_t *cells,
                     const uint8_t *inter, const vfd_mesh_opts &opts)
{
    VFD_REQUIRE(d >= 1 && d <= 3, VFD_EINVAL, "d must be 1, 2 or 3");
    VFD_REQUIRE(d < 3 || opts.tail_mode == 0, VFD_EUNSUPPORTED, "the exterior tail is built for d = 1, 2");
    VFD_REQUIRE(n_vert > 0 && n_cell > 0 && n_vert < (1LL << 30) && n_cell < (1LL << 28), VFD_EINVAL,
                "bad mesh size");
    VFD_REQUIRE(opts.leaf_m >= 2 && opts.leaf_m <= 256, VFD_EINVAL, "leaf_m must be in [2,256]");
    VFD_REQUIRE(opts.rho_leaf_m >= 2 && opts.rho_leaf_m <= 1024, VFD_EINVAL, "rho_leaf_m must be in [2,1024]");
    VFD_REQUIRE(opts.cheb_p >= 1 && opts.cheb_p <= PMAX, VFD_EINVAL, "cheb_p must be in [1,8]");
    VFD_REQUIRE(opts.n_sing >= 1 && opts.n_sing <= NSMAX, VFD_EINVAL, "n_sing must be in [1,16]");
    VFD_REQUIRE(opts.lambda >= 0.0 && opts.rho_lambda >= 0.0, VFD_EINVAL, "lambda must be >= 0");
    VFD_REQUIRE(opts.tail_mode == 0 || (opts.tail_mode == 1 && opts.tail_R > 0.0), VFD_EINVAL, "bad tail options");
    int kk = 1;
    for (int i = 0; i < d; ++i) kk *= opts.cheb_p;
    VFD_REQUIRE(kk <= KMAX, VFD_EINVAL, "rank p^d too large");
    VFD_REQUIRE(opts.inner_p >= 0 && opts.inner_p <= opts.cheb_p, VFD_EINVAL, "inner_p must be in [0, cheb_p]");
    VFD_REQUIRE(opts.recompress_tol >= 0.0 && opts.recompress_tol < 1.0, VFD_EINVAL,
                "recompress_tol must be in [0, 1)");

    auto *m = new MeshData();
    try {
        m->d = d;
        m->M = (int)n_vert;
        m->C = (int)n_cell;
        m->opts = opts;
        m->p = opts.cheb_p;
        m->k = kk;
        const int nv = d + 1, M = m->M, C = m->C;
        m->X.assign(coords, coords + (size_t)M * d);
        m->T.assign(cells, cells + (size_t)C * nv);
        m->inter.assign(inter, inter + C);
        for (int i = 0; i < C * nv; ++i)
            VFD_REQUIRE(m->T[i] >= 0 && m->T[i] < M, VFD_EINVAL, "cell vertex id out of range");

        // ---- cell measures, h_max
        std::vector<double> meas(C);
        for (int c = 0; c < C; ++c) {
            const int *t = &m->T[(size_t)c * nv];
            double mu, diam = 0.0;
            if (d == 1) {
                mu = std::fabs(m->X[t[1]] - m->X[t[0]]);
                diam = mu;
            } else if (d == 3) {
                const double *a = &m->X[3 * t[0]];
                double e[3][3];
                for (int u = 0; u < 3; ++u)
                    for (int c = 0; c < 3; ++c) e[u][c] = m->X[3 * t[u + 1] + c] - a[c];
                mu = std::fabs(e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                               e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                               e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0])) / 6.0;
                for (int u = 0; u < 4; ++u)
                    for (int v = u + 1; v < 4; ++v) {
                        double s2 = 0.0;
                        for (int c = 0; c < 3; ++c) s2 += (m->X[3 * t[u] + c] - m->X[3 * t[v] + c]) * (m->X[3 * t[u] + c] - m->X[3 * t[v] + c]);
                        diam = std::max(diam, std::sqrt(s2));
                    }
            } else {
                const double *a = &m->X[2 * t[0]], *b = &m->X[2 * t[1]], *e = &m->X[2 * t[2]];
                mu = 0.5 * std::fabs((b[0] - a[0]) * (e[1] - a[1]) - (b[1] - a[1]) * (e[0] - a[0]));
                for (int u = 0; u < 3; ++u)
                    for (int v = u + 1; v < 3; ++v) {
                        double dx = m->X[2 * t[u]] - m->X[2 * t[v]], dy = m->X[2 * t[u] + 1] - m->X[2 * t[v] + 1];
                        diam = std::max(diam, std::sqrt(dx * dx + dy * dy));
                    }
            }
            VFD_REQUIRE(mu > 0.0, VFD_EINVAL, "degenerate cell " + std::to_string(c));
            meas[c] = mu;
            m->h_max = std::max(m->h_max, diam);
        }

        // ---- DoFs: vertices of no exterior cell (Sec. 2.3)
        std::vector<char> used(M, 0), ext(M, 0);
        for (int c = 0; c < C; ++c)
            for (int a = 0; a < nv; ++a) {
                used[m->T[(size_t)c * nv + a]] = 1;
                if (!m->inter[c]) ext[m->T[(size_t)c * nv + a]] = 1;
            }
        std::vector<int> dofv;
        for (int v = 0; v < M; ++v)
            if (used[v] && !ext[v]) dofv.push_back(v);
        m->N = (int)dofv.size();
        VFD_REQUIRE(m->N > 0, VFD_EINVAL, "mesh has no interior DoF");
        const int N = m->N;

        // ---- K cluster tree on the DoF positions; DoF numbering = tree order
        {
            std::vector<double> P((size_t)N * d);
            for (int i = 0; i < N; ++i)
                for (int c = 0; c < d; ++c) P[(size_t)i * d + c] = m->X[(size_t)dofv[i] * d + c];
            m->kt = build_kdtree(d, P, N, opts.leaf_m);
            m->vertex_of_dof.resize(N);
            m->dof_of_vertex.assign(M, -1);
            for (int i = 0; i < N; ++i) {
                int v = dofv[m->kt.perm[i]];
                m->vertex_of_dof[i] = v;
                m->dof_of_vertex[v] = i;
            }
        }

        // ---- vertex -> cells
        std::vector<int> vc_ptr(M + 1, 0), vc;
        for (int c = 0; c < C; ++c)
            for (int a = 0; a < nv; ++a) vc_ptr[m->T[(size_t)c * nv + a] + 1]++;
        for (int v = 0; v < M; ++v) vc_ptr[v + 1] += vc_ptr[v];
        vc.resize(vc_ptr[M]);
        {
            std::vector<int> fill(M, 0);
            for (int c = 0; c < C; ++c)
                for (int a = 0; a < nv; ++a) {
                    int v = m->T[(size_t)c * nv + a];
                    vc[vc_ptr[v] + fill[v]++] = c;
                }
        }

        // ---- quadrature cloud: interior cells first (increasing id), then exterior;
        // element rule R3: triangle points with barycentric weight 2/3 on vertex q,
        // interval 3-point Gauss (left to right from stored vertex 0).
        std::vector<int> cell_order;
        for (int c = 0; c < C; ++c)
            if (m->inter[c]) cell_order.push_back(c);
        int nint = (int)cell_order.size();
        for (int c = 0; c < C; ++c)
            if (!m->inter[c]) cell_order.push_back(c);
        std::vector<int> cell_slot(C);
        for (int i = 0; i < C; ++i) cell_slot[cell_order[i]] = i;
        double bq[NQMAX][QB] = {}, wq[NQMAX] = {};
        const int NQ = d == 3 ? 4 : 3;
        m->nqc = NQ;
        if (d == 3) {
            // symmetric 4-point degree-2 rule (reading R20): barycentric (a, b, b, b), weights |tau|/4
            const double a = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, b = (5.0 - std::sqrt(5.0)) / 20.0;
            for (int q = 0; q < 4; ++q) {
                for (int c = 0; c < 4; ++c) bq[q][c] = (c == q) ? a : b;
                wq[q] = 0.25;
            }
        } else if (d == 2) {
            for (int q = 0; q < 3; ++q) {
                for (int a = 0; a < 3; ++a) bq[q][a] = (a == q) ? 2.0 / 3.0 : 1.0 / 6.0;
                wq[q] = 1.0 / 3.0;
            }
        } else {
            double g = 0.5 * std::sqrt(0.6);
            double tt[3] = {0.5 - g, 0.5, 0.5 + g}, ww[3] = {5.0 / 18.0, 8.0 / 18.0, 5.0 / 18.0};
            for (int q = 0; q < 3; ++q) {
                bq[q][0] = 1.0 - tt[q];
                bq[q][1] = tt[q];
                bq[q][2] = 0.0;
                wq[q] = ww[q];
            }
        }
        m->nQ = C * NQ;
        m->nQint = nint * NQ;
        const int nQ = m->nQ;
        std::vector<double> qx((size_t)nQ * d), qw(nQ), qb((size_t)nQ * QB, 0.0);
        m->qcell_host.resize(nQ);
        for (int i = 0; i < C; ++i) {
            int c = cell_order[i];
            const int *t = &m->T[(size_t)c * nv];
            for (int q = 0; q < NQ; ++q) {
                int id = i * NQ + q;
                for (int dim = 0; dim < d; ++dim) {
                    double v = 0.0;
                    for (int a = 0; a < nv; ++a) v += bq[q][a] * m->X[(size_t)t[a] * d + dim];
                    qx[(size_t)dim * nQ + id] = v;
                }
                qw[id] = wq[q] * meas[c];
                m->qcell_host[id] = c;
                for (int a = 0; a < QB; ++a) qb[(size_t)id * QB + a] = bq[q][a];
            }
        }
        auto qpos = [&](int id, int dim) { return qx[(size_t)dim * nQ + id]; };

        // ---- touching unordered pairs with >= 1 interior cell (canonical orientation R1')
        struct Pair {
            int type, w, pv[3], qv[3], loc[5], nl;
        };
        std::vector<Pair> pairs;
        {
            std::vector<int> mark(C, -1);
            for (int c = 0; c < C; ++c) {
                const int *t = &m->T[(size_t)c * nv];
                std::vector<int> nb;
                for (int a = 0; a < nv; ++a)
                    for (int k2 = vc_ptr[t[a]]; k2 < vc_ptr[t[a] + 1]; ++k2) {
                        int c2 = vc[k2];
                        if (mark[c2] != c) {
                            mark[c2] = c;
                            nb.push_back(c2);
                        }
                    }
                std::sort(nb.begin(), nb.end());
                for (int c2 : nb) {
                    if (c2 < c) continue;
                    if (!m->inter[c] && !m->inter[c2]) continue;
                    // tetrahedra: no singular rules (B = 0, reading R20); only the
                    // cells themselves, for the sparsity of the weighted mass matrix
                    if (d == 3 && c2 != c) continue;
                    int first = c, second = c2;
                    if (c != c2 && m->inter[c] != m->inter[c2]) {
                        first = m->inter[c] ? c : c2;
                        second = m->inter[c] ? c2 : c;
                    }
                    const int *u1 = &m->T[(size_t)first * nv], *u2 = &m->T[(size_t)second * nv];
                    Pair pr{};
                    pr.w = (first == second) ? 1 : 2;
                    for (int a = 0; a < 3; ++a) pr.pv[a] = pr.qv[a] = -1;
                    if (first == second) {
                        pr.type = 3;
                        for (int a = 0; a < std::min(nv, 3); ++a) pr.pv[a] = pr.qv[a] = u1[a];
                    } else {
                        int shared[3], ns = 0;
                        for (int a = 0; a < nv; ++a)
                            for (int b = 0; b < nv; ++b)
                                if (u1[a] == u2[b]) shared[ns++] = u1[a];
                        if (ns == 1) {
                            pr.type = 1;
                            int k1 = 1, k3 = 1;
                            pr.pv[0] = pr.qv[0] = shared[0];
                            for (int a = 0; a < nv; ++a) {
                                if (u1[a] != shared[0]) pr.pv[k1++] = u1[a];
                                if (u2[a] != shared[0]) pr.qv[k3++] = u2[a];
                            }
                        } else {
                            VFD_REQUIRE(d == 2 && ns == 2, VFD_EINVAL, "non-conforming cells " + std::to_string(c));
                            pr.type = 2;
                            // shared edge in the first cell's order, apexes last
                            pr.pv[0] = shared[0];
                            pr.pv[1] = shared[1];
                            for (int a = 0; a < 3; ++a)
                                if (u1[a] != shared[0] && u1[a] != shared[1]) pr.pv[2] = u1[a];
                            pr.qv[0] = shared[0];
                            pr.qv[1] = shared[1];
                            for (int a = 0; a < 3; ++a)
                                if (u2[a] != shared[0] && u2[a] != shared[1]) pr.qv[2] = u2[a];
                        }
                    }
                    // local DoF list
                    if (d == 3) {
                        pr.nl = 4;
                        for (int a = 0; a < 4; ++a) pr.loc[a] = u1[a];
                    } else if (d == 2) {
                        if (pr.type == 3) { pr.nl = 3; for (int a = 0; a < 3; ++a) pr.loc[a] = pr.pv[a]; }
                        else if (pr.type == 2) { pr.nl = 4; pr.loc[0] = pr.pv[0]; pr.loc[1] = pr.pv[1]; pr.loc[2] = pr.pv[2]; pr.loc[3] = pr.qv[2]; }
                        else { pr.nl = 5; pr.loc[0] = pr.pv[0]; pr.loc[1] = pr.pv[1]; pr.loc[2] = pr.pv[2]; pr.loc[3] = pr.qv[1]; pr.loc[4] = pr.qv[2]; }
                    } else {
                        if (pr.type == 3) { pr.nl = 2; pr.loc[0] = pr.pv[0]; pr.loc[1] = pr.pv[1]; }
                        else { pr.nl = 3; pr.loc[0] = pr.pv[0]; pr.loc[1] = pr.pv[1]; pr.loc[2] = pr.qv[1]; }
                    }
                    pairs.push_back(pr);
                }
            }
        }
        m->npairs = (int)pairs.size();

        // ---- B/M sparsity over DoFs and deterministic gather lists
        std::vector<std::vector<int>> rows(N);
        for (auto &pr : pairs)
            for (int i = 0; i < pr.nl; ++i) {
                int di = m->dof_of_vertex[pr.loc[i]];
                if (di < 0) continue;
                for (int j = 0; j < pr.nl; ++j) {
                    int dj = m->dof_of_vertex[pr.loc[j]];
                    if (dj >= 0) rows[di].push_back(dj);
                }
            }
        std::vector<int> rowptr(N + 1, 0), colidx;
        for (int i = 0; i < N; ++i) {
            auto &r = rows[i];
            std::sort(r.begin(), r.end());
            r.erase(std::unique(r.begin(), r.end()), r.end());
            rowptr[i + 1] = rowptr[i] + (int)r.size();
        }
        colidx.reserve(rowptr[N]);
        for (auto &r : rows) colidx.insert(colidx.end(), r.begin(), r.end());
        m->nnz = rowptr[N];
        auto entry = [&](int i, int j) {
            auto b = colidx.begin() + rowptr[i], e = colidx.begin() + rowptr[i + 1];
            return (int)(std::lower_bound(b, e, j) - colidx.begin());
        };
        {
            std::vector<int> cnt(m->nnz + 1, 0);
            std::vector<std::pair<int, int>> cont;  // (entry, idx)
            for (int p = 0; p < m->npairs; ++p) {
                auto &pr = pairs[p];
                for (int i = 0; i < pr.nl; ++i) {
                    int di = m->dof_of_vertex[pr.loc[i]];
                    if (di < 0) continue;
                    for (int j = 0; j < pr.nl; ++j) {
                        int dj = m->dof_of_vertex[pr.loc[j]];
                        if (dj < 0) continue;
                        cont.push_back({entry(di, dj), p * 25 + i * 5 + j});
                    }
                }
            }
            std::stable_sort(cont.begin(), cont.end(),
                             [](const std::pair<int, int> &a, const std::pair<int, int> &b) { return a.first < b.first; });
            std::vector<int> ptr(m->nnz + 1, 0), idx(cont.size());
            for (size_t k2 = 0; k2 < cont.size(); ++k2) {
                ptr[cont[k2].first + 1]++;
                idx[k2] = cont[k2].second;
            }
            for (int e = 0; e < m->nnz; ++e) ptr[e + 1] += ptr[e];
            m->ncontribB = (int64_t)cont.size();
            m->cB_ptr.upload(ptr);
            m->cB_idx.upload(idx);
        }
        {
            // mass: entry(i,j) += 2 w_q lam_a(q) lam_b(q) rho(q) over interior cells (eq. e:m)
            struct MC {
                int e, q;
                double c;
            };
            std::vector<MC> cont;
            for (int i = 0; i < nint; ++i) {
                int c = cell_order[i];
                const int *t = &m->T[(size_t)c * nv];
                for (int a = 0; a < nv; ++a) {
                    int di = m->dof_of_vertex[t[a]];
                    if (di < 0) continue;
                    for (int b = 0; b < nv; ++b) {
                        int dj = m->dof_of_vertex[t[b]];
                        if (dj < 0) continue;
                        int e = entry(di, dj);
                        for (int q = 0; q < NQ; ++q) {
                            int id = i * NQ + q;
                            cont.push_back({e, id, 2.0 * qw[id] * qb[(size_t)id * QB + a] * qb[(size_t)id * QB + b]});
                        }
                    }
                }
            }
            std::stable_sort(cont.begin(), cont.end(), [](const MC &a, const MC &b) { return a.e < b.e; });
            std::vector<int> ptr(m->nnz + 1, 0), qi(cont.size());
            std::vector<double> cf(cont.size());
            for (size_t k2 = 0; k2 < cont.size(); ++k2) {
                ptr[cont[k2].e + 1]++;
                qi[k2] = cont[k2].q;
                cf[k2] = cont[k2].c;
            }
            for (int e = 0; e < m->nnz; ++e) ptr[e + 1] += ptr[e];
            m->ncontribM = (int64_t)cont.size();
            m->cM_ptr.upload(ptr);
            m->cM_q.upload(qi);
            m->cM_coef.upload(cf);
        }
        m->rowptr.upload(rowptr);
        m->colidx.upload(colidx);
        {
            std::vector<int> pinfo((size_t)m->npairs * 8);
            for (int p = 0; p < m->npairs; ++p) {
                auto &pr = pairs[p];
                pinfo[(size_t)p * 8 + 0] = pr.type;
                pinfo[(size_t)p * 8 + 1] = pr.w;
                for (int a = 0; a < 3; ++a) {
                    pinfo[(size_t)p * 8 + 2 + a] = pr.pv[a];
                    pinfo[(size_t)p * 8 + 5 + a] = pr.qv[a];
                }
            }
            m->pair_info.upload(pinfo);
            m->pair_info_h = pinfo;
            if (d == 2) {   // regions per pair type: vertex 2, edge 5, identical 3; ns^4 points each
                const int64_t n4 = (int64_t)opts.n_sing * opts.n_sing * opts.n_sing * opts.n_sing;
                m->sing_points = 0;
                for (int p = 0; p < m->npairs; ++p) {
                    const int ty = pinfo[(size_t)p * 8];
                    m->sing_points += n4 * (ty == 1 ? 2 : ty == 2 ? 5 : 3);
                }
            }
        }

        // ---- K tree: support-extended boxes (Sec. 5.1, omega^e), Chebyshev nodes
        Tree &kt = m->kt;
        const int k = m->k, p = m->p, nnode = kt.nnode, nleaf = kt.nleaf, fl = kt.first_leaf();
        for (int lf = 0; lf < nleaf; ++lf) {
            int node = fl + lf;
            double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
            for (int i = kt.begin[node]; i < kt.end[node]; ++i) {
                int v = m->vertex_of_dof[i];
                for (int k2 = vc_ptr[v]; k2 < vc_ptr[v + 1]; ++k2) {
                    const int *t = &m->T[(size_t)vc[k2] * nv];
                    for (int a = 0; a < nv; ++a)
                        for (int c = 0; c < d; ++c) {
                            lo[c] = std::min(lo[c], m->X[(size_t)t[a] * d + c]);
                            hi[c] = std::max(hi[c], m->X[(size_t)t[a] * d + c]);
                        }
                }
            }
            for (int c = 0; c < d; ++c) {
                kt.lo[(size_t)node * d + c] = lo[c];
                kt.hi[(size_t)node * d + c] = hi[c];
            }
        }
        for (int node = fl - 1; node >= 0; --node)
            for (int c = 0; c < d; ++c) {
                kt.lo[(size_t)node * d + c] = std::min(kt.lo[(size_t)(2 * node + 1) * d + c], kt.lo[(size_t)(2 * node + 2) * d + c]);
                kt.hi[(size_t)node * d + c] = std::max(kt.hi[(size_t)(2 * node + 1) * d + c], kt.hi[(size_t)(2 * node + 2) * d + c]);
            }
        pad_boxes(kt, d);
        std::vector<double> kcheb((size_t)nnode * k * d);
        for (int n = 0; n < nnode; ++n) cheb_box(d, p, &kt.lo[(size_t)n * d], &kt.hi[(size_t)n * d], &kcheb[(size_t)n * k * d]);
        m->kt_cheb.upload(kcheb);
        m->kt_cheb_h = kcheb;
        m->kt_begin.upload(kt.begin);
        m->kt_end.upload(kt.end);

        // ---- dual traversal: admissible (far) and inadmissible leaf (near) pairs
        {
            std::vector<std::vector<int>> farl(nnode), nearl(nleaf);
            std::vector<std::pair<int, int>> stack{{0, 0}};
            while (!stack.empty()) {
                auto [a, b] = stack.back();
                stack.pop_back();
                const double *alo = &kt.lo[(size_t)a * d], *ahi = &kt.hi[(size_t)a * d];
                const double *blo = &kt.lo[(size_t)b * d], *bhi = &kt.hi[(size_t)b * d];
                if (admissible(d, opts.lambda, alo, ahi, blo, bhi, 0.0)) {
                    farl[a].push_back(b);
                } else if (kt.is_leaf(a)) {
                    nearl[a - fl].push_back(b - fl);
                } else {
                    for (int ca = 2 * a + 1; ca <= 2 * a + 2; ++ca)
                        for (int cb = 2 * b + 1; cb <= 2 * b + 2; ++cb) stack.push_back({ca, cb});
                }
            }
            for (auto &l : farl) std::sort(l.begin(), l.end());
            for (auto &l : nearl) std::sort(l.begin(), l.end());
            csr_from_lists(farl, m->far_ptr_h, m->far_col_h);
            csr_from_lists(nearl, m->near_ptr_h, m->near_col_h);
            m->nfar = (int)m->far_col_h.size();
            m->nnear = (int)m->near_col_h.size();
            // Near blocks of one row leaf form a row panel (row stride W_a = the
            // partners' column counts, padded to a multiple of 8), so that a row's
            // near entries are contiguous; block e starts at near_off[e].
            m->near_off_h.assign(m->nnear + 1, 0);
            std::vector<int> src(m->nnear, -1), prow(m->nnear), pw(nleaf, 0);
            std::vector<int64_t> poff(nleaf + 1, 0);
            m->near_entries_alg = 0;
            for (int a = 0; a < nleaf; ++a) {
                int na = kt.end[fl + a] - kt.begin[fl + a], w = 0;
                for (int e = m->near_ptr_h[a]; e < m->near_ptr_h[a + 1]; ++e) {
                    int b = m->near_col_h[e];
                    prow[e] = a;
                    int nb = kt.end[fl + b] - kt.begin[fl + b];
                    m->near_off_h[e] = poff[a] + w;
                    w += nb;
                    m->near_entries_alg += (int64_t)na * nb;
                    if (a > b) {
                        auto bb = m->near_col_h.begin() + m->near_ptr_h[b], ee = m->near_col_h.begin() + m->near_ptr_h[b + 1];
                        auto it = std::lower_bound(bb, ee, a);
                        VFD_REQUIRE(it != ee && *it == a, VFD_ECUDA, "near list not symmetric");
                        src[e] = (int)(it - m->near_col_h.begin());
                    }
                }
                w = (w + 7) & ~7;   // rows start on 16 bytes in FP64, FP32 and BF16
                pw[a] = w;
                m->max_panel_w = std::max(m->max_panel_w, w);
                poff[a + 1] = poff[a] + (int64_t)na * w;
            }
            m->near_entries = poff[nleaf];
            m->near_off_h[m->nnear] = m->near_entries;
            m->panel_w.upload(pw);
            m->panel_off.upload(poff);
            // flat gather index of every panel column: the DoF whose x it takes
            // (-1 for the padding); panel a's columns start at gcol_off[a]
            std::vector<int> gcol, goff(nleaf + 1, 0);
            for (int a = 0; a < nleaf; ++a) {
                goff[a] = (int)gcol.size();
                for (int e = m->near_ptr_h[a]; e < m->near_ptr_h[a + 1]; ++e) {
                    int b = m->near_col_h[e];
                    for (int j = kt.begin[fl + b]; j < kt.end[fl + b]; ++j) gcol.push_back(j);
                }
                while ((int)gcol.size() - goff[a] < pw[a]) gcol.push_back(-1);
            }
            goff[nleaf] = (int)gcol.size();
            m->gcol.upload(gcol);
            m->gcol_off.upload(goff);
            // panel position of every B + M entry (flat offset into the near
            // panels, -1 if its column is not among the row leaf's partners), for
            // the batched low-precision apply, which folds B + M into the panels.
            // Touching cells give overlapping support boxes, which are never
            // admissible for lambda < 1, so every entry has a position then.
            {
                std::vector<int> colpos(N, -1);
                std::vector<int64_t> bpos(m->nnz, -1);
                for (int a = 0; a < nleaf; ++a) {
                    const int W = pw[a];
                    for (int c = 0; c < W; ++c)
                        if (gcol[goff[a] + c] >= 0) colpos[gcol[goff[a] + c]] = c;
                    for (int i = kt.begin[fl + a]; i < kt.end[fl + a]; ++i)
                        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
                            const int c = colpos[colidx[e]];
                            if (c >= 0) bpos[e] = poff[a] + (int64_t)(i - kt.begin[fl + a]) * W + c;
                        }
                    for (int c = 0; c < W; ++c)
                        if (gcol[goff[a] + c] >= 0) colpos[gcol[goff[a] + c]] = -1;
                }
                m->bm_in_panels = std::all_of(bpos.begin(), bpos.end(), [](int64_t v) { return v >= 0; });
                m->bm_pos.upload(bpos);
            }
            std::vector<int> vl(N);
            for (int a = 0; a < nleaf; ++a)
                for (int j = kt.begin[fl + a]; j < kt.end[fl + a]; ++j) vl[j] = a;
            m->vleaf.upload(vl);
            m->far_ptr.upload(m->far_ptr_h);
            m->far_col.upload(m->far_col_h);
            m->near_ptr.upload(m->near_ptr_h);
            m->near_col.upload(m->near_col_h);
            m->near_off.upload(m->near_off_h);
            m->near_src.upload(src);
            m->near_pair_row.upload(prow);
        }

        // the far field of the low-precision inner operator may use a lower
        // interpolation order (inner_p); only with admissible blocks
        const int pin = (m->nfar > 0 && opts.inner_p > 0 && opts.inner_p != p) ? opts.inner_p : 0;
        int kin = 0;
        if (pin) {
            kin = 1;
            for (int i = 0; i < d; ++i) kin *= pin;
        }
        m->p_in = pin;
        m->k_in = kin;

        // ---- per-leaf point sets and DoF supports; leaf bases U (Sec. 5.3, R5)
        std::vector<double> Uh;   // N x k, tree order
        {
            std::vector<int> lp_ptr(nleaf + 1, 0), lp_pts;
            std::vector<std::vector<std::pair<int, double>>> supp(N);
            std::vector<double> U, Uin;
            std::vector<int> Uoff(nleaf);
            std::vector<int> mark(C, -1);
            std::vector<double> lag(KMAX);
            for (int lf = 0; lf < nleaf; ++lf) {
                int node = fl + lf;
                std::vector<int> lc;
                for (int i = kt.begin[node]; i < kt.end[node]; ++i) {
                    int v = m->vertex_of_dof[i];
                    for (int k2 = vc_ptr[v]; k2 < vc_ptr[v + 1]; ++k2)
                        if (mark[vc[k2]] != lf) {
                            mark[vc[k2]] = lf;
                            lc.push_back(vc[k2]);
                        }
                }
                std::sort(lc.begin(), lc.end());
                std::vector<int> cpos(lc.size());
                int base = (int)lp_pts.size();
                for (size_t j = 0; j < lc.size(); ++j)
                    for (int q = 0; q < NQ; ++q) lp_pts.push_back(cell_slot[lc[j]] * NQ + q);
                lp_ptr[lf + 1] = (int)lp_pts.size();
                m->max_leaf_pts = std::max(m->max_leaf_pts, lp_ptr[lf + 1] - lp_ptr[lf]);
                m->max_leaf_size = std::max(m->max_leaf_size, kt.end[node] - kt.begin[node]);
                Uoff[lf] = (int)U.size();
                for (int i = kt.begin[node]; i < kt.end[node]; ++i) {
                    int v = m->vertex_of_dof[i];
                    for (int k2 = vc_ptr[v]; k2 < vc_ptr[v + 1]; ++k2) {
                        int c = vc[k2];
                        int j = (int)(std::lower_bound(lc.begin(), lc.end(), c) - lc.begin());
                        const int *t = &m->T[(size_t)c * nv];
                        int a = 0;
                        while (t[a] != v) ++a;
                        for (int q = 0; q < NQ; ++q) {
                            int id = cell_slot[c] * NQ + q;
                            supp[i].push_back({j * NQ + q, qw[id] * qb[(size_t)id * QB + a]});
                        }
                    }
                    m->max_supp = std::max(m->max_supp, (int)supp[i].size());
                    // U_{i,alpha} = sum_{q in supp(i)} w_q psi_i(q) l_alpha(q)
                    std::vector<double> row(k, 0.0), row_in(kin, 0.0);
                    for (auto &sc : supp[i]) {
                        int id = lp_pts[base + sc.first];
                        double x[3];
                        for (int c = 0; c < d; ++c) x[c] = qpos(id, c);
                        lagrange_box(d, p, &kt.lo[(size_t)node * d], &kt.hi[(size_t)node * d], x, lag.data());
                        for (int al = 0; al < k; ++al) row[al] += sc.second * lag[al];
                        if (kin) {
                            lagrange_box(d, pin, &kt.lo[(size_t)node * d], &kt.hi[(size_t)node * d], x, lag.data());
                            for (int al = 0; al < kin; ++al) row_in[al] += sc.second * lag[al];
                        }
                    }
                    U.insert(U.end(), row.begin(), row.end());
                    Uin.insert(Uin.end(), row_in.begin(), row_in.end());
                }
            }
            std::vector<int> sp(N + 1, 0), sl;
            std::vector<double> sc;
            for (int i = 0; i < N; ++i) {
                sp[i + 1] = sp[i] + (int)supp[i].size();
                for (auto &e : supp[i]) {
                    sl.push_back(e.first);
                    sc.push_back(e.second);
                }
            }
            m->near_point_pairs = 0;
            for (int a = 0; a < nleaf; ++a)
                for (int e = m->near_ptr_h[a]; e < m->near_ptr_h[a + 1]; ++e) {
                    const int b = m->near_col_h[e];
                    if (a <= b)
                        m->near_point_pairs += (int64_t)(lp_ptr[a + 1] - lp_ptr[a]) * (lp_ptr[b + 1] - lp_ptr[b]);
                }
            m->lp_ptr.upload(lp_ptr);
            m->lp_pts.upload(lp_pts);
            m->lp_ptr_h = lp_ptr;
            m->lp_pts_h = lp_pts;
            m->supp_ptr.upload(sp);
            m->supp_loc.upload(sl);
            m->supp_coef.upload(sc);
            Uh = U;
            if (kin) m->U_in64.upload(Uin);
            m->kt_Uoff.upload(Uoff);
        }
        // transfers E_c[beta][alpha] = l^parent_alpha(xi^c_beta) (nested bases,
        // Sec. 5.3 last paragraph), and the per-level bases they generate:
        // Ul^(l)[i] = U[i] E_{c_L} ... E_{c_(l+1)} along the path from the leaf
        // of DoF i to its level-(l+1) ancestor, so that the basis of a node at
        // level l is the stack of its rows (used by the apply to avoid a
        // level-by-level transfer chain; stored for the levels with
        // admissible blocks only).
        {
            std::vector<double> E((size_t)nnode * k * k, 0.0), lag(k);
            for (int c = 1; c < nnode; ++c) {
                int par = (c - 1) / 2;
                for (int be = 0; be < k; ++be) {
                    lagrange_box(d, p, &kt.lo[(size_t)par * d], &kt.hi[(size_t)par * d], &kcheb[((size_t)c * k + be) * d], lag.data());
                    for (int al = 0; al < k; ++al) E[((size_t)c * k + be) * k + al] = lag[al];
                }
            }
            int lmin = kt.L + 1;
            for (int a = 0; a < nnode; ++a)
                if (m->far_ptr_h[a + 1] > m->far_ptr_h[a]) {
                    int lev = 0;
                    while ((2 << lev) - 1 <= a) ++lev;
                    lmin = std::min(lmin, lev);
                }
            m->far_lmin = lmin;
            const int nlev = (lmin <= kt.L) ? kt.L - lmin + 1 : 0;
            std::vector<double> Ul((size_t)nlev * N * k, 0.0);
            if (nlev) {
                for (size_t t = 0; t < (size_t)N * k; ++t) Ul[(size_t)(kt.L - lmin) * N * k + t] = Uh[t];
                for (int l = kt.L - 1; l >= lmin; --l)
                    for (int lf = 0; lf < nleaf; ++lf) {
                        int c = ((fl + lf + 1) >> (kt.L - (l + 1))) - 1;   // level-(l+1) ancestor
                        const double *Ec = &E[(size_t)c * k * k];
                        for (int i = kt.begin[fl + lf]; i < kt.end[fl + lf]; ++i) {
                            const double *src = &Ul[((size_t)(l + 1 - lmin) * N + i) * k];
                            double *dst = &Ul[((size_t)(l - lmin) * N + i) * k];
                            for (int al = 0; al < k; ++al) {
                                double v = 0.0;
                                for (int be = 0; be < k; ++be) v += src[be] * Ec[(size_t)be * k + al];
                                dst[al] = v;
                            }
                        }
                    }
            }
            m->Ul64.upload(Ul);
            if (m->nfar > 0) m->E64.upload(E);
            if (kin) {
                // the lower-order interpolation of the inner operator: its Chebyshev
                // nodes on the same boxes and its transfers
                std::vector<double> kcin((size_t)nnode * kin * d), Ein((size_t)nnode * kin * kin, 0.0), lg(KMAX);
                for (int n = 0; n < nnode; ++n)
                    cheb_box(d, pin, &kt.lo[(size_t)n * d], &kt.hi[(size_t)n * d], &kcin[(size_t)n * kin * d]);
                for (int c = 1; c < nnode; ++c) {
                    int par = (c - 1) / 2;
                    for (int be = 0; be < kin; ++be) {
                        lagrange_box(d, pin, &kt.lo[(size_t)par * d], &kt.hi[(size_t)par * d],
                                     &kcin[((size_t)c * kin + be) * d], lg.data());
                        for (int al = 0; al < kin; ++al) Ein[((size_t)c * kin + be) * kin + al] = lg[al];
                    }
                }
                m->kt_cheb_in.upload(kcin);
                m->kt_cheb_in_h = kcin;
                m->E_in64.upload(Ein);
            }
        }

        // ---- density sweep trees (Sec. 6.2): targets = interior points, sources = all points
        {
            std::vector<double> Pt((size_t)m->nQint * d), Ps((size_t)nQ * d);
            for (int i = 0; i < nQ; ++i)
                for (int c = 0; c < d; ++c) {
                    Ps[(size_t)i * d + c] = qpos(i, c);
                    if (i < m->nQint) Pt[(size_t)i * d + c] = qpos(i, c);
                }
            m->tt = build_kdtree(d, Pt, m->nQint, opts.rho_leaf_m);
            m->st = build_kdtree(d, Ps, nQ, opts.rho_leaf_m);
            pad_boxes(m->tt, d);
            pad_boxes(m->st, d);
            Tree &tt = m->tt, &st = m->st;
            std::vector<double> tch((size_t)tt.nnode * k * d), sch((size_t)st.nnode * k * d);
            for (int n = 0; n < tt.nnode; ++n) cheb_box(d, p, &tt.lo[(size_t)n * d], &tt.hi[(size_t)n * d], &tch[(size_t)n * k * d]);
            for (int n = 0; n < st.nnode; ++n) cheb_box(d, p, &st.lo[(size_t)n * d], &st.hi[(size_t)n * d], &sch[(size_t)n * k * d]);
            // source moments xhat_s[beta] = sum_{q in s} l_beta(q) w_q (geometry only)
            std::vector<double> xs((size_t)st.nnode * k, 0.0), lag(k);
            for (int n = 0; n < st.nnode; ++n)
                for (int i = st.begin[n]; i < st.end[n]; ++i) {
                    int id = st.perm[i];
                    double x[3];
                    for (int c = 0; c < d; ++c) x[c] = qpos(id, c);
                    lagrange_box(d, p, &st.lo[(size_t)n * d], &st.hi[(size_t)n * d], x, lag.data());
                    for (int b = 0; b < k; ++b) xs[(size_t)n * k + b] += lag[b] * qw[id];
                }
            // rectangular dual traversal
            std::vector<std::vector<int>> farl(tt.nnode), nearl(tt.nleaf);
            std::vector<std::pair<int, int>> stack{{0, 0}};
            const double mind = 2.0 * m->h_max;
            while (!stack.empty()) {
                auto [a, b] = stack.back();
                stack.pop_back();
                const double *alo = &tt.lo[(size_t)a * d], *ahi = &tt.hi[(size_t)a * d];
                const double *blo = &st.lo[(size_t)b * d], *bhi = &st.hi[(size_t)b * d];
                bool la = tt.is_leaf(a), lb = st.is_leaf(b);
                if (admissible(d, opts.rho_lambda, alo, ahi, blo, bhi, mind)) {
                    farl[a].push_back(b);
                } else if (la && lb) {
                    nearl[a - tt.first_leaf()].push_back(b);
                } else if (la) {
                    stack.push_back({a, 2 * b + 1});
                    stack.push_back({a, 2 * b + 2});
                } else if (lb) {
                    stack.push_back({2 * a + 1, b});
                    stack.push_back({2 * a + 2, b});
                } else {
                    for (int ca = 2 * a + 1; ca <= 2 * a + 2; ++ca)
                        for (int cb = 2 * b + 1; cb <= 2 * b + 2; ++cb) stack.push_back({ca, cb});
                }
            }
            for (auto &l : farl) std::sort(l.begin(), l.end());
            for (auto &l : nearl) std::sort(l.begin(), l.end());
            std::vector<int> fp, fc, np_, nc;
            csr_from_lists(farl, fp, fc);
            csr_from_lists(nearl, np_, nc);
            m->nrfar = (int)fc.size();
            m->nrnear = (int)nc.size();
            m->rnear_pairs = 0;
            for (int a = 0; a < tt.nleaf; ++a)
                for (int e = np_[a]; e < np_[a + 1]; ++e) {
                    int ta = tt.first_leaf() + a, sb = nc[e];
                    m->rnear_pairs += (int64_t)(tt.end[ta] - tt.begin[ta]) * (st.end[sb] - st.begin[sb]);
                }
            m->rfar_ptr.upload(fp);
            m->rfar_col.upload(fc);
            m->rnear_ptr.upload(np_);
            m->rnear_col.upload(nc);
            // transposed lists (by source node / source leaf) for the gradient's
            // source-side sums
            {
                std::vector<std::vector<int>> ft(st.nnode), nt(st.nleaf);
                for (int a = 0; a < tt.nnode; ++a)
                    for (int e = fp[a]; e < fp[a + 1]; ++e) ft[fc[e]].push_back(a);
                for (int a = 0; a < tt.nleaf; ++a)
                    for (int e = np_[a]; e < np_[a + 1]; ++e) nt[nc[e] - st.first_leaf()].push_back(a);
                std::vector<int> tp, tc, up, uc;
                csr_from_lists(ft, tp, tc);
                csr_from_lists(nt, up, uc);
                m->rfarT_ptr.upload(tp);
                m->rfarT_col.upload(tc);
                m->rnearT_ptr.upload(up);
                m->rnearT_col.upload(uc);
            }
            m->tt_begin.upload(tt.begin);
            m->tt_end.upload(tt.end);
            m->tt_perm.upload(tt.perm);
            m->st_begin.upload(st.begin);
            m->st_end.upload(st.end);
            m->st_perm.upload(st.perm);
            m->tt_lo.upload(tt.lo);
            m->tt_hi.upload(tt.hi);
            m->tt_cheb.upload(tch);
            m->st_cheb.upload(sch);
            m->tt_cheb_h = tch;
            m->st_cheb_h = sch;
            m->st_xhat.upload(xs);
        }

        // ---- load-vector gather lists: DoF -> (cell, local vertex) of interior cells
        {
            std::vector<std::vector<int>> l(N);
            for (int c = 0; c < C; ++c) {
                if (!m->inter[c]) continue;
                for (int a = 0; a < nv; ++a) {
                    int di = m->dof_of_vertex[m->T[(size_t)c * nv + a]];
                    if (di >= 0) l[di].push_back(c * nv + a);
                }
            }
            std::vector<int> ptr, idx;
            csr_from_lists(l, ptr, idx);
            m->ld_ptr.upload(ptr);
            m->ld_idx.upload(idx);
        }

        // ---- device geometry
        {
            std::vector<double> vx((size_t)M * d);
            for (int v = 0; v < M; ++v)
                for (int c = 0; c < d; ++c) vx[(size_t)c * M + v] = m->X[(size_t)v * d + c];
            m->vx.upload(vx);
            m->cells.upload(m->T);
            m->vdof.upload(m->dof_of_vertex);
            m->qx.upload(qx);
            m->qw.upload(qw);
            m->qcell.upload(m->qcell_host);
            m->qbary.upload(qb);
            std::vector<double> gx, gw;
            gauss_legendre01(opts.n_sing, gx, gw);
            m->gl_x.upload(gx);
            m->gl_w.upload(gw);
            gauss_legendre01(9, gx, gw);
            m->gl9_x.upload(gx);
            m->gl9_w.upload(gw);
            m->mtab.upload(make_math_tables());
        }
    } catch (...) {
        delete m;
        throw;
    }
    return m;
}

// ---------------------------------------------------------------------------
// Nearest-point location of the Chebyshev nodes (P1 fields at the nodes).
// A node inside the meshed region takes the P1 interpolant of its cell; a
// node outside it (boxes reach past the mesh) takes the value at the nearest
// point of the mesh.  Both are the barycentric coordinates of the closest
// point of the closest cell, found by a bucket grid over the cells' bounding
// boxes searched in rings of growing distance.
// ---------------------------------------------------------------------------
namespace {

// closest point of the simplex V[0..d] (row-major, d coordinates) to x, as
// barycentric coordinates: the orthogonal projections onto the affine hulls
// of all faces, the nearest projection whose coordinates are non-negative
double closest_in_simplex(int d, const double *V, const double *x, double *bary)
{
    const int nvx = d + 1;
    double best = 1e300;
    for (int mask = 1; mask < (1 << nvx); ++mask) {
        int idx[4] = {0, 0, 0, 0}, n = 0;   // mask >= 1: idx[0] is always set below
        for (int a = 0; a < nvx; ++a)
            if (mask >> a & 1) idx[n++] = a;
        const double *v0 = V + (size_t)idx[0] * d;
        double e[3][3], G[3][3], rhs[3], lam[3] = {0, 0, 0};
        const int m = n - 1;
        for (int j = 0; j < m; ++j)
            for (int c = 0; c < d; ++c) e[j][c] = V[(size_t)idx[j + 1] * d + c] - v0[c];
        for (int i = 0; i < m; ++i) {
            rhs[i] = 0.0;
            for (int c = 0; c < d; ++c) rhs[i] += e[i][c] * (x[c] - v0[c]);
            for (int j = 0; j < m; ++j) {
                G[i][j] = 0.0;
                for (int c = 0; c < d; ++c) G[i][j] += e[i][c] * e[j][c];
            }
        }
        // Gaussian elimination with partial pivoting on the m x m Gram system
        bool ok = true;
        for (int c = 0; c < m && ok; ++c) {
            int piv = c;
            for (int r = c + 1; r < m; ++r)
                if (std::fabs(G[r][c]) > std::fabs(G[piv][c])) piv = r;
            if (!(std::fabs(G[piv][c]) > 1e-300)) {
                ok = false;
                break;
            }
            if (piv != c) {
                for (int j = 0; j < m; ++j) std::swap(G[c][j], G[piv][j]);
                std::swap(rhs[c], rhs[piv]);
            }
            for (int r = c + 1; r < m; ++r) {
                const double f = G[r][c] / G[c][c];
                for (int j = c; j < m; ++j) G[r][j] -= f * G[c][j];
                rhs[r] -= f * rhs[c];
            }
        }
        if (!ok) continue;
        for (int c = m - 1; c >= 0; --c) {
            double v = rhs[c];
            for (int j = c + 1; j < m; ++j) v -= G[c][j] * lam[j];
            lam[c] = v / G[c][c];
        }
        double l0 = 1.0;
        bool inside = true;
        for (int j = 0; j < m; ++j) {
            l0 -= lam[j];
            inside &= lam[j] >= -1e-13;
        }
        inside &= l0 >= -1e-13;
        if (!inside) continue;
        double dist2 = 0.0;
        for (int c = 0; c < d; ++c) {
            double pc = v0[c];
            for (int j = 0; j < m; ++j) pc += lam[j] * e[j][c];
            dist2 += (x[c] - pc) * (x[c] - pc);
        }
        if (dist2 < best) {
            best = dist2;
            for (int a = 0; a < nvx; ++a) bary[a] = 0.0;
            bary[idx[0]] = std::max(l0, 0.0);
            for (int j = 0; j < m; ++j) bary[idx[j + 1]] = std::max(lam[j], 0.0);
        }
    }
    double sum = 0.0;
    for (int a = 0; a < nvx; ++a) sum += bary[a];
    for (int a = 0; a < nvx; ++a) bary[a] /= sum;
    return best;
}

struct CellGrid {
    int d = 2, n[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, h = 1.0;
    std::vector<int> ptr, idx;
    int bucket(const int *c) const { return (c[2] * n[1] + c[1]) * n[0] + c[0]; }
};

CellGrid make_cell_grid(const MeshData &m)
{
    CellGrid g;
    const int d = m.d, nv = d + 1;
    g.d = d;
    double hi[3] = {0, 0, 0};
    for (int c = 0; c < d; ++c) {
        g.lo[c] = 1e300;
        hi[c] = -1e300;
    }
    for (int v = 0; v < m.M; ++v)
        for (int c = 0; c < d; ++c) {
            g.lo[c] = std::min(g.lo[c], m.X[(size_t)v * d + c]);
            hi[c] = std::max(hi[c], m.X[(size_t)v * d + c]);
        }
    double ext = 0.0;
    for (int c = 0; c < d; ++c) ext = std::max(ext, hi[c] - g.lo[c]);
    g.h = std::max(m.h_max, ext / (d == 3 ? 128.0 : 1024.0));
    if (!(g.h > 0.0)) g.h = 1.0;
    for (int c = 0; c < d; ++c) g.n[c] = std::max(1, (int)std::ceil((hi[c] - g.lo[c]) / g.h) + 1);
    const size_t nb = (size_t)g.n[0] * g.n[1] * g.n[2];
    std::vector<std::vector<int>> lists(nb);
    for (int cell = 0; cell < m.C; ++cell) {
        int clo[3] = {0, 0, 0}, chi[3] = {0, 0, 0};
        for (int c = 0; c < d; ++c) {
            double a = 1e300, b = -1e300;
            for (int k = 0; k < nv; ++k) {
                const double x = m.X[(size_t)m.T[(size_t)cell * nv + k] * d + c];
                a = std::min(a, x);
                b = std::max(b, x);
            }
            clo[c] = std::min(g.n[c] - 1, std::max(0, (int)std::floor((a - g.lo[c]) / g.h)));
            chi[c] = std::min(g.n[c] - 1, std::max(0, (int)std::floor((b - g.lo[c]) / g.h)));
        }
        int b3[3];
        for (b3[2] = clo[2]; b3[2] <= chi[2]; ++b3[2])
            for (b3[1] = clo[1]; b3[1] <= chi[1]; ++b3[1])
                for (b3[0] = clo[0]; b3[0] <= chi[0]; ++b3[0]) lists[g.bucket(b3)].push_back(cell);
    }
    csr_from_lists(lists, g.ptr, g.idx);
    return g;
}

// closest cell and barycentric coordinates for each of n points (node-major,
// d coords); points split over host threads
void locate(const MeshData &m, const CellGrid &g, const std::vector<double> &pts, NodeLoc &out)
{
    const int d = m.d, nv = d + 1;
    const int n = (int)(pts.size() / d);
    out.cell_h.assign(n, -1);
    out.bary_h.assign((size_t)n * QB, 0.0);
    auto work = [&](int i_begin, int i_end) {
        std::vector<int> stamp(m.C, -1);
        double V[12], bary[4];
        for (int i = i_begin; i < i_end; ++i) {
            const double *x = &pts[(size_t)i * d];
            int c0[3] = {0, 0, 0};
            for (int c = 0; c < d; ++c)
                c0[c] = std::min(g.n[c] - 1, std::max(0, (int)std::floor((x[c] - g.lo[c]) / g.h)));
            double best = 1e300;
            int bcell = -1;
            double bb[4] = {0, 0, 0, 0};
            const int rmax = std::max(g.n[0], std::max(g.n[1], g.n[2]));
            for (int r = 0; r <= rmax && best > 0.0; ++r) {
                int lo3[3] = {0, 0, 0}, hi3[3] = {0, 0, 0};
                for (int c = 0; c < d; ++c) {
                    lo3[c] = c0[c] - r;
                    hi3[c] = c0[c] + r;
                }
                int b3[3];
                for (b3[2] = lo3[2]; b3[2] <= hi3[2] && best > 0.0; ++b3[2])
                    for (b3[1] = lo3[1]; b3[1] <= hi3[1] && best > 0.0; ++b3[1])
                        for (b3[0] = lo3[0]; b3[0] <= hi3[0] && best > 0.0; ++b3[0]) {
                            bool ring = false, in = true;
                            for (int c = 0; c < d; ++c) {
                                ring |= (b3[c] == lo3[c] || b3[c] == hi3[c]);
                                in &= (b3[c] >= 0 && b3[c] < g.n[c]);
                            }
                            if (!ring || !in) continue;
                            const int bk = g.bucket(b3);
                            for (int e = g.ptr[bk]; e < g.ptr[bk + 1] && best > 0.0; ++e) {
                                const int cell = g.idx[e];
                                if (stamp[cell] == i) continue;
                                stamp[cell] = i;
                                for (int a = 0; a < nv; ++a)
                                    for (int c = 0; c < d; ++c)
                                        V[a * d + c] = m.X[(size_t)m.T[(size_t)cell * nv + a] * d + c];
                                const double dist2 = closest_in_simplex(d, V, x, bary);
                                if (dist2 < best) {
                                    best = dist2;
                                    bcell = cell;
                                    for (int a = 0; a < nv; ++a) bb[a] = bary[a];
                                }
                            }
                        }
                // every cell first met in a later ring lies at least r * h away
                if (bcell >= 0 && best <= (r * g.h) * (r * g.h)) break;
            }
            out.cell_h[i] = bcell;
            for (int a = 0; a < nv; ++a) out.bary_h[(size_t)i * QB + a] = bb[a];
        }
    };
    const int nth = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 4096 || nth == 1) {
        work(0, n);
    } else {
        std::vector<std::thread> th;
        for (int t = 0; t < nth; ++t) th.emplace_back(work, (int)((int64_t)n * t / nth), (int)((int64_t)n * (t + 1) / nth));
        for (auto &t : th) t.join();
    }
    for (int i = 0; i < n; ++i) VFD_REQUIRE(out.cell_h[i] >= 0, VFD_EINVAL, "node location: no cell found");
    out.cell.upload(out.cell_h);
    out.bary.upload(out.bary_h);
    out.done = true;
}

}  // namespace

void locate_nodes(MeshData &m)
{
    if (m.nodes_located) return;
    const CellGrid g = make_cell_grid(m);
    if (!m.kt_cheb_h.empty()) locate(m, g, m.kt_cheb_h, m.kt_loc);
    if (!m.kt_cheb_in_h.empty()) locate(m, g, m.kt_cheb_in_h, m.kt_in_loc);
    if (!m.tt_cheb_h.empty()) locate(m, g, m.tt_cheb_h, m.tt_loc);
    if (!m.st_cheb_h.empty()) locate(m, g, m.st_cheb_h, m.st_loc);
    m.nodes_located = true;
}

}  // namespace vfd
