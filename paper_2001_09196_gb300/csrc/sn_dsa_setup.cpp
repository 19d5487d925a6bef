// Host-side setup of the thick-subdomain DSA operator and its multigrid hierarchy.
//
// Operators (paper Sec. 3.1; Sec. 3.2: the heterogeneous operator is the principal submatrix on
// the thick elements):
//   a(u,v) = sum_K (D grad u, grad v)_K + (sigma_a u, v)_K
//          + sum_{interior thick-thick F} <kappa [u],[v]> - <{D grad u.n},[v]> - s <{D grad v.n},[u]>
//          + sum_{F on the thick region's boundary} <kappa u,v> - 1/2<D grad u.n, v> - s/2 <D grad v.n, u>
// D = 1/(3 sigma_t), sigma_a = sigma_t - sigma_s, h = |K|/|F|.  A face to a non-thick neighbour is a
// face to a zero exterior state.
//   SIP (Eq. SIP with a max-floored penalty): s = 1, kappa = max(1/4, c(p) (D-/h- + D+/h+)/2) on
//     interior faces and max(1/4, c(p) D/h) on boundary faces, c(p) = 2 p (p+1).
//   NIP (Eq. NIP): s = 0 (the symmetrising term G^T Sigma_t^{-1} F_1 dropped), kappa = 1/4 (F_0).
//   mNIP (Eq. NIP with Eq. ModifiedF0): s = 0, kappa = (max(c(p)/(sigma_t- h-), 1) + max(c(p)/(sigma_t+ h+),
//     1)) / 8, c(p) = 0.1 p (p+1): each side is upwind for the directions leaving it, and either half of
//     the angular integral of |Omega.n| / (8 pi) is 1/8.  The neighbour's data enter even when it is
//     thin; on the domain boundary the element's own value stands for the missing side; a void
//     neighbour makes the penalty infinite and is an error.
// All integrals use the (p+1)-point Gauss rule per axis, on which the nodal basis lives (so the
// volume terms are collocated).  For the adjoint of a nonsymmetric operator the assembled blocks
// are transposed before the hierarchy is built (the Galerkin hierarchy of A^T is the transpose of
// that of A).
//
// Multigrid (replaces the paper's BoomerAMG, Sec. 4): level 0 is the DG space on the thick
// elements with element block-Jacobi smoothing; level 1 is continuous Q1 on the vertices of
// thick elements (prolongation = the element's own bilinear/trilinear map evaluated at its
// nodes); coarser levels halve the vertex grid per axis with linear interpolation; every
// coarse operator is the Galerkin product P^T A P; the coarsest is inverted densely.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "sn_dsa.h"

namespace sn {

namespace {

struct Csr {
    int rows = 0, cols = 0;
    std::vector<int> ptr, col;
    std::vector<double> val;
};

Csr transpose(const Csr& A) {
    Csr T;
    T.rows = A.cols;
    T.cols = A.rows;
    T.ptr.assign(T.rows + 1, 0);
    for (int c : A.col) T.ptr[c + 1]++;
    for (int r = 0; r < T.rows; ++r) T.ptr[r + 1] += T.ptr[r];
    T.col.resize(A.col.size());
    T.val.resize(A.val.size());
    std::vector<int> fill(T.ptr.begin(), T.ptr.end() - 1);
    for (int r = 0; r < A.rows; ++r)
        for (int k = A.ptr[r]; k < A.ptr[r + 1]; ++k) {
            int pos = fill[A.col[k]]++;
            T.col[pos] = r;
            T.val[pos] = A.val[k];
        }
    return T;
}

// C = A * B, rows in parallel: each output row sums its products in the order A's row entries and
// then B's row entries are met (so the result does not depend on the thread schedule), columns
// ascending.
Csr multiply(const Csr& A, const Csr& B);

// In-place inverse of a small SPD-ish dense matrix (Gauss-Jordan, partial pivoting).
bool invert(std::vector<double>& A, int n) {
    std::vector<double> I(n * n, 0.0);
    for (int i = 0; i < n; ++i) I[i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (A[piv * n + c] == 0.0) return false;
        if (piv != c)
            for (int q = 0; q < n; ++q) {
                std::swap(A[c * n + q], A[piv * n + q]);
                std::swap(I[c * n + q], I[piv * n + q]);
            }
        const double inv = 1.0 / A[c * n + c];
        for (int q = 0; q < n; ++q) {
            A[c * n + q] *= inv;
            I[c * n + q] *= inv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[r * n + c];
            if (f == 0.0) continue;
            for (int q = 0; q < n; ++q) {
                A[r * n + q] -= f * A[c * n + q];
                I[r * n + q] -= f * I[c * n + q];
            }
        }
    }
    A.swap(I);
    return true;
}

struct ElemMap {
    int dim;
    double v[8][3];  // corners, corner c: bit a set -> xi_a = +1
    // x(xi), J(xi) (J[r][c] = dx_r/dxi_c)
    void eval(const double* xi, double* x, double J[3][3]) const {
        for (int r = 0; r < dim; ++r) {
            x[r] = 0.0;
            for (int c = 0; c < dim; ++c) J[r][c] = 0.0;
        }
        const int nc = 1 << dim;
        for (int c = 0; c < nc; ++c) {
            double fac[3], s[3];
            for (int a = 0; a < dim; ++a) {
                s[a] = ((c >> a) & 1) ? 1.0 : -1.0;
                fac[a] = 0.5 * (1.0 + s[a] * xi[a]);
            }
            double N = 1.0;
            for (int a = 0; a < dim; ++a) N *= fac[a];
            for (int r = 0; r < dim; ++r) x[r] += N * v[c][r];
            for (int a = 0; a < dim; ++a) {
                double dN = 0.5 * s[a];
                for (int b = 0; b < dim; ++b)
                    if (b != a) dN *= fac[b];
                for (int r = 0; r < dim; ++r) J[r][a] += dN * v[c][r];
            }
        }
    }
};

double det_inv(int dim, const double J[3][3], double Ji[3][3]) {
    if (dim == 2) {
        const double d = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / d;
        Ji[0][1] = -J[0][1] / d;
        Ji[1][0] = -J[1][0] / d;
        Ji[1][1] = J[0][0] / d;
        return d;
    }
    const double d = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / d;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / d;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / d;
    Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / d;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / d;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / d;
    Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / d;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / d;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / d;
    return d;
}

// Tensor nodal basis values and reference gradients at a reference point.
void basis_at(const GL1D& g, int dim, const double* xi, std::vector<double>& val, std::vector<double>& grad) {
    const int Q = g.p + 1;
    double v1[3][kMaxP + 1], d1[3][kMaxP + 1];
    for (int a = 0; a < dim; ++a) lagrange_eval(g, xi[a], v1[a], d1[a]);
    const int N = dim == 2 ? Q * Q : Q * Q * Q;
    val.assign(N, 0.0);
    grad.assign(N * dim, 0.0);
    for (int i = 0; i < N; ++i) {
        int idx[3] = {i % Q, (i / Q) % Q, i / (Q * Q)};
        double v = 1.0;
        for (int a = 0; a < dim; ++a) v *= v1[a][idx[a]];
        val[i] = v;
        for (int b = 0; b < dim; ++b) {
            double gb = 1.0;
            for (int a = 0; a < dim; ++a) gb *= (a == b ? d1[a][idx[a]] : v1[a][idx[a]]);
            grad[i * dim + b] = gb;
        }
    }
}

}  // namespace

// Runs f(i) for i in [0, n) on the host's cores (fixed chunks claimed from a shared counter; every
// f(i) must touch data of its own index only, so the result does not depend on the schedule).
template <typename F>
void parallel_for(int n, F&& f) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int T = (int)std::max(1u, std::min(hw == 0 ? 1u : hw, 32u));
    if (n < 512 || T == 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::atomic<int> next{0};
    constexpr int chunk = 64;
    auto work = [&]() {
        int s0;
        while ((s0 = next.fetch_add(chunk)) < n)
            for (int i = s0; i < std::min(n, s0 + chunk); ++i) f(i);
    };
    std::vector<std::thread> th;
    for (int k = 1; k < T; ++k) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
}

namespace {

Csr multiply(const Csr& A, const Csr& B) {
    Csr C;
    C.rows = A.rows;
    C.cols = B.cols;
    std::vector<std::vector<std::pair<int, double>>> rows(A.rows);
    parallel_for(A.rows, [&](int r) {
        std::vector<std::pair<int, double>>& row = rows[r];
        for (int k = A.ptr[r]; k < A.ptr[r + 1]; ++k) {
            const double av = A.val[k];
            for (int l = B.ptr[A.col[k]]; l < B.ptr[A.col[k] + 1]; ++l) {
                const int c = B.col[l];
                bool found = false;
                for (auto& pr : row)
                    if (pr.first == c) {
                        pr.second += av * B.val[l];
                        found = true;
                        break;
                    }
                if (!found) row.push_back({c, 0.0 + av * B.val[l]});  // as an accumulator that starts at 0
            }
        }
        std::sort(row.begin(), row.end(), [](const std::pair<int, double>& x, const std::pair<int, double>& y) {
            return x.first < y.first;
        });
    });
    C.ptr.assign(A.rows + 1, 0);
    for (int r = 0; r < A.rows; ++r) C.ptr[r + 1] = C.ptr[r] + (int)rows[r].size();
    C.col.resize(C.ptr[A.rows]);
    C.val.resize(C.ptr[A.rows]);
    parallel_for(A.rows, [&](int r) {
        for (size_t k = 0; k < rows[r].size(); ++k) {
            C.col[C.ptr[r] + k] = rows[r][k].first;
            C.val[C.ptr[r] + k] = rows[r][k].second;
        }
    });
    return C;
}

}  // namespace

DsaHierarchy* dsa_build(const sn_mesh* m, const unsigned char* mask, int dsa_sigma, int dsa_op, bool transposed,
                        std::string& err, bool* void_conflict) {
    if (void_conflict) *void_conflict = false;
    auto* H = new DsaHierarchy();
    const int dim = m->dim, p = m->p, n = m->n, Q = p + 1, nf = 2 * dim;
    H->n = n;
    H->ne = m->ne;
    H->op = dsa_op;
    H->symmetric = dsa_op == SN_DSA_OP_SIP;
    H->transposed = transposed && !H->symmetric;
    const double sym = H->symmetric ? 1.0 : 0.0;  // weight of the symmetrising face term
    for (int e = 0; e < m->ne; ++e)
        if (mask[e]) H->thick.push_back(e);
    const int nt = (int)H->thick.size();
    H->nt = nt;
    if (nt == 0) return H;
    for (int e : H->thick)
        if (!(m->h_sigma_t[e] > 0.0)) {
            err = "DSA on an element with sigma_t = 0";
            delete H;
            return nullptr;
        }
    std::vector<int> local(m->ne, -1);
    for (int t = 0; t < nt; ++t) local[H->thick[t]] = t;
    const GL1D g = gauss_legendre_nodal(p);
    const double cp = 2.0 * p * (p + 1);   // SIP penalty constant
    const double cm = 0.1 * p * (p + 1);   // c(p) of Eq. ModifiedF0

    auto elem_map = [&](int e) {
        ElemMap em;
        em.dim = dim;
        if (dim == 2) {
            const double* c = &m->h_corners[8 * (size_t)e];
            for (int q = 0; q < 4; ++q) {
                em.v[q][0] = c[2 * q];
                em.v[q][1] = c[2 * q + 1];
                em.v[q][2] = 0.0;
            }
        } else {
            const int i = e % m->nx, j = (e / m->nx) % m->ny, k = e / (m->nx * m->ny);
            for (int q = 0; q < 8; ++q) {
                em.v[q][0] = (i + (q & 1)) * m->hx;
                em.v[q][1] = (j + ((q >> 1) & 1)) * m->hy;
                em.v[q][2] = (k + ((q >> 2) & 1)) * m->hz;
            }
        }
        return em;
    };
    auto coord = [&](int e, int ax) {
        return ax == 0 ? e % m->nx : (ax == 1 ? (e / m->nx) % m->ny : e / (m->nx * m->ny));
    };
    auto neighbor = [&](int e, int f) {
        const int ax = f >> 1, side = f & 1;
        int i = e % m->nx, j = (e / m->nx) % m->ny, k = e / (m->nx * m->ny);
        const int dl = side ? 1 : -1;
        if (ax == 0) { i += dl; if (i < 0 || i >= m->nx) return -1; }
        else if (ax == 1) { j += dl; if (j < 0 || j >= m->ny) return -1; }
        else { k += dl; if (k < 0 || k >= m->nz) return -1; }
        return i + m->nx * (j + m->ny * k);
    };
    if (dsa_op == SN_DSA_OP_MNIP)
        for (int e : H->thick)
            for (int f = 0; f < nf; ++f) {
                const int u = neighbor(e, f);
                if (u >= 0 && !(m->h_sigma_t[u] > 0.0)) {
                    err = "the mNIP penalty (Eq. ModifiedF0) is undefined next to a void element";
                    if (void_conflict) *void_conflict = true;
                    delete H;
                    return nullptr;
                }
            }

    // reference basis data, the same for every element: values and reference gradients at the
    // volume nodes and at the face quadrature points of every face
    const int QF = dim == 2 ? Q : Q * Q;
    std::vector<double> vval((size_t)n * n), vgrad((size_t)n * n * dim), vW(n);
    std::vector<double> fval((size_t)nf * QF * n), fgrad((size_t)nf * QF * n * dim), fW((size_t)nf * QF);
    std::vector<double> fxi((size_t)nf * QF * 3);
    {
        std::vector<double> val, grad;
        for (int q = 0; q < n; ++q) {
            const int qi[3] = {q % Q, (q / Q) % Q, q / (Q * Q)};
            double xi[3] = {0, 0, 0}, W = 1.0;
            for (int a = 0; a < dim; ++a) {
                xi[a] = g.x[qi[a]];
                W *= g.w[qi[a]];
            }
            vW[q] = W;
            basis_at(g, dim, xi, val, grad);
            std::copy(val.begin(), val.end(), vval.begin() + (size_t)q * n);
            std::copy(grad.begin(), grad.end(), vgrad.begin() + (size_t)q * n * dim);
        }
        for (int f = 0; f < nf; ++f) {
            const int ax = f >> 1;
            const double s = (f & 1) ? 1.0 : -1.0;
            for (int qf = 0; qf < QF; ++qf) {
                const int tq[2] = {qf % Q, qf / Q};
                double* xi = &fxi[((size_t)f * QF + qf) * 3];
                double Wt = 1.0;
                int c = 0;
                for (int a = 0; a < 3; ++a) xi[a] = 0.0;
                for (int a = 0; a < dim; ++a) {
                    if (a == ax) {
                        xi[a] = s;
                    } else {
                        xi[a] = g.x[tq[c]];
                        Wt *= g.w[tq[c]];
                        ++c;
                    }
                }
                fW[(size_t)f * QF + qf] = Wt;
                basis_at(g, dim, xi, val, grad);
                std::copy(val.begin(), val.end(), fval.begin() + ((size_t)f * QF + qf) * n);
                std::copy(grad.begin(), grad.end(), fgrad.begin() + ((size_t)f * QF + qf) * n * dim);
            }
        }
    }

    // BSR structure: every thick element's row holds its own block and those of its thick face
    // neighbours, columns ascending
    Level0& L0 = H->l0;
    L0.ptr.assign(nt + 1, 0);
    for (int t = 0; t < nt; ++t) {
        int cnt = 1;
        for (int f = 0; f < nf; ++f) {
            const int u = neighbor(H->thick[t], f);
            if (u >= 0 && local[u] >= 0) ++cnt;
        }
        L0.ptr[t + 1] = L0.ptr[t] + cnt;
    }
    L0.col.resize(L0.ptr[nt]);
    parallel_for(nt, [&](int t) {
        int* c = &L0.col[L0.ptr[t]];
        int k = 0;
        c[k++] = t;
        for (int f = 0; f < nf; ++f) {
            const int u = neighbor(H->thick[t], f);
            if (u >= 0 && local[u] >= 0) c[k++] = local[u];
        }
        std::sort(c, c + k);
    });
    L0.val.assign((size_t)L0.ptr[nt] * n * n, 0.0);
    auto block = [&](int r, int c) -> double* {
        for (int k = L0.ptr[r]; k < L0.ptr[r + 1]; ++k)
            if (L0.col[k] == c) return &L0.val[(size_t)k * n * n];
        return nullptr;  // unreachable: the structure holds every face pair
    };

    // volume terms: (D grad u, grad v) + (sigma_a u, v), collocated at the nodes
    std::vector<double> vol(nt), Dc(nt), sa(nt);
    H->h_mass_sig.assign((size_t)nt * n, 0.0);
    parallel_for(nt, [&](int t) {
        const int e = H->thick[t];
        const double st = m->h_sigma_t[e], ss = m->h_sigma_s[e];
        Dc[t] = 1.0 / (3.0 * st);
        sa[t] = st - ss;
        const double sig = dsa_sigma == SN_DSA_SIGMA_T ? st : ss;
        const ElemMap em = elem_map(e);
        double* K = block(t, t);
        double V = 0.0;
        std::vector<double> gp((size_t)n * dim);
        for (int q = 0; q < n; ++q) {
            const int qi[3] = {q % Q, (q / Q) % Q, q / (Q * Q)};
            double xi[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) xi[a] = g.x[qi[a]];
            const double W = vW[q];
            double x[3], J[3][3], Ji[3][3];
            em.eval(xi, x, J);
            const double dJ = det_inv(dim, J, Ji);
            V += W * dJ;
            const double* val = &vval[(size_t)q * n];
            const double* grad = &vgrad[(size_t)q * n * dim];
            for (int i = 0; i < n; ++i)
                for (int r = 0; r < dim; ++r) {
                    double sum = 0.0;
                    for (int k = 0; k < dim; ++k) sum += Ji[k][r] * grad[i * dim + k];
                    gp[i * dim + r] = sum;
                }
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    double sum = 0.0;
                    for (int r = 0; r < dim; ++r) sum += gp[i * dim + r] * gp[j * dim + r];
                    K[i * n + j] += W * dJ * (Dc[t] * sum + sa[t] * val[i] * val[j]);
                }
            H->h_mass_sig[(size_t)t * n + q] = sig * W * dJ;  // collocated mass at node q
        }
        vol[t] = V;
    });

    // volume of any element (the mNIP penalty reads thin neighbours too)
    auto elem_volume = [&](int e) {
        const ElemMap em = elem_map(e);
        double V = 0.0;
        for (int q = 0; q < n; ++q) {
            const int qi[3] = {q % Q, (q / Q) % Q, q / (Q * Q)};
            double xi[3] = {0, 0, 0}, x[3], J[3][3], Ji[3][3];
            for (int a = 0; a < dim; ++a) xi[a] = g.x[qi[a]];
            em.eval(xi, x, J);
            V += vW[q] * det_inv(dim, J, Ji);
        }
        return V;
    };

    // face terms.  An interior thick-thick face is assembled once, from its side-1 element, into
    // the rows of both elements; a face to a non-thick element or the boundary into its own row.
    // Pass (axis, parity) takes the elements whose coordinate along the axis has that parity, so
    // no two faces of one pass write the same row.
    struct FaceData {
        std::vector<double> dS, nrm, B, Dn;
        double area;
    };
    auto face_geometry = [&](const ElemMap& em, int f, FaceData& F) {
        const int ax = f >> 1;
        const double s = (f & 1) ? 1.0 : -1.0;
        F.dS.resize(QF);
        F.nrm.resize((size_t)QF * 3);
        F.area = 0.0;
        for (int qf = 0; qf < QF; ++qf) {
            const double* xi = &fxi[((size_t)f * QF + qf) * 3];
            double x[3], J[3][3], Ji[3][3];
            em.eval(xi, x, J);
            const double dJ = det_inv(dim, J, Ji);
            // Nanson: n dS = det J J^{-T} (s e_ax) dt
            double Nv[3] = {0, 0, 0}, len = 0.0;
            for (int r = 0; r < dim; ++r) {
                Nv[r] = s * dJ * Ji[ax][r];
                len += Nv[r] * Nv[r];
            }
            len = std::sqrt(len);
            F.dS[qf] = len * fW[(size_t)f * QF + qf];
            F.area += F.dS[qf];
            for (int r = 0; r < dim; ++r) F.nrm[qf * 3 + r] = Nv[r] / len;
        }
    };
    // values and normal derivatives on face f of an element with map em, along the normals F.nrm
    auto face_traces = [&](const ElemMap& em, int f, const std::vector<double>& nrm, std::vector<double>& B,
                           std::vector<double>& Dn) {
        B.resize((size_t)QF * n);
        Dn.resize((size_t)QF * n);
        for (int qf = 0; qf < QF; ++qf) {
            const double* xi = &fxi[((size_t)f * QF + qf) * 3];
            double x[3], J[3][3], Ji[3][3];
            em.eval(xi, x, J);
            det_inv(dim, J, Ji);
            const double* val = &fval[((size_t)f * QF + qf) * n];
            const double* grad = &fgrad[((size_t)f * QF + qf) * n * dim];
            for (int i = 0; i < n; ++i) {
                B[qf * n + i] = val[i];
                double dn = 0.0;
                for (int r = 0; r < dim; ++r) {
                    double gr = 0.0;
                    for (int k = 0; k < dim; ++k) gr += Ji[k][r] * grad[i * dim + k];
                    dn += gr * nrm[qf * 3 + r];
                }
                Dn[qf * n + i] = dn;
            }
        }
    };
    for (int ax = 0; ax < dim; ++ax)
        for (int parity = 0; parity < 2; ++parity)
            parallel_for(nt, [&](int t) {
                const int e = H->thick[t];
                if (coord(e, ax) % 2 != parity) return;
                FaceData F;
                std::vector<double> Be, Dne, Bo, Dno;
                for (int side = 0; side < 2; ++side) {
                    const int f = 2 * ax + side;
                    const int u = neighbor(e, f);
                    const int o = u >= 0 ? local[u] : -1;
                    if (o >= 0 && side == 0) continue;  // assembled by the side-1 element
                    const ElemMap em = elem_map(e);
                    face_geometry(em, f, F);
                    face_traces(em, f, F.nrm, Be, Dne);
                    const double h = vol[t] / F.area;
                    // Eq. ModifiedF0 factor of one side: max(c(p) / (sigma_t h), 1)
                    auto mod = [&](double st, double hh) { return std::max(cm / (st * hh), 1.0); };
                    if (o < 0) {
                        double kap = 0.25;
                        if (dsa_op == SN_DSA_OP_SIP) {
                            kap = std::max(0.25, cp * Dc[t] / h);
                        } else if (dsa_op == SN_DSA_OP_MNIP) {
                            const double own = mod(m->h_sigma_t[e], h);
                            const double other = u >= 0 ? mod(m->h_sigma_t[u], elem_volume(u) / F.area) : own;
                            kap = 0.125 * (own + other);
                        }
                        double* K = block(t, t);
                        for (int qf = 0; qf < QF; ++qf)
                            for (int i = 0; i < n; ++i)
                                for (int j = 0; j < n; ++j)
                                    K[i * n + j] += F.dS[qf] * (kap * Be[qf * n + i] * Be[qf * n + j] -
                                                                0.5 * Dc[t] * Dne[qf * n + j] * Be[qf * n + i] -
                                                                sym * 0.5 * Dc[t] * Dne[qf * n + i] * Be[qf * n + j]);
                        continue;
                    }
                    face_traces(elem_map(u), f ^ 1, F.nrm, Bo, Dno);
                    const double ho = vol[o] / F.area;
                    double kap = 0.25;
                    if (dsa_op == SN_DSA_OP_SIP) kap = std::max(0.25, cp * 0.5 * (Dc[t] / h + Dc[o] / ho));
                    else if (dsa_op == SN_DSA_OP_MNIP) kap = 0.125 * (mod(m->h_sigma_t[e], h) + mod(m->h_sigma_t[u], ho));
                    struct Side { int r; const std::vector<double>* B; const std::vector<double>* Dn; double D, sg; };
                    const Side sides[2] = {{t, &Be, &Dne, Dc[t], 1.0}, {o, &Bo, &Dno, Dc[o], -1.0}};
                    for (const Side& A : sides)
                        for (const Side& Bs : sides) {
                            double* K = block(A.r, Bs.r);
                            for (int qf = 0; qf < QF; ++qf)
                                for (int i = 0; i < n; ++i)
                                    for (int j = 0; j < n; ++j)
                                        K[i * n + j] += F.dS[qf] * (kap * A.sg * Bs.sg * (*A.B)[qf * n + i] * (*Bs.B)[qf * n + j] -
                                                                    0.5 * Bs.D * A.sg * (*Bs.Dn)[qf * n + j] * (*A.B)[qf * n + i] -
                                                                    sym * 0.5 * A.D * Bs.sg * (*A.Dn)[qf * n + i] * (*Bs.B)[qf * n + j]);
                        }
                }
            });

    if (H->transposed) {  // block (r, c) of D^T is block (c, r) of D, transposed
        std::vector<double> tv(L0.val.size());
        parallel_for(nt, [&](int r) {
            for (int k = L0.ptr[r]; k < L0.ptr[r + 1]; ++k) {
                const double* src = block(L0.col[k], r);
                double* dst = &tv[(size_t)k * n * n];
                for (int i = 0; i < n; ++i)
                    for (int j = 0; j < n; ++j) dst[i * n + j] = src[j * n + i];
            }
        });
        L0.val.swap(tv);
    }

    // inverse diagonal blocks (block-Jacobi smoother)
    L0.dinv.resize((size_t)nt * n * n);
    std::atomic<int> singular{0};
    parallel_for(nt, [&](int t) {
        const double* K = block(t, t);
        std::vector<double> B(K, K + (size_t)n * n);
        if (!invert(B, n)) singular = 1;
        std::copy(B.begin(), B.end(), L0.dinv.begin() + (size_t)t * n * n);
    });
    if (singular) {
        err = "singular diagonal block in the DSA operator";
        delete H;
        return nullptr;
    }

    // level 1: continuous Q1 on the vertices of thick elements.  The prolongation of an element is
    // its own bilinear (trilinear) map evaluated at its nodes: the same n x 2^dim matrix Pref for
    // every element, so A_1 = P^T A P is accumulated block by block as Pref^T K_tc Pref.
    const int nc = 1 << dim;
    const int vx = m->nx + 1, vy = m->ny + 1, vz = dim == 3 ? m->nz + 1 : 1;
    std::vector<int> vid((size_t)vx * vy * vz, -1);
    std::vector<int> vgrid;  // active vertex -> grid index
    std::vector<int> evid((size_t)nt * nc);
    for (int t = 0; t < nt; ++t) {
        const int e = H->thick[t];
        const int i = e % m->nx, j = (e / m->nx) % m->ny, k = e / (m->nx * m->ny);
        for (int c = 0; c < nc; ++c) {
            const size_t gid = (i + (c & 1)) + (size_t)vx * ((j + ((c >> 1) & 1)) + (size_t)vy * (dim == 3 ? k + ((c >> 2) & 1) : 0));
            if (vid[gid] < 0) {
                vid[gid] = (int)vgrid.size();
                vgrid.push_back((int)gid);
            }
            evid[(size_t)t * nc + c] = vid[gid];
        }
    }
    const int nv = (int)vgrid.size();
    std::vector<double> Pref((size_t)n * nc);
    for (int q = 0; q < n; ++q) {
        const int qi[3] = {q % Q, (q / Q) % Q, q / (Q * Q)};
        for (int c = 0; c < nc; ++c) {
            double N = 1.0;
            for (int a = 0; a < dim; ++a) N *= 0.5 * (1.0 + (((c >> a) & 1) ? 1.0 : -1.0) * g.x[qi[a]]);
            Pref[(size_t)q * nc + c] = N;
        }
    }
    Csr P;
    P.rows = nt * n;
    P.cols = nv;
    P.ptr.resize(P.rows + 1);
    for (int r = 0; r <= P.rows; ++r) P.ptr[r] = r * nc;
    P.col.resize((size_t)P.rows * nc);
    P.val.resize((size_t)P.rows * nc);
    parallel_for(nt, [&](int t) {
        int ord[8];
        for (int c = 0; c < nc; ++c) ord[c] = c;
        std::sort(ord, ord + nc, [&](int a, int b) { return evid[(size_t)t * nc + a] < evid[(size_t)t * nc + b]; });
        for (int q = 0; q < n; ++q)
            for (int k = 0; k < nc; ++k) {
                const size_t pos = ((size_t)t * n + q) * nc + k;
                P.col[pos] = evid[(size_t)t * nc + ord[k]];
                P.val[pos] = Pref[(size_t)q * nc + ord[k]];
            }
    });
    // KP = K_tc Pref for every block
    const size_t nnzb = L0.col.size();
    std::vector<double> KP(nnzb * n * nc);
    parallel_for((int)nnzb, [&](int b) {
        const double* K = &L0.val[(size_t)b * n * n];
        double* o = &KP[(size_t)b * n * nc];
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < nc; ++c) {
                double sum = 0.0;
                for (int j = 0; j < n; ++j) sum += K[i * n + j] * Pref[(size_t)j * nc + c];
                o[i * nc + c] = sum;
            }
    });
    // rows of A_1: vertex v gathers Pref[:, a]^T KP_tc over the (t, a) that touch it
    std::vector<int> vt_ptr(nv + 1, 0), vt((size_t)nt * nc);
    for (size_t k = 0; k < evid.size(); ++k) vt_ptr[evid[k] + 1]++;
    for (int v = 0; v < nv; ++v) vt_ptr[v + 1] += vt_ptr[v];
    {
        std::vector<int> fill(vt_ptr.begin(), vt_ptr.end() - 1);
        for (size_t k = 0; k < evid.size(); ++k) vt[fill[evid[k]]++] = (int)k;  // k = t * nc + a, ascending
    }
    std::vector<std::vector<std::pair<int, double>>> arows(nv);
    parallel_for(nv, [&](int v) {
        std::vector<std::pair<int, double>>& row = arows[v];
        for (int s = vt_ptr[v]; s < vt_ptr[v + 1]; ++s) {
            const int t = vt[s] / nc, a = vt[s] % nc;
            for (int b = L0.ptr[t]; b < L0.ptr[t + 1]; ++b) {
                const int c = L0.col[b];
                const double* kp = &KP[(size_t)b * n * nc];
                for (int cc = 0; cc < nc; ++cc) {
                    double sum = 0.0;
                    for (int i = 0; i < n; ++i) sum += Pref[(size_t)i * nc + a] * kp[i * nc + cc];
                    const int col = evid[(size_t)c * nc + cc];
                    bool found = false;
                    for (auto& pr : row)
                        if (pr.first == col) {
                            pr.second += sum;
                            found = true;
                            break;
                        }
                    if (!found) row.push_back({col, sum});
                }
            }
        }
        std::sort(row.begin(), row.end(), [](const std::pair<int, double>& x, const std::pair<int, double>& y) {
            return x.first < y.first;
        });
    });
    Csr A1;
    A1.rows = A1.cols = nv;
    A1.ptr.assign(nv + 1, 0);
    for (int v = 0; v < nv; ++v) A1.ptr[v + 1] = A1.ptr[v] + (int)arows[v].size();
    A1.col.resize(A1.ptr[nv]);
    A1.val.resize(A1.ptr[nv]);
    parallel_for(nv, [&](int v) {
        for (size_t k = 0; k < arows[v].size(); ++k) {
            A1.col[A1.ptr[v] + k] = arows[v][k].first;
            A1.val[A1.ptr[v] + k] = arows[v][k].second;
        }
    });

    struct GridLevel { int nx, ny, nz; std::vector<int> gids; };  // cells per axis, active vertex grid ids
    GridLevel cur{m->nx, m->ny, dim == 3 ? m->nz : 0, vgrid};
    // restriction to level 1, P^T, row by row: vertex v takes Pref[q][a] from node q of every
    // element t that has v as corner a (the columns come out ascending, as a transpose gives them)
    Csr R1;
    R1.rows = nv;
    R1.cols = P.rows;
    R1.ptr.assign(nv + 1, 0);
    for (int v = 0; v < nv; ++v) R1.ptr[v + 1] = R1.ptr[v] + (vt_ptr[v + 1] - vt_ptr[v]) * n;
    R1.col.resize(R1.ptr[nv]);
    R1.val.resize(R1.ptr[nv]);
    parallel_for(nv, [&](int v) {
        int pos = R1.ptr[v];
        for (int s = vt_ptr[v]; s < vt_ptr[v + 1]; ++s) {
            const int t = vt[s] / nc, a = vt[s] % nc;
            for (int q = 0; q < n; ++q, ++pos) {
                R1.col[pos] = t * n + q;
                R1.val[pos] = Pref[(size_t)q * nc + a];
            }
        }
    });
    Csr Acur;
    Csr Pcur = std::move(P);
    for (int lev = 1; lev < 32; ++lev) {
        Csr Pt = lev == 1 ? std::move(R1) : transpose(Pcur);
        Csr Ac = lev == 1 ? std::move(A1) : multiply(Pt, multiply(Acur, Pcur));
        LevelC L;
        L.n = Ac.rows;
        L.p_ptr = std::move(Pcur.ptr); L.p_col = std::move(Pcur.col); L.p_val = std::move(Pcur.val);
        L.r_ptr = std::move(Pt.ptr); L.r_col = std::move(Pt.col); L.r_val = std::move(Pt.val);
        L.a_ptr = Ac.ptr; L.a_col = Ac.col; L.a_val = Ac.val;
        L.dinv.assign(L.n, 0.0);
        for (int r = 0; r < Ac.rows; ++r)
            for (int k = Ac.ptr[r]; k < Ac.ptr[r + 1]; ++k)
                if (Ac.col[k] == r) L.dinv[r] = 1.0 / Ac.val[k];
        const bool coarsest = Ac.rows <= kCoarseMax || (cur.nx <= 1 && cur.ny <= 1 && cur.nz <= 1);
        if (coarsest) {
            std::vector<double> Dm((size_t)Ac.rows * Ac.rows, 0.0);
            for (int r = 0; r < Ac.rows; ++r)
                for (int k = Ac.ptr[r]; k < Ac.ptr[r + 1]; ++k) Dm[(size_t)r * Ac.rows + Ac.col[k]] = Ac.val[k];
            if (!invert(Dm, Ac.rows)) {
                err = "singular coarsest DSA operator";
                delete H;
                return nullptr;
            }
            L.dense_inv = Dm;
            H->levels.push_back(std::move(L));
            break;
        }
        H->levels.push_back(std::move(L));
        // next vertex grid: half the cells per axis (rounded up), linear interpolation
        GridLevel nxt{(cur.nx + 1) / 2, (cur.ny + 1) / 2, dim == 3 ? (cur.nz + 1) / 2 : 0, {}};
        const int fx = cur.nx + 1, fy = cur.ny + 1;
        const int cx = nxt.nx + 1, cy = nxt.ny + 1, cz = dim == 3 ? nxt.nz + 1 : 1;
        std::vector<int> cid((size_t)cx * cy * cz, -1);
        std::vector<std::vector<std::pair<size_t, double>>> rows(cur.gids.size());
        for (size_t r = 0; r < cur.gids.size(); ++r) {
            const int gidv = cur.gids[r];
            const int I = gidv % fx, J = (gidv / fx) % fy, K = gidv / (fx * fy);
            int ci[3][2];
            double cw[3][2];
            int cnt[3];
            const int idx[3] = {I, J, K};
            for (int a = 0; a < 3; ++a) {
                if (a >= dim) { ci[a][0] = 0; cw[a][0] = 1.0; cnt[a] = 1; continue; }
                if (idx[a] % 2 == 0) { ci[a][0] = idx[a] / 2; cw[a][0] = 1.0; cnt[a] = 1; }
                else { ci[a][0] = (idx[a] - 1) / 2; ci[a][1] = (idx[a] + 1) / 2; cw[a][0] = cw[a][1] = 0.5; cnt[a] = 2; }
            }
            for (int a0 = 0; a0 < cnt[0]; ++a0)
                for (int a1 = 0; a1 < cnt[1]; ++a1)
                    for (int a2 = 0; a2 < cnt[2]; ++a2) {
                        const size_t cg = ci[0][a0] + (size_t)cx * (ci[1][a1] + (size_t)cy * ci[2][a2]);
                        rows[r].push_back({cg, cw[0][a0] * cw[1][a1] * cw[2][a2]});
                        if (cid[cg] < 0) cid[cg] = 0;
                    }
        }
        int nc = 0;
        for (size_t cg = 0; cg < cid.size(); ++cg)
            if (cid[cg] >= 0) {
                cid[cg] = nc++;
                nxt.gids.push_back((int)cg);
            }
        Csr Pn;
        Pn.rows = (int)cur.gids.size();
        Pn.cols = nc;
        Pn.ptr.assign(Pn.rows + 1, 0);
        for (size_t r = 0; r < rows.size(); ++r) {
            std::vector<std::pair<int, double>> ent;
            for (auto& pr : rows[r]) ent.push_back({cid[pr.first], pr.second});
            std::sort(ent.begin(), ent.end());
            for (auto& pr : ent) {
                Pn.col.push_back(pr.first);
                Pn.val.push_back(pr.second);
            }
            Pn.ptr[r + 1] = (int)Pn.col.size();
        }
        if (nc >= (int)cur.gids.size()) {  // no coarsening possible: make this level the coarsest
            LevelC& last = H->levels.back();
            std::vector<double> Dm((size_t)last.n * last.n, 0.0);
            for (int r = 0; r < last.n; ++r)
                for (int k = last.a_ptr[r]; k < last.a_ptr[r + 1]; ++k) Dm[(size_t)r * last.n + last.a_col[k]] = last.a_val[k];
            if (!invert(Dm, last.n)) {
                err = "singular coarsest DSA operator";
                delete H;
                return nullptr;
            }
            last.dense_inv = Dm;
            break;
        }
        Acur = std::move(Ac);
        Pcur = std::move(Pn);
        cur = std::move(nxt);
    }
    return H;
}

}  // namespace sn
