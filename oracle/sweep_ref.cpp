// CPU oracle in plain C++: the transport update, the thick-subdomain DSA operator and source
// iteration with or without the Algorithm 2 step (test infrastructure and timed CPU baseline only;
// the product path never loads it).
//
// What it computes is the update of Sec. 1 (Eq. psi and Eq. phi) in the upwind DG discretisation of
// Sec. 3.1 (Eq. Tmat1), the same steps as oracle/transport.py and independent of the CUDA library:
//   for every direction d: psi_d = L_d^{-1}(M (q/(4 pi) + sigma_s phi/(4 pi)) - inflow terms), solved
//   element by element in a Kahn order of the upwind graph (Omega.n on each face), with
//     A_e = sigma_t M_e - (psi, Omega.grad v)_e + sum_{outflow faces} <(Omega.n) psi, v>,
//     rhs_e = M_e S_e - sum_{inflow faces} <(Omega.n) psi_up, v>  (psi_up = neighbour trace or psi_inc);
//   phi_half = sum_d w_d psi_d.
// Basis: tensor Legendre polynomials (modal), integrals by the (p+2)-point Gauss rule per axis, exact
// on bilinear (2D) and affine (3D) elements.  Element systems by Gaussian elimination with partial
// pivoting.  Input and output scalar fluxes are values at the (p+1)^dim Gauss-Legendre nodes
// ([elem][node], x fastest), converted to and from modal coefficients here.  The direction set and
// both 1D Gauss rules are inputs.  Directions may be swept in parallel (OpenMP); the sum over
// directions always runs in direction order.  The DSA operator (Eq. SIP on the thick elements,
// Sec. 3.1-3.2) and the source iteration (Eq. DSA_fp, Algorithm 2) follow oracle/dsa.py and
// oracle/transport.py; D_ff is solved by block-Jacobi conjugate gradients.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// P_m(x) and P_m'(x) by the three-term recurrence (m P_m = (2m-1) x P_{m-1} - (m-1) P_{m-2})
void legendre_all(int pmax, double x, double* P, double* dP) {
    P[0] = 1.0;
    dP[0] = 0.0;
    if (pmax >= 1) {
        P[1] = x;
        dP[1] = 1.0;
    }
    for (int m = 2; m <= pmax; ++m) {
        P[m] = ((2.0 * m - 1.0) * x * P[m - 1] - (m - 1.0) * P[m - 2]) / m;
        dP[m] = dP[m - 2] + (2.0 * m - 1.0) * P[m - 1];
    }
}

// Gaussian elimination with partial pivoting: solves A x = b (A n x n row-major, overwritten).
void solve_dense(int n, double* A, double* b) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
            std::swap(b[c], b[piv]);
        }
        for (int r = c + 1; r < n; ++r) {
            const double f = A[r * n + c] / A[c * n + c];
            if (f == 0.0) continue;
            for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= A[r * n + k] * b[k];
        b[r] = s / A[r * n + r];
    }
}

struct Problem {
    int dim, nx, ny, nz, p, n, Q, ne, nd;
    std::vector<double> verts;  // vertex coordinates ((nx+1)(ny+1)[(nz+1)] x dim)
    const double *dirs, *w, *st, *ss, *q;
    double psi_inc;
    // reference data: volume rule points/weights, face rule, basis values and gradients
    std::vector<double> vx, vw;       // volume points (nq x dim), weights
    std::vector<double> B, dB;        // basis at volume points (nq x n), gradients (nq x n x dim)
    std::vector<double> fx, fw;       // face points per face (2dim x nqf x dim), face weights (nqf)
    std::vector<double> BF, BFo;      // basis at face points on this side / the opposite side (2dim x nqf x n)
    std::vector<double> V;            // basis at the GL nodes (n x n): nodal = V modal
    std::vector<double> Vinv;
    // per element
    std::vector<int> nbr;             // ne x 2dim
    std::vector<double> M;            // ne x n x n
    std::vector<double> G;            // ne x dim x n x n: G_l[m][k] = -(B_k, d(v_m)/dx_l)
    std::vector<double> FN;           // ne x 2dim x nqf x dim: Omega.n dS = FN . Omega (Nanson)
    int nq, nqf;
};

// corner c of element e: vertex (i + bit0(c), j + bit1(c), k + bit2(c))
void map_point(const Problem& P, int e, const double* xi, double* x, double* J) {
    const int dim = P.dim, nvx = P.nx + 1, nvy = P.ny + 1;
    int ijk[3] = {e % P.nx, (e / P.nx) % P.ny, e / (P.nx * P.ny)};
    for (int r = 0; r < dim; ++r) {
        x[r] = 0.0;
        for (int c = 0; c < dim; ++c) J[r * dim + c] = 0.0;
    }
    for (int c = 0; c < (1 << dim); ++c) {
        double fac[3], s[3];
        int vid = 0, stride = 1;
        for (int a = 0; a < dim; ++a) {
            const int bit = (c >> a) & 1;
            s[a] = bit ? 1.0 : -1.0;
            fac[a] = 0.5 * (1.0 + s[a] * xi[a]);
            vid += (ijk[a] + bit) * stride;
            stride *= a == 0 ? nvx : nvy;
        }
        double Nc = 1.0;
        for (int a = 0; a < dim; ++a) Nc *= fac[a];
        for (int r = 0; r < dim; ++r) {
            const double X = P.verts[(size_t)vid * dim + r];
            x[r] += Nc * X;
            for (int a = 0; a < dim; ++a) {
                double o = 0.5 * s[a];
                for (int b = 0; b < dim; ++b)
                    if (b != a) o *= fac[b];
                J[r * dim + a] += o * X;
            }
        }
    }
}

double det(int dim, const double* J) {
    if (dim == 2) return J[0] * J[3] - J[1] * J[2];
    return J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) + J[2] * (J[3] * J[7] - J[4] * J[6]);
}

// adj(J) = det(J) J^{-1} (cofactor transpose)
void adjugate(int dim, const double* J, double* A) {
    if (dim == 2) {
        A[0] = J[3];
        A[1] = -J[1];
        A[2] = -J[2];
        A[3] = J[0];
        return;
    }
    A[0] = J[4] * J[8] - J[5] * J[7];
    A[1] = J[2] * J[7] - J[1] * J[8];
    A[2] = J[1] * J[5] - J[2] * J[4];
    A[3] = J[5] * J[6] - J[3] * J[8];
    A[4] = J[0] * J[8] - J[2] * J[6];
    A[5] = J[2] * J[3] - J[0] * J[5];
    A[6] = J[3] * J[7] - J[4] * J[6];
    A[7] = J[1] * J[6] - J[0] * J[7];
    A[8] = J[0] * J[4] - J[1] * J[3];
}

// basis values (n) and reference gradients (n x dim) at xi; mode k = (k_0, .., k_{dim-1}), x fastest
void basis(const Problem& P, const double* xi, double* val, double* grad) {
    double Pv[3][8], dPv[3][8];
    for (int a = 0; a < P.dim; ++a) legendre_all(P.p, xi[a], Pv[a], dPv[a]);
    for (int k = 0; k < P.n; ++k) {
        int md[3] = {k % P.Q, (k / P.Q) % P.Q, k / (P.Q * P.Q)};
        double v = 1.0;
        for (int a = 0; a < P.dim; ++a) v *= Pv[a][md[a]];
        val[k] = v;
        if (grad)
            for (int b = 0; b < P.dim; ++b) {
                double g = 1.0;
                for (int a = 0; a < P.dim; ++a) g *= (a == b ? dPv[a][md[a]] : Pv[a][md[a]]);
                grad[k * P.dim + b] = g;
            }
    }
}

void setup(Problem& P, const double* gx, const double* gw, const double* glx) {
    const int dim = P.dim, n = P.n, nqa = P.p + 2;
    P.nq = 1;
    P.nqf = 1;
    for (int a = 0; a < dim; ++a) P.nq *= nqa;
    for (int a = 0; a < dim - 1; ++a) P.nqf *= nqa;
    // volume rule, x fastest
    P.vx.resize((size_t)P.nq * dim);
    P.vw.resize(P.nq);
    for (int t = 0; t < P.nq; ++t) {
        int r = t;
        double wt = 1.0;
        for (int a = 0; a < dim; ++a) {
            P.vx[(size_t)t * dim + a] = gx[r % nqa];
            wt *= gw[r % nqa];
            r /= nqa;
        }
        P.vw[t] = wt;
    }
    P.B.resize((size_t)P.nq * n);
    P.dB.resize((size_t)P.nq * n * dim);
    for (int t = 0; t < P.nq; ++t) basis(P, &P.vx[(size_t)t * dim], &P.B[(size_t)t * n], &P.dB[(size_t)t * n * dim]);
    // face rules: face f = 2a + side, xi_a = -1 (side 0) or +1 (side 1), other coordinates in order
    P.fw.resize(P.nqf);
    P.fx.resize((size_t)2 * dim * P.nqf * dim);
    P.BF.resize((size_t)2 * dim * P.nqf * n);
    P.BFo.resize((size_t)2 * dim * P.nqf * n);
    for (int t = 0; t < P.nqf; ++t) {
        int r = t;
        double wt = 1.0;
        for (int b = 0; b < dim - 1; ++b) {
            wt *= gw[r % nqa];
            r /= nqa;
        }
        P.fw[t] = wt;
    }
    for (int f = 0; f < 2 * dim; ++f) {
        const int a = f / 2, side = f % 2;
        for (int t = 0; t < P.nqf; ++t) {
            double xi[3], xo[3];
            int r = t, b2 = 0;
            for (int b = 0; b < dim; ++b) {
                if (b == a) {
                    xi[b] = side ? 1.0 : -1.0;
                    xo[b] = side ? -1.0 : 1.0;
                } else {
                    xi[b] = xo[b] = gx[r % nqa];
                    r /= nqa;
                    ++b2;
                }
            }
            for (int b = 0; b < dim; ++b) P.fx[((size_t)f * P.nqf + t) * dim + b] = xi[b];
            basis(P, xi, &P.BF[((size_t)f * P.nqf + t) * n], nullptr);
            basis(P, xo, &P.BFo[((size_t)f * P.nqf + t) * n], nullptr);
        }
    }
    // nodal <-> modal
    P.V.resize((size_t)n * n);
    for (int t = 0; t < n; ++t) {
        double xi[3];
        int r = t;
        for (int a = 0; a < dim; ++a) {
            xi[a] = glx[r % P.Q];
            r /= P.Q;
        }
        basis(P, xi, &P.V[(size_t)t * n], nullptr);
    }
    P.Vinv.assign((size_t)n * n, 0.0);
    for (int c = 0; c < n; ++c) {  // column c of V^{-1}
        std::vector<double> A(P.V), b(n, 0.0);
        b[c] = 1.0;
        solve_dense(n, A.data(), b.data());
        for (int r = 0; r < n; ++r) P.Vinv[(size_t)r * n + c] = b[r];
    }
    // neighbours
    const int shape[3] = {P.nx, P.ny, P.nz};
    P.nbr.assign((size_t)P.ne * 2 * dim, -1);
    for (int e = 0; e < P.ne; ++e) {
        int ijk[3] = {e % P.nx, (e / P.nx) % P.ny, e / (P.nx * P.ny)};
        for (int a = 0; a < dim; ++a)
            for (int side = 0; side < 2; ++side) {
                int j[3] = {ijk[0], ijk[1], ijk[2]};
                j[a] += side ? 1 : -1;
                if (j[a] < 0 || j[a] >= shape[a]) continue;
                P.nbr[(size_t)e * 2 * dim + 2 * a + side] = j[0] + P.nx * (j[1] + P.ny * j[2]);
            }
    }
    // element integrals
    P.M.assign((size_t)P.ne * n * n, 0.0);
    P.G.assign((size_t)P.ne * dim * n * n, 0.0);
    P.FN.assign((size_t)P.ne * 2 * dim * P.nqf * dim, 0.0);
    for (int e = 0; e < P.ne; ++e) {
        double x[3], J[9], A[9];
        for (int t = 0; t < P.nq; ++t) {
            map_point(P, e, &P.vx[(size_t)t * dim], x, J);
            const double dJ = det(dim, J);
            adjugate(dim, J, A);
            const double* Bt = &P.B[(size_t)t * n];
            const double* dBt = &P.dB[(size_t)t * n * dim];
            for (int m = 0; m < n; ++m)
                for (int k = 0; k < n; ++k) {
                    P.M[((size_t)e * n + m) * n + k] += P.vw[t] * dJ * Bt[m] * Bt[k];
                    // -(psi, Omega.grad v) detJ = -psi sum_l Omega_l sum_c adj[c][l] dv/dxi_c
                    for (int l = 0; l < dim; ++l) {
                        double gv = 0.0;
                        for (int c = 0; c < dim; ++c) gv += A[c * dim + l] * dBt[m * dim + c];
                        P.G[(((size_t)e * dim + l) * n + m) * n + k] -= P.vw[t] * Bt[k] * gv;
                    }
                }
        }
        for (int f = 0; f < 2 * dim; ++f) {
            const int a = f / 2;
            const double s = (f % 2) ? 1.0 : -1.0;
            for (int t = 0; t < P.nqf; ++t) {
                map_point(P, e, &P.fx[((size_t)f * P.nqf + t) * dim], x, J);
                adjugate(dim, J, A);
                for (int r = 0; r < dim; ++r)
                    P.FN[(((size_t)e * 2 * dim + f) * P.nqf + t) * dim + r] = s * A[a * dim + r] * P.fw[t];
            }
        }
    }
}

// psi (ne x n modal) of direction d for the modal source src (ne x n); returns false on a cycle
bool sweep_direction(const Problem& P, int d, const double* src, double* psi) {
    const int dim = P.dim, n = P.n, nf = 2 * dim, ne = P.ne, nqf = P.nqf;
    const double* Om = P.dirs + 3 * d;
    // face fluxes Omega.n dS at face points and their sums
    std::vector<double> fw((size_t)ne * nf * nqf), fsum((size_t)ne * nf);
    for (int e = 0; e < ne; ++e)
        for (int f = 0; f < nf; ++f) {
            double tot = 0.0;
            for (int t = 0; t < nqf; ++t) {
                const double* N = &P.FN[(((size_t)e * nf + f) * nqf + t) * dim];
                double v = 0.0;
                for (int r = 0; r < dim; ++r) v += N[r] * Om[r];
                fw[((size_t)e * nf + f) * nqf + t] = v;
                tot += v;
            }
            fsum[(size_t)e * nf + f] = tot;
        }
    // Kahn order of the upwind graph
    std::vector<int> indeg(ne, 0), order;
    order.reserve(ne);
    for (int e = 0; e < ne; ++e)
        for (int f = 0; f < nf; ++f)
            if (fsum[(size_t)e * nf + f] < 0 && P.nbr[(size_t)e * nf + f] >= 0) ++indeg[e];
    for (int e = 0; e < ne; ++e)
        if (indeg[e] == 0) order.push_back(e);
    for (size_t h = 0; h < order.size(); ++h) {
        const int e = order[h];
        for (int f = 0; f < nf; ++f) {
            const int u = P.nbr[(size_t)e * nf + f];
            if (u >= 0 && fsum[(size_t)e * nf + f] > 0 && --indeg[u] == 0) order.push_back(u);
        }
    }
    if ((int)order.size() != ne) return false;
    std::vector<double> A((size_t)n * n), b(n), tr(nqf);
    for (int e : order) {
        const double* Me = &P.M[(size_t)e * n * n];
        for (int m = 0; m < n; ++m) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) {
                double a = P.st[e] * Me[m * n + k];
                for (int l = 0; l < dim; ++l) a += Om[l] * P.G[(((size_t)e * dim + l) * n + m) * n + k];
                A[m * n + k] = a;
                s += Me[m * n + k] * src[(size_t)e * n + k];
            }
            b[m] = s;
        }
        for (int f = 0; f < nf; ++f) {
            const double* wq = &fw[((size_t)e * nf + f) * nqf];
            const double* BFf = &P.BF[(size_t)f * nqf * n];
            if (fsum[(size_t)e * nf + f] > 0) {  // outflow face: <(Omega.n) psi, v>
                for (int t = 0; t < nqf; ++t)
                    for (int m = 0; m < n; ++m)
                        for (int k = 0; k < n; ++k) A[m * n + k] += wq[t] * BFf[t * n + m] * BFf[t * n + k];
            } else if (fsum[(size_t)e * nf + f] < 0) {  // inflow face: upwind trace
                const int u = P.nbr[(size_t)e * nf + f];
                const double* BFo = &P.BFo[(size_t)f * nqf * n];
                for (int t = 0; t < nqf; ++t) {
                    if (u >= 0) {
                        double v = 0.0;
                        for (int k = 0; k < n; ++k) v += BFo[t * n + k] * psi[(size_t)u * n + k];
                        tr[t] = v;
                    } else {
                        tr[t] = P.psi_inc;
                    }
                }
                for (int m = 0; m < n; ++m) {
                    double s = 0.0;
                    for (int t = 0; t < nqf; ++t) s += wq[t] * BFf[t * n + m] * tr[t];
                    b[m] -= s;
                }
            }
        }
        solve_dense(n, A.data(), b.data());
        for (int m = 0; m < n; ++m) psi[(size_t)e * n + m] = b[m];
    }
    return true;
}

void build_problem(Problem& P, int dim, int nx, int ny, int nz, int p, const double* vertices, int nd,
                   const double* dirs, const double* w, const double* sigma_t, const double* sigma_s, const double* q,
                   double psi_inc, const double* gx, const double* gw, const double* glx) {
    P.dim = dim;
    P.nx = nx;
    P.ny = ny;
    P.nz = dim == 3 ? nz : 1;
    P.p = p;
    P.Q = p + 1;
    P.n = dim == 2 ? P.Q * P.Q : P.Q * P.Q * P.Q;
    P.ne = nx * ny * P.nz;
    P.nd = nd;
    P.dirs = dirs;
    P.w = w;
    P.st = sigma_t;
    P.ss = sigma_s;
    P.q = q;
    P.psi_inc = psi_inc;
    const int nvx = nx + 1, nvy = ny + 1, nvz = dim == 3 ? nz + 1 : 1;
    P.verts.resize((size_t)nvx * nvy * nvz * dim);
    for (int k = 0; k < nvz; ++k)
        for (int j = 0; j < nvy; ++j)
            for (int i = 0; i < nvx; ++i) {
                const size_t v = (size_t)i + (size_t)nvx * (j + (size_t)nvy * k);
                for (int a = 0; a < dim; ++a) {
                    const int idx[3] = {i, j, k};
                    const int cnt[3] = {nx, ny, nz};
                    P.verts[v * dim + a] = vertices ? vertices[v * dim + a] : (double)idx[a] / cnt[a];
                }
            }
    setup(P, gx, gw, glx);
}

void to_modal(const Problem& P, const double* nodal, double* modal) {
    const int n = P.n;
    for (int e = 0; e < P.ne; ++e)
        for (int m = 0; m < n; ++m) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += P.Vinv[(size_t)m * n + k] * nodal[(size_t)e * n + k];
            modal[(size_t)e * n + m] = s;
        }
}

void to_nodal(const Problem& P, const double* modal, double* nodal) {
    const int n = P.n;
    for (int e = 0; e < P.ne; ++e)
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int m = 0; m < n; ++m) s += P.V[(size_t)r * n + m] * modal[(size_t)e * n + m];
            nodal[(size_t)e * n + r] = s;
        }
}

// The transport update (Eq. source0) in modal coefficients: out = sum over directions
// [d_begin, d_end) of w_d psi_d, psi_d = L_d^{-1}((q + sigma_s phi)/(4 pi)) with the boundary inflow;
// false if an upwind graph has a cycle.
bool update_modal(const Problem& P, const double* phim, double* out, int d_begin, int d_end, int threads) {
    const int n = P.n, ne = P.ne;
    const double four_pi = 4.0 * M_PI;
    std::vector<double> src((size_t)ne * n);
    for (int e = 0; e < ne; ++e)
        for (int m = 0; m < n; ++m)
            src[(size_t)e * n + m] = (P.ss[e] * phim[(size_t)e * n + m]) / four_pi + (m == 0 ? P.q[e] / four_pi : 0.0);
    const int nsweep = d_end - d_begin;
    std::vector<double> psi((size_t)nsweep * ne * n);
    int cycle = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : cycle)
#endif
    for (int t = 0; t < nsweep; ++t)
        if (!sweep_direction(P, d_begin + t, src.data(), &psi[(size_t)t * ne * n])) cycle = 1;
    if (cycle) return false;
    for (size_t i = 0; i < (size_t)ne * n; ++i) out[i] = 0.0;
    for (int t = 0; t < nsweep; ++t)  // in direction order
        for (size_t i = 0; i < (size_t)ne * n; ++i) out[i] += P.w[d_begin + t] * psi[(size_t)t * ne * n + i];
    return true;
}

// ---------------------------------------------------------------- thick-subdomain DSA (SIP)
// D_ff of Sec. 3.1-3.2 with the symmetric interior-penalty face terms (Eq. SIP, the conjugate-
// gradient path), restricted to the thick elements: for thick elements K and thick-thick faces F,
//   sum_K (D grad u, grad v)_K + (sigma_a u, v)_K
//   + sum_F <kappa [u],[v]> - <{D grad u.n},[v]> - <{D grad v.n},[u]>,
// D = 1/(3 sigma_t), sigma_a = sigma_t - sigma_s; a face whose neighbour is not thick is a face to a
// zero exterior state (jump = u, average = u/2); kappa_F = max(1/4, c(p) (D-/h- + D+/h+)/2),
// max(1/4, c(p) D/h) on boundary-type faces, c(p) = 2 p (p+1), h = |K|/|F|.  Integrals by the
// (p+1)-point Gauss rule per axis, the same as oracle/dsa.py.  Stored by block rows of thick
// elements: (column element, n x n block) pairs.
struct Dsa {
    int n = 0, nt = 0;
    std::vector<int> thick, local;                      // thick elements; local index (-1: not thick)
    std::vector<std::vector<std::pair<int, std::vector<double>>>> rows;
    std::vector<double> dinv;                           // inverses of the diagonal blocks (nt x n x n)
};

std::vector<double>& block_at(Dsa& D, int r, int c) {
    for (auto& pr : D.rows[r])
        if (pr.first == c) return pr.second;
    D.rows[r].push_back({c, std::vector<double>((size_t)D.n * D.n, 0.0)});
    return D.rows[r].back().second;
}

void inv3(int dim, const double* J, double* Ji) {  // inverse of a dim x dim matrix
    double A[9];
    adjugate(dim, J, A);
    const double dj = det(dim, J);
    for (int i = 0; i < dim * dim; ++i) Ji[i] = A[i] / dj;
}

void assemble_sip(const Problem& P, const unsigned char* mask, const double* gx1, const double* gw1, Dsa& D) {
    const int dim = P.dim, n = P.n, p = P.p, Q1 = p + 1;
    D.n = n;
    D.local.assign(P.ne, -1);
    for (int e = 0; e < P.ne; ++e)
        if (mask[e]) {
            D.local[e] = (int)D.thick.size();
            D.thick.push_back(e);
        }
    D.nt = (int)D.thick.size();
    D.rows.assign(D.nt, {});
    const double cp = 2.0 * p * (p + 1);
    // (p+1)-point rules: volume (x fastest) and faces
    int nq = 1, nqf = 1;
    for (int a = 0; a < dim; ++a) nq *= Q1;
    for (int a = 0; a < dim - 1; ++a) nqf *= Q1;
    std::vector<double> vx((size_t)nq * dim), vw(nq), B((size_t)nq * n), dB((size_t)nq * n * dim);
    for (int t = 0; t < nq; ++t) {
        int r = t;
        double wt = 1.0;
        for (int a = 0; a < dim; ++a) {
            vx[(size_t)t * dim + a] = gx1[r % Q1];
            wt *= gw1[r % Q1];
            r /= Q1;
        }
        vw[t] = wt;
        basis(P, &vx[(size_t)t * dim], &B[(size_t)t * n], &dB[(size_t)t * n * dim]);
    }
    // element volumes |K| with the same rule (every element: h of non-thick neighbours is not needed)
    std::vector<double> vol(P.ne, 0.0);
    for (int e = 0; e < P.ne; ++e) {
        double x[3], J[9];
        for (int t = 0; t < nq; ++t) {
            map_point(P, e, &vx[(size_t)t * dim], x, J);
            vol[e] += vw[t] * det(dim, J);
        }
    }
    auto Dc = [&](int e) { return 1.0 / (3.0 * P.st[e]); };
    // volume terms
    for (int lt = 0; lt < D.nt; ++lt) {
        const int e = D.thick[lt];
        const double De = Dc(e), sa = P.st[e] - P.ss[e];
        std::vector<double>& K = block_at(D, lt, lt);
        double x[3], J[9], Ji[9];
        std::vector<double> g((size_t)n * dim);
        for (int t = 0; t < nq; ++t) {
            map_point(P, e, &vx[(size_t)t * dim], x, J);
            const double dj = det(dim, J);
            inv3(dim, J, Ji);
            for (int m = 0; m < n; ++m)  // physical gradient: (J^{-T} grad_ref)_r = sum_c Jinv[c][r] d/dxi_c
                for (int r = 0; r < dim; ++r) {
                    double v = 0.0;
                    for (int c = 0; c < dim; ++c) v += Ji[c * dim + r] * dB[((size_t)t * n + m) * dim + c];
                    g[(size_t)m * dim + r] = v;
                }
            for (int m = 0; m < n; ++m)
                for (int k = 0; k < n; ++k) {
                    double gg = 0.0;
                    for (int r = 0; r < dim; ++r) gg += g[(size_t)m * dim + r] * g[(size_t)k * dim + r];
                    K[(size_t)m * n + k] += vw[t] * dj * (De * gg + sa * B[(size_t)t * n + m] * B[(size_t)t * n + k]);
                }
        }
    }
    // face terms
    std::vector<double> fwt(nqf), ft((size_t)nqf * (dim - 1 > 0 ? dim - 1 : 1));
    for (int t = 0; t < nqf; ++t) {
        int r = t;
        double wt = 1.0;
        for (int b = 0; b < dim - 1; ++b) {
            ft[(size_t)t * (dim - 1) + b] = gx1[r % Q1];
            wt *= gw1[r % Q1];
            r /= Q1;
        }
        fwt[t] = wt;
    }
    for (int lt = 0; lt < D.nt; ++lt) {
        const int e = D.thick[lt];
        for (int f = 0; f < 2 * dim; ++f) {
            const int a = f / 2, side = f % 2;
            const double s = side ? 1.0 : -1.0;
            const int u = P.nbr[(size_t)e * 2 * dim + f];
            const int ut = u >= 0 ? D.local[u] : -1;
            if (ut >= 0 && side == 0) continue;  // interior thick-thick faces from the side == 1 element
            // face points on this side (xi) and on the neighbour's side (xo), normals, weights
            std::vector<double> Bf((size_t)nqf * n), Bo((size_t)nqf * n), dn((size_t)nqf * n), dno((size_t)nqf * n),
                dS(nqf);
            double area = 0.0;
            for (int t = 0; t < nqf; ++t) {
                double xi[3], xo[3];
                int b2 = 0;
                for (int b = 0; b < dim; ++b) {
                    if (b == a) {
                        xi[b] = side ? 1.0 : -1.0;
                        xo[b] = side ? -1.0 : 1.0;
                    } else {
                        xi[b] = xo[b] = ft[(size_t)t * (dim - 1) + b2];
                        ++b2;
                    }
                }
                double x[3], J[9], A[9], Ji[9], dBf[27 * 8];
                basis(P, xi, &Bf[(size_t)t * n], dBf);
                map_point(P, e, xi, x, J);
                adjugate(dim, J, A);
                inv3(dim, J, Ji);
                double N[3], nn = 0.0;
                for (int r = 0; r < dim; ++r) {
                    N[r] = s * A[a * dim + r];
                    nn += N[r] * N[r];
                }
                nn = std::sqrt(nn);
                dS[t] = nn * fwt[t];
                area += dS[t];
                double nrm[3];
                for (int r = 0; r < dim; ++r) nrm[r] = N[r] / nn;
                for (int m = 0; m < n; ++m) {
                    double v = 0.0;
                    for (int r = 0; r < dim; ++r) {
                        double gr = 0.0;
                        for (int c = 0; c < dim; ++c) gr += Ji[c * dim + r] * dBf[m * dim + c];
                        v += gr * nrm[r];
                    }
                    dn[(size_t)t * n + m] = v;
                }
                if (ut >= 0) {  // the neighbour's basis and gradient at the same physical point
                    double Jo[9], Jio[9], dBo[27 * 8];
                    basis(P, xo, &Bo[(size_t)t * n], dBo);
                    map_point(P, u, xo, x, Jo);
                    inv3(dim, Jo, Jio);
                    for (int m = 0; m < n; ++m) {
                        double v = 0.0;
                        for (int r = 0; r < dim; ++r) {
                            double gr = 0.0;
                            for (int c = 0; c < dim; ++c) gr += Jio[c * dim + r] * dBo[m * dim + c];
                            v += gr * nrm[r];
                        }
                        dno[(size_t)t * n + m] = v;
                    }
                }
            }
            const double De = Dc(e), he = vol[e] / area;
            if (ut < 0) {  // boundary-type face: <kappa u, v> - 1/2 <D du/dn, v> - 1/2 <D dv/dn, u>
                const double kap = std::max(0.25, cp * De / he);
                std::vector<double>& K = block_at(D, lt, lt);
                for (int t = 0; t < nqf; ++t)
                    for (int m = 0; m < n; ++m)
                        for (int k = 0; k < n; ++k)
                            K[(size_t)m * n + k] += dS[t] * (kap * Bf[(size_t)t * n + m] * Bf[(size_t)t * n + k] -
                                                             0.5 * De * dn[(size_t)t * n + k] * Bf[(size_t)t * n + m] -
                                                             0.5 * De * dn[(size_t)t * n + m] * Bf[(size_t)t * n + k]);
                continue;
            }
            const double Do = Dc(u), ho = vol[u] / area;
            const double kap = std::max(0.25, cp * 0.5 * (De / he + Do / ho));
            struct Side {
                int row;
                const double *Bv, *dnv;
                double Dv, sg;
            };
            const Side sides[2] = {{lt, Bf.data(), dn.data(), De, 1.0}, {ut, Bo.data(), dno.data(), Do, -1.0}};
            for (const Side& ra : sides)
                for (const Side& cb : sides) {
                    std::vector<double>& K = block_at(D, ra.row, cb.row);
                    for (int t = 0; t < nqf; ++t)
                        for (int m = 0; m < n; ++m)
                            for (int k = 0; k < n; ++k)
                                K[(size_t)m * n + k] +=
                                    dS[t] * (kap * ra.sg * cb.sg * ra.Bv[(size_t)t * n + m] * cb.Bv[(size_t)t * n + k] -
                                             0.5 * cb.Dv * ra.sg * cb.dnv[(size_t)t * n + k] * ra.Bv[(size_t)t * n + m] -
                                             0.5 * ra.Dv * cb.sg * ra.dnv[(size_t)t * n + m] * cb.Bv[(size_t)t * n + k]);
                }
        }
    }
    // inverses of the diagonal blocks (block-Jacobi preconditioner of the conjugate gradients)
    D.dinv.assign((size_t)D.nt * n * n, 0.0);
    for (int lt = 0; lt < D.nt; ++lt) {
        const std::vector<double>& K = block_at(D, lt, lt);
        for (int c = 0; c < n; ++c) {
            std::vector<double> A(K), b(n, 0.0);
            b[c] = 1.0;
            solve_dense(n, A.data(), b.data());
            for (int r = 0; r < n; ++r) D.dinv[((size_t)lt * n + r) * n + c] = b[r];
        }
    }
}

void dsa_apply(const Dsa& D, const double* x, double* y) {  // y = D_ff x
    const int n = D.n;
    for (int r = 0; r < D.nt; ++r) {
        double* yr = y + (size_t)r * n;
        for (int m = 0; m < n; ++m) yr[m] = 0.0;
        for (const auto& pr : D.rows[r]) {
            const double* xc = x + (size_t)pr.first * n;
            for (int m = 0; m < n; ++m)
                for (int k = 0; k < n; ++k) yr[m] += pr.second[(size_t)m * n + k] * xc[k];
        }
    }
}

// D_ff x = b by block-Jacobi-preconditioned conjugate gradients to ||b - D x|| <= tol ||b||
int dsa_solve(const Dsa& D, const double* b, double* x, double tol, int max_iters) {
    const size_t N = (size_t)D.nt * D.n;
    const int n = D.n;
    std::vector<double> r(b, b + N), z(N), p(N), q(N);
    for (size_t i = 0; i < N; ++i) x[i] = 0.0;
    auto dot = [&](const std::vector<double>& a, const std::vector<double>& c) {
        double s = 0.0;
        for (size_t i = 0; i < N; ++i) s += a[i] * c[i];
        return s;
    };
    auto precond = [&]() {
        for (int e = 0; e < D.nt; ++e)
            for (int m = 0; m < n; ++m) {
                double s = 0.0;
                for (int k = 0; k < n; ++k) s += D.dinv[((size_t)e * n + m) * n + k] * r[(size_t)e * n + k];
                z[(size_t)e * n + m] = s;
            }
    };
    const double bb = dot(r, r);
    if (bb == 0.0) return 0;
    precond();
    p = z;
    double rz = dot(r, z);
    int it = 0;
    while (it < max_iters) {
        dsa_apply(D, p.data(), q.data());
        const double alpha = rz / dot(p, q);
        for (size_t i = 0; i < N; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        ++it;
        if (dot(r, r) <= tol * tol * bb) break;
        precond();
        const double rz2 = dot(r, z);
        const double beta = rz2 / rz;
        rz = rz2;
        for (size_t i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
    return it;
}

}  // namespace

extern "C" {

// Transport update phi_out = sum over directions [d_begin, d_end) of w_d psi_d (Eq. phi) for
// nodal phi_in; returns 0, or 1 if an upwind graph has a cycle.  vertices: NULL for the uniform
// grid of the unit square/cube.  gx, gw: the (p+2)-point Gauss rule; glx: the (p+1) Gauss-Legendre
// nodes.  threads: OpenMP threads over directions (<= 0: the runtime's default).
int sno_sweep(int dim, int nx, int ny, int nz, int p, const double* vertices, int nd, const double* dirs,
              const double* w, const double* sigma_t, const double* sigma_s, const double* q, double psi_inc,
              const double* gx, const double* gw, const double* glx, const double* phi_in, double* phi_out,
              int d_begin, int d_end, int threads) {
    Problem P;
    build_problem(P, dim, nx, ny, nz, p, vertices, nd, dirs, w, sigma_t, sigma_s, q, psi_inc, gx, gw, glx);
    std::vector<double> phim((size_t)P.ne * P.n), out((size_t)P.ne * P.n);
    to_modal(P, phi_in, phim.data());
    if (!update_modal(P, phim.data(), out.data(), d_begin, d_end, threads)) return 1;
    to_nodal(P, out.data(), phi_out);
    return 0;
}

// The thick-subdomain DSA operator D_ff (SIP) in the modal basis as a dense matrix of the thick
// elements' coefficients (nt n x nt n, row-major; small problems only).  gx1, gw1: the (p+1)-point
// Gauss rule.  Returns nt.
int sno_dsa_matrix(int dim, int nx, int ny, int nz, int p, const double* vertices, const double* sigma_t,
                   const double* sigma_s, const unsigned char* mask, const double* gx, const double* gw,
                   const double* glx, const double* gx1, const double* gw1, double* out) {
    Problem P;
    const double dir0[3] = {0.0, 0.0, 1.0}, w0 = 1.0;
    build_problem(P, dim, nx, ny, nz, p, vertices, 1, dir0, &w0, sigma_t, sigma_s, sigma_t, 0.0, gx, gw, glx);
    Dsa D;
    assemble_sip(P, mask, gx1, gw1, D);
    const size_t N = (size_t)D.nt * D.n;
    if (out) {
        for (size_t i = 0; i < N * N; ++i) out[i] = 0.0;
        for (int r = 0; r < D.nt; ++r)
            for (const auto& pr : D.rows[r])
                for (int m = 0; m < D.n; ++m)
                    for (int k = 0; k < D.n; ++k)
                        out[((size_t)r * D.n + m) * N + (size_t)pr.first * D.n + k] = pr.second[(size_t)m * D.n + k];
    }
    return D.nt;
}

// Source iteration (Eq. DSA_fp) from phi = 0: phi_half = T phi + b (the transport update),
// r = phi_half - phi, then phi = phi_half, or with a thick mask phi = phi_half + E_f D_ff^{-1}
// Sigma_f r_f (Algorithm 2, Sigma = sigma_s M, D_ff the SIP operator above solved by conjugate
// gradients to cg_tol); stops after the iteration whose ||r|| (Euclidean, GL-nodal values) is at most
// tol ||r^0||, or after max_iters.  phi_out: nodal.  Returns 0, 1 on a cycle.
int sno_source_iterate(int dim, int nx, int ny, int nz, int p, const double* vertices, int nd, const double* dirs,
                       const double* w, const double* sigma_t, const double* sigma_s, const double* q,
                       double psi_inc, const double* gx, const double* gw, const double* glx, const double* gx1,
                       const double* gw1, const unsigned char* mask, double tol, int max_iters, double cg_tol,
                       double* phi_out, int* iters, double* rel_out, int threads) {
    Problem P;
    build_problem(P, dim, nx, ny, nz, p, vertices, nd, dirs, w, sigma_t, sigma_s, q, psi_inc, gx, gw, glx);
    const int n = P.n, ne = P.ne;
    Dsa D;
    const bool use_dsa = mask != nullptr;
    if (use_dsa) assemble_sip(P, mask, gx1, gw1, D);
    std::vector<double> phi((size_t)ne * n, 0.0), half((size_t)ne * n), r((size_t)ne * n), rn((size_t)ne * n);
    std::vector<double> rhs((size_t)D.nt * n), corr((size_t)D.nt * n);
    double r0 = -1.0, rel = INFINITY;
    int it = 0;
    while (it < max_iters) {
        if (!update_modal(P, phi.data(), half.data(), 0, P.nd, threads)) return 1;
        for (size_t i = 0; i < r.size(); ++i) r[i] = half[i] - phi[i];
        to_nodal(P, r.data(), rn.data());
        double nrm = 0.0;
        for (double v : rn) nrm += v * v;
        nrm = std::sqrt(nrm);
        if (r0 < 0.0) r0 = nrm > 0.0 ? nrm : 1.0;
        rel = nrm / r0;
        phi = half;
        if (use_dsa && D.nt > 0) {  // Sigma_f r_f = sigma_s M r on the thick elements
            for (int lt = 0; lt < D.nt; ++lt) {
                const int e = D.thick[lt];
                for (int m = 0; m < n; ++m) {
                    double s = 0.0;
                    for (int k = 0; k < n; ++k) s += P.M[((size_t)e * n + m) * n + k] * r[(size_t)e * n + k];
                    rhs[(size_t)lt * n + m] = P.ss[e] * s;
                }
            }
            dsa_solve(D, rhs.data(), corr.data(), cg_tol, 100000);
            for (int lt = 0; lt < D.nt; ++lt)
                for (int m = 0; m < n; ++m) phi[(size_t)D.thick[lt] * n + m] += corr[(size_t)lt * n + m];
        }
        ++it;
        if (rel <= tol) break;
    }
    to_nodal(P, phi.data(), phi_out);
    if (iters) *iters = it;
    if (rel_out) *rel_out = rel;
    return 0;
}

int sno_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
