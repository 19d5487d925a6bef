// CPU oracle of the transport update in plain C++ (test infrastructure and timed CPU baseline only;
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
// directions always runs in direction order.
#include <cmath>
#include <cstring>
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
    const int n = P.n, ne = P.ne;
    // modal source S = (q + sigma_s phi)/(4 pi)
    const double four_pi = 4.0 * M_PI;
    std::vector<double> phim((size_t)ne * n), src((size_t)ne * n);
    for (int e = 0; e < ne; ++e)
        for (int m = 0; m < n; ++m) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += P.Vinv[(size_t)m * n + k] * phi_in[(size_t)e * n + k];
            phim[(size_t)e * n + m] = s;
        }
    for (int e = 0; e < ne; ++e)
        for (int m = 0; m < n; ++m)
            src[(size_t)e * n + m] = (sigma_s[e] * phim[(size_t)e * n + m]) / four_pi + (m == 0 ? q[e] / four_pi : 0.0);
    const int nsweep = d_end - d_begin;
    std::vector<double> psi((size_t)nsweep * ne * n);
    int cycle = 0;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1) reduction(| : cycle)
#endif
    for (int t = 0; t < nsweep; ++t)
        if (!sweep_direction(P, d_begin + t, src.data(), &psi[(size_t)t * ne * n])) cycle = 1;
    if (cycle) return 1;
    std::vector<double> out((size_t)ne * n, 0.0);
    for (int t = 0; t < nsweep; ++t)  // in direction order
        for (size_t i = 0; i < out.size(); ++i) out[i] += w[d_begin + t] * psi[(size_t)t * ne * n + i];
    for (int e = 0; e < ne; ++e)
        for (int r = 0; r < n; ++r) {
            double s = 0.0;
            for (int m = 0; m < n; ++m) s += P.V[(size_t)r * n + m] * out[(size_t)e * n + m];
            phi_out[(size_t)e * n + r] = s;
        }
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
