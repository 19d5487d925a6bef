// Upwind DG S_N sweep kernels for sm_103a.
//
// Discretisation (paper Sec. 1, Eq. sntransport; Sec. 3.1, Eq. Tmat1): on element K and
// direction Omega, with Q_p nodal basis at the (p+1)^dim tensor Gauss-Legendre points,
//   -(psi, Omega.grad v)_K + (sigma_t psi, v)_K + sum_{F outflow} <(Omega.n) psi, v>_F
//        = (S, v)_K - sum_{F inflow} <(Omega.n) psi_up, v>_F,   S = (q + sigma_s phi)/(4 pi).
// Gauss-Legendre collocation integrates every term exactly on bilinear (2D) and affine
// (3D) elements, so the mass matrix is diagonal, M_i = W_i det J(x_i), and the advection
// couples only nodes on a common coordinate line.  With b = adj(J) Omega (the contravariant
// flux; for a bilinear map b_1 depends on xi only and b_2 on eta only):
//   A_ij = sigma_t M_i delta_ij - W_j b(x_j) . grad_ref l_i(x_j) + outflow face terms.
// The face flux factor of face (axis a, side s) is F = s b_a evaluated on the face; it is
// computed from the element's edge vectors so that a face gives exactly -F to its neighbour.
// The transport update (Sec. 1) solves the element systems in upwind order: per direction,
// Kahn level sets are built on the device, and every level of every direction is one
// launch of thread-per-(element, direction) work in which each thread forms A_e in
// registers and solves it by unpivoted LU (A_e has a positive definite symmetric part,
// (sigma_t u,u) + 1/2 <|Omega.n| u, u>, so every leading minor is nonsingular).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <utility>
#include <cstdio>
#include <vector>

#include "sn_internal.h"

namespace sn {

__constant__ double c_x[kMaxP + 1][kMaxP + 1];
__constant__ double c_w[kMaxP + 1][kMaxP + 1];
__constant__ double c_lm[kMaxP + 1][kMaxP + 1];
__constant__ double c_lp[kMaxP + 1][kMaxP + 1];
__constant__ double c_dm[kMaxP + 1][kMaxP + 1][kMaxP + 1];
__constant__ double c_wdm[kMaxP + 1][kMaxP + 1][kMaxP + 1];  // w_a * l_k'(x_a)
__constant__ float c_wf[kMaxP + 1][kMaxP + 1];
__constant__ float c_lmf[kMaxP + 1][kMaxP + 1];
__constant__ float c_lpf[kMaxP + 1][kMaxP + 1];
__constant__ float c_wdmf[kMaxP + 1][kMaxP + 1][kMaxP + 1];

cudaError_t upload_face_coefficients();

cudaError_t upload_gl_constants() {
    double x[kMaxP + 1][kMaxP + 1] = {}, w[kMaxP + 1][kMaxP + 1] = {}, lm[kMaxP + 1][kMaxP + 1] = {},
           lp[kMaxP + 1][kMaxP + 1] = {}, dm[kMaxP + 1][kMaxP + 1][kMaxP + 1] = {},
           wdm[kMaxP + 1][kMaxP + 1][kMaxP + 1] = {};
    float wf[kMaxP + 1][kMaxP + 1] = {}, lmf[kMaxP + 1][kMaxP + 1] = {}, lpf[kMaxP + 1][kMaxP + 1] = {},
          wdmf[kMaxP + 1][kMaxP + 1][kMaxP + 1] = {};
    for (int p = 1; p <= kMaxP; ++p) {
        GL1D g = gauss_legendre_nodal(p);
        for (int k = 0; k <= p; ++k) {
            x[p][k] = g.x[k];
            w[p][k] = g.w[k];
            lm[p][k] = g.lm[k];
            lp[p][k] = g.lp[k];
            wf[p][k] = (float)g.w[k];
            lmf[p][k] = (float)g.lm[k];
            lpf[p][k] = (float)g.lp[k];
            for (int a = 0; a <= p; ++a) {
                dm[p][a][k] = g.dm[a][k];
                wdm[p][a][k] = g.w[a] * g.dm[a][k];
                wdmf[p][a][k] = (float)(g.w[a] * g.dm[a][k]);
            }
        }
    }
    cudaError_t err;
    if ((err = cudaMemcpyToSymbol(c_x, x, sizeof(x))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(c_w, w, sizeof(w))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(c_lm, lm, sizeof(lm))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(c_lp, lp, sizeof(lp))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(c_dm, dm, sizeof(dm))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(c_wdm, wdm, sizeof(wdm))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(c_wf, wf, sizeof(wf))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(c_lmf, lmf, sizeof(lmf))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(c_lpf, lpf, sizeof(lpf))) != cudaSuccess) return err;
    if ((err = cudaMemcpyToSymbol(c_wdmf, wdmf, sizeof(wdmf))) != cudaSuccess) return err;
    return upload_face_coefficients();
}

// Gauss-Legendre tables in the arithmetic type of a kernel.
template <typename R>
struct GLT;
template <>
struct GLT<double> {
    static __device__ __forceinline__ double w(int p, int k) { return c_w[p][k]; }
    static __device__ __forceinline__ double lm(int p, int k) { return c_lm[p][k]; }
    static __device__ __forceinline__ double lp(int p, int k) { return c_lp[p][k]; }
    static __device__ __forceinline__ double wdm(int p, int a, int k) { return c_wdm[p][a][k]; }
};
template <>
struct GLT<float> {
    static __device__ __forceinline__ float w(int p, int k) { return c_wf[p][k]; }
    static __device__ __forceinline__ float lm(int p, int k) { return c_lmf[p][k]; }
    static __device__ __forceinline__ float lp(int p, int k) { return c_lpf[p][k]; }
    static __device__ __forceinline__ float wdm(int p, int a, int k) { return c_wdmf[p][a][k]; }
};

template <int DIM, int P>
struct Shape {
    static constexpr int Q = P + 1;
    static constexpr int N = DIM == 2 ? Q * Q : Q * Q * Q;
    static constexpr int NT = DIM == 2 ? Q : Q * Q;  // nodes on a face
};

// Node index of the node with coordinate index ia on axis a and tangential index t.
template <int DIM, int P>
__device__ __forceinline__ int node_of(int a, int ia, int t) {
    constexpr int Q = P + 1;
    if (DIM == 2) return a == 0 ? ia + Q * t : t + Q * ia;
    const int t0 = t % Q, t1 = t / Q;
    if (a == 0) return ia + Q * (t0 + Q * t1);
    if (a == 1) return t0 + Q * (ia + Q * t1);
    return t0 + Q * (t1 + Q * ia);
}

template <int DIM, int P, typename R = double>
__device__ __forceinline__ R wtan(int t) {
    constexpr int Q = P + 1;
    return DIM == 2 ? GLT<R>::w(P, t) : GLT<R>::w(P, t % Q) * GLT<R>::w(P, t / Q);
}

// Geometry of one element for one direction, in arithmetic type R: face flux factors (the
// float64 value Fd decides inflow/outflow for every precision), b at the nodes and the
// collocated masses W_i det J(x_i) (precomputed per element in float64).
template <int DIM, int P, typename R>
struct ElemGeom {
    double Fd[2 * DIM];
    R F[2 * DIM];
    R b[DIM][P + 1];  // 2D: b[0][a] = b_1(x_a), b[1][a] = b_2(x_a); 3D: constant per axis
    R mass[Shape<DIM, P>::N];
};

// Face flux factor of a 2D face from the half edge vector (ex, ey), rounded without FMA
// contraction so that the level-set build and the sweep see the same value, and a face gives
// exactly the negated value to its neighbour (which computes it from the same vertices).
__device__ __forceinline__ double edge_flux(double Ox, double Oy, double ex, double ey) {
    return __dsub_rn(__dmul_rn(Ox, ey), __dmul_rn(Oy, ex));
}

__device__ __forceinline__ double face_flux_2d(const double* v, int f, double Ox, double Oy) {
    // v = x00 y00 x10 y10 x01 y01 x11 y11; faces 0: xi=-1 (left), 1: xi=+1, 2: eta=-1, 3: eta=+1
    switch (f) {
        case 0: return -edge_flux(Ox, Oy, 0.5 * (v[4] - v[0]), 0.5 * (v[5] - v[1]));
        case 1: return edge_flux(Ox, Oy, 0.5 * (v[6] - v[2]), 0.5 * (v[7] - v[3]));
        case 2: return edge_flux(Ox, Oy, 0.5 * (v[2] - v[0]), 0.5 * (v[3] - v[1]));
        default: return -edge_flux(Ox, Oy, 0.5 * (v[6] - v[4]), 0.5 * (v[7] - v[5]));
    }
}

template <int DIM, int P, typename R>
__device__ __forceinline__ void elem_geom(const SweepArgs& a, int e, double Ox, double Oy, double Oz,
                                          ElemGeom<DIM, P, R>& g) {
    constexpr int Q = P + 1, N = Shape<DIM, P>::N;
    if constexpr (DIM == 2) {
        const double* v = a.corners + 8 * (size_t)e;
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            g.Fd[f] = face_flux_2d(v, f, Ox, Oy);
            g.F[f] = (R)g.Fd[f];
        }
        // b_1(xi) interpolates Omega x (dx/deta) between the left and right edges, b_2(eta) likewise
        const R cl = -g.F[0], cr = g.F[1], cb = g.F[2], ct = -g.F[3];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const R t = (R)c_x[P][k];
            g.b[0][k] = R(0.5) * (R(1) - t) * cl + R(0.5) * (R(1) + t) * cr;
            g.b[1][k] = -(R(0.5) * (R(1) - t) * cb + R(0.5) * (R(1) + t) * ct);
        }
    } else {
        const double bx = 0.25 * Ox * a.hy * a.hz, by = 0.25 * Oy * a.hx * a.hz, bz = 0.25 * Oz * a.hx * a.hy;
        g.Fd[0] = -bx;
        g.Fd[1] = bx;
        g.Fd[2] = -by;
        g.Fd[3] = by;
        g.Fd[4] = -bz;
        g.Fd[5] = bz;
#pragma unroll
        for (int f = 0; f < 6; ++f) g.F[f] = (R)g.Fd[f];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            g.b[0][k] = (R)bx;
            g.b[1][k] = (R)by;
            g.b[2][k] = (R)bz;
        }
    }
    const double* ms = a.mass + (size_t)e * N;
#pragma unroll
    for (int i = 0; i < N; ++i) g.mass[i] = (R)ms[i];
}

template <int DIM, int P>
__device__ __forceinline__ void narrow_geom(const ElemGeom<DIM, P, double>& gd, ElemGeom<DIM, P, float>& gf) {
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        gf.Fd[f] = gd.Fd[f];
        gf.F[f] = (float)gd.F[f];
    }
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int k = 0; k <= P; ++k) gf.b[a][k] = (float)gd.b[a][k];
#pragma unroll
    for (int i = 0; i < Shape<DIM, P>::N; ++i) gf.mass[i] = (float)gd.mass[i];
}

// Collocated masses W_i det J(x_i) of every element (float64, once per mesh).
template <int DIM, int P>
__global__ void mass_kernel(SweepArgs a, double* mass, double* mass4) {
    constexpr int Q = P + 1, N = Shape<DIM, P>::N;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)a.ne * N) return;
    const int e = (int)(idx / N), i = (int)(idx % N);
    const int i0 = i % Q, i1 = (i / Q) % Q, i2 = i / (Q * Q);
    const double W = c_w[P][i0] * c_w[P][i1] * (DIM == 3 ? c_w[P][i2] : 1.0);
    double dj;
    if constexpr (DIM == 2) {
        const double* v = a.corners + 8 * (size_t)e;
        const double ebx = 0.5 * (v[2] - v[0]), eby = 0.5 * (v[3] - v[1]);
        const double etx = 0.5 * (v[6] - v[4]), ety = 0.5 * (v[7] - v[5]);
        const double elx = 0.5 * (v[4] - v[0]), ely = 0.5 * (v[5] - v[1]);
        const double erx = 0.5 * (v[6] - v[2]), ery = 0.5 * (v[7] - v[3]);
        const double xi = c_x[P][i0], eta = c_x[P][i1];
        const double xx = 0.5 * (1.0 - eta) * ebx + 0.5 * (1.0 + eta) * etx;  // dx/dxi
        const double xy = 0.5 * (1.0 - eta) * eby + 0.5 * (1.0 + eta) * ety;
        const double yx = 0.5 * (1.0 - xi) * elx + 0.5 * (1.0 + xi) * erx;    // dx/deta
        const double yy = 0.5 * (1.0 - xi) * ely + 0.5 * (1.0 + xi) * ery;
        dj = xx * yy - yx * xy;
    } else {
        dj = 0.125 * a.hx * a.hy * a.hz;
    }
    mass[idx] = W * dj;
    mass4[idx] = W * dj * (1.0 / kFourPi);  // the source row's scale, M_i / (4 pi)
}

template <int DIM, int P>
__device__ __forceinline__ int neighbor(const SweepArgs& a, int e, int f) {
    const int ax = f >> 1, side = f & 1;
    int i = e % a.nx, j = (e / a.nx) % a.ny, k = e / (a.nx * a.ny);
    const int dl = side ? 1 : -1;
    if (ax == 0) {
        i += dl;
        if (i < 0 || i >= a.nx) return -1;
    } else if (ax == 1) {
        j += dl;
        if (j < 0 || j >= a.ny) return -1;
    } else {
        k += dl;
        if (k < 0 || k >= a.nz) return -1;
    }
    return i + a.nx * (j + a.ny * k);
}

template <int DIM, int P>
__device__ __forceinline__ double face_flux_only(const SweepArgs& a, int e, int f, double Ox, double Oy,
                                                 double Oz) {
    if constexpr (DIM == 2) {
        return face_flux_2d(a.corners + 8 * (size_t)e, f, Ox, Oy);
    } else {
        const double bx = 0.25 * Ox * a.hy * a.hz, by = 0.25 * Oy * a.hx * a.hz, bz = 0.25 * Oz * a.hx * a.hy;
        const double b = (f >> 1) == 0 ? bx : ((f >> 1) == 1 ? by : bz);
        return (f & 1) ? b : -b;
    }
}

// A_e in arithmetic type R (volume + outflow faces); every entry is one FMA on table values.
template <int DIM, int P, typename R>
__device__ __forceinline__ void assemble(const ElemGeom<DIM, P, R>& g, R st, R* A) {
    constexpr int Q = P + 1, N = Shape<DIM, P>::N, NT = Shape<DIM, P>::NT;
    using K = GLT<R>;
#pragma unroll
    for (int i = 0; i < N * N; ++i) A[i] = R(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int j0 = j % Q, j1 = (j / Q) % Q, j2 = j / (Q * Q);
        const R w0 = K::w(P, j0), w1 = K::w(P, j1), w2 = DIM == 3 ? K::w(P, j2) : R(1);
        A[j * N + j] += st * g.mass[j];
        // -W_j b(x_j) . grad_ref l_i(x_j): nodes i on the coordinate lines through j
        const R u0 = w1 * w2 * g.b[0][j0];
#pragma unroll
        for (int ia = 0; ia < Q; ++ia) A[(ia + Q * (j1 + Q * j2)) * N + j] -= u0 * K::wdm(P, j0, ia);
        const R u1 = w0 * w2 * g.b[1][j1];
#pragma unroll
        for (int ia = 0; ia < Q; ++ia) A[(j0 + Q * (ia + Q * j2)) * N + j] -= u1 * K::wdm(P, j1, ia);
        if constexpr (DIM == 3) {
            const R u2 = w0 * w1 * g.b[DIM - 1][j2];
#pragma unroll
            for (int ia = 0; ia < Q; ++ia) A[(j0 + Q * (j1 + Q * ia)) * N + j] -= u2 * K::wdm(P, j2, ia);
        }
    }
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        if (g.Fd[f] > 0.0) {
            const int ax = f >> 1;
            const bool hi = f & 1;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const R ft = g.F[f] * wtan<DIM, P, R>(t);
#pragma unroll
                for (int ia = 0; ia < Q; ++ia) {
                    const R fi = ft * (hi ? K::lp(P, ia) : K::lm(P, ia));
#pragma unroll
                    for (int ja = 0; ja < Q; ++ja)
                        A[node_of<DIM, P>(ax, ia, t) * N + node_of<DIM, P>(ax, ja, t)] += fi * (hi ? K::lp(P, ja) : K::lm(P, ja));
                }
            }
        }
    }
}

// y = A_e x, matrix free, in float64 (the residual of the refinement step).
template <int DIM, int P>
__device__ __forceinline__ void apply_A(const ElemGeom<DIM, P, double>& g, double st, const double* x, double* y) {
    constexpr int Q = P + 1, N = Shape<DIM, P>::N, NT = Shape<DIM, P>::NT;
    using K = GLT<double>;
#pragma unroll
    for (int i = 0; i < N; ++i) y[i] = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int j0 = j % Q, j1 = (j / Q) % Q, j2 = j / (Q * Q);
        const double w0 = K::w(P, j0), w1 = K::w(P, j1), w2 = DIM == 3 ? K::w(P, j2) : 1.0;
        const double xj = x[j];
        y[j] += st * g.mass[j] * xj;
        const double u0 = w1 * w2 * g.b[0][j0] * xj, u1 = w0 * w2 * g.b[1][j1] * xj;
#pragma unroll
        for (int ia = 0; ia < Q; ++ia) y[ia + Q * (j1 + Q * j2)] -= u0 * K::wdm(P, j0, ia);
#pragma unroll
        for (int ia = 0; ia < Q; ++ia) y[j0 + Q * (ia + Q * j2)] -= u1 * K::wdm(P, j1, ia);
        if constexpr (DIM == 3) {
            const double u2 = w0 * w1 * g.b[DIM - 1][j2] * xj;
#pragma unroll
            for (int ia = 0; ia < Q; ++ia) y[j0 + Q * (j1 + Q * ia)] -= u2 * K::wdm(P, j2, ia);
        }
    }
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        if (g.Fd[f] > 0.0) {
            const int ax = f >> 1;
            const bool hi = f & 1;
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                double tr = 0.0;
#pragma unroll
                for (int ja = 0; ja < Q; ++ja) tr += (hi ? K::lp(P, ja) : K::lm(P, ja)) * x[node_of<DIM, P>(ax, ja, t)];
                const double ft = g.F[f] * wtan<DIM, P, double>(t) * tr;
#pragma unroll
                for (int ia = 0; ia < Q; ++ia) y[node_of<DIM, P>(ax, ia, t)] += ft * (hi ? K::lp(P, ia) : K::lm(P, ia));
            }
        }
    }
}

// Structural nonzeros of A_e after unpivoted elimination.  A_e couples only nodes that differ
// in at most one tensor index (mass, line advection, face terms), so part of L and U stays zero;
// the table is evaluated at compile time and the factor/solve loops skip those entries.
template <int DIM, int P>
struct LuPattern {
    static constexpr int Q = P + 1;
    static constexpr int N = DIM == 2 ? Q * Q : Q * Q * Q;
    struct Table {
        unsigned rows[N];  // bit j of rows[i]: entry (i, j) may be nonzero
    };
    __host__ __device__ static constexpr Table build() {
        Table t{};
        for (int i = 0; i < N; ++i) {
            t.rows[i] = 0u;
            for (int j = 0; j < N; ++j) {
                int diff = 0;
                int a = i, b = j;
                for (int ax = 0; ax < DIM; ++ax) {
                    diff += (a % Q) != (b % Q);
                    a /= Q;
                    b /= Q;
                }
                if (diff <= 1) t.rows[i] |= 1u << j;
            }
        }
        for (int k = 0; k < N; ++k)
            for (int i = k + 1; i < N; ++i)
                if ((t.rows[i] >> k) & 1u)
                    for (int j = k + 1; j < N; ++j)
                        if ((t.rows[k] >> j) & 1u) t.rows[i] |= 1u << j;
        return t;
    }
};

template <int DIM, int P, typename R>
__device__ __forceinline__ void lu_factor_s(R* A) {
    constexpr int N = LuPattern<DIM, P>::N;
    constexpr typename LuPattern<DIM, P>::Table pat = LuPattern<DIM, P>::build();
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const R inv = R(1) / A[k * N + k];
        A[k * N + k] = inv;
#pragma unroll
        for (int i = k + 1; i < N; ++i) {
            if (!((pat.rows[i] >> k) & 1u)) continue;
            const R l = A[i * N + k] * inv;
            A[i * N + k] = l;
#pragma unroll
            for (int j = k + 1; j < N; ++j)
                if ((pat.rows[k] >> j) & 1u) A[i * N + j] -= l * A[k * N + j];
        }
    }
}

template <int DIM, int P, typename R>
__device__ __forceinline__ void lu_solve_s(const R* A, R* x) {
    constexpr int N = LuPattern<DIM, P>::N;
    constexpr typename LuPattern<DIM, P>::Table pat = LuPattern<DIM, P>::build();
#pragma unroll
    for (int i = 1; i < N; ++i)
#pragma unroll
        for (int k = 0; k < i; ++k)
            if ((pat.rows[i] >> k) & 1u) x[i] -= A[i * N + k] * x[k];
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
#pragma unroll
        for (int k = i + 1; k < N; ++k)
            if ((pat.rows[i] >> k) & 1u) x[i] -= A[i * N + k] * x[k];
        x[i] *= A[i * N + i];
    }
}

template <int DIM, int P, typename R>
__device__ __forceinline__ void lu_solve_transpose_s(const R* A, R* x) {
    constexpr int N = LuPattern<DIM, P>::N;
    constexpr typename LuPattern<DIM, P>::Table pat = LuPattern<DIM, P>::build();
#pragma unroll
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int k = 0; k < i; ++k)
            if ((pat.rows[k] >> i) & 1u) x[i] -= A[k * N + i] * x[k];
        x[i] *= A[i * N + i];
    }
#pragma unroll
    for (int i = N - 1; i >= 0; --i)
#pragma unroll
        for (int k = i + 1; k < N; ++k)
            if ((pat.rows[k] >> i) & 1u) x[i] -= A[k * N + i] * x[k];
}

// ---------------------------------------------------------------- operator cache
// A_e depends on the direction, the element geometry and sigma_t only, so within a solve every
// transport update would factor the same nd x ne matrices again.  The cache holds A_e^{-1} of
// every (direction, element) pair, column-major (entry (i, j) at [j * N + i]), formed once per
// change of materials by a fully parallel kernel; a cached sweep forms the right-hand side and
// multiplies.  Beside it sit the face flux factors (2D: per pair; 3D: per direction), so that a
// cached sweep needs no geometry.
template <int DIM, int P>
struct CacheShape {
    static constexpr int N = Shape<DIM, P>::N;
    static constexpr int S = (N * N + 3) & ~3;  // entries per cached inverse (16-byte multiple)
};

// A_e^{-1} of every (direction, element) pair, independent work: float64 assembly and unpivoted
// LU (the factorisation the on-the-fly sweep uses), then column j = U^{-1} L^{-1} e_j stored
// contiguously in type R, padding zeroed; the face flux factors are written beside it.
template <int DIM, int P, typename R>
__global__ void __launch_bounds__(128) factor_kernel(SweepArgs a, R* out, double* fflux) {
    constexpr int N = CacheShape<DIM, P>::N, S = CacheShape<DIM, P>::S;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)a.nd * a.ne) return;
    const int d = (int)(t / a.ne), e = (int)(t % a.ne);
    ElemGeom<DIM, P, double> g;
    elem_geom<DIM, P, double>(a, e, a.dirs[3 * d], a.dirs[3 * d + 1], a.dirs[3 * d + 2], g);
    if (DIM == 2) {
#pragma unroll
        for (int f = 0; f < 4; ++f) fflux[t * 4 + f] = g.Fd[f];
    } else if (e == 0) {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) fflux[3 * d + ax] = g.Fd[2 * ax + 1];
    }
    double A[N * N];
    assemble<DIM, P, double>(g, a.sigma_t[e], A);
    lu_factor_s<DIM, P, double>(A);
    R* o = out + t * S;
#pragma unroll 1
    for (int j = 0; j < N; ++j) {
        double x[N];
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = i == j ? 1.0 : 0.0;
        lu_solve_s<DIM, P, double>(A, x);
#pragma unroll
        for (int i = 0; i < N; ++i) o[j * N + i] = (R)x[i];
    }
#pragma unroll
    for (int k = N * N; k < S; ++k) o[k] = R(0);
}

// Face coefficients W_t l_side(i_a) of every node (i_a its index along the face normal axis, t
// its tangential index) and face, per element family, in float64 and float32.
__device__ double g_fcoef[FAM_COUNT][32][6];
__device__ float g_fcoef32[FAM_COUNT][32][6];

// The same coefficient times the weight l_other(k) with which the neighbour's value at its k-th
// node along the face normal enters the face trace: a face term is then -F sum_k fw_k psi_k.
__device__ __align__(16) double g_fw[FAM_COUNT][32][6][4];
__device__ __align__(16) float g_fw32[FAM_COUNT][32][6][4];

template <typename R>
__device__ __forceinline__ R fcoef(int fam, int r, int f);
template <>
__device__ __forceinline__ double fcoef<double>(int fam, int r, int f) { return __ldg(&g_fcoef[fam][r][f]); }
template <>
__device__ __forceinline__ float fcoef<float>(int fam, int r, int f) { return __ldg(&g_fcoef32[fam][r][f]); }
// The Q weights of (r, f) in 16-byte loads.
template <int Q>
__device__ __forceinline__ void fweights(int fam, int r, int f, double* w) {
    const double2* p = reinterpret_cast<const double2*>(&g_fw[fam][r][f][0]);
#pragma unroll
    for (int h = 0; h < (Q + 1) / 2; ++h) {
        const double2 v = __ldg(p + h);
        w[2 * h] = v.x;
        if (2 * h + 1 < Q) w[2 * h + 1] = v.y;
    }
}
template <int Q>
__device__ __forceinline__ void fweights(int fam, int r, int f, float* w) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(&g_fw32[fam][r][f][0]));
    const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < Q; ++k) w[k] = vv[k];
}

// Whether a face with flux factor F = Omega.n |face| is an inflow face (adjoint: an outflow face),
// i.e. F < 0 (F > 0), decided on the bits so that no float64 compare is issued; zeros and NaN are
// on neither side, as with the floating-point compare.
template <bool ADJ>
__device__ __forceinline__ bool upwind_face(double F) {
    const long long b = __double_as_longlong(F);
    const long long m = b & 0x7fffffffffffffffll;
    return (ADJ ? b > 0 : b < 0) && m != 0 && m <= 0x7ff0000000000000ll;
}
template <bool ADJ>
__device__ __forceinline__ bool upwind_face(float F) {
    const int b = __float_as_int(F);
    const int m = b & 0x7fffffff;
    return (ADJ ? b > 0 : b < 0) && m != 0 && m <= 0x7f800000;
}

cudaError_t upload_face_coefficients() {
    static double c[FAM_COUNT][32][6];
    static float c32[FAM_COUNT][32][6];
    static double w[FAM_COUNT][32][6][4];
    static float w32[FAM_COUNT][32][6][4];
    for (int fam = 0; fam < FAM_COUNT; ++fam) {
        const int dim = fam == FAM_3D_P1 ? 3 : 2, p = fam == FAM_3D_P1 ? 1 : fam + 1, Q = p + 1;
        const int n = dim == 2 ? Q * Q : Q * Q * Q;
        const GL1D g = gauss_legendre_nodal(p);
        for (int r = 0; r < 32; ++r)
            for (int f = 0; f < 6; ++f) {
                double v = 0.0;
                if (r < n && f < 2 * dim) {
                    const int ri[3] = {r % Q, (r / Q) % Q, r / (Q * Q)};
                    const int ax = f >> 1;
                    const bool hi = f & 1;
                    double wt = 1.0;
                    for (int b = 0; b < dim; ++b)
                        if (b != ax) wt *= g.w[ri[b]];
                    v = wt * (hi ? g.lp[ri[ax]] : g.lm[ri[ax]]);
                }
                c[fam][r][f] = v;
                c32[fam][r][f] = (float)v;
                // the neighbour's side of the face: its high end for our low face and vice versa
                for (int k = 0; k < 4; ++k) {
                    const double l = k < Q ? ((f & 1) ? g.lm[k] : g.lp[k]) : 0.0;
                    w[fam][r][f][k] = v * l;
                    w32[fam][r][f][k] = (float)(v * l);
                }
            }
    }
    cudaError_t err = cudaMemcpyToSymbol(g_fcoef, c, sizeof(c));
    if (err == cudaSuccess) err = cudaMemcpyToSymbol(g_fcoef32, c32, sizeof(c32));
    if (err == cudaSuccess) err = cudaMemcpyToSymbol(g_fw, w, sizeof(w));
    if (err == cudaSuccess) err = cudaMemcpyToSymbol(g_fw32, w32, sizeof(w32));
    return err;
}

// Cached transport update with one lane per node: a warp holds 32 / N items, lane r of an item
// forms row r of its right-hand side (source and the inflow terms through the faces of node r's
// coordinate lines), the item's right-hand side is exchanged by shuffles and lane r writes
// x_r = sum_j (A_e^{-1})_rj rhs_j.  An item's float64 work on the critical path is then about
// 2N + 5 dim instructions instead of the ~(2/3) N^3 of a factorisation.  ADJ = true is the
// transposed solve of the adjoint (outflow faces, downwind neighbours, A_e^{-T}).
// Face flux factors of (direction d, element e) from the cache: the float64 values the level
// sets were built from, so inflow/outflow decisions agree everywhere.
template <int DIM>
__device__ __forceinline__ void cached_fluxes(const SweepArgs& a, int d, int e, double* F) {
    if constexpr (DIM == 2) {
        const double2* fp = reinterpret_cast<const double2*>(a.fflux + ((size_t)d * a.ne + e) * 4);
        const double2 v0 = __ldg(fp), v1 = __ldg(fp + 1);
        F[0] = v0.x;
        F[1] = v0.y;
        F[2] = v1.x;
        F[3] = v1.y;
    } else {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const double b = __ldg(a.fflux + 3 * d + ax);
            F[2 * ax] = -b;
            F[2 * ax + 1] = b;
        }
    }
}
template <int DIM>
__device__ __forceinline__ void cached_fluxes(const SweepArgs& a, int d, int e, float* F) {
    if constexpr (DIM == 2) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(a.fflux32 + ((size_t)d * a.ne + e) * 4));
        F[0] = v.x;
        F[1] = v.y;
        F[2] = v.z;
        F[3] = v.w;
    } else {
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const float b = __ldg(a.fflux32 + 3 * d + ax);
            F[2 * ax] = -b;
            F[2 * ax + 1] = b;
        }
    }
}

// The part of a node's work that reads no angular flux: the face flux factors, the source row
// (forward: M_r (q + sigma_s phi_r) / (4 pi); adjoint: mu_r) and the N entries of the cached
// inverse this lane multiplies with (forward: row r of A_e^{-1}; adjoint: column r).
template <int DIM, int P, typename R>
struct NodeStage {
    R F[2 * DIM];  // face flux factors (float32 in the FP32 form: its upwind test and face terms)
    R rhs;
    R inv[Shape<DIM, P>::N];
};

template <int DIM, int P, int MODE, bool ADJ>
__device__ __forceinline__ void node_stage(const SweepArgs& a, const double* mu, int d, int e, int r,
                                           NodeStage<DIM, P, typename std::conditional<MODE == 1, float, double>::type>& st) {
    using R = typename std::conditional<MODE == 1, float, double>::type;
    constexpr int N = Shape<DIM, P>::N, S = CacheShape<DIM, P>::S;
    cached_fluxes<DIM>(a, d, e, st.F);
    if constexpr (ADJ) {
        st.rhs = (R)mu[(size_t)e * N + r];
    } else if constexpr (MODE == 1) {
        // float32 source row M_r / (4 pi) (sigma_s phi_r + q): the scattering product is formed in
        // float64 and rounded once, because a sigma_s rounded to float32 would be a systematic
        // change of the absorption sigma_t - sigma_s, which the fixed point amplifies by up to
        // c / (1 - c)
        const float sp = a.phi ? (float)(a.sigma_s[e] * a.phi[(size_t)e * N + r]) : 0.0f;
        const float qe = a.q32 ? __ldg(a.q32 + e) : 0.0f;
        st.rhs = __ldg(a.mass32 + (size_t)e * N + r) * (sp + qe);
    } else {
        // M_r / (4 pi) (sigma_s phi_r + q), q absent (null) in the linear part of the update
        const double qe = a.q ? a.q[e] : 0.0;
        const double S = a.phi ? fma(a.sigma_s[e], a.phi[(size_t)e * N + r], qe) : qe;
        st.rhs = (R)(a.mass4[(size_t)e * N + r] * S);
    }
    const R* inv;
    if constexpr (MODE == 1) inv = a.ainv32;
    else inv = a.ainv;
    inv += ((size_t)d * a.ne + e) * S;
#pragma unroll
    for (int j = 0; j < N; ++j) st.inv[j] = __ldcs(inv + (ADJ ? r * N + j : j * N + r));
}

// Inflow (adjoint: outflow) face terms of node r from the neighbours' angular fluxes.
template <int DIM, int P, typename R, bool ADJ>
__device__ __forceinline__ R node_faces(const SweepArgs& a, const R* F, int d, int e, int r, R rhs) {
    constexpr int Q = P + 1, N = Shape<DIM, P>::N;
    constexpr int FAM = DIM == 3 ? FAM_3D_P1 : P - 1;
    const int ri[3] = {r % Q, (r / Q) % Q, r / (Q * Q)};
    const R* psi = static_cast<const R*>(a.psi);
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        if (!upwind_face<ADJ>(F[f])) continue;
        const int ax = f >> 1;
        const int u = neighbor<DIM, P>(a, e, f);
        const int tt = DIM == 2 ? ri[1 - ax] : (ax == 0 ? ri[1] + Q * ri[2] : (ax == 1 ? ri[0] + Q * ri[2] : ri[0] + Q * ri[1]));
        const R sF = ADJ ? F[f] : -F[f];
        if (u >= 0) {
            const R* pu = psi + ((size_t)d * a.ne + u) * N;
            R w[Q];
            fweights<Q>(FAM, r, f, w);
            R t = R(0);
#pragma unroll
            for (int k = 0; k < Q; ++k) t += w[k] * __ldcg(pu + node_of<DIM, P>(ax, k, tt));
            rhs += sF * t;
        } else if (!ADJ) {
            rhs += (sF * fcoef<R>(FAM, r, f)) * (R)a.psi_inc;
        }
    }
    return rhs;
}

// One node of one item: stage, (PDL: release the next grid, wait for the previous one), face
// terms, x_r = sum_j inv_rj rhs_j with rhs_j shuffled from the item's lane j, store.
// Second half of a node's work: face terms from the neighbours' angular fluxes, then
// x_r = sum_j inv_rj rhs_j with rhs_j shuffled from the item's lane j, and the store.  Every lane
// of the warp must call it (shuffles); `valid` masks lanes without an item.
template <int DIM, int P, int MODE, bool ADJ>
__device__ __forceinline__ void node_finish(const SweepArgs& a,
                                            const NodeStage<DIM, P, typename std::conditional<MODE == 1, float, double>::type>& st,
                                            int d, int e, int r, int src0, bool valid) {
    using R = typename std::conditional<MODE == 1, float, double>::type;
    constexpr int N = Shape<DIM, P>::N;
    const R rhs = valid ? node_faces<DIM, P, R, ADJ>(a, st.F, d, e, r, st.rhs) : R(0);
    R x = R(0);
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const R rj = __shfl_sync(0xffffffffu, rhs, src0 + j);
        if (valid) x += st.inv[j] * rj;
    }
    if (valid) static_cast<R*>(a.psi)[((size_t)d * a.ne + e) * N + r] = x;
}

// One node of one item: stage, (PDL: wait for the previous grid, release the next), finish.
template <int DIM, int P, int MODE, bool ADJ, bool PDL = false>
__device__ __forceinline__ void node_item(const SweepArgs& a, const double* mu, int d, int e, int r, int src0,
                                          bool valid) {
    using R = typename std::conditional<MODE == 1, float, double>::type;
    NodeStage<DIM, P, R> st;
    if (valid) node_stage<DIM, P, MODE, ADJ>(a, mu, d, e, r, st);
    if (PDL) {
        // the next level may launch once this one's inputs are complete: its blocks then run
        // their prologue while this level computes, and the look-ahead stays one level deep
        pdl_wait();
        pdl_launch_dependents();
    }
    node_finish<DIM, P, MODE, ADJ>(a, st, d, e, r, src0, valid);
}

template <int DIM, int P, int MODE, bool ADJ>
__global__ void __launch_bounds__(128, DIM == 3 ? 10 : 1) node_level_kernel(SweepArgs a, const double* mu, long long begin,
                                                        long long end) {
    constexpr int N = Shape<DIM, P>::N, IPW = 32 / N;
    const int lane = threadIdx.x & 31;
    const int slot = lane / N, r = lane - slot * N;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long t = begin + warp * IPW + slot;
    const bool valid = slot < IPW && t < end;
    int d = 0, e = 0;
    if (valid) {
        const int2 it = a.items[t];
        d = it.x;
        e = it.y;
    }
    node_item<DIM, P, MODE, ADJ, true>(a, mu, d, e, r, slot < IPW ? slot * N : 0, valid);
}

// Right-hand side in arithmetic type R: mass-weighted source S = (q + sigma_s phi)/(4 pi) (formed in
// float64, then rounded to R) plus inflow face terms from the upwind neighbours' traces.
template <int DIM, int P, typename RS, typename R>
__device__ __forceinline__ void assemble_rhs(const SweepArgs& a, const ElemGeom<DIM, P, R>& g, int d, int e, R* rhs) {
    constexpr int Q = P + 1, N = Shape<DIM, P>::N, NT = Shape<DIM, P>::NT;
    using K = GLT<R>;
    const double ss = a.sigma_s[e], qe = a.q ? a.q[e] : 0.0;
    const double* phi = a.phi ? a.phi + (size_t)e * N : nullptr;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const double S = (qe + (phi ? ss * phi[i] : 0.0)) * (1.0 / kFourPi);
        rhs[i] = g.mass[i] * (R)S;
    }
    const RS* psi = static_cast<const RS*>(a.psi);
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        if (g.Fd[f] < 0.0) {
            const int ax = f >> 1;
            const bool hi = f & 1;
            const int u = neighbor<DIM, P>(a, e, f);
            R tr[NT];
            if (u >= 0) {
                const RS* pu = psi + ((size_t)d * a.ne + u) * N;
                R vals[N];
#pragma unroll
                for (int i = 0; i < N; ++i) vals[i] = (R)__ldcg(pu + i);
#pragma unroll
                for (int t = 0; t < NT; ++t) {
                    R s = R(0);
#pragma unroll
                    for (int k = 0; k < Q; ++k) s += (hi ? K::lm(P, k) : K::lp(P, k)) * vals[node_of<DIM, P>(ax, k, t)];
                    tr[t] = s;
                }
            } else {
#pragma unroll
                for (int t = 0; t < NT; ++t) tr[t] = (R)a.psi_inc;
            }
#pragma unroll
            for (int t = 0; t < NT; ++t) {
                const R ft = -g.F[f] * wtan<DIM, P, R>(t) * tr[t];
#pragma unroll
                for (int ia = 0; ia < Q; ++ia) rhs[node_of<DIM, P>(ax, ia, t)] += ft * (hi ? K::lp(P, ia) : K::lm(P, ia));
            }
        }
    }
}

// MODE 0: float64 element solve and storage.  MODE 1: float32 geometry, assembly, LU and
// storage (source formed in float64 and rounded).  MODE 2: float32 assembly and LU, then two
// float64 residual corrections x += LU^{-1}(b - A x) with A applied matrix-free in float64;
// float64 storage.
template <int DIM, int P, int MODE>
__device__ __forceinline__ void solve_item(const SweepArgs& a, int d, int e) {
    constexpr int N = Shape<DIM, P>::N;
    const double Ox = a.dirs[3 * d], Oy = a.dirs[3 * d + 1], Oz = a.dirs[3 * d + 2];
    const double st = a.sigma_t[e];
    if constexpr (MODE == 1) {
        ElemGeom<DIM, P, float> g;
        elem_geom<DIM, P, float>(a, e, Ox, Oy, Oz, g);
        float rhs[N], A[N * N];
        assemble_rhs<DIM, P, float, float>(a, g, d, e, rhs);
        assemble<DIM, P, float>(g, (float)st, A);
        lu_factor_s<DIM, P, float>(A);
        lu_solve_s<DIM, P, float>(A, rhs);
        float* out = static_cast<float*>(a.psi) + ((size_t)d * a.ne + e) * N;
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = rhs[i];
    } else if constexpr (MODE == 0) {
        ElemGeom<DIM, P, double> g;
        elem_geom<DIM, P, double>(a, e, Ox, Oy, Oz, g);
        double rhs[N], A[N * N];
        assemble_rhs<DIM, P, double, double>(a, g, d, e, rhs);
        assemble<DIM, P, double>(g, st, A);
        lu_factor_s<DIM, P, double>(A);
        lu_solve_s<DIM, P, double>(A, rhs);
        double* out = static_cast<double*>(a.psi) + ((size_t)d * a.ne + e) * N;
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = rhs[i];
    } else {
        ElemGeom<DIM, P, double> gd;
        elem_geom<DIM, P, double>(a, e, Ox, Oy, Oz, gd);
        double rhs[N], x[N], r[N];
        assemble_rhs<DIM, P, double, double>(a, gd, d, e, rhs);
        float A[N * N], c[N];
        {
            ElemGeom<DIM, P, float> gf;
            narrow_geom<DIM, P>(gd, gf);
            assemble<DIM, P, float>(gf, (float)st, A);
        }
        lu_factor_s<DIM, P, float>(A);
#pragma unroll
        for (int i = 0; i < N; ++i) c[i] = (float)rhs[i];
        lu_solve_s<DIM, P, float>(A, c);
#pragma unroll
        for (int i = 0; i < N; ++i) x[i] = c[i];
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            apply_A<DIM, P>(gd, st, x, r);
#pragma unroll
            for (int i = 0; i < N; ++i) c[i] = (float)(rhs[i] - r[i]);
            lu_solve_s<DIM, P, float>(A, c);
#pragma unroll
            for (int i = 0; i < N; ++i) x[i] += (double)c[i];
        }
        double* out = static_cast<double*>(a.psi) + ((size_t)d * a.ne + e) * N;
#pragma unroll
        for (int i = 0; i < N; ++i) out[i] = x[i];
    }
}

template <int DIM, int P, int MODE>
__global__ void __launch_bounds__(128) sweep_level_kernel(SweepArgs a, long long begin, long long end) {
    const long long t = begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= end) return;
    const int2 it = a.items[t];
    solve_item<DIM, P, MODE>(a, it.x, it.y);
}

// ---------------------------------------------------------------- persistent dataflow sweep
// One launch per transport update.  The work list is padded so that every 32-item chunk lies
// in a single level; warps claim chunks in list order from a global counter, so every item a
// warp waits for belongs to an earlier level and was claimed by a warp that is running.  An
// item waits (bounded, with back-off) until each upwind neighbour's completion word holds the
// current epoch, solves, stores psi and publishes its own word with release semantics.
// Static assignment (SCHED_STATIC): with every warp of the grid resident, warp w takes slices
// w, w + W, w + 2W, ... of the list (W warps in all) instead of claiming them.  Each warp's slices
// are in level order, so the unfinished slice earliest in the list waits only on finished items
// and its warp has finished all of its earlier slices: no deadlock, and no shared counter whose
// atomics every warp would queue on.
__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <int DIM, int P>
__device__ __forceinline__ void adjoint_item(const SweepArgs& a, const double* mu, int d, int e);

// ADJ = false: transport update, waits for upwind neighbours (Omega.n < 0 faces).
// ADJ = true: transposed solve in reverse order, waits for downwind neighbours (Omega.n > 0).
template <int DIM, int P, int MODE, bool ADJ>
__global__ void __launch_bounds__(128) sweep_dataflow_kernel(SweepArgs a, DataflowArgs f, const double* mu) {
    const int lane = threadIdx.x & 31;
    const long long n_chunks = f.n_items >> 5;
    const unsigned long long deadline = globaltimer() + f.timeout_ns;
    if (f.epoch_dev) f.epoch = f.publish = *f.epoch_dev;
    unsigned long long mine = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    while (true) {
        // lane 0 claims the chunk and reads the error word; the warp acts on one broadcast value
        unsigned long long c = 0;
        int failed = 0;
        if (lane == 0) {
            if (f.static_warps > 0) {
                c = mine;
                mine += (unsigned long long)f.static_warps;
            } else {
                c = atomicAdd(f.next, 1ull);
            }
            failed = *(volatile int*)f.error;
        }
        c = __shfl_sync(0xffffffffu, c, 0);
        failed = __shfl_sync(0xffffffffu, failed, 0);
        if ((long long)c >= n_chunks || failed) break;
        const int2 it = f.items[(c << 5) + lane];
        bool ok = true;
        if (it.x >= 0) {
            const int d = it.x, e = it.y;
            const double Ox = a.dirs[3 * d], Oy = a.dirs[3 * d + 1], Oz = a.dirs[3 * d + 2];
#pragma unroll
            for (int fc = 0; fc < 2 * DIM; ++fc) {
                if (!ok) break;
                const double F = face_flux_only<DIM, P>(a, e, fc, Ox, Oy, Oz);
                if (ADJ ? F > 0.0 : F < 0.0) {
                    const int u = neighbor<DIM, P>(a, e, fc);
                    if (u < 0) continue;
                    const int* flag = f.done + (size_t)d * a.ne + u;
                    int polls = 0;
                    while (ld_acquire(flag) != f.epoch) {
                        if (++polls > 64) {  // spin briefly, then back off and watch the deadline
                            if (globaltimer() > deadline) {
                                ok = false;
                                break;
                            }
                            __nanosleep(64);
                        }
                    }
                }
            }
        }
        // reconverge before the solve so the warp issues the element solve once for all its lanes
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicExch(f.error, 1);
            break;
        }
        if (it.x >= 0) {
            if constexpr (ADJ) adjoint_item<DIM, P>(a, mu, it.x, it.y);
            else solve_item<DIM, P, MODE>(a, it.x, it.y);
            st_release(f.done + (size_t)it.x * a.ne + it.y, f.publish);
        }
    }
}

// Bounded wait until every upwind (ADJ: downwind) neighbour of (d, e) holds the current epoch;
// false when the deadline passed.  Face fluxes come from the operator cache.
template <int DIM, int P, bool ADJ>
__device__ __forceinline__ bool wait_neighbours(const SweepArgs& a, const int* done, int epoch, int d, int e,
                                                unsigned long long deadline) {
    double F[2 * DIM];
    cached_fluxes<DIM>(a, d, e, F);
#pragma unroll
    for (int fc = 0; fc < 2 * DIM; ++fc) {
        if (ADJ ? F[fc] > 0.0 : F[fc] < 0.0) {
            const int u = neighbor<DIM, P>(a, e, fc);
            if (u < 0) continue;
            const int* flag = done + (size_t)d * a.ne + u;
            int polls = 0;
            while (ld_acquire(flag) != epoch) {
                if (++polls > 64) {
                    if (globaltimer() > deadline) return false;
                    __nanosleep(64);
                }
            }
        }
    }
    return true;
}

// ---- data-polled dataflow (cached sweeps): before the launch every angular flux of the sweep
// is set to the all-ones bit pattern (a NaN no element solve produces), and a consumer polls the
// upwind values it needs until none is that pattern.  Each value is one 8- (4-) byte word written
// once by a relaxed store and read by relaxed loads, so a value that is seen is the final one; no
// completion words, no fences, and the flag round trip of the completion-word scheme disappears.
__device__ __forceinline__ double ld_relaxed(const double* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return __longlong_as_double((long long)v);
}
__device__ __forceinline__ float ld_relaxed(const float* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return __int_as_float((int)v);
}
__device__ __forceinline__ void st_relaxed(double* p, double x) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"((unsigned long long)__double_as_longlong(x)) : "memory");
}
__device__ __forceinline__ void st_relaxed(float* p, float x) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"((unsigned)__float_as_int(x)) : "memory");
}
__device__ __forceinline__ bool is_unset(double v) { return __double_as_longlong(v) == -1ll; }
__device__ __forceinline__ bool is_unset(float v) { return __float_as_int(v) == -1; }
__device__ __forceinline__ double unset_value(double) { return __longlong_as_double(-1ll); }
__device__ __forceinline__ float unset_value(float) { return __int_as_float(-1); }

// node_faces with the upwind (adjoint: downwind) values polled (bounded); *ok = false when the
// deadline passed or, once a wait has gone on for a while, when another warp has set the launch's
// error word (so a failed launch ends promptly without every item reading the word).
template <int DIM, int P, typename R, bool ADJ>
__device__ __forceinline__ R node_faces_polled(const SweepArgs& a, const R* F, int d, int e, int r, R rhs,
                                               unsigned long long deadline, const int* error, bool* ok) {
    constexpr int Q = P + 1, N = Shape<DIM, P>::N;
    constexpr int FAM = DIM == 3 ? FAM_3D_P1 : P - 1;
    const int ri[3] = {r % Q, (r / Q) % Q, r / (Q * Q)};
    const R* psi = static_cast<const R*>(a.psi);
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        if (!upwind_face<ADJ>(F[f])) continue;
        const int ax = f >> 1;
        const int u = neighbor<DIM, P>(a, e, f);
        const int tt = DIM == 2 ? ri[1 - ax] : (ax == 0 ? ri[1] + Q * ri[2] : (ax == 1 ? ri[0] + Q * ri[2] : ri[0] + Q * ri[1]));
        const R sF = ADJ ? F[f] : -F[f];
        if (u >= 0) {
            const R* pu = psi + ((size_t)d * a.ne + u) * N;
            R v[Q];
            int polls = 0;
            while (true) {
                bool all = true;
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    v[k] = ld_relaxed(pu + node_of<DIM, P>(ax, k, tt));
                    all = all && !is_unset(v[k]);
                }
                if (all) break;
                if (++polls > 64) {
                    if (globaltimer() > deadline || *(volatile const int*)error) {
                        *ok = false;
                        break;
                    }
                    __nanosleep(32);
                }
            }
            R w[Q];
            fweights<Q>(FAM, r, f, w);
            R t = R(0);
#pragma unroll
            for (int k = 0; k < Q; ++k) t += w[k] * v[k];
            rhs += sF * t;
        } else if (!ADJ) {
            rhs += (sF * fcoef<R>(FAM, r, f)) * (R)a.psi_inc;
        }
    }
    return rhs;
}

// Data-polled dataflow item loop of the cached sweeps (schedules 1 and 4; ADJ: the transposed
// solve of the adjoint in reverse level order): claim or take slices as node_dataflow_kernel does,
// stage, then the face terms poll their upwind (downwind) values; the store of x is the
// publication.
template <int DIM, int P, int MODE, bool ADJ>
__global__ void __launch_bounds__(128) node_datapoll_kernel(SweepArgs a, DataflowArgs f, const double* mu) {
    using R = typename std::conditional<MODE == 1, float, double>::type;
    constexpr int N = Shape<DIM, P>::N, IPW = 32 / N, SLICES = (32 + IPW - 1) / IPW;
    const int lane = threadIdx.x & 31;
    const int slot = lane / N, r = lane - slot * N;
    const int src0 = slot < IPW ? slot * N : 0;
    const long long n_slices = (f.n_items >> 5) * SLICES;
    const unsigned long long deadline = globaltimer() + f.timeout_ns;
    const bool withhold = f.publish == -1;  // test hook: store the unset pattern, every wait times out
    // this lane's item of slice c (padding and lanes past the slice's items: (-1, -1))
    auto item_of = [&](unsigned long long c) {
        const long long chunk = (long long)c / SLICES;
        const int k = (int)((long long)c - chunk * SLICES) * IPW + slot;
        return (slot < IPW && k < 32 && (long long)c < n_slices) ? f.items[(chunk << 5) + k] : make_int2(-1, -1);
    };
    const bool fixed = f.static_warps > 0;
    unsigned long long mine = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    // static assignment: the warp's slices are known in advance, so the next one's items are loaded
    // while the current one is solved
    int2 next = fixed ? item_of(mine) : make_int2(-1, -1);
    while (true) {
        unsigned long long c = 0;
        if (fixed) {
            c = mine;
            mine += (unsigned long long)f.static_warps;
        } else {
            if (lane == 0) c = atomicAdd(f.next, 1ull);
            c = __shfl_sync(0xffffffffu, c, 0);
        }
        if ((long long)c >= n_slices) break;
        int2 it;
        if (fixed) {
            it = next;
            next = item_of(mine);
        } else {
            it = item_of(c);
        }
        const bool valid = it.x >= 0;
        const int d = valid ? it.x : 0, e = valid ? it.y : 0;
        NodeStage<DIM, P, R> st;
        if (valid) node_stage<DIM, P, MODE, ADJ>(a, mu, d, e, r, st);
        bool ok = true;
        const R rhs = valid ? node_faces_polled<DIM, P, R, ADJ>(a, st.F, d, e, r, st.rhs, deadline, f.error, &ok)
                            : R(0);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicExch(f.error, 1);
            break;
        }
        R x = R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const R rj = __shfl_sync(0xffffffffu, rhs, src0 + j);
            if (valid) x += st.inv[j] * rj;
        }
        if (valid) st_relaxed(static_cast<R*>(a.psi) + ((size_t)d * a.ne + e) * N + r, withhold ? unset_value(x) : x);
    }
}

// As wait_neighbours with the face fluxes already loaded, every pending word polled in each round
// (their loads in flight together) rather than one face after another.
template <int DIM, int P, bool ADJ, typename T>
__device__ __forceinline__ bool wait_neighbours_all(const SweepArgs& a, const T* F, const int* done, int epoch,
                                                    int d, int e, unsigned long long deadline) {
    const int* flag[2 * DIM];
    int pending = 0;
#pragma unroll
    for (int fc = 0; fc < 2 * DIM; ++fc) {
        flag[fc] = nullptr;
        if (upwind_face<ADJ>(F[fc])) {
            const int u = neighbor<DIM, P>(a, e, fc);
            if (u >= 0) {
                flag[fc] = done + (size_t)d * a.ne + u;
                ++pending;
            }
        }
    }
    int polls = 0;
    while (pending > 0) {
        int v[2 * DIM];
#pragma unroll
        for (int fc = 0; fc < 2 * DIM; ++fc) v[fc] = flag[fc] ? ld_acquire(flag[fc]) : epoch;
#pragma unroll
        for (int fc = 0; fc < 2 * DIM; ++fc)
            if (flag[fc] && v[fc] == epoch) {
                flag[fc] = nullptr;
                --pending;
            }
        if (pending > 0 && ++polls > 64) {
            if (globaltimer() > deadline) return false;
            __nanosleep(64);
        }
    }
    return true;
}

// Dataflow schedule of the cached sweep, one lane per node: a warp claims 32 / N items at a time
// (a slice of a 32-item chunk of the padded list, so claims still follow level order), waits for
// their neighbours, solves, synchronises, and each item's lane 0 fences and publishes the
// completion word, so a waiter that acquires it sees all N lanes' angular fluxes.
template <int DIM, int P, int MODE, bool ADJ>
__global__ void __launch_bounds__(128) node_dataflow_kernel(SweepArgs a, DataflowArgs f, const double* mu) {
    constexpr int N = Shape<DIM, P>::N, IPW = 32 / N, SLICES = (32 + IPW - 1) / IPW;
    const int lane = threadIdx.x & 31;
    const int slot = lane / N, r = lane - slot * N;
    const int src0 = slot < IPW ? slot * N : 0;
    const long long n_slices = (f.n_items >> 5) * SLICES;
    const unsigned long long deadline = globaltimer() + f.timeout_ns;
    if (f.epoch_dev) f.epoch = f.publish = *f.epoch_dev;
    unsigned long long mine = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    while (true) {
        unsigned long long c = 0;
        int failed = 0;
        if (lane == 0) {
            if (f.static_warps > 0) {
                c = mine;
                mine += (unsigned long long)f.static_warps;
            } else {
                c = atomicAdd(f.next, 1ull);
            }
            failed = *(volatile int*)f.error;
        }
        c = __shfl_sync(0xffffffffu, c, 0);
        failed = __shfl_sync(0xffffffffu, failed, 0);
        if ((long long)c >= n_slices || failed) break;
        const long long chunk = (long long)c / SLICES;
        const int k = (int)((long long)c - chunk * SLICES) * IPW + slot;
        int2 it = make_int2(-1, -1);
        if (slot < IPW && k < 32) it = f.items[(chunk << 5) + k];
        const bool valid = it.x >= 0;
        const int d = valid ? it.x : 0, e = valid ? it.y : 0;
        // loads that read no angular flux go out before the waits, so they overlap them
        NodeStage<DIM, P, typename std::conditional<MODE == 1, float, double>::type> st;
        if (valid) node_stage<DIM, P, MODE, ADJ>(a, mu, d, e, r, st);
        // one lane per item polls (all of its upwind words at once); the warp barrier then orders
        // that lane's acquire before every lane's reads of the neighbours
        const bool ok = (valid && r == 0) ? wait_neighbours_all<DIM, P, ADJ>(a, st.F, f.done, f.epoch, d, e, deadline)
                                          : true;
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicExch(f.error, 1);
            break;
        }
        __syncwarp();
        node_finish<DIM, P, MODE, ADJ>(a, st, d, e, r, src0, valid);
        // the warp barrier orders the item's N lanes' stores before lane 0's release store, and a
        // release is cumulative: a waiter that acquires the word sees all N values
        __syncwarp();
        if (valid && r == 0) st_release(f.done + (size_t)d * a.ne + e, f.publish);
    }
}

// ---------------------------------------------------------------- tiled sweep (cached operators)
struct TileArgs {
    const int4* tasks;               // (direction, first item, first level boundary, levels)
    const int* lvl_ptr;
    const int2* items;               // (element, flags)
    long long n_tasks;
    int* done;                       // nd x ne completion words
    int epoch, publish;
    unsigned long long* next;        // task counter, zeroed before each launch
    int* error;                      // set to 1 when a wait times out
    unsigned long long timeout_ns;
};

// Bounded wait for the upwind neighbours through the faces in `bits` (elements of other tasks).
template <int DIM, int P>
__device__ __forceinline__ bool wait_faces(const SweepArgs& a, const int* done, int epoch, int d, int e, int bits,
                                           unsigned long long deadline) {
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        if (!((bits >> f) & 1)) continue;
        const int* flag = done + (size_t)d * a.ne + neighbor<DIM, P>(a, e, f);
        int polls = 0;
        while (ld_acquire(flag) != epoch) {
            if (++polls > 64) {
                if (globaltimer() > deadline) return false;
                __nanosleep(64);
            }
        }
    }
    return true;
}

// A CTA claims tasks in list order and runs each task's local levels one after another, one
// lane per node (node_item), with a CTA barrier between levels.  A failed wait ends the launch
// for every CTA through the error word (all barriers are still reached: waits are bounded).
template <int DIM, int P, int MODE>
__global__ void __launch_bounds__(256) tile_sweep_kernel(SweepArgs a, TileArgs t) {
    using R = typename std::conditional<MODE == 1, float, double>::type;
    constexpr int N = Shape<DIM, P>::N, IPW = 32 / N;
    __shared__ long long s_task;
    __shared__ int s_failed;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = lane / N, r = lane - slot * N, src0 = slot < IPW ? slot * N : 0;
    const int per_pass = (blockDim.x >> 5) * IPW;
    const unsigned long long deadline = globaltimer() + t.timeout_ns;
    while (true) {
        if (threadIdx.x == 0) {
            s_task = (long long)atomicAdd(t.next, 1ull);
            s_failed = *(volatile int*)t.error;
        }
        __syncthreads();
        const long long task = s_task;
        const int failed = s_failed;
        __syncthreads();
        if (task >= t.n_tasks || failed) break;
        const int4 T = t.tasks[task];
        const int d = T.x;
        // the task's passes (level, first item) in order; the stage of the next pass is loaded
        // before the current pass waits and computes (it reads no angular flux)
        int L = 0, lo = t.lvl_ptr[T.z], hi = t.lvl_ptr[T.z + 1], base = lo;
        int idx = base + warp * IPW + slot;
        bool valid = slot < IPW && idx < hi;
        int2 it = valid ? t.items[idx] : make_int2(0, 0);
        NodeStage<DIM, P, R> st;
        if (valid) node_stage<DIM, P, MODE, false>(a, nullptr, d, it.x, r, st);
        bool bad = false, abort = false;
        while (true) {
            // next pass
            int nL = L, nlo = lo, nhi = hi, nbase = base + per_pass;
            if (nbase >= nhi) {
                ++nL;
                if (nL < T.w) {
                    nlo = nhi;
                    nhi = t.lvl_ptr[T.z + nL + 1];
                    nbase = nlo;
                }
            }
            const bool more = nL < T.w;
            const int nidx = nbase + warp * IPW + slot;
            const bool nvalid = more && slot < IPW && nidx < nhi;
            const int2 nit = nvalid ? t.items[nidx] : make_int2(0, 0);
            NodeStage<DIM, P, R> nst;
            if (nvalid) node_stage<DIM, P, MODE, false>(a, nullptr, d, nit.x, r, nst);
            // this pass
            bool ok = true;
            if (valid && (it.y & kTileWaitMask)) ok = wait_faces<DIM, P>(a, t.done, t.epoch, d, it.x, it.y, deadline);
            node_finish<DIM, P, MODE, false>(a, st, d, it.x, r, src0, valid && ok);
            __syncwarp();
            if (valid && ok && r == 0 && (it.y & kTilePublish)) {
                __threadfence();
                st_release(t.done + (size_t)d * a.ne + it.x, t.publish);
            }
            bad = bad || !ok;
            if (nL != L || !more) {  // level boundary: the CTA's angular fluxes of this level are complete
                abort = __syncthreads_or(bad) != 0;
                bad = false;
                if (abort || !more) break;
            }
            L = nL;
            lo = nlo;
            hi = nhi;
            base = nbase;
            valid = nvalid;
            it = nit;
            st = nst;
        }
        if (abort) {
            if (threadIdx.x == 0) atomicExch(t.error, 1);
            break;
        }
    }
}

// ---------------------------------------------------------------- level-barrier sweep (cached operators)
// One cooperative launch per sweep: every CTA takes its share of each level's items (one lane per
// node, node_item) and the CTAs meet at a grid barrier between levels, in place of a kernel
// boundary.  The barrier is an arrival counter: a CTA's thread 0 fences (making the CTA's angular
// fluxes visible), adds one, and polls with acquire loads until every CTA of the level has arrived;
// the poll is bounded and sets the error word when it gives up.
struct BarrierArgs {
    const long long* level_ptr;
    int n_levels;
    int* counter;                    // zeroed before the launch
    int* error;
    int stall;                       // test hook: arrivals are not counted, every wait times out
    unsigned long long timeout_ns;
};

template <int DIM, int P, int MODE>
__global__ void __launch_bounds__(512) barrier_sweep_kernel(SweepArgs a, BarrierArgs b) {
    constexpr int N = Shape<DIM, P>::N, IPW = 32 / N;
    __shared__ int s_fail;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int slot = lane / N, r = lane - slot * N, src0 = slot < IPW ? slot * N : 0;
    using R = typename std::conditional<MODE == 1, float, double>::type;
    const long long per_pass = (long long)(blockDim.x >> 5) * IPW, stride = per_pass * gridDim.x;
    const unsigned long long deadline = globaltimer() + b.timeout_ns;
    // the first pass of a level reads nothing of the previous levels until its face terms, so its
    // stage (item, face fluxes, source row, inverse row) is loaded before the barrier
    auto load_first = [&](int L, int& d, int& e, bool& valid, NodeStage<DIM, P, R>& st) {
        const long long lo = b.level_ptr[L], hi = b.level_ptr[L + 1];
        const long long t = lo + blockIdx.x * per_pass + warp * IPW + slot;
        valid = slot < IPW && t < hi;
        d = e = 0;
        if (valid) {
            const int2 it = a.items[t];
            d = it.x;
            e = it.y;
            node_stage<DIM, P, MODE, false>(a, nullptr, d, e, r, st);
        }
    };
    int d0 = 0, e0 = 0;
    bool v0 = false;
    NodeStage<DIM, P, R> st0;
    if (b.n_levels > 0) load_first(0, d0, e0, v0, st0);
    for (int L = 0; L < b.n_levels; ++L) {
        const long long lo = b.level_ptr[L], hi = b.level_ptr[L + 1];
        node_finish<DIM, P, MODE, false>(a, st0, d0, e0, r, src0, v0);
        for (long long base = lo + blockIdx.x * per_pass + stride; base < hi; base += stride) {
            const long long t = base + warp * IPW + slot;
            const bool valid = slot < IPW && t < hi;
            int d = 0, e = 0;
            if (valid) {
                const int2 it = a.items[t];
                d = it.x;
                e = it.y;
            }
            node_item<DIM, P, MODE, false>(a, nullptr, d, e, r, src0, valid);
        }
        if (L + 1 < b.n_levels) load_first(L + 1, d0, e0, v0, st0);
        __syncthreads();
        if (threadIdx.x == 0) {
            int fail = 0;
            // the CTA barrier orders every thread's stores before this release (cumulative)
            if (!b.stall) asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(b.counter), "r"(1) : "memory");
            const int target = (L + 1) * (int)gridDim.x;
            int polls = 0;
            while (ld_acquire(b.counter) < target) {
                if (++polls > 32) {
                    if (globaltimer() > deadline || *(volatile int*)b.error) {
                        fail = 1;
                        atomicExch(b.error, 1);
                        break;
                    }
                    __nanosleep(32);
                }
            }
            s_fail = fail;
        }
        __syncthreads();
        if (s_fail) return;
    }
}

// Adjoint: A_e^T lam_e = mu_e - sum_{outflow F, downwind u} C(u<-e)^T lam_u, in reverse level order.
template <int DIM, int P>
__device__ __forceinline__ void adjoint_item(const SweepArgs& a, const double* mu, int d, int e) {
    constexpr int Q = P + 1, N = Shape<DIM, P>::N, NT = Shape<DIM, P>::NT;
    const double Ox = a.dirs[3 * d], Oy = a.dirs[3 * d + 1], Oz = a.dirs[3 * d + 2];
    ElemGeom<DIM, P, double> g;
    elem_geom<DIM, P, double>(a, e, Ox, Oy, Oz, g);
    double rhs[N];
#pragma unroll
    for (int i = 0; i < N; ++i) rhs[i] = mu[(size_t)e * N + i];
    const double* lam = static_cast<const double*>(a.psi);
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        if (g.Fd[f] > 0.0) {
            const int u = neighbor<DIM, P>(a, e, f);
            if (u < 0) continue;
            const int ax = f >> 1;
            const bool hi = f & 1;
            const double* lu = lam + ((size_t)d * a.ne + u) * N;
            double vals[N];
#pragma unroll
            for (int i = 0; i < N; ++i) vals[i] = __ldcg(lu + i);
#pragma unroll
            for (int tt = 0; tt < NT; ++tt) {
                double s = 0.0;
#pragma unroll
                for (int k = 0; k < Q; ++k) s += (hi ? c_lm[P][k] : c_lp[P][k]) * vals[node_of<DIM, P>(ax, k, tt)];
                const double ft = g.F[f] * wtan<DIM, P, double>(tt) * s;
#pragma unroll
                for (int ja = 0; ja < Q; ++ja) rhs[node_of<DIM, P>(ax, ja, tt)] += ft * (hi ? c_lp[P][ja] : c_lm[P][ja]);
            }
        }
    }
    double A[N * N];
    assemble<DIM, P, double>(g, a.sigma_t[e], A);
    lu_factor_s<DIM, P, double>(A);
    lu_solve_transpose_s<DIM, P, double>(A, rhs);
    double* out = static_cast<double*>(a.psi) + ((size_t)d * a.ne + e) * N;
#pragma unroll
    for (int i = 0; i < N; ++i) out[i] = rhs[i];
}

template <int DIM, int P>
__global__ void __launch_bounds__(128) adjoint_level_kernel(SweepArgs a, const double* mu, long long begin,
                                                           long long end) {
    const long long t = begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= end) return;
    const int2 it = a.items[t];
    adjoint_item<DIM, P>(a, mu, it.x, it.y);
}

// ---------------------------------------------------------------- level sets (Kahn, on device)
template <int DIM, int P>
__global__ void indegree_kernel(SweepArgs a, int* indeg, int2* frontier, unsigned long long* cursor) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)a.nd * a.ne) return;
    const int d = (int)(t / a.ne), e = (int)(t % a.ne);
    const double Ox = a.dirs[3 * d], Oy = a.dirs[3 * d + 1], Oz = a.dirs[3 * d + 2];
    int c = 0;
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f)
        if (face_flux_only<DIM, P>(a, e, f, Ox, Oy, Oz) < 0.0 && neighbor<DIM, P>(a, e, f) >= 0) ++c;
    indeg[t] = c;
    if (c == 0) {
        const unsigned long long pos = atomicAdd(cursor, 1ull);
        frontier[pos] = make_int2(d, e);
    }
}

template <int DIM, int P>
__global__ void upwind_mask_kernel(SweepArgs a, unsigned char* mask) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)a.nd * a.ne) return;
    const int d = (int)(t / a.ne), e = (int)(t % a.ne);
    const double Ox = a.dirs[3 * d], Oy = a.dirs[3 * d + 1], Oz = a.dirs[3 * d + 2];
    unsigned m = 0;
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f)
        if (face_flux_only<DIM, P>(a, e, f, Ox, Oy, Oz) < 0.0 && neighbor<DIM, P>(a, e, f) >= 0) m |= 1u << f;
    mask[t] = (unsigned char)m;
}

template <int DIM, int P>
__global__ void kahn_level_kernel(SweepArgs a, int* indeg, int2* list, int* level, long long begin, long long end,
                                  int L, unsigned long long* cursor) {
    const long long t = begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= end) return;
    const int2 it = list[t];
    const int d = it.x, e = it.y;
    level[(size_t)d * a.ne + e] = L;
    const double Ox = a.dirs[3 * d], Oy = a.dirs[3 * d + 1], Oz = a.dirs[3 * d + 2];
#pragma unroll
    for (int f = 0; f < 2 * DIM; ++f) {
        if (face_flux_only<DIM, P>(a, e, f, Ox, Oy, Oz) > 0.0) {
            const int u = neighbor<DIM, P>(a, e, f);
            if (u < 0) continue;
            if (atomicSub(&indeg[(size_t)d * a.ne + u], 1) == 1) {
                const unsigned long long pos = atomicAdd(cursor, 1ull);
                list[pos] = make_int2(d, u);
            }
        }
    }
}

// ---------------------------------------------------------------- reductions
// phi_out = sum over directions d0 <= d < d1 of w_d psi_d (in increasing d), and partial sums of
// ||phi_out - phi_in||^2 per block.
template <typename RS>
__global__ void phi_reduce_kernel(const RS* psi, const double* w, int d0, int d1, size_t M, const double* phi_in,
                                  double* phi_out, double* partial) {
    __shared__ double sh[256];
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0.0;
    if (idx < M) {
        double s = 0.0;
        for (int d = d0; d < d1; ++d) s += w[d] * (double)psi[(size_t)d * M + idx];
        const double r = s - (phi_in ? phi_in[idx] : 0.0);
        phi_out[idx] = s;
        rr = r * r;
    }
    sh[threadIdx.x] = rr;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0 && partial) partial[blockIdx.x] = sh[0];
}

__global__ void final_sum_kernel(const double* partial, int n, double* out) {
    __shared__ double sh[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// out = a - b and ||out||^2 partials (b may be null: out = a).
__global__ void diff_norm_kernel(const double* a, const double* b, double* out, size_t M, double* partial) {
    __shared__ double sh[256];
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0.0;
    if (idx < M) {
        const double r = a[idx] - (b ? b[idx] : 0.0);
        if (out) out[idx] = r;
        rr = r * r;
    }
    sh[threadIdx.x] = rr;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// out[e][i] = sigma_s[e] M_i / (4 pi) * sum_d w_d lam_d[e][i]
template <int DIM, int P>
__global__ void adjoint_reduce_kernel(SweepArgs a, const double* lam, const double* w, double* out) {
    constexpr int N = Shape<DIM, P>::N;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t M = (size_t)a.ne * N;
    if (idx >= M) return;
    const int e = (int)(idx / N);
    double s = 0.0;
    for (int d = 0; d < a.nd; ++d) s += w[d] * lam[(size_t)d * M + idx];
    out[idx] = a.sigma_s[e] * a.mass[idx] / kFourPi * s;
}

template <int DIM, int P>
__global__ void gradient_kernel(SweepArgs a, const double* psi, const double* lam, const double* w,
                                const double* phi, double* gt, double* gs, double* gq) {
    constexpr int N = Shape<DIM, P>::N;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.ne) return;
    double M[N];
#pragma unroll
    for (int i = 0; i < N; ++i) M[i] = a.mass[(size_t)e * N + i];
    double st = 0.0, ssum = 0.0, sq = 0.0;
    const size_t stride = (size_t)a.ne * N;
    for (int d = 0; d < a.nd; ++d) {
        const double* l = lam + d * stride + (size_t)e * N;
        const double* p = psi + d * stride + (size_t)e * N;
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const double lm = l[i] * M[i];
            t1 += lm * p[i];
            t2 += lm * phi[(size_t)e * N + i];
            t3 += lm;
        }
        st += w[d] * t1;
        ssum += w[d] * t2;
        sq += w[d] * t3;
    }
    if (gt) gt[e] = -st;
    if (gs) gs[e] = ssum / kFourPi;
    if (gq) gq[e] = sq / kFourPi;
}

// ---------------------------------------------------------------- host launchers
static SweepArgs make_args(const sn_mesh* m) {
    SweepArgs a{};
    a.dim = m->dim;
    a.p = m->p;
    a.nx = m->nx;
    a.ny = m->ny;
    a.nz = m->nz;
    a.ne = m->ne;
    a.nd = m->nd;
    a.hx = m->hx;
    a.hy = m->hy;
    a.hz = m->hz;
    a.psi_inc = m->desc.psi_inc;
    a.dirs = m->d_dirs;
    a.corners = m->d_corners;
    a.sigma_t = m->d_sigma_t;
    a.sigma_s = m->d_sigma_s;
    a.q = m->d_q;
    a.items = m->levels.items;
    a.mass = m->d_mass;
    a.mass4 = m->d_mass4;
    a.q_scale = 1.0;
    a.ainv = m->cache_mode != SN_CACHE_OFF ? m->d_ainv : nullptr;
    a.ainv32 = m->cache_mode != SN_CACHE_OFF ? m->d_ainv32 : nullptr;
    a.fflux = m->d_fflux;
    if (m->d_in32 && m->cache_mode != SN_CACHE_OFF) {  // layout: fflux32, q32 (ne), mass32 (ne n)
        const size_t nf = m->dim == 2 ? (size_t)m->nd * m->ne * 4 : (size_t)m->nd * 3;
        a.fflux32 = m->d_in32;
        a.q32 = m->d_in32 + nf;
        a.mass32 = a.q32 + m->ne;
    }
    return a;
}

// The linear part of the update: no fixed source and vacuum inflow.
static void linear_part(SweepArgs& a) {
    a.q_scale = 0.0;
    a.psi_inc = 0.0;
    a.q = nullptr;
    a.q32 = nullptr;
}

#define SN_DISPATCH(DIMV, PV, CALL)                                             \
    do {                                                                        \
        if ((DIMV) == 2 && (PV) == 1) { constexpr int D_ = 2, P_ = 1; CALL; }   \
        else if ((DIMV) == 2 && (PV) == 2) { constexpr int D_ = 2, P_ = 2; CALL; } \
        else if ((DIMV) == 2 && (PV) == 3) { constexpr int D_ = 2, P_ = 3; CALL; } \
        else if ((DIMV) == 3 && (PV) == 1) { constexpr int D_ = 3, P_ = 1; CALL; } \
        else return cudaErrorInvalidValue;                                      \
    } while (0)

static inline unsigned grid_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

// Blocks of bs threads for n items of the node-per-lane kernels (32 / N items per warp).
static inline unsigned node_grid(const sn_mesh* m, long long n, int bs) {
    const int ipw = 32 / m->n;
    const long long warps = (n + ipw - 1) / ipw;
    return grid_for(warps * 32, bs);
}

cudaError_t compute_mass(sn_mesh* m, cudaStream_t s) {
    SweepArgs a = make_args(m);
    const long long M = (long long)m->ne * m->n;
    SN_COUNT_LAUNCH();
    SN_DISPATCH(m->dim, m->p, (mass_kernel<D_, P_><<<grid_for(M, 256), 256, 0, s>>>(a, m->d_mass, m->d_mass4)));
    return cudaGetLastError();
}

cudaError_t build_levels(sn_mesh* m, cudaStream_t s, bool* cycle) {
    *cycle = false;
    const long long total = (long long)m->nd * m->ne;
    int* indeg = nullptr;
    int* level = nullptr;
    int2* list = nullptr;
    unsigned long long* cursor = nullptr;
    cudaError_t err;
    if ((err = cudaMalloc(&indeg, total * sizeof(int))) != cudaSuccess) return err;
    if ((err = cudaMalloc(&level, total * sizeof(int))) != cudaSuccess) { cudaFree(indeg); return err; }
    if ((err = cudaMalloc(&list, total * sizeof(int2))) != cudaSuccess) { cudaFree(indeg); cudaFree(level); return err; }
    if ((err = cudaMalloc(&cursor, sizeof(unsigned long long))) != cudaSuccess) {
        cudaFree(indeg); cudaFree(level); cudaFree(list);
        return err;
    }
    auto cleanup = [&]() { cudaFree(indeg); cudaFree(level); cudaFree(list); cudaFree(cursor); };
    SweepArgs a = make_args(m);
    cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s);
    cudaMemsetAsync(level, 0xff, total * sizeof(int), s);
    auto run_init = [&]() -> cudaError_t {
        SN_COUNT_LAUNCH();
        SN_DISPATCH(m->dim, m->p, (indegree_kernel<D_, P_><<<grid_for(total, 256), 256, 0, s>>>(a, indeg, list, cursor)));
        return cudaGetLastError();
    };
    if ((err = run_init()) != cudaSuccess) { cleanup(); return err; }
    unsigned long long h_cursor = 0;
    long long begin = 0;
    int L = 0;
    if ((err = cudaMemcpyAsync(&h_cursor, cursor, sizeof(h_cursor), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess) { cleanup(); return err; }
    while ((long long)h_cursor > begin) {
        const long long end = (long long)h_cursor;
        auto run_level = [&]() -> cudaError_t {
            SN_DISPATCH(m->dim, m->p,
                        (kahn_level_kernel<D_, P_><<<grid_for(end - begin, 256), 256, 0, s>>>(a, indeg, list, level, begin, end, L, cursor)));
            return cudaGetLastError();
        };
        if ((err = run_level()) != cudaSuccess) { cleanup(); return err; }
        begin = end;
        ++L;
        if ((err = cudaMemcpyAsync(&h_cursor, cursor, sizeof(h_cursor), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (err = cudaStreamSynchronize(s)) != cudaSuccess) { cleanup(); return err; }
    }
    if (begin != total) {
        *cycle = true;
        cleanup();
        return cudaSuccess;
    }
    // deterministic order: counting sort of (dir, elem) by level on the host
    std::vector<int>& h_level = m->levels.h_level;
    h_level.assign(total, 0);
    if ((err = cudaMemcpyAsync(h_level.data(), level, total * sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess) { cleanup(); return err; }
    std::vector<long long> ptr(L + 1, 0);
    for (long long t = 0; t < total; ++t) ptr[h_level[t] + 1]++;
    for (int l = 0; l < L; ++l) ptr[l + 1] += ptr[l];
    std::vector<long long> fill(ptr.begin(), ptr.end() - 1);
    std::vector<int2> items(total);
    for (long long t = 0; t < total; ++t) {
        const int d = (int)(t / m->ne), e = (int)(t % m->ne);
        items[fill[h_level[t]]++] = make_int2(d, e);
    }
    if (m->levels.items) cudaFree(m->levels.items);
    m->levels.items = nullptr;
    if ((err = cudaMalloc(&m->levels.items, total * sizeof(int2))) != cudaSuccess) { cleanup(); return err; }
    if ((err = cudaMemcpyAsync(m->levels.items, items.data(), total * sizeof(int2), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (err = cudaStreamSynchronize(s)) != cudaSuccess) { cleanup(); return err; }
    m->levels.level_ptr = ptr;
    m->levels.n_levels = L;
    // padded list for the dataflow schedule: no 32-item chunk crosses a level boundary
    std::vector<int2> padded;
    padded.reserve(total + 32 * (size_t)L);
    for (int l = 0; l < L; ++l) {
        for (long long t = ptr[l]; t < ptr[l + 1]; ++t) padded.push_back(items[t]);
        while (padded.size() % 32) padded.push_back(make_int2(-1, -1));
    }
    if (m->levels.padded) cudaFree(m->levels.padded);
    m->levels.padded = nullptr;
    m->levels.n_padded = (long long)padded.size();
    if ((err = cudaMalloc(&m->levels.padded, padded.size() * sizeof(int2))) != cudaSuccess) { cleanup(); return err; }
    if ((err = cudaMemcpyAsync(m->levels.padded, padded.data(), padded.size() * sizeof(int2), cudaMemcpyHostToDevice, s)) != cudaSuccess) { cleanup(); return err; }
    std::vector<int2> padded_rev;
    padded_rev.reserve(padded.size());
    for (int l = L - 1; l >= 0; --l) {
        for (long long t = ptr[l]; t < ptr[l + 1]; ++t) padded_rev.push_back(items[t]);
        while (padded_rev.size() % 32) padded_rev.push_back(make_int2(-1, -1));
    }
    if (m->levels.padded_rev) cudaFree(m->levels.padded_rev);
    m->levels.padded_rev = nullptr;
    if ((err = cudaMalloc(&m->levels.padded_rev, padded_rev.size() * sizeof(int2))) != cudaSuccess) { cleanup(); return err; }
    if ((err = cudaMemcpyAsync(m->levels.padded_rev, padded_rev.data(), padded_rev.size() * sizeof(int2), cudaMemcpyHostToDevice, s)) != cudaSuccess) { cleanup(); return err; }
    if (!m->levels.done) {
        if ((err = cudaMalloc(&m->levels.done, total * sizeof(int))) != cudaSuccess) { cleanup(); return err; }
        if ((err = cudaMalloc(&m->levels.ctrl, 3 * sizeof(unsigned long long))) != cudaSuccess) { cleanup(); return err; }
    }
    cudaMemsetAsync(m->levels.done, 0, total * sizeof(int), s);
    cudaMemsetAsync(m->levels.ctrl, 0, 3 * sizeof(unsigned long long), s);
    m->levels.epoch = 0;
    if ((err = cudaStreamSynchronize(s)) != cudaSuccess) { cleanup(); return err; }
    cleanup();
    return cudaSuccess;
}

void free_level_groups(sn_mesh* m) {
    LevelSets& L = m->levels;
    if (L.gitems) cudaFree(L.gitems);
    L.gitems = nullptr;
    for (cudaStream_t st : L.gstreams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : L.gevents) cudaEventDestroy(ev);
    L.gstreams.clear();
    L.gevents.clear();
    L.gptr.clear();
    L.groups = 0;
}

// Directions are independent, so the level schedule may run G groups of directions as G chains
// of level launches: a chain's levels are those of its own directions, and the deepest direction
// no longer makes every other direction wait at each of its levels.
// Appends the items (d, e) of directions d0 <= d < d1 to `items`, grouped by level (level sets of
// the mesh, directions then elements ascending inside a level); returns the level boundaries.
static std::vector<long long> append_level_list(const sn_mesh* m, int d0, int d1, std::vector<int2>& items) {
    const int ne = m->ne;
    const std::vector<int>& lev = m->levels.h_level;
    int depth = 0;
    for (int d = d0; d < d1; ++d)
        for (int e = 0; e < ne; ++e) depth = std::max(depth, lev[(size_t)d * ne + e] + 1);
    std::vector<long long> cnt(depth + 1, 0);
    for (int d = d0; d < d1; ++d)
        for (int e = 0; e < ne; ++e) cnt[lev[(size_t)d * ne + e] + 1]++;
    for (int l = 0; l < depth; ++l) cnt[l + 1] += cnt[l];
    const long long base = (long long)items.size();
    items.resize(base + cnt[depth]);
    std::vector<long long> fill(cnt.begin(), cnt.end() - 1);
    for (int d = d0; d < d1; ++d)
        for (int e = 0; e < ne; ++e) items[base + fill[lev[(size_t)d * ne + e]]++] = make_int2(d, e);
    for (long long& c : cnt) c += base;
    return cnt;
}

cudaError_t build_level_groups(sn_mesh* m, int G) {
    free_level_groups(m);
    LevelSets& L = m->levels;
    const int nd = m->nd, ne = m->ne;
    G = std::max(1, std::min(G, nd));
    std::vector<int2> items;
    items.reserve((size_t)nd * ne);
    L.gptr.assign(G, {});
    for (int g = 0; g < G; ++g)
        L.gptr[g] = append_level_list(m, (int)((long long)g * nd / G), (int)((long long)(g + 1) * nd / G), items);
    cudaError_t err;
    if ((err = cudaMalloc(&L.gitems, items.size() * sizeof(int2))) != cudaSuccess) {
        L.gitems = nullptr;
        return err;
    }
    if ((err = cudaMemcpy(L.gitems, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice)) != cudaSuccess)
        return err;
    // two sets of fork/join streams and events: a recorded outer iteration captures level chains
    // into two nested graphs at once (outer and inner loop bodies), and a stream joins one capture
    L.gstreams.resize(2 * G, nullptr);
    for (auto& st : L.gstreams)
        if ((err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return err;
    L.gevents.resize(2 * (G + 1), nullptr);
    for (auto& ev : L.gevents)
        if ((err = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return err;
    L.groups = G;
    return cudaSuccess;
}

__global__ void bump_device_epoch_kernel(unsigned long long* ctrl) { ctrl[2] += 1; }

template <int DIM, int P, int MODE, bool ADJ = false>
static cudaError_t launch_dataflow(sn_mesh* m, const SweepArgs& a, cudaStream_t s, const double* mu = nullptr) {
    LevelSets& L = m->levels;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t cerr = cudaStreamIsCapturing(s, &cs);
    if (cerr != cudaSuccess) return cerr;
    const bool recorded = cs == cudaStreamCaptureStatusActive;
    if (!recorded && ++L.epoch == 0x7fffffff) {  // epochs wrap: start over from a cleared table
        cudaMemsetAsync(L.done, 0, (size_t)m->nd * m->ne * sizeof(int), s);
        L.epoch = 1;
    }
    cudaMemsetAsync(L.ctrl, 0, sizeof(unsigned long long), s);
    DataflowArgs f;
    f.epoch_dev = nullptr;
    if (recorded) {
        // inside a recorded iteration the epoch lives on the device (ctrl[2], set from the host's
        // before the graph runs and read back after it): a one-thread kernel advances it per sweep
        SN_COUNT_LAUNCH();
        bump_device_epoch_kernel<<<1, 1, 0, s>>>(L.ctrl);
        f.epoch_dev = reinterpret_cast<const int*>(L.ctrl + 2);
    }
    f.items = ADJ ? L.padded_rev : L.padded;
    f.n_items = L.n_padded;
    f.done = L.done;
    f.epoch = L.epoch;
    f.next = L.ctrl;
    f.error = reinterpret_cast<int*>(L.ctrl + 1);
    f.timeout_ns = 4000000000ull;
    f.publish = L.epoch;
    if (L.stall_timeout_s > 0.0) {  // test hook: completion words never match, every wait times out
        f.publish = -1;
        f.timeout_ns = (unsigned long long)(L.stall_timeout_s * 1e9);
        L.stall_timeout_s = 0.0;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool cached = MODE == 1 ? a.ainv32 != nullptr : (MODE == 0 && a.ainv != nullptr);
    // cached sweeps poll the upwind (adjoint: downwind) angular fluxes themselves (node_datapoll_kernel)
    const bool datapoll = cached;
    if (datapoll) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, node_datapoll_kernel<DIM, P, MODE == 1 ? 1 : 0, ADJ>, m->block, 0);
    else if (cached) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, node_dataflow_kernel<DIM, P, MODE == 1 ? 1 : 0, ADJ>, m->block, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_dataflow_kernel<DIM, P, MODE, ADJ>, m->block, 0);
    if (m->max_blocks_per_sm > 0 && m->max_blocks_per_sm < per_sm) per_sm = m->max_blocks_per_sm;
    per_sm = per_sm < 1 ? 1 : per_sm;
    const long long warps_needed = cached ? (L.n_padded / 32) * ((32 + (32 / m->n) - 1) / (32 / m->n)) : L.n_padded / 32;
    long long blocks = (long long)sms * per_sm;
    const long long cap = (warps_needed * 32 + m->block - 1) / m->block;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    // static assignment needs every warp resident: the grid never exceeds one wave
    f.static_warps = m->schedule == SCHED_STATIC ? blocks * (m->block / 32) : 0;
    if (datapoll) {
        // every angular flux of the sweep starts as the unset pattern (all bits one)
        const size_t bytes = (size_t)m->nd * m->ne * m->n * (MODE == 1 ? sizeof(float) : sizeof(double));
        cudaError_t merr = cudaMemsetAsync(a.psi, 0xFF, bytes, s);
        if (merr != cudaSuccess) return merr;
        SN_COUNT_LAUNCH();
        node_datapoll_kernel<DIM, P, MODE == 1 ? 1 : 0, ADJ><<<(unsigned)blocks, m->block, 0, s>>>(a, f, mu);
        return cudaGetLastError();
    }
    SN_COUNT_LAUNCH();
    if (cached) node_dataflow_kernel<DIM, P, MODE == 1 ? 1 : 0, ADJ><<<(unsigned)blocks, m->block, 0, s>>>(a, f, mu);
    else sweep_dataflow_kernel<DIM, P, MODE, ADJ><<<(unsigned)blocks, m->block, 0, s>>>(a, f, mu);
    return cudaGetLastError();
}

cudaError_t launch_upwind_mask(sn_mesh* m, unsigned char* mask, cudaStream_t s) {
    SweepArgs a = make_args(m);
    const long long total = (long long)m->nd * m->ne;
    SN_COUNT_LAUNCH();
    SN_DISPATCH(m->dim, m->p, (upwind_mask_kernel<D_, P_><<<grid_for(total, 256), 256, 0, s>>>(a, mask)));
    return cudaGetLastError();
}

template <int DIM, int P, int MODE>
static cudaError_t launch_tiles(sn_mesh* m, const SweepArgs& a, cudaStream_t s) {
    LevelSets& L = m->levels;
    if (++L.epoch == 0x7fffffff) {
        cudaMemsetAsync(L.done, 0, (size_t)m->nd * m->ne * sizeof(int), s);
        L.epoch = 1;
    }
    cudaMemsetAsync(L.ctrl, 0, sizeof(unsigned long long), s);
    TileArgs t;
    t.tasks = m->tiles.tasks;
    t.lvl_ptr = m->tiles.lvl_ptr;
    t.items = m->tiles.items;
    t.n_tasks = m->tiles.n_tasks;
    t.done = L.done;
    t.epoch = L.epoch;
    t.publish = L.epoch;
    t.next = L.ctrl;
    t.error = reinterpret_cast<int*>(L.ctrl + 1);
    t.timeout_ns = 4000000000ull;
    if (L.stall_timeout_s > 0.0) {  // test hook: completion words never match, every wait times out
        t.publish = -1;
        t.timeout_ns = (unsigned long long)(L.stall_timeout_s * 1e9);
        L.stall_timeout_s = 0.0;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tile_sweep_kernel<DIM, P, MODE>, m->tile_block, 0);
    per_sm = per_sm < 1 ? 1 : per_sm;
    long long blocks = (long long)sms * per_sm;
    if (blocks > t.n_tasks) blocks = t.n_tasks;
    if (blocks < 1) blocks = 1;
    SN_COUNT_LAUNCH();
    tile_sweep_kernel<DIM, P, MODE><<<(unsigned)blocks, m->tile_block, 0, s>>>(a, t);
    return cudaGetLastError();
}

template <int DIM, int P, int MODE>
static cudaError_t launch_barrier_sweep(sn_mesh* m, const SweepArgs& a, cudaStream_t s) {
    LevelSets& L = m->levels;
    cudaError_t err;
    if (!L.d_level_ptr) {
        if ((err = cudaMalloc(&L.d_level_ptr, L.level_ptr.size() * sizeof(long long))) != cudaSuccess) {
            L.d_level_ptr = nullptr;
            return err;
        }
        if ((err = cudaMemcpy(L.d_level_ptr, L.level_ptr.data(), L.level_ptr.size() * sizeof(long long),
                              cudaMemcpyHostToDevice)) != cudaSuccess)
            return err;
        if ((err = cudaMalloc(&L.d_barrier, sizeof(int))) != cudaSuccess) {
            L.d_barrier = nullptr;
            return err;
        }
    }
    BarrierArgs b;
    b.level_ptr = L.d_level_ptr;
    b.n_levels = L.n_levels;
    b.counter = L.d_barrier;
    b.error = reinterpret_cast<int*>(L.ctrl + 1);
    b.stall = 0;
    b.timeout_ns = 4000000000ull;
    if (L.stall_timeout_s > 0.0) {
        b.stall = 1;
        b.timeout_ns = (unsigned long long)(L.stall_timeout_s * 1e9);
        L.stall_timeout_s = 0.0;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, barrier_sweep_kernel<DIM, P, MODE>, m->barrier_block, 0);
    per_sm = std::min(per_sm, m->barrier_ctas_per_sm);
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if ((err = cudaMemsetAsync(L.d_barrier, 0, sizeof(int), s)) != cudaSuccess) return err;
    void* args[] = {const_cast<SweepArgs*>(&a), &b};
    SN_COUNT_LAUNCH();
    return cudaLaunchCooperativeKernel((const void*)barrier_sweep_kernel<DIM, P, MODE>, dim3(sms * per_sm),
                                       dim3(m->barrier_block), args, 0, s);
}

// One chain of level launches over the level boundaries `ptr` of the items in a.items, in
// increasing order (reverse: decreasing, the adjoint); within a chain every launch after the first
// uses programmatic dependent launch.
static cudaError_t enqueue_chain(sn_mesh* m, int kind, const SweepArgs& a, const std::vector<long long>& ptr,
                                 cudaStream_t s) {
    const int bs = m->block;
    const int nl = (int)ptr.size() - 1;
    bool first = true;
    for (int q = 0; q < nl; ++q) {
        const int L = kind == 3 ? nl - 1 - q : q;
        const long long b = ptr[L], e = ptr[L + 1];
        if (e <= b) continue;
        const unsigned g = grid_for(e - b, bs), gn = node_grid(m, e - b, bs);
        cudaError_t lerr = cudaSuccess;
        const double* none = nullptr;
        const bool pdl = !first && !m->capture_no_pdl;
        first = false;
        if (kind == 3 && a.ainv)
            SN_DISPATCH(m->dim, m->p, (lerr = launch_k(pdl, node_level_kernel<D_, P_, 0, true>, gn, bs, s, a, (const double*)m->d_src, b, e)));
        else if (kind == 3)
            SN_DISPATCH(m->dim, m->p, (adjoint_level_kernel<D_, P_><<<g, bs, 0, s>>>(a, m->d_src, b, e)));
        else if (kind == SN_FP64 && a.ainv)
            SN_DISPATCH(m->dim, m->p, (lerr = launch_k(pdl, node_level_kernel<D_, P_, 0, false>, gn, bs, s, a, none, b, e)));
        else if (kind == SN_FP32 && a.ainv32)
            SN_DISPATCH(m->dim, m->p, (lerr = launch_k(pdl, node_level_kernel<D_, P_, 1, false>, gn, bs, s, a, none, b, e)));
        else if (kind == SN_FP64) SN_DISPATCH(m->dim, m->p, (sweep_level_kernel<D_, P_, 0><<<g, bs, 0, s>>>(a, b, e)));
        else if (kind == SN_FP32) SN_DISPATCH(m->dim, m->p, (sweep_level_kernel<D_, P_, 1><<<g, bs, 0, s>>>(a, b, e)));
        else SN_DISPATCH(m->dim, m->p, (sweep_level_kernel<D_, P_, 2><<<g, bs, 0, s>>>(a, b, e)));
        if (lerr != cudaSuccess) return lerr;
    }
    return cudaGetLastError();
}

// Level schedule: the launches of one sweep are captured once into a CUDA graph per kind
// (forward FP64 / FP32 / FP32+refinement, adjoint, and the forward kinds without the fixed
// source); the kernels read their source vector from the mesh-owned buffer d_src so the captured
// parameters never change.  With direction groups the graph forks into one chain per group.
static cudaError_t enqueue_levels(sn_mesh* m, int kind, cudaStream_t s) {
    SweepArgs a = make_args(m);
    a.q_scale = 1.0;
    if (kind == 3) {
        a.psi = m->d_lambda;
    } else {
        if (kind >= 4) {  // the linear part: no fixed source and vacuum inflow
            linear_part(a);
            kind -= 4;
        }
        a.phi = m->d_src;
        a.psi = kind == SN_FP32 ? m->d_psi32 : m->d_psi;
    }
    LevelSets& L = m->levels;
    if (m->level_groups <= 1) return enqueue_chain(m, kind, a, L.level_ptr, s);
    if (L.groups != m->level_groups) return cudaErrorInvalidValue;  // built before the capture starts
    cudaError_t err;
    a.items = L.gitems;
    const int set = s == m->ig_stream[2] ? 1 : 0;  // the inner loop body of a recorded iteration
    cudaStream_t* gst = L.gstreams.data() + set * L.groups;
    cudaEvent_t* gev = L.gevents.data() + set * (L.groups + 1);
    if ((err = cudaEventRecord(gev[0], s)) != cudaSuccess) return err;
    for (int g = 0; g < L.groups; ++g) {
        cudaStream_t gs = gst[g];
        if ((err = cudaStreamWaitEvent(gs, gev[0], 0)) != cudaSuccess) return err;
        if ((err = enqueue_chain(m, kind, a, L.gptr[g], gs)) != cudaSuccess) return err;
        if ((err = cudaEventRecord(gev[1 + g], gs)) != cudaSuccess) return err;
        if ((err = cudaStreamWaitEvent(s, gev[1 + g], 0)) != cudaSuccess) return err;
    }
    return cudaSuccess;
}

static cudaError_t launch_levels_graph(sn_mesh* m, int kind, cudaStream_t s) {
    cudaError_t err;
    auto kernels_per_sweep = [m]() {
        long long kernels = m->levels.n_levels;
        if (m->level_groups > 1) {
            kernels = 0;
            for (const auto& ptr : m->levels.gptr) kernels += (long long)ptr.size() - 1;
        }
        return kernels;
    };
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((err = cudaStreamIsCapturing(s, &cs)) != cudaSuccess) return err;
    if (cs == cudaStreamCaptureStatusActive) {
        // recorded into an enclosing graph (an outer iteration): the level chain itself, not a
        // nested graph launch; the direction groups must have been built before the capture
        if (m->level_groups > 1 && m->levels.groups != m->level_groups) return cudaErrorStreamCaptureUnsupported;
        g_launches.fetch_add(kernels_per_sweep(), std::memory_order_relaxed);
        return enqueue_levels(m, kind, s);
    }
    if (!m->level_graph[kind]) {
        if (!m->cap_stream && (err = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return err;
        if (m->level_groups > 1 && m->levels.groups != m->level_groups &&
            (err = build_level_groups(m, m->level_groups)) != cudaSuccess)
            return err;
        if ((err = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return err;
        cudaError_t qerr = enqueue_levels(m, kind, m->cap_stream);
        cudaGraph_t graph = nullptr;
        err = cudaStreamEndCapture(m->cap_stream, &graph);
        if (qerr != cudaSuccess) err = qerr;
        if (err == cudaSuccess) err = cudaGraphInstantiate(&m->level_graph[kind], graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (err != cudaSuccess) {
            m->level_graph[kind] = nullptr;
            return err;
        }
    }
    g_launches.fetch_add(kernels_per_sweep(), std::memory_order_relaxed);
    return cudaGraphLaunch(m->level_graph[kind], s);
}

void drop_level_graphs(sn_mesh* m) {
    for (auto& g : m->level_graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    drop_iter_graph(m);  // it holds copies of the level chains
}

void drop_iter_graph(sn_mesh* m) {
    if (m->iter_graph) cudaGraphExecDestroy(m->iter_graph);
    m->iter_graph = nullptr;
    m->iter_key.clear();
}

// Everything a recorded sweep of this precision needs that allocates or launches set-up work: the
// operator cache and the direction-group lists of the level schedule.
cudaError_t prepare_recorded_sweep(sn_mesh* m, int precision, cudaStream_t s) {
    cudaError_t err = prepare_operator_cache(m, precision, s);
    if (err != cudaSuccess) return err;
    if (m->schedule == SCHED_LEVELS && m->level_groups > 1 && m->levels.groups != m->level_groups)
        err = build_level_groups(m, m->level_groups);
    return err;
}

// Float32 copies of the inputs of the FP32 cached solves (layout of SweepArgs::fflux32 .. mass32):
// face flux factors, q per element, mass / (4 pi) per node.
__global__ void fp32_inputs_kernel(const double* fflux, long long nf, const double* q, const double* mass, int ne,
                                   int n, float* out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nf + ne + (long long)ne * n) return;
    double v;
    if (t < nf) v = fflux[t];
    else if (t < nf + ne) v = q[t - nf];
    else v = mass[t - nf - ne] * (1.0 / kFourPi);
    out[t] = (float)v;
}

cudaError_t prepare_operator_cache(sn_mesh* m, int precision, cudaStream_t s) {
    if (m->cache_mode == SN_CACHE_OFF || precision == SN_FP32_REFINE) return cudaSuccess;
    const bool f32 = precision == SN_FP32;
    void** buf = f32 ? reinterpret_cast<void**>(&m->d_ainv32) : reinterpret_cast<void**>(&m->d_ainv);
    bool& valid = f32 ? m->ainv32_valid : m->ainv_valid;
    bool& denied = f32 ? m->ainv32_denied : m->ainv_denied;
    const long long total = (long long)m->nd * m->ne;
    cudaError_t err;
    if (!*buf) {
        if (denied) return cudaSuccess;
        const size_t bytes = (size_t)total * cache_stride(m->dim, m->p) * (f32 ? sizeof(float) : sizeof(double));
        size_t free_b = 0, total_b = 0;
        if ((err = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) return err;
        if (m->cache_mode == SN_CACHE_AUTO && bytes > free_b / 2) {
            denied = true;
            return cudaSuccess;
        }
        if ((err = cudaMalloc(buf, bytes)) != cudaSuccess) {
            *buf = nullptr;
            if (m->cache_mode != SN_CACHE_AUTO) return err;
            cudaGetLastError();  // out of memory is not sticky: fall back to on-the-fly solves
            denied = true;
            return cudaSuccess;
        }
        if (!m->d_fflux) {
            const size_t fb = (m->dim == 2 ? (size_t)total * 4 : (size_t)m->nd * 3) * sizeof(double);
            if ((err = cudaMalloc(&m->d_fflux, fb)) != cudaSuccess) {
                m->d_fflux = nullptr;
                cudaFree(*buf);
                *buf = nullptr;
                if (m->cache_mode != SN_CACHE_AUTO) return err;
                cudaGetLastError();
                denied = true;
                return cudaSuccess;
            }
        }
        drop_level_graphs(m);  // captured launches carry the cache pointers
        valid = false;
    }
    if (!valid) {
        SweepArgs a = make_args(m);
        SN_COUNT_LAUNCH();
        if (f32)
            SN_DISPATCH(m->dim, m->p, (factor_kernel<D_, P_, float><<<grid_for(total, 128), 128, 0, s>>>(a, m->d_ainv32, m->d_fflux)));
        else
            SN_DISPATCH(m->dim, m->p, (factor_kernel<D_, P_, double><<<grid_for(total, 128), 128, 0, s>>>(a, m->d_ainv, m->d_fflux)));
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if (f32) {  // the float32 inputs of the FP32 solves, from the same materials
            const long long nf = m->dim == 2 ? total * 4 : (long long)m->nd * 3;
            const long long n32 = nf + m->ne + (long long)m->ne * m->n;
            if (!m->d_in32) {
                if ((err = cudaMalloc(&m->d_in32, n32 * sizeof(float))) != cudaSuccess) {
                    m->d_in32 = nullptr;
                    return err;
                }
                drop_level_graphs(m);  // captured launches carry the argument pointers
            }
            SN_COUNT_LAUNCH();
            fp32_inputs_kernel<<<grid_for(n32, 256), 256, 0, s>>>(m->d_fflux, nf, m->d_q, m->d_mass, m->ne, m->n,
                                                                  m->d_in32);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
        }
        valid = true;
    }
    return cudaSuccess;
}

void free_operator_cache(sn_mesh* m) {
    if (m->d_ainv) cudaFree(m->d_ainv);
    if (m->d_ainv32) cudaFree(m->d_ainv32);
    if (m->d_fflux) cudaFree(m->d_fflux);
    if (m->d_in32) cudaFree(m->d_in32);
    m->d_ainv = nullptr;
    m->d_ainv32 = nullptr;
    m->d_fflux = nullptr;
    m->d_in32 = nullptr;
    m->ainv_valid = m->ainv32_valid = false;
}

// Brings every instance's cached inverses up to date and points the batch's argument table at
// them.  The batch runs the cached (node-per-lane) kernels only when every instance has a cache
// for this precision; a change of that choice drops the recorded graphs.
cudaError_t batch_refresh_cache(sn_batch* b, int precision, cudaStream_t s) {
    bool changed = false, all = precision != SN_FP32_REFINE;
    for (int i = 0; i < b->count; ++i) {
        sn_mesh* m = b->meshes[i];
        cudaError_t err = prepare_operator_cache(m, precision, s);
        if (err != cudaSuccess) return err;
        const SweepArgs fresh = make_args(m);
        all = all && (precision == SN_FP32 ? fresh.ainv32 != nullptr : fresh.ainv != nullptr);
        SweepArgs& h = b->h_args[i];
        if (fresh.ainv != h.ainv || fresh.ainv32 != h.ainv32 || fresh.fflux != h.fflux || fresh.fflux32 != h.fflux32 ||
            fresh.q32 != h.q32 || fresh.mass32 != h.mass32) {
            h.ainv = fresh.ainv;
            h.ainv32 = fresh.ainv32;
            h.fflux = fresh.fflux;
            h.fflux32 = fresh.fflux32;
            h.q32 = fresh.q32;
            h.mass32 = fresh.mass32;
            changed = true;
        }
    }
    if (all != b->cached) {
        b->cached = all;
        if (b->sweep_graph) cudaGraphExecDestroy(b->sweep_graph);
        if (b->iter_graph) cudaGraphExecDestroy(b->iter_graph);
        b->sweep_graph = b->iter_graph = nullptr;
        ++b->graph_gen;
    }
    // the kernels read the table from device memory, so recorded graphs stay valid
    if (!changed) return cudaSuccess;
    return cudaMemcpyAsync(b->d_args, b->h_args.data(), b->count * sizeof(SweepArgs), cudaMemcpyHostToDevice, s);
}

cudaError_t launch_sweep(sn_mesh* m, const double* phi_in, int precision, double q_scale, cudaStream_t s) {
    cudaError_t cerr = prepare_operator_cache(m, precision, s);
    if (cerr != cudaSuccess) return cerr;
    SweepArgs a = make_args(m);
    a.phi = phi_in;
    if (q_scale != 0.0 && q_scale != 1.0) return cudaErrorInvalidValue;  // the source is on or off
    if (q_scale == 0.0) linear_part(a);
    a.psi = precision == SN_FP32 ? m->d_psi32 : m->d_psi;
    const bool cached = precision == SN_FP64 ? a.ainv != nullptr : (precision == SN_FP32 && a.ainv32 != nullptr);
    if (m->schedule == SCHED_BARRIER && cached) {  // uncached solves fall back to the level schedule
        if (precision == SN_FP64) SN_DISPATCH(m->dim, m->p, (cerr = launch_barrier_sweep<D_, P_, 0>(m, a, s)));
        else SN_DISPATCH(m->dim, m->p, (cerr = launch_barrier_sweep<D_, P_, 1>(m, a, s)));
        return cerr;
    }
    if (m->schedule == SCHED_TILES && cached) {  // uncached solves fall back to the level schedule
        if (m->tiles.edge != m->tile_edge && (cerr = build_tiles(m, m->tile_edge, s)) != cudaSuccess) return cerr;
        if (precision == SN_FP64) SN_DISPATCH(m->dim, m->p, (cerr = launch_tiles<D_, P_, 0>(m, a, s)));
        else SN_DISPATCH(m->dim, m->p, (cerr = launch_tiles<D_, P_, 1>(m, a, s)));
        return cerr;
    }
    if (dataflow_like(m->schedule)) {
        if (precision == SN_FP64) SN_DISPATCH(m->dim, m->p, (launch_dataflow<D_, P_, 0>(m, a, s)));
        else if (precision == SN_FP32) SN_DISPATCH(m->dim, m->p, (launch_dataflow<D_, P_, 1>(m, a, s)));
        else SN_DISPATCH(m->dim, m->p, (launch_dataflow<D_, P_, 2>(m, a, s)));
        return cudaGetLastError();
    }
    const size_t M = (size_t)m->ne * m->n;
    cudaError_t err = phi_in ? cudaMemcpyAsync(m->d_src, phi_in, M * sizeof(double), cudaMemcpyDeviceToDevice, s)
                             : cudaMemsetAsync(m->d_src, 0, M * sizeof(double), s);
    if (err != cudaSuccess) return err;
    return launch_levels_graph(m, q_scale == 0.0 ? precision + 4 : precision, s);
}

// Forward sweep of the directions d0 <= d < d1 only: the level work list of that range (built once
// per range and kept) launched as one chain of level kernels on the stream.  The element solves
// are those of the full sweep, so psi_d of these directions is bitwise the full sweep's.
cudaError_t launch_sweep_range(sn_mesh* m, const double* phi_in, int precision, int d0, int d1, cudaStream_t s,
                               double q_scale) {
    cudaError_t err = prepare_operator_cache(m, precision, s);
    if (err != cudaSuccess) return err;
    if (!m->range_items || m->range_d0 != d0 || m->range_d1 != d1) {
        if ((err = cudaStreamSynchronize(s)) != cudaSuccess) return err;  // a previous list may be in use
        if (m->range_items) cudaFree(m->range_items);
        m->range_items = nullptr;
        std::vector<int2> items;
        m->range_ptr = append_level_list(m, d0, d1, items);
        if ((err = cudaMalloc(&m->range_items, std::max<size_t>(1, items.size()) * sizeof(int2))) != cudaSuccess) {
            m->range_items = nullptr;
            return err;
        }
        if ((err = cudaMemcpy(m->range_items, items.data(), items.size() * sizeof(int2), cudaMemcpyHostToDevice)) !=
            cudaSuccess)
            return err;
        m->range_d0 = d0;
        m->range_d1 = d1;
    }
    SweepArgs a = make_args(m);
    a.phi = phi_in;
    if (q_scale != 0.0 && q_scale != 1.0) return cudaErrorInvalidValue;  // the source is on or off
    if (q_scale == 0.0) linear_part(a);
    a.psi = precision == SN_FP32 ? m->d_psi32 : m->d_psi;
    a.items = m->range_items;
    long long launches = 0;
    for (size_t l = 0; l + 1 < m->range_ptr.size(); ++l) launches += m->range_ptr[l + 1] > m->range_ptr[l];
    g_launches.fetch_add(launches, std::memory_order_relaxed);
    return enqueue_chain(m, precision, a, m->range_ptr, s);
}

cudaError_t launch_adjoint_sweep(sn_mesh* m, const double* mu, cudaStream_t s) {
    cudaError_t cerr = prepare_operator_cache(m, SN_FP64, s);
    if (cerr != cudaSuccess) return cerr;
    SweepArgs a = make_args(m);
    a.psi = m->d_lambda;
    if (dataflow_like(m->schedule)) {
        SN_DISPATCH(m->dim, m->p, (launch_dataflow<D_, P_, 0, true>(m, a, s, mu)));
        return cudaGetLastError();
    }
    const size_t M = (size_t)m->ne * m->n;
    cudaError_t err = cudaMemcpyAsync(m->d_src, mu, M * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (err != cudaSuccess) return err;
    return launch_levels_graph(m, 3, s);
}

// ---------------------------------------------------------------- batched sweeps
// Many meshes (instances) are swept together.  The batch's work list holds every instance's
// (direction, element) items sorted by (level, element family, instance); each (level, family)
// segment is padded to whole 32-item chunks, so a warp always runs one element template.
template <int DIM, int P, int MODE>
__global__ void __launch_bounds__(128) batch_level_kernel(const SweepArgs* args, const BatchItem* items,
                                                         long long begin, long long end, const int* active) {
    const long long t = begin + (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= end) return;
    const BatchItem it = items[t];
    if (it.inst < 0 || !active[it.inst]) return;
    solve_item<DIM, P, MODE>(args[it.inst], it.dir, it.elem);
}

template <int DIM, int P, int MODE>
__device__ __forceinline__ bool batch_chunk_item(const SweepArgs* args, const BatchItem& it, const int* active,
                                                 int* done, const long long* done_off, int epoch,
                                                 unsigned long long deadline, bool run) {
    // wait phase (run = false) or solve phase (run = true) of one lane's item
    if (it.inst < 0 || !active[it.inst]) return true;
    const SweepArgs& a = args[it.inst];
    int* dn = done + done_off[it.inst];
    if (run) {
        solve_item<DIM, P, MODE>(a, it.dir, it.elem);
        st_release(dn + (size_t)it.dir * a.ne + it.elem, epoch);
        return true;
    }
    const double Ox = a.dirs[3 * it.dir], Oy = a.dirs[3 * it.dir + 1], Oz = a.dirs[3 * it.dir + 2];
#pragma unroll
    for (int fc = 0; fc < 2 * DIM; ++fc) {
        if (face_flux_only<DIM, P>(a, it.elem, fc, Ox, Oy, Oz) < 0.0) {
            const int u = neighbor<DIM, P>(a, it.elem, fc);
            if (u < 0) continue;
            const int* flag = dn + (size_t)it.dir * a.ne + u;
            int polls = 0;
            while (ld_acquire(flag) != epoch) {
                if (++polls > 64) {
                    if (globaltimer() > deadline) return false;
                    __nanosleep(64);
                }
            }
        }
    }
    return true;
}

template <int DIM, int P, int MODE>
__device__ __forceinline__ bool batch_chunk(const SweepArgs* args, const BatchItem& it, const int* active, int* done,
                                            const long long* done_off, int epoch, unsigned long long deadline) {
    const bool ok = batch_chunk_item<DIM, P, MODE>(args, it, active, done, done_off, epoch, deadline, false);
    if (!__all_sync(0xffffffffu, ok)) return false;
    batch_chunk_item<DIM, P, MODE>(args, it, active, done, done_off, epoch, deadline, true);
    return true;
}

// Cached batched sweeps, one lane per node (the arithmetic of node_item, so a batched sweep
// equals the single-mesh sweeps bit for bit).  Level schedule: a warp takes 32 / N consecutive
// items of a (level, family) segment.
template <int DIM, int P, int MODE>
__global__ void __launch_bounds__(128) batch_node_level_kernel(const SweepArgs* args, const BatchItem* items,
                                                              long long begin, long long end, const int* active) {
    constexpr int N = Shape<DIM, P>::N, IPW = 32 / N;
    const int lane = threadIdx.x & 31;
    const int slot = lane / N, r = lane - slot * N;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long t = begin + warp * IPW + slot;
    BatchItem it{-1, 0, 0, 0};
    if (slot < IPW && t < end) it = items[t];
    const bool valid = it.inst >= 0 && active[it.inst];
    node_item<DIM, P, MODE, false, true>(args[valid ? it.inst : 0], nullptr, valid ? it.dir : 0, valid ? it.elem : 0,
                                         r, slot < IPW ? slot * N : 0, valid);
}

// Dataflow schedule: a warp claims a 32-item chunk (one family, one level) and runs it in rounds
// of 32 / N items (one claim per chunk keeps the shared counter's traffic low for large batches).
template <int DIM, int P, int MODE>
__device__ __forceinline__ bool batch_node_chunk(const SweepArgs* args, const BatchItem* items, long long chunk,
                                                 const int* active, int* done, const long long* done_off, int epoch,
                                                 unsigned long long deadline) {
    constexpr int N = Shape<DIM, P>::N, IPW = 32 / N, ROUNDS = (32 + IPW - 1) / IPW;
    const int lane = threadIdx.x & 31;
    const int slot = lane / N, r = lane - slot * N;
    const int src0 = slot < IPW ? slot * N : 0;
#pragma unroll 1
    for (int round = 0; round < ROUNDS; ++round) {
        const int k = round * IPW + slot;
        BatchItem it{-1, 0, 0, 0};
        if (slot < IPW && k < 32) it = items[(chunk << 5) + k];
        const bool valid = it.inst >= 0 && active[it.inst];
        const int inst = valid ? it.inst : 0, d = valid ? it.dir : 0, e = valid ? it.elem : 0;
        const SweepArgs& a = args[inst];
        int* dn = done + done_off[inst];
        const bool ok = valid ? wait_neighbours<DIM, P, false>(a, dn, epoch, d, e, deadline) : true;
        if (!__all_sync(0xffffffffu, ok)) return false;
        node_item<DIM, P, MODE, false>(a, nullptr, d, e, r, src0, valid);
        __syncwarp();
        if (valid && r == 0) {
            __threadfence();
            st_release(dn + (size_t)d * a.ne + e, epoch);
        }
    }
    return true;
}

template <int MODE>
__global__ void __launch_bounds__(128) batch_node_dataflow_kernel(const SweepArgs* args, const BatchItem* items,
                                                                 const int* chunk_fam, long long n_items, int* done,
                                                                 const long long* done_off, const int* epoch_ptr,
                                                                 unsigned long long* ctrl, const int* active,
                                                                 unsigned long long timeout_ns) {
    const int lane = threadIdx.x & 31;
    const long long n_chunks = n_items >> 5;
    const int epoch = *epoch_ptr;
    const unsigned long long deadline = globaltimer() + timeout_ns;
    int* error = reinterpret_cast<int*>(ctrl + 1);
    while (true) {
        unsigned long long c = 0;
        int failed = 0;
        if (lane == 0) {
            c = atomicAdd(ctrl, 1ull);
            failed = *(volatile int*)error;
        }
        c = __shfl_sync(0xffffffffu, c, 0);
        failed = __shfl_sync(0xffffffffu, failed, 0);
        if ((long long)c >= n_chunks || failed) break;
        bool ok;
        switch (chunk_fam[c]) {  // uniform across the warp
            case FAM_2D_P1: ok = batch_node_chunk<2, 1, MODE>(args, items, c, active, done, done_off, epoch, deadline); break;
            case FAM_2D_P2: ok = batch_node_chunk<2, 2, MODE>(args, items, c, active, done, done_off, epoch, deadline); break;
            case FAM_2D_P3: ok = batch_node_chunk<2, 3, MODE>(args, items, c, active, done, done_off, epoch, deadline); break;
            default: ok = batch_node_chunk<3, 1, MODE>(args, items, c, active, done, done_off, epoch, deadline); break;
        }
        if (!ok) {
            if (lane == 0) atomicExch(error, 1);
            break;
        }
    }
}

// Data-polled chunk of the batched cached sweep (as node_datapoll_kernel for one mesh): stage, poll
// the upwind angular fluxes (reset to the unset pattern before the launch), solve, store.
template <int DIM, int P, int MODE>
__device__ __forceinline__ bool batch_node_chunk_polled(const SweepArgs* args, const BatchItem* items, long long chunk,
                                                        const int* active, unsigned long long deadline,
                                                        const int* error) {
    using R = typename std::conditional<MODE == 1, float, double>::type;
    constexpr int N = Shape<DIM, P>::N, IPW = 32 / N, ROUNDS = (32 + IPW - 1) / IPW;
    const int lane = threadIdx.x & 31;
    const int slot = lane / N, r = lane - slot * N;
    const int src0 = slot < IPW ? slot * N : 0;
#pragma unroll 1
    for (int round = 0; round < ROUNDS; ++round) {
        const int k = round * IPW + slot;
        BatchItem it{-1, 0, 0, 0};
        if (slot < IPW && k < 32) it = items[(chunk << 5) + k];
        const bool valid = it.inst >= 0 && active[it.inst];
        const int inst = valid ? it.inst : 0, d = valid ? it.dir : 0, e = valid ? it.elem : 0;
        const SweepArgs& a = args[inst];
        NodeStage<DIM, P, R> st;
        if (valid) node_stage<DIM, P, MODE, false>(a, nullptr, d, e, r, st);
        bool ok = true;
        const R rhs = valid ? node_faces_polled<DIM, P, R, false>(a, st.F, d, e, r, st.rhs, deadline, error, &ok) : R(0);
        if (!__all_sync(0xffffffffu, ok)) return false;
        R x = R(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
            const R rj = __shfl_sync(0xffffffffu, rhs, src0 + j);
            if (valid) x += st.inv[j] * rj;
        }
        if (valid) st_relaxed(static_cast<R*>(a.psi) + ((size_t)d * a.ne + e) * N + r, x);
    }
    return true;
}

// Batched data-polled sweep: warps claim 32-item chunks (static_warps > 0: take chunks w, w + W, ...).
template <int MODE>
__global__ void __launch_bounds__(128) batch_node_datapoll_kernel(const SweepArgs* args, const BatchItem* items,
                                                                 const int* chunk_fam, long long n_items,
                                                                 unsigned long long* ctrl, const int* active,
                                                                 unsigned long long timeout_ns, long long static_warps) {
    const int lane = threadIdx.x & 31;
    const long long n_chunks = n_items >> 5;
    const unsigned long long deadline = globaltimer() + timeout_ns;
    int* error = reinterpret_cast<int*>(ctrl + 1);
    unsigned long long mine = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    while (true) {
        unsigned long long c = 0;
        if (static_warps > 0) {
            c = mine;
            mine += (unsigned long long)static_warps;
        } else {
            if (lane == 0) c = atomicAdd(ctrl, 1ull);
            c = __shfl_sync(0xffffffffu, c, 0);
        }
        if ((long long)c >= n_chunks) break;
        bool ok;
        switch (chunk_fam[c]) {  // uniform across the warp
            case FAM_2D_P1: ok = batch_node_chunk_polled<2, 1, MODE>(args, items, c, active, deadline, error); break;
            case FAM_2D_P2: ok = batch_node_chunk_polled<2, 2, MODE>(args, items, c, active, deadline, error); break;
            case FAM_2D_P3: ok = batch_node_chunk_polled<2, 3, MODE>(args, items, c, active, deadline, error); break;
            default: ok = batch_node_chunk_polled<3, 1, MODE>(args, items, c, active, deadline, error); break;
        }
        if (!ok) {
            if (lane == 0) atomicExch(error, 1);
            break;
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(128) batch_dataflow_kernel(const SweepArgs* args, const BatchItem* items,
                                                            const int* chunk_fam, long long n_items, int* done,
                                                            const long long* done_off, const int* epoch_ptr,
                                                            unsigned long long* ctrl, const int* active,
                                                            unsigned long long timeout_ns) {
    const int lane = threadIdx.x & 31;
    const long long n_chunks = n_items >> 5;
    const int epoch = *epoch_ptr;  // advanced on the device before the launch, so graphs can replay it
    const unsigned long long deadline = globaltimer() + timeout_ns;
    int* error = reinterpret_cast<int*>(ctrl + 1);
    while (true) {
        unsigned long long c = 0;
        int failed = 0;
        if (lane == 0) {
            c = atomicAdd(ctrl, 1ull);
            failed = *(volatile int*)error;
        }
        c = __shfl_sync(0xffffffffu, c, 0);
        failed = __shfl_sync(0xffffffffu, failed, 0);
        if ((long long)c >= n_chunks || failed) break;
        const BatchItem it = items[(c << 5) + lane];
        bool ok;
        switch (chunk_fam[c]) {  // uniform across the warp
            case FAM_2D_P1: ok = batch_chunk<2, 1, MODE>(args, it, active, done, done_off, epoch, deadline); break;
            case FAM_2D_P2: ok = batch_chunk<2, 2, MODE>(args, it, active, done, done_off, epoch, deadline); break;
            case FAM_2D_P3: ok = batch_chunk<2, 3, MODE>(args, it, active, done, done_off, epoch, deadline); break;
            default: ok = batch_chunk<3, 1, MODE>(args, it, active, done, done_off, epoch, deadline); break;
        }
        if (!ok) {
            if (lane == 0) atomicExch(error, 1);
            break;
        }
    }
}

cudaError_t batch_build_worklist(sn_batch* b, cudaStream_t s) {
    cudaError_t err;
    const int n = b->count;
    std::vector<std::vector<int2>> items(n);
    int maxL = 0;
    long long done_total = 0;
    std::vector<long long> done_off(n);
    for (int i = 0; i < n; ++i) {
        sn_mesh* m = b->meshes[i];
        const long long total = (long long)m->nd * m->ne;
        items[i].resize(total);
        if ((err = cudaMemcpy(items[i].data(), m->levels.items, total * sizeof(int2), cudaMemcpyDeviceToHost)) != cudaSuccess)
            return err;
        maxL = std::max(maxL, m->levels.n_levels);
        done_off[i] = done_total;
        done_total += total;
    }
    std::vector<BatchItem> list;
    std::vector<int> chunk_fam;
    b->seg_begin.clear();
    b->seg_end.clear();
    b->seg_fam.clear();
    b->seg_level.clear();
    for (int L = 0; L < maxL; ++L)
        for (int fam = 0; fam < FAM_COUNT; ++fam) {
            const long long begin = (long long)list.size();
            for (int i = 0; i < n; ++i) {
                sn_mesh* m = b->meshes[i];
                if (family_of(m->dim, m->p) != fam || L >= m->levels.n_levels) continue;
                for (long long t = m->levels.level_ptr[L]; t < m->levels.level_ptr[L + 1]; ++t)
                    list.push_back({i, items[i][t].x, items[i][t].y, fam});
            }
            if ((long long)list.size() == begin) continue;
            while (list.size() % 32) list.push_back({-1, 0, 0, fam});
            b->seg_begin.push_back(begin);
            b->seg_end.push_back((long long)list.size());
            b->seg_fam.push_back(fam);
            b->seg_level.push_back(L);
            for (long long c = begin / 32; c < (long long)list.size() / 32; ++c) chunk_fam.push_back(fam);
        }
    b->n_items = (long long)list.size();
    if ((err = cudaMalloc(&b->d_items, list.size() * sizeof(BatchItem))) != cudaSuccess) return err;
    if ((err = cudaMemcpy(b->d_items, list.data(), list.size() * sizeof(BatchItem), cudaMemcpyHostToDevice)) != cudaSuccess)
        return err;
    if ((err = cudaMalloc(&b->d_chunk_fam, chunk_fam.size() * sizeof(int))) != cudaSuccess) return err;
    if ((err = cudaMemcpy(b->d_chunk_fam, chunk_fam.data(), chunk_fam.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess)
        return err;
    if ((err = cudaMalloc(&b->d_done, std::max<long long>(1, done_total) * sizeof(int))) != cudaSuccess) return err;
    if ((err = cudaMemset(b->d_done, 0, std::max<long long>(1, done_total) * sizeof(int))) != cudaSuccess) return err;
    if ((err = cudaMalloc(&b->d_done_off, n * sizeof(long long))) != cudaSuccess) return err;
    if ((err = cudaMemcpy(b->d_done_off, done_off.data(), n * sizeof(long long), cudaMemcpyHostToDevice)) != cudaSuccess)
        return err;
    if ((err = cudaMalloc(&b->d_ctrl, 3 * sizeof(unsigned long long))) != cudaSuccess) return err;
    if ((err = cudaMemset(b->d_ctrl, 0, 3 * sizeof(unsigned long long))) != cudaSuccess) return err;
    // per-instance arguments: sources and angular fluxes at fixed addresses
    b->h_args.resize(n);
    for (int i = 0; i < n; ++i) {
        b->h_args[i] = make_args(b->meshes[i]);
        b->h_args[i].phi = b->d_phi + b->dof_off[i];
        b->h_args[i].psi = b->meshes[i]->d_psi;
    }
    if ((err = cudaMalloc(&b->d_args, n * sizeof(SweepArgs))) != cudaSuccess) return err;
    return cudaMemcpyAsync(b->d_args, b->h_args.data(), n * sizeof(SweepArgs), cudaMemcpyHostToDevice, s);
}

// Points every instance's angular-flux storage at the precision's buffer (float32 for SN_FP32).
cudaError_t batch_set_precision(sn_batch* b, int precision, cudaStream_t s) {
    if (b->precision == precision) return cudaSuccess;
    for (int i = 0; i < b->count; ++i)
        b->h_args[i].psi = precision == SN_FP32 ? b->meshes[i]->d_psi32 : b->meshes[i]->d_psi;
    b->precision = precision;
    if (b->sweep_graph) {
        cudaGraphExecDestroy(b->sweep_graph);
        b->sweep_graph = nullptr;
    }
    if (b->iter_graph) {
        cudaGraphExecDestroy(b->iter_graph);
        b->iter_graph = nullptr;
    }
    ++b->graph_gen;
    return cudaMemcpyAsync(b->d_args, b->h_args.data(), b->count * sizeof(SweepArgs), cudaMemcpyHostToDevice, s);
}

cudaError_t batch_enqueue_sweep(sn_batch* b, int precision, cudaStream_t s, const SweepArgs* args, const int* mask) {
    cudaError_t err = batch_set_precision(b, precision, s);
    if (err != cudaSuccess) return err;
    if (!args) args = b->d_args;
    if (!mask) mask = b->d_active;
    const int bs = b->block;
    for (size_t k = 0; k < b->seg_begin.size(); ++k) {
        const long long lo = b->seg_begin[k], hi = b->seg_end[k];
        const unsigned g = grid_for(hi - lo, bs);
        const int fam = b->seg_fam[k];
#define SN_BATCH_LEVEL(MODE_)                                                                                   \
    do {                                                                                                      \
        if (fam == FAM_2D_P1) batch_level_kernel<2, 1, MODE_><<<g, bs, 0, s>>>(args, b->d_items, lo, hi, mask); \
        else if (fam == FAM_2D_P2) batch_level_kernel<2, 2, MODE_><<<g, bs, 0, s>>>(args, b->d_items, lo, hi, mask); \
        else if (fam == FAM_2D_P3) batch_level_kernel<2, 3, MODE_><<<g, bs, 0, s>>>(args, b->d_items, lo, hi, mask); \
        else batch_level_kernel<3, 1, MODE_><<<g, bs, 0, s>>>(args, b->d_items, lo, hi, mask);       \
    } while (0)
#define SN_BATCH_NODE(MODE_)                                                                                    \
    do {                                                                                                      \
        const unsigned gn = grid_for(((hi - lo + ipw - 1) / ipw) * 32, bs);                                   \
        const bool pdl = k > 0;                                                                               \
        cudaError_t lerr;                                                                                     \
        if (fam == FAM_2D_P1) lerr = launch_k(pdl, batch_node_level_kernel<2, 1, MODE_>, gn, bs, s, args, b->d_items, lo, hi, mask); \
        else if (fam == FAM_2D_P2) lerr = launch_k(pdl, batch_node_level_kernel<2, 2, MODE_>, gn, bs, s, args, b->d_items, lo, hi, mask); \
        else if (fam == FAM_2D_P3) lerr = launch_k(pdl, batch_node_level_kernel<2, 3, MODE_>, gn, bs, s, args, b->d_items, lo, hi, mask); \
        else lerr = launch_k(pdl, batch_node_level_kernel<3, 1, MODE_>, gn, bs, s, args, b->d_items, lo, hi, mask); \
        if (lerr != cudaSuccess) return lerr;                                                                 \
    } while (0)
        SN_COUNT_LAUNCH();
        const int ipw = 32 / family_nodes(fam);
        if (precision == SN_FP64 && b->cached) SN_BATCH_NODE(0);
        else if (precision == SN_FP32 && b->cached) SN_BATCH_NODE(1);
        else if (precision == SN_FP64) SN_BATCH_LEVEL(0);
        else if (precision == SN_FP32) SN_BATCH_LEVEL(1);
        else SN_BATCH_LEVEL(2);
#undef SN_BATCH_LEVEL
#undef SN_BATCH_NODE
    }
    return cudaGetLastError();
}

__global__ void bump_epoch_kernel(unsigned long long* ctrl) {
    int* e = reinterpret_cast<int*>(ctrl + 2);
    *e = (*e >= 0x7ffffff0) ? 1 : *e + 1;  // completion words are compared for equality only
    ctrl[0] = 0ull;                          // chunk counter of the coming launch
}

// Persistent dataflow sweep of all instances; capturable (the epoch is advanced on the device).
cudaError_t batch_launch_dataflow(sn_batch* b, int precision, cudaStream_t s, const SweepArgs* args, const int* mask) {
    cudaError_t err = batch_set_precision(b, precision, s);
    if (err != cudaSuccess) return err;
    if (!args) args = b->d_args;
    if (!mask) mask = b->d_active;
    SN_COUNT_LAUNCH();
    bump_epoch_kernel<<<1, 1, 0, s>>>(b->d_ctrl);
    int dev = 0, sms = 0, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool node = b->cached && precision != SN_FP32_REFINE;
    if (node && precision == SN_FP64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_node_datapoll_kernel<0>, b->block, 0);
    else if (node) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_node_datapoll_kernel<1>, b->block, 0);
    else if (precision == SN_FP64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_dataflow_kernel<0>, b->block, 0);
    else if (precision == SN_FP32) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_dataflow_kernel<1>, b->block, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_dataflow_kernel<2>, b->block, 0);
    if (b->max_blocks_per_sm > 0 && b->max_blocks_per_sm < per_sm) per_sm = b->max_blocks_per_sm;
    per_sm = std::max(per_sm, 1);
    long long blocks = std::min<long long>((long long)sms * per_sm, (b->n_items + b->block - 1) / b->block);
    blocks = std::max<long long>(blocks, 1);
    const unsigned long long timeout = 4000000000ull;
    const int* epoch = reinterpret_cast<const int*>(b->d_ctrl + 2);
    if (node) {
        // cached (node-per-lane) solves poll the upwind angular fluxes: every instance's starts unset
        for (int i = 0; i < b->count; ++i) {
            sn_mesh* m = b->meshes[i];
            const size_t bytes = (size_t)m->nd * m->ne * m->n * (precision == SN_FP32 ? sizeof(float) : sizeof(double));
            if ((err = cudaMemsetAsync(b->h_args[i].psi, 0xFF, bytes, s)) != cudaSuccess) return err;
        }
        const long long warps = b->schedule == SCHED_STATIC ? blocks * (b->block / 32) : 0;
        SN_COUNT_LAUNCH();
        if (precision == SN_FP64)
            batch_node_datapoll_kernel<0><<<(unsigned)blocks, b->block, 0, s>>>(args, b->d_items, b->d_chunk_fam,
                                                                               b->n_items, b->d_ctrl, mask,
                                                                               timeout, warps);
        else
            batch_node_datapoll_kernel<1><<<(unsigned)blocks, b->block, 0, s>>>(args, b->d_items, b->d_chunk_fam,
                                                                               b->n_items, b->d_ctrl, mask,
                                                                               timeout, warps);
        return cudaGetLastError();
    }
    SN_COUNT_LAUNCH();
    if (precision == SN_FP64)
        batch_dataflow_kernel<0><<<(unsigned)blocks, b->block, 0, s>>>(args, b->d_items, b->d_chunk_fam, b->n_items,
                                                                      b->d_done, b->d_done_off, epoch, b->d_ctrl,
                                                                      mask, timeout);
    else if (precision == SN_FP32)
        batch_dataflow_kernel<1><<<(unsigned)blocks, b->block, 0, s>>>(args, b->d_items, b->d_chunk_fam, b->n_items,
                                                                      b->d_done, b->d_done_off, epoch, b->d_ctrl,
                                                                      mask, timeout);
    else
        batch_dataflow_kernel<2><<<(unsigned)blocks, b->block, 0, s>>>(args, b->d_items, b->d_chunk_fam, b->n_items,
                                                                      b->d_done, b->d_done_off, epoch, b->d_ctrl,
                                                                      mask, timeout);
    return cudaGetLastError();
}

cudaError_t launch_phi_reduce(sn_mesh* m, int precision, const double* phi_in, double* phi_out, double* d_rr,
                              cudaStream_t s, int d0, int d1) {
    const size_t M = (size_t)m->ne * m->n;
    const unsigned g = (unsigned)((M + 255) / 256);
    if (d1 < 0) d1 = m->nd;
    SN_COUNT_LAUNCH();
    if (precision == SN_FP32)
        phi_reduce_kernel<float><<<g, 256, 0, s>>>(static_cast<const float*>(m->d_psi32), m->d_wts, d0, d1, M, phi_in,
                                                   phi_out, d_rr ? m->d_red : nullptr);
    else
        phi_reduce_kernel<double><<<g, 256, 0, s>>>(static_cast<const double*>(m->d_psi), m->d_wts, d0, d1, M, phi_in,
                                                    phi_out, d_rr ? m->d_red : nullptr);
    if (d_rr) { SN_COUNT_LAUNCH(); final_sum_kernel<<<1, 1024, 0, s>>>(m->d_red, (int)g, d_rr); }
    return cudaGetLastError();
}

cudaError_t launch_axpy_norm(sn_mesh* m, const double* a, const double* b, double* out, double* d_rr,
                             cudaStream_t s) {
    const size_t M = (size_t)m->ne * m->n;
    const unsigned g = (unsigned)((M + 255) / 256);
    SN_COUNT_LAUNCH();
    diff_norm_kernel<<<g, 256, 0, s>>>(a, b, out, M, m->d_red);
    SN_COUNT_LAUNCH();
    final_sum_kernel<<<1, 1024, 0, s>>>(m->d_red, (int)g, d_rr);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_reduce(sn_mesh* m, double* out, cudaStream_t s) {
    SweepArgs a = make_args(m);
    const size_t M = (size_t)m->ne * m->n;
    SN_COUNT_LAUNCH();
    SN_DISPATCH(m->dim, m->p, (adjoint_reduce_kernel<D_, P_><<<grid_for((long long)M, 256), 256, 0, s>>>(a, m->d_lambda, m->d_wts, out)));
    return cudaGetLastError();
}

cudaError_t launch_gradients(sn_mesh* m, const double* phi, double* gt, double* gs, double* gq, cudaStream_t s) {
    SweepArgs a = make_args(m);
    SN_COUNT_LAUNCH();
    SN_DISPATCH(m->dim, m->p,
                (gradient_kernel<D_, P_><<<grid_for(m->ne, 128), 128, 0, s>>>(a, static_cast<const double*>(m->d_psi),
                                                                               m->d_lambda, m->d_wts, phi, gt, gs, gq)));
    return cudaGetLastError();
}

__global__ void add_kernel(double* y, const double* x, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

cudaError_t launch_axpy_add(double* y, const double* x, size_t n, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    add_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, x, n);
    return cudaGetLastError();
}

__global__ void widen_kernel(double* y, const float* x, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (double)x[i];
}

cudaError_t launch_widen(double* y, const float* x, size_t n, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    widen_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(y, x, n);
    return cudaGetLastError();
}

cudaError_t take_sweep_error(sn_mesh* m, cudaStream_t s, bool* timed_out) {
    *timed_out = false;
    if (!m->levels.ctrl) return cudaSuccess;
    unsigned long long w = 0;
    cudaError_t err = cudaMemcpyAsync(&w, m->levels.ctrl + 1, sizeof(w), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return err;
    if (w) {
        *timed_out = true;
        err = cudaMemsetAsync(m->levels.ctrl + 1, 0, sizeof(w), s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    }
    return err;
}

// The device copy of the dataflow epoch (ctrl[2]) follows the host's around a recorded iteration:
// set before the graph runs (after clearing the completion words if the recorded sweeps could run
// past the wrap point), read back after it.
cudaError_t device_epoch_in(sn_mesh* m, long long max_sweeps, cudaStream_t s) {
    LevelSets& L = m->levels;
    if (!L.ctrl) return cudaSuccess;
    cudaError_t err;
    if ((long long)L.epoch + max_sweeps >= 0x7fffffffll) {
        if ((err = cudaMemsetAsync(L.done, 0, (size_t)m->nd * m->ne * sizeof(int), s)) != cudaSuccess) return err;
        L.epoch = 0;
    }
    const unsigned long long e = (unsigned long long)L.epoch;
    if ((err = cudaMemcpyAsync(L.ctrl + 2, &e, sizeof(e), cudaMemcpyHostToDevice, s)) != cudaSuccess) return err;
    return cudaStreamSynchronize(s);  // e lives on this stack frame
}

cudaError_t device_epoch_out(sn_mesh* m, cudaStream_t s) {
    LevelSets& L = m->levels;
    if (!L.ctrl) return cudaSuccess;
    unsigned long long e = 0;
    cudaError_t err = cudaMemcpyAsync(&e, L.ctrl + 2, sizeof(e), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err == cudaSuccess) L.epoch = (int)e;
    return err;
}

cudaError_t launch_copy(double* dst, const double* src, size_t n, cudaStream_t s) {
    return cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}

}  // namespace sn
