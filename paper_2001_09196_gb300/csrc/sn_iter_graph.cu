// Device side of the recorded outer iterations: the convergence tests, the Arnoldi bookkeeping
// and the Givens rotations of flexible GMRES run in single-thread kernels that set the conditional
// handles of the enclosing CUDA graph, so a whole solve is one graph launch and one synchronisation.
//
// Source iteration (Eq. DSA_fp with Algorithm 2 or 1) and flexible GMRES(k) on S x = b (Eq. schur)
// are the host loops of sn_api.cpp step for step; the same floating-point operations run in the
// same order, only the scalars live on the device.  State layout (IterGraphState in sn_internal.h):
//   gd: doubles  [0] r0, [1] rel, [2] beta, [3] hnext, then H ((k+1) x k, column c at c (k+1)),
//       cs (k), sn (k), g (k+1), y (k)
//   gi: ints     [0] iterations, [1] j (Arnoldi step), [2] jj (steps of the last cycle),
//                [3] converged, [4] continue the cycle, [5] restart cycles, [6] checkpoints written
#include <cuda_runtime.h>

#include <cmath>

#include "sn_internal.h"

namespace sn {

namespace {

constexpr int kThreads = 256;
enum { D_R0 = 0, D_REL = 1, D_BETA = 2, D_HNEXT = 3, D_ARR = 4 };
enum { I_IT = 0, I_J = 1, I_JJ = 2, I_CONV = 3, I_CONT = 4, I_CYCLES = 5, I_NCK = 6 };

__device__ __forceinline__ double* gm_H(double* gd) { return gd + D_ARR; }
__device__ __forceinline__ double* gm_cs(double* gd, int k) { return gd + D_ARR + (k + 1) * k; }
__device__ __forceinline__ double* gm_sn(double* gd, int k) { return gm_cs(gd, k) + k; }
__device__ __forceinline__ double* gm_g(double* gd, int k) { return gm_sn(gd, k) + k; }
__device__ __forceinline__ double* gm_y(double* gd, int k) { return gm_g(gd, k) + k + 1; }

__global__ void ig_init_kernel(double* gd, int* gi) {
    gd[D_R0] = 0.0;
    gd[D_REL] = INFINITY;
    for (int i = 0; i < 8; ++i) gi[i] = 0;
}

// ---------------------------------------------------------------- source iteration
// After the transport update of iteration it: rel = ||r|| / ||r^0||, history.
__global__ void si_residual_kernel(const double* rr, double* gd, int* gi, double* hist, int hist_len) {
    const double rn = sqrt(rr[0]);
    const int it = gi[I_IT];
    if (it == 0) gd[D_R0] = rn > 0.0 ? rn : 1.0;
    const double rel = rn / gd[D_R0];
    gd[D_REL] = rel;
    if (hist && it < hist_len) hist[it] = rel;
}

// End of iteration it: count it, stop after the iteration whose residual met tol or at max_iters.
__global__ void si_end_kernel(double* gd, int* gi, double tol, int max_iters, cudaGraphConditionalHandle h) {
    const int it = gi[I_IT] + 1;
    gi[I_IT] = it;
    const bool conv = gd[D_REL] <= tol;
    gi[I_CONV] = conv ? 1 : 0;
    cudaGraphSetConditional(h, (!conv && it < max_iters) ? 1u : 0u);
}

// checkpoints[nck] = phi after every `every`-th iteration (while room is left)
__global__ void si_checkpoint_kernel(const double* phi, double* ckpt, long long M, const int* gi, int every, int max_ck) {
    const int it = gi[I_IT], nck = gi[I_NCK];
    if (it % every != 0 || nck >= max_ck) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < M) ckpt[(size_t)nck * M + t] = phi[t];
}

__global__ void si_checkpoint_count_kernel(int* gi, int every, int max_ck) {
    if (gi[I_IT] % every == 0 && gi[I_NCK] < max_ck) gi[I_NCK] += 1;
}

// ---------------------------------------------------------------- flexible GMRES
// Start of a restart cycle from the true residual norm^2 rr: declares convergence on the true
// residual only, stops at max_iters, else opens the Arnoldi loop with g = beta e_1.
__global__ void gm_cycle_start_kernel(const double* rr, double* gd, int* gi, int k, double tol, int max_iters,
                                      double* hist, int hist_len, cudaGraphConditionalHandle outer,
                                      cudaGraphConditionalHandle inner) {
    const double beta = sqrt(rr[0]);
    if (gd[D_R0] == 0.0) gd[D_R0] = beta > 0.0 ? beta : 1.0;
    const double rel = beta / gd[D_R0];
    gd[D_REL] = rel;
    gd[D_BETA] = beta;
    const int it = gi[I_IT];
    if (hist && hist_len > 0 && it == 0) hist[0] = rel;
    bool stop = false;
    if (rel <= tol || beta == 0.0) {
        gi[I_CONV] = 1;
        stop = true;
    } else if (it >= max_iters) {
        stop = true;
    }
    double* g = gm_g(gd, k);
    for (int i = 0; i <= k; ++i) g[i] = 0.0;
    g[0] = beta;
    gi[I_J] = 0;
    gi[I_JJ] = 0;
    gi[I_CONT] = stop ? 0 : 1;
    if (!stop) gi[I_CYCLES] += 1;
    cudaGraphSetConditional(outer, stop ? 0u : 1u);
    cudaGraphSetConditional(inner, stop ? 0u : 1u);
}

// One Arnoldi step's scalars: column j of H from the two Gram-Schmidt passes, the previous
// rotations applied, a new rotation, the residual estimate; decides whether the cycle continues.
__global__ void gm_arnoldi_kernel(const double* hd, double* gd, int* gi, int k, double tol, int max_iters,
                                  double drop, double* hist, int hist_len, cudaGraphConditionalHandle inner) {
    const int j = gi[I_J];
    double* H = gm_H(gd);
    double* cs = gm_cs(gd, k);
    double* sn_ = gm_sn(gd, k);
    double* g = gm_g(gd, k);
    double* h = H + (size_t)j * (k + 1);
    for (int i = 0; i <= j; ++i) h[i] = hd[i] + hd[k + 1 + i];
    h[j + 1] = sqrt(fmax(hd[2 * (k + 1)], 0.0));
    const double hnext = h[j + 1];
    for (int i = 0; i < j; ++i) {
        const double t = cs[i] * h[i] + sn_[i] * h[i + 1];
        h[i + 1] = -sn_[i] * h[i] + cs[i] * h[i + 1];
        h[i] = t;
    }
    const double rho = hypot(h[j], h[j + 1]);
    cs[j] = rho > 0 ? h[j] / rho : 1.0;
    sn_[j] = rho > 0 ? h[j + 1] / rho : 0.0;
    h[j] = rho;
    h[j + 1] = 0.0;
    g[j + 1] = -sn_[j] * g[j];
    g[j] = cs[j] * g[j];
    const int it = gi[I_IT] + 1;
    gi[I_IT] = it;
    gi[I_JJ] = j + 1;
    const double rel = fabs(g[j + 1]) / gd[D_R0];
    gd[D_REL] = rel;
    if (hist && it < hist_len) hist[it] = rel;
    bool cont = !(rel <= tol || hnext <= 1e-300);
    if (cont && drop > 0.0 && fabs(g[j + 1]) <= drop * gd[D_BETA]) cont = false;
    if (j + 1 >= k || it >= max_iters) cont = false;
    gd[D_HNEXT] = hnext;
    gi[I_J] = j + 1;
    gi[I_CONT] = cont ? 1 : 0;
    cudaGraphSetConditional(inner, cont ? 1u : 0u);
}

// y solves the leading jj x jj triangle of H against g (jj = steps of this cycle)
__global__ void gm_solve_kernel(double* gd, const int* gi, int k) {
    const int jj = gi[I_JJ];
    const double* H = gm_H(gd);
    const double* g = gm_g(gd, k);
    double* y = gm_y(gd, k);
    for (int i = jj - 1; i >= 0; --i) {
        double t = g[i];
        for (int c = i + 1; c < jj; ++c) t -= H[(size_t)c * (k + 1) + i] * y[c];
        y[i] = t / H[(size_t)i * (k + 1) + i];
    }
}

// out = V_j (j on the device, plus `ofs`)
__global__ void gm_get_col_kernel(const double* V, const int* gi, int ofs, long long M, double* out) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    out[t] = V[(size_t)(gi[I_J] + ofs) * M + t];
}

__global__ void gm_set_col_kernel(double* V, const int* gi, long long M, const double* in) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    V[(size_t)gi[I_J] * M + t] = in[t];
}

// V_{j+1} = w / hnext when the cycle continues (gi[I_J] already holds j + 1)
__global__ void gm_next_basis_kernel(const double* w, const double* gd, const int* gi, long long M, double* V) {
    if (!gi[I_CONT]) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    V[(size_t)gi[I_J] * M + t] = w[t] / gd[D_HNEXT];
}

inline unsigned blocks_for(long long n) { return (unsigned)((n + kThreads - 1) / kThreads); }

}  // namespace

size_t iter_graph_doubles(int k) { return D_ARR + (size_t)(k + 1) * k + 2 * k + (k + 1) + k; }
int iter_graph_y_offset(int k) { return D_ARR + (k + 1) * k + 2 * k + (k + 1); }

cudaError_t ig_init(double* gd, int* gi, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    ig_init_kernel<<<1, 1, 0, s>>>(gd, gi);
    return cudaGetLastError();
}

cudaError_t ig_si_residual(const double* rr, double* gd, int* gi, double* hist, int hist_len, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    si_residual_kernel<<<1, 1, 0, s>>>(rr, gd, gi, hist, hist_len);
    return cudaGetLastError();
}

cudaError_t ig_si_end(double* gd, int* gi, double tol, int max_iters, cudaGraphConditionalHandle h, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    si_end_kernel<<<1, 1, 0, s>>>(gd, gi, tol, max_iters, h);
    return cudaGetLastError();
}

cudaError_t ig_si_checkpoint(const double* phi, double* ckpt, long long M, int* gi, int every, int max_ck,
                             cudaStream_t s) {
    SN_COUNT_LAUNCH();
    si_checkpoint_kernel<<<blocks_for(M), kThreads, 0, s>>>(phi, ckpt, M, gi, every, max_ck);
    SN_COUNT_LAUNCH();
    si_checkpoint_count_kernel<<<1, 1, 0, s>>>(gi, every, max_ck);
    return cudaGetLastError();
}

cudaError_t ig_gm_cycle_start(const double* rr, double* gd, int* gi, int k, double tol, int max_iters, double* hist,
                              int hist_len, cudaGraphConditionalHandle outer, cudaGraphConditionalHandle inner,
                              cudaStream_t s) {
    SN_COUNT_LAUNCH();
    gm_cycle_start_kernel<<<1, 1, 0, s>>>(rr, gd, gi, k, tol, max_iters, hist, hist_len, outer, inner);
    return cudaGetLastError();
}

cudaError_t ig_gm_arnoldi(const double* hd, double* gd, int* gi, int k, double tol, int max_iters, double drop,
                          double* hist, int hist_len, cudaGraphConditionalHandle inner, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    gm_arnoldi_kernel<<<1, 1, 0, s>>>(hd, gd, gi, k, tol, max_iters, drop, hist, hist_len, inner);
    return cudaGetLastError();
}

cudaError_t ig_gm_solve(double* gd, const int* gi, int k, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    gm_solve_kernel<<<1, 1, 0, s>>>(gd, gi, k);
    return cudaGetLastError();
}

cudaError_t ig_get_col(const double* V, const int* gi, int ofs, long long M, double* out, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    gm_get_col_kernel<<<blocks_for(M), kThreads, 0, s>>>(V, gi, ofs, M, out);
    return cudaGetLastError();
}

cudaError_t ig_set_col(double* V, const int* gi, long long M, const double* in, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    gm_set_col_kernel<<<blocks_for(M), kThreads, 0, s>>>(V, gi, M, in);
    return cudaGetLastError();
}

cudaError_t ig_next_basis(const double* w, const double* gd, const int* gi, long long M, double* V, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    gm_next_basis_kernel<<<blocks_for(M), kThreads, 0, s>>>(w, gd, gi, M, V);
    return cudaGetLastError();
}

}  // namespace sn
