// Device vector kernels of the flexible GMRES outer iteration (float64, fixed reduction order).
//
// The Krylov basis V (k+1 vectors of length n, contiguous) is orthogonalised by classical
// Gram-Schmidt applied twice; each pass is one batched inner product h = V^T w and one batched
// update w -= V h, so an outer iteration costs a handful of launches and one host read.
#include <cuda_runtime.h>

#include "sn_internal.h"

namespace sn {

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBasis = 64;

// partial[i * nblocks + b] = sum over block b's slice of V_i . w, for i < k
// (kdev non-null: k = *kdev + kofs, read on the device, for the recorded fGMRES iteration)
__global__ void multidot_partial_kernel(const double* V, int k, long long n, const double* w, double* partial,
                                        int nblocks, const int* kdev, int kofs) {
    __shared__ double sh[kThreads];
    if (kdev) k = *kdev + kofs;
    const long long chunk = (n + gridDim.x - 1) / gridDim.x;
    const long long lo = blockIdx.x * chunk, hi = lo + chunk < n ? lo + chunk : n;
    for (int i = 0; i < k; ++i) {
        const double* v = V + (size_t)i * n;
        double s = 0.0;
        for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) s += v[t] * w[t];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(size_t)i * nblocks + blockIdx.x] = sh[0];
        __syncthreads();
    }
}

__global__ void multidot_final_kernel(const double* partial, int nblocks, double* out, const int* kdev, int kofs) {
    __shared__ double sh[kThreads];
    const int i = blockIdx.x;
    if (kdev && i >= *kdev + kofs) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[(size_t)i * nblocks + b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = sh[0];
}

// w += sign * sum_i c[i] V_i  (c on the device)
__global__ void multiaxpy_kernel(const double* V, int k, long long n, const double* c, double sign, double* w,
                                 const int* kdev, int kofs) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (kdev) k = *kdev + kofs;
    double s = 0.0;
    for (int i = 0; i < k; ++i) s += c[i] * V[(size_t)i * n + t];
    w[t] += sign * s;
}

// y = alpha x (alpha = 1 / s[0] read on the device, s[0] = ||x||)
__global__ void scale_inv_kernel(const double* x, const double* s, long long n, double* y) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    y[t] = x[t] / s[0];
}

__global__ void sqrt_kernel(double* s) { s[0] = sqrt(s[0]); }

}  // namespace

int krylov_blocks(long long n) {
    long long b = (n + 4 * kThreads - 1) / (4 * kThreads);
    return (int)(b < 1 ? 1 : (b > 608 ? 608 : b));
}

// h[0..k) = V[0..k)^T w (device), partial holds k * krylov_blocks(n) doubles
cudaError_t launch_multidot(const double* V, int k, long long n, const double* w, double* partial, double* h,
                            cudaStream_t s) {
    if (k < 1 || k > kMaxBasis) return cudaErrorInvalidValue;
    const int nb = krylov_blocks(n);
    SN_COUNT_LAUNCH();
    multidot_partial_kernel<<<nb, kThreads, 0, s>>>(V, k, n, w, partial, nb, nullptr, 0);
    SN_COUNT_LAUNCH();
    multidot_final_kernel<<<k, kThreads, 0, s>>>(partial, nb, h, nullptr, 0);
    return cudaGetLastError();
}

// As launch_multidot with k = *kdev + kofs read on the device (at most kmax)
cudaError_t launch_multidot_dev(const double* V, const int* kdev, int kofs, int kmax, long long n, const double* w,
                                double* partial, double* h, cudaStream_t s) {
    if (kmax < 1 || kmax > kMaxBasis) return cudaErrorInvalidValue;
    const int nb = krylov_blocks(n);
    SN_COUNT_LAUNCH();
    multidot_partial_kernel<<<nb, kThreads, 0, s>>>(V, kmax, n, w, partial, nb, kdev, kofs);
    SN_COUNT_LAUNCH();
    multidot_final_kernel<<<kmax, kThreads, 0, s>>>(partial, nb, h, kdev, kofs);
    return cudaGetLastError();
}

cudaError_t launch_multiaxpy_dev(const double* V, const int* kdev, int kofs, long long n, const double* c, double sign,
                                 double* w, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    multiaxpy_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(V, 0, n, c, sign, w, kdev, kofs);
    return cudaGetLastError();
}

cudaError_t launch_multiaxpy(const double* V, int k, long long n, const double* c, double sign, double* w,
                             cudaStream_t s) {
    SN_COUNT_LAUNCH();
    multiaxpy_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, s>>>(V, k, n, c, sign, w, nullptr, 0);
    return cudaGetLastError();
}

// s[0] = ||x|| (via the multidot machinery), y = x / ||x||
cudaError_t launch_normalize(const double* x, long long n, double* partial, double* s, double* y, cudaStream_t st) {
    cudaError_t err = launch_multidot(x, 1, n, x, partial, s, st);
    if (err != cudaSuccess) return err;
    SN_COUNT_LAUNCH();
    sqrt_kernel<<<1, 1, 0, st>>>(s);
    SN_COUNT_LAUNCH();
    scale_inv_kernel<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(x, s, n, y);
    return cudaGetLastError();
}

}  // namespace sn
