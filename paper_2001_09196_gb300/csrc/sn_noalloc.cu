// Scalar-flux reduction that allocates nothing (sn_scalar_flux_noalloc in include/sn.h).
//
// Same arithmetic as the flux reduction that follows every sweep: phi_out = sum_d w_d psi_d in
// float64, summed over directions in index order, and ||phi_out - phi_prev||^2 reduced in a
// fixed two-stage order.  The first stage's per-block partial sums live in a file-scope
// device array instead of memory owned by a mesh, so the call needs no cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>

#include "sn_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr long long kMaxBlocks = 8192;
constexpr long long kMaxValues = kMaxBlocks * kThreads;  // 2,097,152 flux values per call

// Shared by every call on a device; holds the last call's partial sums until the next call.
static __device__ __align__(256) double g_partials[kMaxBlocks];

__global__ void flux_partial_kernel(const double* psi, const double* w, int nd, long long m, const double* phi_prev,
                                    double* phi_out, double* partials) {
    __shared__ double sh[kThreads];
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double rr = 0.0;
    if (idx < m) {
        double s = 0.0;
        for (int d = 0; d < nd; ++d) s += w[d] * psi[(size_t)d * m + idx];
        phi_out[idx] = s;
        const double r = s - (phi_prev ? phi_prev[idx] : 0.0);
        rr = r * r;
    }
    sh[threadIdx.x] = rr;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void flux_final_kernel(const double* partials, int nblocks, double* out) {
    __shared__ double sh[1024];
    double s = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += partials[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_partials_addr[kMaxDevices] = {};  // device address of g_partials, per device

}  // namespace

extern "C" sn_status sn_scalar_flux_noalloc(const double* psi, const double* weights, int n_dirs, long long n_values,
                                            const double* phi_prev, double* phi_out, double* resid_norm2,
                                            void* stream) {
    if (!psi || !weights || !phi_out) return sn::set_error(SN_ERR_ARG, "psi, weights and phi_out must be non-null");
    if (n_dirs < 1) return sn::set_error(SN_ERR_ARG, "n_dirs must be >= 1");
    if (n_values < 1) return sn::set_error(SN_ERR_ARG, "n_values must be >= 1");
    if (n_values > kMaxValues)
        return sn::set_error(SN_ERR_ARG, "n_values exceeds the no-allocation limit of 2097152 (8192 blocks x 256)");
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return sn::set_error(SN_ERR_CUDA, cudaGetErrorString(err));
    if (dev < 0 || dev >= kMaxDevices) return sn::set_error(SN_ERR_ARG, "device index beyond the supported range");
    double* partials = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_partials_addr[dev]) {
            // one-time set-up on this device (with it current): the host-side symbol is only a
            // stand-in, kernels need the device address.
            void* p = nullptr;
            err = cudaGetSymbolAddress(&p, g_partials);
            if (err != cudaSuccess) return sn::set_error(SN_ERR_CUDA, cudaGetErrorString(err));
            g_partials_addr[dev] = static_cast<double*>(p);
        }
        partials = g_partials_addr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = (int)((n_values + kThreads - 1) / kThreads);
    SN_COUNT_LAUNCH();
    flux_partial_kernel<<<nblocks, kThreads, 0, s>>>(psi, weights, n_dirs, n_values, phi_prev, phi_out, partials);
    if (resid_norm2) {
        SN_COUNT_LAUNCH();
        flux_final_kernel<<<1, 1024, 0, s>>>(partials, nblocks, resid_norm2);
    }
    err = cudaGetLastError();
    if (err != cudaSuccess) return sn::set_error(SN_ERR_CUDA, cudaGetErrorString(err));
    return SN_OK;
}
