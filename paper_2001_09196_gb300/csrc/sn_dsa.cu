// Thick-subdomain DSA on the device (paper Sec. 2.2 Eq. DSA_fp, Algorithm 2, Sec. 3):
// conjugate gradients on the symmetric operator (Eq. SIP), BiCGStab on the nonsymmetric ones
// (Eq. NIP, with or without Eq. ModifiedF0), both preconditioned by one multigrid V-cycle
// (block-Jacobi on the DG level, weighted Jacobi on the continuous levels, dense coarsest).
// All vectors and reductions are float64; dot products reduce in a fixed order.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "sn_dsa.h"

namespace sn {

namespace {

constexpr int kBS = 256;
inline unsigned nblk(long long n) { return (unsigned)((n + kBS - 1) / kBS); }

__global__ void gather_kernel(const double* full, const int* thick, const double* mass, int nt, int n, double* out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nt * n) return;
    const int t = (int)(idx / n), i = (int)(idx % n);
    const double v = full[(size_t)thick[t] * n + i];
    out[idx] = mass ? mass[idx] * v : v;
}

__global__ void scatter_add_kernel(const double* x, const int* thick, const double* mass, int nt, int n, double* full) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nt * n) return;
    const int t = (int)(idx / n), i = (int)(idx % n);
    full[(size_t)thick[t] * n + i] += mass ? mass[idx] * x[idx] : x[idx];
}

__global__ void scatter_set_kernel(const double* x, const int* thick, int nt, int n, double* full) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nt * n) return;
    const int t = (int)(idx / n), i = (int)(idx % n);
    full[(size_t)thick[t] * n + i] = x[idx];
}

// The V-cycle kernels are templated on the arithmetic type T: float64 for the operator products
// of the Krylov solvers and for tight inner tolerances, float32 for the preconditioner when the
// inner tolerance is loose (the Krylov residuals, dot products and tests stay float64).

// out = b - A x (b may be null: out = A x), BSR with n x n blocks; one thread per (row block, node)
template <typename T>
__global__ void bsr_kernel(const int* ptr, const int* col, const T* val, int nt, int n, const T* x, const T* b,
                           T* out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nt * n) return;
    const int t = (int)(idx / n), i = (int)(idx % n);
    T s = T(0);
    for (int k = ptr[t]; k < ptr[t + 1]; ++k) {
        const T* blk = val + (size_t)k * n * n + (size_t)i * n;
        const T* xc = x + (size_t)col[k] * n;
        for (int j = 0; j < n; ++j) s += blk[j] * xc[j];
    }
    out[idx] = b ? b[idx] - s : s;
}

// x (+)= omega Dinv r per block
template <typename T>
__global__ void block_jacobi_kernel(const T* dinv, int nt, int n, T omega, const T* r, T* x, int accumulate) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)nt * n) return;
    const int t = (int)(idx / n), i = (int)(idx % n);
    const T* D = dinv + (size_t)t * n * n + (size_t)i * n;
    const T* rr = r + (size_t)t * n;
    T s = T(0);
    for (int j = 0; j < n; ++j) s += D[j] * rr[j];
    x[idx] = (accumulate ? x[idx] : T(0)) + omega * s;
}

// precision conversions at the entry and exit of a float32 V-cycle
template <typename A, typename B>
__global__ void convert_kernel(const A* in, B* out, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = static_cast<B>(in[i]);
}

// CSR product with G lanes per row (G a power of two dividing 32): the lanes of a group take
// every G-th entry of the row and the group adds its partial sums by a fixed shuffle tree, so a
// row costs about (nnz / G) dependent loads instead of nnz.  mode 0: out = M x; 1: out = b - M x;
// 2: out += M x.
template <int G, typename T>
__global__ void csr_vec_kernel(const int* ptr, const int* col, const T* val, int rows, const T* x, const T* b, T* out,
                               int mode) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int gl = threadIdx.x & (G - 1);
    const long long row = tid / G;
    T s = T(0);
    if (row < rows) {
        const int k1 = ptr[row + 1];
        for (int k = ptr[row] + gl; k < k1; k += G) s += val[k] * x[col[k]];
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (row < rows && gl == 0) {
        if (mode == 0) out[row] = s;
        else if (mode == 1) out[row] = b[row] - s;
        else out[row] += s;
    }
}

// x = A b for the dense coarsest level, one warp per row (lanes stride over the columns)
template <typename T>
__global__ void dense_mv_warp_kernel(const T* A, int n, const T* b, T* x) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const long long row = tid >> 5;
    T s = T(0);
    if (row < n)
        for (int c = lane; c < n; c += 32) s += A[(size_t)row * n + c] * b[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (row < n && lane == 0) x[row] = s;
}

template <typename T>
__global__ void jacobi_kernel(const T* dinv, int rows, T omega, const T* r, T* x, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    x[i] = (accumulate ? x[i] : T(0)) + omega * dinv[i] * r[i];
}

// Algorithm 1 (triangular heterogeneous DSA) helpers on full [elem][node] vectors; emask marks
// the thick elements.
__global__ void select_thick_kernel(const unsigned char* emask, int n, long long M, const double* x, double* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    out[i] = emask[i / n] ? x[i] : 0.0;
}

// thick DOFs: phi += w - r (the DSA correction, w = r + D^{-1} Sigma r there); thin DOFs: phi += y
__global__ void tri_combine_kernel(const unsigned char* emask, int n, long long M, const double* w, const double* r,
                                   const double* y, double* phi) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    phi[i] += emask[i / n] ? w[i] - r[i] : y[i];
}

__global__ void add_thin_kernel(const unsigned char* emask, int n, long long M, const double* y, double* z) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    if (!emask[i / n]) z[i] += y[i];
}

__global__ void dot_partial_kernel(const double* a, const double* b, long long n, double* part) {
    __shared__ double sh[kBS];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        s += a[i] * b[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void dot_final_kernel(const double* part, int n, double* out) {
    __shared__ double sh[kBS];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// x += alpha p, r -= alpha q with alpha = s[0] / s[1]
__global__ void cg_update_xr(double* x, double* r, const double* p, const double* q, long long n, const double* s) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double alpha = s[0] / s[1];
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
}

// p = z + beta p with beta = s[4] / s[0]; the last thread to finish cannot update s, so s[0] is
// refreshed by a separate kernel.
__global__ void cg_update_p(double* p, const double* z, long long n, const double* s) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double beta = s[4] / s[0];
    p[i] = z[i] + beta * p[i];
}

__global__ void copy_scalar(double* s, int dst, int src) { s[dst] = s[src]; }

// Start of the recorded PCG: s[0] (r.z of the previous iteration) = +inf makes the first search
// direction p = z; the loop runs only for b != 0.
__global__ void pcg_start_kernel(double* s, int* it, cudaGraphConditionalHandle h) {
    s[0] = INFINITY;
    it[0] = 0;
    cudaGraphSetConditional(h, s[3] > 0.0 ? 1u : 0u);
}

// End of one recorded PCG iteration: continue while ||r|| > tol ||b|| and fewer than max_iters.
__global__ void pcg_check_kernel(const double* s, int* it, double tol, int max_iters, cudaGraphConditionalHandle h) {
    const int k = ++it[0];
    ++it[1];
    const bool more = sqrt(s[2]) > tol * sqrt(s[3]) && k < max_iters;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

// BiCGStab (right-preconditioned with the V-cycle M) scalars in s: [0] rho of the previous
// iteration, [1] alpha, [2] omega, [3] b.b, [4] rho = rhat.r, [5] rhat.v, [6] t.s, [7] t.t, [8] r.r.
__global__ void bicg_start_kernel(double* s, int* it, cudaGraphConditionalHandle h) {
    s[0] = s[1] = s[2] = 1.0;
    it[0] = 0;
    cudaGraphSetConditional(h, s[3] > 0.0 ? 1u : 0u);
}

// p = r + beta (p - omega v), beta = (rho / rho_prev) (alpha / omega)
__global__ void bicg_update_p(double* p, const double* r, const double* v, long long n, const double* s) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double beta = (s[4] / s[0]) * (s[1] / s[2]);
    p[i] = r[i] + beta * (p[i] - s[2] * v[i]);
}

// alpha = rho / rhat.v; x += alpha M p; r <- s = r - alpha v
__global__ void bicg_update_xs(double* x, double* r, const double* ph, const double* v, long long n, const double* s) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double alpha = s[5] != 0.0 ? s[4] / s[5] : 0.0;
    x[i] += alpha * ph[i];
    r[i] -= alpha * v[i];
}

// omega = t.s / t.t; x += omega M s; r = s - omega t
__global__ void bicg_update_xr(double* x, double* r, const double* sh, const double* t, long long n, const double* s) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double omega = s[7] > 0.0 ? s[6] / s[7] : 0.0;
    x[i] += omega * sh[i];
    r[i] -= omega * t[i];
}

// End of one iteration: keep rho, alpha, omega for the next; continue while ||r|| > tol ||b||,
// fewer than max_iters, and no breakdown (rho, alpha or omega zero, or a non-finite residual).
__global__ void bicg_check_kernel(double* s, int* it, double tol, int max_iters, cudaGraphConditionalHandle h) {
    const double alpha = s[5] != 0.0 ? s[4] / s[5] : 0.0;
    const double omega = s[7] > 0.0 ? s[6] / s[7] : 0.0;
    s[0] = s[4];
    s[1] = alpha;
    s[2] = omega;
    const int k = ++it[0];
    ++it[1];
    const bool ok = s[4] != 0.0 && alpha != 0.0 && omega != 0.0 && isfinite(s[8]);
    const bool more = ok && sqrt(s[8]) > tol * sqrt(s[3]) && k < max_iters;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

constexpr int kDotBlocks = 304;  // 2 x 152 SMs

template <typename T>
cudaError_t up(T** d, const std::vector<T>& h) {
    if (h.empty()) { *d = nullptr; return cudaSuccess; }
    cudaError_t err = cudaMalloc(d, h.size() * sizeof(T));
    if (err != cudaSuccess) return err;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

cudaError_t upload(DsaHierarchy* H) {
    if (H->uploaded) return cudaSuccess;
    const long long N0 = (long long)H->nt * H->n;
    cudaError_t err;
#define UP(dst, src) if ((err = up(&(dst), src)) != cudaSuccess) return err
    UP(H->d_thick, H->thick);
    UP(H->d_mass_sig, H->h_mass_sig);
    UP(H->l0.d_ptr, H->l0.ptr);
    UP(H->l0.d_col, H->l0.col);
    UP(H->l0.d_val, H->l0.val);
    UP(H->l0.d_dinv, H->l0.dinv);
    for (LevelC& L : H->levels) {
        UP(L.d_a_ptr, L.a_ptr);
        UP(L.d_a_col, L.a_col);
        UP(L.d_a_val, L.a_val);
        UP(L.d_p_ptr, L.p_ptr);
        UP(L.d_p_col, L.p_col);
        UP(L.d_p_val, L.p_val);
        UP(L.d_r_ptr, L.r_ptr);
        UP(L.d_r_col, L.r_col);
        UP(L.d_r_val, L.r_val);
        UP(L.d_dinv, L.dinv);
        UP(L.d_dense, L.dense_inv);
        for (double** v : {&L.d_x, &L.d_b, &L.d_r})
            if ((err = cudaMalloc(v, std::max(1, L.n) * sizeof(double))) != cudaSuccess) return err;
    }
#undef UP
    for (double** v : {&H->d_x, &H->d_b, &H->d_r, &H->d_z, &H->d_p, &H->d_q, &H->d_vr, &H->d_vx})
        if ((err = cudaMalloc(v, std::max<long long>(1, N0) * sizeof(double))) != cudaSuccess) return err;
    if (!H->symmetric)
        for (double** v : {&H->d_rh, &H->d_sh, &H->d_t})
            if ((err = cudaMalloc(v, std::max<long long>(1, N0) * sizeof(double))) != cudaSuccess) return err;
    if ((err = cudaMalloc(&H->d_part, kDotBlocks * sizeof(double))) != cudaSuccess) return err;
    if ((err = cudaMalloc(&H->d_s, 16 * sizeof(double))) != cudaSuccess) return err;
    {
        std::vector<unsigned char> em(H->ne, 0);
        for (int e : H->thick) em[e] = 1;
        if ((err = cudaMalloc(&H->d_emask, std::max(1, H->ne))) != cudaSuccess) return err;
        if ((err = cudaMemcpy(H->d_emask, em.data(), H->ne, cudaMemcpyHostToDevice)) != cudaSuccess) return err;
    }
    if ((err = cudaMalloc(&H->d_it, 2 * sizeof(int))) != cudaSuccess) return err;
    if ((err = cudaMemset(H->d_it, 0, 2 * sizeof(int))) != cudaSuccess) return err;
    H->uploaded = true;
    return cudaSuccess;
}

template <typename T>
cudaError_t up32(float** d, const std::vector<T>& h) {
    if (h.empty()) { *d = nullptr; return cudaSuccess; }
    std::vector<float> f(h.begin(), h.end());
    cudaError_t err = cudaMalloc(d, f.size() * sizeof(float));
    if (err != cudaSuccess) return err;
    return cudaMemcpy(*d, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice);
}

// float32 copies of the hierarchy's values and the float32 V-cycle's vectors (made once, on demand)
cudaError_t upload32(DsaHierarchy* H) {
    if (H->uploaded32) return cudaSuccess;
    const long long N0 = (long long)H->nt * H->n;
    cudaError_t err;
#define UP32(dst, src) if ((err = up32(&(dst), src)) != cudaSuccess) return err
    UP32(H->l0.d_val32, H->l0.val);
    UP32(H->l0.d_dinv32, H->l0.dinv);
    for (LevelC& L : H->levels) {
        UP32(L.d_a_val32, L.a_val);
        UP32(L.d_p_val32, L.p_val);
        UP32(L.d_r_val32, L.r_val);
        UP32(L.d_dinv32, L.dinv);
        UP32(L.d_dense32, L.dense_inv);
        for (float** v : {&L.d_x32, &L.d_b32, &L.d_r32})
            if ((err = cudaMalloc(v, std::max(1, L.n) * sizeof(float))) != cudaSuccess) return err;
    }
#undef UP32
    for (float** v : {&H->d_vr32, &H->d_r32, &H->d_z32})
        if ((err = cudaMalloc(v, std::max<long long>(1, N0) * sizeof(float))) != cudaSuccess) return err;
    H->uploaded32 = true;
    return cudaSuccess;
}

cudaError_t dot(DsaHierarchy* H, const double* a, const double* b, long long n, int slot, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    dot_partial_kernel<<<kDotBlocks, kBS, 0, s>>>(a, b, n, H->d_part);
    SN_COUNT_LAUNCH();
    dot_final_kernel<<<1, kBS, 0, s>>>(H->d_part, kDotBlocks, H->d_s + slot);
    return cudaGetLastError();
}

// Pointers of the multigrid hierarchy in one arithmetic type (the index arrays are shared).
template <typename T>
struct VLevel {
    int n = 0;
    long long a_nnz = 0, p_nnz = 0, r_nnz = 0;
    const int *a_ptr, *a_col, *p_ptr, *p_col, *r_ptr, *r_col;
    const T *a_val, *p_val, *r_val, *dinv, *dense;
    T *x, *b, *r;
};
template <typename T>
struct VCycle {
    int nt = 0, n = 0, nu = 2;
    T omega0 = T(0.6), omega = T(0.6);
    const int *l0_ptr, *l0_col;
    const T *l0_val, *l0_dinv;
    T* vr;
    std::vector<VLevel<T>> levels;
};

VCycle<double> view64(const DsaHierarchy* H) {
    VCycle<double> V;
    V.nt = H->nt; V.n = H->n; V.nu = H->nu; V.omega0 = H->omega0; V.omega = H->omega;
    V.l0_ptr = H->l0.d_ptr; V.l0_col = H->l0.d_col; V.l0_val = H->l0.d_val; V.l0_dinv = H->l0.d_dinv; V.vr = H->d_vr;
    for (const LevelC& L : H->levels)
        V.levels.push_back({L.n, (long long)L.a_val.size(), (long long)L.p_val.size(), (long long)L.r_val.size(),
                            L.d_a_ptr, L.d_a_col, L.d_p_ptr, L.d_p_col, L.d_r_ptr, L.d_r_col,
                            L.d_a_val, L.d_p_val, L.d_r_val, L.d_dinv, L.d_dense, L.d_x, L.d_b, L.d_r});
    return V;
}

VCycle<float> view32(const DsaHierarchy* H) {
    VCycle<float> V;
    V.nt = H->nt; V.n = H->n; V.nu = H->nu; V.omega0 = (float)H->omega0; V.omega = (float)H->omega;
    V.l0_ptr = H->l0.d_ptr; V.l0_col = H->l0.d_col; V.l0_val = H->l0.d_val32; V.l0_dinv = H->l0.d_dinv32; V.vr = H->d_vr32;
    for (const LevelC& L : H->levels)
        V.levels.push_back({L.n, (long long)L.a_val.size(), (long long)L.p_val.size(), (long long)L.r_val.size(),
                            L.d_a_ptr, L.d_a_col, L.d_p_ptr, L.d_p_col, L.d_r_ptr, L.d_r_col,
                            L.d_a_val32, L.d_p_val32, L.d_r_val32, L.d_dinv32, L.d_dense32, L.d_x32, L.d_b32, L.d_r32});
    return V;
}

// CSR product with the group width chosen from the rows' average length.
template <typename T>
void csr_mv(const int* ptr, const int* col, const T* val, int rows, long long nnz, const T* x, const T* b, T* out,
            int mode, cudaStream_t s) {
    if (rows <= 0) return;
    const double avg = (double)nnz / rows;
    SN_COUNT_LAUNCH();
    if (avg > 12.0) csr_vec_kernel<8, T><<<nblk((long long)rows * 8), kBS, 0, s>>>(ptr, col, val, rows, x, b, out, mode);
    else if (avg > 3.0) csr_vec_kernel<4, T><<<nblk((long long)rows * 4), kBS, 0, s>>>(ptr, col, val, rows, x, b, out, mode);
    else csr_vec_kernel<1, T><<<nblk(rows), kBS, 0, s>>>(ptr, col, val, rows, x, b, out, mode);
}

// continuous level l: x = V(b)
template <typename T>
void vcycle_c(const VCycle<T>& V, size_t l, cudaStream_t s) {
    const VLevel<T>& L = V.levels[l];
    if (L.dense) {
        SN_COUNT_LAUNCH();
        dense_mv_warp_kernel<T><<<nblk((long long)L.n * 32), kBS, 0, s>>>(L.dense, L.n, L.b, L.x);
        return;
    }
    for (int k = 0; k < V.nu; ++k) {
        if (k == 0) {
            SN_COUNT_LAUNCH();
            jacobi_kernel<T><<<nblk(L.n), kBS, 0, s>>>(L.dinv, L.n, V.omega, L.b, L.x, 0);
        } else {
            csr_mv<T>(L.a_ptr, L.a_col, L.a_val, L.n, L.a_nnz, L.x, L.b, L.r, 1, s);
            SN_COUNT_LAUNCH();
            jacobi_kernel<T><<<nblk(L.n), kBS, 0, s>>>(L.dinv, L.n, V.omega, L.r, L.x, 1);
        }
    }
    csr_mv<T>(L.a_ptr, L.a_col, L.a_val, L.n, L.a_nnz, L.x, L.b, L.r, 1, s);
    const VLevel<T>& C = V.levels[l + 1];
    csr_mv<T>(C.r_ptr, C.r_col, C.r_val, C.n, C.r_nnz, L.r, nullptr, C.b, 0, s);
    vcycle_c<T>(V, l + 1, s);
    csr_mv<T>(C.p_ptr, C.p_col, C.p_val, L.n, C.p_nnz, C.x, nullptr, L.x, 2, s);
    for (int k = 0; k < V.nu; ++k) {
        csr_mv<T>(L.a_ptr, L.a_col, L.a_val, L.n, L.a_nnz, L.x, L.b, L.r, 1, s);
        SN_COUNT_LAUNCH();
        jacobi_kernel<T><<<nblk(L.n), kBS, 0, s>>>(L.dinv, L.n, V.omega, L.r, L.x, 1);
    }
}

// z = V(r) on the DG level
template <typename T>
void vcycle0_t(const VCycle<T>& V, const T* r, T* z, cudaStream_t s) {
    const int nt = V.nt, n = V.n;
    const long long N0 = (long long)nt * n;
    for (int k = 0; k < V.nu; ++k) {
        if (k == 0) {
            SN_COUNT_LAUNCH();
            block_jacobi_kernel<T><<<nblk(N0), kBS, 0, s>>>(V.l0_dinv, nt, n, V.omega0, r, z, 0);
        } else {
            SN_COUNT_LAUNCH();
            bsr_kernel<T><<<nblk(N0), kBS, 0, s>>>(V.l0_ptr, V.l0_col, V.l0_val, nt, n, z, r, V.vr);
            SN_COUNT_LAUNCH();
            block_jacobi_kernel<T><<<nblk(N0), kBS, 0, s>>>(V.l0_dinv, nt, n, V.omega0, V.vr, z, 1);
        }
    }
    if (!V.levels.empty()) {
        SN_COUNT_LAUNCH();
        bsr_kernel<T><<<nblk(N0), kBS, 0, s>>>(V.l0_ptr, V.l0_col, V.l0_val, nt, n, z, r, V.vr);
        const VLevel<T>& C = V.levels[0];
        csr_mv<T>(C.r_ptr, C.r_col, C.r_val, C.n, C.r_nnz, V.vr, nullptr, C.b, 0, s);
        vcycle_c<T>(V, 0, s);
        csr_mv<T>(C.p_ptr, C.p_col, C.p_val, (int)N0, C.p_nnz, C.x, nullptr, z, 2, s);
    }
    for (int k = 0; k < V.nu; ++k) {
        SN_COUNT_LAUNCH();
        bsr_kernel<T><<<nblk(N0), kBS, 0, s>>>(V.l0_ptr, V.l0_col, V.l0_val, nt, n, z, r, V.vr);
        SN_COUNT_LAUNCH();
        block_jacobi_kernel<T><<<nblk(N0), kBS, 0, s>>>(V.l0_dinv, nt, n, V.omega0, V.vr, z, 1);
    }
}

// z = V(r) on float64 vectors, in float64 or (H->pc32) in float32 between two conversions
void vcycle0(DsaHierarchy* H, const double* r, double* z, cudaStream_t s) {
    if (!H->pc32) {
        vcycle0_t<double>(view64(H), r, z, s);
        return;
    }
    const long long N0 = (long long)H->nt * H->n;
    SN_COUNT_LAUNCH();
    convert_kernel<double, float><<<nblk(N0), kBS, 0, s>>>(r, H->d_r32, N0);
    vcycle0_t<float>(view32(H), H->d_r32, H->d_z32, s);
    SN_COUNT_LAUNCH();
    convert_kernel<float, double><<<nblk(N0), kBS, 0, s>>>(H->d_z32, z, N0);
}

// Records the Krylov solve of D_ff x = b (thick-local vectors H->d_b -> H->d_x) into a CUDA graph:
// a prologue and a WHILE conditional node whose body is one iteration; the convergence test runs
// on the device, so a solve is one graph launch.
//   PCG (symmetric operator), the preconditioned CG of the eager form step for step:
//     prologue x = 0, p = 0, r = b, b.b;  body z = M r; rz = r.z; p = z + (rz / rz_prev) p; q = A p;
//     alpha = rz / p.q; x += alpha p; r -= alpha q.
//   BiCGStab (nonsymmetric operators), right-preconditioned by the same V-cycle M:
//     prologue x = 0, r = rhat = b, p = v = 0, b.b;  body rho = rhat.r;
//     p = r + (rho / rho_prev)(alpha / omega)(p - omega v); ph = M p; v = A ph; alpha = rho / rhat.v;
//     x += alpha ph; s = r - alpha v; sh = M s; t = A sh; omega = t.s / t.t; x += omega sh;
//     r = s - omega t.
// Both continue while ||r|| > tol ||b|| and k < max_iters.
// Emits that solve into the graph the stream `cs_stream` is capturing: the prologue on cs_stream, then
// a WHILE node whose body is captured on H->cap2.  Launch counters: the kernels of the prologue and
// of one loop iteration are counted into *pro and *body (g_launches is left as it was).
static cudaError_t emit_krylov(DsaHierarchy* H, cudaStream_t cs_stream, double tol, int max_iters, long long* pro,
                               long long* body_count) {
    const long long N0 = (long long)H->nt * H->n;
    const Level0& A = H->l0;
    cudaError_t err;
    if (!H->cap2 && (err = cudaStreamCreateWithFlags(&H->cap2, cudaStreamNonBlocking)) != cudaSuccess) return err;
    const long long count0 = g_launches.load();
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    if ((err = cudaStreamGetCaptureInfo(cs_stream, &cs, nullptr, &g, nullptr, nullptr, nullptr)) != cudaSuccess) return err;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureUnsupported;
    cudaGraphConditionalHandle h;
    if ((err = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return err;
    cudaMemsetAsync(H->d_x, 0, N0 * sizeof(double), cs_stream);
    cudaMemsetAsync(H->d_p, 0, N0 * sizeof(double), cs_stream);
    cudaMemcpyAsync(H->d_r, H->d_b, N0 * sizeof(double), cudaMemcpyDeviceToDevice, cs_stream);
    if (!H->symmetric) {
        cudaMemsetAsync(H->d_q, 0, N0 * sizeof(double), cs_stream);
        cudaMemcpyAsync(H->d_rh, H->d_b, N0 * sizeof(double), cudaMemcpyDeviceToDevice, cs_stream);
    }
    dot(H, H->d_b, H->d_b, N0, 3, cs_stream);
    SN_COUNT_LAUNCH();
    if (H->symmetric) pcg_start_kernel<<<1, 1, 0, cs_stream>>>(H->d_s, H->d_it, h);
    else bicg_start_kernel<<<1, 1, 0, cs_stream>>>(H->d_s, H->d_it, h);
    *pro = g_launches.load() - count0;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if ((err = cudaStreamGetCaptureInfo(cs_stream, &cs, nullptr, nullptr, &deps, nullptr, &ndeps)) != cudaSuccess) {
        g_launches.store(count0);
        return err;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((err = cudaGraphAddNode(&loop, g, deps, nullptr, ndeps, &cp)) != cudaSuccess ||
        (err = cudaStreamUpdateCaptureDependencies(cs_stream, &loop, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
            cudaSuccess) {
        g_launches.store(count0);
        return err;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((err = cudaStreamBeginCaptureToGraph(H->cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess) {
        g_launches.store(count0);
        return err;
    }
    const long long count1 = g_launches.load();
    cudaStream_t s = H->cap2;
    if (H->symmetric) {
        vcycle0(H, H->d_r, H->d_z, s);
        dot(H, H->d_r, H->d_z, N0, 4, s);
        SN_COUNT_LAUNCH();
        cg_update_p<<<nblk(N0), kBS, 0, s>>>(H->d_p, H->d_z, N0, H->d_s);
        SN_COUNT_LAUNCH();
        copy_scalar<<<1, 1, 0, s>>>(H->d_s, 0, 4);
        SN_COUNT_LAUNCH();
        bsr_kernel<double><<<nblk(N0), kBS, 0, s>>>(A.d_ptr, A.d_col, A.d_val, H->nt, H->n, H->d_p, nullptr, H->d_q);
        dot(H, H->d_p, H->d_q, N0, 1, s);
        SN_COUNT_LAUNCH();
        cg_update_xr<<<nblk(N0), kBS, 0, s>>>(H->d_x, H->d_r, H->d_p, H->d_q, N0, H->d_s);
        dot(H, H->d_r, H->d_r, N0, 2, s);
        SN_COUNT_LAUNCH();
        pcg_check_kernel<<<1, 1, 0, s>>>(H->d_s, H->d_it, tol, max_iters, h);
    } else {
        // vectors: p = d_p, ph = d_z, v = d_q, r (holding s after the first half) = d_r,
        // sh = d_sh, t = d_t, rhat = d_rh
        dot(H, H->d_rh, H->d_r, N0, 4, s);
        SN_COUNT_LAUNCH();
        bicg_update_p<<<nblk(N0), kBS, 0, s>>>(H->d_p, H->d_r, H->d_q, N0, H->d_s);
        vcycle0(H, H->d_p, H->d_z, s);
        SN_COUNT_LAUNCH();
        bsr_kernel<double><<<nblk(N0), kBS, 0, s>>>(A.d_ptr, A.d_col, A.d_val, H->nt, H->n, H->d_z, nullptr, H->d_q);
        dot(H, H->d_rh, H->d_q, N0, 5, s);
        SN_COUNT_LAUNCH();
        bicg_update_xs<<<nblk(N0), kBS, 0, s>>>(H->d_x, H->d_r, H->d_z, H->d_q, N0, H->d_s);
        vcycle0(H, H->d_r, H->d_sh, s);
        SN_COUNT_LAUNCH();
        bsr_kernel<double><<<nblk(N0), kBS, 0, s>>>(A.d_ptr, A.d_col, A.d_val, H->nt, H->n, H->d_sh, nullptr, H->d_t);
        dot(H, H->d_t, H->d_r, N0, 6, s);
        dot(H, H->d_t, H->d_t, N0, 7, s);
        SN_COUNT_LAUNCH();
        bicg_update_xr<<<nblk(N0), kBS, 0, s>>>(H->d_x, H->d_r, H->d_sh, H->d_t, N0, H->d_s);
        dot(H, H->d_r, H->d_r, N0, 8, s);
        SN_COUNT_LAUNCH();
        bicg_check_kernel<<<1, 1, 0, s>>>(H->d_s, H->d_it, tol, max_iters, h);
    }
    *body_count = g_launches.load() - count1;
    g_launches.store(count0);  // recorded, not run: launches are counted when the graph runs
    cudaError_t lerr = cudaGetLastError();
    cudaGraph_t b2 = nullptr;
    err = cudaStreamEndCapture(H->cap2, &b2);
    if (lerr != cudaSuccess) return lerr;
    return err;
}

// Records the solve as a graph of its own (one launch per solve, see emit_krylov).
cudaError_t record_krylov(DsaHierarchy* H, double tol, int max_iters) {
    cudaError_t err;
    if (!H->cap && (err = cudaStreamCreateWithFlags(&H->cap, cudaStreamNonBlocking)) != cudaSuccess) return err;
    if (H->krylov_graph) cudaGraphExecDestroy(H->krylov_graph);
    H->krylov_graph = nullptr;
    if ((err = cudaStreamBeginCapture(H->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return err;
    cudaError_t e = emit_krylov(H, H->cap, tol, max_iters, &H->pro_launches, &H->body_launches);
    cudaGraph_t g2 = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(H->cap, &g2);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&H->krylov_graph, g2, 0);
    if (g2) cudaGraphDestroy(g2);
    if (e != cudaSuccess) H->krylov_graph = nullptr;
    if (e == cudaSuccess) {
        H->krylov_tol = tol;
        H->krylov_max = max_iters;
    }
    return e;
}

// Solves D_ff x = b by one launch of the recorded Krylov solve; the iteration count stays on the
// device (dsa_take_iters reads the running total).
cudaError_t krylov_solve(DsaHierarchy* H, double tol, int max_iters, cudaStream_t s) {
    cudaError_t err;
    const bool want32 = H->vcycle_mode == SN_VCYCLE_FP32 || (H->vcycle_mode == SN_VCYCLE_AUTO && tol >= 1e-8);
    if (want32 && (err = upload32(H)) != cudaSuccess) return err;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if ((err = cudaStreamIsCapturing(s, &cs)) != cudaSuccess) return err;
    if (cs == cudaStreamCaptureStatusActive) {
        // inside an enclosing capture (a recorded outer iteration): the loop becomes a nested WHILE
        // node; its launches are counted when the enclosing graph runs (dsa_take_iters)
        H->pc32 = want32;
        long long pro = 0, body = 0;
        err = emit_krylov(H, s, tol, max_iters, &pro, &body);
        H->body_launches = body;
        H->nested_pro_launches = pro;
        return err;
    }
    if (!H->krylov_graph || H->krylov_tol != tol || H->krylov_max != max_iters || H->krylov_pc32 != want32) {
        H->pc32 = want32;
        H->krylov_pc32 = want32;
        if ((err = record_krylov(H, tol, max_iters)) != cudaSuccess) return err;
    }
    g_launches.fetch_add(H->pro_launches, std::memory_order_relaxed);
    return cudaGraphLaunch(H->krylov_graph, s);
}

}  // namespace

void dsa_free(DsaHierarchy* H) {
    if (!H) return;
    auto f = [](void* p) { if (p) cudaFree(p); };
    f(H->d_thick); f(H->d_mass_sig);
    f(H->l0.d_ptr); f(H->l0.d_col); f(H->l0.d_val); f(H->l0.d_dinv);
    for (LevelC& L : H->levels) {
        f(L.d_a_ptr); f(L.d_a_col); f(L.d_a_val); f(L.d_p_ptr); f(L.d_p_col); f(L.d_p_val);
        f(L.d_r_ptr); f(L.d_r_col); f(L.d_r_val); f(L.d_dinv); f(L.d_dense); f(L.d_x); f(L.d_b); f(L.d_r);
        f(L.d_a_val32); f(L.d_p_val32); f(L.d_r_val32); f(L.d_dinv32); f(L.d_dense32); f(L.d_x32); f(L.d_b32); f(L.d_r32);
    }
    f(H->l0.d_val32); f(H->l0.d_dinv32); f(H->d_vr32); f(H->d_r32); f(H->d_z32);
    f(H->d_x); f(H->d_b); f(H->d_r); f(H->d_z); f(H->d_p); f(H->d_q); f(H->d_vr); f(H->d_vx);
    f(H->d_rh); f(H->d_sh); f(H->d_t);
    f(H->d_part); f(H->d_s); f(H->d_it); f(H->d_emask);
    if (H->krylov_graph) cudaGraphExecDestroy(H->krylov_graph);
    if (H->cap) cudaStreamDestroy(H->cap);
    if (H->cap2) cudaStreamDestroy(H->cap2);
    delete H;
}

int dsa_thick_count(const DsaHierarchy* H) { return H ? H->nt : 0; }

// Device copies a solve to tolerance tol needs (made before a solve is recorded into a graph).
cudaError_t dsa_prepare(DsaHierarchy* H, double tol) {
    cudaError_t err = upload(H);
    if (err != cudaSuccess || H->nt == 0) return err;
    const bool want32 = H->vcycle_mode == SN_VCYCLE_FP32 || (H->vcycle_mode == SN_VCYCLE_AUTO && tol >= 1e-8);
    if (want32) err = upload32(H);
    return err;
}

long long dsa_nested_prologue_launches(const DsaHierarchy* H) { return H ? H->nested_pro_launches : 0; }

cudaError_t dsa_apply(DsaHierarchy* H, const double* x, double* y, cudaStream_t s) {
    cudaError_t err = upload(H);
    if (err != cudaSuccess) return err;
    cudaMemsetAsync(y, 0, (size_t)H->ne * H->n * sizeof(double), s);
    if (H->nt == 0) return cudaGetLastError();
    const long long N0 = (long long)H->nt * H->n;
    SN_COUNT_LAUNCH();
    gather_kernel<<<nblk(N0), kBS, 0, s>>>(x, H->d_thick, nullptr, H->nt, H->n, H->d_p);
    SN_COUNT_LAUNCH();
    bsr_kernel<double><<<nblk(N0), kBS, 0, s>>>(H->l0.d_ptr, H->l0.d_col, H->l0.d_val, H->nt, H->n, H->d_p, nullptr, H->d_q);
    SN_COUNT_LAUNCH();
    scatter_set_kernel<<<nblk(N0), kBS, 0, s>>>(H->d_q, H->d_thick, H->nt, H->n, y);
    return cudaGetLastError();
}

cudaError_t dsa_solve(DsaHierarchy* H, const double* b_full, double* x_full, double tol, int max_iters, cudaStream_t s) {
    cudaError_t err = upload(H);
    if (err != cudaSuccess) return err;
    cudaMemsetAsync(x_full, 0, (size_t)H->ne * H->n * sizeof(double), s);
    if (H->nt == 0) return cudaGetLastError();
    const long long N0 = (long long)H->nt * H->n;
    SN_COUNT_LAUNCH();
    gather_kernel<<<nblk(N0), kBS, 0, s>>>(b_full, H->d_thick, nullptr, H->nt, H->n, H->d_b);
    if ((err = krylov_solve(H, tol, max_iters, s)) != cudaSuccess) return err;
    SN_COUNT_LAUNCH();
    scatter_set_kernel<<<nblk(N0), kBS, 0, s>>>(H->d_x, H->d_thick, H->nt, H->n, x_full);
    return cudaGetLastError();
}

// Forward (Algorithm 2): phi_out[thick] += D_ff^{-1} (Sigma r)_f.
// Transposed: phi_out[thick] += Sigma_f H^{-1} r_f, H = D_ff^T (D_ff itself when symmetric).
cudaError_t dsa_correct(DsaHierarchy* H, const double* r, double* phi_out, double tol, int max_iters, bool transpose,
                        cudaStream_t s) {
    cudaError_t err = upload(H);
    if (err != cudaSuccess) return err;
    if (H->nt == 0) return cudaSuccess;
    const long long N0 = (long long)H->nt * H->n;
    SN_COUNT_LAUNCH();
    gather_kernel<<<nblk(N0), kBS, 0, s>>>(r, H->d_thick, transpose ? nullptr : H->d_mass_sig, H->nt, H->n, H->d_b);
    if ((err = krylov_solve(H, tol, max_iters, s)) != cudaSuccess) return err;
    SN_COUNT_LAUNCH();
    scatter_add_kernel<<<nblk(N0), kBS, 0, s>>>(H->d_x, H->d_thick, transpose ? H->d_mass_sig : nullptr, H->nt, H->n,
                                                phi_out);
    return cudaGetLastError();
}

// Krylov iterations run since the last call (synchronises the stream); 0 before the first solve.
cudaError_t dsa_take_iters(DsaHierarchy* H, cudaStream_t s, int* iters) {
    *iters = 0;
    if (!H || !H->uploaded) return cudaSuccess;
    int h[2] = {0, 0};
    cudaError_t err = cudaMemcpyAsync(h, H->d_it, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return err;
    *iters = h[1];
    g_launches.fetch_add((long long)h[1] * H->body_launches, std::memory_order_relaxed);
    return cudaMemsetAsync(H->d_it + 1, 0, sizeof(int), s);
}

// Algorithm 1 pieces on full vectors (M = ne x n values).
cudaError_t dsa_select_thick(DsaHierarchy* H, const double* x, double* out, cudaStream_t s) {
    cudaError_t err = upload(H);
    if (err != cudaSuccess) return err;
    const long long M = (long long)H->ne * H->n;
    SN_COUNT_LAUNCH();
    select_thick_kernel<<<nblk(M), kBS, 0, s>>>(H->d_emask, H->n, M, x, out);
    return cudaGetLastError();
}

cudaError_t dsa_tri_combine(DsaHierarchy* H, const double* w, const double* r, const double* y, double* phi,
                            cudaStream_t s) {
    const long long M = (long long)H->ne * H->n;
    SN_COUNT_LAUNCH();
    tri_combine_kernel<<<nblk(M), kBS, 0, s>>>(H->d_emask, H->n, M, w, r, y, phi);
    return cudaGetLastError();
}

cudaError_t dsa_add_thin(DsaHierarchy* H, const double* y, double* z, cudaStream_t s) {
    const long long M = (long long)H->ne * H->n;
    SN_COUNT_LAUNCH();
    add_thin_kernel<<<nblk(M), kBS, 0, s>>>(H->d_emask, H->n, M, y, z);
    return cudaGetLastError();
}

}  // namespace sn
