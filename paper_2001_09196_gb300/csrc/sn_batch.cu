// Batched thick-subdomain DSA (paper Algorithm 2 applied to every instance of a batch at once).
//
// The instances' DSA systems D_ff^(i) delta_i = Sigma_f r_f^(i) are independent, so together they
// form one block-diagonal SPD system; conjugate gradients on that union system (one set of scalars)
// is conjugate gradients on an SPD matrix and converges to every instance's solution.  Its
// preconditioner is the union of the instances' multigrid V-cycles: level 0 is the union of the
// DG operators (segmented BSR, a block size per instance), level l the union of the instances'
// continuous level-l operators, and an instance whose hierarchy ends at level l contributes its
// dense coarsest inverse there.  Every kernel takes a device flag that turns it into a no-op once
// the solve has converged, so a fixed number of iterations can be recorded into a CUDA graph and
// still stop early.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "sn_dsa.h"

namespace sn {

struct UnionLevel {              // union continuous level
    int n = 0;
    int *a_ptr = nullptr, *a_col = nullptr, *p_ptr = nullptr, *p_col = nullptr, *r_ptr = nullptr, *r_col = nullptr;
    double *a_val = nullptr, *p_val = nullptr, *r_val = nullptr, *dinv = nullptr;
    double *x = nullptr, *b = nullptr, *r = nullptr;
    int n_dense = 0;             // instances whose coarsest level is this one
    int *dense_off = nullptr, *dense_size = nullptr;
    long long* dense_mat = nullptr;  // offset of each dense inverse in dense_val
    double* dense_val = nullptr;
    int fine_n = 0;              // rows of the finer union level
    int max_dense = 0;           // largest dense block
};

struct UnionDsa {
    int count = 0;
    long long n0 = 0;            // union DG rows
    // maps between the batch's concatenated DOF vectors and union rows
    long long* row_dof = nullptr;
    double* mass_sig = nullptr;
    int* row_inst = nullptr;
    // level 0: segmented BSR
    int* inst_n = nullptr;              // block size per instance
    long long* inst_row0 = nullptr;     // first union row of each instance
    long long* inst_ptr0 = nullptr;     // offset of the instance's block-row pointers in bsr_ptr
    long long* inst_blk0 = nullptr;     // offset of the instance's blocks (in blocks) in bsr_col
    long long* inst_val0 = nullptr;     // offset of the instance's block values (in doubles) in bsr_val
    long long* inst_dinv0 = nullptr;    // offset of the instance's inverse diagonal blocks in dinv
    int *bsr_ptr = nullptr, *bsr_col = nullptr;
    double *bsr_val = nullptr, *dinv = nullptr;
    std::vector<UnionLevel> levels;
    // PCG vectors and scalars
    double *x = nullptr, *b = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *vr = nullptr;
    double* part = nullptr;
    double* s = nullptr;         // [0] rz [1] pq [2] rr [3] bb [4] rz_new
    int* done = nullptr;         // 1 once the solve has converged (or b = 0); 0 in the recorded loop
    int* iters = nullptr;        // PCG iterations performed (device counter)
    int* local_iters = nullptr;  // iterations of the current solve (recorded loop)
    cudaStream_t cap2 = nullptr; // captures the loop body while the batched iteration is recorded
    double omega0 = 0.8, omega = 0.6;  // as the single-mesh V-cycle (sn_dsa.h)
    int nu = 2;
    std::vector<DsaHierarchy*> parts;  // host hierarchies (kept for their sizes)
};

namespace {

constexpr int kBS = 256;
constexpr int kParts = 304;
inline unsigned nb(long long n) { return (unsigned)std::max<long long>(1, (n + kBS - 1) / kBS); }

#define SKIP_IF_DONE \
    if (*done) return

__global__ void u_gather(const double* full, const long long* row_dof, const double* mass, long long n, double* out,
                         const int* done) {
    SKIP_IF_DONE;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = mass[i] * full[row_dof[i]];
}

__global__ void u_scatter_add(const double* x, const long long* row_dof, const int* row_inst, const int* active,
                              long long n, double* full) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !active[row_inst[i]]) return;
    full[row_dof[i]] += x[i];
}

// out = b - A x (b null: out = A x) on the segmented-BSR DG level
__global__ void u_bsr(const int* row_inst, const int* inst_n, const long long* inst_row0, const long long* inst_ptr0,
                      const long long* inst_blk0, const long long* inst_val0, const int* ptr, const int* col,
                      const double* val, long long n, const double* x, const double* b, double* out,
                      const int* done) {
    SKIP_IF_DONE;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int inst = row_inst[r];
    const int bn = inst_n[inst];
    const long long lr = r - inst_row0[inst];
    const long long t = lr / bn;
    const int i = (int)(lr % bn);
    const int* P = ptr + inst_ptr0[inst];
    const long long blk0 = inst_blk0[inst];
    const double* vals = val + inst_val0[inst];
    const double* xi = x + inst_row0[inst];
    double s = 0.0;
    for (int k = P[t]; k < P[t + 1]; ++k) {
        const double* blk = vals + (size_t)k * bn * bn + (size_t)i * bn;
        const double* xc = xi + (size_t)col[blk0 + k] * bn;
        for (int j = 0; j < bn; ++j) s += blk[j] * xc[j];
    }
    out[r] = b ? b[r] - s : s;
}

__global__ void u_block_jacobi(const int* row_inst, const int* inst_n, const long long* inst_row0,
                               const long long* inst_dinv0, const double* dinv, long long n, double omega,
                               const double* res, double* x, int accumulate, const int* done) {
    SKIP_IF_DONE;
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int inst = row_inst[r];
    const int bn = inst_n[inst];
    const long long lr = r - inst_row0[inst];
    const long long t = lr / bn;
    const int i = (int)(lr % bn);
    const double* D = dinv + inst_dinv0[inst] + (size_t)t * bn * bn + (size_t)i * bn;
    const double* rr = res + inst_row0[inst] + (size_t)t * bn;
    double s = 0.0;
    for (int j = 0; j < bn; ++j) s += D[j] * rr[j];
    x[r] = (accumulate ? x[r] : 0.0) + omega * s;
}

// CSR product with 4 lanes per row and a fixed shuffle tree (see csr_vec_kernel of the
// single-mesh DSA); mode 0: out = M x; 1: out = b - M x; 2: out += M x
__global__ void u_csr(const int* ptr, const int* col, const double* val, int rows, const double* x, const double* b,
                      double* out, int mode, const int* done) {
    SKIP_IF_DONE;
    constexpr int G = 4;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int gl = threadIdx.x & (G - 1);
    const long long r = tid / G;
    double s = 0.0;
    if (r < rows) {
        const int k1 = ptr[r + 1];
        for (int k = ptr[r] + gl; k < k1; k += G) s += val[k] * x[col[k]];
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o, G);
    if (r < rows && gl == 0) {
        if (mode == 0) out[r] = s;
        else if (mode == 1) out[r] = b[r] - s;
        else out[r] += s;
    }
}

__global__ void u_jacobi(const double* dinv, int rows, double omega, const double* res, double* x, int accumulate,
                         const int* done) {
    SKIP_IF_DONE;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows) return;
    x[i] = (accumulate ? x[i] : 0.0) + omega * dinv[i] * res[i];
}

// x[off_k + r] = sum_c A_k[r][c] b[off_k + c] for every dense block k, one warp per row
__global__ void u_dense(const int* off, const int* size, const long long* mat, const double* val, int n_dense,
                        const double* b, double* x, const int* done) {
    SKIP_IF_DONE;
    const int k = blockIdx.y;
    if (k >= n_dense) return;
    const int n = size[k];
    const int lane = threadIdx.x & 31;
    const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    double s = 0.0;
    if (r < n) {
        const double* A = val + mat[k] + (size_t)r * n;
        const double* bb = b + off[k];
        for (int c = lane; c < n; c += 32) s += A[c] * bb[c];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (r < n && lane == 0) x[off[k] + r] = s;
}

__global__ void u_dot_partial(const double* a, const double* b, long long n, double* part, const int* done) {
    SKIP_IF_DONE;
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

__global__ void u_dot_final(const double* part, int n, double* out, const int* done) {
    SKIP_IF_DONE;
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

__global__ void u_update_xr(double* x, double* r, const double* p, const double* q, long long n, const double* s,
                            const int* done) {
    SKIP_IF_DONE;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double alpha = s[0] / s[1];
    x[i] += alpha * p[i];
    r[i] -= alpha * q[i];
}

__global__ void u_update_p(double* p, const double* z, long long n, const double* s, const int* done) {
    SKIP_IF_DONE;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    p[i] = z[i] + (s[4] / s[0]) * p[i];
}

__global__ void u_start(double* s, int* done, int* iters) {
    // b = 0 (every instance converged or no residual): nothing to solve
    *iters = 0;
    *done = !(s[3] > 0.0);
}

__global__ void u_check(double* s, double tol2, int* done, int* iters) {
    SKIP_IF_DONE;
    *iters += 1;
    if (!(s[2] > tol2 * s[3])) *done = 1;
}

__global__ void u_shift(double* s, const int* done) {
    SKIP_IF_DONE;
    s[0] = s[4];
}

// Start of the recorded union PCG: s[0] = +inf makes the first search direction p = z; the loop
// body runs only when b != 0.
__global__ void u_loop_start(double* s, int* local_iters, cudaGraphConditionalHandle h) {
    s[0] = INFINITY;
    *local_iters = 0;
    cudaGraphSetConditional(h, s[3] > 0.0 ? 1u : 0u);
}

// End of one recorded union PCG iteration: continue while ||r||^2 > tol^2 ||b||^2 and fewer than
// max_iters iterations; iters accumulates the batch's PCG count.
__global__ void u_loop_check(const double* s, double tol2, int max_iters, int* local_iters, int* iters,
                             cudaGraphConditionalHandle h) {
    const int k = ++*local_iters;
    *iters += 1;
    cudaGraphSetConditional(h, (s[2] > tol2 * s[3] && k < max_iters) ? 1u : 0u);
}

template <typename T>
cudaError_t up(T** d, const std::vector<T>& h) {
    if (h.empty()) {
        *d = nullptr;
        return cudaSuccess;
    }
    cudaError_t err = cudaMalloc(d, h.size() * sizeof(T));
    if (err != cudaSuccess) return err;
    return cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void dot(UnionDsa* U, const double* a, const double* b, long long n, int slot, cudaStream_t s) {
    SN_COUNT_LAUNCH();
    u_dot_partial<<<kParts, kBS, 0, s>>>(a, b, n, U->part, U->done);
    SN_COUNT_LAUNCH();
    u_dot_final<<<1, kBS, 0, s>>>(U->part, kParts, U->s + slot, U->done);
}

void vcycle_union(UnionDsa* U, size_t l, cudaStream_t s) {
    UnionLevel& L = U->levels[l];
    const int* dn = U->done;
    for (int k = 0; k < U->nu; ++k) {
        if (k == 0) {
            SN_COUNT_LAUNCH();
            u_jacobi<<<nb(L.n), kBS, 0, s>>>(L.dinv, L.n, U->omega, L.b, L.x, 0, dn);
        } else {
            SN_COUNT_LAUNCH();
            u_csr<<<nb((long long)(L.n) * 4), kBS, 0, s>>>(L.a_ptr, L.a_col, L.a_val, L.n, L.x, L.b, L.r, 1, dn);
            SN_COUNT_LAUNCH();
            u_jacobi<<<nb(L.n), kBS, 0, s>>>(L.dinv, L.n, U->omega, L.r, L.x, 1, dn);
        }
    }
    if (l + 1 < U->levels.size()) {
        UnionLevel& C = U->levels[l + 1];
        SN_COUNT_LAUNCH();
        u_csr<<<nb((long long)(L.n) * 4), kBS, 0, s>>>(L.a_ptr, L.a_col, L.a_val, L.n, L.x, L.b, L.r, 1, dn);
        SN_COUNT_LAUNCH();
        u_csr<<<nb((long long)(C.n) * 4), kBS, 0, s>>>(C.r_ptr, C.r_col, C.r_val, C.n, L.r, nullptr, C.b, 0, dn);
        vcycle_union(U, l + 1, s);
        SN_COUNT_LAUNCH();
        u_csr<<<nb((long long)(L.n) * 4), kBS, 0, s>>>(C.p_ptr, C.p_col, C.p_val, L.n, C.x, nullptr, L.x, 2, dn);
    }
    for (int k = 0; k < U->nu; ++k) {
        SN_COUNT_LAUNCH();
        u_csr<<<nb((long long)(L.n) * 4), kBS, 0, s>>>(L.a_ptr, L.a_col, L.a_val, L.n, L.x, L.b, L.r, 1, dn);
        SN_COUNT_LAUNCH();
        u_jacobi<<<nb(L.n), kBS, 0, s>>>(L.dinv, L.n, U->omega, L.r, L.x, 1, dn);
    }
    if (L.n_dense > 0) {  // instances whose hierarchy ends here: exact coarsest solve
        SN_COUNT_LAUNCH();
        u_dense<<<dim3(nb((long long)L.max_dense * 32), L.n_dense), kBS, 0, s>>>(L.dense_off, L.dense_size, L.dense_mat, L.dense_val, L.n_dense,
                                                        L.b, L.x, dn);
    }
}

void vcycle0_union(UnionDsa* U, const double* r, double* z, cudaStream_t s) {
    const long long n = U->n0;
    const int* dn = U->done;
    for (int k = 0; k < U->nu; ++k) {
        if (k == 0) {
            SN_COUNT_LAUNCH();
            u_block_jacobi<<<nb(n), kBS, 0, s>>>(U->row_inst, U->inst_n, U->inst_row0, U->inst_dinv0, U->dinv, n, U->omega0,
                                               r, z, 0, dn);
        } else {
            SN_COUNT_LAUNCH();
            u_bsr<<<nb(n), kBS, 0, s>>>(U->row_inst, U->inst_n, U->inst_row0, U->inst_ptr0, U->inst_blk0, U->inst_val0, U->bsr_ptr,
                                       U->bsr_col, U->bsr_val, n, z, r, U->vr, dn);
            SN_COUNT_LAUNCH();
            u_block_jacobi<<<nb(n), kBS, 0, s>>>(U->row_inst, U->inst_n, U->inst_row0, U->inst_dinv0, U->dinv, n, U->omega0,
                                               U->vr, z, 1, dn);
        }
    }
    if (!U->levels.empty()) {
        UnionLevel& C = U->levels[0];
        SN_COUNT_LAUNCH();
        u_bsr<<<nb(n), kBS, 0, s>>>(U->row_inst, U->inst_n, U->inst_row0, U->inst_ptr0, U->inst_blk0, U->inst_val0, U->bsr_ptr,
                                   U->bsr_col, U->bsr_val, n, z, r, U->vr, dn);
        SN_COUNT_LAUNCH();
        u_csr<<<nb((long long)(C.n) * 4), kBS, 0, s>>>(C.r_ptr, C.r_col, C.r_val, C.n, U->vr, nullptr, C.b, 0, dn);
        vcycle_union(U, 0, s);
        SN_COUNT_LAUNCH();
        u_csr<<<nb((long long)(n) * 4), kBS, 0, s>>>(C.p_ptr, C.p_col, C.p_val, (int)n, C.x, nullptr, z, 2, dn);
    }
    for (int k = 0; k < U->nu; ++k) {
        SN_COUNT_LAUNCH();
        u_bsr<<<nb(n), kBS, 0, s>>>(U->row_inst, U->inst_n, U->inst_row0, U->inst_ptr0, U->inst_blk0, U->inst_val0, U->bsr_ptr,
                                   U->bsr_col, U->bsr_val, n, z, r, U->vr, dn);
        SN_COUNT_LAUNCH();
        u_block_jacobi<<<nb(n), kBS, 0, s>>>(U->row_inst, U->inst_n, U->inst_row0, U->inst_dinv0, U->dinv, n, U->omega0,
                                           U->vr, z, 1, dn);
    }
}

}  // namespace

// Builds the union hierarchy from the instances' own (host) hierarchies.
UnionDsa* union_dsa_build(const std::vector<DsaHierarchy*>& parts, const std::vector<long long>& dof_off,
                          std::string& err) {
    auto* U = new UnionDsa();
    U->parts = parts;
    const int n_inst = (int)parts.size();
    U->count = n_inst;
    std::vector<long long> row_dof, inst_row0(n_inst), inst_ptr0(n_inst), inst_blk0(n_inst), inst_val0(n_inst),
        inst_dinv0(n_inst);
    std::vector<int> row_inst, inst_n(n_inst), bsr_ptr, bsr_col;
    std::vector<double> mass, bsr_val, dinv;
    for (int i = 0; i < n_inst; ++i) {
        const DsaHierarchy* H = parts[i];
        inst_n[i] = std::max(H->n, 1);
        inst_row0[i] = (long long)row_dof.size();
        inst_ptr0[i] = (long long)bsr_ptr.size();
        inst_blk0[i] = (long long)bsr_col.size();
        inst_val0[i] = (long long)bsr_val.size();
        inst_dinv0[i] = (long long)dinv.size();
        for (int t = 0; t < H->nt; ++t)
            for (int a = 0; a < H->n; ++a) {
                row_dof.push_back(dof_off[i] + (long long)H->thick[t] * H->n + a);
                row_inst.push_back(i);
                mass.push_back(H->h_mass_sig[(size_t)t * H->n + a]);
            }
        if (H->nt > 0) {
            bsr_ptr.insert(bsr_ptr.end(), H->l0.ptr.begin(), H->l0.ptr.end());
            bsr_col.insert(bsr_col.end(), H->l0.col.begin(), H->l0.col.end());
            bsr_val.insert(bsr_val.end(), H->l0.val.begin(), H->l0.val.end());
            dinv.insert(dinv.end(), H->l0.dinv.begin(), H->l0.dinv.end());
        } else {
            bsr_ptr.push_back(0);
        }
    }
    U->n0 = (long long)row_dof.size();
    // continuous levels: union over instances of their level l
    size_t max_depth = 0;
    for (DsaHierarchy* H : parts) max_depth = std::max(max_depth, H->levels.size());
    std::vector<std::vector<long long>> lvl_off(max_depth + 1, std::vector<long long>(n_inst, -1));
    for (int i = 0; i < n_inst; ++i) lvl_off[0][i] = inst_row0[i];  // level 0 offsets
    cudaError_t cerr;
#define UP(dst, src)                                           \
    if ((cerr = up(&(dst), src)) != cudaSuccess) {             \
        err = cudaGetErrorString(cerr);                        \
        return U;                                              \
    }
    for (size_t l = 0; l < max_depth; ++l) {
        UnionLevel L;
        std::vector<int> a_ptr{0}, a_col, p_ptr{0}, p_col, r_ptr{0}, r_col, doff, dsize;
        std::vector<double> a_val, p_val, r_val, dv, dval;
        std::vector<long long> dmat;
        long long rows = 0;
        for (int i = 0; i < n_inst; ++i) {
            const DsaHierarchy* H = parts[i];
            if (l >= H->levels.size()) continue;
            const LevelC& C = H->levels[l];
            lvl_off[l + 1][i] = rows;
            const bool coarsest = !C.dense_inv.empty();
            for (int r = 0; r < C.n; ++r) {
                if (!coarsest) {
                    for (int k = C.a_ptr[r]; k < C.a_ptr[r + 1]; ++k) {
                        a_col.push_back((int)(rows + C.a_col[k]));
                        a_val.push_back(C.a_val[k]);
                    }
                    dv.push_back(C.dinv[r]);
                } else {
                    dv.push_back(0.0);  // exact dense solve instead of smoothing
                }
                a_ptr.push_back((int)a_col.size());
                for (int k = C.r_ptr[r]; k < C.r_ptr[r + 1]; ++k) {  // restriction from the finer level
                    r_col.push_back((int)(lvl_off[l][i] + C.r_col[k]));
                    r_val.push_back(C.r_val[k]);
                }
                r_ptr.push_back((int)r_col.size());
            }
            if (coarsest) {
                doff.push_back((int)rows);
                dsize.push_back(C.n);
                dmat.push_back((long long)dval.size());
                dval.insert(dval.end(), C.dense_inv.begin(), C.dense_inv.end());
            }
            rows += C.n;
        }
        // prolongation: rows of the finer union level (all instances present there), columns here
        const long long fine_rows = l == 0 ? U->n0 : (long long)U->levels[l - 1].n;
        std::vector<std::vector<std::pair<int, double>>> prow(fine_rows);
        for (int i = 0; i < n_inst; ++i) {
            const DsaHierarchy* H = parts[i];
            if (l >= H->levels.size()) continue;
            const LevelC& C = H->levels[l];
            const long long fo = lvl_off[l][i];
            for (size_t r = 0; r + 1 < C.p_ptr.size(); ++r)
                for (int k = C.p_ptr[r]; k < C.p_ptr[r + 1]; ++k)
                    prow[fo + r].push_back({(int)(lvl_off[l + 1][i] + C.p_col[k]), C.p_val[k]});
        }
        for (long long r = 0; r < fine_rows; ++r) {
            for (auto& pr : prow[r]) {
                p_col.push_back(pr.first);
                p_val.push_back(pr.second);
            }
            p_ptr.push_back((int)p_col.size());
        }
        L.n = (int)rows;
        L.fine_n = (int)fine_rows;
        L.n_dense = (int)doff.size();
        for (int sz : dsize) L.max_dense = std::max(L.max_dense, sz);
        UP(L.a_ptr, a_ptr);
        UP(L.a_col, a_col);
        UP(L.a_val, a_val);
        UP(L.p_ptr, p_ptr);
        UP(L.p_col, p_col);
        UP(L.p_val, p_val);
        UP(L.r_ptr, r_ptr);
        UP(L.r_col, r_col);
        UP(L.r_val, r_val);
        UP(L.dinv, dv);
        UP(L.dense_off, doff);
        UP(L.dense_size, dsize);
        UP(L.dense_mat, dmat);
        UP(L.dense_val, dval);
        for (double** v : {&L.x, &L.b, &L.r})
            if ((cerr = cudaMalloc(v, std::max(1, L.n) * sizeof(double))) != cudaSuccess) {
                err = cudaGetErrorString(cerr);
                return U;
            }
        U->levels.push_back(L);
    }
    UP(U->row_dof, row_dof);
    UP(U->mass_sig, mass);
    UP(U->row_inst, row_inst);
    UP(U->inst_n, inst_n);
    UP(U->inst_row0, inst_row0);
    UP(U->inst_ptr0, inst_ptr0);
    UP(U->inst_blk0, inst_blk0);
    UP(U->inst_val0, inst_val0);
    UP(U->inst_dinv0, inst_dinv0);
    UP(U->bsr_ptr, bsr_ptr);
    UP(U->bsr_col, bsr_col);
    UP(U->bsr_val, bsr_val);
    UP(U->dinv, dinv);
#undef UP
    const long long n0 = std::max<long long>(1, U->n0);
    for (double** v : {&U->x, &U->b, &U->r, &U->z, &U->p, &U->q, &U->vr})
        if ((cerr = cudaMalloc(v, n0 * sizeof(double))) != cudaSuccess) {
            err = cudaGetErrorString(cerr);
            return U;
        }
    if ((cerr = cudaMalloc(&U->part, kParts * sizeof(double))) != cudaSuccess ||
        (cerr = cudaMalloc(&U->s, 8 * sizeof(double))) != cudaSuccess ||
        (cerr = cudaMalloc(&U->done, sizeof(int))) != cudaSuccess ||
        (cerr = cudaMalloc(&U->local_iters, sizeof(int))) != cudaSuccess ||
        (cerr = cudaMalloc(&U->iters, sizeof(int))) != cudaSuccess) {
        err = cudaGetErrorString(cerr);
        return U;
    }
    cudaMemset(U->iters, 0, sizeof(int));
    return U;
}

void union_dsa_free(UnionDsa* U) {
    if (!U) return;
    auto f = [](void* p) {
        if (p) cudaFree(p);
    };
    for (UnionLevel& L : U->levels) {
        for (void* p : {(void*)L.a_ptr, (void*)L.a_col, (void*)L.a_val, (void*)L.p_ptr, (void*)L.p_col, (void*)L.p_val,
                        (void*)L.r_ptr, (void*)L.r_col, (void*)L.r_val, (void*)L.dinv, (void*)L.x, (void*)L.b,
                        (void*)L.r, (void*)L.dense_off, (void*)L.dense_size, (void*)L.dense_mat, (void*)L.dense_val})
            f(p);
    }
    for (void* p : {(void*)U->row_dof, (void*)U->mass_sig, (void*)U->row_inst, (void*)U->inst_n, (void*)U->inst_row0,
                    (void*)U->inst_ptr0, (void*)U->inst_blk0, (void*)U->inst_val0, (void*)U->inst_dinv0, (void*)U->bsr_ptr, (void*)U->bsr_col,
                    (void*)U->bsr_val, (void*)U->dinv, (void*)U->x, (void*)U->b, (void*)U->r, (void*)U->z, (void*)U->p,
                    (void*)U->q, (void*)U->vr, (void*)U->part, (void*)U->s, (void*)U->done, (void*)U->iters,
                    (void*)U->local_iters})
        f(p);
    if (U->cap2) cudaStreamDestroy(U->cap2);
    for (DsaHierarchy* H : U->parts) dsa_free(H);
    delete U;
}

long long union_dsa_rows(const UnionDsa* U) { return U ? U->n0 : 0; }
int* union_dsa_iters(UnionDsa* U) { return U->iters; }

// phi_all[thick rows] += D_ff^{-1} Sigma_f r_all (union of Algorithm 2 over active instances).
// Called while the batched iteration is being recorded: the PCG loop becomes a WHILE conditional
// node whose body is one iteration (z = V(r); rz; p = z + (rz / rz_prev) p; q = A p; x, r update;
// r.r; device-side test), so a converged solve launches nothing more.
cudaError_t union_dsa_correct(UnionDsa* U, const double* r_all, double* phi_all, const int* active, double tol,
                              int max_iters, cudaStream_t s) {
    if (U->n0 == 0) return cudaSuccess;
    const long long n = U->n0;
    cudaError_t err;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    if ((err = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr)) != cudaSuccess) return err;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureUnsupported;
    if (!U->cap2 && (err = cudaStreamCreateWithFlags(&U->cap2, cudaStreamNonBlocking)) != cudaSuccess) return err;
    cudaGraphConditionalHandle h;
    if ((err = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return err;
    cudaMemsetAsync(U->done, 0, sizeof(int), s);  // the loop's kernels never skip
    SN_COUNT_LAUNCH();
    u_gather<<<nb(n), kBS, 0, s>>>(r_all, U->row_dof, U->mass_sig, n, U->b, U->done);
    cudaMemsetAsync(U->x, 0, n * sizeof(double), s);
    cudaMemsetAsync(U->p, 0, n * sizeof(double), s);
    cudaMemcpyAsync(U->r, U->b, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
    dot(U, U->b, U->b, n, 3, s);
    SN_COUNT_LAUNCH();
    u_loop_start<<<1, 1, 0, s>>>(U->s, U->local_iters, h);
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    if ((err = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &ndeps)) != cudaSuccess) return err;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t loop;
    if ((err = cudaGraphAddNode(&loop, g, deps, nullptr, ndeps, &cp)) != cudaSuccess) return err;
    if ((err = cudaStreamUpdateCaptureDependencies(s, &loop, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return err;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaStream_t b = U->cap2;
    if ((err = cudaStreamBeginCaptureToGraph(b, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return err;
    vcycle0_union(U, U->r, U->z, b);
    dot(U, U->r, U->z, n, 4, b);
    SN_COUNT_LAUNCH();
    u_update_p<<<nb(n), kBS, 0, b>>>(U->p, U->z, n, U->s, U->done);
    SN_COUNT_LAUNCH();
    u_shift<<<1, 1, 0, b>>>(U->s, U->done);
    SN_COUNT_LAUNCH();
    u_bsr<<<nb(n), kBS, 0, b>>>(U->row_inst, U->inst_n, U->inst_row0, U->inst_ptr0, U->inst_blk0, U->inst_val0, U->bsr_ptr,
                               U->bsr_col, U->bsr_val, n, U->p, nullptr, U->q, U->done);
    dot(U, U->p, U->q, n, 1, b);
    SN_COUNT_LAUNCH();
    u_update_xr<<<nb(n), kBS, 0, b>>>(U->x, U->r, U->p, U->q, n, U->s, U->done);
    dot(U, U->r, U->r, n, 2, b);
    SN_COUNT_LAUNCH();
    u_loop_check<<<1, 1, 0, b>>>(U->s, tol * tol, max_iters, U->local_iters, U->iters, h);
    cudaError_t lerr = cudaGetLastError();
    cudaGraph_t b2 = nullptr;
    err = cudaStreamEndCapture(b, &b2);
    if (lerr != cudaSuccess) return lerr;
    if (err != cudaSuccess) return err;
    SN_COUNT_LAUNCH();
    u_scatter_add<<<nb(n), kBS, 0, s>>>(U->x, U->row_dof, U->row_inst, active, n, phi_all);
    return cudaGetLastError();
}

}  // namespace sn

// ---------------------------------------------------------------- batched source iteration
namespace sn {
namespace {

__global__ void b_residual(const double* half, const double* phi, double* r, const int* dof_inst, const int* active,
                           long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    r[i] = active[dof_inst[i]] ? half[i] - phi[i] : 0.0;
}

__global__ void b_update(double* phi, const double* half, const int* dof_inst, const int* active, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !active[dof_inst[i]]) return;
    phi[i] = half[i];
}

// per instance: relative residual, iteration count, and whether the next iteration runs
__global__ void b_check(const double* rr, double* r0, double* rel, int* iters, const int* active, int* next, int count,
                        double tol, int max_iters) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    if (!active[i]) {
        next[i] = 0;
        return;
    }
    const double rn = sqrt(rr[i]);
    if (iters[i] == 0) r0[i] = rn > 0.0 ? rn : 1.0;
    rel[i] = rn / r0[i];
    iters[i] += 1;
    next[i] = !(rel[i] <= tol) && iters[i] < max_iters;
}

__global__ void b_advance(int* active, const int* next, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) active[i] = next[i];
}

inline unsigned nbl(long long n) { return (unsigned)std::max<long long>(1, (n + 255) / 256); }

}  // namespace

struct BatchIterState {
    int* d_next = nullptr;
    int* d_dof_inst = nullptr;
};

// One outer iteration of every active instance (Eq. DSA_fp with Algorithm 2), capturable.
cudaError_t batch_enqueue_iteration(sn_batch* b, const sn_iter_opts* o, int* d_next, const int* d_dof_inst,
                                    cudaStream_t s) {
    cudaError_t err = dataflow_like(b->schedule) ? batch_launch_dataflow(b, o->precision, s)
                                                    : batch_enqueue_sweep(b, o->precision, s);
    if (err != cudaSuccess) return err;
    for (int i = 0; i < b->count; ++i) {
        const long long off = b->dof_off[i];
        if ((err = launch_phi_reduce(b->meshes[i], o->precision, b->d_phi + off, b->d_half + off, b->d_rr + i, s)) !=
            cudaSuccess)
            return err;
    }
    SN_COUNT_LAUNCH();
    b_check<<<nbl(b->count), 256, 0, s>>>(b->d_rr, b->d_r0, b->d_rel, b->d_iters, b->d_active, d_next, b->count, o->tol,
                                          o->max_iters);
    SN_COUNT_LAUNCH();
    b_residual<<<nbl(b->n_dof), 256, 0, s>>>(b->d_half, b->d_phi, b->d_r, d_dof_inst, b->d_active, b->n_dof);
    SN_COUNT_LAUNCH();
    b_update<<<nbl(b->n_dof), 256, 0, s>>>(b->d_phi, b->d_half, d_dof_inst, b->d_active, b->n_dof);
    if (o->dsa != SN_DSA_NONE && b->dsa)
        if ((err = union_dsa_correct(b->dsa, b->d_r, b->d_phi, b->d_active, o->inner_tol, o->inner_max_iters, s)) !=
            cudaSuccess)
            return err;
    SN_COUNT_LAUNCH();
    b_advance<<<nbl(b->count), 256, 0, s>>>(b->d_active, d_next, b->count);
    return cudaGetLastError();
}

}  // namespace sn
