// Flexible GMRES(k) over every instance of a batch at once (Eq. schur solved per instance, right-
// preconditioned by the thick-subdomain DSA step of Algorithm 2).
//
// Each instance keeps its own Krylov basis, Hessenberg matrix and Givens rotations; the instances
// advance in lock step, one Arnoldi step of all of them per graph launch:
//   - one batched homogeneous sweep of the extending instances (their own quadratures and meshes),
//   - the union DSA step (one CG on the block-diagonal union system, as in the batched source
//     iteration), applied to the instances' current basis vectors,
//   - classical Gram-Schmidt twice with inner products segmented by instance (every instance's
//     vector is cut into fixed chunks, and each instance's chunk sums are added in chunk order, so
//     an instance's arithmetic does not depend on the rest of the batch),
//   - the Givens update of every instance's least-squares problem on the device.
// An instance stops extending its basis when its residual estimate reaches the tolerance (or its
// iteration budget); a restart recomputes every active instance's true residual with the fixed
// source, and an instance whose true residual is below the tolerance leaves the batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <vector>

#include "sn_dsa.h"

namespace sn {

namespace {

constexpr int kT = 256;
constexpr long long kChunk = 4096;  // DOFs of one inner-product chunk (never spans two instances)

// Offsets of one instance's float64 state (per-instance stride sd).
struct Lay {
    int k, H, cs, sn, g, y, h1, h2, hn, beta, r0, rel, hnext, sd;
};

Lay make_lay(int k) {
    Lay L;
    L.k = k;
    L.H = 0;                        // (k+1) x k, column j at H + j (k+1)
    L.cs = L.H + (k + 1) * k;
    L.sn = L.cs + k;
    L.g = L.sn + k;                 // k + 1
    L.y = L.g + k + 1;              // k
    L.h1 = L.y + k;                 // first Gram-Schmidt pass, k + 1
    L.h2 = L.h1 + k + 1;            // second pass, k + 1
    L.hn = L.h2 + k + 1;            // squared norm
    L.beta = L.hn + 1;
    L.r0 = L.beta + 1;
    L.rel = L.r0 + 1;
    L.hnext = L.rel + 1;
    L.sd = L.hnext + 1;
    return L;
}

inline unsigned nbk(long long n) { return (unsigned)std::max<long long>(1, (n + kT - 1) / kT); }

// Sum over the block in a fixed order (warp shuffles, then the warps' sums in warp order); the
// result is valid in thread 0.
__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
    __syncthreads();
    return t;
}

// part[c * ld + v] = V_v . w over chunk c, v < nv (nv = *jdev + 1 when jdev is set, else nv_fixed);
// chunks of masked-off instances are skipped.
__global__ void bk_dot_partial(const double* V, long long n, const double* w, int nv_fixed, const int* jdev,
                               const int* cinst, const long long* clo, const long long* chi, const int* mask,
                               double* part, int ld) {
    __shared__ double sh[kT / 32];
    const int c = blockIdx.x;
    if (!mask[cinst[c]]) return;
    const int nv = jdev ? *jdev + 1 : nv_fixed;
    const long long lo = clo[c], hi = chi[c];
    for (int v = 0; v < nv; ++v) {
        const double* x = V + (size_t)v * n;
        double s = 0.0;
        for (long long t = lo + threadIdx.x; t < hi; t += blockDim.x) s += x[t] * w[t];
        s = block_sum(s, sh);
        if (threadIdx.x == 0) part[(size_t)c * ld + v] = s;
    }
}

// st[inst * sd + off + v] = sum of the instance's chunks in chunk order (one block per instance)
__global__ void bk_dot_final(const double* part, int ld, const int* c0, const int* c1, int nv_fixed, const int* jdev,
                             const int* mask, double* st, int sd, int off) {
    const int inst = blockIdx.x;
    if (!mask[inst]) return;
    const int nv = jdev ? *jdev + 1 : nv_fixed;
    const int v = threadIdx.x;
    if (v >= nv) return;
    double s = 0.0;
    for (int c = c0[inst]; c < c1[inst]; ++c) s += part[(size_t)c * ld + v];
    st[(size_t)inst * sd + off + v] = s;
}

// w += sign * sum_{v < nv} c_v V_v on the masked instances' DOFs, c_v = st[inst * sd + off + v];
// nv = *jdev + 1, or nv_inst[inst], or nv_fixed
__global__ void bk_axpy(const double* V, long long n, int nv_fixed, const int* jdev, const int* nv_inst,
                        const int* dof_inst, const int* mask, const double* st, int sd, int off, double sign,
                        double* w) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int inst = dof_inst[t];
    if (!mask[inst]) return;
    const int nv = jdev ? *jdev + 1 : (nv_inst ? nv_inst[inst] : nv_fixed);
    const double* c = st + (size_t)inst * sd + off;
    double s = 0.0;
    for (int v = 0; v < nv; ++v) s += c[v] * V[(size_t)v * n + t];
    w[t] += sign * s;
}

// true residual of the fixed-point form: w = (sweep of x with the fixed source) - x
__global__ void bk_residual(const double* tmp, const double* x, long long n, const int* dof_inst, const int* act,
                            double* w) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    w[t] = act[dof_inst[t]] ? tmp[t] - x[t] : 0.0;
}

// w = S z_j = z_j - T z_j and Z_j = z_j on the extending instances (zero elsewhere)
__global__ void bk_apply(const double* zj, const double* tmp, long long n, const int* jdev, const int* dof_inst,
                         const int* ext, double* w, double* Z) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const bool e = ext[dof_inst[t]] != 0;
    const double z = e ? zj[t] : 0.0;
    w[t] = e ? z - tmp[t] : 0.0;
    Z[(size_t)(*jdev) * n + t] = z;
}

// V_j = vj = w / st[inst * sd + off] on the extending instances (zero elsewhere), j = *jdev
__global__ void bk_normalize(const double* w, long long n, const int* jdev, const int* dof_inst, const int* ext,
                             const double* st, int sd, int off, double* V, double* vj) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int inst = dof_inst[t];
    const double v = ext[inst] ? w[t] / st[(size_t)inst * sd + off] : 0.0;
    V[(size_t)(*jdev) * n + t] = v;
    vj[t] = v;
}

// Start of a cycle (one block): beta = ||w|| per active instance, convergence on the true residual,
// g = beta e_1 for the instances that iterate; flags = (j = 0, any active, any extending).
__global__ void bk_cycle_start(int count, Lay L, double* st, int* act, int* ext, int* jj, const int* it, int* conv,
                               int* cyc, int* flags, double tol, int max_iters) {
    int any = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        ext[i] = 0;
        jj[i] = 0;
        if (!act[i]) continue;
        double* d = st + (size_t)i * L.sd;
        const double beta = sqrt(fmax(d[L.hn], 0.0));
        if (d[L.r0] == 0.0) d[L.r0] = beta > 0.0 ? beta : 1.0;
        const double rel = beta / d[L.r0];
        d[L.rel] = rel;
        d[L.beta] = beta;
        if (rel <= tol || beta == 0.0) {  // convergence is declared on the true residual only
            act[i] = 0;
            conv[i] = 1;
            continue;
        }
        if (it[i] >= max_iters) {
            act[i] = 0;
            continue;
        }
        ext[i] = 1;
        cyc[i] += 1;
        d[L.g] = beta;
        for (int r = 1; r <= L.k; ++r) d[L.g + r] = 0.0;
        any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        flags[0] = 0;
        flags[1] = any;
        flags[2] = any;
    }
}

// Arnoldi step j of every extending instance (one block): column j of H from the two Gram-Schmidt
// passes, the previous rotations applied, a new rotation that zeroes H(j+1, j), the residual
// estimate |g_{j+1}|; flags[0] = j + 1, flags[2] = any instance still extending.
__global__ void bk_givens(int count, Lay L, double* st, int* ext, int* jj, int* it, int* flags, double tol,
                          int max_iters) {
    const int j = flags[0];
    const int k = L.k;
    int any = 0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        if (!ext[i]) continue;
        double* d = st + (size_t)i * L.sd;
        double* h = d + L.H + (size_t)j * (k + 1);
        for (int r = 0; r <= j; ++r) h[r] = d[L.h1 + r] + d[L.h2 + r];
        const double hnext = sqrt(fmax(d[L.hn], 0.0));
        h[j + 1] = hnext;
        d[L.hnext] = hnext;
        for (int r = 0; r < j; ++r) {
            const double c = d[L.cs + r], s = d[L.sn + r];
            const double a = c * h[r] + s * h[r + 1];
            h[r + 1] = -s * h[r] + c * h[r + 1];
            h[r] = a;
        }
        const double rho = hypot(h[j], h[j + 1]);
        const double c = rho > 0.0 ? h[j] / rho : 1.0, s = rho > 0.0 ? h[j + 1] / rho : 0.0;
        d[L.cs + j] = c;
        d[L.sn + j] = s;
        h[j] = rho;
        h[j + 1] = 0.0;
        d[L.g + j + 1] = -s * d[L.g + j];
        d[L.g + j] = c * d[L.g + j];
        it[i] += 1;
        jj[i] = j + 1;
        const double rel = fabs(d[L.g + j + 1]) / d[L.r0];
        d[L.rel] = rel;
        if (rel <= tol || hnext <= 1e-300 || it[i] >= max_iters || j + 1 >= k) ext[i] = 0;
        else any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        flags[0] = j + 1;
        flags[2] = any;
    }
}

// y = H^{-1} g (upper triangular, jj x jj) per instance
__global__ void bk_solve(int count, Lay L, double* st, const int* jj) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    double* d = st + (size_t)i * L.sd;
    const int n = jj[i];
    for (int r = n - 1; r >= 0; --r) {
        double t = d[L.g + r];
        for (int c = r + 1; c < n; ++c) t -= d[L.H + (size_t)c * (L.k + 1) + r] * d[L.y + c];
        d[L.y + r] = t / d[L.H + (size_t)r * (L.k + 1) + r];
    }
}

}  // namespace

struct BatchKrylov {
    int k = 0, count = 0, n_chunks = 0;
    long long n = 0;
    Lay L{};
    double *V = nullptr, *Z = nullptr, *w = nullptr, *vj = nullptr, *zj = nullptr, *part = nullptr, *st = nullptr;
    int *ints = nullptr, *act = nullptr, *ext = nullptr, *jj = nullptr, *it = nullptr, *conv = nullptr, *cyc = nullptr;
    int* flags = nullptr;                 // [0] j, [1] any active, [2] any extending
    int *cinst = nullptr, *c0 = nullptr, *c1 = nullptr;
    long long *clo = nullptr, *chi = nullptr;
    SweepArgs* args_h = nullptr;          // homogeneous sweep table: phi = zj, no fixed source, vacuum inflow
    cudaGraphExec_t g_res = nullptr, g_step = nullptr, g_fin = nullptr;
    std::vector<double> key;
    long long gen = -1;
};

void batch_krylov_free(BatchKrylov* K) {
    if (!K) return;
    for (cudaGraphExec_t g : {K->g_res, K->g_step, K->g_fin})
        if (g) cudaGraphExecDestroy(g);
    for (void* p : {(void*)K->V, (void*)K->part, (void*)K->st, (void*)K->ints, (void*)K->cinst, (void*)K->c0,
                    (void*)K->c1, (void*)K->clo, (void*)K->chi, (void*)K->args_h})
        if (p) cudaFree(p);
    delete K;
}

static cudaError_t ensure_workspace(sn_batch* b, int k) {
    if (b->kry && b->kry->k >= k) return cudaSuccess;
    if (b->kry) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return e;
        batch_krylov_free(b->kry);
        b->kry = nullptr;
    }
    BatchKrylov* K = new BatchKrylov();
    K->k = k;
    K->count = b->count;
    K->n = b->n_dof;
    K->L = make_lay(k);
    std::vector<int> cinst, c0(b->count), c1(b->count);
    std::vector<long long> clo, chi;
    for (int i = 0; i < b->count; ++i) {
        const long long lo = b->dof_off[i], hi = lo + (long long)b->meshes[i]->ne * b->meshes[i]->n;
        c0[i] = (int)cinst.size();
        for (long long a = lo; a < hi; a += kChunk) {
            cinst.push_back(i);
            clo.push_back(a);
            chi.push_back(std::min(hi, a + kChunk));
        }
        c1[i] = (int)cinst.size();
    }
    K->n_chunks = (int)cinst.size();
    const long long n = K->n;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    chk(cudaMalloc(&K->V, (size_t)(2 * k + 4) * n * sizeof(double)));
    chk(cudaMalloc(&K->part, (size_t)std::max(1, K->n_chunks) * (k + 1) * sizeof(double)));
    chk(cudaMalloc(&K->st, (size_t)b->count * K->L.sd * sizeof(double)));
    chk(cudaMalloc(&K->ints, (size_t)(6 * b->count + 4) * sizeof(int)));
    chk(cudaMalloc(&K->cinst, std::max<size_t>(1, cinst.size()) * sizeof(int)));
    chk(cudaMalloc(&K->clo, std::max<size_t>(1, clo.size()) * sizeof(long long)));
    chk(cudaMalloc(&K->chi, std::max<size_t>(1, chi.size()) * sizeof(long long)));
    chk(cudaMalloc(&K->c0, b->count * sizeof(int)));
    chk(cudaMalloc(&K->c1, b->count * sizeof(int)));
    chk(cudaMalloc(&K->args_h, b->count * sizeof(SweepArgs)));
    if (e == cudaSuccess) {
        chk(cudaMemcpy(K->cinst, cinst.data(), cinst.size() * sizeof(int), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(K->clo, clo.data(), clo.size() * sizeof(long long), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(K->chi, chi.data(), chi.size() * sizeof(long long), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(K->c0, c0.data(), c0.size() * sizeof(int), cudaMemcpyHostToDevice));
        chk(cudaMemcpy(K->c1, c1.data(), c1.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
    if (e != cudaSuccess) {
        batch_krylov_free(K);
        return e;
    }
    K->Z = K->V + (size_t)(k + 1) * n;
    K->w = K->Z + (size_t)k * n;
    K->vj = K->w + n;
    K->zj = K->vj + n;
    const int c = b->count;
    K->act = K->ints;
    K->ext = K->act + c;
    K->jj = K->ext + c;
    K->it = K->jj + c;
    K->conv = K->it + c;
    K->cyc = K->conv + c;
    K->flags = K->cyc + c;
    b->kry = K;
    return cudaSuccess;
}

// Transport update of every masked instance into tmp (instance blocks at dof_off).
static cudaError_t batch_update(sn_batch* b, int precision, const SweepArgs* args, const int* mask, double* tmp,
                                cudaStream_t s) {
    cudaError_t e = dataflow_like(b->schedule) ? batch_launch_dataflow(b, precision, s, args, mask)
                                                : batch_enqueue_sweep(b, precision, s, args, mask);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < b->count; ++i)
        if ((e = launch_phi_reduce(b->meshes[i], precision, nullptr, tmp + b->dof_off[i], nullptr, s)) != cudaSuccess)
            return e;
    return cudaSuccess;
}

// Segmented inner products st[.. off + v] = V_v . w per masked instance.
static void seg_dots(BatchKrylov* K, const double* V, const double* w, int nv_fixed, const int* jdev, const int* mask,
                     int off, cudaStream_t s) {
    const int ld = K->k + 1;
    SN_COUNT_LAUNCH();
    bk_dot_partial<<<std::max(1, K->n_chunks), kT, 0, s>>>(V, K->n, w, nv_fixed, jdev, K->cinst, K->clo, K->chi, mask,
                                                           K->part, ld);
    SN_COUNT_LAUNCH();
    bk_dot_final<<<K->count, 64, 0, s>>>(K->part, ld, K->c0, K->c1, nv_fixed, jdev, mask, K->st, K->L.sd, off);
}

static cudaError_t capture(cudaStream_t cs, cudaGraphExec_t* out, const std::function<cudaError_t()>& body) {
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    cudaError_t q = body();
    if (q == cudaSuccess) q = cudaGetLastError();
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    if (q != cudaSuccess) e = q;
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) *out = nullptr;
    return e;
}

static cudaError_t record(sn_batch* b, const sn_iter_opts* o, cudaStream_t cs) {
    BatchKrylov* K = b->kry;
    for (cudaGraphExec_t* g : {&K->g_res, &K->g_step, &K->g_fin})
        if (*g) {
            cudaGraphExecDestroy(*g);
            *g = nullptr;
        }
    const Lay L = K->L;
    const long long n = K->n;
    const int prec = o->precision;
    double* x = b->d_phi;
    double* tmp = b->d_half;
    const int* dinst = b->d_dof_inst;
    cudaError_t e = capture(cs, &K->g_res, [&]() -> cudaError_t {
        cudaError_t r = batch_update(b, prec, b->d_args, K->act, tmp, cs);
        if (r != cudaSuccess) return r;
        SN_COUNT_LAUNCH();
        bk_residual<<<nbk(n), kT, 0, cs>>>(tmp, x, n, dinst, K->act, K->w);
        seg_dots(K, K->w, K->w, 1, nullptr, K->act, L.hn, cs);
        SN_COUNT_LAUNCH();
        bk_cycle_start<<<1, kT, 0, cs>>>(K->count, L, K->st, K->act, K->ext, K->jj, K->it, K->conv, K->cyc, K->flags,
                                         o->tol, o->max_iters);
        SN_COUNT_LAUNCH();
        bk_normalize<<<nbk(n), kT, 0, cs>>>(K->w, n, K->flags, dinst, K->ext, K->st, L.sd, L.beta, K->V, K->vj);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    e = capture(cs, &K->g_step, [&]() -> cudaError_t {
        cudaError_t r = cudaMemcpyAsync(K->zj, K->vj, n * sizeof(double), cudaMemcpyDeviceToDevice, cs);
        if (r != cudaSuccess) return r;
        if (o->dsa != SN_DSA_NONE && b->dsa &&
            (r = union_dsa_correct(b->dsa, K->vj, K->zj, K->ext, o->inner_tol, o->inner_max_iters, cs)) != cudaSuccess)
            return r;
        if ((r = batch_update(b, prec, K->args_h, K->ext, tmp, cs)) != cudaSuccess) return r;
        SN_COUNT_LAUNCH();
        bk_apply<<<nbk(n), kT, 0, cs>>>(K->zj, tmp, n, K->flags, dinst, K->ext, K->w, K->Z);
        seg_dots(K, K->V, K->w, 0, K->flags, K->ext, L.h1, cs);
        SN_COUNT_LAUNCH();
        bk_axpy<<<nbk(n), kT, 0, cs>>>(K->V, n, 0, K->flags, nullptr, dinst, K->ext, K->st, L.sd, L.h1, -1.0, K->w);
        seg_dots(K, K->V, K->w, 0, K->flags, K->ext, L.h2, cs);
        SN_COUNT_LAUNCH();
        bk_axpy<<<nbk(n), kT, 0, cs>>>(K->V, n, 0, K->flags, nullptr, dinst, K->ext, K->st, L.sd, L.h2, -1.0, K->w);
        seg_dots(K, K->w, K->w, 1, nullptr, K->ext, L.hn, cs);
        SN_COUNT_LAUNCH();
        bk_givens<<<1, kT, 0, cs>>>(K->count, L, K->st, K->ext, K->jj, K->it, K->flags, o->tol, o->max_iters);
        SN_COUNT_LAUNCH();
        bk_normalize<<<nbk(n), kT, 0, cs>>>(K->w, n, K->flags, dinst, K->ext, K->st, L.sd, L.hnext, K->V, K->vj);
        return cudaSuccess;
    });
    if (e != cudaSuccess) return e;
    return capture(cs, &K->g_fin, [&]() -> cudaError_t {
        SN_COUNT_LAUNCH();
        bk_solve<<<nbk(K->count), kT, 0, cs>>>(K->count, L, K->st, K->jj);
        SN_COUNT_LAUNCH();
        bk_axpy<<<nbk(n), kT, 0, cs>>>(K->Z, n, 0, nullptr, K->jj, dinst, K->act, K->st, L.sd, L.y, 1.0, x);
        return cudaSuccess;
    });
}

// Runs the batched fGMRES from the iterates in b->d_phi.  iters / rel / sweeps / conv receive each
// instance's Arnoldi steps, last relative residual, transport updates and convergence flag.
cudaError_t batch_fgmres(sn_batch* b, const sn_iter_opts* o, cudaStream_t s, std::vector<int>& iters,
                         std::vector<double>& rel, std::vector<int>& sweeps, std::vector<int>& conv) {
    cudaError_t e = ensure_workspace(b, o->restart);
    if (e != cudaSuccess) return e;
    BatchKrylov* K = b->kry;
    // the argument tables are switched to this precision before anything is recorded or copied
    if ((e = batch_set_precision(b, o->precision, s)) != cudaSuccess) return e;
    std::vector<SweepArgs> hom(b->h_args);
    for (int i = 0; i < b->count; ++i) {
        hom[i].phi = K->zj + b->dof_off[i];
        hom[i].q_scale = 0.0;
        hom[i].q = nullptr;
        hom[i].q32 = nullptr;
        hom[i].psi_inc = 0.0;  // the linear part of the update has vacuum inflow
    }
    if ((e = cudaMemcpyAsync(K->args_h, hom.data(), b->count * sizeof(SweepArgs), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(K->st, 0, (size_t)b->count * K->L.sd * sizeof(double), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(K->ints, 0, (size_t)(6 * b->count + 4) * sizeof(int), s)) != cudaSuccess) return e;
    std::vector<int> ones(b->count, 1);
    if ((e = cudaMemcpyAsync(K->act, ones.data(), b->count * sizeof(int), cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return e;
    const std::vector<double> key = {(double)o->precision, (double)o->dsa, o->tol, o->inner_tol,
                                     (double)o->inner_max_iters, (double)o->max_iters, (double)o->restart,
                                     (double)(uintptr_t)b->dsa};
    if (!K->g_res || K->gen != b->graph_gen || K->key != key) {
        if (!b->cap_stream && (e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if ((e = record(b, o, b->cap_stream)) != cudaSuccess) return e;
        K->gen = b->graph_gen;
        K->key = key;
    }
    int flags[3] = {0, 0, 0};
    for (int cycle = 0; cycle <= o->max_iters; ++cycle) {
        if ((e = cudaGraphLaunch(K->g_res, s)) != cudaSuccess) return e;
        if ((e = cudaMemcpyAsync(flags, K->flags, sizeof(flags), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
        if (!flags[1]) break;
        for (int j = 0; j < K->k; ++j) {
            if ((e = cudaGraphLaunch(K->g_step, s)) != cudaSuccess) return e;
            if ((e = cudaMemcpyAsync(flags, K->flags, sizeof(flags), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
                return e;
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
            if (!flags[2]) break;
        }
        if ((e = cudaGraphLaunch(K->g_fin, s)) != cudaSuccess) return e;
    }
    const int c = b->count;
    std::vector<int> h(6 * c);
    std::vector<double> hs((size_t)c * K->L.sd);
    if ((e = cudaMemcpyAsync(h.data(), K->ints, h.size() * sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpyAsync(hs.data(), K->st, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    iters.assign(c, 0);
    rel.assign(c, 0.0);
    sweeps.assign(c, 0);
    conv.assign(c, 0);
    for (int i = 0; i < c; ++i) {
        iters[i] = h[3 * c + i];
        conv[i] = h[4 * c + i];
        sweeps[i] = h[3 * c + i] + h[5 * c + i] + 1;  // Arnoldi steps, restarts, and the first residual
        rel[i] = hs[(size_t)i * K->L.sd + K->L.rel];
    }
    return cudaSuccess;
}

}  // namespace sn
