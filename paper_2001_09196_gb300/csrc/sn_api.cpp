// C ABI of libsn (declared in include/sn.h): argument checking, mesh ownership and the
// outer source iteration.  Every numerical step runs in the CUDA kernels of sn_sweep.cu
// and sn_dsa.cu; this file only sequences them.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <string>
#include <vector>

#include "sn_dsa.h"
#include "sn_internal.h"

namespace sn {
cudaError_t upload_gl_constants();
std::atomic<long long> g_launches{0};
}

namespace {

thread_local std::string g_err;

sn_status fail(sn_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

sn_status cuda_fail(cudaError_t err, const char* where) {
    if (err == cudaErrorMemoryAllocation) return fail(SN_ERR_OOM, "%s: %s", where, cudaGetErrorString(err));
    return fail(SN_ERR_CUDA, "%s: %s", where, cudaGetErrorString(err));
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

bool g_const_ready[64] = {};

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc((void**)p, std::max<size_t>(1, count) * sizeof(T));
}

void free_mesh(sn_mesh* m) {
    if (!m) return;
    sn::drop_level_graphs(m);
    sn::free_operator_cache(m);
    sn::free_tiles(m);
    sn::free_level_groups(m);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    if (m->d_src) cudaFree(m->d_src);
    for (void* p : {(void*)m->d_dirs, (void*)m->d_wts, (void*)m->d_corners, (void*)m->d_sigma_t, (void*)m->d_sigma_s,
                    (void*)m->d_q, m->d_psi, m->d_psi32, (void*)m->d_lambda, (void*)m->d_mass, (void*)m->d_mass4, (void*)m->d_work, (void*)m->d_red,
                    (void*)m->d_scalars, (void*)m->levels.items, (void*)m->levels.padded, (void*)m->levels.padded_rev, (void*)m->levels.done,
                    (void*)m->levels.ctrl, (void*)m->d_krylov, (void*)m->levels.d_level_ptr, (void*)m->levels.d_barrier,
                    (void*)m->range_items})
        if (p) cudaFree(p);
    sn::drop_iter_graph(m);
    for (void* p : {(void*)m->d_ig, (void*)m->d_igi, (void*)m->d_igv})
        if (p) cudaFree(p);
    for (cudaStream_t st : m->ig_stream)
        if (st) cudaStreamDestroy(st);
    sn::dsa_free(m->dsa);
    sn::dsa_free(m->dsa_t);
    delete m;
}

bool finite_nonneg(const std::vector<double>& v) {
    for (double x : v)
        if (!std::isfinite(x) || x < 0.0) return false;
    return true;
}

}  // namespace

sn_status sn::set_error(sn_status st, const char* msg) {
    g_err = msg;
    return st;
}

extern "C" {

const char* sn_last_error(void) { return g_err.c_str(); }
const char* sn_version(void) { return "libsn 0.1 (sm_103a)"; }
long long sn_launch_count(void) { return sn::g_launches.load(); }

void sn_iter_opts_default(sn_iter_opts* o) {
    std::memset(o, 0, sizeof(*o));
    o->dsa = SN_DSA_THICK;
    o->thick_rule = SN_THICK_SIGMA_S;
    o->eta = 1.0;
    o->dsa_sigma = SN_DSA_SIGMA_S;
    o->tol = 1e-8;
    o->inner_tol = 1e-4;
    o->max_iters = 1000;
    o->inner_max_iters = 200;
    o->precision = SN_FP64;
    o->outer = SN_OUTER_SI;
    o->restart = 30;
    o->dsa_operator = SN_DSA_OP_SIP;
}

sn_status sn_mesh_create(const sn_mesh_desc* desc, sn_mesh** out) {
    if (!desc || !out) return fail(SN_ERR_ARG, "null argument");
    *out = nullptr;
    const sn_mesh_desc& d = *desc;
    if (d.dim != 2 && d.dim != 3) return fail(SN_ERR_ARG, "dim must be 2 or 3");
    if (d.nx < 1 || d.ny < 1 || (d.dim == 3 && d.nz < 1)) return fail(SN_ERR_ARG, "element counts must be >= 1");
    if (d.dim == 2 && (d.p < 1 || d.p > 3)) return fail(SN_ERR_ARG, "2D supports p = 1..3");
    if (d.dim == 3 && d.p != 1) return fail(SN_ERR_ARG, "3D supports p = 1");
    if (d.dim == 3 && d.vertices) return fail(SN_ERR_ARG, "3D meshes are uniform (vertices must be NULL)");
    if (!std::isfinite(d.psi_inc) || d.psi_inc < 0) return fail(SN_ERR_ARG, "psi_inc must be finite and >= 0");
    std::unique_ptr<sn_mesh, void (*)(sn_mesh*)> m(new sn_mesh(), free_mesh);
    m->desc = d;
    m->desc.vertices = nullptr;
    m->dim = d.dim;
    m->p = d.p;
    m->nx = d.nx;
    m->ny = d.ny;
    m->nz = d.dim == 3 ? d.nz : 1;
    const int Q = d.p + 1;
    m->n = d.dim == 2 ? Q * Q : Q * Q * Q;
    const long long ne = (long long)m->nx * m->ny * m->nz;
    if (ne > (1ll << 30)) return fail(SN_ERR_ARG, "too many elements");
    m->ne = (int)ne;
    if (!sn::level_symmetric(d.sn_order, d.dim, m->h_dirs, m->h_wts)) return fail(SN_ERR_ARG, "sn_order must be 4, 6 or 8");
    m->nd = (int)m->h_wts.size();
    m->hx = 1.0 / m->nx;
    m->hy = 1.0 / m->ny;
    m->hz = 1.0 / m->nz;
    if (d.dim == 2) {
        m->h_corners.resize((size_t)m->ne * 8);
        const int vx = m->nx + 1;
        for (int j = 0; j < m->ny; ++j)
            for (int i = 0; i < m->nx; ++i) {
                double* c = &m->h_corners[8 * ((size_t)j * m->nx + i)];
                for (int q = 0; q < 4; ++q) {
                    const int I = i + (q & 1), J = j + (q >> 1);
                    if (d.vertices) {
                        c[2 * q] = d.vertices[2 * ((size_t)J * vx + I)];
                        c[2 * q + 1] = d.vertices[2 * ((size_t)J * vx + I) + 1];
                    } else {
                        c[2 * q] = I * m->hx;
                        c[2 * q + 1] = J * m->hy;
                    }
                    if (!std::isfinite(c[2 * q]) || !std::isfinite(c[2 * q + 1])) return fail(SN_ERR_ARG, "non-finite vertex");
                }
                // element must not be inverted: det J > 0 at all four corners
                for (int q = 0; q < 4; ++q) {
                    const double xi = (q & 1) ? 1.0 : -1.0, eta = (q >> 1) ? 1.0 : -1.0;
                    const double ebx = c[2] - c[0], eby = c[3] - c[1], etx = c[6] - c[4], ety = c[7] - c[5];
                    const double elx = c[4] - c[0], ely = c[5] - c[1], erx = c[6] - c[2], ery = c[7] - c[3];
                    const double xx = (1 - eta) * ebx + (1 + eta) * etx, xy = (1 - eta) * eby + (1 + eta) * ety;
                    const double yx = (1 - xi) * elx + (1 + xi) * erx, yy = (1 - xi) * ely + (1 + xi) * ery;
                    if (!(xx * yy - yx * xy > 0)) return fail(SN_ERR_ARG, "element (%d,%d) is inverted or degenerate", i, j);
                }
            }
    }
    int dev = 0;
    CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 64 && !g_const_ready[dev]) {
        CK(sn::upload_gl_constants(), "upload constants");
        g_const_ready[dev] = true;
    }
    const size_t M = (size_t)m->ne * m->n;
    CK(dalloc(&m->d_dirs, m->h_dirs.size()), "alloc");
    CK(dalloc(&m->d_wts, m->h_wts.size()), "alloc");
    CK(cudaMemcpy(m->d_dirs, m->h_dirs.data(), m->h_dirs.size() * sizeof(double), cudaMemcpyHostToDevice), "copy");
    CK(cudaMemcpy(m->d_wts, m->h_wts.data(), m->h_wts.size() * sizeof(double), cudaMemcpyHostToDevice), "copy");
    if (d.dim == 2) {
        CK(dalloc(&m->d_corners, m->h_corners.size()), "alloc");
        CK(cudaMemcpy(m->d_corners, m->h_corners.data(), m->h_corners.size() * sizeof(double), cudaMemcpyHostToDevice), "copy");
    }
    CK(dalloc(&m->d_sigma_t, m->ne), "alloc");
    CK(dalloc(&m->d_sigma_s, m->ne), "alloc");
    CK(dalloc(&m->d_q, m->ne), "alloc");
    CK(cudaMemset(m->d_sigma_t, 0, m->ne * sizeof(double)), "memset");
    CK(cudaMemset(m->d_sigma_s, 0, m->ne * sizeof(double)), "memset");
    CK(cudaMemset(m->d_q, 0, m->ne * sizeof(double)), "memset");
    m->h_sigma_t.assign(m->ne, 0.0);
    m->h_sigma_s.assign(m->ne, 0.0);
    m->h_q.assign(m->ne, 0.0);
    CK(cudaMalloc(&m->d_psi, (size_t)m->nd * M * sizeof(double)), "alloc psi");
    CK(dalloc(&m->d_work, 4 * M), "alloc");
    m->red_blocks = (int)((M + 255) / 256);
    CK(dalloc(&m->d_red, m->red_blocks), "alloc");
    CK(dalloc(&m->d_scalars, 16), "alloc");
    CK(dalloc(&m->d_mass, M), "alloc");
    CK(dalloc(&m->d_mass4, M), "alloc");
    CK(dalloc(&m->d_src, M), "alloc");
    CK(sn::compute_mass(m.get(), 0), "element masses");
    bool cycle = false;
    CK(sn::build_levels(m.get(), 0, &cycle), "level sets");
    if (cycle) return fail(SN_ERR_CYCLE, "an upwind graph has a cycle");
    CK(cudaDeviceSynchronize(), "setup");
    *out = m.release();
    return SN_OK;
}

sn_status sn_mesh_destroy(sn_mesh* m) {
    if (!m) return SN_OK;
    cudaDeviceSynchronize();
    free_mesh(m);
    return SN_OK;
}

sn_status sn_get_levels(const sn_mesh* m, int d, int* levels) {
    if (!m || !levels) return fail(SN_ERR_ARG, "null argument");
    if (d < 0 || d >= m->nd) return fail(SN_ERR_ARG, "direction %d not in [0, %d)", d, m->nd);
    if (m->levels.h_level.size() != (size_t)m->nd * m->ne) return fail(SN_ERR_ARG, "no level sets");
    std::memcpy(levels, m->levels.h_level.data() + (size_t)d * m->ne, m->ne * sizeof(int));
    return SN_OK;
}

sn_status sn_mesh_get_info(const sn_mesh* m, sn_mesh_info* info) {
    if (!m || !info) return fail(SN_ERR_ARG, "null argument");
    info->n_elem = m->ne;
    info->n_nodes = m->n;
    info->n_dirs = m->nd;
    info->n_levels = m->levels.n_levels;
    info->n_items = (long long)m->ne * m->nd;
    return SN_OK;
}

sn_status sn_mesh_quadrature(const sn_mesh* m, double* dirs, double* weights) {
    if (!m) return fail(SN_ERR_ARG, "null mesh");
    if (dirs) std::memcpy(dirs, m->h_dirs.data(), m->h_dirs.size() * sizeof(double));
    if (weights) std::memcpy(weights, m->h_wts.data(), m->h_wts.size() * sizeof(double));
    return SN_OK;
}

static sn_status commit_materials(sn_mesh* m, std::vector<double>& hst, std::vector<double>& hss,
                                  std::vector<double>& hq, cudaStream_t s);

sn_status sn_set_materials(sn_mesh* m, const double* st, const double* ss, const double* q, int mem, void* stream) {
    if (!m || !st || !ss || !q) return fail(SN_ERR_ARG, "null argument");
    if (mem != 0 && mem != 1) return fail(SN_ERR_ARG, "mem must be 0 (host) or 1 (device)");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> hst(m->ne), hss(m->ne), hq(m->ne);
    const cudaMemcpyKind k = mem ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    CK(cudaMemcpyAsync(hst.data(), st, m->ne * sizeof(double), k, s), "copy");
    CK(cudaMemcpyAsync(hss.data(), ss, m->ne * sizeof(double), k, s), "copy");
    CK(cudaMemcpyAsync(hq.data(), q, m->ne * sizeof(double), k, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    return commit_materials(m, hst, hss, hq, s);
}

sn_status sn_set_pseudo_scattering(sn_mesh* m, const double* sigma, const double* cv, const double* T, double dt,
                                   double a_rad, double c_light, int mem, void* stream) {
    if (!m || !sigma || !cv || !T) return fail(SN_ERR_ARG, "null argument");
    if (mem != 0 && mem != 1) return fail(SN_ERR_ARG, "mem must be 0 (host) or 1 (device)");
    if (!(dt > 0) || !(a_rad > 0) || !(c_light > 0) || !std::isfinite(dt) || !std::isfinite(a_rad) ||
        !std::isfinite(c_light))
        return fail(SN_ERR_ARG, "dt, a_rad and c_light must be finite and > 0");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ne = (size_t)m->ne;
    // inputs and outputs in the work vector (4 n_elem n_nodes doubles >= 6 n_elem)
    double* in = m->d_work;
    double* out = m->d_work + 3 * ne;
    std::vector<double> h(3 * ne);
    const cudaMemcpyKind k = mem ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
    CK(cudaMemcpyAsync(h.data(), sigma, ne * sizeof(double), k, s), "copy");
    CK(cudaMemcpyAsync(h.data() + ne, cv, ne * sizeof(double), k, s), "copy");
    CK(cudaMemcpyAsync(h.data() + 2 * ne, T, ne * sizeof(double), k, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    for (size_t e = 0; e < ne; ++e)
        if (!(std::isfinite(h[e]) && h[e] >= 0.0 && std::isfinite(h[ne + e]) && h[ne + e] > 0.0 &&
              std::isfinite(h[2 * ne + e]) && h[2 * ne + e] >= 0.0))
            return fail(SN_ERR_ARG, "need finite sigma >= 0, C_v > 0, T >= 0 (element %zu)", e);
    // sigma b = 16 pi a c sigma T^3 and the emission sigma a c T^4 must stay finite (Eq. hohlraum_q)
    for (size_t e = 0; e < ne; ++e) {
        const double t = h[2 * ne + e], t3 = t * t * t;
        const double sb = h[e] * (16.0 * M_PI * a_rad * c_light * t3);
        if (!std::isfinite(sb) || !std::isfinite(h[e] * a_rad * c_light * t3 * t * 4.0 * M_PI))
            return fail(SN_ERR_ARG, "sigma b = 16 pi a c sigma T^3 overflows at element %zu (T = %g)", e, t);
    }
    CK(cudaMemcpyAsync(in, h.data(), 3 * ne * sizeof(double), cudaMemcpyHostToDevice, s), "copy");
    CK(sn::launch_pseudo_scattering(in, in + ne, in + 2 * ne, m->ne, dt, a_rad, c_light, out, out + ne, out + 2 * ne, s),
       "pseudo-scattering kernel");
    std::vector<double> hst(ne), hss(ne), hq(ne);
    CK(cudaMemcpyAsync(hst.data(), out, ne * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaMemcpyAsync(hss.data(), out + ne, ne * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaMemcpyAsync(hq.data(), out + 2 * ne, ne * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    return commit_materials(m, hst, hss, hq, s);
}

sn_status sn_get_materials(const sn_mesh* m, double* st, double* ss, double* q) {
    if (!m) return fail(SN_ERR_ARG, "null mesh");
    if (st) std::memcpy(st, m->h_sigma_t.data(), m->ne * sizeof(double));
    if (ss) std::memcpy(ss, m->h_sigma_s.data(), m->ne * sizeof(double));
    if (q) std::memcpy(q, m->h_q.data(), m->ne * sizeof(double));
    return SN_OK;
}

// Validates host copies of the materials and makes them the mesh's (invalidating what depends on them).
static sn_status commit_materials(sn_mesh* m, std::vector<double>& hst, std::vector<double>& hss,
                                  std::vector<double>& hq, cudaStream_t s) {
    if (!finite_nonneg(hst) || !finite_nonneg(hss) || !finite_nonneg(hq))
        return fail(SN_ERR_ARG, "materials must be finite and >= 0");
    for (int e = 0; e < m->ne; ++e)
        if (hss[e] > hst[e]) return fail(SN_ERR_ARG, "sigma_s > sigma_t at element %d", e);
    m->h_sigma_t = hst;
    m->h_sigma_s = hss;
    m->h_q = hq;
    CK(cudaMemcpyAsync(m->d_sigma_t, hst.data(), m->ne * sizeof(double), cudaMemcpyHostToDevice, s), "copy");
    CK(cudaMemcpyAsync(m->d_sigma_s, hss.data(), m->ne * sizeof(double), cudaMemcpyHostToDevice, s), "copy");
    CK(cudaMemcpyAsync(m->d_q, hq.data(), m->ne * sizeof(double), cudaMemcpyHostToDevice, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    sn::drop_iter_graph(m);
    sn::dsa_free(m->dsa);
    sn::dsa_free(m->dsa_t);
    m->dsa = m->dsa_t = nullptr;
    m->dsa_key_dsa = -1;
    m->ainv_valid = m->ainv32_valid = false;  // the cached inverses depend on sigma_t
    return SN_OK;
}

static sn_status ensure_psi32(sn_mesh* m) {
    if (m->d_psi32) return SN_OK;
    CK(cudaMalloc(&m->d_psi32, (size_t)m->nd * m->ne * m->n * sizeof(float)), "alloc psi32");
    sn::drop_level_graphs(m);
    return SN_OK;
}

static sn_status ensure_lambda(sn_mesh* m) {
    if (m->d_lambda) return SN_OK;
    CK(cudaMalloc(&m->d_lambda, (size_t)m->nd * m->ne * m->n * sizeof(double)), "alloc lambda");
    sn::drop_level_graphs(m);
    return SN_OK;
}

sn_status sn_sweep(sn_mesh* m, const double* phi_in, double* phi_out, int precision, void* stream) {
    if (!m || !phi_out) return fail(SN_ERR_ARG, "null argument");
    if (precision < SN_FP64 || precision > SN_FP32_REFINE) return fail(SN_ERR_ARG, "bad precision");
    if (phi_in == phi_out) return fail(SN_ERR_ARG, "phi_in and phi_out must not alias");
    if (precision == SN_FP32) {
        sn_status st = ensure_psi32(m);
        if (st != SN_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CK(sn::launch_sweep(m, phi_in, precision, 1.0, s), "sweep");
    CK(sn::launch_phi_reduce(m, precision, nullptr, phi_out, nullptr, s), "phi reduce");
    if (m->schedule != sn::SCHED_LEVELS) {
        bool timed_out = false;
        CK(sn::take_sweep_error(m, s, &timed_out), "sweep status");
        if (timed_out) return fail(SN_ERR_TIMEOUT, "a sweep dependency wait timed out");
    }
    return SN_OK;
}

sn_status sn_sweep_directions(sn_mesh* m, const double* phi_in, double* phi_out, int d_begin, int d_end, int precision,
                              void* stream) {
    if (!m || !phi_out) return fail(SN_ERR_ARG, "null argument");
    if (precision < SN_FP64 || precision > SN_FP32_REFINE) return fail(SN_ERR_ARG, "bad precision");
    if (phi_in == phi_out) return fail(SN_ERR_ARG, "phi_in and phi_out must not alias");
    if (d_begin < 0 || d_end > m->nd || d_begin >= d_end)
        return fail(SN_ERR_ARG, "direction range [%d, %d) not inside [0, %d)", d_begin, d_end, m->nd);
    if (precision == SN_FP32) {
        sn_status st = ensure_psi32(m);
        if (st != SN_OK) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CK(sn::launch_sweep_range(m, phi_in, precision, d_begin, d_end, s), "sweep");
    CK(sn::launch_phi_reduce(m, precision, nullptr, phi_out, nullptr, s, d_begin, d_end), "phi reduce");
    return SN_OK;
}

sn_status sn_mesh_set_operator_cache(sn_mesh* m, int mode) {
    if (!m) return fail(SN_ERR_ARG, "null mesh");
    if (mode < SN_CACHE_OFF || mode > SN_CACHE_AUTO) return fail(SN_ERR_ARG, "bad cache mode %d", mode);
    CK(cudaDeviceSynchronize(), "sync");  // no sweep may still read the buffers freed below
    if (mode == SN_CACHE_OFF) sn::free_operator_cache(m);
    m->ainv_denied = m->ainv32_denied = false;
    m->cache_mode = mode;
    sn::drop_level_graphs(m);
    return SN_OK;
}

sn_status sn_debug_stall_next_sweep(sn_mesh* m, double timeout_seconds) {
    if (!m) return fail(SN_ERR_ARG, "null mesh");
    if (!(timeout_seconds > 0.0 && timeout_seconds <= 4.0)) return fail(SN_ERR_ARG, "timeout must be in (0, 4] s");
    if (m->schedule == sn::SCHED_LEVELS) return fail(SN_ERR_ARG, "only the dataflow and tiled schedules wait");
    m->levels.stall_timeout_s = timeout_seconds;
    return SN_OK;
}

sn_status sn_mesh_set_schedule(sn_mesh* m, int schedule, int block, int param) {
    if (!m) return fail(SN_ERR_ARG, "null mesh");
    if (schedule < sn::SCHED_LEVELS || schedule > sn::SCHED_STATIC) return fail(SN_ERR_ARG, "bad schedule");
    const int max_block = schedule == sn::SCHED_TILES ? 256 : (schedule == sn::SCHED_BARRIER ? 512 : 128);
    if (block < 32 || block > max_block || block % 32)
        return fail(SN_ERR_ARG, "block must be a multiple of 32 in [32, %d]", max_block);
    if (param < 0) return fail(SN_ERR_ARG, "the schedule parameter must be >= 0");
    if (schedule == sn::SCHED_TILES && param > 64) return fail(SN_ERR_ARG, "tile edge must be <= 64");
    if (schedule == sn::SCHED_LEVELS && param > m->nd) return fail(SN_ERR_ARG, "more direction groups than directions");
    const int groups = schedule == sn::SCHED_LEVELS ? std::max(param, 1) : m->level_groups;
    const bool own_block = schedule == sn::SCHED_LEVELS || sn::dataflow_like(schedule);
    if ((own_block && m->block != block) || groups != m->level_groups) sn::drop_level_graphs(m);
    m->schedule = schedule;
    if (own_block) m->block = block;
    if (schedule == sn::SCHED_TILES) {
        m->tile_block = block;
        m->tile_edge = param > 0 ? param : (m->dim == 2 ? 16 : 8);
    } else if (schedule == sn::SCHED_LEVELS) {
        m->level_groups = groups;
    } else if (schedule == sn::SCHED_BARRIER) {
        m->barrier_block = block;
        m->barrier_ctas_per_sm = std::max(param, 1);
    } else {
        m->max_blocks_per_sm = param;
    }
    return SN_OK;
}

// Thick mask selected by opts (Sec. 3.2: sigma_s >= eta; or sigma_t h > eta; or explicit; all for full DSA).
static sn_status thick_mask_for(const sn_mesh* m, const sn_iter_opts* o, std::vector<unsigned char>& mask) {
    mask.assign(m->ne, 0);
    if (o->dsa == SN_DSA_FULL) {
        for (int e = 0; e < m->ne; ++e) {
            if (!(m->h_sigma_t[e] > 0.0))
                return fail(SN_ERR_VOID_FULL_DSA, "full DSA needs sigma_t > 0 everywhere (element %d is void)", e);
            mask[e] = 1;
        }
    } else if (o->thick_rule == SN_THICK_SIGMA_S) {
        for (int e = 0; e < m->ne; ++e) mask[e] = m->h_sigma_s[e] >= o->eta && m->h_sigma_t[e] > 0.0;
    } else if (o->thick_rule == SN_THICK_SIGMA_T_H) {
        const double h = m->hx;
        for (int e = 0; e < m->ne; ++e) mask[e] = m->h_sigma_t[e] * h > o->eta;
    } else if (o->thick_rule == SN_THICK_MASK) {
        if (!o->mask) return fail(SN_ERR_ARG, "thick_rule MASK needs opts->mask");
        for (int e = 0; e < m->ne; ++e) {
            mask[e] = o->mask[e] ? 1 : 0;
            if (mask[e] && !(m->h_sigma_t[e] > 0.0)) return fail(SN_ERR_ARG, "masked element %d is void", e);
        }
    } else {
        return fail(SN_ERR_ARG, "bad thick_rule");
    }
    return SN_OK;
}

// Builds (or reuses) the DSA hierarchy selected by opts.
static sn_status ensure_dsa(sn_mesh* m, const sn_iter_opts* o) {
    std::vector<unsigned char> mask;
    sn_status st = thick_mask_for(m, o, mask);
    if (st != SN_OK) return st;
    if (m->dsa && m->dsa_key_mask == mask && m->dsa_key_sigma == o->dsa_sigma && m->dsa_key_op == o->dsa_operator) {
        m->dsa->vcycle_mode = o->dsa_vcycle;
        if (m->dsa_t) m->dsa_t->vcycle_mode = o->dsa_vcycle;
        return SN_OK;
    }
    sn::drop_iter_graph(m);
    sn::dsa_free(m->dsa);
    sn::dsa_free(m->dsa_t);
    m->dsa = m->dsa_t = nullptr;
    std::string err;
    bool void_conflict = false;
    m->dsa = sn::dsa_build(m, mask.data(), o->dsa_sigma, o->dsa_operator, false, err, &void_conflict);
    if (!m->dsa) return fail(void_conflict ? SN_ERR_VOID_FULL_DSA : SN_ERR_ARG, "DSA setup: %s", err.c_str());
    m->dsa_key_mask = mask;
    m->dsa_key_sigma = o->dsa_sigma;
    m->dsa_key_op = o->dsa_operator;
    m->dsa->vcycle_mode = o->dsa_vcycle;
    return SN_OK;
}

// The adjoint iteration's DSA step solves with D_ff^T: for a nonsymmetric operator (Eq. NIP) a
// second hierarchy built from the transposed blocks, kept beside the forward one.
static sn_status ensure_dsa_adjoint(sn_mesh* m, const sn_iter_opts* o) {
    sn_status st = ensure_dsa(m, o);
    if (st != SN_OK || !m->dsa || m->dsa->symmetric || m->dsa_t) return st;
    std::string err;
    m->dsa_t = sn::dsa_build(m, m->dsa_key_mask.data(), o->dsa_sigma, o->dsa_operator, true, err);
    if (!m->dsa_t) return fail(SN_ERR_ARG, "DSA setup (transposed): %s", err.c_str());
    m->dsa_t->vcycle_mode = o->dsa_vcycle;
    return SN_OK;
}

// Hierarchy of the DSA step: D_ff, or D_ff^T in the adjoint iteration.
static sn::DsaHierarchy* dsa_for(sn_mesh* m, bool adjoint) { return adjoint && m->dsa_t ? m->dsa_t : m->dsa; }

// Direction sharding (sn_iter_opts.dir_begin / dir_end / exchange): this process sweeps a range of
// directions and the caller's exchange sums the partial updates over processes (Eq. phi).
static bool sharded(const sn_iter_opts* o) { return o->exchange != nullptr || o->dir_begin != 0 || o->dir_end != 0; }

static sn_status check_shard(const sn_mesh* m, const sn_iter_opts* o) {
    if (!sharded(o)) return SN_OK;
    if (!o->exchange) return fail(SN_ERR_ARG, "a direction range needs an exchange function");
    const int d1 = o->dir_begin == 0 && o->dir_end == 0 ? m->nd : o->dir_end;
    if (o->dir_begin < 0 || d1 > m->nd || o->dir_begin >= d1)
        return fail(SN_ERR_ARG, "direction range [%d, %d) not inside [0, %d)", o->dir_begin, d1, m->nd);
    return SN_OK;
}

// out = sum_d w_d L_d^{-1}(q_scale q/(4 pi) + sigma_s phi_in/(4 pi)) over all directions: swept here,
// or this process's range swept here and completed by the caller's exchange.
static sn_status transport_update(sn_mesh* m, const sn_iter_opts* o, const double* phi_in, double* out, double q_scale,
                                  cudaStream_t s, int precision = -1) {
    if (precision < 0) precision = o->precision;
    if (!sharded(o)) {
        CK(sn::launch_sweep(m, phi_in, precision, q_scale, s), "sweep");
        CK(sn::launch_phi_reduce(m, precision, nullptr, out, nullptr, s), "phi reduce");
        return SN_OK;
    }
    const int d0 = o->dir_begin, d1 = o->dir_begin == 0 && o->dir_end == 0 ? m->nd : o->dir_end;
    const long long M = (long long)m->ne * m->n;
    double* buf = o->exchange_buf ? o->exchange_buf : out;
    CK(sn::launch_sweep_range(m, phi_in, precision, d0, d1, s, q_scale), "sweep");
    CK(sn::launch_phi_reduce(m, precision, nullptr, buf, nullptr, s, d0, d1), "phi reduce");
    const sn_status st = o->exchange(buf, M, (void*)s, o->exchange_ctx);
    if (st != SN_OK) return fail(st, "the exchange of a partial transport update returned status %d", (int)st);
    if (buf != out) CK(cudaMemcpyAsync(out, buf, M * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    return SN_OK;
}

static sn_status check_opts(const sn_iter_opts* o) {
    if (!o) return fail(SN_ERR_ARG, "null opts");
    if (o->dsa < SN_DSA_NONE || o->dsa > SN_DSA_TRIANGULAR) return fail(SN_ERR_ARG, "bad dsa");
    if (o->dsa_operator < SN_DSA_OP_SIP || o->dsa_operator > SN_DSA_OP_MNIP) return fail(SN_ERR_ARG, "bad dsa_operator");
    if (o->dsa_vcycle < SN_VCYCLE_AUTO || o->dsa_vcycle > SN_VCYCLE_FP32) return fail(SN_ERR_ARG, "bad dsa_vcycle");
    if (o->precision < SN_FP64 || o->precision > SN_FP32_MIXED) return fail(SN_ERR_ARG, "bad precision");
    if (o->precision == SN_FP32_MIXED && o->outer != SN_OUTER_FGMRES)
        return fail(SN_ERR_ARG, "SN_FP32_MIXED refines around fGMRES (outer = SN_OUTER_FGMRES)");
    if (o->precision == SN_FP32_MIXED && !(o->refine_drop >= 0.0 && o->refine_drop < 1.0))
        return fail(SN_ERR_ARG, "refine_drop must be in [0, 1)");
    if (!(o->tol >= 0) || o->max_iters < 1) return fail(SN_ERR_ARG, "bad tol / max_iters");
    if (o->dsa != SN_DSA_NONE && (!(o->inner_tol > 0) || o->inner_max_iters < 1))
        return fail(SN_ERR_ARG, "bad inner_tol / inner_max_iters");
    if (o->checkpoint_every > 0 && (!o->checkpoints || o->max_checkpoints < 1))
        return fail(SN_ERR_ARG, "checkpointing needs a buffer");
    if (o->outer != SN_OUTER_SI && o->outer != SN_OUTER_FGMRES) return fail(SN_ERR_ARG, "bad outer iteration");
    if (o->outer == SN_OUTER_FGMRES && (o->restart < 1 || o->restart > 60))
        return fail(SN_ERR_ARG, "restart must be in 1..60");
    return SN_OK;
}

// Device time of one kind of work over a solve: CUDA event pairs recorded on the stream around
// each segment, their elapsed times summed at the synchronisation points the iterations already
// have (harvest() is called only after the stream has been synchronised).
struct SegmentClock {
    static constexpr int kPairs = 8;
    cudaEvent_t a[kPairs] = {}, b[kPairs] = {};
    int n = 0;
    double ms = 0.0;
    bool ok = true;
    SegmentClock() {
        for (int i = 0; i < kPairs && ok; ++i)
            ok = cudaEventCreate(&a[i]) == cudaSuccess && cudaEventCreate(&b[i]) == cudaSuccess;
    }
    ~SegmentClock() {
        for (int i = 0; i < kPairs; ++i) {
            if (a[i]) cudaEventDestroy(a[i]);
            if (b[i]) cudaEventDestroy(b[i]);
        }
    }
    void begin(cudaStream_t s) {
        if (!ok) return;
        if (n == kPairs) {  // more segments than pairs between two synchronisations
            cudaEventSynchronize(b[kPairs - 1]);
            harvest();
        }
        cudaEventRecord(a[n], s);
    }
    void end(cudaStream_t s) {
        if (!ok) return;
        cudaEventRecord(b[n], s);
        ++n;
    }
    void harvest() {
        for (int i = 0; i < n; ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, a[i], b[i]) == cudaSuccess) ms += t;
        }
        n = 0;
    }
};

// Workspace of flexible GMRES(k): basis V ((k+1) x M), preconditioned basis Z (k x M), w (M),
// partial sums ((k+1) x blocks) and small device scalars.
static sn_status ensure_krylov(sn_mesh* m, int k) {
    const long long M = (long long)m->ne * m->n;
    const int nb = sn::krylov_blocks(M);
    const size_t need = (size_t)(2 * k + 2) * M + (size_t)(k + 1) * nb + 4 * (k + 2);
    if (!m->d_krylov || m->krylov_restart < k) {
        if (m->d_krylov) {
            CK(cudaDeviceSynchronize(), "sync");
            cudaFree(m->d_krylov);
        }
        m->d_krylov = nullptr;
        sn::drop_iter_graph(m);  // a recorded iteration holds the old workspace's addresses
        CK(cudaMalloc(&m->d_krylov, need * sizeof(double)), "alloc fGMRES workspace");
        m->krylov_restart = k;
    }
    return SN_OK;
}

// Flexible GMRES(k) on S x = b (Eq. schur), right-preconditioned by the DSA step
// P v = v + E_f D_ff^{-1} Sigma_f E_f^T v (Algorithm 2 applied to a residual); classical
// Gram-Schmidt twice, Givens rotations on the host.
// adjoint = true solves S^T x = g instead: operator x - T^T x (reverse sweeps), preconditioner
// v + Sigma_f D_ff^{-1} E_f^T v (the transposed DSA step), residual g + T^T x - x.
static sn_status fgmres(sn_mesh* m, const sn_iter_opts* o, double* x, sn_iter_stats* stats, cudaStream_t s,
                        std::chrono::steady_clock::time_point t0, bool adjoint = false, const double* g_rhs = nullptr) {
    const long long M = (long long)m->ne * m->n;
    const int k = o->restart;
    const int nb = sn::krylov_blocks(M);
    sn_status wst = ensure_krylov(m, k);
    if (wst != SN_OK) return wst;
    double* V = m->d_krylov;                    // (k+1) x M
    double* Z = V + (size_t)(k + 1) * M;        // k x M
    double* w = Z + (size_t)k * M;              // M
    double* part = w + M;                       // (k+1) x nb
    double* hd = part + (size_t)(k + 1) * nb;   // h (k+1), h2 (k+1), norm, y (k)
    double* tmp = m->d_work + 2 * (size_t)M;
    std::vector<double> H((size_t)(k + 1) * k, 0.0), cs(k), sn_(k), g(k + 1), hh(2 * (k + 1) + 1), y(k);
    double r0 = 0.0, rel = INFINITY;
    int it = 0, inner_total = 0, sweeps = 0;
    bool converged = false;
    bool timed_out = false;
    SegmentClock sweep_clock, dsa_clock;
    // SN_FP32_MIXED: float64 sweeps for the true residual, float32 sweeps inside the cycle, and a
    // cycle ends once its residual estimate fell by `drop` (iterative refinement around fGMRES)
    const bool mixed = o->precision == SN_FP32_MIXED;
    const int prec_res = mixed ? SN_FP64 : o->precision, prec_op = mixed ? SN_FP32 : o->precision;
    const double drop = mixed ? (o->refine_drop > 0.0 ? o->refine_drop : 1e-4) : 0.0;
    while (true) {
        // true residual r = sweep(x) - x (with the fixed source); adjoint: g + T^T x - x
        ++sweeps;
        sweep_clock.begin(s);
        if (adjoint) {
            CK(sn::launch_adjoint_sweep(m, x, s), "adjoint sweep");
            CK(sn::launch_adjoint_reduce(m, tmp, s), "adjoint reduce");
            CK(sn::launch_axpy_add(tmp, g_rhs, M, s), "add g");
        } else {
            sn_status ust = transport_update(m, o, x, tmp, 1.0, s, prec_res);
            if (ust != SN_OK) return ust;
        }
        sweep_clock.end(s);
        CK(sn::launch_axpy_norm(m, tmp, x, w, m->d_scalars, s), "residual");
        double rr = 0.0;
        CK(cudaMemcpyAsync(&rr, m->d_scalars, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
        CK(cudaStreamSynchronize(s), "sync");
        sweep_clock.harvest();
        dsa_clock.harvest();
        if (m->schedule != sn::SCHED_LEVELS) {
            CK(sn::take_sweep_error(m, s, &timed_out), "sweep status");
            if (timed_out) return fail(SN_ERR_TIMEOUT, "a sweep dependency wait timed out");
        }
        const double beta = std::sqrt(rr);
        if (r0 == 0.0) r0 = beta > 0 ? beta : 1.0;
        rel = beta / r0;
        if (stats && stats->residual_history && it < stats->history_len && it == 0) stats->residual_history[0] = rel;
        if (rel <= o->tol || beta == 0.0) {  // convergence is declared on the true residual only
            converged = true;
            break;
        }
        if (it >= o->max_iters) break;
        CK(sn::launch_normalize(w, M, part, hd, V, s), "normalize");
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jj = 0;
        for (int j = 0; j < k && it < o->max_iters; ++j) {
            double* Vj = V + (size_t)j * M;
            double* Zj = Z + (size_t)j * M;
            CK(sn::launch_copy(Zj, Vj, M, s), "copy");
            if (o->dsa != SN_DSA_NONE && m->dsa && sn::dsa_thick_count(m->dsa) > 0) {
                dsa_clock.begin(s);
                CK(sn::dsa_correct(dsa_for(m, adjoint), Vj, Zj, o->inner_tol, o->inner_max_iters, adjoint, s), "DSA");
                dsa_clock.end(s);
                if (o->dsa == SN_DSA_TRIANGULAR) {
                    // Algorithm 1, step 2: the zero-source transport update of [0; Z_f], kept on the
                    // thin DOFs (Z_f = V_f + D_ff^{-1} Sigma_f V_f after step 1)
                    double* w = m->d_work;
                    double* y = m->d_work + M;
                    CK(sn::dsa_select_thick(m->dsa, Zj, w, s), "Algorithm 1");
                    sweep_clock.begin(s);
                    sn_status ust = transport_update(m, o, w, y, 0.0, s, prec_op);
                    if (ust != SN_OK) return ust;
                    sweep_clock.end(s);
                    CK(sn::dsa_add_thin(m->dsa, y, Zj, s), "Algorithm 1");
                    ++sweeps;
                }
            }
            // w = S Zj = Zj - T Zj (T: sweep without the fixed source)
            sweep_clock.begin(s);
            if (adjoint) {
                CK(sn::launch_adjoint_sweep(m, Zj, s), "adjoint sweep");
                CK(sn::launch_adjoint_reduce(m, tmp, s), "adjoint reduce");
            } else {
                sn_status ust = transport_update(m, o, Zj, tmp, 0.0, s, prec_op);
                if (ust != SN_OK) return ust;
            }
            sweep_clock.end(s);
            ++sweeps;
            CK(sn::launch_axpy_norm(m, Zj, tmp, w, m->d_scalars, s), "apply S");
            CK(sn::launch_multidot(V, j + 1, M, w, part, hd, s), "orthogonalise");
            CK(sn::launch_multiaxpy(V, j + 1, M, hd, -1.0, w, s), "orthogonalise");
            CK(sn::launch_multidot(V, j + 1, M, w, part, hd + (k + 1), s), "orthogonalise");
            CK(sn::launch_multiaxpy(V, j + 1, M, hd + (k + 1), -1.0, w, s), "orthogonalise");
            CK(sn::launch_multidot(w, 1, M, w, part, hd + 2 * (k + 1), s), "norm");
            CK(cudaMemcpyAsync(hh.data(), hd, hh.size() * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
            CK(cudaStreamSynchronize(s), "sync");
            sweep_clock.harvest();
            dsa_clock.harvest();
            if (m->schedule != sn::SCHED_LEVELS) {
                CK(sn::take_sweep_error(m, s, &timed_out), "sweep status");
                if (timed_out) return fail(SN_ERR_TIMEOUT, "a sweep dependency wait timed out");
            }
            double* h = &H[(size_t)j * (k + 1)];
            for (int i = 0; i <= j; ++i) h[i] = hh[i] + hh[k + 1 + i];
            h[j + 1] = std::sqrt(std::max(hh[2 * (k + 1)], 0.0));
            const double hnext = h[j + 1];
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * h[i] + sn_[i] * h[i + 1];
                h[i + 1] = -sn_[i] * h[i] + cs[i] * h[i + 1];
                h[i] = t;
            }
            const double rho = std::hypot(h[j], h[j + 1]);
            cs[j] = rho > 0 ? h[j] / rho : 1.0;
            sn_[j] = rho > 0 ? h[j + 1] / rho : 0.0;
            h[j] = rho;
            h[j + 1] = 0.0;
            g[j + 1] = -sn_[j] * g[j];
            g[j] = cs[j] * g[j];
            ++it;
            jj = j + 1;
            rel = std::fabs(g[j + 1]) / r0;
            if (stats && stats->residual_history && it < stats->history_len) stats->residual_history[it] = rel;
            if (rel <= o->tol || hnext <= 1e-300) break;
            if (mixed && std::fabs(g[j + 1]) <= drop * beta) break;  // this cycle's correction is done
            CK(sn::launch_normalize(w, M, part, hd + 2 * (k + 1), V + (size_t)(j + 1) * M, s), "normalize");
        }
        // x += Z y with H y = g (upper triangular)
        for (int i = jj - 1; i >= 0; --i) {
            double t = g[i];
            for (int c = i + 1; c < jj; ++c) t -= H[(size_t)c * (k + 1) + i] * y[c];
            y[i] = t / H[(size_t)i * (k + 1) + i];
        }
        CK(cudaMemcpyAsync(hd, y.data(), jj * sizeof(double), cudaMemcpyHostToDevice, s), "copy");
        CK(sn::launch_multiaxpy(Z, jj, M, hd, 1.0, x, s), "update");
        // the restart (or the final check) recomputes the true residual with one more sweep
    }
    CK(cudaStreamSynchronize(s), "sync");
    sweep_clock.harvest();
    dsa_clock.harvest();
    if (m->dsa) CK(sn::dsa_take_iters(dsa_for(m, adjoint), s, &inner_total), "DSA iterations");
    if (stats) {
        stats->iters = it;
        stats->rel_residual = rel;
        stats->inner_iters_total = inner_total;
        stats->thick_fraction = m->dsa && o->dsa != SN_DSA_NONE ? (double)sn::dsa_thick_count(m->dsa) / m->ne : 0.0;
        stats->n_checkpoints = 0;
        stats->n_sweeps = sweeps;
        stats->ms_sweep = sweep_clock.ms;
        stats->ms_dsa = dsa_clock.ms;
        stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!converged) return fail(SN_ERR_NOT_CONVERGED, "fGMRES not converged after %d iterations (%.3e)", it, rel);
    return SN_OK;
}

// ---------------------------------------------------------------- recorded outer iterations
// A whole source iteration or flexible GMRES solve recorded once into a CUDA graph and launched as
// one graph: the loops are WHILE conditional nodes whose conditions are set by device kernels
// (sn_iter_graph.cu), the DSA solve is a nested WHILE node, and the host synchronises once per
// solve instead of once per outer iteration.  Used for the level and dataflow schedules on one
// process (the tiled and level-barrier schedules carry host-side state, and a sharded iteration
// calls back to the host).

// WHILE node (handle h) appended to the graph `s` is capturing; its body graph in *body.
static cudaError_t add_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t* body) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t err = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps);
    if (err != cudaSuccess) return err;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if ((err = cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &cp)) != cudaSuccess) return err;
    if ((err = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return err;
    *body = cp.conditional.phGraph_out[0];
    return cudaSuccess;
}

static cudaError_t new_handle(cudaStream_t s, unsigned dflt, cudaGraphConditionalHandle* h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    cudaError_t err = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr);
    if (err != cudaSuccess) return err;
    return cudaGraphConditionalHandleCreate(h, g, dflt, cudaGraphCondAssignDefault);
}

static bool recordable(const sn_mesh* m, const sn_iter_opts* o) {
    return !o->host_loop && !sharded(o) && (m->schedule == sn::SCHED_LEVELS || sn::dataflow_like(m->schedule));
}

// What a recorded iteration depends on: a graph is reused only for the same key.
static std::vector<double> iteration_key(const sn_mesh* m, const sn_iter_opts* o, int hist_len) {
    auto addr = [](const void* p) { return (double)(uintptr_t)p; };
    return {(double)o->outer, (double)o->restart, (double)o->dsa, (double)o->precision, o->tol, o->inner_tol,
            (double)o->inner_max_iters, (double)o->max_iters, o->refine_drop, (double)hist_len,
            (double)o->checkpoint_every, addr(o->checkpoints), (double)o->max_checkpoints, addr(m->dsa),
            m->dsa ? (double)m->dsa->vcycle_mode : -1.0, (double)m->level_groups, (double)m->block,
            (double)m->schedule, (double)m->max_blocks_per_sm,
            addr(m->d_krylov), addr(m->d_ig), addr(m->d_igv), addr(m->d_psi32)};
}

// Records the iteration (fgmres: flexible GMRES, else source iteration) into m->iter_graph.
static cudaError_t record_iteration(sn_mesh* m, const sn_iter_opts* o, bool fg, int hist_len) {
    const long long M = (long long)m->ne * m->n;
    const int k = o->restart;
    cudaError_t err;
    for (auto& st : m->ig_stream)
        if (!st && (err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return err;
    cudaStream_t s0 = m->ig_stream[0], s1 = m->ig_stream[1], s2 = m->ig_stream[2];
    double* gd = m->d_ig;
    int* gi = m->d_igi;
    double* hist = hist_len > 0 ? m->d_ig + m->ig_doubles : nullptr;
    double* x = m->d_igv;
    double* vt = x + M;
    double* zt = x + 2 * M;
    const bool mixed = o->precision == SN_FP32_MIXED;
    const int prec_res = mixed ? SN_FP64 : o->precision, prec_op = mixed ? SN_FP32 : o->precision;
    const double drop = mixed ? (o->refine_drop > 0.0 ? o->refine_drop : 1e-4) : 0.0;
    const bool dsa = o->dsa != SN_DSA_NONE && m->dsa && sn::dsa_thick_count(m->dsa) > 0;
    const long long c0 = sn::g_launches.load();
    int open = 0;  // captures in progress (s0, s1, s2)
    cudaGraph_t graph = nullptr;
    auto unwind = [&](cudaError_t e) {
        cudaGraph_t g2 = nullptr;
        if (open > 2) cudaStreamEndCapture(s2, &g2);
        if (open > 1) cudaStreamEndCapture(s1, &g2);
        if (open > 0) {
            cudaStreamEndCapture(s0, &g2);
            if (g2) cudaGraphDestroy(g2);
        }
        cudaGetLastError();
        sn::g_launches.store(c0);
        return e;
    };
#define RK(call)                                \
    do {                                        \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) return unwind(e_); \
    } while (0)
#define RS(call)                                                    \
    do {                                                            \
        if ((call) != SN_OK) return unwind(cudaErrorUnknown);       \
    } while (0)
    RK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
    open = 1;
    RK(sn::ig_init(gd, gi, s0));
    m->ig_pro = sn::g_launches.load() - c0;
    cudaGraphConditionalHandle ho, hi;
    cudaGraph_t body_o = nullptr, body_i = nullptr;
    RK(new_handle(s0, 1, &ho));
    RK(add_while(s0, ho, &body_o));
    RK(cudaStreamBeginCaptureToGraph(s1, body_o, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    open = 2;
    const long long c1 = sn::g_launches.load();
    long long inner = 0;
    if (fg) {
        double* V = m->d_krylov;
        double* Z = V + (size_t)(k + 1) * M;
        double* w = Z + (size_t)k * M;
        double* part = w + M;
        double* hd = part + (size_t)(k + 1) * sn::krylov_blocks(M);
        double* tmp = m->d_work + 2 * (size_t)M;
        // cycle start: true residual w = b - S x with the fixed source, then V_0 = w / ||w||
        RS(transport_update(m, o, x, tmp, 1.0, s1, prec_res));
        RK(sn::launch_axpy_norm(m, tmp, x, w, m->d_scalars, s1));
        RK(new_handle(s1, 0, &hi));
        RK(sn::ig_gm_cycle_start(m->d_scalars, gd, gi, k, o->tol, o->max_iters, hist, hist_len, ho, hi, s1));
        RK(sn::launch_normalize(w, M, part, hd + 2 * (k + 1), V, s1));
        RK(add_while(s1, hi, &body_i));
        RK(cudaStreamBeginCaptureToGraph(s2, body_i, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        open = 3;
        const long long c2 = sn::g_launches.load();
        // Arnoldi step j: Z_j = P V_j (DSA step, Algorithm 2 or 1), w = S Z_j, two Gram-Schmidt passes
        RK(sn::ig_get_col(V, gi, 0, M, vt, s2));
        RK(sn::launch_copy(zt, vt, M, s2));
        if (dsa) {
            RK(sn::dsa_correct(m->dsa, vt, zt, o->inner_tol, o->inner_max_iters, false, s2));
            inner += sn::dsa_nested_prologue_launches(m->dsa);
            if (o->dsa == SN_DSA_TRIANGULAR) {
                double* tw = m->d_work;
                double* ty = m->d_work + M;
                RK(sn::dsa_select_thick(m->dsa, zt, tw, s2));
                RS(transport_update(m, o, tw, ty, 0.0, s2, prec_op));
                RK(sn::dsa_add_thin(m->dsa, ty, zt, s2));
            }
        }
        RK(sn::ig_set_col(Z, gi, M, zt, s2));
        RS(transport_update(m, o, zt, tmp, 0.0, s2, prec_op));
        RK(sn::launch_axpy_norm(m, zt, tmp, w, m->d_scalars, s2));
        RK(sn::launch_multidot_dev(V, gi + 1, 1, k + 1, M, w, part, hd, s2));
        RK(sn::launch_multiaxpy_dev(V, gi + 1, 1, M, hd, -1.0, w, s2));
        RK(sn::launch_multidot_dev(V, gi + 1, 1, k + 1, M, w, part, hd + (k + 1), s2));
        RK(sn::launch_multiaxpy_dev(V, gi + 1, 1, M, hd + (k + 1), -1.0, w, s2));
        RK(sn::launch_multidot(w, 1, M, w, part, hd + 2 * (k + 1), s2));
        RK(sn::ig_gm_arnoldi(hd, gd, gi, k, o->tol, o->max_iters, drop, hist, hist_len, hi, s2));
        RK(sn::ig_next_basis(w, gd, gi, M, V, s2));
        RK(cudaGetLastError());
        inner += sn::g_launches.load() - c2;
        {
            cudaGraph_t g2 = nullptr;
            open = 2;
            RK(cudaStreamEndCapture(s2, &g2));
        }
        // x += Z y with H y = g over the steps of this cycle
        RK(sn::ig_gm_solve(gd, gi, k, s1));
        RK(sn::launch_multiaxpy_dev(Z, gi + 2, 0, M, gd + sn::iter_graph_y_offset(k), 1.0, x, s1));
    } else {
        double* half = m->d_work;
        double* r = m->d_work + M;
        RK(sn::launch_sweep(m, x, o->precision, 1.0, s1));
        RK(sn::launch_phi_reduce(m, o->precision, x, half, m->d_scalars, s1));
        RK(sn::ig_si_residual(m->d_scalars, gd, gi, hist, hist_len, s1));
        if (dsa) {
            RK(sn::launch_axpy_norm(m, half, x, r, m->d_scalars + 1, s1));
            RK(sn::launch_copy(x, half, M, s1));
            if (o->dsa != SN_DSA_TRIANGULAR) {
                RK(sn::dsa_correct(m->dsa, r, x, o->inner_tol, o->inner_max_iters, false, s1));
                inner += sn::dsa_nested_prologue_launches(m->dsa);
            } else {
                double* tw = m->d_work + 2 * M;
                double* ty = m->d_work + 3 * M;
                RK(sn::dsa_select_thick(m->dsa, r, tw, s1));
                RK(sn::dsa_correct(m->dsa, r, tw, o->inner_tol, o->inner_max_iters, false, s1));
                inner += sn::dsa_nested_prologue_launches(m->dsa);
                RK(sn::launch_sweep(m, tw, o->precision, 0.0, s1));
                RK(sn::launch_phi_reduce(m, o->precision, nullptr, ty, nullptr, s1));
                RK(sn::dsa_tri_combine(m->dsa, tw, r, ty, x, s1));
            }
        } else {
            RK(sn::launch_copy(x, half, M, s1));
        }
        RK(sn::ig_si_end(gd, gi, o->tol, o->max_iters, ho, s1));
        if (o->checkpoint_every > 0)
            RK(sn::ig_si_checkpoint(x, o->checkpoints, M, gi, o->checkpoint_every, o->max_checkpoints, s1));
    }
    RK(cudaGetLastError());
    // the outer body's own kernels (the inner body counted apart, per Arnoldi step)
    const long long outer = sn::g_launches.load() - c1 - (fg ? inner - (dsa ? sn::dsa_nested_prologue_launches(m->dsa) : 0) : 0);
    {
        cudaGraph_t g2 = nullptr;
        open = 1;
        RK(cudaStreamEndCapture(s1, &g2));
    }
    open = 0;
    RK(cudaStreamEndCapture(s0, &graph));
#undef RK
#undef RS
    sn::g_launches.store(c0);  // recorded, not run
    if (m->iter_graph) cudaGraphExecDestroy(m->iter_graph);
    m->iter_graph = nullptr;
    err = cudaGraphInstantiate(&m->iter_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) {
        m->iter_graph = nullptr;
        cudaGetLastError();
        return err;
    }
    m->ig_outer = fg ? outer : outer + inner;
    m->ig_inner = fg ? inner : 0;
    return cudaSuccess;
}

// Solve by one launch of the recorded iteration.  Returns SN_ERR_NOT_CONVERGED like the host loops;
// *done = false when the iteration cannot be recorded (the caller then runs the host loop).
static sn_status run_recorded(sn_mesh* m, const sn_iter_opts* o, double* phi, sn_iter_stats* stats, cudaStream_t s,
                              std::chrono::steady_clock::time_point t0, bool* done) {
    *done = false;
    const bool fg = o->outer == SN_OUTER_FGMRES;
    const long long M = (long long)m->ne * m->n;
    const int hist_len = stats && stats->residual_history ? stats->history_len : 0;
    sn_status st;
    if (fg && (st = ensure_krylov(m, o->restart)) != SN_OK) return st;
    const size_t doubles = sn::iter_graph_doubles(60);
    const size_t need = doubles + (size_t)std::max(hist_len, 0);
    if (!m->d_ig || m->ig_doubles + (size_t)0 < doubles || need > m->ig_doubles + m->ig_hist_cap) {
        if (m->d_ig) {
            CK(cudaDeviceSynchronize(), "sync");
            cudaFree(m->d_ig);
        }
        m->d_ig = nullptr;
        m->ig_doubles = doubles;
        m->ig_hist_cap = std::max<size_t>(need - doubles, 1024);
        CK(cudaMalloc(&m->d_ig, (m->ig_doubles + m->ig_hist_cap) * sizeof(double)), "alloc iteration state");
    }
    if (!m->d_igi) CK(cudaMalloc(&m->d_igi, 8 * sizeof(int)), "alloc iteration state");
    if (!m->d_igv) CK(cudaMalloc(&m->d_igv, 3 * (size_t)M * sizeof(double)), "alloc iteration vectors");
    // set-up that allocates or launches work happens before the recording
    const bool mixed = o->precision == SN_FP32_MIXED;
    CK(sn::prepare_recorded_sweep(m, mixed ? SN_FP64 : o->precision, s), "operator cache");
    if (mixed) CK(sn::prepare_recorded_sweep(m, SN_FP32, s), "operator cache");
    if (o->dsa != SN_DSA_NONE && m->dsa) CK(sn::dsa_prepare(m->dsa, o->inner_tol), "DSA set-up");
    const std::vector<double> key = iteration_key(m, o, hist_len);
    if (!m->iter_graph || m->iter_key != key) {
        CK(cudaStreamSynchronize(s), "sync");
        m->capture_no_pdl = false;
        cudaError_t err = record_iteration(m, o, fg, hist_len);
        if (err != cudaSuccess) {  // e.g. programmatic edges inside conditional bodies: retry without
            m->capture_no_pdl = true;
            err = record_iteration(m, o, fg, hist_len);
            m->capture_no_pdl = false;
        }
        if (err != cudaSuccess) {
            sn::drop_iter_graph(m);
            cudaGetLastError();
            return SN_OK;  // not recordable here: the host loop runs instead
        }
        m->iter_key = key;
    }
    double* x = m->d_igv;
    if (o->warm_start) CK(cudaMemcpyAsync(x, phi, M * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    else CK(cudaMemsetAsync(x, 0, M * sizeof(double), s), "memset");
    const bool df = sn::dataflow_like(m->schedule);
    if (df) {  // every recorded sweep advances the device epoch once
        const long long most = 4ll * (o->max_iters + 2) + 8;  // at most 3 sweeps per iteration
        CK(sn::device_epoch_in(m, most, s), "epoch");
    }
    CK(cudaGraphLaunch(m->iter_graph, s), "recorded iteration");
    CK(cudaMemcpyAsync(phi, x, M * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    int hi[8] = {};
    double hd[4] = {};
    CK(cudaMemcpyAsync(hi, m->d_igi, sizeof(hi), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaMemcpyAsync(hd, m->d_ig, sizeof(hd), cudaMemcpyDeviceToHost, s), "copy");
    if (hist_len > 0)
        CK(cudaMemcpyAsync(stats->residual_history, m->d_ig + m->ig_doubles, hist_len * sizeof(double),
                           cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    *done = true;
    if (df) {
        CK(sn::device_epoch_out(m, s), "epoch");
        bool timed_out = false;
        CK(sn::take_sweep_error(m, s, &timed_out), "sweep status");
        if (timed_out) return fail(SN_ERR_TIMEOUT, "a sweep dependency wait timed out");
    }
    const int it = hi[0], cycles = hi[5];
    const bool converged = hi[3] != 0;
    if (hist_len > 0) {  // entries the solve did not reach stay zero, as in the host loops
        const int written = std::min(hist_len, fg ? it + 1 : it);
        for (int i = written; i < hist_len; ++i) stats->residual_history[i] = 0.0;
    }
    sn::g_launches.fetch_add(m->ig_pro + (fg ? (long long)(cycles + 1) * m->ig_outer + (long long)it * m->ig_inner
                                             : (long long)it * m->ig_outer),
                             std::memory_order_relaxed);
    int inner_total = 0;
    if (m->dsa) CK(sn::dsa_take_iters(m->dsa, s, &inner_total), "DSA iterations");
    const bool tri = o->dsa == SN_DSA_TRIANGULAR && m->dsa && sn::dsa_thick_count(m->dsa) > 0;
    if (stats) {
        stats->iters = it;
        stats->rel_residual = hd[1];
        stats->inner_iters_total = inner_total;
        stats->thick_fraction = m->dsa && o->dsa != SN_DSA_NONE ? (double)sn::dsa_thick_count(m->dsa) / m->ne : 0.0;
        stats->n_checkpoints = fg ? 0 : hi[6];
        stats->n_sweeps = fg ? (cycles + 1) + it * (tri ? 2 : 1) : it * (tri ? 2 : 1);
        stats->ms_sweep = 0.0;  // not split in a recorded solve (one graph launch)
        stats->ms_dsa = 0.0;
        stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!converged)
        return fail(SN_ERR_NOT_CONVERGED, "%s not converged after %d iterations (%.3e)", fg ? "fGMRES" : "source iteration",
                    it, hd[1]);
    return SN_OK;
}

sn_status sn_source_iterate(sn_mesh* m, const sn_iter_opts* o, double* phi, sn_iter_stats* stats, void* stream) {
    if (!m || !phi) return fail(SN_ERR_ARG, "null argument");
    sn_status st = check_opts(o);
    if (st != SN_OK) return st;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = check_shard(m, o)) != SN_OK) return st;
    if ((o->precision == SN_FP32 || o->precision == SN_FP32_MIXED) && (st = ensure_psi32(m)) != SN_OK) return st;
    if (o->dsa != SN_DSA_NONE && (st = ensure_dsa(m, o)) != SN_OK) return st;
    if (m->dsa) {  // the PCG iteration counter starts from zero for this solve
        int stale = 0;
        CK(sn::dsa_take_iters(m->dsa, (cudaStream_t)stream, &stale), "DSA iterations");
    }
    if (recordable(m, o)) {
        bool done = false;
        st = run_recorded(m, o, phi, stats, s, t0, &done);
        if (done || st != SN_OK) return st;
    }
    if (o->outer == SN_OUTER_FGMRES) {
        if (!o->warm_start) CK(cudaMemsetAsync(phi, 0, (size_t)m->ne * m->n * sizeof(double), s), "memset");
        return fgmres(m, o, phi, stats, s, t0);
    }
    const size_t M = (size_t)m->ne * m->n;
    double* half = m->d_work;
    double* r = m->d_work + M;
    if (!o->warm_start) CK(cudaMemsetAsync(phi, 0, M * sizeof(double), s), "memset");
    double r0 = 0.0, rel = INFINITY;
    int it = 0, inner_total = 0, nck = 0, extra_sweeps = 0;
    bool converged = false;
    SegmentClock sweep_clock, dsa_clock;
    const bool shard = sharded(o);
    while (it < o->max_iters) {
        sweep_clock.begin(s);
        if (!shard) {
            CK(sn::launch_sweep(m, phi, o->precision, 1.0, s), "sweep");
            CK(sn::launch_phi_reduce(m, o->precision, phi, half, m->d_scalars, s), "phi reduce");
        } else {
            if ((st = transport_update(m, o, phi, half, 1.0, s)) != SN_OK) return st;
            CK(sn::launch_axpy_norm(m, half, phi, r, m->d_scalars, s), "residual");
        }
        sweep_clock.end(s);
        double rr = 0.0;
        CK(cudaMemcpyAsync(&rr, m->d_scalars, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
        CK(cudaStreamSynchronize(s), "sync");
        sweep_clock.harvest();
        dsa_clock.harvest();
        if (m->schedule != sn::SCHED_LEVELS) {
            bool timed_out = false;
            CK(sn::take_sweep_error(m, s, &timed_out), "sweep status");
            if (timed_out) return fail(SN_ERR_TIMEOUT, "a sweep dependency wait timed out");
        }
        const double rn = std::sqrt(rr);
        if (it == 0) r0 = rn > 0 ? rn : 1.0;
        rel = rn / r0;
        if (stats && stats->residual_history && it < stats->history_len) stats->residual_history[it] = rel;
        if (o->dsa != SN_DSA_NONE && m->dsa && sn::dsa_thick_count(m->dsa) > 0) {
            CK(sn::launch_axpy_norm(m, half, phi, r, m->d_scalars + 1, s), "residual");
            CK(sn::launch_copy(phi, half, M, s), "copy");
            if (o->dsa != SN_DSA_TRIANGULAR) {
                dsa_clock.begin(s);
                CK(sn::dsa_correct(m->dsa, r, phi, o->inner_tol, o->inner_max_iters, false, s), "DSA");
                dsa_clock.end(s);
            } else {
                // Algorithm 1: w = E_f (r_f + D_ff^{-1} Sigma_f r_f) (step 1), y = zero-source transport
                // update of w (step 2); phi gets w - r on the thick DOFs and y on the thin ones
                double* w = m->d_work + 2 * M;
                double* y = m->d_work + 3 * M;
                CK(sn::dsa_select_thick(m->dsa, r, w, s), "Algorithm 1");
                dsa_clock.begin(s);
                CK(sn::dsa_correct(m->dsa, r, w, o->inner_tol, o->inner_max_iters, false, s), "DSA");
                dsa_clock.end(s);
                sweep_clock.begin(s);
                if ((st = transport_update(m, o, w, y, 0.0, s)) != SN_OK) return st;
                sweep_clock.end(s);
                CK(sn::dsa_tri_combine(m->dsa, w, r, y, phi, s), "Algorithm 1");
                ++extra_sweeps;
            }
        } else {
            CK(sn::launch_copy(phi, half, M, s), "copy");
        }
        ++it;
        if (o->checkpoint_every > 0 && it % o->checkpoint_every == 0 && nck < o->max_checkpoints) {
            CK(sn::launch_copy(o->checkpoints + (size_t)nck * M, phi, M, s), "checkpoint");
            ++nck;
        }
        if (rel <= o->tol) {
            converged = true;
            break;
        }
    }
    CK(cudaStreamSynchronize(s), "sync");
    sweep_clock.harvest();
    dsa_clock.harvest();
    if (m->dsa) CK(sn::dsa_take_iters(m->dsa, s, &inner_total), "DSA iterations");
    if (stats) {
        stats->iters = it;
        stats->rel_residual = rel;
        stats->inner_iters_total = inner_total;
        stats->thick_fraction = m->dsa && o->dsa != SN_DSA_NONE ? (double)sn::dsa_thick_count(m->dsa) / m->ne : 0.0;
        stats->n_checkpoints = nck;
        stats->n_sweeps = it + extra_sweeps;
        stats->ms_sweep = sweep_clock.ms;
        stats->ms_dsa = dsa_clock.ms;
        stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!converged) return fail(SN_ERR_NOT_CONVERGED, "not converged after %d iterations (rel. residual %.3e)", it, rel);
    return SN_OK;
}

sn_status sn_adjoint_sweep(sn_mesh* m, const double* mu, double* out, int precision, void* stream) {
    if (!m || !mu || !out) return fail(SN_ERR_ARG, "null argument");
    if (mu == out) return fail(SN_ERR_ARG, "mu_in and out must not alias");
    if (precision != SN_FP64) return fail(SN_ERR_ARG, "the adjoint sweep is float64 only");
    sn_status st = ensure_lambda(m);
    if (st != SN_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CK(sn::launch_adjoint_sweep(m, mu, s), "adjoint sweep");
    CK(sn::launch_adjoint_reduce(m, out, s), "adjoint reduce");
    if (m->schedule != sn::SCHED_LEVELS) {
        bool timed_out = false;
        CK(sn::take_sweep_error(m, s, &timed_out), "sweep status");
        if (timed_out) return fail(SN_ERR_TIMEOUT, "an adjoint sweep dependency wait timed out");
    }
    return SN_OK;
}

sn_status sn_adjoint_iterate(sn_mesh* m, const sn_iter_opts* o, const double* g, double* mu, sn_iter_stats* stats,
                             void* stream) {
    if (!m || !g || !mu) return fail(SN_ERR_ARG, "null argument");
    sn_status st = check_opts(o);
    if (st != SN_OK) return st;
    if (o->dsa == SN_DSA_TRIANGULAR) return fail(SN_ERR_ARG, "the adjoint iteration has no triangular DSA");
    if (sharded(o)) return fail(SN_ERR_ARG, "direction sharding is available in sn_source_iterate only");
    if ((st = ensure_lambda(m)) != SN_OK) return st;
    if (o->dsa != SN_DSA_NONE && (st = ensure_dsa_adjoint(m, o)) != SN_OK) return st;
    if (m->dsa) {  // the inner iteration counter starts from zero for this solve
        int stale = 0;
        CK(sn::dsa_take_iters(dsa_for(m, true), (cudaStream_t)stream, &stale), "DSA iterations");
    }
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    const size_t M = (size_t)m->ne * m->n;
    if (o->outer == SN_OUTER_FGMRES) {
        if (o->precision != SN_FP64) return fail(SN_ERR_ARG, "the adjoint solve is float64 only");
        if (!o->warm_start) CK(cudaMemsetAsync(mu, 0, M * sizeof(double), s), "memset");
        return fgmres(m, o, mu, stats, s, t0, true, g);
    }
    double* half = m->d_work;
    double* r = m->d_work + M;
    double* tmp = m->d_work + 2 * M;
    if (!o->warm_start) CK(cudaMemsetAsync(mu, 0, M * sizeof(double), s), "memset");
    double r0 = 0.0, rel = INFINITY;
    int it = 0, inner_total = 0;
    bool converged = false;
    SegmentClock sweep_clock, dsa_clock;
    while (it < o->max_iters) {
        sweep_clock.begin(s);
        CK(sn::launch_adjoint_sweep(m, mu, s), "adjoint sweep");
        CK(sn::launch_adjoint_reduce(m, tmp, s), "adjoint reduce");
        sweep_clock.end(s);
        // half = g + T^T mu ; r = half - mu
        CK(cudaMemcpyAsync(half, g, M * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
        CK(sn::launch_axpy_add(half, tmp, M, s), "axpy");
        CK(sn::launch_axpy_norm(m, half, mu, r, m->d_scalars, s), "residual");
        double rr = 0.0;
        CK(cudaMemcpyAsync(&rr, m->d_scalars, sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
        CK(cudaStreamSynchronize(s), "sync");
        sweep_clock.harvest();
        dsa_clock.harvest();
        const double rn = std::sqrt(rr);
        if (it == 0) r0 = rn > 0 ? rn : 1.0;
        rel = rn / r0;
        if (stats && stats->residual_history && it < stats->history_len) stats->residual_history[it] = rel;
        CK(sn::launch_copy(mu, half, M, s), "copy");
        if (o->dsa != SN_DSA_NONE && m->dsa && sn::dsa_thick_count(m->dsa) > 0) {
            dsa_clock.begin(s);
            CK(sn::dsa_correct(dsa_for(m, true), r, mu, o->inner_tol, o->inner_max_iters, true, s), "DSA");
            dsa_clock.end(s);
        }
        ++it;
        if (rel <= o->tol) {
            converged = true;
            break;
        }
    }
    CK(cudaStreamSynchronize(s), "sync");
    sweep_clock.harvest();
    dsa_clock.harvest();
    if (m->dsa) CK(sn::dsa_take_iters(dsa_for(m, true), s, &inner_total), "DSA iterations");
    if (stats) {
        stats->iters = it;
        stats->rel_residual = rel;
        stats->inner_iters_total = inner_total;
        stats->thick_fraction = m->dsa && o->dsa != SN_DSA_NONE ? (double)sn::dsa_thick_count(m->dsa) / m->ne : 0.0;
        stats->n_sweeps = it;
        stats->ms_sweep = sweep_clock.ms;
        stats->ms_dsa = dsa_clock.ms;
        stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    if (!converged) return fail(SN_ERR_NOT_CONVERGED, "adjoint not converged after %d iterations (%.3e)", it, rel);
    return SN_OK;
}

sn_status sn_gradients(sn_mesh* m, const double* phi, const double* mu, double* gt, double* gs, double* gq,
                       void* stream) {
    if (!m || !phi || !mu) return fail(SN_ERR_ARG, "null argument");
    sn_status st = ensure_lambda(m);
    if (st != SN_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    CK(sn::launch_sweep(m, phi, SN_FP64, 1.0, s), "sweep");
    CK(sn::launch_adjoint_sweep(m, mu, s), "adjoint sweep");
    CK(sn::launch_gradients(m, phi, gt, gs, gq, s), "gradients");
    return SN_OK;
}

// Reverse accumulation through K unaccelerated transport updates phi_{k+1} = T phi_k + b (see sn.h).
sn_status sn_unrolled_gradients(sn_mesh* m, const double* phi0, int K, int every, const double* checkpoints,
                                const double* g, double* gt, double* gs, double* gq, void* stream) {
    if (!m || !g) return fail(SN_ERR_ARG, "null argument");
    if (K < 1) return fail(SN_ERR_ARG, "K must be >= 1");
    if (every < 1) return fail(SN_ERR_ARG, "checkpoint_every must be >= 1");
    every = std::min(every, K);  // one segment either way; no workspace beyond K iterates
    sn_status st = ensure_lambda(m);
    if (st != SN_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t M = (size_t)m->ne * m->n, ne = (size_t)m->ne;
    const int nseg = (K + every - 1) / every;  // segment j starts at iterate j * every
    // workspace: phi_0 (when none is given), own checkpoints (when none are given), one segment of
    // iterates, two scratch vectors, two adjoint vectors, one step's gradients
    const size_t n_own = checkpoints ? 0 : (size_t)nseg * M;
    const size_t need = M + n_own + (size_t)every * M + 4 * M + 3 * ne;
    double* work = nullptr;
    CK(cudaMalloc(&work, need * sizeof(double)), "alloc unrolled-gradient workspace");
    std::unique_ptr<double, decltype(&cudaFree)> hold(work, &cudaFree);
    double* zero = work;
    double* own = zero + M;
    double* seg = own + n_own;
    double* scr = seg + (size_t)every * M;
    double* mu = scr + 2 * M;
    double* tg = mu + 2 * M;
    if (!phi0) {
        CK(cudaMemsetAsync(zero, 0, M * sizeof(double), s), "memset");
        phi0 = zero;
    }
    // iterate j * every: phi_0, then the caller's checkpoints (source iteration's, which hold
    // iterates every, 2 every, ...) or this call's own
    auto start = [&](int j) -> const double* {
        if (j == 0) return phi0;
        return checkpoints ? checkpoints + (size_t)(j - 1) * M : own + (size_t)j * M;
    };
    auto update = [&](const double* in, double* out) -> sn_status {  // out = T in + b
        CK(sn::launch_sweep(m, in, SN_FP64, 1.0, s), "sweep");
        CK(sn::launch_phi_reduce(m, SN_FP64, nullptr, out, nullptr, s), "phi reduce");
        return SN_OK;
    };
    if (!checkpoints) {  // forward pass keeping every `every`-th iterate below K
        const double* cur = phi0;
        for (int k = 0; k + 1 < K; ++k) {
            double* out = (k + 1) % every == 0 ? own + (size_t)((k + 1) / every) * M : scr + (size_t)(k % 2) * M;
            if ((st = update(cur, out)) != SN_OK) return st;
            cur = out;
        }
    }
    for (double* o : {gt, gs, gq})
        if (o) CK(cudaMemsetAsync(o, 0, ne * sizeof(double), s), "memset");
    double* mu_cur = mu;
    double* mu_next = mu + M;
    CK(cudaMemcpyAsync(mu_cur, g, M * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    for (int j = nseg - 1; j >= 0; --j) {
        const int base = j * every, end = std::min(K, base + every);
        // the segment's iterates, recomputed from its first
        CK(cudaMemcpyAsync(seg, start(j), M * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
        for (int i = 1; i < end - base; ++i)
            if ((st = update(seg + (size_t)(i - 1) * M, seg + (size_t)i * M)) != SN_OK) return st;
        for (int k = end - 1; k >= base; --k) {
            const double* phik = seg + (size_t)(k - base) * M;
            // update k at (phi_k, mu_{k+1}): psi of the update, lambda_d = w_d L_d^{-T} mu_{k+1}
            CK(sn::launch_sweep(m, phik, SN_FP64, 1.0, s), "sweep");
            CK(sn::launch_adjoint_sweep(m, mu_cur, s), "adjoint sweep");
            CK(sn::launch_gradients(m, phik, gt ? tg : nullptr, gs ? tg + ne : nullptr, gq ? tg + 2 * ne : nullptr, s),
               "gradients");
            if (gt) CK(sn::launch_axpy_add(gt, tg, ne, s), "accumulate");
            if (gs) CK(sn::launch_axpy_add(gs, tg + ne, ne, s), "accumulate");
            if (gq) CK(sn::launch_axpy_add(gq, tg + 2 * ne, ne, s), "accumulate");
            if (k > 0) {  // mu_k = T^T mu_{k+1}, from the same lambda
                CK(sn::launch_adjoint_reduce(m, mu_next, s), "adjoint reduce");
                std::swap(mu_cur, mu_next);
            }
        }
    }
    CK(cudaStreamSynchronize(s), "sync");
    if (m->schedule != sn::SCHED_LEVELS) {
        bool timed_out = false;
        CK(sn::take_sweep_error(m, s, &timed_out), "sweep status");
        if (timed_out) return fail(SN_ERR_TIMEOUT, "a sweep dependency wait timed out");
    }
    return SN_OK;
}

sn_status sn_dsa_apply(sn_mesh* m, const sn_iter_opts* o, const double* x, double* y, void* stream) {
    if (!m || !o || !x || !y) return fail(SN_ERR_ARG, "null argument");
    sn_iter_opts oo = *o;
    if (oo.dsa == SN_DSA_NONE) oo.dsa = SN_DSA_THICK;
    sn_status st = ensure_dsa(m, &oo);
    if (st != SN_OK) return st;
    CK(sn::dsa_apply(m->dsa, x, y, (cudaStream_t)stream), "DSA apply");
    return SN_OK;
}

sn_status sn_dsa_solve(sn_mesh* m, const sn_iter_opts* o, const double* b, double* x, int* iters, void* stream) {
    if (!m || !o || !b || !x) return fail(SN_ERR_ARG, "null argument");
    sn_iter_opts oo = *o;
    if (oo.dsa == SN_DSA_NONE) oo.dsa = SN_DSA_THICK;
    sn_status st = ensure_dsa(m, &oo);
    if (st != SN_OK) return st;
    int its = 0;
    CK(sn::dsa_take_iters(m->dsa, (cudaStream_t)stream, &its), "DSA iterations");  // drop earlier counts
    CK(sn::dsa_solve(m->dsa, b, x, oo.inner_tol, oo.inner_max_iters, (cudaStream_t)stream), "DSA solve");
    CK(sn::dsa_take_iters(m->dsa, (cudaStream_t)stream, &its), "DSA iterations");
    if (iters) *iters = its;
    return SN_OK;
}

sn_status sn_get_angular_flux(sn_mesh* m, int d, int adjoint, int precision, double* out, void* stream) {
    if (!m || !out) return fail(SN_ERR_ARG, "null argument");
    if (d < 0 || d >= m->nd) return fail(SN_ERR_ARG, "direction out of range");
    const size_t M = (size_t)m->ne * m->n;
    cudaStream_t s = (cudaStream_t)stream;
    if (adjoint) {
        if (!m->d_lambda) return fail(SN_ERR_ARG, "no adjoint sweep has run");
        CK(sn::launch_copy(out, m->d_lambda + (size_t)d * M, M, s), "copy");
    } else if (precision == SN_FP32) {
        if (!m->d_psi32) return fail(SN_ERR_ARG, "no FP32 sweep has run");
        CK(sn::launch_widen(out, static_cast<const float*>(m->d_psi32) + (size_t)d * M, M, s), "copy");
    } else {
        CK(sn::launch_copy(out, static_cast<const double*>(m->d_psi) + (size_t)d * M, M, s), "copy");
    }
    return SN_OK;
}

// ---------------------------------------------------------------- batches
static void free_batch(sn_batch* b) {
    if (!b) return;
    if (b->sweep_graph) cudaGraphExecDestroy(b->sweep_graph);
    if (b->iter_graph) cudaGraphExecDestroy(b->iter_graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void* p : {(void*)b->d_items, (void*)b->d_chunk_fam, (void*)b->d_args, (void*)b->d_done, (void*)b->d_done_off,
                    (void*)b->d_ctrl, (void*)b->d_active, (void*)b->d_phi, (void*)b->d_half, (void*)b->d_r,
                    (void*)b->d_rr, (void*)b->d_r0, (void*)b->d_iters, (void*)b->d_rel, (void*)b->d_next,
                    (void*)b->d_dof_inst})
        if (p) cudaFree(p);
    sn::union_dsa_free(b->dsa);
    sn::batch_krylov_free(b->kry);
    delete b;
}

sn_status sn_batch_create(sn_mesh* const* meshes, int count, sn_batch** out) {
    if (!meshes || !out || count < 1) return fail(SN_ERR_ARG, "need at least one mesh");
    *out = nullptr;
    std::unique_ptr<sn_batch, void (*)(sn_batch*)> b(new sn_batch(), free_batch);
    b->count = count;
    b->meshes.assign(meshes, meshes + count);
    long long off = 0;
    std::vector<int> dof_inst;
    for (int i = 0; i < count; ++i) {
        if (!meshes[i]) return fail(SN_ERR_ARG, "mesh %d is null", i);
        for (int j = 0; j < i; ++j)
            if (meshes[j] == meshes[i]) return fail(SN_ERR_ARG, "mesh %d appears twice", i);
        b->dof_off.push_back(off);
        const long long M = (long long)meshes[i]->ne * meshes[i]->n;
        dof_inst.insert(dof_inst.end(), M, i);
        off += M;
    }
    b->n_dof = off;
    CK(dalloc(&b->d_phi, off), "alloc");
    CK(dalloc(&b->d_half, off), "alloc");
    CK(dalloc(&b->d_r, off), "alloc");
    CK(dalloc(&b->d_dof_inst, off), "alloc");
    CK(cudaMemcpy(b->d_dof_inst, dof_inst.data(), off * sizeof(int), cudaMemcpyHostToDevice), "copy");
    CK(dalloc(&b->d_rr, count), "alloc");
    CK(dalloc(&b->d_r0, count), "alloc");
    CK(dalloc(&b->d_rel, count), "alloc");
    CK(dalloc(&b->d_iters, count), "alloc");
    CK(dalloc(&b->d_active, count), "alloc");
    CK(dalloc(&b->d_next, count), "alloc");
    CK(cudaMemset(b->d_phi, 0, off * sizeof(double)), "memset");
    CK(sn::batch_build_worklist(b.get(), 0), "batch work list");
    CK(cudaDeviceSynchronize(), "setup");
    *out = b.release();
    return SN_OK;
}

sn_status sn_batch_destroy(sn_batch* b) {
    if (!b) return SN_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    return SN_OK;
}

sn_status sn_batch_set_schedule(sn_batch* b, int schedule, int block, int max_blocks_per_sm) {
    if (!b) return fail(SN_ERR_ARG, "null batch");
    if (schedule != sn::SCHED_LEVELS && !sn::dataflow_like(schedule)) return fail(SN_ERR_ARG, "bad schedule");
    if (block < 32 || block > 128 || block % 32) return fail(SN_ERR_ARG, "block must be 32, 64, 96 or 128");
    if (max_blocks_per_sm < 0) return fail(SN_ERR_ARG, "max_blocks_per_sm must be >= 0");
    if (b->schedule != schedule || b->block != block || b->max_blocks_per_sm != max_blocks_per_sm) {
        if (b->sweep_graph) cudaGraphExecDestroy(b->sweep_graph);
        if (b->iter_graph) cudaGraphExecDestroy(b->iter_graph);
        b->sweep_graph = b->iter_graph = nullptr;
        ++b->graph_gen;
    }
    b->schedule = schedule;
    b->block = block;
    b->max_blocks_per_sm = max_blocks_per_sm;
    return SN_OK;
}

static sn_status batch_prepare(sn_batch* b, int precision, cudaStream_t s) {
    for (sn_mesh* m : b->meshes)
        if (precision == SN_FP32) {
            sn_status st = ensure_psi32(m);
            if (st != SN_OK) return st;
        }
    CK(sn::batch_refresh_cache(b, precision, s), "operator cache");
    return SN_OK;
}

static sn_status batch_timeout_check(sn_batch* b, cudaStream_t s) {
    unsigned long long w = 0;
    CK(cudaMemcpyAsync(&w, b->d_ctrl + 1, sizeof(w), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    if (w) {
        CK(cudaMemsetAsync(b->d_ctrl + 1, 0, sizeof(w), s), "memset");
        return fail(SN_ERR_TIMEOUT, "a batched sweep dependency wait timed out");
    }
    return SN_OK;
}

sn_status sn_batch_sweep(sn_batch* b, const double* const* phi_in, double* const* phi_out, int precision, void* stream) {
    if (!b || !phi_out) return fail(SN_ERR_ARG, "null argument");
    if (precision < SN_FP64 || precision > SN_FP32_REFINE) return fail(SN_ERR_ARG, "bad precision");
    cudaStream_t s = (cudaStream_t)stream;
    sn_status st = batch_prepare(b, precision, s);
    if (st != SN_OK) return st;
    for (int i = 0; i < b->count; ++i) {
        const size_t M = (size_t)b->meshes[i]->ne * b->meshes[i]->n;
        if (phi_in && phi_in[i])
            CK(cudaMemcpyAsync(b->d_phi + b->dof_off[i], phi_in[i], M * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
        else
            CK(cudaMemsetAsync(b->d_phi + b->dof_off[i], 0, M * sizeof(double), s), "memset");
    }
    std::vector<int> ones(b->count, 1);
    CK(cudaMemcpyAsync(b->d_active, ones.data(), b->count * sizeof(int), cudaMemcpyHostToDevice, s), "copy");
    if (sn::dataflow_like(b->schedule)) {
        CK(sn::batch_launch_dataflow(b, precision, s), "batched sweep");
    } else {
        CK(sn::batch_enqueue_sweep(b, precision, s), "batched sweep");
    }
    for (int i = 0; i < b->count; ++i)
        CK(sn::launch_phi_reduce(b->meshes[i], precision, nullptr, phi_out[i], nullptr, s), "phi reduce");
    if (sn::dataflow_like(b->schedule)) return batch_timeout_check(b, s);
    CK(cudaStreamSynchronize(s), "sync");
    return SN_OK;
}

static sn_status batch_ensure_dsa(sn_batch* b, const sn_iter_opts* o) {
    if (o->dsa == SN_DSA_TRIANGULAR) return fail(SN_ERR_ARG, "batches use the diagonal (Algorithm 2) DSA only");
    if (o->dsa_operator != SN_DSA_OP_SIP) return fail(SN_ERR_ARG, "batches use the symmetric (SIP) DSA operator only");
    std::vector<std::vector<unsigned char>> masks(b->count);
    for (int i = 0; i < b->count; ++i) {
        sn_iter_opts oi = *o;
        if (o->thick_rule == SN_THICK_MASK) return fail(SN_ERR_ARG, "explicit masks are not supported for batches");
        sn_status st = thick_mask_for(b->meshes[i], &oi, masks[i]);
        if (st != SN_OK) return st;
    }
    if (b->dsa && b->dsa_masks == masks && b->dsa_sigma == o->dsa_sigma) return SN_OK;
    sn::union_dsa_free(b->dsa);
    b->dsa = nullptr;
    std::vector<sn::DsaHierarchy*> parts;
    std::string err;
    for (int i = 0; i < b->count; ++i) {
        sn::DsaHierarchy* H = sn::dsa_build(b->meshes[i], masks[i].data(), o->dsa_sigma, SN_DSA_OP_SIP, false, err);
        if (!H) {
            for (sn::DsaHierarchy* P : parts) sn::dsa_free(P);
            return fail(SN_ERR_ARG, "DSA setup of instance %d: %s", i, err.c_str());
        }
        parts.push_back(H);
    }
    b->dsa = sn::union_dsa_build(parts, b->dof_off, err);
    if (!err.empty()) {
        sn::union_dsa_free(b->dsa);
        b->dsa = nullptr;
        return fail(SN_ERR_CUDA, "batched DSA upload: %s", err.c_str());
    }
    b->dsa_masks = masks;
    b->dsa_sigma = o->dsa_sigma;
    if (b->iter_graph) {
        cudaGraphExecDestroy(b->iter_graph);
        b->iter_graph = nullptr;
    }
    ++b->graph_gen;
    return SN_OK;
}

// Flexible GMRES(restart) of every instance at once (sn_batch_krylov.cu) from the iterates in
// b->d_phi; the solutions are copied to phis.
static sn_status batch_fgmres_solve(sn_batch* b, const sn_iter_opts* o, double* const* phis, sn_iter_stats* stats,
                                    cudaStream_t s, std::chrono::steady_clock::time_point t0) {
    std::vector<int> iters, sweeps, conv;
    std::vector<double> rel;
    CK(sn::batch_fgmres(b, o, s, iters, rel, sweeps, conv), "batched fGMRES");
    if (sn::dataflow_like(b->schedule)) {
        sn_status st = batch_timeout_check(b, s);
        if (st != SN_OK) return st;
    }
    for (int i = 0; i < b->count; ++i) {
        const size_t M = (size_t)b->meshes[i]->ne * b->meshes[i]->n;
        CK(cudaMemcpyAsync(phis[i], b->d_phi + b->dof_off[i], M * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    }
    CK(cudaStreamSynchronize(s), "sync");
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    bool all = true;
    for (int i = 0; i < b->count; ++i) {
        all &= conv[i] != 0;
        if (stats) {
            stats[i].iters = iters[i];
            stats[i].rel_residual = rel[i];
            stats[i].inner_iters_total = 0;
            stats[i].thick_fraction = 0.0;
            stats[i].n_checkpoints = 0;
            stats[i].n_sweeps = sweeps[i];
            stats[i].ms_total = ms;
            stats[i].ms_sweep = stats[i].ms_dsa = 0.0;
        }
    }
    if (!all) return fail(SN_ERR_NOT_CONVERGED, "some batch instances did not converge in %d iterations", o->max_iters);
    return SN_OK;
}

sn_status sn_batch_source_iterate(sn_batch* b, const sn_iter_opts* o, double* const* phis, sn_iter_stats* stats,
                                  void* stream) {
    if (!b || !phis) return fail(SN_ERR_ARG, "null argument");
    sn_status st = check_opts(o);
    if (st != SN_OK) return st;
    if (o->precision == SN_FP32_MIXED) return fail(SN_ERR_ARG, "SN_FP32_MIXED is for single meshes");
    if (sharded(o)) return fail(SN_ERR_ARG, "batches shard by instance, not by direction");
    if (o->checkpoint_every > 0) return fail(SN_ERR_ARG, "checkpoints are not supported for batches");
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = batch_prepare(b, o->precision, s)) != SN_OK) return st;
    if (o->dsa != SN_DSA_NONE && (st = batch_ensure_dsa(b, o)) != SN_OK) return st;
    for (int i = 0; i < b->count; ++i) {
        const size_t M = (size_t)b->meshes[i]->ne * b->meshes[i]->n;
        if (o->warm_start)
            CK(cudaMemcpyAsync(b->d_phi + b->dof_off[i], phis[i], M * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
        else
            CK(cudaMemsetAsync(b->d_phi + b->dof_off[i], 0, M * sizeof(double), s), "memset");
    }
    if (o->outer == SN_OUTER_FGMRES) return batch_fgmres_solve(b, o, phis, stats, s, t0);
    std::vector<int> ones(b->count, 1);
    CK(cudaMemcpyAsync(b->d_active, ones.data(), b->count * sizeof(int), cudaMemcpyHostToDevice, s), "copy");
    CK(cudaMemsetAsync(b->d_iters, 0, b->count * sizeof(int), s), "memset");
    // one outer iteration of all instances is recorded once into a CUDA graph and replayed
    const bool same_key = b->iter_graph && b->g_prec == o->precision && b->g_sched == b->schedule &&
                          b->g_dsa == o->dsa && b->g_tol == o->tol && b->g_inner_tol == o->inner_tol &&
                          b->g_inner_max == o->inner_max_iters && b->g_max_iters == o->max_iters;
    if (!same_key) {
        if (b->iter_graph) cudaGraphExecDestroy(b->iter_graph);
        b->iter_graph = nullptr;
        if (!b->cap_stream) CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking), "stream");
        CK(cudaStreamSynchronize(s), "sync");
        // the argument table is switched to this precision before recording (host copies stay out)
        CK(sn::batch_set_precision(b, o->precision, s), "precision");
        CK(cudaStreamSynchronize(s), "sync");
        CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal), "capture");
        cudaError_t qerr = sn::batch_enqueue_iteration(b, o, b->d_next, b->d_dof_inst, b->cap_stream);
        cudaGraph_t graph = nullptr;
        cudaError_t err = cudaStreamEndCapture(b->cap_stream, &graph);
        if (qerr != cudaSuccess) err = qerr;
        if (err == cudaSuccess) err = cudaGraphInstantiate(&b->iter_graph, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (err != cudaSuccess) {
            b->iter_graph = nullptr;
            return cuda_fail(err, "capture of the batched iteration");
        }
        b->g_prec = o->precision;
        b->g_sched = b->schedule;
        b->g_dsa = o->dsa;
        b->g_tol = o->tol;
        b->g_inner_tol = o->inner_tol;
        b->g_inner_max = o->inner_max_iters;
        b->g_max_iters = o->max_iters;
    }
    const int check_every = 4;
    std::vector<int> active(b->count);
    int launches = 0;
    bool any = true;
    while (any && launches < o->max_iters) {
        CK(cudaGraphLaunch(b->iter_graph, s), "graph launch");
        ++launches;
        if (launches % check_every == 0 || launches == o->max_iters) {
            CK(cudaMemcpyAsync(active.data(), b->d_active, b->count * sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
            CK(cudaStreamSynchronize(s), "sync");
            any = false;
            for (int a : active) any |= a != 0;
        }
    }
    if (sn::dataflow_like(b->schedule) && (st = batch_timeout_check(b, s)) != SN_OK) return st;
    for (int i = 0; i < b->count; ++i) {
        const size_t M = (size_t)b->meshes[i]->ne * b->meshes[i]->n;
        CK(cudaMemcpyAsync(phis[i], b->d_phi + b->dof_off[i], M * sizeof(double), cudaMemcpyDeviceToDevice, s), "copy");
    }
    std::vector<int> iters(b->count);
    std::vector<double> rel(b->count);
    CK(cudaMemcpyAsync(iters.data(), b->d_iters, b->count * sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaMemcpyAsync(rel.data(), b->d_rel, b->count * sizeof(double), cudaMemcpyDeviceToHost, s), "copy");
    CK(cudaStreamSynchronize(s), "sync");
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    bool all = true;
    for (int i = 0; i < b->count; ++i) {
        const bool conv = rel[i] <= o->tol;
        all &= conv;
        if (stats) {
            stats[i].iters = iters[i];
            stats[i].rel_residual = rel[i];
            stats[i].inner_iters_total = 0;
            stats[i].thick_fraction = 0.0;
            stats[i].n_checkpoints = 0;
            stats[i].n_sweeps = iters[i];
            stats[i].ms_total = ms;
            stats[i].ms_sweep = stats[i].ms_dsa = 0.0;  // one recorded iteration for all instances: no split
        }
    }
    if (!all) return fail(SN_ERR_NOT_CONVERGED, "some batch instances did not converge in %d iterations", o->max_iters);
    return SN_OK;
}

// ---------------------------------------------------------------- schedule autotuner
}  // extern "C"

namespace {
struct TuneKey {
    int kind, dim, p, nd, precision;
    long long size;
    bool operator<(const TuneKey& o) const {
        return std::tie(kind, dim, p, nd, precision, size) < std::tie(o.kind, o.dim, o.p, o.nd, o.precision, o.size);
    }
};
struct TuneChoice {
    int schedule, block, cap;
    float ms;
};
std::map<TuneKey, TuneChoice> g_tune_cache;
std::mutex g_tune_mutex;
const TuneChoice kCandidates[] = {{0, 32, 0, 0}, {0, 64, 0, 0}, {0, 128, 0, 0}, {4, 32, 0, 0}, {4, 64, 0, 0},
                                  {4, 128, 0, 0}, {1, 128, 0, 0},
                                  {1, 128, 1, 0}, {1, 64, 2, 0}, {1, 32, 4, 0}};
// meshes also try the tiled schedule (cached solves) with a few tile edges and CTA sizes
const TuneChoice kMeshCandidates[] = {{0, 32, 0, 0}, {0, 64, 0, 0}, {0, 128, 0, 0}, {0, 32, 2, 0},
                                      {0, 32, 4, 0}, {0, 64, 8, 0}, {1, 128, 0, 0}, {1, 64, 2, 0},
                                      {2, 128, 8, 0}, {2, 256, 16, 0}, {3, 256, 1, 0}, {3, 512, 1, 0},
                                      {3, 256, 2, 0}, {3, 128, 4, 0}, {4, 128, 0, 0}, {4, 64, 0, 0},
                                      {4, 128, 4, 0}, {4, 128, 2, 0}, {4, 32, 0, 0}};

template <typename F>
float time_ms(F&& run, cudaStream_t s, int reps) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    run();  // warm-up (also records graphs)
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a, s);
        run();
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        best = std::min(best, ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}
}  // namespace

extern "C" {

sn_status sn_mesh_autotune(sn_mesh* m, int precision, void* stream, int* schedule, int* block, int* cap) {
    if (!m) return fail(SN_ERR_ARG, "null mesh");
    if (precision < SN_FP64 || precision > SN_FP32_REFINE) return fail(SN_ERR_ARG, "bad precision");
    cudaStream_t s = (cudaStream_t)stream;
    const TuneKey key{0, m->dim, m->p, m->nd, precision, (long long)m->ne};
    TuneChoice best{-1, 0, 0, 1e30f};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) best = it->second;
    }
    if (best.schedule < 0) {
        if (precision == SN_FP32) {
            sn_status st = ensure_psi32(m);
            if (st != SN_OK) return st;
        }
        double* out = m->d_work + 3 * (size_t)m->ne * m->n;
        for (const TuneChoice& c : kMeshCandidates) {
            sn_status st = sn_mesh_set_schedule(m, c.schedule, c.block, c.cap);
            if (st != SN_OK) return st;
            cudaError_t err = cudaSuccess;
            const float ms = time_ms([&] {
                if (err == cudaSuccess) err = sn::launch_sweep(m, nullptr, precision, 1.0, s);
                if (err == cudaSuccess) err = sn::launch_phi_reduce(m, precision, nullptr, out, nullptr, s);
            }, s, 2);
            CK(err, "autotune sweep");
            if (m->schedule != sn::SCHED_LEVELS) {
                bool timed_out = false;
                CK(sn::take_sweep_error(m, s, &timed_out), "sweep status");
                if (timed_out) return fail(SN_ERR_TIMEOUT, "a sweep dependency wait timed out while tuning");
            }
            if (ms < best.ms) best = {c.schedule, c.block, c.cap, ms};
        }
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = best;
    }
    sn_status st = sn_mesh_set_schedule(m, best.schedule, best.block, best.cap);
    if (st != SN_OK) return st;
    if (schedule) *schedule = best.schedule;
    if (block) *block = best.block;
    if (cap) *cap = best.cap;
    return SN_OK;
}

sn_status sn_batch_autotune(sn_batch* b, int precision, void* stream, int* schedule, int* block, int* cap) {
    if (!b) return fail(SN_ERR_ARG, "null batch");
    if (precision < SN_FP64 || precision > SN_FP32_REFINE) return fail(SN_ERR_ARG, "bad precision");
    cudaStream_t s = (cudaStream_t)stream;
    sn_status st = batch_prepare(b, precision, s);
    if (st != SN_OK) return st;
    std::vector<int> ones(b->count, 1);
    CK(cudaMemcpyAsync(b->d_active, ones.data(), b->count * sizeof(int), cudaMemcpyHostToDevice, s), "copy");
    CK(cudaMemsetAsync(b->d_phi, 0, (size_t)b->n_dof * sizeof(double), s), "memset");
    TuneChoice best{-1, 0, 0, 1e30f};
    for (const TuneChoice& c : kCandidates) {
        if ((st = sn_batch_set_schedule(b, c.schedule, c.block, c.cap)) != SN_OK) return st;
        cudaError_t err = cudaSuccess;
        const float ms = time_ms([&] {
            if (err != cudaSuccess) return;
            err = sn::dataflow_like(b->schedule) ? sn::batch_launch_dataflow(b, precision, s)
                                                    : sn::batch_enqueue_sweep(b, precision, s);
        }, s, 2);
        CK(err, "autotune batched sweep");
        if (sn::dataflow_like(b->schedule) && (st = batch_timeout_check(b, s)) != SN_OK) return st;
        if (ms < best.ms) best = {c.schedule, c.block, c.cap, ms};
    }
    if ((st = sn_batch_set_schedule(b, best.schedule, best.block, best.cap)) != SN_OK) return st;
    if (schedule) *schedule = best.schedule;
    if (block) *block = best.block;
    if (cap) *cap = best.cap;
    return SN_OK;
}

}  // extern "C"
