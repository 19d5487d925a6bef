// Internal declarations of libsn (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sn.h"

namespace sn {

constexpr int kMaxP = 3;

// Number of kernels this library has launched (reported by sn_launch_count).
extern std::atomic<long long> g_launches;
#define SN_COUNT_LAUNCH() (::sn::g_launches.fetch_add(1, std::memory_order_relaxed))
constexpr double kFourPi = 12.566370614359172953850573533118;

// 1D Gauss-Legendre nodal data for one polynomial order p (p+1 nodes).
struct GL1D {
    int p = 0;
    double x[kMaxP + 1] = {};               // nodes on [-1, 1]
    double w[kMaxP + 1] = {};               // weights
    double lm[kMaxP + 1] = {};              // l_k(-1)
    double lp[kMaxP + 1] = {};              // l_k(+1)
    double dm[kMaxP + 1][kMaxP + 1] = {};   // dm[a][k] = l_k'(x_a)
    double dlm[kMaxP + 1] = {};             // l_k'(-1)
    double dlp[kMaxP + 1] = {};             // l_k'(+1)
};

GL1D gauss_legendre_nodal(int p);
void lagrange_eval(const GL1D& g, double t, double* val, double* der);

// Level-symmetric S_N set; returns false for an unsupported order.
bool level_symmetric(int N, int dim, std::vector<double>& dirs, std::vector<double>& wts);

// Directed graph helpers of the tiled schedule (host).  to_csr sorts and de-duplicates the edges
// (source, target) and builds the CSR arrays ptr (n + 1) and adj; strong_components labels every
// vertex with its strongly connected component (comp, n values) and returns how many there are.
void to_csr(int n, std::vector<std::pair<int, int>>& edges, std::vector<int>& ptr, std::vector<int>& adj);
int strong_components(int n, const std::vector<int>& ptr, const std::vector<int>& adj, std::vector<int>& comp);

// Everything a sweep kernel reads, by value.
struct SweepArgs {
    int dim, p, nx, ny, nz, ne, nd;
    double hx, hy, hz;              // 3D uniform spacing
    double psi_inc;
    const double* dirs;             // nd x 3
    const double* corners;          // 2D: ne x 8 = (x00,y00,x10,y10,x01,y01,x11,y11); 3D: null
    const double* sigma_t;
    const double* sigma_s;
    const double* q;
    const double* phi;              // scattering source (nodal), may be null (= 0)
    const double* mass;             // ne x n collocated masses W_i det J(x_i)
    const double* mass4;            // the same divided by 4 pi (the scale of a source row)
    void* psi;                      // nd x ne x n, float64 or float32
    const int2* items;              // (dir, elem) sorted by level
    double q_scale;                 // 1 normally, 0 for homogeneous solves (q and q32 are then null)
    const double* ainv;             // operator cache: nd x ne inverses A_e^{-1} (float64), or null
    const float* ainv32;            // the same rounded to float32 (FP32 form), or null
    const double* fflux;            // face flux factors beside the cache: 2D nd x ne x 4, 3D nd x 3 (b_x, b_y, b_z)
    // float32 copies read by the FP32 cached solves (built with the float32 cache): face flux
    // factors (as fflux), q per element, mass / (4 pi) per node; q32 is null for the linear part
    // of the update (no fixed source)
    const float* fflux32;
    const float* q32;
    const float* mass32;
};

// Entries of one cached inverse: N*N rounded up to a multiple of 4 (16-byte vector loads).  The
// inverse is stored column-major: entry (i, j) of A_e^{-1} at [j * N + i].
inline int cache_stride(int dim, int p) {
    const int q = p + 1, n = dim == 2 ? q * q : q * q * q;
    return (n * n + 3) & ~3;
}

// Persistent dataflow sweep: padded work list and completion words.
struct DataflowArgs {
    const int2* items;               // chunks of 32 items, each chunk inside one level; padding = (-1, -1)
    long long n_items;               // multiple of 32
    int* done;                       // nd x ne completion epochs
    int epoch;                       // value that marks "done in this sweep"
    int publish;                     // value an item writes when done (== epoch except in the stall test)
    unsigned long long* next;        // chunk counter, zeroed before each launch
    int* error;                      // set to 1 when a wait times out
    unsigned long long timeout_ns;   // per-launch wait budget
    long long static_warps;          // > 0: static assignment, warp w takes slices w, w + static_warps, ...
                                     // (every warp of the grid resident); 0: slices claimed from `next`
    const int* epoch_dev;            // non-null (recorded sweeps): epoch and publish value read here
};

struct LevelSets {
    std::vector<long long> level_ptr;   // host copy, n_levels + 1
    int2* items = nullptr;              // device, sorted by (level, dir, elem)
    int n_levels = 0;
    int2* padded = nullptr;             // device, each level padded to a multiple of 32 with (-1, -1)
    long long n_padded = 0;
    int2* padded_rev = nullptr;         // device, levels in reverse order (adjoint), padded the same way
    int* done = nullptr;                // device, nd x ne completion epochs (dataflow schedule)
    unsigned long long* ctrl = nullptr; // device: [0] chunk counter, [1] error word
    int epoch = 0;
    double stall_timeout_s = 0.0;       // > 0: the next dataflow sweep publishes a value nobody waits for
    std::vector<int> h_level;           // host copy of the level of every (dir, elem), dir-major
    long long* d_level_ptr = nullptr;   // device copy of level_ptr (level-barrier schedule)
    int* d_barrier = nullptr;           // arrival counter of the level-barrier schedule
    // direction groups of the level schedule: group g sweeps directions [g nd / G, (g + 1) nd / G)
    // as its own chain of level launches (items sorted by (group, level, dir, elem))
    int groups = 0;                     // G the group lists were built for (0: not built)
    int2* gitems = nullptr;
    std::vector<std::vector<long long>> gptr;  // per group: level boundaries into gitems
    std::vector<cudaStream_t> gstreams;        // fork/join streams of the captured graph
    std::vector<cudaEvent_t> gevents;          // [0] fork, [1 + g] join of group g
};

enum { SCHED_LEVELS = 0, SCHED_DATAFLOW = 1, SCHED_TILES = 2, SCHED_BARRIER = 3, SCHED_STATIC = 4 };
// Schedules whose kernels wait (bounded) on completion words of the dataflow kind.
inline bool dataflow_like(int schedule) { return schedule == SCHED_DATAFLOW || schedule == SCHED_STATIC; }

// Tiled schedule of the cached sweep: the mesh is cut into tiles of edge^dim elements; per
// direction, the tiles of every strongly connected component of the tile upwind graph form one
// task (a component of several tiles appears only where vertex jitter reverses faces on a tile
// boundary), and tasks are listed in a topological order of the component graph.  A CTA runs a
// task's elements in increasing global level, synchronising the CTA between levels, and waits
// (bounded) on the completion words of upwind elements in other tasks.
struct TileSets {
    int edge = 0;                       // tile edge the tasks were built for (0: not built)
    int4* tasks = nullptr;              // device: (direction, first item, first level boundary, levels)
    int* lvl_ptr = nullptr;             // device: item offsets of every task's local levels
    int2* items = nullptr;              // device: (element, flags) flags bit f < 6: wait for the upwind
                                        // neighbour through face f; bit 6: publish the completion word
    long long n_tasks = 0;
    int max_level_items = 0;            // largest local level of any task
};
constexpr int kTileWaitMask = 63, kTilePublish = 64;

struct DsaHierarchy;  // sn_dsa.cu
struct UnionDsa;      // sn_batch.cu
struct BatchKrylov;   // sn_batch_krylov.cu

// Element families a batch can mix; a 32-item chunk of the batched work list never mixes them.
enum { FAM_2D_P1 = 0, FAM_2D_P2 = 1, FAM_2D_P3 = 2, FAM_3D_P1 = 3, FAM_COUNT = 4 };
inline int family_of(int dim, int p) { return dim == 3 ? FAM_3D_P1 : p - 1; }
inline int family_nodes(int fam) { return fam == FAM_3D_P1 ? 8 : (fam + 2) * (fam + 2); }

// Batched work item: instance, direction, element, family.
struct BatchItem {
    int inst, dir, elem, fam;
};

}  // namespace sn

struct sn_mesh {
    sn_mesh_desc desc{};
    int dim = 2, p = 1, n = 4, ne = 0, nd = 0;
    int nx = 0, ny = 0, nz = 1;
    double hx = 0, hy = 0, hz = 0;
    std::vector<double> h_dirs, h_wts, h_corners;
    std::vector<double> h_sigma_t, h_sigma_s, h_q;  // host mirrors for setup
    double* d_dirs = nullptr;
    double* d_wts = nullptr;
    double* d_corners = nullptr;
    double* d_sigma_t = nullptr;
    double* d_sigma_s = nullptr;
    double* d_q = nullptr;
    void* d_psi = nullptr;          // forward angular fluxes (float64 storage)
    void* d_psi32 = nullptr;        // float32 angular fluxes of the FP32 form
    double* d_lambda = nullptr;     // adjoint angular fluxes
    double* d_mass = nullptr;       // ne x n collocated masses
    double* d_mass4 = nullptr;      // the same divided by 4 pi
    double* d_work = nullptr;       // 4 x ne x n scratch vectors for iterations
    double* d_red = nullptr;        // reduction partials
    int red_blocks = 0;
    double* d_scalars = nullptr;    // small device scalars
    sn::LevelSets levels;
    sn::TileSets tiles;
    int schedule = sn::SCHED_LEVELS;    // sweep schedule (see sn_mesh_set_schedule)
    int level_groups = 1;               // direction groups of the level schedule (parallel chains)
    int tile_edge = 16;                 // tile edge of the tiled schedule
    int tile_block = 128;               // threads per CTA of the tiled schedule
    int barrier_block = 256;            // threads per CTA of the level-barrier schedule
    int barrier_ctas_per_sm = 1;        // CTAs per SM of the level-barrier schedule
    int block = 128;                    // threads per block of the sweep kernels
    int max_blocks_per_sm = 0;          // 0: occupancy limit
    int cache_mode = SN_CACHE_AUTO;     // operator cache (see sn_mesh_set_operator_cache)
    double* d_ainv = nullptr;           // cached inverses, float64 (FP64 form and adjoint)
    float* d_ainv32 = nullptr;          // cached inverses, float32 (FP32 form)
    double* d_fflux = nullptr;          // face flux factors read with the cache (see SweepArgs::fflux)
    float* d_in32 = nullptr;            // float32 inputs of the FP32 cached solves (see SweepArgs::fflux32)
    bool ainv_valid = false, ainv32_valid = false;    // match the current materials
    bool ainv_denied = false, ainv32_denied = false;  // AUTO mode found no room for them
    double* d_src = nullptr;            // ne x n source vector read by the graph-captured level launches
    cudaGraphExec_t level_graph[7] = {};  // level-schedule sweeps: FP64, FP32, refine, adjoint, and the
                                          // three forward kinds without the fixed source
    cudaStream_t cap_stream = nullptr;  // private stream used only for graph capture
    sn::DsaHierarchy* dsa = nullptr;
    int2* range_items = nullptr;        // level work list of the direction range of sn_sweep_directions
    std::vector<long long> range_ptr;
    int range_d0 = -1, range_d1 = -1;
    sn::DsaHierarchy* dsa_t = nullptr;  // D_ff^T for the adjoint of a nonsymmetric operator (built on demand)
    double* d_krylov = nullptr;     // flexible GMRES workspace (basis, preconditioned basis, scratch)
    int krylov_restart = 0;
    // recorded outer iteration (one graph launch per solve; sn_api.cpp)
    cudaGraphExec_t iter_graph = nullptr;
    std::vector<double> iter_key;       // options and buffers the graph was recorded for
    long long ig_pro = 0, ig_outer = 0, ig_inner = 0;  // kernels in the prologue / outer body / inner body
    double* d_ig = nullptr;             // device scalars (sn_iter_graph.cu layout) + residual history
    int* d_igi = nullptr;               // device integers
    size_t ig_doubles = 0, ig_hist_cap = 0;
    double* d_igv = nullptr;            // 3 x ne x n: iterate, V_j copy, Z_j work vector
    cudaStream_t ig_stream[3] = {};     // capture streams: graph, outer body, inner body
    bool capture_no_pdl = false;        // record level chains without programmatic dependent launch
    int dsa_key_dsa = -1, dsa_key_rule = -1, dsa_key_sigma = -1, dsa_key_op = -1;
    double dsa_key_eta = 0;
    std::vector<unsigned char> dsa_key_mask;
};

struct sn_batch {
    std::vector<sn_mesh*> meshes;
    int count = 0;
    int precision = -1;                      // precision the graphs were captured for
    // batched work list: sorted by (level, family, instance, dir, elem); every (level, family)
    // segment padded to a multiple of 32 with inst = -1
    sn::BatchItem* d_items = nullptr;
    long long n_items = 0;
    std::vector<long long> seg_begin, seg_end;
    std::vector<int> seg_fam, seg_level;
    int* d_chunk_fam = nullptr;              // family of each 32-item chunk (dataflow)
    sn::SweepArgs* d_args = nullptr;         // per-instance sweep arguments (fixed pointers)
    std::vector<sn::SweepArgs> h_args;
    int* d_done = nullptr;                   // completion words, instance blocks at done_off
    long long* d_done_off = nullptr;
    unsigned long long* d_ctrl = nullptr;    // chunk counter, error word
    int epoch = 0;
    int* d_active = nullptr;                 // per instance: 1 = still iterating
    int schedule = 0, block = 64, max_blocks_per_sm = 0;
    bool cached = false;                     // every instance has an operator cache: node-per-lane kernels
    cudaGraphExec_t sweep_graph = nullptr;   // level schedule, all instances
    cudaGraphExec_t iter_graph = nullptr;    // one whole outer iteration
    long long graph_gen = 0;                 // advanced whenever recorded batch graphs go stale
    cudaStream_t cap_stream = nullptr;
    // concatenated iteration vectors (instance blocks at dof_off)
    std::vector<long long> dof_off;
    long long n_dof = 0;
    double *d_phi = nullptr, *d_half = nullptr, *d_r = nullptr;
    double* d_rr = nullptr;                  // per-instance squared residual norms
    double* d_r0 = nullptr;                  // per-instance first residual norm
    int* d_iters = nullptr;                  // per-instance iteration counts
    double* d_rel = nullptr;                 // per-instance last relative residual
    int* d_next = nullptr;                   // per-instance "iterate again" flags
    int* d_dof_inst = nullptr;               // instance of every concatenated DOF
    sn::UnionDsa* dsa = nullptr;
    sn::BatchKrylov* kry = nullptr;          // batched flexible GMRES workspace and graphs
    std::vector<std::vector<unsigned char>> dsa_masks;  // thick masks the union DSA was built for
    int dsa_sigma = -1;
    // key of the captured iteration graph
    int g_prec = -1, g_sched = -1, g_dsa = -1, g_inner_max = -1;
    double g_tol = -1, g_inner_tol = -1;
    int g_max_iters = -1;
};

namespace sn {
// Launch with programmatic stream serialisation when pdl is set: the kernel may start while its
// predecessor in the stream still runs (it waits in griddepcontrol.wait before reading the
// predecessor's results).  The first launch of a sequence passes pdl = false, so everything
// written before the sequence is complete before any of its kernels starts.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(bool pdl, void (*kernel)(KArgs...), unsigned grid, int block, cudaStream_t s,
                            Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

#ifdef __CUDACC__
// Programmatic dependent launch: a kernel does the work that reads nothing its predecessor writes
// before griddepcontrol.wait, which returns when every prerequisite grid has completed and its
// writes are visible; griddepcontrol.launch_dependents lets the next kernel in the stream start
// its own blocks.  Without a programmatic dependency both instructions do nothing.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

#endif

// sn_api.cpp: records the thread-local message returned by sn_last_error
sn_status set_error(sn_status st, const char* msg);
// sn_sweep.cu
cudaError_t build_levels(sn_mesh* m, cudaStream_t s, bool* cycle);
// group lists of the level schedule for G direction groups (needs the level sets)
cudaError_t build_level_groups(sn_mesh* m, int G);
void free_level_groups(sn_mesh* m);
// upwind face bits of every (dir, elem): bit f set when Omega.n_f < 0 and face f has a neighbour
cudaError_t launch_upwind_mask(sn_mesh* m, unsigned char* mask, cudaStream_t s);
// sn_tiles.cpp: builds m->tiles for tile edge `edge` (needs the level sets)
cudaError_t build_tiles(sn_mesh* m, int edge, cudaStream_t s);
void free_tiles(sn_mesh* m);
cudaError_t compute_mass(sn_mesh* m, cudaStream_t s);
void drop_level_graphs(sn_mesh* m);
void drop_iter_graph(sn_mesh* m);
cudaError_t prepare_recorded_sweep(sn_mesh* m, int precision, cudaStream_t s);
// batched sweep over all instances of a batch (sn_sweep.cu)
cudaError_t batch_build_worklist(sn_batch* b, cudaStream_t s);
// (args / mask: argument table and per-instance mask other than the batch's own, e.g. the
// homogeneous table of the batched fGMRES; null = b->d_args / b->d_active)
cudaError_t batch_enqueue_sweep(sn_batch* b, int precision, cudaStream_t s, const SweepArgs* args = nullptr,
                                const int* mask = nullptr);  // level schedule, capturable
cudaError_t batch_launch_dataflow(sn_batch* b, int precision, cudaStream_t s, const SweepArgs* args = nullptr,
                                  const int* mask = nullptr);
cudaError_t batch_set_precision(sn_batch* b, int precision, cudaStream_t s);
// union DSA of a batch (sn_batch.cu)
UnionDsa* union_dsa_build(const std::vector<DsaHierarchy*>& parts, const std::vector<long long>& dof_off,
                          std::string& err);
void union_dsa_free(UnionDsa* U);
long long union_dsa_rows(const UnionDsa* U);
int* union_dsa_iters(UnionDsa* U);
cudaError_t union_dsa_correct(UnionDsa* U, const double* r_all, double* phi_all, const int* active, double tol,
                              int max_iters, cudaStream_t s);
cudaError_t batch_enqueue_iteration(sn_batch* b, const sn_iter_opts* o, int* d_next, const int* d_dof_inst,
                                    cudaStream_t s);
// batched flexible GMRES (sn_batch_krylov.cu): per-instance Arnoldi steps, last relative
// residuals, transport updates and convergence flags
cudaError_t batch_fgmres(sn_batch* b, const sn_iter_opts* o, cudaStream_t s, std::vector<int>& iters,
                         std::vector<double>& rel, std::vector<int>& sweeps, std::vector<int>& conv);
void batch_krylov_free(BatchKrylov* K);
cudaError_t launch_sweep(sn_mesh* m, const double* phi_in, int precision, double q_scale, cudaStream_t s);
cudaError_t prepare_operator_cache(sn_mesh* m, int precision, cudaStream_t s);
void free_operator_cache(sn_mesh* m);
cudaError_t batch_refresh_cache(sn_batch* b, int precision, cudaStream_t s);
cudaError_t launch_adjoint_sweep(sn_mesh* m, const double* mu, cudaStream_t s);
// phi_out = sum_{d0 <= d < d1} w_d psi_d (d1 < 0: every direction), optional ||phi_out - phi_in||^2
cudaError_t launch_phi_reduce(sn_mesh* m, int precision, const double* phi_in, double* phi_out, double* d_rr,
                              cudaStream_t s, int d0 = 0, int d1 = -1);
// forward sweep of directions d0 <= d < d1 only (level chain on the stream, any schedule)
// (q_scale = 0: the linear part of the update, no fixed source and vacuum inflow)
cudaError_t launch_sweep_range(sn_mesh* m, const double* phi_in, int precision, int d0, int d1, cudaStream_t s,
                               double q_scale = 1.0);
cudaError_t launch_adjoint_reduce(sn_mesh* m, double* out, cudaStream_t s);
cudaError_t launch_gradients(sn_mesh* m, const double* phi, double* gt, double* gs, double* gq, cudaStream_t s);
cudaError_t launch_axpy_norm(sn_mesh* m, const double* a, const double* b, double* out, double* d_rr,
                             cudaStream_t s);
cudaError_t launch_copy(double* dst, const double* src, size_t n, cudaStream_t s);
// Reads and clears the dataflow error word (synchronises the stream).
cudaError_t take_sweep_error(sn_mesh* m, cudaStream_t s, bool* timed_out);
// device copy of the dataflow epoch around a recorded iteration (see sn_sweep.cu)
cudaError_t device_epoch_in(sn_mesh* m, long long max_sweeps, cudaStream_t s);
cudaError_t device_epoch_out(sn_mesh* m, cudaStream_t s);
cudaError_t launch_axpy_add(double* y, const double* x, size_t n, cudaStream_t s);  // y += x
// sn_materials.cu: per-element sigma_t, sigma_s, q of the pseudo-scattering time step
cudaError_t launch_pseudo_scattering(const double* sigma, const double* cv, const double* T, int ne, double dt,
                                     double a_rad, double c_light, double* sigma_t, double* sigma_s, double* q,
                                     cudaStream_t s);
cudaError_t launch_widen(double* y, const float* x, size_t n, cudaStream_t s);
// sn_krylov.cu
int krylov_blocks(long long n);
cudaError_t launch_multidot(const double* V, int k, long long n, const double* w, double* partial, double* h,
                            cudaStream_t s);
cudaError_t launch_multiaxpy(const double* V, int k, long long n, const double* c, double sign, double* w,
                             cudaStream_t s);
cudaError_t launch_normalize(const double* x, long long n, double* partial, double* s, double* y, cudaStream_t st);
// the same with the basis size k = *kdev + kofs read on the device (recorded fGMRES)
cudaError_t launch_multidot_dev(const double* V, const int* kdev, int kofs, int kmax, long long n, const double* w,
                                double* partial, double* h, cudaStream_t s);
cudaError_t launch_multiaxpy_dev(const double* V, const int* kdev, int kofs, long long n, const double* c, double sign,
                                 double* w, cudaStream_t s);
// sn_iter_graph.cu: device scalars of the recorded outer iterations (layout in that file)
size_t iter_graph_doubles(int k);
int iter_graph_y_offset(int k);
cudaError_t ig_init(double* gd, int* gi, cudaStream_t s);
cudaError_t ig_si_residual(const double* rr, double* gd, int* gi, double* hist, int hist_len, cudaStream_t s);
cudaError_t ig_si_end(double* gd, int* gi, double tol, int max_iters, cudaGraphConditionalHandle h, cudaStream_t s);
cudaError_t ig_si_checkpoint(const double* phi, double* ckpt, long long M, int* gi, int every, int max_ck,
                             cudaStream_t s);
cudaError_t ig_gm_cycle_start(const double* rr, double* gd, int* gi, int k, double tol, int max_iters, double* hist,
                              int hist_len, cudaGraphConditionalHandle outer, cudaGraphConditionalHandle inner,
                              cudaStream_t s);
cudaError_t ig_gm_arnoldi(const double* hd, double* gd, int* gi, int k, double tol, int max_iters, double drop,
                          double* hist, int hist_len, cudaGraphConditionalHandle inner, cudaStream_t s);
cudaError_t ig_gm_solve(double* gd, const int* gi, int k, cudaStream_t s);
cudaError_t ig_get_col(const double* V, const int* gi, int ofs, long long M, double* out, cudaStream_t s);
cudaError_t ig_set_col(double* V, const int* gi, long long M, const double* in, cudaStream_t s);
cudaError_t ig_next_basis(const double* w, const double* gd, const int* gi, long long M, double* V, cudaStream_t s);
// sn_dsa.cu
// Assembles D_ff (dsa_op: SN_DSA_OP_SIP / NIP / MNIP; transposed: D_ff^T, for the adjoint of a
// nonsymmetric operator) and its multigrid hierarchy.  Returns null with err set; *void_conflict
// is set when the operator is undefined next to a void element (mNIP, Eq. ModifiedF0).
DsaHierarchy* dsa_build(const sn_mesh* m, const unsigned char* mask, int dsa_sigma, int dsa_op, bool transposed,
                        std::string& err, bool* void_conflict = nullptr);
void dsa_free(DsaHierarchy* h);
int dsa_thick_count(const DsaHierarchy* h);
cudaError_t dsa_prepare(DsaHierarchy* h, double tol);
long long dsa_nested_prologue_launches(const DsaHierarchy* h);
// y = D_ff x (scatter into [elem][node], zeros elsewhere)
cudaError_t dsa_apply(DsaHierarchy* h, const double* x, double* y, cudaStream_t s);
// phi_out += E_f D_ff^{-1} Sigma_f r (transpose = false) or E_f Sigma_f H^{-1} r (transpose = true, with H
// the hierarchy of D_ff^T for a nonsymmetric operator); inner iterations accumulate on the device.
cudaError_t dsa_correct(DsaHierarchy* h, const double* r, double* phi_out, double tol, int max_iters,
                        bool transpose, cudaStream_t s);
cudaError_t dsa_solve(DsaHierarchy* h, const double* b_full, double* x_full, double tol, int max_iters,
                      cudaStream_t s);
// inner Krylov iterations run since the last call (synchronises the stream)
cudaError_t dsa_take_iters(DsaHierarchy* h, cudaStream_t s, int* iters);
// Algorithm 1 on full [elem][node] vectors: out = x on thick elements, 0 elsewhere;
// phi += (w - r) on thick elements and y elsewhere; z += y on thin elements
cudaError_t dsa_select_thick(DsaHierarchy* h, const double* x, double* out, cudaStream_t s);
cudaError_t dsa_tri_combine(DsaHierarchy* h, const double* w, const double* r, const double* y, double* phi,
                            cudaStream_t s);
cudaError_t dsa_add_thin(DsaHierarchy* h, const double* y, double* z, cudaStream_t s);
}  // namespace sn
