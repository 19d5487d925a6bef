/*
 * libsn: GB300 (sm_103a) upwind-DG S_N transport sweep, source iteration and
 * thick-subdomain-only diffusion synthetic acceleration (Southworth, Holec & Haut,
 * "Diffusion synthetic acceleration for heterogeneous domains, compatible with voids").
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Every call returns an sn_status; none aborts.  On failure sn_last_error() returns a
 *    thread-local message.  SN_ERR_CUDA leaves the mesh usable unless the CUDA context
 *    itself was lost.
 *  - Meshes are structured nx x ny (x nz) grids of the unit square / cube; elements are
 *    numbered lexicographically with x fastest.  The discrete space is Q_p on each element,
 *    represented by values at the (p+1)^dim tensor Gauss-Legendre nodes, lexicographic with
 *    x fastest inside the element.  A scalar-flux array has layout [elem][node] (float64).
 *  - Directions: level-symmetric S_N, N in {4, 6, 8}; N(N+2) directions in 3D and the
 *    N(N+2)/2 with positive z component in 2D; weights sum to 4*pi.  Order: octant o
 *    (x negative if bit 0, y if bit 1, z if bit 2), then points (i, j, k) of the octant,
 *    i ascending, then j ascending.
 *  - Array arguments marked "device" are caller-owned device pointers (e.g. a torch
 *    tensor's data_ptr()); the library never frees them.  "mem" arguments choose host (0)
 *    or device (1) for inputs that accept both.
 *  - stream is a cudaStream_t (NULL = legacy default stream).  Calls enqueue work on it
 *    and return when the results are ready in device memory unless stated otherwise.
 *  - All device buffers a mesh needs (angular fluxes, work lists, the DSA hierarchy) are
 *    owned by the mesh and freed by sn_mesh_destroy.
 *  - Sizes are not checked: a scalar-flux argument must hold n_elem x n_nodes doubles and a
 *    per-element argument n_elem doubles (sn_mesh_get_info); a shorter buffer is overrun.
 *  - Unless an entry point says more: SN_ERR_ARG for a null mesh or required pointer or an
 *    out-of-range option (nothing is enqueued), SN_ERR_CUDA for a failed CUDA call, and
 *    SN_ERR_TIMEOUT when a bounded wait of the dataflow or tiled schedules gave up.
 */
#ifndef SN_H
#define SN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SN_OK = 0,
    SN_ERR_ARG = 1,                 /* invalid argument or unsupported combination */
    SN_ERR_CUDA = 2,                /* a CUDA call failed */
    SN_ERR_OOM = 3,                 /* device allocation failed */
    SN_ERR_CYCLE = 4,               /* an upwind graph has a cycle (no sweep order) */
    SN_ERR_VOID_FULL_DSA = 5,       /* full DSA on a mesh with sigma_t = 0, or the mNIP penalty next to a void */
    SN_ERR_NOT_CONVERGED = 6,       /* max_iters reached; phi still holds the last iterate */
    SN_ERR_TIMEOUT = 7,             /* a bounded device wait gave up; outputs undefined */
    SN_ERR_INNER_NOT_CONVERGED = 8  /* a DSA solve hit inner_max_iters (only if strict) */
} sn_status;

enum { SN_FP64 = 0, SN_FP32 = 1, SN_FP32_REFINE = 2, SN_FP32_MIXED = 3 };  /* element-solve precision */
enum { SN_DSA_NONE = 0, SN_DSA_FULL = 1, SN_DSA_THICK = 2, SN_DSA_TRIANGULAR = 3 };  /* DSA variant */
enum { SN_THICK_SIGMA_S = 0, SN_THICK_SIGMA_T_H = 1, SN_THICK_MASK = 2 };
enum { SN_DSA_SIGMA_S = 0, SN_DSA_SIGMA_T = 1 };
enum { SN_DSA_OP_SIP = 0, SN_DSA_OP_NIP = 1, SN_DSA_OP_MNIP = 2 };  /* DSA operator (Sec. 3.1) */
enum { SN_VCYCLE_AUTO = 0, SN_VCYCLE_FP64 = 1, SN_VCYCLE_FP32 = 2 };  /* DSA preconditioner arithmetic */
enum { SN_OUTER_SI = 0, SN_OUTER_FGMRES = 1 };                  /* outer iteration */
enum { SN_CACHE_OFF = 0, SN_CACHE_ON = 1, SN_CACHE_AUTO = 2 };  /* operator cache */

typedef struct sn_mesh sn_mesh;

typedef struct {
    int dim;                 /* 2 or 3 */
    int nx, ny, nz;          /* elements per axis (nz ignored in 2D) */
    int p;                   /* polynomial order: 1..3 in 2D, 1 in 3D */
    int sn_order;            /* 4, 6 or 8 */
    const double* vertices;  /* host, 2D only: ((ny+1)*(nx+1)) x 2, x fastest; NULL = uniform grid */
    double psi_inc;          /* isotropic inflow on every boundary face; 0 = vacuum */
} sn_mesh_desc;

typedef struct {
    int n_elem, n_nodes, n_dirs, n_levels;
    long long n_items;       /* n_elem * n_dirs */
} sn_mesh_info;

/*
 * sn_mesh_create: Eq. (sntransport) semi-discretisation (Sec. 1) on a structured mesh.
 * Builds the S_N quadrature, the per-element geometry and, on the device, the upwind
 * level sets of every direction (the topological order that makes each transport update
 * a forward block solve, Sec. 1).  Returns SN_ERR_CYCLE if a direction's upwind graph
 * has a cycle.  *out is owned by the caller and released with sn_mesh_destroy.
 * Materials default to sigma_t = sigma_s = q = 0 until sn_set_materials.
 */
sn_status sn_mesh_create(const sn_mesh_desc* desc, sn_mesh** out);
sn_status sn_mesh_destroy(sn_mesh* mesh);
sn_status sn_mesh_get_info(const sn_mesh* mesh, sn_mesh_info* info);

/*
 * Sweep schedule (tuning; every schedule computes the same element solves in the same arithmetic,
 * so results are bitwise identical):
 *   schedule 0 (default): one launch per wavefront level, captured once into a CUDA graph so that
 *   a sweep is a single graph launch (programmatic dependent launch overlaps a level's prologue
 *   with the previous level); with param = G > 1 the directions are split into G groups of
 *   consecutive directions whose level launches form G independent chains of the graph;
 *   schedule 1: one persistent launch per sweep in which warps claim items in level order and
 *   wait (bounded, SN_ERR_TIMEOUT after 4 s) for their upwind neighbours;
 *   schedule 2 (operator cache on): one persistent launch in which a CTA of `block` threads runs
 *   a whole tile of param^dim elements of one direction (param = tile edge, 0 = 16 in 2D and 8 in
 *   3D), synchronising itself between the tile's levels and waiting (bounded) only for upwind
 *   elements of other tiles; tiles whose upwind graph is cyclic (jittered faces) run as one task.
 *   schedule 3 (operator cache on): one cooperative launch per sweep; every CTA takes its share of
 *   each level's items and the CTAs meet at a grid barrier between levels (bounded wait,
 *   SN_ERR_TIMEOUT after 4 s); param = CTAs per SM (at least 1).
 *   schedule 4: as schedule 1, but with every warp of the grid resident and the work list dealt
 *   out statically (warp w takes slices w, w + W, w + 2W, ... of the level-ordered list, W warps in
 *   all) instead of claimed through a shared counter.
 *   In schedules 1 and 4 with the operator cache, the angular fluxes of the sweep are first set to
 *   the all-ones bit pattern and each element solve polls the upwind (adjoint: downwind) values it
 *   needs until none is that pattern (relaxed loads and stores; the stored values are their own
 *   completion signal); uncached solves wait on per-element completion words.
 *   Uncached solves (SN_FP32_REFINE, cache off) and the adjoint use schedule 0 instead of 2 or 3.
 * block: threads per block, a multiple of 32 in [32, 128] (schedules 0, 1, 4), [32, 256] (2),
 * [32, 512] (3).
 * param: schedule 0: direction groups (0 or 1 = one chain, at most the number of directions);
 * schedules 1 and 4: blocks per SM (0 = occupancy limit); schedule 2: tile edge (<= 64); schedule 3:
 * CTAs per SM.
 * Errors: SN_ERR_ARG for an unknown schedule, a block outside its range or a param out of range.
 */
sn_status sn_mesh_set_schedule(sn_mesh* mesh, int schedule, int block, int param);

/*
 * Operator cache.  The element operator A_e of Eq. (sntransport) (volume terms plus outflow
 * faces, Sec. 1) depends on the direction, the element geometry and sigma_t only, so within a
 * solve every transport update re-solves the same nd x ne small systems.  With the cache on, one
 * fully parallel kernel forms every A_e^{-1} in float64 (from its LU factors) after each change
 * of materials, and a sweep then builds the right-hand side and applies the stored inverse (the
 * adjoint applies its transpose); on the level schedule one lane per element node does this, so
 * an element's solve takes O(N) dependent steps instead of O(N^3).  Storage: nd x ne x s values,
 * s = N^2 rounded up to a multiple of 4 (N = nodes per element), float64 for SN_FP64 and the
 * adjoint, a float32 copy for SN_FP32, plus the face flux factors (2D: 4 float64 per direction
 * and element; 3D: 3 per direction).  SN_FP32_REFINE always assembles on the fly.  Results agree
 * with on-the-fly solves to rounding.
 *   SN_CACHE_OFF: assemble and factor in every sweep (frees any cached inverses);
 *   SN_CACHE_ON: always cache (an allocation failure is returned as SN_ERR_CUDA);
 *   SN_CACHE_AUTO (default): cache when the inverses take at most half of the free device memory.
 * Synchronises the device.  Errors: SN_ERR_ARG for a null mesh or an unknown mode.
 */
sn_status sn_mesh_set_operator_cache(sn_mesh* mesh, int mode);

/*
 * Test hook for the bounded waits of the dataflow schedule: the next sweep's items publish a
 * completion value that no waiter accepts, so every dependent item waits timeout_seconds
 * (0 < t <= 4), the kernel records the failure and exits, and the call returns SN_ERR_TIMEOUT.
 * The context stays usable; later sweeps are unaffected.  The paper has no counterpart (a hook of
 * the device-side wait limits).  Errors: SN_ERR_ARG for t outside (0, 4] or a mesh on the level
 * schedule, which never waits.
 */
sn_status sn_debug_stall_next_sweep(sn_mesh* mesh, double timeout_seconds);

/* Quadrature readback (the level-symmetric set of Eq. sntransport, Sec. 1): dirs (host, n_dirs x 3,
 * Omega_d row by row) and weights (host, n_dirs, summing to 4 pi).  Errors: SN_ERR_ARG for a null
 * mesh. */
sn_status sn_mesh_quadrature(const sn_mesh* mesh, double* dirs, double* weights);

/*
 * sn_set_materials: per-element sigma_t, sigma_s and isotropic emission density q
 * (Eq. 1: 0 <= sigma_s <= sigma_t; q_d = q / (4 pi)).  Copied into the mesh (n_elem
 * doubles each, host if mem = 0, device if mem = 1).  Invalidates any DSA hierarchy.
 * Returns SN_ERR_ARG on NaN/Inf, negative values or sigma_s > sigma_t.
 */
sn_status sn_set_materials(sn_mesh* mesh, const double* sigma_t, const double* sigma_s,
                           const double* q, int mem, void* stream);

/*
 * sn_set_pseudo_scattering: the materials of one implicit time step of gray thermal radiative
 * transfer written as a steady transport problem (Sec. 4.2, Eq. hohlraum_sigma, Eq. hohlraum_q),
 * computed per element on the device from the opacity sigma (= sigma_a), the heat capacity C_v
 * and the temperature T:
 *     b = 16 pi a c T^3,  sigma_t = sigma,  sigma_s = sigma^2 b / (C_v/dt + sigma b),
 *     q = 4 pi q_ps,  q_ps = sigma a c T^4 - sigma^2 b a c T^4 / (C_v/dt + sigma b)
 * (q_d = q_ps per direction; the library's q is total emission, q_d = q / (4 pi)).  q_ps is
 * evaluated in the equal form sigma a c T^4 (C_v/dt) / (C_v/dt + sigma b), free of the
 * cancellation of the printed difference.  sigma, cv, T: n_elem doubles each, host if mem = 0,
 * device if mem = 1; dt, a_rad, c_light: the time step, the radiation constant and the speed of
 * light (the paper: 1e-3, 137.199, 2.9979e4 in NIF units).  Then as sn_set_materials.
 * Synchronises the stream and uses the mesh's work vectors, so no other call on this mesh may be
 * in flight.  SN_ERR_ARG unless sigma >= 0, C_v > 0, T >= 0 (finite) and dt, a_rad, c_light > 0;
 * a refused call leaves the materials unchanged.
 */
sn_status sn_set_pseudo_scattering(sn_mesh* mesh, const double* sigma, const double* cv, const double* T,
                                   double dt, double a_rad, double c_light, int mem, void* stream);

/* Current materials sigma_t, sigma_s, q of Eq. sntransport (host arrays of n_elem doubles, written;
 * any may be NULL).  Errors: SN_ERR_ARG for a null mesh. */
sn_status sn_get_materials(const sn_mesh* mesh, double* sigma_t, double* sigma_s, double* q);

/*
 * sn_sweep: one transport update, Eq. (source0) / Eq. (phi):
 *     phi_out = sum_d w_d L_d^{-1} ( q/(4 pi) + sigma_s phi_in / (4 pi) ),
 * the element systems solved in the given precision (SN_FP64, SN_FP32 or SN_FP32_REFINE;
 * the scalar-flux sum is always float64).  phi_in, phi_out: device, [elem][node],
 * must not alias.  phi_in may be NULL (phi_in = 0).  The angular fluxes psi_d of this sweep
 * stay in the mesh (used by sn_gradients).  Errors: SN_ERR_ARG for a null mesh or phi_out, an
 * unknown precision (SN_FP32_MIXED is an iteration, not a sweep) or phi_in == phi_out.
 */
sn_status sn_sweep(sn_mesh* mesh, const double* phi_in, double* phi_out, int precision, void* stream);

/*
 * sn_sweep_directions: the part of the transport update that directions d_begin <= d < d_end
 * contribute, phi_out = sum_{d in range} w_d L_d^{-1}( q/(4 pi) + sigma_s phi_in/(4 pi) ).
 * Directions are independent within one update (Eq. psi), so the partial updates of a partition
 * of the directions sum to sn_sweep's phi_out (up to the order of the float64 additions): the
 * decomposition behind sharding the sweep by direction, where each process sweeps its range and
 * one sum-reduction of phi_out completes the update.  psi_d of the range is stored as sn_sweep
 * stores it (bitwise the same values); the other directions' psi_d are left as they were.  Runs as
 * a chain of level launches whatever the mesh's schedule.  Errors: SN_ERR_ARG for a range outside
 * [0, n_dirs), an empty range, a bad precision or aliasing buffers.
 */
sn_status sn_sweep_directions(sn_mesh* mesh, const double* phi_in, double* phi_out, int d_begin, int d_end,
                              int precision, void* stream);

/*
 * Exchange step of a direction-sharded iteration (sn_iter_opts.exchange).  The transport update
 * is a sum over directions (Eq. phi), so processes that each sweep their own range of directions
 * complete one update by summing their partial scalar fluxes.  The library calls the function
 * after it has enqueued this process's partial update on `stream`: phi_partial (device, n doubles,
 * [elem][node]) holds sum_{d in range} w_d psi_d when the stream reaches that point, and must hold
 * the sum over all processes when the stream continues past the call (for example an NCCL
 * all-reduce enqueued on `stream`, or a synchronise, host all-reduce and copy back).  Every process
 * must receive bitwise the same sum, so that all of them take the same convergence decisions.
 * Return SN_OK, or any other status to end the iteration with that status.
 */
typedef sn_status (*sn_exchange_fn)(double* phi_partial, long long n, void* stream, void* ctx);

typedef struct {
    int dsa;                 /* SN_DSA_NONE | SN_DSA_FULL | SN_DSA_THICK (Algorithm 2) | SN_DSA_TRIANGULAR (Algorithm 1) */
    int thick_rule;          /* SN_THICK_SIGMA_S (sigma_s >= eta, Sec. 3.2) | SN_THICK_SIGMA_T_H | SN_THICK_MASK */
    double eta;              /* threshold of the thick rule; the paper uses eta = 1 (Sec. 4.1) */
    const unsigned char* mask; /* host, n_elem, used with SN_THICK_MASK */
    int dsa_sigma;           /* SN_DSA_SIGMA_S (default) | SN_DSA_SIGMA_T: mass matrix of the DSA rhs */
    double tol;              /* relative residual ||r^i|| / ||r^0|| (Euclidean, nodal) */
    double inner_tol;        /* relative residual of each DSA solve (PCG, or BiCGStab for NIP / mNIP) */
    int max_iters, inner_max_iters;
    int precision;           /* SN_FP64 | SN_FP32 | SN_FP32_REFINE | SN_FP32_MIXED (fGMRES only): float32
                                element solves in every Arnoldi step, float64 element solves for the true
                                residual that starts each restart cycle; a cycle ends once its residual
                                estimate fell by refine_drop (or after `restart` steps), so the float32
                                operator error enters only as the inexactness of a correction and the
                                iteration converges to the float64 fixed point (mixed-precision iterative
                                refinement around flexible GMRES) */
    int checkpoint_every;    /* >0: copy phi^{k} to checkpoints after every k-th iteration */
    double* checkpoints;     /* device, max_checkpoints x n_elem x n_nodes, or NULL */
    int max_checkpoints;
    int warm_start;          /* 1: start from phi_inout, 0: from phi = 0 */
    int outer;               /* SN_OUTER_SI (fixed point, Eq. DSA_fp) | SN_OUTER_FGMRES (Sec. 4) */
    int restart;             /* fGMRES restart length (1..60; the paper uses 30) */
    int dsa_operator;        /* SN_DSA_OP_SIP (default) | SN_DSA_OP_NIP (Eq. NIP) | SN_DSA_OP_MNIP (Eq. NIP with
                                the penalty of Eq. ModifiedF0); see sn_source_iterate */
    int dsa_vcycle;          /* arithmetic of the multigrid V-cycle that preconditions each DSA solve:
                                SN_VCYCLE_AUTO (default: float32 when inner_tol >= 1e-8, else float64),
                                SN_VCYCLE_FP64 or SN_VCYCLE_FP32.  The Krylov residuals, dot products and
                                convergence test are float64 in every mode. */
    int dir_begin, dir_end;  /* direction sharding (sn_source_iterate only): this process sweeps the
                                directions dir_begin <= d < dir_end of every transport update and
                                `exchange` sums the partial updates over processes; both 0 = all
                                directions, no exchange.  The DSA step, the Krylov work and the
                                convergence test run replicated on every process. */
    sn_exchange_fn exchange; /* required with a direction range; see sn_exchange_fn */
    void* exchange_ctx;      /* passed through to exchange */
    double* exchange_buf;    /* optional device buffer (n_elem x n_nodes doubles) that the partial
                                updates are written to and exchanged in; NULL = library scratch */
    double refine_drop;      /* SN_FP32_MIXED: residual reduction that ends a restart cycle (0 = 1e-4) */
    int host_loop;           /* 0 (default): on the level schedule of one process, the whole solve is
                                recorded once into a CUDA graph (WHILE conditional nodes, convergence
                                tests on the device) and runs as one graph launch with one host
                                synchronisation; 1: a host loop with one synchronisation per outer
                                iteration, which also splits the device time into ms_sweep / ms_dsa */
} sn_iter_opts;

typedef struct {
    int iters;               /* outer iterations performed */
    double rel_residual;     /* last ||r^i|| / ||r^0|| */
    int inner_iters_total;   /* inner Krylov iterations summed over all DSA solves */
    double thick_fraction;   /* thick elements / all elements */
    double* residual_history; /* host, history_len entries, or NULL */
    int history_len;
    int n_checkpoints;       /* checkpoints written */
    double ms_total;         /* wall time of the call (stream-synchronised) */
    int n_sweeps;            /* transport updates performed (all directions each) */
    double ms_sweep;         /* device time of the transport updates and their flux reductions (CUDA events) */
    double ms_dsa;           /* device time of the DSA solves (CUDA events); both 0 for batches */
} sn_iter_stats;

/* Defaults: dsa thick, sigma_s >= 1, tol 1e-8, inner_tol 1e-4 (Sec. 4), FP64, cold start. */
void sn_iter_opts_default(sn_iter_opts* opts);

/*
 * sn_source_iterate: source iteration with diffusion synthetic acceleration,
 * Eq. (DSA_fp) with the diagonal heterogeneous preconditioner of Algorithm 2:
 *     phi_half^i = sweep(phi^i),  r^i = phi_half^i - phi^i,
 *     phi^{i+1} = phi_half^i + E_f D_ff^{-1} Sigma_f r^i_f     (nothing added for SN_DSA_NONE),
 * with D_ff the symmetric interior-penalty diffusion operator on the thick elements
 * (Sec. 3.1-3.2; SN_DSA_FULL uses every element) solved by conjugate gradients
 * preconditioned with a geometric multigrid V-cycle.  Stops after the iteration whose
 * ||r^i|| <= tol ||r^0||.  phi_inout: device [elem][node]; receives phi^{i+1}.
 * With outer = SN_OUTER_FGMRES the same system S phi = b (Eq. schur) is solved by flexible
 * GMRES(restart) right-preconditioned by the same DSA step, I + E_f D_ff^{-1} Sigma_f E_f^T (the paper's
 * outer solver, Sec. 4; "flexible" because each DSA solve is inexact).  Its residual b - S phi equals
 * the source-iteration residual, so tol means the same; iters counts Krylov iterations.
 * SN_DSA_TRIANGULAR is the block upper-triangular preconditioner of Algorithm 1 (Eq. approxS): the
 * thick-only DSA step above, then a transport update with zero fixed source and vacuum inflow of
 * [0; corrected thick part] whose result is added on the thin DOFs only (one extra sweep per outer
 * iteration).  It uses the same thick rule; it is not available for the adjoint or for batches
 * (SN_ERR_ARG).
 * opts->dsa_operator picks D_ff (Sec. 3.1; D = 1/(3 sigma_t), sigma_a = sigma_t - sigma_s, all
 * integrals on the (p+1)-point Gauss rule; a face to a non-thick element or the boundary is a face
 * to a zero exterior state, as in a principal submatrix):
 *   SN_DSA_OP_SIP: symmetric interior penalty with kappa = max(1/4, 2 p(p+1) {D/h}), h = |K|/|F|;
 *     SPD, solved by conjugate gradients.
 *   SN_DSA_OP_NIP: Eq. NIP, the SIP form without the symmetrising face term -<{D dv/dn},[u]> and
 *     with the penalty of F_0, kappa = 1/4; nonsymmetric, solved by BiCGStab right-preconditioned
 *     with the same V-cycle (the adjoint builds D_ff^T and its own hierarchy).
 *   SN_DSA_OP_MNIP: Eq. NIP with the penalty of Eq. ModifiedF0,
 *     kappa = [max(0.1 p(p+1)/(sigma_t^- h^-), 1) + max(0.1 p(p+1)/(sigma_t^+ h^+), 1)] / 8 with
 *     the neighbour's data even when it is thin (the element's own on the domain boundary);
 *     SN_ERR_VOID_FULL_DSA if a thick element has a void neighbour.
 * Batches take SN_DSA_OP_SIP only (SN_ERR_ARG).
 * SN_ERR_VOID_FULL_DSA if dsa = FULL and some sigma_t = 0; SN_ERR_NOT_CONVERGED after
 * max_iters (phi_inout still written).  stats may be NULL.
 */
sn_status sn_source_iterate(sn_mesh* mesh, const sn_iter_opts* opts, double* phi_inout,
                            sn_iter_stats* stats, void* stream);

/*
 * sn_adjoint_sweep: transpose of the linear part of sn_sweep (in the nodal coordinates
 * of the interface): out = sum_d w_d Sigma_s L_d^{-T} mu_in, where Sigma_s is the nodal
 * mass matrix with coefficient sigma_s/(4 pi).  L_d^T is solved by a sweep in reversed
 * upwind order with transposed element and face blocks (adjoint of Eq. system).
 * mu_in, out: device [elem][node]; the lambda_d = w_d L_d^{-T} mu_in stay in the mesh.
 * Errors: SN_ERR_ARG for a null pointer, mu_in == out or a precision other than SN_FP64.
 */
sn_status sn_adjoint_sweep(sn_mesh* mesh, const double* mu_in, double* out, int precision, void* stream);

/*
 * sn_adjoint_iterate: solves S^T mu = g (S = I - T, Eq. schur) by the adjoint source
 * iteration mu <- g + T^T mu with the transposed DSA step, or (outer = SN_OUTER_FGMRES) by
 * flexible GMRES right-preconditioned by that transposed step.  g, mu_inout: device.
 * Errors: as sn_source_iterate for the options; SN_ERR_ARG for SN_DSA_TRIANGULAR or a direction
 * range (the adjoint runs on one process); SN_ERR_NOT_CONVERGED after max_iters (mu_inout written).
 */
sn_status sn_adjoint_iterate(sn_mesh* mesh, const sn_iter_opts* opts, const double* g, double* mu_inout,
                             sn_iter_stats* stats, void* stream);

/*
 * sn_gradients: for J = g^T phi with phi converged and mu = S^{-T} g, per element
 *   d_sigma_t[e] = -sum_d lambda_d,e^T M_e psi_d,e,
 *   d_sigma_s[e] =  sum_d lambda_d,e^T M_e phi_e / (4 pi),
 *   d_q[e]       =  sum_d lambda_d,e^T M_e 1 / (4 pi),
 * with psi_d = L_d^{-1}(q_d + Sigma_s phi) and lambda_d = w_d L_d^{-T} mu (one forward and
 * one adjoint sweep, FP64).  All pointers device; outputs n_elem doubles (NULL to skip).
 * The paper computes no gradients: these follow from Eq. (system) by the adjoint method.
 * Errors: SN_ERR_ARG for a null mesh, phi or mu.
 */
sn_status sn_gradients(sn_mesh* mesh, const double* phi, const double* mu, double* d_sigma_t,
                       double* d_sigma_s, double* d_q, void* stream);

/*
 * sn_unrolled_gradients: gradients of J = g^T phi_K with respect to sigma_t, sigma_s and q, where
 * phi_K is the K-th iterate of source iteration without acceleration from phi_0, phi_{k+1} =
 * T phi_k + b (one transport update, sn_sweep; Eq. source0), i.e. the derivative of the map that a
 * fixed number of updates computes, not of the converged solution.  Reverse accumulation through
 * the K updates: mu_K = g; for k = K-1 .. 0 the update at (phi_k, mu_{k+1}) contributes the
 * sn_gradients contractions (one forward sweep from phi_k, one adjoint sweep of mu_{k+1}), and
 * mu_k = T^T mu_{k+1} (sn_adjoint_sweep's reduction of the same adjoint sweep).
 * Iterate checkpointing: the phi_k are needed in reverse order; they are recomputed segment by
 * segment from every `checkpoint_every`-th iterate.  checkpoints: NULL (this call runs the K - 1
 * forward updates first and keeps its own), or the buffer that sn_source_iterate filled with
 * dsa = SN_DSA_NONE, max_iters = K, checkpoint_every = the same value (iterates checkpoint_every,
 * 2 checkpoint_every, ...; at least ceil(K / checkpoint_every) - 1 of them).  phi0: device, or NULL
 * for phi_0 = 0 (sn_source_iterate's cold start).  g: device [elem][node].  Outputs n_elem doubles
 * each (NULL to skip), overwritten.  Memory: min(checkpoint_every, K) + 5 vectors of n_elem x n_nodes
 * doubles, plus ceil(K / checkpoint_every) more when checkpoints is NULL, allocated for the call.
 * Cost: K forward and K adjoint sweeps in the backward pass, K - ceil(K / checkpoint_every) forward
 * sweeps recomputing segments, and K - 1 more when checkpoints is NULL.  FP64.
 * Errors: SN_ERR_ARG for K < 1 or checkpoint_every < 1; SN_ERR_TIMEOUT as sn_sweep.
 */
sn_status sn_unrolled_gradients(sn_mesh* mesh, const double* phi0, int K, int checkpoint_every,
                                const double* checkpoints, const double* g, double* d_sigma_t, double* d_sigma_s,
                                double* d_q, void* stream);

/*
 * Diagnostics of the DSA operator (Sec. 3): y = D_ff x on the elements selected by opts
 * (x, y device, [elem][node]; entries outside the thick set are ignored / set to 0), and the
 * PCG + V-cycle solve of D_ff x = b to opts->inner_tol.  *iters receives the PCG count.
 * Errors: SN_ERR_ARG for a null pointer or bad options; SN_ERR_VOID_FULL_DSA as sn_source_iterate.
 */
sn_status sn_dsa_apply(sn_mesh* mesh, const sn_iter_opts* opts, const double* x, double* y, void* stream);
sn_status sn_dsa_solve(sn_mesh* mesh, const sn_iter_opts* opts, const double* b, double* x, int* iters,
                       void* stream);

/*
 * Diagnostic: copies psi_d (direction d) of the last forward sweep (or lambda_d of the last
 * adjoint sweep if adjoint != 0) into out (device, [elem][node], float64; the FP32 form's
 * float32 values are widened).  Used to check the element equations of Sec. 3.1 at full size.
 * Errors: SN_ERR_ARG for a null pointer, d outside [0, n_dirs), or no sweep of that kind yet.
 */
sn_status sn_get_angular_flux(sn_mesh* mesh, int d, int adjoint, int precision, double* out, void* stream);

/*
 * Diagnostic: the upwind level of every element for direction d (host, n_elem ints), as the
 * device's Kahn pass computed it when the mesh was created (Sec. 1: the transport update is a
 * forward solve in an upwind order; level 0 has no upwind neighbour, an element's level is one
 * more than its highest upwind neighbour's).  SN_ERR_ARG for d outside [0, n_dirs).
 */
sn_status sn_get_levels(const sn_mesh* mesh, int d, int* levels);

/*
 * sn_scalar_flux_noalloc: the scalar-flux reduction of a transport update without any device
 * allocation.  The paper has no counterpart; it exists for callers that cannot call cudaMalloc:
 * frameworks whose caching allocator owns all device memory (a cudaMalloc behind its back can fail
 * or fragment the pool it manages), latency-critical loops that cannot afford cudaMalloc's implicit
 * device synchronisation, and embedded hosts whose device memory budget is fixed at start-up.
 * Computes, in float64 with the same summation order as sn_sweep,
 *     phi_out[i] = sum_d weights[d] * psi[d * n_values + i],
 *     *resid_norm2 = sum_i (phi_out[i] - phi_prev[i])^2     (phi_prev NULL means 0; resid_norm2 may be NULL).
 * psi (n_dirs x n_values), weights (n_dirs), phi_prev, phi_out (n_values) and resid_norm2 (1) are
 * caller-owned device pointers; phi_out must not alias the inputs.
 * Scratch: the per-block partial sums live in one file-scope device array of 8192 doubles (64 KB),
 * held by every GPU that loads the library until the process exits, which limits n_values to
 * 2,097,152 (larger sizes return SN_ERR_ARG before any GPU work).  The array is shared by all calls
 * and keeps the last call's partial sums; each call overwrites every slot it reads, so nothing
 * needs clearing, but calls whose kernels overlap on the GPU (different streams, no ordering)
 * race on it.  The first call on each device (with that device current) resolves the array's
 * device address with cudaGetSymbolAddress; make that first call before any stream capture.
 * No cudaMalloc, cudaFree or allocating library routine is called.
 */
sn_status sn_scalar_flux_noalloc(const double* psi, const double* weights, int n_dirs, long long n_values,
                                 const double* phi_prev, double* phi_out, double* resid_norm2, void* stream);

/* Number of CUDA kernels the library has launched since it was loaded (diagnostic). */
long long sn_launch_count(void);

/*
 * Batches (task form 2): many meshes of different size, order p and S_N order swept together.
 * sn_batch_create: the meshes stay owned by the caller and must outlive the batch.  The batch builds
 * one work list of every instance's (direction, element) items ordered by (upwind level, element
 * family, instance); a level never mixes element templates inside a warp.
 * sn_batch_sweep: one transport update of every instance, phi_out[i] = sweep_i(phi_in[i]) (arrays of
 * count device pointers; phi_in may be NULL), as one persistent launch (schedule 1: warps claim
 * 32-item chunks; schedule 4: chunks dealt out statically to resident warps) or one set of level
 * launches (schedule 0).  In the persistent launches with cached operators every instance's angular
 * fluxes are reset to an unset bit pattern before the sweep and consumers poll the upwind values
 * (see sn_mesh_set_schedule); an instance that has converged in a batched iteration keeps its
 * iterate, but its stored angular fluxes are then not those of a sweep.  Synchronises the stream.
 * sn_batch_source_iterate: Eq. (DSA_fp) with Algorithm 2 for every instance at once: the batched sweep,
 * per-instance flux reductions and residual norms, and one conjugate-gradient solve of the union of
 * the instances' thick-DSA systems (block diagonal, one multigrid V-cycle over the union of their
 * hierarchies), with per-instance convergence masks (a converged instance's items become no-ops).
 * With opts->outer = SN_OUTER_SI one whole outer iteration is recorded once into a CUDA graph and
 * replayed; the host checks the masks every 4 iterations.  With SN_OUTER_FGMRES every instance runs
 * its own flexible GMRES(opts->restart) on Eq. (schur), right-preconditioned by the same union DSA
 * step, in lock step: one recorded graph per Arnoldi step of all instances (the batched homogeneous
 * sweep, the union DSA solve, Gram-Schmidt with inner products segmented by instance, the Givens
 * updates on the device) and one per restart (true residuals with the fixed source); the host reads
 * two flags after each.  An instance stops extending its basis at the tolerance or its iteration
 * budget and leaves the batch when its true residual is below opts->tol; stats[i].iters counts its
 * Arnoldi steps.  phis: count device pointers (warm start if opts->warm_start), receive the
 * results; stats: count entries or NULL.  Precision SN_FP64, SN_FP32 or SN_FP32_REFINE (not
 * SN_FP32_MIXED); no checkpoints, no direction sharding; the thick rule must not be SN_THICK_MASK.
 * SN_ERR_NOT_CONVERGED if any instance stops at max_iters.
 */
typedef struct sn_batch sn_batch;
sn_status sn_batch_create(sn_mesh* const* meshes, int count, sn_batch** out);
sn_status sn_batch_destroy(sn_batch* batch);
sn_status sn_batch_set_schedule(sn_batch* batch, int schedule, int block, int max_blocks_per_sm);
sn_status sn_batch_sweep(sn_batch* batch, const double* const* phi_in, double* const* phi_out, int precision,
                         void* stream);
sn_status sn_batch_source_iterate(sn_batch* batch, const sn_iter_opts* opts, double* const* phis,
                                  sn_iter_stats* stats, void* stream);

/*
 * Schedule autotuner: times the candidate sweep schedules (level graphs with 32/64/128-thread blocks;
 * persistent dataflow launches with several per-SM occupancy caps; for meshes, tiled launches with
 * several tile edges and CTA sizes) for this mesh / batch and precision
 * with CUDA events, keeps the fastest and reports it (any output pointer may be NULL).  Results of
 * sn_mesh_autotune are cached per (dim, p, directions, precision, element count), so meshes of the same
 * shape reuse them.  Schedules give bitwise-identical results; tuning changes only the time.
 */
sn_status sn_mesh_autotune(sn_mesh* mesh, int precision, void* stream, int* schedule, int* block, int* cap);
sn_status sn_batch_autotune(sn_batch* batch, int precision, void* stream, int* schedule, int* block, int* cap);

const char* sn_last_error(void);
const char* sn_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SN_H */
