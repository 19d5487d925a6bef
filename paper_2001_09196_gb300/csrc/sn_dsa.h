// Internal: data of the thick-subdomain DSA operator and its multigrid hierarchy.
#pragma once

#include <vector>

#include "sn_internal.h"

namespace sn {

constexpr int kCoarseMax = 256;  // rows at which the hierarchy stops and inverts densely

struct Level0 {                  // DG space on the thick elements, BSR with n x n blocks
    std::vector<int> ptr, col;
    std::vector<double> val;     // nnzb x n x n (row-major blocks)
    std::vector<double> dinv;    // nt x n x n inverse diagonal blocks
    int *d_ptr = nullptr, *d_col = nullptr;
    double *d_val = nullptr, *d_dinv = nullptr;
    float *d_val32 = nullptr, *d_dinv32 = nullptr;  // float32 copies for the float32 V-cycle
};

struct LevelC {                  // a continuous level: operator, prolongation to the finer level
    int n = 0;
    std::vector<int> a_ptr, a_col, p_ptr, p_col, r_ptr, r_col;
    std::vector<double> a_val, p_val, r_val, dinv, dense_inv;
    int *d_a_ptr = nullptr, *d_a_col = nullptr, *d_p_ptr = nullptr, *d_p_col = nullptr, *d_r_ptr = nullptr,
        *d_r_col = nullptr;
    double *d_a_val = nullptr, *d_p_val = nullptr, *d_r_val = nullptr, *d_dinv = nullptr, *d_dense = nullptr;
    double *d_x = nullptr, *d_b = nullptr, *d_r = nullptr;
    float *d_a_val32 = nullptr, *d_p_val32 = nullptr, *d_r_val32 = nullptr, *d_dinv32 = nullptr, *d_dense32 = nullptr;
    float *d_x32 = nullptr, *d_b32 = nullptr, *d_r32 = nullptr;
};

struct DsaHierarchy {
    int n = 0, ne = 0, nt = 0;
    int op = 0;                           // SN_DSA_OP_SIP | SN_DSA_OP_NIP | SN_DSA_OP_MNIP
    bool symmetric = true;                // SIP: conjugate gradients; NIP / mNIP: BiCGStab
    bool transposed = false;              // holds D_ff^T
    std::vector<int> thick;               // thick element ids
    std::vector<double> h_mass_sig;       // nt x n: sigma_Sigma * collocated mass
    Level0 l0;
    std::vector<LevelC> levels;           // level 1 .. coarsest
    int* d_thick = nullptr;
    double* d_mass_sig = nullptr;
    // PCG vectors on the thick DOFs (nt x n)
    double *d_x = nullptr, *d_b = nullptr, *d_r = nullptr, *d_z = nullptr, *d_p = nullptr, *d_q = nullptr;
    double *d_vr = nullptr, *d_vx = nullptr;  // V-cycle level-0 residual / correction
    double *d_rh = nullptr, *d_sh = nullptr, *d_t = nullptr;  // BiCGStab: shadow residual, M s, A M s
    double* d_part = nullptr;                 // reduction partials
    double* d_s = nullptr;                    // device scalars
    bool uploaded = false;
    // V-cycle arithmetic: SN_VCYCLE_AUTO (float32 when the inner tolerance is >= 1e-8), _FP64, _FP32
    int vcycle_mode = 0;
    bool pc32 = false;                        // the recorded solve uses the float32 V-cycle
    bool uploaded32 = false;
    float *d_vr32 = nullptr, *d_r32 = nullptr, *d_z32 = nullptr;
    // damping of block-Jacobi (level 0) / Jacobi (levels >= 1).  Level 0: 0.8 keeps the smoother
    // convergent with margin for the largest eigenvalue of the block-Jacobi-preconditioned SIP
    // operator measured on the jittered Q2 configuration (between 2 and 2.2: damping 1.0 made the
    // PCG diverge, 0.9 converged) and takes fewer PCG iterations than 0.6 (336 against 391 per solve)
    double omega0 = 0.8, omega = 0.6;
    int nu = 2;                               // pre- and post-smoothing steps
    // The Krylov solve (PCG or BiCGStab) recorded as a CUDA graph whose WHILE conditional node
    // repeats one iteration until the device-side convergence test fails (no host
    // synchronisation per iteration)
    cudaGraphExec_t krylov_graph = nullptr;
    double krylov_tol = -1.0;
    int krylov_max = -1;
    int* d_it = nullptr;                      // [0] iterations of the current solve, [1] running total
    unsigned char* d_emask = nullptr;         // per element: 1 = thick (Algorithm 1's restrictions)
    long long pro_launches = 0, body_launches = 0;  // kernels in the prologue / one loop iteration
    long long nested_pro_launches = 0;              // prologue kernels of a solve recorded inside another graph
    bool krylov_pc32 = false;                       // V-cycle arithmetic krylov_graph was recorded with
    cudaStream_t cap = nullptr, cap2 = nullptr;     // private capture streams
};

}  // namespace sn
