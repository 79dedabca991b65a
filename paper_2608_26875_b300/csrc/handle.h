// Internal definition of ms_handle shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ms_b300.h"

// One translation family (near pairs, P2M, M2M, M2L, L2L or L2P) for one wave: CSR over
// destination entities; each task names a source entity and the offset of its sequence.
struct DevList {
    int ndst = 0, ntask = 0;
    int* ptr = nullptr;
    int* src = nullptr;
    long long* seq = nullptr;
};

// Arguments of the generic Toeplitz translation kernel (see fmm.cu).
struct TransArgs {
    const int* dst_ptr;
    const int* task_src;
    const long long* task_seq;
    int K, Pd, Ps;   // K: centre of each stored sequence (h_k at offset K + k), >= Pd + Ps
    int adj;         // 1: apply the adjoint of the reverse-direction translation (see fmm.cu)
    void* dst;
    long long dst_stride;
    const void* src;
    long long src_stride;
    const int* ad;
    long long ad_stride;
    int sd;
    const int* as;
    long long as_stride;
    int ss;
    int nrhs;
    int accumulate;
};

struct FmmHost {
    int nbox[13] = {0};
    double w[13] = {0};
    int P[2][13] = {{0}};
    int* expo[2][13] = {{nullptr}};    // device exponent profile per level, [2P+1]
    void* mexp[2][13] = {{nullptr}};   // multipole expansions [box][2P+1][nrhs]
    void* lexp[2][13] = {{nullptr}};   // local expansions
    DevList near[2], p2m[2], l2p[2];
    DevList m2m[2][13], m2l[2][13], l2l[2][13];
};

struct MsDeviceTables {
    // geometry
    double2* centre = nullptr;     // [M] (x_m, y_m)
    int* expo = nullptr;           // [M][2][nc] binary exponent a of the per-order scale 2^a
    // scattering matrices in the scaled basis (S~ = D^-1 S D^-1, D = diag(2^a))
    double2* sdisc = nullptr;      // [M][nc][2][2] for disc particles (zero block for prototypes)
    float2* sdisc_f = nullptr;
    int* proto = nullptr;          // [M] -1 disc, else prototype index
    double* rot = nullptr;         // [M] rotation angle
    double2* sproto = nullptr;     // [Q][2nc][2nc] unscaled prototype tables
    // Sommerfeld contour (Sec. 5.1)
    double2* node = nullptr;       // [NS] per node: xi_q
    double2* wq = nullptr;         // [NS] quadrature weight w_q xi'(t_q)
    double2* sq = nullptr;         // [NS][2] s_b(xi_q), b = P, S (lower layer)
    double2* qq = nullptr;         // [NS][2] q_b = (xi_q - s_b)/k_b
    double2* refl = nullptr;       // [NS][2][2] reflection matrix R(xi_q): (U_P,U_S) -> (D_P,D_S)
    double2* qpow_m2s = nullptr;   // [2][NS][nc] (-i)^n q_b^n / (i pi s_b)
    double2* qpow_s2l = nullptr;   // [2][NS][nc] i^n q_b^n W_q
    float2* qpm_m = nullptr;       // FP32 mantissa / binary exponent copies of the two tables
    int* qpm_e = nullptr;
    float2* qps_m = nullptr;
    int* qps_e = nullptr;
    // translation sequences h_k = Z_k(k|v|) e^{ik arg v}: FP64 and FP32 mantissa / exponent copies
    double2* seq64 = nullptr;
    float2* seqm = nullptr;
    int* seqe = nullptr;
};

struct ms_handle {
    int M = 0, p = 0, nc = 0, NS = 0;
    double omega = 0;
    double lam_u = 0, mu_u = 0, lam_l = 0, mu_l = 0;
    double kp_u = 0, ks_u = 0, kp_l = 0, ks_l = 0;
    int n_proto = 0;
    bool any_proto = false;
    ms_options opt{};
    MsDeviceTables d;
    std::vector<double> h_centres, h_radius;
    std::vector<int> h_expo;       // host copy of the exponents
    int nnz_near = 0;
    int fmm_levels = 0;            // 0: direct sum over all pairs
    long long seq_len = 0;
    FmmHost fmm;
    // workspace sized for ws_nrhs columns
    int ws_nrhs = 0;
    void* ws_x = nullptr;          // scaled input  [M][2][nc][nrhs] (double2 or float2)
    void* ws_a = nullptr;          // scaled local  [M][2][nc][nrhs]
    void* ws_y = nullptr;          // scaled output [M][2][nc][nrhs]
    void* ws_part = nullptr;       // M2S split-K partials [chunks][2][NS][nrhs] (double2)
    void* ws_u = nullptr;          // [2][NS][nrhs] double2 upgoing amplitudes, then reflected D
    int last_cuda = 0;
};

// internal helpers implemented across the .cu files
int ms_check(ms_handle* h, cudaError_t e);
int ms_ensure_workspace(ms_handle* h, int nrhs);
template <typename T>
int ms_apply_scaled(ms_handle* h, const void* xs, void* ys, int nrhs, int parts, bool identity,
                    cudaStream_t st);
template <typename T>
int ms_local_scaled(ms_handle* h, const void* xs, int nrhs, int parts, cudaStream_t st);
template <typename T>
int ms_sapply_scaled(ms_handle* h, const void* xs, void* ys, int nrhs, bool identity, bool apply_s,
                     cudaStream_t st);
int ms_build_translations(ms_handle* h, int use_fmm, int leaf_target);
template <typename T>
int ms_translate_scaled(ms_handle* h, const void* xs, int nrhs, bool near, bool far, cudaStream_t st);
int ms_fmm_workspace(ms_handle* h, int nrhs);
void ms_fmm_free(ms_handle* h);
int ms_to_scaled(ms_handle* h, const void* x, void* xs, int nrhs, int prec, cudaStream_t st);
int ms_from_scaled(ms_handle* h, const void* ys, void* y, int nrhs, int prec, cudaStream_t st,
                   bool local = false);
