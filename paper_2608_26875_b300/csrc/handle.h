// Internal definition of ms_handle shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <tuple>
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
    int deriv;       // 1: entries c1 h_{k-1} + c2 h_{k+1} (derivative in the translation vector)
    double2 dc1, dc2;
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

// Tiles of a tensor-core translation launch.
struct TcTiles {
    int n = 0;
    int4* tile = nullptr;          // [n] {target offset, targets, source offset, sources}
    int* tgt = nullptr;            // target entities of every tile
    int* self = nullptr;           // position of each target in its source list (-1: none)
    int* src = nullptr;            // source entities (near: one list per leaf)
    int* row = nullptr;            // per tile: first output order (M2L), or NULL
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
    // tensor-core tiles of the near lists (up to 256 / nc target particles of one leaf against the
    // particles of the 3 x 3 leaves around it, the target included, in near-list order: near task =
    // ptr[m] + s - (s > self position)) and of the M2L lists (256-row ranges of one box)
    TcTiles near_tc;
    TcTiles m2l_tc[2][13];
    long long near_seq_base[2] = {0, 0};   // near task t's sequence starts at base + t (4p + 3)
    // algorithmic complex multiply-adds per right-hand-side column of one application (both waves):
    // direct near pairs, and the FMM's P2M + M2M + M2L + L2L + L2P tasks
    double work_near = 0, work_far = 0;
    // stored 3xTF32 B tiles of the near tiles (ms_options.store_near): wave b at near_store + b *
    // near_store_wave, tile t at near_store_off[t], chunk c at + c * 2 * (n * KC * 4) (hi, then lo)
    unsigned char* near_store = nullptr;
    long long* near_store_off = nullptr;
    long long near_store_wave = 0;
};

// group-block Jacobi preconditioner (precond.cu): group g's inverse block (D_g = 2 nc n_g square,
// row-major, rows (position in group, wave, order)) at goff[g]
struct PrecondDev {
    double2* inv64 = nullptr;
    float2* inv32 = nullptr;
    long long* goff = nullptr;
    int* gptr = nullptr;           // [ng + 1] into gpart
    int* gpart = nullptr;          // particles by group
    int* pgrp = nullptr;           // group of each particle
    int* ppos = nullptr;           // position of each particle in its group
    int ng = 0, dmax = 0;
    long long total = 0;
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
    double2* sps64 = nullptr;      // [Q][2nc][2nc] scaled prototype tables S~_q = 2^-e_ref S_q 2^-e_ref
    float2* sps32 = nullptr;       // FP32 copy, and its conjugate transpose (adjoint, tensor cores)
    float2* spsH32 = nullptr;
    int* plist = nullptr;          // [n_plist] the prototype particles
    int* pref = nullptr;           // [Q] reference particle of each prototype (whose scales S~_q carries)
    // Sommerfeld contour (Sec. 5.1)
    double2* node = nullptr;       // [NS] per node: xi_q
    double2* wq = nullptr;         // [NS] quadrature weight w_q xi'(t_q)
    double2* sq = nullptr;         // [NS][2] s_b(xi_q), b = P, S (lower layer)
    double2* qq = nullptr;         // [NS][2] q_b = (xi_q - s_b)/k_b
    double2* refl = nullptr;       // [NS][2][2] reflection matrix R(xi_q): (U_P,U_S) -> (D_P,D_S)
    double2* trans = nullptr;      // [NS][2][2] transmission into the upper layer: (U_P,U_S) -> (E_P,E_S)
    double2* squ = nullptr;        // [NS][2] s_b(xi_q) of the upper layer
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
    int* zexp = nullptr;           // zeros: exponent table of the unscaled (gradient) path
    double2* dsdr = nullptr;       // [M][nc][2][2] derivative of the disc scattering matrix in R_m
    // tensor-core spectral path (FP32): exponential factors per (wave, particle, node), rows padded
    // to NSp nodes with zeros, and node-contiguous copies of the FP32 power tables
    float2* es2l = nullptr;        // [2][M][NSp] e^{i xi_q x_m + s_b y_m}
    float2* em2s = nullptr;        // [2][M][NSp] e^{s_b y_m - i xi_q x_m}
    float2* qpmT_m = nullptr;      // [2][nc][NSp] mantissa / exponent of (-i)^n q^n / (i pi s)
    int* qpmT_e = nullptr;
    float2* qpsT_m = nullptr;      // [2][nc][NSp] mantissa / exponent of i^n q^n W_q
    int* qpsT_e = nullptr;
    float2* rho_m2s = nullptr;     // [2][NSp] -i q_b(xi_q): ratio of consecutive M2S powers
    float2* rho_s2l = nullptr;     // [2][NSp]  i q_b(xi_q): ratio of consecutive S2L powers
    int* tc_err = nullptr;         // set by a tensor-core kernel whose pipeline wait gave up
};

struct ms_handle {
    int M = 0, p = 0, nc = 0, NS = 0;
    int NSp = 0;                   // NS rounded up to the tensor-core K chunk (16 nodes)
    double omega = 0;
    double lam_u = 0, mu_u = 0, lam_l = 0, mu_l = 0;
    double kp_u = 0, ks_u = 0, kp_l = 0, ks_l = 0;
    int n_proto = 0;
    bool any_proto = false;
    int n_plist = 0;
    int m2s_rows = 0;              // tensor-core multipole-to-Sommerfeld: rows per K split (0: 2048)
    int tc_kind = 0;               // operand kind of the tensor-core operator kernels in the current call:
                                   // 0 3xTF32 (MS_PREC_FP32), 1 BF16-split (MS_PREC_BF16)
    ms_options opt{};
    MsDeviceTables d;
    std::vector<double> h_centres, h_radius, h_rot, h_protoS;
    std::vector<int> h_bc, h_proto;
    ms_media media{};
    std::vector<int> h_expo;       // host copy of the exponents
    int nnz_near = 0;
    int fmm_levels = 0;            // 0: direct sum over all pairs
    long long seq_len = 0;
    FmmHost fmm;
    PrecondDev pc;
    // workspace sized for ws_nrhs columns
    int ws_nrhs = 0;
    void* ws_x = nullptr;          // scaled input  [M][2][nc][nrhs] (double2 or float2)
    void* ws_a = nullptr;          // scaled local  [M][2][nc][nrhs]
    void* ws_y = nullptr;          // scaled output [M][2][nc][nrhs]
    void* ws_part = nullptr;       // M2S split-K partials [chunks][2][NS][nrhs] (double2)
    void* ws_u = nullptr;          // [2][NS][nrhs] double2 upgoing amplitudes, then reflected D
    void* ws_uf = nullptr;         // [2][NSp][nrhs] float2 copy of the reflected amplitudes (tensor cores)
    int last_cuda = 0;
    // captured operator graphs (ms_options.cuda_graph): key (nrhs, data precision, operand kind, parts,
    // identity / adjoint), workspace input ws_x (ws_y for the adjoint) to output ws_y
    std::map<std::tuple<int, int, int, int, int>, cudaGraphExec_t> graphs;
    cudaStream_t cap_stream = nullptr;
};

// MS_PREC_BF16 runs the FP32 data path with BF16-split operands on the tensor cores: sets h->tc_kind
// and returns the data precision (MS_PREC_FP64 or MS_PREC_FP32), or a negative status.
inline int ms_resolve_prec(ms_handle* h, int prec) {
    if (prec == MS_PREC_BF16) {
        if (!h->opt.tensor_cores) return MS_ERR_UNSUPPORTED;
        h->tc_kind = 1;
        return MS_PREC_FP32;
    }
    if (prec != MS_PREC_FP64 && prec != MS_PREC_FP32) return MS_ERR_ARG;
    h->tc_kind = 0;
    return prec;
}

// internal helpers implemented across the .cu files
int ms_check(ms_handle* h, cudaError_t e);
int ms_ensure_workspace(ms_handle* h, int nrhs);
template <typename T>
int ms_apply_scaled(ms_handle* h, const void* xs, void* ys, int nrhs, int parts, bool identity,
                    cudaStream_t st);
template <typename T>
int ms_local_scaled(ms_handle* h, const void* xs, int nrhs, int parts, cudaStream_t st, int adj = 0);
template <typename T>
int ms_sapply_scaled(ms_handle* h, const void* xs, void* ys, int nrhs, bool identity, bool apply_s,
                     cudaStream_t st, int adj = 0, const void* in = nullptr);
template <typename T>
int ms_apply_adjoint_scaled(ms_handle* h, const void* xs, void* ys, int nrhs, cudaStream_t st);
int ms_sapply_setup(ms_handle* h);
void ms_graphs_free(ms_handle* h);
template <typename T>
int ms_operator_ws(ms_handle* h, int nrhs, int parts, bool identity, bool adjoint, cudaStream_t st);
template <typename T>
int ms_operator_op(ms_handle* h, const void* in, void* out, int nrhs, bool adjoint, cudaStream_t st);
void ms_near_tc_attributes();
int ms_precond_build(ms_handle* h);
void ms_precond_free(ms_handle* h);
template <typename T>
int ms_precond_apply(ms_handle* h, const void* x, void* y, int nrhs, bool adjoint, cudaStream_t st);
int ms_near_store_build(ms_handle* h);
void ms_near_store_free(ms_handle* h);
void ms_sapply_free(ms_handle* h);
template <typename T>
int ms_sapply_proto_launch(ms_handle* h, const void* xs, const void* as, void* ys, int nrhs, bool identity,
                           bool apply_s, int adj, cudaStream_t st);
template <typename T>
int ms_m2s_launch(ms_handle* h, const void* xs, int nrhs, const int* expo, int adj, int* nchunks, cudaStream_t st);
int ms_reflect_launch(ms_handle* h, const double2* part, int nchunks, double2* out, int nrhs, int adj,
                      cudaStream_t st, const double2* table = nullptr);
template <typename T>
int ms_s2l_launch(ms_handle* h, const double2* ud, void* out, int nrhs, const int* expo, int adj, int accumulate,
                  cudaStream_t st);
int ms_fields_upper_impl(ms_handle* h, const void* gamma, int nrhs, const double* rx, int R, void* u, cudaStream_t st);
int ms_build_translations(ms_handle* h, int use_fmm, int leaf_target);
template <typename T>
int ms_translate_scaled(ms_handle* h, const void* xs, int nrhs, bool near, bool far, cudaStream_t st);
template <typename T>
int ms_translate_gen(ms_handle* h, const void* xs, void* dst, int nrhs, bool near, bool far, int adj, int deriv_axis,
                     bool unscaled, cudaStream_t st);
int ms_fmm_workspace(ms_handle* h, int nrhs);
void ms_fmm_free(ms_handle* h);
int ms_to_scaled(ms_handle* h, const void* x, void* xs, int nrhs, int prec, cudaStream_t st, bool local = false);
int ms_spectral_tc_setup(ms_handle* h);
void ms_spectral_tc_free(ms_handle* h);
int ms_m2s_tc_launch(ms_handle* h, const float2* xs, int nrhs, int adj, int* nchunks, cudaStream_t st);
int ms_s2l_tc_launch(ms_handle* h, const double2* ud, float2* out, int nrhs, int adj, int accumulate,
                     cudaStream_t st);
int ms_spectral_tc_status(ms_handle* h, cudaStream_t st);
bool ms_s2l_tc_ok(const ms_handle* h);
int ms_near_tc_launch(ms_handle* h, const float2* xs, float2* dst, int nrhs, cudaStream_t st);
int ms_m2l_tc_launch(ms_handle* h, int b, int lev, const float2* mexp, float2* lexp, int nrhs, cudaStream_t st);
int ms_m2l_tc_tiles(ms_handle* h, int b, int lev, const std::vector<int>& ptr);
void ms_tc_tiles_free(TcTiles& T);
int ms_refine_solve(ms_handle* h, const double2* b, double2* x, int nrhs, double tol, int prec, bool adjoint,
                    ms_solve_info* info, cudaStream_t st, bool guess = false);
template <typename T>
int ms_block_inner(ms_handle* h, int nrhs, long long N, const void* rs, void* ds, double tol, int max_iters,
                   bool adjoint, int& iters, int& matvecs, std::vector<double>& relres, cudaStream_t st,
                   void** cache);
template <typename T>
void ms_block_free(void* cache);
int ms_from_scaled(ms_handle* h, const void* ys, void* y, int nrhs, int prec, cudaStream_t st,
                   bool local = false);
