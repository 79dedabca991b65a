/*
 * ms_b300.h - C ABI of the B300 layered-medium elastic multiple-scattering library.
 *
 * The library applies and solves the coupled multiple-scattering system of
 * arxiv 2608.26875 for M rigid or traction-free particles buried in the lower
 * half-space of a welded two-layer elastic medium (Sec. 2), with the layered
 * response written as Sommerfeld integrals (Sec. 3, 5):
 *
 *     gamma^m = S_m ( a0^m + sum_{l != m} T^{ml} gamma^l + (R gamma)^m )      (mul2, Sec. 4.2;
 *                                                                             Schur complement, Sec. 5.2)
 *
 *   S_m     single-particle scattering matrix (Sec. 4.1, 4.3)
 *   T^{ml}  Graf multipole-to-local translation (Sec. 4.2)
 *   R       interface-reflected operator: multipole-to-Sommerfeld (Sec. 5.4, pts1/sed1/sed2),
 *           2x2 P/S reflection per quadrature node (Sec. 3, aa), Sommerfeld-to-local
 *           (Sec. 5.3, ja/stm/eee1); it includes the self term l = m
 *   a0      local expansion of the transmitted plane wave (Sec. 7.3, bplan)
 *
 * Conventions
 *   - Every call returns an int status: MS_OK (0), a positive warning or a negative error.
 *     No C++ exception crosses the ABI.
 *   - Coefficient blocks are complex, interleaved (re, im) double, in the layout
 *         x[((m * 2 + b) * nc + (n + p)) * nrhs + r]
 *     m particle, b = 0 compressional (alpha / a) or 1 shear (beta / b), n in [-p, p],
 *     r right-hand side; nc = 2p + 1.  The basis is the paper's unscaled one (scatspan, Sec. 4.1).
 *   - "device" pointers are CUDA device memory owned by the caller; "host" pointers are
 *     ordinary host memory owned by the caller.  The handle owns its own tables and workspace.
 *   - Work is ordered on the CUDA stream passed in (cudaStream_t as void*, NULL = default stream).
 *     Calls that need host decisions (ms_solve, ms_grad) synchronise that stream.  A handle must not be
 *     used from two threads at once.
 */
#ifndef MS_B300_H
#define MS_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status codes */
#define MS_OK                    0
#define MS_NOT_CONVERGED         1    /* warning: a column did not reach tol; info holds residuals */
#define MS_ERR_ARG              -1    /* NULL pointer, non-positive size, unknown enum */
#define MS_ERR_CUDA             -2    /* a CUDA runtime call failed; see ms_last_cuda_error */
#define MS_ERR_OVERLAP          -3    /* two enclosing discs closer than 1.1 (R_l + R_m) (Sec. 2) */
#define MS_ERR_NOT_BURIED       -4    /* a particle with y_m + 1.1 R_m > 0 (must lie in x2 < 0, Sec. 2) */
#define MS_ERR_UNSUPPORTED      -5    /* request outside what this library implements */
#define MS_ERR_RECEIVER_INSIDE  -6    /* a receiver inside some particle's enclosing disc, or above y = 0 */
#define MS_ERR_ALLOC            -7    /* device or host allocation failed */
#define MS_ERR_NONFINITE        -9    /* NaN or Inf met in a right-hand side or residual */
#define MS_ERR_BREAKDOWN       -10    /* GMRES breakdown with a non-zero residual */
#define MS_ERR_TOO_LARGE       -11    /* request exceeds the fixed scratch of ms_fields_noalloc */
#define MS_ERR_TIMEOUT         -12    /* a tensor-core kernel gave up waiting on its own pipeline (the
                                         result of that call is invalid; the context stays usable).  A CTA
                                         that gave up still waits, bounded, for its last committed multiplies
                                         before it frees its tensor memory; if that wait also runs out, the
                                         results of other kernels running at the same time are suspect too */

/* ------------------------------------------------------------------ precision of an apply / solve */
#define MS_PREC_FP64   0   /* every operator step in FP64 */
#define MS_PREC_FP32   1   /* translations and spectral contractions in FP32 (scaled basis); solves
                              use FP64 iterative refinement around an FP32 inner GMRES */
#define MS_PREC_BF16   2   /* BF16-split: as MS_PREC_FP32, with the tensor-core contractions of the operator
                              (near pairs, FMM M2L, M2S, S2L, prototype S-apply) on bf16 hi/lo operands,
                              three products (hi hi + hi lo + lo hi) accumulated in FP32: about 2^-16
                              relative error per product.  Needs ms_options.tensor_cores = 1
                              (MS_ERR_UNSUPPORTED otherwise); solves refine in FP64 as for FP32 */

/* ------------------------------------------------------------------ operator parts (ms_operator) */
#define MS_PART_T      1   /* free-space particle-to-particle translation sum_{l != m} T^{ml} */
#define MS_PART_R      2   /* interface-reflected operator R (includes l = m) */
#define MS_PART_S      4   /* left-multiply the selected sum by the scattering matrices S_m */
#define MS_PART_T_NEAR 8   /* only the directly summed near pairs of T (adjacent FMM leaves) */
#define MS_PART_T_FAR 16   /* only the FMM far field of T (zero when the FMM is off) */

/* ------------------------------------------------------------------ inputs */
typedef struct {
    int32_t        M;          /* number of particles (>= 1) */
    const double*  centres;    /* host [M][2]: (x_m, y_m), y_m < 0 */
    const double*  radius;     /* host [M]: enclosing radius R_m > 0 (Sec. 4.3) */
    const int32_t* bc;         /* host [M]: 0 rigid, 1 traction-free (Sec. 2) */
    const int32_t* proto;      /* host [M] or NULL: -1 = disc of radius R_m (closed-form S);
                                  q >= 0 = dense prototype table q below */
    const double*  rotation;   /* host [M] or NULL: rotation angle phi_m of prototype particles (Sec. 4.3) */
    int32_t        n_proto;    /* number of prototype tables (0 if none) */
    const double*  proto_S;    /* host [n_proto][2nc][2nc] complex interleaved, row (b,n) -> column (b',n'),
                                  the unrotated prototype's scattering matrix in its own frame */
} ms_geometry;

typedef struct {
    double lam_u, mu_u;        /* upper layer Lame constants (x2 > 0); density 1 (Sec. 2) */
    double lam_l, mu_l;        /* lower layer Lame constants (x2 < 0) */
} ms_media;

typedef struct {
    int32_t n_panels;          /* uniform Gauss-Legendre panels on [-t_max, t_max] (default 32) */
    int32_t nodes_per_panel;   /* nodes per panel (default 16); N_S = panels * nodes_per_panel, the panels
                                  being the uniform ones split at the graded edges (see grade);
                                  n_panels * nodes_per_panel <= 2^20 */
    double  t_max;             /* contour xi(t) = t - i tanh(t)/2, |t| <= t_max (Sec. 5.1; default 20) */
    int32_t restart;           /* GMRES restart length (default 50; block iterations with block_krylov) */
    int32_t max_iters;         /* total GMRES iteration cap per solve (default 2000) */
    int32_t check_geometry;    /* 1 = validate separation / burial (default 1) */
    int32_t use_fmm;           /* 1 = quadtree FMM for non-adjacent leaves when M is large enough
                                  (default 1); 0 = direct Graf sum over every pair */
    int32_t leaf_target;       /* FMM: target particles per leaf box (default 10) */
    double  depth;             /* contour depth d: xi(t) = t - i d tanh(t) (paper: d = 1/2, the default).
                                  Spectral factors grow like e^{d |x_m - x_l|}: wide domains need
                                  d ~ 3 / (horizontal extent) and panels narrow enough for e^{i t dx} */
    int32_t grade;             /* extra panel edges at each branch point +-kp, +-ks of both layers and
                                  at c +- d 2^j, j < grade (default 0: none) */
    int32_t tensor_cores;      /* MS_PREC_FP32 contractions (near-pair Graf sum, FMM M2L, M2S, S2L, the dense
                                  prototype scattering-matrix apply; the adjoints of the spectral maps):
                                  1 = tcgen05 tensor cores, 3xTF32 split with FP32 accumulation (default);
                                  0 = CUDA-core FP32.  Costs 16 M N_S bytes of device tables. */
    double  inner_tol;         /* ms_solve / ms_grad: relative tolerance of each inner GMRES solve of the
                                  FP64 iterative refinement; 0 = default (1e-3 for MS_PREC_FP32,
                                  1e-7 for MS_PREC_FP64) */
    int32_t block_krylov;      /* ms_solve / ms_solve_rhs / ms_grad: 1 = block GMRES, the right-hand sides
                                  share one Krylov space (default); 0 = one Krylov space per column.  With
                                  block GMRES, restart counts block iterations and the basis holds
                                  (restart + 1) blocks of M (4p + 2) nrhs complex values (FP32 or FP64 as
                                  the inner precision); if they do not fit, restart is halved until they do */
    int32_t cuda_graph;        /* 1 = the operator's kernel sequence (from the handle's scaled input workspace
                                  to its output workspace) is captured into a CUDA graph once per column
                                  count, precision and operator part set, and replayed on the caller's stream
                                  by ms_apply, ms_operator, ms_apply_adjoint and the solves' inner
                                  iterations (default 1); 0 = plain launches.  The graphs are rebuilt when
                                  the workspace grows. */
    int32_t tc_wait_test;      /* test hook for the tensor-core kernels' failure path (default 0 = off).
                                  n > 0: every tensor-core CTA first waits, bounded by n microseconds, on a
                                  barrier that nothing arrives at, gives up, issues no multiply, and the call
                                  returns MS_ERR_TIMEOUT.  Valid range 0..1000000. */
    int32_t store_near;        /* tensor_cores = 1: device-memory budget in GB (0..1024) for the near-pair
                                  Graf operator of the FP32 path, stored as its 3xTF32 tensor-core tiles at
                                  setup (and again when ms_autotune rebuilds the tree) instead of being
                                  generated in every application (default 0 = generate).  Not stored
                                  (silently) when the tiles need more than the budget or would leave less
                                  than 8 GB of the device free.  Same arithmetic either way. */
    int32_t precond_group;     /* ms_solve / ms_solve_rhs / ms_grad with block_krylov: n > 0 = right group-block
                                  Jacobi preconditioner: particles grouped by a uniform grid of cells holding
                                  about n particles (a fuller cell cut into runs of at most 2n), each group's
                                  block I - S T (free-space translations inside the group) inverted in FP64
                                  at setup; costs 24 (2 (2p+1) n_g)^2 bytes per group.  0 = none (default).
                                  Valid range 0..64; ms_setup returns MS_ERR_UNSUPPORTED for more than 65535
                                  groups or a group block wider than 12800 unknowns. */
} ms_options;

typedef struct {
    int32_t       nrhs;
    const int32_t* kind;       /* host [nrhs]: 0 plane P-wave, 1 plane S-wave, from the upper layer */
    const double*  angle;      /* host [nrhs]: direction (cos t, -sin t), t in (0, pi) (Sec. 7.3) */
} ms_incidence;

typedef struct {
    int32_t iterations;        /* total inner GMRES iterations (max over columns) */
    int32_t refinements;       /* FP64 refinement steps (MS_PREC_FP32 solves) */
    int32_t matvecs;           /* operator applications */
    double  max_rel_residual;  /* max over columns of ||b - A x|| / ||b|| in FP64 at exit */
    double  seconds;           /* wall time of the solve */
} ms_solve_info;

typedef struct ms_handle ms_handle;

/* Fill *o with the defaults listed above. */
void ms_default_options(ms_options* o);

/* Build a handle for one geometry, medium, finite frequency omega > 0 and expansion order 0 <= p <= 30
 * (truncation Z_p of Sec. 4.1): wavenumbers (Sec. 2), scattering matrices (closed-form discs,
 * Sec. 4.1; caller prototypes, Sec. 4.3), the Sommerfeld contour and the 2x2 reflection table per
 * node (Sec. 3, 5.1), and device workspace.  Errors: MS_ERR_ARG, MS_ERR_OVERLAP,
 * MS_ERR_NOT_BURIED, MS_ERR_ALLOC, MS_ERR_CUDA.  On error *out is NULL. */
int ms_setup(const ms_geometry* g, const ms_media* md, double omega, int32_t p,
             const ms_options* o, ms_handle** out);

/* y = A x = x - S (T + R) x for nrhs columns (mul2 with the layered Schur complement).
 * x, y: device [M][2][nc][nrhs] complex double; x and y must not overlap.
 * prec: MS_PREC_FP64 or MS_PREC_FP32 (operator steps in FP32; input/output stay FP64). */
int ms_apply(ms_handle* h, const void* x, void* y, int32_t nrhs, int32_t prec, void* stream);

/* y = A^H x = x - (T^H + R^H) S^H x, the conjugate transpose of ms_apply (the system of the adjoint
 * gradient).  Same layouts, precisions and errors as ms_apply. */
int ms_apply_adjoint(ms_handle* h, const void* x, void* y, int32_t nrhs, int32_t prec, void* stream);

/* Building block view of the same operator: y = [S] (T_sel + R_sel) x with parts a mask of
 * MS_PART_T (or its halves MS_PART_T_NEAR, MS_PART_T_FAR) | MS_PART_R | MS_PART_S.  Without
 * MS_PART_S the result is a block of local (incoming) coefficients.  Same layouts and errors as
 * ms_apply. */
int ms_operator(ms_handle* h, const void* x, void* y, int32_t nrhs, int32_t prec, int32_t parts,
                void* stream);

/* b = S a0: right-hand side for plane-wave incidences from the upper layer (Sec. 7.3, bplan).
 * b: device [M][2][nc][inc->nrhs] complex double. */
int ms_rhs(ms_handle* h, const ms_incidence* inc, void* b, void* stream);

/* Solve A gamma = S a0 for the given incidences to relative residual tol (per column, 2-norm)
 * with restarted GMRES (MS_PREC_FP64) or GMRES with FP64 iterative refinement around an FP32
 * inner solve (MS_PREC_FP32).  gamma: device [M][2][nc][nrhs] complex double, overwritten.
 * info may be NULL.  Returns MS_OK, MS_NOT_CONVERGED (positive) or an error. */
int ms_solve(ms_handle* h, const ms_incidence* inc, double tol, int32_t prec, void* gamma,
             ms_solve_info* info, void* stream);

/* b = S a0 for point forces in the upper layer (the point-source incidence of Sec. 7.2): source j at
 * src[2j], src[2j+1] (host, y > 0) with force vector force[2j], force[2j+1] (host; unit density of the
 * upper layer's fundamental solution).  Each source's downgoing spectrum (som1) is transmitted through
 * the welded interface node by node on the handle's contour and expanded about every centre by the
 * Sommerfeld-to-local map.  b: device [M][2][nc][nsrc] complex double, nsrc <= 64.  Errors: MS_ERR_ARG
 * (a source not above the interface, non-finite input), MS_ERR_UNSUPPORTED (nsrc > 64). */
int ms_rhs_point(ms_handle* h, const double* src, const double* force, int32_t nsrc, void* b, void* stream);

/* Solve A gamma = b for a caller-supplied right-hand side b (device [M][2][nc][nrhs] complex double,
 * not modified; e.g. S a0 of ms_rhs, or the coefficients of any incident field), by the same iterative
 * refinement as ms_solve.  gamma: device, same layout; if guess != 0 it holds the initial guess on
 * entry (zero otherwise), and it is overwritten by the solution.  info may be NULL.  Returns MS_OK,
 * MS_NOT_CONVERGED, MS_ERR_NONFINITE (a NaN or Inf in b or in a residual), or another error. */
int ms_solve_rhs(ms_handle* h, const void* b, int32_t nrhs, double tol, int32_t prec, void* gamma, int32_t guess,
                 ms_solve_info* info, void* stream);

/* Scattered displacement at R receivers in the lower layer (Sec. 5, total-field representation):
 * direct outgoing sum of every particle plus the interface-reflected Sommerfeld field.
 * gamma: device [M][2][nc][nrhs]; rx: device [R][2] double; u: device [nrhs][R][2] complex double.
 * Errors: MS_ERR_RECEIVER_INSIDE if a receiver lies in an enclosing disc or at y >= 0. */
int ms_fields(ms_handle* h, const void* gamma, int32_t nrhs, const double* rx, int32_t R, void* u,
              void* stream);

/* Scattered displacement at R receivers in the upper layer (y > 0): the particles' upgoing spectra
 * (multipole-to-Sommerfeld, Sec. 5.4) transmitted through the welded interface (Sec. 3) node by node
 * and summed as upgoing plane waves of the upper layer.  Same layouts as ms_fields; a receiver with
 * y <= 0 gives MS_ERR_RECEIVER_INSIDE. */
int ms_fields_upper(ms_handle* h, const void* gamma, int32_t nrhs, const double* rx, int32_t R, void* u,
                    void* stream);

/* Time-reversal matrix of a mirror of n points in the upper layer (the DORT method of Sec. 7.5):
 * trm host [n][2] (y > 0), 2n <= 64.  The 2n incident fields are point forces at the mirror points,
 * x then y polarised (ms_rhs_point); one batched solve to tol in precision prec; the response
 *     F[(2i + c)][(2j + d)] = component c at mirror point i of the field scattered under force e_d at point j
 * (ms_fields_upper), and T = conj(F)^T F.  Outputs (host, any may be NULL but not all):
 *   F   [2n][2n] complex interleaved;
 *   eig [2n] eigenvalues of T, descending;
 *   vec [2n][2n] complex interleaved, column k the eigenvector of eig[k] (the focusing density).
 * Returns the solve's status (MS_OK or MS_NOT_CONVERGED) or an error. */
int ms_time_reversal(ms_handle* h, const double* trm, int32_t n, double tol, int32_t prec, double* F, double* eig,
                     double* vec, ms_solve_info* info, void* stream);

/* Adjoint gradient of a real loss L of the receiver fields u = ms_fields(gamma) of the solution
 * gamma of ms_solve for the same incidences (the inverse-scattering use, Sec. 7.5): given
 * w = dL/d conj(u) (so that dL = Re sum conj(w) du; for L = 1/2 |u - d|^2, w = u - d), returns
 * dL/d(centres), dL/d(radii) and dL/d(omega) through one transposed solve A^H lambda = F^H w with the
 * adjoint kernels and the position derivatives of the translation and Sommerfeld factors.
 *   gamma: device [M][2][nc][nrhs] (the converged solution); w: device [nrhs][R][2] complex double;
 *   rx: device [R][2]; tol: relative residual of the transposed solve; prec: its inner precision.
 *   g_centres: device [M][2] double or NULL; g_radii: device [M] double or NULL (0 for prototype
 *   particles); g_omega: host double or NULL (central differences of the assembled operator at
 *   omega +- 1e-6 omega, which builds two temporary handles).
 *   info (may be NULL) reports the transposed solve.  Returns MS_OK, MS_NOT_CONVERGED or an error. */
int ms_grad(ms_handle* h, const ms_incidence* inc, const void* gamma, const void* w, const double* rx, int32_t R,
            double tol, int32_t prec, double* g_centres, double* g_radii, double* g_omega, ms_solve_info* info,
            void* stream);

/* Allocation-free variant of ms_fields (the paper has no counterpart: this is a service for
 * callers).  Some callers cannot call cudaMalloc: real-time loops that must never wait on the
 * allocator (cudaMalloc and cudaFree can synchronise the device), or processes whose device memory is
 * owned by a pool sized in advance by the host application.  This call computes exactly what
 * ms_fields computes, with the
 * same arguments, layouts and receiver validation, but allocates nothing: no cudaMalloc, cudaFree
 * or allocating library routine.  Its scratch -- the multipole-to-Sommerfeld partial sums, the
 * reflected spectral amplitudes, a device copy of the radii and a validation flag -- lives in fixed
 * device arrays of about 10 MiB that every GPU which loads the library keeps until the process
 * exits.
 *   Limits: nrhs <= 64, M <= 131072, min(16, M) * 2 * N_S * nrhs <= 524288 and
 *   2 * N_S * nrhs <= 65536 (e.g. N_S = 512 allows nrhs <= 32); beyond them it returns
 *   MS_ERR_TOO_LARGE and touches nothing.
 *   The first call on each device looks up the addresses of the fixed arrays (with that device
 *   current) and keeps them for the rest of the process: they assume that the device's primary
 *   context lives as long as the process (after a cudaDeviceReset they are stale).  Make that first
 *   call before any stream capture.
 *   Every call shares the same arrays and leaves its contents behind: calls that overlap on the
 *   GPU (several streams, several handles or several host threads at once) race and corrupt each
 *   other's results.  Like ms_fields it synchronises `stream` once to read the validation flag. */
int ms_fields_noalloc(ms_handle* h, const void* gamma, int32_t nrhs, const double* rx, int32_t R, void* u,
                      void* stream);

/* Autotuner of the operator's launch shapes for nrhs columns in precision prec: the FMM leaf level (the
 * candidates M / 4^L for L one below, at and one above the current level) and, for the tensor-core FP32
 * path, the K-split size of the multipole-to-Sommerfeld contraction (1024, 2048, 4096 or 8192 rows).
 * Every candidate is timed on this handle (median of three applications of a seeded block after a
 * warm-up); the fastest is kept in the handle and cached for the process by (M, p, N_S, nrhs,
 * precision, tensor cores), so that a later call for a handle of the same sizes applies the cached
 * choice after one timing.  Rebuilding the tree reallocates the handle's translation tables.
 * Outputs (host, may be NULL): the chosen leaf target and split size, and the time of one application
 * in milliseconds with them.  Synchronises the stream. */
int ms_autotune(ms_handle* h, int32_t nrhs, int32_t prec, int32_t* leaf_target, int32_t* m2s_rows,
                double* ms_per_apply, void* stream);

/* Dense tensor-core rate of this GPU for the operand kind of prec (MS_PREC_FP32: kind::tf32;
 * MS_PREC_BF16: kind::f16 with bf16 inputs), measured by a project microkernel with the operator's MMA
 * shapes (M = 128, N = 256, K-major shared-memory operands, FP32 accumulation): one CTA per SM issues
 * iters groups of 32-deep MMAs back to back (the current device; no handle needed).  Outputs (host):
 * TFLOP/s counting 2 M N K flops per MMA, and the milliseconds of the timed launch (may be NULL). */
int ms_tensor_peak(int32_t prec, int32_t iters, double* tflops, double* ms);

/* Sizes of the handle: M, p, N_S, FMM levels (0 = direct sum over all pairs) and the number of
 * ordered particle pairs summed directly.  Any output pointer may be NULL. */
int ms_info(const ms_handle* h, int32_t* M, int32_t* p, int32_t* n_nodes, int32_t* fmm_levels,
            int64_t* near_pairs);

/* Algorithmic work of one application per right-hand-side column, in complex multiply-adds (a
 * complex multiply-add is 8 real flops): near, the directly summed near pairs (nc^2 per ordered pair and
 * wave); far, the FMM's P2M, M2M, M2L, L2L and L2P tasks ((2P_dst + 1)(2P_src + 1) each); refl, the two
 * spectral maps (2 waves x N_S x M x nc each); sapply, the scattering matrices ((2nc)^2 per prototype
 * particle, 4 nc per disc).  Any output may be NULL. */
int ms_work(const ms_handle* h, double* near, double* far, double* refl, double* sapply);

/* Device bytes of the stored near-pair operator (ms_options.store_near) into *bytes: 0 when the
   operator is generated in each application.  MS_ERR_ARG for a NULL argument. */
int ms_near_stored(const ms_handle* h, int64_t* bytes);

/* Release every device buffer of the handle.  NULL is ignored. */
void ms_destroy(ms_handle* h);

/* Static string for a status code. */
const char* ms_status_string(int status);

/* Last CUDA error code (cudaError_t value) recorded by the handle, 0 if none. */
int ms_last_cuda_error(const ms_handle* h);

#ifdef __cplusplus
}
#endif
#endif /* MS_B300_H */
