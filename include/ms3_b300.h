/*
 * ms3_b300.h - C ABI of the 3D extension (Sec. 6): rigid or traction-free spheres buried in the lower
 * half-space z < 0 of two welded elastic half-spaces, vector spherical wave expansions, and the layered
 * response as 2D Sommerfeld integrals in polar form (Sec. 6.1).  The coupled system has the same three
 * parts as in 2D (Sec. 6.2, 6.3; the block system aequ2):
 *
 *     tau^m = S_m ( a0^m + sum_{l != m} T^{ml} tau^l + (R tau)^m )
 *
 *   tau^m   outgoing coefficients of sphere m: alpha_nm (N-type shear waves curl curl(x v^{ks'}) / (i ks')),
 *           beta_nm (M-type shear waves curl(x v^{ks'})), n = 1..p, and gamma_nm (L-type compressional
 *           waves grad v^{kp'}), n = 0..p, |m| <= n; v^k_nm = h_n(k r) Y_n^m with
 *           Y_n^m = sqrt((2n+1)/(4 pi) (n-|m|)!/(n+|m|)!) P_n^|m|(cos theta) e^{i m phi}, P_n^|m| without
 *           the Condon-Shortley sign (so Y_n^-m = conj(Y_n^m), as the plane-wave coefficients of Sec. 6.3
 *           require)
 *   S_m     closed-form sphere scattering matrix: per order n a 2 x 2 block on (alpha, gamma) and a
 *           scalar on beta, from u = 0 (rigid) or sigma n = 0 (traction-free) on r = R_m
 *   T^{ml}  free-space translation of sphere l's outgoing field into regular waves about sphere m
 *           (the homogeneous-medium part, block D)
 *   R       the interface-reflected part: outgoing waves to upgoing P, SV, SH plane waves at each
 *           Sommerfeld node (block B, Sec. 6.2), their reflection at z = 0, and the downgoing waves to
 *           regular waves about every sphere (block C, Sec. 6.3), self term included
 *   a0      regular expansion of the transmitted field of a plane wave from the upper layer
 *
 * Coefficient blocks: complex interleaved double, x[(m * T + k) * nrhs + r], T = 2 p (p + 2) + (p + 1)^2,
 * k = idx(n, m) - 1 for alpha (n >= 1), p (p + 2) + idx(n, m) - 1 for beta, 2 p (p + 2) + idx(n, m) for
 * gamma, idx(n, m) = n^2 + n + m.  Device pointers are caller-owned CUDA memory; work is ordered on the
 * stream passed in (NULL = default); status codes are those of ms_b300.h.
 */
#ifndef MS3_B300_H
#define MS3_B300_H

#include <stdint.h>

#include "ms_b300.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ms3_handle ms3_handle;

typedef struct {
    int32_t        M;          /* number of spheres (>= 1) */
    const double*  centres;    /* host [M][3]: (x, y, z), z + 1.1 R < 0 */
    const double*  radius;     /* host [M]: R_m > 0 */
    const int32_t* bc;         /* host [M]: 0 rigid (u = 0), 1 traction-free (sigma n = 0) */
} ms3_geometry;

typedef struct {
    int32_t n_r;               /* Gauss-Legendre nodes in t on [0, t_max] (default 128) */
    int32_t n_theta;           /* equispaced angles (default 64); n_r * n_theta <= 2^18 */
    int32_t n_panels;          /* equal panels the n_r nodes are split into (default 4; must divide n_r) */
    double  t_max;             /* radial contour k_rho = t - i alpha tanh(beta t), t in [0, t_max] (default 10) */
    double  alpha;             /* contour depth (default 1; wide clouds need ~3 / horizontal extent) */
    double  beta;              /* contour steepness (default 1) */
    int32_t restart;           /* block GMRES restart length in block iterations (default 60) */
    int32_t max_iters;         /* block GMRES iteration cap (default 1000) */
} ms3_options;

typedef struct {
    int32_t        nrhs;       /* plane waves (1..64) */
    const int32_t* kind;       /* host [nrhs]: 0 P, 1 SV, 2 SH wave in the upper layer */
    const double*  theta;      /* host [nrhs]: angle from the downward vertical, [0, pi/2) */
    const double*  phi;        /* host [nrhs]: azimuth of the horizontal direction */
} ms3_incidence;

/* Operator parts for ms3_operator */
#define MS3_PART_T 1           /* free-space translations between spheres */
#define MS3_PART_R 2           /* the interface-reflected part (self terms included) */
#define MS3_PART_S 4           /* apply S and form tau - S(...) (else the incoming coefficients themselves) */

/* Defaults into *o.  NULL is ignored. */
void ms3_default_options(ms3_options* o);

/* Handle for the geometry, media (Lame pairs of both layers, unit density), finite omega > 0 and order
 * 1 <= p <= 10.  Host-side validation (MS_ERR_ARG, MS_ERR_NOT_BURIED, MS_ERR_OVERLAP: centres closer
 * than 1.1 (R_l + R_m)) precedes any device work.  Tables: the sphere matrices, per-node spectral
 * factors of blocks B and C and the reflection matrices (about 16 (2 (T + p(p+2)) + 9) N_S bytes,
 * N_S = n_r n_theta), translation coefficient tables.  MS_ERR_ALLOC if a device or host allocation fails.  *out is NULL on
 * failure. */
int ms3_setup(const ms3_geometry* g, const ms_media* md, double omega, int32_t p, const ms3_options* o,
              ms3_handle** out);

/* y = x - S (T + R) x for nrhs (1..64) columns: prec MS_PREC_FP64 (FP64 tables and arithmetic) or
 * MS_PREC_FP32 (FP32 tables and arithmetic, blocks converted on the way in and out).
 * x, y: device [M][T][nrhs] complex double, y != x. */
int ms3_apply(ms3_handle* h, const void* x, void* y, int32_t nrhs, int32_t prec, void* stream);

/* The parts selected by MS3_PART_* bits: with MS3_PART_S, y = x - S (sum of parts) x; without it,
 * y = (sum of parts) x (incoming coefficients).  Same layouts, precisions and limits as ms3_apply. */
int ms3_operator(ms3_handle* h, const void* x, void* y, int32_t nrhs, int32_t parts, int32_t prec, void* stream);

/* b = S a0 for plane waves from the upper layer (their transmitted field's regular expansion about each
 * sphere).  b: device [M][T][inc->nrhs]. */
int ms3_rhs(ms3_handle* h, const ms3_incidence* inc, void* b, void* stream);

/* Solve A tau = S a0 to relative residual tol per column (FP64 residuals) with block GMRES over the
 * columns: prec MS_PREC_FP64 (FP64 operator and basis) or MS_PREC_FP32 (FP64 iterative refinement around
 * FP32 block GMRES solves to 1e-3).  tau: device [M][T][nrhs], overwritten.  info may be NULL.  MS_OK,
 * MS_NOT_CONVERGED or an error.  Synchronises the stream. */
int ms3_solve(ms3_handle* h, const ms3_incidence* inc, double tol, int32_t prec, void* tau, ms_solve_info* info,
              void* stream);

/* M, p, coefficients per sphere T, Sommerfeld nodes N_S.  Any output may be NULL. */
int ms3_info(const ms3_handle* h, int32_t* M, int32_t* p, int32_t* T, int32_t* n_nodes);

/* Release the handle's device buffers.  NULL is ignored. */
void ms3_destroy(ms3_handle* h);

#ifdef __cplusplus
}
#endif

#endif
