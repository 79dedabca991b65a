// C ABI entry points other than setup and solve: apply, operator parts, right-hand side,
// sizes, teardown and status strings.
#include <algorithm>
#include <complex>
#include <vector>

#include "common.cuh"
#include "handle.h"

typedef std::complex<double> cd;
bool ms_plane_wave_transmission(const ms_handle* h, int kind, double angle, double* xi_out, cd D[2]);
bool ms_point_force_transmission(const ms_handle* h, cd xi, const double z[2], const double q[2], cd D[2]);

int ms_check(ms_handle* h, cudaError_t e) {
    if (e == cudaSuccess) return MS_OK;
    if (h) h->last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? MS_ERR_ALLOC : MS_ERR_CUDA;
}

static void dfree(void*& p) {
    if (p) cudaFree(p);
    p = nullptr;
}
template <typename X>
static void dfree_t(X*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

int ms_ensure_workspace(ms_handle* h, int nrhs) {
    if (h->ws_nrhs >= nrhs) return MS_OK;
    ms_graphs_free(h);              // captured graphs hold the old workspace addresses
    dfree(h->ws_x);
    dfree(h->ws_a);
    dfree(h->ws_y);
    dfree(h->ws_part);
    dfree(h->ws_u);
    dfree(h->ws_uf);
    h->ws_nrhs = 0;
    size_t nvec = (size_t)h->M * 2 * h->nc * nrhs * sizeof(double2);
    size_t npart = (size_t)64 * 2 * h->NS * nrhs * sizeof(double2);
    size_t nu = (size_t)2 * h->NS * nrhs * sizeof(double2);
    cudaError_t e;
    if ((e = cudaMalloc(&h->ws_x, nvec)) != cudaSuccess || (e = cudaMalloc(&h->ws_a, nvec)) != cudaSuccess ||
        (e = cudaMalloc(&h->ws_y, nvec)) != cudaSuccess || (e = cudaMalloc(&h->ws_part, npart)) != cudaSuccess ||
        (e = cudaMalloc(&h->ws_u, nu)) != cudaSuccess ||
        (e = cudaMalloc(&h->ws_uf, (size_t)2 * std::max(h->NSp, h->NS) * nrhs * sizeof(float2))) != cudaSuccess) {
        h->last_cuda = (int)e;
        return MS_ERR_ALLOC;
    }
    if (int rc = ms_fmm_workspace(h, nrhs)) return rc;
    h->ws_nrhs = nrhs;
    return MS_OK;
}

static int check_call(ms_handle* h, const void* x, void* y, int nrhs, int prec) {
    if (!h || !x || !y || nrhs < 1) return MS_ERR_ARG;
    if (prec != MS_PREC_FP64 && prec != MS_PREC_FP32) return MS_ERR_ARG;     // (after ms_resolve_prec)
    if (nrhs > 64) return MS_ERR_UNSUPPORTED;
    return ms_ensure_workspace(h, nrhs);
}

static int apply_common(ms_handle* h, const void* x, void* y, int nrhs, int prec, int parts, bool identity,
                        cudaStream_t st) {
    int rc;
    if ((rc = ms_to_scaled(h, x, h->ws_x, nrhs, prec, st))) return rc;
    if (prec == MS_PREC_FP64)
        rc = ms_operator_ws<double>(h, nrhs, parts, identity, false, st);
    else
        rc = ms_operator_ws<float>(h, nrhs, parts, identity, false, st);
    if (rc) return rc;
    // without S the result is a local (incoming) block, scaled the other way
    bool local = !(parts & MS_PART_S) && (parts & (MS_PART_T | MS_PART_R | MS_PART_T_NEAR | MS_PART_T_FAR));
    if ((rc = ms_from_scaled(h, h->ws_y, y, nrhs, prec, st, local))) return rc;
    if (prec == MS_PREC_FP32 && h->opt.tensor_cores) return ms_spectral_tc_status(h, st);
    return MS_OK;
}

extern "C" int ms_apply(ms_handle* h, const void* x, void* y, int32_t nrhs, int32_t prec, void* stream) {
    if (!h) return MS_ERR_ARG;
    if ((prec = ms_resolve_prec(h, prec)) < 0) return prec;
    int rc = check_call(h, x, y, nrhs, prec);
    if (rc) return rc;
    return apply_common(h, x, y, nrhs, prec, MS_PART_T | MS_PART_R | MS_PART_S, true, (cudaStream_t)stream);
}

extern "C" int ms_operator(ms_handle* h, const void* x, void* y, int32_t nrhs, int32_t prec, int32_t parts,
                           void* stream) {
    if (!h) return MS_ERR_ARG;
    if ((prec = ms_resolve_prec(h, prec)) < 0) return prec;
    int rc = check_call(h, x, y, nrhs, prec);
    if (rc) return rc;
    if (parts & ~(MS_PART_T | MS_PART_R | MS_PART_S | MS_PART_T_NEAR | MS_PART_T_FAR)) return MS_ERR_ARG;
    return apply_common(h, x, y, nrhs, prec, parts, false, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ plane-wave right-hand side
// a~0[m,b,n,r] (+)= 2^{a_{m,b,n}} D_b(r) e^{i xi_r x_m + s_{b,r} y_m} i^n q_{b,r}^n  (Jacobi-Anger about
// x_m); expo = zeros gives the unscaled a0.
__global__ void k_incident(double2* __restrict__ as, const double2* __restrict__ centre, const int* __restrict__ expo,
                           const double* __restrict__ xi, const double2* __restrict__ amp,
                           const double2* __restrict__ s, const double2* __restrict__ q, int M, int p, int nrhs,
                           int accumulate) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int nc = 2 * p + 1;
    long long total = (long long)M * 2 * nc * nrhs;
    if (i >= total) return;
    int r = (int)(i % nrhs);
    long long row = i / nrhs;
    int ni = (int)(row % nc);
    int b = (int)((row / nc) % 2);
    int m = (int)(row / (2 * nc));
    int n = ni - p;
    double2 c = centre[m];
    double2 sb = s[r * 2 + b], qb = q[r * 2 + b];
    double re = sb.x * c.y;
    double im = xi[r] * c.x + sb.y * c.y;
    double mag = exp(re), sn, cs;
    sincos(im, &sn, &cs);
    double2 v = cmul(amp[r * 2 + b], make_double2(mag * cs, mag * sn));
    // i^n q^n by repeated multiplication (|n| <= 30)
    double2 f = make_double2(1.0, 0.0);
    double2 iq = cmul(make_double2(0.0, 1.0), qb);
    if (n < 0) iq = cdiv(make_double2(1.0, 0.0), iq);
    int an = n < 0 ? -n : n;
    for (int k = 0; k < an; ++k) f = cmul(f, iq);
    double sc = pow2d(expo[row]);
    v = cmul(v, f);
    v = make_double2(v.x * sc, v.y * sc);
    as[i] = accumulate ? cadd(as[i], v) : v;
}

void ms_incident_launch(ms_handle* h, const double* xi, const double2* amp, const double2* s, const double2* q,
                        double2* out, const int* expo, int nrhs, int accumulate, cudaStream_t st) {
    long long total = (long long)h->M * 2 * h->nc * nrhs;
    k_incident<<<(int)((total + 255) / 256), 256, 0, st>>>(out, h->d.centre, expo, xi, amp, s, q, h->M, h->p, nrhs,
                                                          accumulate);
}

extern "C" int ms_rhs(ms_handle* h, const ms_incidence* inc, void* b, void* stream) {
    if (!h || !inc || !b || !inc->kind || !inc->angle) return MS_ERR_ARG;
    const int nrhs = inc->nrhs;
    int rc = check_call(h, b, b, nrhs, MS_PREC_FP64);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<double> xi(nrhs);
    std::vector<double2> amp(nrhs * 2), s(nrhs * 2), q(nrhs * 2);
    for (int r = 0; r < nrhs; ++r) {
        if ((inc->kind[r] != 0 && inc->kind[r] != 1) || !(inc->angle[r] > 0) || !(inc->angle[r] < M_PI))
            return MS_ERR_ARG;
        cd D[2];
        if (!ms_plane_wave_transmission(h, inc->kind[r], inc->angle[r], &xi[r], D)) return MS_ERR_ARG;
        for (int bb = 0; bb < 2; ++bb) {
            double k = bb ? h->ks_l : h->kp_l;
            cd x(xi[r], 0.0);
            cd sv = cd(0, -1) * std::sqrt(cd(k * k - xi[r] * xi[r], 0.0));
            cd qv = (x - sv) / k;
            amp[r * 2 + bb] = make_double2(D[bb].real(), D[bb].imag());
            s[r * 2 + bb] = make_double2(sv.real(), sv.imag());
            q[r * 2 + bb] = make_double2(qv.real(), qv.imag());
        }
    }
    double *d_xi = nullptr;
    double2 *d_amp = nullptr, *d_s = nullptr, *d_q = nullptr;
    cudaError_t e;
    if ((e = cudaMalloc(&d_xi, nrhs * sizeof(double))) || (e = cudaMalloc(&d_amp, nrhs * 2 * sizeof(double2))) ||
        (e = cudaMalloc(&d_s, nrhs * 2 * sizeof(double2))) || (e = cudaMalloc(&d_q, nrhs * 2 * sizeof(double2)))) {
        cudaFree(d_xi); cudaFree(d_amp); cudaFree(d_s); cudaFree(d_q);
        return ms_check(h, e);
    }
    cudaMemcpyAsync(d_xi, xi.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_amp, amp.data(), nrhs * 2 * sizeof(double2), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_s, s.data(), nrhs * 2 * sizeof(double2), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_q, q.data(), nrhs * 2 * sizeof(double2), cudaMemcpyHostToDevice, st);
    ms_incident_launch(h, d_xi, d_amp, d_s, d_q, (double2*)h->ws_a, h->d.expo, nrhs, 0, st);
    rc = ms_check(h, cudaGetLastError());
    // b~ = S~ a~0 (identity off, S on, no operator part: the workspace a~ is used as is)
    if (!rc) rc = ms_sapply_scaled<double>(h, h->ws_x, h->ws_y, nrhs, false, true, st);
    if (!rc) rc = ms_from_scaled(h, h->ws_y, b, nrhs, MS_PREC_FP64, st);
    cudaStreamSynchronize(st);
    cudaFree(d_xi); cudaFree(d_amp); cudaFree(d_s); cudaFree(d_q);
    return rc;
}

// b = S a0 for point forces in the upper layer (Sec. 7.2): per node the transmitted amplitudes of each
// source (host, FP64), then the Sommerfeld-to-local map and the scattering matrices on the device.
extern "C" int ms_rhs_point(ms_handle* h, const double* src, const double* force, int32_t nsrc, void* b,
                            void* stream) {
    if (!h || !src || !force || !b || nsrc < 1) return MS_ERR_ARG;
    if (nsrc > 64) return MS_ERR_UNSUPPORTED;
    for (int j = 0; j < nsrc; ++j)
        if (!std::isfinite(src[2 * j]) || !(src[2 * j + 1] > 0) || !std::isfinite(src[2 * j + 1]) ||
            !std::isfinite(force[2 * j]) || !std::isfinite(force[2 * j + 1]))
            return MS_ERR_ARG;
    int rc = check_call(h, b, b, nsrc, MS_PREC_FP64);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int NS = h->NS;
    std::vector<double2> node(NS), ud((size_t)2 * NS * nsrc);
    if ((rc = ms_check(h, cudaMemcpy(node.data(), h->d.node, NS * sizeof(double2), cudaMemcpyDeviceToHost))))
        return rc;
    for (int q = 0; q < NS; ++q) {
        const cd xi(node[q].x, node[q].y);
        for (int r = 0; r < nsrc; ++r) {
            cd D[2];
            if (!ms_point_force_transmission(h, xi, src + 2 * r, force + 2 * r, D)) return MS_ERR_ARG;
            ud[((size_t)0 * NS + q) * nsrc + r] = make_double2(D[0].real(), D[0].imag());
            ud[((size_t)1 * NS + q) * nsrc + r] = make_double2(D[1].real(), D[1].imag());
        }
    }
    if ((rc = ms_check(h, cudaMemcpyAsync(h->ws_u, ud.data(), ud.size() * sizeof(double2), cudaMemcpyHostToDevice,
                                          st))))
        return rc;
    if ((rc = ms_s2l_launch<double>(h, (const double2*)h->ws_u, h->ws_a, nsrc, h->d.expo, 0, 0, st))) return rc;
    if ((rc = ms_sapply_scaled<double>(h, h->ws_x, h->ws_y, nsrc, false, true, st))) return rc;
    if ((rc = ms_from_scaled(h, h->ws_y, b, nsrc, MS_PREC_FP64, st))) return rc;
    return ms_check(h, cudaStreamSynchronize(st));
}

extern "C" int ms_info(const ms_handle* h, int32_t* M, int32_t* p, int32_t* n_nodes, int32_t* fmm_levels,
                       int64_t* near_pairs) {
    if (!h) return MS_ERR_ARG;
    if (M) *M = h->M;
    if (p) *p = h->p;
    if (n_nodes) *n_nodes = h->NS;
    if (fmm_levels) *fmm_levels = h->fmm_levels;
    if (near_pairs) *near_pairs = h->nnz_near;
    return MS_OK;
}

extern "C" int ms_work(const ms_handle* h, double* near, double* far, double* refl, double* sapply) {
    if (!h) return MS_ERR_ARG;
    const double nc = h->nc;
    if (near) *near = h->fmm.work_near;
    if (far) *far = h->fmm.work_far;
    if (refl) *refl = 2.0 * 2.0 * h->NS * h->M * nc;                // M2S and S2L, both waves
    if (sapply) {
        const double np = h->n_plist;
        *sapply = np * (2 * nc) * (2 * nc) + (h->M - np) * nc * 4.0;   // dense prototypes, 2 x 2 disc blocks
    }
    return MS_OK;
}

extern "C" int ms_near_stored(const ms_handle* h, int64_t* bytes) {
    if (!h || !bytes) return MS_ERR_ARG;
    *bytes = h->fmm.near_store ? 2 * h->fmm.near_store_wave : 0;
    return MS_OK;
}

extern "C" void ms_destroy(ms_handle* h) {
    if (!h) return;
    dfree_t(h->d.centre); dfree_t(h->d.expo); dfree_t(h->d.sdisc); dfree_t(h->d.sdisc_f);
    dfree_t(h->d.proto); dfree_t(h->d.rot); ms_sapply_free(h); dfree_t(h->d.node); dfree_t(h->d.wq);
    dfree_t(h->d.sq); dfree_t(h->d.qq); dfree_t(h->d.refl); dfree_t(h->d.trans); dfree_t(h->d.squ); dfree_t(h->d.qpow_m2s); dfree_t(h->d.qpow_s2l);
    dfree_t(h->d.qpm_m); dfree_t(h->d.qpm_e); dfree_t(h->d.qps_m); dfree_t(h->d.qps_e);
    dfree_t(h->d.zexp); dfree_t(h->d.dsdr);
    ms_graphs_free(h);
    ms_spectral_tc_free(h);
    ms_fmm_free(h);
    ms_precond_free(h);
    dfree(h->ws_x); dfree(h->ws_a); dfree(h->ws_y); dfree(h->ws_part); dfree(h->ws_u); dfree(h->ws_uf);
    delete h;
}

extern "C" const char* ms_status_string(int s) {
    switch (s) {
        case MS_OK: return "ok";
        case MS_NOT_CONVERGED: return "not converged";
        case MS_ERR_ARG: return "invalid argument";
        case MS_ERR_CUDA: return "CUDA error";
        case MS_ERR_OVERLAP: return "enclosing discs closer than 1.1 (R_l + R_m)";
        case MS_ERR_NOT_BURIED: return "particle not buried below the interface";
        case MS_ERR_UNSUPPORTED: return "unsupported request";
        case MS_ERR_RECEIVER_INSIDE: return "receiver inside an enclosing disc or not below the interface";
        case MS_ERR_ALLOC: return "device allocation failed";
        case MS_ERR_NONFINITE: return "non-finite value";
        case MS_ERR_BREAKDOWN: return "GMRES breakdown";
        case MS_ERR_TOO_LARGE: return "request exceeds the fixed scratch of the allocation-free call";
        case MS_ERR_TIMEOUT: return "a tensor-core kernel gave up waiting on its pipeline";
        default: return "unknown status";
    }
}

extern "C" int ms_last_cuda_error(const ms_handle* h) { return h ? h->last_cuda : 0; }
