// Scattered displacement at receivers in the lower layer (Sec. 5, total-field representation):
//   u(x) = sum_m sum_n alpha^m_n grad(H_n(kp' r_m) e^{in th_m}) + beta^m_n grad_perp(H_n(ks' r_m) e^{in th_m})
//        + int [D_P grad(e^{i xi x + s'_p y}) + D_S grad_perp(e^{i xi x + s'_s y})] dxi,
// with (D_P, D_S) = R(xi) (U_P, U_S) the interface-reflected amplitudes of the same outgoing
// coefficients.  Derivatives of cylindrical waves use the order shifts of DLMF 10.6:
//   d/dx (H_n e^{in th}) = (k/2)(h_{n-1} - h_{n+1}),  d/dy = (ik/2)(h_{n-1} + h_{n+1}).
// Everything here is FP64.
#include <algorithm>
#include <mutex>

#include "bessel.cuh"
#include "common.cuh"
#include "handle.h"

namespace {

__global__ void k_check_receivers(const double2* __restrict__ rx, const double2* __restrict__ centre,
                                   const double* __restrict__ radius, int R, int M, int* flag) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)R * M) return;
    int k = (int)(i / M), m = (int)(i % M);
    double2 x = rx[k];
    if (m == 0 && !(x.y < 0.0)) atomicExch(flag, 1);
    double dx = x.x - centre[m].x, dy = x.y - centre[m].y;
    double lim = 1.1 * radius[m];
    if (dx * dx + dy * dy < lim * lim) atomicExch(flag, 1);
}

constexpr int FLD_NB = 16;

__global__ void __launch_bounds__(256)
k_fields_direct(const double2* __restrict__ gam, const double2* __restrict__ rx, const double2* __restrict__ centre,
                double2* __restrict__ u, int M, int p, int nrhs, int R, double kp, double ks) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = p + 1, nh = 2 * K + 1, nc = 2 * p + 1;
    double2* hs = reinterpret_cast<double2*>(smem_raw);                 // [NB][2][nh]
    double* scratch = reinterpret_cast<double*>(hs + FLD_NB * 2 * nh);   // [NB*2][2][K+1]
    const int k = blockIdx.x;
    const double2 x = rx[k];
    const int t = threadIdx.x;
    const int r = t >> 1, comp = t & 1;
    double2 acc = make_double2(0, 0);
    for (int base = 0; base < M; base += FLD_NB) {
        const int nb = min(FLD_NB, M - base);
        __syncthreads();
        if (t < 2 * nb) {
            int s = t >> 1, b = t & 1;
            double2 c = centre[base + s];
            double dx = x.x - c.x, dy = x.y - c.y;
            double d = sqrt(dx * dx + dy * dy);
            double* J = scratch + (size_t)t * 2 * (K + 1);
            hankel_phase_seq(K, (b ? ks : kp) * d, dx / d, dy / d, hs + (s * 2 + b) * nh, J, J + (K + 1));
        }
        __syncthreads();
        if (r < nrhs) {
            for (int s = 0; s < nb; ++s) {
                const int m = base + s;
                const double2* hp = hs + (s * 2 + 0) * nh;
                const double2* hv = hs + (s * 2 + 1) * nh;
                const double2* ga = gam + ((size_t)(m * 2 + 0) * nc) * nrhs + r;
                const double2* gb = gam + ((size_t)(m * 2 + 1) * nc) * nrhs + r;
                for (int i = 0; i < nc; ++i) {
                    int n = i - p;
                    double2 a = ga[(size_t)i * nrhs], be = gb[(size_t)i * nrhs];
                    double2 pm = hp[n - 1 + K], pp = hp[n + 1 + K];
                    double2 sm = hv[n - 1 + K], sp = hv[n + 1 + K];
                    // dx, dy of the P wave and of the S wave
                    double2 pdx = cscale(csub(pm, pp), 0.5 * kp);
                    double2 pdy = cmul(make_double2(0.0, 0.5 * kp), cadd(pm, pp));
                    double2 sdx = cscale(csub(sm, sp), 0.5 * ks);
                    double2 sdy = cmul(make_double2(0.0, 0.5 * ks), cadd(sm, sp));
                    if (comp == 0) {            // u1 = dphi/dx - dpsi/dy
                        cfma(acc, a, pdx);
                        cfma(acc, be, make_double2(-sdy.x, -sdy.y));
                    } else {                    // u2 = dphi/dy + dpsi/dx
                        cfma(acc, a, pdy);
                        cfma(acc, be, sdx);
                    }
                }
            }
        }
    }
    if (r < nrhs) u[((size_t)r * R + k) * 2 + comp] = acc;
}

// u += sum_q W_q [D_P (i xi, s_p) e^{i xi X + s_p Y} + D_S (-s_s, i xi) e^{i xi X + s_s Y}]
__global__ void k_fields_refl(const double2* __restrict__ ud, const double2* __restrict__ rx,
                              const double2* __restrict__ node, const double2* __restrict__ wq,
                              const double2* __restrict__ sq, double2* __restrict__ u, int NS, int nrhs, int R) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * nrhs) return;
    int k = i / nrhs, r = i % nrhs;
    double2 x = rx[k];
    double2 u1 = make_double2(0, 0), u2 = make_double2(0, 0);
    for (int q = 0; q < NS; ++q) {
        double2 xi = node[q], w = wq[q];
        double2 ixi = make_double2(-xi.y, xi.x);
        for (int b = 0; b < 2; ++b) {
            double2 s = sq[q * 2 + b];
            // exponent i xi X + s Y
            double re = -xi.y * x.x + s.x * x.y;
            double im = xi.x * x.x + s.y * x.y;
            double mag = exp(re), sn, cs;
            sincos(im, &sn, &cs);
            double2 e = cmul(cmul(make_double2(mag * cs, mag * sn), w), ud[((size_t)b * NS + q) * nrhs + r]);
            if (b == 0) {
                u1 = cadd(u1, cmul(ixi, e));
                u2 = cadd(u2, cmul(s, e));
            } else {
                u1 = csub(u1, cmul(s, e));
                u2 = cadd(u2, cmul(ixi, e));
            }
        }
    }
    u[((size_t)r * R + k) * 2 + 0] = cadd(u[((size_t)r * R + k) * 2 + 0], u1);
    u[((size_t)r * R + k) * 2 + 1] = cadd(u[((size_t)r * R + k) * 2 + 1], u2);
}

// Upper layer: u = sum_q W_q [E_P (i xi, -s_p) e^{i xi X - s_p Y} + E_S (s_s, i xi) e^{i xi X - s_s Y}] with
// (E_P, E_S) = T(xi)(U_P, U_S) the transmitted upgoing amplitudes (upper-layer s).
__global__ void k_fields_upper(const double2* __restrict__ ue, const double2* __restrict__ rx,
                               const double2* __restrict__ node, const double2* __restrict__ wq,
                               const double2* __restrict__ squ, double2* __restrict__ u, int NS, int nrhs, int R) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R * nrhs) return;
    int k = i / nrhs, r = i % nrhs;
    double2 x = rx[k];
    double2 u1 = make_double2(0, 0), u2 = make_double2(0, 0);
    for (int q = 0; q < NS; ++q) {
        double2 xi = node[q], w = wq[q];
        double2 ixi = make_double2(-xi.y, xi.x);
        for (int b = 0; b < 2; ++b) {
            double2 s = squ[q * 2 + b];
            // exponent i xi X - s Y
            double re = -xi.y * x.x - s.x * x.y;
            double im = xi.x * x.x - s.y * x.y;
            double mag = exp(re), sn, cs;
            sincos(im, &sn, &cs);
            double2 e = cmul(cmul(make_double2(mag * cs, mag * sn), w), ue[((size_t)b * NS + q) * nrhs + r]);
            if (b == 0) {
                u1 = cadd(u1, cmul(ixi, e));
                u2 = csub(u2, cmul(s, e));
            } else {
                u1 = cadd(u1, cmul(s, e));
                u2 = cadd(u2, cmul(ixi, e));
            }
        }
    }
    u[((size_t)r * R + k) * 2 + 0] = u1;
    u[((size_t)r * R + k) * 2 + 1] = u2;
}

__global__ void k_check_upper(const double2* __restrict__ rx, int R, int* flag) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < R && !(rx[k].y > 0.0)) atomicExch(flag, 1);
}

}  // namespace

// Scattered displacement at receivers in the upper layer (shared by ms_fields_upper and the time
// reversal): multipole-to-Sommerfeld of gamma, transmission per node, the upgoing plane-wave sum.
int ms_fields_upper_impl(ms_handle* h, const void* gamma, int nrhs, const double* rx, int R, void* u,
                         cudaStream_t st) {
    int rc = ms_ensure_workspace(h, nrhs);
    if (rc) return rc;
    int* flag = nullptr;
    if ((rc = ms_check(h, cudaMalloc(&flag, sizeof(int))))) return rc;
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    k_check_upper<<<(R + 255) / 256, 256, 0, st>>>((const double2*)rx, R, flag);
    int hflag = 0;
    cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    rc = ms_check(h, cudaStreamSynchronize(st));
    cudaFree(flag);
    if (rc) return rc;
    if (hflag) return MS_ERR_RECEIVER_INSIDE;
    if ((rc = ms_to_scaled(h, gamma, h->ws_x, nrhs, MS_PREC_FP64, st))) return rc;
    int chunks = 0;
    if ((rc = ms_m2s_launch<double>(h, h->ws_x, nrhs, h->d.expo, 0, &chunks, st))) return rc;
    if ((rc = ms_reflect_launch(h, (const double2*)h->ws_part, chunks, (double2*)h->ws_u, nrhs, 0, st, h->d.trans)))
        return rc;
    k_fields_upper<<<(R * nrhs + 127) / 128, 128, 0, st>>>((const double2*)h->ws_u, (const double2*)rx, h->d.node,
                                                           h->d.wq, h->d.squ, (double2*)u, h->NS, nrhs, R);
    return ms_check(h, cudaGetLastError());
}

extern "C" int ms_fields_upper(ms_handle* h, const void* gamma, int32_t nrhs, const double* rx, int32_t R, void* u,
                               void* stream) {
    if (!h || !gamma || !rx || !u || nrhs < 1 || R < 1) return MS_ERR_ARG;
    if (nrhs > 64) return MS_ERR_UNSUPPORTED;
    return ms_fields_upper_impl(h, gamma, nrhs, rx, R, u, (cudaStream_t)stream);
}

extern "C" int ms_fields(ms_handle* h, const void* gamma, int32_t nrhs, const double* rx, int32_t R, void* u,
                         void* stream) {
    if (!h || !gamma || !rx || !u || nrhs < 1 || R < 1) return MS_ERR_ARG;
    if (nrhs > 64) return MS_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ms_ensure_workspace(h, nrhs);
    if (rc) return rc;
    // receiver validation
    int* flag = nullptr;
    double* rad = nullptr;
    if ((rc = ms_check(h, cudaMalloc(&flag, sizeof(int))))) return rc;
    if ((rc = ms_check(h, cudaMalloc(&rad, h->M * sizeof(double))))) { cudaFree(flag); return rc; }
    cudaMemcpyAsync(rad, h->h_radius.data(), h->M * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(flag, 0, sizeof(int), st);
    long long npair = (long long)R * h->M;
    k_check_receivers<<<(int)((npair + 255) / 256), 256, 0, st>>>((const double2*)rx, h->d.centre, rad, R, h->M, flag);
    int hflag = 0;
    cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    rc = ms_check(h, cudaStreamSynchronize(st));
    cudaFree(flag);
    cudaFree(rad);
    if (rc) return rc;
    if (hflag) return MS_ERR_RECEIVER_INSIDE;
    // reflected amplitudes D = R U(gamma)
    if ((rc = ms_to_scaled(h, gamma, h->ws_x, nrhs, MS_PREC_FP64, st))) return rc;
    if ((rc = ms_local_scaled<double>(h, h->ws_x, nrhs, MS_PART_R, st))) return rc;   // leaves D in ws_u
    const int K = h->p + 1, nh = 2 * K + 1;
    size_t smem = (size_t)FLD_NB * 2 * nh * sizeof(double2) + (size_t)FLD_NB * 2 * 2 * (K + 1) * sizeof(double);
    cudaFuncSetAttribute(k_fields_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fields_direct<<<R, 256, smem, st>>>((const double2*)gamma, (const double2*)rx, h->d.centre, (double2*)u, h->M,
                                          h->p, nrhs, R, h->kp_l, h->ks_l);
    if ((rc = ms_check(h, cudaGetLastError()))) return rc;
    k_fields_refl<<<(R * nrhs + 127) / 128, 128, 0, st>>>((const double2*)h->ws_u, (const double2*)rx, h->d.node,
                                                          h->d.wq, h->d.sq, (double2*)u, h->NS, nrhs, R);
    return ms_check(h, cudaGetLastError());
}

// ====================================================================== allocation-free fields
// ms_fields_noalloc: the receiver-field computation of ms_fields for callers that cannot call
// cudaMalloc (for example real-time loops that must not synchronise with the allocator, or
// processes whose device memory is owned by a pool sized in advance).
// Everything ms_fields allocates per call -- the validation flag, a device copy of the radii, the
// multipole-to-Sommerfeld partial sums and the reflected spectral amplitudes -- lives instead in
// the fixed arrays below, which every GPU that loads this library holds until the process exits.
// The handle's own tables (made by ms_setup) are only read.
namespace {

constexpr long long NAL_PART_MAX = 1LL << 19;   // split-K partials: chunks * 2 * N_S * nrhs complex (8 MiB)
constexpr long long NAL_D_MAX = 1LL << 16;      // reflected amplitudes: 2 * N_S * nrhs complex (1 MiB)
constexpr int NAL_M_MAX = 1 << 17;              // particles (radii copy, 1 MiB)
constexpr int NAL_CHUNK_MAX = 16;               // source chunks of the partial sums

static __device__ __align__(256) double2 g_nal_part[NAL_PART_MAX];
static __device__ __align__(256) double2 g_nal_d[NAL_D_MAX];
static __device__ __align__(256) double g_nal_radius[NAL_M_MAX];
static __device__ __align__(256) int g_nal_flag[64];

struct NalPtrs {
    double2* part = nullptr;
    double2* d = nullptr;
    double* radius = nullptr;
    int* flag = nullptr;
    bool ready = false;
};
constexpr int NAL_MAX_DEVICES = 64;
NalPtrs g_nal_ptrs[NAL_MAX_DEVICES];
std::mutex g_nal_mutex;

// part[chunk][b][q][r] = sum_{l in chunk} e^{s_b y_l - i xi_q x_l} sum_n Q_b(q,n) gamma^l_{b,n,r},
// Q_b(q,n) = (-i)^n q_b^n / (i pi s_b): the multipole-to-Sommerfeld sums (Sec. 5.4, pts1 / sed1 /
// sed2) on the caller's unscaled FP64 coefficients.  One thread per (chunk, b, q, r).
__global__ void k_nal_m2s(const double2* __restrict__ gam, double2* __restrict__ part,
                          const double2* __restrict__ centre, const double2* __restrict__ node,
                          const double2* __restrict__ sq, const double2* __restrict__ qpow, int M, int p, int NS,
                          int nrhs, int nchunks, int chunk_len) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)nchunks * 2 * NS * nrhs;
    if (i >= total) return;
    const int r = (int)(i % nrhs);
    const int q = (int)((i / nrhs) % NS);
    const int b = (int)((i / ((long long)nrhs * NS)) % 2);
    const int c = (int)(i / ((long long)nrhs * NS * 2));
    const int nc = 2 * p + 1;
    const double2 xi = node[q], s = sq[q * 2 + b];
    const double2* Q = qpow + ((size_t)b * NS + q) * nc;
    double2 acc = make_double2(0, 0);
    const int l0 = c * chunk_len, l1 = min(M, l0 + chunk_len);
    for (int l = l0; l < l1; ++l) {
        double2 cl = centre[l];
        double re = s.x * cl.y + xi.y * cl.x;
        double im = s.y * cl.y - xi.x * cl.x;
        double mag = exp(re), sn, cs;
        sincos(im, &sn, &cs);
        const double2* g = gam + ((size_t)(l * 2 + b) * nc) * nrhs + r;
        double2 inner = make_double2(0, 0);
        for (int n = 0; n < nc; ++n) cfma(inner, Q[n], g[(size_t)n * nrhs]);
        cfma(acc, make_double2(mag * cs, mag * sn), inner);
    }
    part[i] = acc;
}

// D(q, r) = R(xi_q) sum_chunks part(q, r)   (2x2 reflection per node, Sec. 3 / 5.2)
__global__ void k_nal_reflect(const double2* __restrict__ part, double2* __restrict__ d,
                              const double2* __restrict__ refl, int nchunks, int NS, int nrhs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NS * nrhs) return;
    int q = i / nrhs, r = i % nrhs;
    double2 up = make_double2(0, 0), us = make_double2(0, 0);
    for (int c = 0; c < nchunks; ++c) {
        up = cadd(up, part[(((size_t)c * 2 + 0) * NS + q) * nrhs + r]);
        us = cadd(us, part[(((size_t)c * 2 + 1) * NS + q) * nrhs + r]);
    }
    const double2* R = refl + (size_t)q * 4;
    d[(size_t)(0 * NS + q) * nrhs + r] = cadd(cmul(R[0], up), cmul(R[1], us));
    d[(size_t)(1 * NS + q) * nrhs + r] = cadd(cmul(R[2], up), cmul(R[3], us));
}

// Device addresses of the fixed arrays, looked up once per device with that device current and kept
// for the rest of the process: the cache assumes the device's primary context lives as long as the
// process (a cudaDeviceReset would leave these addresses stale).
int nal_pointers(ms_handle* h, NalPtrs** out) {
    int dev = 0;
    if (int rc = ms_check(h, cudaGetDevice(&dev))) return rc;
    if (dev < 0 || dev >= NAL_MAX_DEVICES) return MS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_nal_mutex);
    NalPtrs& P = g_nal_ptrs[dev];
    if (!P.ready) {
        int rc;
        if ((rc = ms_check(h, cudaGetSymbolAddress((void**)&P.part, g_nal_part))) ||
            (rc = ms_check(h, cudaGetSymbolAddress((void**)&P.d, g_nal_d))) ||
            (rc = ms_check(h, cudaGetSymbolAddress((void**)&P.radius, g_nal_radius))) ||
            (rc = ms_check(h, cudaGetSymbolAddress((void**)&P.flag, g_nal_flag))))
            return rc;
        P.ready = true;
    }
    *out = &P;
    return MS_OK;
}

}  // namespace

extern "C" int ms_fields_noalloc(ms_handle* h, const void* gamma, int32_t nrhs, const double* rx, int32_t R,
                                 void* u, void* stream) {
    if (!h || !gamma || !rx || !u || nrhs < 1 || R < 1) return MS_ERR_ARG;
    const int M = h->M, NS = h->NS;
    int nchunks = std::min(NAL_CHUNK_MAX, M);
    int chunk_len = (M + nchunks - 1) / nchunks;
    nchunks = (M + chunk_len - 1) / chunk_len;
    if (nrhs > 64 || M > NAL_M_MAX || (long long)nchunks * 2 * NS * nrhs > NAL_PART_MAX ||
        2LL * NS * nrhs > NAL_D_MAX)
        return MS_ERR_TOO_LARGE;
    NalPtrs* P = nullptr;
    int rc = nal_pointers(h, &P);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // receiver validation: flag cleared, radii copied into the fixed array, flag read back
    if ((rc = ms_check(h, cudaMemsetAsync(P->flag, 0, sizeof(int), st)))) return rc;
    if ((rc = ms_check(h, cudaMemcpyAsync(P->radius, h->h_radius.data(), M * sizeof(double),
                                          cudaMemcpyHostToDevice, st))))
        return rc;
    long long npair = (long long)R * M;
    k_check_receivers<<<(int)((npair + 255) / 256), 256, 0, st>>>((const double2*)rx, h->d.centre, P->radius, R, M,
                                                                 P->flag);
    if ((rc = ms_check(h, cudaGetLastError()))) return rc;
    int hflag = 0;
    if ((rc = ms_check(h, cudaMemcpyAsync(&hflag, P->flag, sizeof(int), cudaMemcpyDeviceToHost, st))) ||
        (rc = ms_check(h, cudaStreamSynchronize(st))))
        return rc;
    if (hflag) return MS_ERR_RECEIVER_INSIDE;
    // reflected amplitudes into the fixed arrays (every partial slot is written, no clearing needed)
    long long tot = (long long)nchunks * 2 * NS * nrhs;
    k_nal_m2s<<<(int)((tot + 127) / 128), 128, 0, st>>>((const double2*)gamma, P->part, h->d.centre, h->d.node,
                                                       h->d.sq, h->d.qpow_m2s, M, h->p, NS, nrhs, nchunks,
                                                       chunk_len);
    if ((rc = ms_check(h, cudaGetLastError()))) return rc;
    k_nal_reflect<<<(NS * nrhs + 255) / 256, 256, 0, st>>>(P->part, P->d, h->d.refl, nchunks, NS, nrhs);
    if ((rc = ms_check(h, cudaGetLastError()))) return rc;
    // field sums: the same kernels as ms_fields
    const int K = h->p + 1, nh = 2 * K + 1;
    size_t smem = (size_t)FLD_NB * 2 * nh * sizeof(double2) + (size_t)FLD_NB * 2 * 2 * (K + 1) * sizeof(double);
    cudaFuncSetAttribute(k_fields_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_fields_direct<<<R, 256, smem, st>>>((const double2*)gamma, (const double2*)rx, h->d.centre, (double2*)u, M,
                                          h->p, nrhs, R, h->kp_l, h->ks_l);
    if ((rc = ms_check(h, cudaGetLastError()))) return rc;
    k_fields_refl<<<(R * nrhs + 127) / 128, 128, 0, st>>>(P->d, (const double2*)rx, h->d.node, h->d.wq, h->d.sq,
                                                          (double2*)u, NS, nrhs, R);
    return ms_check(h, cudaGetLastError());
}
