// Scattered displacement at receivers in the lower layer (Sec. 5, total-field representation):
//   u(x) = sum_m sum_n alpha^m_n grad(H_n(kp' r_m) e^{in th_m}) + beta^m_n grad_perp(H_n(ks' r_m) e^{in th_m})
//        + int [D_P grad(e^{i xi x + s'_p y}) + D_S grad_perp(e^{i xi x + s'_s y})] dxi,
// with (D_P, D_S) = R(xi) (U_P, U_S) the interface-reflected amplitudes of the same outgoing
// coefficients.  Derivatives of cylindrical waves use the order shifts of DLMF 10.6:
//   d/dx (H_n e^{in th}) = (k/2)(h_{n-1} - h_{n+1}),  d/dy = (ik/2)(h_{n-1} + h_{n+1}).
// Everything here is FP64.
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

}  // namespace

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

