// Adjoint gradient of a real receiver loss with respect to particle centres, radii and the
// frequency (ms_grad).
//
// With u = F gamma the scattered field at the receivers (Sec. 5), A gamma = b (mul2 with the layered
// Schur complement, Sec. 4.2 / 5.2; b = S a0, Sec. 7.3) and w = dL/d conj(u) (so dL = Re w^H du):
//     dL/dtheta = Re[w^H (dF) gamma] + Re[lambda^H (db - (dA) gamma)],   A^H lambda = F^H w,
// and with mu = S^H lambda, -Re[lambda^H (dA) gamma] = Re[mu^H d(T + R) gamma] (S does not depend on
// the centres).  The centre derivatives of every factor are local:
//   * Graf entries h_k(v) = Z_k(k|v|) e^{ik arg v}, v = x_dst - x_src: d/dv_x h_k = (k/2)(h_{k-1} - h_{k+1}),
//     d/dv_y h_k = (ik/2)(h_{k-1} + h_{k+1}) (DLMF 10.6).  The target-side term is the forward translation
//     in derivative mode (near pairs and the L2P stage of the FMM), dotted with mu; the source-side term
//     is the adjoint translation in derivative mode applied to mu, dotted with gamma;
//   * spectral factors: target e^{i xi x + s y} -> (i xi, s), source e^{-i xi x + s y} -> (-i xi, s);
//   * right-hand side a0 ~ e^{i xi_inc x + s y}: (i xi_inc, s);
//   * receiver field of a particle: minus its receiver gradient (second-order shifts).
// Radii: Re[lambda^{m H} (dS_m/dR) (a0 + (T + R) gamma)^m] with the closed-form disc derivative.
// Frequency: central differences of A gamma, b and F gamma on handles built at omega +- h.
// All arithmetic here is FP64 in the unscaled basis.
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "bessel.cuh"
#include "common.cuh"
#include "handle.h"

typedef std::complex<double> cd;
bool ms_plane_wave_transmission(const ms_handle* h, int kind, double angle, double* xi_out, cd D[2]);

namespace {

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// block-wide sum of a double (blockDim.x <= 1024, multiple of 32)
__device__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;   // valid on thread 0
}

// g[m * gstride + goff] += Re sum_{b,n,r} conj(a) b over particle m's block.
__global__ void k_dot_particles(const double2* __restrict__ a, const double2* __restrict__ b, double* __restrict__ g,
                                int per, int gstride, int goff) {
    __shared__ double sh[32];
    const int m = blockIdx.x;
    const double2* pa = a + (size_t)m * per;
    const double2* pb = b + (size_t)m * per;
    double v = 0;
    for (int i = threadIdx.x; i < per; i += blockDim.x) v += pa[i].x * pb[i].x + pa[i].y * pb[i].y;
    double s = block_sum(v, sh);
    if (threadIdx.x == 0) g[(size_t)m * gstride + goff] += s;
}

// Re sum conj(a) b over n elements, one partial per block (summed on the host).
__global__ void k_dot_all(const double2* __restrict__ a, const double2* __restrict__ b, double* __restrict__ part,
                          long long n) {
    __shared__ double sh[32];
    double v = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v += a[i].x * b[i].x + a[i].y * b[i].y;
    double s = block_sum(v, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// out[b][q][r] = f_b(q) v[b][q][r]; mode 0: i xi, 1: s_b, 2: i conj(xi), 3: conj(s_b)
__global__ void k_scale_nodes(const double2* __restrict__ v, double2* __restrict__ out, const double2* __restrict__ node,
                              const double2* __restrict__ sq, int mode, int NS, int nrhs) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= 2LL * NS * nrhs) return;
    int q = (int)((i / nrhs) % NS), b = (int)(i / ((long long)nrhs * NS));
    double2 xi = node[q], s = sq[q * 2 + b], f;
    if (mode == 0) f = make_double2(-xi.y, xi.x);
    else if (mode == 1) f = s;
    else if (mode == 2) f = make_double2(xi.y, xi.x);      // i conj(xi)
    else f = cconj(s);
    out[i] = cmul(f, v[i]);
}

__global__ void k_cadd(double2* __restrict__ y, const double2* __restrict__ x, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = cadd(y[i], x[i]);
}

constexpr int GNB = 16;   // receivers per batch

// out^m_{b,n,r} = sum_k conj(psi_{b,n}(x_k - x_m)) . w_{r,k}: the adjoint of the direct receiver map,
// psi_P = grad(H_n(kp r) e^{in th}), psi_S = grad_perp(H_n(ks r) e^{in th}).  CTA per particle.
__global__ void __launch_bounds__(256)
k_fieldsT_direct(const double2* __restrict__ w, const double2* __restrict__ rx, const double2* __restrict__ centre,
                 double2* __restrict__ out, int p, int nrhs, int R, double kp, double ks) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = p + 1, nh = 2 * K + 1, nc = 2 * p + 1;
    double2* hs = reinterpret_cast<double2*>(smem_raw);                  // [GNB][2][nh]
    double* scratch = reinterpret_cast<double*>(hs + GNB * 2 * nh);       // [GNB*2][2][K+1]
    double2* acc = reinterpret_cast<double2*>(scratch + GNB * 2 * 2 * (K + 1));   // [2][nc][nrhs]
    const int m = blockIdx.x;
    const double2 cm = centre[m];
    const int nout = 2 * nc * nrhs;
    for (int t = threadIdx.x; t < nout; t += blockDim.x) acc[t] = make_double2(0, 0);
    for (int base = 0; base < R; base += GNB) {
        const int nbk = min(GNB, R - base);
        __syncthreads();
        if (threadIdx.x < 2 * nbk) {
            int s = threadIdx.x >> 1, b = threadIdx.x & 1;
            double2 x = rx[base + s];
            double dx = x.x - cm.x, dy = x.y - cm.y, d = sqrt(dx * dx + dy * dy);
            double* J = scratch + (size_t)threadIdx.x * 2 * (K + 1);
            hankel_phase_seq(K, (b ? ks : kp) * d, dx / d, dy / d, hs + (s * 2 + b) * nh, J, J + (K + 1));
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nout; t += blockDim.x) {
            const int r = t % nrhs, bn = t / nrhs, b = bn / nc, n = bn % nc - p;
            const double k = b ? ks : kp;
            double2 sum = acc[t];
            for (int s = 0; s < nbk; ++s) {
                const double2* hh = hs + (s * 2 + b) * nh;
                double2 hm = hh[n - 1 + K], hp = hh[n + 1 + K];
                double2 dxv = cscale(csub(hm, hp), 0.5 * k);
                double2 dyv = cmul(make_double2(0.0, 0.5 * k), cadd(hm, hp));
                double2 v1 = b ? make_double2(-dyv.x, -dyv.y) : dxv;      // psi components
                double2 v2 = b ? dxv : dyv;
                const double2* wk = w + ((size_t)r * R + base + s) * 2;
                cfma_conj(sum, v1, wk[0]);
                cfma_conj(sum, v2, wk[1]);
            }
            acc[t] = sum;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nout; t += blockDim.x) out[(size_t)m * nout + t] = acc[t];
}

// V[b][q][r] = sum_k conj(W_q vec_b(q, x_k)) . w_{r,k}: the adjoint of the reflected receiver map,
// vec_P = (i xi, s_p) e^{i xi X + s_p Y}, vec_S = (-s_s, i xi) e^{i xi X + s_s Y}.
__global__ void k_fieldsT_refl(const double2* __restrict__ w, const double2* __restrict__ rx,
                               const double2* __restrict__ node, const double2* __restrict__ wq,
                               const double2* __restrict__ sq, double2* __restrict__ V, int NS, int nrhs, int R) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= 2LL * NS * nrhs) return;
    const int r = (int)(i % nrhs), q = (int)((i / nrhs) % NS), b = (int)(i / ((long long)nrhs * NS));
    const double2 xi = node[q], wt = wq[q], s = sq[q * 2 + b];
    const double2 ixi = make_double2(-xi.y, xi.x);
    double2 acc = make_double2(0, 0);
    for (int k = 0; k < R; ++k) {
        double2 x = rx[k];
        double re = -xi.y * x.x + s.x * x.y, im = xi.x * x.x + s.y * x.y;
        double mag = exp(re), sn, cs;
        sincos(im, &sn, &cs);
        double2 e = cmul(make_double2(mag * cs, mag * sn), wt);
        double2 c1 = b ? make_double2(-s.x, -s.y) : ixi;
        double2 c2 = b ? ixi : s;
        const double2* wk = w + ((size_t)r * R + k) * 2;
        cfma_conj(acc, cmul(c1, e), wk[0]);
        cfma_conj(acc, cmul(c2, e), wk[1]);
    }
    V[i] = acc;
}

// g[m*2 + axis] += Re sum_{k,r,c} conj(w) (d/dc_m F_direct gamma): minus the receiver derivative of
// particle m's outgoing field (second derivatives by order shifts, orders up to p + 2).
__global__ void __launch_bounds__(256)
k_grad_fdirect(const double2* __restrict__ gam, const double2* __restrict__ w, const double2* __restrict__ rx,
               const double2* __restrict__ centre, double* __restrict__ g, int p, int nrhs, int R, double kp,
               double ks) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int K = p + 2, nh = 2 * K + 1, nc = 2 * p + 1;
    double2* hs = reinterpret_cast<double2*>(smem_raw);                  // [GNB][2][nh]
    double* scratch = reinterpret_cast<double*>(hs + GNB * 2 * nh);       // [GNB*2][2][K+1]
    __shared__ double sh[32];
    const int m = blockIdx.x;
    const double2 cm = centre[m];
    double gx = 0, gy = 0;
    for (int base = 0; base < R; base += GNB) {
        const int nbk = min(GNB, R - base);
        __syncthreads();
        if (threadIdx.x < 2 * nbk) {
            int s = threadIdx.x >> 1, b = threadIdx.x & 1;
            double2 x = rx[base + s];
            double dx = x.x - cm.x, dy = x.y - cm.y, d = sqrt(dx * dx + dy * dy);
            double* J = scratch + (size_t)threadIdx.x * 2 * (K + 1);
            hankel_phase_seq(K, (b ? ks : kp) * d, dx / d, dy / d, hs + (s * 2 + b) * nh, J, J + (K + 1));
        }
        __syncthreads();
        for (int t = threadIdx.x; t < nbk * nrhs; t += blockDim.x) {
            const int s = t / nrhs, r = t % nrhs;
            double2 dd[2][3];   // [wave][xx, xy, yy] of the potential sum
            for (int b = 0; b < 2; ++b) {
                const double k = b ? ks : kp;
                const double2* hh = hs + (s * 2 + b) * nh;
                const double2* ga = gam + ((size_t)(m * 2 + b) * nc) * nrhs + r;
                double2 xx = make_double2(0, 0), xy = xx, yy = xx;
                for (int i = 0; i < nc; ++i) {
                    int n = i - p;
                    double2 c = ga[(size_t)i * nrhs];
                    double2 m2 = hh[n - 2 + K], z = hh[n + K], p2 = hh[n + 2 + K];
                    double2 vxx = cscale(cadd(csub(m2, cscale(z, 2.0)), p2), 0.25 * k * k);
                    double2 vxy = cmul(make_double2(0.0, 0.25 * k * k), csub(m2, p2));
                    double2 vyy = cscale(cadd(cadd(m2, cscale(z, 2.0)), p2), -0.25 * k * k);
                    cfma(xx, c, vxx);
                    cfma(xy, c, vxy);
                    cfma(yy, c, vyy);
                }
                dd[b][0] = xx; dd[b][1] = xy; dd[b][2] = yy;
            }
            // u1 = phi_x - psi_y, u2 = phi_y + psi_x; d/dc_m = -d/dX
            double2 du1x = csub(dd[0][0], dd[1][1]), du2x = cadd(dd[0][1], dd[1][0]);
            double2 du1y = csub(dd[0][1], dd[1][2]), du2y = cadd(dd[0][2], dd[1][1]);
            const double2* wk = w + ((size_t)r * R + base + s) * 2;
            gx -= wk[0].x * du1x.x + wk[0].y * du1x.y + wk[1].x * du2x.x + wk[1].y * du2x.y;
            gy -= wk[0].x * du1y.x + wk[0].y * du1y.y + wk[1].x * du2y.x + wk[1].y * du2y.y;
        }
    }
    double sx = block_sum(gx, sh);
    if (threadIdx.x == 0) g[(size_t)m * 2 + 0] += sx;
    double sy = block_sum(gy, sh);
    if (threadIdx.x == 0) g[(size_t)m * 2 + 1] += sy;
}

// g[m*2 + axis] += Re sum conj(mu) c a0 with a0^m_{b,n,r} = D_b(r) e^{i xi_r x_m + s y_m} i^n q^n and
// c = i xi_r (axis 0) or s_{b,r} (axis 1).
__global__ void k_grad_rhs(const double2* __restrict__ mu, const double2* __restrict__ centre,
                           const double* __restrict__ xi, const double2* __restrict__ amp, const double2* __restrict__ s,
                           const double2* __restrict__ q, double* __restrict__ g, int p, int nrhs) {
    __shared__ double sh[32];
    const int m = blockIdx.x, nc = 2 * p + 1;
    const double2 c = centre[m];
    double gx = 0, gy = 0;
    for (int t = threadIdx.x; t < 2 * nc * nrhs; t += blockDim.x) {
        int r = t % nrhs, row = t / nrhs, b = row / nc, n = row % nc - p;
        double2 sb = s[r * 2 + b], qb = q[r * 2 + b];
        double re = sb.x * c.y, im = xi[r] * c.x + sb.y * c.y;
        double mag = exp(re), sn, cs;
        sincos(im, &sn, &cs);
        double2 v = cmul(amp[r * 2 + b], make_double2(mag * cs, mag * sn));
        double2 f = make_double2(1.0, 0.0), iq = cmul(make_double2(0.0, 1.0), qb);
        if (n < 0) iq = cdiv(make_double2(1.0, 0.0), iq);
        for (int k = 0; k < (n < 0 ? -n : n); ++k) f = cmul(f, iq);
        v = cmul(v, f);
        double2 mv = mu[((size_t)m * 2 * nc + row) * nrhs + r];
        double2 ax = cmul(make_double2(0.0, xi[r]), v), ay = cmul(sb, v);
        gx += mv.x * ax.x + mv.y * ax.y;
        gy += mv.x * ay.x + mv.y * ay.y;
    }
    double sx = block_sum(gx, sh);
    if (threadIdx.x == 0) g[(size_t)m * 2 + 0] += sx;
    double sy = block_sum(gy, sh);
    if (threadIdx.x == 0) g[(size_t)m * 2 + 1] += sy;
}

// gr[m] = Re sum_{n,r} conj(lambda^m_n) (dS_m/dR)_n atot^m_n for disc particles (0 for prototypes).
__global__ void k_grad_radius(const double2* __restrict__ lam, const double2* __restrict__ atot,
                              const double2* __restrict__ dsdr, const int* __restrict__ proto, double* __restrict__ gr,
                              int nc, int nrhs) {
    __shared__ double sh[32];
    const int m = blockIdx.x;
    double v = 0;
    if (proto[m] < 0) {
        for (int t = threadIdx.x; t < nc * nrhs; t += blockDim.x) {
            int n = t / nrhs, r = t % nrhs;
            const double2* D = dsdr + ((size_t)m * nc + n) * 4;
            size_t ip = ((size_t)(m * 2 + 0) * nc + n) * nrhs + r, is = ((size_t)(m * 2 + 1) * nc + n) * nrhs + r;
            double2 ap = atot[ip], as = atot[is];
            double2 yp = cadd(cmul(D[0], ap), cmul(D[1], as)), ys = cadd(cmul(D[2], ap), cmul(D[3], as));
            double2 lp = lam[ip], ls = lam[is];
            v += lp.x * yp.x + lp.y * yp.y + ls.x * ys.x + ls.y * ys.y;
        }
    }
    double s = block_sum(v, sh);
    if (threadIdx.x == 0) gr[m] = s;
}

}  // namespace

// a0 (unscaled, written or added) for the incidences, and the per-column device data of the
// transmitted plane waves (used by the right-hand-side derivative).
struct IncDev {
    double* xi = nullptr;
    double2 *amp = nullptr, *s = nullptr, *q = nullptr;
    ~IncDev() { cudaFree(xi); cudaFree(amp); cudaFree(s); cudaFree(q); }
};
void ms_incident_launch(ms_handle* h, const double* xi, const double2* amp, const double2* s, const double2* q,
                        double2* out, const int* expo, int nrhs, int accumulate, cudaStream_t st);

static int inc_device(ms_handle* h, const ms_incidence* inc, IncDev& D, cudaStream_t st) {
    const int nrhs = inc->nrhs;
    std::vector<double> xi(nrhs);
    std::vector<double2> amp(nrhs * 2), s(nrhs * 2), q(nrhs * 2);
    for (int r = 0; r < nrhs; ++r) {
        if ((inc->kind[r] != 0 && inc->kind[r] != 1) || !(inc->angle[r] > 0) || !(inc->angle[r] < M_PI))
            return MS_ERR_ARG;
        cd Dm[2];
        if (!ms_plane_wave_transmission(h, inc->kind[r], inc->angle[r], &xi[r], Dm)) return MS_ERR_ARG;
        for (int b = 0; b < 2; ++b) {
            double k = b ? h->ks_l : h->kp_l;
            cd sv = cd(0, -1) * std::sqrt(cd(k * k - xi[r] * xi[r], 0.0));
            cd qv = (cd(xi[r], 0.0) - sv) / k;
            amp[r * 2 + b] = make_double2(Dm[b].real(), Dm[b].imag());
            s[r * 2 + b] = make_double2(sv.real(), sv.imag());
            q[r * 2 + b] = make_double2(qv.real(), qv.imag());
        }
    }
    int rc;
    if ((rc = ms_check(h, cudaMalloc(&D.xi, nrhs * sizeof(double)))) ||
        (rc = ms_check(h, cudaMalloc(&D.amp, nrhs * 2 * sizeof(double2)))) ||
        (rc = ms_check(h, cudaMalloc(&D.s, nrhs * 2 * sizeof(double2)))) ||
        (rc = ms_check(h, cudaMalloc(&D.q, nrhs * 2 * sizeof(double2)))))
        return rc;
    cudaMemcpyAsync(D.xi, xi.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(D.amp, amp.data(), nrhs * 2 * sizeof(double2), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(D.s, s.data(), nrhs * 2 * sizeof(double2), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(D.q, q.data(), nrhs * 2 * sizeof(double2), cudaMemcpyHostToDevice, st);
    return ms_check(h, cudaStreamSynchronize(st));
}

static int dot_all(ms_handle* h, const double2* a, const double2* b, long long n, double* out, cudaStream_t st) {
    const int nb = 296;
    double* part = nullptr;
    int rc = ms_check(h, cudaMalloc(&part, nb * sizeof(double)));
    if (rc) return rc;
    k_dot_all<<<nb, 256, 0, st>>>(a, b, part, n);
    std::vector<double> hp(nb);
    rc = ms_check(h, cudaMemcpyAsync(hp.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (!rc) rc = ms_check(h, cudaStreamSynchronize(st));
    cudaFree(part);
    double s = 0;
    for (double v : hp) s += v;
    *out = s;
    return rc;
}

extern "C" int ms_grad(ms_handle* h, const ms_incidence* inc, const void* gamma_, const void* w_, const double* rx_,
                       int32_t R, double tol, int32_t prec, double* g_centres, double* g_radii, double* g_omega,
                       ms_solve_info* info, void* stream) {
    if (!h || !inc || !gamma_ || !w_ || !rx_ || R < 1 || !(tol > 0)) return MS_ERR_ARG;
    if ((prec = ms_resolve_prec(h, prec)) < 0) return prec;
    const int nrhs = inc->nrhs;
    if (nrhs < 1) return MS_ERR_ARG;
    if (nrhs > 64) return MS_ERR_UNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ms_ensure_workspace(h, nrhs);
    if (rc) return rc;
    const int M = h->M, p = h->p, nc = h->nc, NS = h->NS;
    const long long N = (long long)M * 2 * nc, tot = N * nrhs, nsp = 2LL * NS * nrhs;
    const double2* gamma = (const double2*)gamma_;
    const double2* w = (const double2*)w_;
    const double2* rx = (const double2*)rx_;
    // receivers must lie below the interface and outside every enclosing disc (as in ms_fields)
    {
        std::vector<double2> hrx(R);
        if ((rc = ms_check(h, cudaMemcpyAsync(hrx.data(), rx, R * sizeof(double2), cudaMemcpyDeviceToHost, st))) ||
            (rc = ms_check(h, cudaStreamSynchronize(st))))
            return rc;
        for (int j = 0; j < R; ++j) {
            if (!(hrx[j].y < 0)) return MS_ERR_RECEIVER_INSIDE;
            for (int m = 0; m < M; ++m) {
                double dx = hrx[j].x - h->h_centres[2 * m], dy = hrx[j].y - h->h_centres[2 * m + 1];
                double lim = 1.1 * h->h_radius[m];
                if (dx * dx + dy * dy < lim * lim) return MS_ERR_RECEIVER_INSIDE;
            }
        }
    }
    std::vector<void*> bufs;
    auto alloc = [&](size_t bytes) -> void* {
        void* p2 = nullptr;
        if (cudaMalloc(&p2, bytes) != cudaSuccess) return nullptr;
        bufs.push_back(p2);
        return p2;
    };
    auto cleanup = [&]() {
        for (void* b : bufs) cudaFree(b);
    };
    double2* gv = (double2*)alloc(tot * sizeof(double2));
    double2* lam = (double2*)alloc(tot * sizeof(double2));
    double2* mu = (double2*)alloc(tot * sizeof(double2));
    double2* out = (double2*)alloc(tot * sizeof(double2));
    double2* VF = (double2*)alloc(nsp * sizeof(double2));
    double2* V1 = (double2*)alloc(nsp * sizeof(double2));
    double2* Dfw = (double2*)alloc(nsp * sizeof(double2));
    double2* Vt = (double2*)alloc(nsp * sizeof(double2));
    double2* tmp = (double2*)alloc(nsp * sizeof(double2));
    double* gc = (double*)alloc((size_t)M * 2 * sizeof(double));
    if (!gv || !lam || !mu || !out || !VF || !V1 || !Dfw || !Vt || !tmp || !gc) { cleanup(); return MS_ERR_ALLOC; }
    IncDev inc_d;
    if ((rc = inc_device(h, inc, inc_d, st))) { cleanup(); return rc; }
    const int* z = h->d.zexp;
#define CK(x) do { if ((rc = (x))) { cleanup(); return rc; } } while (0)
#define CKL() CK(ms_check(h, cudaGetLastError()))
    // ---- 1. g = F^H w
    {
        const int K = p + 1, nh = 2 * K + 1;
        size_t smem = (size_t)GNB * 2 * nh * sizeof(double2) + (size_t)GNB * 2 * 2 * (K + 1) * sizeof(double) +
                      (size_t)2 * nc * nrhs * sizeof(double2);
        cudaFuncSetAttribute(k_fieldsT_direct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_fieldsT_direct<<<M, 256, smem, st>>>(w, rx, h->d.centre, gv, p, nrhs, R, h->kp_l, h->ks_l);
        CKL();
        k_fieldsT_refl<<<nblk(nsp, 128), 128, 0, st>>>(w, rx, h->d.node, h->d.wq, h->d.sq, VF, NS, nrhs, R);
        CKL();
        CK(ms_reflect_launch(h, VF, 1, V1, nrhs, 1, st));                       // V1 = R^H E^H w
        CK(ms_s2l_launch<double>(h, V1, gv, nrhs, z, 1, 1, st));                 // g += B^H V1
    }
    // ---- 2. adjoint solve A^H lambda = g
    ms_solve_info sinfo{};
    rc = ms_refine_solve(h, gv, lam, nrhs, tol, prec, true, &sinfo, st);
    if (info) *info = sinfo;
    if (rc < 0) { cleanup(); return rc; }
    const int solve_status = rc;
    // ---- 3. mu = S^H lambda (through the scaled tables: mu = D S~^H (D lambda))
    CK(ms_to_scaled(h, lam, h->ws_y, nrhs, MS_PREC_FP64, st, true));
    CK(ms_sapply_scaled<double>(h, nullptr, h->ws_x, nrhs, false, true, st, 1, h->ws_y));
    CK(ms_from_scaled(h, h->ws_x, mu, nrhs, MS_PREC_FP64, st));
    // ---- 4. forward spectral amplitudes D = R B gamma and adjoint ones Vt = R^H (C^H mu + E^H w)
    int chunks = 0;
    CK(ms_m2s_launch<double>(h, gamma, nrhs, z, 0, &chunks, st));
    CK(ms_reflect_launch(h, (const double2*)h->ws_part, chunks, Dfw, nrhs, 0, st));
    CK(ms_m2s_launch<double>(h, mu, nrhs, z, 1, &chunks, st));
    CK(ms_reflect_launch(h, (const double2*)h->ws_part, chunks, Vt, nrhs, 1, st));
    k_cadd<<<nblk(nsp, 256), 256, 0, st>>>(Vt, V1, nsp);
    CKL();
    // ---- 5. centre gradient
    if (g_centres) {
        CK(ms_check(h, cudaMemsetAsync(gc, 0, (size_t)M * 2 * sizeof(double), st)));
        const int per = 2 * nc * nrhs;
        for (int axis = 0; axis < 2; ++axis) {
            // target side of T: (D T) gamma . mu
            CK(ms_translate_gen<double>(h, gamma, out, nrhs, true, true, 0, axis + 1, true, st));
            k_dot_particles<<<M, 256, 0, st>>>(mu, out, gc, per, 2, axis);
            CKL();
            // source side of T: gamma . (D T)^H mu
            CK(ms_translate_gen<double>(h, mu, out, nrhs, true, true, 1, axis + 1, true, st));
            k_dot_particles<<<M, 256, 0, st>>>(out, gamma, gc, per, 2, axis);
            CKL();
            // target side of R: S2L(f D) . mu, f = (i xi, s)
            k_scale_nodes<<<nblk(nsp, 256), 256, 0, st>>>(Dfw, tmp, h->d.node, h->d.sq, axis, NS, nrhs);
            CKL();
            CK(ms_s2l_launch<double>(h, tmp, out, nrhs, z, 0, 0, st));
            k_dot_particles<<<M, 256, 0, st>>>(mu, out, gc, per, 2, axis);
            CKL();
            // source side of R and of the reflected receiver map: gamma . B^H (conj(f') Vt), f' = (-i xi, s)
            k_scale_nodes<<<nblk(nsp, 256), 256, 0, st>>>(Vt, tmp, h->d.node, h->d.sq, axis + 2, NS, nrhs);
            CKL();
            CK(ms_s2l_launch<double>(h, tmp, out, nrhs, z, 1, 0, st));
            k_dot_particles<<<M, 256, 0, st>>>(out, gamma, gc, per, 2, axis);
            CKL();
        }
        // direct receiver map and right-hand side
        {
            const int K = p + 2, nh = 2 * K + 1;
            size_t smem = (size_t)GNB * 2 * nh * sizeof(double2) + (size_t)GNB * 2 * 2 * (K + 1) * sizeof(double);
            cudaFuncSetAttribute(k_grad_fdirect, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_grad_fdirect<<<M, 256, smem, st>>>(gamma, w, rx, h->d.centre, gc, p, nrhs, R, h->kp_l, h->ks_l);
            CKL();
            k_grad_rhs<<<M, 256, 0, st>>>(mu, h->d.centre, inc_d.xi, inc_d.amp, inc_d.s, inc_d.q, gc, p, nrhs);
            CKL();
        }
        CK(ms_check(h, cudaMemcpyAsync(g_centres, gc, (size_t)M * 2 * sizeof(double), cudaMemcpyDeviceToDevice, st)));
    }
    // ---- 6. radius gradient: Re lambda^H (dS/dR) (a0 + (T + R) gamma)
    if (g_radii) {
        CK(ms_translate_gen<double>(h, gamma, out, nrhs, true, true, 0, 0, true, st));
        CK(ms_s2l_launch<double>(h, Dfw, out, nrhs, z, 0, 1, st));
        ms_incident_launch(h, inc_d.xi, inc_d.amp, inc_d.s, inc_d.q, out, z, nrhs, 1, st);
        CKL();
        k_grad_radius<<<M, 256, 0, st>>>(lam, out, h->d.dsdr, h->d.proto, g_radii, nc, nrhs);
        CKL();
    }
    // ---- 7. frequency: central differences of A gamma, b and F gamma on neighbouring handles
    if (g_omega) {
        const double hw = 1e-6 * h->omega;
        double2* Ag[2] = {(double2*)alloc(tot * sizeof(double2)), (double2*)alloc(tot * sizeof(double2))};
        double2* bg[2] = {(double2*)alloc(tot * sizeof(double2)), (double2*)alloc(tot * sizeof(double2))};
        double2* Fg[2] = {(double2*)alloc((size_t)nrhs * R * 2 * sizeof(double2)),
                          (double2*)alloc((size_t)nrhs * R * 2 * sizeof(double2))};
        if (!Ag[0] || !Ag[1] || !bg[0] || !bg[1] || !Fg[0] || !Fg[1]) { cleanup(); return MS_ERR_ALLOC; }
        ms_geometry g2{};
        g2.M = M;
        g2.centres = h->h_centres.data();
        g2.radius = h->h_radius.data();
        g2.bc = h->h_bc.data();
        g2.proto = h->h_proto.empty() ? nullptr : h->h_proto.data();
        g2.rotation = h->h_rot.empty() ? nullptr : h->h_rot.data();
        g2.n_proto = h->n_proto;
        g2.proto_S = h->h_protoS.empty() ? nullptr : h->h_protoS.data();
        ms_options o2 = h->opt;
        o2.check_geometry = 0;
        for (int sgn = 0; sgn < 2; ++sgn) {
            ms_handle* h2 = nullptr;
            double om = h->omega + (sgn == 0 ? hw : -hw);
            CK(ms_setup(&g2, &h->media, om, p, &o2, &h2));
            int r2 = ms_apply(h2, gamma, Ag[sgn], nrhs, MS_PREC_FP64, stream);
            if (!r2) r2 = ms_rhs(h2, inc, bg[sgn], stream);
            if (!r2) r2 = ms_fields(h2, gamma, nrhs, rx_, R, Fg[sgn], stream);
            cudaStreamSynchronize(st);
            ms_destroy(h2);
            CK(r2);
        }
        double t1 = 0, t2 = 0, t3 = 0, t4 = 0, t5 = 0, t6 = 0;
        long long nf = (long long)nrhs * R * 2;
        CK(dot_all(h, w, Fg[0], nf, &t1, st));
        CK(dot_all(h, w, Fg[1], nf, &t2, st));
        CK(dot_all(h, lam, bg[0], tot, &t3, st));
        CK(dot_all(h, lam, bg[1], tot, &t4, st));
        CK(dot_all(h, lam, Ag[0], tot, &t5, st));
        CK(dot_all(h, lam, Ag[1], tot, &t6, st));
        *g_omega = ((t1 - t2) + (t3 - t4) - (t5 - t6)) / (2.0 * hw);
    }
#undef CK
#undef CKL
    cudaStreamSynchronize(st);
    cleanup();
    return solve_status;
}
