// Hot-path kernels of one mat-vec y = x - S (T + R) x, in the scaled basis.
//
// Scaled basis: every coefficient of particle m, wave b, order n carries an exact power-of-two
// scale tau = 2^a, a = round(log2((k_b R_m / 2)^|n| / |n|!)).  Outgoing blocks are stored as
// x~ = x / tau, local blocks as a~ = a * tau, so that the translation entries
// tau_i H_{j-i}(k d) e^{i(j-i)theta} tau_j, the spectral factors and the scattering blocks
// tau^-1 S tau^-1 all stay O(1) and fit FP32; in FP64 the scaling is exact.
//
// Kernels (one template per precision T = double or float):
//   k_to_scaled / k_from_scaled  precision staging (row a1)
//   (free-space translation, rows a2/a3, lives in fmm.cu)
//   k_m2s                        multipole-to-Sommerfeld, split over source chunks (row a4, Sec. 5.4)
//   k_reflect                    chunk reduction + 2x2 reflection per node (row a5, Sec. 3 / 5.2)
//   k_s2l                        Sommerfeld-to-local (row a6, Sec. 5.3)
//   k_sapply_disc                scattering-matrix apply and combine for discs (row a7, Sec. 4.2 mul2, 4.1);
//                                prototype particles in sapply.cu
#include <algorithm>

#include "bessel.cuh"
#include "common.cuh"
#include "handle.h"

namespace {

// ------------------------------------------------------------------ precision staging
// outgoing-type blocks: x~ = x 2^-a (sign = +1); local-type blocks: a~ = a 2^a (sign = -1)
template <typename T>
__global__ void k_to_scaled(const double2* __restrict__ x, typename CT<T>::c* __restrict__ xs,
                            const int* __restrict__ expo, long long total, int nrhs, int sign) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    int row = (int)(i / nrhs);
    double s = pow2d(-sign * expo[row]);
    double2 v = x[i];
    xs[i] = to_c<T>(make_double2(v.x * s, v.y * s));
}

// outgoing-type blocks: y = y~ 2^a (sign = +1); local-type blocks: a = a~ 2^-a (sign = -1)
template <typename T>
__global__ void k_from_scaled(const typename CT<T>::c* __restrict__ ys, double2* __restrict__ y,
                              const int* __restrict__ expo, long long total, int nrhs, int sign) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    int row = (int)(i / nrhs);
    double s = pow2d(sign * expo[row]);
    double2 v = to_d(ys[i]);
    y[i] = make_double2(v.x * s, v.y * s);
}

// ------------------------------------------------------------------ spectral factors
// e^{z} for the exponents of the spectral factors, with z = re + i im built in FP64 from the
// node and the particle position.  FP64 path: FP64 exp / sincos.  FP32 path: the phase is reduced
// mod 2 pi in FP64 (|im| reaches ~|xi| |x| ~ 10^3), then expf / sincosf in FP32.
template <typename T> struct SpecExp;
template <> struct SpecExp<double> {
    __device__ static double2 eval(double re, double im) {
        double m = exp(re), sn, cs;
        sincos(im, &sn, &cs);
        return make_double2(m * cs, m * sn);
    }
};
template <> struct SpecExp<float> {
    __device__ static float2 eval(double re, double im) {
        const double twopi = 6.283185307179586476925286766559;
        double red = im - twopi * rint(im * (1.0 / twopi));
        float m = expf((float)re), sn, cs;
        sincosf((float)red, &sn, &cs);
        return make_float2(m * cs, m * sn);
    }
};
// A table factor (double2, or FP32 mantissa + exponent) times 2^scale, in the precision T.
template <typename T> struct QRef;
template <> struct QRef<double> {
    const double2* q;
    __device__ double2 get(long long idx, int scale) const {
        double2 v = q[idx];
        double f = pow2d(scale);
        return make_double2(v.x * f, v.y * f);
    }
};
template <> struct QRef<float> {
    const float2* m;
    const int* e;
    __device__ float2 get(long long idx, int scale) const {
        float2 v = m[idx];
        float f = pow2f(e[idx] + scale);
        return make_float2(v.x * f, v.y * f);
    }
};

// ------------------------------------------------------------------ multipole-to-Sommerfeld
// part[chunk][b][q][r] = sum_{l in chunk} sum_n F(q,l,n) x~^l_{b,n,r},
// F(q,l,n) = e^{s_b y_l - i xi_q x_l} * [(-i)^n q_b^n / (i pi s_b)] * tau_{l,b,n}   (pts1 / sed1 / sed2)
// A generated-operand GEMM: CTA = (tile of M2S_QT nodes, chunk of particles, wave b), thread tile
// M2S_QB nodes x M2S_RB columns; per particle the CTA stages the source block (cp.async when the
// rows are 16-byte aligned) and builds F for its nodes in shared memory.
constexpr int M2S_QT = 32;
constexpr int M2S_QB = 4;
constexpr int M2S_RB = 4;
constexpr int M2S_THREADS = 128;

// ADJ = 1 computes the adjoint of the Sommerfeld-to-local map instead (C^H): factor
// conj(e^{i xi x + s y} [i^n q^n W_q]) tau = e^{-i conj(xi) x + conj(s) y} conj(.) tau, read from the
// S2L table and conjugated.
template <typename T, int ADJ>
__global__ void __launch_bounds__(M2S_THREADS)
k_m2s(const typename CT<T>::c* __restrict__ xs, double2* __restrict__ part,
      const double2* __restrict__ centre, const int* __restrict__ expo, const double2* __restrict__ node,
      const double2* __restrict__ sq, QRef<T> qpow, int M, int p, int NS, int nrhs, int chunk_len) {
    typedef typename CT<T>::c C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = 2 * p + 1;
    C* F = reinterpret_cast<C*>(smem_raw);            // [nc][M2S_QT + 1]
    C* X = F + nc * (M2S_QT + 1);                     // [nc][nrhs]
    C* Eq = X + nc * nrhs;                            // [M2S_QT]
    const int b = blockIdx.z;
    const int q0 = blockIdx.x * M2S_QT;
    const int chunk = blockIdx.y;
    const int l0 = chunk * chunk_len, l1 = min(M, l0 + chunk_len);
    const int n_rb = (nrhs + M2S_RB - 1) / M2S_RB;
    const int tile = threadIdx.x;
    const bool act = tile < (M2S_QT / M2S_QB) * n_rb;
    const int qb = act ? tile / n_rb : 0, rb = act ? tile % n_rb : 0;
    const int qi0 = qb * M2S_QB, r0 = rb * M2S_RB;
    C acc[M2S_QB][M2S_RB];
#pragma unroll
    for (int u = 0; u < M2S_QB; ++u)
#pragma unroll
        for (int v = 0; v < M2S_RB; ++v) acc[u][v] = mk((T)0, (T)0);

    for (int l = l0; l < l1; ++l) {
        __syncthreads();
        const C* xl = xs + ((size_t)(l * 2 + b) * nc) * nrhs;
        for (int e = threadIdx.x; e < nc * nrhs; e += blockDim.x) X[e] = xl[e];
        const double2 cl = centre[l];
        for (int qi = threadIdx.x; qi < M2S_QT; qi += blockDim.x) {
            int q = q0 + qi;
            C ev = mk((T)0, (T)0);
            if (q < NS) {
                double2 xi = node[q], s = sq[q * 2 + b];
                ev = ADJ ? SpecExp<T>::eval(s.x * cl.y - xi.y * cl.x, -s.y * cl.y - xi.x * cl.x)
                         : SpecExp<T>::eval(s.x * cl.y + xi.y * cl.x, s.y * cl.y - xi.x * cl.x);
            }
            Eq[qi] = ev;
        }
        __syncthreads();
        const int* al = expo + (l * 2 + b) * nc;
        for (int e = threadIdx.x; e < nc * M2S_QT; e += blockDim.x) {
            int n = e / M2S_QT, qi = e % M2S_QT;
            int q = q0 + qi;
            C f = mk((T)0, (T)0);
            if (q < NS) {
                C qv = qpow.get(((long long)b * NS + q) * nc + n, al[n]);
                f = cmul(Eq[qi], ADJ ? cconj(qv) : qv);
            }
            F[n * (M2S_QT + 1) + qi] = f;
        }
        __syncthreads();
        if (act) {
            const int nr = min(M2S_RB, nrhs - r0);
            for (int n = 0; n < nc; ++n) {
                C xv[M2S_RB], fv[M2S_QB];
#pragma unroll
                for (int v = 0; v < M2S_RB; ++v) xv[v] = v < nr ? X[n * nrhs + r0 + v] : mk((T)0, (T)0);
#pragma unroll
                for (int u = 0; u < M2S_QB; ++u) fv[u] = F[n * (M2S_QT + 1) + qi0 + u];
#pragma unroll
                for (int u = 0; u < M2S_QB; ++u)
#pragma unroll
                    for (int v = 0; v < M2S_RB; ++v) cfma(acc[u][v], fv[u], xv[v]);
            }
        }
    }
    if (act) {
#pragma unroll
        for (int u = 0; u < M2S_QB; ++u) {
            int q = q0 + qi0 + u;
            if (q >= NS) continue;
#pragma unroll
            for (int v = 0; v < M2S_RB; ++v) {
                int r = r0 + v;
                if (r < nrhs) part[(((size_t)chunk * 2 + b) * NS + q) * nrhs + r] = to_d(acc[u][v]);
            }
        }
    }
}

// ------------------------------------------------------------------ reduce chunks + reflect
// U_b(q,r) = sum_chunks part; D(q,r) = R(xi_q) U(q,r).  Output ud[b][q][r] holds D.
// adj = 1: D = R(xi_q)^H U (conjugate transpose, for the adjoint operator).
__global__ void k_reflect(const double2* __restrict__ part, double2* __restrict__ ud,
                          const double2* __restrict__ refl, int nchunks, int NS, int nrhs, int adj) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NS * nrhs) return;
    int q = i / nrhs, r = i % nrhs;
    double2 up = make_double2(0, 0), us = make_double2(0, 0);
    for (int c = 0; c < nchunks; ++c) {
        up = cadd(up, part[(((size_t)c * 2 + 0) * NS + q) * nrhs + r]);
        us = cadd(us, part[(((size_t)c * 2 + 1) * NS + q) * nrhs + r]);
    }
    const double2* R = refl + (size_t)q * 4;
    if (adj) {
        ud[(size_t)(0 * NS + q) * nrhs + r] = cadd(cmul(cconj(R[0]), up), cmul(cconj(R[2]), us));
        ud[(size_t)(1 * NS + q) * nrhs + r] = cadd(cmul(cconj(R[1]), up), cmul(cconj(R[3]), us));
    } else {
        ud[(size_t)(0 * NS + q) * nrhs + r] = cadd(cmul(R[0], up), cmul(R[1], us));
        ud[(size_t)(1 * NS + q) * nrhs + r] = cadd(cmul(R[2], up), cmul(R[3], us));
    }
}

// ------------------------------------------------------------------ Sommerfeld-to-local
// a~^m_{b,n,r} (+)= sum_q G(q,m,n) D_b(q,r),
// G(q,m,n) = e^{i xi_q x_m + s_b y_m} * [i^n q_b^n W_q] * tau_{m,b,n}    (ja / stm / eee1)
// CTA = (target m, wave b); thread tile S2L_NB orders x S2L_RB columns; nodes in chunks of S2L_QC
// with the reflected amplitudes and the generated factor staged in shared memory.
constexpr int S2L_QC = 32;
constexpr int S2L_NB = 3;
constexpr int S2L_RB = 8;
constexpr int S2L_THREADS = 128;

// ADJ = 1 computes the adjoint of the multipole-to-Sommerfeld map instead (B^H): factor
// conj(e^{-i xi x + s y} [(-i)^n q^n / (i pi s)]) tau = e^{i conj(xi) x + conj(s) y} conj(.) tau.
template <typename T, int ADJ>
__global__ void __launch_bounds__(S2L_THREADS)
k_s2l(const double2* __restrict__ ud, typename CT<T>::c* __restrict__ as,
      const double2* __restrict__ centre, const int* __restrict__ expo, const double2* __restrict__ node,
      const double2* __restrict__ sq, QRef<T> qpow, int p, int NS, int nrhs, int accumulate) {
    typedef typename CT<T>::c C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = 2 * p + 1;
    C* G = reinterpret_cast<C*>(smem_raw);          // [S2L_QC][nc + 1]
    C* Ds = G + S2L_QC * (nc + 1);                  // [S2L_QC][nrhs]
    C* Eq = Ds + S2L_QC * nrhs;                     // [S2L_QC]
    const int m = blockIdx.x, b = blockIdx.y;
    const double2 cm = centre[m];
    const int* am = expo + (m * 2 + b) * nc;
    const int n_rb = (nrhs + S2L_RB - 1) / S2L_RB;
    const int n_nb = (nc + S2L_NB - 1) / S2L_NB;
    const int tile = threadIdx.x;
    const bool act = tile < n_nb * n_rb;
    const int nb = act ? tile / n_rb : 0, rb = act ? tile % n_rb : 0;
    const int n0 = nb * S2L_NB, r0 = rb * S2L_RB;
    C acc[S2L_NB][S2L_RB];
#pragma unroll
    for (int u = 0; u < S2L_NB; ++u)
#pragma unroll
        for (int v = 0; v < S2L_RB; ++v) acc[u][v] = mk((T)0, (T)0);

    for (int qb = 0; qb < NS; qb += S2L_QC) {
        const int nq = min(S2L_QC, NS - qb);
        __syncthreads();
        for (int e = threadIdx.x; e < nq * nrhs; e += blockDim.x) {
            int r = e % nrhs, qi = e / nrhs;
            Ds[qi * nrhs + r] = to_c<T>(ud[((size_t)b * NS + qb + qi) * nrhs + r]);
        }
        for (int qi = threadIdx.x; qi < nq; qi += blockDim.x) {
            double2 xi = node[qb + qi], s = sq[(qb + qi) * 2 + b];
            Eq[qi] = ADJ ? SpecExp<T>::eval(xi.y * cm.x + s.x * cm.y, xi.x * cm.x - s.y * cm.y)
                         : SpecExp<T>::eval(-xi.y * cm.x + s.x * cm.y, xi.x * cm.x + s.y * cm.y);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nq * nc; e += blockDim.x) {
            int n = e % nc, qi = e / nc;
            C qv = qpow.get(((long long)b * NS + qb + qi) * nc + n, am[n]);
            G[qi * (nc + 1) + n] = cmul(Eq[qi], ADJ ? cconj(qv) : qv);
        }
        __syncthreads();
        if (act) {
            const int nr = min(S2L_RB, nrhs - r0);
            for (int qi = 0; qi < nq; ++qi) {
                C dv[S2L_RB], gv[S2L_NB];
#pragma unroll
                for (int v = 0; v < S2L_RB; ++v) dv[v] = v < nr ? Ds[qi * nrhs + r0 + v] : mk((T)0, (T)0);
#pragma unroll
                for (int u = 0; u < S2L_NB; ++u) gv[u] = (n0 + u) < nc ? G[qi * (nc + 1) + n0 + u] : mk((T)0, (T)0);
#pragma unroll
                for (int u = 0; u < S2L_NB; ++u)
#pragma unroll
                    for (int v = 0; v < S2L_RB; ++v) cfma(acc[u][v], gv[u], dv[v]);
            }
        }
    }
    if (act) {
        C* out = as + ((size_t)(m * 2 + b) * nc) * nrhs;
#pragma unroll
        for (int u = 0; u < S2L_NB; ++u) {
            int n = n0 + u;
            if (n >= nc) continue;
#pragma unroll
            for (int v = 0; v < S2L_RB; ++v) {
                int r = r0 + v;
                if (r >= nrhs) continue;
                size_t o = (size_t)n * nrhs + r;
                out[o] = accumulate ? cadd(out[o], acc[u][v]) : acc[u][v];
            }
        }
    }
}

// ------------------------------------------------------------------ scattering-matrix apply
// y~ = (identity ? x~ : 0) - S~ a~ for disc particles: 2x2 per mode (Sec. 4.1).  With
// negate = 0 the sign is + (plain S~ a~, used by the operator-parts view).
template <typename T>
__global__ void k_sapply_disc(const typename CT<T>::c* __restrict__ xs, const typename CT<T>::c* __restrict__ as,
                              typename CT<T>::c* __restrict__ ys, const typename CT<T>::c* __restrict__ sd,
                              const int* __restrict__ proto, int M, int nc, int nrhs, int identity,
                              int apply_s, int adj) {
    typedef typename CT<T>::c C;
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long total = (long long)M * nc * nrhs;
    if (i >= total) return;
    int r = (int)(i % nrhs);
    long long mn = i / nrhs;
    int n = (int)(mn % nc), m = (int)(mn / nc);
    if (proto[m] >= 0) return;
    size_t ip = ((size_t)(m * 2 + 0) * nc + n) * nrhs + r;
    size_t is = ((size_t)(m * 2 + 1) * nc + n) * nrhs + r;
    C ap = as[ip], a2 = as[is];
    C yp, y2;
    if (apply_s) {
        const C* S = sd + ((size_t)m * nc + n) * 4;
        if (adj) {   // S~^H per mode
            yp = cadd(cmul(cconj(S[0]), ap), cmul(cconj(S[2]), a2));
            y2 = cadd(cmul(cconj(S[1]), ap), cmul(cconj(S[3]), a2));
        } else {
            yp = cadd(cmul(S[0], ap), cmul(S[1], a2));
            y2 = cadd(cmul(S[2], ap), cmul(S[3], a2));
        }
    } else {
        yp = ap;
        y2 = a2;
    }
    if (identity) {
        ys[ip] = csub(xs[ip], yp);
        ys[is] = csub(xs[is], y2);
    } else {
        ys[ip] = yp;
        ys[is] = y2;
    }
}

template <typename T>
__global__ void k_zero(typename CT<T>::c* a, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) a[i] = mk((T)0, (T)0);
}

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ------------------------------------------------------------------ host launchers

int ms_to_scaled(ms_handle* h, const void* x, void* xs, int nrhs, int prec, cudaStream_t st, bool local) {
    long long total = (long long)h->M * 2 * h->nc * nrhs;
    int sign = local ? -1 : 1;
    if (prec == MS_PREC_FP64)
        k_to_scaled<double><<<nblk(total, 256), 256, 0, st>>>((const double2*)x, (double2*)xs, h->d.expo, total, nrhs,
                                                             sign);
    else
        k_to_scaled<float><<<nblk(total, 256), 256, 0, st>>>((const double2*)x, (float2*)xs, h->d.expo, total, nrhs,
                                                            sign);
    return ms_check(h, cudaGetLastError());
}

int ms_from_scaled(ms_handle* h, const void* ys, void* y, int nrhs, int prec, cudaStream_t st, bool local) {
    long long total = (long long)h->M * 2 * h->nc * nrhs;
    int sign = local ? -1 : 1;
    if (prec == MS_PREC_FP64)
        k_from_scaled<double><<<nblk(total, 256), 256, 0, st>>>((const double2*)ys, (double2*)y, h->d.expo, total, nrhs,
                                                               sign);
    else
        k_from_scaled<float><<<nblk(total, 256), 256, 0, st>>>((const float2*)ys, (double2*)y, h->d.expo, total, nrhs,
                                                              sign);
    return ms_check(h, cudaGetLastError());
}

template <typename T> QRef<T> qref_m2s(ms_handle* h);
template <> QRef<double> qref_m2s<double>(ms_handle* h) { return QRef<double>{h->d.qpow_m2s}; }
template <> QRef<float> qref_m2s<float>(ms_handle* h) { return QRef<float>{h->d.qpm_m, h->d.qpm_e}; }
template <typename T> QRef<T> qref_s2l(ms_handle* h);
template <> QRef<double> qref_s2l<double>(ms_handle* h) { return QRef<double>{h->d.qpow_s2l}; }
template <> QRef<float> qref_s2l<float>(ms_handle* h) { return QRef<float>{h->d.qps_m, h->d.qps_e}; }

static int m2s_chunks(ms_handle* h) {
    int chunks = (h->M + 63) / 64;
    if (chunks > 64) chunks = 64;
    return chunks;
}

// ------------------------------------------------------------------ spectral part, host side
// M2S (or, adj = 1, its Sommerfeld-to-local adjoint C^H) into the chunk partials of the workspace;
// returns the number of chunks.  expo: the scale exponents (zeros for the unscaled FP64 path).
template <typename T>
int ms_m2s_launch(ms_handle* h, const void* xs_, int nrhs, const int* expo, int adj, int* nchunks,
                  cudaStream_t st) {
    typedef typename CT<T>::c C;
    const int M = h->M, p = h->p, nc = h->nc, NS = h->NS;
    int chunks = m2s_chunks(h);
    int chunk_len = (M + chunks - 1) / chunks;
    chunks = (M + chunk_len - 1) / chunk_len;
    *nchunks = chunks;
    dim3 g((NS + M2S_QT - 1) / M2S_QT, chunks, 2);
    size_t smem = ((size_t)nc * (M2S_QT + 1) + (size_t)nc * nrhs + M2S_QT) * sizeof(C);
    int tiles = (M2S_QT / M2S_QB) * ((nrhs + M2S_RB - 1) / M2S_RB);
    int thr = std::max(32, std::min(M2S_THREADS, (tiles + 31) / 32 * 32));
    const C* xs = (const C*)xs_;
    if (!adj) {
        cudaFuncSetAttribute(k_m2s<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_m2s<T, 0><<<g, thr, smem, st>>>(xs, (double2*)h->ws_part, h->d.centre, expo, h->d.node, h->d.sq,
                                          qref_m2s<T>(h), M, p, NS, nrhs, chunk_len);
    } else {
        cudaFuncSetAttribute(k_m2s<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_m2s<T, 1><<<g, thr, smem, st>>>(xs, (double2*)h->ws_part, h->d.centre, expo, h->d.node, h->d.sq,
                                          qref_s2l<T>(h), M, p, NS, nrhs, chunk_len);
    }
    return ms_check(h, cudaGetLastError());
}

int ms_reflect_launch(ms_handle* h, const double2* part, int nchunks, double2* out, int nrhs, int adj,
                      cudaStream_t st, const double2* table) {
    k_reflect<<<nblk((long long)h->NS * nrhs, 256), 256, 0, st>>>(part, out, table ? table : h->d.refl, nchunks, h->NS,
                                                                  nrhs, adj);
    return ms_check(h, cudaGetLastError());
}

// S2L of the amplitudes ud[2][N_S][nrhs] (or, adj = 1, the multipole-to-Sommerfeld adjoint B^H) into
// the particle block out (written, or added when accumulate).
template <typename T>
int ms_s2l_launch(ms_handle* h, const double2* ud, void* out, int nrhs, const int* expo, int adj, int accumulate,
                  cudaStream_t st) {
    typedef typename CT<T>::c C;
    const int M = h->M, p = h->p, nc = h->nc, NS = h->NS;
    size_t smem2 = ((size_t)S2L_QC * (nc + 1) + (size_t)S2L_QC * nrhs + S2L_QC) * sizeof(C);
    int tiles2 = ((nc + S2L_NB - 1) / S2L_NB) * ((nrhs + S2L_RB - 1) / S2L_RB);
    int thr2 = std::max(32, std::min(256, (tiles2 + 31) / 32 * 32));
    if (!adj) {
        cudaFuncSetAttribute(k_s2l<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        k_s2l<T, 0><<<dim3(M, 2), thr2, smem2, st>>>(ud, (C*)out, h->d.centre, expo, h->d.node, h->d.sq,
                                                     qref_s2l<T>(h), p, NS, nrhs, accumulate);
    } else {
        cudaFuncSetAttribute(k_s2l<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
        k_s2l<T, 1><<<dim3(M, 2), thr2, smem2, st>>>(ud, (C*)out, h->d.centre, expo, h->d.node, h->d.sq,
                                                     qref_m2s<T>(h), p, NS, nrhs, accumulate);
    }
    return ms_check(h, cudaGetLastError());
}

// a~ (workspace) = (T~ + R~) xs for the parts selected (scaled basis); zero if none.  With adj = 1
// the adjoints T~^H and R~^H = D B^H R^H C^H D instead.
template <typename T>
int ms_local_scaled(ms_handle* h, const void* xs_, int nrhs, int parts, cudaStream_t st, int adj) {
    typedef typename CT<T>::c C;
    C* as = (C*)h->ws_a;
    const int M = h->M, nc = h->nc;
    long long nall = (long long)M * 2 * nc * nrhs;
    bool have = false;
    if (parts & (MS_PART_T | MS_PART_T_NEAR | MS_PART_T_FAR)) {
        bool near = (parts & (MS_PART_T | MS_PART_T_NEAR)) != 0;
        bool far = (parts & (MS_PART_T | MS_PART_T_FAR)) != 0;
        if (int rc = ms_translate_gen<T>(h, xs_, h->ws_a, nrhs, near, far, adj, 0, false, st)) return rc;
        have = true;
    }
    if (parts & MS_PART_R) {
        int chunks = 0;
        const bool tcore = sizeof(T) == 4 && h->opt.tensor_cores;
        if (tcore) {
            if (int rc = ms_m2s_tc_launch(h, (const float2*)xs_, nrhs, adj, &chunks, st)) return rc;
        } else if (int rc = ms_m2s_launch<T>(h, xs_, nrhs, h->d.expo, adj, &chunks, st)) {
            return rc;
        }
        if (int rc = ms_reflect_launch(h, (const double2*)h->ws_part, chunks, (double2*)h->ws_u, nrhs, adj, st))
            return rc;
        if (tcore && ms_s2l_tc_ok(h)) {
            if (int rc = ms_s2l_tc_launch(h, (const double2*)h->ws_u, (float2*)as, nrhs, adj, have ? 1 : 0, st))
                return rc;
        } else if (int rc = ms_s2l_launch<T>(h, (const double2*)h->ws_u, as, nrhs, h->d.expo, adj, have ? 1 : 0, st)) {
            return rc;
        }
        have = true;
    }
    if (!have) {
        k_zero<T><<<nblk(nall, 256), 256, 0, st>>>(as, nall);
        if (int rc = ms_check(h, cudaGetLastError())) return rc;
    }
    return MS_OK;
}

// ys = [xs -] [S~ or S~^H] in, with `in` the workspace a~ unless given.
template <typename T>
int ms_sapply_scaled(ms_handle* h, const void* xs_, void* ys_, int nrhs, bool identity, bool apply_s,
                     cudaStream_t st, int adj, const void* in) {
    typedef typename CT<T>::c C;
    const C* xs = (const C*)xs_;
    C* ys = (C*)ys_;
    const C* as = (const C*)(in ? in : h->ws_a);
    const int M = h->M, p = h->p, nc = h->nc;
    const C* sd = (const C*)(sizeof(T) == 8 ? (const void*)h->d.sdisc : (const void*)h->d.sdisc_f);
    long long nd = (long long)M * nc * nrhs;
    k_sapply_disc<T><<<nblk(nd, 256), 256, 0, st>>>(xs, as, ys, sd, h->d.proto, M, nc, nrhs, identity ? 1 : 0,
                                                    apply_s ? 1 : 0, adj);
    if (int rc = ms_check(h, cudaGetLastError())) return rc;
    return ms_sapply_proto_launch<T>(h, xs, as, ys, nrhs, identity, apply_s, adj, st);
}

// ys = [xs -] [S~] (T~ + R~) xs for the parts selected (all in the scaled basis).
template <typename T>
int ms_apply_scaled(ms_handle* h, const void* xs, void* ys, int nrhs, int parts, bool identity, cudaStream_t st) {
    int rc = ms_local_scaled<T>(h, xs, nrhs, parts, st, 0);
    if (rc) return rc;
    return ms_sapply_scaled<T>(h, xs, ys, nrhs, identity, (parts & MS_PART_S) != 0, st, 0, nullptr);
}

template <typename T>
__global__ void k_csub(const typename CT<T>::c* a, const typename CT<T>::c* b, typename CT<T>::c* y, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) y[i] = csub(a[i], b[i]);
}

// Adjoint operator in the scaled basis: ys = y - (T~^H + R~^H) S~^H y, y = xs.  Uses ws_x as scratch,
// so xs and ys must not be ws_x.
template <typename T>
int ms_apply_adjoint_scaled(ms_handle* h, const void* xs, void* ys, int nrhs, cudaStream_t st) {
    typedef typename CT<T>::c C;
    int rc;
    if ((rc = ms_sapply_scaled<T>(h, nullptr, h->ws_x, nrhs, false, true, st, 1, xs))) return rc;
    if ((rc = ms_local_scaled<T>(h, h->ws_x, nrhs, MS_PART_T | MS_PART_R, st, 1))) return rc;
    long long n = (long long)h->M * 2 * h->nc * nrhs;
    k_csub<T><<<nblk(n, 256), 256, 0, st>>>((const C*)xs, (const C*)h->ws_a, (C*)ys, n);
    return ms_check(h, cudaGetLastError());
}

template int ms_local_scaled<double>(ms_handle*, const void*, int, int, cudaStream_t, int);
template int ms_local_scaled<float>(ms_handle*, const void*, int, int, cudaStream_t, int);
template int ms_sapply_scaled<double>(ms_handle*, const void*, void*, int, bool, bool, cudaStream_t, int, const void*);
template int ms_sapply_scaled<float>(ms_handle*, const void*, void*, int, bool, bool, cudaStream_t, int, const void*);
template int ms_apply_scaled<double>(ms_handle*, const void*, void*, int, int, bool, cudaStream_t);
template int ms_apply_scaled<float>(ms_handle*, const void*, void*, int, int, bool, cudaStream_t);
template int ms_apply_adjoint_scaled<double>(ms_handle*, const void*, void*, int, cudaStream_t);
template int ms_apply_adjoint_scaled<float>(ms_handle*, const void*, void*, int, cudaStream_t);
template int ms_m2s_launch<double>(ms_handle*, const void*, int, const int*, int, int*, cudaStream_t);
template int ms_s2l_launch<double>(ms_handle*, const double2*, void*, int, const int*, int, int, cudaStream_t);

// ------------------------------------------------------------------ captured operator graphs
void ms_graphs_free(ms_handle* h) {
    for (auto& kv : h->graphs) cudaGraphExecDestroy(kv.second);
    h->graphs.clear();
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
}

// Workspace to workspace: ws_y = [ws_x -] [S~] (T~ + R~) ws_x for the parts (adjoint: ws_y = A~^H ws_y in
// place), as a replay of a graph captured on the handle's private stream the first time a key is seen.
template <typename T>
int ms_operator_ws(ms_handle* h, int nrhs, int parts, bool identity, bool adjoint, cudaStream_t st) {
    auto direct = [&](cudaStream_t s) -> int {
        if (adjoint) return ms_apply_adjoint_scaled<T>(h, h->ws_y, h->ws_y, nrhs, s);
        return ms_apply_scaled<T>(h, h->ws_x, h->ws_y, nrhs, parts, identity, s);
    };
    if (!h->opt.cuda_graph) return direct(st);
    const auto key = std::make_tuple(nrhs, (int)sizeof(T), h->tc_kind, parts, (identity ? 1 : 0) + (adjoint ? 2 : 0));
    auto it = h->graphs.find(key);
    if (it == h->graphs.end()) {
        int rc;
        if (!h->cap_stream && (rc = ms_check(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking))))
            return rc;
        if ((rc = ms_check(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal)))) return rc;
        rc = direct(h->cap_stream);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return rc ? rc : ms_check(h, e);
        }
        cudaGraphExec_t ex = nullptr;
        const cudaError_t e2 = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        if ((rc = ms_check(h, e2))) return rc;
        it = h->graphs.emplace(key, ex).first;
    }
    return ms_check(h, cudaGraphLaunch(it->second, st));
}

// out = A~ in (or A~^H in) for scaled blocks at any address: copied through the workspace so that the
// captured graph of the whole operator can run (two block copies against the operator's work).
template <typename T>
int ms_operator_op(ms_handle* h, const void* in, void* out, int nrhs, bool adjoint, cudaStream_t st) {
    typedef typename CT<T>::c C;
    const int parts = MS_PART_T | MS_PART_R | MS_PART_S;
    if (!h->opt.cuda_graph) {
        if (adjoint) return ms_apply_adjoint_scaled<T>(h, in, out, nrhs, st);
        return ms_apply_scaled<T>(h, in, out, nrhs, parts, true, st);
    }
    const size_t bytes = (size_t)h->M * 2 * h->nc * nrhs * sizeof(C);
    void* wi = adjoint ? h->ws_y : h->ws_x;
    int rc;
    if (in != wi && (rc = ms_check(h, cudaMemcpyAsync(wi, in, bytes, cudaMemcpyDeviceToDevice, st)))) return rc;
    if ((rc = ms_operator_ws<T>(h, nrhs, parts, true, adjoint, st))) return rc;
    if (out != h->ws_y) return ms_check(h, cudaMemcpyAsync(out, h->ws_y, bytes, cudaMemcpyDeviceToDevice, st));
    return MS_OK;
}

template int ms_operator_ws<double>(ms_handle*, int, int, bool, bool, cudaStream_t);
template int ms_operator_ws<float>(ms_handle*, int, int, bool, bool, cudaStream_t);
template int ms_operator_op<double>(ms_handle*, const void*, void*, int, bool, cudaStream_t);
template int ms_operator_op<float>(ms_handle*, const void*, void*, int, bool, cudaStream_t);
