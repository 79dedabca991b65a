// GMRES on the multiple-scattering system (Sec. 4.2 mul2: solved by GMRES) and the solve entry
// point (row a8).  All right-hand sides iterate together as one block; each column has its own
// Hessenberg matrix, Givens rotations and convergence flag.  Orthogonalisation is classical
// Gram-Schmidt applied twice (CGS2) with FP64 accumulation of every inner product, whatever the
// vector precision.  The small Hessenberg / Givens work runs on the host in FP64.
//
// Both precisions use iterative refinement (ms_refine_solve), for A and for A^H.
#include <math.h>

#include <chrono>
#include <complex>
#include <vector>

#include "common.cuh"
#include "handle.h"

typedef std::complex<double> cd;

namespace {

constexpr int GRAM_THREADS = 256;
constexpr int GRAM_TILE = 4;

// partial[blk][i][r] = sum over this block's rows of conj(V_i[row,r]) w[row,r], i in [i0, i0+ni)
template <typename T>
__global__ void __launch_bounds__(GRAM_THREADS)
k_gram(const typename CT<T>::c* __restrict__ V, long long vstride, const typename CT<T>::c* __restrict__ w,
       double2* __restrict__ partial, int nvec, long long N, int nrhs) {
    __shared__ double2 red[GRAM_THREADS];
    const int rpp = GRAM_THREADS / nrhs;           // row groups per pass
    const int r = threadIdx.x % nrhs, rg = threadIdx.x / nrhs;
    const bool act = rg < rpp;
    long long rows_per_blk = (N + gridDim.x - 1) / gridDim.x;
    long long row0 = blockIdx.x * rows_per_blk;
    long long row1 = min(N, row0 + rows_per_blk);
    for (int i0 = 0; i0 < nvec; i0 += GRAM_TILE) {
        double2 acc[GRAM_TILE];
#pragma unroll
        for (int t = 0; t < GRAM_TILE; ++t) acc[t] = make_double2(0, 0);
        if (act) {
            for (long long row = row0 + rg; row < row1; row += rpp) {
                double2 wv = to_d(w[row * nrhs + r]);
#pragma unroll
                for (int t = 0; t < GRAM_TILE; ++t)
                    if (i0 + t < nvec) cfma_conj(acc[t], to_d(V[(i0 + t) * vstride + row * nrhs + r]), wv);
            }
        }
#pragma unroll
        for (int t = 0; t < GRAM_TILE; ++t) {
            if (i0 + t >= nvec) break;
            __syncthreads();
            red[threadIdx.x] = act ? acc[t] : make_double2(0, 0);
            __syncthreads();
            if (threadIdx.x < nrhs) {
                double2 s = make_double2(0, 0);
                for (int g = 0; g < rpp; ++g) s = cadd(s, red[g * nrhs + threadIdx.x]);
                partial[((size_t)blockIdx.x * nvec + i0 + t) * nrhs + threadIdx.x] = s;
            }
        }
    }
}

__global__ void k_gram_reduce(const double2* __restrict__ partial, double2* __restrict__ out, int nblk, int nvec,
                              int nrhs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nvec * nrhs) return;
    double2 s = make_double2(0, 0);
    for (int b = 0; b < nblk; ++b) s = cadd(s, partial[(size_t)b * nvec * nrhs + i]);
    out[i] = s;
}

// w[row,r] -= sum_i coef[i][r] V_i[row,r]
template <typename T>
__global__ void k_update(const typename CT<T>::c* __restrict__ V, long long vstride, typename CT<T>::c* __restrict__ w,
                         const double2* __restrict__ coef, int nvec, long long total, int nrhs, double sign) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    int r = (int)(e % nrhs);
    double2 acc = to_d(w[e]);
    for (int i = 0; i < nvec; ++i) {
        double2 c = coef[i * nrhs + r];
        double2 v = to_d(V[i * vstride + e]);
        acc.x -= sign * (c.x * v.x - c.y * v.y);
        acc.y -= sign * (c.x * v.y + c.y * v.x);
    }
    w[e] = to_c<T>(acc);
}

// out[row,r] = w[row,r] * s[r]
template <typename T>
__global__ void k_colscale(const typename CT<T>::c* __restrict__ w, typename CT<T>::c* __restrict__ out,
                           const double* __restrict__ s, long long total, int nrhs) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= total) return;
    double2 v = to_d(w[e]);
    double f = s[e % nrhs];
    out[e] = to_c<T>(make_double2(v.x * f, v.y * f));
}

// y = a - b (FP64)
__global__ void k_sub(const double2* a, const double2* b, double2* y, long long n) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e < n) y[e] = csub(a[e], b[e]);
}

// scaled FP32 copy of an unscaled FP64 vector (r 2^{-sign a}), and back-accumulation
// x += 2^{sign a} d~ (sign = +1 for outgoing-type unknowns, -1 for the local-type adjoint ones)
__global__ void k_scale_down_f(const double2* __restrict__ r, float2* __restrict__ rs, const int* __restrict__ expo,
                               long long n, int nrhs, int sign) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s = pow2d(-sign * expo[e / nrhs]);
    rs[e] = make_float2((float)(r[e].x * s), (float)(r[e].y * s));
}
__global__ void k_add_up_f(double2* __restrict__ x, const float2* __restrict__ ds, const int* __restrict__ expo,
                           long long n, int nrhs, int sign) {
    long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s = pow2d(sign * expo[e / nrhs]);
    x[e].x += (double)ds[e].x * s;
    x[e].y += (double)ds[e].y * s;
}

inline int nb(long long n, int t) { return (int)((n + t - 1) / t); }

// GMRES state for nrhs independent columns advanced together (one Krylov space per column).
template <typename T>
struct Krylov {
    typedef typename CT<T>::c C;
    ms_handle* h;
    cudaStream_t st;
    long long N;        // rows per column
    int nrhs, m;
    C* V = nullptr;     // [(m+1)][N][nrhs]
    C* w = nullptr;     // [N][nrhs]
    double2* part = nullptr;
    double2* coef = nullptr;
    double* dscale = nullptr;
    int gblk;
    int err = MS_OK;

    int init() {
        size_t vec = (size_t)N * nrhs * sizeof(C);
        gblk = 4 * 148;
        if (cudaMalloc(&V, vec * (m + 1)) != cudaSuccess || cudaMalloc(&w, vec) != cudaSuccess ||
            cudaMalloc(&part, (size_t)gblk * (m + 2) * nrhs * sizeof(double2)) != cudaSuccess ||
            cudaMalloc(&coef, (size_t)(m + 2) * nrhs * sizeof(double2)) != cudaSuccess ||
            cudaMalloc(&dscale, nrhs * sizeof(double)) != cudaSuccess)
            return MS_ERR_ALLOC;
        return MS_OK;
    }
    ~Krylov() {
        cudaFree(V); cudaFree(w); cudaFree(part); cudaFree(coef); cudaFree(dscale);
    }
    C* vec(int i) { return V + (size_t)i * N * nrhs; }
    // out[i][r] = <V_i, x>_r for i < nvec (basis base pointer b0)
    int gram(const C* b0, int nvec, const C* x, std::vector<cd>& out) {
        k_gram<T><<<gblk, GRAM_THREADS, 0, st>>>(b0, N * nrhs, x, part, nvec, N, nrhs);
        k_gram_reduce<<<nb(nvec * nrhs, 128), 128, 0, st>>>(part, coef, gblk, nvec, nrhs);
        if (int rc = ms_check(h, cudaGetLastError())) return rc;
        out.resize((size_t)nvec * nrhs);
        if (int rc = ms_check(h, cudaMemcpyAsync(out.data(), coef, out.size() * sizeof(double2),
                                                 cudaMemcpyDeviceToHost, st)))
            return rc;
        return ms_check(h, cudaStreamSynchronize(st));
    }
    int update(const C* b0, int nvec, C* x, const std::vector<cd>& c, double sign) {
        if (int rc = ms_check(h, cudaMemcpyAsync(coef, c.data(), c.size() * sizeof(double2), cudaMemcpyHostToDevice,
                                                 st)))
            return rc;
        long long tot = N * nrhs;
        k_update<T><<<nb(tot, 256), 256, 0, st>>>(b0, N * nrhs, x, coef, nvec, tot, nrhs, sign);
        return ms_check(h, cudaGetLastError());
    }
    int colscale(const C* x, C* out, const std::vector<double>& s) {
        if (int rc = ms_check(h, cudaMemcpyAsync(dscale, s.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st)))
            return rc;
        long long tot = N * nrhs;
        k_colscale<T><<<nb(tot, 256), 256, 0, st>>>(x, out, dscale, tot, nrhs);
        return ms_check(h, cudaGetLastError());
    }
    int norms(const C* x, std::vector<double>& out) {
        std::vector<cd> g;
        if (int rc = gram(x, 1, x, g)) return rc;
        out.resize(nrhs);
        // (a NaN inner product must stay NaN: std::max(0.0, NaN) would return 0)
        for (int r = 0; r < nrhs; ++r) out[r] = std::isnan(g[r].real()) ? g[r].real() : sqrt(std::max(0.0, g[r].real()));
        return MS_OK;
    }
};

// FP32 operator on the tensor cores: read (and clear) their timeout flag after every application, so
// that a pipeline wait that gave up ends the solve with MS_ERR_TIMEOUT at once (one small device-to-
// host copy next to the inner products' own synchronisations).
template <typename T>
int tc_check(ms_handle* h, cudaStream_t st) {
    if (sizeof(T) == 4 && h->opt.tensor_cores) return ms_spectral_tc_status(h, st);
    return MS_OK;
}

// Restarted GMRES: solve A x = b for every column; x holds the initial guess on entry.
// op(in, out) applies A.  Stops a column when its residual estimate drops below tol * ||b||.
template <typename T, typename Op>
int gmres(Krylov<T>& K, Op op, const typename CT<T>::c* b, typename CT<T>::c* x, double tol, int max_iters,
          int& iters_out, int& matvecs, std::vector<double>& relres) {
    typedef typename CT<T>::c C;
    const int nrhs = K.nrhs, m = K.m;
    int rc;
    std::vector<double> bn;
    if ((rc = K.norms(b, bn))) return rc;
    for (int r = 0; r < nrhs; ++r)
        if (!std::isfinite(bn[r])) return MS_ERR_NONFINITE;
    relres.assign(nrhs, 0.0);
    int total = 0;
    std::vector<bool> done(nrhs, false);
    std::vector<cd> H((size_t)(m + 1) * m * nrhs), cs((size_t)m * nrhs), sn((size_t)m * nrhs), g((size_t)(m + 1) * nrhs);
    std::vector<int> kcol(nrhs);
    while (true) {
        // r0 = b - A x  (into V_0, then normalised)
        if ((rc = op(x, K.w)) || (rc = tc_check<T>(K.h, K.st))) return rc;
        ++matvecs;
        long long tot = K.N * nrhs;
        // V_0 = b - w
        {
            std::vector<cd> one(nrhs, cd(1.0, 0.0));
            if ((rc = ms_check(K.h, cudaMemcpyAsync(K.vec(0), b, tot * sizeof(C), cudaMemcpyDeviceToDevice, K.st))))
                return rc;
            if ((rc = K.update(K.w, 1, K.vec(0), one, 1.0))) return rc;
        }
        std::vector<double> beta;
        if ((rc = K.norms(K.vec(0), beta))) return rc;
        bool all = true;
        for (int r = 0; r < nrhs; ++r) {
            if (!std::isfinite(beta[r])) return MS_ERR_NONFINITE;
            relres[r] = bn[r] > 0 ? beta[r] / bn[r] : 0.0;
            done[r] = relres[r] <= tol;
            all = all && done[r];
        }
        if (all || total >= max_iters) break;
        std::vector<double> inv(nrhs);
        for (int r = 0; r < nrhs; ++r) inv[r] = (!done[r] && beta[r] > 0) ? 1.0 / beta[r] : 0.0;
        if ((rc = K.colscale(K.vec(0), K.vec(0), inv))) return rc;
        std::fill(g.begin(), g.end(), cd(0));
        std::fill(H.begin(), H.end(), cd(0));
        for (int r = 0; r < nrhs; ++r) {
            g[(size_t)r * (m + 1)] = done[r] ? 0.0 : beta[r];   // g_0 of column r
            kcol[r] = 0;
        }
        int j = 0;
        for (; j < m && total < max_iters; ++j) {
            if ((rc = op(K.vec(j), K.w)) || (rc = tc_check<T>(K.h, K.st))) return rc;
            ++matvecs;
            std::vector<cd> h1, h2;
            if ((rc = K.gram(K.vec(0), j + 1, K.w, h1))) return rc;
            if ((rc = K.update(K.vec(0), j + 1, K.w, h1, 1.0))) return rc;
            if ((rc = K.gram(K.vec(0), j + 1, K.w, h2))) return rc;
            if ((rc = K.update(K.vec(0), j + 1, K.w, h2, 1.0))) return rc;
            std::vector<double> hn;
            if ((rc = K.norms(K.w, hn))) return rc;
            std::vector<double> invn(nrhs);
            ++total;
            bool alldone = true;
            for (int r = 0; r < nrhs; ++r) {
                if (done[r]) { invn[r] = 0.0; continue; }
                cd* Hc = &H[(size_t)r * (m + 1) * m];
                for (int i = 0; i <= j; ++i) Hc[i * m + j] = h1[(size_t)i * nrhs + r] + h2[(size_t)i * nrhs + r];
                Hc[(j + 1) * m + j] = hn[r];
                for (int i = 0; i < j; ++i) {
                    cd c = cs[(size_t)r * m + i], s = sn[(size_t)r * m + i];
                    cd a = Hc[i * m + j], bq = Hc[(i + 1) * m + j];
                    Hc[i * m + j] = std::conj(c) * a + std::conj(s) * bq;
                    Hc[(i + 1) * m + j] = -s * a + c * bq;
                }
                cd a = Hc[j * m + j];
                double den = std::hypot(std::abs(a), hn[r]);
                cd c = den > 0 ? a / den : cd(1.0), s = den > 0 ? cd(hn[r] / den) : cd(0.0);
                cs[(size_t)r * m + j] = c;
                sn[(size_t)r * m + j] = s;
                Hc[j * m + j] = den;
                Hc[(j + 1) * m + j] = 0.0;
                cd* gc = &g[(size_t)r * (m + 1)];
                gc[j + 1] = -s * gc[j];
                gc[j] = std::conj(c) * gc[j];
                kcol[r] = j + 1;
                double est = std::abs(gc[j + 1]) / bn[r];
                relres[r] = est;
                bool brk = !(hn[r] > 1e-300) || !(den > 0);
                if (est <= tol || brk) done[r] = true;
                invn[r] = done[r] ? 0.0 : 1.0 / hn[r];
                alldone = alldone && done[r];
            }
            if ((rc = K.colscale(K.w, K.vec(j + 1), invn))) return rc;
            if (alldone) { ++j; break; }
        }
        // x += V y per column, y from the triangular system of its first kcol[r] rows
        int kmax = 0;
        for (int r = 0; r < nrhs; ++r) kmax = std::max(kmax, kcol[r]);
        std::vector<cd> y((size_t)std::max(kmax, 1) * nrhs, cd(0));
        for (int r = 0; r < nrhs; ++r) {
            int k = kcol[r];
            cd* Hc = &H[(size_t)r * (m + 1) * m];
            cd* gc = &g[(size_t)r * (m + 1)];
            for (int i = k - 1; i >= 0; --i) {
                cd s = gc[i];
                for (int l = i + 1; l < k; ++l) s -= Hc[i * m + l] * y[(size_t)l * nrhs + r];
                y[(size_t)i * nrhs + r] = Hc[i * m + i] != 0.0 ? s / Hc[i * m + i] : 0.0;
            }
        }
        if (kmax > 0 && (rc = K.update(K.vec(0), kmax, x, y, -1.0))) return rc;
        // loop back: the true residual is formed at the top and re-checked
        for (int r = 0; r < nrhs; ++r) done[r] = false;
    }
    iters_out = total;
    return MS_OK;
}

}  // namespace

// Solve A x = b (adjoint = false) or A^H x = b (adjoint = true) for every column to relative residual
// tol by iterative refinement.  The outer loop keeps x and r = b - op x in FP64 in the ABI basis; each
// step solves the diagonally scaled system (D^-1 A D, or its adjoint D A^H D^-1 for the local-type
// adjoint unknowns) for the correction with restarted GMRES in FP64 (inner tolerance 1e-7) or FP32
// (1e-3); ms_options.inner_tol overrides both.  x is overwritten; it holds the initial guess on entry
// when guess is set (zero otherwise).
int ms_refine_solve(ms_handle* h, const double2* b, double2* x, int nrhs, double tol, int prec, bool adjoint,
                    ms_solve_info* info, cudaStream_t st, bool guess) {
    auto t0 = std::chrono::steady_clock::now();
    int rc = ms_ensure_workspace(h, nrhs);
    if (rc) return rc;
    const long long N = (long long)h->M * 2 * h->nc;
    const long long tot = N * nrhs;
    const bool local = adjoint;                 // adjoint unknowns scale like local coefficients
    const int sgn = local ? -1 : 1;
    if (!guess && (rc = ms_check(h, cudaMemsetAsync(x, 0, tot * sizeof(double2), st)))) return rc;
    int iters = 0, matvecs = 0, refinements = 0;
    std::vector<double> relres;
    auto op64 = [&](const double2* in, double2* out) -> int {
        int r2;
        if (!adjoint) {
            if ((r2 = ms_to_scaled(h, in, h->ws_x, nrhs, MS_PREC_FP64, st))) return r2;
            if ((r2 = ms_operator_ws<double>(h, nrhs, MS_PART_T | MS_PART_R | MS_PART_S, true, false, st))) return r2;
            return ms_from_scaled(h, h->ws_y, out, nrhs, MS_PREC_FP64, st);
        }
        if ((r2 = ms_to_scaled(h, in, h->ws_y, nrhs, MS_PREC_FP64, st, true))) return r2;
        if ((r2 = ms_operator_ws<double>(h, nrhs, MS_PART_T | MS_PART_R | MS_PART_S, true, true, st))) return r2;
        return ms_from_scaled(h, h->ws_y, out, nrhs, MS_PREC_FP64, st, true);
    };
    auto op32 = [&](const float2* in, float2* out) -> int { return ms_operator_op<float>(h, in, out, nrhs, adjoint, st); };
    auto op64s = [&](const double2* in, double2* out) -> int {
        return ms_operator_op<double>(h, in, out, nrhs, adjoint, st);
    };
    Krylov<double> K64{h, st, N, nrhs, 1};
    double2* r = nullptr;
    void *rs = nullptr, *ds = nullptr;
    const size_t esz = prec == MS_PREC_FP64 ? sizeof(double2) : sizeof(float2);
    if ((rc = K64.init()) || (rc = ms_check(h, cudaMalloc(&r, tot * sizeof(double2)))) ||
        (rc = ms_check(h, cudaMalloc(&rs, tot * esz))) || (rc = ms_check(h, cudaMalloc(&ds, tot * esz)))) {
        cudaFree(r); cudaFree(rs); cudaFree(ds);
        return rc ? rc : MS_ERR_ALLOC;
    }
    Krylov<double>* K64i = nullptr;
    Krylov<float>* K32 = nullptr;
    void* bk = nullptr;                      // block Krylov state (allocated by the first inner solve)
    const bool block = h->opt.block_krylov != 0;
    if (!rc && !block) {
        if (prec == MS_PREC_FP64) {
            K64i = new Krylov<double>{h, st, N, nrhs, h->opt.restart};
            rc = K64i->init();
        } else {
            K32 = new Krylov<float>{h, st, N, nrhs, h->opt.restart};
            rc = K32->init();
        }
    }
    std::vector<double> bn, rn;
    if (!rc) rc = K64.norms(b, bn);
    // inner solves: FP64 to 1e-7; FP32 to 1e-3, since the FP32 operator (3xTF32 products on the tensor
    // cores) bounds what one correction can gain, and tighter inner targets stall (measured: 200
    // particles, 64 columns to 1e-8 in 4307 iterations at 1e-3, 4724 at 1e-4, > 8000 at 1e-5)
    const double inner_tol = h->opt.inner_tol > 0 ? h->opt.inner_tol : (prec == MS_PREC_FP64 ? 1e-7 : 1e-3);
    const int max_ref = 40;
    int left = h->opt.max_iters;
    while (!rc) {
        if ((rc = op64(x, K64.w))) break;
        ++matvecs;
        k_sub<<<nb(tot, 256), 256, 0, st>>>(b, K64.w, r, tot);
        if ((rc = K64.norms(r, rn))) break;
        bool all = true;
        relres.assign(nrhs, 0.0);
        for (int c = 0; c < nrhs; ++c) {
            if (!std::isfinite(rn[c]) || !std::isfinite(bn[c])) { rc = MS_ERR_NONFINITE; break; }
            relres[c] = bn[c] > 0 ? rn[c] / bn[c] : 0.0;
            all = all && relres[c] <= tol;
        }
        if (rc || all || refinements >= max_ref || left <= 0) break;
        int it = 0;
        std::vector<double> inner_res;
        if (prec == MS_PREC_FP64) {
            if ((rc = ms_to_scaled(h, r, rs, nrhs, MS_PREC_FP64, st, local))) break;
            if ((rc = ms_check(h, cudaMemsetAsync(ds, 0, tot * esz, st)))) break;
            rc = block ? ms_block_inner<double>(h, nrhs, N, rs, ds, inner_tol, left, adjoint, it, matvecs, inner_res,
                                                st, &bk)
                       : gmres<double>(*K64i, op64s, (const double2*)rs, (double2*)ds, inner_tol, left, it, matvecs,
                                       inner_res);
            if (rc) break;
            if ((rc = ms_from_scaled(h, ds, K64.w, nrhs, MS_PREC_FP64, st, local))) break;
            std::vector<cd> one(nrhs, cd(1.0, 0.0));
            if ((rc = K64.update(K64.w, 1, x, one, -1.0))) break;       // x += D d~ (or D^-1 d~)
        } else {
            k_scale_down_f<<<nb(tot, 256), 256, 0, st>>>(r, (float2*)rs, h->d.expo, tot, nrhs, sgn);
            if ((rc = ms_check(h, cudaMemsetAsync(ds, 0, tot * esz, st)))) break;
            rc = block ? ms_block_inner<float>(h, nrhs, N, rs, ds, inner_tol, left, adjoint, it, matvecs, inner_res, st,
                                               &bk)
                       : gmres<float>(*K32, op32, (const float2*)rs, (float2*)ds, inner_tol, left, it, matvecs,
                                      inner_res);
            if (rc) break;
            if (h->opt.tensor_cores && (rc = ms_spectral_tc_status(h, st))) break;
            k_add_up_f<<<nb(tot, 256), 256, 0, st>>>(x, (const float2*)ds, h->d.expo, tot, nrhs, sgn);
        }
        iters += it;
        left -= it;
        ++refinements;
    }
    delete K64i;
    delete K32;
    if (bk) {
        if (prec == MS_PREC_FP64)
            ms_block_free<double>(bk);
        else
            ms_block_free<float>(bk);
    }
    cudaFree(r); cudaFree(rs); cudaFree(ds);
    cudaStreamSynchronize(st);
    double worst = 0;
    for (double v : relres) worst = std::max(worst, v);
    if (info) {
        info->iterations = iters;
        info->refinements = refinements;
        info->matvecs = matvecs;
        info->max_rel_residual = worst;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (rc) return rc;
    return worst <= tol ? MS_OK : MS_NOT_CONVERGED;
}

extern "C" int ms_solve(ms_handle* h, const ms_incidence* inc, double tol, int32_t prec, void* gamma,
                        ms_solve_info* info, void* stream) {
    if (!h || !inc || !gamma || !(tol > 0)) return MS_ERR_ARG;
    if ((prec = ms_resolve_prec(h, prec)) < 0) return prec;
    const int nrhs = inc->nrhs;
    if (nrhs < 1) return MS_ERR_ARG;
    if (nrhs > 64) return MS_ERR_UNSUPPORTED;
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t st = (cudaStream_t)stream;
    int rc = ms_ensure_workspace(h, nrhs);
    if (rc) return rc;
    const long long tot = (long long)h->M * 2 * h->nc * nrhs;
    double2* b = nullptr;
    if ((rc = ms_check(h, cudaMalloc(&b, tot * sizeof(double2))))) return rc;
    if ((rc = ms_rhs(h, inc, b, stream))) { cudaFree(b); return rc; }
    rc = ms_refine_solve(h, b, (double2*)gamma, nrhs, tol, prec, false, info, st);
    cudaFree(b);
    if (info) info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}

extern "C" int ms_solve_rhs(ms_handle* h, const void* b, int32_t nrhs, double tol, int32_t prec, void* gamma,
                            int32_t guess, ms_solve_info* info, void* stream) {
    if (!h || !b || !gamma || !(tol > 0) || nrhs < 1) return MS_ERR_ARG;
    if ((prec = ms_resolve_prec(h, prec)) < 0) return prec;
    if (nrhs > 64) return MS_ERR_UNSUPPORTED;
    return ms_refine_solve(h, (const double2*)b, (double2*)gamma, nrhs, tol, prec, false, info, (cudaStream_t)stream,
                           guess != 0);
}

// y = A^H x in the ABI basis (the transposed system of the gradient), through the adjoint kernels.
extern "C" int ms_apply_adjoint(ms_handle* h, const void* x, void* y, int32_t nrhs, int32_t prec, void* stream) {
    if (!h || !x || !y || nrhs < 1) return MS_ERR_ARG;
    if ((prec = ms_resolve_prec(h, prec)) < 0) return prec;
    if (nrhs > 64) return MS_ERR_UNSUPPORTED;
    int rc = ms_ensure_workspace(h, nrhs);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = ms_to_scaled(h, x, h->ws_y, nrhs, prec, st, true))) return rc;
    if (prec == MS_PREC_FP64)
        rc = ms_operator_ws<double>(h, nrhs, MS_PART_T | MS_PART_R | MS_PART_S, true, true, st);
    else
        rc = ms_operator_ws<float>(h, nrhs, MS_PART_T | MS_PART_R | MS_PART_S, true, true, st);
    if (rc) return rc;
    if ((rc = ms_from_scaled(h, h->ws_y, y, nrhs, prec, st, true))) return rc;
    if (prec == MS_PREC_FP32 && h->opt.tensor_cores) return ms_spectral_tc_status(h, st);
    return MS_OK;
}
