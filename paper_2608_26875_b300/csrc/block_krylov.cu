// Block GMRES over the right-hand sides (row a8; Sec. 4.2: the coupled system is solved by GMRES).
//
// The plane waves of one solve share one Krylov space: with the s-column residual block R0 = V0 S0,
//     K_j = span{V0, A V0, ..., A^j V0},  A V_{0:j} = V_{0:j+1} Hbar_j  (block Arnoldi),
// and each column's iterate minimises its own residual over the shared space.  Every block iteration
// costs one s-column application of the operator -- the batched mat-vec -- so a block iteration
// costs what one per-column GMRES iteration costs, and far fewer are needed when the waves excite
// the same slowly converging multiple-scattering modes.
//
// Orthogonalisation is block classical Gram-Schmidt applied twice (CGS2) followed by Cholesky QR
// applied twice (CholQR2) of the new block; the two dense contractions
//     G = V_{0:j}^H W   (Gram, contracted over the N rows)      and      W (+)= V_{0:j} H   (update)
// run on the tensor cores for FP32 bases (tcgen05 kind::tf32, 3xTF32, tc_pipeline.cuh) and on the CUDA
// cores for FP64 ones.  The small dense work -- Cholesky factors, the block Householder QR of the
// block Hessenberg matrix, the residual estimates and the final triangular solve -- runs on the host
// in FP64, parallel over the s columns.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <functional>
#include <vector>

#include "common.cuh"
#include "dense_host.h"
#include "handle.h"
#include "tc_pipeline.cuh"

typedef std::complex<double> cd;

using dense::chol_upper;
using dense::matmul;
using dense::StepQR;
using dense::tri_inv_upper;

namespace {

using tcp::KCC;
using tcp::Stage;

// basis vector k = i s + r of block i, row `row`: V + (i N + row) s + r
__host__ __device__ __forceinline__ size_t vidx(int k, long long row, long long N, int s) {
    const int i = k / s, r = k - i * s;
    return ((size_t)i * N + row) * s + r;
}

// ------------------------------------------------------------------ tensor cores (FP32 bases)
// Gram: part[split][k][r] = sum_{row in split} conj(V_k[row]) W[row][r]; tile = 256 basis vectors.
struct GramPolicy {
    static constexpr bool kStaged = false;
    const float2* V;
    const float2* W;
    double2* part;
    long long N, row0, row1;
    int s, nb, k0, split;
    int k;
    bool valid;
    float2 ya[4];
    float2 vb[8];

    __device__ void init() {
        k = k0 + tcp::brow();
        valid = k < nb;
    }
    __device__ void fetch(int c) {
        const int r = tcp::arow() & 63;
        const long long ra = row0 + (long long)c * KCC + 4 * tcp::aq();
#pragma unroll
        for (int v = 0; v < 4; ++v)
            ya[v] = (r < s && ra + v < row1) ? W[(ra + v) * s + r] : make_float2(0.f, 0.f);
        const long long rb = row0 + (long long)c * KCC + 8 * tcp::bhalf();
#pragma unroll
        for (int v = 0; v < 8; ++v) vb[v] = (valid && rb + v < row1) ? V[vidx(k, rb + v, N, s)] : make_float2(0.f, 0.f);
    }
    __device__ void build(const Stage& st) {
#pragma unroll
        for (int u = 0; u < 2; ++u) tcp::put_a(st, tcp::arow(), 2 * tcp::aq() + u, ya[2 * u], ya[2 * u + 1]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            tcp::put_b(st, tcp::brow(), 4 * tcp::bhalf() + u, make_float2(vb[2 * u].x, -vb[2 * u].y),
                       make_float2(vb[2 * u + 1].x, -vb[2 * u + 1].y));
    }
    __device__ void epilogue(uint32_t tmem, bool ok) {
        const int ncol = min(tcp::NMAX, (nb - k0 + 15) / 16 * 16);
        tcp::for_each_acc(tmem, ncol, [&](int rp, int col, float v) {
            const int r = rp & 63, comp = rp >> 6;
            const int kk = k0 + col;
            if (r >= s || kk >= nb) return;
            reinterpret_cast<double*>(part + ((size_t)split * nb + kk) * s + r)[comp] = ok ? (double)v : 0.0;
        });
    }
};

__global__ void __launch_bounds__(tcp::THREADS, 1)
k_bgram_tc(const float2* __restrict__ V, const float2* __restrict__ W, double2* __restrict__ part, long long N,
           int s, int nb, long long rows_per_split, int* err) {
    GramPolicy pol;
    pol.V = V;
    pol.W = W;
    pol.part = part;
    pol.N = N;
    pol.s = s;
    pol.nb = nb;
    pol.k0 = blockIdx.x * tcp::NMAX;
    pol.split = blockIdx.y;
    pol.row0 = (long long)blockIdx.y * rows_per_split;
    pol.row1 = min(N, pol.row0 + rows_per_split);
    pol.init();
    const int nchunks = pol.row1 > pol.row0 ? (int)((pol.row1 - pol.row0 + KCC - 1) / KCC) : 0;
    tcp::run(pol, nchunks, min(tcp::NMAX, (nb - pol.k0 + 15) / 16 * 16), err);
}

// Update: out[row][r] = (accumulate ? out : 0) + sign sum_k V_k[row] H[k][r]; tile = 256 rows.
struct UpdPolicy {
    static constexpr bool kStaged = false;
    const float2* V;
    const float2* H;       // [nb][s]
    float2* out;
    long long N, row0;
    int s, nb, accumulate;
    float sign;
    long long row;
    bool valid;
    float2 ya[4];
    float2 vb[8];

    __device__ void init() {
        row = row0 + tcp::brow();
        valid = row < N;
    }
    __device__ void fetch(int c) {
        const int r = tcp::arow() & 63;
        const int ka = c * KCC + 4 * tcp::aq();
#pragma unroll
        for (int v = 0; v < 4; ++v) ya[v] = (r < s && ka + v < nb) ? H[(size_t)(ka + v) * s + r] : make_float2(0.f, 0.f);
        const int kb = c * KCC + 8 * tcp::bhalf();
#pragma unroll
        for (int v = 0; v < 8; ++v) vb[v] = (valid && kb + v < nb) ? V[vidx(kb + v, row, N, s)] : make_float2(0.f, 0.f);
    }
    __device__ void build(const Stage& st) {
#pragma unroll
        for (int u = 0; u < 2; ++u) tcp::put_a(st, tcp::arow(), 2 * tcp::aq() + u, ya[2 * u], ya[2 * u + 1]);
#pragma unroll
        for (int u = 0; u < 4; ++u) tcp::put_b(st, tcp::brow(), 4 * tcp::bhalf() + u, vb[2 * u], vb[2 * u + 1]);
    }
    __device__ void epilogue(uint32_t tmem, bool ok) {
        if (!ok) return;
        tcp::for_each_acc(tmem, tcp::NMAX, [&](int rp, int col, float v) {
            const int r = rp & 63, comp = rp >> 6;
            const long long rr = row0 + col;
            if (r >= s || rr >= N) return;
            float* dst = reinterpret_cast<float*>(out + rr * s + r) + comp;
            *dst = accumulate ? *dst + sign * v : sign * v;
        });
    }
};

__global__ void __launch_bounds__(tcp::THREADS, 1)
k_bupdate_tc(const float2* V, const float2* __restrict__ H, float2* out, long long N, int s, int nb,
             int accumulate, float sign, int* err) {
    UpdPolicy pol;
    pol.V = V;
    pol.H = H;
    pol.out = out;
    pol.N = N;
    pol.row0 = (long long)blockIdx.x * tcp::NMAX;
    pol.s = s;
    pol.nb = nb;
    pol.accumulate = accumulate;
    pol.sign = sign;
    pol.init();
    tcp::run(pol, (nb + KCC - 1) / KCC, tcp::NMAX, err);
}

// ------------------------------------------------------------------ CUDA cores (FP64 and FP32 bases)
constexpr int CC_T = 16;            // 16 x 16 threads, 4 x 4 outputs each: 64 x 64 output tile
constexpr int CC_K = 16;            // contracted entries per staged chunk

// part[split][k][r] over a 64-basis-vector x 64-column tile (k = k0 + tk + 16 a, r = tr + 16 b), with
// products and sums in the accumulation type A (double for the exact Gram of an FP32 block: FP32
// products are exact in FP64)
template <typename T, typename A = T>
__global__ void __launch_bounds__(256)
k_bgram_cc(const typename CT<T>::c* __restrict__ V, const typename CT<T>::c* __restrict__ W,
           double2* __restrict__ part, long long N, int s, int nb, long long rows_per_split) {
    typedef typename CT<T>::c CI;
    typedef typename CT<A>::c C;
    __shared__ CI Vs[CC_K][64];
    __shared__ CI Ws[CC_K][64];
    const int k0 = blockIdx.x * 64, split = blockIdx.y;
    const long long row0 = (long long)split * rows_per_split, row1 = min(N, row0 + rows_per_split);
    const int tk = threadIdx.x / CC_T, tr = threadIdx.x % CC_T;
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mk((A)0, (A)0);
    for (long long rc = row0; rc < row1; rc += CC_K) {
        __syncthreads();
        for (int e = threadIdx.x; e < CC_K * 64; e += blockDim.x) {
            const int rr = e / 64, q = e % 64;
            const long long row = rc + rr;
            const bool inrow = row < row1;
            Vs[rr][q] = (inrow && k0 + q < nb) ? cconj(V[vidx(k0 + q, row, N, s)]) : mk((T)0, (T)0);
            Ws[rr][q] = (inrow && q < s) ? W[row * s + q] : mk((T)0, (T)0);
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < CC_K; ++rr) {
            C vv[4], ww[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) vv[a] = to_c<A>(to_d(Vs[rr][tk + 16 * a]));
#pragma unroll
            for (int b = 0; b < 4; ++b) ww[b] = to_c<A>(to_d(Ws[rr][tr + 16 * b]));
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) cfma(acc[a][b], vv[a], ww[b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int k = k0 + tk + 16 * a, r = tr + 16 * b;
            if (k < nb && r < s) part[((size_t)split * nb + k) * s + r] = to_d(acc[a][b]);
        }
}

// out[row][r] = (accumulate ? out : 0) + sign sum_k V_k[row] H[k][r] over a 64-row x 64-column tile
template <typename T>
__global__ void __launch_bounds__(256)
k_bupdate_cc(const typename CT<T>::c* V, const typename CT<T>::c* __restrict__ H,
             typename CT<T>::c* out, long long N, int s, int nb, int accumulate, double sign) {
    typedef typename CT<T>::c C;
    __shared__ C Vs[64][CC_K + 1];
    __shared__ C Hs[CC_K][64];
    const long long r0 = (long long)blockIdx.x * 64;
    const int tw = threadIdx.x / CC_T, tr = threadIdx.x % CC_T;
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = mk((T)0, (T)0);
    for (int kc = 0; kc < nb; kc += CC_K) {
        __syncthreads();
        for (int e = threadIdx.x; e < 64 * CC_K; e += blockDim.x) {
            const int w = e / CC_K, kk = e % CC_K;
            const long long row = r0 + w;
            Vs[w][kk] = (row < N && kc + kk < nb) ? V[vidx(kc + kk, row, N, s)] : mk((T)0, (T)0);
        }
        for (int e = threadIdx.x; e < CC_K * 64; e += blockDim.x) {
            const int kk = e / 64, q = e % 64;
            Hs[kk][q] = (kc + kk < nb && q < s) ? H[(size_t)(kc + kk) * s + q] : mk((T)0, (T)0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < CC_K; ++kk) {
            C vv[4], hh[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) vv[a] = Vs[tw + 16 * a][kk];
#pragma unroll
            for (int b = 0; b < 4; ++b) hh[b] = Hs[kk][tr + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) cfma(acc[a][b], vv[a], hh[b]);
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const long long row = r0 + tw + 16 * a;
            const int r = tr + 16 * b;
            if (row >= N || r >= s) continue;
            double2 v = to_d(acc[a][b]);
            v = make_double2(sign * v.x, sign * v.y);
            C* dst = out + row * s + r;
            *dst = accumulate ? to_c<T>(cadd(to_d(*dst), v)) : to_c<T>(v);
        }
}

// G[k][r] = sum over splits of part[split][k][r]
__global__ void k_bgram_sum(const double2* __restrict__ part, double2* __restrict__ G, int nsplit, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 a = make_double2(0, 0);
    for (int sp = 0; sp < nsplit; ++sp) a = cadd(a, part[(size_t)sp * n + i]);
    G[i] = a;
}

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// Columns c0..s-1 of an N x s block: pseudo-random entries in [-1, 1) + i [-1, 1) from a 64-bit mix
// (splitmix64) of the entry index and the call's seed.
template <typename T>
__global__ void k_fill_random(typename CT<T>::c* __restrict__ dst, long long N, int s, int c0,
                              unsigned long long seed, double scale) {
    const int w = s - c0;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= N * w) return;
    const long long row = i / w;
    const int c = c0 + (int)(i - row * w);
    unsigned long long z = ((unsigned long long)row * s + c) * 0x9E3779B97F4A7C15ull + seed;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    dst[row * s + c] = to_c<T>(make_double2(((z & 0xffffffff) * 0x1p-31 - 1.0) * scale, ((z >> 32) * 0x1p-31 - 1.0) * scale));
}

}  // namespace

// ------------------------------------------------------------------ the block Krylov solver
template <typename T>
struct BlockKrylov {
    typedef typename CT<T>::c C;
    ms_handle* h;
    cudaStream_t st;
    long long N;
    int s, m;
    bool tc;
    C* V = nullptr;          // (m + 1) blocks of N x s
    C* W = nullptr;          // N x s
    C* Hd = nullptr;         // (m + 1) s x s coefficients of an update
    double2* part = nullptr;
    double2* G = nullptr;
    int nsplit_max = 1;
    int deflations = 0;      // rank-deficient blocks met (orth)
    int exhausted = 0;       // of which the basis left no room for filler columns
    int reverted = 0;        // restart cycles undone by the residual safeguard

    C* Z = nullptr;          // N x s: preconditioned block (group-block Jacobi), when the handle has one
    C* Xprev = nullptr;      // N x s: the iterate before the last restart cycle's update

    ~BlockKrylov() {
        cudaFree(V); cudaFree(W); cudaFree(Hd); cudaFree(part); cudaFree(G); cudaFree(Z); cudaFree(Xprev);
    }
    int init() {
        const size_t blk = (size_t)N * s * sizeof(C);
        nsplit_max = std::max(1, std::min(2 * 148, (int)((N + 4095) / 4096)));
        const size_t nbmax = (size_t)(m + 1) * s;
        // split-K partials: a launch uses nsplit <= 296 / ntile + 1 splits of its nb vectors in tiles of
        // <= 256, so nsplit * nb <= 296 * 256 + nb + 256
        const size_t part_cap = ((size_t)2 * 148 * tcp::NMAX + nbmax + tcp::NMAX) * s;
        if (cudaMalloc(&V, blk * (m + 1)) != cudaSuccess || cudaMalloc(&W, blk) != cudaSuccess ||
            cudaMalloc(&Hd, nbmax * s * sizeof(C)) != cudaSuccess ||
            cudaMalloc(&part, part_cap * sizeof(double2)) != cudaSuccess ||
            cudaMalloc(&G, nbmax * s * sizeof(double2)) != cudaSuccess || cudaMalloc(&Xprev, blk) != cudaSuccess ||
            (h->pc.ng > 0 && cudaMalloc(&Z, blk) != cudaSuccess)) {
            cudaGetLastError();
            return MS_ERR_ALLOC;
        }
        return MS_OK;
    }
    C* blk(int i) { return V + (size_t)i * N * s; }

    // out[k * s + r] = <basis_k, Wp[:, r]> for the nb basis vectors starting at block pointer Vb; exact:
    // on the CUDA cores with FP64 products and sums whatever the basis precision
    int gram(const C* Vb, int nb, const C* Wp, std::vector<cd>& out, bool exact = false) {
        int nsplit;
        if (tc && !exact) {
            const int ntile = (nb + tcp::NMAX - 1) / tcp::NMAX;
            nsplit = std::max(1, std::min(nsplit_max, (2 * 148 + ntile - 1) / ntile));
            long long per = (N + nsplit - 1) / nsplit;
            per = (per + KCC - 1) / KCC * KCC;
            nsplit = (int)((N + per - 1) / per);
            cudaFuncSetAttribute(k_bgram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcp::SMEM);
            k_bgram_tc<<<dim3(ntile, nsplit), tcp::THREADS, tcp::SMEM, st>>>(
                (const float2*)Vb, (const float2*)Wp, part, N, s, nb, per, h->d.tc_err);
        } else {
            const int ntile = (nb + 63) / 64;
            nsplit = std::max(1, std::min(nsplit_max, (2 * 148 + ntile - 1) / ntile));
            long long per = (N + nsplit - 1) / nsplit;
            nsplit = (int)((N + per - 1) / per);
            if (exact)
                k_bgram_cc<T, double><<<dim3(ntile, nsplit), 256, 0, st>>>(Vb, Wp, part, N, s, nb, per);
            else
                k_bgram_cc<T><<<dim3(ntile, nsplit), 256, 0, st>>>(Vb, Wp, part, N, s, nb, per);
        }
        const int n = nb * s;
        k_bgram_sum<<<nblk(n, 256), 256, 0, st>>>(part, G, nsplit, n);
        if (int rc = ms_check(h, cudaGetLastError())) return rc;
        out.resize(n);
        if (int rc = ms_check(h, cudaMemcpyAsync(out.data(), G, n * sizeof(double2), cudaMemcpyDeviceToHost, st)))
            return rc;
        if (int rc = ms_check(h, cudaStreamSynchronize(st))) return rc;
        if (tc && !exact) return ms_spectral_tc_status(h, st);
        return MS_OK;
    }
    // out (+)= sign * Vb[:, 0:nb] Hc, Hc = nb x s row-major
    int update(const C* Vb, int nb, const std::vector<cd>& Hc, C* out, bool accumulate, double sign) {
        std::vector<C> hc((size_t)nb * s);
        for (size_t i = 0; i < hc.size(); ++i) hc[i] = to_c<T>(make_double2(Hc[i].real(), Hc[i].imag()));
        if (int rc = ms_check(h, cudaMemcpyAsync(Hd, hc.data(), hc.size() * sizeof(C), cudaMemcpyHostToDevice, st)))
            return rc;
        if (tc) {
            cudaFuncSetAttribute(k_bupdate_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcp::SMEM);
            k_bupdate_tc<<<nblk(N, tcp::NMAX), tcp::THREADS, tcp::SMEM, st>>>(
                (const float2*)Vb, (const float2*)Hd, (float2*)out, N, s, nb, accumulate ? 1 : 0, (float)sign,
                h->d.tc_err);
        } else
            k_bupdate_cc<T><<<nblk(N, 64), 256, 0, st>>>(Vb, Hd, out, N, s, nb, accumulate ? 1 : 0, sign);
        // (a copy from pageable host memory returns once the data are staged: hc may go out of scope)
        return ms_check(h, cudaGetLastError());
    }
    // relative eigenvalue floor of a Gram matrix: below it a direction of the block is rounding noise.
    // For a Gram from the tensor cores (FP32 sums) 64 u of the FP32 basis; for an exact Gram (FP64
    // products and sums) (64 u)^2 for an FP32 basis -- the block's own rounding -- and 64 u for FP64.
    double floor_rel(bool exact = false) const {
        const double u = sizeof(T) == 8 ? 1.11e-16 : 5.96e-8;
        return (exact && sizeof(T) == 4) ? (64.0 * u) * (64.0 * u) : 64.0 * u;
    }
    // Cholesky factor of the leading k x k block of a Gram matrix, refused when a column is negligible
    // against the largest or (nearly) dependent on the columns before it (R_ii^2 below the floor times
    // its own G_ii).  Returns R (k x k, row-major).
    bool chol_checked(const std::vector<cd>& Gm, int k, double floor, std::vector<cd>& R) {
        std::vector<cd> Gk((size_t)k * k);
        double dmax = 0;
        for (int i = 0; i < k; ++i) {
            for (int j = 0; j < k; ++j) Gk[(size_t)i * k + j] = Gm[(size_t)i * s + j];
            dmax = std::max(dmax, Gm[(size_t)i * s + i].real());
        }
        if (!(dmax > 0) || !chol_upper(Gk, k, 0.0, R)) return false;
        for (int i = 0; i < k; ++i) {
            const double gii = Gk[(size_t)i * k + i].real();
            if (!(gii >= floor * dmax) || !(std::norm(R[(size_t)i * k + i]) >= floor * gii)) return false;
        }
        return true;
    }
    // the s x s matrix [R_k^{-1} 0; 0 0] that orthonormalises the leading k columns and zeroes the rest
    std::vector<cd> inv_lead(const std::vector<cd>& Rk, int k) {
        std::vector<cd> Ri, out((size_t)s * s, cd(0));
        tri_inv_upper(Rk, k, Ri);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) out[(size_t)i * s + j] = Ri[(size_t)i * k + j];
        return out;
    }
    // Cholesky QR of the leading k columns of a block in place (the rest zeroed), twice; the first
    // factor from G1 when given.  ok = false when a factor is refused.
    // With k = s and Rout given, Rout = R2 R1 (blk_in = blk_out Rout).
    int cholqr2_lead(C* blk, int k, const std::vector<cd>* G1, double floor1, bool& ok,
                     std::vector<cd>* Rout = nullptr) {
        std::vector<cd> Gm, R1, R2;
        ok = false;
        if (G1) Gm = *G1;
        else if (int rc = gram(blk, s, blk, Gm)) return rc;
        if (!chol_checked(Gm, k, floor1, R1)) return MS_OK;
        if (int rc = update(blk, s, inv_lead(R1, k), blk, false, 1.0)) return rc;
        if (int rc = gram(blk, s, blk, Gm)) return rc;
        if (!chol_checked(Gm, k, floor_rel(), R2)) return MS_OK;
        if (int rc = update(blk, s, inv_lead(R2, k), blk, false, 1.0)) return rc;
        if (Rout && k == s) *Rout = matmul(R2, R1, s);
        ok = true;
        return MS_OK;
    }
    // Orthonormal block dst with src = dst R (R s x s), orthogonal to the nprev basis blocks before it.
    //  1. CholQR2 with tensor-core Grams (well-conditioned blocks).
    //  2. CholQR2 whose first factor comes from an exact Gram (FP64 products and sums): FP32 blocks with
    //     condition numbers up to ~1/u.
    //  3. A (numerically) rank-deficient block -- the Krylov space has (nearly) closed, or the
    //     right-hand sides are dependent: the exact Gram's eigenvectors with eigenvalues above the floor
    //     give its independent directions at unit length; the other columns take pseudo-random vectors
    //     orthogonalised against the basis, or, when the basis leaves no room for them (it spans the
    //     space), zeros.
    // R = dst^H src throughout, so the Arnoldi relation holds up to the dropped noise.  dst may equal src.
    int orth(const C* src, C* dst, int nprev, std::vector<cd>& R) {
        int rc;
        if (src == dst) {
            if ((rc = ms_check(h, cudaMemcpyAsync(W, src, (size_t)N * s * sizeof(C), cudaMemcpyDeviceToDevice, st))))
                return rc;
            src = W;
        }
        auto restart_from_src = [&]() {
            return ms_check(h, cudaMemcpyAsync(dst, src, (size_t)N * s * sizeof(C), cudaMemcpyDeviceToDevice, st));
        };
        if ((rc = restart_from_src())) return rc;
        bool ok;
        if ((rc = cholqr2_lead(dst, s, nullptr, floor_rel(), ok, &R))) return rc;
        if (ok) return MS_OK;
        std::vector<cd> Gx;
        if ((rc = gram(src, s, src, Gx, true))) return rc;
        if ((rc = restart_from_src())) return rc;
        if ((rc = cholqr2_lead(dst, s, &Gx, floor_rel(true), ok, &R))) return rc;
        if (ok) return MS_OK;
        ++deflations;
        // eigenpairs of the Hermitian Gram by one-sided Jacobi: the squared column norms are the
        // eigenvalues of G^2, the accumulated rotations the eigenvectors
        std::vector<cd> A((size_t)s * s), V;
        for (int r = 0; r < s; ++r)
            for (int c = 0; c < s; ++c) A[(size_t)c * s + r] = Gx[(size_t)r * s + c];
        std::vector<double> ev;
        dense::jacobi_svd(A, s, ev, V);
        std::vector<int> order(s);
        for (int i = 0; i < s; ++i) order[i] = i;
        std::sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] > ev[b]; });
        const double lmax = sqrt(std::max(0.0, ev[order[0]]));
        int k = 0;
        std::vector<cd> Y((size_t)s * s, cd(0));
        for (; k < s; ++k) {
            const double lk = sqrt(std::max(0.0, ev[order[k]]));
            if (!(lmax > 0) || !(lk > floor_rel(true) * lmax)) break;
            for (int i = 0; i < s; ++i) Y[(size_t)i * s + k] = V[(size_t)order[k] * s + i] / sqrt(lk);
        }
        auto project_out = [&]() -> int {
            for (int pass = 0; pass < 2 && nprev > 0; ++pass) {
                std::vector<cd> Gp;
                if (int e = gram(blk(0), nprev * s, dst, Gp)) return e;
                if (int e = update(blk(0), nprev * s, Gp, dst, true, -1.0)) return e;
            }
            return MS_OK;
        };
        if ((rc = update(src, s, Y, dst, false, 1.0))) return rc;
        if (k < s) {
            // entries of variance 2/3 per component: unit expected column norm with the 1 / sqrt(4N/3) scale
            k_fill_random<T><<<nblk(N * (s - k), 256), 256, 0, st>>>(dst, N, s, k, 0x632BE59BD9B4E019ull + 977ull * deflations,
                                                                     1.0 / sqrt(4.0 * N / 3.0));
            if ((rc = ms_check(h, cudaGetLastError()))) return rc;
        }
        if ((rc = project_out())) return rc;
        if ((rc = cholqr2_lead(dst, s, nullptr, floor_rel(), ok))) return rc;
        if (!ok) {
            // no room for the filler columns: keep the k independent directions, zero the rest
            ++exhausted;
            if ((rc = update(src, s, Y, dst, false, 1.0))) return rc;
            if ((rc = project_out())) return rc;
            if (k > 0) {
                if ((rc = cholqr2_lead(dst, k, nullptr, floor_rel(), ok))) return rc;
                if (!ok) return MS_ERR_BREAKDOWN;
            }
        }
        return gram(dst, s, src, R);             // R[k][r] = <dst_k, src_r>
    }
};

// Block GMRES(m): solve A x = b for the s columns of b; x holds the initial guess.  op(in, out)
// applies A to an s-column block.  Stops when every column's residual estimate is <= tol ||b_c||.
template <typename T, typename Op>
int block_gmres(BlockKrylov<T>& K, Op op, const typename CT<T>::c* b, typename CT<T>::c* x, double tol,
                int max_iters, bool zero_guess, int& iters_out, int& matvecs, std::vector<double>& relres) {
    typedef typename CT<T>::c C;
    const int s = K.s, m = K.m;
    int rc;
    std::vector<cd> gb;
    if ((rc = K.gram(b, s, b, gb))) return rc;
    std::vector<double> bn(s);
    for (int c = 0; c < s; ++c) {
        const double g2 = gb[(size_t)c * s + c].real();
        bn[c] = std::isnan(g2) ? g2 : sqrt(std::max(0.0, g2));      // a NaN must not read as zero
        if (!std::isfinite(bn[c])) return MS_ERR_NONFINITE;
    }
    relres.assign(s, 0.0);
    int total = 0;
    bool first = true;
    // safeguard: a restart cycle whose update raised the worst true residual (an inaccurate basis or
    // least-squares solution) is undone and the solve returns the previous iterate
    std::vector<double> prev_res;
    double prev_worst = 0;
    while (true) {
        // R0 = b - A x into V_0 (the first cycle of a zero initial guess needs no product)
        if (first && zero_guess) {
            if ((rc = ms_check(K.h, cudaMemcpyAsync(K.blk(0), b, (size_t)K.N * s * sizeof(C),
                                                    cudaMemcpyDeviceToDevice, K.st))))
                return rc;
        } else {
            if ((rc = op(x, K.W))) return rc;
            ++matvecs;
            if ((rc = ms_check(K.h, cudaMemcpyAsync(K.blk(0), b, (size_t)K.N * s * sizeof(C),
                                                    cudaMemcpyDeviceToDevice, K.st))))
                return rc;
            std::vector<cd> I((size_t)s * s, cd(0));
            for (int c = 0; c < s; ++c) I[(size_t)c * s + c] = 1.0;
            if ((rc = K.update(K.W, s, I, K.blk(0), true, -1.0))) return rc;
        }
        first = false;
        std::vector<cd> S0;
        if ((rc = K.orth(K.blk(0), K.blk(0), 0, S0))) return rc;
        // transformed right-hand side of the least-squares problem: (m + 1) s x s, column-major per column c
        const int rows_max = (m + 1) * s;
        std::vector<cd> g((size_t)rows_max * s, cd(0));     // g[row * s + c]
        for (int i = 0; i < s; ++i)
            for (int c = 0; c < s; ++c) g[(size_t)i * s + c] = S0[(size_t)i * s + c];
        bool all = true;
        double worst = 0;
        for (int c = 0; c < s; ++c) {
            double r2 = 0;
            for (int i = 0; i < s; ++i) r2 += std::norm(g[(size_t)i * s + c]);
            relres[c] = bn[c] > 0 ? sqrt(r2) / bn[c] : 0.0;
            all = all && relres[c] <= tol;
            worst = std::max(worst, relres[c]);
        }
        if (!prev_res.empty() && !(worst <= 1.05 * prev_worst)) {
            if ((rc = ms_check(K.h, cudaMemcpyAsync(x, K.Xprev, (size_t)K.N * s * sizeof(C), cudaMemcpyDeviceToDevice,
                                                    K.st))))
                return rc;
            relres = prev_res;
            ++K.reverted;
            break;
        }
        prev_res = relres;
        prev_worst = worst;
        if (all || total >= max_iters) break;
        std::vector<std::vector<cd>> Rcol;      // R block column j: (j + 1) s x s, row-major
        std::vector<StepQR> qr;
        int j = 0;
        for (; j < m && total < max_iters; ++j) {
            if ((rc = op(K.blk(j), K.W))) return rc;
            ++matvecs;
            const int nb = (j + 1) * s;
            std::vector<cd> hcol((size_t)(nb + s) * s, cd(0));      // (j + 2) s x s
            for (int pass = 0; pass < 2; ++pass) {
                std::vector<cd> Gp;
                if ((rc = K.gram(K.blk(0), nb, K.W, Gp))) return rc;
                if ((rc = K.update(K.blk(0), nb, Gp, K.W, true, -1.0))) return rc;
                for (size_t i = 0; i < Gp.size(); ++i) hcol[i] += Gp[i];
            }
            std::vector<cd> Rn;
            if ((rc = K.orth(K.W, K.blk(j + 1), j + 1, Rn))) return rc;
            for (int i = 0; i < s; ++i)
                for (int c = 0; c < s; ++c) hcol[(size_t)(nb + i) * s + c] = Rn[(size_t)i * s + c];
            ++total;
            // previous steps' reflectors on the new block column, then this step's QR, applied to g too
            dense::apply_steps(qr, 0, j, s, hcol.data());
            StepQR q;
            dense::step_qr(&hcol[(size_t)(j * s) * s], s, q);      // the 2s x s panel, row stride s
            qr.push_back(std::move(q));
            dense::apply_steps(qr, j, j + 1, s, g.data());
            Rcol.emplace_back(hcol.begin(), hcol.begin() + (size_t)nb * s);
            all = true;
            for (int c = 0; c < s; ++c) {
                double r2 = 0;
                for (int i = 0; i < s; ++i) r2 += std::norm(g[(size_t)(nb + i) * s + c]);
                relres[c] = bn[c] > 0 ? sqrt(r2) / bn[c] : 0.0;
                if (!std::isfinite(relres[c])) return MS_ERR_NONFINITE;
                all = all && relres[c] <= tol;
            }
            if (all) {
                ++j;
                break;
            }
        }
        // x += V_{0:j} Y with R Y = g[0 : j s] (block upper-triangular back substitution per column)
        const int nbj = j * s;
        if (nbj > 0) {
            std::vector<cd> Y;
            dense::block_back_substitute(Rcol, g, s, j, K.floor_rel(), Y);
            if ((rc = ms_check(K.h, cudaMemcpyAsync(K.Xprev, x, (size_t)K.N * s * sizeof(C), cudaMemcpyDeviceToDevice,
                                                    K.st))))
                return rc;
            if ((rc = K.update(K.blk(0), nbj, Y, x, true, 1.0))) return rc;
        }
        if (all) break;
        if (total >= max_iters) {
            // the cap ended a cycle: its update is checked against the true residual like any other
            if ((rc = op(x, K.W))) return rc;
            ++matvecs;
            if ((rc = ms_check(K.h, cudaMemcpyAsync(K.blk(0), b, (size_t)K.N * s * sizeof(C), cudaMemcpyDeviceToDevice,
                                                    K.st))))
                return rc;
            std::vector<cd> I((size_t)s * s, cd(0));
            for (int c = 0; c < s; ++c) I[(size_t)c * s + c] = 1.0;
            if ((rc = K.update(K.W, s, I, K.blk(0), true, -1.0))) return rc;
            std::vector<cd> gr;
            if ((rc = K.gram(K.blk(0), s, K.blk(0), gr, true))) return rc;
            double worst = 0;
            std::vector<double> now(s);
            for (int c = 0; c < s; ++c) {
                now[c] = bn[c] > 0 ? sqrt(std::max(0.0, gr[(size_t)c * s + c].real())) / bn[c] : 0.0;
                worst = std::max(worst, now[c]);
            }
            if (!(worst <= 1.05 * prev_worst)) {
                if ((rc = ms_check(K.h, cudaMemcpyAsync(x, K.Xprev, (size_t)K.N * s * sizeof(C), cudaMemcpyDeviceToDevice,
                                                        K.st))))
                    return rc;
                ++K.reverted;
            } else {
                relres = now;
            }
            break;
        }
    }
    iters_out = total;
    return MS_OK;
}

// Inner solve of the refinement with block GMRES (scaled basis); see ms_refine_solve.
template <typename T>
int ms_block_inner(ms_handle* h, int nrhs, long long N, const void* rs, void* ds, double tol, int max_iters,
                   bool adjoint, int& iters, int& matvecs, std::vector<double>& relres, cudaStream_t st,
                   void** cache) {
    typedef typename CT<T>::c C;
    BlockKrylov<T>* K = (BlockKrylov<T>*)*cache;
    if (!K) {
        int m = std::max(1, h->opt.restart);
        while (true) {
            K = new BlockKrylov<T>{h, st, N, nrhs, m, sizeof(T) == 4 && h->opt.tensor_cores != 0};
            if (K->init() == MS_OK) break;
            delete K;
            K = nullptr;
            if (m <= 4) return MS_ERR_ALLOC;
            m /= 2;                     // the basis does not fit: restart more often
        }
        *cache = K;
    }
    // right preconditioning: iterate on A~ P^{-1} (A~^H P^{-H}) and map the result back, d = P^{-1} z
    const bool pc = h->pc.ng > 0;
    auto op = [&](const C* in, C* out) -> int {
        int rc;
        if (pc) {
            if ((rc = ms_precond_apply<T>(h, in, K->Z, nrhs, adjoint, st))) return rc;
            in = K->Z;
        }
        if ((rc = ms_operator_op<T>(h, in, out, nrhs, adjoint, st))) return rc;
        if (sizeof(T) == 4 && h->opt.tensor_cores) return ms_spectral_tc_status(h, st);
        return MS_OK;
    };
    int rc = block_gmres<T>(*K, op, (const C*)rs, (C*)ds, tol, max_iters, true, iters, matvecs, relres);
    if (rc || !pc) return rc;
    if ((rc = ms_precond_apply<T>(h, ds, K->Z, nrhs, adjoint, st))) return rc;
    return ms_check(h, cudaMemcpyAsync(ds, K->Z, (size_t)N * nrhs * sizeof(C), cudaMemcpyDeviceToDevice, st));
}

// Block GMRES on the CUDA cores (FP64 or FP32 basis) for an operator given as a callable (the 3D
// system): x holds the initial guess (zero here) and receives the solution; restart in block iterations.
template <typename T>
int ms_block_solve(ms_handle* herr, long long N, int nrhs, int restart,
                   const std::function<int(const typename CT<T>::c*, typename CT<T>::c*)>& op,
                   const typename CT<T>::c* b, typename CT<T>::c* x, double tol, int max_iters, int& iters, int& matvecs,
                   std::vector<double>& relres, cudaStream_t st) {
    int m = std::max(1, restart);
    BlockKrylov<T>* K = nullptr;
    while (true) {
        K = new BlockKrylov<T>{herr, st, N, nrhs, m, false};
        if (K->init() == MS_OK) break;
        delete K;
        K = nullptr;
        if (m <= 4) return MS_ERR_ALLOC;
        m /= 2;
    }
    auto opc = [&](const typename CT<T>::c* in, typename CT<T>::c* out) -> int { return op(in, out); };
    const int rc = block_gmres<T>(*K, opc, b, x, tol, max_iters, true, iters, matvecs, relres);
    delete K;
    return rc;
}

template int ms_block_solve<double>(ms_handle*, long long, int, int, const std::function<int(const double2*, double2*)>&,
                                    const double2*, double2*, double, int, int&, int&, std::vector<double>&, cudaStream_t);
template int ms_block_solve<float>(ms_handle*, long long, int, int, const std::function<int(const float2*, float2*)>&,
                                   const float2*, float2*, double, int, int&, int&, std::vector<double>&, cudaStream_t);

template <typename T>
void ms_block_free(void* cache) {
    delete (BlockKrylov<T>*)cache;
}

template int ms_block_inner<double>(ms_handle*, int, long long, const void*, void*, double, int, bool, int&, int&,
                                    std::vector<double>&, cudaStream_t, void**);
template int ms_block_inner<float>(ms_handle*, int, long long, const void*, void*, double, int, bool, int&, int&,
                                   std::vector<double>&, cudaStream_t, void**);
template void ms_block_free<double>(void*);
template void ms_block_free<float>(void*);
