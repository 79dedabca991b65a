// Group-block Jacobi preconditioner of the coupled system (row a8; Sec. 4.2 solves the system by GMRES).
//
// The strongest couplings of A = I - S (T + R) are the free-space translations between close
// neighbours.  Particles are grouped by a uniform grid (cells sized for about `precond_group` particles;
// a fuller cell is cut into runs of at most twice that, in x order), and per group g
//     B_g = I - S~_g T~_gg            (scaled basis; T~_gg: the Graf blocks between the group's own particles)
// is assembled on the device, inverted in FP64 (Gauss-Jordan with partial pivoting, one CTA per group)
// and kept in FP64 and FP32.  The block GMRES iterates on A~ P^{-1} (right preconditioning, P =
// blockdiag B_g; the adjoint system on A~^H P^{-H}), and the inner solution is d = P^{-1} z.
//
// Assembly: the Graf entries T~^{ml}_{ij} = H_{j-i}(k |c_m - c_l|) e^{i (j-i) arg(c_m - c_l)} 2^{a_m(i) + a_l(j)}
// of every ordered pair of a group are written block by block (the Hankel sequence of a pair comes from
// the same FP64 recurrences as the operator's tables); then, 64 columns of every group at a time, the
// columns are gathered into the operator's vector layout, multiplied by S~ with the operator's own
// scattering-matrix apply, and written back as the columns of I - S~ T~.
#include <math.h>

#include <algorithm>
#include <vector>

#include "bessel.cuh"
#include "common.cuh"
#include "handle.h"

namespace {

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

// Graf blocks of every ordered pair (m, l), m != l, of a group: one CTA per (group, target position,
// source position, wave).  Zero diagonal blocks and zero wave-coupling blocks are written too.
__global__ void k_pc_graf(double2* __restrict__ B, const long long* __restrict__ goff, const int* __restrict__ gptr,
                          const int* __restrict__ gpart, const double* __restrict__ centre_xy,
                          const int* __restrict__ expo, double kp, double ks, int p, int gmax) {
    const int g = blockIdx.z;
    const int ng = gptr[g + 1] - gptr[g];
    const int tm = blockIdx.x / 2, b = blockIdx.x % 2, tl = blockIdx.y;
    if (tm >= ng || tl >= ng) return;
    const int nc = 2 * p + 1, D = ng * 2 * nc;
    const int m = gpart[gptr[g] + tm], l = gpart[gptr[g] + tl];
    __shared__ double2 hs[4 * MS_PMAX + 3];
    __shared__ double Js[2 * MS_PMAX + 2], Ys[2 * MS_PMAX + 2];
    const int K = 2 * p;
    if (threadIdx.x == 0 && m != l) {
        const double vx = centre_xy[2 * m] - centre_xy[2 * l], vy = centre_xy[2 * m + 1] - centre_xy[2 * l + 1];
        const double d = sqrt(vx * vx + vy * vy);
        hankel_phase_seq(K, (b ? ks : kp) * d, vx / d, vy / d, hs, Js, Ys);
    }
    __syncthreads();
    double2* Bg = B + goff[g];
    for (int e = threadIdx.x; e < 2 * nc * nc; e += blockDim.x) {
        const int bb = e / (nc * nc), ij = e % (nc * nc), i = ij / nc, j = ij % nc;
        double2 v = make_double2(0.0, 0.0);
        if (m != l && bb == b) {
            const int ex = expo[((size_t)m * 2 + b) * nc + i] + expo[((size_t)l * 2 + b) * nc + j];
            const double f = pow2d(ex);
            const double2 hv = hs[(j - i) + K];
            v = make_double2(hv.x * f, hv.y * f);
        }
        // row (tm, b, i), column (tl, bb, j)
        Bg[(size_t)(tm * 2 * nc + b * nc + i) * D + tl * 2 * nc + bb * nc + j] = v;
    }
}

// columns c0 .. c0 + 63 of every group into the operator layout x[(m, b, n)][r] (zero past the group)
__global__ void k_pc_gather(const double2* __restrict__ B, const long long* __restrict__ goff, const int* __restrict__ pgrp,
                            const int* __restrict__ ppos, const int* __restrict__ gptr, double2* __restrict__ x, int M,
                            int nc, int c0) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)M * 2 * nc * 64) return;
    const int r = (int)(i % 64);
    const long long row = i / 64;
    const int m = (int)(row / (2 * nc)), bn = (int)(row % (2 * nc));
    const int g = pgrp[m];
    const int D = (gptr[g + 1] - gptr[g]) * 2 * nc;
    const int col = c0 + r;
    x[i] = col < D ? B[goff[g] + (size_t)(ppos[m] * 2 * nc + bn) * D + col] : make_double2(0.0, 0.0);
}

// B_g[:, c0 + r] = e_{c0 + r} - y[:, r]
__global__ void k_pc_scatter(double2* __restrict__ B, const long long* __restrict__ goff, const int* __restrict__ pgrp,
                             const int* __restrict__ ppos, const int* __restrict__ gptr, const double2* __restrict__ y,
                             int M, int nc, int c0) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)M * 2 * nc * 64) return;
    const int r = (int)(i % 64);
    const long long row = i / 64;
    const int m = (int)(row / (2 * nc)), bn = (int)(row % (2 * nc));
    const int g = pgrp[m];
    const int D = (gptr[g + 1] - gptr[g]) * 2 * nc;
    const int col = c0 + r;
    if (col >= D) return;
    const int lr = ppos[m] * 2 * nc + bn;
    const double2 v = y[i];
    B[goff[g] + (size_t)lr * D + col] = make_double2((lr == col ? 1.0 : 0.0) - v.x, -v.y);
}

// In-place Gauss-Jordan inversion with partial pivoting of every group's block (one CTA per group):
// per pivot k, the largest |a_ik|, i >= k, is swapped into row k, row k is scaled by 1/a_kk, every other
// row i loses a_ik times row k (its column k becoming -a_ik / a_kk), and at the end the columns are
// swapped back in reverse order.  A zero pivot column sets *singular and leaves that block.
constexpr int PC_THREADS = 1024;

__global__ void __launch_bounds__(PC_THREADS) k_pc_invert(double2* __restrict__ B, const long long* __restrict__ goff,
                                                          const int* __restrict__ gptr, int nc, int* __restrict__ ipiv_all,
                                                          const long long* __restrict__ poff, int* __restrict__ singular) {
    extern __shared__ double2 fcol[];                 // [D] the pivot column before the update
    __shared__ double redv[PC_THREADS / 32];
    __shared__ int redi[PC_THREADS / 32];
    __shared__ int piv_s;
    const int g = blockIdx.x;
    const int D = (gptr[g + 1] - gptr[g]) * 2 * nc;
    double2* A = B + goff[g];
    int* ipiv = ipiv_all + poff[g];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int k = 0; k < D; ++k) {
        // pivot search over rows k..D-1 of column k
        double best = -1.0;
        int bi = k;
        for (int i = k + tid; i < D; i += PC_THREADS) {
            const double2 v = A[(size_t)i * D + k];
            const double a = v.x * v.x + v.y * v.y;
            if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { redv[wid] = best; redi[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            double bb = -1.0;
            int ii = k;
            for (int w = 0; w < PC_THREADS / 32; ++w)
                if (redv[w] > bb || (redv[w] == bb && redi[w] < ii)) { bb = redv[w]; ii = redi[w]; }
            piv_s = bb > 0.0 ? ii : -1;
            ipiv[k] = ii;
        }
        __syncthreads();
        const int piv = piv_s;
        if (piv < 0) {
            if (tid == 0) atomicExch(singular, 1);
            return;
        }
        if (piv != k)
            for (int j = tid; j < D; j += PC_THREADS) {
                const double2 t = A[(size_t)k * D + j];
                A[(size_t)k * D + j] = A[(size_t)piv * D + j];
                A[(size_t)piv * D + j] = t;
            }
        __syncthreads();
        const double2 akk = A[(size_t)k * D + k];
        const double den = akk.x * akk.x + akk.y * akk.y;
        const double2 c = make_double2(akk.x / den, -akk.y / den);      // 1 / a_kk
        __syncthreads();
        for (int j = tid; j < D; j += PC_THREADS) {
            const double2 v = j == k ? make_double2(1.0, 0.0) : A[(size_t)k * D + j];
            A[(size_t)k * D + j] = cmul(v, c);
        }
        for (int i = tid; i < D; i += PC_THREADS) fcol[i] = i == k ? make_double2(0.0, 0.0) : A[(size_t)i * D + k];
        __syncthreads();
        // rows i != k: a_ij -= f_i a_kj (j != k); a_ik = -f_i c
        const long long n2 = (long long)D * D;
        for (long long e = tid; e < n2; e += PC_THREADS) {
            const int i = (int)(e / D), j = (int)(e - (long long)i * D);
            if (i == k) continue;
            const double2 f = fcol[i];
            if (j == k)
                A[e] = make_double2(-(f.x * c.x - f.y * c.y), -(f.x * c.y + f.y * c.x));
            else
                A[e] = csub(A[e], cmul(f, A[(size_t)k * D + j]));
        }
        __syncthreads();
    }
    for (int k = D - 1; k >= 0; --k) {
        const int pv = ipiv[k];
        if (pv != k)
            for (int i = tid; i < D; i += PC_THREADS) {
                const double2 t = A[(size_t)i * D + k];
                A[(size_t)i * D + k] = A[(size_t)i * D + pv];
                A[(size_t)i * D + pv] = t;
            }
        __syncthreads();
    }
}

__global__ void k_pc_to_f32(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// y_g = Binv_g x_g (adj = 0) or Binv_g^H x_g (adj = 1) for every group, x and y in the operator layout
// [M][2][nc][nrhs] (y != x).  CTA = (64-row tile, group); K staged in tiles of AP_K.
constexpr int AP_ROWS = 64, AP_K = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_pc_apply(const typename CT<T>::c* __restrict__ Binv,
                                                  const long long* __restrict__ goff, const int* __restrict__ gptr,
                                                  const int* __restrict__ gpart, const typename CT<T>::c* __restrict__ x,
                                                  typename CT<T>::c* __restrict__ y, int nc, int nrhs, int adj) {
    typedef typename CT<T>::c C;
    __shared__ C As[AP_ROWS][AP_K + 1];
    __shared__ C Xs[AP_K][64];
    const int g = blockIdx.y;
    const int ng = gptr[g + 1] - gptr[g];
    const int D = ng * 2 * nc;
    const int r0 = blockIdx.x * AP_ROWS;
    if (r0 >= D) return;
    const C* Bg = Binv + goff[g];
    const int* part = gpart + gptr[g];
    const int tid = threadIdx.x;
    // thread: rows tr + 16 u (u < 4), columns tc + 16 v (v < 4)
    const int tr = tid >> 4, tc = tid & 15;
    C acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = mk((T)0, (T)0);
    for (int k0 = 0; k0 < D; k0 += AP_K) {
        for (int e = tid; e < AP_ROWS * AP_K; e += 256) {
            const int rr = e / AP_K, kk = e % AP_K;
            const int row = r0 + rr, col = k0 + kk;
            C v = mk((T)0, (T)0);
            if (row < D && col < D) v = adj ? cconj(Bg[(size_t)col * D + row]) : Bg[(size_t)row * D + col];
            As[rr][kk] = v;
        }
        for (int e = tid; e < AP_K * 64; e += 256) {
            const int kk = e / 64, r = e % 64;
            const int col = k0 + kk;
            C v = mk((T)0, (T)0);
            if (col < D && r < nrhs) {
                const int pos = col / (2 * nc), bn = col % (2 * nc);
                v = x[((size_t)part[pos] * 2 * nc + bn) * nrhs + r];
            }
            Xs[kk][r] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < AP_K; ++kk) {
            C a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[tr + 16 * u][kk];
#pragma unroll
            for (int v = 0; v < 4; ++v) b[v] = Xs[kk][tc + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = cadd(acc[u][v], cmul(a[u], b[v]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int row = r0 + tr + 16 * u;
        if (row >= D) continue;
        const int pos = row / (2 * nc), bn = row % (2 * nc);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = tc + 16 * v;
            if (r < nrhs) y[((size_t)part[pos] * 2 * nc + bn) * nrhs + r] = acc[u][v];
        }
    }
}

template <typename T>
int upv(ms_handle* h, T** dst, const std::vector<T>& v) {
    *dst = nullptr;
    if (v.empty()) return MS_OK;
    if (cudaMalloc((void**)dst, v.size() * sizeof(T)) != cudaSuccess) return MS_ERR_ALLOC;
    return ms_check(h, cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
}

}  // namespace

void ms_precond_free(ms_handle* h) {
    PrecondDev& P = h->pc;
    cudaFree(P.inv64); cudaFree(P.inv32); cudaFree(P.goff); cudaFree(P.gptr); cudaFree(P.gpart);
    cudaFree(P.pgrp); cudaFree(P.ppos);
    P = PrecondDev{};
}

// Groups, assembly and inversion (ms_options.precond_group > 0).  Called from ms_setup.
int ms_precond_build(ms_handle* h) {
    ms_precond_free(h);
    const int target = h->opt.precond_group;
    if (target <= 0) return MS_OK;
    const int M = h->M, nc = h->nc;
    const double* c = h->h_centres.data();
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int m = 0; m < M; ++m) {
        xmin = std::min(xmin, c[2 * m]); xmax = std::max(xmax, c[2 * m]);
        ymin = std::min(ymin, c[2 * m + 1]); ymax = std::max(ymax, c[2 * m + 1]);
    }
    const double Sx = xmax - xmin + 1e-9, Sy = ymax - ymin + 1e-9;
    const double ncell = std::max(1.0, (double)M / target);
    int nx = std::max(1, (int)lround(sqrt(ncell * Sx / Sy)));
    int ny = std::max(1, (int)lround(ncell / nx));
    std::vector<std::vector<int>> cells((size_t)nx * ny);
    for (int m = 0; m < M; ++m) {
        const int ix = std::min(nx - 1, (int)((c[2 * m] - xmin) / Sx * nx));
        const int iy = std::min(ny - 1, (int)((c[2 * m + 1] - ymin) / Sy * ny));
        cells[(size_t)iy * nx + ix].push_back(m);
    }
    const int gmax = 2 * target;
    std::vector<int> gptr{0}, gpart, pgrp(M), ppos(M);
    for (auto& cl : cells) {
        if (cl.empty()) continue;
        std::sort(cl.begin(), cl.end(), [&](int a, int b) { return c[2 * a] < c[2 * b]; });
        const int nch = ((int)cl.size() + gmax - 1) / gmax;
        const int per = ((int)cl.size() + nch - 1) / nch;
        for (size_t s = 0; s < cl.size(); s += per) {
            const int g = (int)gptr.size() - 1;
            for (size_t t = s; t < std::min(cl.size(), s + per); ++t) {
                pgrp[cl[t]] = g;
                ppos[cl[t]] = (int)(t - s);
                gpart.push_back(cl[t]);
            }
            gptr.push_back((int)gpart.size());
        }
    }
    const int ng = (int)gptr.size() - 1;
    std::vector<long long> goff(ng + 1, 0), poff(ng + 1, 0);
    int dmax = 0;
    for (int g = 0; g < ng; ++g) {
        const long long D = (long long)(gptr[g + 1] - gptr[g]) * 2 * nc;
        goff[g + 1] = goff[g] + D * D;
        poff[g + 1] = poff[g] + D;
        dmax = std::max(dmax, (int)D);
    }
    // the inversion keeps one pivot column of the largest block in shared memory; groups index grid z
    // (assembly) and grid y (apply), at most 65535
    if ((size_t)dmax * sizeof(double2) > (size_t)200 * 1024 || ng > 65535) return MS_ERR_UNSUPPORTED;
    PrecondDev& P = h->pc;
    P.ng = ng;
    P.total = goff[ng];
    P.dmax = dmax;
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    if ((size_t)P.total * 24 + ((size_t)4 << 30) > freeb) return MS_ERR_ALLOC;
    int rc;
    if ((rc = upv(h, &P.goff, goff)) || (rc = upv(h, &P.gptr, gptr)) || (rc = upv(h, &P.gpart, gpart)) ||
        (rc = upv(h, &P.pgrp, pgrp)) || (rc = upv(h, &P.ppos, ppos))) {
        ms_precond_free(h);
        return rc;
    }
    if (cudaMalloc(&P.inv64, (size_t)P.total * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&P.inv32, (size_t)P.total * sizeof(float2)) != cudaSuccess) {
        ms_precond_free(h);
        return MS_ERR_ALLOC;
    }
    double* dxy = nullptr;
    long long* dpoff = nullptr;
    int *ipiv = nullptr, *sing = nullptr;
    double2 *xg = nullptr, *yg = nullptr;
    const size_t vec = (size_t)M * 2 * nc * 64;
    if (cudaMalloc(&dxy, 2 * M * sizeof(double)) != cudaSuccess || cudaMalloc(&dpoff, (ng + 1) * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&ipiv, std::max<long long>(1, poff[ng]) * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&sing, sizeof(int)) != cudaSuccess || cudaMalloc(&xg, vec * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&yg, vec * sizeof(double2)) != cudaSuccess) {
        cudaFree(dxy); cudaFree(dpoff); cudaFree(ipiv); cudaFree(sing); cudaFree(xg); cudaFree(yg);
        ms_precond_free(h);
        return MS_ERR_ALLOC;
    }
    rc = ms_check(h, cudaMemcpy(dxy, c, 2 * M * sizeof(double), cudaMemcpyHostToDevice));
    if (!rc) rc = ms_check(h, cudaMemcpy(dpoff, poff.data(), (ng + 1) * sizeof(long long), cudaMemcpyHostToDevice));
    if (!rc) rc = ms_check(h, cudaMemset(sing, 0, sizeof(int)));
    const int gm = gmax;
    if (!rc) {
        k_pc_graf<<<dim3(2 * gm, gm, ng), 256>>>(P.inv64, P.goff, P.gptr, P.gpart, dxy, h->d.expo, h->kp_l, h->ks_l,
                                                 h->p, gm);
        rc = ms_check(h, cudaGetLastError());
    }
    for (int c0 = 0; !rc && c0 < dmax; c0 += 64) {
        k_pc_gather<<<nblk((long long)vec, 256), 256>>>(P.inv64, P.goff, P.pgrp, P.ppos, P.gptr, xg, M, nc, c0);
        if ((rc = ms_check(h, cudaGetLastError()))) break;
        if ((rc = ms_sapply_scaled<double>(h, nullptr, yg, 64, false, true, 0, 0, xg))) break;
        k_pc_scatter<<<nblk((long long)vec, 256), 256>>>(P.inv64, P.goff, P.pgrp, P.ppos, P.gptr, yg, M, nc, c0);
        rc = ms_check(h, cudaGetLastError());
    }
    if (!rc) {
        rc = ms_check(h, cudaFuncSetAttribute(k_pc_invert, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              dmax * (int)sizeof(double2)));
        if (!rc) {
            k_pc_invert<<<ng, PC_THREADS, dmax * sizeof(double2)>>>(P.inv64, P.goff, P.gptr, nc, ipiv, dpoff, sing);
            rc = ms_check(h, cudaGetLastError());
        }
    }
    if (!rc) {
        k_pc_to_f32<<<nblk(P.total, 256), 256>>>(P.inv64, P.inv32, P.total);
        rc = ms_check(h, cudaGetLastError());
    }
    int hs = 0;
    if (!rc) rc = ms_check(h, cudaMemcpy(&hs, sing, sizeof(int), cudaMemcpyDeviceToHost));
    cudaFree(dxy); cudaFree(dpoff); cudaFree(ipiv); cudaFree(sing); cudaFree(xg); cudaFree(yg);
    if (!rc && hs) rc = MS_ERR_BREAKDOWN;
    if (rc) ms_precond_free(h);
    return rc;
}

// y = P^{-1} x (adjoint: P^{-H} x) in the scaled basis, FP64 or FP32 blocks as T.
template <typename T>
int ms_precond_apply(ms_handle* h, const void* x, void* y, int nrhs, bool adjoint, cudaStream_t st) {
    typedef typename CT<T>::c C;
    const PrecondDev& P = h->pc;
    const C* Bi = (const C*)(sizeof(T) == 8 ? (const void*)P.inv64 : (const void*)P.inv32);
    if (nrhs < 1 || nrhs > 64) return MS_ERR_UNSUPPORTED;           // one block of at most 64 columns
    k_pc_apply<T><<<dim3(nblk(P.dmax, AP_ROWS), P.ng), 256, 0, st>>>(Bi, P.goff, P.gptr, P.gpart, (const C*)x, (C*)y,
                                                                     h->nc, nrhs, adjoint ? 1 : 0);
    return ms_check(h, cudaGetLastError());
}

template int ms_precond_apply<double>(ms_handle*, const void*, void*, int, bool, cudaStream_t);
template int ms_precond_apply<float>(ms_handle*, const void*, void*, int, bool, cudaStream_t);
