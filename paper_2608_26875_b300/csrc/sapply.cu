// Scattering-matrix apply for prototype particles (row a7; Sec. 4.3: a small number of prototype
// shapes, rotated copies obtained by a rotation of the basis).
//
// In the scaled basis the matrix of particle m with prototype q and rotation phi_m is
//     S~_m = 2^{-e_m} P S_q P^* 2^{-e_m},   P = diag(e^{-i n phi_m}),  2^{e_m} = diag of its scales,
// which factors through the prototype's own scaled table S~_q = 2^{-e_ref} S_q 2^{-e_ref} (e_ref: the
// scales of the first particle that uses q) as
//     S~_m = R_m S~_q C_m,  R_m = diag(e^{-i n_j phi} 2^{e_ref,j - e_m,j}),  C_m = diag(e^{+i n_k phi} 2^{e_ref,k - e_m,k}),
// so a launch reads one shared table per prototype and two length-2nc factor vectors per particle;
// the adjoint uses S~_m^H = R_m S~_q^H C_m with the conjugate-transposed table.  Particles of one
// prototype and one radius have e_m = e_ref and the powers of two are 1.
//
//   k_sapply_tc      FP32 on the tensor cores (tcgen05 kind::tf32, 3xTF32): one CTA per particle,
//                    C = (R_m S~_q C_m) a~_m as a 128 x (2nc) x (2nc) MMA tile; the generated operand
//                    is the rotated table row, the data operand the particle's 64-column block.
//   k_sapply_cc<T>   CUDA cores (FP64, and FP32 with the tensor cores off): one CTA per particle, the
//                    table and the phased block staged in shared memory in chunks of the contracted index.
//   k_sapply_copy    the operator-parts view without S: y = [x -] a on prototype particles.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "tc_pipeline.cuh"

namespace {

using tcp::KC;
using tcp::KCC;
using tcp::Stage;

// Row and column factors of particle m: rowf[j] = e^{-i n_j phi} 2^{s_j}, colf[j] = e^{+i n_j phi} 2^{s_j},
// s_j = e_ref,j - e_m,j, j = (b, n) over 2nc entries.  The phase is formed in FP64.
__device__ __forceinline__ void factors(int j, int nc, int p, double phi, const int* expo, int m, int ref,
                                        double2& rowf, double2& colf) {
    const int n = (j % nc) - p;
    double s, c;
    sincos((double)n * phi, &s, &c);
    const double f = pow2d(expo[(size_t)ref * 2 * nc + j] - expo[(size_t)m * 2 * nc + j]);
    rowf = make_double2(c * f, -s * f);
    colf = make_double2(c * f, s * f);
}

// ------------------------------------------------------------------ tensor cores (FP32)
struct SapplyPolicy {
    static constexpr bool kStaged = false;
    const float2* a;       // a~ block [M][2nc][nrhs]
    const float2* x;       // x~ block (identity) or NULL
    float2* y;
    const float2* S;       // S~_q or S~_q^H, [2nc][2nc] row-major
    int m, n2, nrhs, identity;
    float2* colf;          // shared [n2]
    float2 rowf;           // this thread's B row
    int j;
    float2 ya[4];
    float2 sb[8];

    __device__ void fetch(int c) {
        const int r = tcp::arow() & 63;
        const int k0 = c * KCC + 4 * tcp::aq();
#pragma unroll
        for (int v = 0; v < 4; ++v)
            ya[v] = (r < nrhs && k0 + v < n2) ? a[((size_t)m * n2 + k0 + v) * nrhs + r] : make_float2(0.f, 0.f);
        const int k1 = c * KCC + 8 * tcp::bhalf();
#pragma unroll
        for (int v = 0; v < 8; ++v) sb[v] = (j < n2 && k1 + v < n2) ? S[(size_t)j * n2 + k1 + v] : make_float2(0.f, 0.f);
    }
    template <class St>
    __device__ void build(const St& st) {
#pragma unroll
        for (int u = 0; u < 2; ++u) tcp::put_a(st, tcp::arow(), 2 * tcp::aq() + u, ya[2 * u], ya[2 * u + 1]);
        const int k1 = (cur_chunk++ * KCC) + 8 * tcp::bhalf();
        if (j >= n2) return;     // B rows past 2nc feed only output columns that are discarded
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float2 g[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int k = k1 + 2 * u + v;
                g[v] = (k < n2) ? tcp::cmulf(tcp::cmulf(rowf, sb[2 * u + v]), colf[k]) : make_float2(0.f, 0.f);
            }
            tcp::put_b(st, j, 4 * tcp::bhalf() + u, g[0], g[1]);
        }
    }
    int cur_chunk = 0;
    __device__ void epilogue(uint32_t tmem, bool ok) {
        if (!ok) return;
        tcp::for_each_acc(tmem, (n2 + 15) / 16 * 16, [&](int rp, int col, float v) {
            const int r = rp & 63, comp = rp >> 6;
            if (r >= nrhs || col >= n2) return;
            const size_t o = ((size_t)m * n2 + col) * nrhs + r;
            const float xv = identity ? reinterpret_cast<const float*>(x + o)[comp] : 0.f;
            reinterpret_cast<float*>(y + o)[comp] = xv - (identity ? v : -v);
        });
    }
};

template <class K>
__global__ void __launch_bounds__(tcp::THREADS, 1)
k_sapply_tc(const float2* __restrict__ a, const float2* __restrict__ x, float2* __restrict__ y,
            const float2* __restrict__ tab, const int* __restrict__ plist, const int* __restrict__ proto,
            const int* __restrict__ pref, const double* __restrict__ rot, const int* __restrict__ expo, int p,
            int nrhs, int identity, int* err) {
    const int nc = 2 * p + 1, n2 = 2 * nc;
    const int m = plist[blockIdx.x];
    const int q = proto[m];
    const int ref = pref[q];
    float2* colf = reinterpret_cast<float2*>(tcp::raw_base());
    const double phi = rot[m];
    if (threadIdx.x < n2) {
        double2 rf, cf;
        factors(threadIdx.x, nc, p, phi, expo, m, ref, rf, cf);
        colf[threadIdx.x] = make_float2((float)cf.x, (float)cf.y);
    }
    SapplyPolicy pol;
    pol.a = a;
    pol.x = x;
    pol.y = y;
    pol.S = tab + (size_t)q * n2 * n2;
    pol.m = m;
    pol.n2 = n2;
    pol.nrhs = nrhs;
    pol.identity = identity;
    pol.colf = colf;
    pol.j = tcp::brow();
    pol.rowf = make_float2(0.f, 0.f);
    if (pol.j < n2) {
        double2 rf, cf;
        factors(pol.j, nc, p, phi, expo, m, ref, rf, cf);
        pol.rowf = make_float2((float)rf.x, (float)rf.y);
    }
    const int nchunks = (n2 + KCC - 1) / KCC;
    // (the pipeline's first barrier, after its tensor-memory allocation, publishes colf)
    tcp::run<SapplyPolicy, K>(pol, nchunks, (n2 + 15) / 16 * 16, err);
}

// ------------------------------------------------------------------ CUDA cores (FP64 / FP32)
constexpr int CC_THREADS = 256;
constexpr int CC_KC = 16;          // contracted entries per staged chunk
constexpr int CC_JV = 8;           // rows per thread (2nc <= 16 * 8 = 128)

template <typename T>
__global__ void __launch_bounds__(CC_THREADS)
k_sapply_cc(const typename CT<T>::c* __restrict__ a, const typename CT<T>::c* __restrict__ x,
            typename CT<T>::c* __restrict__ y, const double2* __restrict__ tab, const int* __restrict__ plist,
            const int* __restrict__ proto, const int* __restrict__ pref, const double* __restrict__ rot,
            const int* __restrict__ expo, int p, int nrhs, int identity, int adj) {
    typedef typename CT<T>::c C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = 2 * p + 1, n2 = 2 * nc;
    C* rowf = reinterpret_cast<C*>(smem_raw);
    C* colf = rowf + n2;
    C* Sc = colf + n2;                 // [n2][CC_KC]
    C* Ac = Sc + n2 * CC_KC;           // [CC_KC][64]
    const int m = plist[blockIdx.x];
    const int q = proto[m];
    const int ref = pref[q];
    const double2* S = tab + (size_t)q * n2 * n2;
    for (int j = threadIdx.x; j < n2; j += blockDim.x) {
        double2 rf, cf;
        factors(j, nc, p, rot[m], expo, m, ref, rf, cf);
        rowf[j] = to_c<T>(rf);
        colf[j] = to_c<T>(cf);
    }
    const int tr = threadIdx.x & 15, tj = threadIdx.x >> 4;   // columns tr + 16 u, rows tj + 16 v
    C acc[CC_JV][4];
#pragma unroll
    for (int v = 0; v < CC_JV; ++v)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[v][u] = mk((T)0, (T)0);
    for (int k0 = 0; k0 < n2; k0 += CC_KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < n2 * CC_KC; e += blockDim.x) {
            const int j = e / CC_KC, k = k0 + e % CC_KC;
            double2 v = make_double2(0.0, 0.0);
            if (k < n2) v = adj ? cconj(S[(size_t)k * n2 + j]) : S[(size_t)j * n2 + k];
            Sc[e] = to_c<T>(v);
        }
        for (int e = threadIdx.x; e < CC_KC * 64; e += blockDim.x) {
            const int k = k0 + e / 64, r = e % 64;
            C v = mk((T)0, (T)0);
            if (k < n2 && r < nrhs) v = cmul(colf[k], a[((size_t)m * n2 + k) * nrhs + r]);
            Ac[e] = v;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < CC_KC; ++k) {
            C av[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) av[u] = Ac[k * 64 + tr + 16 * u];
#pragma unroll
            for (int v = 0; v < CC_JV; ++v) {
                const int j = tj + 16 * v;
                if (j < n2) {
                    const C s = Sc[j * CC_KC + k];
#pragma unroll
                    for (int u = 0; u < 4; ++u) cfma(acc[v][u], s, av[u]);
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < CC_JV; ++v) {
        const int j = tj + 16 * v;
        if (j >= n2) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = tr + 16 * u;
            if (r >= nrhs) continue;
            const size_t o = ((size_t)m * n2 + j) * nrhs + r;
            const C s = cmul(rowf[j], acc[v][u]);
            y[o] = identity ? csub(x[o], s) : s;
        }
    }
}

// y = [x -] a on the prototype particles (operator-parts view without S)
template <typename T>
__global__ void k_sapply_copy(const typename CT<T>::c* __restrict__ a, const typename CT<T>::c* __restrict__ x,
                              typename CT<T>::c* __restrict__ y, const int* __restrict__ plist, int n2, int nrhs,
                              int identity) {
    const int m = plist[blockIdx.x];
    for (int e = threadIdx.x; e < n2 * nrhs; e += blockDim.x) {
        const size_t o = (size_t)m * n2 * nrhs + e;
        y[o] = identity ? csub(x[o], a[o]) : a[o];
    }
}

}  // namespace

// ------------------------------------------------------------------ host side

// Scaled prototype tables S~_q = 2^{-e_ref} S_q 2^{-e_ref} (FP64; FP32 and its conjugate transpose for
// the tensor cores), the reference particle of each prototype and the list of prototype particles.
int ms_sapply_setup(ms_handle* h) {
    const int M = h->M, nc = h->nc, n2 = 2 * nc, Q = h->n_proto;
    if (!h->any_proto) return MS_OK;
    std::vector<int> ref(Q, -1), plist;
    for (int m = 0; m < M; ++m) {
        const int q = h->h_proto[m];
        if (q < 0) continue;
        plist.push_back(m);
        if (ref[q] < 0) ref[q] = m;
    }
    std::vector<double2> t64((size_t)Q * n2 * n2, make_double2(0.0, 0.0));
    std::vector<float2> t32(t64.size()), tH32(t64.size());
    for (int q = 0; q < Q; ++q) {
        if (ref[q] < 0) continue;
        const int* e = &h->h_expo[(size_t)ref[q] * n2];
        for (int j = 0; j < n2; ++j)
            for (int k = 0; k < n2; ++k) {
                const size_t s = ((size_t)q * n2 + j) * n2 + k;
                const double f = pow2d(-e[j] - e[k]);
                t64[s] = make_double2(h->h_protoS[2 * s] * f, h->h_protoS[2 * s + 1] * f);
            }
        for (int j = 0; j < n2; ++j)
            for (int k = 0; k < n2; ++k) {
                const double2 v = t64[((size_t)q * n2 + j) * n2 + k];
                t32[((size_t)q * n2 + j) * n2 + k] = make_float2((float)v.x, (float)v.y);
                tH32[((size_t)q * n2 + k) * n2 + j] = make_float2((float)v.x, -(float)v.y);
            }
    }
    for (int q = 0; q < Q; ++q)
        if (ref[q] < 0) ref[q] = 0;
    h->n_plist = (int)plist.size();
    cudaError_t e;
    if ((e = cudaMalloc(&h->d.sps64, t64.size() * sizeof(double2))) ||
        (e = cudaMalloc(&h->d.sps32, t32.size() * sizeof(float2))) ||
        (e = cudaMalloc(&h->d.spsH32, tH32.size() * sizeof(float2))) ||
        (e = cudaMalloc(&h->d.plist, plist.size() * sizeof(int))) ||
        (e = cudaMalloc(&h->d.pref, ref.size() * sizeof(int))))
        return ms_check(h, e);
    if ((e = cudaMemcpy(h->d.sps64, t64.data(), t64.size() * sizeof(double2), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d.sps32, t32.data(), t32.size() * sizeof(float2), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d.spsH32, tH32.data(), tH32.size() * sizeof(float2), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d.plist, plist.data(), plist.size() * sizeof(int), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(h->d.pref, ref.data(), ref.size() * sizeof(int), cudaMemcpyHostToDevice)))
        return ms_check(h, e);
    return MS_OK;
}

void ms_sapply_free(ms_handle* h) {
    cudaFree(h->d.sps64); cudaFree(h->d.sps32); cudaFree(h->d.spsH32); cudaFree(h->d.plist); cudaFree(h->d.pref);
    h->d.sps64 = nullptr; h->d.sps32 = h->d.spsH32 = nullptr; h->d.plist = h->d.pref = nullptr;
}

template <typename T>
int ms_sapply_proto_launch(ms_handle* h, const void* xs, const void* as, void* ys, int nrhs, bool identity,
                           bool apply_s, int adj, cudaStream_t st) {
    typedef typename CT<T>::c C;
    if (!h->any_proto || h->n_plist == 0) return MS_OK;
    const int n2 = 2 * h->nc, np = h->n_plist;
    if (!apply_s) {
        k_sapply_copy<T><<<np, 256, 0, st>>>((const C*)as, (const C*)xs, (C*)ys, h->d.plist, n2, nrhs,
                                             identity ? 1 : 0);
        return ms_check(h, cudaGetLastError());
    }
    if (sizeof(T) == 4 && h->opt.tensor_cores) {
        const size_t smem = tcp::SMEM + (size_t)n2 * sizeof(float2);
        auto kern = h->tc_kind ? k_sapply_tc<tcp::BF16> : k_sapply_tc<tcp::TF32>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        kern<<<np, tcp::THREADS, smem, st>>>((const float2*)as, (const float2*)xs, (float2*)ys,
                                                    adj ? h->d.spsH32 : h->d.sps32, h->d.plist, h->d.proto,
                                                    h->d.pref, h->d.rot, h->d.expo, h->p, nrhs, identity ? 1 : 0,
                                                    h->d.tc_err);
        return ms_check(h, cudaGetLastError());
    }
    const size_t smem = ((size_t)2 * n2 + (size_t)n2 * CC_KC + (size_t)CC_KC * 64) * sizeof(C);
    cudaFuncSetAttribute(k_sapply_cc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_sapply_cc<T><<<np, CC_THREADS, smem, st>>>((const C*)as, (const C*)xs, (C*)ys, h->d.sps64, h->d.plist,
                                                 h->d.proto, h->d.pref, h->d.rot, h->d.expo, h->p, nrhs,
                                                 identity ? 1 : 0, adj);
    return ms_check(h, cudaGetLastError());
}

template int ms_sapply_proto_launch<double>(ms_handle*, const void*, const void*, void*, int, bool, bool, int,
                                            cudaStream_t);
template int ms_sapply_proto_launch<float>(ms_handle*, const void*, const void*, void*, int, bool, bool, int,
                                           cudaStream_t);
