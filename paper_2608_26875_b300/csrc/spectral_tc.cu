// Spectral part of the FP32 operator on the fifth-generation tensor cores (tcgen05, kind::tf32),
// with FP32-level accuracy from the 3xTF32 split (a b ~ ah bh + ah bl + al bh, FP32 accumulation
// in tensor memory).
//
// Both spectral maps are dense complex contractions across the block of right-hand sides:
//   S2L (Sec. 5.3):  a~_b[(m,n), r] (+)= sum_q G_b(q, m, n) D_b(q, r)
//   M2S (Sec. 5.4):  U_b[q, r]       =  sum_(l,n) F_b(q, l, n) x~_b[(l,n), r]
// with generated operator entries  G = E_s2l(q, m) Qs(q, n) 2^{a(m,b,n)},  F = E_m2s(q, l) Qm(q, n) 2^{a(l,b,n)},
//   E_s2l(q, m) = e^{i xi_q x_m + s_b y_m},  E_m2s(q, l) = e^{s_b y_l - i xi_q x_l},
//   Qs(q, n) = i^n q_b^n W_q,  Qm(q, n) = (-i)^n q_b^n / (i pi s_b)          (ja/stm/eee1, pts1/sed1/sed2).
// The adjoints (B^H for S2L-shaped, C^H for M2S-shaped launches) take the other map's tables, conjugated.
//
// Both run on the shared tcgen05 pipeline of tc_pipeline.cuh: the data (amplitudes D or coefficients
// x~) form the 128-row A operand, the generated operator entries the 256-row B operand.
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
constexpr int NT = tcp::NMAX;
constexpr int THREADS = tcp::THREADS;
constexpr size_t SMEM = tcp::SMEM;

__device__ __forceinline__ float2 gen_entry(float2 e, float2 qm, int ex, int conj) {
    float2 v = tcp::cmulf(e, qm);
    float f = pow2f(ex);
    return make_float2(v.x * f, conj ? -v.y * f : v.y * f);
}

// ------------------------------------------------------------------ S2L-shaped launch
// out_b[(m,n), r] (+)= sum_q Z(q, m, n) D_b(q, r);  tile = 256 consecutive rows j = m nc + n.
// The K chunk's distinct operator data -- E of the tile's particles and Q of every order, for the
// chunk's 16 nodes -- are fetched cooperatively (one or two 16-byte loads per thread) and staged in
// shared memory: rows of E (16 nodes), Q mantissas (padded to 18 nodes) and Q exponents (padded to
// 20), so that a warp's 16-byte reads of neighbouring orders spread over the banks.
constexpr int QS_STRIDE = 18;   // float2 per staged Q row
constexpr int QE_STRIDE = 20;   // int per staged exponent row

__host__ __device__ inline int s2l_parts_per_tile(int nc) { return (tcp::NMAX + nc - 1) / nc + 1; }
__host__ __device__ inline size_t s2l_raw_bytes(int nc) {
    return (size_t)s2l_parts_per_tile(nc) * 16 * 8 + (size_t)nc * QS_STRIDE * 8 + (size_t)nc * QE_STRIDE * 4;
}

struct S2LPolicy {
    static constexpr bool kStaged = true;
    const float2* D;       // [NSp][nrhs] this wave (zero beyond NS)
    const float2* E;       // [M][NSp] this wave
    const float2* Qm;      // [nc][NSp] this wave
    const int* Qe;
    const int* expo;       // [M][2][nc]
    float2* out;           // [M][2][nc][nrhs]
    int M, nc, NSp, nrhs, b, j0, accumulate, conj;
    int j, m, n, a, m0, npt, nitems;
    bool valid;
    // one fetched chunk: this thread's data rows and its share of the staged items
    float2 ya[4];
    float4 it[2];

    __device__ void init() {
        j = j0 + tcp::brow();
        valid = j < M * nc;
        m = valid ? j / nc : 0;
        n = valid ? j - m * nc : 0;
        a = valid ? expo[((size_t)m * 2 + b) * nc + n] : 0;
        m0 = j0 / nc;
        npt = s2l_parts_per_tile(nc);
        nitems = npt * 8 + nc * 8 + nc * 4;
    }
    // staged item e: E (npt x 8 float4), then Q mantissas (nc x 8 float4), then exponents (nc x 4 int4)
    __device__ float4 load_item(int e, int q0) const {
        if (e < npt * 8) {
            const int mi = e >> 3, part = e & 7;
            if (m0 + mi >= M) return make_float4(0.f, 0.f, 0.f, 0.f);
            return *reinterpret_cast<const float4*>(E + (size_t)(m0 + mi) * NSp + q0 + 2 * part);
        }
        e -= npt * 8;
        if (e < nc * 8) return *reinterpret_cast<const float4*>(Qm + (size_t)(e >> 3) * NSp + q0 + 2 * (e & 7));
        e -= nc * 8;
        const int4 v = *reinterpret_cast<const int4*>(Qe + (size_t)(e >> 2) * NSp + q0 + 4 * (e & 3));
        return make_float4(__int_as_float(v.x), __int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w));
    }
    __device__ void store_item(unsigned char* raw, int e, float4 v) const {
        float2* Es = reinterpret_cast<float2*>(raw);
        float2* Qs = Es + npt * 16;
        int* Qx = reinterpret_cast<int*>(Qs + nc * QS_STRIDE);
        if (e < npt * 8) {
            *reinterpret_cast<float4*>(Es + (e >> 3) * 16 + 2 * (e & 7)) = v;
            return;
        }
        e -= npt * 8;
        if (e < nc * 8) {
            *reinterpret_cast<float4*>(Qs + (e >> 3) * QS_STRIDE + 2 * (e & 7)) = v;
            return;
        }
        e -= nc * 8;
        *reinterpret_cast<float4*>(Qx + (e >> 2) * QE_STRIDE + 4 * (e & 3)) = v;
    }
    __device__ unsigned char* raw(int c) const {
        return tcp::raw_base() + (size_t)(c & 1) * ((s2l_raw_bytes(nc) + 15) / 16 * 16);
    }
    __device__ void fetch(int c) {
        const int r = tcp::arow() & 63;
        const int qa = c * KCC + 4 * tcp::aq();
#pragma unroll
        for (int v = 0; v < 4; ++v) ya[v] = r < nrhs ? D[(size_t)(qa + v) * nrhs + r] : make_float2(0.f, 0.f);
        const int q0 = c * KCC;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int e = threadIdx.x + k * tcp::THREADS;
            if (e < nitems) it[k] = load_item(e, q0);
        }
    }
    __device__ void stage(int c) {
        unsigned char* rb = raw(c);
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int e = threadIdx.x + k * tcp::THREADS;
            if (e < nitems) store_item(rb, e, it[k]);
        }
        cur = rb;
    }
    template <class St>
    __device__ void build(const St& st) {
#pragma unroll
        for (int u = 0; u < 2; ++u) tcp::put_a(st, tcp::arow(), 2 * tcp::aq() + u, ya[2 * u], ya[2 * u + 1]);
        // the chunk being built is the one staged last: its buffer is raw(c) with c from the stage call
        const float2* Es = reinterpret_cast<const float2*>(cur);
        const float2* Qs = Es + npt * 16;
        const int* Qx = reinterpret_cast<const int*>(Qs + nc * QS_STRIDE);
        const int h8 = 8 * tcp::bhalf();
        const float4* er = reinterpret_cast<const float4*>(Es + (m - m0) * 16 + h8);
        const float4* qr = reinterpret_cast<const float4*>(Qs + n * QS_STRIDE + h8);
        const int4* xr = reinterpret_cast<const int4*>(Qx + n * QE_STRIDE + h8);
        const int4 x0 = xr[0], x1 = xr[1];
        const int xe[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float2 g0 = make_float2(0.f, 0.f), g1 = g0;
            if (valid) {
                const float4 e4 = er[u], q4 = qr[u];
                g0 = gen_entry(make_float2(e4.x, e4.y), make_float2(q4.x, q4.y), xe[2 * u] + a, conj);
                g1 = gen_entry(make_float2(e4.z, e4.w), make_float2(q4.z, q4.w), xe[2 * u + 1] + a, conj);
            }
            tcp::put_b(st, tcp::brow(), 4 * tcp::bhalf() + u, g0, g1);
        }
    }
    unsigned char* cur = nullptr;   // raw buffer of the chunk last staged
    __device__ void epilogue(uint32_t tmem, bool ok) {
        if (!ok) return;
        tcp::for_each_acc(tmem, NT, [&](int rp, int col, float v) {
            const int r = rp & 63, comp = rp >> 6;
            const int jj = j0 + col;
            if (r >= nrhs || jj >= M * nc) return;
            const int m2 = jj / nc, n2 = jj - m2 * nc;
            float* dst = reinterpret_cast<float*>(out + (((size_t)m2 * 2 + b) * nc + n2) * nrhs + r) + comp;
            *dst = accumulate ? *dst + v : v;
        });
    }
};

template <class K>
__global__ void __launch_bounds__(THREADS, 1)
k_s2l_tc(const float2* __restrict__ D, const float2* __restrict__ E, const float2* __restrict__ Qm,
         const int* __restrict__ Qe, const int* __restrict__ expo, float2* __restrict__ out, int M, int nc, int NSp,
         int nrhs, int accumulate, int conj, int* err) {
    const int b = blockIdx.y;
    S2LPolicy pol{D + (size_t)b * NSp * nrhs, E + (size_t)b * M * NSp, Qm + (size_t)b * nc * NSp,
                  Qe + (size_t)b * nc * NSp, expo, out, M, nc, NSp, nrhs, b, (int)blockIdx.x * NT, accumulate, conj};
    pol.init();
    tcp::run<S2LPolicy, K>(pol, NSp / KCC, NT, err);
}

// ------------------------------------------------------------------ M2S-shaped launch
// part[split][b][q][r] = sum_{(l,n) in split's rows} Z(q, l, n) x~_b[(l,n), r];  tile = 256 nodes.
// Along the orders of one particle the entries obey Z(q, l, n+1) = Z(q, l, n) rho_q 2^{a(l,n+1) - a(l,n)}
// with rho_q = -i q (multipole-to-Sommerfeld powers) or i q (the Sommerfeld-to-local ones of the
// adjoint): a thread reads the power table once per particle segment of its 8 entries and steps the
// rest by one complex multiply and an exact power-of-two scale (relative error ~1e-6 after 7 steps).
struct M2SPolicy {
    static constexpr bool kStaged = false;
    const float2* xs;      // [M][2][nc][nrhs]
    const float2* E;       // [M][NSp] this wave
    const float2* Qm;      // [nc][NSp] this wave (node-contiguous: neighbouring threads, neighbouring nodes)
    const int* Qe;
    const float2* rho;     // [NSp] this wave: ratio of consecutive powers
    const int* expo;
    double2* part;         // [nsplit][2][NS][nrhs]
    int M, nc, NS, NSp, nrhs, b, q0, i0, i1, split, conj;
    int q;
    bool valid;
    float2 rq;
    // one fetched chunk (this thread's share)
    float2 ya[4];
    float2 ee[8], qm[8];
    int qe[8], ax[8];
    unsigned vmask, smask;     // entries present; entries that start a particle segment

    __device__ void init() {
        q = q0 + tcp::brow();
        valid = q < NS;
        rq = valid ? rho[q] : make_float2(0.f, 0.f);
    }
    __device__ void fetch(int c) {
        const int r = tcp::arow() & 63;
        const bool ok = r < nrhs;
        const int ia = i0 + c * KCC + 4 * tcp::aq();
        int l = ia / nc, n = ia - l * nc;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            ya[v] = (ok && ia + v < i1) ? xs[(((size_t)l * 2 + b) * nc + n) * nrhs + r] : make_float2(0.f, 0.f);
            if (++n == nc) { n = 0; ++l; }
        }
        const int ib = i0 + c * KCC + 8 * tcp::bhalf();
        l = ib / nc;
        n = ib - l * nc;
        vmask = smask = 0;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            if (valid && ib + v < i1) {
                vmask |= 1u << v;
                ax[v] = expo[((size_t)l * 2 + b) * nc + n];
                if (v == 0 || n == 0) {
                    smask |= 1u << v;
                    ee[v] = E[(size_t)l * NSp + q];
                    qm[v] = Qm[(size_t)n * NSp + q];
                    qe[v] = Qe[(size_t)n * NSp + q];
                }
            }
            if (++n == nc) { n = 0; ++l; }
        }
    }
    template <class St>
    __device__ void build(const St& st) {
#pragma unroll
        for (int u = 0; u < 2; ++u) tcp::put_a(st, tcp::arow(), 2 * tcp::aq() + u, ya[2 * u], ya[2 * u + 1]);
        float2 w = make_float2(0.f, 0.f);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float2 g[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int e = 2 * u + v;
                g[v] = make_float2(0.f, 0.f);
                if ((vmask >> e) & 1u) {
                    if ((smask >> e) & 1u) {
                        const float2 t = tcp::cmulf(ee[e], qm[e]);
                        const float f = pow2f(qe[e] + ax[e]);
                        w = make_float2(t.x * f, t.y * f);
                    } else {
                        const float2 t = tcp::cmulf(w, rq);
                        const float f = pow2f(ax[e] - ax[e > 0 ? e - 1 : 0]);
                        w = make_float2(t.x * f, t.y * f);
                    }
                    g[v] = conj ? make_float2(w.x, -w.y) : w;
                }
            }
            tcp::put_b(st, tcp::brow(), 4 * tcp::bhalf() + u, g[0], g[1]);
        }
    }
    __device__ void epilogue(uint32_t tmem, bool ok) {
        tcp::for_each_acc(tmem, NT, [&](int rp, int col, float v) {
            const int r = rp & 63, comp = rp >> 6;
            const int qq = q0 + col;
            if (r >= nrhs || qq >= NS) return;
            double* dst = reinterpret_cast<double*>(part + (((size_t)split * 2 + b) * NS + qq) * nrhs + r) + comp;
            *dst = ok ? (double)v : 0.0;
        });
    }
};

template <class K>
__global__ void __launch_bounds__(THREADS, 1)
k_m2s_tc(const float2* __restrict__ xs, const float2* __restrict__ E, const float2* __restrict__ Qm,
         const int* __restrict__ Qe, const float2* __restrict__ rho, const int* __restrict__ expo,
         double2* __restrict__ part, int M, int nc, int NS, int NSp, int nrhs, int rows_per_split, int conj,
         int* err) {
    const int b = blockIdx.z, split = blockIdx.y;
    const int i0 = split * rows_per_split, i1 = min(M * nc, i0 + rows_per_split);
    M2SPolicy pol{xs, E + (size_t)b * M * NSp, Qm + (size_t)b * nc * NSp, Qe + (size_t)b * nc * NSp,
                  rho + (size_t)b * NSp, expo, part, M, nc, NS, NSp, nrhs, b, (int)blockIdx.x * NT, i0, i1, split, conj};
    pol.init();
    const int nchunks = i1 > i0 ? (i1 - i0 + KCC - 1) / KCC : 0;
    tcp::run<M2SPolicy, K>(pol, nchunks, NT, err);
}

// ------------------------------------------------------------------ setup-time tables
// E_s2l[b][m][q] = e^{i xi_q x_m + s_b y_m},  E_m2s[b][m][q] = e^{s_b y_m - i xi_q x_m}  (FP64, rounded)
__global__ void k_etab(const double2* __restrict__ centre, const double2* __restrict__ node,
                       const double2* __restrict__ sq, float2* __restrict__ es2l, float2* __restrict__ em2s, int M,
                       int NS, int NSp) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= 2LL * M * NSp) return;
    const int q = (int)(i % NSp);
    const long long bm = i / NSp;
    const int m = (int)(bm % M), b = (int)(bm / M);
    if (q >= NS) {
        es2l[i] = make_float2(0.f, 0.f);
        em2s[i] = make_float2(0.f, 0.f);
        return;
    }
    const double2 c = centre[m], xi = node[q], s = sq[q * 2 + b];
    double re = -xi.y * c.x + s.x * c.y, im = xi.x * c.x + s.y * c.y;
    double mg = exp(re), sn, cs;
    sincos(im, &sn, &cs);
    es2l[i] = make_float2((float)(mg * cs), (float)(mg * sn));
    re = s.x * c.y + xi.y * c.x;
    im = s.y * c.y - xi.x * c.x;
    mg = exp(re);
    sincos(im, &sn, &cs);
    em2s[i] = make_float2((float)(mg * cs), (float)(mg * sn));
}

// amplitudes [2][NS][nrhs] FP64 -> [2][NSp][nrhs] FP32, zero beyond NS
__global__ void k_amp_f(const double2* __restrict__ ud, float2* __restrict__ uf, int NS, int NSp, int nrhs) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= 2LL * NSp * nrhs) return;
    const int r = (int)(i % nrhs);
    const long long bq = i / nrhs;
    const int q = (int)(bq % NSp), b = (int)(bq / NSp);
    uf[i] = q < NS ? make_float2((float)ud[((size_t)b * NS + q) * nrhs + r].x,
                                 (float)ud[((size_t)b * NS + q) * nrhs + r].y)
                   : make_float2(0.f, 0.f);
}

inline int nblk(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

int ms_spectral_tc_setup(ms_handle* h) {
    const int M = h->M, NS = h->NS, nc = h->nc;
    const int NSp = (NS + KCC - 1) / KCC * KCC;
    h->NSp = NSp;
    MsDeviceTables& d = h->d;
    size_t ne = (size_t)2 * M * NSp;
    if (cudaMalloc(&d.es2l, ne * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&d.em2s, ne * sizeof(float2)) != cudaSuccess)
        return MS_ERR_ALLOC;
    k_etab<<<nblk((long long)ne, 256), 256>>>(d.centre, d.node, d.sq, d.es2l, d.em2s, M, NS, NSp);
    if (int rc = ms_check(h, cudaGetLastError())) return rc;
    // node-contiguous copies [b][n][NSp] of the FP32 power tables
    std::vector<float2> hm((size_t)2 * NS * nc), hs((size_t)2 * NS * nc);
    std::vector<int> em((size_t)2 * NS * nc), es((size_t)2 * NS * nc);
    cudaMemcpy(hm.data(), d.qpm_m, hm.size() * sizeof(float2), cudaMemcpyDeviceToHost);
    cudaMemcpy(hs.data(), d.qps_m, hs.size() * sizeof(float2), cudaMemcpyDeviceToHost);
    cudaMemcpy(em.data(), d.qpm_e, em.size() * sizeof(int), cudaMemcpyDeviceToHost);
    if (int rc = ms_check(h, cudaMemcpy(es.data(), d.qps_e, es.size() * sizeof(int), cudaMemcpyDeviceToHost)))
        return rc;
    size_t nt = (size_t)2 * nc * NSp;
    std::vector<float2> tm(nt, make_float2(0.f, 0.f)), ts(nt, make_float2(0.f, 0.f));
    std::vector<int> tme(nt, 0), tse(nt, 0);
    for (int b = 0; b < 2; ++b)
        for (int q = 0; q < NS; ++q)
            for (int n = 0; n < nc; ++n) {
                size_t src = ((size_t)b * NS + q) * nc + n, dst = ((size_t)b * nc + n) * NSp + q;
                tm[dst] = hm[src];
                ts[dst] = hs[src];
                tme[dst] = em[src];
                tse[dst] = es[src];
            }
    // ratios of consecutive powers per (wave, node): -i q (M2S table) and i q (S2L table)
    std::vector<double2> hq((size_t)NS * 2);
    if (int rc = ms_check(h, cudaMemcpy(hq.data(), d.qq, hq.size() * sizeof(double2), cudaMemcpyDeviceToHost)))
        return rc;
    std::vector<float2> rm((size_t)2 * NSp, make_float2(0.f, 0.f)), rs((size_t)2 * NSp, make_float2(0.f, 0.f));
    for (int b = 0; b < 2; ++b)
        for (int q = 0; q < NS; ++q) {
            const double2 v = hq[(size_t)q * 2 + b];
            rm[(size_t)b * NSp + q] = make_float2((float)v.y, (float)-v.x);
            rs[(size_t)b * NSp + q] = make_float2((float)-v.y, (float)v.x);
        }
    if (cudaMalloc(&d.rho_m2s, rm.size() * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&d.rho_s2l, rs.size() * sizeof(float2)) != cudaSuccess)
        return MS_ERR_ALLOC;
    cudaMemcpy(d.rho_m2s, rm.data(), rm.size() * sizeof(float2), cudaMemcpyHostToDevice);
    cudaMemcpy(d.rho_s2l, rs.data(), rs.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (cudaMalloc(&d.qpmT_m, nt * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&d.qpsT_m, nt * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&d.qpmT_e, nt * sizeof(int)) != cudaSuccess || cudaMalloc(&d.qpsT_e, nt * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&d.tc_err, 2 * sizeof(int)) != cudaSuccess)
        return MS_ERR_ALLOC;
    cudaMemcpy(d.qpmT_m, tm.data(), nt * sizeof(float2), cudaMemcpyHostToDevice);
    cudaMemcpy(d.qpsT_m, ts.data(), nt * sizeof(float2), cudaMemcpyHostToDevice);
    cudaMemcpy(d.qpmT_e, tme.data(), nt * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(d.qpsT_e, tse.data(), nt * sizeof(int), cudaMemcpyHostToDevice);
    // tc_err[0]: the timeout flag; tc_err[1]: the test hook's wait in microseconds (ms_options.tc_wait_test)
    const int flags[2] = {0, h->opt.tc_wait_test};
    cudaMemcpy(d.tc_err, flags, sizeof(flags), cudaMemcpyHostToDevice);
    cudaFuncSetAttribute(k_m2s_tc<tcp::TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    cudaFuncSetAttribute(k_m2s_tc<tcp::BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM);
    ms_near_tc_attributes();
    return ms_check(h, cudaDeviceSynchronize());
}

void ms_spectral_tc_free(ms_handle* h) {
    MsDeviceTables& d = h->d;
    cudaFree(d.es2l);
    cudaFree(d.em2s);
    cudaFree(d.qpmT_m);
    cudaFree(d.qpsT_m);
    cudaFree(d.qpmT_e);
    cudaFree(d.qpsT_e);
    cudaFree(d.tc_err);
    cudaFree(d.rho_m2s);
    cudaFree(d.rho_s2l);
    d.rho_m2s = d.rho_s2l = nullptr;
    d.es2l = d.em2s = d.qpmT_m = d.qpsT_m = nullptr;
    d.qpmT_e = d.qpsT_e = d.tc_err = nullptr;
}

// M2S (adj = 0) or C^H (adj = 1) of the FP32 scaled block into the chunk partials; *nchunks = splits.
int ms_m2s_tc_launch(ms_handle* h, const float2* xs, int nrhs, int adj, int* nchunks, cudaStream_t st) {
    const int M = h->M, nc = h->nc, NS = h->NS, NSp = h->NSp;
    const int rows = M * nc;
    const int ntile = (NS + NT - 1) / NT;
    const int rows_per = h->m2s_rows > 0 ? h->m2s_rows : 2048;          // ms_autotune may change it
    int nsplit = std::max(1, std::min(64, (rows + rows_per - 1) / rows_per));
    int per = (rows + nsplit - 1) / nsplit;
    per = (per + KCC - 1) / KCC * KCC;
    nsplit = (rows + per - 1) / per;
    *nchunks = nsplit;
    const MsDeviceTables& d = h->d;
    auto kern = h->tc_kind ? k_m2s_tc<tcp::BF16> : k_m2s_tc<tcp::TF32>;
    kern<<<dim3(ntile, nsplit, 2), THREADS, SMEM, st>>>(xs, adj ? d.es2l : d.em2s, adj ? d.qpsT_m : d.qpmT_m,
                                                        adj ? d.qpsT_e : d.qpmT_e, adj ? d.rho_s2l : d.rho_m2s,
                                                        d.expo, (double2*)h->ws_part, M, nc, NS, NSp, nrhs, per,
                                                        adj, d.tc_err);
    return ms_check(h, cudaGetLastError());
}

// S2L (adj = 0) or B^H (adj = 1) of the amplitudes ud[2][NS][nrhs] into the FP32 block out.
int ms_s2l_tc_launch(ms_handle* h, const double2* ud, float2* out, int nrhs, int adj, int accumulate,
                     cudaStream_t st) {
    const int M = h->M, nc = h->nc, NS = h->NS, NSp = h->NSp;
    const MsDeviceTables& d = h->d;
    float2* uf = (float2*)h->ws_uf;
    k_amp_f<<<nblk(2LL * NSp * nrhs, 256), 256, 0, st>>>(ud, uf, NS, NSp, nrhs);
    if (int rc = ms_check(h, cudaGetLastError())) return rc;
    const int ntile = (M * nc + NT - 1) / NT;
    const size_t smem = SMEM + 2 * ((s2l_raw_bytes(nc) + 15) / 16 * 16);
    auto kern = h->tc_kind ? k_s2l_tc<tcp::BF16> : k_s2l_tc<tcp::TF32>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<dim3(ntile, 2), THREADS, smem, st>>>(uf, adj ? d.em2s : d.es2l, adj ? d.qpmT_m : d.qpsT_m,
                                                adj ? d.qpmT_e : d.qpsT_e, d.expo, out, M, nc, NSp, nrhs,
                                                accumulate, adj, d.tc_err);
    return ms_check(h, cudaGetLastError());
}

// The staged Sommerfeld-to-local kernel fits in shared memory for p >= 1 (two raw buffers of E, Q rows).
bool ms_s2l_tc_ok(const ms_handle* h) {
    const int nitems = s2l_parts_per_tile(h->nc) * 8 + h->nc * 12;     // staged 16-byte items per chunk
    return h->p >= 1 && nitems <= 2 * THREADS && SMEM + 2 * ((s2l_raw_bytes(h->nc) + 15) / 16 * 16) <= 227 * 1024;
}

// Reads and clears the tensor-core kernels' timeout flag (MS_ERR_TIMEOUT if a wait gave up).
int ms_spectral_tc_status(ms_handle* h, cudaStream_t st) {
    int v = 0;
    if (int rc = ms_check(h, cudaMemcpyAsync(&v, h->d.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st))) return rc;
    if (int rc = ms_check(h, cudaStreamSynchronize(st))) return rc;
    if (v) {
        cudaMemsetAsync(h->d.tc_err, 0, sizeof(int), st);
        return MS_ERR_TIMEOUT;
    }
    return MS_OK;
}
