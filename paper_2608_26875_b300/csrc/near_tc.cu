// Near-field Graf sum of the FP32 operator on the tensor cores (row a2, Sec. 4.2):
//   a~^m_{b,i,r} = sum_{l in N(m), l != m} sum_j h^{ml}_{j-i} 2^{a(m,b,i) + a(l,b,j)} x~^l_{b,j,r},
// h^{ml}_k = H_k(kappa_b |x_m - x_l|) e^{ik arg(x_m - x_l)} (DLMF 10.23.7), read from the per-pair
// sequences built at setup (FP32 mantissa and binary exponent).
//
// Targets of one leaf share their sources (the particles of the 3 x 3 leaves around it), so a tile of
// up to 256 / nc targets of a leaf is one dense contraction: output rows (m, i), contracted index
// (s, j) over the leaf's source list, with the self block set to zero.  The coefficients form the
// 128-row A operand, the Toeplitz blocks h_{j-i} of every (target, source) pair the B operand; see
// tc_pipeline.cuh.
#include <algorithm>

#include "common.cuh"
#include "handle.h"
#include "tc_pipeline.cuh"

namespace {

using tcp::KCC;
using tcp::Stage;

struct NearPolicy {
    const float2* xs;          // [M][2][nc][nrhs] scaled coefficients
    const float2* seqm;        // sequence mantissas
    const int* seqe;           // sequence exponents
    const long long* tseq;     // [near tasks] sequence offset of each (target, source) task
    const int* nptr;           // [M + 1] near tasks of each target
    const int* tgt;            // this tile's targets
    const int* self;           // their positions in the source list
    const int* src;            // this tile's source list
    const int* expo;           // [M][2][nc]
    float2* out;               // [M][2][nc][nrhs]
    int nc, nrhs, b, ntgt, nsrc, K;
    int i, a_mi, ptr_m, self_m;
    bool valid;

    __device__ void init() {
        const int row = threadIdx.x;
        const int tt = row / nc;
        i = row - tt * nc;
        valid = tt < ntgt;
        a_mi = ptr_m = 0;
        self_m = -1;
        if (valid) {
            const int m = tgt[tt];
            a_mi = expo[((size_t)m * 2 + b) * nc + i];
            ptr_m = nptr[m];
            self_m = self[tt];
        }
    }
    __device__ void load_a(const Stage& st, int c) {
        const int rp = threadIdx.x & 127, h = threadIdx.x >> 7, r = rp & 63;
        const bool ok = r < nrhs;
        const int f0 = c * KCC + h * 8;
        int s = f0 / nc, j = f0 - s * nc;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float2 y[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                y[v] = make_float2(0.f, 0.f);
                if (ok && s < nsrc) y[v] = xs[(((size_t)src[s] * 2 + b) * nc + j) * nrhs + r];
                if (++j == nc) { j = 0; ++s; }
            }
            tcp::put_a(st, rp, h * 4 + u, y[0], y[1]);
        }
    }
    __device__ void gen_b(const Stage& st, int c) {
        const int f0 = c * KCC;
        int s = f0 / nc, j = f0 - s * nc;
        int cs = -1, l = 0;
        long long off = 0;
#pragma unroll
        for (int kk = 0; kk < tcp::KC / 4; ++kk) {
            float2 z[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                z[v] = make_float2(0.f, 0.f);
                if (valid && s < nsrc && s != self_m) {
                    if (s != cs) {
                        cs = s;
                        l = src[s];
                        off = tseq[ptr_m + s - (s > self_m ? 1 : 0)];
                    }
                    const long long idx = off + K + (j - i);
                    const float2 mv = seqm[idx];
                    const float f = pow2f(seqe[idx] + a_mi + expo[((size_t)l * 2 + b) * nc + j]);
                    z[v] = make_float2(mv.x * f, mv.y * f);
                }
                if (++j == nc) { j = 0; ++s; }
            }
            tcp::put_b(st, threadIdx.x, kk, z[0], z[1]);
        }
    }
    __device__ void epilogue(uint32_t tmem, bool ok) {
        if (!ok) return;
        const int n = ((ntgt * nc + 15) / 16) * 16;
        tcp::for_each_acc(tmem, n, [&](int rp, int col, float v) {
            const int r = rp & 63, comp = rp >> 6;
            if (r >= nrhs) return;
            const int tt = col / nc;
            if (tt >= ntgt) return;
            const int i2 = col - tt * nc, m2 = tgt[tt];
            reinterpret_cast<float*>(out + (((size_t)m2 * 2 + b) * nc + i2) * nrhs + r)[comp] = v;
        });
    }
};

__global__ void __launch_bounds__(tcp::THREADS, 1)
k_near_tc(const float2* __restrict__ xs, const float2* __restrict__ seqm, const int* __restrict__ seqe,
          const long long* __restrict__ tseq0, const long long* __restrict__ tseq1, const int* __restrict__ nptr,
          const int4* __restrict__ tiles, const int* __restrict__ ttgt, const int* __restrict__ tself,
          const int* __restrict__ tsrc, const int* __restrict__ expo, float2* __restrict__ out, int nc, int nrhs,
          int K, int* err) {
    const int b = blockIdx.y;
    const int4 t = tiles[blockIdx.x];
    NearPolicy pol{xs, seqm, seqe, b ? tseq1 : tseq0, nptr, ttgt + t.x, tself + t.x, tsrc + t.z, expo, out,
                   nc, nrhs, b, t.y, t.w, K};
    pol.init();
    const int n = ((t.y * nc + 15) / 16) * 16;
    const int nchunks = (t.w * nc + KCC - 1) / KCC;
    tcp::run(pol, nchunks, n, err);
}

}  // namespace

// a~ = near-pair Graf sum of the FP32 scaled block xs into dst (written, both waves).
int ms_near_tc_launch(ms_handle* h, const float2* xs, float2* dst, int nrhs, cudaStream_t st) {
    const FmmHost& F = h->fmm;
    cudaFuncSetAttribute(k_near_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcp::SMEM);
    k_near_tc<<<dim3(F.ntile, 2), tcp::THREADS, tcp::SMEM, st>>>(
        xs, h->d.seqm, h->d.seqe, F.near[0].seq, F.near[1].seq, F.near[0].ptr, F.tile, F.ttgt, F.tself, F.tsrc,
        h->d.expo, dst, h->nc, nrhs, 2 * h->p + 1, h->d.tc_err);
    return ms_check(h, cudaGetLastError());
}
