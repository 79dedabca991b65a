// A tcgen05 pipeline for complex contractions across a block of right-hand sides, shared by the
// spectral maps and the near-field Graf sum.
//
// C = A B^T on the tensor cores (kind::tf32, FP32 accumulation in tensor memory), 3xTF32:
// A B ~ Ah Bh + Ah Bl + Al Bh with X = Xh + Xl, Xh exactly representable in tf32.
// With k = 2 kappa + t running over the contracted complex index kappa,
//   A[r][2k]    = Re Y(kappa, r),  A[r][2k+1]    = -Im Y(kappa, r),   r < 64
//   A[64+r][2k] = Im Y(kappa, r),  A[64+r][2k+1] =  Re Y(kappa, r)
//   B[j][2k]    = Re Z(j, kappa),  B[j][2k+1]    =  Im Z(j, kappa)
// gives C[r][j] = Re sum_kappa Z(j, kappa) Y(kappa, r) and C[64+r][j] = Im of the same.
// A (the data, M = 128 rows = 2 x 64 columns) and B (the generated operator, N <= 256 rows) are
// written into shared memory by the CTA's 512 threads one K chunk (16 complex) at a time, in a
// two-stage pipeline; one thread issues the MMAs and commits them to the stage's mbarrier, which the
// threads wait on (time-bounded) before reusing the stage.
#pragma once
#include "tc.cuh"

namespace tcp {

constexpr int KC = 32;                         // real K per chunk (16 complex)
constexpr int KCC = KC / 2;
constexpr int NMAX = 256;                      // MMA N: generated-operator rows per tile (max)
constexpr int MA = 128;                        // MMA M: 2 x 64 right-hand-side columns
constexpr int THREADS = 512;                   // 16 warps: two per B row, four per A row
constexpr int NSTAGE = 2;
constexpr uint32_t A_TILE = MA * KC * 4;       // 16 KB (hi or lo)
constexpr uint32_t B_TILE = NMAX * KC * 4;     // 32 KB
constexpr uint32_t STAGE = 2 * A_TILE + 2 * B_TILE;
constexpr size_t SMEM = (size_t)NSTAGE * STAGE + 64;   // + stage barriers, tensor-memory slot, flag, probe,
                                                         //   copy barriers and the last-commit index
constexpr uint32_t LBO = 128, SBO = (KC / 4) * 128;
constexpr uint32_t TMEM_COLS = 256;
static_assert(SMEM <= 227 * 1024, "shared memory");

// Shared memory after the stages, the two mbarriers and the tensor-memory slot: raw buffers of
// policies that stage chunk data (16-byte aligned).
__device__ __forceinline__ unsigned char* raw_base() {
    extern __shared__ __align__(1024) unsigned char smem[];
    return smem + (size_t)NSTAGE * (2 * MA * KC * 4 + 2 * NMAX * KC * 4) + 64;
}

// Operand kinds.  TF32: 32-bit tf32 hi/lo tiles, kind::tf32 (K = 8 per MMA).  BF16: 16-bit bf16 hi/lo
// tiles, kind::f16 with bf16 inputs (K = 16 per MMA), half the tile bytes; the BF16-split variant.
// Both keep the TF32 stage stride, so that the shared-memory map (barriers, raw buffers) is one.
struct TF32 {
    static constexpr int ELEM = 4;
    static constexpr int KMMA = 8;
    static constexpr uint32_t SBO_ = (KC / 4) * 128;     // 8-row groups: K / 4 core matrices apart
    __device__ static uint32_t idesc(int M, int N) { return tc::idesc_tf32(M, N); }
    __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
        tc::mma_tf32(d, a, b, id, acc);
    }
};
struct BF16 {
    static constexpr int ELEM = 2;
    static constexpr int KMMA = 16;
    static constexpr uint32_t SBO_ = (KC / 8) * 128;
    __device__ static uint32_t idesc(int M, int N) { return tc::idesc_bf16(M, N); }
    __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
        tc::mma_bf16(d, a, b, id, acc);
    }
};

template <class K>
struct StageT {
    K* kind_tag;           // (type carrier only)
    unsigned char *ah, *al, *bh, *bl;
};
typedef StageT<TF32> Stage;

template <class K>
__device__ __forceinline__ StageT<K> stage_ptrs(unsigned char* base, int s) {
    unsigned char* p = base + (size_t)s * STAGE;
    const size_t at = (size_t)MA * KC * K::ELEM, bt = (size_t)NMAX * KC * K::ELEM;
    return {nullptr, p, p + at, p + 2 * at, p + 2 * at + bt};
}

__device__ __forceinline__ void put4(float* hi, float* lo, int off, float a, float b, float c, float d) {
    float4 h, l;
    tc::split(a, h.x, l.x);
    tc::split(b, h.y, l.y);
    tc::split(c, h.z, l.z);
    tc::split(d, h.w, l.w);
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
}

// four consecutive K values of one row as bf16 hi and lo (8 bytes each)
__device__ __forceinline__ void put4_bf16(unsigned char* hi, unsigned char* lo, int off, float a, float b, float c,
                                          float d) {
    uint2 h, l;
    tc::split_bf16(a, b, h.x, l.x);
    tc::split_bf16(c, d, h.y, l.y);
    *reinterpret_cast<uint2*>(hi + 2 * off) = h;
    *reinterpret_cast<uint2*>(lo + 2 * off) = l;
}

// A row rp (= r or 64 + r) of k-group kk from two consecutive complex values y0, y1 of column r
__device__ __forceinline__ void put_a(const StageT<TF32>& st, int rp, int kk, float2 y0, float2 y1) {
    const int off = tc::kmajor_off(rp, 4 * kk, KC);
    float* ah = reinterpret_cast<float*>(st.ah);
    float* al = reinterpret_cast<float*>(st.al);
    if (rp < 64)
        put4(ah, al, off, y0.x, -y0.y, y1.x, -y1.y);
    else
        put4(ah, al, off, y0.y, y0.x, y1.y, y1.x);
}
__device__ __forceinline__ void put_a(const StageT<BF16>& st, int rp, int kk, float2 y0, float2 y1) {
    const int off = tc::kmajor_off16(rp, 4 * kk, KC);
    if (rp < 64)
        put4_bf16(st.ah, st.al, off, y0.x, -y0.y, y1.x, -y1.y);
    else
        put4_bf16(st.ah, st.al, off, y0.y, y0.x, y1.y, y1.x);
}
// B row j of k-group kk from two consecutive complex operator entries
__device__ __forceinline__ void put_b(const StageT<TF32>& st, int j, int kk, float2 z0, float2 z1) {
    put4(reinterpret_cast<float*>(st.bh), reinterpret_cast<float*>(st.bl), tc::kmajor_off(j, 4 * kk, KC), z0.x,
         z0.y, z1.x, z1.y);
}
__device__ __forceinline__ void put_b(const StageT<BF16>& st, int j, int kk, float2 z0, float2 z1) {
    put4_bf16(st.bh, st.bl, tc::kmajor_off16(j, 4 * kk, KC), z0.x, z0.y, z1.x, z1.y);
}

// Thread roles in building a chunk: B row brow() (one of 256) and its half bhalf() of the 16
// complex K entries (k-groups 4 bhalf() .. 4 bhalf() + 3); A row arow() (one of 128) and its
// quarter aq() of the entries (k-groups 2 aq(), 2 aq() + 1).
__device__ __forceinline__ int brow() { return threadIdx.x & 255; }
__device__ __forceinline__ int bhalf() { return threadIdx.x >> 8; }
__device__ __forceinline__ int arow() { return threadIdx.x & 127; }
__device__ __forceinline__ int aq() { return threadIdx.x >> 7; }

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// P provides fetch(chunk) (issue the global loads of one K chunk into registers), build(Stage)
// (write the A and B tiles of the fetched chunk) and epilogue(tmem, ok); n is the MMA N of this
// tile (a multiple of 16 in [16, 256]).  The loads of chunk c + 1 are issued right after chunk c is
// built, so their latency overlaps the MMAs in flight.  A policy with kStaged = true also has
// stage(chunk): it stores the cooperatively fetched data of the chunk into a shared-memory raw
// buffer (two, alternating) that build() then reads after a barrier.  Sets *err on a timed-out wait.
template <class P, class K = TF32>
__device__ __forceinline__ void run(P& pol, int nchunks, int n, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)NSTAGE * STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + NSTAGE);
    int* fail = reinterpret_cast<int*>(tslot + 1);
    uint64_t* probe = bar + NSTAGE + 1;            // test hook: a barrier that nothing arrives at
    const int tid = threadIdx.x;
    const uint32_t idesc = K::idesc(MA, n);
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) tc::mbar_init(&bar[s], 1);
        tc::mbar_init(probe, 1);
        tc::mbar_fence_init();
        *fail = 0;
        // err[1] > 0 (ms_options.tc_wait_test): wait that many microseconds for a phase that never
        // completes, give up, and leave the CTA on its failure path before any multiply is issued
        const int test_us = err[1];
        if (test_us > 0 && !tc::mbar_wait(probe, 0, (uint64_t)test_us * 1000ull)) *fail = 1;
    }
    if (tid < 32) tc::tmem_alloc(tslot, TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    int issued = 0;
    if (nchunks > 0) pol.fetch(0);
    for (int c = 0; c < nchunks; ++c) {
        const int s = c % NSTAGE;
        if (c >= NSTAGE && !tc::mbar_wait(&bar[s], ((c / NSTAGE) - 1) & 1)) *fail = 1;
        const StageT<K> st = stage_ptrs<K>(smem, s);
        if constexpr (P::kStaged) {
            pol.stage(c);
            __syncthreads();
        }
        pol.build(st);
        if (c + 1 < nchunks) pol.fetch(c + 1);
        tc::fence_proxy_async();
        __syncthreads();
        if (*fail) break;
        if (tid == 0) {
            tc::fence_after();
#pragma unroll
            for (int pass = 0; pass < 3; ++pass) {
                const uint32_t a0 = tc::smem_u32(pass == 2 ? st.al : st.ah);
                const uint32_t b0 = tc::smem_u32(pass == 1 ? st.bl : st.bh);
                // one MMA covers K::KMMA values = two core matrices (256 bytes) along K
#pragma unroll
                for (int ks = 0; ks < KC / K::KMMA; ++ks)
                    K::mma(tmem, tc::smem_desc(a0 + ks * 256, LBO, K::SBO_), tc::smem_desc(b0 + ks * 256, LBO, K::SBO_),
                           idesc, (c > 0 || pass > 0 || ks > 0) ? 1u : 0u);
            }
            tc::mma_commit(&bar[s]);
        }
        issued = c + 1;
    }
    // the last commit covers every MMA issued before it
    bool ok = !*fail && issued == nchunks;
    if (issued > 0) {
        const int c = issued - 1;
        if (!tc::mbar_wait(&bar[c % NSTAGE], (c / NSTAGE) & 1)) ok = false;
    }
    tc::fence_after();
    if (!ok && tid == 0) atomicExch(err, 1);
    pol.epilogue(tmem, ok && nchunks > 0);
    tc::fence_before();
    __syncthreads();
    if (tid < 32) tc::tmem_free(tmem, TMEM_COLS);
}

// As run(), for an operator stored in global memory in the stage layout: chunk c's B tiles (hi, then
// lo, half_bytes each; rows 0..n-1 of the 256-row tile, 8-row groups SBO apart) are at
// bsrc + c * 2 * half_bytes.  Thread 0 issues two bulk asynchronous copies per chunk into the stage as
// soon as the multiplies that last read it have completed; they complete on the stage's copy barrier,
// which thread 0 waits on (bounded) before it issues the chunk's multiplies.  The policy's build_a()
// writes only the A tiles.  Every wait is bounded; a CTA that gave up waits, bounded, for its issued
// copies and multiplies before it frees tensor memory.
template <class P, class K = TF32>
__device__ __forceinline__ void run_stored(P& pol, int nchunks, int n, int* err, const unsigned char* bsrc,
                                           uint32_t half_bytes) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + (size_t)NSTAGE * STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + NSTAGE);
    int* fail = reinterpret_cast<int*>(tslot + 1);
    uint64_t* probe = bar + NSTAGE + 1;
    uint64_t* cbar = bar + NSTAGE + 2;             // [NSTAGE] copy barriers
    int* last = reinterpret_cast<int*>(cbar + NSTAGE);   // last committed chunk (thread 0 writes)
    const int tid = threadIdx.x;
    const uint32_t idesc = K::idesc(MA, n);
    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            tc::mbar_init(&bar[s], 1);
            tc::mbar_init(&cbar[s], 1);
        }
        tc::mbar_init(probe, 1);
        tc::mbar_fence_init();
        *fail = 0;
        *last = -1;
        const int test_us = err[1];
        if (test_us > 0 && !tc::mbar_wait(probe, 0, (uint64_t)test_us * 1000ull)) *fail = 1;
    }
    if (tid < 32) tc::tmem_alloc(tslot, TMEM_COLS);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    int copied = -1;                               // thread 0: last chunk whose copies were issued
    int waited = -1;                               // thread 0: last chunk whose copies were waited for
    // thread 0 issues the hi and lo copies of chunk c into stage c % NSTAGE
    auto issue_copy = [&](int c) {
        const StageT<K> st = stage_ptrs<K>(smem, c % NSTAGE);
        const unsigned char* src = bsrc + (size_t)c * 2 * half_bytes;
        tc::mbar_expect_tx(&cbar[c % NSTAGE], 2 * half_bytes);
        tc::bulk_g2s(st.bh, src, half_bytes, &cbar[c % NSTAGE]);
        tc::bulk_g2s(st.bl, src + half_bytes, half_bytes, &cbar[c % NSTAGE]);
        copied = c;
    };
    if (nchunks > 0) pol.fetch(0);
    if (tid == 0 && nchunks > 0 && !*fail) issue_copy(0);
    for (int c = 0; c < nchunks; ++c) {
        const int s = c % NSTAGE;
        if (c >= NSTAGE && !tc::mbar_wait(&bar[s], ((c / NSTAGE) - 1) & 1)) *fail = 1;
        const StageT<K> st = stage_ptrs<K>(smem, s);
        pol.build_a(st);
        if (c + 1 < nchunks) pol.fetch(c + 1);
        tc::fence_proxy_async();
        __syncthreads();
        if (*fail) break;
        if (tid == 0) {
            if (!tc::mbar_wait(&cbar[s], (c / NSTAGE) & 1)) {
                *fail = 1;
            } else {
                waited = c;
                tc::fence_after();
#pragma unroll
                for (int pass = 0; pass < 3; ++pass) {
                    const uint32_t a0 = tc::smem_u32(pass == 2 ? st.al : st.ah);
                    const uint32_t b0 = tc::smem_u32(pass == 1 ? st.bl : st.bh);
#pragma unroll
                    for (int ks = 0; ks < KC / K::KMMA; ++ks)
                        K::mma(tmem, tc::smem_desc(a0 + ks * 256, LBO, K::SBO_),
                               tc::smem_desc(b0 + ks * 256, LBO, K::SBO_), idesc, (c > 0 || pass > 0 || ks > 0) ? 1u : 0u);
                }
                tc::mma_commit(&bar[s]);
                *last = c;
                // the next chunk's copies go out now, overlapping this chunk's multiplies; its stage is free
                // once the multiplies of chunk c + 1 - NSTAGE have completed
                const int cn = c + 1;
                if (cn < nchunks) {
                    if (cn >= NSTAGE && !tc::mbar_wait(&bar[cn % NSTAGE], ((cn / NSTAGE) - 1) & 1))
                        *fail = 1;
                    else
                        issue_copy(cn);
                }
            }
        }
    }
    if (tid == 0 && copied > waited) {             // copies issued but never waited for (failure path)
        if (!tc::mbar_wait(&cbar[copied % NSTAGE], (copied / NSTAGE) & 1)) *fail = 1;
    }
    __syncthreads();
    bool ok = !*fail && *last == nchunks - 1;
    if (*last >= 0) {
        const int c = *last;
        if (!tc::mbar_wait(&bar[c % NSTAGE], (c / NSTAGE) & 1)) ok = false;
    }
    tc::fence_after();
    if (!ok && tid == 0) atomicExch(err, 1);
    pol.epilogue(tmem, ok && nchunks > 0);
    tc::fence_before();
    __syncthreads();
    if (tid < 32) tc::tmem_free(tmem, TMEM_COLS);
}

// Epilogue helper: warp w reads accumulator rows 32 (w & 3) + lane (the A rows rp) and the 64
// columns of its block w >> 2; f(rp, col, value) is called for every column < n.
template <class F>
__device__ __forceinline__ void for_each_acc(uint32_t tmem, int n, F&& f) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = w & 3, blk = w >> 2;
    const int rp = 32 * quarter + lane;
#pragma unroll 1
    for (int cb = 0; cb < 4; ++cb) {
        const int col0 = 64 * blk + 16 * cb;
        if (col0 >= n) break;                          // uniform per warp
        float v[16];
        tc::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)col0, v);
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (col0 + i < n) f(rp, col0 + i, v[i]);
    }
}

}  // namespace tcp
