// Toeplitz translation lists of the FP32 operator on the tensor cores: the near-field Graf sum
// (row a2, Sec. 4.2) and the FMM's multipole-to-local stage (row a3).  Both have the form
//   out^d_{i,r} = sum_{e in list(d)} sum_j h^{de}_{(j - Ps) - (i - Pd)} 2^{a_d(i) + a_e(j)} in^e_{j,r},
// with h^{de}_k = Z_k(kappa |v|) e^{ik arg v}, v = c_d - c_e (DLMF 10.23.7), read from the per-task
// sequences built at setup (FP32 mantissa and binary exponent, entries k in [-K, K]).
//
// A tile is up to 256 output rows: several targets sharing one source list (the particles of one
// leaf against the 3 x 3 leaves around it; the self block is zero), or a row range of one box (M2L:
// 2P + 1 rows against its interaction list).  Each tile is one dense contraction over (source,
// order): the input expansions form the 128-row A operand and the Toeplitz blocks the B operand
// (tc_pipeline.cuh).  Task of target d and source slot s: tptr[d] + s, minus one past the target's
// own slot self(d) when it has one (near lists; self(d) = -1 for M2L).
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "handle.h"
#include "tc_pipeline.cuh"

namespace {

using tcp::KCC;
using tcp::Stage;

struct ListArgs {
    const float2* in;            // source entity e, order j: in + e * in_stride + j * nrhs
    long long in_stride;
    float2* out;                 // target entity d, order i: out + d * out_stride + i * nrhs
    long long out_stride;
    const float2* seqm;
    const int* seqe;
    const long long* tseq;       // per task: sequence offset (used when seq_len == 0)
    long long seq_base;          // seq_len > 0: task t's sequence starts at seq_base + t * seq_len
    int seq_len;
    const int* tptr;             // per target entity: first task
    const int* ad;               // target exponents ad[d * ad_stride + i]
    long long ad_stride;
    const int* as;               // source exponents as[e * as_stride + j]
    long long as_stride;
    const int4* tiles;           // {target offset, targets, source offset, sources}
    const int* ttgt;             // target entities of the tiles
    const int* tself;            // position of each target in its source list (-1: none)
    const int* tsrc;             // source entities, indexed by the tile's source offset
    const int* trow;             // per tile: first output order (NULL: 0)
    int Pd, Ps, K, nrhs;
};

constexpr int MAX_TABLE = 64;    // task offsets staged per single-target tile (M2L lists <= 27)

struct ListPolicy {
    static constexpr bool kStaged = false;
    const ListArgs& a;
    const int* tgt;
    const int* self;
    const int* src;
    const long long* toff;       // staged task offsets of a single-target tile, or NULL
    int ntgt, nsrc, nrow, i0, nd, ns;
    int i, ad_i, ptr_t, self_t, kbase;
    bool valid;
    // one fetched chunk (this thread's share)
    float2 ya[4];
    float2 mv[8];
    int ex[8];
    unsigned vmask;

    __device__ void init() {
        const int row = tcp::brow();
        const int tt = row / nrow;
        i = i0 + (row - tt * nrow);
        valid = tt < ntgt && i < nd;
        ad_i = ptr_t = 0;
        self_t = -1;
        if (valid) {
            const int d = tgt[tt];
            ad_i = a.ad[(long long)d * a.ad_stride + i];
            ptr_t = a.tptr[d];
            self_t = self[tt];
        }
        kbase = a.K - a.Ps - (i - a.Pd);         // sequence index = task offset + kbase + j
    }
    __device__ long long task_off(int s) const {
        const int t = ptr_t + s - ((self_t >= 0 && s > self_t) ? 1 : 0);
        if (a.seq_len > 0) return a.seq_base + (long long)t * a.seq_len;
        return toff ? toff[s] : a.tseq[t];
    }
    bool load_b = true;          // false: the B tiles come from a stored copy (run_stored)
    __device__ void fetch(int c) {
        const int r = tcp::arow() & 63;
        const bool ok = r < a.nrhs && a.in != nullptr;
        const int fa = c * KCC + 4 * tcp::aq();
        int s = fa / ns, j = fa - s * ns;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            ya[v] = (ok && s < nsrc) ? a.in[(long long)src[s] * a.in_stride + (long long)j * a.nrhs + r]
                                     : make_float2(0.f, 0.f);
            if (++j == ns) { j = 0; ++s; }
        }
        if (!load_b) return;
        const int f0 = c * KCC + 8 * tcp::bhalf();
        s = f0 / ns;
        j = f0 - s * ns;
        vmask = 0;
        int cs = -1, e = 0;
        long long off = 0;
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            if (valid && s < nsrc && s != self_t) {
                if (s != cs) {
                    cs = s;
                    e = src[s];
                    off = task_off(s);
                }
                const long long idx = off + kbase + j;
                vmask |= 1u << v;
                mv[v] = a.seqm[idx];
                ex[v] = a.seqe[idx] + a.as[(long long)e * a.as_stride + j];
            }
            if (++j == ns) { j = 0; ++s; }
        }
    }
    template <class St>
    __device__ void build_a(const St& st) {
#pragma unroll
        for (int u = 0; u < 2; ++u) tcp::put_a(st, tcp::arow(), 2 * tcp::aq() + u, ya[2 * u], ya[2 * u + 1]);
    }
    template <class St>
    __device__ void build(const St& st) {
        build_a(st);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float2 z[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int q = 2 * u + v;
                z[v] = make_float2(0.f, 0.f);
                if ((vmask >> q) & 1u) {
                    const float f = pow2f(ex[q] + ad_i);
                    z[v] = make_float2(mv[q].x * f, mv[q].y * f);
                }
            }
            tcp::put_b(st, tcp::brow(), 4 * tcp::bhalf() + u, z[0], z[1]);
        }
    }
    __device__ void epilogue(uint32_t tmem, bool ok) {
        const int n = ((ntgt * nrow + 15) / 16) * 16;
        if (!ok) return;
        tcp::for_each_acc(tmem, n, [&](int rp, int col, float v) {
            const int r = rp & 63, comp = rp >> 6;
            if (r >= a.nrhs) return;
            const int tt = col / nrow;
            const int i2 = i0 + (col - tt * nrow);
            if (tt >= ntgt || i2 >= nd) return;
            reinterpret_cast<float*>(a.out + (long long)tgt[tt] * a.out_stride + (long long)i2 * a.nrhs + r)[comp] = v;
        });
    }
};

template <class K>
__global__ void __launch_bounds__(tcp::THREADS, 1) k_list_tc(ListArgs a, int* err) {
    __shared__ long long toff[MAX_TABLE];
    const int4 t = a.tiles[blockIdx.x];
    const int nd = 2 * a.Pd + 1, ns = 2 * a.Ps + 1;
    const int i0 = a.trow ? a.trow[blockIdx.x] : 0;
    const int nrow = t.y == 1 ? min(tcp::NMAX, nd - i0) : nd;
    // single-target lists with looked-up offsets: stage the task offsets once per tile
    const bool staged = a.seq_len == 0 && t.y == 1 && t.w <= MAX_TABLE;
    if (staged) {
        const int p0 = a.tptr[a.ttgt[t.x]];
        for (int s = threadIdx.x; s < t.w; s += blockDim.x) toff[s] = a.tseq[p0 + s];
        __syncthreads();
    }
    ListPolicy pol{a, a.ttgt + t.x, a.tself + t.x, a.tsrc + t.z, staged ? toff : nullptr, t.y, t.w, nrow, i0, nd, ns};
    pol.init();
    const int n = ((t.y * nrow + 15) / 16) * 16;
    const int nchunks = (t.w * ns + KCC - 1) / KCC;
    tcp::run<ListPolicy, K>(pol, nchunks, n, err);
}

// Stored operator of the near tiles: one CTA per tile generates every chunk's B tiles exactly as
// k_list_tc builds them (same policy, same split) and writes rows 0..n-1 of the hi and lo tiles to
// out + off[tile] + chunk * 2 * half, half = n * KC * ELEM bytes.
template <class K>
__global__ void __launch_bounds__(tcp::THREADS, 1) k_list_store(ListArgs a, unsigned char* out,
                                                                const long long* off) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int4 t = a.tiles[blockIdx.x];
    const int nd = 2 * a.Pd + 1, ns = 2 * a.Ps + 1;
    const int nrow = nd;
    ListPolicy pol{a, a.ttgt + t.x, a.tself + t.x, a.tsrc + t.z, nullptr, t.y, t.w, nrow, 0, nd, ns};
    pol.init();
    const int n = ((t.y * nrow + 15) / 16) * 16;
    const size_t half = (size_t)n * tcp::KC * K::ELEM;
    const int nchunks = (t.w * ns + KCC - 1) / KCC;
    const tcp::StageT<K> st = tcp::stage_ptrs<K>(smem, 0);
    unsigned char* dst = out + off[blockIdx.x];
    for (int c = 0; c < nchunks; ++c) {
        pol.fetch(c);
        pol.build(st);
        __syncthreads();
        uint4* d = reinterpret_cast<uint4*>(dst + (size_t)c * 2 * half);
        const uint4* bh = reinterpret_cast<const uint4*>(st.bh);
        const uint4* bl = reinterpret_cast<const uint4*>(st.bl);
        for (int i = threadIdx.x; i < (int)(half / 16); i += blockDim.x) {
            d[i] = bh[i];
            d[half / 16 + i] = bl[i];
        }
        __syncthreads();
    }
}

// Near tiles against the stored operator: only the data operand is built in the loop.
template <class K>
__global__ void __launch_bounds__(tcp::THREADS, 1) k_list_stored(ListArgs a, const unsigned char* bstore,
                                                                 const long long* off, int* err) {
    const int4 t = a.tiles[blockIdx.x];
    const int nd = 2 * a.Pd + 1, ns = 2 * a.Ps + 1;
    const int nrow = nd;
    ListPolicy pol{a, a.ttgt + t.x, a.tself + t.x, a.tsrc + t.z, nullptr, t.y, t.w, nrow, 0, nd, ns};
    pol.init();
    pol.load_b = false;
    const int n = ((t.y * nrow + 15) / 16) * 16;
    const uint32_t half = (uint32_t)n * tcp::KC * K::ELEM;
    const int nchunks = (t.w * ns + KCC - 1) / KCC;
    tcp::run_stored<ListPolicy, K>(pol, nchunks, n, err, bstore + off[blockIdx.x], half);
}

inline int upv(ms_handle* h, void** dst, const void* src, size_t bytes) {
    *dst = nullptr;
    if (!bytes) return MS_OK;
    if (cudaMalloc(dst, bytes) != cudaSuccess) return MS_ERR_ALLOC;
    return ms_check(h, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
}

}  // namespace

// Shared-memory limits of the tensor-core list kernels (both operand kinds), set once at setup.
void ms_near_tc_attributes() {
    cudaFuncSetAttribute(k_list_tc<tcp::TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcp::SMEM);
    cudaFuncSetAttribute(k_list_tc<tcp::BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcp::SMEM);
    cudaFuncSetAttribute(k_list_store<tcp::TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcp::SMEM);
    cudaFuncSetAttribute(k_list_stored<tcp::TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tcp::SMEM);
}

namespace {
void near_args(ms_handle* h, int b, const float2* xs, float2* dst, int nrhs, ListArgs& a) {
    const FmmHost& F = h->fmm;
    const int nc = h->nc;
    a = ListArgs{};
    a.in = xs ? xs + (long long)b * nc * nrhs : nullptr; a.in_stride = 2LL * nc * nrhs;
    a.out = dst ? dst + (long long)b * nc * nrhs : nullptr; a.out_stride = 2LL * nc * nrhs;
    a.seqm = h->d.seqm; a.seqe = h->d.seqe;
    a.tseq = F.near[b].seq; a.tptr = F.near[b].ptr;
    a.seq_base = F.near_seq_base[b]; a.seq_len = 4 * h->p + 3;
    a.ad = h->d.expo + b * nc; a.ad_stride = 2LL * nc;
    a.as = h->d.expo + b * nc; a.as_stride = 2LL * nc;
    a.tiles = F.near_tc.tile; a.ttgt = F.near_tc.tgt; a.tself = F.near_tc.self; a.tsrc = F.near_tc.src;
    a.trow = nullptr;
    a.Pd = h->p; a.Ps = h->p; a.K = 2 * h->p + 1; a.nrhs = nrhs;
}
}  // namespace

// Stored near operator (ms_options.store_near): the 3xTF32 B tiles of every near tile and chunk, for
// both waves, generated once here.  Skipped (MS_OK, nothing stored) when the tiles exceed the budget
// of opt.store_near gigabytes or the free device memory.
int ms_near_store_build(ms_handle* h) {
    FmmHost& F = h->fmm;
    ms_near_store_free(h);
    if (!h->opt.store_near || !h->opt.tensor_cores || F.near_tc.n == 0) return MS_OK;
    const int nc = h->nc, ntile = F.near_tc.n;
    std::vector<int4> tiles(ntile);
    if (int rc = ms_check(h, cudaMemcpy(tiles.data(), F.near_tc.tile, ntile * sizeof(int4), cudaMemcpyDeviceToHost)))
        return rc;
    std::vector<long long> off(ntile);
    long long total = 0;
    for (int t = 0; t < ntile; ++t) {
        const long long n = ((long long)tiles[t].y * nc + 15) / 16 * 16;
        const long long nchunks = ((long long)tiles[t].w * nc + KCC - 1) / KCC;
        off[t] = total;
        total += nchunks * 2 * n * tcp::KC * 4;
    }
    size_t freeb = 0, totb = 0;
    cudaMemGetInfo(&freeb, &totb);
    const double budget = (double)h->opt.store_near * 1e9;
    if ((double)(2 * total) > budget || (size_t)(2 * total) + ((size_t)8 << 30) > freeb) return MS_OK;
    int rc;
    if ((rc = ms_check(h, cudaMalloc(&F.near_store, (size_t)2 * total))) ||
        (rc = ms_check(h, cudaMalloc(&F.near_store_off, ntile * sizeof(long long)))) ||
        (rc = ms_check(h, cudaMemcpy(F.near_store_off, off.data(), ntile * sizeof(long long),
                                     cudaMemcpyHostToDevice)))) {
        ms_near_store_free(h);
        return rc;
    }
    F.near_store_wave = total;
    for (int b = 0; b < 2; ++b) {
        ListArgs a;
        near_args(h, b, nullptr, nullptr, 1, a);
        k_list_store<tcp::TF32><<<ntile, tcp::THREADS, tcp::SMEM>>>(a, F.near_store + (size_t)b * total,
                                                                    F.near_store_off);
        if ((rc = ms_check(h, cudaGetLastError()))) { ms_near_store_free(h); return rc; }
    }
    return ms_check(h, cudaDeviceSynchronize());
}

void ms_near_store_free(ms_handle* h) {
    FmmHost& F = h->fmm;
    cudaFree(F.near_store);
    cudaFree(F.near_store_off);
    F.near_store = nullptr;
    F.near_store_off = nullptr;
    F.near_store_wave = 0;
}

// Tiles of the FMM multipole-to-local stage for (wave b, level lev): one tile per 256-row range of
// every box that has an interaction list; its sources are the box's M2L tasks.  Boxes without a list
// keep zero local expansions (the launch clears the level first).
int ms_m2l_tc_tiles(ms_handle* h, int b, int lev, const std::vector<int>& ptr) {
    FmmHost& F = h->fmm;
    const int nd = 2 * F.P[b][lev] + 1;
    std::vector<int4> tiles;
    std::vector<int> tgt, self, row;
    for (int d = 0; d + 1 < (int)ptr.size(); ++d) {
        if (ptr[d + 1] == ptr[d]) continue;
        for (int i0 = 0; i0 < nd; i0 += tcp::NMAX) {
            tiles.push_back(make_int4((int)tgt.size(), 1, ptr[d], ptr[d + 1] - ptr[d]));
            tgt.push_back(d);
            self.push_back(-1);
            row.push_back(i0);
        }
    }
    TcTiles& T = F.m2l_tc[b][lev];
    T.n = (int)tiles.size();
    int rc;
    if ((rc = upv(h, (void**)&T.tile, tiles.data(), tiles.size() * sizeof(int4))) ||
        (rc = upv(h, (void**)&T.tgt, tgt.data(), tgt.size() * sizeof(int))) ||
        (rc = upv(h, (void**)&T.self, self.data(), self.size() * sizeof(int))) ||
        (rc = upv(h, (void**)&T.row, row.data(), row.size() * sizeof(int))))
        return rc;
    return MS_OK;
}

void ms_tc_tiles_free(TcTiles& T) {
    cudaFree(T.tile); cudaFree(T.tgt); cudaFree(T.self); cudaFree(T.src); cudaFree(T.row);
    T = TcTiles{};
}

// a~ = near-pair Graf sum of the FP32 scaled block xs into dst (written, both waves).
int ms_near_tc_launch(ms_handle* h, const float2* xs, float2* dst, int nrhs, cudaStream_t st) {
    const FmmHost& F = h->fmm;
    const int nc = h->nc;
    for (int b = 0; b < 2; ++b) {
        ListArgs a;
        near_args(h, b, xs, dst, nrhs, a);
        if (!h->tc_kind && F.near_store)
            k_list_stored<tcp::TF32><<<F.near_tc.n, tcp::THREADS, tcp::SMEM, st>>>(
                a, F.near_store + (size_t)b * F.near_store_wave, F.near_store_off, h->d.tc_err);
        else if (h->tc_kind)
            k_list_tc<tcp::BF16><<<F.near_tc.n, tcp::THREADS, tcp::SMEM, st>>>(a, h->d.tc_err);
        else
            k_list_tc<tcp::TF32><<<F.near_tc.n, tcp::THREADS, tcp::SMEM, st>>>(a, h->d.tc_err);
        if (int rc = ms_check(h, cudaGetLastError())) return rc;
    }
    return MS_OK;
}

// Multipole-to-local of (wave b, level lev) from the FP32 multipole block into the local block.
int ms_m2l_tc_launch(ms_handle* h, int b, int lev, const float2* mexp, float2* lexp, int nrhs, cudaStream_t st) {
    const FmmHost& F = h->fmm;
    const int P = F.P[b][lev], nd = 2 * P + 1;
    if (int rc = ms_check(h, cudaMemsetAsync(lexp, 0, (size_t)F.nbox[lev] * nd * nrhs * sizeof(float2), st)))
        return rc;
    const TcTiles& T = F.m2l_tc[b][lev];
    if (T.n == 0) return MS_OK;
    ListArgs a{};
    a.in = mexp; a.in_stride = (long long)nd * nrhs;
    a.out = lexp; a.out_stride = (long long)nd * nrhs;
    a.seqm = h->d.seqm; a.seqe = h->d.seqe;
    a.tseq = F.m2l[b][lev].seq; a.tptr = F.m2l[b][lev].ptr;
    a.seq_base = 0; a.seq_len = 0;
    a.ad = F.expo[b][lev]; a.ad_stride = 0;
    a.as = F.expo[b][lev]; a.as_stride = 0;
    a.tiles = T.tile; a.ttgt = T.tgt; a.tself = T.self; a.tsrc = F.m2l[b][lev].src; a.trow = T.row;
    a.Pd = P; a.Ps = P; a.K = 2 * P; a.nrhs = nrhs;
    if (h->tc_kind)
        k_list_tc<tcp::BF16><<<T.n, tcp::THREADS, tcp::SMEM, st>>>(a, h->d.tc_err);
    else
        k_list_tc<tcp::TF32><<<T.n, tcp::THREADS, tcp::SMEM, st>>>(a, h->d.tc_err);
    return ms_check(h, cudaGetLastError());
}
