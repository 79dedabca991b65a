// Autotuner of the operator's launch shapes: the FMM leaf level (which sets the near-pair tiles, the
// M2L tiles and how much work is direct) and the K-split size of the tensor-core multipole-to-
// Sommerfeld contraction.  Each candidate is timed on the live handle (one warm-up, then the median of
// three mat-vecs of a seeded block with CUDA events); the fastest stays.  Choices are cached per
// process by (M, p, N_S, columns, data precision, operand kind, tensor cores), so that another handle
// of the same sizes adopts them without timing.
#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "handle.h"

namespace {

typedef std::tuple<int, int, int, int, int, int, int> Key;
std::map<Key, std::pair<int, int>> g_cache;     // -> (leaf target, M2S rows per split)
std::mutex g_mutex;

// deterministic block: entries in [-1, 1) from a 64-bit mix of the index, scaled down with the order
__global__ void k_seed_block(double2* x, long long n, int nrhs, int nc) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    unsigned long long z = (unsigned long long)i * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const int n_abs = abs((int)((i / nrhs) % nc) - nc / 2);
    const double f = pow2d(-n_abs);
    x[i] = make_double2(((z & 0xffffffff) * 0x1p-31 - 1.0) * f, ((z >> 32) * 0x1p-31 - 1.0) * f);
}

int rebuild(ms_handle* h, int leaf) {
    ms_graphs_free(h);
    ms_fmm_free(h);
    if (int rc = ms_build_translations(h, h->opt.use_fmm, leaf)) return rc;
    h->opt.leaf_target = leaf;
    if (h->opt.tensor_cores)
        if (int rc = ms_near_store_build(h)) return rc;
    return ms_fmm_workspace(h, h->ws_nrhs);
}

}  // namespace

extern "C" int ms_autotune(ms_handle* h, int32_t nrhs, int32_t prec, int32_t* leaf_target, int32_t* m2s_rows,
                           double* ms_per_apply, void* stream) {
    if (!h || nrhs < 1) return MS_ERR_ARG;
    if (nrhs > 64) return MS_ERR_UNSUPPORTED;
    const int kind_prec = prec;
    if ((prec = ms_resolve_prec(h, prec)) < 0) return prec;
    int rc = ms_ensure_workspace(h, nrhs);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const Key key{h->M, h->p, h->NS, nrhs, prec, h->tc_kind, h->opt.tensor_cores};
    const size_t n = (size_t)h->M * 2 * h->nc * nrhs;
    double2 *x = nullptr, *y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaFree(x); cudaFree(y);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if ((rc = ms_check(h, cudaMalloc(&x, n * sizeof(double2)))) || (rc = ms_check(h, cudaMalloc(&y, n * sizeof(double2)))) ||
        (rc = ms_check(h, cudaEventCreate(&e0))) || (rc = ms_check(h, cudaEventCreate(&e1)))) {
        cleanup();
        return rc;
    }
    k_seed_block<<<(int)((n + 255) / 256), 256, 0, st>>>(x, (long long)n, nrhs, h->nc);
    auto timed = [&](double& ms) -> int {
        if (int r = ms_apply(h, x, y, nrhs, kind_prec, stream)) return r;
        std::vector<float> t(3);
        for (float& v : t) {
            cudaEventRecord(e0, st);
            if (int r = ms_apply(h, x, y, nrhs, kind_prec, stream)) return r;
            cudaEventRecord(e1, st);
            if (int r = ms_check(h, cudaEventSynchronize(e1))) return r;
            cudaEventElapsedTime(&v, e0, e1);
        }
        std::sort(t.begin(), t.end());
        ms = t[1];
        return MS_OK;
    };
    int best_leaf = h->opt.leaf_target, best_rows = h->m2s_rows > 0 ? h->m2s_rows : 2048;
    double best = 1e300;
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            cached = true;
            best_leaf = it->second.first;
            best_rows = it->second.second;
        }
    }
    if (cached) {
        if (best_leaf != h->opt.leaf_target && (rc = rebuild(h, best_leaf))) { cleanup(); return rc; }
        h->m2s_rows = best_rows;
        rc = timed(best);
    } else {
        // leaf levels around the current one: leaf targets M / 4^L for L = L0 - 1, L0, L0 + 1
        const int L0 = h->fmm_levels;
        std::vector<int> leaves;
        if (L0 >= 2 && h->opt.use_fmm) {
            for (int L = std::max(2, L0 - 1); L <= std::min(12, L0 + 1); ++L) {
                double v = (double)h->M;
                for (int k = 0; k < L; ++k) v /= 4.0;
                leaves.push_back(std::max(1, (int)lround(v)));
            }
        } else {
            leaves.push_back(h->opt.leaf_target);
        }
        int seen_levels[13] = {0};
        for (int leaf : leaves) {
            if ((rc = rebuild(h, leaf))) { cleanup(); return rc; }
            if (seen_levels[h->fmm_levels]++) continue;           // the width rule merged two candidates
            double t;
            if ((rc = timed(t))) { cleanup(); return rc; }
            if (t < best) { best = t; best_leaf = leaf; }
        }
        if (best_leaf != h->opt.leaf_target && (rc = rebuild(h, best_leaf))) { cleanup(); return rc; }
        // K-split size of the tensor-core multipole-to-Sommerfeld contraction
        if (h->opt.tensor_cores && prec == MS_PREC_FP32) {
            best = 1e300;
            for (int rows : {1024, 2048, 4096, 8192}) {
                h->m2s_rows = rows;
                ms_graphs_free(h);
                double t;
                if ((rc = timed(t))) { cleanup(); return rc; }
                if (t < best) { best = t; best_rows = rows; }
            }
            h->m2s_rows = best_rows;
            ms_graphs_free(h);
        } else {
            double t;
            if ((rc = timed(t))) { cleanup(); return rc; }
            best = t;
        }
        std::lock_guard<std::mutex> lock(g_mutex);
        g_cache[key] = {best_leaf, best_rows};
    }
    cleanup();
    if (leaf_target) *leaf_target = best_leaf;
    if (m2s_rows) *m2s_rows = best_rows;
    if (ms_per_apply) *ms_per_apply = best;
    return MS_OK;
}
