// Free-space particle-to-particle translation: direct Graf sum for near pairs (row a2) and a
// quadtree fast multipole method for the rest (row a3), Sec. 4.2 (FMM cited there, O(M p^2)).
//
// Every translation in this file has the same Toeplitz form (Graf's addition theorem,
// DLMF 10.23.7, for H and J):
//     dst[i] += sum_j Z_{j-i}(k |v|) e^{i (j-i) arg v} src[j],   v = c_dst - c_src,
// with Z = H^(1) from outgoing to local (particle near pairs, M2L) and Z = J for shifts of
// outgoing expansions (P2M, M2M) and of local expansions (L2L, L2P).  The sequences
// h_k = Z_k(k|v|) e^{ik arg v}, |k| <= K = P_dst + P_src, are computed once per geometry in FP64
// on the device and stored in HBM (an FP32 mantissa / binary-exponent copy serves the FP32 path).
// Coefficients live in the scaled basis: outgoing x~ = x / tau, local a~ = a tau, tau = 2^a, so
// the entry applied is  h_{j-i} 2^{s_dst a_dst,i + s_src a_src,j}  with the signs s of each side.
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "handle.h"

namespace {

// ------------------------------------------------------------------ sequence generation
// h[K + k] = Z_k(x) e^{ik phi}, k in [-K, K], Z = J (kind 0) or H^(1) (kind 1).  The recurrences
// are those of bessel.cuh, run in place in the output row: first (J_k, Y_k) are written at
// h[K + k], k >= 0, then phases are applied and negative orders filled from Z_{-k} = (-1)^k Z_k.
__device__ void zseq_inplace(int K, double x, double ux, double uy, int kind, double2* h) {
    double2* o = h + K;
    // Y upward (stable), kept in .y
    if (kind == 1) {
        o[0].y = y0(x);
        if (K >= 1) o[1].y = y1(x);
        for (int k = 1; k < K; ++k) o[k + 1].y = (2.0 * k / x) * o[k].y - o[k - 1].y;
    }
    if (x > (double)K) {
        o[0].x = j0(x);
        if (K >= 1) o[1].x = j1(x);
        for (int k = 1; k < K; ++k) o[k + 1].x = (2.0 * k / x) * o[k].x - o[k - 1].x;
    } else {
        int ns = K + 16 + (int)ceil(x) + (int)sqrt(40.0 * K);
        ns += ns & 1;
        double jp1 = 0.0, j = 1e-300;
        for (int k = ns; k >= 1; --k) {
            double jm1 = (2.0 * k / x) * j - jp1;
            jp1 = j;
            j = jm1;
            if (k - 1 <= K) o[k - 1].x = jm1;
            if (fabs(j) > 1e250) {
                j *= 1e-250;
                jp1 *= 1e-250;
                for (int i = k - 1; i <= K; ++i) o[i].x *= 1e-250;
            }
        }
        double j0s = o[0].x, j1s = K >= 1 ? o[1].x : jp1;
        double c = (fabs(j0s) > fabs(j1s)) ? j0(x) / j0s : j1(x) / j1s;
        for (int k = 0; k <= K; ++k) o[k].x *= c;
    }
    if (kind == 0)
        for (int k = 0; k <= K; ++k) o[k].y = 0.0;
    // phases; walk k downward so that the (J, Y) pairs at o[k] are read before h[K - k] is written
    // (h[K - k] for k > 0 lies below o[0]).
    double2 u = make_double2(ux, uy);
    // e^{iK phi} by repeated squaring would lose nothing here; plain powers are accurate to ~K ulp
    double2 eK = make_double2(1.0, 0.0);
    for (int k = 0; k < K; ++k) eK = cmul(eK, u);
    double2 e = eK;
    double2 ub = cconj(u);
    for (int k = K; k >= 0; --k) {
        double2 Z = o[k];
        o[k] = cmul(Z, e);
        if (k > 0) {
            double2 w = cmul(Z, cconj(e));
            if (k & 1) w = make_double2(-w.x, -w.y);
            h[K - k] = w;
        }
        e = cmul(e, ub);
    }
}

struct SeqSpec {
    double vx, vy, k;
    int K, kind;
    long long off;
};

__global__ void k_gen_seq(const SeqSpec* __restrict__ spec, int n, double2* __restrict__ seq) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    SeqSpec s = spec[i];
    double d = sqrt(s.vx * s.vx + s.vy * s.vy);
    double ux = d > 0 ? s.vx / d : 1.0, uy = d > 0 ? s.vy / d : 0.0;
    if (d == 0.0) {
        // zero shift: J_k(0) = delta_k0 (only J sequences are ever asked for at d = 0)
        for (int k = -s.K; k <= s.K; ++k) seq[s.off + s.K + k] = make_double2(k == 0 ? 1.0 : 0.0, 0.0);
        return;
    }
    zseq_inplace(s.K, s.k * d, ux, uy, s.kind, seq + s.off);
}

__global__ void k_split_seq(const double2* __restrict__ seq, float2* __restrict__ m, int* __restrict__ e,
                            long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float2 mm;
    int ee;
    split_exp(seq[i], mm, ee);
    m[i] = mm;
    e[i] = ee;
}

// ------------------------------------------------------------------ generic translation
constexpr int TR_IB = 3;
constexpr int TR_RB = 8;
constexpr int TR_ICH = 42;     // dst orders per CTA (14 x TR_IB)
constexpr int TR_JCH = 41;     // src orders per staged tile
constexpr int TR_ES = 43;      // row stride of the operator tile (bank-conflict-free for rows 3*ib)
constexpr int TR_SEQ = TR_ICH + TR_JCH + 2;   // sequence entries a tile needs (<= ni + nj + 1)
constexpr int TR_THREADS = 128;

template <typename T> struct SeqRef;
template <> struct SeqRef<double> {
    const double2* s;
    typedef double2 M;
    __device__ void stage(long long idx, double2* m, int* e) const { *m = s[idx]; *e = 0; }
    __device__ static double2 make(double2 v, int e, int scale) {
        double f = pow2d(scale);
        return make_double2(v.x * f, v.y * f);
    }
};
template <> struct SeqRef<float> {
    const float2* m;
    const int* e;
    typedef float2 M;
    __device__ void stage(long long idx, float2* mm, int* ee) const { *mm = m[idx]; *ee = e[idx]; }
    __device__ static float2 make(float2 v, int e, int scale) {
        float f = pow2f(e + scale);
        return make_float2(v.x * f, v.y * f);
    }
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// Adjoint mode (a.adj = 1).  For a translation with vector v from s to d, the reverse one (from d
// to s, vector -v) has h^rev_k = (-1)^k h_k, since Z_k(x) e^{ik(phi + pi)} = (-1)^k Z_k(x) e^{ik phi}.
// So the adjoint, out_s[j] += sum_i conj(h_{n_j - n_i}) in_d[i], is the reverse-direction launch
// (reverse list: dst s, src d) with entries (-1)^k conj(h^rev_{-k}), k = n_src - n_dst.  Run on the
// mirrored lists (near <-> near, P2M <-> L2P, M2M <-> L2L, M2L <-> M2L) with the mirrored scale
// signs, the forward pipeline code in adjoint mode applies T^H.
//
// CTA = (dst entity d, dst order chunk).  Work items are (task, source-order chunk) pairs: each
// stages the sequence segment and the scale exponents it needs, builds the scaled operator tile
// E[i][j] = h_{n_j - n_i} 2^{s_d a_d,i + s_s a_s,j} in shared memory, and accumulates
// E x (source block) into a TR_IB x TR_RB register tile per thread.  The source block of the next
// item is fetched with cp.async while the current one is multiplied (when rows are 16-byte aligned).
template <typename T>
__global__ void __launch_bounds__(TR_THREADS)
k_translate(TransArgs a, SeqRef<T> seq) {
    typedef typename CT<T>::c C;
    typedef typename SeqRef<T>::M SM;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nrhs = a.nrhs;
    C* Eb = reinterpret_cast<C*>(smem_raw);                    // [TR_ICH][TR_ES]
    C* Xb = Eb + TR_ICH * TR_ES;                               // [2][TR_JCH][nrhs]
    SM* sq = reinterpret_cast<SM*>(Xb + 2 * TR_JCH * nrhs);    // [TR_SEQ]
    int* se = reinterpret_cast<int*>(sq + TR_SEQ);             // [TR_SEQ]
    int* sad = se + TR_SEQ;                                    // [TR_ICH]
    int* sas = sad + TR_ICH;                                   // [TR_JCH]

    const int nd = 2 * a.Pd + 1, ns = 2 * a.Ps + 1, K = a.K;
    const int d = blockIdx.x;
    const int ic0 = blockIdx.y * TR_ICH;
    const int ni = min(TR_ICH, nd - ic0);
    const int n_rb = (nrhs + TR_RB - 1) / TR_RB;
    const int tile = threadIdx.x;
    const bool act = tile < ((ni + TR_IB - 1) / TR_IB) * n_rb;
    const int ib = act ? tile / n_rb : 0, rb = act ? tile % n_rb : 0;
    const int i0 = ib * TR_IB, r0 = rb * TR_RB;
    const bool vec = (nrhs % 2) == 0;            // 16-byte rows for cp.async and paired loads
    const int* ad = a.ad + (long long)d * a.ad_stride;
    for (int t = threadIdx.x; t < ni; t += blockDim.x) sad[t] = ad[ic0 + t];

    C acc[TR_IB][TR_RB];
#pragma unroll
    for (int u = 0; u < TR_IB; ++u)
#pragma unroll
        for (int v = 0; v < TR_RB; ++v) acc[u][v] = mk((T)0, (T)0);

    const int t0 = a.dst_ptr[d], t1 = a.dst_ptr[d + 1];
    const int nch = (ns + TR_JCH - 1) / TR_JCH;
    const int nitems = (t1 - t0) * nch;

    // issue the copy of item it's source block into buffer buf
    auto fetch = [&](int it, int buf) {
        const int t = t0 + it / nch, jc = (it % nch) * TR_JCH;
        const int nj = min(TR_JCH, ns - jc);
        const C* src = reinterpret_cast<const C*>(a.src) + (long long)a.task_src[t] * a.src_stride + (long long)jc * nrhs;
        C* dstb = Xb + buf * TR_JCH * nrhs;
        if (vec) {
            const int n16 = nj * nrhs * (int)sizeof(C) / 16;
            for (int e = threadIdx.x; e < n16; e += blockDim.x)
                cp_async16(reinterpret_cast<char*>(dstb) + 16 * e, reinterpret_cast<const char*>(src) + 16 * e);
            cp_async_commit();
        } else {
            for (int e = threadIdx.x; e < nj * nrhs; e += blockDim.x) dstb[e] = src[e];
        }
    };
    if (nitems > 0) fetch(0, 0);
    for (int it = 0; it < nitems; ++it) {
        const int buf = it & 1;
        const int t = t0 + it / nch, jc = (it % nch) * TR_JCH;
        const int nj = min(TR_JCH, ns - jc);
        const int s = a.task_src[t];
        const long long so = a.task_seq[t];
        // sequence segment: k = (j - Ps) - (i - Pd) for i in [ic0, ic0+ni), j in [jc, jc+nj); the
        // adjoint reads index -k of the reverse-direction sequence
        const int klo = (jc - a.Ps) - (ic0 + ni - 1 - a.Pd), khi = (jc + nj - 1 - a.Ps) - (ic0 - a.Pd);
        const int kmin = (a.adj ? -khi : klo) - a.deriv;      // one more entry each side for derivatives
        const int nk = ni + nj - 1 + 2 * a.deriv;
        for (int e = threadIdx.x; e < nk; e += blockDim.x) seq.stage(so + K + kmin + e, &sq[e], &se[e]);
        const int* as = a.as + (long long)s * a.as_stride;
        for (int e = threadIdx.x; e < nj; e += blockDim.x) sas[e] = as[jc + e];
        if (vec) cp_async_wait_all();
        __syncthreads();                                   // sequence, exponents, block `buf` ready
        if (it + 1 < nitems) fetch(it + 1, buf ^ 1);
        for (int e = threadIdx.x; e < ni * nj; e += blockDim.x) {
            int ii = e / nj, jj = e % nj;
            int k = (jj + jc - a.Ps) - (ii + ic0 - a.Pd);
            if (a.adj) k = -k;
            const int sc = a.sd * sad[ii] + a.ss * sas[jj];
            C v;
            if (a.deriv) {
                // d/dv of h_k = Z_k(kap|v|) e^{ik arg v}: c1 h_{k-1} + c2 h_{k+1} (DLMF 10.6)
                C lo = SeqRef<T>::make(sq[k - 1 - kmin], se[k - 1 - kmin], sc);
                C hi = SeqRef<T>::make(sq[k + 1 - kmin], se[k + 1 - kmin], sc);
                v = cadd(cmul(to_c<T>(a.dc1), lo), cmul(to_c<T>(a.dc2), hi));
            } else {
                v = SeqRef<T>::make(sq[k - kmin], se[k - kmin], sc);
            }
            if (a.adj) {
                v = cconj(v);
                if (k & 1) v = mk(-v.x, -v.y);
            }
            Eb[ii * TR_ES + jj] = v;
        }
        __syncthreads();                                   // operator tile ready
        if (act) {
            const C* X = Xb + buf * TR_JCH * nrhs + r0;
            const C* E = Eb + i0 * TR_ES;
            const int nr = min(TR_RB, nrhs - r0);
            if (vec && nr == TR_RB) {
#pragma unroll 2
                for (int jj = 0; jj < nj; ++jj) {
                    C xv[TR_RB];
                    const C* xr = X + jj * nrhs;
#pragma unroll
                    for (int v = 0; v < TR_RB; ++v) xv[v] = xr[v];
                    C ev[TR_IB];
#pragma unroll
                    for (int u = 0; u < TR_IB; ++u) ev[u] = E[u * TR_ES + jj];
#pragma unroll
                    for (int u = 0; u < TR_IB; ++u)
#pragma unroll
                        for (int v = 0; v < TR_RB; ++v) cfma(acc[u][v], ev[u], xv[v]);
                }
            } else {
                for (int jj = 0; jj < nj; ++jj) {
                    C xv[TR_RB];
#pragma unroll
                    for (int v = 0; v < TR_RB; ++v) xv[v] = v < nr ? X[jj * nrhs + v] : mk((T)0, (T)0);
#pragma unroll
                    for (int u = 0; u < TR_IB; ++u) {
                        C e = (i0 + u) < ni ? E[u * TR_ES + jj] : mk((T)0, (T)0);
#pragma unroll
                        for (int v = 0; v < TR_RB; ++v) cfma(acc[u][v], e, xv[v]);
                    }
                }
            }
        }
        __syncthreads();                                   // tile and block `buf` free again
    }
    if (act) {
        C* dst = reinterpret_cast<C*>(a.dst) + (long long)d * a.dst_stride;
#pragma unroll
        for (int u = 0; u < TR_IB; ++u) {
            int ii = i0 + u;
            if (ii >= ni) continue;
#pragma unroll
            for (int v = 0; v < TR_RB; ++v) {
                int r = r0 + v;
                if (r >= nrhs) continue;
                long long o = (long long)(ic0 + ii) * nrhs + r;
                dst[o] = a.accumulate ? cadd(dst[o], acc[u][v]) : acc[u][v];
            }
        }
    }
}

}  // namespace

static double fmm_order_tail(double k, double rho, double dist) {
    // smallest P with |J_{P+1}(k rho)| |H_{P+1}(k (dist - rho))| < 1e-14 and |J_{P+1}(k rho)| < 1e-3
    for (int P = 5; P < 1000; ++P) {
        double j = fabs(jn(P + 1, k * rho));
        double hx = k * (dist - rho);
        double hy = hypot(jn(P + 1, hx), yn(P + 1, hx));
        if (j * hy < 1e-14 && j < 1e-3) return P;
    }
    return 1000;
}

int ms_translate_launch(ms_handle* h, const TransArgs& a, int ndst, bool fp32, cudaStream_t st) {
    if (ndst == 0) return MS_OK;
    int nd = 2 * a.Pd + 1;
    dim3 grid(ndst, (nd + TR_ICH - 1) / TR_ICH);
    int tiles = (TR_ICH / TR_IB) * ((a.nrhs + TR_RB - 1) / TR_RB);
    int threads = std::max(32, std::min(TR_THREADS, (tiles + 31) / 32 * 32));
    size_t tail = (size_t)TR_SEQ * sizeof(int) + (size_t)(TR_ICH + TR_JCH) * sizeof(int);
    if (fp32) {
        size_t smem = (size_t)TR_ICH * TR_ES * sizeof(float2) + (size_t)2 * TR_JCH * a.nrhs * sizeof(float2) +
                      (size_t)TR_SEQ * sizeof(float2) + tail;
        cudaFuncSetAttribute(k_translate<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        SeqRef<float> s{h->d.seqm, h->d.seqe};
        k_translate<float><<<grid, threads, smem, st>>>(a, s);
    } else {
        size_t smem = (size_t)TR_ICH * TR_ES * sizeof(double2) + (size_t)2 * TR_JCH * a.nrhs * sizeof(double2) +
                      (size_t)TR_SEQ * sizeof(double2) + tail;
        cudaFuncSetAttribute(k_translate<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        SeqRef<double> s{h->d.seq64};
        k_translate<double><<<grid, threads, smem, st>>>(a, s);
    }
    return ms_check(h, cudaGetLastError());
}

// ------------------------------------------------------------------ host: tree and task lists
namespace {

struct HostList {
    std::vector<int> ptr, src;
    std::vector<long long> seq;
};

struct Builder {
    ms_handle* h;
    std::vector<SeqSpec> specs;
    long long total = 0;
    long long add(double vx, double vy, double k, int K, int kind) {
        SeqSpec s{vx, vy, k, K, kind, total};
        specs.push_back(s);
        total += 2 * K + 1;
        return s.off;
    }
};

template <typename X>
int up(ms_handle* h, X** dst, const std::vector<X>& v) {
    if (v.empty()) { *dst = nullptr; return MS_OK; }
    if (cudaMalloc((void**)dst, v.size() * sizeof(X)) != cudaSuccess) return MS_ERR_ALLOC;
    return ms_check(h, cudaMemcpy(*dst, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice));
}

int upload_list(ms_handle* h, const HostList& L, DevList& D) {
    D.ndst = (int)L.ptr.size() - 1;
    D.ntask = (int)L.src.size();
    int rc;
    if ((rc = up(h, &D.ptr, L.ptr)) || (rc = up(h, &D.src, L.src)) || (rc = up(h, &D.seq, L.seq))) return rc;
    return MS_OK;
}

}  // namespace

// Build the near-field pair lists (all pairs when the FMM is off) and, with the FMM on, the
// quadtree, interaction lists and translation sequences.  Called once from ms_setup.
int ms_build_translations(ms_handle* h, int use_fmm, int leaf_target) {
    const int M = h->M, p = h->p;
    const double* c = h->h_centres.data();
    double rmax = 0;
    for (double r : h->h_radius) rmax = std::max(rmax, r);
    double xmin = 1e300, xmax = -1e300, ymin = 1e300, ymax = -1e300;
    for (int m = 0; m < M; ++m) {
        xmin = std::min(xmin, c[2 * m]); xmax = std::max(xmax, c[2 * m]);
        ymin = std::min(ymin, c[2 * m + 1]); ymax = std::max(ymax, c[2 * m + 1]);
    }
    double S = std::max(xmax - xmin, ymax - ymin) * (1.0 + 1e-9) + 1e-9;
    // leaf level: about leaf_target particles per leaf, >= 2, leaf width > 3.5 R_max (so that
    // non-adjacent leaves are separated for the expansions, particle discs included)
    int L = 0;
    if (use_fmm) {
        L = (int)lround(log((double)M / leaf_target) / log(4.0));
        while (L >= 2 && S / (1 << L) <= 3.5 * rmax) --L;
        if (L < 2) L = 0;
    }
    h->fmm_levels = L;
    Builder B{h};
    const double kb[2] = {h->kp_l, h->ks_l};

    // leaf index of each particle (or a single leaf)
    int nL = L ? (1 << L) : 1;
    double wL = S / nL;
    std::vector<int> leaf(M);
    for (int m = 0; m < M; ++m) {
        int ix = std::min(nL - 1, std::max(0, (int)((c[2 * m] - xmin) / wL)));
        int iy = std::min(nL - 1, std::max(0, (int)((c[2 * m + 1] - ymin) / wL)));
        leaf[m] = iy * nL + ix;
    }
    std::vector<int> lptr(nL * nL + 1, 0), lidx(M);
    for (int m = 0; m < M; ++m) lptr[leaf[m] + 1]++;
    for (int i = 0; i < nL * nL; ++i) lptr[i + 1] += lptr[i];
    {
        std::vector<int> fill(lptr.begin(), lptr.end() - 1);
        for (int m = 0; m < M; ++m) lidx[fill[leaf[m]]++] = m;
    }

    // near lists: sources in the 3 x 3 leaves around the target's leaf (all pairs if one leaf)
    HostList nearL;
    nearL.ptr.assign(M + 1, 0);
    std::vector<long long> seq_near[2];
    for (int m = 0; m < M; ++m) {
        nearL.ptr[m] = (int)nearL.src.size();
        int ix = leaf[m] % nL, iy = leaf[m] / nL;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int jx = ix + dx, jy = iy + dy;
                if (jx < 0 || jy < 0 || jx >= nL || jy >= nL) continue;
                int bx = jy * nL + jx;
                for (int t = lptr[bx]; t < lptr[bx + 1]; ++t) {
                    int l = lidx[t];
                    if (l == m) continue;
                    nearL.src.push_back(l);
                }
            }
    }
    nearL.ptr[M] = (int)nearL.src.size();
    h->nnz_near = (int)nearL.src.size();
    for (int b = 0; b < 2; ++b) {
        seq_near[b].resize(nearL.src.size());
        for (int m = 0; m < M; ++m)
            for (int t = nearL.ptr[m]; t < nearL.ptr[m + 1]; ++t) {
                int l = nearL.src[t];
                // one order beyond 2p so that order-shifted (derivative) expansions reuse the table
                seq_near[b][t] = B.add(c[2 * m] - c[2 * l], c[2 * m + 1] - c[2 * l + 1], kb[b], 2 * p + 1, 1);
            }
    }
    int rc;
    for (int b = 0; b < 2; ++b) {
        HostList hl = nearL;
        hl.seq = seq_near[b];
        if ((rc = upload_list(h, hl, h->fmm.near[b]))) return rc;
        h->fmm.work_near += (double)h->fmm.near[b].ntask * (2 * p + 1) * (2 * p + 1);
    }
    if (h->opt.tensor_cores) {
        // the near sequences of each wave are consecutive (the tensor-core tiles compute offsets)
        for (int b = 0; b < 2; ++b) {
            const long long len = 4LL * p + 3;
            h->fmm.near_seq_base[b] = seq_near[b].empty() ? 0 : seq_near[b][0];
            for (size_t t = 0; t < seq_near[b].size(); ++t)
                if (seq_near[b][t] != h->fmm.near_seq_base[b] + (long long)t * len) return MS_ERR_UNSUPPORTED;
        }
        // tiles of the tensor-core near field (same source order as the near lists above)
        const int tpt = std::max(1, 256 / h->nc);
        std::vector<int4> tinfo;
        std::vector<int> ttgt, tself, tsrc;
        for (int bx = 0; bx < nL * nL; ++bx) {
            if (lptr[bx] == lptr[bx + 1]) continue;
            const int src_off = (int)tsrc.size();
            const int ix = bx % nL, iy = bx / nL;
            int self_base = -1;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int jx = ix + dx, jy = iy + dy;
                    if (jx < 0 || jy < 0 || jx >= nL || jy >= nL) continue;
                    int by = jy * nL + jx;
                    if (by == bx) self_base = (int)tsrc.size() - src_off;
                    for (int t = lptr[by]; t < lptr[by + 1]; ++t) tsrc.push_back(lidx[t]);
                }
            const int nsrc = (int)tsrc.size() - src_off;
            for (int t0 = lptr[bx]; t0 < lptr[bx + 1]; t0 += tpt) {
                const int nt = std::min(tpt, lptr[bx + 1] - t0);
                tinfo.push_back(make_int4((int)ttgt.size(), nt, src_off, nsrc));
                for (int u = 0; u < nt; ++u) {
                    ttgt.push_back(lidx[t0 + u]);
                    tself.push_back(self_base + (t0 + u - lptr[bx]));
                }
            }
        }
        TcTiles& T = h->fmm.near_tc;
        T.n = (int)tinfo.size();
        if ((rc = up(h, &T.tile, tinfo)) || (rc = up(h, &T.tgt, ttgt)) || (rc = up(h, &T.self, tself)) ||
            (rc = up(h, &T.src, tsrc)))
            return rc;
    }

    if (L) {
        // ---------------------------------------------------------- tree
        FmmHost& F = h->fmm;
        std::vector<std::vector<int>> nonempty(L + 1);
        for (int lev = 0; lev <= L; ++lev) {
            int n = 1 << lev;
            F.nbox[lev] = n * n;
            F.w[lev] = S / n;
            nonempty[lev].assign(n * n, 0);
        }
        for (int m = 0; m < M; ++m) {
            int ix = leaf[m] % nL, iy = leaf[m] / nL;
            for (int lev = L; lev >= 0; --lev) {
                int sh = L - lev;
                nonempty[lev][(iy >> sh) * (1 << lev) + (ix >> sh)] = 1;
            }
        }
        auto centre = [&](int lev, int id, double& cx, double& cy) {
            int n = 1 << lev;
            cx = xmin + ((id % n) + 0.5) * F.w[lev];
            cy = ymin + ((id / n) + 0.5) * F.w[lev];
        };
        for (int b = 0; b < 2; ++b)
            for (int lev = 2; lev <= L; ++lev) {
                double rho = F.w[lev] * sqrt(2.0) / 2.0 + rmax;
                int P = (int)fmm_order_tail(kb[b], rho, 2.0 * F.w[lev]);
                P = std::min(P, 480);
                F.P[b][lev] = P;
                // scale exponents of the box expansions: round(log2((k rho / 2)^|n| / |n|!)) where that is
                // below 1, else 0.  Box expansions of a physical field are O(1) up to |n| ~ k rho and decay
                // like the profile beyond; scaling the lower orders up as well (by up to 2^108 on the
                // 36-wide boxes of the 10^4-particle cloud) pushes the products of two profiles in the M2L
                // entries past the FP32 exponent range
                std::vector<int> e(2 * P + 1);
                for (int i = 0; i <= 2 * P; ++i) {
                    int n = abs(i - P);
                    double l2 = n * log2(kb[b] * rho / 2.0) - lgamma(n + 1.0) / log(2.0);
                    e[i] = (int)std::max(-900L, std::min(0L, lround(l2)));
                }
                if ((rc = up(h, &F.expo[b][lev], e))) return rc;
            }
        // ---------------------------------------------------------- lists per wave
        for (int b = 0; b < 2; ++b) {
            const double k = kb[b];
            // P2M: leaf <- its particles, v = c_leaf - x_l
            HostList p2m;
            p2m.ptr.assign(nL * nL + 1, 0);
            for (int bx = 0; bx < nL * nL; ++bx) {
                p2m.ptr[bx] = (int)p2m.src.size();
                double cx, cy;
                centre(L, bx, cx, cy);
                for (int t = lptr[bx]; t < lptr[bx + 1]; ++t) {
                    int l = lidx[t];
                    p2m.src.push_back(l);
                    p2m.seq.push_back(B.add(cx - c[2 * l], cy - c[2 * l + 1], k, F.P[b][L] + p, 0));
                }
            }
            p2m.ptr[nL * nL] = (int)p2m.src.size();
            if ((rc = upload_list(h, p2m, F.p2m[b]))) return rc;
            F.work_far += (double)F.p2m[b].ntask * (2 * F.P[b][L] + 1) * (2 * p + 1);
            // L2P: particle <- its leaf, v = x_m - c_leaf
            HostList l2p;
            l2p.ptr.assign(M + 1, 0);
            for (int m = 0; m < M; ++m) {
                l2p.ptr[m] = m;
                double cx, cy;
                centre(L, leaf[m], cx, cy);
                l2p.src.push_back(leaf[m]);
                l2p.seq.push_back(B.add(c[2 * m] - cx, c[2 * m + 1] - cy, k, p + 1 + F.P[b][L], 0));
            }
            l2p.ptr[M] = M;
            if ((rc = upload_list(h, l2p, F.l2p[b]))) return rc;
            F.work_far += (double)F.l2p[b].ntask * (2 * p + 1) * (2 * F.P[b][L] + 1);
            for (int lev = 2; lev <= L; ++lev) {
                int n = 1 << lev;
                double w = F.w[lev];
                // M2L table: offsets (dx, dy) in [-3, 3]^2 with max(|dx|,|dy|) >= 2
                long long tab[7][7];
                for (int dy = -3; dy <= 3; ++dy)
                    for (int dx = -3; dx <= 3; ++dx)
                        tab[dy + 3][dx + 3] = (std::max(abs(dx), abs(dy)) >= 2)
                                                  ? B.add(dx * w, dy * w, k, 2 * F.P[b][lev], 1) : -1;
                HostList m2l;
                m2l.ptr.assign(n * n + 1, 0);
                for (int id = 0; id < n * n; ++id) {
                    m2l.ptr[id] = (int)m2l.src.size();
                    if (!nonempty[lev][id]) continue;
                    int ix = id % n, iy = id / n;
                    int px = ix >> 1, py = iy >> 1;
                    for (int qy = py - 1; qy <= py + 1; ++qy)
                        for (int qx = px - 1; qx <= px + 1; ++qx) {
                            if (qx < 0 || qy < 0 || qx >= n / 2 || qy >= n / 2) continue;
                            for (int cyy = 0; cyy < 2; ++cyy)
                                for (int cxx = 0; cxx < 2; ++cxx) {
                                    int sx = 2 * qx + cxx, sy = 2 * qy + cyy;
                                    int dx = ix - sx, dy = iy - sy;
                                    if (std::max(abs(dx), abs(dy)) < 2) continue;
                                    int sid = sy * n + sx;
                                    if (!nonempty[lev][sid]) continue;
                                    m2l.src.push_back(sid);
                                    m2l.seq.push_back(tab[dy + 3][dx + 3]);
                                }
                        }
                }
                m2l.ptr[n * n] = (int)m2l.src.size();
                if ((rc = upload_list(h, m2l, F.m2l[b][lev]))) return rc;
                F.work_far += (double)F.m2l[b][lev].ntask * (2 * F.P[b][lev] + 1) * (2 * F.P[b][lev] + 1);
                if (h->opt.tensor_cores && (rc = ms_m2l_tc_tiles(h, b, lev, m2l.ptr))) return rc;
                if (lev < L) {
                    // M2M: parent (lev) <- children (lev+1); v = c_parent - c_child = (+-w/4, +-w/4)
                    int nc2 = 2 * n;
                    long long tabc[2][2], tabp[2][2];
                    for (int cyy = 0; cyy < 2; ++cyy)
                        for (int cxx = 0; cxx < 2; ++cxx) {
                            // c_parent - c_child: the child centre sits (cxx - 1/2) child widths
                            // from the parent centre
                            double vx = (0.5 - cxx) * F.w[lev + 1];
                            double vy = (0.5 - cyy) * F.w[lev + 1];
                            tabc[cyy][cxx] = B.add(vx, vy, k, F.P[b][lev] + F.P[b][lev + 1], 0);
                            tabp[cyy][cxx] = B.add(-vx, -vy, k, F.P[b][lev + 1] + F.P[b][lev], 0);
                        }
                    HostList m2m, l2l;
                    m2m.ptr.assign(n * n + 1, 0);
                    for (int id = 0; id < n * n; ++id) {
                        m2m.ptr[id] = (int)m2m.src.size();
                        int ix = id % n, iy = id / n;
                        for (int cyy = 0; cyy < 2; ++cyy)
                            for (int cxx = 0; cxx < 2; ++cxx) {
                                int cid = (2 * iy + cyy) * nc2 + 2 * ix + cxx;
                                if (!nonempty[lev + 1][cid]) continue;
                                m2m.src.push_back(cid);
                                m2m.seq.push_back(tabc[cyy][cxx]);
                            }
                    }
                    m2m.ptr[n * n] = (int)m2m.src.size();
                    l2l.ptr.assign(nc2 * nc2 + 1, 0);
                    for (int cid = 0; cid < nc2 * nc2; ++cid) {
                        l2l.ptr[cid] = (int)l2l.src.size();
                        if (!nonempty[lev + 1][cid]) continue;
                        int cx = cid % nc2, cy = cid / nc2;
                        l2l.src.push_back((cy / 2) * n + cx / 2);
                        l2l.seq.push_back(tabp[cy & 1][cx & 1]);
                    }
                    l2l.ptr[nc2 * nc2] = (int)l2l.src.size();
                    if ((rc = upload_list(h, m2m, F.m2m[b][lev])) || (rc = upload_list(h, l2l, F.l2l[b][lev + 1])))
                        return rc;
                    F.work_far += (double)(F.m2m[b][lev].ntask + F.l2l[b][lev + 1].ntask) * (2 * F.P[b][lev] + 1) *
                                  (2 * F.P[b][lev + 1] + 1);
                }
            }
        }
    }

    // ---------------------------------------------------------- sequences on the device
    h->seq_len = B.total;
    if (B.total == 0) return MS_OK;   // a single particle and no FMM: nothing to translate
    if (cudaMalloc(&h->d.seq64, B.total * sizeof(double2)) != cudaSuccess ||
        cudaMalloc(&h->d.seqm, B.total * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&h->d.seqe, B.total * sizeof(int)) != cudaSuccess)
        return MS_ERR_ALLOC;
    SeqSpec* dspec = nullptr;
    const size_t chunk = 1 << 20;
    if (cudaMalloc(&dspec, std::min(chunk, B.specs.size() + 1) * sizeof(SeqSpec)) != cudaSuccess) return MS_ERR_ALLOC;
    for (size_t s0 = 0; s0 < B.specs.size(); s0 += chunk) {
        size_t n = std::min(chunk, B.specs.size() - s0);
        if ((rc = ms_check(h, cudaMemcpy(dspec, B.specs.data() + s0, n * sizeof(SeqSpec), cudaMemcpyHostToDevice)))) {
            cudaFree(dspec);
            return rc;
        }
        k_gen_seq<<<(int)((n + 127) / 128), 128>>>(dspec, (int)n, h->d.seq64);
        if ((rc = ms_check(h, cudaGetLastError()))) { cudaFree(dspec); return rc; }
    }
    cudaFree(dspec);
    k_split_seq<<<(int)((B.total + 255) / 256), 256>>>(h->d.seq64, h->d.seqm, h->d.seqe, B.total);
    if ((rc = ms_check(h, cudaGetLastError()))) return rc;
    return ms_check(h, cudaDeviceSynchronize());
}

// Translation part of the operator in the scaled basis: a~ (workspace) = T~ xs (written, not
// accumulated).  Near pairs directly; with the FMM, far pairs through P2M, M2M, M2L, L2L, L2P.
// `near` / `far` select the two halves (both for the full T).
__global__ void k_zero_c(double2* a, long long n) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) a[i] = make_double2(0, 0);
}

template <typename T>
int ms_translate_gen(ms_handle* h, const void* xs, void* dst_, int nrhs, bool near, bool far, int adj, int deriv_axis,
                     bool unscaled, cudaStream_t st) {
    typedef typename CT<T>::c C;
    const bool f32 = sizeof(T) == 4;
    const int M = h->M, p = h->p, nc = h->nc;
    C* dst = (C*)dst_;
    const int* pexp = unscaled ? h->d.zexp : h->d.expo;      // particle exponents (zeros: unscaled)
    const long long pstride = unscaled ? 0 : 2 * nc;
    const double kb[2] = {h->kp_l, h->ks_l};
    int rc;
    auto set_deriv = [&](TransArgs& a, int b) {
        if (!deriv_axis) return;
        a.deriv = 1;
        double k = kb[b];
        if (deriv_axis == 1) { a.dc1 = make_double2(0.5 * k, 0.0); a.dc2 = make_double2(-0.5 * k, 0.0); }
        else { a.dc1 = make_double2(0.0, 0.5 * k); a.dc2 = make_double2(0.0, 0.5 * k); }
    };
    if (!near) {
        // far field only: start from zero
        long long n = (long long)M * 2 * nc * nrhs * (long long)sizeof(C) / (long long)sizeof(double2);
        k_zero_c<<<(int)((n + 255) / 256), 256, 0, st>>>((double2*)dst, n);
        if ((rc = ms_check(h, cudaGetLastError()))) return rc;
    }
    const bool tcore = f32 && !adj && !deriv_axis && !unscaled && h->opt.tensor_cores;
    const bool near_tc = near && tcore && h->fmm.near_tc.n > 0;
    if (near_tc && (rc = ms_near_tc_launch(h, (const float2*)xs, (float2*)dst, nrhs, st))) return rc;
    for (int b = 0; b < 2 && near && !near_tc; ++b) {
        TransArgs a{};
        const DevList& nl = h->fmm.near[b];
        a.dst_ptr = nl.ptr; a.task_src = nl.src; a.task_seq = nl.seq;
        a.K = 2 * p + 1; a.Pd = p; a.Ps = p;
        a.dst = dst + (long long)b * nc * nrhs; a.dst_stride = 2LL * nc * nrhs;
        a.src = (const C*)xs + (long long)b * nc * nrhs; a.src_stride = 2LL * nc * nrhs;
        a.ad = pexp + (unscaled ? 0 : b * nc); a.ad_stride = pstride; a.sd = 1;
        a.as = pexp + (unscaled ? 0 : b * nc); a.as_stride = pstride; a.ss = 1;
        a.nrhs = nrhs; a.accumulate = 0; a.adj = adj;
        set_deriv(a, b);
        if ((rc = ms_translate_launch(h, a, M, f32, st))) return rc;
    }
    const int L = h->fmm_levels;
    if (!L || !far) return MS_OK;
    FmmHost& F = h->fmm;
    for (int b = 0; b < 2; ++b) {
        auto mexp = [&](int lev) { return (C*)F.mexp[b][lev]; };
        auto lexp = [&](int lev) { return (C*)F.lexp[b][lev]; };
        auto ncl = [&](int lev) { return 2 * F.P[b][lev] + 1; };
        auto bexp = [&](int lev) { return unscaled ? (const int*)h->d.zexp : (const int*)F.expo[b][lev]; };
        // P2M
        {
            TransArgs a{};
            a.dst_ptr = F.p2m[b].ptr; a.task_src = F.p2m[b].src; a.task_seq = F.p2m[b].seq;
            a.Pd = F.P[b][L]; a.Ps = p; a.K = a.Pd + a.Ps;
            a.dst = mexp(L); a.dst_stride = (long long)ncl(L) * nrhs;
            a.src = (const C*)xs + (long long)b * nc * nrhs; a.src_stride = 2LL * nc * nrhs;
            a.ad = bexp(L); a.ad_stride = 0; a.sd = -1;
            a.as = pexp + (unscaled ? 0 : b * nc); a.as_stride = pstride; a.ss = 1;
            a.nrhs = nrhs; a.accumulate = 0; a.adj = adj;
            if ((rc = ms_translate_launch(h, a, F.p2m[b].ndst, f32, st))) return rc;
        }
        // M2M upward
        for (int lev = L - 1; lev >= 2; --lev) {
            TransArgs a{};
            a.dst_ptr = F.m2m[b][lev].ptr; a.task_src = F.m2m[b][lev].src; a.task_seq = F.m2m[b][lev].seq;
            a.Pd = F.P[b][lev]; a.Ps = F.P[b][lev + 1]; a.K = a.Pd + a.Ps;
            a.dst = mexp(lev); a.dst_stride = (long long)ncl(lev) * nrhs;
            a.src = mexp(lev + 1); a.src_stride = (long long)ncl(lev + 1) * nrhs;
            a.ad = bexp(lev); a.ad_stride = 0; a.sd = -1;
            a.as = bexp(lev + 1); a.as_stride = 0; a.ss = 1;
            a.nrhs = nrhs; a.accumulate = 0; a.adj = adj;
            if ((rc = ms_translate_launch(h, a, F.m2m[b][lev].ndst, f32, st))) return rc;
        }
        // M2L and L2L downward
        for (int lev = 2; lev <= L; ++lev) {
            TransArgs a{};
            a.dst_ptr = F.m2l[b][lev].ptr; a.task_src = F.m2l[b][lev].src; a.task_seq = F.m2l[b][lev].seq;
            a.Pd = F.P[b][lev]; a.Ps = F.P[b][lev]; a.K = 2 * a.Pd;
            a.dst = lexp(lev); a.dst_stride = (long long)ncl(lev) * nrhs;
            a.src = mexp(lev); a.src_stride = (long long)ncl(lev) * nrhs;
            a.ad = bexp(lev); a.ad_stride = 0; a.sd = 1;
            a.as = bexp(lev); a.as_stride = 0; a.ss = 1;
            a.nrhs = nrhs; a.accumulate = 0; a.adj = adj;
            if (tcore) {
                if ((rc = ms_m2l_tc_launch(h, b, lev, (const float2*)mexp(lev), (float2*)lexp(lev), nrhs, st))) return rc;
            } else if ((rc = ms_translate_launch(h, a, F.m2l[b][lev].ndst, f32, st))) {
                return rc;
            }
            if (lev > 2) {
                TransArgs c{};
                c.dst_ptr = F.l2l[b][lev].ptr; c.task_src = F.l2l[b][lev].src; c.task_seq = F.l2l[b][lev].seq;
                c.Pd = F.P[b][lev]; c.Ps = F.P[b][lev - 1]; c.K = c.Pd + c.Ps;
                c.dst = lexp(lev); c.dst_stride = (long long)ncl(lev) * nrhs;
                c.src = lexp(lev - 1); c.src_stride = (long long)ncl(lev - 1) * nrhs;
                c.ad = bexp(lev); c.ad_stride = 0; c.sd = 1;
                c.as = bexp(lev - 1); c.as_stride = 0; c.ss = -1;
                c.nrhs = nrhs; c.accumulate = 1; c.adj = adj;
                if ((rc = ms_translate_launch(h, c, F.l2l[b][lev].ndst, f32, st))) return rc;
            }
        }
        // L2P (in adjoint mode: the adjoint of P2M); the particle-position derivative acts here
        {
            TransArgs a{};
            a.dst_ptr = F.l2p[b].ptr; a.task_src = F.l2p[b].src; a.task_seq = F.l2p[b].seq;
            a.Pd = p; a.Ps = F.P[b][L]; a.K = p + 1 + F.P[b][L];
            a.dst = dst + (long long)b * nc * nrhs; a.dst_stride = 2LL * nc * nrhs;
            a.src = lexp(L); a.src_stride = (long long)ncl(L) * nrhs;
            a.ad = pexp + (unscaled ? 0 : b * nc); a.ad_stride = pstride; a.sd = 1;
            a.as = bexp(L); a.as_stride = 0; a.ss = -1;
            a.nrhs = nrhs; a.accumulate = 1; a.adj = adj;
            set_deriv(a, b);
            if ((rc = ms_translate_launch(h, a, M, f32, st))) return rc;
        }
    }
    return MS_OK;
}

template <typename T>
int ms_translate_scaled(ms_handle* h, const void* xs, int nrhs, bool near, bool far, cudaStream_t st) {
    return ms_translate_gen<T>(h, xs, h->ws_a, nrhs, near, far, 0, 0, false, st);
}

template int ms_translate_gen<double>(ms_handle*, const void*, void*, int, bool, bool, int, int, bool, cudaStream_t);
template int ms_translate_gen<float>(ms_handle*, const void*, void*, int, bool, bool, int, int, bool, cudaStream_t);
template int ms_translate_scaled<double>(ms_handle*, const void*, int, bool, bool, cudaStream_t);
template int ms_translate_scaled<float>(ms_handle*, const void*, int, bool, bool, cudaStream_t);

// Expansion buffers for nrhs columns (called from the workspace allocator).
int ms_fmm_workspace(ms_handle* h, int nrhs) {
    FmmHost& F = h->fmm;
    for (int b = 0; b < 2; ++b)
        for (int lev = 0; lev <= 12; ++lev) {
            if (F.mexp[b][lev]) cudaFree(F.mexp[b][lev]);
            if (F.lexp[b][lev]) cudaFree(F.lexp[b][lev]);
            F.mexp[b][lev] = F.lexp[b][lev] = nullptr;
        }
    for (int b = 0; b < 2; ++b)
        for (int lev = 2; lev <= h->fmm_levels; ++lev) {
            size_t n = (size_t)F.nbox[lev] * (2 * F.P[b][lev] + 1) * nrhs * sizeof(double2);
            if (cudaMalloc(&F.mexp[b][lev], n) != cudaSuccess || cudaMalloc(&F.lexp[b][lev], n) != cudaSuccess)
                return MS_ERR_ALLOC;
            cudaMemset(F.mexp[b][lev], 0, n);
            cudaMemset(F.lexp[b][lev], 0, n);
        }
    return MS_OK;
}

void ms_fmm_free(ms_handle* h) {
    FmmHost& F = h->fmm;
    F.work_near = F.work_far = 0;
    auto fl = [](DevList& D) { cudaFree(D.ptr); cudaFree(D.src); cudaFree(D.seq); D = DevList{}; };
    for (int b = 0; b < 2; ++b) {
        fl(F.near[b]); fl(F.p2m[b]); fl(F.l2p[b]);
        for (int lev = 0; lev <= 12; ++lev) {
            fl(F.m2m[b][lev]); fl(F.m2l[b][lev]); fl(F.l2l[b][lev]);
            cudaFree(F.expo[b][lev]); F.expo[b][lev] = nullptr;
            cudaFree(F.mexp[b][lev]); cudaFree(F.lexp[b][lev]);
            F.mexp[b][lev] = F.lexp[b][lev] = nullptr;
        }
    }
    ms_near_store_free(h);
    ms_tc_tiles_free(F.near_tc);
    for (int b = 0; b < 2; ++b)
        for (int lev = 0; lev <= 12; ++lev) ms_tc_tiles_free(F.m2l_tc[b][lev]);
    cudaFree(h->d.seq64); cudaFree(h->d.seqm); cudaFree(h->d.seqe);
    h->d.seq64 = nullptr; h->d.seqm = nullptr; h->d.seqe = nullptr;
}
