// Tensor-core throughput microkernel: the dense MMA rate of this GPU for the two operand kinds the
// operator uses (kind::tf32 and kind::f16 with bf16 inputs), measured with the same instruction shapes
// (M = 128, N = 256, K-major no-swizzle shared-memory operands, FP32 accumulation in tensor memory).
// One CTA per SM; one thread issues `iters` groups of MMAs over a 32-deep K chunk and commits each
// group to one of four mbarriers in turn, waiting (bounded) on the group issued three before, so that
// up to four groups are in flight.  The operand contents do not matter to the rate; shared memory is
// zeroed.
#include "common.cuh"
#include "handle.h"
#include "tc_pipeline.cuh"

namespace {

template <class K>
__global__ void __launch_bounds__(128, 1) k_mma_rate(int iters, int* err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + tcp::STAGE);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 4);
    for (int i = threadIdx.x; i < (int)(tcp::STAGE / 16); i += blockDim.x)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        for (int b = 0; b < 4; ++b) tc::mbar_init(&bar[b], 1);
        tc::mbar_fence_init();
    }
    if (threadIdx.x < 32) tc::tmem_alloc(tslot, tcp::TMEM_COLS);
    tc::fence_proxy_async();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    if (threadIdx.x == 0) {
        const tcp::StageT<K> st = tcp::stage_ptrs<K>(smem, 0);
        const uint32_t idesc = K::idesc(tcp::MA, tcp::NMAX);
        const uint32_t a0 = tc::smem_u32(st.ah), b0 = tc::smem_u32(st.bh);
        bool ok = true;
        for (int it = 0; it < iters && ok; ++it) {
#pragma unroll
            for (int ks = 0; ks < tcp::KC / K::KMMA; ++ks)
                K::mma(tmem, tc::smem_desc(a0 + ks * 256, tcp::LBO, K::SBO_), tc::smem_desc(b0 + ks * 256, tcp::LBO, K::SBO_),
                       idesc, (it > 0 || ks > 0) ? 1u : 0u);
            tc::mma_commit(&bar[it & 3]);
            // group g completes phase (g >> 2) & 1 of barrier g & 3
            if (it >= 3 && !tc::mbar_wait(&bar[(it - 3) & 3], ((it - 3) >> 2) & 1)) ok = false;
        }
        // the last commit covers every group before it
        if (ok && !tc::mbar_wait(&bar[(iters - 1) & 3], ((iters - 1) >> 2) & 1)) ok = false;
        if (!ok) atomicExch(err, 1);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x < 32) tc::tmem_free(tmem, tcp::TMEM_COLS);
}

}  // namespace

extern "C" int ms_tensor_peak(int32_t kind, int32_t iters, double* tflops, double* ms) {
    if ((kind != MS_PREC_FP32 && kind != MS_PREC_BF16) || iters < 1 || !tflops) return MS_ERR_ARG;
    int dev = 0, nsm = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)))
        return MS_ERR_CUDA;
    int* err = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc(&err, 2 * sizeof(int)) != cudaSuccess) return MS_ERR_ALLOC;
    cudaMemset(err, 0, 2 * sizeof(int));
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const size_t smem = tcp::STAGE + 64;
    auto launch = [&](int n) {
        if (kind == MS_PREC_BF16) {
            cudaFuncSetAttribute(k_mma_rate<tcp::BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_mma_rate<tcp::BF16><<<nsm, 128, smem>>>(n, err);
        } else {
            cudaFuncSetAttribute(k_mma_rate<tcp::TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_mma_rate<tcp::TF32><<<nsm, 128, smem>>>(n, err);
        }
    };
    launch(std::min(iters, 64));                     // warm-up
    cudaEventRecord(e0);
    launch(iters);
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return MS_ERR_CUDA;
    if (herr) return MS_ERR_TIMEOUT;
    // each MMA: 2 M N K flops with K = KMMA values; KC values per group
    const double flops = 2.0 * tcp::MA * tcp::NMAX * tcp::KC * (double)iters * nsm;
    *tflops = flops / (t * 1e-3) / 1e12;
    if (ms) *ms = t;
    return MS_OK;
}
