// Measured dense rate of the two tcgen05 MMA kinds the Boolean product can use on sm_103a,
// with the tile shape of the product kernels (M = 128, N = 256, A in tensor memory, B in
// 128-byte-swizzled K-major shared memory, F32 accumulator in tensor memory):
//   kind::f8f6f4             E4M3 x E4M3, K = 32 per instruction
//   kind::mxf4.block_scale   E2M1 x E2M1 (packed, two per byte) with UE8M0 scale factors
//                            per 32 K elements (scale_vec::2X), K = 64 per instruction
// One CTA per SM; one thread issues the MMAs back to back (4 instructions per 128-byte K
// row of the operands, repeated), the others only set up the operands. Every operand is
// 1.0 (and every scale factor 2^0), so after r instructions each accumulator element must
// be exactly r K: the probe also checks that the kind's operand encoding, instruction
// descriptor and scale-factor set-up are what the product kernels assume. The MMA-only
// rate is the ceiling of a product kernel of that kind (it unpacks nothing).
#include "cfpq_tcgen05.cuh"

namespace cfpq {
namespace tc {
namespace probe {

constexpr int kThreads = 128;
constexpr uint32_t kACol = 256, kSfaCol = 384, kSfbCol = 416, kTmemCols = 512;
constexpr size_t kSmemBytes = 116 * 1024;  // more than half of an SM: one CTA per SM

// kind::f8f6f4, E4M3 x E4M3 -> F32, K-major, M = 128, N = 256 (bits 4-5: D is F32)
constexpr uint32_t kIdescF8 = (1u << 4) | (0u << 7) | (0u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24);
// kind::mxf4 block-scaled: bits 4-5 the B scale-factor id (0), 7-9 / 10-12 A / B type
// (E2M1 = 1), 17-22 N >> 3, 23 scale type (UE8M0 = 1), 24-28 M >> 4, 29-30 the A
// scale-factor id (0)
constexpr uint32_t kIdescF4 = (1u << 7) | (1u << 10) | ((256u >> 3) << 17) | (1u << 23) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_f8(uint32_t d, uint32_t a, uint64_t bd, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
        "r"(a), "l"(bd), "r"(kIdescF8), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_f4(uint32_t d, uint32_t a, uint64_t bd, uint32_t sfa, uint32_t sfb, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
        " tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], [%1], %2, %3, [%4], [%5], p;\n}" ::"r"(d),
        "r"(a), "l"(bd), "r"(kIdescF4), "r"(sfa), "r"(sfb), "r"(acc)
        : "memory");
}

template <int KIND>  // 0: kind::f8f6f4, 1: kind::mxf4
__global__ void __launch_bounds__(kThreads, 1) k_tc_rate(int iters, int *bad, unsigned long long *cycles) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *b_tile = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) unsigned long long done;
    const int warp = threadIdx.x >> 5;
    const uint32_t one4 = KIND == 0 ? 0x38383838u : 0x22222222u;  // four E4M3 1.0 / eight E2M1 1.0
    for (int i = threadIdx.x; i < 256 * 128 / 16; i += kThreads)
        reinterpret_cast<uint4 *>(b_tile)[i] = make_uint4(one4, one4, one4, one4);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(&done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;  // this warp's quadrant of lanes
    uint32_t v[32];
#pragma unroll
    for (int j = 0; j < 32; j++) v[j] = one4;
    tmem_st32(tmem + lanes + kACol, v);  // A: 128 lanes x 128 bytes
    if (KIND == 1) {
#pragma unroll
        for (int j = 0; j < 32; j++) v[j] = 0x7F7F7F7Fu;  // UE8M0 127 = 2^0
        tmem_st32(tmem + lanes + kSfaCol, v);
        tmem_st32(tmem + lanes + kSfbCol, v);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
        const uint32_t b0 = sa(b_tile);
        const unsigned long long t0 = clock64();
        for (int it = 0; it < iters; it++)
#pragma unroll
            for (int kk = 0; kk < 4; kk++) {
                const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                if (KIND == 0)
                    mma_f8(tmem, tmem + kACol + kk * 8, sdesc(b0 + kk * 32), acc);
                else
                    mma_f4(tmem, tmem + kACol + kk * 8, sdesc(b0 + kk * 32), tmem + kSfaCol, tmem + kSfbCol, acc);
            }
        mma_commit(&done);
        volatile int e = 0;
        if (!mbar_wait(&done, 0u, &e, 10ull * 1000 * 1000 * 1000)) atomicAdd(bad, 1 << 20);
        const unsigned long long t1 = clock64();
        if (blockIdx.x == 0) *cycles = t1 - t0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const float expect = (float)iters * 4.0f * (KIND == 0 ? 32.0f : 64.0f);
    tmem_ld32(tmem + lanes, v);  // accumulator columns 0..31 of this warp's lanes
    int wrong = 0;
#pragma unroll
    for (int j = 0; j < 32; j++) wrong += __uint_as_float(v[j]) != expect;
    tmem_ld32(tmem + lanes + 224, v);  // and the last 32 columns
#pragma unroll
    for (int j = 0; j < 32; j++) wrong += __uint_as_float(v[j]) != expect;
    if (wrong) atomicAdd(bad, wrong);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

template <int KIND>
static int measure(int sms, int iters, double *tflops, double *per_clk, int *exact) {
    auto fn = k_tc_rate<KIND>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes) != cudaSuccess)
        return CFPQ_ERR_CUDA;
    int *bad = nullptr;
    unsigned long long *cyc = nullptr;
    if (cudaMalloc(&bad, sizeof(int)) != cudaSuccess) return CFPQ_ERR_NOMEM;
    if (cudaMalloc(&cyc, sizeof(unsigned long long)) != cudaSuccess) {
        cudaFree(bad);
        return CFPQ_ERR_NOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = CFPQ_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = CFPQ_ERR_CUDA;
    int h_bad = 0;
    unsigned long long h_cyc = 0;
    float ms = 0.f;
    if (rc == CFPQ_OK) {
        cudaMemset(bad, 0, sizeof(int));
        fn<<<sms, kThreads, kSmemBytes>>>(iters / 8 > 0 ? iters / 8 : 1, bad, cyc);  // warm-up
        cudaEventRecord(e0);
        fn<<<sms, kThreads, kSmemBytes>>>(iters, bad, cyc);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaMemcpy(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&h_cyc, cyc, sizeof(h_cyc), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = CFPQ_ERR_CUDA;
    }
    if (rc == CFPQ_OK) {
        const double ops = (double)iters * 4.0 * 2.0 * 128.0 * 256.0 * (KIND == 0 ? 32.0 : 64.0);
        *tflops = (double)sms * ops / (ms * 1e-3) / 1e12;
        *per_clk = h_cyc ? ops / (double)h_cyc : 0.0;
        *exact = h_bad == 0 ? 1 : 0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(bad);
    cudaFree(cyc);
    return rc;
}

}  // namespace probe
}  // namespace tc
}  // namespace cfpq

extern "C" int cfpq_measure_tensor_peaks(cfpq_tensor_peaks *out) {
    using namespace cfpq::tc::probe;
    if (!out) return CFPQ_ERR_INVALID;
    int dev = 0, sms = 0;
    cudaDeviceProp p;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess) return CFPQ_ERR_CUDA;
    if (p.major != 10 || p.minor != 3) return CFPQ_ERR_UNSUPPORTED;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) return CFPQ_ERR_CUDA;
    *out = cfpq_tensor_peaks{};
    int rc = measure<0>(sms, 16384, &out->f8f6f4_tflops, &out->f8f6f4_ops_per_clk_sm, &out->f8f6f4_exact);
    if (rc == CFPQ_OK) rc = measure<1>(sms, 16384, &out->mxf4_tflops, &out->mxf4_ops_per_clk_sm, &out->mxf4_exact);
    return rc;
}
