// Measured peaks of the warp-level integer tensor instructions (mma.sync): on sm_103a the
// 8-bit integer and 1-bit AND/popc tensor paths exist only in this legacy form (tcgen05
// has no 8-bit integer kind there), so they are the integer references against which the
// Boolean product's throughput is also reported. Each warp runs independent accumulator
// chains of one instruction back to back; operand values do not matter for the rate.
#include "cfpq_internal.h"

namespace cfpq {
namespace peaks {

constexpr int kChains = 8;          // independent accumulators per warp (covers the MMA latency)
constexpr int kBlocksPerSM = 4, kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_mma_s8(int iters, int *sink) {
    uint32_t a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; i++) a[i] = (threadIdx.x + 1u) * 0x01010101u + (uint32_t)i;
    b[0] = threadIdx.x * 0x00010203u;
    b[1] = ~b[0];
    int d[kChains][4];
#pragma unroll
    for (int c = 0; c < kChains; c++) d[c][0] = d[c][1] = d[c][2] = d[c][3] = c;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kChains; c++)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
                "{%0, %1, %2, %3};"
                : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) acc ^= d[c][0] ^ d[c][1] ^ d[c][2] ^ d[c][3];
    if (acc == 0x7ffffff1) sink[0] = acc;  // keeps the results live
}

__global__ void __launch_bounds__(kThreads) k_mma_b1(int iters, int *sink) {
    uint32_t a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; i++) a[i] = (threadIdx.x + 7u) * 0x9E3779B9u + (uint32_t)i;
    b[0] = threadIdx.x * 0x85EBCA6Bu;
    b[1] = ~b[0];
    int d[kChains][4];
#pragma unroll
    for (int c = 0; c < kChains; c++) d[c][0] = d[c][1] = d[c][2] = d[c][3] = c;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int c = 0; c < kChains; c++)
            asm volatile(
                "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                "{%8, %9}, {%0, %1, %2, %3};"
                : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
    int acc = 0;
#pragma unroll
    for (int c = 0; c < kChains; c++) acc ^= d[c][0] ^ d[c][1] ^ d[c][2] ^ d[c][3];
    if (acc == 0x7ffffff1) sink[0] = acc;
}

// Device time of one launch of kernel `fn` (after one warm-up launch), in ms.
template <typename K>
static int time_launch(K fn, int grid, int iters, int *sink, float *ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CFPQ_ERR_CUDA;
    fn<<<grid, kThreads>>>(iters / 8 > 0 ? iters / 8 : 1, sink);
    cudaEventRecord(e0);
    fn<<<grid, kThreads>>>(iters, sink);
    cudaEventRecord(e1);
    const cudaError_t e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) cudaEventElapsedTime(ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return e == cudaSuccess && cudaGetLastError() == cudaSuccess ? CFPQ_OK : CFPQ_ERR_CUDA;
}

}  // namespace peaks
}  // namespace cfpq

using namespace cfpq;

extern "C" int cfpq_measure_mma_sync_peaks(double *s8_tops, double *b1_tops) {
    if (!s8_tops || !b1_tops) return CFPQ_ERR_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CFPQ_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) return CFPQ_ERR_CUDA;
    int *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(int)) != cudaSuccess) return CFPQ_ERR_NOMEM;
    const int grid = sms * peaks::kBlocksPerSM;
    const double mmas_per_iter = (double)grid * (peaks::kThreads / 32) * peaks::kChains;
    const int it_s8 = 16384, it_b1 = 4096;
    float ms = 0.f;
    int rc = peaks::time_launch(peaks::k_mma_s8, grid, it_s8, sink, &ms);
    if (rc == CFPQ_OK) *s8_tops = mmas_per_iter * it_s8 * (2.0 * 16 * 8 * 32) / (ms * 1e-3) / 1e12;
    if (rc == CFPQ_OK) rc = peaks::time_launch(peaks::k_mma_b1, grid, it_b1, sink, &ms);
    if (rc == CFPQ_OK) *b1_tops = mmas_per_iter * it_b1 * (2.0 * 16 * 8 * 256) / (ms * 1e-3) / 1e12;
    cudaFree(sink);
    return rc;
}
