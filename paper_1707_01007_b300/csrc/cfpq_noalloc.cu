// Pair extraction that allocates nothing (cfpq_extract_pairs_noalloc).
//
// Some callers cannot allocate device memory themselves: code running under an external
// memory manager that owns the whole device heap, allocation-free real-time paths, or
// plug-ins whose host forbids cudaMalloc after start-up. For them this file provides a
// variant of the library's pair extraction (per-row popcount, exclusive scan, emission
// of (A, m, n) triples in row-major order) whose scratch -- the per-row counts and
// offsets and the total -- lives in one file-scope device array instead of memory the
// library would allocate. The caller passes the bit-packed matrix and the output buffer.
//
// The array is a property of the loaded library: every GPU that loads it holds the array
// (kScratchBytes) until the process exits, and all calls on a device share it. A call
// overwrites every part of the array it reads before reading it, so nothing carries over
// from the previous call, but two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on the array and must be serialised by the
// caller.
//
// In host code the array's name is only a host-side stand-in, not a device address; the
// device address is looked up with cudaGetSymbolAddress while the device is current, once
// per device and CUDA context (a device reset, or a primary context released and created
// again, loads the module anew and gets a new context id, so the address is looked up
// again), and passed to the kernels.
//
// Every call synchronises its stream and reads the total on the host, so it cannot be
// part of a stream capture: a call on a capturing stream is refused before any device work.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "../../include/cfpq.h"

namespace cfpq {
namespace noalloc {

constexpr uint32_t kMaxRows = CFPQ_NOALLOC_MAX_ROWS;
// layout: [total: 8 B, padded to 256][offsets: kMaxRows x 8 B][counts: kMaxRows x 4 B]
constexpr size_t kOffsetsAt = 256;
constexpr size_t kCountsAt = kOffsetsAt + (size_t)kMaxRows * 8;
constexpr size_t kScratchBytes = kCountsAt + (size_t)kMaxRows * 4;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
static unsigned char *g_dev_ptr[kMaxDevices];
static unsigned long long g_dev_ctx[kMaxDevices];  // context id the cached address belongs to
static std::mutex g_mu;

__device__ __forceinline__ uint32_t masked_word(const uint32_t *row, uint32_t w, uint32_t n_cols) {
    uint32_t x = row[w];
    const uint32_t lo = w * 32u;
    if (lo + 32u > n_cols) x = (lo >= n_cols) ? 0u : (x & ((1u << (n_cols - lo)) - 1u));
    return x;
}

__global__ void k_count(const uint32_t *bits, uint32_t n_rows, uint32_t n_cols, uint32_t row_words,
                        unsigned char *scratch) {
    uint32_t *counts = reinterpret_cast<uint32_t *>(scratch + kCountsAt);
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_rows) return;
    const uint32_t *row = bits + warp * row_words;
    uint32_t c = 0;
    for (uint32_t w = lane; w < row_words; w += 32) c += __popc(masked_word(row, w, n_cols));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) counts[warp] = c;
}

__global__ void __launch_bounds__(1024) k_scan(uint32_t n_rows, unsigned char *scratch) {
    const uint32_t *counts = reinterpret_cast<const uint32_t *>(scratch + kCountsAt);
    unsigned long long *offsets = reinterpret_cast<unsigned long long *>(scratch + kOffsetsAt);
    unsigned long long *total = reinterpret_cast<unsigned long long *>(scratch);
    __shared__ unsigned long long part[1024];
    const uint32_t per = (n_rows + 1023) / 1024;
    const uint32_t lo = threadIdx.x * per, hi = min(n_rows, lo + per);
    unsigned long long s = 0;
    for (uint32_t i = lo; i < hi; i++) s += counts[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const unsigned long long v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0ull;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = part[threadIdx.x] - s;
    for (uint32_t i = lo; i < hi; i++) {
        offsets[i] = run;
        run += counts[i];
    }
    if (threadIdx.x == 1023) *total = part[1023];
}

__global__ void k_emit(const uint32_t *bits, uint32_t n_rows, uint32_t n_cols, uint32_t row_words, int32_t a,
                       const unsigned char *scratch, cfpq_triple *out) {
    const uint32_t *counts = reinterpret_cast<const uint32_t *>(scratch + kCountsAt);
    const unsigned long long *offsets = reinterpret_cast<const unsigned long long *>(scratch + kOffsetsAt);
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= n_rows || counts[warp] == 0) return;
    const uint32_t *row = bits + warp * row_words;
    unsigned long long off = offsets[warp];
    for (uint32_t w0 = 0; w0 < row_words; w0 += 32) {
        uint32_t x = (w0 + lane < row_words) ? masked_word(row, w0 + lane, n_cols) : 0u;
        const uint32_t c = __popc(x);
        uint32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        unsigned long long pos = off + incl - c;
        while (x) {
            const uint32_t j = (w0 + lane) * 32u + (uint32_t)(__ffs(x) - 1);
            x &= x - 1;
            out[pos++] = cfpq_triple{a, (uint32_t)warp, j};
        }
        off += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// Unique id of the CUDA context current on this thread (cuCtxGetId), 0 if there is none yet
// or the driver entry points are unavailable.
static unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &qr) == cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &qr) == cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
        cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array on the current device: looked up once per device and
// context (every call where the context id cannot be read).
static int scratch_address(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CFPQ_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long ctx = current_context_id();
    if (ctx != 0 && g_dev_ptr[dev] && g_dev_ctx[dev] == ctx) {
        *out = g_dev_ptr[dev];
        return CFPQ_OK;
    }
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return CFPQ_ERR_CUDA;
    }
    // the look-up makes the device's primary context current if it was not yet
    const unsigned long long ctx_now = ctx != 0 ? ctx : current_context_id();
    g_dev_ptr[dev] = ctx_now != 0 ? static_cast<unsigned char *>(p) : nullptr;
    g_dev_ctx[dev] = ctx_now;
    *out = static_cast<unsigned char *>(p);
    return CFPQ_OK;
}

}  // namespace noalloc
}  // namespace cfpq

extern "C" int cfpq_extract_pairs_noalloc(const uint32_t *bits, uint32_t n_rows, uint32_t n_cols,
                                          uint32_t row_words, int32_t A, cfpq_triple *out, size_t cap,
                                          size_t *count, void *stream) {
    using namespace cfpq::noalloc;
    if (!count || (!bits && n_rows > 0)) return CFPQ_ERR_INVALID;
    if (n_rows > kMaxRows) return CFPQ_ERR_INVALID;  // beyond the fixed scratch array
    if ((uint64_t)row_words * 32u < n_cols) return CFPQ_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the call synchronises the stream: never inside a stream capture (on the legacy stream
    // while another stream captures, the query itself reports an error: refused as well)
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap_status) != cudaSuccess) {
        cudaGetLastError();
        return CFPQ_ERR_INVALID;
    }
    if (cap_status != cudaStreamCaptureStatusNone) return CFPQ_ERR_INVALID;
    if (n_rows == 0) {
        *count = 0;
        return CFPQ_OK;
    }
    unsigned char *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != CFPQ_OK) return rc;
    const uint32_t blocks = (uint32_t)(((uint64_t)n_rows * 32 + 255) / 256);
    k_count<<<blocks, 256, 0, s>>>(bits, n_rows, n_cols, row_words, scratch);
    k_scan<<<1, 1024, 0, s>>>(n_rows, scratch);
    unsigned long long total = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&total, scratch, sizeof(total), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CFPQ_ERR_CUDA;
    *count = (size_t)total;
    if (!out) return CFPQ_OK;
    if (cap < total) return CFPQ_ERR_BUFFER;
    if (total == 0) return CFPQ_OK;
    k_emit<<<blocks, 256, 0, s>>>(bits, n_rows, n_cols, row_words, A, scratch, out);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return CFPQ_ERR_CUDA;
    return CFPQ_OK;
}
