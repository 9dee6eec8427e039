// gs_noalloc.cu -- gs_sort_pairs_noalloc: the stand-alone radix sort of gs_sort_pairs with its
// scratch (digit histograms, digit offsets, look-back descriptors, tickets) in one fixed device
// array defined in this file, so that the call itself allocates nothing.
//
// Who needs it: code that is handed device buffers by a host application which owns the whole
// device-memory budget (an embedded renderer, a plugin, a real-time loop) and is not allowed to
// call cudaMalloc/cudaFree: those calls can synchronise the device, and fail outright when the
// host application has already reserved all memory for its own pool.
//
// The array is part of the library's device image: every GPU that loads the library holds it
// (kScratchBytes below, about 2 MiB) until the process exits.  In host code the array's name is
// only a host-side stand-in, not a device address, so the device address is looked up once per
// device with cudaGetSymbolAddress and passed to the kernels.
#include <cstddef>
#include <cstdio>
#include <mutex>

#include "gs_internal.cuh"

namespace gs {
void set_error_message(const char *msg);   // gs_last_error() text, defined with the C ABI
}

using namespace gs;

namespace {

constexpr long long kNoAllocMaxPairs = 1ll << 21;                 // 2,097,152 pairs
constexpr size_t kCtrWords = (sizeof(FrameCounters) + 7) / 8;     // tickets, epoch, status
constexpr size_t kHistWords = (8 * 256 * sizeof(unsigned)) / 8;   // one [8][256] u32 table
constexpr size_t kDescTiles = 960;   // tiles of 3072 pairs: room for kNoAllocMaxPairs (683 tiles)
constexpr size_t kDescWords = (kDescTiles + kDescTiles / 16) * 256;  // look-back descriptors (tile + block)
constexpr size_t kScratchWords = kCtrWords + 2 * kHistWords + kDescWords;
constexpr size_t kScratchBytes = kScratchWords * 8;
static_assert(kScratchBytes <= (2u << 20) + (32u << 10), "the fixed scratch stays near 2 MiB");

// Shared by every call on a device; zero at module load.
static __device__ __align__(256) unsigned long long g_sort_scratch[kScratchWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned long long *g_scratch_dev[kMaxDevices] = {};              // device address per device

thread_local char g_msg[256];

gs_status report(gs_status code) {
    set_error_message(g_msg);
    return code;
}

}  // namespace

extern "C" gs_status gs_sort_pairs_noalloc(uint64_t *keys, uint32_t *vals, uint64_t *keys_tmp, uint32_t *vals_tmp,
                                           int64_t n, int32_t end_bit, int32_t *in_tmp, gs_stream stream) {
    g_msg[0] = 0;
    if (!in_tmp) {
        snprintf(g_msg, sizeof(g_msg), "in_tmp is NULL");
        return report(GS_ERR_INVALID_ARG);
    }
    if (n < 0) {
        snprintf(g_msg, sizeof(g_msg), "n = %lld is negative", (long long)n);
        return report(GS_ERR_INVALID_ARG);
    }
    if (n > kNoAllocMaxPairs) {
        snprintf(g_msg, sizeof(g_msg), "n = %lld exceeds the no-allocation sort's maximum of %lld pairs",
                 (long long)n, kNoAllocMaxPairs);
        return report(GS_ERR_CAPACITY);
    }
    if (end_bit < 1 || end_bit > 64) {
        snprintf(g_msg, sizeof(g_msg), "end_bit %d not in 1..64", end_bit);
        return report(GS_ERR_INVALID_ARG);
    }
    if (n > 0 && (!keys || !vals || !keys_tmp || !vals_tmp)) {
        snprintf(g_msg, sizeof(g_msg), "NULL buffer");
        return report(GS_ERR_INVALID_ARG);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "cudaGetDevice: %s", cudaGetErrorString(e));
        return report(GS_ERR_CUDA);
    }
    if (dev < 0 || dev >= kMaxDevices) {
        snprintf(g_msg, sizeof(g_msg), "device %d: the allocation-free sort serves devices 0..%d", dev,
                 kMaxDevices - 1);
        return report(GS_ERR_INVALID_ARG);
    }
    unsigned long long *base = nullptr;
    {
        // first call on a device: look the array's device address up with that device current
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_dev[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_sort_scratch);
            if (e != cudaSuccess || !p) {
                snprintf(g_msg, sizeof(g_msg), "cudaGetSymbolAddress(sort scratch): %s", cudaGetErrorString(e));
                return report(GS_ERR_CUDA);
            }
            g_scratch_dev[dev] = (unsigned long long *)p;
        }
        base = g_scratch_dev[dev];
    }
    SortScratch scr;
    FrameCounters *ctr = (FrameCounters *)base;
    scr.hist = (unsigned *)(base + kCtrWords);
    scr.offs = (unsigned *)(base + kCtrWords + kHistWords);
    scr.desc = base + kCtrWords + 2 * kHistWords;
    scr.max_tiles = (long long)kDescTiles;
    if (sort_max_tiles_for(n > 0 ? n : 1) > scr.max_tiles) {
        snprintf(g_msg, sizeof(g_msg), "descriptor area too small for %lld pairs", (long long)n);
        return report(GS_ERR_CAPACITY);
    }
    cudaStream_t s = (cudaStream_t)stream;
    // The array keeps the previous call's contents: clear the histograms and the tickets/status
    // (the look-back descriptors are tagged with a per-sort epoch and need no clearing).
    e = cudaMemsetAsync(scr.hist, 0, kHistWords * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, offsetof(FrameCounters, sort_epoch), s);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "clearing sort scratch: %s", cudaGetErrorString(e));
        return report(GS_ERR_CUDA);
    }
    const int passes = launch_sort((unsigned long long *)keys, vals, (unsigned long long *)keys_tmp, vals_tmp,
                                   nullptr, n, n, end_bit, scr, ctr, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "sort launch: %s", cudaGetErrorString(e));
        return report(GS_ERR_CUDA);
    }
    *in_tmp = passes & 1;
    return GS_OK;
}

extern "C" gs_status gs_sort_pairs_noalloc_status(gs_stream stream) {
    g_msg[0] = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        snprintf(g_msg, sizeof(g_msg), "no usable current device");
        return report(GS_ERR_CUDA);
    }
    unsigned long long *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        base = g_scratch_dev[dev];
    }
    if (!base) {
        snprintf(g_msg, sizeof(g_msg), "no allocation-free sort has run on device %d", dev);
        return report(GS_ERR_INVALID_ARG);
    }
    e = cudaStreamSynchronize((cudaStream_t)stream);
    unsigned status = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&status, (const char *)base + offsetof(FrameCounters, status), sizeof(status),
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "reading the sort status: %s", cudaGetErrorString(e));
        return report(GS_ERR_CUDA);
    }
    if (status & kStTimeout) {
        snprintf(g_msg, sizeof(g_msg), "a bounded wait of the last allocation-free sort gave up: its output is invalid");
        return report(GS_ERR_DEVICE_TIMEOUT);
    }
    return GS_OK;
}
