// gs_probe.cu -- gs_measure_alu_peaks: the FP32 FMA and ex2.approx throughput of the device, the
// measured denominator of the blend stage's roofline.
//
// Each thread runs kChains independent dependency chains so that the pipes stay full at any
// latency; the grid is a multiple of the SM count at full occupancy (kThreads x kCtasPerSm per SM).
// The chains' values are data dependent (seeded from the thread index) and their sum is stored
// only when it equals a value it can never take, so nothing is folded away and nothing is written.
#include <cstdio>
#include <cuda_runtime.h>

#include "gs.h"

namespace gs {
void set_error_message(const char *msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int kCtasPerSm = 8;          // 2048 threads per SM
constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(kThreads) k_probe_fma(float *sink, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0f) sink[threadIdx.x] = s;      // a <= 1, b >= 0: the chains stay >= 0
}

__device__ __forceinline__ float ex2_probe(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kThreads) k_probe_ex2(float *sink, int iters) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = -(float)((threadIdx.x + c) & 63) * (1.0f / 64.0f);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = ex2_probe(-x[c]);    // bounded: after two steps x stays in [1/4, 1]
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == -1.0f) sink[threadIdx.x] = s;
}

thread_local char g_msg[256];

gs_status fail(gs_status code, const char *what, cudaError_t e) {
    snprintf(g_msg, sizeof(g_msg), "%s: %s", what, cudaGetErrorString(e));
    gs::set_error_message(g_msg);
    return code;
}

// Runs one probe with `iters` loop trips and returns its event-timed duration in ms.
template <class Launch>
cudaError_t timed(Launch launch, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    cudaEventRecord(e0, s);
    launch();
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) return e;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaEventElapsedTime(ms, e0, e1);
}

}  // namespace

extern "C" gs_status gs_measure_alu_peaks(int32_t device, double target_ms, gs_alu_peaks *out) {
    if (!out) {
        gs::set_error_message("out is NULL");
        return GS_ERR_INVALID_ARG;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        gs::set_error_message("no such CUDA device");
        return GS_ERR_NO_DEVICE;
    }
    if (!(target_ms > 0.0)) target_ms = 200.0;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(device);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int grid = sms * kCtasPerSm;
    float *sink = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    gs_status st = GS_OK;
    cudaError_t e = cudaMalloc(&sink, kThreads * sizeof(float) * 4);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    double res[2] = {0, 0}, dur[2] = {0, 0};
    for (int probe = 0; probe < 2 && e == cudaSuccess; ++probe) {
        auto run = [&](int iters, float *ms) {
            return timed(
                [&] {
                    if (probe == 0)
                        k_probe_fma<<<grid, kThreads, 0, s>>>(sink, iters, 0.999f, 0.25f);
                    else
                        k_probe_ex2<<<grid, kThreads, 0, s>>>(sink, iters);
                },
                s, e0, e1, ms);
        };
        // calibrate: grow the trip count until one launch takes >= 5 ms, then scale to the target
        int iters = 64;
        float ms = 0.f;
        while (e == cudaSuccess) {
            e = run(iters, &ms);
            if (e != cudaSuccess || ms >= 5.0f || iters >= (1 << 24)) break;
            iters *= 4;
        }
        if (e != cudaSuccess) break;
        double scale = target_ms / (double)ms;
        long long it2 = (long long)(iters * scale);
        iters = (int)(it2 < 1 ? 1 : (it2 > (1 << 26) ? (1 << 26) : it2));
        e = run(iters, &ms);
        if (e != cudaSuccess) break;
        const double ops = (double)grid * kThreads * (double)iters * kUnroll * kChains;
        res[probe] = ops / (ms * 1e-3) / 1e12;
        dur[probe] = ms;
    }
    if (e != cudaSuccess) st = fail(GS_ERR_CUDA, "alu probe", e);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (sink) cudaFree(sink);
    cudaSetDevice(prev);
    if (st == GS_OK) {
        out->fma_tops = res[0];
        out->ex2_tops = res[1];
        out->fma_ms = dur[0];
        out->ex2_ms = dur[1];
        out->sm_count = sms;
        out->pad = 0;
    }
    return st;
}
