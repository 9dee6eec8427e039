// gs_mathcheck.cu -- gs_eval_decision_math: the binary32 functions whose bits decide pairs,
// evaluated by the very device code the preprocess kernel runs, over caller arrays.
//
// The pair set depends on t = 2 ln(alpha0 / tau) (Eq. 2-3) and, for raw parameters, on the
// exponential behind exp(log-scale) and sigmoid(logit).  These are the library's own binary32
// routines (range reduction plus a fixed polynomial, every operation explicitly rounded), so a
// host implementation of the same published method can reproduce them bit for bit; this entry
// point lets a test compare every input of a domain exhaustively.
#include <cstdio>

#include "gs_internal.cuh"

namespace gs {
void set_error_message(const char *msg);
}

using namespace gs;

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) k_decision_math(int fn, const float *__restrict__ x,
                                                            float *__restrict__ y, long long n, float param) {
    const long long stride = (long long)gridDim.x * kThreads;
    for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
        const float v = x[i];
        y[i] = fn == 0 ? threshold_t(v, param) : fn == 1 ? exp_rn(v) : sigmoid_rn(v);
    }
}

thread_local char g_msg[256];

gs_status fail(gs_status code) {
    set_error_message(g_msg);
    return code;
}

}  // namespace

extern "C" gs_status gs_eval_decision_math(int32_t fn, const float *x_dev, float *y_dev, int64_t n, float param,
                                           gs_stream stream) {
    if (fn < 0 || fn > 2) {
        snprintf(g_msg, sizeof(g_msg), "fn %d not 0, 1 or 2", fn);
        return fail(GS_ERR_INVALID_ARG);
    }
    if (n < 0) {
        snprintf(g_msg, sizeof(g_msg), "n = %lld is negative", (long long)n);
        return fail(GS_ERR_INVALID_ARG);
    }
    if (n == 0) return GS_OK;
    if (!x_dev || !y_dev) {
        snprintf(g_msg, sizeof(g_msg), "NULL array");
        return fail(GS_ERR_INVALID_ARG);
    }
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "device query: %s", cudaGetErrorString(e));
        return fail(GS_ERR_CUDA);
    }
    const long long want = (n + kThreads - 1) / kThreads;
    const long long cap = 8ll * (sms > 0 ? sms : 1);
    const unsigned grid = (unsigned)(want < cap ? want : cap);
    k_decision_math<<<grid, kThreads, 0, (cudaStream_t)stream>>>(fn, x_dev, y_dev, n, param);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        snprintf(g_msg, sizeof(g_msg), "launch: %s", cudaGetErrorString(e));
        return fail(GS_ERR_CUDA);
    }
    return GS_OK;
}
