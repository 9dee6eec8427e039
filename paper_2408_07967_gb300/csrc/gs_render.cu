// gs_render.cu -- per-tile front-to-back alpha blending (the render stage of Section 2.2, with
// the Section 5.2 / 5.3.2 ideas: staged Gaussian batches, one CTA-wide vote to stop, the
// exponent folded into one FMA in the log2 domain and evaluated by ex2.approx.ftz.f32).
//
// Per pixel sample (i + 1/2, j + 1/2) and list entry (u, v, a, b2, c, t, G, rgb):
//   q = fma(fma(a, dx, b2 dy), dx, (c dy) dy)     (binary32; skip the entry when !(q <= t))
//   alpha = min(alpha_max, 2^(G - q log2(e)/2))   (G = log2 alpha0, so alpha = alpha0 e^(-q/2))
//   T' = T (1 - alpha); stop before the entry if T' < T_min; C += rgb alpha T; T = T'.
#include "gs_internal.cuh"

namespace gs {

constexpr int kBlendThreads = 256;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(kBlendThreads) k_blend(const __grid_constant__ BlendArgs A) {
    __shared__ float4 s_r0[kBlendThreads];
    __shared__ float4 s_r1[kBlendThreads];
    __shared__ float2 s_r2[kBlendThreads];
    const int tile = blockIdx.x;
    const int tx = tile % A.tiles_x, ty = tile / A.tiles_x;
    const int px = tx * kTile + (threadIdx.x & 15), py = ty * kTile + (threadIdx.x >> 4);
    const bool inside = px < A.W && py < A.H;
    long long n = (long long)*A.n_dev;
    if (n > A.cap) n = A.cap;
    const long long start = min((long long)A.starts[tile], n);
    const long long end = min((long long)A.starts[tile + 1], n);
    const float fpx = (float)px + 0.5f, fpy = (float)py + 0.5f;
    const float HALF_LOG2E = 0.72134752044448170f;
    const float amax = A.opt.alpha_max, tmin = A.opt.T_min;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    unsigned last = 0;
    bool done = !inside;
    for (long long b = start; b < end; b += kBlendThreads) {
        if (__syncthreads_count(!done) == 0) break;
        const long long i = b + threadIdx.x;
        if (i < end) {
            const unsigned g = A.vals[i];
            const Rec r = A.recs[g];
            s_r0[threadIdx.x] = r.r0;
            s_r1[threadIdx.x] = r.r1;
            s_r2[threadIdx.x] = make_float2(r.r2.x, r.r2.y);
        }
        __syncthreads();
        const int cnt = (int)min((long long)kBlendThreads, end - b);
        if (!done) {
            for (int j = 0; j < cnt; ++j) {
                const float4 r0 = s_r0[j];
                const float4 r1 = s_r1[j];
                const float dx = fsub(fpx, r0.x);
                const float dy = fsub(fpy, r0.y);
                const float q = pixel_q(r0.z, r0.w, r1.x, dx, dy);
                if (!(q <= r1.y)) continue;
                const float al = fminf(amax, ex2_approx(fmaf(q, -HALF_LOG2E, r1.z)));
                const float Tn = T * (1.0f - al);
                if (Tn < tmin) {
                    done = true;
                    break;
                }
                const float w = al * T;
                const float2 r2 = s_r2[j];
                C0 = fmaf(w, r1.w, C0);
                C1 = fmaf(w, r2.x, C1);
                C2 = fmaf(w, r2.y, C2);
                T = Tn;
                last = (unsigned)(b - start) + (unsigned)j + 1u;
            }
        }
    }
    if (inside) {
        const long long npx = (long long)A.W * A.H;
        const long long o = (long long)py * A.W + px;
        A.rgb[o] = C0 + T * A.opt.bg[0];
        A.rgb[npx + o] = C1 + T * A.opt.bg[1];
        A.rgb[2 * npx + o] = C2 + T * A.opt.bg[2];
        if (A.T) A.T[o] = T;
        if (A.last) A.last[o] = last;
    }
}

void launch_blend(const BlendArgs &a, cudaStream_t s) {
    const int ntiles = a.tiles_x * a.tiles_y;
    if (ntiles <= 0) return;
    k_blend<<<ntiles, kBlendThreads, 0, s>>>(a);
}

}  // namespace gs
