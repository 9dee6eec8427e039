// gs_render.cu -- per-tile front-to-back alpha blending (the render stage of Section 2.2, with
// the ideas of Sections 5.2-5.3 realised for sm_103a):
//   * coarse-grained partition (Section 5.2.3): each thread owns PX horizontally adjacent pixels
//     of one row, so the row terms of the quadratic form and the shared-memory reads of a
//     Gaussian are computed once for PX pixels;
//   * two-level prefetch (Section 5.2.1): while batch b is blended, the records of batch b+1
//     are in flight to shared memory (cp.async, double buffer) and the Gaussian ids of batch
//     b+2 are in flight to registers;
//   * divergence control (Section 5.2.2): a warp-uniform vote skips a Gaussian that reaches
//     alpha >= tau at none of the warp's pixels, and one CTA-wide count stops the tile when
//     every pixel has saturated;
//   * the exponent is folded into one FMA in the log2 domain and evaluated by
//     ex2.approx.ftz.f32 (Section 5.3.2).
//
// Per pixel sample (i + 1/2, j + 1/2) and list entry (u, v, a, b2, c, t, G, rgb):
//   q = fma(fma(a, dx, b2 dy), dx, (c dy) dy)     (binary32; skip the entry when !(q <= t))
//   alpha = min(alpha_max, 2^(G - q log2(e)/2))   (G = log2 alpha0, so alpha = alpha0 e^(-q/2))
//   T' = T (1 - alpha); stop before the entry if T' < T_min; C += rgb alpha T; T = T'.
#include "gs_internal.cuh"

namespace gs {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int PX, int BATCH>
struct BlendSmem {
    float4 r0[2][BATCH];
    float4 r1[2][BATCH];
    float4 r2[2][BATCH];
};

// PX pixels per thread along a row; 256/PX threads per 16x16 tile; BATCH records per stage.
template <int PX, int BATCH>
__global__ void __launch_bounds__(256 / PX) k_blend(const __grid_constant__ BlendArgs A) {
    constexpr int NT = 256 / PX;            // threads per tile
    constexpr int PER = BATCH / NT;         // records each thread stages per batch
    static_assert(BATCH % NT == 0, "batch must be a multiple of the thread count");
    __shared__ BlendSmem<PX, BATCH> S;
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int tx = tile % A.tiles_x, ty = tile / A.tiles_x;
    constexpr int GROUPS = 16 / PX;         // thread groups per row
    const int row = tid / GROUPS, grp = tid % GROUPS;
    const int py = ty * kTile + row;
    const int px0 = tx * kTile + grp * PX;
    long long n = (long long)*A.n_dev;
    if (n > A.cap) n = A.cap;
    const long long start = min((long long)A.starts[tile], n);
    const long long end = min((long long)A.starts[tile + 1], n);
    const float fpy = (float)py + 0.5f;
    float fpx[PX];
    bool done[PX];
    float T[PX], C0[PX], C1[PX], C2[PX];
    unsigned last[PX], stop[PX];
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        fpx[k] = (float)(px0 + k) + 0.5f;
        done[k] = !(px0 + k < A.W && py < A.H);
        T[k] = 1.0f;
        C0[k] = C1[k] = C2[k] = 0.0f;
        last[k] = 0;
        stop[k] = 0;
    }
    const float HALF_LOG2E = 0.72134752044448170f;
    const float amax = A.opt.alpha_max, tmin = A.opt.T_min;
    const unsigned FULL = 0xffffffffu;

    // ---- pipeline prologue: ids of batches 0 and 1, records of batch 0
    unsigned ids[PER], ids_next[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const long long i0 = start + r * NT + tid, i1 = start + BATCH + r * NT + tid;
        ids[r] = i0 < end ? __ldg(A.vals + i0) : 0u;
        ids_next[r] = i1 < end ? __ldg(A.vals + i1) : 0u;
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const int e = r * NT + tid;
        if (start + e < end) {
            const Rec *src = A.recs + ids[r];
            cp_async16(&S.r0[0][e], &src->r0);
            cp_async16(&S.r1[0][e], &src->r1);
            cp_async16(&S.r2[0][e], &src->r2);
        }
    }
    cp_async_commit();

    int buf = 0;
    for (long long b = start; b < end; b += BATCH) {
        // records of batch b+1 into the other buffer, ids of batch b+2 into registers
        const long long bn = b + BATCH;
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = r * NT + tid;
            if (bn + e < end) {
                const Rec *src = A.recs + ids_next[r];
                cp_async16(&S.r0[buf ^ 1][e], &src->r0);
                cp_async16(&S.r1[buf ^ 1][e], &src->r1);
                cp_async16(&S.r2[buf ^ 1][e], &src->r2);
            }
        }
        cp_async_commit();
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const long long i2 = bn + BATCH + r * NT + tid;
            ids_next[r] = i2 < end ? __ldg(A.vals + i2) : 0u;
        }
        cp_async_wait<1>();
        __syncthreads();
        const int cnt = (int)min((long long)BATCH, end - b);
        const unsigned pos0 = (unsigned)(b - start);
        bool alive = false;
#pragma unroll
        for (int k = 0; k < PX; ++k) alive |= !done[k];
        if (__any_sync(FULL, alive)) {
            for (int j = 0; j < cnt; ++j) {
                const float4 r0 = S.r0[buf][j];
                const float4 r1 = S.r1[buf][j];
                const float dy = fsub(fpy, r0.y);
                const float By = fmul(r0.w, dy);
                const float Cy = fmul(fmul(r1.x, dy), dy);
                float q[PX];
                bool pass[PX];
                bool anyp = false;
#pragma unroll
                for (int k = 0; k < PX; ++k) {
                    const float dx = fsub(fpx[k], r0.x);
                    q[k] = ffma(ffma(r0.z, dx, By), dx, Cy);
                    pass[k] = (q[k] <= r1.y) && !done[k];
                    anyp |= pass[k];
                }
                if (!__any_sync(FULL, anyp)) continue;
                const float4 r2 = S.r2[buf][j];
                const unsigned pos = pos0 + (unsigned)j + 1u;
#pragma unroll
                for (int k = 0; k < PX; ++k) {
                    if (pass[k]) {
                        const float al = fminf(amax, ex2_approx(fmaf(q[k], -HALF_LOG2E, r1.z)));
                        const float Tn = T[k] * (1.0f - al);
                        if (Tn < tmin) {
                            done[k] = true;
                            stop[k] = pos;
                        } else {
                            const float w = al * T[k];
                            C0[k] = fmaf(w, r1.w, C0[k]);
                            C1[k] = fmaf(w, r2.x, C1[k]);
                            C2[k] = fmaf(w, r2.y, C2[k]);
                            T[k] = Tn;
                            last[k] = pos;
                        }
                    }
                }
            }
        }
        bool alive2 = false;
#pragma unroll
        for (int k = 0; k < PX; ++k) alive2 |= !done[k];
        if (__syncthreads_count(alive2) == 0) break;   // also orders buffer reuse
        buf ^= 1;
    }
    cp_async_wait<0>();

    // evaluation count for the roofline: entries walked per pixel, skipped ones included
    unsigned long long walked = 0;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const bool in = px0 + k < A.W && py < A.H;
        if (in) walked += stop[k] ? stop[k] : (unsigned long long)(end - start);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) walked += __shfl_xor_sync(FULL, walked, o);
    if ((tid & 31) == 0 && walked) atomicAdd(A.evals, walked);

    const long long npx = (long long)A.W * A.H;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const int px = px0 + k;
        if (px < A.W && py < A.H) {
            const long long o = (long long)py * A.W + px;
            A.rgb[o] = C0[k] + T[k] * A.opt.bg[0];
            A.rgb[npx + o] = C1[k] + T[k] * A.opt.bg[1];
            A.rgb[2 * npx + o] = C2[k] + T[k] * A.opt.bg[2];
            if (A.T) A.T[o] = T[k];
            if (A.last) A.last[o] = last[k];
        }
    }
}

// Launch shapes (pixels per thread, records per staged batch); the autotuner picks one.
// Every variant evaluates each pixel's list with the same operations in the same order, so
// the outputs are bit-identical across variants.
int blend_variant_count() { return 6; }

void launch_blend(const BlendArgs &a, cudaStream_t s) {
    const int ntiles = a.tiles_x * a.tiles_y;
    if (ntiles <= 0) return;
    switch (a.variant) {
        case 0: k_blend<1, 256><<<ntiles, 256, 0, s>>>(a); break;
        case 1: k_blend<2, 128><<<ntiles, 128, 0, s>>>(a); break;
        case 2: k_blend<4, 128><<<ntiles, 64, 0, s>>>(a); break;
        case 3: k_blend<2, 256><<<ntiles, 128, 0, s>>>(a); break;
        case 4: k_blend<4, 64><<<ntiles, 64, 0, s>>>(a); break;
        default: k_blend<4, 256><<<ntiles, 64, 0, s>>>(a); break;
    }
}

}  // namespace gs
