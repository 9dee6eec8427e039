// gs_render.cu -- per-tile front-to-back alpha blending (the render stage of Section 2.2, with
// the ideas of Sections 5.2-5.3 realised for sm_103a):
//   * coarse-grained partition (Section 5.2.3): each thread owns PX horizontally adjacent pixels
//     of one row, so the row terms of the quadratic form and the shared-memory reads of a
//     Gaussian are computed once for PX pixels;
//   * two-level prefetch (Section 5.2.1): while batch b is blended, the records of batch b+1
//     are in flight to shared memory (cp.async, double buffer) and the Gaussian ids of batch
//     b+2 are in flight to registers;
//   * divergence control (Section 5.2.2): each warp filters every staged batch against its own
//     pixel region with the exact ellipse/rectangle test of Algorithm 3 (one Gaussian per lane,
//     one ballot per 32 entries) and walks only the entries that can reach its pixels -- the
//     paper's tile-level exact intersection applied again at warp granularity (with one pixel
//     per thread, a warp-uniform vote also skips an entry that passes q <= t at none of the
//     warp's pixels); a saturated pixel is parked at x = +inf, and one CTA-wide count stops the
//     tile when every pixel has saturated;
//   * with two or four pixels per thread, the pixels are processed in pairs by the packed
//     binary32 operations of sm_100-class GPUs (add/mul/fma .f32x2: one instruction for both
//     pixels, each lane rounded exactly as the scalar operation), halving the issue slots of the
//     per-pixel arithmetic in this issue-bound loop;
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

// Warp region of a launch shape: RC columns x RR rows of pixels, RC * RR = 32 * PX.
template <int PX>
struct WarpRegion {
    static constexpr int RC = PX == 4 ? 16 : 8;
    static constexpr int RR = 32 * PX / RC;
    static constexpr int LANES_PER_ROW = RC / PX;
};

// PX pixels per thread along a row; 256/PX threads per 16x16 tile; BATCH records per stage.
// Each warp owns an RR x RC pixel region of the tile.  Per staged batch, lane l tests entries
// l, l+32, ... exactly against the region's rectangle shrunk by a quarter pixel; the warp then walks only the
// entries that meet it, in list order, so a pixel's entries are still evaluated in order and
// with the same arithmetic.  (A pixel sample passing q <= t lies inside the ellipse, a quarter
// pixel inside the tested rectangle, so no contributing entry is filtered out.)  COUNT adds the
// per-pixel evaluation and contribution counters used for the roofline (not in timed runs).
template <int PX, int BATCH, bool COUNT>
__global__ void __launch_bounds__(256 / PX) k_blend(const __grid_constant__ BlendArgs A) {
    constexpr int NT = 256 / PX;            // threads per tile
    constexpr int PER = BATCH / NT;         // records each thread stages per batch
    constexpr int WORDS = BATCH / 32;       // filter mask words per batch
    using WR = WarpRegion<PX>;
    static_assert(BATCH % NT == 0 && BATCH % 32 == 0, "batch must be a multiple of the thread count");
    __shared__ BlendSmem<PX, BATCH> S;
    if (upstream_timed_out(A.ctr)) return;   // the sort gave up: its ids may be garbage
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int gtile = A.order ? (int)A.order[blockIdx.x] : (int)blockIdx.x;   // global tile of the batch
    const ReqDesc &R = A.B.r[req_of_tile(A.B, gtile)];
    const int tile = gtile - R.tile0;
    const int W = R.cam.W, H = R.cam.H;
    const int tx = tile % R.cam.tiles_x, ty = tile / R.cam.tiles_x;
    constexpr int REGIONS_PER_ROW = 16 / WR::RC;
    const int rx0 = tx * kTile + (warp % REGIONS_PER_ROW) * WR::RC;    // region origin (pixels)
    const int ry0 = ty * kTile + (warp / REGIONS_PER_ROW) * WR::RR;
    const int py = ry0 + lane / WR::LANES_PER_ROW;
    const int px0 = rx0 + (lane % WR::LANES_PER_ROW) * PX;
    // the rectangle the filter tests: the region's pixel samples lie a quarter pixel inside it (far
    // above binary32 rounding, so a sample that passes q <= t always finds its entry kept)
    const float qx0 = (float)rx0 + 0.25f, qx1 = (float)(rx0 + WR::RC) - 0.25f, qy0 = (float)ry0 + 0.25f,
                qy1 = (float)(ry0 + WR::RR) - 0.25f;
    long long n = (long long)*A.n_dev;
    if (n > A.cap) n = A.cap;
    const long long start = min((long long)A.starts[gtile], n);
    const long long end = min((long long)A.starts[gtile + 1], n);
    const float fpy = (float)py + 0.5f;
    const float INF = __int_as_float(0x7f800000);
    float fpx[PX];
    bool inside[PX];
    float T[PX], C0[PX], C1[PX], C2[PX];
    unsigned last[PX];
    unsigned stop[PX], contrib[PX];
    int alive_px = 0;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        inside[k] = px0 + k < W && py < H;
        // a finished pixel keeps x = +inf: its q is +inf or NaN and never passes q <= t
        fpx[k] = inside[k] ? (float)(px0 + k) + 0.5f : INF;
        alive_px += inside[k];
        T[k] = 1.0f;
        C0[k] = C1[k] = C2[k] = 0.0f;
        last[k] = 0;
        stop[k] = 0;
        contrib[k] = 0;
    }
    // PX >= 2: the state of pixels 2h, 2h+1 as float2 pairs, updated by packed f32x2 operations
    // (one instruction for both pixels; each lane of the pair is the binary32 operation above)
    constexpr int NP = PX / 2 > 0 ? PX / 2 : 1;
    float2 fx2[NP], T2[NP], C02[NP], C12[NP], C22[NP];
#pragma unroll
    for (int h = 0; h < NP; ++h) {
        fx2[h] = make_float2(fpx[2 * h < PX ? 2 * h : 0], fpx[2 * h + 1 < PX ? 2 * h + 1 : 0]);
        T2[h] = make_float2(1.0f, 1.0f);
        C02[h] = C12[h] = C22[h] = make_float2(0.0f, 0.0f);
    }
    const float HALF_LOG2E = 0.72134752044448170f;
    const float amax = R.opt.alpha_max, tmin = R.opt.T_min;
    const float2 nhl2 = make_float2(-HALF_LOG2E, -HALF_LOG2E);
    const unsigned FULL = 0xffffffffu;

    // ---- pipeline prologue: ids of batches 0 and 1, records of batch 0
    unsigned ids_next[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const long long i0 = start + r * NT + tid, i1 = start + BATCH + r * NT + tid;
        const unsigned id0 = i0 < end ? __ldg(A.vals + i0) : 0u;
        ids_next[r] = i1 < end ? __ldg(A.vals + i1) : 0u;
        if (i0 < end) {
            const Rec *src = A.recs + id0;
            const int e = r * NT + tid;
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
        if (__any_sync(FULL, alive_px > 0)) {
            // per-warp filter of the batch against the warp's pixel region
            unsigned mask[WORDS];
#pragma unroll
            for (int w = 0; w < WORDS; ++w) {
                const int e = w * 32 + lane;
                bool rel = false;
                if (e < cnt) {
                    // exact ellipse / rectangle test (Algorithm 3) of {q <= t} against the region
                    const float4 a0 = S.r0[buf][e];
                    const float4 a1 = S.r1[buf][e];
                    rel = tile_hits(a0.x, a0.y, a0.z, 0.5f * a0.w, a1.x, a1.y, qx0, qx1, qy0, qy1);
                }
                mask[w] = __ballot_sync(FULL, rel);
            }
#pragma unroll
            for (int w = 0; w < WORDS; ++w) {
                unsigned m = mask[w];
                auto step = [&](const int j) {
                    const float4 r0 = S.r0[buf][j];
                    const float4 r1 = S.r1[buf][j];
                    const float dy = fsub(fpy, r0.y);
                    const float By = fmul(r0.w, dy);
                    const float Cy = fmul(fmul(r1.x, dy), dy);
                    const unsigned pos = pos0 + (unsigned)j + 1u;
                    if constexpr (PX >= 2) {
                        // both pixels of a pair in one packed operation per step; the filter
                        // already dropped the entries that reach no pixel of the warp, so with
                        // two pixels per thread the rest are blended without a per-entry vote
                        // (with four, the warp's 128 pixels leave more entries that reach none
                        // of them and the vote pays)
                        float2 q2[NP];
                        bool pass[PX];
#pragma unroll
                        for (int h = 0; h < NP; ++h) {
                            const float2 dx2 = __fadd2_rn(fx2[h], make_float2(-r0.x, -r0.x));
                            q2[h] = __ffma2_rn(__ffma2_rn(make_float2(r0.z, r0.z), dx2, make_float2(By, By)), dx2,
                                               make_float2(Cy, Cy));
                            pass[2 * h] = q2[h].x <= r1.y;
                            pass[2 * h + 1] = q2[h].y <= r1.y;
                        }
                        if (PX == 4) {
                            bool anyp = false;
#pragma unroll
                            for (int k = 0; k < PX; ++k) anyp |= pass[k];
                            if (!__any_sync(FULL, anyp)) return;
                        }
                        const float4 r2 = S.r2[buf][j];
#pragma unroll
                        for (int h = 0; h < NP; ++h) {
                            const bool p0 = pass[2 * h], p1 = pass[2 * h + 1];
                            const float2 e2 = __ffma2_rn(q2[h], nhl2, make_float2(r1.z, r1.z));
                            // nal = -alpha and nau = -alpha where the pixel takes the entry, else 0:
                            // T' = fma(nau, T, T) is the scalar fma(-alpha, T, T) or T itself, and
                            // C += (nau T)(-rgb) is the scalar fma(alpha T, rgb, C) bit for bit
                            const float2 nal2 =make_float2(fmaxf(-amax, -ex2_approx(e2.x)), fmaxf(-amax, -ex2_approx(e2.y)));
                            const float2 Tn2 = __ffma2_rn(nal2, T2[h], T2[h]);
                            const bool s0 = p0 && Tn2.x < tmin, s1 = p1 && Tn2.y < tmin;
                            const bool u0 = p0 && !(Tn2.x < tmin), u1 = p1 && !(Tn2.y < tmin);
                            if (COUNT) {
                                contrib[2 * h] += p0;
                                contrib[2 * h + 1] += p1;
                                if (s0) stop[2 * h] = pos;
                                if (s1) stop[2 * h + 1] = pos;
                            }
                            const float2 nau = make_float2(u0 ? nal2.x : 0.0f, u1 ? nal2.y : 0.0f);
                            const float2 nw2 = __fmul2_rn(nau, T2[h]);
                            C02[h] = __ffma2_rn(nw2, make_float2(-r1.w, -r1.w), C02[h]);
                            C12[h] = __ffma2_rn(nw2, make_float2(-r2.x, -r2.x), C12[h]);
                            C22[h] = __ffma2_rn(nw2, make_float2(-r2.y, -r2.y), C22[h]);
                            T2[h] = __ffma2_rn(nau, T2[h], T2[h]);
                            last[2 * h] = u0 ? pos : last[2 * h];
                            last[2 * h + 1] = u1 ? pos : last[2 * h + 1];
                            fx2[h] = make_float2(s0 ? INF : fx2[h].x, s1 ? INF : fx2[h].y);
                        }
                        return;
                    }
                    float q[PX];
                    bool pass[PX];
                    bool anyp = false;
#pragma unroll
                    for (int k = 0; k < PX; ++k) {
                        const float dx = fsub(fpx[k], r0.x);
                        q[k] = ffma(ffma(r0.z, dx, By), dx, Cy);
                        pass[k] = q[k] <= r1.y;
                        anyp |= pass[k];
                    }
                    if (!__any_sync(FULL, anyp)) return;
                    const float4 r2 = S.r2[buf][j];
                    // branch-free: a pixel that does not pass adds a zero weight and keeps its state
#pragma unroll
                    for (int k = 0; k < PX; ++k) {
                        const float al = fminf(amax, ex2_approx(fmaf(q[k], -HALF_LOG2E, r1.z)));
                        const float Tn = fmaf(-al, T[k], T[k]);
                        const bool stp = pass[k] && Tn < tmin;
                        const bool upd = pass[k] && !(Tn < tmin);
                        if (COUNT) contrib[k] += pass[k];
                        if (COUNT && stp) stop[k] = pos;
                        const float w = upd ? al * T[k] : 0.0f;
                        C0[k] = fmaf(w, r1.w, C0[k]);
                        C1[k] = fmaf(w, r2.x, C1[k]);
                        C2[k] = fmaf(w, r2.y, C2[k]);
                        T[k] = upd ? Tn : T[k];
                        last[k] = upd ? pos : last[k];
                        fpx[k] = stp ? INF : fpx[k];
                        alive_px -= stp;
                    }
                };
                // four pixels per thread: two entries per trip (fewer loop steps a walked entry;
                // measured faster there, slower with two pixels per thread)
                while (m) {
                    step(w * 32 + __ffs(m) - 1);
                    m &= m - 1;
                    if constexpr (PX == 4) {
                        if (!m) break;
                        step(w * 32 + __ffs(m) - 1);
                        m &= m - 1;
                    }
                }
            }
        }
        if constexpr (PX >= 2) {
            // pixels still running: the ones not parked at x = +inf (outside pixels start there)
            alive_px = 0;
#pragma unroll
            for (int h = 0; h < NP; ++h) alive_px += (fx2[h].x != INF) + (fx2[h].y != INF);
        }
        if (__syncthreads_count(alive_px > 0) == 0) break;   // also orders buffer reuse
        buf ^= 1;
    }
    cp_async_wait<0>();
    if constexpr (PX >= 2) {
#pragma unroll
        for (int h = 0; h < NP; ++h) {
            T[2 * h] = T2[h].x;
            T[2 * h + 1] = T2[h].y;
            C0[2 * h] = C02[h].x;
            C0[2 * h + 1] = C02[h].y;
            C1[2 * h] = C12[h].x;
            C1[2 * h + 1] = C12[h].y;
            C2[2 * h] = C22[h].x;
            C2[2 * h + 1] = C22[h].y;
        }
    }

    if (COUNT) {
        // entries walked per pixel (skipped ones included) and entries that passed q <= t
        unsigned long long walked = 0, contributed = 0;
#pragma unroll
        for (int k = 0; k < PX; ++k) {
            if (inside[k]) {
                walked += stop[k] ? stop[k] : (unsigned long long)(end - start);
                contributed += contrib[k];
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            walked += __shfl_xor_sync(FULL, walked, o);
            contributed += __shfl_xor_sync(FULL, contributed, o);
        }
        if (lane == 0) {
            if (walked) atomicAdd(A.evals, walked);
            if (contributed) atomicAdd(A.evals + 1, contributed);
        }
    }

    const long long npx = (long long)W * H;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const int px = px0 + k;
        if (inside[k]) {
            const long long o = (long long)py * W + px;
            R.rgb[o] = C0[k] + T[k] * R.opt.bg[0];
            R.rgb[npx + o] = C1[k] + T[k] * R.opt.bg[1];
            R.rgb[2 * npx + o] = C2[k] + T[k] * R.opt.bg[2];
            if (R.T) R.T[o] = T[k];
            if (R.last) R.last[o] = last[k];
        }
    }
}

// Blend order: the tiles by decreasing class of list length (floor log2(length + 1)), so the
// longest lists start first and short ones fill the end of the launch -- a long list that starts
// late would otherwise set the blend's makespan (one 1165-entry tile started at 134 us of a room
// frame's 209 us median SM finish ran to 250 us).  Within a class any order: tiles are
// independent, so the images do not depend on it.  One CTA of 1024 threads, sixteen consecutive
// tiles per thread (up to 16384 tiles, the limit the caller applies): the seventeen starts a
// thread needs arrive in one round of loads, the classes stay in registers, a class histogram in
// shared memory gives the class bases from the longest class down, and each tile takes the next
// slot of its class by a shared-memory atomic (the order within a class is whatever the atomics
// give).
constexpr int kOrderThreads = 1024;
constexpr int kOrderPer = 16;
__global__ void __launch_bounds__(kOrderThreads) k_tile_order(const unsigned *starts, int ntiles, unsigned *order) {
    __shared__ unsigned s_cnt[33], s_base[33];
    const int tid = threadIdx.x;
    if (tid < 33) s_cnt[tid] = 0;
    const int t0 = tid * kOrderPer;
    unsigned st[kOrderPer + 1];
#pragma unroll
    for (int k = 0; k <= kOrderPer; ++k) st[k] = t0 + k <= ntiles ? __ldg(starts + t0 + k) : 0u;
    unsigned cls[kOrderPer];
#pragma unroll
    for (int k = 0; k < kOrderPer; ++k)
        cls[k] = t0 + k < ntiles ? 31u - (unsigned)__clz(st[k + 1] - st[k] + 1u) : 32u;   // 32: past the end
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kOrderPer; ++k)
        if (cls[k] < 32u) atomicAdd(&s_cnt[cls[k]], 1u);
    __syncthreads();
    if (tid == 0) {
        unsigned base = 0;
        for (int c = 31; c >= 0; --c) {
            s_base[c] = base;
            base += s_cnt[c];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kOrderPer; ++k)
        if (cls[k] < 32u) order[atomicAdd(&s_base[cls[k]], 1u)] = (unsigned)(t0 + k);
}

void launch_tile_order(const unsigned *starts, int ntiles, unsigned *order, cudaStream_t s) {
    if (ntiles > 0 && ntiles <= kOrderThreads * kOrderPer) k_tile_order<<<1, kOrderThreads, 0, s>>>(starts, ntiles, order);
}

// Launch shapes (pixels per thread, records per staged batch); the autotuner picks one.
// Every variant evaluates each pixel's list with the same operations in the same order, so
// the outputs are bit-identical across variants.
int blend_variant_count() { return 6; }

template <bool COUNT>
static void launch_blend_t(const BlendArgs &a, int ntiles, cudaStream_t s) {
    switch (a.variant) {
        case 0: k_blend<1, 256, COUNT><<<ntiles, 256, 0, s>>>(a); break;
        case 1: k_blend<2, 128, COUNT><<<ntiles, 128, 0, s>>>(a); break;
        case 2: k_blend<4, 128, COUNT><<<ntiles, 64, 0, s>>>(a); break;
        case 3: k_blend<2, 256, COUNT><<<ntiles, 128, 0, s>>>(a); break;
        case 4: k_blend<4, 64, COUNT><<<ntiles, 64, 0, s>>>(a); break;
        default: k_blend<4, 256, COUNT><<<ntiles, 64, 0, s>>>(a); break;
    }
}

void launch_blend(const BlendArgs &a, cudaStream_t s) {
    const int ntiles = a.B.total_tiles;
    if (ntiles <= 0) return;
    if (a.count)
        launch_blend_t<true>(a, ntiles, s);
    else
        launch_blend_t<false>(a, ntiles, s);
}

}  // namespace gs
