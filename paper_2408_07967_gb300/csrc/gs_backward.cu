// gs_backward.cu -- gradient of the forward rasterizer (the paper claims a differentiable
// rasterizer but describes no backward pass; this is the exact derivative of the forward with its
// decisions held: which entries contribute to a pixel, where the walk stops, whether alpha or a
// colour channel or the Jacobian's x/z, y/z were clamped).
//
// k_blend_backward: per 16x16 tile, every pixel walks its list back to front from its last
//   contributor, recovering the transmittance before each contribution by division
//   (T_before = T_after / (1 - alpha)) from the final T stored by the forward.  With g = dL/dC:
//     dL/drgb   += alpha T g
//     dL/dalpha  = T (g . rgb) - S / (1 - alpha),   S = g . (sum of later contributions + T_final bg)
//     alpha = alpha0 e^(-q/2):  dL/dalpha0 = dL/dalpha e^(-q/2),  dL/dq = -alpha/2 dL/dalpha
//     q = a dx^2 + 2 b dx dy + c dy^2 with dx = px - u, dy = py - v.
//   Each thread takes PX pixels of a row; the nine per-Gaussian sums (u, v, a, b, c, alpha0, r, g,
//   b) of its pixels are added in the thread, reduced over the warp with shuffles, accumulated
//   over the CTA in shared memory, then added to global memory once per CTA and entry (warp-level
//   reduction before atomics, the idea DISTWAR applies to 3DGS).  With two pixels a thread the
//   pair's states are float2s updated by packed f32x2 operations, and a pixel that does not take
//   an entry gets alpha = 0 (no branch), which leaves its T and S unchanged and adds nothing.
// k_gauss_backward: per Gaussian, the chain from those 2D gradients to the parameters: colour ->
//   SH coefficients and the view direction; alpha0 -> opacity (logit); conic -> Sigma'
//   (dQ = -Q dSigma' Q) -> Sigma and J W -> scales, quaternion and the camera-space mean; (u, v)
//   -> camera-space mean -> mean.
#include "gs_internal.cuh"

namespace gs {

constexpr int kBwdPx = 2;  // pixels per thread of the reverse blend
constexpr int kG2 = 10;   // floats per Gaussian in the 2D-gradient buffer

__device__ __forceinline__ float ex2_approx_b(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Reverse blend, laid out like the forward blend: PX pixels per thread along a row (256 / PX
// threads per tile), each warp owning an RR x RC pixel region; entries are staged kBwdBatch at a
// time, each warp keeps those whose {q <= t} meets its region (the exact test of Algorithm 3 on the
// region's rectangle: an entry that meets none of the warp's pixel samples changes none of their
// states) and walks them from the highest list position down.  A thread sums its pixels' terms
// before the warp reduction, so a (warp, entry) pays one nine-value reduction for 32 PX pixels.
template <int PX>
struct BwdRegion {
    static constexpr int RC = PX == 4 ? 16 : 8;
    static constexpr int RR = 32 * PX / RC;
    static constexpr int LANES_PER_ROW = RC / PX;
};
constexpr int kBwdBatch = 128;

// Warp sums of the nine per-entry terms d, accumulated into s_acc[jj]: d[0..7] by halving
// exchanges -- across lanes 16 apart each lane keeps four values (its half's) and adds its
// partner's copy of them, then two, then one; two butterfly steps finish, leaving value
// 4 b4 + 2 b3 + b2 (bits of the lane) in every lane of a group of four -- 9 shuffles instead of
// 40; d[8] by a butterfly.
__device__ __forceinline__ void bwd_warp_sums(const float d[9], int lane, int jj, float (*s_acc)[9]) {
    const unsigned FULL = 0xffffffffu;
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    float k4[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = h4 ? d[i] : d[i + 4];
        k4[i] = (h4 ? d[i + 4] : d[i]) + __shfl_xor_sync(FULL, send, 16);
    }
    float k2[2];
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = h3 ? k4[i] : k4[i + 2];
        k2[i] = (h3 ? k4[i + 2] : k4[i]) + __shfl_xor_sync(FULL, send, 8);
    }
    float v = (h2 ? k2[1] : k2[0]) + __shfl_xor_sync(FULL, h2 ? k2[0] : k2[1], 4);
    v += __shfl_xor_sync(FULL, v, 2);
    v += __shfl_xor_sync(FULL, v, 1);
    float v8 = d[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v8 += __shfl_xor_sync(FULL, v8, o);
    if ((lane & 3) == 0 && v != 0.0f) atomicAdd(&s_acc[jj][lane >> 2], v);
    if (lane == 0 && v8 != 0.0f) atomicAdd(&s_acc[jj][8], v8);
}

template <int PX>
__global__ void __launch_bounds__(256 / PX) k_blend_backward(const __grid_constant__ BwdArgs A) {
    constexpr int NT = 256 / PX;
    constexpr int PER = kBwdBatch / NT;
    constexpr int WORDS = kBwdBatch / 32;
    using WR = BwdRegion<PX>;
    __shared__ float4 s_r0[kBwdBatch], s_r1[kBwdBatch], s_r2[kBwdBatch];
    __shared__ unsigned s_gid[kBwdBatch];
    __shared__ float s_acc[kBwdBatch][9];
    __shared__ unsigned s_maxlast;
    if (upstream_timed_out(A.ctr)) return;   // the forward's sort gave up: its ids may be garbage
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const int tile = blockIdx.x;
    const int tx = tile % A.tiles_x, ty = tile / A.tiles_x;
    constexpr int REGIONS_PER_ROW = 16 / WR::RC;
    const int rx0 = tx * kTile + (warp % REGIONS_PER_ROW) * WR::RC;
    const int ry0 = ty * kTile + (warp / REGIONS_PER_ROW) * WR::RR;
    const int py = ry0 + lane / WR::LANES_PER_ROW;
    const int px0 = rx0 + (lane % WR::LANES_PER_ROW) * PX;
    const float qx0 = (float)rx0, qx1 = (float)(rx0 + WR::RC), qy0 = (float)ry0, qy1 = (float)(ry0 + WR::RR);
    long long n = (long long)*A.n_dev;
    if (n > A.cap) n = A.cap;
    const long long start = min((long long)A.starts[tile], n);
    const long long npx = (long long)A.W * A.H;
    float fpx[PX], T[PX], S[PX], g0[PX], g1[PX], g2[PX];
    unsigned last[PX];
    unsigned my_max = 0;
#pragma unroll
    for (int k = 0; k < PX; ++k) {
        const bool inside = px0 + k < A.W && py < A.H;
        const long long o = (long long)py * A.W + px0 + k;
        fpx[k] = (float)(px0 + k) + 0.5f;
        last[k] = inside ? A.last[o] : 0u;
        g0[k] = inside ? A.dL_drgb[o] : 0.f;
        g1[k] = inside ? A.dL_drgb[npx + o] : 0.f;
        g2[k] = inside ? A.dL_drgb[2 * npx + o] : 0.f;
        T[k] = inside ? A.T_final[o] : 1.f;
        S[k] = T[k] * (g0[k] * A.opt.bg[0] + g1[k] * A.opt.bg[1] + g2[k] * A.opt.bg[2]);
        my_max = max(my_max, last[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_max = max(my_max, __shfl_xor_sync(FULL, my_max, o));
    if (tid == 0) s_maxlast = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&s_maxlast, my_max);
    __syncthreads();
    const int max_last = (int)s_maxlast;
    const float fpy = (float)py + 0.5f;
    const float HALF_LOG2E = 0.72134752044448170f;
    const float amax = A.opt.alpha_max;
    // two pixels a thread: their states as float2 pairs, updated by packed f32x2 operations
    float2 fx2 = make_float2(fpx[0], fpx[PX > 1 ? 1 : 0]), T2 = make_float2(T[0], T[PX > 1 ? 1 : 0]);
    float2 S2 = make_float2(S[0], S[PX > 1 ? 1 : 0]);
    const float2 G0 = make_float2(g0[0], g0[PX > 1 ? 1 : 0]), G1 = make_float2(g1[0], g1[PX > 1 ? 1 : 0]),
                 G2 = make_float2(g2[0], g2[PX > 1 ? 1 : 0]);
    const float2 nhl2 = make_float2(-HALF_LOG2E, -HALF_LOG2E), one2 = make_float2(1.0f, 1.0f),
                 neg1 = make_float2(-1.0f, -1.0f);

    for (int hi = max_last; hi > 0; hi -= kBwdBatch) {
        const int lo = max(0, hi - kBwdBatch);
        const int cnt = hi - lo;
        __syncthreads();                     // the previous batch has been flushed
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            const int e = r * NT + tid;
            if (e < cnt) {
                const unsigned g = A.vals[start + lo + e];
                const Rec rc = A.recs[g];
                s_r0[e] = rc.r0;
                s_r1[e] = rc.r1;
                const float a0v = ex2_approx_b(rc.r1.z);                           // alpha0
                s_r2[e] = make_float4(rc.r2.x, rc.r2.y, a0v, 1.0f / a0v);
                s_gid[e] = g;
            }
#pragma unroll
            for (int k = 0; k < 9; ++k) s_acc[e][k] = 0.0f;
        }
        __syncthreads();
        unsigned mask[WORDS];
#pragma unroll
        for (int w = 0; w < WORDS; ++w) {
            const int e = w * 32 + lane;
            bool rel = false;
            if (e < cnt) {
                const float4 a0 = s_r0[e], a1 = s_r1[e];
                rel = tile_hits(a0.x, a0.y, a0.z, 0.5f * a0.w, a1.x, a1.y, qx0, qx1, qy0, qy1);
            }
            mask[w] = __ballot_sync(FULL, rel);
        }
        // back to front: highest list position first
#pragma unroll
        for (int w = WORDS - 1; w >= 0; --w) {
            unsigned m = mask[w];
            while (m) {
                const int bit = 31 - __clz(m);
                m &= ~(1u << bit);
                const int jj = w * 32 + bit;
                const unsigned j = (unsigned)(lo + jj);
                const float4 r0 = s_r0[jj], r1 = s_r1[jj];
                const float dy = fsub(fpy, r0.y);
                const float By = fmul(r0.w, dy);
                const float Cy = fmul(fmul(r1.x, dy), dy);
                if constexpr (PX == 2) {
                    // the two pixels in packed steps; a pixel that does not take the entry gets
                    // alpha = 0, which leaves T and S as they are and adds zero to every sum
                    const float2 dx2 = __fadd2_rn(fx2, make_float2(-r0.x, -r0.x));
                    const float2 q2 = __ffma2_rn(__ffma2_rn(make_float2(r0.z, r0.z), dx2, make_float2(By, By)), dx2,
                                                 make_float2(Cy, Cy));
                    const bool p0 = j < last[0] && q2.x <= r1.y, p1 = j < last[1] && q2.y <= r1.y;
                    if (!__any_sync(FULL, p0 || p1)) continue;
                    const float4 r2 = s_r2[jj];
                    const float2 e2a = __ffma2_rn(q2, nhl2, make_float2(r1.z, r1.z));
                    const float e0 = ex2_approx_b(e2a.x), e1 = ex2_approx_b(e2a.y);   // alpha0 e^(-q/2), as forward
                    const float2 al2 = make_float2(p0 ? fminf(amax, e0) : 0.0f, p1 ? fminf(amax, e1) : 0.0f);
                    const float2 om2 = __ffma2_rn(al2, neg1, one2);                   // 1 - alpha >= 0.01
                    const float2 inv2 = make_float2(__fdividef(1.0f, om2.x), __fdividef(1.0f, om2.y));
                    const float2 Tb2 = __fmul2_rn(T2, inv2);
                    const float2 gc2 = __ffma2_rn(G0, make_float2(r1.w, r1.w),
                                                  __ffma2_rn(G1, make_float2(r2.x, r2.x), __fmul2_rn(G2, make_float2(r2.y, r2.y))));
                    const float2 wgt2 = __fmul2_rn(al2, Tb2);
                    const float2 si2 = __fmul2_rn(S2, inv2);
                    const float2 dal2 = __ffma2_rn(Tb2, gc2, make_float2(-si2.x, -si2.y));
                    S2 = __ffma2_rn(gc2, wgt2, S2);
                    T2 = Tb2;
                    // alpha not clamped: the geometry and alpha0 terms, h = alpha dL/dalpha
                    const float2 h2 = make_float2(p0 && e0 <= amax ? al2.x * dal2.x : 0.0f,
                                                  p1 && e1 <= amax ? al2.y * dal2.y : 0.0f);
                    const float2 P0 = __ffma2_rn(make_float2(2.0f * r0.z, 2.0f * r0.z), dx2,
                                                 make_float2(r0.w * dy, r0.w * dy));
                    const float2 P1 = __ffma2_rn(make_float2(r0.w, r0.w), dx2,
                                                 make_float2(2.0f * r1.x * dy, 2.0f * r1.x * dy));
                    const float2 D0 = __fmul2_rn(h2, P0), D1 = __fmul2_rn(h2, P1);
                    const float2 D2 = __fmul2_rn(h2, __fmul2_rn(dx2, dx2)), D3 = __fmul2_rn(h2, dx2);
                    const float2 D6 = __fmul2_rn(wgt2, G0), D7 = __fmul2_rn(wgt2, G1), D8 = __fmul2_rn(wgt2, G2);
                    const float hs = h2.x + h2.y;
                    float d[9];
                    d[0] = 0.5f * (D0.x + D0.y);            // -dq (2 a dx + 2 b dy), dq = -h / 2
                    d[1] = 0.5f * (D1.x + D1.y);            // -dq (2 b dx + 2 c dy)
                    d[2] = -0.5f * (D2.x + D2.y);           // dq dx^2
                    d[3] = -(D3.x + D3.y) * dy;             // dq 2 dx dy
                    d[4] = -0.5f * hs * dy * dy;            // dq dy^2
                    d[5] = hs * r2.w;                       // dL/dalpha e^(-q/2) = h / alpha0
                    d[6] = D6.x + D6.y;
                    d[7] = D7.x + D7.y;
                    d[8] = D8.x + D8.y;
                    bwd_warp_sums(d, lane, jj, s_acc);
                    continue;
                }
                float q[PX], dx[PX];
                bool pass[PX];
                bool anyp = false;
#pragma unroll
                for (int k = 0; k < PX; ++k) {
                    dx[k] = fsub(fpx[k], r0.x);
                    q[k] = ffma(ffma(r0.z, dx[k], By), dx[k], Cy);
                    pass[k] = j < last[k] && q[k] <= r1.y;
                    anyp |= pass[k];
                }
                if (!__any_sync(FULL, anyp)) continue;
                const float4 r2 = s_r2[jj];
                float d[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) d[k] = 0.0f;
#pragma unroll
                for (int k = 0; k < PX; ++k) {
                    if (!pass[k]) continue;
                    const float e2 = ex2_approx_b(fmaf(q[k], -HALF_LOG2E, r1.z));   // alpha0 e^(-q/2), as forward
                    const float al = fminf(amax, e2);
                    const float inv = __fdividef(1.0f, 1.0f - al);      // 1 - al >= 0.01
                    const float Tb = T[k] * inv;
                    const float gc = g0[k] * r1.w + g1[k] * r2.x + g2[k] * r2.y;
                    const float wgt = al * Tb;
                    d[6] += wgt * g0[k];
                    d[7] += wgt * g1[k];
                    d[8] += wgt * g2[k];
                    const float dal = Tb * gc - S[k] * inv;
                    S[k] = fmaf(gc, wgt, S[k]);
                    T[k] = Tb;
                    if (e2 <= amax) {
                        d[5] += dal * (al / r2.z);
                        const float dq = -0.5f * al * dal;
                        const float ddy = dy, ddx = dx[k];
                        d[0] += -dq * (2.0f * r0.z * ddx + r0.w * ddy);
                        d[1] += -dq * (r0.w * ddx + 2.0f * r1.x * ddy);
                        d[2] += dq * ddx * ddx;
                        d[3] += dq * 2.0f * ddx * ddy;
                        d[4] += dq * ddy * ddy;
                    }
                }
                bwd_warp_sums(d, lane, jj, s_acc);
            }
        }
        __syncthreads();
        for (int e = tid; e < cnt; e += NT) {
            float *dst = A.grad2d + (long long)s_gid[e] * kG2;
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float v = s_acc[e][k];
                if (v != 0.0f) atomicAdd(dst + k, v);
            }
        }
    }
}

// ------------------------------------------------------------------------------------------ per Gaussian
__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16]) {
    const float K0 = 0.28209479177387814f, K1 = 0.48860251190291992f;
    const float K2a = 1.0925484305920792f, K2b = 0.31539156525252005f, K2c = 0.54627421529603959f;
    const float K3a = 0.59004358992664352f, K3b = 2.8906114426405538f, K3c = 0.45704579946446572f;
    const float K3d = 0.3731763325901154f, K3e = 1.4453057213202769f;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = K0;
    Y[1] = -K1 * y;
    Y[2] = K1 * z;
    Y[3] = -K1 * x;
    Y[4] = K2a * x * y;
    Y[5] = -K2a * y * z;
    Y[6] = K2b * (2.0f * zz - xx - yy);
    Y[7] = -K2a * x * z;
    Y[8] = K2c * (xx - yy);
    Y[9] = -K3a * y * (3.0f * xx - yy);
    Y[10] = K3b * x * y * z;
    Y[11] = -K3c * y * (4.0f * zz - xx - yy);
    Y[12] = K3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -K3c * x * (4.0f * zz - xx - yy);
    Y[14] = K3e * z * (xx - yy);
    Y[15] = -K3a * x * (xx - 3.0f * yy);
}

// sum_i c_i grad Y_i(d) with respect to the (unnormalised) components of d, the partial derivatives
// of the basis above written out.
__device__ __forceinline__ void sh_dir_grad(float x, float y, float z, const float c[16], float g[3]) {
    const float K1 = 0.48860251190291992f;
    const float K2a = 1.0925484305920792f, K2b = 0.31539156525252005f, K2c = 0.54627421529603959f;
    const float K3a = 0.59004358992664352f, K3b = 2.8906114426405538f, K3c = 0.45704579946446572f;
    const float K3d = 0.3731763325901154f, K3e = 1.4453057213202769f;
    const float xx = x * x, yy = y * y, zz = z * z;
    g[0] = -K1 * c[3] + K2a * y * c[4] - 2.0f * K2b * x * c[6] - K2a * z * c[7] + 2.0f * K2c * x * c[8] -
           6.0f * K3a * x * y * c[9] + K3b * y * z * c[10] + 2.0f * K3c * x * y * c[11] - 6.0f * K3d * x * z * c[12] -
           K3c * (4.0f * zz - 3.0f * xx - yy) * c[13] + 2.0f * K3e * x * z * c[14] - K3a * (3.0f * xx - 3.0f * yy) * c[15];
    g[1] = -K1 * c[1] + K2a * x * c[4] - K2a * z * c[5] - 2.0f * K2b * y * c[6] - 2.0f * K2c * y * c[8] -
           K3a * (3.0f * xx - 3.0f * yy) * c[9] + K3b * x * z * c[10] - K3c * (4.0f * zz - xx - 3.0f * yy) * c[11] -
           6.0f * K3d * y * z * c[12] + 2.0f * K3c * x * y * c[13] - 2.0f * K3e * y * z * c[14] + 6.0f * K3a * x * y * c[15];
    g[2] = K1 * c[2] - K2a * y * c[5] + 4.0f * K2b * z * c[6] - K2a * x * c[7] + K3b * x * y * c[10] -
           8.0f * K3c * y * z * c[11] + K3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * c[12] - 8.0f * K3c * x * z * c[13] +
           K3e * (xx - yy) * c[14];
}

// SH gradients 4k .. 4k+3 of Gaussian gid: overwritten, or added to when accumulating; a 16-byte
// store when the caller's array allows.
__device__ __forceinline__ void store_sh_plane(const BwdArgs &A, long long gid, int k, const float g[4]) {
    if (A.vec16) {
        float4 *p = reinterpret_cast<float4 *>(A.g_sh) + 12 * gid + k;
        float4 w4 = make_float4(g[0], g[1], g[2], g[3]);
        if (A.accumulate) {
            const float4 o = *p;
            w4 = make_float4(o.x + w4.x, o.y + w4.y, o.z + w4.z, o.w + w4.w);
        }
        *p = w4;
    } else {
        float *p = A.g_sh + 48 * gid + 4 * k;
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = A.accumulate ? p[j] + g[j] : g[j];
    }
}

__global__ void __launch_bounds__(128, 6) k_gauss_backward(const __grid_constant__ BwdArgs A) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= A.scene.P) return;
    const float *d2 = A.grad2d + gid * kG2;
    float D[9];
    bool any = false;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        D[k] = d2[k];
        any |= D[k] != 0.0f;
    }
    float gm[3] = {0, 0, 0}, gsc[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, gop = 0.0f;
    if (any) {
        const Cam &cam = A.cam;
        const SceneView &S = A.scene;
        const float4 po = S.pos_opa[gid];
        const float *Rc = cam.R;
        float p[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) p[i] = Rc[3 * i] * po.x + Rc[3 * i + 1] * po.y + Rc[3 * i + 2] * po.z + cam.t[i];
        const float alpha0 = S.activated ? po.w : 1.0f / (1.0f + __expf(-po.w));
        const float4 sc4 = rs_of(S, gid)[0];
        float s[3] = {sc4.x, sc4.y, sc4.z};
        if (!S.activated) {
            s[0] = __expf(s[0]);
            s[1] = __expf(s[1]);
            s[2] = __expf(s[2]);
        }
        const float4 q4 = rs_of(S, gid)[1];
        const float qlen = sqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
        const float w = q4.x / qlen, x = q4.y / qlen, y = q4.z / qlen, z = q4.w / qlen;
        float R[9];
        R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
        R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
        R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
        float Sg[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                Sg[3 * i + j] = R[3 * i] * s[0] * s[0] * R[3 * j] + R[3 * i + 1] * s[1] * s[1] * R[3 * j + 1] +
                                R[3 * i + 2] * s[2] * s[2] * R[3 * j + 2];
        const float fx = cam.fx, fy = cam.fy, pz = p[2];
        float txz = p[0] / pz, tyz = p[1] / pz;
        bool clx = false, cly = false;
        if (A.opt.clamp_fov) {
            if (txz < -cam.limx) { txz = -cam.limx; clx = true; }
            if (txz > cam.limx) { txz = cam.limx; clx = true; }
            if (tyz < -cam.limy) { tyz = -cam.limy; cly = true; }
            if (tyz > cam.limy) { tyz = cam.limy; cly = true; }
        }
        const float J00 = fx / pz, J02 = -fx * txz / pz, J11 = fy / pz, J12 = -fy * tyz / pz;
        float M[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            M[k] = J00 * Rc[k] + J02 * Rc[6 + k];
            M[3 + k] = J11 * Rc[3 + k] + J12 * Rc[6 + k];
        }
        float S2[4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int l = 0; l < 2; ++l) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 3; ++k)
#pragma unroll
                    for (int m = 0; m < 3; ++m) acc += M[3 * i + k] * Sg[3 * k + m] * M[3 * l + m];
                S2[2 * i + l] = acc;
            }
        S2[0] += A.opt.dilation;
        S2[3] += A.opt.dilation;
        const float det = S2[0] * S2[3] - S2[1] * S2[2];
        const float Q[4] = {S2[3] / det, -S2[1] / det, -S2[2] / det, S2[0] / det};

        // colour -> SH and direction.  Pass 1 over the SH planes: each channel's colour (a channel
        // clamped at 0 passes no gradient).  Pass 2: the coefficient gradients Y_i dr, written plane
        // by plane, and c_i = sum over the live channels of dr k_i, from which the direction's
        // gradient is sum_i c_i grad Y_i -- no 48-value arrays held in registers.
        float dvec[3] = {po.x - cam.campos[0], po.y - cam.campos[1], po.z - cam.campos[2]};
        const float dlen = sqrtf(dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2]);
        const float dir[3] = {dvec[0] / dlen, dvec[1] / dlen, dvec[2] / dlen};
        float Y[16];
        sh_basis(dir[0], dir[1], dir[2], Y);
        const int ncoef = (S.sh_degree + 1) * (S.sh_degree + 1);
        float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kShPlanes; ++k) {
            const float4 v4 = sh_plane(S, gid, k);
            const float e[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int f = 4 * k + j, i = f / 3, ch = f - 3 * (f / 3);
                if (i < ncoef) acc[ch] += Y[i] * e[j];
            }
        }
        float dr[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) dr[ch] = acc[ch] + 0.5f < 0.0f ? 0.0f : D[6 + ch];
        float cc[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) cc[i] = 0.0f;
#pragma unroll
        for (int k = 0; k < kShPlanes; ++k) {
            const float4 v4 = sh_plane(S, gid, k);
            const float e[4] = {v4.x, v4.y, v4.z, v4.w};
            float gk[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int f = 4 * k + j, i = f / 3, ch = f - 3 * (f / 3);
                gk[j] = i < ncoef ? Y[i] * dr[ch] : 0.0f;
                if (i < ncoef) cc[i] += dr[ch] * e[j];
            }
            store_sh_plane(A, gid, k, gk);
        }
        float ddir[3];
        sh_dir_grad(dir[0], dir[1], dir[2], cc, ddir);
        const float dd = ddir[0] * dir[0] + ddir[1] * dir[1] + ddir[2] * dir[2];
        float dmean[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) dmean[a] = (ddir[a] - dir[a] * dd) / dlen;
        // opacity
        gop = S.activated ? D[5] : D[5] * alpha0 * (1.0f - alpha0);
        // conic -> Sigma'
        const float GQ[4] = {D[2], 0.5f * D[3], 0.5f * D[3], D[4]};
        float T1[4], GS2[4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) T1[2 * i + j] = Q[2 * i] * GQ[j] + Q[2 * i + 1] * GQ[2 + j];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) GS2[2 * i + j] = -(T1[2 * i] * Q[j] + T1[2 * i + 1] * Q[2 + j]);
        float GSg[9], GM[6];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                float acc = 0.f;
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 2; ++b) acc += M[3 * a + i] * GS2[2 * a + b] * M[3 * b + j];
                GSg[3 * i + j] = acc;
            }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int m = 0; m < 3; ++m) acc += GS2[2 * a + b] * M[3 * b + m] * Sg[3 * m + k];
                GM[3 * a + k] = 2.0f * acc;
            }
        float GJ[6];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int j = 0; j < 3; ++j) GJ[3 * a + j] = GM[3 * a] * Rc[3 * j] + GM[3 * a + 1] * Rc[3 * j + 1] +
                                                        GM[3 * a + 2] * Rc[3 * j + 2];
        float dp[3] = {0.f, 0.f, 0.f};
        dp[2] += GJ[0] * (-fx / (pz * pz)) + GJ[4] * (-fy / (pz * pz));
        if (!clx) {
            dp[0] += GJ[2] * (-fx / (pz * pz));
            dp[2] += GJ[2] * (2.0f * fx * p[0] / (pz * pz * pz));
        } else {
            dp[2] += GJ[2] * (fx * txz / (pz * pz));
        }
        if (!cly) {
            dp[1] += GJ[5] * (-fy / (pz * pz));
            dp[2] += GJ[5] * (2.0f * fy * p[1] / (pz * pz * pz));
        } else {
            dp[2] += GJ[5] * (fy * tyz / (pz * pz));
        }
        dp[0] += D[0] * fx / pz;
        dp[1] += D[1] * fy / pz;
        dp[2] += D[0] * (-fx * p[0] / (pz * pz)) + D[1] * (-fy * p[1] / (pz * pz));
#pragma unroll
        for (int a = 0; a < 3; ++a) gm[a] = dmean[a] + Rc[a] * dp[0] + Rc[3 + a] * dp[1] + Rc[6 + a] * dp[2];
        // Sigma = R diag(s^2) R^T
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float acc = 0.f;
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) acc += R[3 * i + k] * GSg[3 * i + j] * R[3 * j + k];
            const float ds = 2.0f * s[k] * acc;
            gsc[k] = S.activated ? ds : ds * s[k];
        }
        float GR[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k)
                GR[3 * i + k] = 2.0f * (GSg[3 * i] * R[k] + GSg[3 * i + 1] * R[3 + k] + GSg[3 * i + 2] * R[6 + k]) *
                                s[k] * s[k];
        float dq[4];
        dq[0] = GR[1] * (-2 * z) + GR[2] * (2 * y) + GR[3] * (2 * z) + GR[5] * (-2 * x) + GR[6] * (-2 * y) + GR[7] * (2 * x);
        dq[1] = GR[1] * (2 * y) + GR[2] * (2 * z) + GR[3] * (2 * y) + GR[4] * (-4 * x) + GR[5] * (-2 * w) +
                GR[6] * (2 * z) + GR[7] * (2 * w) + GR[8] * (-4 * x);
        dq[2] = GR[0] * (-4 * y) + GR[1] * (2 * x) + GR[2] * (2 * w) + GR[3] * (2 * x) + GR[5] * (2 * z) +
                GR[6] * (-2 * w) + GR[7] * (2 * z) + GR[8] * (-4 * y);
        dq[3] = GR[0] * (-4 * z) + GR[1] * (-2 * w) + GR[2] * (2 * x) + GR[3] * (2 * w) + GR[4] * (-4 * z) +
                GR[5] * (2 * y) + GR[6] * (2 * x) + GR[7] * (2 * y);
        const float proj = dq[0] * w + dq[1] * x + dq[2] * y + dq[3] * z;
        gq[0] = (dq[0] - w * proj) / qlen;
        gq[1] = (dq[1] - x * proj) / qlen;
        gq[2] = (dq[2] - y * proj) / qlen;
        gq[3] = (dq[3] - z * proj) / qlen;
    }
    if (!any && A.accumulate) return;
    const bool add = A.accumulate != 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        A.g_means[3 * gid + a] = add ? A.g_means[3 * gid + a] + gm[a] : gm[a];
        A.g_scales[3 * gid + a] = add ? A.g_scales[3 * gid + a] + gsc[a] : gsc[a];
    }
    A.g_opacity[gid] = add ? A.g_opacity[gid] + gop : gop;
    if (A.vec16) {
        // the quaternion gradient as one 16-byte store (the array is 16-byte aligned)
        float4 *gq4 = reinterpret_cast<float4 *>(A.g_quats) + gid;
        float4 v = make_float4(gq[0], gq[1], gq[2], gq[3]);
        if (add) {
            const float4 o = *gq4;
            v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
        }
        *gq4 = v;
    } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) A.g_quats[4 * gid + a] = add ? A.g_quats[4 * gid + a] + gq[a] : gq[a];
    }
    if (!any) {
        // an unused Gaussian's SH gradients (written here; a used one's went out with pass 2)
        const float z4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < kShPlanes; ++k) store_sh_plane(A, gid, k, z4);
    }
}

void launch_backward(const BwdArgs &a, cudaStream_t s, cudaEvent_t between) {
    const int ntiles = a.tiles_x * a.tiles_y;
    if (ntiles > 0) k_blend_backward<kBwdPx><<<ntiles, 256 / kBwdPx, 0, s>>>(a);
    if (between) cudaEventRecord(between, s);
    const long long P = a.scene.P;
    if (P > 0) k_gauss_backward<<<(unsigned)((P + 127) / 128), 128, 0, s>>>(a);
}

int grad2d_floats() { return kG2; }

}  // namespace gs
