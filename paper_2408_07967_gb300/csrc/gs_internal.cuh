// gs_internal.cuh -- device-side structures and helpers shared by the sm_103a kernels.
//
// Decision arithmetic.  Every quantity that decides an integer outcome (cull, candidate
// tiles, the exact tile test, key bits, the per-pixel alpha >= tau skip) is computed with
// explicitly rounded binary32 intrinsics (__fadd_rn, __fmul_rn, __fdiv_rn, __fsqrt_rn and,
// where the definition fuses, __fmaf_rn), so the compiler can neither contract nor reorder
// it.  The rest (SH colour, blending values) uses ordinary float arithmetic.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr int kTile = 16;            // 16x16-pixel tiles (Section 2.2)
constexpr int kShPlanes = 12;        // 48 SH floats as twelve float4

// device-side status bits, collected in FrameCounters::status
enum : unsigned { kStPairOverflow = 1u, kStTimeout = 2u };

// Bounded waits: a spin gives up after this many polls and sets kStTimeout.  Waits on other CTAs
// (look-back descriptors, grid barriers) take the process-wide limit wait_limit() (this value
// unless gs_set_wait_limit changed it); waits of a CTA on its own bulk copies always take this one,
// so a CTA never leaves while a copy into its shared memory is in flight.
constexpr unsigned kSpinLimit = 1u << 22;
unsigned wait_limit();

struct Cam {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    float near_z;
    float limx, limy;      // 1.3 tan(half fov) bounds of x/z, y/z for the Jacobian
    float campos[3];       // camera centre in world space (for SH directions)
    int W, H;
    int tiles_x, tiles_y;
};

struct Opts {
    float bg[3];
    float tau, alpha_max, T_min, dilation;
    int cap_3sigma, clamp_fov;
    int intersect;           // 0 exact tiles, 1 every tile of the 3DGS 3-sigma square
};

// Internal scene layout, three arrays sized by how sparsely each is read:
//   pos_opa[i]          (x, y, z, opacity or logit): read by the cull of every Gaussian;
//   rs[2 i], rs[2 i+1]  (sx, sy, sz, 0) or log-scales, and the quaternion (w, x, y, z): read by
//                       every Gaussian that passes the cull (most of them), so a dense plane;
//   sh[kShPlanes i + k] SH floats 4k .. 4k+3: read only for paired Gaussians, which are scattered
//                       over the id range, so each Gaussian's 192 bytes are contiguous (three
//                       64-byte bursts) instead of twelve planes with one burst each.  With
//                       binary16 storage (opt-in) plane k is four halves, 96 bytes a Gaussian.
struct SceneView {
    const float4 *pos_opa;
    const float4 *rs;
    const void *sh;
    int64_t P;
    int sh_degree;
    int activated;
    int sh_half;             // SH kept as binary16
};
__device__ __forceinline__ const float4 *rs_of(const SceneView &S, long long gid) { return S.rs + 2 * gid; }
// SH floats 4k .. 4k+3 of Gaussian gid (k < kShPlanes), from either storage.
__device__ __forceinline__ float4 sh_plane(const SceneView &S, long long gid, int k) {
    if (S.sh_half) {
        const uint2 h = __ldg(reinterpret_cast<const uint2 *>(S.sh) + kShPlanes * gid + k);
        const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&h.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&h.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
    return __ldg(reinterpret_cast<const float4 *>(S.sh) + kShPlanes * gid + k);
}

// Render record of a paired Gaussian (48 bytes, three float4):
//   r0 = (u, v, a, b2)   centre and conic, b2 = 2 b
//   r1 = (c, t, G, red)  t = pixel threshold on q; G = log2(alpha0) = log2(tau) + t_full log2(e)/2
//   r2 = (green, blue, hx + 1, hy + 1)  half extents of the {q <= t} box plus one pixel
struct Rec {
    float4 r0, r1, r2;
};

// A batch of render requests, passed by value to every forward kernel (Section 5.3.1: parameters
// shared by all threads live in the kernel-parameter constant bank).  Request r owns chunks
// [chunk0, next chunk0) of 256 Gaussians, records rec0 + Gaussian id and global tiles
// [tile0, tile0 + tiles_x * tiles_y); a single render is a batch of one with all offsets 0.
constexpr int kMaxBatch = 16;
struct ReqDesc {
    Cam cam;
    Opts opt;
    SceneView scene;
    long long chunk0;
    long long rec0;
    int tile0;
    int pad;
    float *rgb;          // blend outputs ([3,H,W], [H,W], [H,W])
    float *T;
    unsigned *last;
};
struct BatchDesc {
    int n;
    int total_tiles;
    long long total_chunks;
    long long total_recs;
    ReqDesc r[kMaxBatch];
};
__device__ __forceinline__ int req_of_chunk(const BatchDesc &B, long long chunk) {
    int r = 0;
    for (int i = 1; i < B.n; ++i)
        if (B.r[i].chunk0 <= chunk) r = i;
    return r;
}
__device__ __forceinline__ int req_of_rec(const BatchDesc &B, long long rec) {
    int r = 0;
    for (int i = 1; i < B.n; ++i)
        if (B.r[i].rec0 <= rec) r = i;
    return r;
}
__device__ __forceinline__ int req_of_tile(const BatchDesc &B, int tile) {
    int r = 0;
    for (int i = 1; i < B.n; ++i)
        if (B.r[i].tile0 <= tile) r = i;
    return r;
}

// Device counters of one frame.  Everything before sort_epoch is cleared at the start of every
// frame; sort_epoch only grows (it tags the sort's look-back descriptors).
struct FrameCounters {
    unsigned long long n_pairs;      // pairs found by preprocess (may exceed capacity)
    unsigned long long evals[2];     // counted blend: entries walked, entries passing q <= t
    unsigned int n_visible;          // Gaussians with >= 1 pair
    unsigned int n_culled_in;        // Gaussians passing the near-plane / opacity cull
    unsigned int status;             // kSt* bits
    unsigned int chunk_ticket;       // preprocess chunk ticket
    unsigned long long n_vis64;      // paired Gaussians (two-level order)
    unsigned long long scratch64;    // unused scan total
    unsigned long long mask_used;    // bytes of unit hit masks taken by the count pass
    unsigned int n_big;              // two-level order: Gaussians left to k_emit_big
    unsigned int big_ticket;
    unsigned int n_mid;              // two-level order: Gaussians left to k_emit_mid (one warp each)
    unsigned int mid_ticket;
    unsigned int sort_ticket[8];     // scatter-pass tickets
    unsigned int sort_bar[9];        // fused sort: arrivals at grid barrier b (0..7) and exits (8);
                                     // the last CTA out zeroes them for the next sort
    unsigned int sort_epoch;         // bumped once per sort; tags look-back descriptors
    unsigned int pad1[4];
};

// True when a bounded wait of this frame gave up earlier in the stream: the sort output that a
// consumer would read may then be incomplete (wrong ids, tile keys out of range), so consumers
// return at once.  For kernels that never set the timeout bit themselves, so every thread reads
// the same value and may branch on it without a barrier.
__device__ __forceinline__ bool upstream_timed_out(const FrameCounters *ctr) {
    return (*(const volatile unsigned *)&ctr->status & kStTimeout) != 0u;
}

// ----------------------------------------------------------------------------------------------
// explicit IEEE binary32 operations (never contracted)
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ float ffma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// ln(x) for positive normal x: x = m 2^e with m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s),
// s = (m - 1)/(m + 1), by the odd Taylor series of atanh through s^11 in Horner form; e ln 2
// added with a two-part constant whose high part has 16 significant bits.
__device__ __forceinline__ float log_rn(float x) {
    unsigned bits = __float_as_uint(x);
    int e = (int)((bits >> 23) & 0xffu) - 127;
    float m = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);
    if (m > 1.41421353816986083984375f) {
        m = fmul(m, 0.5f);
        e += 1;
    }
    const float k3 = 0.3333333432674407958984375f;    // 1/3 rounded
    const float k5 = 0.20000000298023223876953125f;   // 1/5
    const float k7 = 0.14285714924335479736328125f;   // 1/7
    const float k9 = 0.111111111938953399658203125f;  // 1/9
    const float k11 = 0.0909090936183929443359375f;   // 1/11
    float s = fdiv(fsub(m, 1.0f), fadd(m, 1.0f));
    float s2 = fmul(s, s);
    float p = fmul(k11, s2);
    p = fmul(fadd(p, k9), s2);
    p = fmul(fadd(p, k7), s2);
    p = fmul(fadd(p, k5), s2);
    p = fmul(fadd(p, k3), s2);
    float s_2 = fadd(s, s);
    float lnm = fadd(s_2, fmul(s_2, p));
    float ef = (float)e;
    const float ln2_hi = 0.693145751953125f;
    const float ln2_lo = 1.428606765330187045037746429443359375e-06f;
    return fadd(fmul(ef, ln2_hi), fadd(fmul(ef, ln2_lo), lnm));
}

// e^x: x = k ln 2 + r with k = floor(x log2 e + 1/2), r reduced with the same two-part ln 2;
// e^r by its Taylor polynomial through r^8/8! (Horner); scaled by 2^k as two exact factors.
__device__ __forceinline__ float exp_rn(float x) {
    if (!(x == x)) return x;
    if (x < -87.0f) return 0.0f;
    if (x > 88.0f) return __uint_as_float(0x7f800000u);
    const float log2e = 1.44269502162933349609375f;
    const float ln2_hi = 0.693145751953125f;
    const float ln2_lo = 1.428606765330187045037746429443359375e-06f;
    float kf = floorf(fadd(fmul(x, log2e), 0.5f));
    float r = fsub(x, fmul(kf, ln2_hi));
    r = fsub(r, fmul(kf, ln2_lo));
    const float c2 = 0.5f;
    const float c3 = 0.16666667163372039794921875f;      // 1/3!
    const float c4 = 0.0416666679084300994873046875f;    // 1/4!
    const float c5 = 0.008333333767950534820556640625f;  // 1/5!
    const float c6 = 0.001388888922519981861114501953125f;       // 1/6!
    const float c7 = 0.0001984127011382952332496643066406f;      // 1/7!
    const float c8 = 2.48015876422868669033050537109375e-05f;    // 1/8!
    float p = fmul(c8, r);
    p = fmul(fadd(p, c7), r);
    p = fmul(fadd(p, c6), r);
    p = fmul(fadd(p, c5), r);
    p = fmul(fadd(p, c4), r);
    p = fmul(fadd(p, c3), r);
    p = fmul(fadd(p, c2), r);
    p = fmul(fadd(p, 1.0f), r);
    p = fadd(p, 1.0f);
    int k = (int)kf;
    int k1 = k / 2, k2 = k - k1;
    float s1 = __uint_as_float((unsigned)(k1 + 127) << 23);
    float s2 = __uint_as_float((unsigned)(k2 + 127) << 23);
    return fmul(fmul(p, s1), s2);
}

// Eq. 3: alpha0 exp(-q/2) >= tau  <=>  q <= t = 2 ln(alpha0 / tau), in binary32 with the own ln.
__device__ __forceinline__ float threshold_t(float alpha0, float tau) { return fmul(2.0f, log_rn(fdiv(alpha0, tau))); }

// Opacity from its logit, 1 / (1 + e^-x), with the own exp.
__device__ __forceinline__ float sigmoid_rn(float x) { return fdiv(1.0f, fadd(1.0f, exp_rn(-x))); }

// Exact ellipse/tile test (Algorithm 3, Eq. 9 with the linear coefficient halved): the tile
// [x0,x1] x [y0,y1] meets {a X^2 + 2 b X Y + c Y^2 <= t} about (u, v) iff the centre is inside,
// or some edge line's chord (roots of A s^2 + 2 B s + C) overlaps the edge.
__device__ __forceinline__ bool chord_hits(float A, float B, float C, float lo, float hi) {
    float D = fsub(fmul(B, B), fmul(A, C));
    if (!(D >= 0.0f)) return false;
    float e1 = fadd(fmul(A, lo), B);
    float e2 = fadd(fmul(A, hi), B);
    bool left = (e1 <= 0.0f) || (fmul(e1, e1) <= D);
    bool right = (e2 >= 0.0f) || (fmul(e2, e2) <= D);
    return left && right;
}

__device__ __forceinline__ bool tile_hits(float u, float v, float a, float b, float c, float t,
                                          float x0, float x1, float y0, float y1) {
    if (x0 <= u && u <= x1 && y0 <= v && v <= y1) return true;
    float lo = fsub(x0, u), hi = fsub(x1, u);
    float dy = fsub(y0, v);
    if (chord_hits(a, fmul(b, dy), fsub(fmul(fmul(c, dy), dy), t), lo, hi)) return true;
    dy = fsub(y1, v);
    if (chord_hits(a, fmul(b, dy), fsub(fmul(fmul(c, dy), dy), t), lo, hi)) return true;
    lo = fsub(y0, v);
    hi = fsub(y1, v);
    float dx = fsub(x0, u);
    if (chord_hits(c, fmul(b, dx), fsub(fmul(fmul(a, dx), dx), t), lo, hi)) return true;
    dx = fsub(x1, u);
    if (chord_hits(c, fmul(b, dx), fsub(fmul(fmul(a, dx), dx), t), lo, hi)) return true;
    return false;
}

// The exact test of a run of n <= 32 consecutive tiles tx_begin .. tx_begin+n-1 of tile row ty,
// bit j of the result for tile tx_begin + j.  Every sub-test evaluates the same binary32
// operations on the same operands as tile_hits, so each bit equals tile_hits of that tile; the
// quantities that depend only on the row (the top and bottom edge chords) are formed once, and the
// side chord at x = 16 (tx + 1) is shared by the right edge of tile tx and the left edge of tile
// tx + 1.
__device__ __forceinline__ bool chord_eval(float A, float B, float D, float lo, float hi) {
    float e1 = fadd(fmul(A, lo), B);
    float e2 = fadd(fmul(A, hi), B);
    bool left = (e1 <= 0.0f) || (fmul(e1, e1) <= D);
    bool right = (e2 >= 0.0f) || (fmul(e2, e2) <= D);
    return left && right;
}

__device__ __forceinline__ bool side_hits(float u, float a, float b, float c, float t, float x, float loy,
                                          float hiy) {
    const float dx = fsub(x, u);
    const float B = fmul(b, dx);
    const float C = fsub(fmul(fmul(a, dx), dx), t);
    const float D = fsub(fmul(B, B), fmul(c, C));
    if (!(D >= 0.0f)) return false;
    return chord_eval(c, B, D, loy, hiy);
}

__device__ __forceinline__ unsigned run_hits(int W, int H, float u, float v, float a, float b, float c, float t,
                                             int tx_begin, int n, int ty) {
    const float y0 = (float)(16 * ty), y1 = (float)min(16 * ty + 16, H);
    const bool cy = y0 <= v && v <= y1;
    const float dyt = fsub(y0, v), dyb = fsub(y1, v);
    const float Bt = fmul(b, dyt), Ct = fsub(fmul(fmul(c, dyt), dyt), t);
    const float Bb = fmul(b, dyb), Cb = fsub(fmul(fmul(c, dyb), dyb), t);
    const float Dt = fsub(fmul(Bt, Bt), fmul(a, Ct));
    const float Db = fsub(fmul(Bb, Bb), fmul(a, Cb));
    const bool top = Dt >= 0.0f, bot = Db >= 0.0f;
    const float loy = dyt, hiy = dyb;
    unsigned mask = 0;
    bool have = false, cached = false;        // side chord at the current tile's left edge
    for (int j = 0; j < n; ++j) {
        const int tx = tx_begin + j;
        const float x0 = (float)(16 * tx), x1 = (float)min(16 * tx + 16, W);
        bool h = cy && x0 <= u && u <= x1;
        const float lo = fsub(x0, u), hi = fsub(x1, u);
        if (!h && top) h = chord_eval(a, Bt, Dt, lo, hi);
        if (!h && bot) h = chord_eval(a, Bb, Db, lo, hi);
        if (!h) h = have ? cached : side_hits(u, a, b, c, t, x0, loy, hiy);
        have = false;
        if (!h) {
            cached = side_hits(u, a, b, c, t, x1, loy, hiy);
            have = true;
            h = cached;
        }
        mask |= (unsigned)h << j;
    }
    return mask;
}

// run_hits with most decisions taken without evaluating the test.  A tile spans its row's whole
// band [y0, y1], so it meets the ellipse {q <= t} iff its x-range [x0, x1] meets the x-range of the
// ellipse within the band -- an interval [xmin, xmax] about u, found in closed form: x as a function
// of dy on the ellipse's left boundary, (-b dy - sqrt(a t - det dy^2)) / a with det = a c - b^2, is
// convex with its minimum at dy = b hx / c (hx = the half width, sqrt(t c / det)), so its least value
// over the band is at that dy clamped into the band (likewise the right boundary, concave, greatest
// at dy = -b hx / c).  A tile that overlaps [xmin, xmax] by more than a margin eps meets the ellipse
// with room to spare, and so does the binary32 test (one of its edge chords or its centre test holds
// with a slack far above binary32 rounding); one that misses the interval, or whose band misses
// [-hy, hy], by more than eps fails every part of the test likewise.  Only tiles within eps of the
// interval's ends (at most two or three a row end) are tested, with tile_hits, which equals each bit
// of run_hits.  eps = 1/2 pixel plus 2^-8 of hx + hy bounds the interval's own error (approximate
// division and square root, relative ~1e-6; cancellation in a t - det dy^2 near the band ends, about
// 3.5e-4 hx) many times over.  Ellipses with det < 2^-12 a c (thin ones, where det cancels) and
// non-finite extents take run_hits.
__device__ __forceinline__ unsigned run_hits_banded(int W, int H, float u, float v, float a, float b, float c,
                                                    float t, float hx, float hy, int tx_begin, int n, int ty) {
    const float det = a * c - b * b;
    if (!(det > 2.44140625e-4f * a * c) || !(hx + hy < 1.0e6f)) return run_hits(W, H, u, v, a, b, c, t, tx_begin, n, ty);
    const float y0 = (float)(16 * ty), y1 = (float)min(16 * ty + 16, H);
    const float eps = 0.5f + 3.90625e-3f * (hx + hy);
    const float p0 = y0 - v, p1 = y1 - v;
    if (p0 > hy + eps || p1 < -hy - eps) return 0u;             // the band misses the ellipse
    const bool band_in = p0 < hy - eps && p1 > -hy + eps;        // ... or crosses it with room
    const float lo_dy = fmaxf(p0, -hy), hi_dy = fminf(p1, hy);
    const float ia = __fdividef(1.0f, a);
    const float ky = __fdividef(b * hx, c);
    const float dl = fminf(fmaxf(ky, lo_dy), hi_dy), dr = fminf(fmaxf(-ky, lo_dy), hi_dy);
    const float rl = fmaxf(a * t - det * dl * dl, 0.0f), rr = fmaxf(a * t - det * dr * dr, 0.0f);
    const float sl = rl > 0.0f ? rl * rsqrtf(rl) : 0.0f, sr = rr > 0.0f ? rr * rsqrtf(rr) : 0.0f;
    const float xmin = u + (-b * dl - sl) * ia, xmax = u + (-b * dr + sr) * ia;
    unsigned mask = 0;
    for (int j = 0; j < n; ++j) {
        const int tx = tx_begin + j;
        const float x0 = (float)(16 * tx), x1 = (float)min(16 * tx + 16, W);
        bool h;
        if (x1 < xmin - eps || x0 > xmax + eps)
            h = false;
        else if (band_in && x1 > xmin + eps && x0 < xmax - eps)
            h = true;
        else
            h = tile_hits(u, v, a, b, c, t, x0, x1, y0, y1);
        mask |= (unsigned)h << j;
    }
    return mask;
}

// The decisions of n <= 64 consecutive tiles tx_begin .. of row ty as a 64-bit mask, by the band
// interval of run_hits_banded turned into tile-index ranges: with y = x + eps, z = x - eps,
//   tiles tx >= floor((xmin + eps) / 16) have x1 > xmin + eps and tiles tx <= ceil((xmax - eps)/16) - 1
//   have x0 < xmax - eps (certain hits between, when the band crosses the ellipse with room);
//   tiles tx <= ceil((xmin - eps) / 16) - 2 have x1 < xmin - eps and tiles tx >= floor((xmax + eps)/16)
//   + 1 have x0 > xmax + eps (certain misses);
// the last image column's x1 is W, not 16 tx + 16, so its certain hit is checked directly.  Only the
// tiles between the two ranges (a few a row end) take tile_hits.  Thin ellipses take run_hits.
__device__ __forceinline__ unsigned long long run_hits_long(int W, int H, float u, float v, float a, float b,
                                                            float c, float t, float hx, float hy, int tx_begin,
                                                            int n, int ty) {
    const float det = a * c - b * b;
    if (!(det > 2.44140625e-4f * a * c) || !(hx + hy < 1.0e6f)) {
        unsigned long long m = 0;
        for (int k = 0; k < n; k += 8)
            m |= (unsigned long long)run_hits(W, H, u, v, a, b, c, t, tx_begin + k, min(8, n - k), ty) << k;
        return m;
    }
    const float y0 = (float)(16 * ty), y1 = (float)min(16 * ty + 16, H);
    const float eps = 0.5f + 3.90625e-3f * (hx + hy);
    const float p0 = y0 - v, p1 = y1 - v;
    if (p0 > hy + eps || p1 < -hy - eps) return 0ull;
    const bool band_in = p0 < hy - eps && p1 > -hy + eps;
    const float lo_dy = fmaxf(p0, -hy), hi_dy = fminf(p1, hy);
    const float ia = __fdividef(1.0f, a);
    const float ky = __fdividef(b * hx, c);
    const float dl = fminf(fmaxf(ky, lo_dy), hi_dy), dr = fminf(fmaxf(-ky, lo_dy), hi_dy);
    const float rl = fmaxf(a * t - det * dl * dl, 0.0f), rr = fmaxf(a * t - det * dr * dr, 0.0f);
    const float sl = rl > 0.0f ? rl * rsqrtf(rl) : 0.0f, sr = rr > 0.0f ? rr * rsqrtf(rr) : 0.0f;
    const float xmin = u + (-b * dl - sl) * ia, xmax = u + (-b * dr + sr) * ia;
    const int tx_end = tx_begin + n - 1;
    const int last_col = (W - 1) / 16;
    int m0 = (int)ceilf((xmin - eps) * 0.0625f) - 2;   // tiles <= m0 miss
    int m1 = (int)floorf((xmax + eps) * 0.0625f) + 1;  // tiles >= m1 miss
    int h0 = (int)floorf((xmin + eps) * 0.0625f);      // tiles in [h0, h1] hit (band_in)
    int h1 = (int)ceilf((xmax - eps) * 0.0625f) - 1;
    if (h0 == last_col && !((float)W > xmin + eps)) h0 = last_col + 1;
    if (!band_in || h1 < h0) {
        h0 = m1;                                       // no certain hits: [m0 + 1, m1 - 1] is open
        h1 = m1 - 1;
    }
    unsigned long long mask = 0;
    const int a0 = max(h0, tx_begin), a1 = min(h1, tx_end);
    if (a0 <= a1) {
        const int len = a1 - a0 + 1;
        mask = (len == 64 ? ~0ull : ((1ull << len) - 1ull)) << (a0 - tx_begin);
    }
    // the open tiles: (m0, h0) and (h1, m1), clipped to the run
    const int o0 = max(m0 + 1, tx_begin), o1 = min(h0 - 1, tx_end);
    for (int tx = o0; tx <= o1; ++tx) {
        const float x0 = (float)(16 * tx), x1 = (float)min(16 * tx + 16, W);
        if (tile_hits(u, v, a, b, c, t, x0, x1, y0, y1)) mask |= 1ull << (tx - tx_begin);
    }
    const int q0 = max(max(h1 + 1, h0), tx_begin), q1 = min(m1 - 1, tx_end);
    for (int tx = q0; tx <= q1; ++tx) {
        const float x0 = (float)(16 * tx), x1 = (float)min(16 * tx + 16, W);
        if (tile_hits(u, v, a, b, c, t, x0, x1, y0, y1)) mask |= 1ull << (tx - tx_begin);
    }
    return mask;
}

// Pixel-area rectangle of tile (tx, ty), clipped to the image.
__device__ __forceinline__ void tile_rect(const Cam &cam, int tx, int ty, float &x0, float &x1,
                                          float &y0, float &y1) {
    int xe = min(kTile * tx + kTile, cam.W), ye = min(kTile * ty + kTile, cam.H);
    x0 = (float)(kTile * tx);
    x1 = (float)xe;
    y0 = (float)(kTile * ty);
    y1 = (float)ye;
}

// Per-pixel skip decision: q = fma(fma(a, dx, b2 dy), dx, (c dy) dy) at the pixel sample,
// skipped when !(q <= t).
__device__ __forceinline__ float pixel_q(float a, float b2, float c, float dx, float dy) {
    float By = fmul(b2, dy);
    float Cy = fmul(fmul(c, dy), dy);
    return ffma(ffma(a, dx, By), dx, Cy);
}

// ----------------------------------------------------------------------------------------------
// host-side launchers (defined in the .cu files)
struct PreprocessArgs {
    BatchDesc B;
    Rec *recs;
    unsigned long long *keys;
    unsigned *vals;
    float4 *geo0, *geo1;             // per Gaussian: (u, v, a, b), (c, t, z bits, mask offset bits)
    int4 *geo2;                      // per Gaussian: (tx0, ty0, w, h) of the candidate box, 0 if unpaired
    unsigned *chunk_hits;            // pairs per 256-Gaussian chunk
    unsigned long long *chunk_base;  // exclusive scan of chunk_hits
    unsigned *counts;                // pairs per Gaussian
    // two-level order
    unsigned *tkeys;                 // 32-bit tile keys (aliases the pair key buffer)
    unsigned *chunk_vis;             // paired Gaussians per chunk
    unsigned long long *vis_base;    // exclusive scan of chunk_vis
    unsigned *dkey, *dval, *dkey_tmp, *dval_tmp;   // (depth bits, id) of paired Gaussians + ping-pong
    const unsigned *dsorted;         // ids in depth order (== dval after the sort)
    unsigned *chunk_hits2;           // pairs per chunk of 256 depth-sorted Gaussians
    unsigned long long *chunk_base2; // exclusive scan of chunk_hits2
    uint4 *big;                      // (record, request, output base lo, hi) of large Gaussians
    uint4 *mid;                      // the same for medium Gaussians
    // The count pass keeps each candidate unit's hit mask (one byte per run of kSeg tiles, a
    // Gaussian's units row-major from its offset in geo1.w; kNoMasks when the area was full) so
    // that emission reads the decisions instead of repeating the tests.
    unsigned char *masks;
    long long mask_cap;              // bytes, < 2^32
    FrameCounters *ctr;
    long long pair_cap;
    long long n_chunks;
};

void launch_pack_scene(const gs_gaussians &g, float4 *pos_opa, float4 *rs, void *sh, cudaStream_t s);
void launch_pre_count(const PreprocessArgs &a, cudaStream_t s);
void launch_req_pairs(const PreprocessArgs &a, unsigned long long *out, cudaStream_t s);
void launch_preprocess(const PreprocessArgs &a, cudaStream_t s, bool counted);
struct SortScratch;
int launch_preprocess_depth(const PreprocessArgs &a, const SortScratch &scr, cudaStream_t s, bool counted);
void launch_make_keys(const unsigned *tkeys, const unsigned *vals, const float4 *geo1, long long n,
                      unsigned long long *out, const FrameCounters *ctr, cudaStream_t s);
int preprocess_chunk();

struct SortScratch {
    unsigned *hist;                  // [8][256] digit counts
    unsigned *offs;                  // [8][256] exclusive digit offsets
    unsigned long long *desc;        // [sort_desc_words(max_tiles)] epoch-tagged look-back
                                     // descriptors: per tile, then per block of tiles
    long long max_tiles;
    unsigned *counts = nullptr;      // [256][rts_stride(max_tiles)] per-tile digit counts
                                     // (reduce-then-scan)
    int algo = 0;                    // 0 onesweep (decoupled look-back), 1 reduce-then-scan,
                                     // 2 onesweep passes fused into one cooperative launch
};

long long sort_max_tiles_for(long long n);
long long sort_desc_words(long long max_tiles);
long long rts_stride(long long max_tiles);
// Sorts by key bits [0, end_bit).  n_dev: device pointer to the pair count (clamped to cap);
// returns the number of passes (result in the tmp buffers when odd).
int launch_sort(unsigned long long *keys, unsigned *vals, unsigned long long *keys_tmp, unsigned *vals_tmp,
                const unsigned long long *n_dev, long long n_host, long long cap, int end_bit,
                const SortScratch &scr, FrameCounters *ctr, cudaStream_t s);
void launch_ranges(const unsigned long long *keys, const unsigned long long *n_dev, long long cap, int ntiles,
                   unsigned *starts, const FrameCounters *ctr, cudaStream_t s);
// 32-bit-key forms (depth bits alone, tile id alone) used by the two-level sort.
int launch_sort32(unsigned *keys, unsigned *vals, unsigned *keys_tmp, unsigned *vals_tmp,
                  const unsigned long long *n_dev, long long cap, int end_bit, const SortScratch &scr,
                  FrameCounters *ctr, cudaStream_t s);
void launch_ranges32(const unsigned *keys, const unsigned long long *n_dev, long long cap, int ntiles,
                     unsigned *starts, const FrameCounters *ctr, cudaStream_t s);
// Blend order of the tiles: decreasing list length class (see gs_render.cu).
void launch_tile_order(const unsigned *starts, int ntiles, unsigned *order, cudaStream_t s);

struct BlendArgs {
    BatchDesc B;
    const FrameCounters *ctr;        // status of the frame (a timed-out sort leaves nothing to blend)
    const Rec *recs;
    const unsigned *vals;
    const unsigned *starts;
    const unsigned *order;           // [total_tiles]: tile of each CTA (nullable: CTA i takes tile i)
    const unsigned long long *n_dev;
    long long cap;
    unsigned long long *evals;       // [2]: entries walked, entries passing q <= t (count mode)
    int variant;                     // launch shape, see launch_blend
    int count;                       // 1: instrumented variant filling evals
};
void launch_blend(const BlendArgs &a, cudaStream_t s);
int blend_variant_count();

struct BwdArgs {
    const FrameCounters *ctr;        // status of the forward's frame
    const Rec *recs;
    const unsigned *vals;
    const unsigned *starts;
    const unsigned long long *n_dev;
    long long cap;
    Opts opt;
    Cam cam;
    SceneView scene;
    int W, H, tiles_x, tiles_y;
    const float *dL_drgb;            // [3,H,W]
    const float *T_final;            // [H,W]
    const unsigned *last;            // [H,W]
    float *grad2d;                   // [P][10]: u, v, a, b, c, alpha0, r, g, b, -
    float *g_means, *g_scales, *g_quats, *g_opacity, *g_sh;
    int accumulate;
    int vec16;                       // g_quats and g_sh are 16-byte aligned: vector stores
};
// between (nullable): recorded after the reverse blend, before the per-Gaussian chain rule.
void launch_backward(const BwdArgs &a, cudaStream_t s, cudaEvent_t between);
int grad2d_floats();

}  // namespace gs
