// gs_preprocess.cu -- scene packing and the preprocess / exact-intersection / key-emission stage
// (Algorithm 4 of FlashGS, with the exact tile test of Algorithm 3 and Eq. 9, the opacity-aware
// threshold of Eq. 2-3 and the tight bounding box of Section 4.1).
//
// Kernels over chunks of 256 consecutive Gaussians:
//   k_pre_count  each thread culls and projects its Gaussian and finds its candidate tiles (tight
//                box); then the exact tile tests run load-balanced over the whole CTA: the
//                candidate box of every Gaussian is cut into units (runs of up to 8 tiles of one
//                tile row), a block scan numbers the units of the chunk, and each step the 256
//                threads take 256 consecutive units, whatever Gaussians they belong to, testing a
//                unit's tiles with the row's shared terms formed once (run_hits).  This
//                generalises the paper's size-aware remapping of a large ellipse onto a warp
//                (Section 5.1.2) to any mix of sizes.  It writes the chunk's hit count, the
//                geometry of paired Gaussians, and their render records with the SH colour
//                (Algorithm 4, last step: colour only for Gaussians that are used);
//   k_chunk_scan exclusive scan of the chunk hit counts (CTAs that each sum their predecessors' counts);
//   k_pre_emit   repeats the tests and writes every hit at its chunk's base + its rank in unit
//                order, so pairs land in (Gaussian id, tile row-major) order -- deterministic,
//                unlike the paper's atomicAdd slots, and without any inter-CTA waiting, so a
//                chunk holding a huge Gaussian delays nobody else.
// The depth-ordered variant (k_vis_compact, k_emit_sum, k_pre_emit<true>, k_emit_big) emits the
// same pairs Gaussian by Gaussian in depth order for the two-level sort.
#include "gs_internal.cuh"

namespace gs {

constexpr int kPreBlock = 256;
constexpr int kPackBlock = 128;

int preprocess_chunk() { return kPreBlock; }

// ------------------------------------------------------------------------------------------ pack
// Canonical AoS arrays -> the internal position, scale/rotation and SH arrays.  The SH block of
// a CTA is contiguous in both layouts (48 floats per Gaussian), so it is copied four floats at a
// time -- as float4s, or as four binary16 values (round to nearest even) when g.sh_half.
__global__ void __launch_bounds__(kPackBlock) k_pack_scene(gs_gaussians g, float4 *pos_opa, float4 *rs, void *sh) {
    const long long base = (long long)blockIdx.x * kPackBlock;
    const int n = (int)min((long long)kPackBlock, g.P - base);
    const float *src = g.sh + base * 48;
    if (g.sh_half) {
        uint2 *dst = reinterpret_cast<uint2 *>(sh) + base * kShPlanes;
        for (int k = threadIdx.x; k < n * kShPlanes; k += kPackBlock) {
            const __half2 a = __floats2half2_rn(src[4 * k], src[4 * k + 1]);
            const __half2 b = __floats2half2_rn(src[4 * k + 2], src[4 * k + 3]);
            dst[k] = make_uint2(*reinterpret_cast<const unsigned *>(&a), *reinterpret_cast<const unsigned *>(&b));
        }
    } else {
        float4 *dst = reinterpret_cast<float4 *>(sh) + base * kShPlanes;
        for (int k = threadIdx.x; k < n * kShPlanes; k += kPackBlock)
            dst[k] = make_float4(src[4 * k], src[4 * k + 1], src[4 * k + 2], src[4 * k + 3]);
    }
    const long long i = base + threadIdx.x;
    if (threadIdx.x < n) {
        const float *m = g.means + 3 * i;
        const float *s = g.scales + 3 * i;
        const float *q = g.quats + 4 * i;
        pos_opa[i] = make_float4(m[0], m[1], m[2], g.opacity[i]);
        rs[2 * i] = make_float4(s[0], s[1], s[2], 0.0f);
        rs[2 * i + 1] = make_float4(q[0], q[1], q[2], q[3]);
    }
}

void launch_pack_scene(const gs_gaussians &g, float4 *pos_opa, float4 *rs, void *sh, cudaStream_t s) {
    long long blocks = (g.P + kPackBlock - 1) / kPackBlock;
    k_pack_scene<<<(unsigned)blocks, kPackBlock, 0, s>>>(g, pos_opa, rs, sh);
}

// ------------------------------------------------------------------------------------------ SH
// Real SH basis through degree 3 (3DGS sign/order convention), constants are the closed forms
// 1/(2 sqrt pi), sqrt(3/(4 pi)), sqrt(15/pi)/2, sqrt(5/pi)/4, sqrt(15/pi)/4, sqrt(35/(2 pi))/4,
// sqrt(105/pi)/2, sqrt(21/(2 pi))/4, sqrt(7/pi)/4, sqrt(105/pi)/4 evaluated to float.
//
// A Gaussian's colour is evaluated by four consecutive lanes: lane `part` reads SH planes 3 part ..
// 3 part + 2 (floats 12 part .. 12 part + 11, i.e. coefficients 4 part .. 4 part + 3 of the three
// channels) -- three 16-byte loads in flight per lane instead of twelve in one lane, whose
// registers the count pass does not have -- and its partial sums are added across the four
// lanes in a fixed order.  Returns the clamped colour (identical on the four lanes).
__device__ __forceinline__ void sh_colour4(const SceneView &S, long long gid, const Cam &cam, float mx, float my,
                                           float mz, int part, unsigned gmask, float rgb[3]) {
    const int deg = S.sh_degree;
    const int ncoef = (deg + 1) * (deg + 1);
    const int nplanes = (3 * ncoef + 3) / 4;
    float4 pl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int plane = 3 * part + k;
        pl[k] = plane < nplanes ? sh_plane(S, gid, plane) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float K0 = 0.28209479177387814f;
    const float K1 = 0.48860251190291992f;
    const float K2a = 1.0925484305920792f, K2b = 0.31539156525252005f, K2c = 0.54627421529603959f;
    const float K3a = 0.59004358992664352f, K3b = 2.8906114426405538f, K3c = 0.45704579946446572f;
    const float K3d = 0.3731763325901154f, K3e = 1.4453057213202769f;
    const float dx = mx - cam.campos[0], dy = my - cam.campos[1], dz = mz - cam.campos[2];
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    const float x = dx * inv, y = dy * inv, z = dz * inv;
    const float xx = x * x, yy = y * y, zz = z * z;
    // the four basis functions of this lane's coefficients
    float Y[4];
    if (part == 0) {
        Y[0] = K0;
        Y[1] = -K1 * y;
        Y[2] = K1 * z;
        Y[3] = -K1 * x;
    } else if (part == 1) {
        Y[0] = K2a * x * y;
        Y[1] = -K2a * y * z;
        Y[2] = K2b * (2.0f * zz - xx - yy);
        Y[3] = -K2a * x * z;
    } else if (part == 2) {
        Y[0] = K2c * (xx - yy);
        Y[1] = -K3a * y * (3.0f * xx - yy);
        Y[2] = K3b * x * y * z;
        Y[3] = -K3c * y * (4.0f * zz - xx - yy);
    } else {
        Y[0] = K3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
        Y[1] = -K3c * x * (4.0f * zz - xx - yy);
        Y[2] = K3e * z * (xx - yy);
        Y[3] = -K3a * x * (xx - 3.0f * yy);
    }
    // float f = 12 part + j belongs to coefficient 4 part + j / 3 of channel j % 3
    float acc[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float e[4] = {pl[k].x, pl[k].y, pl[k].z, pl[k].w};
#pragma unroll
        for (int j4 = 0; j4 < 4; ++j4) {
            const int j = 4 * k + j4, i = j / 3, ch = j - 3 * (j / 3);
            acc[ch] += (4 * part + i < ncoef ? Y[i] : 0.0f) * e[j4];
        }
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float a = acc[ch];
        a += __shfl_xor_sync(gmask, a, 1);    // (p0 + p1), (p2 + p3)
        a += __shfl_xor_sync(gmask, a, 2);    // (p0 + p1) + (p2 + p3) on every lane
        rgb[ch] = fmaxf(a + 0.5f, 0.0f);
    }
}

// ------------------------------------------------------------------------------------------ geometry
struct Geom {
    float u, v, a, b, c, t, t_full, z, alpha0, hx, hy;
    int tx0, tx1, ty0, ty1;
};

// Phase 1 of a Gaussian's geometry, run by every thread of the count pass: the cull (Alg. 4: z >
// near, opacity > tau) and a conservative off-screen bound.  Returns true when the Gaussian may
// have a candidate tile; p (camera-space mean) and alpha0 are left for phase 2.  Binary32
// evaluation order of the definition (see the header).
__device__ __forceinline__ bool cull_and_bound(const SceneView &S, long long gid, const Cam &cam, const Opts &o,
                                               float p[3], float &alpha0, bool &passed_cull) {
    const float4 po = __ldg(S.pos_opa + gid);
    // the scales are loaded with the position, before the cull decides whether they are needed:
    // one memory round trip for the phase instead of two
    const float4 sc = __ldg(rs_of(S, gid));
    const float *R = cam.R;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float s = fmul(R[3 * i], po.x);
        s = fadd(s, fmul(R[3 * i + 1], po.y));
        s = fadd(s, fmul(R[3 * i + 2], po.z));
        p[i] = fadd(s, cam.t[i]);
    }
    alpha0 = S.activated ? po.w : sigmoid_rn(po.w);
    if (!(p[2] > cam.near_z)) return false;
    if (!(alpha0 > o.tau)) return false;
    passed_cull = true;
    // Conservative screen-extent test, before any exact arithmetic of the covariance.
    // Sigma <= s_max^2 I, so Sigma'00 <= s_max^2 |M0|^2 + dilation (M0 = first row of J W) and
    // {q <= t} lies within u +- sqrt(t Sigma'00).  Every factor here is an upper estimate from
    // the fast approximate unit (relative errors near 1e-6), padded by 2% and two pixels: a
    // Gaussian whose bound misses the image can have no candidate tile, and skipping it
    // changes no result.  (NaN bounds compare false and keep the Gaussian.)
    float tb = 2.0f * __logf(__fdividef(alpha0, o.tau)) * 1.01f + 0.01f;
    if (o.cap_3sigma && tb > 9.01f) tb = 9.01f;
    const float sraw = fmaxf(fmaxf(sc.x, sc.y), sc.z);
    const float smax = S.activated ? sraw : __expf(sraw) * 1.01f;
    const float iz = __fdividef(1.0f, p[2]);
    float rx = p[0] * iz, ry = p[1] * iz;
    if (o.clamp_fov) {
        rx = fminf(fmaxf(rx, -cam.limx), cam.limx);
        ry = fminf(fmaxf(ry, -cam.limy), cam.limy);
    }
    const float a00 = cam.fx * iz, a02 = -cam.fx * rx * iz;
    const float a11 = cam.fy * iz, a12 = -cam.fy * ry * iz;
    float m0 = 0.0f, m1 = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float e0 = a00 * R[k] + a02 * R[6 + k];
        const float e1 = a11 * R[3 + k] + a12 * R[6 + k];
        m0 += e0 * e0;
        m1 += e1 * e1;
    }
    const float x2 = tb * (smax * smax * m0 + o.dilation), y2 = tb * (smax * smax * m1 + o.dilation);
    float hxb = (x2 > 0.0f ? x2 * rsqrtf(x2) : 0.0f) * 1.02f + 2.0f;
    float hyb = (y2 > 0.0f ? y2 * rsqrtf(y2) : 0.0f) * 1.02f + 2.0f;
    if (o.intersect == 1) {
        // 3DGS square: r <= ceil(3 sqrt(trace Sigma')), trace <= s_max^2 (|M0|^2 + |M1|^2) + 2 dilation
        const float r2 = smax * smax * (m0 + m1) + 2.0f * o.dilation;
        const float rb = 3.0f * (r2 > 0.0f ? r2 * rsqrtf(r2) : 0.0f) * 1.02f + 3.0f;
        hxb = rb;
        hyb = rb;
    }
    const float uu = cam.fx * p[0] * iz + cam.cx, vv = cam.fy * p[1] * iz + cam.cy;
    return !(uu + hxb < 0.0f || uu - hxb >= (float)(kTile * cam.tiles_x) || vv + hyb < 0.0f ||
             vv - hyb >= (float)(kTile * cam.tiles_y));
}

// Phase 2, run only for the Gaussians that passed phase 1 (compacted across the CTA): the exact
// threshold, 3D covariance, EWA projection, conic and candidate tile box; false if the conic is
// degenerate or the box is empty.
__device__ __forceinline__ bool exact_geometry(const SceneView &S, long long gid, const Cam &cam, const Opts &o,
                                               const float p[3], float alpha0, Geom &G) {
    const float *R = cam.R;
    const float4 sc = __ldg(rs_of(S, gid));
    // Eq. 3: alpha0 exp(-q/2) >= tau  <=>  q <= 2 ln(alpha0 / tau)
    const float t_full = threshold_t(alpha0, o.tau);
    float t = t_full;
    if (o.cap_3sigma && t > 9.0f) t = 9.0f;
    // Sigma = R_q diag(s^2) R_q^T
    float s0 = sc.x, s1 = sc.y, s2 = sc.z;
    if (!S.activated) {
        s0 = exp_rn(s0);
        s1 = exp_rn(s1);
        s2 = exp_rn(s2);
    }
    const float4 q4 = __ldg(rs_of(S, gid) + 1);
    float qw = q4.x, qx = q4.y, qy = q4.z, qz = q4.w;
    float n2 = fmul(qw, qw);
    n2 = fadd(n2, fmul(qx, qx));
    n2 = fadd(n2, fmul(qy, qy));
    n2 = fadd(n2, fmul(qz, qz));
    if (!(n2 > 0.0f)) return false;
    const float qn = fsqrt(n2);
    qw = fdiv(qw, qn);
    qx = fdiv(qx, qn);
    qy = fdiv(qy, qn);
    qz = fdiv(qz, qn);
    const float yy = fmul(qy, qy), zz = fmul(qz, qz), xx = fmul(qx, qx);
    const float xy = fmul(qx, qy), xz = fmul(qx, qz), yz = fmul(qy, qz);
    const float wx = fmul(qw, qx), wy = fmul(qw, qy), wz = fmul(qw, qz);
    float r[9];
    r[0] = fsub(1.0f, fmul(2.0f, fadd(yy, zz)));
    r[1] = fmul(2.0f, fsub(xy, wz));
    r[2] = fmul(2.0f, fadd(xz, wy));
    r[3] = fmul(2.0f, fadd(xy, wz));
    r[4] = fsub(1.0f, fmul(2.0f, fadd(xx, zz)));
    r[5] = fmul(2.0f, fsub(yz, wx));
    r[6] = fmul(2.0f, fsub(xz, wy));
    r[7] = fmul(2.0f, fadd(yz, wx));
    r[8] = fsub(1.0f, fmul(2.0f, fadd(xx, yy)));
    const float d0 = fmul(s0, s0), d1 = fmul(s1, s1), d2 = fmul(s2, s2);
    float Sg[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            float acc = fmul(fmul(r[3 * i], d0), r[3 * j]);
            acc = fadd(acc, fmul(fmul(r[3 * i + 1], d1), r[3 * j + 1]));
            acc = fadd(acc, fmul(fmul(r[3 * i + 2], d2), r[3 * j + 2]));
            Sg[3 * i + j] = acc;
            Sg[3 * j + i] = acc;
        }
    // projection to pixel-area coordinates
    const float u = fadd(fdiv(fmul(cam.fx, p[0]), p[2]), cam.cx);
    const float v = fadd(fdiv(fmul(cam.fy, p[1]), p[2]), cam.cy);
    // EWA Jacobian of the perspective map, with the 1.3 tan(half fov) clamp
    float tx = p[0], ty = p[1];
    if (o.clamp_fov) {
        float txz = fdiv(p[0], p[2]), tyz = fdiv(p[1], p[2]);
        txz = txz < -cam.limx ? -cam.limx : (txz > cam.limx ? cam.limx : txz);
        tyz = tyz < -cam.limy ? -cam.limy : (tyz > cam.limy ? cam.limy : tyz);
        tx = fmul(txz, p[2]);
        ty = fmul(tyz, p[2]);
    }
    const float zsq = fmul(p[2], p[2]);
    const float j00 = fdiv(cam.fx, p[2]);
    const float j02 = -fdiv(fmul(cam.fx, tx), zsq);
    const float j11 = fdiv(cam.fy, p[2]);
    const float j12 = -fdiv(fmul(cam.fy, ty), zsq);
    float M[6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        M[k] = fadd(fmul(j00, R[k]), fmul(j02, R[6 + k]));
        M[3 + k] = fadd(fmul(j11, R[3 + k]), fmul(j12, R[6 + k]));
    }
    float N[6];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float acc = fmul(M[3 * i], Sg[k]);
            acc = fadd(acc, fmul(M[3 * i + 1], Sg[3 + k]));
            acc = fadd(acc, fmul(M[3 * i + 2], Sg[6 + k]));
            N[3 * i + k] = acc;
        }
    float s00 = fmul(N[0], M[0]);
    s00 = fadd(s00, fmul(N[1], M[1]));
    s00 = fadd(s00, fmul(N[2], M[2]));
    s00 = fadd(s00, o.dilation);
    float s01 = fmul(N[0], M[3]);
    s01 = fadd(s01, fmul(N[1], M[4]));
    s01 = fadd(s01, fmul(N[2], M[5]));
    float s11 = fmul(N[3], M[3]);
    s11 = fadd(s11, fmul(N[4], M[4]));
    s11 = fadd(s11, fmul(N[5], M[5]));
    s11 = fadd(s11, o.dilation);
    const float det = fsub(fmul(s00, s11), fmul(s01, s01));
    if (!(det > 0.0f)) return false;
    G.a = fdiv(s11, det);
    G.b = fdiv(-s01, det);
    G.c = fdiv(s00, det);
    // tight box of {q <= t}: half extents sqrt(t Sigma'00), sqrt(t Sigma'11), padded by 1 px
    const float hx = fsqrt(fmul(t, s00));
    const float hy = fsqrt(fmul(t, s11));
    float fx0 = floorf(fmul(fsub(fsub(u, hx), 1.0f), 0.0625f));
    float fx1 = floorf(fmul(fadd(fadd(u, hx), 1.0f), 0.0625f));
    float fy0 = floorf(fmul(fsub(fsub(v, hy), 1.0f), 0.0625f));
    float fy1 = floorf(fmul(fadd(fadd(v, hy), 1.0f), 0.0625f));
    if (o.intersect == 1) {
        // 3DGS pairs (Eq. 1; Alg. 1 radii; Alg. 2): r = ceil(3 sqrt(lambda_max)) of Sigma', every
        // tile of [u - r, u + r] x [v - r, v + r] (the discriminant clamped at 0 against rounding)
        const float mid = fmul(0.5f, fadd(s00, s11));
        const float disc = fsub(fmul(mid, mid), det);
        const float lam = fadd(mid, fsqrt(disc > 0.0f ? disc : 0.0f));
        const float rad = ceilf(fmul(3.0f, fsqrt(lam)));
        fx0 = floorf(fmul(fsub(u, rad), 0.0625f));
        fx1 = floorf(fmul(fadd(u, rad), 0.0625f));
        fy0 = floorf(fmul(fsub(v, rad), 0.0625f));
        fy1 = floorf(fmul(fadd(v, rad), 0.0625f));
    }
    const float mxx = (float)(cam.tiles_x - 1), mxy = (float)(cam.tiles_y - 1);
    if (!(fx1 >= 0.0f) || !(fy1 >= 0.0f) || !(fx0 <= mxx) || !(fy0 <= mxy)) return false;
    G.tx0 = fx0 < 0.0f ? 0 : (int)fx0;
    G.tx1 = fx1 > mxx ? cam.tiles_x - 1 : (int)fx1;
    G.ty0 = fy0 < 0.0f ? 0 : (int)fy0;
    G.ty1 = fy1 > mxy ? cam.tiles_y - 1 : (int)fy1;
    G.u = u;
    G.v = v;
    G.hx = hx;
    G.hy = hy;
    G.t = t;
    G.t_full = t_full;
    G.z = p[2];
    G.alpha0 = alpha0;
    return true;
}

// ------------------------------------------------------------------------------------------ kernels
struct PreSmem {
    float u[kPreBlock], v[kPreBlock], a[kPreBlock], b[kPreBlock], c[kPreBlock], t[kPreBlock];
    unsigned zb[kPreBlock];
    int tx0[kPreBlock], ty0[kPreBlock], w[kPreBlock];
    int cstart[kPreBlock + 1];        // exclusive scan of candidate-tile counts
    unsigned cnt[kPreBlock];          // pairs of each Gaussian of the chunk
    unsigned char req[kPreBlock];     // request of each Gaussian (batch index)
    unsigned wsum[kPreBlock / 32];
    unsigned long long pbase[kPreBlock];   // depth order: first output position of each Gaussian
    unsigned run[kPreBlock];               // depth order: hits of each Gaussian written so far
    unsigned xr[kPreBlock];                // depth order: exclusive hit rank of each slot of a step
    unsigned moff[kPreBlock];              // first hit-mask byte of each Gaussian (emission)
    unsigned long long mbase;              // first hit-mask byte of the chunk (count pass)
};

constexpr unsigned kNoMasks = 0xffffffffu;   // geo1.w: the unit masks were not kept

// Depth-ordered emission by footprint: Gaussians with more candidate tiles than kBigCand are
// emitted by k_emit_big (a CTA each), those above kMidCand by k_emit_mid (a warp each), the rest
// by their rank chunk in k_pre_emit.  Near Gaussians are large and neighbours in depth order, so a
// rank chunk full of them would otherwise hold up the whole pass.
constexpr int kBigCand = 4096;
constexpr int kMidCand = 64;

// Work unit of the exact tests: a run of up to kSeg consecutive candidate tiles of one tile row
// of one Gaussian (row-major), tested by one thread with the row's shared terms (run_hits).
constexpr int kSeg = 8;

// Emission stages each step's hits (tile id and Gaussian slot, in output order) in shared memory
// and then writes them as consecutive runs, so global stores are coalesced.
struct EmitSmem {
    PreSmem P;
    unsigned stile[kPreBlock * kSeg];
    unsigned char sg[kPreBlock * kSeg];
};
__device__ __forceinline__ int units_of(int w, int h) { return h * ((w + kSeg - 1) / kSeg); }

struct Unit {
    int g, tx, ty, n;
};

// Unit slot -> (Gaussian g of the CTA, first tile, row, length); slot s belongs to the last g with
// cstart[g] <= s and is its k-th unit in row-major order.
__device__ __forceinline__ Unit unit_of(const PreSmem &S, int slot) {
    int lo = 0, hi = kPreBlock - 1;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int mid = (lo + hi + 1) >> 1;
        if (S.cstart[mid] <= slot)
            lo = mid;
        else
            hi = mid - 1;
    }
    Unit U;
    U.g = lo;
    const int k = slot - S.cstart[lo];
    const int w = S.w[lo];
    const int segs = (w + kSeg - 1) / kSeg;
    const int dy = k / segs;
    const int seg = k - dy * segs;
    U.tx = S.tx0[lo] + seg * kSeg;
    U.ty = S.ty0[lo] + dy;
    U.n = min(kSeg, w - seg * kSeg);
    return U;
}

__device__ __forceinline__ unsigned unit_hits(const PreSmem &S, const BatchDesc &B, const Unit &U) {
    if (B.r[S.req[U.g]].opt.intersect == 1) return (1u << U.n) - 1u;    // 3DGS square: every tile
    const Cam &cam = B.r[S.req[U.g]].cam;
    return run_hits(cam.W, cam.H, S.u[U.g], S.v[U.g], S.a[U.g], S.b[U.g], S.c[U.g], S.t[U.g], U.tx, U.n, U.ty);
}

// Emission: the count pass's decision for a unit (its kept mask byte), else the test again.
__device__ __forceinline__ unsigned kept_hits(const PreSmem &S, const PreprocessArgs &A, const Unit &U, int slot) {
    const unsigned mo = S.moff[U.g];
    return mo != kNoMasks ? (unsigned)A.masks[(unsigned long long)mo + (unsigned)(slot - S.cstart[U.g])]
                          : unit_hits(S, A.B, U);
}

// Block exclusive scan of one unsigned per thread (uses S.wsum); returns the exclusive prefix and
// writes the block total to *total.
__device__ __forceinline__ unsigned block_excl(PreSmem &S, unsigned x, unsigned *total) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) S.wsum[warp] = incl;
    __syncthreads();
    unsigned wex = 0, tot = 0;
#pragma unroll
    for (int w2 = 0; w2 < kPreBlock / 32; ++w2) {
        const unsigned y = S.wsum[w2];
        wex += w2 < warp ? y : 0u;
        tot += y;
    }
    __syncthreads();
    *total = tot;
    return wex + incl - x;
}

// Block exclusive scan of one int per thread into S.cstart; returns the block total.
__device__ __forceinline__ int block_scan_cand(PreSmem &S, int ncand) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int incl = ncand;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) S.wsum[warp] = (unsigned)incl;
    __syncthreads();
    int wex = 0, total = 0;
#pragma unroll
    for (int w2 = 0; w2 < kPreBlock / 32; ++w2) {
        const int x = (int)S.wsum[w2];
        wex += w2 < warp ? x : 0;
        total += x;
    }
    S.cstart[tid] = wex + incl - ncand;
    if (tid == 0) S.cstart[kPreBlock] = total;
    __syncthreads();
    return total;
}

// Shared state of the count pass.  The exact work is done on compact slots: slot k holds the k-th
// Gaussian of the chunk (in id order) that passed the cull and the off-screen bound, so warps
// running the exact geometry, the tile tests and the colour are full however sparse the
// survivors are (a city frame keeps about one Gaussian in six of a chunk).
struct CountSmem {
    float u[kPreBlock], v[kPreBlock], a[kPreBlock], b[kPreBlock], c[kPreBlock], t[kPreBlock];
    int tx0[kPreBlock], ty0[kPreBlock], w[kPreBlock];
    int cstart[kPreBlock + 1];        // exclusive scan of the slots' unit counts (mask bytes)
    int istart[kPreBlock + 1];        // exclusive scan of the slots' work items
    unsigned cnt[kPreBlock];          // pairs of each slot
    float4 pa[kPreBlock];             // slot: camera-space mean and opacity from phase 1
    float z[kPreBlock], gl[kPreBlock];    // slot: depth and log2(alpha0) (the record's G)
    float2 hxy[kPreBlock];                // slot: half extents of the {q <= t} box
    int h[kPreBlock];                     // slot: candidate rows
    short sl[kPreBlock];              // slot -> Gaussian (thread) of the chunk
    short slot_of[kPreBlock];         // Gaussian -> slot, -1 when it has none
    short vlist[kPreBlock];           // paired slots in slot order
    unsigned wsum[kPreBlock / 32], wsum2[kPreBlock / 32];
    unsigned long long mbase;         // first hit-mask byte of the chunk
};

// Work items of the count pass: a box at least kWideBox tiles wide is cut into items of up to
// kLong tiles of one row (kLong / kSeg mask bytes, decided by run_hits_long); narrower boxes into
// the units themselves.  The mask bytes keep the unit layout either way.
constexpr int kLong = 64;
constexpr int kWideBox = 16;
static_assert(kLong % kSeg == 0, "a long item covers whole units");

// Pass 1: geometry, exact tests counted over all candidate tiles of the chunk (load-balanced),
// render records of paired Gaussians, the chunk's pair count, and each paired Gaussian's
// geometry for emission.  Phase 1 (cull and off-screen bound) runs on every thread; the survivors
// are compacted into slots; phase 2 (exact geometry), the tile tests and the records run on slots.
__global__ void __launch_bounds__(kPreBlock, 8) k_pre_count(const __grid_constant__ PreprocessArgs A) {
    __shared__ CountSmem S;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long chunk = blockIdx.x;
    const int ri = req_of_chunk(A.B, chunk);
    const ReqDesc &R = A.B.r[ri];
    const long long g0 = (chunk - R.chunk0) * kPreBlock;     // first Gaussian of the chunk
    const Cam &cam = R.cam;

    // ---- phase 1 on every Gaussian, then compaction of the survivors (id order kept)
    float p[3] = {0.f, 0.f, 0.f}, alpha0 = 0.f;
    bool passed_cull = false, cand = false;
    if (g0 + tid < R.scene.P) cand = cull_and_bound(R.scene, g0 + tid, cam, R.opt, p, alpha0, passed_cull);
    const unsigned bal = __ballot_sync(0xffffffffu, cand);
    if (lane == 0) S.wsum[warp] = __popc(bal);
    const unsigned n_in_block = (unsigned)__syncthreads_count(passed_cull);
    int before = 0, ns = 0;
#pragma unroll
    for (int w2 = 0; w2 < kPreBlock / 32; ++w2) {
        const int x = (int)S.wsum[w2];
        before += w2 < warp ? x : 0;
        ns += x;
    }
    const int myslot = cand ? before + __popc(bal & ((1u << lane) - 1u)) : -1;
    S.slot_of[tid] = (short)myslot;
    if (cand) {
        S.sl[myslot] = (short)tid;
        S.pa[myslot] = make_float4(p[0], p[1], p[2], alpha0);
    }
    __syncthreads();

    // ---- phase 2 on slot tid; its geometry goes to shared memory (registers stay free for the tests)
    int units = 0, items = 0;
    if (tid < ns) {
        Geom G;
        const float4 pa = S.pa[tid];
        const float pp[3] = {pa.x, pa.y, pa.z};
        if (exact_geometry(R.scene, g0 + S.sl[tid], cam, R.opt, pp, pa.w, G)) {
            const int w = G.tx1 - G.tx0 + 1, h = G.ty1 - G.ty0 + 1;
            S.u[tid] = G.u;
            S.v[tid] = G.v;
            S.a[tid] = G.a;
            S.b[tid] = G.b;
            S.c[tid] = G.c;
            S.t[tid] = G.t;
            S.tx0[tid] = G.tx0;
            S.ty0[tid] = G.ty0;
            S.w[tid] = w;
            S.h[tid] = h;
            S.z[tid] = G.z;
            S.gl[tid] = log_rn(G.alpha0) * 1.4426950408889634f;     // log2(alpha0)
            S.hxy[tid] = make_float2(G.hx, G.hy);
            units = units_of(w, h);
            // the colour reads this Gaussian's SH block once the tile tests have run: start
            // bringing the (at most two) 128-byte lines it spans into L2 now
            {
                const long long gid = g0 + S.sl[tid];
                const size_t bytes = R.scene.sh_half ? kShPlanes * 8 : kShPlanes * 16;
                const char *sp = (const char *)R.scene.sh + (size_t)gid * bytes;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(sp));
                asm volatile("prefetch.global.L2 [%0];" ::"l"(sp + bytes - 1));
            }
            items = w >= kWideBox ? h * ((w + kLong - 1) / kLong) : units;
        }
    }
    if (units == 0) S.w[tid] = 1;
    S.cnt[tid] = 0;
    // block scans of the slots' units and items (wsum and wsum2: every read of phase 1's counts is
    // behind the barrier)
    int ctotal, itotal;
    {
        int incl = units, incl2 = items;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            const int y2 = __shfl_up_sync(0xffffffffu, incl2, o);
            if (lane >= o) {
                incl += y;
                incl2 += y2;
            }
        }
        if (lane == 31) {
            S.wsum[warp] = (unsigned)incl;
            S.wsum2[warp] = (unsigned)incl2;
        }
        __syncthreads();
        int wex = 0, wex2 = 0;
        ctotal = 0;
        itotal = 0;
#pragma unroll
        for (int w2 = 0; w2 < kPreBlock / 32; ++w2) {
            const int x = (int)S.wsum[w2], x2 = (int)S.wsum2[w2];
            wex += w2 < warp ? x : 0;
            wex2 += w2 < warp ? x2 : 0;
            ctotal += x;
            itotal += x2;
        }
        S.cstart[tid] = wex + incl - units;
        S.istart[tid] = wex2 + incl2 - items;
        if (tid == 0) {
            S.cstart[kPreBlock] = ctotal;
            S.istart[kPreBlock] = itotal;
            // one range of mask bytes per chunk (kept only while the area lasts)
            S.mbase = ctotal > 0 ? atomicAdd(&A.ctr->mask_used, (unsigned long long)ctotal) : 0ull;
        }
        __syncthreads();
    }
    const bool keep = S.mbase + (unsigned long long)ctotal <= (unsigned long long)A.mask_cap;

    // ---- exact tile tests, 256 work items per step over all slots
    const bool square = R.opt.intersect == 1;
    for (int base = 0; base < itotal; base += kPreBlock) {
        const int s = base + tid;
        if (s >= itotal) continue;
        // slot of item s: the last slot g with istart[g] <= s
        int g = 0, hi = kPreBlock - 1;
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const int mid = (g + hi + 1) >> 1;
            if (S.istart[mid] <= s)
                g = mid;
            else
                hi = mid - 1;
        }
        const int k = s - S.istart[g];
        const int w = S.w[g];
        const float2 hxy = S.hxy[g];
        unsigned pc;
        if (w >= kWideBox) {
            const int ipr = (w + kLong - 1) / kLong;
            const int dy = k / ipr, j = k - dy * ipr;
            const int tx = S.tx0[g] + kLong * j, n = min(kLong, w - kLong * j);
            const unsigned long long m =
                square ? (n == 64 ? ~0ull : (1ull << n) - 1ull)
                       : run_hits_long(cam.W, cam.H, S.u[g], S.v[g], S.a[g], S.b[g], S.c[g], S.t[g], hxy.x, hxy.y,
                                       tx, n, S.ty0[g] + dy);
            if (keep) {
                const unsigned long long mo =
                    S.mbase + (unsigned long long)(S.cstart[g] + dy * ((w + kSeg - 1) / kSeg) + (kLong / kSeg) * j);
                for (int q = 0; q * kSeg < n; ++q) A.masks[mo + q] = (unsigned char)(m >> (kSeg * q));
            }
            pc = (unsigned)__popcll(m);
        } else {
            const int segs = (w + kSeg - 1) / kSeg;
            const int dy = k / segs, seg = k - dy * segs;
            const int tx = S.tx0[g] + seg * kSeg, ty = S.ty0[g] + dy, n = min(kSeg, w - seg * kSeg);
            // boxes three or more tiles wide: most tiles decided by the band interval
            const unsigned m = square ? (1u << n) - 1u
                               : w >= 3 ? run_hits_banded(cam.W, cam.H, S.u[g], S.v[g], S.a[g], S.b[g], S.c[g], S.t[g],
                                                          hxy.x, hxy.y, tx, n, ty)
                                        : run_hits(cam.W, cam.H, S.u[g], S.v[g], S.a[g], S.b[g], S.c[g], S.t[g], tx, n,
                                                   ty);
            if (keep) A.masks[S.mbase + (unsigned long long)(S.cstart[g] + k)] = (unsigned char)m;
            pc = (unsigned)__popc(m);
        }
        if (pc) atomicAdd(&S.cnt[g], pc);
    }
    __syncthreads();
    const unsigned mine = S.cnt[tid];                  // pairs of slot tid (0 beyond ns)
    const bool vis = mine != 0;
    unsigned hits = 0, nvis_block = 0;
    {
        unsigned v = mine;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const unsigned vb = __ballot_sync(0xffffffffu, vis);
        if (lane == 0) {
            S.wsum[warp] = v;
            S.wsum2[warp] = (unsigned)__popc(vb);
        }
        __syncthreads();
        unsigned vbefore = 0;
#pragma unroll
        for (int w2 = 0; w2 < kPreBlock / 32; ++w2) {
            const unsigned c = S.wsum2[w2];
            hits += S.wsum[w2];
            vbefore += w2 < warp ? c : 0u;
            nvis_block += c;
        }
        // the paired slots in slot (= id) order
        if (vis) S.vlist[vbefore + __popc(vb & ((1u << lane) - 1u))] = (short)tid;
    }
    if (tid == 0) {
        A.chunk_hits[chunk] = hits;
        A.chunk_vis[chunk] = nvis_block;
        if (nvis_block) atomicAdd(&A.ctr->n_visible, nvis_block);
        if (n_in_block) atomicAdd(&A.ctr->n_culled_in, n_in_block);
    }
    // pairs of every Gaussian of the chunk (id order, coalesced)
    if (g0 + tid < R.scene.P) {
        const int k = S.slot_of[tid];
        A.counts[R.rec0 + g0 + tid] = k >= 0 ? S.cnt[k] : 0u;
    }
    __syncthreads();
    // render record and emission geometry of every paired slot, four lanes a slot: the colour's SH
    // loads are spread over the lanes, then lane 0 writes the record and lanes 1-3 the geometry
    for (int q = tid; q < 4 * (int)nvis_block; q += kPreBlock) {
        const int slot = S.vlist[q >> 2], part = q & 3;
        const unsigned gmask = 0xfu << (lane & ~3);
        const long long gid = g0 + S.sl[slot];
        const long long rec = R.rec0 + gid;
        const float4 po = __ldg(R.scene.pos_opa + gid);
        float rgb[3];
        sh_colour4(R.scene, gid, cam, po.x, po.y, po.z, part, gmask, rgb);
        const float u = S.u[slot], v = S.v[slot], a = S.a[slot], b = S.b[slot], c = S.c[slot], t = S.t[slot];
        if (part == 0) {
            const float2 hxy = S.hxy[slot];
            Rec rc;
            rc.r0 = make_float4(u, v, a, b + b);
            rc.r1 = make_float4(c, t, S.gl[slot], rgb[0]);
            rc.r2 = make_float4(rgb[1], rgb[2], hxy.x + 1.0f, hxy.y + 1.0f);
            A.recs[rec] = rc;
        } else if (part == 1) {
            A.geo0[rec] = make_float4(u, v, a, b);
        } else if (part == 2) {
            const unsigned moff = keep ? (unsigned)(S.mbase + (unsigned long long)S.cstart[slot]) : kNoMasks;
            A.geo1[rec] = make_float4(c, t, S.z[slot], __uint_as_float(moff));
        } else {
            A.geo2[rec] = make_int4(S.tx0[slot], S.ty0[slot], S.w[slot], S.h[slot]);
        }
    }
}

// Exclusive scans of chunk counts over many CTAs in one launch, with no CTA waiting on another:
// CTA j scans counts [2048 j, 2048 j + 2048) (eight consecutive counts per thread, two 16-byte
// loads) and finds its base by summing every count before its span itself (16-byte loads, all
// CTAs in parallel; a city frame's 39k chunks take 20 CTAs, the last reading 39k counts from L2).
// The CTA holding the last count writes the total.  Counts arrays are 16-byte aligned.
constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr long long kScanSpan = (long long)kScanThreads * kScanPer;
__device__ unsigned long long block_sum64(unsigned long long x, unsigned long long *s_w) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_w[warp] = x;
    __syncthreads();
    unsigned long long t = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) t += s_w[w];
    __syncthreads();
    return t;
}
__device__ void chunk_scan(const unsigned *in, unsigned long long *out, long long n, unsigned long long *total) {
    __shared__ unsigned long long s_w[kScanThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long j = blockIdx.x, base = j * kScanSpan;
    const long long jlast = n > 0 ? (n - 1) / kScanSpan : 0;
    if (j > jlast || (!out && j != jlast)) return;      // uniform over the CTA
    // sum of the counts before the span (base is a multiple of 4)
    unsigned long long pre = 0;
    {
        const uint4 *in4 = reinterpret_cast<const uint4 *>(in);
        const long long nb4 = base / 4;
        long long i = tid;
        for (; i + 3 * kScanThreads < nb4; i += 4 * kScanThreads) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = __ldcg(in4 + i + u * kScanThreads);
#pragma unroll
            for (int u = 0; u < 4; ++u) pre += (unsigned long long)v[u].x + v[u].y + v[u].z + v[u].w;
        }
        for (; i < nb4; i += kScanThreads) {
            const uint4 v = __ldcg(in4 + i);
            pre += (unsigned long long)v.x + v.y + v.z + v.w;
        }
    }
    pre = block_sum64(pre, s_w);
    // this thread's eight counts
    const long long e0 = base + (long long)tid * kScanPer;
    unsigned c[kScanPer];
    if (e0 + kScanPer <= n) {
        const uint4 a = __ldcg(reinterpret_cast<const uint4 *>(in + e0));
        const uint4 b = __ldcg(reinterpret_cast<const uint4 *>(in + e0) + 1);
        c[0] = a.x; c[1] = a.y; c[2] = a.z; c[3] = a.w; c[4] = b.x; c[5] = b.y; c[6] = b.z; c[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) c[k] = e0 + k < n ? __ldcg(in + e0 + k) : 0u;
    }
    unsigned long long tsum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) tsum += c[k];
    // block exclusive scan of the thread sums
    unsigned long long incl = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    unsigned long long wex = 0, btot = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const unsigned long long y = s_w[w];
        wex += w < warp ? y : 0ull;
        btot += y;
    }
    if (out) {
        unsigned long long run = pre + wex + incl - tsum;
        if (e0 + kScanPer <= n) {
            ulonglong2 *o2 = reinterpret_cast<ulonglong2 *>(out + e0);
#pragma unroll
            for (int k = 0; k < kScanPer; k += 2) {
                const unsigned long long o0 = run, o1 = run + c[k];
                run = o1 + c[k + 1];
                o2[k / 2] = make_ulonglong2(o0, o1);
            }
        } else {
#pragma unroll
            for (int k = 0; k < kScanPer; ++k) {
                if (e0 + k < n) out[e0 + k] = run;
                run += c[k];
            }
        }
    }
    if (j == jlast && tid == 0) *total = pre + btot;
}

// n_items (nullable, device): when given, array a holds counts of ceil(*n_items / kPreBlock) chunks
// only (at most n), e.g. the rank chunks of the paired Gaussians.  Grid: ceil(n / kScanSpan) CTAs.
__global__ void __launch_bounds__(kScanThreads) k_chunk_scan(const unsigned *in_a, unsigned long long *out_a,
                                                             unsigned long long *tot_a, const unsigned *in_b,
                                                             unsigned long long *out_b, unsigned long long *tot_b,
                                                             long long n, long long pair_cap, unsigned *status,
                                                             const unsigned long long *n_items) {
    long long na = n;
    if (n_items) {
        const long long c = ((long long)*(const volatile unsigned long long *)n_items + kPreBlock - 1) / kPreBlock;
        na = c < n ? c : n;
    }
    chunk_scan(in_a, out_a, na, tot_a);
    if (in_b) {
        __syncthreads();
        chunk_scan(in_b, out_b, n, tot_b);
    }
    const long long jlast = na > 0 ? (na - 1) / kScanSpan : 0;
    if (status && blockIdx.x == jlast && threadIdx.x == 0) {
        __threadfence_block();
        if ((long long)*(volatile unsigned long long *)tot_a > pair_cap) atomicOr(status, kStPairOverflow);
    }
}
static unsigned scan_grid(long long n) { return (unsigned)(n > 0 ? (n + kScanSpan - 1) / kScanSpan : 1); }

// Two-level order, step 1: the paired Gaussians of each chunk, compacted in id order, as
// (depth bits, id) for the depth sort.  One warp a chunk (no block-wide step): its eight count
// loads go out together, then eight ballots place the paired ones after the chunk's base; a
// resident grid's warps walk the chunks, skipping those without paired Gaussians.
__global__ void __launch_bounds__(kPreBlock) k_vis_compact(const __grid_constant__ PreprocessArgs A) {
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long chunk = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; chunk < A.n_chunks;
         chunk += nwarps) {
        if (A.chunk_vis[chunk] == 0) continue;            // uniform over the warp
        const ReqDesc &R = A.B.r[req_of_chunk(A.B, chunk)];
        const long long g0 = (chunk - R.chunk0) * kPreBlock;
        constexpr int K = kPreBlock / 32;
        unsigned c[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const long long gid = g0 + 32 * k + lane;
            c[k] = gid < R.scene.P ? A.counts[R.rec0 + gid] : 0u;
        }
        unsigned long long base = A.vis_base[chunk];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool vis = c[k] != 0u;
            const unsigned bal = __ballot_sync(FULL, vis);
            if (vis) {
                const long long rec = R.rec0 + g0 + 32 * k + lane;
                const unsigned long long pos = base + __popc(bal & ((1u << lane) - 1u));
                A.dkey[pos] = __float_as_uint(A.geo1[rec].z);
                A.dval[pos] = (unsigned)rec;
            }
            base += __popc(bal);
        }
    }
}

// Two-level order, step 2: pairs per chunk of 256 depth-sorted Gaussians.
__global__ void __launch_bounds__(kPreBlock) k_emit_sum(const __grid_constant__ PreprocessArgs A) {
    if (upstream_timed_out(A.ctr)) return;   // the depth sort gave up: its ids may be garbage
    __shared__ unsigned s_w[kPreBlock / 32];
    const long long V = (long long)A.ctr->n_vis64;
    const long long nch = (V + kPreBlock - 1) / kPreBlock;
    for (long long c = blockIdx.x; c < nch; c += gridDim.x) {
        const long long r = c * kPreBlock + threadIdx.x;
        unsigned v = r < V ? A.counts[A.dsorted[r]] : 0u;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned t = 0;
            for (int w2 = 0; w2 < kPreBlock / 32; ++w2) t += s_w[w2];
            A.chunk_hits2[c] = t;
        }
        __syncthreads();
    }
}

// Emission: the same load-balanced units, their decisions read from the count pass's masks; every
// hit is written at the chunk's base + its rank in slot order.  DEPTH = false: chunk c holds
// Gaussians 256c .. 256c+255 and the pairs land in (Gaussian id, tile row-major) order with
// 64-bit (tile, depth) keys.  DEPTH = true: chunk c holds
// the depth-sorted Gaussians of ranks 256c .. 256c+255 and the pairs land in (depth, id, tile)
// order with the tile id alone as a 32-bit key -- a stable sort by tile then yields exactly the
// (tile, depth, id) order of the 64-bit keys.
template <bool DEPTH>
__device__ __forceinline__ void emit_chunk(const PreprocessArgs &A, EmitSmem &E, const long long chunk) {
    PreSmem &S = E.P;
    const int tid = threadIdx.x;
    long long gid;                    // here: the record index (request rec0 + Gaussian id)
    bool in_range;
    int ri;
    if (DEPTH) {
        const long long rank = chunk * kPreBlock + tid;
        in_range = rank < (long long)A.ctr->n_vis64;
        gid = in_range ? (long long)A.dsorted[rank] : 0;
        ri = req_of_rec(A.B, gid);
    } else {
        ri = req_of_chunk(A.B, chunk);
        const ReqDesc &R = A.B.r[ri];
        const long long lg = (chunk - R.chunk0) * kPreBlock + tid;
        in_range = lg < R.scene.P;
        gid = R.rec0 + lg;
    }
    S.req[tid] = (unsigned char)ri;
    int ncand = 0;
    S.cnt[tid] = (unsigned)gid;
    // geometry exists only for paired Gaussians (count > 0; every depth-ordered one is)
    if (in_range && (DEPTH || A.counts[gid] != 0u)) {
        const int4 g2 = A.geo2[gid];
        ncand = g2.z * g2.w;
        if (ncand > 0) {
            const float4 g0 = A.geo0[gid], g1 = A.geo1[gid];
            S.u[tid] = g0.x;
            S.v[tid] = g0.y;
            S.a[tid] = g0.z;
            S.b[tid] = g0.w;
            S.c[tid] = g1.x;
            S.t[tid] = g1.y;
            S.zb[tid] = __float_as_uint(g1.z);
            S.moff[tid] = __float_as_uint(g1.w);
            S.tx0[tid] = g2.x;
            S.ty0[tid] = g2.y;
        }
        S.w[tid] = g2.z > 0 ? g2.z : 1;
    } else {
        S.w[tid] = 1;
    }
    const long long cap = A.pair_cap;
    const int nunits = ncand > 0 ? units_of(S.w[tid], ncand / S.w[tid]) : 0;
    if (DEPTH) {
        // Each Gaussian's pairs start at the chunk base + the pairs of the Gaussians before it in
        // depth order.  Large Gaussians go to k_emit_big (one CTA each) so that a chunk of
        // consecutive depth ranks -- where large footprints cluster -- does not serialise them.
        const unsigned c = in_range ? A.counts[gid] : 0u;
        unsigned tot;
        const unsigned pre = block_excl(S, c, &tot);
        const unsigned long long pb = A.chunk_base2[chunk] + pre;
        S.pbase[tid] = pb;
        S.run[tid] = 0;
        const bool big = ncand > kBigCand, mid = !big && ncand > kMidCand;
        // this CTA's large and medium Gaussians take consecutive slots of their lists: one atomic
        // per CTA and list
        unsigned nbig_blk, nmid_blk;
        const unsigned bslot = block_excl(S, (big && c > 0) ? 1u : 0u, &nbig_blk);
        const unsigned mslot = block_excl(S, (mid && c > 0) ? 1u : 0u, &nmid_blk);
        if (tid == 0 && nbig_blk) S.xr[0] = atomicAdd(&A.ctr->n_big, nbig_blk);
        if (tid == 32 && nmid_blk) S.xr[1] = atomicAdd(&A.ctr->n_mid, nmid_blk);
        __syncthreads();
        const uint4 item = make_uint4((unsigned)gid, (unsigned)ri, (unsigned)(pb & 0xffffffffu), (unsigned)(pb >> 32));
        if (big && c > 0) A.big[S.xr[0] + bslot] = item;
        if (mid && c > 0) A.mid[S.xr[1] + mslot] = item;
        __syncthreads();
        const int ctotal = block_scan_cand(S, (big || mid) ? 0 : nunits);
        for (int base = 0; base < ctotal; base += kPreBlock) {
            const int slot = base + tid;
            unsigned m = 0;
            Unit U{-1, 0, 0, 0};
            if (slot < ctotal) {
                U = unit_of(S, slot);
                m = kept_hits(S, A, U, slot);
            }
            unsigned step_tot;
            const unsigned xr = block_excl(S, (unsigned)__popc(m), &step_tot);   // exclusive hit rank in the step
            S.xr[tid] = xr;
            if (m) {
                const ReqDesc &R = A.B.r[S.req[U.g]];
                const unsigned trow = (unsigned)(R.tile0 + U.ty * R.cam.tiles_x);
                unsigned i = xr;
                for (unsigned mm = m; mm; mm &= mm - 1, ++i) {
                    E.stile[i] = trow + (unsigned)(U.tx + __ffs(mm) - 1);
                    E.sg[i] = (unsigned char)U.g;
                }
            }
            __syncthreads();
            // hit i of Gaussian g lands at g's base + g's hits in earlier steps + its rank among
            // g's hits of this step (g's first unit of the step starts at staged index xr[first])
            for (unsigned i = tid; i < step_tot; i += kPreBlock) {
                const int g = E.sg[i];
                const int first = max(S.cstart[g], base) - base;
                const unsigned long long pos = S.pbase[g] + S.run[g] + (i - S.xr[first]);
                if ((long long)pos < cap) {
                    A.tkeys[pos] = E.stile[i];
                    A.vals[pos] = S.cnt[g];
                }
            }
            __syncthreads();
            // advance each Gaussian's running count by its hits in this step
            if (m) atomicAdd(&S.run[U.g], (unsigned)__popc(m));
            __syncthreads();
        }
        return;
    }
    const int ctotal = block_scan_cand(S, nunits);
    unsigned long long run = A.chunk_base[chunk];
    for (int base = 0; base < ctotal; base += kPreBlock) {
        const int slot = base + tid;
        unsigned m = 0;
        Unit U{0, 0, 0, 0};
        if (slot < ctotal) {
            U = unit_of(S, slot);
            m = kept_hits(S, A, U, slot);
        }
        unsigned step_tot;
        const unsigned xr = block_excl(S, (unsigned)__popc(m), &step_tot);
        if (m) {
            const ReqDesc &R = A.B.r[S.req[U.g]];
            const unsigned trow = (unsigned)(R.tile0 + U.ty * R.cam.tiles_x);
            unsigned i = xr;
            for (unsigned mm = m; mm; mm &= mm - 1, ++i) {
                E.stile[i] = trow + (unsigned)(U.tx + __ffs(mm) - 1);
                E.sg[i] = (unsigned char)U.g;
            }
        }
        __syncthreads();
        for (unsigned i = tid; i < step_tot; i += kPreBlock) {
            const unsigned long long pos = run + i;
            if ((long long)pos < cap) {
                const int g = E.sg[i];
                A.keys[pos] = ((unsigned long long)E.stile[i] << 32) | S.zb[g];
                A.vals[pos] = S.cnt[g];        // record index of Gaussian g
            }
        }
        run += step_tot;
        __syncthreads();
    }
}

// DEPTH = false: one CTA per chunk of 256 Gaussians.  DEPTH = true: a resident grid walks the rank
// chunks that hold paired Gaussians (ceil(V / 256) of them, V known only on the device).
template <bool DEPTH>
__global__ void __launch_bounds__(kPreBlock, DEPTH ? 4 : 8) k_pre_emit(const __grid_constant__ PreprocessArgs A) {
    __shared__ EmitSmem E;
    if (!DEPTH) {
        emit_chunk<false>(A, E, blockIdx.x);
        return;
    }
    if (upstream_timed_out(A.ctr)) return;   // the depth sort gave up: its ids may be garbage
    const long long V = (long long)A.ctr->n_vis64;
    for (long long chunk = blockIdx.x; chunk * kPreBlock < V; chunk += gridDim.x) {
        emit_chunk<true>(A, E, chunk);
        __syncthreads();
    }
}

// Depth order, medium Gaussians: one warp per Gaussian (warps take items in ticket order), its
// units tested 32 at a time, hits staged per warp and written as coalesced runs from the
// Gaussian's base.
__global__ void __launch_bounds__(kPreBlock) k_emit_mid(const __grid_constant__ PreprocessArgs A) {
    // four consecutive units a lane and step (128 units): a 4096-tile Gaussian takes four steps
    constexpr int U = 4;
    constexpr int kWarps = kPreBlock / 32;
    __shared__ unsigned s_tile[kWarps][32 * kSeg * U];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    const unsigned nmid = *(volatile unsigned *)&A.ctr->n_mid;
    const long long cap = A.pair_cap;
    while (true) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(&A.ctr->mid_ticket, 1u);
        item = __shfl_sync(FULL, item, 0);
        if (item >= nmid) break;
        const uint4 it = A.mid[item];
        const long long rec = it.x;
        const ReqDesc &R = A.B.r[it.y];
        unsigned long long run = ((unsigned long long)it.w << 32) | it.z;
        const float4 g0 = A.geo0[rec], g1 = A.geo1[rec];
        const int4 g2 = A.geo2[rec];
        const unsigned mo = __float_as_uint(g1.w);
        const int segs = (g2.z + kSeg - 1) / kSeg;
        const int nunits = segs * g2.w;
        for (int base = 0; base < nunits; base += 32 * U) {
            unsigned m[U];
            int tx[U], ty[U];
            unsigned c = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = base + lane * U + u;
                m[u] = 0;
                tx[u] = ty[u] = 0;
                if (k < nunits) {
                    const int dy = k / segs, seg = k - dy * segs;
                    tx[u] = g2.x + seg * kSeg;
                    ty[u] = g2.y + dy;
                    const int nrun = min(kSeg, g2.z - seg * kSeg);
                    m[u] = mo != kNoMasks       ? (unsigned)A.masks[(unsigned long long)mo + (unsigned)k]
                           : R.opt.intersect == 1 ? (1u << nrun) - 1u
                                                  : run_hits(R.cam.W, R.cam.H, g0.x, g0.y, g0.z, g0.w, g1.x, g1.y,
                                                             tx[u], nrun, ty[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) c += (unsigned)__popc(m[u]);
            unsigned incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            const unsigned tot = __shfl_sync(FULL, incl, 31);
            unsigned i = incl - c;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const unsigned trow = (unsigned)(R.tile0 + ty[u] * R.cam.tiles_x);
                for (unsigned mm = m[u]; mm; mm &= mm - 1, ++i) s_tile[warp][i] = trow + (unsigned)(tx[u] + __ffs(mm) - 1);
            }
            __syncwarp();
            for (unsigned j = lane; j < tot; j += 32) {
                const unsigned long long pos = run + j;
                if ((long long)pos < cap) {
                    A.tkeys[pos] = s_tile[warp][j];
                    A.vals[pos] = (unsigned)rec;
                }
            }
            run += tot;
            __syncwarp();
        }
    }
}

// Depth order, large Gaussians: one CTA per Gaussian (persistent grid, ticketed), its candidate
// tiles tested 256 at a time, hits written in row-major order from the Gaussian's base.
__global__ void __launch_bounds__(kPreBlock) k_emit_big(const __grid_constant__ PreprocessArgs A) {
    // four consecutive units a thread and step (1024 units, 8192 candidate tiles): a Gaussian
    // that covers the whole image takes four steps, each with its loads in flight together
    constexpr int U = 4;
    __shared__ unsigned s_item, s_w[kPreBlock / 32];
    __shared__ unsigned s_tile[kPreBlock * kSeg * U];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned FULL = 0xffffffffu;
    const unsigned nbig = *(volatile unsigned *)&A.ctr->n_big;
    const long long cap = A.pair_cap;
    // items in ticket order, so that CTAs that drew small Gaussians take more of them
    while (true) {
        if (tid == 0) s_item = atomicAdd(&A.ctr->big_ticket, 1u);
        __syncthreads();
        const unsigned item = s_item;
        __syncthreads();
        if (item >= nbig) break;
        const uint4 it = A.big[item];
        const long long rec = it.x;
        const ReqDesc &R = A.B.r[it.y];
        unsigned long long run = ((unsigned long long)it.w << 32) | it.z;
        const float4 g0 = A.geo0[rec], g1 = A.geo1[rec];
        const int4 g2 = A.geo2[rec];
        const unsigned mo = __float_as_uint(g1.w);
        const int segs = (g2.z + kSeg - 1) / kSeg;
        const int nunits = segs * g2.w;
        for (int base = 0; base < nunits; base += kPreBlock * U) {
            unsigned m[U];
            int tx[U], ty[U];
            unsigned c = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = base + tid * U + u;
                m[u] = 0;
                tx[u] = ty[u] = 0;
                if (k < nunits) {
                    const int dy = k / segs, seg = k - dy * segs;
                    tx[u] = g2.x + seg * kSeg;
                    ty[u] = g2.y + dy;
                    const int nrun = min(kSeg, g2.z - seg * kSeg);
                    m[u] = mo != kNoMasks       ? (unsigned)A.masks[(unsigned long long)mo + (unsigned)k]
                           : R.opt.intersect == 1 ? (1u << nrun) - 1u
                                                  : run_hits(R.cam.W, R.cam.H, g0.x, g0.y, g0.z, g0.w, g1.x, g1.y,
                                                             tx[u], nrun, ty[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) c += (unsigned)__popc(m[u]);
            // block exclusive scan of the hit counts (thread order = unit order)
            unsigned incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(FULL, incl, o);
                if (lane >= o) incl += y;
            }
            if (lane == 31) s_w[warp] = incl;
            __syncthreads();
            unsigned wpre = 0, tot = 0;
#pragma unroll
            for (int w2 = 0; w2 < kPreBlock / 32; ++w2) {
                const unsigned x = s_w[w2];
                wpre += w2 < warp ? x : 0u;
                tot += x;
            }
            unsigned i = wpre + incl - c;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const unsigned trow = (unsigned)(R.tile0 + ty[u] * R.cam.tiles_x);
                for (unsigned mm = m[u]; mm; mm &= mm - 1, ++i) s_tile[i] = trow + (unsigned)(tx[u] + __ffs(mm) - 1);
            }
            __syncthreads();
            for (unsigned j = tid; j < tot; j += kPreBlock) {
                const unsigned long long pos = run + j;
                if ((long long)pos < cap) {
                    A.tkeys[pos] = s_tile[j];
                    A.vals[pos] = (unsigned)rec;
                }
            }
            run += tot;
            __syncthreads();
        }
    }
}

// k CTAs per SM of the current device.
static int resident_grid(int k) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return k * sms;
}

void launch_pre_count(const PreprocessArgs &a, cudaStream_t s) {
    if (a.n_chunks <= 0) return;
    k_pre_count<<<(unsigned)a.n_chunks, kPreBlock, 0, s>>>(a);
}

void launch_preprocess(const PreprocessArgs &a, cudaStream_t s, bool counted) {
    if (a.n_chunks <= 0) return;
    if (!counted) k_pre_count<<<(unsigned)a.n_chunks, kPreBlock, 0, s>>>(a);
    k_chunk_scan<<<scan_grid(a.n_chunks), kScanThreads, 0, s>>>(a.chunk_hits, a.chunk_base, &a.ctr->n_pairs, nullptr, nullptr, nullptr,
                                            a.n_chunks, a.pair_cap, &a.ctr->status, nullptr);
    k_pre_emit<false><<<(unsigned)a.n_chunks, kPreBlock, 0, s>>>(a);
}

int launch_preprocess_depth(const PreprocessArgs &a, const SortScratch &scr, cudaStream_t s, bool counted) {
    if (a.n_chunks <= 0) return 0;
    if (!counted) k_pre_count<<<(unsigned)a.n_chunks, kPreBlock, 0, s>>>(a);
    k_chunk_scan<<<scan_grid(a.n_chunks), kScanThreads, 0, s>>>(a.chunk_hits, nullptr, &a.ctr->n_pairs, a.chunk_vis, a.vis_base,
                                            &a.ctr->n_vis64, a.n_chunks, a.pair_cap, &a.ctr->status, nullptr);
    k_vis_compact<<<(unsigned)min(a.n_chunks, (long long)resident_grid(8)), kPreBlock, 0, s>>>(a);
    // depth sort of the paired Gaussians: 32-bit float bits of z (positive, so bit order = value order)
    // (always the fused onesweep: a few hundred thousand to a few million keys, where its single
    // launch beats the per-pass forms; the frame's sort_algo applies to the pair sort)
    SortScratch dscr = scr;
    dscr.algo = 2;
    const int dp = launch_sort32(a.dkey, a.dval, a.dkey_tmp, a.dval_tmp, &a.ctr->n_vis64, a.B.total_recs, 32, dscr,
                                 a.ctr, s);
    (void)dp;   // four passes: the result is back in dkey / dval
    // depth ranks run over all records of the batch: size the rank chunks by total_recs
    const long long rank_chunks = (a.B.total_recs + kPreBlock - 1) / kPreBlock;
    k_emit_sum<<<(unsigned)min(rank_chunks, (long long)resident_grid(8)), kPreBlock, 0, s>>>(a);
    unsigned long long *unused_total = &a.ctr->scratch64;
    // only the rank chunks that hold paired Gaussians: ceil(V / 256) of them
    k_chunk_scan<<<scan_grid(rank_chunks), kScanThreads, 0, s>>>(a.chunk_hits2, a.chunk_base2, unused_total, nullptr, nullptr, nullptr,
                                            rank_chunks, 1ll << 62, nullptr, &a.ctr->n_vis64);
    k_pre_emit<true><<<(unsigned)min(rank_chunks, (long long)resident_grid(4)), kPreBlock, 0, s>>>(a);
    k_emit_mid<<<resident_grid(8), kPreBlock, 0, s>>>(a);
    k_emit_big<<<resident_grid(8), kPreBlock, 0, s>>>(a);
    return 4;
}

// Pairs of each request of the batch (sums of its chunks' counts), for admission decisions.
__global__ void __launch_bounds__(256) k_req_pairs(const __grid_constant__ PreprocessArgs A, unsigned long long *out) {
    const int r = blockIdx.x;
    const long long c0 = A.B.r[r].chunk0;
    const long long c1 = r + 1 < A.B.n ? A.B.r[r + 1].chunk0 : A.B.total_chunks;
    unsigned long long sum = 0;
    for (long long c = c0 + threadIdx.x; c < c1; c += blockDim.x) sum += A.chunk_hits[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    __shared__ unsigned long long s_w[8];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < 8; ++w) t += s_w[w];
        out[r] = t;
    }
}

void launch_req_pairs(const PreprocessArgs &a, unsigned long long *out, cudaStream_t s) {
    if (a.B.n > 0) k_req_pairs<<<a.B.n, 256, 0, s>>>(a, out);
}

__global__ void k_make_keys(const unsigned *tkeys, const unsigned *vals, const float4 *geo1, long long n,
                            unsigned long long *out, const FrameCounters *ctr) {
    if (upstream_timed_out(ctr)) return;     // the sort gave up: its ids may be garbage
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = ((unsigned long long)tkeys[i] << 32) | __float_as_uint(geo1[vals[i]].z);
}

void launch_make_keys(const unsigned *tkeys, const unsigned *vals, const float4 *geo1, long long n,
                      unsigned long long *out, const FrameCounters *ctr, cudaStream_t s) {
    if (n <= 0) return;
    k_make_keys<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tkeys, vals, geo1, n, out, ctr);
}

}  // namespace gs
