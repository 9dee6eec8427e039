/*
 * gs_oracle.c -- CPU oracle for the FlashGS forward rasterizer (arXiv 2408.07967).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of what the rasterizer computes.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant with the CUDA library and neither side
 * includes the other.
 *
 * Structure (one function per step, each citing the passage it follows):
 *   or_preprocess      cull, projection, EWA covariance, conic, opacity-aware
 *                      threshold, SH colour          (Alg. 1; Alg. 4; Eq. 2-3)
 *   or_tile_hit        exact ellipse / tile test      (Alg. 3; Eq. 6-9)
 *   or_emit_pairs      (tile, depth) keys of every intersecting tile (Alg. 4)
 *   or_sort_pairs      order by (key, Gaussian id)    (Section 2.2, sort)
 *   or_tile_ranges     [start, end) of each tile in the sorted list
 *   or_blend_tiled     front-to-back alpha blending with early stop
 *                      (Section 2.2 render; Section 5.2)
 *   or_blend_brute     the same blend over *every* Gaussian per pixel, the
 *                      plain definition the tiled result must equal.
 *
 * Precision.  Every step that decides an integer outcome -- whether a
 * Gaussian is culled, whether a tile is paired, the key bits, whether a pixel
 * skips a Gaussian (alpha < tau) -- is taken in IEEE binary32 with the
 * evaluation order written out below (compile with -ffp-contract=off; the one
 * fused multiply-add, in the per-pixel quadratic form, is an explicit fmaf).
 * The blended values are computed either in binary32 ("mode 32") or in
 * binary64 from binary64 geometry ("mode 64", the image reference).  The
 * early-stop test (T < T_min) uses the mode's own transmittance.
 *
 * Readings of the paper (where it is silent or garbled) are listed in the
 * design notes of the repository; the ones that matter here:
 *   - 3D covariance, EWA 2D covariance, SH basis: the 3DGS formulation the
 *     paper builds on (Section 2.2), with 0.3 px dilation and the 1.3 x tan
 *     frustum clamp of the Jacobian.
 *   - Effective ellipse (Eq. 2-3) generalised to 2D: alpha0*exp(-q/2) >= tau
 *     <=> q <= t = 2 ln(alpha0/tau), q the conic quadratic form.  Uncapped by
 *     default; cap_3sigma applies the paper's min(3 sigma, Eq. 3) rule (t<=9).
 *   - Eq. 6 is read max(a_i, a_j), Eq. 7 a_j <= b_i (typeset garbles).
 *   - Ties in depth are broken by Gaussian id.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    float R[9];             /* world -> camera rotation, row-major */
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_z;           /* 0.2 in the paper (Alg. 4) */
} OrCamera;

typedef struct {
    float bg[3];
    float tau;              /* 1/255 (Section 4.1) */
    float alpha_max;        /* 0.99 */
    float T_min;            /* 1e-4 */
    float dilation;         /* 0.3 px^2 low-pass */
    int32_t cap_3sigma;     /* 1: t = min(9, 2 ln(alpha0/tau)) */
    int32_t clamp_fov;      /* 1: clamp x/z, y/z to 1.3 tan(half fov) in the Jacobian */
    int32_t intersect;      /* 0: exact tiles (Alg. 3); 1: every tile of the 3DGS square (Eq. 1, Alg. 2) */
} OrOpts;

/* FP32 per-Gaussian record (floats). */
/* F_ALL = 1: every tile of the rectangle is paired (3DGS square); 0: the exact test decides. */
enum { F_U, F_V, F_A, F_B, F_C, F_T, F_Z, F_S00, F_S01, F_S11, F_ALPHA, F_R, F_G, F_BL, F_TFULL, F_ALL, REC32 };
/* FP64 per-Gaussian record (doubles). */
enum { D_U, D_V, D_A, D_B, D_C, D_ALPHA, D_R, D_G, D_BL, D_S00, D_S01, D_S11, D_Z, D_PAD0, D_PAD1, D_PAD2, REC64 };

#define TILE 16

int or_version(void) { return 3; }

void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int or_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static uint32_t f2u(float x) { uint32_t u; memcpy(&u, &x, 4); return u; }
static float u2f(uint32_t u) { float x; memcpy(&x, &u, 4); return x; }

/* ------------------------------------------------------------------------------------------
 * Natural logarithm in binary32 (own routine; the per-Gaussian threshold t feeds pair
 * decisions, so it must not depend on a platform libm).  Method: x = m * 2^e with
 * m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s), s = (m-1)/(m+1), by the odd series
 * 2 (s + s^3/3 + s^5/5 + ... + s^11/11) (|s| <= 0.1716, truncation < 2^-30 relative);
 * e*ln2 is added with a split constant (ln2_hi has 16 significant bits so e*ln2_hi is
 * exact).  Domain: positive normal finite x.
 * ---------------------------------------------------------------------------------------- */
float or_logf(float x)
{
    uint32_t bits = f2u(x);
    int e = (int)((bits >> 23) & 0xffu) - 127;
    float m = u2f((bits & 0x007fffffu) | 0x3f800000u);       /* [1, 2) */
    const float sqrt2 = 1.41421353816986083984375f;
    if (m > sqrt2) { m = m * 0.5f; e = e + 1; }
    const float ln2_hi = 0.693145751953125f;                 /* 0x3f317200 */
    const float ln2_lo = 1.42860676533018704503775e-06f;     /* ln 2 - ln2_hi */
    const float c3 = (float)(1.0 / 3.0), c5 = (float)(1.0 / 5.0), c7 = (float)(1.0 / 7.0);
    const float c9 = (float)(1.0 / 9.0), c11 = (float)(1.0 / 11.0);
    float num = m - 1.0f;
    float den = m + 1.0f;
    float s = num / den;
    float s2 = s * s;
    float p = c11 * s2;
    p = p + c9;  p = p * s2;
    p = p + c7;  p = p * s2;
    p = p + c5;  p = p * s2;
    p = p + c3;  p = p * s2;
    float two_s = s + s;
    float lnm = two_s + two_s * p;
    float ef = (float)e;
    float lo = ef * ln2_lo;
    lo = lo + lnm;
    return ef * ln2_hi + lo;
}

/* ------------------------------------------------------------------------------------------
 * exp in binary32 (own routine, used for log-scale and logit activation).  Cody-Waite
 * reduction x = k ln2 + r, k = floor(x log2(e) + 1/2), r = (x - k ln2_hi) - k ln2_lo,
 * |r| <= 0.35; e^r by its Taylor series to r^8/8! (truncation < 3e-10 relative) in
 * Horner form; result r * 2^k.  Returns 0 for x < -87, +inf for x > 88.
 * ---------------------------------------------------------------------------------------- */
float or_expf(float x)
{
    if (!(x == x)) return x;
    if (x < -87.0f) return 0.0f;
    if (x > 88.0f) return u2f(0x7f800000u);
    const float log2e = 1.44269502162933349609375f;
    const float ln2_hi = 0.693145751953125f;
    const float ln2_lo = 1.42860676533018704503775e-06f;
    float kf = floorf(x * log2e + 0.5f);
    float r = x - kf * ln2_hi;
    r = r - kf * ln2_lo;
    const float i2 = (float)(1.0 / 2.0), i3 = (float)(1.0 / 6.0), i4 = (float)(1.0 / 24.0);
    const float i5 = (float)(1.0 / 120.0), i6 = (float)(1.0 / 720.0), i7 = (float)(1.0 / 5040.0);
    const float i8 = (float)(1.0 / 40320.0);
    float p = i8 * r;
    p = p + i7;  p = p * r;
    p = p + i6;  p = p * r;
    p = p + i5;  p = p * r;
    p = p + i4;  p = p * r;
    p = p + i3;  p = p * r;
    p = p + i2;  p = p * r;
    p = p + 1.0f; p = p * r;
    p = p + 1.0f;
    int k = (int)kf;
    /* 2^k as two factors so that k = -127 .. 127 stays exact */
    int k1 = k / 2, k2 = k - k1;
    float s1 = u2f((uint32_t)(k1 + 127) << 23);
    float s2 = u2f((uint32_t)(k2 + 127) << 23);
    return (p * s1) * s2;
}

/* Opacity-aware threshold of Eq. 3 in binary32: alpha0 exp(-q/2) >= tau <=> q <= 2 ln(alpha0/tau). */
float or_threshold(float alpha0, float tau)
{
    float ratio = alpha0 / tau;
    return 2.0f * or_logf(ratio);
}

/* Opacity from its logit in binary32: 1 / (1 + e^-x) with or_expf. */
float or_sigmoidf(float x)
{
    float e = or_expf(-x);
    return 1.0f / (1.0f + e);
}

/* The three functions above over an array (fn 0: or_threshold(x[i], param); 1: or_expf(x[i]);
 * 2: or_sigmoidf(x[i])), for exhaustive comparisons over whole input domains. */
void or_eval_decision_math(int32_t fn, int64_t n, const float *x, float param, float *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        y[i] = fn == 0 ? or_threshold(x[i], param) : fn == 1 ? or_expf(x[i]) : or_sigmoidf(x[i]);
}

/* Max ulp error of or_logf against binary64 log over every float in [lo, hi]. */
double or_logf_max_ulp(float lo, float hi, float *worst_x)
{
    double worst = 0.0;
    float wx = lo;
    for (uint32_t b = f2u(lo); b <= f2u(hi); ++b) {
        float x = u2f(b);
        float y = or_logf(x);
        double ref = log((double)x);
        float rf = (float)ref;
        double ulp = fabs((double)nextafterf(rf, INFINITY) - (double)rf);
        if (ulp == 0.0) ulp = 1e-45;
        double err = fabs((double)y - ref) / ulp;
        if (err > worst) { worst = err; wx = x; }
    }
    if (worst_x) *worst_x = wx;
    return worst;
}

double or_expf_max_ulp(float lo, float hi, int32_t stride, float *worst_x)
{
    double worst = 0.0;
    float wx = lo;
    if (stride < 1) stride = 1;
    /* walk the float line in order (both signs) */
    float x = lo;
    while (x <= hi) {
        float y = or_expf(x);
        double ref = exp((double)x);
        float rf = (float)ref;
        double ulp = fabs((double)nextafterf(rf, INFINITY) - (double)rf);
        double err = fabs((double)y - ref) / ulp;
        if (err > worst) { worst = err; wx = x; }
        for (int s = 0; s < stride; ++s) x = nextafterf(x, INFINITY);
    }
    if (worst_x) *worst_x = wx;
    return worst;
}

/* ------------------------------------------------------------------------------------------
 * Real SH basis of degree <= 3 in the 3DGS sign/order convention, constants from their
 * closed forms: l=0 1/(2 sqrt(pi)); l=1 sqrt(3/(4pi)) (-y, z, -x); l=2 and l=3 as below.
 * ---------------------------------------------------------------------------------------- */
static void sh_consts(double k[16])
{
    const double pi = 3.14159265358979323846;
    k[0] = 0.5 / sqrt(pi);
    double c1 = sqrt(3.0 / (4.0 * pi));
    k[1] = -c1; k[2] = c1; k[3] = -c1;
    k[4] = 0.5 * sqrt(15.0 / pi);
    k[5] = -0.5 * sqrt(15.0 / pi);
    k[6] = 0.25 * sqrt(5.0 / pi);
    k[7] = -0.5 * sqrt(15.0 / pi);
    k[8] = 0.25 * sqrt(15.0 / pi);
    k[9] = -0.25 * sqrt(35.0 / (2.0 * pi));
    k[10] = 0.5 * sqrt(105.0 / pi);
    k[11] = -0.25 * sqrt(21.0 / (2.0 * pi));
    k[12] = 0.25 * sqrt(7.0 / pi);
    k[13] = -0.25 * sqrt(21.0 / (2.0 * pi));
    k[14] = 0.25 * sqrt(105.0 / pi);
    k[15] = -0.25 * sqrt(35.0 / (2.0 * pi));
}

/* basis values Y_i(d) (i = l^2 + l + m) for a unit direction d, FP64 */
void or_sh_basis(const double d[3], double Y[16])
{
    double k[16];
    sh_consts(k);
    double x = d[0], y = d[1], z = d[2];
    double xx = x * x, yy = y * y, zz = z * z;
    Y[0] = k[0];
    Y[1] = k[1] * y; Y[2] = k[2] * z; Y[3] = k[3] * x;
    Y[4] = k[4] * x * y;
    Y[5] = k[5] * y * z;
    Y[6] = k[6] * (2.0 * zz - xx - yy);
    Y[7] = k[7] * x * z;
    Y[8] = k[8] * (xx - yy);
    Y[9] = k[9] * y * (3.0 * xx - yy);
    Y[10] = k[10] * x * y * z;
    Y[11] = k[11] * y * (4.0 * zz - xx - yy);
    Y[12] = k[12] * z * (2.0 * zz - 3.0 * xx - 3.0 * yy);
    Y[13] = k[13] * x * (4.0 * zz - xx - yy);
    Y[14] = k[14] * z * (xx - yy);
    Y[15] = k[15] * x * (xx - 3.0 * yy);
}

static void sh_basis_f(const float d[3], float Y[16])
{
    double k[16];
    sh_consts(k);
    float kf[16];
    for (int i = 0; i < 16; ++i) kf[i] = (float)k[i];
    float x = d[0], y = d[1], z = d[2];
    float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = kf[0];
    Y[1] = kf[1] * y; Y[2] = kf[2] * z; Y[3] = kf[3] * x;
    Y[4] = kf[4] * x * y;
    Y[5] = kf[5] * y * z;
    Y[6] = kf[6] * (2.0f * zz - xx - yy);
    Y[7] = kf[7] * x * z;
    Y[8] = kf[8] * (xx - yy);
    Y[9] = kf[9] * y * (3.0f * xx - yy);
    Y[10] = kf[10] * x * y * z;
    Y[11] = kf[11] * y * (4.0f * zz - xx - yy);
    Y[12] = kf[12] * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = kf[13] * x * (4.0f * zz - xx - yy);
    Y[14] = kf[14] * z * (xx - yy);
    Y[15] = kf[15] * x * (xx - 3.0f * yy);
}

static int sh_count(int degree)
{
    if (degree < 0) degree = 0;
    if (degree > 3) degree = 3;
    return (degree + 1) * (degree + 1);
}

/* ------------------------------------------------------------------------------------------
 * Exact ellipse / tile test (Alg. 3 with the division- and root-free form of Eq. 9).
 * Ellipse {d : a dx^2 + 2 b dx dy + c dy^2 <= t} about (u, v); rectangle [x0,x1] x [y0,y1].
 * Hit if the centre is in the rectangle, or, for some edge, the chord the ellipse cuts
 * from the edge's line overlaps the edge.  On the line y = y_e the chord solves
 * A X^2 + 2 B X + C <= 0 with A = a, B = b dy, C = c dy^2 - t (X = x - u); with D =
 * B^2 - A C >= 0 its roots are (-B -+ sqrt D)/A, and overlap with [lo, hi] is
 * (e1 <= 0 or e1^2 <= D) and (e2 >= 0 or e2^2 <= D), e1 = A lo + B, e2 = A hi + B
 * (Eq. 8-9 with B halved and DELTA quartered; A > 0).  Binary32, evaluated as written.
 * ---------------------------------------------------------------------------------------- */
static int chord_overlaps(float A, float B, float C, float lo, float hi)
{
    float BB = B * B;
    float AC = A * C;
    float D = BB - AC;
    if (!(D >= 0.0f)) return 0;
    float e1 = A * lo;
    e1 = e1 + B;
    float e2 = A * hi;
    e2 = e2 + B;
    int left = (e1 <= 0.0f) || (e1 * e1 <= D);
    int right = (e2 >= 0.0f) || (e2 * e2 <= D);
    return left && right;
}

int or_tile_hit(float u, float v, float a, float b, float c, float t,
                float x0, float x1, float y0, float y1)
{
    if (x0 <= u && u <= x1 && y0 <= v && v <= y1) return 1;
    float lo = x0 - u, hi = x1 - u;
    for (int k = 0; k < 2; ++k) {                 /* horizontal edges */
        float ye = k ? y1 : y0;
        float dy = ye - v;
        float B = b * dy;
        float C = c * dy;
        C = C * dy;
        C = C - t;
        if (chord_overlaps(a, B, C, lo, hi)) return 1;
    }
    lo = y0 - v; hi = y1 - v;
    for (int k = 0; k < 2; ++k) {                 /* vertical edges */
        float xe = k ? x1 : x0;
        float dx = xe - u;
        float B = b * dx;
        float C = a * dx;
        C = C * dx;
        C = C - t;
        if (chord_overlaps(c, B, C, lo, hi)) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Per-Gaussian preprocess (Alg. 1 steps in_frustum/project/computeCov3D/computeCov2D/
 * computeColorFromSH; Alg. 4 cull z > 0.2 and opacity > 1/255; Eq. 2-3 threshold; the
 * tight bounding box of Section 4.1).
 *
 * Outputs per Gaussian g:
 *   valid[g]  1 when the Gaussian passes the cull and has a positive-definite 2D covariance
 *   rec32[g]  FP32 record (u, v, conic a b c, t, z, Sigma'00 01 11, alpha0, rgb, t uncapped)
 *   rec64[g]  FP64 values for the image reference (NULL to skip)
 *   rect[g]   candidate tile range tx0, tx1, ty0, ty1 (inclusive; tx0 > tx1 if empty)
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    const float *means, *scales, *quats, *opac, *sh;
    int32_t sh_degree, activated;
} OrGauss;

static void quat_to_R_f(const float q_in[4], float r[9], int *ok)
{
    float w = q_in[0], x = q_in[1], y = q_in[2], z = q_in[3];
    float n2 = w * w;
    n2 = n2 + x * x;
    n2 = n2 + y * y;
    n2 = n2 + z * z;
    if (!(n2 > 0.0f)) { *ok = 0; return; }
    float n = sqrtf(n2);
    w = w / n; x = x / n; y = y / n; z = z / n;
    float yy = y * y, zz = z * z, xx = x * x;
    float xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y, wz = w * z;
    r[0] = 1.0f - 2.0f * (yy + zz); r[1] = 2.0f * (xy - wz);         r[2] = 2.0f * (xz + wy);
    r[3] = 2.0f * (xy + wz);         r[4] = 1.0f - 2.0f * (xx + zz); r[5] = 2.0f * (yz - wx);
    r[6] = 2.0f * (xz - wy);         r[7] = 2.0f * (yz + wx);         r[8] = 1.0f - 2.0f * (xx + yy);
    *ok = 1;
}

static void quat_to_R_d(const double q_in[4], double r[9])
{
    double w = q_in[0], x = q_in[1], y = q_in[2], z = q_in[3];
    double n = sqrt(w * w + x * x + y * y + z * z);
    w /= n; x /= n; y /= n; z /= n;
    r[0] = 1 - 2 * (y * y + z * z); r[1] = 2 * (x * y - w * z);     r[2] = 2 * (x * z + w * y);
    r[3] = 2 * (x * y + w * z);     r[4] = 1 - 2 * (x * x + z * z); r[5] = 2 * (y * z - w * x);
    r[6] = 2 * (x * z - w * y);     r[7] = 2 * (y * z + w * x);     r[8] = 1 - 2 * (x * x + y * y);
}

static int preprocess_one(const OrGauss *G, int64_t g, const OrCamera *cam, const OrOpts *o,
                          float *rec, double *rec64, int32_t rect[4])
{
    const float *m = G->means + 3 * g;
    memset(rec, 0, sizeof(float) * REC32);
    rect[0] = 0; rect[1] = -1; rect[2] = 0; rect[3] = -1;
    const float *Rc = cam->R;
    /* camera-space mean, each row summed in index order */
    float p[3];
    for (int i = 0; i < 3; ++i) {
        float s = Rc[3 * i + 0] * m[0];
        s = s + Rc[3 * i + 1] * m[1];
        s = s + Rc[3 * i + 2] * m[2];
        p[i] = s + cam->t[i];
    }
    float alpha0;
    if (G->activated) {
        alpha0 = G->opac[g];
    } else {
        alpha0 = or_sigmoidf(G->opac[g]);
    }
    /* cull (Alg. 4): z > near and opacity > tau */
    if (!(p[2] > cam->near_z)) return 0;
    if (!(alpha0 > o->tau)) return 0;
    /* opacity-aware threshold (Eq. 3): q <= t = 2 ln(alpha0 / tau) */
    float t_full = or_threshold(alpha0, o->tau);
    float t = t_full;
    if (o->cap_3sigma && t > 9.0f) t = 9.0f;
    /* 3D covariance Sigma = R S S^T R^T */
    float s[3];
    for (int k = 0; k < 3; ++k) s[k] = G->activated ? G->scales[3 * g + k] : or_expf(G->scales[3 * g + k]);
    float r[9];
    int ok;
    quat_to_R_f(G->quats + 4 * g, r, &ok);
    if (!ok) return 0;
    float d2[3] = {s[0] * s[0], s[1] * s[1], s[2] * s[2]};
    float S[9];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            float acc = (r[3 * i + 0] * d2[0]) * r[3 * j + 0];
            acc = acc + (r[3 * i + 1] * d2[1]) * r[3 * j + 1];
            acc = acc + (r[3 * i + 2] * d2[2]) * r[3 * j + 2];
            S[3 * i + j] = acc;
            S[3 * j + i] = acc;
        }
    /* projection to pixel-area coordinates */
    float u = (cam->fx * p[0]) / p[2] + cam->cx;
    float v = (cam->fy * p[1]) / p[2] + cam->cy;
    /* EWA: J of the perspective map at p, with the 1.3 tan(half-fov) clamp */
    float tx = p[0], ty = p[1];
    if (o->clamp_fov) {
        float limx = 1.3f * ((0.5f * (float)cam->width) / cam->fx);
        float limy = 1.3f * ((0.5f * (float)cam->height) / cam->fy);
        float txz = p[0] / p[2], tyz = p[1] / p[2];
        txz = txz < -limx ? -limx : (txz > limx ? limx : txz);
        tyz = tyz < -limy ? -limy : (tyz > limy ? limy : tyz);
        tx = txz * p[2];
        ty = tyz * p[2];
    }
    float zz = p[2] * p[2];
    float j00 = cam->fx / p[2];
    float j02 = -((cam->fx * tx) / zz);
    float j11 = cam->fy / p[2];
    float j12 = -((cam->fy * ty) / zz);
    /* M = J Rc (2x3) */
    float M[6];
    for (int k = 0; k < 3; ++k) {
        M[k] = j00 * Rc[k] + j02 * Rc[6 + k];
        M[3 + k] = j11 * Rc[3 + k] + j12 * Rc[6 + k];
    }
    /* N = M Sigma, Sigma' = N M^T + dilation I */
    float N[6];
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k) {
            float acc = M[3 * i + 0] * S[0 + k];
            acc = acc + M[3 * i + 1] * S[3 + k];
            acc = acc + M[3 * i + 2] * S[6 + k];
            N[3 * i + k] = acc;
        }
    float s00 = N[0] * M[0];
    s00 = s00 + N[1] * M[1];
    s00 = s00 + N[2] * M[2];
    s00 = s00 + o->dilation;
    float s01 = N[0] * M[3];
    s01 = s01 + N[1] * M[4];
    s01 = s01 + N[2] * M[5];
    float s11 = N[3] * M[3];
    s11 = s11 + N[4] * M[4];
    s11 = s11 + N[5] * M[5];
    s11 = s11 + o->dilation;
    float det = s00 * s11 - s01 * s01;
    if (!(det > 0.0f)) return 0;
    float a = s11 / det;
    float b = (-s01) / det;
    float c = s00 / det;
    /* tight bounding box of {q <= t}: half extents sqrt(t Sigma'00), sqrt(t Sigma'11) (Sec. 4.1),
       padded by one pixel; the exact test decides inside it */
    float hx = sqrtf(t * s00);
    float hy = sqrtf(t * s11);
    int tiles_x = (cam->width + TILE - 1) / TILE, tiles_y = (cam->height + TILE - 1) / TILE;
    float fx0 = floorf(((u - hx) - 1.0f) * 0.0625f), fx1 = floorf(((u + hx) + 1.0f) * 0.0625f);
    float fy0 = floorf(((v - hy) - 1.0f) * 0.0625f), fy1 = floorf(((v + hy) + 1.0f) * 0.0625f);
    rec[F_ALL] = 0.0f;
    if (o->intersect == 1) {
        /* 3DGS pairs (Eq. 1; Alg. 1 radii, Alg. 2): radius r = ceil(3 sqrt(lambda_max)) of
           Sigma' (lambda_max = mid + sqrt(mid^2 - det), the discriminant clamped at 0 against
           rounding), and every tile of the square [u - r, u + r] x [v - r, v + r] */
        float mid = 0.5f * (s00 + s11);
        float disc = mid * mid - det;
        float lam = mid + sqrtf(disc > 0.0f ? disc : 0.0f);
        float rad = ceilf(3.0f * sqrtf(lam));
        fx0 = floorf((u - rad) * 0.0625f); fx1 = floorf((u + rad) * 0.0625f);
        fy0 = floorf((v - rad) * 0.0625f); fy1 = floorf((v + rad) * 0.0625f);
        rec[F_ALL] = 1.0f;
    }
    rec[F_U] = u; rec[F_V] = v; rec[F_A] = a; rec[F_B] = b; rec[F_C] = c; rec[F_T] = t;
    rec[F_Z] = p[2]; rec[F_S00] = s00; rec[F_S01] = s01; rec[F_S11] = s11; rec[F_ALPHA] = alpha0;
    rec[F_TFULL] = t_full;
    int empty = !(fx1 >= 0.0f) || !(fy1 >= 0.0f) || !(fx0 <= (float)(tiles_x - 1)) || !(fy0 <= (float)(tiles_y - 1));
    if (!empty) {
        rect[0] = fx0 < 0.0f ? 0 : (int)fx0;
        rect[1] = fx1 > (float)(tiles_x - 1) ? tiles_x - 1 : (int)fx1;
        rect[2] = fy0 < 0.0f ? 0 : (int)fy0;
        rect[3] = fy1 > (float)(tiles_y - 1) ? tiles_y - 1 : (int)fy1;
    }
    /* colour from SH (FP32), direction from the camera centre to the mean */
    float cpos[3];
    for (int i = 0; i < 3; ++i) {
        float acc = Rc[0 + i] * cam->t[0];
        acc = acc + Rc[3 + i] * cam->t[1];
        acc = acc + Rc[6 + i] * cam->t[2];
        cpos[i] = -acc;
    }
    float dir[3] = {m[0] - cpos[0], m[1] - cpos[1], m[2] - cpos[2]};
    float len = sqrtf(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
    dir[0] /= len; dir[1] /= len; dir[2] /= len;
    float Y[16];
    sh_basis_f(dir, Y);
    int nsh = sh_count(G->sh_degree);
    const float *sh = G->sh + 48 * g;
    for (int ch = 0; ch < 3; ++ch) {
        float acc = 0.0f;
        for (int i = 0; i < nsh; ++i) acc += Y[i] * sh[3 * i + ch];
        acc += 0.5f;
        rec[F_R + ch] = acc < 0.0f ? 0.0f : acc;
    }
    if (rec64) {
        /* the same quantities in binary64 for the image reference */
        double pd[3];
        for (int i = 0; i < 3; ++i)
            pd[i] = (double)Rc[3 * i] * m[0] + (double)Rc[3 * i + 1] * m[1] + (double)Rc[3 * i + 2] * m[2] + cam->t[i];
        double al = G->activated ? (double)G->opac[g] : 1.0 / (1.0 + exp(-(double)G->opac[g]));
        double sd[3];
        for (int k = 0; k < 3; ++k) sd[k] = G->activated ? (double)G->scales[3 * g + k] : exp((double)G->scales[3 * g + k]);
        double qd[4] = {G->quats[4 * g], G->quats[4 * g + 1], G->quats[4 * g + 2], G->quats[4 * g + 3]};
        double rd[9];
        quat_to_R_d(qd, rd);
        double Sd[9];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0;
                for (int k = 0; k < 3; ++k) acc += rd[3 * i + k] * sd[k] * sd[k] * rd[3 * j + k];
                Sd[3 * i + j] = acc;
            }
        double fx = cam->fx, fy = cam->fy;
        double ud = fx * pd[0] / pd[2] + cam->cx, vd = fy * pd[1] / pd[2] + cam->cy;
        double txd = pd[0], tyd = pd[1];
        if (o->clamp_fov) {
            double limx = 1.3 * (0.5 * cam->width / fx), limy = 1.3 * (0.5 * cam->height / fy);
            double a1 = pd[0] / pd[2], a2 = pd[1] / pd[2];
            a1 = a1 < -limx ? -limx : (a1 > limx ? limx : a1);
            a2 = a2 < -limy ? -limy : (a2 > limy ? limy : a2);
            txd = a1 * pd[2]; tyd = a2 * pd[2];
        }
        double J[6] = {fx / pd[2], 0.0, -fx * txd / (pd[2] * pd[2]), 0.0, fy / pd[2], -fy * tyd / (pd[2] * pd[2])};
        double Md[6];
        for (int i = 0; i < 2; ++i)
            for (int k = 0; k < 3; ++k)
                Md[3 * i + k] = J[3 * i] * Rc[k] + J[3 * i + 1] * Rc[3 + k] + J[3 * i + 2] * Rc[6 + k];
        double C2[4];
        for (int i = 0; i < 2; ++i)
            for (int l = 0; l < 2; ++l) {
                double acc = 0;
                for (int k = 0; k < 3; ++k)
                    for (int n = 0; n < 3; ++n) acc += Md[3 * i + k] * Sd[3 * k + n] * Md[3 * l + n];
                C2[2 * i + l] = acc;
            }
        C2[0] += o->dilation; C2[3] += o->dilation;
        double dd = C2[0] * C2[3] - C2[1] * C2[2];
        rec64[D_U] = ud; rec64[D_V] = vd;
        rec64[D_A] = C2[3] / dd; rec64[D_B] = -C2[1] / dd; rec64[D_C] = C2[0] / dd;
        rec64[D_ALPHA] = al;
        rec64[D_S00] = C2[0]; rec64[D_S01] = C2[1]; rec64[D_S11] = C2[3]; rec64[D_Z] = pd[2];
        double cp[3];
        for (int i = 0; i < 3; ++i)
            cp[i] = -((double)Rc[i] * cam->t[0] + (double)Rc[3 + i] * cam->t[1] + (double)Rc[6 + i] * cam->t[2]);
        double dv[3] = {m[0] - cp[0], m[1] - cp[1], m[2] - cp[2]};
        double ln = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
        dv[0] /= ln; dv[1] /= ln; dv[2] /= ln;
        double Yd[16];
        or_sh_basis(dv, Yd);
        for (int ch = 0; ch < 3; ++ch) {
            double acc = 0.0;
            for (int i = 0; i < nsh; ++i) acc += Yd[i] * sh[3 * i + ch];
            acc += 0.5;
            rec64[D_R + ch] = acc < 0.0 ? 0.0 : acc;
        }
    }
    return 1;
}

int64_t or_preprocess(int64_t P, const float *means, const float *scales, const float *quats,
                      const float *opac, const float *sh, int32_t sh_degree, int32_t activated,
                      const OrCamera *cam, const OrOpts *opts,
                      float *rec32, double *rec64, int32_t *rect, uint8_t *valid)
{
    OrGauss G = {means, scales, quats, opac, sh, sh_degree, activated};
    int64_t nvalid = 0;
#pragma omp parallel for schedule(static) reduction(+ : nvalid)
    for (int64_t g = 0; g < P; ++g) {
        int ok = preprocess_one(&G, g, cam, opts, rec32 + REC32 * g, rec64 ? rec64 + REC64 * g : NULL, rect + 4 * g);
        valid[g] = (uint8_t)ok;
        nvalid += ok;
    }
    return nvalid;
}

/* ------------------------------------------------------------------------------------------
 * Pair emission (Alg. 4 key/value generation, keeping only tiles passing Alg. 3).
 * key = (tile_id << 32) | bits(z) with tile_id = ty * tiles_x + tx; value = Gaussian id.
 * Order: Gaussian id, then the candidate tiles row-major.  counts[g] receives the pair
 * count of every Gaussian.  Returns N; keys/vals are written only when cap >= N.
 * ---------------------------------------------------------------------------------------- */
static void tile_rect(const OrCamera *cam, int tx, int ty, float r[4])
{
    int x1 = TILE * tx + TILE, y1 = TILE * ty + TILE;
    if (x1 > cam->width) x1 = cam->width;
    if (y1 > cam->height) y1 = cam->height;
    r[0] = (float)(TILE * tx); r[1] = (float)x1; r[2] = (float)(TILE * ty); r[3] = (float)y1;
}

static int32_t count_one(const float *rec, const int32_t *rc, const OrCamera *cam)
{
    if (rec[F_ALL] != 0.0f) return (rc[1] - rc[0] + 1) * (rc[3] - rc[2] + 1);
    int32_t n = 0;
    for (int ty = rc[2]; ty <= rc[3]; ++ty)
        for (int tx = rc[0]; tx <= rc[1]; ++tx) {
            float r[4];
            tile_rect(cam, tx, ty, r);
            n += or_tile_hit(rec[F_U], rec[F_V], rec[F_A], rec[F_B], rec[F_C], rec[F_T], r[0], r[1], r[2], r[3]);
        }
    return n;
}

int64_t or_emit_pairs(int64_t P, const float *rec32, const int32_t *rect, const uint8_t *valid,
                      const OrCamera *cam, int32_t *counts, uint64_t *keys, uint32_t *vals, int64_t cap)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t g = 0; g < P; ++g)
        counts[g] = valid[g] ? count_one(rec32 + REC32 * g, rect + 4 * g, cam) : 0;
    int64_t N = 0;
    for (int64_t g = 0; g < P; ++g) N += counts[g];
    if (!keys || cap < N) return N;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(P + 1));
    off[0] = 0;
    for (int64_t g = 0; g < P; ++g) off[g + 1] = off[g] + counts[g];
    int tiles_x = (cam->width + TILE - 1) / TILE;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t g = 0; g < P; ++g) {
        if (!counts[g]) continue;
        const float *rec = rec32 + REC32 * g;
        const int32_t *rc = rect + 4 * g;
        int64_t o = off[g];
        uint64_t zb = f2u(rec[F_Z]);
        for (int ty = rc[2]; ty <= rc[3]; ++ty)
            for (int tx = rc[0]; tx <= rc[1]; ++tx) {
                float r[4];
                tile_rect(cam, tx, ty, r);
                if (rec[F_ALL] != 0.0f ||
                    or_tile_hit(rec[F_U], rec[F_V], rec[F_A], rec[F_B], rec[F_C], rec[F_T], r[0], r[1], r[2], r[3])) {
                    keys[o] = ((uint64_t)(ty * tiles_x + tx) << 32) | zb;
                    vals[o] = (uint32_t)g;
                    ++o;
                }
            }
    }
    free(off);
    return N;
}

/* ------------------------------------------------------------------------------------------
 * Sort of the pairs by (key, value): the order the renderer walks (tile, then depth front to
 * back, then Gaussian id for equal depths).  A plain comparison sort.
 * ---------------------------------------------------------------------------------------- */
typedef struct { uint64_t k; uint32_t v; } OrPair;

static int pair_cmp(const void *pa, const void *pb)
{
    const OrPair *a = (const OrPair *)pa, *b = (const OrPair *)pb;
    if (a->k != b->k) return a->k < b->k ? -1 : 1;
    if (a->v != b->v) return a->v < b->v ? -1 : 1;
    return 0;
}

void or_sort_pairs(int64_t n, uint64_t *keys, uint32_t *vals)
{
    OrPair *p = (OrPair *)malloc(sizeof(OrPair) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { p[i].k = keys[i]; p[i].v = vals[i]; }
    qsort(p, (size_t)n, sizeof(OrPair), pair_cmp);
    for (int64_t i = 0; i < n; ++i) { keys[i] = p[i].k; vals[i] = p[i].v; }
    free(p);
}

/* ranges[2*tile], ranges[2*tile+1] = first and one-past-last position of the tile */
void or_tile_ranges(int64_t n, const uint64_t *keys, int32_t ntiles, int64_t *ranges)
{
    for (int32_t i = 0; i < 2 * ntiles; ++i) ranges[i] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t tile = (int64_t)(keys[i] >> 32);
        if (tile < 0 || tile >= ntiles) continue;
        if (i == 0 || (int64_t)(keys[i - 1] >> 32) != tile) ranges[2 * tile] = i;
        if (i == n - 1 || (int64_t)(keys[i + 1] >> 32) != tile) ranges[2 * tile + 1] = i + 1;
    }
}

/* ------------------------------------------------------------------------------------------
 * Per-pixel skip decision, binary32: q = fmaf(fmaf(a, dx, 2b dy), dx, (c dy) dy) with
 * dx = px - u, dy = py - v at the pixel sample (i + 1/2, j + 1/2); the Gaussian is skipped
 * when q > t (equivalently alpha0 exp(-q/2) < tau, Eq. 2-3), or when q is not a number.
 * ---------------------------------------------------------------------------------------- */
static int pixel_skip(const float *rec, float px, float py)
{
    float dx = px - rec[F_U];
    float dy = py - rec[F_V];
    float b2 = rec[F_B] + rec[F_B];
    float By = b2 * dy;
    float Cy = rec[F_C] * dy;
    Cy = Cy * dy;
    float q = fmaf(fmaf(rec[F_A], dx, By), dx, Cy);
    return !(q <= rec[F_T]);
}

/* State of one pixel's front-to-back walk. */
typedef struct {
    double C[3];
    double T;
    float Cf[3];
    float Tf;
    uint32_t last;
    int done;
    int64_t evals;
} PixState;

/* One list entry at position `pos` (1-based count of entries walked) for pixel (px, py).
   Blend rule: alpha = min(alpha_max, alpha0 exp(-q/2)); skip if alpha < tau (decided in
   binary32 as above); T' = T (1 - alpha); stop without this Gaussian if T' < T_min;
   else C += rgb alpha T, T = T'. */
static void blend_step(PixState *s, int mode, const float *rec, const double *rec64,
                       float px, float py, const OrOpts *o, uint32_t pos)
{
    s->evals++;
    if (pixel_skip(rec, px, py)) return;
    if (mode == 32) {
        float dx = px - rec[F_U], dy = py - rec[F_V];
        float q = rec[F_A] * dx * dx + 2.0f * rec[F_B] * dx * dy + rec[F_C] * dy * dy;
        float al = rec[F_ALPHA] * expf(-0.5f * q);
        if (al > o->alpha_max) al = o->alpha_max;
        float Tn = s->Tf * (1.0f - al);
        if (Tn < o->T_min) { s->done = 1; return; }
        for (int ch = 0; ch < 3; ++ch) s->Cf[ch] += rec[F_R + ch] * al * s->Tf;
        s->Tf = Tn;
    } else {
        double dx = (double)px - rec64[D_U], dy = (double)py - rec64[D_V];
        double q = rec64[D_A] * dx * dx + 2.0 * rec64[D_B] * dx * dy + rec64[D_C] * dy * dy;
        double al = rec64[D_ALPHA] * exp(-0.5 * q);
        if (al > (double)o->alpha_max) al = (double)o->alpha_max;
        double Tn = s->T * (1.0 - al);
        if (Tn < (double)o->T_min) { s->done = 1; return; }
        for (int ch = 0; ch < 3; ++ch) s->C[ch] += rec64[D_R + ch] * al * s->T;
        s->T = Tn;
    }
    s->last = pos;
}

static void pix_init(PixState *s)
{
    memset(s, 0, sizeof(*s));
    s->T = 1.0;
    s->Tf = 1.0f;
}

static void pix_store(const PixState *s, int mode, const OrOpts *o, int64_t idx, int64_t npx,
                      double *rgb, double *T_out, uint32_t *last)
{
    for (int ch = 0; ch < 3; ++ch) {
        if (mode == 32) {
            float val = s->Cf[ch] + s->Tf * o->bg[ch];
            rgb[ch * npx + idx] = (double)val;
        } else {
            rgb[ch * npx + idx] = s->C[ch] + s->T * (double)o->bg[ch];
        }
    }
    if (T_out) T_out[idx] = mode == 32 ? (double)s->Tf : s->T;
    if (last) last[idx] = s->last;
}

/* Tiled blend: each pixel walks its tile's sorted list (Section 2.2, Section 5.2). */
int64_t or_blend_tiled(int32_t mode, const OrCamera *cam, const OrOpts *o,
                       const int64_t *ranges, const uint32_t *vals,
                       const float *rec32, const double *rec64,
                       double *rgb, double *T_out, uint32_t *last)
{
    int W = cam->width, H = cam->height;
    int tiles_x = (W + TILE - 1) / TILE, tiles_y = (H + TILE - 1) / TILE;
    int64_t npx = (int64_t)W * H;
    int64_t evals = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : evals)
    for (int tile = 0; tile < tiles_x * tiles_y; ++tile) {
        int tx = tile % tiles_x, ty = tile / tiles_x;
        int64_t s0 = ranges[2 * tile], s1 = ranges[2 * tile + 1];
        for (int j = TILE * ty; j < TILE * ty + TILE && j < H; ++j)
            for (int i = TILE * tx; i < TILE * tx + TILE && i < W; ++i) {
                PixState st;
                pix_init(&st);
                float px = (float)i + 0.5f, py = (float)j + 0.5f;
                for (int64_t k = s0; k < s1 && !st.done; ++k) {
                    uint32_t g = vals[k];
                    blend_step(&st, mode, rec32 + REC32 * (int64_t)g, rec64 ? rec64 + REC64 * (int64_t)g : NULL,
                               px, py, o, (uint32_t)(k - s0 + 1));
                }
                evals += st.evals;
                pix_store(&st, mode, o, (int64_t)j * W + i, npx, rgb, T_out, last);
            }
    }
    return evals;
}

/* Brute force: every pixel walks every Gaussian that passed the cull, in the order
   `order` (Gaussian ids sorted by (bits(z), id)); no tiles, no pairs.  `last` here counts
   positions in `order`, so only rgb and T are comparable with the tiled walk. */
void or_blend_brute(int32_t mode, const OrCamera *cam, const OrOpts *o, int64_t n_order,
                    const uint32_t *order, const float *rec32, const double *rec64,
                    int32_t x0, int32_t y0, int32_t w, int32_t h,
                    double *rgb, double *T_out)
{
    int W = cam->width;
    (void)W;
    int64_t npx = (int64_t)w * h;
#pragma omp parallel for schedule(dynamic, 1)
    for (int jj = 0; jj < h; ++jj)
        for (int ii = 0; ii < w; ++ii) {
            PixState st;
            pix_init(&st);
            float px = (float)(x0 + ii) + 0.5f, py = (float)(y0 + jj) + 0.5f;
            for (int64_t k = 0; k < n_order && !st.done; ++k) {
                uint32_t g = order[k];
                blend_step(&st, mode, rec32 + REC32 * (int64_t)g, rec64 ? rec64 + REC64 * (int64_t)g : NULL,
                           px, py, o, (uint32_t)(k + 1));
            }
            pix_store(&st, mode, o, (int64_t)jj * w + ii, npx, rgb, T_out, NULL);
        }
}

/* ------------------------------------------------------------------------------------------
 * Whole frame in one call (preprocess -> pairs -> sort -> ranges -> blend), the form the
 * CPU baseline times.  Returns N (pairs) or -1 on allocation failure.  keys/vals, when
 * non-NULL and cap >= N, receive the sorted pair list; stats[0..3] = visible Gaussians
 * (>= 1 pair), N, evaluations, Gaussians passing the cull.
 * ---------------------------------------------------------------------------------------- */
int64_t or_render(int32_t mode, int64_t P, const float *means, const float *scales, const float *quats,
                  const float *opac, const float *sh, int32_t sh_degree, int32_t activated,
                  const OrCamera *cam, const OrOpts *o,
                  double *rgb, double *T_out, uint32_t *last,
                  uint64_t *keys_out, uint32_t *vals_out, int64_t cap, int64_t *stats)
{
    float *rec32 = (float *)malloc(sizeof(float) * REC32 * (size_t)(P > 0 ? P : 1));
    double *rec64 = mode == 64 ? (double *)malloc(sizeof(double) * REC64 * (size_t)(P > 0 ? P : 1)) : NULL;
    int32_t *rect = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(P > 0 ? P : 1));
    uint8_t *valid = (uint8_t *)malloc((size_t)(P > 0 ? P : 1));
    int32_t *counts = (int32_t *)malloc(sizeof(int32_t) * (size_t)(P > 0 ? P : 1));
    if (!rec32 || !rect || !valid || !counts || (mode == 64 && !rec64)) return -1;
    int64_t ncull = or_preprocess(P, means, scales, quats, opac, sh, sh_degree, activated, cam, o, rec32, rec64, rect, valid);
    int64_t N = or_emit_pairs(P, rec32, rect, valid, cam, counts, NULL, NULL, 0);
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(N > 0 ? N : 1));
    uint32_t *vals = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(N > 0 ? N : 1));
    if (!keys || !vals) return -1;
    or_emit_pairs(P, rec32, rect, valid, cam, counts, keys, vals, N);
    or_sort_pairs(N, keys, vals);
    int tiles = ((cam->width + TILE - 1) / TILE) * ((cam->height + TILE - 1) / TILE);
    int64_t *ranges = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)tiles);
    or_tile_ranges(N, keys, tiles, ranges);
    int64_t evals = or_blend_tiled(mode, cam, o, ranges, vals, rec32, rec64, rgb, T_out, last);
    if (keys_out && vals_out && cap >= N) {
        memcpy(keys_out, keys, sizeof(uint64_t) * (size_t)N);
        memcpy(vals_out, vals, sizeof(uint32_t) * (size_t)N);
    }
    if (stats) {
        int64_t vis = 0;
        for (int64_t g = 0; g < P; ++g) vis += counts[g] > 0;
        stats[0] = vis; stats[1] = N; stats[2] = evals; stats[3] = ncull;
    }
    free(rec32); free(rec64); free(rect); free(valid); free(counts); free(keys); free(vals); free(ranges);
    return N;
}
