/*
 * gs_oracle_grad.c -- binary64 gradient of the rasterizer for the oracle.  TEST INFRASTRUCTURE
 * ONLY (see gs_oracle.c).  The paper claims differentiability (abstract) but describes no
 * backward pass; this file is the exact derivative of the forward definition in gs_oracle.c
 * with every decision held fixed:
 *   - which Gaussians contribute to which pixel, in which order, and where the walk stops
 *     (the per-pixel contributor lists of a reference render);
 *   - whether alpha was clamped at alpha_max (then d alpha = 0), whether an RGB channel was
 *     clamped at 0 (then d rgb = 0), whether x/z or y/z was clamped in the Jacobian.
 * The frozen function is smooth in the parameters, so its gradient is checked here against
 * central finite differences in binary64, and the GPU's gradient against it.
 *
 * Parameters (binary64): means [P,3], scales or log-scales [P,3], quaternions [P,4] (any
 * length), opacities or logits [P], SH [P,16,3]; activated = 0 means log-scales and logits.
 * Loss: any L with dL/dimage given ([3,H,W]).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float near_z;
} OrCamera;

typedef struct {
    float bg[3];
    float tau;
    float alpha_max;
    float T_min;
    float dilation;
    int32_t cap_3sigma;
    int32_t clamp_fov;
    int32_t intersect;      /* pair rule of the forward; the gradient does not depend on it */
} OrOpts;

void or_sh_basis(const double d[3], double Y[16]);

/* flags per Gaussian: bit 0/1/2 rgb channel clamped at 0, bit 3 x/z clamped low, bit 4 x/z
   clamped high, bit 5 y/z clamped low, bit 6 y/z clamped high */
enum { FL_R = 1, FL_G = 2, FL_B = 4, FL_XLO = 8, FL_XHI = 16, FL_YLO = 32, FL_YHI = 64 };

typedef struct {
    const double *means, *scales, *quats, *opac, *sh;
    int32_t activated, sh_degree;
} GParams;

/* Everything the forward of one Gaussian computes, kept for the backward. */
typedef struct {
    double p[3];          /* camera-space mean */
    double s[3];          /* scales */
    double qn[4], qlen;   /* normalised quaternion and the input's length */
    double Rq[9];         /* rotation of the normalised quaternion */
    double Sg[9];         /* 3D covariance */
    double txz, tyz;      /* x/z, y/z after the clamp */
    double J[6];          /* 2x3 Jacobian */
    double M[6];          /* J Rc */
    double S2[4];         /* Sigma' (2x2, with dilation) */
    double Q[4];          /* its inverse: [[a, b], [b, c]] */
    double u, v;
    double alpha0;
    double dir[3], dlen;  /* unit direction camera -> mean, and the distance */
    double Y[16];
    double rgb[3];
} G64;

static int sh_count(int degree)
{
    if (degree < 0) degree = 0;
    if (degree > 3) degree = 3;
    return (degree + 1) * (degree + 1);
}

/* forward of one Gaussian in binary64 under the given flags (flags_out: set flags instead) */
static void geom64(const GParams *G, int64_t g, const OrCamera *cam, const OrOpts *o, int flags, int *flags_out,
                   G64 *r)
{
    const double *m = G->means + 3 * g;
    const float *Rc = cam->R;
    for (int i = 0; i < 3; ++i)
        r->p[i] = (double)Rc[3 * i] * m[0] + (double)Rc[3 * i + 1] * m[1] + (double)Rc[3 * i + 2] * m[2] + cam->t[i];
    for (int k = 0; k < 3; ++k) r->s[k] = G->activated ? G->scales[3 * g + k] : exp(G->scales[3 * g + k]);
    const double *q = G->quats + 4 * g;
    r->qlen = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) r->qn[k] = q[k] / r->qlen;
    double w = r->qn[0], x = r->qn[1], y = r->qn[2], z = r->qn[3];
    double *R = r->Rq;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * r->s[k] * r->s[k] * R[3 * j + k];
            r->Sg[3 * i + j] = acc;
        }
    const double fx = cam->fx, fy = cam->fy;
    double pz = r->p[2];
    r->u = fx * r->p[0] / pz + cam->cx;
    r->v = fy * r->p[1] / pz + cam->cy;
    double txz = r->p[0] / pz, tyz = r->p[1] / pz;
    int fl = 0;
    if (o->clamp_fov) {
        double limx = 1.3 * (0.5 * cam->width / fx), limy = 1.3 * (0.5 * cam->height / fy);
        if (flags_out) {
            if (txz < -limx) fl |= FL_XLO;
            if (txz > limx) fl |= FL_XHI;
            if (tyz < -limy) fl |= FL_YLO;
            if (tyz > limy) fl |= FL_YHI;
        } else {
            fl = flags;
        }
        if (fl & FL_XLO) txz = -limx;
        if (fl & FL_XHI) txz = limx;
        if (fl & FL_YLO) tyz = -limy;
        if (fl & FL_YHI) tyz = limy;
    }
    r->txz = txz;
    r->tyz = tyz;
    /* J02 = -fx x~/z^2 with x~ = txz z, i.e. -fx txz / z */
    double *J = r->J;
    J[0] = fx / pz; J[1] = 0.0; J[2] = -fx * txz / pz;
    J[3] = 0.0; J[4] = fy / pz; J[5] = -fy * tyz / pz;
    for (int i = 0; i < 2; ++i)
        for (int k = 0; k < 3; ++k)
            r->M[3 * i + k] = J[3 * i] * Rc[k] + J[3 * i + 1] * Rc[3 + k] + J[3 * i + 2] * Rc[6 + k];
    for (int i = 0; i < 2; ++i)
        for (int l = 0; l < 2; ++l) {
            double acc = 0;
            for (int k = 0; k < 3; ++k)
                for (int n = 0; n < 3; ++n) acc += r->M[3 * i + k] * r->Sg[3 * k + n] * r->M[3 * l + n];
            r->S2[2 * i + l] = acc;
        }
    r->S2[0] += o->dilation;
    r->S2[3] += o->dilation;
    double det = r->S2[0] * r->S2[3] - r->S2[1] * r->S2[2];
    r->Q[0] = r->S2[3] / det;
    r->Q[1] = -r->S2[1] / det;
    r->Q[2] = -r->S2[2] / det;
    r->Q[3] = r->S2[0] / det;
    r->alpha0 = G->activated ? G->opac[g] : 1.0 / (1.0 + exp(-G->opac[g]));
    double cp[3];
    for (int i = 0; i < 3; ++i) cp[i] = -((double)Rc[i] * cam->t[0] + (double)Rc[3 + i] * cam->t[1] + (double)Rc[6 + i] * cam->t[2]);
    double dv[3] = {m[0] - cp[0], m[1] - cp[1], m[2] - cp[2]};
    r->dlen = sqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
    for (int i = 0; i < 3; ++i) r->dir[i] = dv[i] / r->dlen;
    or_sh_basis(r->dir, r->Y);
    int nsh = sh_count(G->sh_degree);
    const double *sh = G->sh + 48 * g;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int i = 0; i < nsh; ++i) acc += r->Y[i] * sh[3 * i + ch];
        acc += 0.5;
        int clamped = flags_out ? (acc < 0.0) : ((flags >> ch) & 1);
        if (flags_out && clamped) fl |= (1 << ch);
        r->rgb[ch] = clamped ? 0.0 : acc;
    }
    if (flags_out) *flags_out = fl;
}

/* flags of every Gaussian at the given parameters */
void or_grad_flags(int64_t P, const double *means, const double *scales, const double *quats, const double *opac,
                   const double *sh, int32_t sh_degree, int32_t activated, const OrCamera *cam, const OrOpts *o,
                   const uint8_t *valid, int32_t *flags)
{
    GParams G = {means, scales, quats, opac, sh, activated, sh_degree};
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < P; ++g) {
        G64 r;
        int fl = 0;
        if (valid[g]) geom64(&G, g, cam, o, 0, &fl, &r);
        flags[g] = fl;
    }
}

static double alpha_of(const G64 *r, double px, double py, double *qout)
{
    double dx = px - r->u, dy = py - r->v;
    double q = r->Q[0] * dx * dx + 2.0 * r->Q[1] * dx * dy + r->Q[3] * dy * dy;
    *qout = q;
    return r->alpha0 * exp(-0.5 * q);
}

/* Forward under frozen decisions: pixel p blends contributors gid[off[p] .. off[p+1]) in order;
   aclamp marks contributions whose alpha is clamped at alpha_max.  Writes rgb [3,H,W] and T. */
void or_forward_fixed(int64_t P, const double *means, const double *scales, const double *quats, const double *opac,
                      const double *sh, int32_t sh_degree, int32_t activated, const OrCamera *cam, const OrOpts *o,
                      const uint8_t *valid, const int32_t *flags, const int64_t *off, const int32_t *gid,
                      const uint8_t *aclamp, double *rgb, double *T_out)
{
    GParams G = {means, scales, quats, opac, sh, activated, sh_degree};
    G64 *rs = (G64 *)malloc(sizeof(G64) * (size_t)(P > 0 ? P : 1));
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < P; ++g)
        if (valid[g]) geom64(&G, g, cam, o, flags[g], NULL, &rs[g]);
    const int W = cam->width, H = cam->height;
    const int64_t npx = (int64_t)W * H;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t pix = 0; pix < npx; ++pix) {
        double px = (double)(pix % W) + 0.5, py = (double)(pix / W) + 0.5;
        double C[3] = {0, 0, 0}, T = 1.0;
        for (int64_t k = off[pix]; k < off[pix + 1]; ++k) {
            const G64 *r = &rs[gid[k]];
            double q;
            double al = aclamp[k] ? (double)o->alpha_max : alpha_of(r, px, py, &q);
            for (int ch = 0; ch < 3; ++ch) C[ch] += r->rgb[ch] * al * T;
            T *= 1.0 - al;
        }
        for (int ch = 0; ch < 3; ++ch) rgb[ch * npx + pix] = C[ch] + T * (double)o->bg[ch];
        if (T_out) T_out[pix] = T;
    }
    free(rs);
}

/* d Y_i / d (x, y, z) of the SH polynomials (as functions on R^3) */
static void sh_basis_grad(const double d[3], double dY[16][3])
{
    const double pi = 3.14159265358979323846;
    double k[16];
    k[0] = 0.5 / sqrt(pi);
    double c1 = sqrt(3.0 / (4.0 * pi));
    k[1] = -c1; k[2] = c1; k[3] = -c1;
    k[4] = 0.5 * sqrt(15.0 / pi); k[5] = -0.5 * sqrt(15.0 / pi); k[6] = 0.25 * sqrt(5.0 / pi);
    k[7] = -0.5 * sqrt(15.0 / pi); k[8] = 0.25 * sqrt(15.0 / pi);
    k[9] = -0.25 * sqrt(35.0 / (2.0 * pi)); k[10] = 0.5 * sqrt(105.0 / pi); k[11] = -0.25 * sqrt(21.0 / (2.0 * pi));
    k[12] = 0.25 * sqrt(7.0 / pi); k[13] = -0.25 * sqrt(21.0 / (2.0 * pi)); k[14] = 0.25 * sqrt(105.0 / pi);
    k[15] = -0.25 * sqrt(35.0 / (2.0 * pi));
    double x = d[0], y = d[1], z = d[2];
    double xx = x * x, yy = y * y, zz = z * z;
    memset(dY, 0, sizeof(double) * 48);
    dY[1][1] = k[1];
    dY[2][2] = k[2];
    dY[3][0] = k[3];
    dY[4][0] = k[4] * y; dY[4][1] = k[4] * x;
    dY[5][1] = k[5] * z; dY[5][2] = k[5] * y;
    dY[6][0] = -2 * k[6] * x; dY[6][1] = -2 * k[6] * y; dY[6][2] = 4 * k[6] * z;
    dY[7][0] = k[7] * z; dY[7][2] = k[7] * x;
    dY[8][0] = 2 * k[8] * x; dY[8][1] = -2 * k[8] * y;
    dY[9][0] = 6 * k[9] * x * y; dY[9][1] = k[9] * (3 * xx - 3 * yy);
    dY[10][0] = k[10] * y * z; dY[10][1] = k[10] * x * z; dY[10][2] = k[10] * x * y;
    dY[11][0] = -2 * k[11] * x * y; dY[11][1] = k[11] * (4 * zz - xx - 3 * yy); dY[11][2] = 8 * k[11] * y * z;
    dY[12][0] = -6 * k[12] * x * z; dY[12][1] = -6 * k[12] * y * z; dY[12][2] = k[12] * (6 * zz - 3 * xx - 3 * yy);
    dY[13][0] = k[13] * (4 * zz - 3 * xx - yy); dY[13][1] = -2 * k[13] * x * y; dY[13][2] = 8 * k[13] * x * z;
    dY[14][0] = 2 * k[14] * x * z; dY[14][1] = -2 * k[14] * y * z; dY[14][2] = k[14] * (xx - yy);
    dY[15][0] = k[15] * (3 * xx - 3 * yy); dY[15][1] = -6 * k[15] * x * y;
}

/* Backward of one Gaussian from its 2D gradients (u, v, conic a, b, c, alpha0, rgb) to the
   parameters.  Chain: rgb -> SH coefficients and the direction -> mean; alpha0 -> opacity
   (logit); conic -> Sigma' (dQ = -Q dSigma' Q) -> (Sigma, M) -> (scales, quaternion) and J ->
   camera-space mean; (u, v) -> camera-space mean; camera-space mean -> mean. */
static void back64(const GParams *G, int64_t g, const OrCamera *cam, const OrOpts *o, int flags, const G64 *r,
                   const double d2[9], double *gm, double *gs, double *gq, double *go, double *gsh)
{
    (void)o;
    const float *Rc = cam->R;
    const double du = d2[0], dv = d2[1], da = d2[2], db = d2[3], dc = d2[4], dal = d2[5];
    const double drgb[3] = {d2[6], d2[7], d2[8]};
    double dp[3] = {0, 0, 0};     /* dL / d(camera-space mean) */
    double dmean[3] = {0, 0, 0};  /* dL / d(world mean), direct terms */
    /* colour */
    int nsh = sh_count(G->sh_degree);
    double ddir[3] = {0, 0, 0};
    double dY[16][3];
    sh_basis_grad(r->dir, dY);
    const double *sh = G->sh + 48 * g;
    for (int ch = 0; ch < 3; ++ch) {
        if ((flags >> ch) & 1) continue;
        for (int i = 0; i < nsh; ++i) {
            gsh[48 * g + 3 * i + ch] += r->Y[i] * drgb[ch];
            for (int a = 0; a < 3; ++a) ddir[a] += drgb[ch] * sh[3 * i + ch] * dY[i][a];
        }
    }
    double dd = ddir[0] * r->dir[0] + ddir[1] * r->dir[1] + ddir[2] * r->dir[2];
    for (int a = 0; a < 3; ++a) dmean[a] += (ddir[a] - r->dir[a] * dd) / r->dlen;
    /* opacity */
    go[g] += G->activated ? dal : dal * r->alpha0 * (1.0 - r->alpha0);
    /* conic -> Sigma' */
    double GQ[4] = {da, 0.5 * db, 0.5 * db, dc};
    double T1[4], GS2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) T1[2 * i + j] = r->Q[2 * i] * GQ[j] + r->Q[2 * i + 1] * GQ[2 + j];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) GS2[2 * i + j] = -(T1[2 * i] * r->Q[j] + T1[2 * i + 1] * r->Q[2 + j]);
    /* Sigma' = M Sigma M^T (+ dilation): dSigma = M^T G M, dM = 2 G M Sigma */
    double GSg[9], GM[6];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) acc += r->M[3 * a + i] * GS2[2 * a + b] * r->M[3 * b + j];
            GSg[3 * i + j] = acc;
        }
    for (int a = 0; a < 2; ++a)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int b = 0; b < 2; ++b)
                for (int n = 0; n < 3; ++n) acc += GS2[2 * a + b] * r->M[3 * b + n] * r->Sg[3 * n + k];
            GM[3 * a + k] = 2.0 * acc;
        }
    /* M = J Rc: dJ = dM Rc^T */
    double GJ[6];
    for (int a = 0; a < 2; ++a)
        for (int j = 0; j < 3; ++j) {
            double acc = 0;
            for (int k = 0; k < 3; ++k) acc += GM[3 * a + k] * Rc[3 * j + k];
            GJ[3 * a + j] = acc;
        }
    /* J entries as functions of p: J00 = fx/z, J02 = -fx txz/z, J11 = fy/z, J12 = -fy tyz/z,
       txz = x/z unless clamped (then constant) */
    const double fx = cam->fx, fy = cam->fy, z = r->p[2];
    dp[2] += GJ[0] * (-fx / (z * z)) + GJ[4] * (-fy / (z * z));
    if (!(flags & (FL_XLO | FL_XHI))) {
        /* J02 = -fx x / z^2 */
        dp[0] += GJ[2] * (-fx / (z * z));
        dp[2] += GJ[2] * (2.0 * fx * r->p[0] / (z * z * z));
    } else {
        dp[2] += GJ[2] * (fx * r->txz / (z * z));
    }
    if (!(flags & (FL_YLO | FL_YHI))) {
        dp[1] += GJ[5] * (-fy / (z * z));
        dp[2] += GJ[5] * (2.0 * fy * r->p[1] / (z * z * z));
    } else {
        dp[2] += GJ[5] * (fy * r->tyz / (z * z));
    }
    /* projection u = fx x/z + cx, v = fy y/z + cy */
    dp[0] += du * fx / z;
    dp[1] += dv * fy / z;
    dp[2] += du * (-fx * r->p[0] / (z * z)) + dv * (-fy * r->p[1] / (z * z));
    /* camera-space mean -> world mean: p = Rc m + t */
    for (int a = 0; a < 3; ++a) {
        double acc = dmean[a];
        for (int i = 0; i < 3; ++i) acc += (double)Rc[3 * i + a] * dp[i];
        gm[3 * g + a] += acc;
    }
    /* Sigma = R diag(s^2) R^T: ds_k = 2 s_k r_k^T G r_k ; dR = 2 G R D */
    const double *R = r->Rq;
    for (int k = 0; k < 3; ++k) {
        double acc = 0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) acc += R[3 * i + k] * GSg[3 * i + j] * R[3 * j + k];
        double ds = 2.0 * r->s[k] * acc;
        gs[3 * g + k] += G->activated ? ds : ds * r->s[k];
    }
    double GR[9];
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) {
            double acc = 0;
            for (int j = 0; j < 3; ++j) acc += GSg[3 * i + j] * R[3 * j + k];
            GR[3 * i + k] = 2.0 * acc * r->s[k] * r->s[k];
        }
    double w = r->qn[0], x = r->qn[1], y = r->qn[2], zq = r->qn[3];
    double dqn[4];
    dqn[0] = GR[1] * (-2 * zq) + GR[2] * (2 * y) + GR[3] * (2 * zq) + GR[5] * (-2 * x) + GR[6] * (-2 * y) + GR[7] * (2 * x);
    dqn[1] = GR[1] * (2 * y) + GR[2] * (2 * zq) + GR[3] * (2 * y) + GR[4] * (-4 * x) + GR[5] * (-2 * w) + GR[6] * (2 * zq) +
             GR[7] * (2 * w) + GR[8] * (-4 * x);
    dqn[2] = GR[0] * (-4 * y) + GR[1] * (2 * x) + GR[2] * (2 * w) + GR[3] * (2 * x) + GR[5] * (2 * zq) + GR[6] * (-2 * w) +
             GR[7] * (2 * zq) + GR[8] * (-4 * y);
    dqn[3] = GR[0] * (-4 * zq) + GR[1] * (-2 * w) + GR[2] * (2 * x) + GR[3] * (2 * w) + GR[4] * (-4 * zq) + GR[5] * (2 * y) +
             GR[6] * (2 * x) + GR[7] * (2 * y);
    double proj = dqn[0] * w + dqn[1] * x + dqn[2] * y + dqn[3] * zq;
    gq[4 * g + 0] += (dqn[0] - w * proj) / r->qlen;
    gq[4 * g + 1] += (dqn[1] - x * proj) / r->qlen;
    gq[4 * g + 2] += (dqn[2] - y * proj) / r->qlen;
    gq[4 * g + 3] += (dqn[3] - zq * proj) / r->qlen;
}

/* Gradient of L under frozen decisions.  d2d (nullable, [P,9]) receives the per-Gaussian 2D
   gradients (u, v, a, b, c, alpha0, r, g, b) that the blend backward accumulates. */
void or_backward_fixed(int64_t P, const double *means, const double *scales, const double *quats,
                       const double *opac, const double *sh, int32_t sh_degree, int32_t activated,
                       const OrCamera *cam, const OrOpts *o, const uint8_t *valid, const int32_t *flags,
                       const int64_t *off, const int32_t *gid, const uint8_t *aclamp, const double *dimg,
                       double *gm, double *gs, double *gq, double *go, double *gsh, double *d2d_out)
{
    GParams G = {means, scales, quats, opac, sh, activated, sh_degree};
    G64 *rs = (G64 *)malloc(sizeof(G64) * (size_t)(P > 0 ? P : 1));
    double *d2 = (double *)calloc((size_t)(P > 0 ? P : 1) * 9, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < P; ++g)
        if (valid[g]) geom64(&G, g, cam, o, flags[g], NULL, &rs[g]);
    const int W = cam->width, H = cam->height;
    const int64_t npx = (int64_t)W * H;
    /* blend backward, per pixel back to front (serial over pixels: exact accumulation order) */
    for (int64_t pix = 0; pix < npx; ++pix) {
        const int64_t k0 = off[pix], k1 = off[pix + 1];
        if (k1 == k0) continue;
        double px = (double)(pix % W) + 0.5, py = (double)(pix / W) + 0.5;
        double gpx[3];
        for (int ch = 0; ch < 3; ++ch) gpx[ch] = dimg[ch * npx + pix];
        /* forward pass to get T before every contribution */
        int64_t n = k1 - k0;
        double *Tb = (double *)malloc(sizeof(double) * (size_t)(n + 1));
        double *al = (double *)malloc(sizeof(double) * (size_t)n);
        double *qv = (double *)malloc(sizeof(double) * (size_t)n);
        Tb[0] = 1.0;
        for (int64_t k = 0; k < n; ++k) {
            const G64 *r = &rs[gid[k0 + k]];
            al[k] = aclamp[k0 + k] ? (double)o->alpha_max : alpha_of(r, px, py, &qv[k]);
            Tb[k + 1] = Tb[k] * (1.0 - al[k]);
        }
        double S = Tb[n] * (gpx[0] * o->bg[0] + gpx[1] * o->bg[1] + gpx[2] * o->bg[2]);
        for (int64_t k = n - 1; k >= 0; --k) {
            const int32_t g = gid[k0 + k];
            const G64 *r = &rs[g];
            double gc = gpx[0] * r->rgb[0] + gpx[1] * r->rgb[1] + gpx[2] * r->rgb[2];
            double *D = d2 + 9 * (int64_t)g;
            for (int ch = 0; ch < 3; ++ch) D[6 + ch] += al[k] * Tb[k] * gpx[ch];
            double dalpha = Tb[k] * gc - S / (1.0 - al[k]);
            S += gc * al[k] * Tb[k];
            if (aclamp[k0 + k]) continue;
            double e = exp(-0.5 * qv[k]);
            D[5] += dalpha * e;
            double dq = -0.5 * al[k] * dalpha;
            double dx = px - r->u, dy = py - r->v;
            D[2] += dq * dx * dx;
            D[3] += dq * 2.0 * dx * dy;
            D[4] += dq * dy * dy;
            D[0] += dq * (-2.0 * (r->Q[0] * dx + r->Q[1] * dy));
            D[1] += dq * (-2.0 * (r->Q[1] * dx + r->Q[3] * dy));
        }
        free(Tb);
        free(al);
        free(qv);
    }
    memset(gm, 0, sizeof(double) * 3 * (size_t)P);
    memset(gs, 0, sizeof(double) * 3 * (size_t)P);
    memset(gq, 0, sizeof(double) * 4 * (size_t)P);
    memset(go, 0, sizeof(double) * (size_t)P);
    memset(gsh, 0, sizeof(double) * 48 * (size_t)P);
#pragma omp parallel for schedule(static)
    for (int64_t g = 0; g < P; ++g)
        if (valid[g]) back64(&G, g, cam, o, flags[g], &rs[g], d2 + 9 * g, gm, gs, gq, go, gsh);
    if (d2d_out) memcpy(d2d_out, d2, sizeof(double) * 9 * (size_t)P);
    free(d2);
    free(rs);
}

/* Per-pixel contributor lists of a reference render: walks the sorted tile lists exactly like
   the binary64 blend (binary32 skip decision q <= t, binary64 transmittance and stop), and
   records the contributing Gaussians in order, with alpha-clamp flags.  off has npx + 1
   entries; returns the number of contributions (gid/aclamp written only when cap suffices). */
int64_t or_contrib_lists(const OrCamera *cam, const OrOpts *o, const int64_t *ranges, const uint32_t *vals,
                         const float *rec32, const double *rec64, int64_t *off, int32_t *gid, uint8_t *aclamp,
                         int64_t cap)
{
    enum { F_U, F_V, F_A, F_B, F_C, F_T, REC32 = 16 };
    enum { D_U, D_V, D_A, D_B, D_C, D_ALPHA, REC64 = 16 };
    const int W = cam->width, H = cam->height;
    const int tiles_x = (W + 15) / 16;
    const int64_t npx = (int64_t)W * H;
    int64_t total = 0;
    for (int64_t pix = 0; pix < npx; ++pix) {
        int i = (int)(pix % W), j = (int)(pix / W);
        int tile = (j / 16) * tiles_x + (i / 16);
        float pxf = (float)i + 0.5f, pyf = (float)j + 0.5f;
        double T = 1.0;
        off[pix] = total;
        for (int64_t k = ranges[2 * tile]; k < ranges[2 * tile + 1]; ++k) {
            uint32_t g = vals[k];
            const float *rc = rec32 + REC32 * (int64_t)g;
            float dx = pxf - rc[F_U], dy = pyf - rc[F_V];
            float b2 = rc[F_B] + rc[F_B];
            float By = b2 * dy;
            float Cy = rc[F_C] * dy;
            Cy = Cy * dy;
            float q = fmaf(fmaf(rc[F_A], dx, By), dx, Cy);
            if (!(q <= rc[F_T])) continue;
            const double *r = rec64 + REC64 * (int64_t)g;
            double ddx = (double)pxf - r[D_U], ddy = (double)pyf - r[D_V];
            double qq = r[D_A] * ddx * ddx + 2.0 * r[D_B] * ddx * ddy + r[D_C] * ddy * ddy;
            double a = r[D_ALPHA] * exp(-0.5 * qq);
            int cl = a > (double)o->alpha_max;
            if (cl) a = (double)o->alpha_max;
            double Tn = T * (1.0 - a);
            if (Tn < (double)o->T_min) break;
            if (total < cap) {
                gid[total] = (int32_t)g;
                aclamp[total] = (uint8_t)cl;
            }
            ++total;
            T = Tn;
        }
    }
    off[npx] = total;
    return total;
}
