"""Pins for the CPU oracle: each test ties it to something other than itself -- a value the
paper prints, a closed form, a library routine, an independent construction (Monte-Carlo
projection, minimisation over a rectangle, the SH addition theorem, quadrature) or brute
force on a small input.  CPU only."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2408_07967_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")
TAU32 = float(np.float32(1.0 / 255.0))


def golden():
    vals = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, value = line.split()[:2]
        vals[name] = eval(value, {})  # numbers or simple fractions only
    return vals


def cam_simple(W=64, H=64, f=50.0, cx=None, cy=None, R=None, t=None):
    return synth.Camera(np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32),
                        np.zeros(3, np.float32) if t is None else np.asarray(t, np.float32),
                        f, f, W / 2 if cx is None else cx, H / 2 if cy is None else cy, W, H)


def scene_of(means, scales, quats=None, opac=None, dc=None, activated=True, sh=None):
    means = np.asarray(means, np.float32).reshape(-1, 3)
    P = means.shape[0]
    scales = np.asarray(scales, np.float32).reshape(P, 3)
    quats = np.tile(np.array([1, 0, 0, 0], np.float32), (P, 1)) if quats is None else np.asarray(quats, np.float32)
    opac = np.full(P, 0.5, np.float32) if opac is None else np.asarray(opac, np.float32).reshape(P)
    if sh is None:
        sh = np.zeros((P, 16, 3), np.float32)
        if dc is not None:
            sh[:, 0, :] = np.asarray(dc, np.float32).reshape(P, 3)
    return synth.Scene(means, scales, quats, opac, np.asarray(sh, np.float32), activated)


C0 = 0.5 / math.sqrt(math.pi)


# ------------------------------------------------------------------ own log / exp (library pins)

def test_logf_exhaustive_ratio_domain(oracle_lib):
    # t = 2 ln(alpha0 / tau) is evaluated for alpha0/tau in (1, 255]: every float there
    err, worst = oracle.logf_max_ulp(1.0, 256.0)
    assert err <= 2.0, (err, worst)


def test_logf_wide_range(oracle_lib):
    err, worst = oracle.logf_max_ulp(2.0 ** -20, 2.0 ** -19)
    assert err <= 2.0, (err, worst)
    for x in [1e-30, 1e-3, 0.5, 0.75, 1.0, 1.5, 3.0, 1e10, 3e38]:
        y = oracle.logf(x)
        assert abs(y - math.log(x)) <= 3 * abs(math.log(x)) * 2 ** -24 + 1e-30


def test_expf_range(oracle_lib):
    err, worst = oracle.expf_max_ulp(-80.0, 80.0, 4099)
    assert err <= 2.0, (err, worst)
    err, worst = oracle.expf_max_ulp(-1.0, 1.0, 97)
    assert err <= 2.0, (err, worst)
    assert oracle.expf(0.0) == 1.0
    assert oracle.expf(-100.0) == 0.0 and math.isinf(oracle.expf(100.0))


# ------------------------------------------------------------------ Eq. 3 threshold and the paper's 0.35

def t_full_of(alpha0, cap=False):
    sc = scene_of([[0, 0, 2.0]], [[0.05] * 3], opac=[alpha0])
    valid, rec32, _, _ = oracle.preprocess(sc, cam_simple(), oracle.opts(cap_3sigma=cap), want64=False)
    assert valid[0] == 1
    return float(rec32[0, oracle.F["TFULL"]]), float(rec32[0, oracle.F["T"]])


def test_threshold_matches_eq3_and_paper_crossover(oracle_lib):
    g = golden()
    assert abs(g["tau"] - 1 / 255) < 1e-15
    for a in [0.004, 0.01, 0.1, 0.35, 0.5, 0.9, 1.0]:
        tf, _ = t_full_of(a)
        a32 = float(np.float32(a))
        assert abs(tf - 2.0 * math.log(a32 / TAU32)) < 4e-6 * max(1.0, tf)
    # Eq. 3 radius equals the 3-sigma radius (Eq. 1) where 2 ln(alpha0/tau) = 9:
    cross = math.exp(4.5) / 255.0
    assert abs(cross - g["crossover_alpha0"]) < 0.005          # the paper prints 0.35
    assert t_full_of(g["crossover_alpha0"])[0] < 9.0 < t_full_of(0.36)[0]
    # cap_3sigma applies min(3 sigma, Eq. 3): t never exceeds 9
    assert t_full_of(0.9, cap=True)[1] == 9.0
    assert t_full_of(0.2, cap=True)[1] == t_full_of(0.2, cap=True)[0] < 9.0


def test_cull_near_plane_and_opacity(oracle_lib):
    g = golden()
    cam = cam_simple()
    sc = scene_of([[0, 0, 0.19], [0, 0, 0.21], [0, 0, 2.0], [0, 0, 2.0], [0, 0, -1.0]], [[0.05] * 3] * 5,
                  opac=[0.5, 0.5, g["opacity_cull"], 0.0040, 0.9])
    valid, _, _, _ = oracle.preprocess(sc, cam)
    assert list(valid) == [0, 1, 0, 1, 0]


# ------------------------------------------------------------------ closed forms of the blend

def test_single_gaussian_at_pixel_centre(oracle_lib):
    """A Gaussian whose mean projects onto a pixel sample gives alpha = min(0.99, alpha0) there and
    pixel = alpha * rgb + (1 - alpha) * bg with rgb = max(0, C0 k00 + 1/2) for DC-only SH."""
    cam = cam_simple(cx=31.5, cy=31.5)
    bg = (0.1, 0.2, 0.3)
    dc = np.array([0.3, -0.2, 0.9])
    for a0 in [0.7, 1.0, 0.05]:
        sc = scene_of([[0, 0, 2.0]], [[0.05, 0.03, 0.02]], quats=[[0.9, 0.1, 0.3, -0.2]], opac=[a0], dc=[dc])
        for mode, tol in [(64, 1e-12), (32, 2e-6)]:
            f = oracle.Frame(sc, cam, oracle.opts(bg=bg), mode=mode)
            al = min(float(np.float32(0.99)), float(np.float32(a0)))
            rgb = np.maximum(0.0, C0 * dc.astype(np.float32).astype(np.float64) + 0.5)
            exp = al * rgb + (1 - al) * np.array(bg, np.float32).astype(np.float64)
            assert np.allclose(f.rgb[:, 31, 31], exp, atol=tol, rtol=0), (mode, a0, f.rgb[:, 31, 31], exp)
            assert abs(f.T[31, 31] - (1 - al)) < tol
            assert f.last[31, 31] == 1


def test_early_stop_stack_closed_form(oracle_lib):
    """Five alpha=0.95 layers on one pixel: T goes 1, .05, .0025, 1.25e-4 after three layers and the
    fourth would leave 6.25e-6 < 1e-4, so the walk stops after three contributors (front to back)."""
    cam = cam_simple(cx=31.5, cy=31.5)
    z = np.array([4.0, 2.0, 3.5, 2.5, 3.0])            # shuffled ids: depth decides the order
    dcs = np.array([[0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5], [0.5, 0.5, 0], [0, 0.5, 0.5]])
    sc = scene_of(np.c_[np.zeros(5), np.zeros(5), z], [[0.05] * 3] * 5, opac=[0.95] * 5, dc=dcs)
    f = oracle.Frame(sc, cam, mode=64)
    a = float(np.float32(0.95))
    order = np.argsort(z)
    C, T = np.zeros(3), 1.0
    for k in order[:3]:
        C += (C0 * dcs[k].astype(np.float32).astype(np.float64) + 0.5) * a * T
        T *= 1 - a
    assert np.allclose(f.rgb[:, 31, 31], C, atol=1e-12)
    assert abs(f.T[31, 31] - T) < 1e-15
    assert f.last[31, 31] == 3


def test_equal_depth_ties_broken_by_id(oracle_lib):
    cam = cam_simple(cx=31.5, cy=31.5)
    dcs = np.array([[1.0, -1.0, -1.0], [-1.0, -1.0, 1.0]])
    sc = scene_of([[0, 0, 2.0], [0, 0, 2.0]], [[0.05] * 3] * 2, opac=[0.5, 0.5], dc=dcs)
    f = oracle.Frame(sc, cam, mode=64)
    c = np.maximum(0, C0 * dcs.astype(np.float32).astype(np.float64) + 0.5)
    a = 0.5
    exp = c[0] * a + c[1] * a * (1 - a)
    assert np.allclose(f.rgb[:, 31, 31], exp, atol=1e-12)
    assert list(f.vals) == [0, 1] * (f.N // 2) or np.all(np.diff(f.vals.reshape(-1, 2), axis=1) > 0)


# ------------------------------------------------------------------ EWA projection by Monte Carlo

def rotate_by_quat(q, v):
    """Rotate vectors v [n,3] by unit quaternion q=(w,x,y,z) with v' = v + 2w (u x v) + 2 u x (u x v)."""
    w, u = q[0], q[1:]
    uv = np.cross(u, v)
    return v + 2 * w * uv + 2 * np.cross(u, uv)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ewa_covariance_monte_carlo(oracle_lib, seed):
    """Sigma' - dilation I equals the covariance of projected samples of the 3D Gaussian (to first
    order), and (u, v) the projection of the mean: the Jacobian, the rotation, the scales and the
    world-to-camera transform all enter, each independently of the oracle's matrix code."""
    rng = np.random.default_rng(100 + seed)
    cam = synth.look_at((0.3, -2.5, 1.2), (0.1, 0.2, 0.9), 320, 240, 60.0)
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    s = np.array([0.012, 0.006, 0.002]) * rng.uniform(0.7, 1.3, 3)
    mu = np.array([0.25, 0.1, 0.95])
    sc = scene_of([mu], [s], quats=[q], opac=[0.6])
    valid, rec32, rec64, _ = oracle.preprocess(sc, cam)
    assert valid[0] == 1
    mu32 = sc.means[0].astype(np.float64)
    s32 = sc.scales[0].astype(np.float64)
    q32 = sc.quats[0].astype(np.float64)
    q32 /= np.linalg.norm(q32)
    n = 400_000
    eps = rng.standard_normal((n, 3)) * s32
    X = mu32 + rotate_by_quat(q32, eps)
    R, t = cam.R.astype(np.float64), cam.t.astype(np.float64)
    Xc = X @ R.T + t
    uv = np.c_[cam.fx * Xc[:, 0] / Xc[:, 2] + cam.cx, cam.fy * Xc[:, 1] / Xc[:, 2] + cam.cy]
    emp = np.cov(uv.T)
    D = oracle.D
    model = np.array([[rec64[0, D["S00"]] - 0.3, rec64[0, D["S01"]]], [rec64[0, D["S01"]], rec64[0, D["S11"]] - 0.3]])
    scale = np.sqrt(np.diag(emp))
    rel = np.abs(model - emp) / np.outer(scale, scale)
    assert rel.max() < 0.02, (model, emp)
    pc = R @ mu32 + t
    assert abs(rec64[0, D["U"]] - (cam.fx * pc[0] / pc[2] + cam.cx)) < 1e-9
    assert abs(rec64[0, D["V"]] - (cam.fy * pc[1] / pc[2] + cam.cy)) < 1e-9
    # the binary32 path agrees with the binary64 one to rounding
    F = oracle.F
    for kf, kd in [("U", "U"), ("V", "V"), ("S00", "S00"), ("S01", "S01"), ("S11", "S11"), ("A", "A"), ("B", "B"), ("C", "C")]:
        ref = rec64[0, D[kd]]
        assert abs(rec32[0, F[kf]] - ref) <= 1e-4 * max(1.0, abs(ref)), kf
    # conic is the inverse of Sigma'
    Sg = np.array([[rec64[0, D["S00"]], rec64[0, D["S01"]]], [rec64[0, D["S01"]], rec64[0, D["S11"]]]])
    Q = np.array([[rec64[0, D["A"]], rec64[0, D["B"]]], [rec64[0, D["B"]], rec64[0, D["C"]]]])
    assert np.allclose(Q @ Sg, np.eye(2), atol=1e-12)


def test_fov_clamp_only_beyond_1p3_tan(oracle_lib):
    """Inside the frustum the clamp is inactive (same Sigma' with and without it); far outside it
    bounds the Jacobian's off-axis term."""
    cam = cam_simple(W=64, H=64, f=50.0)
    inside = scene_of([[0.5, 0.2, 2.0]], [[0.05, 0.02, 0.01]], quats=[[0.8, 0.2, 0.5, 0.1]])
    a = oracle.preprocess(inside, cam, oracle.opts(clamp_fov=True))[2]
    b = oracle.preprocess(inside, cam, oracle.opts(clamp_fov=False))[2]
    assert np.array_equal(a[0], b[0])
    outside = scene_of([[10.0, 0.0, 2.0]], [[0.05, 0.05, 0.05]])
    a = oracle.preprocess(outside, cam, oracle.opts(clamp_fov=True))[2]
    b = oracle.preprocess(outside, cam, oracle.opts(clamp_fov=False))[2]
    assert a[0, oracle.D["S00"]] < b[0, oracle.D["S00"]]


def test_fov_clamp_sits_at_1p3_tan_half_fov(oracle_lib):
    """The Jacobian clamp bites exactly beyond x/z = 1.3 tan(half fov) = 1.3 (W/2)/fx (and the
    same for y with H and fy): just inside, Sigma' is that of the unclamped projection; just
    outside, Sigma' no longer depends on how far out the Gaussian is (the off-axis Jacobian term
    is frozen at the bound), while the unclamped Sigma' keeps changing.  The crossing found by
    bisection on that behaviour lands on 1.3 (W/2)/fx."""
    W, H, f = 64, 48, 50.0
    cam = cam_simple(W=W, H=H, f=f)
    z = 2.0
    shape = dict(scales=[[0.05, 0.02, 0.01]], quats=[[0.8, 0.2, 0.5, 0.1]])
    D = oracle.D

    def sig(xz, yz, clamp=True):
        sc = scene_of([[xz * z, yz * z, z]], **shape)
        r = oracle.preprocess(sc, cam, oracle.opts(clamp_fov=clamp))[2][0]
        return np.array([r[D["S00"]], r[D["S01"]], r[D["S11"]]])

    for axis, lim in ((0, 1.3 * (W / 2) / f), (1, 1.3 * (H / 2) / f)):
        def at(k, clamp=True):
            return sig(k, 0.0, clamp) if axis == 0 else sig(0.0, k, clamp)
        for sgn in (1.0, -1.0):
            inside = sgn * lim * (1 - 1e-3)
            assert np.array_equal(at(inside), at(inside, clamp=False))
            out1, out2 = sgn * lim * (1 + 1e-3), sgn * lim * 1.5
            assert np.array_equal(at(out1), at(out2))
            assert not np.array_equal(at(out1, clamp=False), at(out2, clamp=False))
            # bisection on "clamped == unclamped" between 0.5 lim and 1.5 lim
            lo, hi = 0.5 * lim, 1.5 * lim
            ref_out = at(sgn * hi)
            for _ in range(40):
                mid = 0.5 * (lo + hi)
                if np.array_equal(at(sgn * mid), ref_out):
                    hi = mid
                else:
                    lo = mid
            assert abs(hi - lim) <= 1e-6 * lim, (axis, sgn, hi, lim)


# ------------------------------------------------------------------ SH basis

def test_sh_orthonormal_by_quadrature(oracle_lib):
    xg, wg = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for ct, w in zip(xg, wg):
        st = math.sqrt(1 - ct * ct)
        for k in range(nphi):
            ph = 2 * math.pi * k / nphi
            Y = oracle.sh_basis([st * math.cos(ph), st * math.sin(ph), ct])
            G += np.outer(Y, Y) * w * (2 * math.pi / nphi)
    assert np.allclose(G, np.eye(16), atol=1e-12)


def test_sh_addition_theorem(oracle_lib):
    """sum_m Y_lm(d)^2 = (2l+1)/(4 pi) for every unit d and every band l."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        Y = oracle.sh_basis(d)
        for l in range(4):
            band = Y[l * l:(l + 1) * (l + 1)]
            assert abs((band ** 2).sum() - (2 * l + 1) / (4 * math.pi)) < 1e-12


def real_sh_from_complex(d):
    """Real SH of degree <= 3 built from scipy's complex spherical harmonics (which carry the
    Condon-Shortley phase): m > 0 -> sqrt(2) Re Y_l^m, m < 0 -> sqrt(2) Im Y_l^|m|, m = 0 -> Y_l^0,
    at index l^2 + l + m.  This is the sign and order convention of the 3DGS colour model (its
    l = 1 band reads (-y, z, -x) times sqrt(3 / 4 pi)); nothing here comes from the oracle."""
    special = pytest.importorskip("scipy.special")
    x, y, z = d
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x)
    out = np.zeros(16)
    for l in range(4):
        for m in range(-l, l + 1):
            Y = complex(special.sph_harm_y(l, abs(m), theta, phi))
            out[l * l + l + m] = (math.sqrt(2) * Y.real if m > 0 else math.sqrt(2) * Y.imag if m < 0 else Y.real)
    return out


def test_sh_basis_sign_and_order_vs_scipy(oracle_lib):
    """Index by index, the oracle's basis equals the real SH built from scipy's complex ones, at
    random directions and at the axes (where a sign or an index swap within a band shows)."""
    rng = np.random.default_rng(21)
    dirs = [np.array(v, float) for v in ([1, 0, 0], [0, 1, 0], [0, 0, 1], [-1, 0, 0], [0, 0, -1])]
    for _ in range(40):
        d = rng.standard_normal(3)
        dirs.append(d / np.linalg.norm(d))
    for d in dirs:
        ref = real_sh_from_complex(d)
        got = oracle.sh_basis(d)
        assert np.allclose(got, ref, atol=1e-12, rtol=0), (d, got - ref)
    # the l = 1 band of the convention, written out: sqrt(3 / 4 pi) (-y, z, -x)
    d = np.array([0.36, -0.48, 0.8])
    assert np.allclose(real_sh_from_complex(d)[1:4], math.sqrt(3 / (4 * math.pi)) * np.array([0.48, 0.8, -0.36]))


def test_sh_coefficient_layout_in_colour(oracle_lib):
    """The colour of a Gaussian whose only SH coefficient is k_i (channel c of coefficient i at
    sh[:, i, c], the [P,16,3] layout) is max(0, Y_i(d) k_i + 1/2) with Y_i from scipy and d the
    unit vector from the camera centre -- for every i and channel."""
    cam = synth.look_at((0.3, -2.5, 1.2), (0.1, 0.2, 0.9), 64, 64)
    mean = np.array([0.1, 0.1, 0.9])
    d = mean - cam.position()
    Ysc = real_sh_from_complex(d / np.linalg.norm(d))
    for i in range(16):
        for c in range(3):
            sh = np.zeros((1, 16, 3), np.float32)
            sh[0, i, c] = 0.4 - 0.1 * c
            sc = scene_of([mean], [[0.02] * 3], sh=sh)
            valid, rec32, rec64, _ = oracle.preprocess(sc, cam)
            assert valid[0] == 1
            exp = np.full(3, 0.5)
            exp[c] = max(0.0, Ysc[i] * float(sh[0, i, c]) + 0.5)
            assert np.allclose(rec64[0, 6:9], exp, atol=1e-7), (i, c, rec64[0, 6:9], exp)


def test_sh_colour_in_record(oracle_lib):
    """The preprocess colour is max(0, sum_i Y_i(d) k_i + 1/2) with d from the camera centre."""
    rng = np.random.default_rng(3)
    cam = synth.look_at((0.3, -2.5, 1.2), (0.1, 0.2, 0.9), 64, 64)
    sh = rng.normal(0, 0.3, (1, 16, 3)).astype(np.float32)
    sc = scene_of([[0.1, 0.1, 0.9]], [[0.02] * 3], sh=sh)
    valid, rec32, rec64, _ = oracle.preprocess(sc, cam)
    d = sc.means[0].astype(np.float64) - cam.position()
    Y = oracle.sh_basis(d / np.linalg.norm(d))
    exp = np.maximum(0.0, Y @ sh[0].astype(np.float64) + 0.5)
    assert np.allclose(rec64[0, 6:9], exp, atol=1e-6)
    assert np.allclose(rec32[0, 11:14], exp, atol=1e-5)


# ------------------------------------------------------------------ exact tile test (Alg. 3, Eq. 6-9)

def min_q_over_rect(u, v, a, b, c, x0, x1, y0, y1):
    """min over the closed rectangle of a X^2 + 2b X Y + c Y^2 (X = x-u, Y = y-v), by convexity:
    0 if the centre is inside, else the least of the four edge minima (vertex of a 1D parabola,
    clamped to the edge)."""
    if x0 <= u <= x1 and y0 <= v <= y1:
        return 0.0
    best = math.inf
    for ye in (y0, y1):
        Y = ye - v
        X = min(max(-b * Y / a, x0 - u), x1 - u)
        best = min(best, a * X * X + 2 * b * X * Y + c * Y * Y)
    for xe in (x0, x1):
        X = xe - u
        Y = min(max(-b * X / c, y0 - v), y1 - v)
        best = min(best, a * X * X + 2 * b * X * Y + c * Y * Y)
    return best


def test_tile_hit_equals_rectangle_minimisation(oracle_lib):
    rng = np.random.default_rng(11)
    n, mism, near = 20000, 0, 0
    for _ in range(n):
        sx, sy = np.exp(rng.uniform(-1, 4, 2))
        th = rng.uniform(0, math.pi)
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        S = R @ np.diag([sx * sx, sy * sy]) @ R.T + 0.3 * np.eye(2)
        Q = np.linalg.inv(S)
        a, b, c = (float(np.float32(x)) for x in (Q[0, 0], Q[0, 1], Q[1, 1]))
        if a * c - b * b <= 0:
            continue
        t = float(np.float32(rng.uniform(0.0, 11.0)))
        u, v = (float(np.float32(x)) for x in rng.uniform(-60, 76, 2))
        x0, y0 = 16.0 * rng.integers(0, 2), 16.0 * rng.integers(0, 2)
        x1, y1 = x0 + 16.0, y0 + (16.0 if rng.random() < 0.8 else 7.0)
        m = min_q_over_rect(u, v, a, b, c, x0, x1, y0, y1)
        if abs(m - t) <= 1e-4 * max(t, 1e-3):
            near += 1
            continue
        mism += oracle.tile_hit(u, v, a, b, c, t, x0, x1, y0, y1) != (m <= t)
    assert mism == 0
    assert near < n * 0.001


def test_tile_hit_edge_cases(oracle_lib):
    # circle of radius 3 (a=c=1, t=9) about (20, 8) against the tile [0,16]x[0,16]
    hit = lambda u, v: oracle.tile_hit(u, v, 1, 0, 1, 9, 0, 16, 0, 16)
    assert hit(8, 8)              # centre inside
    assert hit(18.5, 8)           # chord of the right edge inside the edge
    assert hit(19.0, 8)           # tangent
    assert not hit(19.01, 8)      # just outside
    assert hit(8, -3.0)           # tangent to the top edge from above
    assert not hit(8, -3.01)
    assert not hit(-2.5, -2.5)    # corner at distance sqrt(12.5) > 3


def test_tile_hit_corner(oracle_lib):
    # a circle whose centre is diagonal to the corner hits only if the corner is within the radius
    assert oracle.tile_hit(-2.0, -2.0, 1, 0, 1, 9, 0, 16, 0, 16)         # 8 <= 9
    assert not oracle.tile_hit(-2.2, -2.2, 1, 0, 1, 9, 0, 16, 0, 16)     # 9.68 > 9
    # a long thin ellipse passing diagonally across the tile without containing its centre
    th = math.pi / 4
    R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
    Q = np.linalg.inv(R @ np.diag([400.0, 0.25]) @ R.T)
    assert oracle.tile_hit(-10.0, -10.0, Q[0, 0], Q[0, 1], Q[1, 1], 9.0, 0, 16, 0, 16)
    assert not oracle.tile_hit(-10.0, 10.0, Q[0, 0], Q[0, 1], Q[1, 1], 9.0, 16, 32, 0, 16)


# ------------------------------------------------------------------ pairs, sort, ranges

def test_sort_and_ranges_match_numpy(oracle_lib):
    sc, cam = synth.random_small_scene(400, 3, 100, 76, log_scale_mu=-2.5)
    f = oracle.Frame(sc, cam, mode=32)
    order = np.lexsort((f.vals_unsorted, f.keys_unsorted))
    assert np.array_equal(f.keys, f.keys_unsorted[order])
    assert np.array_equal(f.vals, f.vals_unsorted[order])
    tiles = np.arange(f.ranges.shape[0], dtype=np.uint64)
    hi = (f.keys >> np.uint64(32))
    st = np.searchsorted(hi, tiles, side="left")
    en = np.searchsorted(hi, tiles, side="right")
    nz = en > st
    assert np.array_equal(f.ranges[nz, 0], st[nz]) and np.array_equal(f.ranges[nz, 1], en[nz])
    assert np.all(f.ranges[~nz] == 0)
    # emission order: Gaussian id, then tiles row-major
    assert np.all(np.diff(f.vals_unsorted.astype(np.int64)) >= 0)
    same = np.diff(f.vals_unsorted.astype(np.int64)) == 0
    assert np.all(np.diff((f.keys_unsorted >> np.uint64(32)).astype(np.int64))[same] > 0)
    # key low word is the depth bits of the Gaussian
    zb = f.rec32[f.vals_unsorted, oracle.F["Z"]].view(np.uint32)
    assert np.array_equal((f.keys_unsorted & np.uint64(0xffffffff)).astype(np.uint32), zb)


# ------------------------------------------------------------------ brute force == tiled (bitwise)

@pytest.mark.parametrize("mode", [32, 64])
def test_bruteforce_equals_tiled_tiny_crop(oracle_lib, mode):
    sc, cams = synth.load_config("tiny")
    cam = cams[0]
    f = oracle.Frame(sc, cam, mode=mode)
    crop = (96, 100, 48, 40)
    rgb, T = oracle.blend_brute(mode, cam, f.valid, f.rec32, f.rec64, crop=crop)
    x0, y0, w, h = crop
    assert np.array_equal(rgb, f.rgb[:, y0:y0 + h, x0:x0 + w])
    assert np.array_equal(T, f.T[y0:y0 + h, x0:x0 + w])


@pytest.mark.parametrize("cap", [False, True])
def test_bruteforce_equals_tiled_large_gaussians(oracle_lib, cap):
    sc, cam = synth.random_small_scene(300, 5, 100, 76, log_scale_mu=-2.0, log_scale_sigma=1.0)
    o = oracle.opts(cap_3sigma=cap, bg=(0.2, 0.1, 0.05))
    for mode in (32, 64):
        f = oracle.Frame(sc, cam, o, mode=mode)
        rgb, T = oracle.blend_brute(mode, cam, f.valid, f.rec32, f.rec64, o)
        assert np.array_equal(rgb, f.rgb) and np.array_equal(T, f.T)
        assert np.all(f.T <= 1.0) and np.all(f.T >= 1e-4 * (1 - 1e-6))
        lastzero = f.last == 0
        assert np.all(f.T[lastzero] == 1.0)
        assert f.evals >= int(f.last.sum())


def test_transmittance_non_increasing_along_the_depth_order(oracle_lib):
    """Invariant: a pixel's transmittance never rises as the list grows -- rendering only the k
    nearest Gaussians (a prefix of every pixel's front-to-back list) gives T_k >= T_k' for k < k'
    (each further entry multiplies T by 1 - alpha in [0.01, 1], is skipped, or meets the stop)."""
    sc, cam = synth.random_small_scene(400, 23, 64, 48, log_scale_mu=-2.2, log_scale_sigma=0.8)
    f = oracle.Frame(sc, cam, mode=64)
    order = oracle.depth_order(f.valid, f.rec32)
    prev = None
    for k in (0, 1, 5, 20, 80, 200, len(order)):
        valid = np.zeros_like(f.valid)
        valid[order[:k]] = f.valid[order[:k]]
        rgb, T = oracle.blend_brute(64, cam, valid, f.rec32, f.rec64)
        if k == 0:
            assert np.all(T == 1.0)
        else:
            assert np.all(T <= prev)
        assert np.all(T >= 1e-4 * (1 - 1e-12)) and np.all(rgb >= 0.0)
        prev = T
    assert np.array_equal(prev, f.T)     # the whole list is the tiled frame


def test_pairs_cover_every_alpha_above_tau(oracle_lib):
    """Invariant: every (pixel, Gaussian) with alpha0 exp(-q/2) >= tau in binary64 has its tile in
    the Gaussian's pair set (Section 4.1: only false positives are removed)."""
    sc, cam = synth.random_small_scene(250, 9, 100, 76, log_scale_mu=-2.2, log_scale_sigma=1.0)
    f = oracle.Frame(sc, cam, mode=64)
    D = oracle.D
    W, H = cam.width, cam.height
    tx_n = (W + 15) // 16
    px = np.arange(W) + 0.5
    py = np.arange(H) + 0.5
    tiles_of_px = (np.arange(H)[:, None] // 16) * tx_n + (np.arange(W)[None, :] // 16)
    paired = {}
    for k, v in zip((f.keys_unsorted >> np.uint64(32)).astype(np.int64), f.vals_unsorted):
        paired.setdefault(int(v), set()).add(int(k))
    checked = 0
    for g in np.nonzero(f.valid)[0]:
        r = f.rec64[g]
        dx = px[None, :] - r[D["U"]]
        dy = py[:, None] - r[D["V"]]
        q = r[D["A"]] * dx * dx + 2 * r[D["B"]] * dx * dy + r[D["C"]] * dy * dy
        al = r[D["ALPHA"]] * np.exp(-0.5 * q)
        need = set(np.unique(tiles_of_px[al >= TAU32 * (1 + 1e-5)]).tolist())
        assert need <= paired.get(int(g), set()), g
        checked += len(need)
    assert checked > 100


def test_exact_pairs_subset_of_3dgs_aabb(oracle_lib):
    """With the paper's min(3 sigma, Eq. 3) rule the exact pairs are a subset of the 3DGS pairs
    (square of side 2 ceil(3 sqrt(lambda_max)) about the mean, Eq. 1 and Alg. 2), and fewer."""
    sc, cam = synth.random_small_scene(400, 12, 160, 128, log_scale_mu=-2.3, log_scale_sigma=0.9)
    f = oracle.Frame(sc, cam, oracle.opts(cap_3sigma=True), mode=64)
    D = oracle.D
    tx_n, ty_n = oracle.tiles_of(cam)
    total_aabb = 0
    for g in np.nonzero(f.valid)[0]:
        r = f.rec64[g]
        mid = 0.5 * (r[D["S00"]] + r[D["S11"]])
        lam = mid + math.sqrt(max(0.1, mid * mid - (r[D["S00"]] * r[D["S11"]] - r[D["S01"]] ** 2)))
        rad = math.ceil(3.0 * math.sqrt(lam))
        xs = [tx for tx in range(tx_n) if 16 * tx <= r[D["U"]] + rad + 1e-3 and 16 * tx + 16 >= r[D["U"]] - rad - 1e-3]
        ys = [ty for ty in range(ty_n) if 16 * ty <= r[D["V"]] + rad + 1e-3 and 16 * ty + 16 >= r[D["V"]] - rad - 1e-3]
        aabb = {ty * tx_n + tx for ty in ys for tx in xs}
        total_aabb += len(aabb)
        mine = set((f.keys_unsorted[f.vals_unsorted == g] >> np.uint64(32)).astype(np.int64).tolist())
        assert mine <= aabb, g
    assert f.N < total_aabb


def last_gaussian(fr, cam):
    """Gaussian id of each pixel's last contributor (-1 for none) from the list positions."""
    tx_n, _ = oracle.tiles_of(cam)
    ty = np.arange(cam.height)[:, None] // 16
    tx = np.arange(cam.width)[None, :] // 16
    start = fr.ranges[ty * tx_n + tx, 0]
    last = fr.last.astype(np.int64)
    idx = np.where(last > 0, start + last - 1, 0)
    return np.where(last > 0, fr.vals[idx].astype(np.int64), -1)


def test_aabb_mode_is_the_3sigma_square_closed_form(oracle_lib):
    """3DGS pairs (Eq. 1; Alg. 1 radii = ceil(3 sqrt(max eigenvalue)); Alg. 2): an isotropic
    Gaussian of scale s at depth z has Sigma' = ((f s / z)^2 + 0.3) I at the image centre, so
    r = ceil(3 sqrt((f s / z)^2 + 0.3)) and the pairs are every tile of [u - r, u + r]^2 --
    counted here from the closed form alone (offsets small enough that the Jacobian's x/z term
    changes no radius)."""
    W = H = 256
    f, z = 100.0, 4.0
    for s_ in (0.05, 0.13, 0.31, 0.62):
        for du in (0.0, 5.3, -9.7):
            cam = cam_simple(W, H, f=f)
            sc = scene_of([[du * z / f, 0.0, z]], [[s_, s_, s_]], opac=[0.9])
            fr = oracle.Frame(sc, cam, oracle.opts(intersect=1), mode=32)
            sig2 = (f * s_ / z) ** 2 + 0.3
            r = math.ceil(3.0 * math.sqrt(sig2))
            u, v = W / 2 + du, H / 2
            tx = range(max(0, math.floor((u - r) / 16)), min(W // 16 - 1, math.floor((u + r) / 16)) + 1)
            ty = range(max(0, math.floor((v - r) / 16)), min(H // 16 - 1, math.floor((v + r) / 16)) + 1)
            expect = sorted(y * (W // 16) + x for y in ty for x in tx)
            got = sorted((fr.keys >> np.uint64(32)).astype(np.int64).tolist())
            assert got == expect, (s_, du, r)


def test_aabb_mode_superset_same_image_under_3sigma_cap(oracle_lib):
    """Under the paper's min(3 sigma, Eq. 3) rule every contribution (q <= t <= 9) lies in the
    3-sigma ellipse, which the 3DGS square contains: the exact pairs are a subset of the square's,
    fewer, and the image is the same bit for bit (both precisions).  Brute force: every pixel with
    q <= 9 of a Gaussian falls in one of its square's tiles."""
    sc, cam = synth.random_small_scene(500, 31, 176, 144, log_scale_mu=-2.3, log_scale_sigma=0.9)
    for mode in (32, 64):
        fe = oracle.Frame(sc, cam, oracle.opts(cap_3sigma=True), mode=mode)
        fa = oracle.Frame(sc, cam, oracle.opts(cap_3sigma=True, intersect=1), mode=mode)
        assert fe.N < fa.N
        assert np.array_equal(fe.rgb, fa.rgb) and np.array_equal(fe.T, fa.T)
        # `last` is a position in the tile's list: compare the Gaussians it names
        assert np.array_equal(last_gaussian(fe, cam), last_gaussian(fa, cam))
    tx_n, _ = oracle.tiles_of(cam)
    pe = {}
    for k, v in zip(fe.keys_unsorted >> np.uint64(32), fe.vals_unsorted):
        pe.setdefault(int(v), set()).add(int(k))
    pa = {}
    for k, v in zip(fa.keys_unsorted >> np.uint64(32), fa.vals_unsorted):
        pa.setdefault(int(v), set()).add(int(k))
    for g, tiles in pe.items():
        assert tiles <= pa.get(g, set()), g
    D = oracle.D
    px = np.arange(cam.width) + 0.5
    py = np.arange(cam.height) + 0.5
    tiles_of_px = (py[:, None] // 16).astype(int) * tx_n + (px[None, :] // 16).astype(int)
    checked = 0
    for g in list(pa)[:150]:
        r = fa.rec64[g]
        dx = px[None, :] - r[D["U"]]
        dy = py[:, None] - r[D["V"]]
        q = r[D["A"]] * dx * dx + 2 * r[D["B"]] * dx * dy + r[D["C"]] * dy * dy
        inside = set(np.unique(tiles_of_px[q <= 9.0 * (1 - 1e-4)]).tolist())
        assert inside <= pa[g], g
        checked += len(inside)
    assert checked > 100


# ------------------------------------------------------------------ activation

def test_raw_parameters_activate_with_own_exp(oracle_lib):
    rng = np.random.default_rng(5)
    ls = rng.normal(-3, 1, 2000).astype(np.float32)
    own = np.array([oracle.expf(x) for x in ls], np.float32)
    ref = np.exp(ls.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(own - ref) / ulp) <= 2.0
    raw, cam = synth.random_small_scene(200, 21, 64, 48, activated=False)
    act = raw.subset(slice(None))
    act.activated = True
    act.scales = np.vectorize(oracle.expf, otypes=[np.float32])(raw.scales)
    e = np.vectorize(oracle.expf, otypes=[np.float32])(-raw.opacity)
    act.opacity = (np.float32(1.0) / (np.float32(1.0) + e)).astype(np.float32)
    a = oracle.preprocess(raw, cam, want64=False)
    b = oracle.preprocess(act, cam, want64=False)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and np.array_equal(a[3], b[3])


def test_tiny_frame_statistics(oracle_lib):
    sc, cams = synth.load_config("tiny")
    f = oracle.Frame(sc, cams[0], mode=64)
    assert f.N > f.visible > 0
    assert 0.0 < f.T.mean() < 1.0
    assert np.all(f.rgb >= 0)
