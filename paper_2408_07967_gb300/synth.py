"""Seeded synthetic scenes and cameras for the 3DGS forward rasterizer.

This module only *draws inputs*: Gaussian parameters and pinhole cameras shaped
like the paper's workloads (room-scale indoor scenes of Tanks&Temples /
DeepBlending size up to city-scale aerial scenes of MatrixCity / Mill19 size,
FlashGS Section 6.1.2).  The paper's trained models and datasets are not
available, so these seeded stand-ins replace them.  Nothing here performs any
step of the rasterizer itself: it holds no projection, covariance, SH,
intersection, sort or blending arithmetic, so both the CPU oracle and the CUDA
path can be fed from it.

Conventions shared by every scene:
  * world space is right-handed with +z up (the tiny scene is axis-aligned);
  * a camera is (R, t, fx, fy, cx, cy, width, height): x_cam = R @ x_world + t,
    camera looks down +z_cam, x_cam right, y_cam down, pixel (i, j) covers
    [i, i+1) x [j, j+1) (pixel-area coordinates);
  * Gaussian arrays are float32, canonical AoS: means [P,3], scales or
    log-scales [P,3], quaternions [P,4] as (w, x, y, z), opacities or logits
    [P], SH coefficients [P,16,3] (coefficient-major, RGB-minor).

Activated scenes carry scale = exp(log_scale) and opacity = sigmoid(logit),
computed here in float64 and rounded once to float32, so both sides of every
parity test read identical bits.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SH_COEFFS = 16


@dataclasses.dataclass
class Camera:
    R: np.ndarray          # [3,3] float32, world -> camera rotation (row-major)
    t: np.ndarray          # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2

    def position(self) -> np.ndarray:
        """Camera centre in world space (float64)."""
        R = self.R.astype(np.float64)
        return -R.T @ self.t.astype(np.float64)


@dataclasses.dataclass
class Scene:
    means: np.ndarray      # [P,3] f32
    scales: np.ndarray     # [P,3] f32 (activated) or log-scales when activated=False
    quats: np.ndarray      # [P,4] f32 (w,x,y,z), not necessarily unit length
    opacity: np.ndarray    # [P] f32 (activated) or logits when activated=False
    sh: np.ndarray         # [P,16,3] f32
    activated: bool = True
    name: str = ""

    @property
    def P(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(self.means[idx].copy(), self.scales[idx].copy(), self.quats[idx].copy(),
                     self.opacity[idx].copy(), self.sh[idx].copy(), self.activated, self.name)


def _sigmoid64(x):
    return 1.0 / (1.0 + np.exp(-x))


def _finish(rng, means, log_scales, logit_sigma, name, activated=True, dc_sigma=0.5, hi_sigma=0.05):
    P = means.shape[0]
    q = rng.standard_normal((P, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logits = rng.normal(0.0, logit_sigma, P)
    sh = np.empty((P, SH_COEFFS, 3), dtype=np.float64)
    sh[:, 0, :] = rng.normal(0.0, dc_sigma, (P, 3))
    sh[:, 1:, :] = rng.normal(0.0, hi_sigma, (P, SH_COEFFS - 1, 3))
    if activated:
        scales = np.exp(log_scales)
        opac = _sigmoid64(logits)
    else:
        scales = log_scales
        opac = logits
    return Scene(means.astype(np.float32), scales.astype(np.float32), q.astype(np.float32),
                 opac.astype(np.float32), sh.astype(np.float32), activated, name)


# ----------------------------------------------------------------------------------- cameras

def _look(C, forward, right, width, height, hfov_deg):
    """Camera at world point C with unit forward / right vectors (down = forward x right)."""
    f = np.asarray(forward, np.float64)
    f = f / np.linalg.norm(f)
    r = np.asarray(right, np.float64)
    r = r - f * (r @ f)
    r = r / np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f])
    t = -R @ np.asarray(C, np.float64)
    fx = 0.5 * width / math.tan(math.radians(hfov_deg) * 0.5)
    return Camera(R.astype(np.float32), t.astype(np.float32), float(np.float32(fx)), float(np.float32(fx)),
                  0.5 * width, 0.5 * height, int(width), int(height))


def look_at(C, target, width, height, hfov_deg=60.0, up=(0.0, 0.0, 1.0)):
    C = np.asarray(C, np.float64)
    f = np.asarray(target, np.float64) - C
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:
        r = np.array([1.0, 0.0, 0.0])
    return _look(C, f, r, width, height, hfov_deg)


def yaw_pitch_camera(C, yaw, pitch_down, width, height, hfov_deg=60.0):
    """Camera whose forward has heading `yaw` and is pitched `pitch_down` radians below horizontal."""
    cp, sp = math.cos(pitch_down), math.sin(pitch_down)
    cy, sy = math.cos(yaw), math.sin(yaw)
    f = np.array([cp * cy, cp * sy, -sp])
    r = np.array([sy, -cy, 0.0])
    return _look(C, f, r, width, height, hfov_deg)


def tiny_camera(width=256, height=256, hfov_deg=60.0):
    """Camera at (0,0,-3) looking at the origin along +z with y down (axis-aligned)."""
    return _look((0.0, 0.0, -3.0), (0.0, 0.0, 1.0), (1.0, 0.0, 0.0), width, height, hfov_deg)


# ----------------------------------------------------------------------------------- scenes

def tiny_scene(P=10_000, seed=0, activated=True):
    """10k Gaussians, means U[-1,1]^3, log-scales N(-4,0.5), opacity sigmoid(N(0,1.5))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-1.0, 1.0, (P, 3))
    log_scales = rng.normal(-4.0, 0.5, (P, 3))
    return _finish(rng, means, log_scales, 1.5, "tiny", activated)


ROOM_LO = np.array([-5.0, -5.0, 0.0])
ROOM_HI = np.array([5.0, 5.0, 3.0])


def room_scene(P=1_000_000, seed=1, patches=200, activated=True):
    """Gaussians on random planar patches inside a 10 x 10 x 3 m room (z up).

    Each patch: centre uniform in the room box, normal uniform on the sphere,
    square side U[0.5, 3] m; points uniform on the square plus N(0, 0.01) along
    the normal.  Log-scales N(-5, 0.7) per axis, opacity sigmoid(N(0, 2)).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    centres = rng.uniform(ROOM_LO, ROOM_HI, (patches, 3))
    normals = rng.standard_normal((patches, 3))
    normals /= np.linalg.norm(normals, axis=1, keepdims=True)
    sides = rng.uniform(0.5, 3.0, patches)
    helper = np.where(np.abs(normals[:, :1]) < 0.9, np.array([[1.0, 0.0, 0.0]]), np.array([[0.0, 1.0, 0.0]]))
    e1 = np.cross(normals, helper)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(normals, e1)
    pid = rng.integers(0, patches, P)
    uv = rng.uniform(-0.5, 0.5, (P, 2)) * sides[pid, None]
    jitter = rng.normal(0.0, 0.01, P)
    means = centres[pid] + uv[:, :1] * e1[pid] + uv[:, 1:] * e2[pid] + jitter[:, None] * normals[pid]
    log_scales = rng.normal(-5.0, 0.7, (P, 3))
    return _finish(rng, means, log_scales, 2.0, "room", activated)


def room_cameras(n=32, width=1920, height=1080, hfov_deg=60.0):
    """n cameras evenly spaced on a circle of radius 2.5 m at height 1.6 m, looking through (0,0,1.5)."""
    cams = []
    for k in range(n):
        a = 2.0 * math.pi * k / n
        C = (2.5 * math.cos(a), 2.5 * math.sin(a), 1.6)
        # look through the room centre: the target is on the far side of the axis
        cams.append(look_at(C, (0.0, 0.0, 1.5), width, height, hfov_deg))
    return cams


CITY_HALF = 1000.0
CITY_TOP = 100.0


def city_scene(P=10_000_000, seed=2, buildings=400, activated=True):
    """City-scale scene over a 2000 x 2000 x 100 m box (z up).

    80% of the Gaussians lie on planes (half on the ground z=0, half on the
    facades of axis-aligned buildings with footprint U[20,80]^2 m and height
    U[10,100] m), 20% float uniformly in the box.  Log-scales N(-1, 1.2);
    1% of the Gaussians are very large: scale U[20, 60] m on every axis.
    Opacity sigmoid(N(0, 2)).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_plane = int(0.8 * P)
    n_ground = n_plane // 2
    n_facade = n_plane - n_ground
    n_free = P - n_plane
    means = np.empty((P, 3), np.float64)
    # ground
    means[:n_ground, :2] = rng.uniform(-CITY_HALF, CITY_HALF, (n_ground, 2))
    means[:n_ground, 2] = 0.0
    # facades
    bc = rng.uniform(-CITY_HALF + 40.0, CITY_HALF - 40.0, (buildings, 2))
    bsz = rng.uniform(20.0, 80.0, (buildings, 2))
    bh = rng.uniform(10.0, 100.0, buildings)
    b = rng.integers(0, buildings, n_facade)
    face = rng.integers(0, 4, n_facade)
    s = rng.uniform(-0.5, 0.5, n_facade)
    h = rng.uniform(0.0, 1.0, n_facade) * bh[b]
    half = 0.5 * bsz[b]
    fx_ = np.where(face < 2, np.where(face == 0, -1.0, 1.0) * half[:, 0], s * 2.0 * half[:, 0])
    fy_ = np.where(face < 2, s * 2.0 * half[:, 1], np.where(face == 2, -1.0, 1.0) * half[:, 1])
    sl = slice(n_ground, n_ground + n_facade)
    means[sl, 0] = bc[b, 0] + fx_
    means[sl, 1] = bc[b, 1] + fy_
    means[sl, 2] = h
    # free-floating
    means[n_plane:, :2] = rng.uniform(-CITY_HALF, CITY_HALF, (n_free, 2))
    means[n_plane:, 2] = rng.uniform(0.0, CITY_TOP, n_free)
    log_scales = rng.normal(-1.0, 1.2, (P, 3))
    big = rng.random(P) < 0.01
    log_scales[big] = np.log(rng.uniform(20.0, 60.0, (int(big.sum()), 1)))
    return _finish(rng, means, log_scales, 2.0, "city", activated)


def city_cameras(n_aerial=16, n_street=16, width=3840, height=2160, hfov_deg=60.0, seed=2):
    """16 aerial cameras (altitude U[300,600] m, pitch U[45,90] deg down, random yaw) and
    16 street cameras (2 m high, horizontal, random yaw), positions uniform over the city."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    cams = []
    for _ in range(n_aerial):
        xy = rng.uniform(-0.8 * CITY_HALF, 0.8 * CITY_HALF, 2)
        alt = rng.uniform(300.0, 600.0)
        pitch = math.radians(rng.uniform(45.0, 89.0))
        yaw = rng.uniform(0.0, 2.0 * math.pi)
        cams.append(yaw_pitch_camera((xy[0], xy[1], alt), yaw, pitch, width, height, hfov_deg))
    for _ in range(n_street):
        xy = rng.uniform(-0.9 * CITY_HALF, 0.9 * CITY_HALF, 2)
        yaw = rng.uniform(0.0, 2.0 * math.pi)
        cams.append(yaw_pitch_camera((xy[0], xy[1], 2.0), yaw, 0.0, width, height, hfov_deg))
    return cams


def rescaled(cam: Camera, width: int, height: int, hfov_deg: float = 60.0) -> Camera:
    """The same pose with a pinhole of another resolution and the given horizontal FOV."""
    fx = 0.5 * width / math.tan(math.radians(hfov_deg) * 0.5)
    return Camera(cam.R.copy(), cam.t.copy(), float(np.float32(fx)), float(np.float32(fx)), 0.5 * width, 0.5 * height,
                  int(width), int(height), cam.near)


def poisson_requests(n, rate, seed=3, resolutions=((1280, 720), (1920, 1080), (3840, 2160)), n_scenes=2):
    """Open-loop arrival schedule: exponential inter-arrival times at `rate` per second, each
    request a uniformly drawn scene index, camera index (0..31) and resolution."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    scene = rng.integers(0, n_scenes, n)
    cam = rng.integers(0, 32, n)
    res = rng.integers(0, len(resolutions), n)
    return [(float(t[i]), int(scene[i]), int(cam[i]), resolutions[int(res[i])]) for i in range(n)]


def perturbed(scene: Scene, seed=4, mean_sigma=0.01, dc_sigma=0.05, logit_sigma=0.2) -> Scene:
    """Target scene for the differentiable workload: means += N(0,0.01), DC += N(0,0.05),
    logits += N(0,0.2).  `scene` must hold raw (log-scale / logit) parameters."""
    assert not scene.activated
    rng = np.random.Generator(np.random.PCG64(seed))
    s = scene.subset(slice(None))
    s.means = (scene.means + rng.normal(0, mean_sigma, scene.means.shape)).astype(np.float32)
    sh = scene.sh.copy()
    sh[:, 0, :] += rng.normal(0, dc_sigma, (scene.P, 3)).astype(np.float32)
    s.sh = sh
    s.opacity = (scene.opacity + rng.normal(0, logit_sigma, scene.P)).astype(np.float32)
    return s


def grad_subset(P=2000, seed=5, size=64):
    """Small raw-parameter scene for gradient checks: Gaussians drawn like the room
    scene but re-centred in front of a size x size camera at the origin."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = np.empty((P, 3))
    means[:, :2] = rng.uniform(-0.45, 0.45, (P, 2)) * 2.0
    means[:, 2] = rng.uniform(2.5, 3.5, P)
    log_scales = rng.normal(-3.2, 0.4, (P, 3))
    scene = _finish(rng, means, log_scales, 2.0, "grad", activated=False)
    cam = _look((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), (1.0, 0.0, 0.0), size, size, 60.0)
    return scene, cam


def random_small_scene(P, seed, width, height, activated=True, log_scale_mu=-3.0, log_scale_sigma=0.8,
                       logit_sigma=1.5, depth=(1.5, 4.0)):
    """Generic seeded scene in front of an axis-aligned camera at the origin (for parity sweeps)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = np.empty((P, 3))
    means[:, 2] = rng.uniform(depth[0], depth[1], P)
    ext = rng.uniform(-0.8, 0.8, (P, 2)) * means[:, 2:3] * 0.6
    means[:, 0] = ext[:, 0] * (width / max(width, height))
    means[:, 1] = ext[:, 1] * (height / max(width, height))
    log_scales = rng.normal(log_scale_mu, log_scale_sigma, (P, 3))
    scene = _finish(rng, means, log_scales, logit_sigma, "small", activated)
    cam = _look((0.0, 0.0, 0.0), (0.0, 0.0, 1.0), (1.0, 0.0, 0.0), width, height, 60.0)
    return scene, cam


CONFIGS = {
    "tiny": "10k Gaussians, 256x256, one camera (seed 0)",
    "room": "1M Gaussians on 200 planar patches, 32 cameras at 1920x1080 (seed 1)",
    "city": "10M Gaussians over a 2 km city box, 16 aerial + 16 street cameras at 3840x2160 (seed 2)",
}


def load_config(name, P=None):
    """(scene, cameras) for one of the named workloads."""
    if name == "tiny":
        return tiny_scene(P or 10_000), [tiny_camera()]
    if name == "room":
        return room_scene(P or 1_000_000), room_cameras()
    if name == "city":
        return city_scene(P or 10_000_000), city_cameras()
    raise KeyError(name)
