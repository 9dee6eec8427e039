"""CPU oracle for the FlashGS forward rasterizer -- TEST INFRASTRUCTURE ONLY.

Plain C (``gs_oracle.c``, binary64 image reference with binary32 decisions)
loaded through ctypes.  Only the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the product
library never does, and this package imports nothing from the product.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_SRC_GRAD = os.path.join(_HERE, "gs_oracle_grad.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
          "-fno-associative-math", "-Wall", "-Wno-unused-function"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no contraction: binary32 decisions must be reproducible)."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_GRAD))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, _SRC_GRAD, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_z", C.c_float)]


class OrOpts(C.Structure):
    _fields_ = [("bg", C.c_float * 3), ("tau", C.c_float), ("alpha_max", C.c_float), ("T_min", C.c_float),
                ("dilation", C.c_float), ("cap_3sigma", C.c_int32), ("clamp_fov", C.c_int32),
                ("intersect", C.c_int32)]


REC32 = 16
REC64 = 16
F = dict(U=0, V=1, A=2, B=3, C=4, T=5, Z=6, S00=7, S01=8, S11=9, ALPHA=10, R=11, G=12, BL=13, TFULL=14)
D = dict(U=0, V=1, A=2, B=3, C=4, ALPHA=5, R=6, G=7, BL=8, S00=9, S01=10, S11=11, Z=12)

_fp = C.POINTER(C.c_float)
_dp = C.POINTER(C.c_double)
_i64 = C.c_int64


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.or_logf.restype = C.c_float
            L.or_logf.argtypes = [C.c_float]
            L.or_expf.restype = C.c_float
            L.or_expf.argtypes = [C.c_float]
            L.or_logf_max_ulp.restype = C.c_double
            L.or_logf_max_ulp.argtypes = [C.c_float, C.c_float, _fp]
            L.or_expf_max_ulp.restype = C.c_double
            L.or_expf_max_ulp.argtypes = [C.c_float, C.c_float, C.c_int32, _fp]
            L.or_eval_decision_math.restype = None
            L.or_eval_decision_math.argtypes = [C.c_int32, _i64, C.c_void_p, C.c_float, C.c_void_p]
            L.or_sh_basis.restype = None
            L.or_sh_basis.argtypes = [_dp, _dp]
            L.or_tile_hit.restype = C.c_int
            L.or_tile_hit.argtypes = [C.c_float] * 10
            L.or_preprocess.restype = _i64
            L.or_preprocess.argtypes = [_i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_int32, C.c_int32, C.POINTER(OrCamera), C.POINTER(OrOpts),
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_emit_pairs.restype = _i64
            L.or_emit_pairs.argtypes = [_i64, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(OrCamera),
                                        C.c_void_p, C.c_void_p, C.c_void_p, _i64]
            L.or_sort_pairs.restype = None
            L.or_sort_pairs.argtypes = [_i64, C.c_void_p, C.c_void_p]
            L.or_tile_ranges.restype = None
            L.or_tile_ranges.argtypes = [_i64, C.c_void_p, C.c_int32, C.c_void_p]
            L.or_blend_tiled.restype = _i64
            L.or_blend_tiled.argtypes = [C.c_int32, C.POINTER(OrCamera), C.POINTER(OrOpts), C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p]
            L.or_blend_brute.restype = None
            L.or_blend_brute.argtypes = [C.c_int32, C.POINTER(OrCamera), C.POINTER(OrOpts), _i64, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                         C.c_void_p, C.c_void_p]
            L.or_render.restype = _i64
            L.or_render.argtypes = [C.c_int32, _i64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_int32, C.c_int32, C.POINTER(OrCamera), C.POINTER(OrOpts),
                                    C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, _i64,
                                    C.c_void_p]
            _vp = C.c_void_p
            L.or_grad_flags.restype = None
            L.or_grad_flags.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(OrCamera),
                                        C.POINTER(OrOpts), _vp, _vp]
            L.or_forward_fixed.restype = None
            L.or_forward_fixed.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(OrCamera),
                                           C.POINTER(OrOpts), _vp, _vp, _vp, _vp, _vp, _vp, _vp]
            L.or_backward_fixed.restype = None
            L.or_backward_fixed.argtypes = [_i64, _vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.POINTER(OrCamera),
                                            C.POINTER(OrOpts), _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                            _vp, _vp]
            L.or_contrib_lists.restype = _i64
            L.or_contrib_lists.argtypes = [C.POINTER(OrCamera), C.POINTER(OrOpts), _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                           _i64]
            L.or_set_threads.restype = None
            L.or_set_threads.argtypes = [C.c_int]
            L.or_get_threads.restype = C.c_int
            L.or_get_threads.argtypes = []
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def camera(cam) -> OrCamera:
    c = OrCamera()
    for i, x in enumerate(np.asarray(cam.R, np.float32).reshape(9)):
        c.R[i] = float(x)
    for i, x in enumerate(np.asarray(cam.t, np.float32).reshape(3)):
        c.t[i] = float(x)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_z = float(getattr(cam, "near", 0.2))
    return c


def opts(bg=(0.0, 0.0, 0.0), tau=1.0 / 255.0, alpha_max=0.99, T_min=1e-4, dilation=0.3, cap_3sigma=False,
         clamp_fov=True, intersect=0) -> OrOpts:
    """intersect 0: exact tile pairs (Alg. 3); 1: every tile of the 3DGS 3-sigma square (Eq. 1, Alg. 2)."""
    o = OrOpts()
    for i in range(3):
        o.bg[i] = float(bg[i])
    o.tau, o.alpha_max, o.T_min, o.dilation = float(tau), float(alpha_max), float(T_min), float(dilation)
    o.cap_3sigma, o.clamp_fov, o.intersect = int(bool(cap_3sigma)), int(bool(clamp_fov)), int(intersect)
    return o


def set_threads(n: int):
    lib().or_set_threads(int(n))


def get_threads() -> int:
    return int(lib().or_get_threads())


def logf(x: float) -> float:
    return float(lib().or_logf(float(x)))


def expf(x: float) -> float:
    return float(lib().or_expf(float(x)))


def logf_max_ulp(lo, hi):
    w = C.c_float()
    e = lib().or_logf_max_ulp(float(lo), float(hi), C.byref(w))
    return e, w.value


def expf_max_ulp(lo, hi, stride=1):
    w = C.c_float()
    e = lib().or_expf_max_ulp(float(lo), float(hi), int(stride), C.byref(w))
    return e, w.value


def eval_decision_math(fn: int, x, param: float = 0.0):
    """The oracle's binary32 decision arithmetic over an array: fn 0 the Eq. 3 threshold
    2 ln(x / param), fn 1 e^x, fn 2 1 / (1 + e^-x) -- the routines its preprocess runs."""
    x = np.ascontiguousarray(x, np.float32)
    y = np.empty_like(x)
    lib().or_eval_decision_math(int(fn), x.shape[0], _ptr(x), float(param), _ptr(y))
    return y


def sh_basis(d):
    d = np.ascontiguousarray(d, np.float64)
    out = np.empty(16, np.float64)
    lib().or_sh_basis(d.ctypes.data_as(_dp), out.ctypes.data_as(_dp))
    return out


def tile_hit(u, v, a, b, c, t, x0, x1, y0, y1) -> bool:
    return bool(lib().or_tile_hit(*(float(x) for x in (u, v, a, b, c, t, x0, x1, y0, y1))))


def _scene_arrays(scene):
    m = np.ascontiguousarray(scene.means, np.float32)
    s = np.ascontiguousarray(scene.scales, np.float32)
    q = np.ascontiguousarray(scene.quats, np.float32)
    o = np.ascontiguousarray(scene.opacity, np.float32)
    sh = np.ascontiguousarray(scene.sh, np.float32)
    return m, s, q, o, sh


def preprocess(scene, cam, o=None, want64=True, sh_degree=3):
    """Per-Gaussian records: (valid[P] u8, rec32[P,16] f32, rec64[P,16] f64 | None, rect[P,4] i32)."""
    o = o or opts()
    P = scene.P
    m, s, q, op, sh = _scene_arrays(scene)
    rec32 = np.zeros((P, REC32), np.float32)
    rec64 = np.zeros((P, REC64), np.float64) if want64 else None
    rect = np.zeros((P, 4), np.int32)
    valid = np.zeros(P, np.uint8)
    cc = camera(cam)
    lib().or_preprocess(P, _ptr(m), _ptr(s), _ptr(q), _ptr(op), _ptr(sh), sh_degree, int(bool(scene.activated)),
                        C.byref(cc), C.byref(o), _ptr(rec32), _ptr(rec64), _ptr(rect), _ptr(valid))
    return valid, rec32, rec64, rect


def emit_pairs(rec32, rect, valid, cam):
    """Unsorted pairs in emission order (Gaussian id, tiles row-major) and per-Gaussian counts."""
    P = rec32.shape[0]
    cc = camera(cam)
    counts = np.zeros(P, np.int32)
    N = lib().or_emit_pairs(P, _ptr(rec32), _ptr(rect), _ptr(valid), C.byref(cc), _ptr(counts), None, None, 0)
    keys = np.zeros(max(N, 1), np.uint64)
    vals = np.zeros(max(N, 1), np.uint32)
    lib().or_emit_pairs(P, _ptr(rec32), _ptr(rect), _ptr(valid), C.byref(cc), _ptr(counts), _ptr(keys), _ptr(vals), N)
    return keys[:N], vals[:N], counts


def sort_pairs(keys, vals):
    k = np.ascontiguousarray(keys, np.uint64).copy()
    v = np.ascontiguousarray(vals, np.uint32).copy()
    lib().or_sort_pairs(k.shape[0], _ptr(k), _ptr(v))
    return k, v


def tiles_of(cam):
    tx = (cam.width + 15) // 16
    ty = (cam.height + 15) // 16
    return tx, ty


def tile_ranges(keys, cam):
    tx, ty = tiles_of(cam)
    r = np.zeros((tx * ty, 2), np.int64)
    k = np.ascontiguousarray(keys, np.uint64)
    lib().or_tile_ranges(k.shape[0], _ptr(k), tx * ty, _ptr(r))
    return r


def blend_tiled(mode, cam, ranges, vals, rec32, rec64, o=None):
    o = o or opts()
    H, W = cam.height, cam.width
    rgb = np.zeros((3, H, W), np.float64)
    T = np.zeros((H, W), np.float64)
    last = np.zeros((H, W), np.uint32)
    cc = camera(cam)
    ev = lib().or_blend_tiled(int(mode), C.byref(cc), C.byref(o), _ptr(np.ascontiguousarray(ranges, np.int64)),
                              _ptr(np.ascontiguousarray(vals, np.uint32)), _ptr(rec32),
                              _ptr(rec64) if mode == 64 else None, _ptr(rgb), _ptr(T), _ptr(last))
    return rgb, T, last, int(ev)


def depth_order(valid, rec32):
    """Gaussian ids passing the cull, sorted by (bits(z), id)."""
    ids = np.nonzero(valid)[0].astype(np.uint32)
    zb = rec32[ids, F["Z"]].view(np.uint32)
    order = np.lexsort((ids, zb))
    return ids[order]


def blend_brute(mode, cam, valid, rec32, rec64, o=None, crop=None):
    o = o or opts()
    x0, y0, w, h = crop or (0, 0, cam.width, cam.height)
    order = depth_order(valid, rec32)
    rgb = np.zeros((3, h, w), np.float64)
    T = np.zeros((h, w), np.float64)
    cc = camera(cam)
    lib().or_blend_brute(int(mode), C.byref(cc), C.byref(o), order.shape[0], _ptr(order), _ptr(rec32),
                         _ptr(rec64) if mode == 64 else None, x0, y0, w, h, _ptr(rgb), _ptr(T))
    return rgb, T


class Frame:
    """Everything the oracle computes for one (scene, camera)."""

    def __init__(self, scene, cam, o=None, mode=64, sh_degree=3):
        self.o = o or opts()
        self.cam = cam
        self.valid, self.rec32, self.rec64, self.rect = preprocess(scene, cam, self.o, want64=(mode == 64),
                                                                   sh_degree=sh_degree)
        self.keys_unsorted, self.vals_unsorted, self.counts = emit_pairs(self.rec32, self.rect, self.valid, cam)
        self.keys, self.vals = sort_pairs(self.keys_unsorted, self.vals_unsorted)
        self.ranges = tile_ranges(self.keys, cam)
        self.rgb, self.T, self.last, self.evals = blend_tiled(mode, cam, self.ranges, self.vals, self.rec32,
                                                              self.rec64, self.o)
        self.N = int(self.keys.shape[0])
        self.visible = int((self.counts > 0).sum())


def render(scene, cam, o=None, mode=64, sh_degree=3, want_pairs=False):
    """One whole frame through the single C entry point (the timed CPU baseline)."""
    o = o or opts()
    P = scene.P
    m, s, q, op, sh = _scene_arrays(scene)
    H, W = cam.height, cam.width
    rgb = np.zeros((3, H, W), np.float64)
    T = np.zeros((H, W), np.float64)
    last = np.zeros((H, W), np.uint32)
    stats = np.zeros(4, np.int64)
    cc = camera(cam)
    keys = vals = None
    cap = 0
    if want_pairs:
        cap = 1 << 26
        keys = np.zeros(cap, np.uint64)
        vals = np.zeros(cap, np.uint32)
    N = lib().or_render(int(mode), P, _ptr(m), _ptr(s), _ptr(q), _ptr(op), _ptr(sh), sh_degree,
                        int(bool(scene.activated)), C.byref(cc), C.byref(o), _ptr(rgb), _ptr(T), _ptr(last),
                        _ptr(keys), _ptr(vals), cap, _ptr(stats))
    if N < 0:
        raise MemoryError("oracle allocation failed")
    out = dict(rgb=rgb, T=T, last=last, N=int(N), visible=int(stats[0]), evals=int(stats[2]), culled_in=int(stats[3]))
    if want_pairs:
        out["keys"] = keys[:N]
        out["vals"] = vals[:N]
    return out


# ---------------------------------------------------------------------------------------- gradients
class Params64:
    """Binary64 copies of a scene's parameters (the variables of the gradient)."""

    def __init__(self, scene):
        self.means = np.ascontiguousarray(scene.means, np.float64)
        self.scales = np.ascontiguousarray(scene.scales, np.float64)
        self.quats = np.ascontiguousarray(scene.quats, np.float64)
        self.opacity = np.ascontiguousarray(scene.opacity, np.float64)
        self.sh = np.ascontiguousarray(scene.sh, np.float64).reshape(-1, 16, 3)
        self.activated = bool(scene.activated)
        self.P = self.means.shape[0]

    def arrays(self):
        return [self.means, self.scales, self.quats, self.opacity, self.sh]

    def copy(self):
        c = Params64.__new__(Params64)
        c.means, c.scales, c.quats, c.opacity, c.sh = (a.copy() for a in self.arrays())
        c.activated, c.P = self.activated, self.P
        return c


class Frozen:
    """The decisions of a reference render (binary64 mode): per-pixel contributor lists with
    alpha-clamp flags, and per-Gaussian colour / FOV clamp flags.  forward() and backward() are
    the frozen-decision image and its exact gradient."""

    def __init__(self, scene, cam, o=None, sh_degree=3):
        self.o = o or opts()
        self.cam = cam
        self.cc = camera(cam)
        self.sh_degree = sh_degree
        self.ref = Frame(scene, cam, self.o, mode=64, sh_degree=sh_degree)
        self.valid = self.ref.valid
        npx = cam.width * cam.height
        self.off = np.zeros(npx + 1, np.int64)
        n = lib().or_contrib_lists(C.byref(self.cc), C.byref(self.o), _ptr(self.ref.ranges), _ptr(self.ref.vals),
                                   _ptr(self.ref.rec32), _ptr(self.ref.rec64), _ptr(self.off), None, None, 0)
        self.gid = np.zeros(max(n, 1), np.int32)
        self.aclamp = np.zeros(max(n, 1), np.uint8)
        lib().or_contrib_lists(C.byref(self.cc), C.byref(self.o), _ptr(self.ref.ranges), _ptr(self.ref.vals),
                               _ptr(self.ref.rec32), _ptr(self.ref.rec64), _ptr(self.off), _ptr(self.gid),
                               _ptr(self.aclamp), n)
        self.n_contrib = int(n)
        self.p0 = Params64(scene)
        self.flags = np.zeros(scene.P, np.int32)
        a = self.p0.arrays()
        lib().or_grad_flags(scene.P, *(_ptr(x) for x in a), sh_degree, int(self.p0.activated), C.byref(self.cc),
                            C.byref(self.o), _ptr(self.valid), _ptr(self.flags))

    def forward(self, p: Params64):
        H, W = self.cam.height, self.cam.width
        rgb = np.zeros((3, H, W), np.float64)
        T = np.zeros((H, W), np.float64)
        lib().or_forward_fixed(p.P, *(_ptr(x) for x in p.arrays()), self.sh_degree, int(p.activated),
                               C.byref(self.cc), C.byref(self.o), _ptr(self.valid), _ptr(self.flags), _ptr(self.off),
                               _ptr(self.gid), _ptr(self.aclamp), _ptr(rgb), _ptr(T))
        return rgb, T

    def backward(self, p: Params64, dimg):
        dimg = np.ascontiguousarray(dimg, np.float64)
        g = [np.zeros_like(x) for x in p.arrays()]
        d2 = np.zeros((p.P, 9), np.float64)
        lib().or_backward_fixed(p.P, *(_ptr(x) for x in p.arrays()), self.sh_degree, int(p.activated),
                                C.byref(self.cc), C.byref(self.o), _ptr(self.valid), _ptr(self.flags),
                                _ptr(self.off), _ptr(self.gid), _ptr(self.aclamp), _ptr(dimg),
                                *(_ptr(x) for x in g), _ptr(d2))
        return dict(means=g[0], scales=g[1], quats=g[2], opacity=g[3], sh=g[4], d2=d2)
