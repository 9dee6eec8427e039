"""GB300 (sm_103a) 3D Gaussian Splatting forward rasterizer with FlashGS's opacity-aware exact
intersection (arXiv 2408.07967).

Thin Python binding over the C ABI of include/gs.h: the functions carry the C names and only
marshal arguments (torch CUDA tensors -> device pointers, the current torch stream ->
cudaStream_t).  Every stage of the rasterizer runs in the library's CUDA kernels; when
libgs.so is missing the binding raises -- there is no CPU fallback.

Importing this package loads neither torch nor the library; both happen on first use.
"""
from __future__ import annotations

import ctypes as C

from . import _native

__all__ = ["GsError", "Context", "Scene", "Frame", "Server", "Router", "gs_camera_from", "gs_opts", "gs_sort_pairs", "gs_eval_decision_math", "lib"]

GS_OK = 0
STATUS_NAMES = {0: "GS_OK", -1: "GS_ERR_INVALID_ARG", -2: "GS_ERR_OOM", -3: "GS_ERR_PAIR_OVERFLOW", -4: "GS_ERR_CUDA",
                -5: "GS_ERR_DEVICE_TIMEOUT", -6: "GS_ERR_BUSY", -7: "GS_ERR_CAPACITY", -8: "GS_ERR_NO_DEVICE"}


class GsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    return _native.load()


def _check(status):
    if status != GS_OK:
        raise GsError(status, lib().gs_last_error().decode(errors="replace"))


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "tensors must be contiguous CUDA tensors"
    return C.c_void_p(t.data_ptr())


def gs_camera_from(cam) -> _native.gs_camera:
    """gs_camera from any object with R, t, fx, fy, cx, cy, width, height (and optional near)."""
    import numpy as np
    c = _native.gs_camera()
    R = np.asarray(cam.R, np.float32).reshape(9)
    t = np.asarray(cam.t, np.float32).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_z = float(getattr(cam, "near", 0.2))
    return c


def gs_opts(bg=(0.0, 0.0, 0.0), tau=None, alpha_max=None, T_min=None, dilation=None, cap_3sigma=False,
            clamp_fov=True, intersect=0) -> _native.gs_render_opts:
    o = _native.gs_render_opts()
    _check(lib().gs_default_opts(C.byref(o)))
    for i in range(3):
        o.bg[i] = float(bg[i])
    if tau is not None:
        o.tau = float(tau)
    if alpha_max is not None:
        o.alpha_max = float(alpha_max)
    if T_min is not None:
        o.T_min = float(T_min)
    if dilation is not None:
        o.dilation = float(dilation)
    o.cap_3sigma = int(bool(cap_3sigma))
    o.clamp_fov = int(bool(clamp_fov))
    o.intersect = int(intersect)    # 0 exact tile pairs; 1 the 3DGS 3-sigma square (the paper's baseline)
    return o


class Context:
    """gs_context: one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        h = C.c_void_p()
        _check(lib().gs_context_create(self.device, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().gs_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """gs_scene: device-resident Gaussians (position plane, scale/rotation plane, SH blocks).
    sh_half=True keeps the SH coefficients as binary16 (opt-in reduced precision)."""

    def __init__(self, ctx: Context, means, scales, quats, opacity, sh, sh_degree=3, activated=True, stream=None,
                 sh_half=False):
        self.ctx = ctx
        self.sh_half = bool(sh_half)
        g = self._struct(means, scales, quats, opacity, sh, sh_degree, activated, self.sh_half)
        h = C.c_void_p()
        _check(lib().gs_scene_create(ctx.h, C.byref(g), _stream(stream), C.byref(h)))
        self.h = h
        self.P = int(g.P)

    @staticmethod
    def _struct(means, scales, quats, opacity, sh, sh_degree, activated, sh_half=False):
        g = _native.gs_gaussians()
        g.means, g.scales, g.quats, g.opacity, g.sh = (_ptr(x) for x in (means, scales, quats, opacity, sh))
        g.P = int(means.shape[0])
        g.sh_degree = int(sh_degree)
        g.activated = int(bool(activated))
        g.sh_half = int(bool(sh_half))
        for x, k in ((means, 3), (scales, 3), (quats, 4), (sh, 48)):
            assert x.numel() == g.P * k, "array size does not match P"
        assert opacity.numel() == g.P
        return g

    def gs_scene_update(self, means, scales, quats, opacity, sh, sh_degree=3, activated=True, stream=None):
        g = self._struct(means, scales, quats, opacity, sh, sh_degree, activated, self.sh_half)
        _check(lib().gs_scene_update(self.h, C.byref(g), _stream(stream)))

    @classmethod
    def from_numpy(cls, ctx, scene, device="cuda", stream=None, sh_half=False):
        """Upload a synth.Scene-like object (numpy float32 arrays) and build the device scene."""
        import torch
        arrs = [torch.from_numpy(a.reshape(a.shape[0], -1) if a.ndim > 1 else a).to(device).contiguous()
                for a in (scene.means, scene.scales, scene.quats, scene.opacity, scene.sh)]
        s = cls(ctx, *arrs, sh_degree=3, activated=scene.activated, stream=stream, sh_half=sh_half)
        s._inputs = arrs          # kept alive until the pack kernel has run
        return s

    def close(self):
        if getattr(self, "h", None):
            lib().gs_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Frame:
    """gs_frame: per-frame device state allocated once."""

    def __init__(self, ctx: Context, max_gaussians: int, max_pairs: int, max_width: int, max_height: int):
        self.ctx = ctx
        h = C.c_void_p()
        _check(lib().gs_frame_create(ctx.h, int(max_gaussians), int(max_pairs), int(max_width), int(max_height),
                                     C.byref(h)))
        self.h = h
        self.max_pairs = int(max_pairs)

    # ---- stages (C names)
    def gs_preprocess(self, scene: Scene, cam, opts=None, stream=None):
        o = opts or gs_opts()
        _check(lib().gs_preprocess(self.h, scene.h, C.byref(gs_camera_from(cam)), C.byref(o), _stream(stream)))

    def gs_sort(self, stream=None):
        _check(lib().gs_sort(self.h, _stream(stream)))

    def gs_ranges(self, stream=None):
        _check(lib().gs_ranges(self.h, _stream(stream)))

    def gs_blend(self, rgb, T=None, last=None, opts=None, stream=None):
        o = opts or gs_opts()
        _check(lib().gs_blend(self.h, C.byref(o), _ptr(rgb), _ptr(T), _ptr(last), _stream(stream)))

    def gs_render(self, scene: Scene, cam, rgb, T=None, last=None, opts=None, stream=None):
        o = opts or gs_opts()
        _check(lib().gs_render(self.h, scene.h, C.byref(gs_camera_from(cam)), C.byref(o), _ptr(rgb), _ptr(T),
                               _ptr(last), _stream(stream)))

    def gs_render_backward(self, scene: Scene, dL_drgb, T, last, grads=None, accumulate=False, stream=None):
        """Gradients of the last render w.r.t. the scene parameters (dict of tensors)."""
        import torch
        P = scene.P
        if grads is None:
            dev = dL_drgb.device
            grads = dict(means=torch.empty((P, 3), device=dev), scales=torch.empty((P, 3), device=dev),
                         quats=torch.empty((P, 4), device=dev), opacity=torch.empty((P,), device=dev),
                         sh=torch.empty((P, 16, 3), device=dev))
        g = _native.gs_gaussian_grads()
        g.means, g.scales, g.quats, g.opacity, g.sh = (_ptr(grads[k]) for k in
                                                       ("means", "scales", "quats", "opacity", "sh"))
        _check(lib().gs_render_backward(self.h, scene.h, _ptr(dL_drgb), _ptr(T), _ptr(last), C.byref(g),
                                        int(bool(accumulate)), _stream(stream)))
        return grads

    def gs_render_batch(self, scenes, cams, opts=None, stream=None, want_T=False, want_last=False):
        """Render several requests (scenes and cameras of any sizes) in one pass of every stage.
        Returns a list of (rgb, T, last) tensors."""
        import torch
        n = len(cams)
        sc = (C.c_void_p * n)(*[s.h.value for s in scenes])
        cm = (_native.gs_camera * n)(*[gs_camera_from(c) for c in cams])
        op = None
        if opts is not None:
            op = (_native.gs_render_opts * n)(*opts)
        outs = []
        for c in cams:
            H, W = int(c.height), int(c.width)
            outs.append((torch.empty((3, H, W), device="cuda"),
                         torch.empty((H, W), device="cuda") if want_T else None,
                         torch.empty((H, W), dtype=torch.int32, device="cuda") if want_last else None))
        rgb = (C.c_void_p * n)(*[o[0].data_ptr() for o in outs])
        T = (C.c_void_p * n)(*[o[1].data_ptr() for o in outs]) if want_T else None
        last = (C.c_void_p * n)(*[o[2].data_ptr() for o in outs]) if want_last else None
        _check(lib().gs_render_batch(self.h, n, sc, cm, op, rgb, T, last, _stream(stream)))
        return outs

    def gs_frame_use_graph(self, enable: bool):
        _check(lib().gs_frame_use_graph(self.h, int(bool(enable))))

    def gs_frame_set_tuning(self, blend_variant: int | None = None, sort_mode: int | None = None,
                            sort_algo: int | None = None):
        t = _native.gs_tuning()
        _check(lib().gs_frame_get_tuning(self.h, C.byref(t)))
        if blend_variant is not None:
            t.blend_variant = int(blend_variant)
        if sort_mode is not None:
            t.sort_mode = int(sort_mode)
        if sort_algo is not None:
            t.sort_algo = int(sort_algo)
        _check(lib().gs_frame_set_tuning(self.h, C.byref(t)))

    def gs_frame_get_tuning(self) -> dict:
        t = _native.gs_tuning()
        _check(lib().gs_frame_get_tuning(self.h, C.byref(t)))
        return {"blend_variant": t.blend_variant, "sort_mode": t.sort_mode, "sort_algo": t.sort_algo}

    def gs_autotune(self, scene: Scene, cams, opts=None, cache_path=None, stream=None) -> dict:
        """Pick the fastest launch shape for this scene and image size (cached per device, P, W, H)."""
        arr = (_native.gs_camera * len(cams))(*[gs_camera_from(c) for c in cams])
        o = opts or gs_opts()
        t = _native.gs_tuning()
        path = None if cache_path is None else str(cache_path).encode()
        _check(lib().gs_autotune(self.h, scene.h, arr, len(cams), C.byref(o), path, C.byref(t), _stream(stream)))
        return {"blend_variant": t.blend_variant, "sort_mode": t.sort_mode, "sort_algo": t.sort_algo}

    def gs_frame_set_counting(self, enable: bool):
        _check(lib().gs_frame_set_counting(self.h, int(bool(enable))))

    def gs_frame_enable_timing(self, enable: bool):
        _check(lib().gs_frame_enable_timing(self.h, int(bool(enable))))

    def gs_frame_stage_ms(self):
        ms = (C.c_float * 4)()
        _check(lib().gs_frame_stage_ms(self.h, ms))
        return list(ms)

    def gs_frame_backward_ms(self):
        """[reverse blend ms, per-Gaussian chain rule ms] of the last timed backward."""
        ms = (C.c_float * 2)()
        _check(lib().gs_frame_backward_ms(self.h, ms))
        return [ms[0], ms[1]]

    def gs_render_host(self, scene: Scene, cam, rgb_host, T_host=None, last_host=None, opts=None, stream=None):
        """Render and copy into host tensors (page-locked for asynchronous copies)."""
        o = opts or gs_opts()
        hp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
        _check(lib().gs_render_host(self.h, scene.h, C.byref(gs_camera_from(cam)), C.byref(o), hp(rgb_host),
                                    hp(T_host), hp(last_host), _stream(stream)))

    # ---- conveniences
    def render(self, scene: Scene, cam, opts=None, stream=None, want_T=True, want_last=True):
        import torch
        H, W = int(cam.height), int(cam.width)
        rgb = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
        T = torch.empty((H, W), dtype=torch.float32, device="cuda") if want_T else None
        last = torch.empty((H, W), dtype=torch.int32, device="cuda") if want_last else None
        self.gs_render(scene, cam, rgb, T, last, opts, stream)
        return rgb, T, last

    def stats(self, stream=None) -> dict:
        s = _native.gs_frame_stats()
        _check(lib().gs_frame_get_stats(self.h, C.byref(s), _stream(stream)))
        return {k: getattr(s, k) for k, _ in _native.gs_frame_stats._fields_}

    def pairs(self, which: int = 1, stream=None):
        """(keys uint64 as int64 tensor, values int32 tensor) of the emission-order (0) or sorted (1) list."""
        import torch
        n_total = self.stats(stream)["pairs"]
        cap = max(1, min(n_total, self.max_pairs))
        keys = torch.empty(cap, dtype=torch.int64, device="cuda")
        vals = torch.empty(cap, dtype=torch.int32, device="cuda")
        n = C.c_int64()
        _check(lib().gs_frame_pairs(self.h, int(which), _ptr(keys), _ptr(vals), cap, C.byref(n), _stream(stream)))
        return keys[: n.value], vals[: n.value]

    def starts(self, stream=None):
        import torch
        st = self.stats(stream)
        n = st["tiles_x"] * st["tiles_y"] + 1
        out = torch.empty(n, dtype=torch.int32, device="cuda")
        _check(lib().gs_frame_ranges(self.h, _ptr(out), n, _stream(stream)))
        return out

    def nbytes(self) -> int:
        return int(lib().gs_frame_bytes(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().gs_frame_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """gs_server: continuous-batching request loop (worker thread inside the library)."""

    def __init__(self, ctx: Context, plain=False, **cfg):
        c = _native.gs_server_cfg()
        _check(lib().gs_default_server_cfg(C.byref(c)))
        for k, v in cfg.items():
            setattr(c, k, int(v))
        c.plain = int(bool(plain))
        h = C.c_void_p()
        _check(lib().gs_server_create(ctx.h, C.byref(c), C.byref(h)))
        self.h = h
        self.ctx = ctx
        self.cfg = c
        self._bufs = {}

    @staticmethod
    def clock() -> float:
        return float(lib().gs_clock_s())

    def gs_server_hold(self, hold: bool = True):
        """Stop admitting (and wait for the batches in flight), or resume."""
        _check(lib().gs_server_hold(self.h, int(bool(hold))))

    def gs_server_submit(self, scene: Scene, cam, rgb_host, opts=None, arrival_s=0.0) -> int:
        """rgb_host: a CPU float32 tensor [3,H,W] (page-locked for asynchronous copies)."""
        assert rgb_host.dtype.is_floating_point and not rgb_host.is_cuda and rgb_host.is_contiguous()
        t = C.c_uint64()
        o = opts or gs_opts()
        _check(lib().gs_server_submit(self.h, scene.h, C.byref(gs_camera_from(cam)), C.byref(o),
                                      C.c_void_p(rgb_host.data_ptr()), float(arrival_s), C.byref(t)))
        self._bufs[t.value] = rgb_host
        return t.value

    def gs_server_wait(self, ticket: int, timeout_ms: int = -1) -> dict:
        st = _native.gs_request_stats()
        status = lib().gs_server_wait(self.h, C.c_uint64(ticket), int(timeout_ms), C.byref(st))
        if status == -5:
            raise GsError(status, lib().gs_last_error().decode())
        self._bufs.pop(ticket, None)
        return {k: getattr(st, k) for k, _ in _native.gs_request_stats._fields_}

    def stats(self) -> dict:
        st = _native.gs_server_stats()
        _check(lib().gs_server_get_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in _native.gs_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            lib().gs_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Router:
    """gs_router: requests routed across replicas (one server per GPU) by scene placement and
    fewest outstanding pixels.  Router.on_servers(...) drives gs_server objects; Router(replicas,
    submit, wait) takes Python callables (submit(replica, scene, cam_ptr, opts_ptr, rgb_ptr,
    arrival_s) -> (status, ticket); wait(replica, ticket, timeout_ms, stats) -> status)."""

    def __init__(self, replicas: int, submit=None, wait=None, _servers=None):
        h = C.c_void_p()
        self._keep = []
        if _servers is not None:
            arr = (C.c_void_p * replicas)(*[sv.h.value for sv in _servers])
            self._keep.append((arr, _servers))
            _check(lib().gs_router_create_on_servers(int(replicas), arr, C.byref(h)))
        else:
            def c_submit(user, replica, scene, cam, opts, rgb, arrival, ticket):
                st, t = submit(replica, scene, cam, opts, rgb, arrival)
                ticket[0] = t
                return st

            def c_wait(user, replica, ticket, timeout_ms, out):
                return wait(replica, ticket, timeout_ms, _native.gs_request_stats.from_address(out))

            cs, cw = _native.ROUTER_SUBMIT(c_submit), _native.ROUTER_WAIT(c_wait)
            be = _native.gs_router_backend(cs, cw, None)
            self._keep += [cs, cw, be]
            _check(lib().gs_router_create(int(replicas), C.byref(be), C.byref(h)))
        self.h = h
        self.replicas = replicas

    @classmethod
    def on_servers(cls, servers) -> "Router":
        return cls(len(servers), _servers=list(servers))

    def place_scene(self, scene_id: int, replica: int, scene: Scene | None = None):
        _check(lib().gs_router_place_scene(self.h, int(scene_id), int(replica), scene.h if scene else None))

    def submit(self, scene_id: int, cam, rgb_host=None, opts=None, arrival_s: float = 0.0) -> int:
        t = C.c_uint64()
        o = opts or gs_opts()
        ptr = C.c_void_p(rgb_host.data_ptr()) if rgb_host is not None else None
        _check(lib().gs_router_submit(self.h, int(scene_id), C.byref(gs_camera_from(cam)), C.byref(o), ptr,
                                      float(arrival_s), C.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        st = _native.gs_request_stats()
        rep = C.c_int32(-1)
        status = lib().gs_router_wait(self.h, C.c_uint64(ticket), int(timeout_ms), C.byref(st), C.byref(rep))
        if status in (-1, -5):
            raise GsError(status, lib().gs_last_error().decode(errors="replace"))
        d = {k: getattr(st, k) for k, _ in _native.gs_request_stats._fields_}
        d["status"] = status
        return d, rep.value

    def outstanding(self, replica: int):
        r, p = C.c_int64(), C.c_int64()
        _check(lib().gs_router_outstanding(self.h, int(replica), C.byref(r), C.byref(p)))
        return r.value, p.value

    def close(self):
        if getattr(self, "h", None):
            lib().gs_router_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gs_measure_alu_peaks(device: int = 0, target_ms: float = 200.0) -> dict:
    """Measured FP32 FMA and ex2.approx throughput (lane-operations/s / 1e12) of a device."""
    out = _native.gs_alu_peaks()
    _check(lib().gs_measure_alu_peaks(int(device), float(target_ms), C.byref(out)))
    return {"fma_tops": out.fma_tops, "ex2_tops": out.ex2_tops, "fma_ms": out.fma_ms, "ex2_ms": out.ex2_ms,
            "sm_count": out.sm_count}


def gs_sort_pairs(ctx: Context, keys, vals, end_bit: int = 64, stream=None):
    """Stable radix sort of (int64-viewed uint64 keys, int32 values) by key bits [0, end_bit).
    Returns the sorted (keys, vals) tensors (inputs are used as ping-pong storage)."""
    import torch
    n = int(keys.numel())
    kt = torch.empty_like(keys)
    vt = torch.empty_like(vals)
    in_tmp = C.c_int32()
    _check(lib().gs_sort_pairs(ctx.h, _ptr(keys), _ptr(vals), _ptr(kt), _ptr(vt), n, int(end_bit), C.byref(in_tmp),
                               _stream(stream)))
    return (kt, vt) if in_tmp.value else (keys, vals)


def gs_eval_decision_math(fn: int, x, param: float = 0.0, stream=None):
    """The device's binary32 decision arithmetic over a float32 CUDA tensor: fn 0 the Eq. 3
    threshold 2 ln(x / param), fn 1 e^x, fn 2 1 / (1 + e^-x).  Returns a new tensor."""
    import torch
    y = torch.empty_like(x)
    _check(lib().gs_eval_decision_math(int(fn), _ptr(x), _ptr(y), int(x.numel()), float(param), _stream(stream)))
    return y
