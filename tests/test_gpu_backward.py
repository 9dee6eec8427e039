"""GPU gradients through the C ABI against the binary64 oracle gradient (the exact derivative of
the frozen-decision forward, itself pinned by finite differences) and against central finite
differences of that forward; bar: relative error <= 1e-3 per parameter group, and per element
with an absolute floor of 1e-5 of the group's largest value."""
import numpy as np
import pytest

import oracle
from paper_2408_07967_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2408_07967_gb300 as gs  # noqa: E402
from paper_2408_07967_gb300.autograd import GaussianRasterizer  # noqa: E402

GROUPS = ("means", "scales", "quats", "opacity", "sh")


@pytest.fixture(scope="module")
def ctx():
    from paper_2408_07967_gb300 import build
    build.build()
    return gs.Context(0)


def gpu_grads(ctx, scene, cam, w, opts_kw=None, sort_mode=None):
    sc = gs.Scene.from_numpy(ctx, scene)
    fr = gs.Frame(ctx, scene.P, 1 << 22, cam.width, cam.height)
    fr.gs_frame_set_tuning(sort_mode=sort_mode)
    o = gs.gs_opts(**(opts_kw or {}))
    rgb, T, last = fr.render(sc, cam, o)
    dl = torch.from_numpy(w.astype(np.float32)).cuda().contiguous()
    g = fr.gs_render_backward(sc, dl, T, last)
    torch.cuda.synchronize()
    return {k: v.double().cpu().numpy().reshape(scene.P, -1) for k, v in g.items()}


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("sort_mode", [0, 1])
@pytest.mark.parametrize("seed", [5, 6])
def test_gradients_match_oracle(ctx, seed, sort_mode):
    scene, cam = synth.grad_subset(P=2000, seed=seed, size=64)
    bg = (0.1, 0.2, 0.3)
    fz = oracle.Frozen(scene, cam, oracle.opts(bg=bg))
    w = np.random.default_rng(seed).normal(0, 1, (3, 64, 64))
    ref = fz.backward(fz.p0, w)
    got = gpu_grads(ctx, scene, cam, w, dict(bg=bg), sort_mode)
    for k in GROUPS:
        r = ref[k].reshape(scene.P, -1)
        assert rel(got[k], r) <= 1e-3, (k, rel(got[k], r))


@pytest.mark.parametrize("sort_mode", [0, 1])
def test_gradients_match_oracle_per_element(ctx, sort_mode):
    """Element by element: |gpu - oracle| <= 1e-3 |oracle| + 1e-5 max|oracle| of the group.  The
    floor is for elements that are sums of many terms cancelling to almost nothing, where binary32
    accumulation (atomics over up to ~10^4 pixels a Gaussian) leaves an absolute error far below the
    group's scale but a large relative one."""
    scene, cam = synth.grad_subset(P=2000, seed=5, size=64)
    bg = (0.1, 0.2, 0.3)
    fz = oracle.Frozen(scene, cam, oracle.opts(bg=bg))
    w = np.random.default_rng(11).normal(0, 1, (3, 64, 64))
    ref = fz.backward(fz.p0, w)
    got = gpu_grads(ctx, scene, cam, w, dict(bg=bg), sort_mode)
    for k in GROUPS:
        r = ref[k].reshape(scene.P, -1)
        g = got[k]
        floor = 1e-5 * np.abs(r).max()
        excess = np.abs(g - r) - (1e-3 * np.abs(r) + floor)
        i = np.unravel_index(np.argmax(excess), r.shape)
        assert excess.max() <= 0, (k, i, g[i], r[i], floor)
        assert np.count_nonzero(r) > 100, k


@pytest.mark.parametrize("accumulate", [False, True])
def test_unaligned_gradient_buffers(ctx, accumulate):
    """Caller buffers that are not 16-byte aligned take scalar stores; the result is the same as
    with aligned ones (and accumulation adds to what is there).  The 2D gradients are summed with
    float atomics in no fixed order, so two runs agree to rounding, not bit for bit."""
    scene, cam = synth.grad_subset(P=1200, seed=9, size=48)
    sc = gs.Scene.from_numpy(ctx, scene)
    fr = gs.Frame(ctx, scene.P, 1 << 22, cam.width, cam.height)
    rgb, T, last = fr.render(sc, cam)
    dl = torch.randn_like(rgb)
    shapes = dict(means=(scene.P, 3), scales=(scene.P, 3), quats=(scene.P, 4), opacity=(scene.P,),
                  sh=(scene.P, 16, 3))
    base = {k: torch.randn(v, device="cuda") for k, v in shapes.items()}
    aligned = {k: v.clone() for k, v in base.items()}
    store = {k: torch.empty(int(np.prod(v)) + 1, device="cuda") for k, v in shapes.items()}
    unaligned = {k: store[k][1:].view(shapes[k]) for k in shapes}
    for k in shapes:
        unaligned[k].copy_(base[k])
    assert unaligned["sh"].data_ptr() % 16 != 0 and unaligned["quats"].data_ptr() % 16 != 0
    a = fr.gs_render_backward(sc, dl, T, last, grads=aligned, accumulate=accumulate)
    b = fr.gs_render_backward(sc, dl, T, last, grads=unaligned, accumulate=accumulate)
    torch.cuda.synchronize()
    for k in shapes:
        scale = float(a[k].abs().max())
        assert torch.allclose(a[k], b[k], rtol=1e-4, atol=1e-6 * scale), k
    if accumulate:
        fresh = fr.gs_render_backward(sc, dl, T, last)
        torch.cuda.synchronize()
        assert torch.allclose(a["sh"], base["sh"] + fresh["sh"], rtol=1e-4, atol=1e-5)


def test_gradients_match_finite_differences(ctx):
    scene, cam = synth.grad_subset(P=2000, seed=7, size=64)
    fz = oracle.Frozen(scene, cam)
    w = np.random.default_rng(7).normal(0, 1, (3, 64, 64))
    got = gpu_grads(ctx, scene, cam, w)
    used = np.unique(fz.gid[: fz.n_contrib])
    rng = np.random.default_rng(1)
    h = 1e-6

    def L(p):
        rgb, _ = fz.forward(p)
        return float((rgb * w).sum())

    for k in GROUPS:
        g = got[k]
        scale = np.linalg.norm(g) / np.sqrt(np.count_nonzero(g) or 1)
        for _ in range(12):
            gi = int(rng.choice(used))
            j = int(rng.integers(0, g.shape[1]))
            pp, pm = fz.p0.copy(), fz.p0.copy()
            arr_p, arr_m = getattr(pp, k).reshape(scene.P, -1), getattr(pm, k).reshape(scene.P, -1)
            arr_p[gi, j] += h
            arr_m[gi, j] -= h
            fd = (L(pp) - L(pm)) / (2 * h)
            assert abs(g[gi, j] - fd) <= 1e-3 * (abs(fd) + scale), (k, gi, j, g[gi, j], fd)


def test_autograd_batch_accumulates(ctx):
    scene, cam0 = synth.grad_subset(P=1500, seed=8, size=48)
    cam1 = synth.look_at((0.3, -0.2, 0.1), (0.0, 0.0, 3.0), 48, 48, 60.0)
    dev = "cuda"
    params = [torch.tensor(a, device=dev, requires_grad=True) for a in
              (scene.means, scene.scales, scene.quats, scene.opacity, scene.sh)]
    rast = GaussianRasterizer(ctx, scene.P, 48, 48, batch=2)
    img = rast(*params, [cam0, cam1])
    assert img.shape == (2, 3, 48, 48)
    wt = torch.randn_like(img)
    (img * wt).sum().backward()
    # per-camera gradients through the C ABI must sum to the batch gradient
    tot = None
    for i, cam in enumerate((cam0, cam1)):
        g = gpu_grads(ctx, scene, cam, wt[i].detach().cpu().numpy().astype(np.float64))
        tot = g if tot is None else {k: tot[k] + g[k] for k in g}
    for k, p in zip(GROUPS, params):
        a = p.grad.double().cpu().numpy().reshape(scene.P, -1)
        assert rel(a, tot[k]) <= 1e-5, k
