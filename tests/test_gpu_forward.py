"""GPU parity of the forward path against the CPU oracle, through the C ABI.

Bars: pair counts, the emission-order and the sorted (tile, depth) key lists, their Gaussian
ids and the tile ranges are bit-exact against the oracle's binary32 decisions; images are
within max-abs 2e-3 and mean-abs 1e-5 per RGB channel of the oracle's binary64 image (the
transmittance likewise); the last-contributor index may differ only where the early-stop test
T' < T_min is a near tie (binary32 vs binary64 transmittance)."""
import numpy as np
import pytest

import oracle
from paper_2408_07967_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2408_07967_gb300 as gs  # noqa: E402

RGB_MAX, RGB_MEAN = 2e-3, 1e-5


@pytest.fixture(scope="module")
def ctx():
    from paper_2408_07967_gb300 import build
    build.build()
    return gs.Context(0)


def run_gpu(ctx, scene, cam, opts_kw=None, max_pairs=1 << 22, graph=False, variant=None, sort_mode=None,
            sort_algo=None, sh_half=False):
    sc = gs.Scene.from_numpy(ctx, scene, sh_half=sh_half)
    fr = gs.Frame(ctx, scene.P, max_pairs, cam.width, cam.height)
    fr.gs_frame_set_tuning(blend_variant=variant, sort_mode=sort_mode, sort_algo=sort_algo)
    o = gs.gs_opts(**(opts_kw or {}))
    H, W = cam.height, cam.width
    rgb = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
    T = torch.empty((H, W), dtype=torch.float32, device="cuda")
    last = torch.empty((H, W), dtype=torch.int32, device="cuda")
    if graph:
        s = torch.cuda.Stream()
        fr.gs_frame_use_graph(True)
        with torch.cuda.stream(s):
            fr.gs_render(sc, cam, rgb, T, last, o)
        s.synchronize()
        ku = vu = None
    else:
        fr.gs_preprocess(sc, cam, o)
        ku, vu = fr.pairs(0)
        fr.gs_sort()
        fr.gs_ranges()
        fr.gs_blend(rgb, T, last, o)
    torch.cuda.synchronize()
    st = fr.stats()
    ks, vs = fr.pairs(1)
    out = dict(stats=st, rgb=rgb.double().cpu().numpy(), T=T.double().cpu().numpy(),
               last=last.cpu().numpy().view(np.uint32), keys=ks.cpu().numpy().view(np.uint64),
               vals=vs.cpu().numpy().view(np.uint32), starts=fr.starts().cpu().numpy().view(np.uint32))
    if ku is not None:
        out["keys_unsorted"] = ku.cpu().numpy().view(np.uint64)
        out["vals_unsorted"] = vu.cpu().numpy().view(np.uint32)
    out["sort_mode"] = fr.gs_frame_get_tuning()["sort_mode"]
    fr.close()
    sc.close()
    return out


def check(res, ref, check_unsorted=True, t_min=1e-4, alpha_max=0.99):
    st = res["stats"]
    assert st["status"] == 0, st
    assert st["pairs"] == ref.N
    assert st["visible"] == ref.visible
    if check_unsorted and "keys_unsorted" in res:
        ku, vu = ref.keys_unsorted, ref.vals_unsorted
        if res["sort_mode"] == 1:
            # two-level order: pairs emitted in (depth bits, Gaussian id, tile) order
            order = np.lexsort((ku >> np.uint64(32), vu, ku & np.uint64(0xffffffff)))
            ku, vu = ku[order], vu[order]
        assert np.array_equal(res["keys_unsorted"], ku)
        assert np.array_equal(res["vals_unsorted"], vu)
    assert np.array_equal(res["keys"], ref.keys)
    assert np.array_equal(res["vals"], ref.vals)
    starts = res["starts"].astype(np.int64)
    nz = ref.ranges[:, 1] > ref.ranges[:, 0]
    assert np.array_equal(starts[:-1][nz], ref.ranges[nz, 0])
    assert np.array_equal(starts[1:][nz], ref.ranges[nz, 1])
    assert np.all(starts[1:][~nz] == starts[:-1][~nz])
    err = np.abs(res["rgb"] - ref.rgb)
    assert err.max() <= RGB_MAX, err.max()
    assert err.mean(axis=(1, 2)).max() <= RGB_MEAN, err.mean(axis=(1, 2))
    assert np.abs(res["T"] - ref.T).max() <= RGB_MAX
    diff = res["last"] != ref.last
    assert diff.mean() <= 1e-3, diff.mean()
    # where the index differs, the early-stop decision T (1 - alpha) < T_min was a near tie: the
    # pixel's transmittance is within the stop regime T <= T_min / (1 - alpha_max) on both sides
    if diff.any():
        stop_regime = t_min / (1.0 - alpha_max) * 1.01
        assert np.all(ref.T[diff] <= stop_regime) and np.all(res["T"][diff] <= stop_regime)


@pytest.mark.parametrize("sort_algo", [0, 1, 2])
@pytest.mark.parametrize("sort_mode", [0, 1])
def test_tiny_config_parity(ctx, sort_mode, sort_algo):
    scene, cams = synth.load_config("tiny")
    ref = oracle.Frame(scene, cams[0], mode=64)
    check(run_gpu(ctx, scene, cams[0], sort_mode=sort_mode, sort_algo=sort_algo), ref)


@pytest.mark.parametrize("sort_mode", [0, 1])
@pytest.mark.parametrize("W,H", [(100, 76), (17, 33), (1, 1), (256, 130)])
def test_ragged_images(ctx, W, H, sort_mode):
    scene, cam = synth.random_small_scene(2500, 31 + W, W, H, log_scale_mu=-2.6, log_scale_sigma=1.0)
    ref = oracle.Frame(scene, cam, mode=64)
    check(run_gpu(ctx, scene, cam, sort_mode=sort_mode), ref)


@pytest.mark.parametrize("sort_mode", [0, 1])
@pytest.mark.parametrize("opts_kw", [dict(cap_3sigma=True), dict(bg=(0.3, 0.6, 0.1)),
                                     dict(clamp_fov=False, dilation=0.1), dict(tau=0.02, T_min=1e-3)])
def test_options(ctx, opts_kw, sort_mode):
    scene, cam = synth.random_small_scene(3000, 11, 128, 96, log_scale_mu=-2.4, log_scale_sigma=1.0)
    ref = oracle.Frame(scene, cam, oracle.opts(**opts_kw), mode=64)
    check(run_gpu(ctx, scene, cam, opts_kw, sort_mode=sort_mode), ref, t_min=opts_kw.get("T_min", 1e-4))


def test_raw_parameters_activated_on_device(ctx):
    scene, cam = synth.random_small_scene(3000, 12, 128, 96, activated=False, log_scale_mu=-2.6)
    ref = oracle.Frame(scene, cam, mode=64)
    check(run_gpu(ctx, scene, cam), ref)


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("sort_mode", [0, 1])
def test_sh_half_storage(ctx, sort_mode, graph):
    """Opt-in binary16 SH storage: against the oracle given the same rounded coefficients (numpy's
    IEEE round to nearest even, as the device's conversion) every forward bar holds as for binary32
    storage -- pairs and keys do not depend on SH; against the unrounded coefficients the image
    moves by the rounding alone, within the image bar."""
    import dataclasses
    scene, cam = synth.random_small_scene(3000, 21, 128, 96, log_scale_mu=-2.4)
    rounded = dataclasses.replace(scene, sh=scene.sh.astype(np.float16).astype(np.float32))
    res = run_gpu(ctx, scene, cam, sort_mode=sort_mode, graph=graph, sh_half=True)
    check(res, oracle.Frame(rounded, cam, mode=64))
    full = oracle.Frame(scene, cam, mode=64)
    moved = np.abs(res["rgb"] - full.rgb)
    assert 0 < moved.max() <= RGB_MAX, moved.max()


def test_sh_half_fixed_at_creation(ctx):
    scene, cam = synth.random_small_scene(100, 22, 64, 64)
    sc = gs.Scene.from_numpy(ctx, scene, sh_half=True)
    arrs = sc._inputs
    sc.sh_half = False          # an update must keep the creation's storage
    with pytest.raises(gs.GsError):
        sc.gs_scene_update(*arrs)


@pytest.mark.parametrize("sort_algo", [0, 1, 2])
@pytest.mark.parametrize("sort_mode", [0, 1])
def test_large_gaussians_many_candidate_tiles(ctx, sort_mode, sort_algo):
    """Gaussians with hundreds of candidate tiles spread over many load-balanced steps."""
    scene, cam = synth.random_small_scene(400, 13, 320, 240, log_scale_mu=-1.2, log_scale_sigma=0.5)
    ref = oracle.Frame(scene, cam, mode=64)
    big = ((ref.rect[:, 1] - ref.rect[:, 0] + 1) * (ref.rect[:, 3] - ref.rect[:, 2] + 1) > 256) & (ref.valid > 0)
    assert big.sum() > 10
    check(run_gpu(ctx, scene, cam, sort_mode=sort_mode, sort_algo=sort_algo), ref)


@pytest.mark.parametrize("sort_algo", [0, 1, 2])
@pytest.mark.parametrize("sort_mode", [0, 1])
def test_elongated_gaussians_row_runs(ctx, sort_mode, sort_algo):
    """Thin rotated ellipses up to a few hundred pixels long: many tiles are hit only through a
    side edge, box widths are not multiples of the 8-tile run, and the largest take the
    one-CTA-per-Gaussian emission of the depth-ordered mode."""
    scene, cam = synth.random_small_scene(700, 17, 700, 610, log_scale_mu=-2.2, log_scale_sigma=0.5)
    rng = np.random.Generator(np.random.PCG64(5))
    s = scene.scales.astype(np.float64)
    axis = rng.integers(0, 3, scene.P)
    s *= 0.08
    s[np.arange(scene.P), axis] *= rng.uniform(10.0, 400.0, scene.P)
    scene.scales = s.astype(np.float32)
    # Conics this ill-conditioned carry binary32 rounding far above the image tolerance against
    # binary64 values, so the image is compared with the oracle's binary32 blend; the pair lists
    # are exact either way.
    ref = oracle.Frame(scene, cam, mode=32)
    ncand = (ref.rect[:, 1] - ref.rect[:, 0] + 1) * (ref.rect[:, 3] - ref.rect[:, 2] + 1) * (ref.valid > 0)
    assert (ncand > 1024).sum() >= 5 and ((ncand > 8) & (ncand < 200)).sum() >= 50
    check(run_gpu(ctx, scene, cam, sort_mode=sort_mode, sort_algo=sort_algo), ref)


@pytest.mark.parametrize("seed,mu", [(0, -1.6), (1, -3.0)])
def test_large_ellipses_every_tile_decision(ctx, seed, mu):
    """Thousands of ellipses from tens to hundreds of pixels across, axis ratios from 1 to about
    60 (on both sides of the count pass's switch to the full test for thin ellipses), centres on
    and off the image: every tile decision, taken by the band interval or by the binary32 test,
    must equal the oracle's binary32 test of that tile (the emission-order pair lists are
    compared element by element)."""
    scene, cam = synth.random_small_scene(2500, 40 + seed, 1920, 1080, log_scale_mu=mu, log_scale_sigma=0.6)
    rng = np.random.Generator(np.random.PCG64(60 + seed))
    s = scene.scales.astype(np.float64)
    s[np.arange(scene.P), rng.integers(0, 3, scene.P)] *= rng.uniform(0.015, 1.0, scene.P)
    scene.scales = s.astype(np.float32)
    ref = oracle.Frame(scene, cam, mode=32)
    ncand = (ref.rect[:, 1] - ref.rect[:, 0] + 1) * (ref.rect[:, 3] - ref.rect[:, 2] + 1) * (ref.valid > 0)
    assert (ncand > 400).sum() >= 100 and ref.N > 300_000
    check(run_gpu(ctx, scene, cam, sort_mode=0, max_pairs=1 << 24), ref)


@pytest.mark.parametrize("sort_mode", [0, 1])
def test_offscreen_centres_reaching_in(ctx, sort_mode):
    """Centres projected just outside every image edge, footprints from a few pixels to far
    across the border: the off-screen early-out must keep every Gaussian whose ellipse reaches a
    tile, and only those."""
    W, H = 240, 180
    scene, cam = synth.random_small_scene(1500, 23, W, H, log_scale_mu=-2.0, log_scale_sigma=1.0)
    rng = np.random.Generator(np.random.PCG64(29))
    m = scene.means.astype(np.float64)
    z = m[:, 2]
    fx, cx, cy = cam.fx, cam.cx, cam.cy
    side = rng.integers(0, 4, scene.P)
    off = rng.uniform(0.0, 120.0, scene.P)                  # pixels beyond the edge
    u = rng.uniform(-20.0, W + 20.0, scene.P)
    v = rng.uniform(-20.0, H + 20.0, scene.P)
    u = np.where(side == 0, -off, np.where(side == 1, W + off, u))
    v = np.where(side == 2, -off, np.where(side == 3, H + off, v))
    m[:, 0] = (u - cx) * z / fx
    m[:, 1] = (v - cy) * z / cam.fy
    scene.means = m.astype(np.float32)
    ref = oracle.Frame(scene, cam, mode=32)
    assert ref.visible > 100 and ref.N > 1000
    check(run_gpu(ctx, scene, cam, sort_mode=sort_mode), ref)


@pytest.mark.parametrize("sort_mode", [0, 1])
@pytest.mark.parametrize("cap", [False, True])
def test_3dgs_square_pairs(ctx, sort_mode, cap):
    """The paper's baseline pairs (every tile of the 3-sigma square, Eq. 1, Alg. 1-2): pair lists
    bit-exact against the oracle; under the 3-sigma cap the image equals the exact pairs' image
    bit for bit, with fewer pairs for the exact test."""
    scene, cam = synth.random_small_scene(3000, 41, 200, 150, log_scale_mu=-2.4, log_scale_sigma=1.0)
    kw = dict(cap_3sigma=cap)
    ref = oracle.Frame(scene, cam, oracle.opts(intersect=1, **kw), mode=64)
    res = run_gpu(ctx, scene, cam, dict(intersect=1, **kw), sort_mode=sort_mode)
    check(res, ref)
    ex = run_gpu(ctx, scene, cam, dict(intersect=0, **kw), sort_mode=sort_mode)
    assert ex["stats"]["pairs"] < res["stats"]["pairs"]
    if cap:
        assert np.array_equal(ex["rgb"], res["rgb"]) and np.array_equal(ex["T"], res["T"])


@pytest.mark.parametrize("sort_algo", [0, 1, 2])
@pytest.mark.parametrize("sort_mode", [0, 1])
def test_empty_view(ctx, sort_mode, sort_algo):
    scene, cam = synth.random_small_scene(1000, 14, 64, 48)
    cam.R = (-np.eye(3)).astype(np.float32)        # looking the other way
    cam.R[1, 1] = 1.0
    ref = oracle.Frame(scene, cam, oracle.opts(bg=(0.2, 0.3, 0.4)), mode=64)
    assert ref.N == 0
    res = run_gpu(ctx, scene, cam, dict(bg=(0.2, 0.3, 0.4)), sort_mode=sort_mode, sort_algo=sort_algo)
    check(res, ref)
    assert np.allclose(res["rgb"][0], np.float32(0.2)) and np.all(res["T"] == 1.0)


@pytest.mark.parametrize("sort_algo", [0, 1, 2])
@pytest.mark.parametrize("sort_mode", [0, 1])
def test_single_gaussian_and_tiny_scene_sizes(ctx, sort_mode, sort_algo):
    for P in (1, 255, 257):
        scene, cam = synth.random_small_scene(P, 15 + P, 64, 64, log_scale_mu=-2.0)
        ref = oracle.Frame(scene, cam, mode=64)
        check(run_gpu(ctx, scene, cam, sort_mode=sort_mode, sort_algo=sort_algo), ref)


@pytest.mark.parametrize("sort_algo", [0, 2])
@pytest.mark.parametrize("sort_mode", [0, 1])
def test_pair_overflow_is_reported(ctx, sort_mode, sort_algo):
    scene, cam = synth.random_small_scene(2000, 16, 128, 96, log_scale_mu=-2.4)
    ref = oracle.Frame(scene, cam, mode=32)
    res = run_gpu(ctx, scene, cam, max_pairs=ref.N // 3, sort_mode=sort_mode, sort_algo=sort_algo)
    assert res["stats"]["status"] == -3, res["stats"]
    assert res["stats"]["pairs"] == ref.N
    # the frame stays usable
    check(run_gpu(ctx, scene, cam), oracle.Frame(scene, cam, mode=64))


def test_deterministic_graph_replay_and_modes_agree(ctx):
    scene, cam = synth.random_small_scene(4000, 17, 160, 120, log_scale_mu=-2.5)
    a = run_gpu(ctx, scene, cam, sort_mode=0)
    b = run_gpu(ctx, scene, cam, sort_mode=0)
    c = run_gpu(ctx, scene, cam, graph=True, sort_mode=0)
    d = run_gpu(ctx, scene, cam, sort_mode=1)
    e = run_gpu(ctx, scene, cam, graph=True, sort_mode=1)
    for k in ("rgb", "T", "last", "keys", "vals", "starts"):
        for other in (b, c, d, e):
            assert np.array_equal(a[k], other[k]), k


@pytest.mark.parametrize("variant", range(6))
def test_blend_variants_bit_identical(ctx, variant):
    """Every launch shape evaluates each pixel's list identically: outputs equal bit for bit,
    and match the oracle."""
    scene, cam = synth.random_small_scene(5000, 23, 200, 150, log_scale_mu=-2.6, log_scale_sigma=1.0)
    base = run_gpu(ctx, scene, cam, variant=2)
    res = run_gpu(ctx, scene, cam, variant=variant)
    for k in ("rgb", "T", "last"):
        assert np.array_equal(base[k], res[k]), k
    check(res, oracle.Frame(scene, cam, mode=64))


def test_counting_blend_same_image_and_oracle_walk_count(ctx):
    """The instrumented blend gives the same image, and its count of (pixel, entry) pairs walked
    before early stop equals the oracle's (up to early-stop near ties)."""
    scene, cams = synth.load_config("tiny")
    cam = cams[0]
    ref = oracle.Frame(scene, cam, mode=32)
    sc = gs.Scene.from_numpy(ctx, scene)
    fr = gs.Frame(ctx, scene.P, 1 << 20, cam.width, cam.height)
    a, _, _ = fr.render(sc, cam)
    fr.gs_frame_set_counting(True)
    b, _, _ = fr.render(sc, cam)
    st = fr.stats()
    assert torch.equal(a, b)
    assert abs(st["evaluations"] - ref.evals) <= 1e-4 * ref.evals
    assert 0 < st["contributions"] <= st["evaluations"]


def test_autotune_picks_a_shape_and_caches_it(ctx, tmp_path):
    scene, cams = synth.load_config("tiny")
    sc = gs.Scene.from_numpy(ctx, scene)
    fr = gs.Frame(ctx, scene.P, 1 << 20, 256, 256)
    ref, _, _ = fr.render(sc, cams[0])
    cache = tmp_path / "tune.txt"
    t1 = fr.gs_autotune(sc, cams, cache_path=cache)
    assert 0 <= t1["blend_variant"] < 6 and t1["sort_mode"] in (0, 1) and t1["sort_algo"] in (0, 1, 2)
    assert fr.gs_frame_get_tuning() == t1
    line = cache.read_text().strip().split()
    assert line[0] == "gs-autotune-v2"
    assert [int(x) for x in line[-3:]] == [t1["blend_variant"], t1["sort_mode"], t1["sort_algo"]]
    fr2 = gs.Frame(ctx, scene.P, 1 << 20, 256, 256)
    assert fr2.gs_autotune(sc, cams, cache_path=cache) == t1          # served from the cache
    out, _, _ = fr2.render(sc, cams[0])
    assert torch.equal(out, ref)


def test_graph_replay_many_cameras(ctx):
    scene, cams = synth.load_config("tiny")
    sc = gs.Scene.from_numpy(ctx, scene)
    fr = gs.Frame(ctx, scene.P, 1 << 20, 256, 256)
    fr.gs_frame_use_graph(True)
    s = torch.cuda.Stream()
    rng = np.random.default_rng(0)
    for k in range(4):
        C = rng.normal(0, 1, 3)
        C = 3.2 * C / np.linalg.norm(C)
        cam = synth.look_at(C, (0, 0, 0), 256, 256, 60.0)
        with torch.cuda.stream(s):
            rgb, T, last = fr.render(sc, cam)
        s.synchronize()
        ref = oracle.Frame(scene, cam, mode=64)
        err = np.abs(rgb.double().cpu().numpy() - ref.rgb)
        assert err.max() <= RGB_MAX and fr.stats()["pairs"] == ref.N


@pytest.mark.parametrize("n", [0, 1, 5, 3071, 3072, 3073, 100_003, 1_000_001])
def test_sort_pairs_primitive(ctx, n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 2 ** 63, n, dtype=np.int64).astype(np.uint64) * np.uint64(2)
    keys[: n // 3] = keys[n // 2: n // 2 + n // 3]       # duplicates: stability is observable
    keys ^= rng.integers(0, 2, n).astype(np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    order = np.lexsort((vals, keys))
    k_t = torch.from_numpy(keys.view(np.int64)).cuda()
    v_t = torch.from_numpy(vals.view(np.int32)).cuda()
    ks, vs = gs.gs_sort_pairs(ctx, k_t, v_t, 64)
    torch.cuda.synchronize()
    assert np.array_equal(ks.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(vs.cpu().numpy().view(np.uint32), vals[order])


@pytest.mark.parametrize("end_bit", [8, 13, 40, 47])
def test_sort_pairs_partial_bits(ctx, end_bit):
    n = 200_000
    rng = np.random.default_rng(end_bit)
    keys = rng.integers(0, 2 ** min(end_bit, 62), n, dtype=np.int64).astype(np.uint64)
    vals = np.arange(n, dtype=np.uint32)
    order = np.lexsort((vals, keys))
    ks, vs = gs.gs_sort_pairs(ctx, torch.from_numpy(keys.view(np.int64)).cuda(),
                              torch.from_numpy(vals.view(np.int32)).cuda(), end_bit)
    assert np.array_equal(ks.cpu().numpy().view(np.uint64), keys[order])
    assert np.array_equal(vs.cpu().numpy().view(np.uint32), vals[order])
