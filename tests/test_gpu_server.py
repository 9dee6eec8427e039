"""The serving loop through the C ABI: requests of mixed scenes and sizes submitted together are
batched (continuous batching over several slots), every image equals the standalone render bit for
bit, admission by pair-buffer memory splits batches that do not fit and fails a request that alone
exceeds the capacity, and the plain baseline loop runs one request at a time."""
import numpy as np
import pytest

import oracle
from paper_2408_07967_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2408_07967_gb300 as gs  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    from paper_2408_07967_gb300 import build
    build.build()
    ctx = gs.Context(0)
    sa, ca = synth.random_small_scene(6000, 51, 160, 120, log_scale_mu=-2.6, log_scale_sigma=1.0)
    sb, cb = synth.random_small_scene(3000, 52, 96, 64, log_scale_mu=-2.2, log_scale_sigma=0.8)
    A = gs.Scene.from_numpy(ctx, sa)
    B = gs.Scene.from_numpy(ctx, sb)
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(24):
        sc = (A, B)[i % 2]
        W, H = [(160, 120), (96, 64), (200, 90), (64, 64)][i % 4]
        C = rng.normal(0, 0.2, 3)
        cam = synth.look_at(C, (rng.normal(0, 0.2), rng.normal(0, 0.2), 3.0), W, H)
        reqs.append((sc, cam))
    alone = []
    for sc, cam in reqs:
        fr = gs.Frame(ctx, sc.P, 1 << 22, cam.width, cam.height)
        rgb, _, _ = fr.render(sc, cam)
        alone.append(rgb.cpu())
    return ctx, A, B, reqs, alone


def run(server, reqs, release=None):
    outs, tickets = [], []
    for sc, cam in reqs:
        buf = torch.empty((3, cam.height, cam.width), dtype=torch.float32).pin_memory()
        outs.append(buf)
        tickets.append(server.gs_server_submit(sc, cam, buf))
    if release is not None:
        assert release.stats()["pending"] == len(reqs)      # held: nothing admitted yet
        release.gs_server_hold(False)
    stats = [server.gs_server_wait(t, 60000) for t in tickets]
    return outs, stats


@pytest.mark.parametrize("sort_mode", [0, 1])
def test_batched_results_equal_alone(setup, sort_mode):
    ctx, A, B, reqs, alone = setup
    sv = gs.Server(ctx, slots=3, max_batch=8, pair_capacity=1 << 22, max_gaussians=1 << 20, max_width=256,
                   max_height=256, sort_mode=sort_mode)
    sv.gs_server_hold(True)          # let the whole burst queue, so that it runs in full batches
    outs, stats = run(sv, reqs, release=sv)
    assert all(s["status"] == 0 for s in stats)
    for o, a in zip(outs, alone):
        assert torch.equal(o, a)
    assert max(s["batch_size"] for s in stats) > 1           # requests were batched
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["batched_requests"] == len(reqs)
    assert all(s["done_s"] >= s["admit_s"] >= s["arrival_s"] for s in stats)
    sv.close()


def test_served_images_match_the_oracle(setup):
    """Every image of a batched burst against the oracle's binary64 render of that request: max-abs
    2e-3 and mean-abs 1e-5 per channel (the forward parity bars)."""
    ctx, A, B, reqs, alone = setup
    scenes = {id(A): None, id(B): None}
    sa, _ = synth.random_small_scene(6000, 51, 160, 120, log_scale_mu=-2.6, log_scale_sigma=1.0)
    sb, _ = synth.random_small_scene(3000, 52, 96, 64, log_scale_mu=-2.2, log_scale_sigma=0.8)
    scenes[id(A)], scenes[id(B)] = sa, sb
    sv = gs.Server(ctx, slots=3, max_batch=8, pair_capacity=1 << 22, max_gaussians=1 << 20, max_width=256,
                   max_height=256)
    sv.gs_server_hold(True)
    outs, stats = run(sv, reqs[:12], release=sv)
    assert max(s["batch_size"] for s in stats) > 1
    for (sc, cam), o, s in zip(reqs[:12], outs, stats):
        assert s["status"] == 0
        ref = oracle.Frame(scenes[id(sc)], cam, mode=64)
        assert s["pairs"] == ref.N
        err = np.abs(o.double().numpy() - ref.rgb)
        assert err.max() <= 2e-3 and err.mean(axis=(1, 2)).max() <= 1e-5, (err.max(), err.mean(axis=(1, 2)))
    sv.close()


def test_admission_by_pair_memory(setup):
    ctx, A, B, reqs, alone = setup
    # capacity below the largest request's pairs: that one fails, the others are split into fitting batches
    fr = gs.Frame(ctx, A.P, 1 << 22, 200, 120)
    pairs = []
    for sc, cam in reqs:
        f = gs.Frame(ctx, sc.P, 1 << 22, cam.width, cam.height)
        f.render(sc, cam)
        pairs.append(f.stats()["pairs"])
    cap = int(sorted(pairs)[-2]) + 1          # the largest request does not fit
    sv = gs.Server(ctx, slots=2, max_batch=8, pair_capacity=cap, max_gaussians=1 << 20, max_width=256, max_height=256)
    outs, stats = run(sv, reqs)
    big = int(np.argmax(pairs))
    for i, (o, a, s) in enumerate(zip(outs, alone, stats)):
        if pairs[i] > cap:
            assert s["status"] == -3 and s["pairs"] == pairs[i]
        else:
            assert s["status"] == 0 and torch.equal(o, a)
            assert s["pairs"] == pairs[i]
    assert stats[big]["status"] == -3
    sv.close()


def test_plain_loop_one_at_a_time(setup):
    ctx, A, B, reqs, alone = setup
    sv = gs.Server(ctx, plain=True, pair_capacity=1 << 22, max_gaussians=1 << 20, max_width=256, max_height=256)
    outs, stats = run(sv, reqs[:8])
    assert all(s["status"] == 0 and s["batch_size"] == 1 for s in stats)
    for o, a in zip(outs, alone[:8]):
        assert torch.equal(o, a)
    done = sorted(s["done_s"] for s in stats)
    admits = sorted(s["admit_s"] for s in stats)
    assert all(admits[i + 1] >= done[i] - 1e-6 for i in range(7))   # strictly one after another
    sv.close()


def test_plain_loop_reports_overflow(setup):
    """The one-at-a-time loop renders without an admission pass: a request whose pairs exceed the
    capacity must still fail (from the frame's device status), and the others succeed."""
    ctx, A, B, reqs, alone = setup
    pairs = []
    for sc, cam in reqs[:8]:
        f = gs.Frame(ctx, sc.P, 1 << 22, cam.width, cam.height)
        f.render(sc, cam)
        pairs.append(f.stats()["pairs"])
    cap = int(sorted(pairs)[-2]) + 1
    sv = gs.Server(ctx, plain=True, pair_capacity=cap, max_gaussians=1 << 20, max_width=256, max_height=256)
    outs, stats = run(sv, reqs[:8])
    for i, (o, a, s) in enumerate(zip(outs, alone[:8], stats)):
        assert s["pairs"] == pairs[i]
        if pairs[i] > cap:
            assert s["status"] == -3
        else:
            assert s["status"] == 0 and torch.equal(o, a)
    sv.close()


def test_router_over_two_servers(setup):
    """The router's server backend: two servers (both on this GPU, independent of each other)
    hold scene A, only the second holds scene B; every routed request renders bit-identical to
    rendering it alone and lands where its scene is."""
    ctx, A, B, reqs, alone = setup
    kw = dict(slots=2, max_batch=4, pair_capacity=1 << 22, max_gaussians=1 << 20, max_width=256, max_height=256)
    s0, s1 = gs.Server(ctx, **kw), gs.Server(ctx, **kw)
    r = gs.Router.on_servers([s0, s1])
    r.place_scene(0, 0, A)
    r.place_scene(0, 1, A)
    r.place_scene(1, 1, B)
    outs, tickets = [], []
    for sc, cam in reqs:
        buf = torch.empty((3, cam.height, cam.width), dtype=torch.float32).pin_memory()
        outs.append(buf)
        tickets.append(r.submit(0 if sc is A else 1, cam, buf))
    placed = []
    for t in tickets:
        st, rep = r.wait(t, 60000)
        assert st["status"] == 0
        placed.append(rep)
    for (sc, cam), o, a, rep in zip(reqs, outs, alone, placed):
        assert torch.equal(o, a)
        if sc is B:
            assert rep == 1
    assert 0 in placed and all(r.outstanding(i) == (0, 0) for i in range(2))
    r.close()
    s0.close()
    s1.close()


def test_wait_timeout_and_bad_requests(setup):
    ctx, A, B, reqs, alone = setup
    sv = gs.Server(ctx, slots=1, max_batch=2, pair_capacity=1 << 22, max_gaussians=1 << 20, max_width=128,
                   max_height=128)
    big = synth.look_at((0, 0, 0), (0, 0, 3), 512, 512)
    buf = torch.empty((3, 512, 512)).pin_memory()
    with pytest.raises(gs.GsError):
        sv.gs_server_submit(A, big, buf)
    sv.close()
