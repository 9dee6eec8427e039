"""Batched rendering through the C ABI: a batch mixing two resident scenes and several image sizes
renders every request bit-identically to rendering it alone (each request's pairs and arithmetic
are request-local), in both pair orderings; and one request matches the oracle."""
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
    sa, ca = synth.random_small_scene(6000, 41, 160, 120, log_scale_mu=-2.6, log_scale_sigma=1.0)
    sb, cb = synth.random_small_scene(3000, 42, 96, 64, log_scale_mu=-2.2, log_scale_sigma=0.8)
    A = gs.Scene.from_numpy(ctx, sa)
    B = gs.Scene.from_numpy(ctx, sb)
    cams = [ca, cb, synth.look_at((0.2, 0.1, 0.0), (0.0, 0.0, 3.0), 200, 90), cb,
            synth.look_at((-0.3, 0.0, 0.2), (0.1, 0.0, 2.5), 33, 47)]
    scenes = [A, B, A, A, B]
    return ctx, sa, sb, A, B, scenes, cams


@pytest.mark.parametrize("sort_mode", [0, 1])
def test_batch_equals_alone(setup, sort_mode):
    ctx, sa, sb, A, B, scenes, cams = setup
    total_px = sum(c.width * c.height for c in cams)
    fb = gs.Frame(ctx, sum(s.P for s in scenes), 1 << 22, 1024, 1024)
    fb.gs_frame_set_tuning(sort_mode=sort_mode)
    outs = fb.gs_render_batch(scenes, cams, want_T=True, want_last=True)
    torch.cuda.synchronize()
    for s, c, (rgb, T, last) in zip(scenes, cams, outs):
        fa = gs.Frame(ctx, s.P, 1 << 22, c.width, c.height)
        fa.gs_frame_set_tuning(sort_mode=sort_mode)
        r1, T1, l1 = fa.render(s, c)
        assert torch.equal(rgb, r1) and torch.equal(T, T1) and torch.equal(last, l1)
    assert total_px > 0


def test_batch_request_matches_oracle(setup):
    ctx, sa, sb, A, B, scenes, cams = setup
    fb = gs.Frame(ctx, sum(s.P for s in scenes), 1 << 22, 1024, 1024)
    outs = fb.gs_render_batch(scenes, cams)
    ref = oracle.Frame(sa, cams[2], mode=64)
    err = np.abs(outs[2][0].double().cpu().numpy() - ref.rgb)
    assert err.max() <= 2e-3 and err.mean(axis=(1, 2)).max() <= 1e-5


def test_batch_capacity_errors(setup):
    ctx, sa, sb, A, B, scenes, cams = setup
    small = gs.Frame(ctx, sa.P, 1 << 20, 200, 200)
    with pytest.raises(gs.GsError) as e:
        small.gs_render_batch([A, B], cams[:2])
    assert e.value.status == -7
    with pytest.raises(gs.GsError):
        small.gs_render_batch([A] * 17, [cams[0]] * 17)
