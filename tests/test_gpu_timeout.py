"""The failure path of the bounded waits, made to happen on purpose without faulting anything.

Kernels that wait on other thread blocks (the onesweep look-back between tiles, the grid barriers
of the fused sort) give up after gs_set_wait_limit polls, flag a device status and return; every
kernel launched after that which would read the incomplete output writes nothing.  Here the limit
is set to one poll, so that such a wait runs out in an ordinary sort or render: the status must
come back as GS_ERR_DEVICE_TIMEOUT, and after the default limit is restored the same objects must
sort and render correctly again (the context stays usable).  A wait that gives up early leaves
the result wrong but every write in bounds (a tile's partial prefix is at most its true one)."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_2408_07967_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2408_07967_gb300 as gs  # noqa: E402

TIMEOUT = -5


@pytest.fixture(scope="module")
def ctx():
    from paper_2408_07967_gb300 import build
    build.build()
    c = gs.Context(0)
    yield c
    gs.lib().gs_set_wait_limit(0)


def stream_ptr():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def random_pairs(n, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2 ** 62, n, dtype=np.int64)
    keys[: n // 4] = keys[n // 2: n // 2 + n // 4]
    vals = rng.permutation(n).astype(np.int32)
    return keys, vals


def stable_sorted(keys, vals, end_bit):
    k = keys.view(np.uint64)
    masked = k & np.uint64((1 << end_bit) - 1) if end_bit < 64 else k
    order = np.argsort(masked, kind="stable")
    return keys[order], vals[order]


def test_wait_limit_roundtrip(ctx):
    L = gs.lib()
    assert L.gs_get_wait_limit() == 1 << 22
    L.gs_set_wait_limit(7)
    assert L.gs_get_wait_limit() == 7
    L.gs_set_wait_limit(0)
    assert L.gs_get_wait_limit() == 1 << 22


def test_sort_gives_up_and_recovers(ctx):
    keys, vals = random_pairs(1_500_001, 3)
    ek, ev = stable_sorted(keys, vals, 64)
    kd, vd = torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda()
    seen = False
    try:
        gs.lib().gs_set_wait_limit(1)
        for _ in range(8):
            ok, ov = gs.gs_sort_pairs(ctx, kd.clone(), vd.clone(), 64)
            st = gs.lib().gs_sort_pairs_status(ctx.h, stream_ptr())
            assert st in (0, TIMEOUT), st
            if st == TIMEOUT:
                assert b"gave up" in gs.lib().gs_last_error()
                seen = True
                break
            assert np.array_equal(ok.cpu().numpy(), ek) and np.array_equal(ov.cpu().numpy(), ev)
    finally:
        gs.lib().gs_set_wait_limit(0)
    assert seen, "a one-poll limit never ran out over eight sorts of 1.5M pairs"
    ok, ov = gs.gs_sort_pairs(ctx, kd.clone(), vd.clone(), 64)
    assert gs.lib().gs_sort_pairs_status(ctx.h, stream_ptr()) == 0
    assert np.array_equal(ok.cpu().numpy(), ek) and np.array_equal(ov.cpu().numpy(), ev)


@pytest.mark.parametrize("sort_algo", [0, 2])
def test_frame_reports_timeout_then_renders(ctx, sort_algo):
    """A whole render whose sort gives up reports GS_ERR_DEVICE_TIMEOUT in the frame's stats (ranges
    and blend write nothing); with the default limit back, the next render of the same frame
    matches the oracle."""
    scene, cam = synth.random_small_scene(150_000, 11, 1280, 720, log_scale_mu=-4.0)
    sc = gs.Scene.from_numpy(ctx, scene)
    fr = gs.Frame(ctx, scene.P, 1 << 23, cam.width, cam.height)
    fr.gs_frame_set_tuning(sort_mode=0, sort_algo=sort_algo)
    seen = False
    try:
        gs.lib().gs_set_wait_limit(1)
        for _ in range(8):
            fr.render(sc, cam)
            st = fr.stats()
            assert st["status"] in (0, TIMEOUT), st
            if st["status"] == TIMEOUT:
                seen = True
                break
    finally:
        gs.lib().gs_set_wait_limit(0)
    assert seen
    rgb, T, last = fr.render(sc, cam)
    torch.cuda.synchronize()
    st = fr.stats()
    assert st["status"] == 0
    ref = oracle.Frame(scene, cam, mode=64)
    assert st["pairs"] == ref.N
    keys, vals = fr.pairs(1)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), ref.keys)
    assert np.array_equal(vals.cpu().numpy().view(np.uint32), ref.vals)
    err = np.abs(rgb.double().cpu().numpy() - ref.rgb)
    assert err.max() <= 2e-3 and err.mean(axis=(1, 2)).max() <= 1e-5
    fr.close()
    sc.close()
