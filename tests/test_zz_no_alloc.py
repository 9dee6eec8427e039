"""The allocation-free sort entry point, for callers that must not allocate device memory (code
embedded in a host application that owns the device-memory budget, where cudaMalloc/cudaFree could
synchronise the device or fail).  It is checked through the C ABI against the allocating entry
point gs_sort_pairs, on two calls in a row (the second reuses the fixed scratch the first left
behind), and it must refuse sizes beyond its stated maximum.  A sort is exact, so the comparison
is bit for bit.  This file is collected last so that a failure here leaves every other test run."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2408_07967_gb300 as gs  # noqa: E402

MAX_PAIRS = 1 << 21


@pytest.fixture(scope="module")
def ctx():
    from paper_2408_07967_gb300 import build
    build.build()
    return gs.Context(0)


def noalloc_sort(keys, vals, end_bit):
    kt, vt = torch.empty_like(keys), torch.empty_like(vals)
    in_tmp = C.c_int32(-1)
    st = gs.lib().gs_sort_pairs_noalloc(C.c_void_p(keys.data_ptr()), C.c_void_p(vals.data_ptr()),
                                        C.c_void_p(kt.data_ptr()), C.c_void_p(vt.data_ptr()), keys.numel(),
                                        end_bit, C.byref(in_tmp), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, gs.lib().gs_last_error()
    return (kt, vt) if in_tmp.value == 1 else (keys, vals)


def random_pairs(n, seed):
    rng = np.random.default_rng(seed)
    keys = rng.integers(0, 2 ** 62, n, dtype=np.int64)
    keys[: n // 4] = keys[n // 2: n // 2 + n // 4]          # duplicate keys: stability shows
    vals = rng.permutation(n).astype(np.int32)
    return torch.from_numpy(keys).cuda(), torch.from_numpy(vals).cuda()


def status():
    return gs.lib().gs_sort_pairs_noalloc_status(C.c_void_p(torch.cuda.current_stream().cuda_stream))


def host_stable_sort(keys, vals, end_bit):
    """Stable sort by key bits [0, end_bit) on the host (numpy), the reference for exactness."""
    k = keys.cpu().numpy().view(np.uint64)
    masked = k & np.uint64((1 << end_bit) - 1) if end_bit < 64 else k
    order = np.argsort(masked, kind="stable")
    return k[order], vals.cpu().numpy()[order]


def test_noalloc_sort_matches_allocating_sort_twice(ctx):
    for n, end_bit, seed in ((1_500_001, 64, 1), (MAX_PAIRS, 47, 2)):
        keys, vals = random_pairs(n, seed)
        ref_k, ref_v = gs.gs_sort_pairs(ctx, keys.clone(), vals.clone(), end_bit)
        out_k, out_v = noalloc_sort(keys.clone(), vals.clone(), end_bit)
        torch.cuda.synchronize()
        assert status() == 0
        assert torch.equal(out_k, ref_k) and torch.equal(out_v, ref_v)


@pytest.mark.parametrize("n,end_bit", [(0, 64), (1, 64), (5000, 40), (3072 * 7 + 11, 33), (200_003, 40)])
def test_noalloc_sort_against_host_stable_sort(ctx, n, end_bit):
    """Odd pass counts (end_bit 40 and 33 take five passes, leaving the result in the ping-pong
    buffers), the empty input and sizes that are not a whole number of 3072-pair tiles, each
    against numpy's stable sort of the masked keys."""
    keys, vals = random_pairs(n, 40 + n % 97)
    ek, ev = host_stable_sort(keys, vals, end_bit)
    out_k, out_v = noalloc_sort(keys.clone(), vals.clone(), end_bit)
    torch.cuda.synchronize()
    if n:
        assert status() == 0
    got_k = out_k.cpu().numpy().view(np.uint64)
    assert np.array_equal(got_k, ek) and np.array_equal(out_v.cpu().numpy(), ev)


def test_noalloc_sort_reports_a_wait_that_gave_up(ctx):
    """With the bounded waits cut to one poll, a sort's look-back gives up: the status call
    reports GS_ERR_DEVICE_TIMEOUT, and with the default limit back the next call sorts correctly."""
    keys, vals = random_pairs(1_500_001, 9)
    ek, ev = host_stable_sort(keys, vals, 64)
    seen = False
    try:
        gs.lib().gs_set_wait_limit(1)
        for _ in range(8):
            noalloc_sort(keys.clone(), vals.clone(), 64)
            st = status()
            assert st in (0, -5), st
            if st == -5:
                seen = True
                break
    finally:
        gs.lib().gs_set_wait_limit(0)
    assert seen
    out_k, out_v = noalloc_sort(keys.clone(), vals.clone(), 64)
    assert status() == 0
    assert np.array_equal(out_k.cpu().numpy().view(np.uint64), ek) and np.array_equal(out_v.cpu().numpy(), ev)


def test_noalloc_sort_rejects_oversize(ctx):
    in_tmp = C.c_int32(0)
    st = gs.lib().gs_sort_pairs_noalloc(None, None, None, None, MAX_PAIRS + 1, 64, C.byref(in_tmp), None)
    assert st == -7
    assert b"maximum" in gs.lib().gs_last_error()
