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


def test_noalloc_sort_matches_allocating_sort_twice(ctx):
    for n, end_bit, seed in ((1_500_001, 64, 1), (MAX_PAIRS, 47, 2)):
        keys, vals = random_pairs(n, seed)
        ref_k, ref_v = gs.gs_sort_pairs(ctx, keys.clone(), vals.clone(), end_bit)
        out_k, out_v = noalloc_sort(keys.clone(), vals.clone(), end_bit)
        torch.cuda.synchronize()
        assert torch.equal(out_k, ref_k) and torch.equal(out_v, ref_v)


def test_noalloc_sort_rejects_oversize(ctx):
    in_tmp = C.c_int32(0)
    st = gs.lib().gs_sort_pairs_noalloc(None, None, None, None, MAX_PAIRS + 1, 64, C.byref(in_tmp), None)
    assert st == -7
    assert b"maximum" in gs.lib().gs_last_error()
