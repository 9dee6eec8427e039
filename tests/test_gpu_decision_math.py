"""Exhaustive GPU-vs-host checks of the binary32 arithmetic whose bits decide the pair set.

The threshold t = 2 ln(alpha0 / tau) of Eq. 3 (Section 4.1) decides which tiles a Gaussian
pairs with, and for raw parameters e^x decides the scales (exp of the log-scales) and the
opacities (1 / (1 + e^-logit)).  The device and the oracle each implement ln and exp from the same
published method in their own code; here every binary32 input of each domain goes through both
and the results must be identical bit for bit:
  * t for every alpha0 in (tau, 1] (about 6.7e7 values; alpha0 <= tau is culled first);
  * e^x and the sigmoid for every x with 2^-30 <= |x| <= 32 (about 5.9e8 values each), which
    covers log-scales of scenes from millimetres to tens of metres and every logit whose
    opacity is not rounded to 0 or 1.
Inputs are made from their bit patterns in chunks of 2^24; both sides see the same floats."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2408_07967_gb300 as gs  # noqa: E402

CHUNK = 1 << 24
TAU = np.float32(1.0 / 255.0)


@pytest.fixture(scope="module")
def lib():
    from paper_2408_07967_gb300 import build
    build.build()
    oracle.build()
    return gs.lib()


def bits(x):
    return int(np.array([x], np.float32).view(np.uint32)[0])


def compare_range(fn, lo_bits, hi_bits, param=0.0, sign=1.0):
    """Every float whose bit pattern lies in [lo_bits, hi_bits] (times `sign`) through the device
    and the oracle; returns the number of values compared."""
    total = 0
    for b0 in range(lo_bits, hi_bits + 1, CHUNK):
        b1 = min(hi_bits + 1, b0 + CHUNK)
        x = np.arange(b0, b1, dtype=np.uint32).view(np.float32)
        if sign < 0:
            x = -x
        y_dev = gs.gs_eval_decision_math(fn, torch.from_numpy(x).cuda(), param).cpu().numpy()
        y_ref = oracle.eval_decision_math(fn, x, param)
        same = y_dev.view(np.uint32) == y_ref.view(np.uint32)
        if not same.all():
            i = int(np.flatnonzero(~same)[0])
            pytest.fail(f"fn {fn}: x = {x[i]!r} ({x[i].view(np.uint32):#010x}): device {y_dev[i]!r}, "
                        f"oracle {y_ref[i]!r}; {int((~same).sum())} mismatches in the chunk")
        total += x.shape[0]
    return total


def test_threshold_bitwise_every_alpha0_above_tau(lib):
    n = compare_range(0, bits(TAU) + 1, bits(1.0), param=float(TAU))
    assert n == bits(1.0) - bits(TAU)
    assert n > 6.5e7


@pytest.mark.parametrize("fn", [1, 2], ids=["exp", "sigmoid"])
def test_activation_bitwise_whole_domain(lib, fn):
    lo, hi = bits(2.0 ** -30), bits(32.0)
    n = compare_range(fn, lo, hi) + compare_range(fn, lo, hi, sign=-1.0)
    assert n == 2 * (hi - lo + 1)


def test_decision_math_argument_checks(lib):
    x = torch.zeros(4, device="cuda")
    with pytest.raises(gs.GsError):
        gs.gs_eval_decision_math(3, x)
    assert gs.lib().gs_eval_decision_math(0, None, None, 0, 1.0, None) == 0
    assert gs.lib().gs_eval_decision_math(0, None, None, 5, 1.0, None) == -1
