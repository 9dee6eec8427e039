"""gs_measure_alu_peaks: the measured FP32 FMA and ex2 rates that divide the blend's work."""
import pytest

from conftest import cuda_available

pytestmark = pytest.mark.gpu


@pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")
def test_alu_peaks_plausible():
    import paper_2408_07967_gb300 as gs
    import torch
    props = torch.cuda.get_device_properties(0)
    r = gs.gs_measure_alu_peaks(0, 50.0)
    assert r["sm_count"] == props.multi_processor_count
    # 128 FP32 lanes per SM at 0.5 .. 3 GHz bounds the FMA rate; ex2 runs on fewer lanes
    lo = r["sm_count"] * 128 * 0.5e9 / 1e12
    hi = r["sm_count"] * 128 * 3.0e9 / 1e12
    assert lo < r["fma_tops"] < hi, r
    assert 0 < r["ex2_tops"] < r["fma_tops"], r
    assert 20.0 < r["fma_ms"] < 500.0 and 20.0 < r["ex2_ms"] < 500.0, r


@pytest.mark.skipif(not cuda_available(), reason="needs a CUDA GPU")
def test_alu_peaks_bad_args():
    import paper_2408_07967_gb300 as gs
    with pytest.raises(gs.GsError):
        gs.gs_measure_alu_peaks(1 << 20, 10.0)
