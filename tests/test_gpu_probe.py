"""The measured ALU ceilings used beside the derived peak in the line sum's roofline."""
import pytest

pytestmark = pytest.mark.gpu


def test_alu_probe_is_plausible():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_cs_0703028_gb300 as rt
    r = rt.alu_probe()
    props = torch.cuda.get_device_properties(0)
    # 128 FP32 lanes per SM at no more than 2.2 GHz bound the FMA rate from above;
    # a full-occupancy chain kernel reaches well over half of it at any clock above 1.2 GHz
    top = props.multi_processor_count * 128 * 2.2e9
    assert 0.5 * top * (1.2 / 2.2) < r["fma_lane_ops_per_s"] < top
    assert 0 < r["rcp_lane_ops_per_s"] < r["fma_lane_ops_per_s"]
