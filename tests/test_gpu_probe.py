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


def test_bounded_wait_gives_up_and_reports_timeout():
    # Failure detection without a fault: an mbarrier wait that nothing completes gives up
    # after its iteration limit, the block leaves, the host reads RT_E_TIMEOUT from the
    # status word, and the context stays usable (a kappa build afterwards succeeds).
    import ctypes as ct
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_cs_0703028_gb300 as rt
    import synth
    L = rt.lib()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert L.rt_wait_probe(1000, 0, ct.c_void_p(st.data_ptr()), None) == rt.RT_OK
    assert L.rt_status_read(ct.c_void_p(st.data_ptr()), None) == rt.RT_E_TIMEOUT
    st.zero_()
    assert L.rt_wait_probe(1000, 1, ct.c_void_p(st.data_ptr()), None) == rt.RT_OK
    assert L.rt_status_read(ct.c_void_p(st.data_ptr()), None) == rt.RT_OK
    assert L.rt_wait_probe(0, 0, ct.c_void_p(st.data_ptr()), None) == rt.RT_E_INVAL
    c0 = synth.config(0)
    kap = rt.build_kappa(c0.lines, c0.spec)
    torch.cuda.synchronize()
    assert bool(torch.all(kap > 0))
