"""Measurement and self-test entry points: rsi_fp32_peak, the FP32 ceiling
the benchmark compares the traversal's arithmetic with (the measured rate
must be plausible for the device: well above zero, not above its FP32 units
at the maximum clock), and rsi_selftest_wait, the bounded device-side wait
running out."""
import pytest
import torch

import paper_2209_02878_gb300 as rsi

pytestmark = pytest.mark.gpu


def test_fp32_peak_is_plausible():
    props = torch.cuda.get_device_properties(0)
    # 128 FP32 lanes per SM, 2 flops per FMA, at most 2.2 GHz
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12
    v = rsi.fp32_peak(1 << 16)
    assert 0.2 * ceiling < v <= ceiling, (v, ceiling)
    # the rate does not depend on the length of the run
    v2 = rsi.fp32_peak(1 << 17)
    assert abs(v2 - v) <= 0.15 * v, (v, v2)


def test_bounded_wait_times_out_and_the_context_survives():
    """The bounded wait that the streamed host path uses, on a flag that
    nothing sets: it gives up, latches RSI_ERR_TIMEOUT, and the device is
    still usable afterwards."""
    import ctypes as C

    from paper_2209_02878_gb300 import _abi, synth
    lib = _abi.load()
    st = C.c_int32(-1)
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.rsi_selftest_wait(2000, s, C.byref(st)) == _abi.RSI_OK
    assert st.value == _abi.RSI_ERR_TIMEOUT
    mesh, seg = synth.workload_small_bool()
    dev = torch.device("cuda:0")
    bvh = rsi.BVH(torch.from_numpy(mesh.V).to(dev), torch.from_numpy(mesh.T).to(dev))
    flag = bvh.intersect(torch.from_numpy(seg.A).to(dev), torch.from_numpy(seg.B).to(dev))["flag"]
    torch.cuda.synchronize()
    assert bvh.status() == 0 and 0 < int(flag.sum()) < seg.n


def test_streamed_launch_gives_up_after_one_wait():
    """A whole persistent BOOL traversal whose warps wait for ready flags
    that no copy sets (rsi_selftest_stream_wait): the first wait that gives
    up ends the launch for every warp, so 4M segments in 128-segment chunks
    (tens of thousands of chunks, several per resident warp) take about as
    long as one chunk's wait, not one wait per chunk."""
    import ctypes as C

    from paper_2209_02878_gb300 import _abi
    lib = _abi.load()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    polls = 20000
    res = {}
    for n in (32, 4_000_000):
        st, ms = C.c_int32(-1), C.c_float(-1.0)
        assert lib.rsi_selftest_stream_wait(polls, n, s, C.byref(st), C.byref(ms)) == _abi.RSI_OK
        assert st.value == _abi.RSI_ERR_TIMEOUT, (n, st.value)
        res[n] = ms.value
    assert res[32] > 0.5, res            # one wait of 20k polls takes a while
    assert res[4_000_000] < 3 * res[32] + 5.0, res
    # the device is still usable
    x = torch.arange(10, device="cuda:0").sum()
    assert int(x) == 45
