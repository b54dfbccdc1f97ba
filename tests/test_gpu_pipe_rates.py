"""GPU test of the pipe-rate probe (lens_sim_pipe_rates), the measured denominators of the
ALU-bound kernels' rooflines: every rate is positive and within what one SM can issue per
clock (128 FP32 lanes; the MUFU unit far fewer), and bad arguments are refused."""
import ctypes

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sim():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_01547_gb300 import lenssim
    s = lenssim.Simulator(device=0)
    yield s
    s.close()


def test_pipe_rates_are_within_one_sm_per_clock(sim):
    r = sim.pipe_rates()
    # FP32: 4 sub-partitions x 32 lanes per clock; packed and scalar chains both reach most of it
    for k in ("fp32_lane_ops_ffma2", "fp32_lane_ops_ffma"):
        assert 96.0 <= r[k] <= 129.0, (k, r[k])
    # MUFU: a fraction of the FP32 rate, at least 4 results per clock per SM
    for k in ("mufu_rsqrt", "mufu_ex2", "mufu_lg2", "mufu_rcp"):
        assert 4.0 <= r[k] <= 64.0, (k, r[k])
    # the probe leaves the handle usable and nothing allocated
    assert sim.pipe_rates()["mufu_rsqrt"] > 0.0


def test_pipe_rates_partial_and_bad_arguments(sim):
    from paper_2606_01547_gb300 import lenssim
    L = sim._L
    one = (ctypes.c_double * 3)(-1.0, -1.0, -1.0)
    assert L.lens_sim_pipe_rates(sim.h, one, 1) == lenssim.LENS_OK
    assert one[0] > 0.0 and one[1] == -1.0 and one[2] == -1.0
    many = (ctypes.c_double * (len(lenssim.PIPE_RATES) + 2))()
    assert L.lens_sim_pipe_rates(sim.h, many, len(many)) == lenssim.LENS_OK
    assert all(v > 0.0 for v in many[:len(lenssim.PIPE_RATES)]) and many[-1] == 0.0 and many[-2] == 0.0
    assert L.lens_sim_pipe_rates(sim.h, None, 6) == lenssim.LENS_ERR_INVALID_ARG
    assert L.lens_sim_pipe_rates(sim.h, one, 0) == lenssim.LENS_ERR_INVALID_ARG
    assert L.lens_sim_pipe_rates(None, one, 1) == lenssim.LENS_ERR_INVALID_ARG
