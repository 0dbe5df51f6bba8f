"""The pipe micro-benchmarks behind the pair kernels' ALU roofline (od_measure_peaks):
rates in the range of one GB300 SM and the SFU's relative speeds the roofline uses."""
import pytest

import paper_2205_06557_gb300 as od

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2205_06557_gb300 import build

    build.build()
    od.lib()


def test_pipe_rates_are_in_range():
    pk = od.od_measure_peaks()
    c = pk["per_clk_per_sm"]
    # per clock at the maximum clock: a lower running clock only lowers them
    assert 48 < c["ffma"] <= 1.05 * 128, c
    for k in ("rsqrt", "rcp", "lg2"):
        assert 6 < c[k] <= 1.05 * 16, (k, c)
    # the roofline counts ex2 at twice the rate of rsqrt
    assert 1.7 < c["ex2"] / c["rsqrt"] < 2.3, c
    assert 0 < c["dfma"] < c["ffma"]
    assert 1 < pk["dfma_latency_ns"] < 1000 and pk["dfma_latency_ns"] < pk["dexp_latency_ns"] < 1e5
