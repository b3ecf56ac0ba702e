"""Pipe-rate probe (lsp_probe_pipes): the rates it measures are those the
kernels' roofline denominators assume -- FP32 FMA near 128 lanes per clock per
SM, packed FP32x2 FMA moving the same lanes, the sin/cos pair at the SFU rate
(16 SFU ops, i.e. 8 pairs, per clock per SM) -- and the SM count and clock are
the device's."""
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lsp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_1658_gb300 import build, lsp as L
    build.build()
    return L


def test_probe_rates_match_the_pipe_widths(lsp):
    with lsp.Context(0) as ctx:
        r = ctx.probe_pipes()
    assert r["sms"] == torch.cuda.get_device_properties(0).multi_processor_count
    assert 96.0 <= r["ffma_per_clk_sm"] <= 132.0, r
    assert 96.0 <= r["ffma2_lanes_per_clk_sm"] <= 132.0, r
    assert 4.0 <= r["sincos_per_clk_sm"] <= 17.0, r
    # an FP32 FMA lane is at least as fast as a sin/cos pair by a wide margin
    assert r["ffma_per_clk_sm"] >= 6.0 * r["sincos_per_clk_sm"], r
    assert 300.0 <= r["sm_mhz"] <= 3000.0, r
