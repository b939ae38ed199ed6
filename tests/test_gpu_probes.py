"""Measurement utilities (needs a GPU): the gather and streaming ceilings
count their work exactly and report rates in the physically possible range."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lg():
    import paper_2303_06150_gb300 as lg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return lg


@pytest.mark.parametrize("width", [4, 8, 16, 32])
def test_gather_probe_counts_and_rate(lg, width):
    buf = torch.randn((20 << 20) // 32, 8, device="cuda")
    p = lg.probe_gather(buf, 64, width)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert p["loads"] == sms * 2048 * 64 and p["ms"] > 0
    assert 1e10 < p["loads_per_s"] < 2e12


def test_stream_probe_counts_and_rate(lg):
    buf = torch.randn(20 << 18, device="cuda")            # 20 MB
    p = lg.probe_stream(buf, 10)
    assert p["bytes"] == buf.numel() * 4 * 10 and p["ms"] > 0
    assert 500 < p["gbs"] < 100000


def test_probes_reject_bad_arguments(lg):
    buf = torch.randn(1024, device="cuda")
    with pytest.raises(lg.LigenError):
        lg.probe_stream(buf, 0)
    with pytest.raises(lg.LigenError):
        lg.probe_gather(buf.view(-1, 8), 64, 12)
