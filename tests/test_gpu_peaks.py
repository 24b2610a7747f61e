"""The measured peaks the roofline figures divide by: the MUFU issue rate (sqrt and rsqrt, the epilogues'
per-bin operations) and the cost of one tensor-core MMA by width.  Checked for plausibility against the
pipes' unit counts: at most 16 MUFU results per clock and SM, and an MMA of 256 columns (M = 128, K = 16:
524,288 multiply-adds) no faster than the 4096 multiply-adds per clock and SM of the dense FP16 peak,
with narrower MMAs no slower than the widest."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sal():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2201_06174_gb300 as s
    s.load()
    return s


def test_mufu_rate_is_plausible(sal):
    clk = torch.cuda.get_device_properties(0).multi_processor_count
    for op in ("sqrt", "rsqrt"):
        rate, sms = sal.sal_measure_mufu_rate(op)
        assert sms == clk
        per_clk_sm = rate / (sms * 2.2e9)   # above the highest clock this part runs at
        assert 4.0 < per_clk_sm <= 16.5, (op, rate)


def test_mma_cost_by_width(sal):
    cyc = {nc: sal.sal_measure_mma_rate(nc)[0] for nc in (16, 32, 64, 128, 256)}
    assert cyc[256] >= 128 * 0.95, cyc                        # 524,288 MACs at <= 4096 per clock
    assert all(cyc[nc] <= cyc[256] * 1.05 for nc in (16, 32, 64, 128)), cyc
    assert all(10.0 < c < 10000.0 for c in cyc.values()), cyc
    with pytest.raises(sal.SalError):
        sal.sal_measure_mma_rate(48)
