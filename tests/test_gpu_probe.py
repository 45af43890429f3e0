"""The bandwidth probe (the L2 denominator of the DFS kernel's roofline):
positive readings for an L2-sized and a DRAM-sized working set, and the
argument checks."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2401_17018_gb300 import gamma
    return gamma


def test_probe_reads_l2_and_dram_sized_buffers(G):
    l2 = G.gamma_probe_bandwidth(0, 32 << 20, reps=8, trials=3)
    dram = G.gamma_probe_bandwidth(0, 2 << 30, reps=1, trials=3)
    assert 0 < l2 < 1e6 and 0 < dram < 1e6
    with pytest.raises(G.GammaError):
        G.gamma_probe_bandwidth(0, 1024, reps=1, trials=1)  # below the 1 MiB minimum
