"""The L2 random-gather probe: a plausible rate on an L2-resident array, and
its argument checks."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_20735_gb300 as pkg
    pkg.build()
    return pkg


def test_probe_rate_plausible(g):
    import torch
    table = torch.zeros(1 << 24, dtype=torch.int32, device="cuda")     # 64 MiB
    rate = g.probe_l2_gather(table, 1 << 26)
    # one request per read: well above 1e9/s and below what the L2 could serve at
    # one request per slice and clock (a few 1e11/s)
    assert 1e9 < rate < 5e12


def test_probe_rejects_bad_sizes(g):
    import torch
    table = torch.zeros(3 * (1 << 20), dtype=torch.int32, device="cuda")   # 12 MiB: not a power of two
    with pytest.raises(g.DfaError) as e:
        g.probe_l2_gather(table, 1 << 20)
    assert e.value.status == g.DFA_EINVAL
