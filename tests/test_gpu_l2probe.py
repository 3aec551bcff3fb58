"""The bench's L2 random-gather probe (bench_l2probe.cu, outside the product
library): a plausible rate on an L2-resident array, and its argument checks."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bench():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench as b
    b.build_l2probe()
    return b


def test_probe_rate_plausible(bench):
    import torch
    table = torch.zeros(1 << 24, dtype=torch.int32, device="cuda")     # 64 MiB
    rate = bench.l2probe_gather(table, 1 << 26)
    # one request per read: well above 1e9/s and below what the L2 could serve at
    # one request per slice and clock (a few 1e11/s)
    assert 1e9 < rate < 5e12


def test_probe_rejects_bad_sizes(bench):
    import torch
    table = torch.zeros(3 * (1 << 20), dtype=torch.int32, device="cuda")   # 12 MiB: not a power of two
    with pytest.raises(ValueError):
        bench.l2probe_gather(table, 1 << 20)
