"""GPU parity: naivePR (Algorithm 2) and transPR (Algorithm 5) through the C ABI,
bit for bit against the CPU oracle (partition in canonical numbering and round
counts), plus the deep-round chain workload of n = 2^20 states."""
import numpy as np
import pytest

import dfagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_20735_gb300 as pkg
    pkg.build()
    return pkg


def _run(g, A, algo, **kw):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda()
    a = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
    block, res = g.minimise(d, a, algo=algo, **kw)
    return block.cpu().numpy().view(np.uint32), res


def _parity(g, A, algo):
    ref = oracle.naive_pr(A.delta, A.accept) if algo == "naive" else oracle.trans_pr(A.delta, A.accept)
    got, res = _run(g, A, algo)
    assert np.array_equal(got, ref.block)
    assert res.num_blocks == ref.num_blocks
    assert (res.rounds_changed, res.rounds_executed) == (ref.rounds_changed, ref.rounds_executed)
    return res


@pytest.mark.parametrize("algo", ["naive", "trans"])
@pytest.mark.parametrize("n,k,p", [(1, 2, 0.5), (2, 1, 0.5), (7, 3, 0.5), (100, 2, 0.5), (1000, 3, 0.3),
                                   (4097, 2, 0.5), (10_000, 2, 0.5), (3000, 0, 0.5), (2000, 5, 0.0)])
def test_random(g, algo, n, k, p):
    _parity(g, dfagen.random_dfa(n, k, p, 500 + n + k), algo)


@pytest.mark.parametrize("algo", ["naive", "trans"])
@pytest.mark.parametrize("i", [5, 9, 13, 17])
def test_fibonacci(g, algo, i):
    A = dfagen.fibonacci_dfa(i)
    res = _parity(g, A, algo)
    if algo == "naive":
        assert res.rounds_executed == A.n - 1          # Table concur: N-1 iterations


@pytest.mark.parametrize("algo", ["naive", "trans"])
@pytest.mark.parametrize("m", [3, 8, 14])
def test_bit_splitters(g, algo, m):
    _parity(g, dfagen.bit_splitter(m), algo)


@pytest.mark.parametrize("algo", ["naive", "trans"])
def test_fig1_and_cycle(g, algo):
    _parity(g, dfagen.fig1_chain(), algo)
    _parity(g, dfagen.cycle_dfa(12), algo)


@pytest.mark.parametrize("algo", ["naive", "trans"])
@pytest.mark.parametrize("seed", [1, 2])
def test_planted(g, algo, seed):
    base = dfagen.random_dfa(400, 3, 0.5, seed + 60)
    P, origin = dfagen.planted_redundancy(base, 5, seed)
    res = _parity(g, P, algo)
    assert res.num_blocks == base.n


@pytest.mark.parametrize("lg", [6, 10, 14])
def test_chain_trans(g, lg):
    C = dfagen.chain_dfa(1 << lg)
    res = _parity(g, C, "trans")
    assert res.num_blocks == 1 << lg


def test_chain_2p20_trans_full_size(g):
    """The deep-round workload at full size with the closure: parity with the oracle."""
    C = dfagen.chain_dfa(1 << 20)
    res = _parity(g, C, "trans")
    assert res.num_blocks == 1 << 20


def test_chain_2p20_moore_closed_form(g):
    """Plain signature refinement on the chain: n-2 growing rounds, all states
    distinct (closed form; the oracle would need ~10^12 steps at this size)."""
    n = 1 << 20
    C = dfagen.chain_dfa(n)
    got, res = _run(g, C, "moore")
    assert res.num_blocks == n
    assert (res.rounds_changed, res.rounds_executed) == (n - 2, n - 1)
    assert np.array_equal(got, np.arange(n, dtype=np.uint32))


def test_naive_host_buffers(g):
    A = dfagen.random_dfa(5000, 2, 0.5, 77)
    ref = oracle.trans_pr(A.delta, A.accept)
    block, res = g.minimise(A.delta, A.accept, algo="trans")
    assert np.array_equal(block, ref.block) and res.rounds_executed == ref.rounds_executed


def test_naive_max_rounds_and_bad_delta(g):
    A = dfagen.fibonacci_dfa(10)
    got, res = _run(g, A, "naive", max_rounds=7, check=False)
    assert res.call_status == g.DFA_EMAXROUNDS and res.rounds_executed == 7
    ref = oracle.naive_pr(A.delta, A.accept, max_rounds=7)
    assert np.array_equal(got, ref.block)
    B = dfagen.random_dfa(100, 2, 0.5, 3)
    B.delta[0][5] = 100
    with pytest.raises(g.DfaError):
        _run(g, B, "trans")
