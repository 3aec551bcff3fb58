"""GPU parity: signature refinement on the closure DFA (DFA_ALGO_CLOSURE_MOORE),
bit for bit against the CPU oracle, and the chain's closed-form round count at
full size (n = 2^20)."""
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


def _run(g, A, **kw):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda()
    a = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
    block, res = g.minimise(d, a, algo="closure_moore", **kw)
    return block.cpu().numpy().view(np.uint32), res


def _parity(g, A, **kw):
    ref = oracle.closure_moore(A.delta, A.accept)
    got, res = _run(g, A, **kw)
    assert np.array_equal(got, ref.block)
    assert res.num_blocks == ref.num_blocks
    assert (res.rounds_changed, res.rounds_executed) == (ref.rounds_changed, ref.rounds_executed)
    return res


@pytest.mark.parametrize("n,k,p", [(1, 2, 0.5), (2, 1, 0.5), (7, 3, 0.5), (100, 2, 0.5), (1000, 3, 0.3),
                                   (4097, 2, 0.5), (10_000, 2, 0.5), (3000, 0, 0.5), (2000, 5, 0.0)])
def test_random(g, n, k, p):
    _parity(g, dfagen.random_dfa(n, k, p, 700 + n + k))


@pytest.mark.parametrize("i", [5, 9, 13, 17])
def test_fibonacci(g, i):
    _parity(g, dfagen.fibonacci_dfa(i))


@pytest.mark.parametrize("m", [3, 8, 12])
def test_bit_splitters(g, m):
    _parity(g, dfagen.bit_splitter(m))


def test_fig1_cycle_planted(g):
    _parity(g, dfagen.fig1_chain())
    _parity(g, dfagen.cycle_dfa(12))
    base = dfagen.random_dfa(400, 3, 0.5, 62)
    P, _ = dfagen.planted_redundancy(base, 5, 1)
    res = _parity(g, P)
    assert res.num_blocks == base.n


@pytest.mark.parametrize("lg", [6, 10, 14])
def test_chain(g, lg):
    _parity(g, dfagen.chain_dfa(1 << lg))


def test_chain_2p20_closed_form(g):
    """Full-size chain: the identity partition after max popcount(x), x <= n-2,
    growing rounds (19 for n = 2^20), against 1,048,574 for plain refinement."""
    n = 1 << 20
    got, res = _run(g, dfagen.chain_dfa(n))
    R = max(bin(x).count("1") for x in range(1, n - 1))
    assert R == 19
    assert np.array_equal(got, np.arange(n, dtype=np.uint32))
    assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == (n, R, R + 1)


def test_host_buffers_max_rounds_bad_delta(g):
    A = dfagen.random_dfa(5000, 2, 0.5, 78)
    ref = oracle.closure_moore(A.delta, A.accept)
    block, res = g.minimise(A.delta, A.accept, algo="closure_moore")
    assert np.array_equal(block, ref.block) and res.rounds_executed == ref.rounds_executed
    F = dfagen.fibonacci_dfa(12)
    got, res = _run(g, F, max_rounds=2, check=False)
    assert res.call_status == g.DFA_EMAXROUNDS and res.rounds_executed == 2
    assert np.array_equal(got, oracle.closure_moore(F.delta, F.accept, max_rounds=2).block)
    B = dfagen.random_dfa(100, 2, 0.5, 3)
    B.delta[1][5] = 100
    with pytest.raises(g.DfaError) as e:
        _run(g, B)
    assert e.value.status == g.DFA_EINVAL
