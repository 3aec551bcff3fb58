"""GPU parity: sortPR with the radix-sort renumbering (DFA_ALGO_SORT, the
paper's own sort + adjacent difference + scan per round) against the oracle's
Moore refinement: partition element by element, rounds_changed and
rounds_executed."""
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


def _sort(g, A, device=True, flags=0, max_rounds=0):
    import torch
    if device:
        d = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda()
        a = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
        blk, res = g.minimise(d, a, algo="sort", flags=flags, max_rounds=max_rounds)
        return blk.cpu().numpy().view(np.uint32), res
    return g.minimise(A.delta, A.accept, algo="sort", flags=flags, max_rounds=max_rounds)


def _check(g, A, device=True, flags=0):
    ref = oracle.moore(A.delta, A.accept, stop_discrete=bool(flags & g.DFA_FLAG_STOP_DISCRETE))
    blk, res = _sort(g, A, device, flags)
    assert np.array_equal(blk, ref.block)
    assert res.num_blocks == int(ref.block.max()) + 1
    assert (res.rounds_changed, res.rounds_executed) == (ref.rounds_changed, ref.rounds_executed)


def _cases():
    yield dfagen.random_dfa(1, 2, 0.5, 1)
    yield dfagen.random_dfa(2, 1, 0.5, 2)
    yield dfagen.random_dfa(100, 2, 0.5, 3)
    yield dfagen.random_dfa(10_000, 2, 0.5, 1)          # the small workload
    yield dfagen.random_dfa(4097, 3, 0.3, 4)
    yield dfagen.random_dfa(70_000, 8, 0.5, 5)          # 9 components of 17 bits: 27 passes a round
    yield dfagen.random_dfa(3000, 0, 0.5, 6)
    yield dfagen.random_dfa(500, 2, 0.0, 7)
    yield dfagen.random_dfa(500, 2, 1.0, 8)
    yield dfagen.planted_redundancy(dfagen.random_dfa(2000, 3, 0.5, 9), 5, 2)[0]
    yield dfagen.chain_dfa(600)                          # 598 growing rounds
    yield dfagen.fibonacci_dfa_with_states(233)
    yield dfagen.bit_splitter(10)
    yield dfagen.random_dfa(300_001, 4, 0.5, 10)        # a ragged final chunk


@pytest.mark.parametrize("idx", range(14))
def test_parity_with_oracle(g, idx):
    _check(g, list(_cases())[idx])


@pytest.mark.parametrize("idx", [2, 9, 12])
def test_host_buffers(g, idx):
    _check(g, list(_cases())[idx], device=False)


@pytest.mark.parametrize("idx", [3, 11, 12])
def test_stop_discrete(g, idx):
    _check(g, list(_cases())[idx], flags=g.DFA_FLAG_STOP_DISCRETE)


def test_full_size_2p22(g):
    """2^22 states, 4 letters: 4 rounds of 5 components x 3 passes."""
    _check(g, dfagen.random_dfa(1 << 22, 4, 0.5, 2))


def test_max_rounds(g):
    A = dfagen.chain_dfa(200)
    blk, res = g.minimise(A.delta, A.accept, algo="sort", max_rounds=5, check=False)
    assert res.call_status == g.DFA_EMAXROUNDS
    ref = oracle.moore(A.delta, A.accept, max_rounds=5)
    assert np.array_equal(blk, ref.block)


def test_bad_target(g):
    A = dfagen.random_dfa(1000, 2, 0.5, 5)
    bad = A.delta.copy()
    bad[1][999] = 1000
    with pytest.raises(g.DfaError) as e:
        g.minimise(bad, A.accept, algo="sort")
    assert e.value.status == g.DFA_EINVAL
    _check(g, A)
