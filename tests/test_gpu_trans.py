"""GPU parity: dfa_trans (Algorithm 1, transitive closure of the pair graph)
against the oracle's trans on small DFAs (partition and iteration count), and
on the larger ones the dense oracle cannot reach against Hopcroft's partition
and the closed form of the iteration count; Table 1's Fibonacci rows."""
import os

import numpy as np
import pytest

import dfagen
import oracle
from conftest import GOLDEN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_20735_gb300 as pkg
    pkg.build()
    return pkg


def _run(g, A, device=True):
    import torch
    if device:
        d = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda()
        a = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
        blk, it = g.trans(d, a)
        return blk.cpu().numpy().view(np.uint32), it
    return g.trans(A.delta, A.accept)


def _closed_form(D):
    """Iteration i ends with Apart = the pairs within 2^(i+1) - 2 edges of an
    initially Apart pair; D = the distance of the farthest separable pair."""
    i = 0
    while (1 << (i + 1)) - 2 < D:
        i += 1
    return i + 1


def _table():
    rows = {}
    with open(os.path.join(GOLDEN, "trans_table1.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                N, it = map(int, line.split())
                rows[N] = it
    return rows


def _small_cases():
    for n, k, p, seed in [(1, 2, 0.5, 1), (2, 1, 0.5, 2), (5, 2, 0.5, 3), (12, 3, 0.5, 4), (20, 2, 0.3, 5),
                          (31, 1, 0.5, 6), (33, 2, 0.5, 7), (16, 0, 0.5, 8), (10, 2, 0.0, 9), (10, 2, 1.0, 10)]:
        yield dfagen.random_dfa(n, k, p, seed)
    yield dfagen.bit_splitter(4)
    yield dfagen.chain_dfa(16)
    yield dfagen.cycle_dfa(9)
    yield dfagen.planted_redundancy(dfagen.random_dfa(6, 2, 0.5, 9), 4, 1)[0]
    yield dfagen.planted_redundancy(dfagen.random_dfa(8, 3, 0.5, 3), 3, 2)[0]


@pytest.mark.parametrize("idx", range(15))
def test_small_against_oracle(g, idx):
    A = list(_small_cases())[idx]
    ref = oracle.trans(A.delta, A.accept)
    for device in (True, False):
        blk, it = _run(g, A, device)
        assert np.array_equal(blk, ref.block), device
        assert it == ref.iterations, device


@pytest.mark.parametrize("N", [8, 13, 21, 34, 55, 89])
def test_table_fibonacci_rows(g, N):
    """Every Fibonacci state is its own block; the iteration counts are the
    table's (the synchronous count on N = 34, one above the printed 5)."""
    A = dfagen.fibonacci_dfa_with_states(N)
    blk, it = _run(g, A)
    assert np.array_equal(blk, np.arange(N, dtype=np.uint32))
    assert it == _closed_form(N - 2)
    printed = _table()[N]
    assert it == printed or (N == 34 and it == 6 and printed == 5)
    if N <= 34:
        assert it == oracle.trans(A.delta, A.accept).iterations


def _large_cases():
    yield dfagen.fibonacci_dfa_with_states(144)       # printed as a timeout in the table
    yield dfagen.fibonacci_dfa_with_states(233)
    yield dfagen.random_dfa(256, 2, 0.5, 11)
    yield dfagen.planted_redundancy(dfagen.random_dfa(50, 2, 0.5, 12), 4, 3)[0]
    yield dfagen.bit_splitter(7)
    yield dfagen.chain_dfa(100)


@pytest.mark.parametrize("idx", range(6))
def test_large_against_hopcroft_and_closed_form(g, idx):
    A = list(_large_cases())[idx]
    assert A.n <= g.DFA_TRANS_MAX_STATES
    blk, it = _run(g, A)
    assert np.array_equal(blk, oracle.hopcroft(A.delta, A.accept))
    assert it == _closed_form(oracle.moore(A.delta, A.accept).rounds_changed)


def test_errors(g):
    A = dfagen.random_dfa(257, 2, 0.5, 1)
    with pytest.raises(g.DfaError) as e:
        g.trans(A.delta, A.accept)
    assert e.value.status == g.DFA_EINVAL
    B = dfagen.random_dfa(20, 2, 0.5, 2)
    bad = B.delta.copy()
    bad[1][7] = 20
    for device in (True, False):
        C = dfagen.DFA(bad, B.accept, 0)
        with pytest.raises(g.DfaError) as e:
            _run(g, C, device)
        assert e.value.status == g.DFA_EINVAL
    # the context is still usable
    blk, it = _run(g, B)
    assert np.array_equal(blk, oracle.trans(B.delta, B.accept).block)
