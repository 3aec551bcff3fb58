"""GPU parity: dfa_product_check (product exploration, Section 4) against the
oracle's exploration and the paper's inclusion table."""
import os

import numpy as np
import pytest

import dfagen
import oracle

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_20735_gb300 as pkg
    pkg.build()
    return pkg


def _dev(X):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(X.delta).view(np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(X.accept)).cuda(), X.start)


def _table():
    rows = {}
    with open(os.path.join(GOLDEN, "memory_inclusion.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, c = map(int, line.split())
            rows[n] = c
    return rows


@pytest.mark.parametrize("n", list(range(5, 25)))
def test_memory_inclusion_table(g, n):
    """The inclusion table (memory_5 .. memory_24): holds, with the printed
    number of explored product states."""
    F, P = dfagen.memory_dfa(n, True), dfagen.memory_dfa(n, False)
    holds, pairs, cex = g.product_check(_dev(F), _dev(P), inclusion=True)
    assert holds and cex == -1 and pairs == _table()[n]


@pytest.mark.parametrize("n", [25, 26, 27])
def test_memory_inclusion_table_largest(g, n):
    """The table's largest rows (up to 1.85e9 product states, 64 GB of search
    state), with max_pairs set to the printed count: a larger product would
    end with DFA_ENOMEM."""
    import torch
    F, P = dfagen.memory_dfa(n, True), dfagen.memory_dfa(n, False)
    want = _table()[n]
    holds, pairs, cex = g.product_check(_dev(F), _dev(P), inclusion=True, max_pairs=want)
    assert holds and cex == -1 and pairs == want
    torch.cuda.empty_cache()


@pytest.mark.parametrize("n", [3, 6, 10])
def test_memory_reverse_inclusion(g, n):
    F, P = dfagen.memory_dfa(n, True), dfagen.memory_dfa(n, False)
    ref = oracle.product_explore(P.delta, P.accept, P.start, F.delta, F.accept, F.start, inclusion=True)
    assert g.product_check(_dev(P), _dev(F), inclusion=True) == (ref.holds, ref.pairs, ref.cex_len)


@pytest.mark.parametrize("req", range(10))
def test_equivalence_pairs(g, req):
    A, B, expect = dfagen.equivalence_pair(req, 13, n_lo=100, n_hi=30_000)
    ref = oracle.product_explore(A.delta, A.accept, A.start, B.delta, B.accept, B.start)
    got = g.product_check(_dev(A), _dev(B))
    assert got == (ref.holds, ref.pairs, ref.cex_len)
    assert got[0] == expect


@pytest.mark.parametrize("idx", range(5))
def test_self_product(g, idx):
    A = [dfagen.random_dfa(3000, 2, 0.5, 3), dfagen.fibonacci_dfa(14), dfagen.bit_splitter(10),
         dfagen.chain_dfa(2000), dfagen.cycle_dfa(9)][idx]
    holds, pairs, cex = g.product_check(_dev(A), _dev(A))
    assert holds and cex == -1 and pairs == int(oracle.reachable(A.delta, A.start).sum())


def test_large_equivalent_pair(g):
    """A million-state DFA against a renamed copy with junk: one explored pair per
    reachable state of A (the renaming is a bijection on them)."""
    A, B, _ = dfagen.equivalence_pair(0, 17, n_lo=1_000_000, n_hi=1_000_001, force="equivalent")
    holds, pairs, cex = g.product_check(_dev(A), _dev(B))
    assert holds and cex == -1 and pairs == int(oracle.reachable(A.delta, A.start).sum())


def test_inclusion_random_and_host_inputs(g):
    for seed in range(6):
        A = dfagen.random_dfa(60, 2, 0.3, 500 + seed)
        B = dfagen.random_dfa(40, 2, 0.7, 600 + seed)
        ref = oracle.product_explore(A.delta, A.accept, A.start, B.delta, B.accept, B.start, inclusion=True)
        got = g.product_check((A.delta, A.accept, A.start), (B.delta, B.accept, B.start), inclusion=True)
        assert got == (ref.holds, ref.pairs, ref.cex_len)


def test_errors(g):
    F, P = dfagen.memory_dfa(8, True), dfagen.memory_dfa(8, False)
    with pytest.raises(g.DfaError) as e:
        g.product_check(_dev(F), _dev(P), inclusion=True, max_pairs=100)   # 1,088 pairs reachable
    assert e.value.status == g.DFA_ENOMEM
    A = dfagen.random_dfa(100, 2, 0.5, 3)
    A.delta[1][5] = 100
    with pytest.raises(g.DfaError) as e:
        g.product_check((A.delta, A.accept, 0), (A.delta, A.accept, 0))
    assert e.value.status == g.DFA_EINVAL
