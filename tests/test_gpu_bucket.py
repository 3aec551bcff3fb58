"""GPU parity of the bucketed gather (DFA_FLAG_BUCKETED): the transitions are
sorted once per call by (source range, target range), and every round reads
its labels from shared-memory slices instead of the label array.  Forced here
at every size, so that small state spaces exercise many buckets, empty and
ragged segments, partial last buckets and every round mode (direct, filter,
single-stage table, multi-stage table through the direct reads).  Integer
work: partitions bit for bit in canonical numbering, round counts exactly.
"""
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


def _dev(A):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(A.accept)).cuda())


def _parity(g, A, ref=None, flags=0):
    ref = ref or oracle.moore(A.delta, A.accept)
    d, a = _dev(A)
    block, res = g.minimise(d, a, flags=g.DFA_FLAG_BUCKETED | flags)
    got = block.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, ref.block)
    assert res.num_blocks == ref.num_blocks
    assert (res.rounds_changed, res.rounds_executed) == (ref.rounds_changed, ref.rounds_executed), ref.counts
    return res


@pytest.mark.parametrize("n", [1, 2, 7, 8, 9, 63, 511, 1000, 4097, 10_000, 65_537, 100_003, 262_144])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 16])
def test_random_sizes(g, n, k):
    A = dfagen.random_dfa(n, k, 0.5, 7000 + n + k)
    _parity(g, A)


@pytest.mark.parametrize("n,k", [(10_000, 2), (300_000, 4), (65_536, 3), (4097, 8), (50_000, 16)])
def test_table_only(g, n, k):
    """Every round through the exact table: single-stage rounds from the tiles,
    multi-stage ones (k >= 5 after the first round) through direct reads."""
    A = dfagen.random_dfa(n, k, 0.5, n + k)
    _parity(g, A, flags=g.DFA_FLAG_TABLE_ONLY)


@pytest.mark.parametrize("p", [0.0, 1.0, 0.01, 0.3])
def test_acceptance_extremes(g, p):
    A = dfagen.random_dfa(20_000, 3, p, 70)
    _parity(g, A)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_planted_redundancy(g, seed):
    """Real merges: filter rounds whose listed states are true duplicates."""
    base = dfagen.random_dfa(3000, 3 + seed % 3, 0.5, seed + 40)
    P, origin = dfagen.planted_redundancy(base, 6, seed)
    ref = oracle.moore(P.delta, P.accept)
    assert np.array_equal(ref.block, oracle.canonical(origin))
    _parity(g, P, ref)


def test_few_targets_heavy_merging(g):
    """Huge blocks: partitions of the uniqueness test overflow and list all their states."""
    n, k = 200_000, 3
    d = dfagen.bounded(9, 91, n * k, 5).reshape(k, n)
    acc = dfagen.bernoulli(9, 92, n, 0.5)
    _parity(g, dfagen.DFA(d, acc, 0))


@pytest.mark.parametrize("fam", ["fib", "bits", "chain", "cycle"])
def test_families(g, fam):
    A = {"fib": lambda: dfagen.fibonacci_dfa(14), "bits": lambda: dfagen.bit_splitter(12),
         "chain": lambda: dfagen.chain_dfa(1 << 10), "cycle": lambda: dfagen.cycle_dfa(14)}[fam]()
    _parity(g, A)


@pytest.mark.parametrize("idx", range(4))
def test_stop_discrete(g, idx):
    A = [dfagen.random_dfa(300_000, 4, 0.5, 2), dfagen.bit_splitter(12),
         dfagen.planted_redundancy(dfagen.random_dfa(300, 3, 0.5, 61), 5, 2)[0],
         dfagen.random_dfa(65_537, 3, 0.3, 8)][idx]
    ref = oracle.moore(A.delta, A.accept, stop_discrete=True)
    _parity(g, A, ref=ref, flags=g.DFA_FLAG_STOP_DISCRETE)


def test_bad_transition_target(g):
    A = dfagen.random_dfa(1000, 2, 0.5, 5)
    A.delta[1][123] = 1000
    d, a = _dev(A)
    with pytest.raises(g.DfaError) as e:
        g.minimise(d, a, flags=g.DFA_FLAG_BUCKETED)
    assert e.value.status == g.DFA_EINVAL


def test_host_buffers(g):
    A = dfagen.random_dfa(50_000, 3, 0.5, 17)
    ref = oracle.moore(A.delta, A.accept)
    block, res = g.minimise(A.delta, A.accept, flags=g.DFA_FLAG_BUCKETED)
    assert np.array_equal(block, ref.block) and res.rounds_executed == ref.rounds_executed


@pytest.mark.parametrize("req", range(6))
def test_equivalence(g, req):
    A, B, expect = dfagen.equivalence_pair(req, 5, n_lo=1000, n_hi=60_000)
    args = (A.delta, A.accept, A.start, B.delta, B.accept, B.start)
    for early in (False, True):
        eq, res = g.equivalent(args[:3], args[3:], early_exit=early, flags=g.DFA_FLAG_BUCKETED)
        ref = oracle.equivalent(*args, early_exit=early)
        assert eq == expect == ref.equivalent
        assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
            (ref.refine.num_blocks, ref.refine.rounds_changed, ref.refine.rounds_executed)


def test_default_and_bucketed_same_result_2p20(g):
    """Above 2^20 states: the bucketed gather (opt-in) and the default direct
    label reads give the same partition and rounds, both equal to the oracle's."""
    A = dfagen.random_dfa((1 << 20) + 5, 4, 0.5, 23)
    ref = oracle.moore(A.delta, A.accept)
    _parity(g, A, ref)
    d, a = _dev(A)
    b2, r2 = g.minimise(d, a)
    assert np.array_equal(b2.cpu().numpy().view(np.uint32), ref.block)
    assert (r2.num_blocks, r2.rounds_changed, r2.rounds_executed) == \
        (ref.num_blocks, ref.rounds_changed, ref.rounds_executed)


def test_gather_flag_overrides(g):
    """DFA_FLAG_GATHER with DFA_FLAG_BUCKETED: the direct reads run (no bucket
    workspace needed), same result."""
    A = dfagen.random_dfa(30_000, 3, 0.5, 24)
    d, a = _dev(A)
    dd, keep = g.make_dfa(d, a)
    both = g.make_opts("moore", flags=g.DFA_FLAG_BUCKETED | g.DFA_FLAG_GATHER)
    assert g.dfa_workspace_size(dd, both) == g.dfa_workspace_size(dd, g.make_opts("moore"))
    ref = oracle.moore(A.delta, A.accept)
    block, res = g.minimise(d, a, flags=g.DFA_FLAG_BUCKETED | g.DFA_FLAG_GATHER)
    assert np.array_equal(block.cpu().numpy().view(np.uint32), ref.block)
