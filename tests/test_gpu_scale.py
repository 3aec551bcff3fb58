"""GPU parity with real merges at scale.

Random complete DFAs are almost always minimal, so the full-size random
workloads check only the identity partition.  Here a minimal random base DFA
is blown up by planted redundancy (every state copied 1..c times, each copy's
transitions pointing at random copies of the targets): the coarsest partition
is exactly "copies of the same base state" (a closed form), the oracle's Moore
refinement reaches it, and the GPU must equal the oracle bit for bit with the
same round counts.  Rounds of these inputs take every renumbering mode at
scale: direct rounds, filter rounds whose listed states are mostly true
duplicates, and table rounds after the filter gives up.
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


def _gpu(g, A, **kw):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda()
    a = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
    block, res = g.minimise(d, a, **kw)
    out = block.cpu().numpy().view(np.uint32)
    del d, a, block
    torch.cuda.empty_cache()
    return out, res


def _check(got, res, ref):
    assert np.array_equal(got, ref.block)
    assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
        (ref.num_blocks, ref.rounds_changed, ref.rounds_executed), ref.counts


@pytest.fixture(scope="module")
def base20():
    base = dfagen.random_dfa(1 << 20, 4, 0.5, 901)
    assert oracle.hopcroft(base.delta, base.accept).max() + 1 == base.n   # minimal: the closed form holds
    return base


@pytest.fixture(scope="module")
def planted22(base20):
    P, origin = dfagen.planted_redundancy(base20, 7, 902)            # about 2^22 states
    ref = oracle.moore(P.delta, P.accept)
    assert np.array_equal(ref.block, oracle.canonical(origin))
    return P, ref


@pytest.mark.parametrize("mode", ["default", "table_only", "stop_discrete", "bucketed"])
def test_planted_2p22(g, planted22, mode):
    P, ref = planted22
    flags = {"default": 0, "table_only": g.DFA_FLAG_TABLE_ONLY, "stop_discrete": g.DFA_FLAG_STOP_DISCRETE,
             "bucketed": g.DFA_FLAG_BUCKETED}[mode]
    if mode == "stop_discrete":
        ref = oracle.moore(P.delta, P.accept, stop_discrete=True)
    got, res = _gpu(g, P, flags=flags)
    _check(got, res, ref)


def test_planted_2p24(g, base20):
    """About 2^24 states (16 copies on average): the headline size with real merges."""
    P, origin = dfagen.planted_redundancy(base20, 31, 903)
    ref = oracle.moore(P.delta, P.accept)
    assert np.array_equal(ref.block, oracle.canonical(origin))
    got, res = _gpu(g, P)
    _check(got, res, ref)


def test_planted_many_letters_sparse_filter(g):
    """k = 8 and about 2^20 states: from 2^20 states on, a round whose previous
    blocks allow B^(k+1) >= 64 n combinations takes the filter path although the
    blocks are large; here its listed states are true duplicates."""
    base = dfagen.random_dfa(1 << 17, 8, 0.5, 904)
    assert oracle.hopcroft(base.delta, base.accept).max() + 1 == base.n
    P, origin = dfagen.planted_redundancy(base, 16, 905)
    assert P.n >= 1 << 20
    ref = oracle.moore(P.delta, P.accept)
    assert np.array_equal(ref.block, oracle.canonical(origin))
    got, res = _gpu(g, P)
    _check(got, res, ref)


def test_epoch_wraparound_table_rounds(g):
    """2^24 states and 4 letters leave 3 epoch bits in the exact table's keys
    ((k+1) * 25 = 125 key bits), so table-only rounds wrap the epoch every 7
    passes.  A deep-round chain (letters a, b doubled into 4) run for 20 rounds
    through the table only must equal the oracle's first 20 rounds."""
    n = 1 << 24
    C = dfagen.chain_dfa(n)
    D = dfagen.DFA(np.concatenate([C.delta, C.delta]), C.accept, 0)
    ref = oracle.moore(D.delta, D.accept, max_rounds=20)
    got, res = _gpu(g, D, flags=g.DFA_FLAG_TABLE_ONLY, max_rounds=20, check=False)
    assert res.call_status == g.DFA_EMAXROUNDS and res.rounds_executed == 20
    assert np.array_equal(got, oracle.canonical(ref.block))
