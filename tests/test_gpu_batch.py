"""GPU parity: dfa_minimise_batch.  Each DFA's partition (numbered within the
DFA) and round counts must equal the oracle's and dfa_minimise's on that DFA
alone, under every schedule and under the autotuner."""
import os

import numpy as np
import pytest

import dfagen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    os.environ["DFA_AUTOTUNE_CACHE"] = str(tmp_path_factory.mktemp("tune") / "autotune.json")
    import paper_2508_20735_gb300 as pkg
    pkg.build()
    return pkg


def _dev(A):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(A.accept)).cuda())


def _batch(g, dfas, schedule=-1, host=False, **kw):
    items = [(A.delta, A.accept) if host else _dev(A) for A in dfas]
    out, res = g.minimise_batch(items, schedule=schedule, **kw)
    blocks = out.cpu().numpy().view(np.uint32)
    offs = np.concatenate([[0], np.cumsum([A.n for A in dfas])])
    return [blocks[offs[i]:offs[i + 1]] for i in range(len(dfas))], res


def _mixed():
    dfas = [dfagen.random_dfa(n, k, p, 900 + i) for i, (n, k, p) in enumerate(
        [(1, 2, 0.5), (2, 1, 0.5), (3, 0, 0.5), (5, 3, 0.5), (64, 2, 0.3), (257, 4, 0.3), (1000, 8, 0.3),
         (3000, 40, 0.5), (4096, 2, 0.0), (777, 3, 1.0), (10_000, 5, 0.3), (14_462, 8, 0.3),
         (300, 130, 0.5)])]
    dfas.append(dfagen.fibonacci_dfa(11))
    dfas.append(dfagen.bit_splitter(9))
    base = dfagen.random_dfa(300, 3, 0.5, 61)
    dfas.append(dfagen.planted_redundancy(base, 5, 2)[0])
    dfas.append(dfagen.chain_dfa(300))
    dfas.append(dfagen.planted_redundancy(dfagen.random_dfa(200, 30, 0.5, 63), 5, 3)[0])   # wide keys, duplicates
    return dfas


@pytest.mark.parametrize("schedule", list(range(12)) + [-1])
def test_mixed_batch_against_oracle(g, schedule):
    dfas = _mixed()
    blocks, res = _batch(g, dfas, schedule=schedule)
    for A, b, r in zip(dfas, blocks, res):
        ref = oracle.moore(A.delta, A.accept)
        assert np.array_equal(b, ref.block)
        assert (r.num_blocks, r.rounds_changed, r.rounds_executed) == \
            (ref.num_blocks, ref.rounds_changed, ref.rounds_executed)


@pytest.mark.parametrize("schedule", [0, 5, 6, 11, -1])
def test_mixed_batch_stop_discrete(g, schedule):
    dfas = _mixed()
    blocks, res = _batch(g, dfas, schedule=schedule, flags=g.DFA_FLAG_STOP_DISCRETE)
    for A, b, r in zip(dfas, blocks, res):
        ref = oracle.moore(A.delta, A.accept, stop_discrete=True)
        assert np.array_equal(b, ref.block)
        assert (r.num_blocks, r.rounds_changed, r.rounds_executed) == \
            (ref.num_blocks, ref.rounds_changed, ref.rounds_executed)


def test_autotuner_records_every_schedule(g):
    """The autotuner times all twelve schedules once per batch shape, keeps the
    fastest, and writes the choice and every time to its cache file."""
    import json
    dfas = [dfagen.random_dfa(n, k, 0.3, 950 + i) for i, (n, k) in enumerate(
        [(3000, 3), (20_000, 5), (777, 2), (40_000, 7)])]
    blocks, res = _batch(g, dfas, schedule=-1)
    for A, b in zip(dfas, blocks):
        assert np.array_equal(b, oracle.moore(A.delta, A.accept).block)
    with open(os.environ["DFA_AUTOTUNE_CACHE"]) as f:
        cache = json.load(f)
    kmax = [key for key in cache if key.startswith("batch|") and key.endswith("|kmax7")]
    assert kmax, cache
    entry = cache[kmax[0]]
    choice, times = entry[0], entry[1:]
    assert len(times) == 12 and all(t > 0 for t in times)
    assert 0 <= choice < 12 and times[choice] == min(times)


def test_batch_schedule_out_of_range(g):
    with pytest.raises(g.DfaError) as e:
        _batch(g, [dfagen.random_dfa(100, 2, 0.5, 3)], schedule=12)
    assert e.value.status == g.DFA_EINVAL


def test_batch_graph_is_reused(g):
    """Repeated calls in one thread update the kept graph instead of
    instantiating a new one."""
    dfas = _mixed()[:6]
    _batch(g, dfas, schedule=0)
    i0, u0 = g.batch_graph_stats()
    for _ in range(3):
        blocks, _ = _batch(g, dfas, schedule=0)
    i1, u1 = g.batch_graph_stats()
    assert i1 == i0 and u1 - u0 == 3
    for A, b in zip(dfas, blocks):
        assert np.array_equal(b, oracle.moore(A.delta, A.accept).block)


def test_batch_equals_alone_and_host_inputs(g):
    dfas = _mixed()[:10]
    blocks, res = _batch(g, dfas, host=True)
    for A, b, r in zip(dfas, blocks, res):
        d, a = _dev(A)
        alone, ra = g.minimise(d, a)
        assert np.array_equal(b, alone.cpu().numpy().view(np.uint32))
        assert (r.num_blocks, r.rounds_executed) == (ra.num_blocks, ra.rounds_executed)


def test_batch_recipe_sample(g):
    """256 DFAs of the batch recipe (n log-uniform in [64, 65536], k in 2..8)."""
    dfas = dfagen.batch_dfas(256, 64, 65_536, 2, 8, 0.3, 4)
    blocks, res = _batch(g, dfas)
    for A, b, r in zip(dfas, blocks, res):
        ref = oracle.moore(A.delta, A.accept)
        assert np.array_equal(b, ref.block)
        assert r.rounds_executed == ref.rounds_executed


def test_batch_4096_full_size(g):
    """The full 4,096-DFA workload: every DFA's partition equals the oracle's
    Moore refinement and Hopcroft's partition, its round counts equal the
    oracle's, and it equals the DFA's stand-alone refinement on the GPU."""
    dfas = dfagen.batch_dfas(4096, 64, 65_536, 2, 8, 0.3, 4)
    blocks, res = _batch(g, dfas)
    for i, (A, b, r) in enumerate(zip(dfas, blocks, res)):
        ref = oracle.moore(A.delta, A.accept)
        assert np.array_equal(b, ref.block), i
        assert (r.num_blocks, r.rounds_changed, r.rounds_executed) == \
            (ref.num_blocks, ref.rounds_changed, ref.rounds_executed), i
        assert np.array_equal(b, oracle.hopcroft(A.delta, A.accept)), i
        d, a = _dev(A)
        alone, ra = g.minimise(d, a)
        assert np.array_equal(b, alone.cpu().numpy().view(np.uint32)), i


def test_batch_medium_dfas_planted(g):
    """DFAs of 16,385 to 65,536 states with true merges (planted redundancy)
    and with many letters, on the block-per-DFA path with the table in global
    memory, against the oracle and Hopcroft's partition."""
    dfas = [dfagen.planted_redundancy(dfagen.random_dfa(n, k, 0.5, 70 + n), c, 71 + k)[0]
            for n, k, c in ((5000, 3, 7), (8000, 2, 8), (2000, 8, 30), (13_000, 5, 5))]
    dfas.append(dfagen.random_dfa(60_000, 2, 0.0, 9))       # no accepting state: one block
    dfas.append(dfagen.chain_dfa(20_000))                   # 19,999 rounds: the round tags wrap
    assert all(16_384 < A.n <= 65_536 for A in dfas)
    blocks, res = _batch(g, dfas, schedule=6)
    for i, (A, b, r) in enumerate(zip(dfas, blocks, res)):
        ref = oracle.moore(A.delta, A.accept)
        assert np.array_equal(b, ref.block), i
        assert (r.num_blocks, r.rounds_changed, r.rounds_executed) == \
            (ref.num_blocks, ref.rounds_changed, ref.rounds_executed), i
        if A.n < 30_000:
            assert np.array_equal(b, oracle.hopcroft(A.delta, A.accept)), i


@pytest.mark.parametrize("schedule", [0, 6])
def test_batch_recipe_both_paths(g, schedule):
    """512 DFAs of the batch recipe (64 to 65,536 states) and two beyond 65,536:
    with schedule 6 the DFAs that fit one block's shared memory, and those of
    up to 65,536 states with the table in global memory, are refined one per
    block, the two largest by the cooperative kernel, in the same call; every
    partition and round count equals the oracle's."""
    dfas = dfagen.batch_dfas(512, 64, 65_536, 2, 8, 0.3, 41)
    dfas += [dfagen.random_dfa(70_000, 3, 0.3, 42), dfagen.random_dfa(66_000, 8, 0.3, 43)]
    assert any(A.n > 16_384 for A in dfas) and any(A.n <= 16_384 for A in dfas)
    blocks, res = _batch(g, dfas, schedule=schedule)
    for i, (A, b, r) in enumerate(zip(dfas, blocks, res)):
        ref = oracle.moore(A.delta, A.accept)
        assert np.array_equal(b, ref.block), i
        assert (r.num_blocks, r.rounds_changed, r.rounds_executed) == \
            (ref.num_blocks, ref.rounds_changed, ref.rounds_executed), i


def test_batch_block_per_dfa_limits(g):
    """Round limit and an invalid target on the block-per-DFA path (both the
    shared-memory and the global-table refinement)."""
    dfas = [dfagen.chain_dfa(50), dfagen.random_dfa(100, 2, 0.5, 3), dfagen.random_dfa(30_000, 3, 0.5, 4),
            dfagen.chain_dfa(40_000)]
    blocks, res = _batch(g, dfas, schedule=6, max_rounds=3, check=False)
    for A, b, r in zip(dfas, blocks, res):
        ref = oracle.moore(A.delta, A.accept, max_rounds=3)
        assert np.array_equal(b, oracle.canonical(ref.block))
        assert r.rounds_executed == ref.rounds_executed
    assert res[0].status == g.DFA_EMAXROUNDS
    for nB in (50, 40_000):   # a DFA held in shared memory, and one with its table in global memory
        B = dfagen.random_dfa(nB, 2, 0.5, 4)
        B.delta[1][7] = nB
        with pytest.raises(g.DfaError):
            _batch(g, [dfagen.random_dfa(100, 2, 0.5, 3), B], schedule=6)
    _batch(g, [dfagen.random_dfa(100, 2, 0.5, 3)], schedule=6)   # the context survives


def test_batch_max_rounds(g):
    dfas = [dfagen.chain_dfa(50), dfagen.random_dfa(100, 2, 0.5, 3)]
    blocks, res = _batch(g, dfas, max_rounds=3, check=False)
    assert res[0].status == g.DFA_EMAXROUNDS and res[0].rounds_executed == 3
    ref = oracle.moore(dfas[0].delta, dfas[0].accept, max_rounds=3)
    assert np.array_equal(blocks[0], ref.block)


def test_batch_bad_delta(g):
    A = dfagen.random_dfa(100, 2, 0.5, 3)
    B = dfagen.random_dfa(50, 2, 0.5, 4)
    B.delta[1][7] = 50
    with pytest.raises(g.DfaError):
        _batch(g, [A, B])


# ---------------------------------------------------------------- packed (segment-offset) form

def _packed(g, dfas, device="cuda", **kw):
    n, k, d, a = g.pack_batch([(A.delta, A.accept) for A in dfas], device=device)
    out, res = g.minimise_batch_packed(n, k, d, a, **kw)
    blocks = out.cpu().numpy().view(np.uint32)
    offs = np.concatenate([[0], np.cumsum([A.n for A in dfas])])
    return [blocks[offs[i]:offs[i + 1]] for i in range(len(dfas))], res


@pytest.mark.parametrize("device", ["cuda", None])
def test_packed_equals_list_form(g, device):
    dfas = _mixed()
    pb, pr = _packed(g, dfas, device=device)
    lb, lr = _batch(g, dfas)
    for A, x, y, rx, ry in zip(dfas, pb, lb, pr, lr):
        assert np.array_equal(x, y)
        assert (rx.num_blocks, rx.rounds_changed, rx.rounds_executed) == \
            (ry.num_blocks, ry.rounds_changed, ry.rounds_executed)
        ref = oracle.moore(A.delta, A.accept)
        assert np.array_equal(x, ref.block)


@pytest.mark.parametrize("device", ["cuda", None])
def test_packed_letterless_dfas(g, device):
    """DFAs with no letters anywhere in the batch, first included (the packed
    delta then starts at the first DFA that has letters)."""
    dfas = [dfagen.random_dfa(5, 0, 0.5, 1), dfagen.random_dfa(300, 3, 0.5, 2), dfagen.random_dfa(7, 0, 0.5, 3),
            dfagen.random_dfa(1000, 2, 0.3, 4)]
    pb, pr = _packed(g, dfas, device=device)
    for A, b, r in zip(dfas, pb, pr):
        ref = oracle.moore(A.delta, A.accept)
        assert np.array_equal(b, ref.block)
        assert (r.rounds_changed, r.rounds_executed) == (ref.rounds_changed, ref.rounds_executed)
    only = [dfagen.random_dfa(9, 0, 0.5, 5), dfagen.random_dfa(4, 0, 0.5, 6)]
    ob, _ = _packed(g, only, device=device)
    for A, b in zip(only, ob):
        assert np.array_equal(b, oracle.moore(A.delta, A.accept).block)


def test_packed_bad_target_and_sizes(g):
    A = dfagen.random_dfa(100, 2, 0.5, 3)
    B = dfagen.random_dfa(50, 2, 0.5, 4)
    n, k, d, a = g.pack_batch([(A.delta, A.accept), (B.delta, B.accept)])
    d[2 * 100 + 7] = 50                      # DFA 1's targets are local: 50 is out of range
    with pytest.raises(g.DfaError) as e:
        g.minimise_batch_packed(n, k, d, a)
    assert e.value.status == g.DFA_EINVAL
    n2 = n.copy()
    n2[1] = 0
    with pytest.raises(g.DfaError):
        g.minimise_batch_packed(n2, k, d, a)


def test_packed_4096_full_size(g):
    """The 4,096-DFA workload in packed form equals the list form, DFA by DFA."""
    dfas = dfagen.batch_dfas(4096, 64, 65_536, 2, 8, 0.3, 4)
    pb, pr = _packed(g, dfas)
    lb, lr = _batch(g, dfas)
    for i in range(len(dfas)):
        assert np.array_equal(pb[i], lb[i]), i
        assert (pr[i].num_blocks, pr[i].rounds_executed) == (lr[i].num_blocks, lr[i].rounds_executed), i
