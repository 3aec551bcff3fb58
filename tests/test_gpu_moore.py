"""GPU parity: signature refinement (Moore / sortPR semantics) and equivalence
through the C ABI, element by element against the CPU oracle.

All partitions are compared bit for bit in canonical numbering; round counts
must match exactly.  Integer work: the tolerance is zero.
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


def _gpu_moore(g, A, **kw):
    d, a = _dev(A)
    block, res = g.minimise(d, a, **kw)
    return block.cpu().numpy().view(np.uint32), res


def _assert_parity(g, A, ref=None, **kw):
    ref = ref or oracle.moore(A.delta, A.accept)
    got, res = _gpu_moore(g, A, **kw)
    assert np.array_equal(got, ref.block)
    assert res.num_blocks == ref.num_blocks
    assert (res.rounds_changed, res.rounds_executed) == (ref.rounds_changed, ref.rounds_executed), ref.counts
    return res


def test_config1_random_n10000_k2(g):
    A = dfagen.random_dfa(10_000, 2, 0.5, 1)
    _assert_parity(g, A)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 7, 63, 64, 65, 511, 512, 513, 1000, 4097, 65_537, 100_003, 262_144])
@pytest.mark.parametrize("k", [0, 1, 2, 3, 5])
def test_random_sizes_ragged(g, n, k):
    A = dfagen.random_dfa(n, k, 0.5, 1000 + n + k)
    _assert_parity(g, A)


@pytest.mark.parametrize("n", [1, 2, 7, 8, 9, 63, 65, 127, 129, 513, 4097, 10_000, 16_383, 16_384])
@pytest.mark.parametrize("k", [0, 1, 2, 5, 9])
def test_small_sizes_all_kernels(g, n, k):
    """Up to 16,384 states the default call picks the single-block or the
    cluster kernel; DFA_FLAG_ONE_BLOCK and DFA_FLAG_CLUSTER force either (the
    cooperative kernel where it does not fit), and an explicit schedule (1)
    runs the cooperative kernel.  All equal the oracle.  Sizes span slices
    that end inside a CTA, CTAs with no states, and signatures wide enough for
    the representative comparison (k = 9)."""
    A = dfagen.random_dfa(n, k, 0.5, 5000 + n + k)
    ref = oracle.moore(A.delta, A.accept)
    _assert_parity(g, A, ref)
    _assert_parity(g, A, ref, flags=g.DFA_FLAG_ONE_BLOCK)
    _assert_parity(g, A, ref, flags=g.DFA_FLAG_CLUSTER)
    _assert_parity(g, A, ref, schedule=1)


@pytest.mark.parametrize("n,k,copies", [(2000, 2, 8), (500, 4, 30), (300, 12, 40), (3000, 3, 5)])
def test_small_kernels_real_merges(g, n, k, copies):
    """Planted redundancy (every block has several members) on the cluster and
    single-block kernels, against the oracle and Hopcroft's partition."""
    base = dfagen.random_dfa(n, k, 0.5, 70 + n)
    A, _ = dfagen.planted_redundancy(base, copies, 71 + k)
    if A.n > 16_384:
        pytest.skip("beyond the small kernels")
    ref = oracle.moore(A.delta, A.accept)
    assert np.array_equal(ref.block, oracle.hopcroft(A.delta, A.accept))
    stop = oracle.moore(A.delta, A.accept, stop_discrete=True)
    for flags in (g.DFA_FLAG_CLUSTER, g.DFA_FLAG_ONE_BLOCK):
        _assert_parity(g, A, ref, flags=flags)
        _assert_parity(g, A, stop, flags=flags | g.DFA_FLAG_STOP_DISCRETE)


@pytest.mark.parametrize("one_block", [False, True])
def test_small_kernel_deep_chain_and_limits(g, one_block):
    """The small kernels on the 16,384-state chain: 16,383 rounds to the
    fixpoint; a round limit and a time limit end them with their statuses."""
    flags = g.DFA_FLAG_ONE_BLOCK if one_block else g.DFA_FLAG_CLUSTER
    C = dfagen.chain_dfa(16_384)
    res = _assert_parity(g, C, flags=flags)
    assert res.rounds_changed == 16_382
    d, a = _dev(C)
    block, res = g.minimise(d, a, max_rounds=7, check=False, flags=flags)
    assert res.call_status == g.DFA_EMAXROUNDS and res.rounds_executed == 7
    ref = oracle.moore(C.delta, C.accept, max_rounds=7)
    assert np.array_equal(block.cpu().numpy().view(np.uint32), oracle.canonical(ref.block))
    _, res = g.minimise(d, a, timeout_ns=200_000, check=False, flags=flags)   # 0.2 ms: far below the work
    assert res.call_status == g.DFA_ETIMEOUT
    _assert_parity(g, dfagen.random_dfa(4096, 2, 0.5, 1), flags=flags)     # the context survives


def test_small_kernels_bad_target(g):
    """An invalid transition target is reported by both small kernels (staged
    δ and δ read from global memory), and the context survives."""
    for n, k in ((1000, 2), (16_000, 12)):
        A = dfagen.random_dfa(n, k, 0.5, 77)
        A.delta[k - 1][n // 2] = n
        d, a = _dev(A)
        for flags in (0, g.DFA_FLAG_ONE_BLOCK, g.DFA_FLAG_CLUSTER):
            _, res = g.minimise(d, a, check=False, flags=flags)
            assert res.call_status == g.DFA_EINVAL
    _assert_parity(g, dfagen.random_dfa(1000, 2, 0.5, 78))


@pytest.mark.parametrize("schedule", [1, 2, 4])
@pytest.mark.parametrize("n,k", [(4096, 2), (100_000, 4), (30_001, 3)])
def test_vector_widths(g, schedule, n, k):
    """Every kernel width (states per thread) gives the same result."""
    A = dfagen.random_dfa(n, k, 0.5, 31 + n)
    _assert_parity(g, A, schedule=schedule)


@pytest.mark.parametrize("n,k,seed", [(10_000, 2, 1), (300_000, 4, 2), (65_536, 3, 3), (4097, 8, 4)])
def test_table_only_path(g, n, k, seed):
    """Renumbering through the exact table in every round (no direct or filter
    rounds) gives the same partition and round counts."""
    A = dfagen.random_dfa(n, k, 0.5, seed)
    _assert_parity(g, A, flags=g.DFA_FLAG_TABLE_ONLY)


@pytest.mark.parametrize("p", [0.0, 1.0, 0.01, 0.3, 0.9])
def test_acceptance_extremes(g, p):
    A = dfagen.random_dfa(5000, 3, p, 7)
    _assert_parity(g, A)


@pytest.mark.parametrize("n,k", [(10_000, 8), (20_000, 12), (3000, 40), (777, 100), (14_462, 8), (300, 130),
                                 (1000, 200)])
def test_multi_stage_keys(g, n, k):
    """Signatures wider than one 128-bit key are renumbered in several exact stages."""
    A = dfagen.random_dfa(n, k, 0.5, n + k)
    _assert_parity(g, A)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_planted_redundancy(g, seed):
    """Real merges: the expected partition is 'copies of the same state'."""
    base = dfagen.random_dfa(3000, 3 + seed % 3, 0.5, seed + 40)
    assert oracle.hopcroft(base.delta, base.accept).max() + 1 == base.n     # the base is minimal
    P, origin = dfagen.planted_redundancy(base, 6, seed)
    ref = oracle.moore(P.delta, P.accept)
    assert np.array_equal(ref.block, oracle.canonical(origin))
    _assert_parity(g, P, ref)


@pytest.mark.parametrize("k", [30, 60])
def test_planted_wide_keys(g, k):
    """Copies of a minimal DFA whose signatures are wider than one 125-bit key:
    filter rounds join the copies through the hashed exact insert (signature
    hash plus full comparison)."""
    base = dfagen.random_dfa(400, k, 0.5, 40 + k)
    P, origin = dfagen.planted_redundancy(base, 5, k)
    res = _assert_parity(g, P)
    assert res.num_blocks == base.n
    assert np.array_equal(_gpu_moore(g, P)[0], oracle.canonical(origin))


def test_few_targets_heavy_merging(g):
    """Targets restricted to a few states: most states are equivalent, blocks are huge."""
    n, k = 200_000, 3
    d = dfagen.bounded(9, 91, n * k, 5).reshape(k, n)
    acc = dfagen.bernoulli(9, 92, n, 0.5)
    _assert_parity(g, dfagen.DFA(d, acc, 0))


@pytest.mark.parametrize("i", [8, 12, 16])
def test_fibonacci(g, i):
    A = dfagen.fibonacci_dfa(i)
    res = _assert_parity(g, A)
    assert res.num_blocks == A.n and res.rounds_executed == A.n - 1


@pytest.mark.parametrize("m", [3, 8, 12, 15])
def test_bit_splitters(g, m):
    B = dfagen.bit_splitter(m)
    res = _assert_parity(g, B)
    assert res.rounds_changed == m - 1


def test_chain_deep_rounds(g):
    C = dfagen.chain_dfa(1 << 12)
    res = _assert_parity(g, C)
    assert res.rounds_changed == (1 << 12) - 2


def test_cycle(g):
    C = dfagen.cycle_dfa(14)
    _assert_parity(g, C)


def test_host_buffers_e2e(g):
    """Host (numpy) inputs and output go through the same call: staged copies."""
    A = dfagen.random_dfa(50_000, 3, 0.5, 17)
    ref = oracle.moore(A.delta, A.accept)
    block, res = g.minimise(A.delta, A.accept)
    assert isinstance(block, np.ndarray)
    assert np.array_equal(block, ref.block)
    assert res.rounds_executed == ref.rounds_executed


def test_deterministic(g):
    A = dfagen.random_dfa(300_000, 4, 0.5, 3)
    a, r1 = _gpu_moore(g, A)
    b, r2 = _gpu_moore(g, A)
    assert np.array_equal(a, b) and r1.rounds_executed == r2.rounds_executed


def test_large_random_2p22(g):
    """A quarter of the 2^24-state workload, compared in full with the oracle."""
    A = dfagen.random_dfa(1 << 22, 4, 0.5, 2)
    _assert_parity(g, A)


def test_bench_workload_2p24(g):
    """The bench workload itself (2^24 states, 4 letters, seed 2), in full."""
    A = dfagen.random_dfa(1 << 24, 4, 0.5, 2)
    _assert_parity(g, A)


# ---------------------------------------------------------------- stopping at n blocks

def _stop_cases():
    return [dfagen.random_dfa(10_000, 2, 0.5, 1), dfagen.random_dfa(300_000, 4, 0.5, 2),
            dfagen.random_dfa(1, 2, 0.5, 4), dfagen.random_dfa(2, 1, 0.5, 5), dfagen.random_dfa(5000, 0, 0.5, 6),
            dfagen.fibonacci_dfa(12), dfagen.bit_splitter(12), dfagen.chain_dfa(4096),
            dfagen.planted_redundancy(dfagen.random_dfa(300, 3, 0.5, 61), 5, 2)[0],
            dfagen.random_dfa(3000, 40, 0.5, 7), dfagen.random_dfa(65_537, 3, 0.3, 8)]


@pytest.mark.parametrize("table_only", [False, True])
@pytest.mark.parametrize("idx", range(11))
def test_stop_discrete(g, idx, table_only):
    A = _stop_cases()[idx]
    ref = oracle.moore(A.delta, A.accept, stop_discrete=True)
    flags = g.DFA_FLAG_STOP_DISCRETE | (g.DFA_FLAG_TABLE_ONLY if table_only else 0)
    _assert_parity(g, A, ref=ref, flags=flags)


def test_stop_discrete_bench_workload_2p24(g):
    """The 2^24-state workload ends discrete: stopping at n blocks gives the
    identity partition one round earlier than the plain loop (itself checked in
    full against the oracle above)."""
    A = dfagen.random_dfa(1 << 24, 4, 0.5, 2)
    plain, rp = _gpu_moore(g, A)
    got, rs = _gpu_moore(g, A, flags=g.DFA_FLAG_STOP_DISCRETE)
    assert rp.num_blocks == A.n and rs.num_blocks == A.n
    assert np.array_equal(got, np.arange(A.n, dtype=np.uint32))
    assert rs.rounds_changed == rp.rounds_changed == rs.rounds_executed == rp.rounds_executed - 1


# ---------------------------------------------------------------- errors

def test_bad_transition_target(g):
    A = dfagen.random_dfa(1000, 2, 0.5, 5)
    A.delta[1][123] = 1000
    with pytest.raises(g.DfaError) as e:
        _gpu_moore(g, A)
    assert e.value.status == g.DFA_EINVAL


def test_workspace_too_small(g):
    import torch
    A = dfagen.random_dfa(1000, 2, 0.5, 5)
    d, a = _dev(A)
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(g.DfaError) as e:
        g.minimise(d, a, workspace=ws)
    assert e.value.status == g.DFA_EINVAL and "workspace too small" in str(e.value)


def test_max_rounds(g):
    C = dfagen.chain_dfa(256)
    d, a = _dev(C)
    block, res = g.minimise(d, a, max_rounds=5, check=False)
    assert res.call_status == g.DFA_EMAXROUNDS and res.rounds_executed == 5
    ref = oracle.moore(C.delta, C.accept, max_rounds=5)
    assert np.array_equal(block.cpu().numpy().view(np.uint32), oracle.canonical(ref.block))


def test_timeout_returns_status_and_context_survives(g):
    """A call-time limit far below the work needed ends the launch with
    DFA_ETIMEOUT (device-side, no fault); the next call on the context works."""
    C = dfagen.chain_dfa(1 << 16)             # 65,535 rounds
    d, a = _dev(C)
    _, res = g.minimise(d, a, timeout_ns=2_000_000, check=False)   # 2 ms
    assert res.call_status == g.DFA_ETIMEOUT
    A = dfagen.random_dfa(4096, 2, 0.5, 1)
    _assert_parity(g, A)


# ---------------------------------------------------------------- equivalence

@pytest.mark.parametrize("req", range(12))
def test_equivalence_pairs(g, req):
    A, B, expect = dfagen.equivalence_pair(req, 5, n_lo=1000, n_hi=60_000)
    eq, res = g.equivalent((A.delta, A.accept, A.start), (B.delta, B.accept, B.start))
    assert eq == expect
    ref = oracle.equivalent(A.delta, A.accept, A.start, B.delta, B.accept, B.start)
    assert eq == ref.equivalent
    assert (res.num_blocks, res.rounds_executed) == (ref.refine.num_blocks, ref.refine.rounds_executed)
    eq2, res2 = g.equivalent((A.delta, A.accept, A.start), (B.delta, B.accept, B.start), early_exit=True)
    assert eq2 == expect
    if not expect:
        cex = oracle.shortest_cex(A.delta, A.accept, A.start, B.delta, B.accept, B.start)
        assert res2.rounds_executed == cex


@pytest.mark.parametrize("req", range(6))
def test_equivalence_stop_discrete(g, req):
    A, B, expect = dfagen.equivalence_pair(100 + req, 5, n_lo=1000, n_hi=60_000)
    args = (A.delta, A.accept, A.start, B.delta, B.accept, B.start)
    for early in (False, True):
        eq, res = g.equivalent(args[:3], args[3:], early_exit=early, flags=g.DFA_FLAG_STOP_DISCRETE)
        ref = oracle.equivalent(*args, early_exit=early, stop_discrete=True)
        assert eq == expect == ref.equivalent
        assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
            (ref.refine.num_blocks, ref.refine.rounds_changed, ref.refine.rounds_executed)


def test_equivalence_start_acceptance_differs(g):
    C = dfagen.cycle_dfa(7)
    s2 = int(np.nonzero(C.accept)[0][0])
    eq, res = g.equivalent((C.delta, C.accept, 0), (C.delta, C.accept, s2), early_exit=True)
    assert not eq and res.rounds_executed == 0
    eq, res = g.equivalent((C.delta, C.accept, 0), (C.delta, C.accept, s2))
    assert not eq


def test_equivalence_self(g):
    A = dfagen.random_dfa(12_345, 2, 0.5, 8)
    eq, _ = g.equivalent((A.delta, A.accept, 3), (A.delta, A.accept, 3))
    assert eq


# ---------------------------------------------------------------- stream-ordered calls

def test_async_pipeline_equals_oracle(g):
    """dfa_minimise_async on two streams with two workspaces, each call issued
    before the previous one on the other stream has finished, host and device
    buffers alternating: every partition and round count equals the oracle's."""
    import torch
    dfas = [dfagen.random_dfa(n, k, 0.5, s) for n, k, s in ((10_000, 2, 1), (300_000, 4, 2), (4097, 3, 3),
                                                             (65_536, 8, 4), (1, 2, 5), (200_000, 2, 6))]
    dfas.append(dfagen.planted_redundancy(dfagen.random_dfa(3000, 3, 0.5, 7), 5, 2)[0])
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    opts = g.make_opts("moore")
    nmax, kmax = max(A.n for A in dfas), max(A.k for A in dfas)
    probe, _ = g.make_dfa(np.zeros((kmax, nmax), np.uint32), np.zeros(nmax, np.uint8))
    wsb = g.dfa_workspace_size(probe, opts)
    ws = [g._workspace(wsb), g._workspace(wsb)]
    keep, pending = [], {}
    for i, A in enumerate(dfas):
        s = i % 2
        if s in pending:
            j = pending.pop(s)
            _check_async(g, dfas[j], keep[j], ws[s], streams[s])
        if i % 4 < 2:   # host buffers (pinned)
            arrs = (torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).pin_memory(),
                    torch.from_numpy(np.ascontiguousarray(A.accept)).pin_memory())
            out = torch.empty(A.n, dtype=torch.int32).pin_memory()
        else:
            arrs = (torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda(),
                    torch.from_numpy(np.ascontiguousarray(A.accept)).cuda())
            out = torch.empty(A.n, dtype=torch.int32, device="cuda")
        d, k2 = g.make_dfa(arrs[0], arrs[1])
        keep.append((d, k2, arrs, out))
        assert g.minimise_async(d, opts, out.data_ptr(), ws[s].data_ptr(), wsb, streams[s].cuda_stream) == g.DFA_OK
        pending[s] = i
    for s, j in pending.items():
        _check_async(g, dfas[j], keep[j], ws[s], streams[s])


def _check_async(g, A, kept, ws, stream):
    st, res = g.minimise_result(ws.data_ptr(), stream.cuda_stream)
    assert st == g.DFA_OK, g.last_error()
    out = kept[3]
    got = out.cpu().numpy().view(np.uint32) if out.is_cuda else out.numpy().view(np.uint32)
    ref = oracle.moore(A.delta, A.accept)
    assert np.array_equal(got, ref.block)
    assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
        (ref.num_blocks, ref.rounds_changed, ref.rounds_executed)


def test_async_reports_device_errors(g):
    import torch
    A = dfagen.random_dfa(1000, 2, 0.5, 5)
    bad = A.delta.copy()
    bad[0][3] = 5000
    d, keep = g.make_dfa(bad, A.accept)
    opts = g.make_opts("moore")
    wsb = g.dfa_workspace_size(d, opts)
    ws = g._workspace(wsb)
    out = np.empty(A.n, dtype=np.uint32)
    s = torch.cuda.Stream()
    assert g.minimise_async(d, opts, out.ctypes.data, ws.data_ptr(), wsb, s.cuda_stream) == g.DFA_OK
    st, _ = g.minimise_result(ws.data_ptr(), s.cuda_stream)
    assert st == g.DFA_EINVAL
    opts_naive = g.make_opts("naive")
    assert g.minimise_async(d, opts_naive, out.ctypes.data, ws.data_ptr(), wsb, s.cuda_stream) == g.DFA_EINVAL


def test_many_letters_large_against_oracle(g):
    """From 2^20 states on, a DFA with many letters takes filter rounds while the
    previous round's blocks are still few (B^(k+1) >= 64 n): the partition and
    rounds still equal the oracle's."""
    A = dfagen.random_dfa((1 << 20) + 3, 8, 0.5, 21)
    _assert_parity(g, A, ref=oracle.moore(A.delta, A.accept))



@pytest.mark.parametrize("n,k", [(1000, 2), (10_000, 3), (333, 5)])
def test_small_kernels_unaligned_inputs(g, n, k):
    """δ and the acceptance bytes at addresses that are not 16-byte aligned
    (4 bytes and 1 byte past an aligned start): the small kernels stage them
    with plain loads instead of 16-byte ones, and the cooperative kernel picks
    its narrow width; the results equal the oracle's."""
    import torch
    A = dfagen.random_dfa(n, k, 0.5, 600 + n + k)
    ref = oracle.moore(A.delta, A.accept)
    dbuf = torch.zeros(k * n + 1, dtype=torch.int32, device="cuda")
    dbuf[1:] = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32).ravel()).cuda()
    abuf = torch.zeros(n + 3, dtype=torch.uint8, device="cuda")
    abuf[3:] = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
    d, a = dbuf[1:], abuf[3:]
    assert d.data_ptr() % 16 != 0 and a.data_ptr() % 16 != 0
    for kw in ({"flags": g.DFA_FLAG_ONE_BLOCK}, {"flags": g.DFA_FLAG_CLUSTER}, {}, {"schedule": 1}):
        block, res = g.minimise(d.view(k, n), a, **kw)
        assert np.array_equal(block.cpu().numpy().view(np.uint32), ref.block)
        assert (res.rounds_changed, res.rounds_executed) == (ref.rounds_changed, ref.rounds_executed)


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_small_union_equivalence_all_kernels(g, seed):
    """Equivalence by union for unions of at most 16,384 states: the single
    block, the cluster and the cooperative kernel give the same verdict and
    the same refinement (rounds, blocks), with and without early exit, and
    the verdict equals the oracle's; start states apart by acceptance alone
    take round 0."""
    pairs = [dfagen.equivalence_pair(seed * 10 + i, 17, n_lo=200, n_hi=7000) for i in range(3)]
    A = dfagen.random_dfa(900 + seed, 2, 0.5, seed)
    B_acc = A.accept.copy()
    B_acc[A.start] ^= 1
    pairs.append((A, dfagen.DFA(A.delta.copy(), B_acc, A.start), False))
    for A, B, expect in pairs:
        if A.n + B.n > 16_384:
            continue
        args = ((A.delta, A.accept, A.start), (B.delta, B.accept, B.start))
        ref = oracle.equivalent(A.delta, A.accept, A.start, B.delta, B.accept, B.start)
        assert ref.equivalent == bool(expect)
        for early in (False, True):
            base_eq, base = g.equivalent(*args, early_exit=early, schedule=1)   # cooperative kernel
            assert base_eq == bool(expect)
            for flags in (0, g.DFA_FLAG_ONE_BLOCK, g.DFA_FLAG_CLUSTER):
                eq, res = g.equivalent(*args, early_exit=early, flags=flags)
                assert eq == base_eq, (flags, early)
                assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
                    (base.num_blocks, base.rounds_changed, base.rounds_executed), (flags, early)
