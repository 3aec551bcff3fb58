"""dfa_minimise_noalloc: the entry point for callers that cannot allocate.

Some callers cannot give the library a workspace: a host framework may own
every device allocation, or a latency-critical path may be forbidden to call
cudaMalloc because it can synchronise the device.  This test calls the
no-allocation entry point through the C ABI twice in a row (the second call on
a smaller DFA, after the first has left its data in the shared scratch) and
checks each result against dfa_minimise, bit for bit, and that sizes beyond
the fixed scratch are rejected with a clear error; concurrent calls from two
host threads serialise on the shared scratch, and a call under stream capture
is refused.

The file is named to be collected last.
"""
import numpy as np
import pytest

import dfagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2508_20735_gb300 as pkg
    pkg.build()
    return pkg


def _noalloc(g, A):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda()
    a = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
    out = torch.full((A.n,), -1, dtype=torch.int32, device="cuda")
    dd, keep = g.make_dfa(d, a)
    st, res = g.dfa_minimise_noalloc(dd, None, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, res, out.cpu().numpy().view(np.uint32)


def _reference(g, A):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda()
    a = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
    block, res = g.minimise(d, a)
    return res, block.cpu().numpy().view(np.uint32)


def test_noalloc_matches_dfa_minimise_twice(g):
    big = dfagen.random_dfa(60_000, 3, 0.5, 71)
    base = dfagen.random_dfa(500, 3, 0.5, 72)
    small, _ = dfagen.planted_redundancy(base, 4, 73)      # real merges, fewer states
    for A in (big, small):
        st, res, got = _noalloc(g, A)
        assert st == g.DFA_OK, g.last_error()
        ref_res, ref = _reference(g, A)
        assert np.array_equal(got, ref)
        assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
            (ref_res.num_blocks, ref_res.rounds_changed, ref_res.rounds_executed)


def test_noalloc_small_case_matches_oracle(g):
    """Independently of the GPU's own dfa_minimise: the canonical partition and
    round counts of a small planted-redundancy DFA equal the oracle's Moore
    refinement, on two calls in a row."""
    import oracle
    base = dfagen.random_dfa(400, 3, 0.5, 75)
    A, origin = dfagen.planted_redundancy(base, 5, 76)
    ref = oracle.moore(A.delta, A.accept)
    for _ in range(2):
        st, res, got = _noalloc(g, A)
        assert st == g.DFA_OK, g.last_error()
        assert np.array_equal(got, ref.block)
        assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
            (ref.num_blocks, ref.rounds_changed, ref.rounds_executed)


def test_noalloc_at_the_state_limit(g):
    """Exactly DFA_NOALLOC_MAX_STATES states fit the fixed scratch."""
    A = dfagen.random_dfa(65_536, 4, 0.5, 77)
    st, res, got = _noalloc(g, A)
    assert st == g.DFA_OK, g.last_error()
    ref_res, ref = _reference(g, A)
    assert np.array_equal(got, ref)
    assert res.rounds_executed == ref_res.rounds_executed


def test_noalloc_rejects_too_many_states(g):
    A = dfagen.random_dfa(65_537, 2, 0.5, 74)
    st, res, _ = _noalloc(g, A)
    assert st == g.DFA_EINVAL
    assert "at most 65536 states" in g.last_error()


def test_noalloc_concurrent_threads_on_two_streams(g):
    """Two host threads, each on its own stream, call the no-allocation entry
    point in a loop on different DFAs.  The calls share one scratch array; the
    per-device lock makes them run one after another, so every result equals
    the oracle's."""
    import threading
    import torch
    import oracle
    As = []
    for i in range(2):
        base = dfagen.random_dfa(300 + 200 * i, 3, 0.5, 80 + i)
        A, _ = dfagen.planted_redundancy(base, 4 + i, 90 + i)
        As.append(A)
    refs = [oracle.moore(A.delta, A.accept) for A in As]
    results = [[], []]

    def work(i):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for _ in range(6):
                st, res, got = _noalloc(g, As[i])
                results[i].append((st, res.num_blocks, res.rounds_executed, got))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for i in range(2):
        assert len(results[i]) == 6
        for st, nb, rx, got in results[i]:
            assert st == g.DFA_OK
            assert np.array_equal(got, refs[i].block)
            assert (nb, rx) == (refs[i].num_blocks, refs[i].rounds_executed)


def test_noalloc_refuses_graph_capture(g):
    """On a stream that is being captured the call enqueues nothing and
    returns DFA_EINVAL; the next ordinary call still works."""
    import torch
    A = dfagen.random_dfa(1_000, 2, 0.5, 78)
    d = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda()
    a = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
    out = torch.full((A.n,), -1, dtype=torch.int32, device="cuda")
    dd, keep = g.make_dfa(d, a)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        st, _ = g.dfa_minimise_noalloc(dd, None, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == g.DFA_EINVAL
    assert "captured" in g.last_error()
    assert int((out == -1).sum()) == A.n     # nothing ran
    st, res, got = _noalloc(g, A)
    assert st == g.DFA_OK, g.last_error()
    ref_res, ref = _reference(g, A)
    assert np.array_equal(got, ref)
