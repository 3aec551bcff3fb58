"""GPU parity: dfa_quotient (the minimal DFA from the partition) against the
oracle's quotient, element by element, on device and host buffers."""
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


def _check(g, A, device=True):
    import torch
    blk = oracle.moore(A.delta, A.accept).block
    ref = oracle.quotient(A.delta, A.accept, A.start, blk)
    if device:
        d = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda()
        a = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
        b = torch.from_numpy(blk.view(np.int32)).cuda()
        qd, qa, qs = g.quotient(d, a, A.start, b)
        qd, qa = qd.cpu().numpy().view(np.uint32), qa.cpu().numpy()
    else:
        qd, qa, qs = g.quotient(A.delta, A.accept, A.start, blk)
    assert qs == ref.start
    assert qd.shape == ref.delta.shape
    assert np.array_equal(qd, ref.delta) and np.array_equal(qa, ref.accept)
    return ref


@pytest.mark.parametrize("n,k,p", [(1, 2, 0.5), (2, 1, 0.5), (7, 3, 0.5), (100, 2, 0.5), (1000, 3, 0.3),
                                   (4097, 2, 0.5), (100_000, 4, 0.5), (3000, 0, 0.5), (2000, 5, 0.0)])
def test_random(g, n, k, p):
    _check(g, dfagen.random_dfa(n, k, p, 900 + n + k))


@pytest.mark.parametrize("req", range(6))
def test_equivalence_pairs_with_junk(g, req):
    A, B, _ = dfagen.equivalence_pair(req, 11, n_lo=200, n_hi=20_000)
    for X in (A, B):
        ref = _check(g, X)
        assert ref.n <= int(oracle.reachable(X.delta, X.start).sum())


def test_planted_fibonacci_chain_cycle(g):
    base = dfagen.random_dfa(500, 3, 0.5, 81)
    P, _ = dfagen.planted_redundancy(base, 5, 4)
    _check(g, P)
    _check(g, dfagen.fibonacci_dfa(16))        # a unary cycle: deep search, block 0 alone
    _check(g, dfagen.chain_dfa(5000))
    _check(g, dfagen.cycle_dfa(11))


def test_deep_unary_fibonacci_full(g):
    """Fibonacci with 121,393 states, minimal (Table 2) and a single cycle: the
    search runs 121,392 levels and the quotient of the identity partition is the
    DFA itself."""
    import torch
    A = dfagen.fibonacci_dfa(25)
    d = torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda()
    a = torch.from_numpy(np.ascontiguousarray(A.accept)).cuda()
    b = torch.arange(A.n, dtype=torch.int32, device="cuda")
    qd, qa, qs = g.quotient(d, a, A.start, b)
    assert qs == A.start
    assert np.array_equal(qd.cpu().numpy().view(np.uint32), A.delta)
    assert np.array_equal(qa.cpu().numpy(), A.accept)


def test_host_buffers_and_errors(g):
    _check(g, dfagen.random_dfa(3000, 2, 0.5, 82), device=False)
    A = dfagen.random_dfa(100, 2, 0.5, 83)
    blk = oracle.moore(A.delta, A.accept).block.copy()
    blk[7] = 100
    with pytest.raises(g.DfaError) as e:
        g.quotient(A.delta, A.accept, A.start, blk)
    assert e.value.status == g.DFA_EINVAL
