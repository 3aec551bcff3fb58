"""GPU: the serving loop (continuous batching).  Every request's result in a
mix -- requests submitted while others are being refined, admitted as slots
and arena space free up -- equals the stand-alone call's and the oracle's."""
import time

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


def _requests():
    reqs = []
    for i in range(24):
        if i % 3 == 0:
            A = dfagen.random_dfa(200 + 397 * i, 2 + i % 3, 0.5, 300 + i)
            reqs.append(("min", A))
        else:
            A, B, eq = dfagen.equivalence_pair(i, 5, n_lo=500, n_hi=40_000)
            reqs.append(("eq", (A, B, eq)))
    base = dfagen.random_dfa(500, 3, 0.5, 71)
    reqs.append(("min", dfagen.planted_redundancy(base, 4, 3)[0]))
    reqs.append(("min", dfagen.fibonacci_dfa(12)))
    reqs.append(("min", dfagen.random_dfa(3000, 40, 0.5, 5)))      # multi-stage keys
    return reqs


@pytest.mark.parametrize("slots,budget_mb", [(64, 2048), (3, 64)])
def test_mix_equals_alone(g, slots, budget_mb):
    reqs = _requests()
    with g.Server(budget_mb << 20, max_slots=slots) as srv:
        tickets = []
        for j, (kind, item) in enumerate(reqs):
            if kind == "min":
                tickets.append(srv.submit_minimise(item.delta, item.accept))
            else:
                A, B, _ = item
                tickets.append(srv.submit_equivalent((A.delta, A.accept, A.start), (B.delta, B.accept, B.start),
                                                     early_exit=(j % 2 == 0)))
            if j % 5 == 4:
                time.sleep(0.002)          # later requests arrive while earlier ones run
        for j, ((kind, item), t) in enumerate(zip(reqs, tickets)):
            if kind == "min":
                st, res, _, blocks = srv.wait(t, n=item.n)
                assert st == g.DFA_OK, g.last_error()
                ref = oracle.moore(item.delta, item.accept)
                assert np.array_equal(blocks, ref.block)
                assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
                    (ref.num_blocks, ref.rounds_changed, ref.rounds_executed)
            else:
                A, B, expect = item
                st, res, eq, _ = srv.wait(t)
                assert st == g.DFA_OK, g.last_error()
                assert eq == int(expect)
                alone_eq, alone = g.equivalent((A.delta, A.accept, A.start), (B.delta, B.accept, B.start),
                                               early_exit=(j % 2 == 0))
                assert bool(eq) == alone_eq
                assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
                    (alone.num_blocks, alone.rounds_changed, alone.rounds_executed)
        s = srv.stats()
        assert s["p50_us"] > 0 and s["p99_us"] >= s["p50_us"] and s["throughput_rps"] > 0
        c = srv.counters()
        assert c["steps"] > 0 and c["request_rounds"] >= len(reqs) and c["step_us"] > 0
        assert c["state_rounds"] == c["state_rounds_direct"] + c["state_rounds_filter"] + c["state_rounds_table"]


def test_poll_busy_then_done(g):
    C = dfagen.chain_dfa(1 << 12)      # thousands of rounds: still running at the first poll
    with g.Server(256 << 20, max_slots=4) as srv:
        t = srv.submit_minimise(C.delta, C.accept)
        st, *_ = srv.poll(t)
        assert st == g.DFA_EBUSY
        st, res, _, blocks = srv.wait(t, n=C.n)
        assert st == g.DFA_OK and res.rounds_changed == C.n - 2
        assert np.array_equal(blocks, np.arange(C.n, dtype=np.uint32))


def test_request_beyond_budget_and_destroy_with_pending(g):
    big = dfagen.random_dfa(1 << 20, 4, 0.5, 1)
    srv = g.Server(16 << 20, max_slots=2)
    with pytest.raises(g.DfaError) as e:
        srv.submit_minimise(big.delta, big.accept)
    assert e.value.status == g.DFA_ENOMEM
    for i in range(6):
        A = dfagen.random_dfa(20_000, 2, 0.5, i)
        srv.submit_minimise(A.delta, A.accept)
    srv.close()        # cancels what is still queued; must not hang


def _as(kind, X):
    """X's arrays as numpy (pageable host), pinned host tensors or device tensors."""
    import torch
    d = np.ascontiguousarray(X.delta)
    a = np.ascontiguousarray(X.accept)
    if kind == "numpy":
        return d, a
    td, ta = torch.from_numpy(d.view(np.int32)), torch.from_numpy(a)
    if kind == "pinned":
        return td.pin_memory(), ta.pin_memory()
    return td.cuda(), ta.cuda()


def test_concurrent_submitters_and_input_kinds(g):
    """Four client threads submit at once (the C call releases the GIL), with
    pageable, pinned and device inputs; every verdict and round count equals the
    stand-alone call's."""
    import threading
    pairs = [dfagen.equivalence_pair(i, 23, n_lo=300, n_hi=30_000) for i in range(24)]
    kinds = ("numpy", "pinned", "device")
    results = {}
    with g.Server(1 << 30, max_slots=16) as srv:
        def client(c):
            for i in range(c, len(pairs), 4):
                A, B, _ = pairs[i]
                ka, kb = kinds[i % 3], kinds[(i + c) % 3]
                t = srv.submit_equivalent(_as(ka, A) + (A.start,), _as(kb, B) + (B.start,))
                results[i] = srv.wait(t)
        threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
    assert sorted(results) == list(range(len(pairs)))
    for i, (A, B, expect) in enumerate(pairs):
        st, res, eq, _ = results[i]
        assert st == g.DFA_OK
        assert eq == int(expect)
        alone_eq, alone = g.equivalent((A.delta, A.accept, A.start), (B.delta, B.accept, B.start))
        assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
            (alone.num_blocks, alone.rounds_changed, alone.rounds_executed)


def test_start_states_apart_with_early_exit(g):
    """Start states of different acceptance: with early exit the verdict needs
    no round (the empty word separates them), for host and device inputs."""
    A = dfagen.random_dfa(1000, 2, 0.5, 3)
    B_acc = A.accept.copy()
    B_acc[A.start] ^= 1
    B = dfagen.DFA(A.delta.copy(), B_acc, A.start)
    with g.Server(256 << 20, max_slots=4) as srv:
        for kind in ("numpy", "device"):
            t = srv.submit_equivalent(_as(kind, A) + (A.start,), _as(kind, B) + (B.start,), early_exit=True)
            st, res, eq, _ = srv.wait(t)
            assert st == g.DFA_OK and eq == 0 and res.rounds_executed == 0
            t = srv.submit_equivalent(_as(kind, A) + (A.start,), _as(kind, B) + (B.start,))
            st, res, eq, _ = srv.wait(t)
            assert st == g.DFA_OK and eq == 0
            assert res.rounds_executed == oracle.equivalent(A.delta, A.accept, A.start, B.delta, B.accept,
                                                            B.start).refine.rounds_executed


def test_bad_targets_fail_alone(g):
    """A request whose targets are out of range finishes with DFA_EINVAL
    (validated on the device); requests beside it are unaffected."""
    good = dfagen.random_dfa(5000, 3, 0.5, 8)
    bad_delta = good.delta.copy()
    bad_delta[2][17] = good.n + 5
    with g.Server(512 << 20, max_slots=8) as srv:
        t_bad = srv.submit_minimise(bad_delta, good.accept)
        t_good = srv.submit_minimise(good.delta, good.accept)
        st, *_ = srv.wait(t_bad)
        assert st == g.DFA_EINVAL
        st, res, _, blocks = srv.wait(t_good, n=good.n)
        assert st == g.DFA_OK
        assert np.array_equal(blocks, oracle.moore(good.delta, good.accept).block)


def test_served_equivalence_recipe_full_sizes(g):
    """The served-equivalence workload at its full sizes (A: n log-uniform in
    [1e3, 1e6], k in {2, 4}; B a renamed copy plus junk, half with a reachable
    accepting bit flipped): 2,000 Poisson-free requests cycling through 32
    generated pairs; every verdict is the generator's and every round count
    equals the stand-alone dfa_equivalent call's."""
    import torch
    pairs = [dfagen.equivalence_pair(i, 5) for i in range(32)]
    dev = [((torch.from_numpy(A.delta.view(np.int32)).cuda(), torch.from_numpy(A.accept).cuda(), A.start),
            (torch.from_numpy(B.delta.view(np.int32)).cuda(), torch.from_numpy(B.accept).cuda(), B.start), eq)
           for A, B, eq in pairs]
    alone = [g.equivalent(a, b)[1] for a, b, _ in dev]
    with g.Server(24 << 30, max_slots=64) as srv:
        tickets = [srv.submit_equivalent(dev[i % 32][0], dev[i % 32][1]) for i in range(2000)]
        for i, t in enumerate(tickets):
            st, res, eq, _ = srv.wait(t)
            assert st == g.DFA_OK
            assert eq == int(dev[i % 32][2])
            ref = alone[i % 32]
            assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
                (ref.num_blocks, ref.rounds_changed, ref.rounds_executed)


def test_small_and_large_requests_with_limits(g):
    """A mix of small and large requests (unions from a few hundred to over
    100,000 states; minimisation, equivalence with and without early exit,
    round limits on a small and a large chain) gives every request the
    stand-alone call's result and the oracle's partition."""
    reqs = []
    for i in range(10):
        A, B, eq = dfagen.equivalence_pair(100 + i, 9, n_lo=300, n_hi=60_000)
        reqs.append(("eq", (A, B, eq), i % 2 == 0))
    for i, n in enumerate((700, 9000, 16_384, 16_385, 50_000)):
        reqs.append(("min", dfagen.random_dfa(n, 2 + i % 3, 0.5, 800 + i), 0))
    chain = dfagen.chain_dfa(3000)
    reqs.append(("min", chain, 5))            # small path, stopped by the round limit
    reqs.append(("min", dfagen.chain_dfa(20_000), 7))   # step path, stopped by the round limit
    assert any(kind == "eq" and x[0].n + x[1].n <= 16_384 for kind, x, _ in reqs)
    assert any(kind == "eq" and x[0].n + x[1].n > 16_384 for kind, x, _ in reqs)
    with g.Server(4 << 30, max_slots=16) as srv:
        tickets = []
        for kind, item, opt in reqs:
            if kind == "min":
                tickets.append(srv.submit_minimise(item.delta, item.accept, max_rounds=opt))
            else:
                A, B, _ = item
                tickets.append(srv.submit_equivalent((A.delta, A.accept, A.start), (B.delta, B.accept, B.start),
                                                     early_exit=opt))
        for (kind, item, opt), t in zip(reqs, tickets):
            if kind == "min":
                st, res, _, blocks = srv.wait(t, n=item.n)
                ref = oracle.moore(item.delta, item.accept, max_rounds=opt or None)
                # the limit ends the call only while every round still splits a block
                assert st == (g.DFA_EMAXROUNDS if opt and ref.rounds_changed == opt else g.DFA_OK)
                assert np.array_equal(blocks, oracle.canonical(ref.block))
                assert (res.rounds_changed, res.rounds_executed) == (ref.rounds_changed, ref.rounds_executed)
            else:
                A, B, expect = item
                st, res, eq, _ = srv.wait(t)
                assert st == g.DFA_OK and eq == int(expect)
                alone_eq, alone = g.equivalent((A.delta, A.accept, A.start), (B.delta, B.accept, B.start),
                                               early_exit=opt)
                assert (res.num_blocks, res.rounds_changed, res.rounds_executed) == \
                    (alone.num_blocks, alone.rounds_changed, alone.rounds_executed)
        c = srv.counters()
        assert c["state_rounds"] == c["state_rounds_direct"] + c["state_rounds_filter"] + c["state_rounds_table"]
