"""Pins for the CPU oracle (CPU only).

The oracle is checked against things other than itself: the paper's printed
outcomes (Table "table:concur", the claims around Figure "fig:dfalong"),
closed forms, independent algorithms (Hopcroft's n log n method, the pair-graph
characterisation of Section 3.1, word enumeration, Hopcroft-Karp with
union-find, breadth-first product search), and invariants.  The last tests
plant mistakes in the oracle and check that the pins catch them.
"""
import os

import numpy as np
import pytest

import dfagen
import oracle
from conftest import GOLDEN


def _table_rows():
    rows = {}
    with open(os.path.join(GOLDEN, "table_concur.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows[p[0]] = dict(N=int(p[1]), k=int(p[2]), size=int(p[3]), naive=p[4], sort=p[5], trans=p[6])
    return rows


def _tiny_random(seed, n, k, p=0.5):
    return dfagen.random_dfa(n, k, p, seed)


# ---------------------------------------------------------------- whole partition

@pytest.mark.parametrize("n,k,p,seed", [(50, 1, 0.5, 1), (200, 2, 0.5, 2), (1000, 3, 0.3, 3),
                                        (5000, 4, 0.5, 4), (3000, 8, 0.1, 5), (777, 2, 0.9, 6)])
def test_moore_equals_hopcroft_random(n, k, p, seed):
    A = dfagen.random_dfa(n, k, p, seed)
    assert np.array_equal(oracle.moore(A.delta, A.accept).block, oracle.hopcroft(A.delta, A.accept))


def test_moore_equals_brute_force_tiny():
    """n <= 7, k <= 3: Moore = pair-table backward search = word enumeration."""
    checked = 0
    for seed in range(120):
        n = 1 + seed % 7
        k = 1 + (seed // 7) % 3
        A = _tiny_random(seed, n, k, p=[0.5, 0.3, 0.7][seed % 3])
        m = oracle.moore(A.delta, A.accept).block
        assert np.array_equal(m, oracle.pair_table(A.delta, A.accept))
        assert np.array_equal(m, oracle.word_enumeration(A.delta, A.accept))
        checked += 1
    assert checked == 120


def test_tiny_dfas_with_merges_brute_force():
    """Small DFAs with few targets have many equivalent states; all three agree."""
    for seed in range(60):
        n, k = 6 + seed % 3, 1 + seed % 2
        d = dfagen.bounded(seed, 77, n * k, 3).reshape(k, n)    # targets only among states 0..2
        acc = dfagen.bernoulli(seed, 78, n, 0.5)
        m = oracle.moore(d, acc).block
        assert np.array_equal(m, oracle.pair_table(d, acc))
        assert np.array_equal(m, oracle.word_enumeration(d, acc))
        assert np.array_equal(m, oracle.hopcroft(d, acc))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_planted_redundancy_closed_form(seed):
    """Blowing every state of a minimal DFA up into copies: the coarsest partition
    is exactly 'copies of the same state'."""
    base = dfagen.random_dfa(400, 2 + seed, 0.5, seed + 10)
    assert oracle.hopcroft(base.delta, base.accept).max() + 1 == base.n      # base is minimal
    P, origin = dfagen.planted_redundancy(base, 5, seed)
    expect = oracle.canonical(origin)
    m = oracle.moore(P.delta, P.accept)
    assert m.num_blocks == base.n
    assert np.array_equal(m.block, expect)
    assert np.array_equal(oracle.hopcroft(P.delta, P.accept), expect)
    assert np.array_equal(oracle.naive_pr(P.delta, P.accept).block, expect)
    assert np.array_equal(oracle.trans_pr(P.delta, P.accept).block, expect)


# ---------------------------------------------------------------- paper's outcomes

def test_table_concur_fib18_row():
    """Fib_18 row: N = 6,765, output size N, naivePR and sortPR iterations N-1."""
    row = _table_rows()["Fib_18"]
    A = dfagen.fibonacci_dfa_with_states(row["N"])
    m = oracle.moore(A.delta, A.accept)
    assert m.num_blocks == row["size"]
    assert m.rounds_executed == int(row["sort"])
    assert m.rounds_changed == row["N"] - 2          # shortest distinguishing word has length n-2 (Section 3.3)
    nv = oracle.naive_pr(A.delta, A.accept)
    assert nv.num_blocks == row["size"] and nv.rounds_executed == int(row["naive"])


@pytest.mark.parametrize("name", ["B_15", "B_16", "B_17"])
def test_table_concur_bit_splitter_rows(name):
    """B_m rows: output size 2^m; the printed iteration count m-1 is the number of
    rounds that grow the partition; every round doubles the block count."""
    row = _table_rows()[name]
    m_ = int(name.split("_")[1])
    B = dfagen.bit_splitter(m_)
    assert B.n == row["N"] and B.k == row["k"]
    r = oracle.moore(B.delta, B.accept)
    assert r.num_blocks == row["size"]
    assert r.rounds_changed == int(row["sort"])
    assert r.counts[:-1] == [2 ** (i + 1) for i in range(m_)]
    nv = oracle.naive_pr(B.delta, B.accept)
    assert nv.rounds_changed == int(row["naive"]) and nv.num_blocks == row["size"]
    # stopping at n singleton blocks reproduces the printed count as the number
    # of rounds run, with the same partition
    rd = oracle.moore(B.delta, B.accept, stop_discrete=True)
    assert rd.rounds_executed == int(row["sort"]) == rd.rounds_changed
    assert np.array_equal(rd.block, r.block)


def _stop_discrete_cases():
    yield dfagen.random_dfa(10_000, 2, 0.5, 1)
    yield dfagen.random_dfa(3000, 4, 0.5, 2)
    yield dfagen.random_dfa(2000, 2, 0.0, 3)          # one block
    yield dfagen.random_dfa(1, 2, 0.5, 4)
    yield dfagen.random_dfa(2, 1, 0.5, 5)
    yield dfagen.fibonacci_dfa(9)
    yield dfagen.bit_splitter(6)
    yield dfagen.chain_dfa(64)
    yield dfagen.cycle_dfa(10)
    yield dfagen.planted_redundancy(dfagen.random_dfa(300, 3, 0.5, 61), 5, 2)[0]


@pytest.mark.parametrize("idx", range(10))
def test_stop_discrete_invariants(idx):
    """Stopping at n blocks changes nothing but the confirming round: same
    partition and block-count history; one round fewer exactly when the final
    partition is discrete (and was reached by a growing round)."""
    A = list(_stop_discrete_cases())[idx]
    plain = oracle.moore(A.delta, A.accept)
    fast = oracle.moore(A.delta, A.accept, stop_discrete=True)
    assert np.array_equal(fast.block, plain.block)
    assert fast.rounds_changed == plain.rounds_changed
    assert fast.counts == plain.counts[:len(fast.counts)]
    if plain.num_blocks == A.n and plain.rounds_changed > 0:
        assert fast.rounds_executed == plain.rounds_executed - 1 == fast.rounds_changed
        assert fast.counts[-1] == A.n
    else:
        assert fast.rounds_executed == plain.rounds_executed


def test_stop_discrete_fib_row():
    """Fib_N ends discrete, so stopping at n blocks runs N-2 rounds where
    Table 2 prints N-1: the table counts Fib with the confirming round."""
    A = dfagen.fibonacci_dfa(10)
    r = oracle.moore(A.delta, A.accept, stop_discrete=True)
    assert r.num_blocks == A.n and r.rounds_executed == r.rounds_changed == A.n - 2


@pytest.mark.parametrize("seed", range(6))
def test_stop_discrete_equivalence(seed):
    """The verdict does not depend on stopping at n blocks (Hopcroft-Karp decides)."""
    A, B, _ = dfagen.equivalence_pair(seed, 7, n_lo=20, n_hi=200)
    args = (A.delta, A.accept, A.start, B.delta, B.accept, B.start)
    expect = oracle.hk_equivalent(*args)
    for early in (False, True):
        assert oracle.equivalent(*args, early_exit=early, stop_discrete=True).equivalent == expect


@pytest.mark.parametrize("i", range(3, 14))
def test_fibonacci_rounds(i):
    A = dfagen.fibonacci_dfa(i)
    m = oracle.moore(A.delta, A.accept)
    assert m.num_blocks == A.n and m.rounds_changed == A.n - 2 and m.rounds_executed == A.n - 1


def test_fig1_claims():
    """Section 3.4: without the closure, q0 and q1 need at least eight iterations;
    with it, the first iteration already separates them."""
    C = dfagen.fig1_chain()
    m = oracle.moore(C.delta, C.accept, history=True)
    sep = [h[0] != h[1] for h in m.history]
    assert sep.index(True) == 8
    assert m.rounds_changed == 8 and m.num_blocks == 10
    nv = oracle.naive_pr(C.delta, C.accept, history=True)
    assert [h[0] != h[1] for h in nv.history].index(True) == 8
    t = oracle.naive_pr(oracle.closure(C.delta), C.accept, history=True)
    assert t.history[1][0] != t.history[1][1]
    assert t.num_blocks == 10


@pytest.mark.parametrize("m", [6, 8, 10])
def test_chain_transpr_rounds_closed_form(m):
    """transPR (Algorithm 5) on the chain with n = 2^m states, under the
    synchronous min-leader reading of Algorithm 2.  The closure letter a^(2^j)
    sends i to min(i + 2^j, n - 1) and every b-level sends i to 0, so a
    non-accepting state differs from its block's leader exactly when some
    a^(2^j) reaches n - 1 from one of them and not from the other: each round
    cuts every interval of non-accepting states at one more bit of the distance
    to n - 1, doubling their number, while {n - 1} stays alone.  Hence
    B_r = min(2^r + 1, n): m rounds that add blocks, one that confirms,
    rounds_executed = log2 n + 1 (and the leader-election split gives at most
    one new block per old block per round, B_r <= 2 B_(r-1))."""
    n = 1 << m
    C = dfagen.chain_dfa(n)
    t = oracle.trans_pr(C.delta, C.accept)
    assert t.num_blocks == n
    assert t.counts == [min((1 << r) + 1, n) for r in range(m + 1)] + [n]
    assert (t.rounds_changed, t.rounds_executed) == (m, m + 1)
    assert all(b <= 2 * a for a, b in zip(t.counts, t.counts[1:]))


def test_fig1_transpr_rounds():
    """Figure 1's 10-state unary chain (q9 accepting): with the closure
    (letters a, a^2, a^4, a^8) the min-leader naivePR needs 4 splitting rounds
    and one confirming round, 5 executed, against 8 + 1 without it."""
    C = dfagen.fig1_chain()
    t = oracle.trans_pr(C.delta, C.accept)
    assert t.num_blocks == 10
    assert (t.rounds_changed, t.rounds_executed) == (4, 5)
    assert t.counts == [2, 3, 4, 6, 10, 10]
    plain = oracle.naive_pr(C.delta, C.accept)
    assert (plain.rounds_changed, plain.rounds_executed) == (8, 9)


@pytest.mark.parametrize("lg", [3, 5, 8, 10])
def test_chain_closed_forms(lg):
    n = 1 << lg
    C = dfagen.chain_dfa(n)
    T = oracle.closure(C.delta)
    L = lg
    i = np.arange(n)
    for j in range(L + 1):
        assert np.array_equal(T[0 * (L + 1) + j], np.minimum(i + (1 << j), n - 1))
        assert (T[1 * (L + 1) + j] == 0).all()
    m = oracle.moore(C.delta, C.accept)
    assert m.num_blocks == n and m.rounds_changed == n - 2


@pytest.mark.parametrize("n,k,seed", [(1, 2, 1), (2, 1, 2), (37, 3, 3), (300, 2, 4), (1025, 1, 5)])
def test_closure_equals_repeated_application(n, k, seed):
    A = dfagen.random_dfa(n, k, 0.5, seed)
    T = oracle.closure(A.delta)
    L = oracle.closure_levels(n)
    assert T.shape == (k * (L + 1), n)
    for a in range(k):
        for lvl in range(L + 1):
            cur = np.arange(n)
            for _ in range(1 << lvl):
                cur = A.delta[a][cur]
            assert np.array_equal(T[a * (L + 1) + lvl], cur)


# ---------------------------------------------------------------- naivePR / transPR

@pytest.mark.parametrize("n,k,seed", [(300, 2, 1), (1000, 3, 2), (2000, 1, 3)])
def test_naive_and_trans_equal_hopcroft(n, k, seed):
    A = dfagen.random_dfa(n, k, 0.5, seed)
    h = oracle.hopcroft(A.delta, A.accept)
    assert np.array_equal(oracle.naive_pr(A.delta, A.accept).block, h)
    assert np.array_equal(oracle.trans_pr(A.delta, A.accept).block, h)


def test_naive_invariants():
    """Leaders are the smallest member of their block; a round splits a block into
    at most two parts; block counts never decrease."""
    A = dfagen.random_dfa(500, 2, 0.5, 9)
    r = oracle.naive_pr(A.delta, A.accept, history=True)
    for prev, cur in zip(r.history, r.history[1:]):
        assert oracle.is_refinement(cur, prev)
        for b in np.unique(prev):
            assert np.unique(cur[prev == b]).shape[0] <= 2
    for h in r.history:
        for b in np.unique(h):
            assert b == np.nonzero(h == b)[0].min()
    assert all(x <= y for x, y in zip(r.counts, r.counts[1:]))


# ---------------------------------------------------------------- invariants, edges

def test_moore_invariants():
    A = dfagen.random_dfa(3000, 3, 0.5, 12)
    r = oracle.moore(A.delta, A.accept, history=True)
    for prev, cur in zip(r.history, r.history[1:]):
        assert oracle.is_refinement(cur, prev)
    assert all(x <= y for x, y in zip(r.counts, r.counts[1:]))
    assert oracle.is_congruence(A.delta, r.block) and oracle.respects(A.accept, r.block)
    assert oracle.is_canonical(r.block)


def test_edge_cases():
    # n = 1
    r = oracle.moore(np.zeros((2, 1), np.uint32), np.array([1], np.uint8))
    assert (r.num_blocks, r.rounds_changed, r.rounds_executed) == (1, 0, 1)
    # k = 0: the result is {F, Q\F}
    acc = np.array([0, 1, 1, 0, 1], np.uint8)
    r = oracle.moore(np.zeros((0, 5), np.uint32), acc)
    assert (r.num_blocks, r.rounds_changed, r.rounds_executed) == (2, 0, 1)
    assert list(r.block) == [0, 1, 1, 0, 1]
    # F empty / F = Q: one block
    A = dfagen.random_dfa(100, 2, 0.0, 3)
    assert oracle.moore(A.delta, A.accept).num_blocks == 1
    A = dfagen.random_dfa(100, 2, 1.0, 3)
    assert oracle.moore(A.delta, A.accept).num_blocks == 1
    assert oracle.naive_pr(A.delta, A.accept).num_blocks == 1
    with pytest.raises(ValueError):
        oracle.moore(np.array([[5]], np.uint32), np.array([0], np.uint8))


# ---------------------------------------------------------------- equivalence

@pytest.mark.parametrize("req", range(10))
def test_equivalence_recipe(req):
    A, B, expect = dfagen.equivalence_pair(req, 5, n_lo=100, n_hi=3000)
    e = oracle.equivalent(A.delta, A.accept, A.start, B.delta, B.accept, B.start)
    assert e.equivalent == expect                                 # by construction
    assert oracle.hk_equivalent(A.delta, A.accept, A.start, B.delta, B.accept, B.start) == expect
    cex = oracle.shortest_cex(A.delta, A.accept, A.start, B.delta, B.accept, B.start)
    assert (cex == -1) == expect
    assert e.separated_round == cex                                # Moore round r = words of length <= r
    ee = oracle.equivalent(A.delta, A.accept, A.start, B.delta, B.accept, B.start, early_exit=True)
    assert ee.equivalent == expect and ee.separated_round == cex
    if not expect:
        assert ee.refine.rounds_executed == cex


def test_equivalence_self_and_cycle():
    C = dfagen.cycle_dfa(8)
    assert oracle.equivalent(C.delta, C.accept, 0, C.delta, C.accept, 0).equivalent
    # different start states of a minimal DFA are inequivalent
    assert not oracle.equivalent(C.delta, C.accept, 0, C.delta, C.accept, 1).equivalent
    assert not oracle.hk_equivalent(C.delta, C.accept, 0, C.delta, C.accept, 1)


# ---------------------------------------------------------------- planted mistakes

def test_pins_catch_dropped_letter(monkeypatch):
    """A signature that forgets the last letter must fail the Hopcroft pin."""
    def bad_round(delta, block):
        cols = [block] + [block[delta[a]] for a in range(delta.shape[0] - 1)]
        return oracle.kernel_of(cols)
    A = dfagen.random_dfa(400, 3, 0.5, 2)
    good = oracle.moore(A.delta, A.accept).block
    monkeypatch.setattr(oracle, "moore_round", bad_round)
    assert not np.array_equal(oracle.moore(A.delta, A.accept).block, good)


def test_pins_catch_missing_own_block(monkeypatch):
    """Dropping block[q] from the signature breaks the refinement invariant on a
    DFA where it matters (Fibonacci), caught by the table pin."""
    def bad_round(delta, block):
        return oracle.kernel_of([block[delta[a]] for a in range(delta.shape[0])])
    A = dfagen.fibonacci_dfa(7)
    monkeypatch.setattr(oracle, "moore_round", bad_round)
    r = oracle.moore(A.delta, A.accept, history=True)
    ok = all(oracle.is_refinement(c, p) for p, c in zip(r.history, r.history[1:]))
    assert not ok or r.rounds_changed != A.n - 2


def test_pins_catch_wrong_leader(monkeypatch):
    """naivePR that compares q's successor with the leader itself (instead of the
    leader's successor) must fail the Hopcroft pin."""
    A = dfagen.random_dfa(300, 2, 0.5, 7)
    h = oracle.hopcroft(A.delta, A.accept)
    monkeypatch.setattr(oracle, "naive_differs", lambda d, block: block[d] != block[block])
    assert not np.array_equal(oracle.naive_pr(A.delta, A.accept, max_rounds=3 * A.n).block, h)


def test_pins_catch_broken_closure():
    """A closure that squares the wrong row fails the repeated-application pin."""
    A = dfagen.random_dfa(64, 2, 0.5, 4)
    T = oracle.closure(A.delta)
    L = oracle.closure_levels(64)
    broken = T.copy()
    broken[0 * (L + 1) + 2] = T[0 * (L + 1) + 1][T[1 * (L + 1) + 1]]   # mixes letters
    cur = np.arange(64)
    for _ in range(4):
        cur = A.delta[0][cur]
    assert np.array_equal(T[2], cur) and not np.array_equal(broken[2], cur)


# ---------------------------------------------------------------- closure + signature refinement

def _closure_moore_cases():
    yield dfagen.random_dfa(500, 2, 0.5, 11)
    yield dfagen.random_dfa(300, 3, 0.3, 12)
    yield dfagen.random_dfa(200, 0, 0.5, 13)
    yield dfagen.fibonacci_dfa(10)
    yield dfagen.bit_splitter(5)
    yield dfagen.chain_dfa(100)
    yield dfagen.cycle_dfa(9)
    yield dfagen.fig1_chain()
    yield dfagen.planted_redundancy(dfagen.random_dfa(120, 3, 0.5, 14), 4, 3)[0]


@pytest.mark.parametrize("idx", range(9))
def test_closure_moore_partition_is_nerode(idx):
    """The closure letters are words over Σ, so refining A' gives A's coarsest
    congruence: the same partition as Hopcroft and as plain refinement."""
    A = list(_closure_moore_cases())[idx]
    r = oracle.closure_moore(A.delta, A.accept)
    assert np.array_equal(r.block, oracle.hopcroft(A.delta, A.accept))
    assert np.array_equal(r.block, oracle.moore(A.delta, A.accept).block)
    assert r.rounds_executed <= oracle.moore(A.delta, A.accept).rounds_executed


@pytest.mark.parametrize("n", [3, 5, 10, 64, 100, 256, 1000])
def test_closure_moore_chain_closed_form(n):
    """Chain: state q is at distance d = n-1-q from the accepting state; only
    powers a^s separate states (b resets to state 0), and a^s accepts from
    distance d iff s >= d.  r closure letters spell a^s iff popcount(s) <= r,
    so distances d and d-1 first differ in round popcount(d-1): the refinement
    grows in every round up to max popcount(x), 1 <= x <= n-2."""
    C = dfagen.chain_dfa(n)
    r = oracle.closure_moore(C.delta, C.accept)
    R = max(bin(x).count("1") for x in range(1, n - 1))
    assert r.num_blocks == n
    assert (r.rounds_changed, r.rounds_executed) == (R, R + 1)


def test_closure_moore_fig1_first_round():
    """Section 3.4's example: with the closure, q0 and q1 part in the first round."""
    C = dfagen.fig1_chain()
    r = oracle.closure_moore(C.delta, C.accept, history=True)
    assert r.history[1][0] != r.history[1][1]


# ---------------------------------------------------------------- quotient (the minimal DFA itself)

def test_reachable_small_cases():
    """Hand-made graphs: the chain reaches every state from anywhere (b leads to
    0); two separate components stay separate."""
    C = dfagen.chain_dfa(6)
    assert oracle.reachable(C.delta, 0).all()
    assert oracle.reachable(C.delta, 5).all()                           # b leads back to 0
    d = np.array([[1, 1, 3, 3]], dtype=np.uint32)                       # 0->1->1; 2->3->3
    assert oracle.reachable(d, 0).tolist() == [True, True, False, False]
    assert oracle.reachable(d, 2).tolist() == [False, False, True, True]


def test_quotient_of_minimal_reachable_dfa_is_itself():
    """All states reachable and pairwise inequivalent: the quotient is the DFA
    with identical numbering (each block is a singleton numbered by its state)."""
    A = dfagen.fibonacci_dfa(12)          # a unary cycle: every state reachable, minimal (Table 2)
    blk = oracle.hopcroft(A.delta, A.accept)
    assert blk.max() + 1 == A.n and oracle.reachable(A.delta, A.start).all()
    Q = oracle.quotient(A.delta, A.accept, A.start, blk)
    assert Q.n == A.n and Q.start == A.start
    assert np.array_equal(Q.delta, A.delta) and np.array_equal(Q.accept, A.accept)


@pytest.mark.parametrize("seed", range(6))
def test_quotient_is_minimal_and_equivalent(seed):
    """Same language (Hopcroft-Karp), no two states equivalent (Hopcroft), every
    state reachable, and unreachable junk dropped."""
    A, B, _ = dfagen.equivalence_pair(seed, 9, n_lo=30, n_hi=400)
    for X in (A, B):
        blk = oracle.moore(X.delta, X.accept).block
        Q = oracle.quotient(X.delta, X.accept, X.start, blk)
        assert oracle.hk_equivalent(Q.delta, Q.accept, Q.start, X.delta, X.accept, X.start)
        assert oracle.hopcroft(Q.delta, Q.accept).max() + 1 == Q.n
        assert oracle.reachable(Q.delta, Q.start).all()
        assert Q.n <= int(oracle.reachable(X.delta, X.start).sum())
    # B is a renamed copy of A plus junk: the same minimal DFA up to renaming
    QA = oracle.quotient(A.delta, A.accept, A.start, oracle.moore(A.delta, A.accept).block)
    QB = oracle.quotient(B.delta, B.accept, B.start, oracle.moore(B.delta, B.accept).block)
    if oracle.hk_equivalent(A.delta, A.accept, A.start, B.delta, B.accept, B.start):
        assert QA.n == QB.n


def test_quotient_planted_redundancy():
    """Copies of a minimal DFA collapse onto it: the quotient has the base's size."""
    base = dfagen.random_dfa(200, 3, 0.5, 72)
    P, origin = dfagen.planted_redundancy(base, 4, 5)
    Q = oracle.quotient(P.delta, P.accept, P.start, oracle.canonical(origin))
    reach_base = int(oracle.reachable(base.delta, base.start).sum())
    assert Q.n == reach_base
    assert oracle.hk_equivalent(Q.delta, Q.accept, Q.start, base.delta, base.accept, base.start)


# ---------------------------------------------------------------- product exploration (Section 4)

def _memory_table():
    rows = {}
    with open(os.path.join(GOLDEN, "memory_inclusion.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, count = map(int, line.split())
            rows[n] = count
    return rows


def test_memory3_generator_matches_figure():
    """Both memory_3 DFAs edge by edge against the figure."""
    edges = {"P": {}, "F": {}}
    with open(os.path.join(GOLDEN, "memory3_figure.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v, src, a, dst = line.split()
            edges[v][(int(src, 2), int(a))] = int(dst, 2)
    for v, forgetful in (("P", False), ("F", True)):
        M = dfagen.memory_dfa(3, forgetful)
        assert len(edges[v]) == 16
        for (s, a), t in edges[v].items():
            assert M.delta[a][s] == t, (v, s, a)
        assert M.accept.tolist() == [0, 0, 0, 0, 1, 1, 1, 1] and M.start == 0


@pytest.mark.parametrize("n", list(range(5, 19)))
def test_memory_inclusion_table(n):
    """Inclusion table: forgetful memory_n is included in perfect memory_n, and
    the explored product has the printed state count."""
    F, P = dfagen.memory_dfa(n, True), dfagen.memory_dfa(n, False)
    r = oracle.product_explore(F.delta, F.accept, F.start, P.delta, P.accept, P.start, inclusion=True)
    assert r.holds and r.cex_len == -1
    assert r.pairs == _memory_table()[n]


def test_memory_reverse_inclusion_fails():
    """Perfect memory remembers more: it accepts words the forgetful one rejects."""
    for n in (3, 5, 8):
        F, P = dfagen.memory_dfa(n, True), dfagen.memory_dfa(n, False)
        r = oracle.product_explore(P.delta, P.accept, P.start, F.delta, F.accept, F.start, inclusion=True)
        assert not r.holds and r.cex_len >= n


@pytest.mark.parametrize("idx", range(5))
def test_self_product_is_reachable_part(idx):
    """Comparing a DFA with itself explores one pair per reachable state (the
    equivalence table's observation that the product has the input's size)."""
    A = [dfagen.random_dfa(300, 2, 0.5, 3), dfagen.fibonacci_dfa(9), dfagen.bit_splitter(6),
         dfagen.chain_dfa(50), dfagen.cycle_dfa(8)][idx]
    r = oracle.product_explore(A.delta, A.accept, A.start, A.delta, A.accept, A.start)
    assert r.holds and r.pairs == int(oracle.reachable(A.delta, A.start).sum())


@pytest.mark.parametrize("seed", range(8))
def test_product_equivalence_against_hk_and_bfs(seed):
    """Verdict = Hopcroft-Karp with union-find; a failing check stops at the
    level of a shortest counterexample (BFS over the product in C)."""
    A, B, _ = dfagen.equivalence_pair(seed, 12, n_lo=20, n_hi=400)
    args = (A.delta, A.accept, A.start, B.delta, B.accept, B.start)
    r = oracle.product_explore(*args)
    assert r.holds == oracle.hk_equivalent(*args)
    assert r.cex_len == oracle.shortest_cex(*args)


def _brute_included(A, B, L):
    """L(A) ⊆ L(B) on all words of length <= L, by enumeration."""
    states = {(A.start, B.start)}
    for _ in range(L + 1):
        if any(A.accept[p] and not B.accept[q] for p, q in states):
            return False
        states = {(int(A.delta[a][p]), int(B.delta[a][q])) for p, q in states for a in range(A.k)}
    return True


@pytest.mark.parametrize("seed", range(10))
def test_product_inclusion_brute_force(seed):
    """Inclusion on tiny DFAs against enumeration of all words up to n_A n_B."""
    A = dfagen.random_dfa(5, 2, 0.4, 300 + seed)
    B = dfagen.random_dfa(4, 2, 0.6, 400 + seed)
    r = oracle.product_explore(A.delta, A.accept, A.start, B.delta, B.accept, B.start, inclusion=True)
    assert r.holds == _brute_included(A, B, A.n * B.n)


# ---------------------------------------------------------------- trans (Algorithm 1)

def _trans_rows():
    rows = {}
    with open(os.path.join(GOLDEN, "trans_table1.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            N, it = map(int, line.split())
            rows[N] = it
    return rows


def _trans_iterations_closed_form(D):
    """Iteration i ends with Reach = paths of 1..2^i edges, so Apart then holds
    every pair within 2^(i+1) - 2 edges of an initially Apart pair; the pairs
    first separated by Moore's round r are exactly those at distance r, so with
    D = the last round that splits, the loop labels something new in iterations
    1..i* (i* the least i with 2^(i+1) - 2 >= D) and stops after i* + 1."""
    i = 0
    while (1 << (i + 1)) - 2 < D:
        i += 1
    return i + 1


def _trans_cases():
    yield dfagen.random_dfa(12, 2, 0.5, 1)
    yield dfagen.random_dfa(20, 3, 0.3, 2)
    yield dfagen.random_dfa(25, 1, 0.5, 3)
    yield dfagen.bit_splitter(4)
    yield dfagen.chain_dfa(16)
    yield dfagen.cycle_dfa(9)
    yield dfagen.planted_redundancy(dfagen.random_dfa(6, 2, 0.5, 9), 3, 1)[0]
    yield dfagen.random_dfa(15, 2, 0.0, 4)


@pytest.mark.parametrize("idx", range(8))
def test_trans_partition_and_closed_form(idx):
    """trans gives Hopcroft's partition, and its iteration count is the closed
    form in the distance to the first Apart pair (from Moore's rounds)."""
    A = list(_trans_cases())[idx]
    r = oracle.trans(A.delta, A.accept)
    assert np.array_equal(r.block, oracle.hopcroft(A.delta, A.accept))
    D = oracle.moore(A.delta, A.accept).rounds_changed
    assert r.iterations == _trans_iterations_closed_form(D)
    # Apart is symmetric, irreflexive, and exactly "different blocks"
    assert np.array_equal(r.apart, r.apart.T) and not r.apart.diagonal().any()
    assert np.array_equal(r.apart, r.block[:, None] != r.block[None, :])


def test_trans_table_rows():
    """The table's iteration counts for N = 8, 13, 21 and 55 come out of the
    oracle; for N = 89 (too large for the dense oracle) out of the closed form
    with D = N - 2 (Moore's rounds on Fibonacci).  N = 34 is printed as 5 where the
    synchronous reading gives 6: the paper's code updates Reach and Apart in
    place, which can only label pairs earlier, so the printed count never
    exceeds the synchronous one."""
    rows = _trans_rows()
    for N, printed in rows.items():
        A = dfagen.fibonacci_dfa_with_states(N)
        if N <= 21 or N == 55:
            r = oracle.trans(A.delta, A.accept)
            assert r.iterations == printed, N
            assert len(set(r.block.tolist())) == N
        ours = _trans_iterations_closed_form(N - 2)
        assert printed <= ours
        assert (printed == ours) == (N != 34), N


def test_trans_fib34_synchronous():
    A = dfagen.fibonacci_dfa_with_states(34)
    r = oracle.trans(A.delta, A.accept)
    assert r.iterations == 6 and oracle.moore(A.delta, A.accept).rounds_changed == 32


def test_pins_catch_trans_without_squaring(monkeypatch):
    """Leaving out the closure step makes trans a one-edge-per-iteration search,
    which the table rows (and the closed form) catch."""
    A = dfagen.fibonacci_dfa_with_states(21)
    monkeypatch.setattr(oracle, "trans_square", lambda reach: reach)
    assert oracle.trans(A.delta, A.accept).iterations != _trans_rows()[21]


def test_pins_catch_trans_label_from_wrong_side(monkeypatch):
    """Labelling the Apart node's predecessors through Reach transposed (t -> s
    instead of s -> t) gives a wrong partition."""
    A = dfagen.random_dfa(12, 2, 0.5, 1)
    h = oracle.hopcroft(A.delta, A.accept)
    monkeypatch.setattr(oracle, "trans_label",
                        lambda reach, apart: apart | ((reach.T @ apart.astype(np.float64)) > 0))
    try:
        r = oracle.trans(A.delta, A.accept)
    except IndexError:          # a state Apart from itself: no representative
        return
    assert not np.array_equal(r.block, h) or r.apart.diagonal().any() or not np.array_equal(r.apart, r.apart.T)


# ---------------------------------------------------------------- the C Moore refinement (CPU baseline)

def _moore_c_cases():
    yield dfagen.random_dfa(1, 2, 0.5, 1)
    yield dfagen.random_dfa(7, 0, 0.5, 2)
    yield dfagen.random_dfa(5000, 3, 0.0, 3)
    yield dfagen.random_dfa(5000, 3, 1.0, 4)
    yield dfagen.random_dfa(10_000, 2, 0.5, 1)
    yield dfagen.random_dfa(30_001, 5, 0.3, 6)
    yield dfagen.fibonacci_dfa(12)
    yield dfagen.bit_splitter(10)
    yield dfagen.chain_dfa(300)
    yield dfagen.cycle_dfa(14)
    yield dfagen.planted_redundancy(dfagen.random_dfa(2000, 3, 0.5, 61), 6, 2)[0]
    yield dfagen.DFA(dfagen.bounded(9, 91, 3 * 20_000, 5).reshape(3, 20_000),
                     dfagen.bernoulli(9, 92, 20_000, 0.5), 0)


@pytest.mark.parametrize("idx", range(12))
@pytest.mark.parametrize("threads", [1, 0])
def test_moore_c_equals_moore_and_hopcroft(idx, threads):
    """The C refinement (one thread, and OpenMP on all host cores) reaches the
    definition-level oracle's partition with the same round counts, and
    Hopcroft's partition."""
    A = list(_moore_c_cases())[idx]
    ref = oracle.moore(A.delta, A.accept)
    got = oracle.moore_c(A.delta, A.accept, threads=threads)
    assert np.array_equal(got.block, ref.block)
    assert (got.num_blocks, got.rounds_changed, got.rounds_executed) == \
        (ref.num_blocks, ref.rounds_changed, ref.rounds_executed)
    assert np.array_equal(got.block, oracle.hopcroft(A.delta, A.accept))


def test_moore_c_rejects_bad_targets():
    A = dfagen.random_dfa(100, 2, 0.5, 3)
    bad = A.delta.copy()
    bad[1][7] = 100
    with pytest.raises((RuntimeError, ValueError)):
        oracle.moore_c(bad, A.accept)
