"""The seeded input generators against the paper's figures and definitions (CPU)."""
import os

import numpy as np
import pytest

import dfagen
from conftest import GOLDEN, read_golden_dfa


def _figure_to_arrays(name, state_index):
    header, edges = read_golden_dfa(name)
    n = int(header["states"][0])
    k = int(header["letters"][0])
    delta = np.full((k, n), -1, dtype=np.int64)
    for s, a, t in edges:
        assert delta[a, state_index(s)] == -1, "figure lists an edge twice"
        delta[a, state_index(s)] = state_index(t)
    accept = np.zeros(n, dtype=np.uint8)
    for s in header["accepting"]:
        accept[state_index(s)] = 1
    return delta, accept, header


def test_fibonacci_words_as_printed():
    with open(os.path.join(GOLDEN, "fibonacci_words.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for idx, word in rows:
        assert dfagen.fibonacci_word(int(idx)) == word


def test_fib5_matches_figure():
    delta, accept, header = _figure_to_arrays("fib5_figure.txt", int)
    A = dfagen.fibonacci_dfa(5)
    assert np.array_equal(A.delta, delta) and np.array_equal(A.accept, accept)
    assert A.start == int(header["start"][0])


def test_bit_splitter_b3_matches_figure():
    delta, accept, _ = _figure_to_arrays("b3_figure.txt", lambda s: int(s, 2))
    B = dfagen.bit_splitter(3)
    assert np.array_equal(B.delta, delta)
    assert np.array_equal(B.accept, accept)


def test_cycle_c5_matches_figure():
    delta, accept, header = _figure_to_arrays("c5_figure.txt", int)
    C = dfagen.cycle_dfa(5)
    assert np.array_equal(C.delta, delta) and np.array_equal(C.accept, accept)


def test_fig1_chain_matches_figure():
    delta, accept, header = _figure_to_arrays("fig1_chain.txt", int)
    C = dfagen.fig1_chain()
    assert np.array_equal(C.delta, delta) and np.array_equal(C.accept, accept)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 7, 10])
def test_bit_splitter_sizes(m):
    B = dfagen.bit_splitter(m)
    assert B.n == 2 ** m and B.k == m - 1
    assert int(B.accept.sum()) == 2 ** (m - 1)


def test_bit_splitter_recursion():
    """B_{m+1} on letters a_1..a_{m-1} behaves as B_m on the low m bits (Section 5.1)."""
    for m in range(2, 8):
        small, big = dfagen.bit_splitter(m), dfagen.bit_splitter(m + 1)
        n = 2 ** m
        for a in range(m - 1):
            for b in (0, 1):
                q = np.arange(n) + b * n
                assert np.array_equal(big.delta[a][q], small.delta[a] + b * n)


def test_cycle_sizes():
    for i, (N, letters) in {2: (2, 2), 5: (8, 2), 10: (89, 3), 20: (10946, 5)}.items():
        C = dfagen.cycle_dfa(i)
        assert C.n == N and C.k == letters
        assert C.accept.sum() == 1 and C.accept[dfagen.fib_number(i - 1)] == 1


def test_chain_definition():
    C = dfagen.chain_dfa(16)
    assert C.delta[0][3] == 4 and C.delta[0][15] == 15 and (C.delta[1] == 0).all()
    assert C.accept.sum() == 1 and C.accept[15] == 1


def test_splitmix64_known_answers():
    """SplitMix64 from state 0 produces 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
    0x06C45D188009454F (the generator's published reference outputs)."""
    v = dfagen._mix64(np.arange(1, 4, dtype=np.uint64) * dfagen.GAMMA)
    assert [int(x) for x in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_bounded_range_and_uniformity():
    x = dfagen.bounded(7, 3, 200_000, 10)
    assert x.min() >= 0 and x.max() < 10
    counts = np.bincount(x, minlength=10)
    chi2 = float(((counts - 20_000) ** 2 / 20_000).sum())
    assert chi2 < 40.0           # 9 dof; p ~ 1e-5
    big = dfagen.bounded(7, 4, 100_000, (1 << 32) - 1)
    assert big.max() < (1 << 32) - 1
    # deterministic and counter-based: a slice equals the same range of a longer draw
    y = dfagen.bounded(7, 3, 100, 10, start=50)
    assert np.array_equal(y, x[50:150])


def test_bernoulli_rate():
    b = dfagen.bernoulli(3, 1, 100_000, 0.3)
    assert abs(b.mean() - 0.3) < 0.01
    assert dfagen.bernoulli(3, 1, 10, 1.0).all() and not dfagen.bernoulli(3, 1, 10, 0.0).any()


def test_random_dfa_shapes_and_determinism():
    A = dfagen.random_dfa(1000, 3, 0.5, 1)
    B = dfagen.random_dfa(1000, 3, 0.5, 1)
    assert A.delta.shape == (3, 1000) and A.delta.dtype == np.uint32
    assert np.array_equal(A.delta, B.delta) and np.array_equal(A.accept, B.accept)
    assert A.delta.max() < 1000


def test_batch_recipe_ranges():
    ns, ks = dfagen.batch_recipe(4096, 64, 65536, 2, 8, 0.3, 4)
    assert min(ns) >= 64 and max(ns) <= 65536 and min(ks) >= 2 and max(ks) <= 8
    # log-uniform: about half the DFAs below the geometric mean
    gm = (64 * 65537) ** 0.5
    assert 0.45 < np.mean(np.array(ns) < gm) < 0.55


def test_equivalence_pair_structure():
    for r in range(8):
        A, B, eq = dfagen.equivalence_pair(r, 5, n_lo=30, n_hi=300)
        assert B.k == A.k and B.n > A.n
        # every state reachable from B's start is a renamed copy of an A state (junk is unreachable)
        seen = {B.start}
        stack = [B.start]
        while stack:
            s = stack.pop()
            for a in range(B.k):
                t = int(B.delta[a][s])
                if t not in seen:
                    seen.add(t)
                    stack.append(t)
        seenA = {A.start}
        stack = [A.start]
        while stack:
            s = stack.pop()
            for a in range(A.k):
                t = int(A.delta[a][s])
                if t not in seenA:
                    seenA.add(t)
                    stack.append(t)
        assert len(seen) == len(seenA)


def test_planted_redundancy_structure():
    base = dfagen.random_dfa(50, 2, 0.5, 3)
    P, origin = dfagen.planted_redundancy(base, 3, 5)
    assert P.n == origin.shape[0] and P.n >= 50
    for a in range(2):
        assert np.array_equal(origin[P.delta[a]], base.delta[a][origin])
    assert np.array_equal(P.accept, base.accept[origin])
