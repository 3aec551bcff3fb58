"""Seeded, synthetic DFA inputs shared by the CPU oracle tests and the GPU tests.

This module only *builds inputs*.  It holds none of the refinement arithmetic:
no partition, signature, closure or equivalence computation lives here, so the
oracle and the CUDA path can both consume it without sharing any method code.

Random numbers
--------------
All randomness comes from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): value
``i`` of stream ``(seed, stream)`` is ``mix64(key(seed, stream) + (i+1)*GAMMA)``
where ``mix64`` is SplitMix64's output finaliser.  Bounded integers use
Lemire's multiply-shift method with rejection ("Fast random integer generation
in an interval", ACM TOMACS 2019).  Bernoulli(p) is ``u < floor(p * 2**64)``.

Representation
--------------
A DFA is ``(delta, accept, start)`` with ``delta`` a ``uint32`` array of shape
``(k, n)`` in letter-major order, ``delta[a, q] = δ(q, a)`` (the paper's
"Representation" paragraph in Section 2), ``accept`` a ``uint8`` array of 0/1
and ``start`` an int.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "DFA", "u64_stream", "bounded", "bernoulli", "random_dfa", "fibonacci_word",
    "fibonacci_dfa", "bit_splitter", "cycle_dfa", "chain_dfa", "fig1_chain",
    "planted_redundancy", "batch_recipe", "equivalence_pair", "log_uniform_int",
    "CONFIGS",
]

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK32 = np.uint64(0xFFFFFFFF)

# Stream purpose codes; the stream id of instance i is (i << 8) | code.
S_DELTA, S_ACCEPT, S_N, S_K, S_PERM, S_JUNKN, S_JUNKD, S_JUNKA, S_COIN, S_WALK, S_COPIES, S_ARRIVAL, S_LETTER = range(1, 14)


@dataclass
class DFA:
    delta: np.ndarray   # (k, n) uint32, letter-major
    accept: np.ndarray  # (n,) uint8
    start: int = 0

    @property
    def n(self) -> int:
        return int(self.accept.shape[0])

    @property
    def k(self) -> int:
        return int(self.delta.shape[0])


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        t = np.array([stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return _mix64(s * GAMMA + _mix64(t + GAMMA))[0]


def u64_stream(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Values start..start+count-1 of SplitMix64 stream (seed, stream), as uint64."""
    key = _key(seed, stream)
    idx = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + idx * GAMMA)


def _lemire(x: np.ndarray, s: int):
    """(high, low) 64-bit halves of the 128-bit product x*s, for s < 2**32."""
    su = np.uint64(s)
    with np.errstate(over="ignore"):
        p1 = (x & _MASK32) * su
        p2 = (x >> np.uint64(32)) * su
        t = (p2 & _MASK32) << np.uint64(32)
        lo = t + p1
        carry = (lo < t).astype(np.uint64)
        hi = (p2 >> np.uint64(32)) + carry
    return hi, lo


def bounded(seed: int, stream: int, count: int, s: int, start: int = 0) -> np.ndarray:
    """count unbiased integers in [0, s) (s <= 2**32-1), Lemire's method with rejection."""
    assert 1 <= s < (1 << 32)
    x = u64_stream(seed, stream, start, count)
    hi, lo = _lemire(x, s)
    thr = np.uint64(((1 << 64) - s) % s)
    bad = np.nonzero(lo < thr)[0]
    attempt = 1
    while bad.size:
        # Rejected draws are redrawn from a per-attempt side stream at the same index.
        x2 = np.array([u64_stream(seed, stream ^ (attempt << 48), start + int(i), 1)[0] for i in bad], dtype=np.uint64)
        h2, l2 = _lemire(x2, s)
        ok = l2 >= thr
        hi[bad[ok]] = h2[ok]
        bad = bad[~ok]
        attempt += 1
    return hi.astype(np.uint32) if s <= (1 << 32) else hi


def bernoulli(seed: int, stream: int, count: int, p: float, start: int = 0) -> np.ndarray:
    thr = int(p * float(1 << 64)) if p < 1.0 else (1 << 64)
    x = u64_stream(seed, stream, start, count)
    if thr >= (1 << 64):
        return np.ones(count, dtype=np.uint8)
    return (x < np.uint64(thr)).astype(np.uint8)


def uniform01(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits."""
    x = u64_stream(seed, stream, start, count)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / float(1 << 53))


def log_uniform_int(u: float, lo: int, hi: int) -> int:
    """clamp(floor(exp(ln lo + u*(ln(hi+1) - ln lo))), lo, hi), computed on the host."""
    v = math.floor(math.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo))))
    return int(min(max(v, lo), hi))


def _sid(instance: int, code: int) -> int:
    return (instance << 8) | code


def random_dfa(n: int, k: int, p_accept: float, seed: int, instance: int = 0, start: int = 0) -> DFA:
    """Random complete DFA: δ(q, a) uniform over [0, n), q accepting w.p. p_accept."""
    delta = bounded(seed, _sid(instance, S_DELTA), n * k, n).reshape(k, n) if k > 0 else np.zeros((0, n), np.uint32)
    accept = bernoulli(seed, _sid(instance, S_ACCEPT), n, p_accept)
    return DFA(np.ascontiguousarray(delta, dtype=np.uint32), accept, start)


# ----------------------------------------------------------------------------
# The paper's benchmark families (Section 5.1)
# ----------------------------------------------------------------------------

def fibonacci_word(i: int) -> str:
    """w_0 = 1, w_1 = 0, w_{i+1} = w_i w_{i-1} (Section 5.1, Fibonacci DFAs)."""
    a, b = "1", "0"
    if i == 0:
        return a
    for _ in range(i - 1):
        a, b = b, b + a
    return b


def fibonacci_dfa(i: int) -> DFA:
    """Fib_i: unary cycle over |w_i| states, q_j accepting iff w_i[j] = 1."""
    w = fibonacci_word(i)
    n = len(w)
    delta = ((np.arange(n, dtype=np.uint64) + 1) % n).astype(np.uint32).reshape(1, n)
    accept = np.frombuffer(w.encode(), dtype=np.uint8) - ord("0")
    return DFA(delta, accept.astype(np.uint8), 0)


def fibonacci_dfa_with_states(n_states: int) -> DFA:
    """The Fibonacci DFA whose word has exactly n_states letters."""
    i = 0
    while len(fibonacci_word(i)) < n_states:
        i += 1
    if len(fibonacci_word(i)) != n_states:
        raise ValueError(f"{n_states} is not the length of a Fibonacci word")
    return fibonacci_dfa(i)


def bit_splitter(m: int) -> DFA:
    """B_m: 2^m states (bit strings, most significant bit first), letters a_1..a_{m-1}.

    Built from the recursive definition in Section 5.1: B_{j+1} keeps B_j's
    letters on the low j bits and adds a_j, which sends b·σ to (not b)·0^j when
    σ[0] = 1 (σ[0] is the leftmost bit of σ) and leaves it in place otherwise.
    F = states whose leading bit is 1.  The family has no initial state; start = 0.
    """
    n = 1 << m
    q = np.arange(n, dtype=np.uint64)
    k = m - 1
    delta = np.zeros((max(k, 0), n), dtype=np.uint32)
    for letter in range(1, m):          # a_letter introduced when going from B_letter to B_{letter+1}
        j = letter                      # sigma has j bits, b is bit j (counting from 0 at the LSB)
        low = q & np.uint64((1 << j) - 1)
        b = (q >> np.uint64(j)) & np.uint64(1)
        high = q >> np.uint64(j + 1)    # bits above b, kept unchanged by a_letter
        sigma0 = (low >> np.uint64(j - 1)) & np.uint64(1)
        moved = (high << np.uint64(j + 1)) | ((b ^ np.uint64(1)) << np.uint64(j))
        delta[letter - 1] = np.where(sigma0 == 1, moved, q).astype(np.uint32)
    accept = ((q >> np.uint64(m - 1)) & np.uint64(1)).astype(np.uint8)
    return DFA(delta, accept, 0)


def fib_number(i: int) -> int:
    """fib(0) = fib(1) = 1, fib(i) = fib(i-1) + fib(i-2) (Section 5.1, Cycle DFAs)."""
    a, b = 1, 1
    for _ in range(i - 1):
        a, b = b, a + b
    return b if i >= 1 else a


def cycle_dfa(i: int) -> DFA:
    """C_i: fib(i) states, letters a_0..a_m with m = max(round(log10 fib(i)), 1),
    δ(q_j, a_l) = q_{(j + 100 l + 1) mod fib(i)}, F = {q_fib(i-1)}."""
    N = fib_number(i)
    m = max(int(math.floor(math.log10(N) + 0.5)), 1)
    j = np.arange(N, dtype=np.int64)
    delta = np.stack([((j + 100 * l + 1) % N) for l in range(m + 1)]).astype(np.uint32)
    accept = np.zeros(N, dtype=np.uint8)
    accept[fib_number(i - 1)] = 1
    return DFA(delta, accept, 0)


def chain_dfa(n: int) -> DFA:
    """Deep-round chain: letter a maps i -> min(i+1, n-1), letter b maps i -> 0, F = {n-1}."""
    i = np.arange(n, dtype=np.int64)
    a = np.minimum(i + 1, n - 1)
    b = np.zeros(n, dtype=np.int64)
    accept = np.zeros(n, dtype=np.uint8)
    accept[n - 1] = 1
    return DFA(np.stack([a, b]).astype(np.uint32), accept, 0)


def fig1_chain() -> DFA:
    """Figure 1 of Section 3.4: q_0 -a-> q_1 -a-> ... -a-> q_9 with a loop on q_9, F = {q_9}."""
    i = np.arange(10, dtype=np.int64)
    delta = np.minimum(i + 1, 9).astype(np.uint32).reshape(1, 10)
    accept = np.zeros(10, dtype=np.uint8)
    accept[9] = 1
    return DFA(delta, accept, 0)


def memory_dfa(n: int, forgetful: bool = False) -> DFA:
    """memory_n (Section 5.1): states are the last n bits read (state s = the
    bitstring, most significant bit first), 0...0 initial, accepting iff the
    most significant bit is 1; reading bit b appends it and drops the most
    significant bit.  The forgetful variant resets all bits (state b) when the
    two most significant bits are 10."""
    N = 1 << n
    s = np.arange(N, dtype=np.int64)
    rows = []
    for b in (0, 1):
        t = ((s << 1) | b) & (N - 1)
        if forgetful and n >= 2:
            t = np.where((s >> (n - 2)) == 0b10, b, t)
        rows.append(t)
    accept = ((s >> (n - 1)) & 1).astype(np.uint8)
    return DFA(np.stack(rows).astype(np.uint32), accept, 0)


def planted_redundancy(base: DFA, max_copies: int, seed: int, instance: int = 0):
    """Blow every state s of `base` up into c_s in [1, max_copies] copies.

    Each copy of s keeps s's acceptance bit, and its a-transition goes to a
    uniformly chosen copy of δ(s, a).  States are then shuffled.  Returns the new
    DFA and origin[q'] = the base state that q' copies.  If `base` is minimal, the
    coarsest partition of the result is exactly "same origin".
    """
    nb, k = base.n, base.k
    copies = bounded(seed, _sid(instance, S_COPIES), nb, max_copies).astype(np.int64) + 1
    first = np.concatenate([[0], np.cumsum(copies)[:-1]])
    n = int(copies.sum())
    origin_unshuffled = np.repeat(np.arange(nb), copies)
    # random permutation: sort random keys (index breaks ties)
    keys = u64_stream(seed, _sid(instance, S_PERM), 0, n)
    perm = np.lexsort((np.arange(n), keys))        # perm[new_pos] = old index
    pos_of = np.empty(n, dtype=np.int64)
    pos_of[perm] = np.arange(n)
    delta = np.empty((k, n), dtype=np.uint32)
    for a in range(k):
        tgt_base = base.delta[a][origin_unshuffled]
        pick = bounded(seed, _sid(instance, S_DELTA) ^ (a << 40), n, max_copies).astype(np.int64) % copies[tgt_base]
        tgt_old = first[tgt_base] + pick
        delta[a][pos_of] = pos_of[tgt_old]
    accept = np.empty(n, dtype=np.uint8)
    accept[pos_of] = base.accept[origin_unshuffled]
    origin = np.empty(n, dtype=np.int64)
    origin[pos_of] = origin_unshuffled
    return DFA(delta, accept, int(pos_of[first[base.start]])), origin


# ----------------------------------------------------------------------------
# Workload recipes: batch of uneven DFAs and equivalence pairs
# ----------------------------------------------------------------------------

def batch_recipe(count: int, n_lo: int, n_hi: int, k_lo: int, k_hi: int, p_accept: float, seed: int):
    """Sizes of a batch: n_i log-uniform in [n_lo, n_hi], k_i uniform in [k_lo, k_hi]."""
    us = uniform01(seed, S_N, count)
    ns = [log_uniform_int(float(u), n_lo, n_hi) for u in us]
    ks = (bounded(seed, S_K, count, k_hi - k_lo + 1).astype(np.int64) + k_lo).tolist()
    return ns, ks


def batch_dfas(count: int, n_lo: int, n_hi: int, k_lo: int, k_hi: int, p_accept: float, seed: int):
    ns, ks = batch_recipe(count, n_lo, n_hi, k_lo, k_hi, p_accept, seed)
    return [random_dfa(n, k, p_accept, seed, instance=i + 1) for i, (n, k) in enumerate(zip(ns, ks))]


def _random_perm(seed: int, stream: int, n: int) -> np.ndarray:
    keys = u64_stream(seed, stream, 0, n)
    return np.lexsort((np.arange(n), keys)).astype(np.int64)


def equivalence_pair(request: int, seed: int, n_lo: int = 1000, n_hi: int = 1_000_000, ks=(2, 4),
                     p_accept: float = 0.5, force: str | None = None):
    """One equivalence request: (A, B, expected_equivalent).

    A is a random DFA (n log-uniform in [n_lo, n_hi], k drawn from `ks`).  B is
    a random renaming of A's states plus J unreachable junk states, J uniform in
    [1, ceil(n/16)], whose out-edges go anywhere in B.  With probability 1/2
    (or as forced) the acceptance bit of one state of B reached from B's start by
    a random walk is flipped, which makes B inequivalent to A.
    """
    inst = request + 1
    u = float(uniform01(seed, _sid(inst, S_N), 1)[0])
    n = log_uniform_int(u, n_lo, n_hi)
    k = int(ks[int(bounded(seed, _sid(inst, S_K), 1, len(ks))[0])])
    A = random_dfa(n, k, p_accept, seed, instance=inst)
    J = int(bounded(seed, _sid(inst, S_JUNKN), 1, (n + 15) // 16)[0]) + 1
    nb = n + J
    perm = _random_perm(seed, _sid(inst, S_PERM), nb)   # A state q -> B state perm[q]; junk j -> perm[n+j]
    dB = np.empty((k, nb), dtype=np.uint32)
    accB = np.empty(nb, dtype=np.uint8)
    for a in range(k):
        dB[a][perm[:n]] = perm[A.delta[a].astype(np.int64)]
        dB[a][perm[n:]] = bounded(seed, _sid(inst, S_JUNKD) ^ (a << 40), J, nb)
    accB[perm[:n]] = A.accept
    accB[perm[n:]] = bernoulli(seed, _sid(inst, S_JUNKA), J, 0.5)
    startB = int(perm[A.start])
    if force is None:
        equivalent = bool(bernoulli(seed, _sid(inst, S_COIN), 1, 0.5)[0])
    else:
        equivalent = force == "equivalent"
    if not equivalent:
        # walk a random word from B's start; the state reached is reachable by construction
        steps = int(bounded(seed, _sid(inst, S_WALK), 1, 65)[0])
        letters = bounded(seed, _sid(inst, S_LETTER), max(steps, 1), k)
        s = startB
        for t in range(steps):
            s = int(dB[int(letters[t])][s])
        accB[s] ^= 1
    return A, DFA(dB, accB, startB), equivalent


# The five workloads this library is measured on (sizes and seeds).
CONFIGS = {
    "random_n1e4_k2": dict(n=10_000, k=2, p=0.5, seed=1),
    "random_n2p24_k4": dict(n=1 << 24, k=4, p=0.5, seed=2),
    "chain_n2p20": dict(n=1 << 20),
    "batch_4096": dict(count=4096, n_lo=64, n_hi=65_536, k_lo=2, k_hi=8, p=0.3, seed=4),
    "serve_equiv_10000": dict(requests=10_000, n_lo=1000, n_hi=1_000_000, ks=(2, 4), seed=5),
}
