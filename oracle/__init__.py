"""CPU oracle for DFA partition refinement.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library (``paper_2508_20735_gb300``) and never imports it.

Plain, slow and obviously correct.  Every function cites the passage of the
paper it follows.  Arithmetic is exact integer throughout (state and block
indices); there is no floating point in the method.

Definition-level functions (numpy; a library sort is the only primitive):
  * :func:`moore`      Moore-style signature refinement, the result of
                       ``sortPR`` (Section 3.3, Algorithm 4).
  * :func:`naive_pr`   leader-election refinement ``naivePR`` (Section 3.2,
                       Algorithm 2) under the synchronous PRAM reading.
  * :func:`closure`    the partial transitive closure δT (Section 3.4,
                       Algorithm 5) by pointer doubling.
  * :func:`trans_pr`   ``transPR`` = closure, then naivePR on A' (Algorithm 5).
  * :func:`trans`      ``trans``: transitive closure of the pair graph
                       (Section 3.1, Algorithm 1), tiny n only.
  * :func:`equivalent` language equivalence by refining the disjoint union
                       (Section 4: equivalence via minimisation).
  * :func:`canonical`  blocks renumbered 0..B-1 in increasing order of their
                       smallest state.

Independent cross-checks (plain C in ``oracle.c``, loaded with ctypes):
  * :func:`hopcroft`, :func:`hk_equivalent`, :func:`shortest_cex`,
    :func:`pair_table`; plus :func:`word_enumeration` in pure Python.

CPU baseline (plain C in ``moore.c``): :func:`moore_c`, Moore refinement with
hash partitions and exact signature comparison, on one thread or with OpenMP
on all host cores (bench.py times it; tests pin it to :func:`moore`).

Readings of the paper where it is silent or inconsistent (also listed in the
design notes):
  * Round counts: ``rounds_changed`` counts rounds whose block count grew;
    ``rounds_executed`` also counts the final round that confirms the fixpoint
    (Algorithm 4 stops after a round in which the count did not grow).
  * Initial partition: the non-empty classes among {F, Q \\ F}; if F = ∅ or
    F = Q there is one initial block (Algorithm 4 assumes two).
  * naivePR's concurrent write elects the smallest writer (priority CRCW); the
    initial leaders are min F and min Q \\ F.  Every read in a parallel step sees
    the values from before the step.
  * transPR: log is base 2, levels i = 0..floor(log2 n); row a*(L+1)+i of δT is
    the letter a^(2^i).
  * All n states are partitioned; unreachable states are kept.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c and moore.c into liboracle.so next to them (plain gcc,
    with OpenMP when the compiler has it; no GPU)."""
    srcs = [os.path.join(_HERE, f) for f in ("oracle.c", "moore.c")]
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(f) for f in srcs):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:] + srcs, stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:   # no OpenMP: the single-threaded build
            subprocess.check_call(base + srcs)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P32 = ctypes.POINTER(ctypes.c_uint32)
        P8 = ctypes.POINTER(ctypes.c_uint8)
        u32 = ctypes.c_uint32
        lib.oracle_hopcroft.argtypes = [u32, u32, P32, P8, P32]
        lib.oracle_hopcroft.restype = ctypes.c_int
        lib.oracle_pair_table.argtypes = [u32, u32, P32, P8, P32]
        lib.oracle_pair_table.restype = ctypes.c_int
        lib.oracle_hk_equivalent.argtypes = [u32, u32, P32, P8, u32, u32, P32, P8, u32]
        lib.oracle_hk_equivalent.restype = ctypes.c_int
        lib.oracle_shortest_cex.argtypes = [u32, u32, P32, P8, u32, u32, P32, P8, u32]
        lib.oracle_shortest_cex.restype = ctypes.c_int64
        lib.oracle_moore_c.argtypes = [u32, u32, P32, P8, ctypes.c_int, P32, P32, P32, P32]
        lib.oracle_moore_c.restype = ctypes.c_int
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p32(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _p8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


def _prep(delta, accept):
    delta = np.ascontiguousarray(delta, dtype=np.uint32)
    accept = np.ascontiguousarray(accept, dtype=np.uint8)
    if delta.ndim != 2 or delta.shape[1] != accept.shape[0]:
        raise ValueError("delta must have shape (k, n) matching accept (n,)")
    n = accept.shape[0]
    if n == 0:
        raise ValueError("n must be positive")
    if delta.size and int(delta.max()) >= n:
        raise ValueError("transition target out of range")
    return delta, accept


# ----------------------------------------------------------------------------
# Canonical numbering
# ----------------------------------------------------------------------------

def canonical(labels: np.ndarray) -> np.ndarray:
    """Renumber a partition given by arbitrary labels: block ids 0..B-1 in
    increasing order of each block's smallest state (the output convention)."""
    labels = np.asarray(labels)
    n = labels.shape[0]
    order = np.lexsort((np.arange(n), labels))          # by label, then by state
    sl = labels[order]
    first = np.ones(n, dtype=bool)
    first[1:] = sl[1:] != sl[:-1]
    min_member = order[first]                           # smallest state of each block
    group = np.cumsum(first) - 1
    rank = np.empty(min_member.shape[0], dtype=np.int64)
    rank[np.argsort(min_member, kind="stable")] = np.arange(min_member.shape[0])
    out = np.empty(n, dtype=np.uint32)
    out[order] = rank[group]
    return out


def kernel_of(columns) -> np.ndarray:
    """Partition of states by equality of the tuple (columns[0][q], columns[1][q], ...),
    returned in canonical numbering.  Columns hold block numbers < 2**32; they are
    packed losslessly into as few 64-bit words as fit, then sorted."""
    cols = [np.asarray(c, dtype=np.uint64) for c in columns]
    n = cols[0].shape[0]
    width = max(1, max(int(c.max()).bit_length() if n else 1 for c in cols))
    per_word = max(1, 64 // width)
    words = []
    for i in range(0, len(cols), per_word):
        w = np.zeros(n, dtype=np.uint64)
        for c in cols[i:i + per_word]:
            w = (w << np.uint64(width)) | c
        words.append(w)
    order = np.lexsort([np.arange(n)] + words[::-1])   # primary key words[0]; ties by state
    first = np.zeros(n, dtype=bool)     # first[i]: sorted position i starts a new block
    first[0] = True
    for w in words:
        sw = w[order]
        first[1:] |= sw[1:] != sw[:-1]
    min_member = order[first]
    group = np.cumsum(first) - 1
    rank = np.empty(min_member.shape[0], dtype=np.int64)
    rank[np.argsort(min_member, kind="stable")] = np.arange(min_member.shape[0])
    out = np.empty(n, dtype=np.uint32)
    out[order] = rank[group]
    return out


# ----------------------------------------------------------------------------
# Moore / sortPR (Section 3.3, Algorithm 4)
# ----------------------------------------------------------------------------

@dataclass
class RefineResult:
    block: np.ndarray                 # canonical block numbers, shape (n,)
    num_blocks: int
    rounds_changed: int
    rounds_executed: int
    counts: list = field(default_factory=list)   # block count before round 1, after each round


def initial_partition(accept: np.ndarray) -> np.ndarray:
    """Algorithm 4's initialisation: accepting states in one block, the rest in another
    (only non-empty classes exist)."""
    return canonical(np.asarray(accept, dtype=np.uint8))


def moore_round(delta: np.ndarray, block: np.ndarray) -> np.ndarray:
    """One iteration of Algorithm 4: signature[q] = (block[q], block[δ(q,a0)], ...,
    block[δ(q,a_{k-1})]); states with equal signatures share a new block."""
    cols = [block] + [block[delta[a]] for a in range(delta.shape[0])]
    return kernel_of(cols)


def moore(delta, accept, max_rounds: int | None = None, history: bool = False,
          stop_discrete: bool = False) -> RefineResult:
    """Signature refinement until the number of blocks stops growing (Algorithm 4).

    The result is the coarsest partition of all n states that respects F and is a
    congruence for δ (Nerode equivalence over Q).  With stop_discrete the loop also
    ends after a round that leaves n blocks: singletons cannot split, so the
    until-test's confirming round is skipped (Table 2 counts B_n this way)."""
    delta, accept = _prep(delta, accept)
    block = initial_partition(accept)
    count = int(block.max()) + 1
    counts = [count]
    hist = [block] if history else None
    changed = executed = 0
    while max_rounds is None or executed < max_rounds:
        new = moore_round(delta, block)
        executed += 1
        new_count = int(new.max()) + 1
        counts.append(new_count)
        if history:
            hist.append(new)
        if new_count == count:        # until-condition of Algorithm 4
            block = new
            break
        changed += 1
        block, count = new, new_count
        if stop_discrete and count == block.shape[0]:
            break
    res = RefineResult(block, int(block.max()) + 1, changed, executed, counts)
    if history:
        res.history = hist
    return res


# ----------------------------------------------------------------------------
# naivePR (Section 3.2, Algorithm 2), transPR (Section 3.4, Algorithm 5)
# ----------------------------------------------------------------------------

def naive_differs(d: np.ndarray, block: np.ndarray) -> np.ndarray:
    """Algorithm 2's test for one letter a with d = δ(·, a):
    block[δ(q,a)] ≠ block[δ(block[q],a)], i.e. q's a-successor and its leader's
    a-successor lie in different blocks."""
    return block[d] != block[d[block]]


def naive_pr(delta, accept, max_rounds: int | None = None, history: bool = False) -> RefineResult:
    """Leader-election refinement.  block[q] is the leader (a state) of q's block.

    Each round, in parallel: diff(q) = ∃a: block[δ(q,a)] ≠ block[δ(block[q],a)];
    new_leader[b] = the smallest q with diff(q) and block[q] = b; then every q with
    diff(q) moves to new_leader[block[q]].  Stops when no state differs (stable)."""
    delta, accept = _prep(delta, accept)
    k, n = delta.shape
    q = np.arange(n, dtype=np.int64)
    F = accept.astype(bool)
    qf = int(q[F].min()) if F.any() else -1
    qn = int(q[~F].min()) if (~F).any() else -1
    block = np.where(F, qf, qn).astype(np.int64)
    counts = [int(np.unique(block).shape[0])]
    hist = [block.copy()] if history else None
    changed = executed = 0
    while max_rounds is None or executed < max_rounds:
        executed += 1
        diff = np.zeros(n, dtype=bool)
        for a in range(k):
            diff |= naive_differs(delta[a].astype(np.int64), block)
        if not diff.any():
            counts.append(counts[-1])
            break
        # leader election: smallest differing state per old block (priority CRCW)
        cand_blocks = block[diff]
        cand_states = q[diff]                 # ascending, so the first per block is the minimum
        uniq, first_idx = np.unique(cand_blocks, return_index=True)
        new_leader = np.full(n, -1, dtype=np.int64)
        new_leader[uniq] = cand_states[first_idx]
        block = np.where(diff, new_leader[block], block)
        changed += 1
        counts.append(int(np.unique(block).shape[0]))
        if history:
            hist.append(block.copy())
    res = RefineResult(canonical(block), 0, changed, executed, counts)
    res.num_blocks = int(res.block.max()) + 1
    res.leaders = block
    if history:
        res.history = hist
    return res


def closure_levels(n: int) -> int:
    """floor(log2 n): the largest level i with a^(2^i) in Σ^T (n >= 1)."""
    return int(n).bit_length() - 1


def closure(delta) -> np.ndarray:
    """δT of Algorithm 5: row a*(L+1)+i is δ(·, a^(2^i)), L = floor(log2 n).

    δT(q, a^(2^i)) = δT(δT(q, a^(2^(i-1))), a^(2^(i-1))) for i = 1..L."""
    delta = np.ascontiguousarray(delta, dtype=np.uint32)
    k, n = delta.shape
    L = closure_levels(n)
    out = np.empty((k * (L + 1), n), dtype=np.uint32)
    for a in range(k):
        out[a * (L + 1)] = delta[a]
    for i in range(1, L + 1):
        for a in range(k):
            prev = out[a * (L + 1) + i - 1]
            out[a * (L + 1) + i] = prev[prev]
    return out


def trans_pr(delta, accept, max_rounds: int | None = None) -> RefineResult:
    """Algorithm 5: build δT, then run naivePR on A' = (Q, Σ^T, δT, F, q0)."""
    delta, accept = _prep(delta, accept)
    return naive_pr(closure(delta), accept, max_rounds=max_rounds)


def closure_moore(delta, accept, max_rounds: int | None = None, history: bool = False,
                  stop_discrete: bool = False) -> RefineResult:
    """Signature refinement (Algorithm 4) on the extended DFA A' of Algorithm 5
    (letters a^(2^i), i = 0..floor(log2 n)) instead of naivePR.  The extra letters
    are words over Σ and Σ's own letters are level 0 of δT, so A' and A have the
    same coarsest congruence (the Nerode partition); a round of A' tests words
    of up to 2^L letters of A at once."""
    delta, accept = _prep(delta, accept)
    return moore(closure(delta), accept, max_rounds=max_rounds, history=history, stop_discrete=stop_discrete)


# ----------------------------------------------------------------------------
# trans: transitive closure of the pair graph (Section 3.1, Algorithm 1)
# ----------------------------------------------------------------------------

def trans_square(reach: np.ndarray) -> np.ndarray:
    """Algorithm 1's first parallel step: Reach[s][u] := true wherever
    Reach[s][t] and Reach[t][u] for some t (0/1 matrices)."""
    return ((reach + reach @ reach) > 0).astype(np.float64)


def trans_label(reach: np.ndarray, apart: np.ndarray) -> np.ndarray:
    """Algorithm 1's second parallel step: s becomes Apart if Reach[s][t] for an
    Apart node t."""
    return apart | ((reach @ apart.astype(np.float64)) > 0)


@dataclass
class TransResult:
    block: np.ndarray        # canonical partition: q, q' share a block iff not Apart(q, q')
    iterations: int          # executions of the while loop, the last one labelling nothing new
    apart: np.ndarray        # bool[n, n]


def trans(delta, accept, max_iterations: int | None = None) -> TransResult:
    """Algorithm 1 (trans).  The pair graph has the nodes (q, q') in Q x Q,
    numbered q*n + q', and an edge (q, q') -> (δ(q,a), δ(q',a)) for every
    letter a; Apart starts with the pairs on which F disagrees.  Each iteration
    of the while loop (i) extends Reach by every path Reach[s][t], Reach[t][u]
    and (ii) labels s Apart if Reach[s][t] for an Apart t; the loop ends after
    an iteration in which (ii) labels nothing new.  Synchronous reading: each
    parallel step reads the values from before the step, so iteration i ends
    with Reach = paths of 1..2^i edges.  The boolean products are 0/1 matrix
    products (a library matmul, exact: the sums stay far below 2^53)."""
    delta, accept = _prep(delta, accept)
    k, n = delta.shape
    V = n * n
    q, qp = np.divmod(np.arange(V, dtype=np.int64), n)
    reach = np.zeros((V, V), dtype=np.float64)
    for a in range(k):
        reach[np.arange(V), delta[a][q].astype(np.int64) * n + delta[a][qp]] = 1.0
    apart = accept[q] != accept[qp]
    it = 0
    while max_iterations is None or it < max_iterations:
        it += 1
        reach = trans_square(reach)
        new = trans_label(reach, apart)
        grew = bool((new & ~apart).any())
        apart = new
        if not grew:
            break
    A = apart.reshape(n, n)
    rep = np.array([int(np.flatnonzero(~A[x])[0]) for x in range(n)], dtype=np.int64) if n else \
        np.zeros(0, dtype=np.int64)
    return TransResult(canonical(rep), it, A)


# ----------------------------------------------------------------------------
# The minimal DFA itself: reachable part, quotient by the partition
# ----------------------------------------------------------------------------

def reachable(delta, start: int) -> np.ndarray:
    """States reachable from `start` (breadth-first search), as a bool array."""
    delta = np.ascontiguousarray(delta, dtype=np.uint32)
    k, n = delta.shape
    seen = np.zeros(n, dtype=bool)
    seen[start] = True
    frontier = np.array([start], dtype=np.int64)
    while frontier.size:
        nxt = np.unique(delta[:, frontier].reshape(-1).astype(np.int64))
        nxt = nxt[~seen[nxt]]
        seen[nxt] = True
        frontier = nxt
    return seen


@dataclass
class Quotient:
    delta: np.ndarray      # (k, n') letter-major
    accept: np.ndarray     # (n',)
    start: int
    n: int


def quotient(delta, accept, start: int, block) -> Quotient:
    """The minimal DFA A' with L(A') = L(A) (Section 2's problem statement) from
    the coarsest partition: its states are the blocks holding a state reachable
    from `start`, numbered in order of their smallest reachable state; a block's
    transitions and acceptance are those of that representative."""
    delta, accept = _prep(delta, accept)
    block = np.asarray(block, dtype=np.int64)
    reach = reachable(delta, start)
    states = np.nonzero(reach)[0]                       # ascending
    blocks_in_order, first = np.unique(block[states], return_index=True)
    reps = states[first]                                # smallest reachable state of each block
    order = np.argsort(reps, kind="stable")
    reps = reps[order]
    newid = np.full(int(block.max()) + 1, -1, dtype=np.int64)
    newid[block[reps]] = np.arange(reps.size)
    qd = newid[block[delta[:, reps].astype(np.int64)]]
    assert (qd >= 0).all()
    return Quotient(qd.astype(np.uint32), accept[reps].copy(), int(newid[block[start]]), int(reps.size))


# ----------------------------------------------------------------------------
# Equivalence (Section 4): refine the disjoint union
# ----------------------------------------------------------------------------

def disjoint_union(dA, accA, dB, accB):
    dA = np.ascontiguousarray(dA, dtype=np.uint32)
    dB = np.ascontiguousarray(dB, dtype=np.uint32)
    if dA.shape[0] != dB.shape[0]:
        raise ValueError("alphabets differ")
    nA = dA.shape[1]
    d = np.concatenate([dA, (dB.astype(np.uint64) + nA).astype(np.uint32)], axis=1)
    acc = np.concatenate([np.asarray(accA, np.uint8), np.asarray(accB, np.uint8)])
    return d, acc


@dataclass
class EquivResult:
    equivalent: bool
    refine: RefineResult
    separated_round: int      # round in which the two start states first differ, -1 if never


def equivalent(dA, accA, sA, dB, accB, sB, early_exit: bool = False,
               stop_discrete: bool = False) -> EquivResult:
    """L(A) = L(B) iff q0A and q0B end in the same block of the coarsest partition of
    A ⊎ B.  With early_exit, refinement stops at the first round whose partition
    separates the two start states (that round number is the length of a shortest
    distinguishing word)."""
    d, acc = disjoint_union(dA, accA, dB, accB)
    nA = np.asarray(accA).shape[0]
    sBu = nA + int(sB)
    if not early_exit:
        r = moore(d, acc, history=True, stop_discrete=stop_discrete)
        sep = -1
        for i, h in enumerate(r.history):
            if h[sA] != h[sBu]:
                sep = i
                break
        return EquivResult(bool(r.block[sA] == r.block[sBu]), r, sep)
    block = initial_partition(acc)
    count = int(block.max()) + 1
    counts = [count]
    changed = executed = 0
    if block[sA] != block[sBu]:
        return EquivResult(False, RefineResult(block, count, 0, 0, counts), 0)
    while True:
        new = moore_round(d, block)
        executed += 1
        new_count = int(new.max()) + 1
        counts.append(new_count)
        if new_count == count:
            block = new
            break
        changed += 1
        block, count = new, new_count
        if block[sA] != block[sBu]:
            return EquivResult(False, RefineResult(block, count, changed, executed, counts), executed)
        if stop_discrete and count == block.shape[0]:
            break
    return EquivResult(True, RefineResult(block, int(block.max()) + 1, changed, executed, counts), -1)


# ----------------------------------------------------------------------------
# Product exploration (Section 4): the naive Hopcroft-Karp variant
# ----------------------------------------------------------------------------

@dataclass
class ProductResult:
    holds: bool            # L(A) = L(B) (equivalence) or L(A) ⊆ L(B) (inclusion)
    pairs: int             # state pairs explored (all reachable ones if `holds`)
    cex_len: int           # breadth-first level of a first violating pair (a shortest
                           # counterexample's length); -1 if `holds`


def product_explore(dA, accA, sA, dB, accB, sB, inclusion: bool = False) -> ProductResult:
    """Algorithm 6 without R+: the set R of explored state pairs grows from
    <q0A, q0B> by following every letter in both DFAs at once, breadth first; a
    pair with exactly one accepting state (equivalence), or with the first
    accepting and the second not (inclusion, the condition of Section 4's
    variant), ends the search with `False` once its level is complete."""
    dA, accA = _prep(dA, accA)
    dB, accB = _prep(dB, accB)
    if dA.shape[0] != dB.shape[0]:
        raise ValueError("alphabets differ")
    k = dA.shape[0]
    nB = np.int64(accB.shape[0])
    def bad(p, q):
        a, b = accA[p] != 0, accB[q] != 0
        return (a & ~b) if inclusion else (a != b)
    frontier = np.array([int(sA) * nB + int(sB)], dtype=np.int64)
    seen = set(frontier.tolist())
    total, level = 1, 0
    while frontier.size:
        p, q = frontier // nB, frontier % nB
        if bad(p, q).any():
            return ProductResult(False, total, level)
        nxt = []
        for a in range(k):
            nxt.append(dA[a][p].astype(np.int64) * nB + dB[a][q].astype(np.int64))
        cand = np.unique(np.concatenate(nxt)) if nxt else np.zeros(0, dtype=np.int64)
        new = [c for c in cand.tolist() if c not in seen]
        seen.update(new)
        total += len(new)
        frontier = np.array(new, dtype=np.int64)
        level += 1
    return ProductResult(True, total, -1)


# ----------------------------------------------------------------------------
# Independent cross-checks
# ----------------------------------------------------------------------------

def moore_c(delta, accept, threads: int = 1) -> "RefineResult":
    """Moore refinement in plain C (moore.c): the same partition and round
    counts as :func:`moore`, for the CPU baseline.  threads = 1: one thread;
    0: all host cores (OpenMP); else that many."""
    delta, accept = _prep(delta, accept)
    k, n = delta.shape
    out = np.empty(n, dtype=np.uint32)
    ch, ex, nb = ctypes.c_uint32(0), ctypes.c_uint32(0), ctypes.c_uint32(0)
    rc = _load().oracle_moore_c(n, k, _p32(delta), _p8(accept), int(threads), _p32(out), ctypes.byref(ch),
                                ctypes.byref(ex), ctypes.byref(nb))
    if rc != 0:
        raise RuntimeError(f"oracle_moore_c failed: {rc}")
    res = RefineResult(out, int(nb.value), int(ch.value), int(ex.value), [])
    return res


def host_threads() -> int:
    """Threads moore_c uses with threads = 0 (the host cores OpenMP sees)."""
    return int(_load().oracle_threads())


def hopcroft(delta, accept) -> np.ndarray:
    """Hopcroft's n log n coarsest partition (C), canonical numbering."""
    delta, accept = _prep(delta, accept)
    k, n = delta.shape
    out = np.empty(n, dtype=np.uint32)
    rc = _load().oracle_hopcroft(n, k, _p32(delta), _p8(accept), _p32(out))
    if rc != 0:
        raise RuntimeError(f"oracle_hopcroft failed: {rc}")
    return canonical(out)


def pair_table(delta, accept) -> np.ndarray:
    """Section 3.1's pair-graph characterisation (C, n <= 4096), canonical numbering."""
    delta, accept = _prep(delta, accept)
    k, n = delta.shape
    out = np.empty(n, dtype=np.uint32)
    rc = _load().oracle_pair_table(n, k, _p32(delta), _p8(accept), _p32(out))
    if rc != 0:
        raise RuntimeError(f"oracle_pair_table failed: {rc}")
    return canonical(out)


def hk_equivalent(dA, accA, sA, dB, accB, sB) -> bool:
    """Hopcroft-Karp with union-find (Algorithm 6)."""
    dA, accA = _prep(dA, accA)
    dB, accB = _prep(dB, accB)
    if dA.shape[0] != dB.shape[0]:
        raise ValueError("alphabets differ")
    r = _load().oracle_hk_equivalent(accA.shape[0], dA.shape[0], _p32(dA), _p8(accA), int(sA),
                                     accB.shape[0], _p32(dB), _p8(accB), int(sB))
    if r < 0:
        raise RuntimeError(f"oracle_hk_equivalent failed: {r}")
    return bool(r)


def shortest_cex(dA, accA, sA, dB, accB, sB) -> int:
    """Length of a shortest word accepted by exactly one of A, B; -1 if equivalent."""
    dA, accA = _prep(dA, accA)
    dB, accB = _prep(dB, accB)
    r = _load().oracle_shortest_cex(accA.shape[0], dA.shape[0], _p32(dA), _p8(accA), int(sA),
                                    accB.shape[0], _p32(dB), _p8(accB), int(sB))
    if r < -1:
        raise RuntimeError(f"oracle_shortest_cex failed: {r}")
    return int(r)


def word_enumeration(delta, accept, max_len: int | None = None) -> np.ndarray:
    """Pure-Python brute force for tiny DFAs: p ~ q iff every word of length
    <= max_len (default n-2, which suffices for n states) leads both to the same
    acceptance.  Canonical numbering."""
    delta, accept = _prep(delta, accept)
    k, n = delta.shape
    L = max(n - 2, 0) if max_len is None else max_len
    # behaviour vector of each state: acceptance after every word, in a fixed word order
    behaviour = [[int(accept[q])] for q in range(n)]
    frontier = list(range(n))          # frontier[q] = state reached from q by the current word
    words = [frontier]
    for _length in range(1, L + 1):
        nxt = []
        for reached in words:
            for a in range(k):
                r2 = [int(delta[a][s]) for s in reached]
                nxt.append(r2)
                for q in range(n):
                    behaviour[q].append(int(accept[r2[q]]))
        words = nxt
    keys = {}
    labels = np.empty(n, dtype=np.uint32)
    for q in range(n):
        labels[q] = keys.setdefault(tuple(behaviour[q]), len(keys))
    return canonical(labels)


# ----------------------------------------------------------------------------
# Invariants of a refinement run
# ----------------------------------------------------------------------------

def is_refinement(finer: np.ndarray, coarser: np.ndarray) -> bool:
    """Every block of `finer` lies inside one block of `coarser`."""
    pairs = np.unique(np.stack([finer.astype(np.int64), coarser.astype(np.int64)]), axis=1)
    return pairs.shape[1] == np.unique(finer).shape[0]


def is_congruence(delta, block) -> bool:
    """Same block ⇒ same block of successors, for every letter."""
    delta = np.asarray(delta)
    for a in range(delta.shape[0]):
        succ = block[delta[a]]
        pairs = np.unique(np.stack([block.astype(np.int64), succ.astype(np.int64)]), axis=1)
        if pairs.shape[1] != np.unique(block).shape[0]:
            return False
    return True


def respects(accept, block) -> bool:
    pairs = np.unique(np.stack([block.astype(np.int64), np.asarray(accept, np.int64)]), axis=1)
    return pairs.shape[1] == np.unique(block).shape[0]


def is_canonical(block) -> bool:
    """Ids dense 0..B-1 and ordered by smallest member."""
    block = np.asarray(block)
    return bool(np.array_equal(canonical(block), block))
