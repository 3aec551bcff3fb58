"""Benchmark of the DFA partition-refinement hot path on GB300.

One step = one dfa_minimise call (signature refinement, every round until the
fixpoint, plus canonical numbering) on the 2^24-state, 4-letter random DFA
(uniform uint32 targets, acceptance Bernoulli(0.5), seed 2), inputs resident
in HBM.  The metric is transitions refined per second, n*|Σ|*rounds / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun, one process per GPU): every rank refines its own copy of the
workload (independent problems, no collective on the data path); the value
is the sum over ranks divided by the slowest rank's time ("weak" scaling).

--impl reference times the CPU oracle's Moore refinement in plain C with
OpenMP on all of the machine's host cores (oracle/moore.c), one whole refinement
of the same workload per step.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = dict(workload="random_dfa_n2^24_k4", n=1 << 24, k=4, p_accept=0.5, seed=2)
METRIC = "transitions refined/sec (n*|Sigma|*rounds/s)"
UNIT = "transitions/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the CPU-oracle leg (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads (batch, chain, serve)")
    ap.add_argument("--lg", type=int, default=24,
                    help="profiling cases: 2^lg states instead of 2^24 (same k, seed and acceptance)")
    ap.add_argument("--stop-discrete", action="store_true",
                    help="profiling cases: time the call with DFA_FLAG_STOP_DISCRETE")
    ap.add_argument("--bucketed", action="store_true",
                    help="profiling cases: time the call with DFA_FLAG_BUCKETED (the bucketed gather)")
    ap.add_argument("--case", default="headline", choices=["headline", "batch", "serve"],
                    help="batch: time only the packed batched call on --batch-dfas DFAs of the batch recipe")
    ap.add_argument("--batch-dfas", type=int, default=4096)
    ap.add_argument("--serve-requests", type=int, default=10_000)
    ap.add_argument("--serve-pairs", type=int, default=1000, help="serve case: distinct generated pairs")
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-budget-gb", type=float, default=24.0)
    ap.add_argument("--schedule", type=int, default=-1, help="batch case: kernel schedule (-1 = autotuned)")
    args = ap.parse_args()
    if args.lg != 24:
        WORKLOAD.update(workload=f"random_dfa_n2^{args.lg}_k4", n=1 << args.lg)
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "10"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx = float(p[1])
            except ValueError:
                continue
            for nm, v in zip(names, p[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def whole_job(units: float, elapsed_s: float, dist=None, device="cpu"):
    """Whole-job throughput over ranks: the units every rank processed divided
    by the slowest rank's time (every rank gets the same value)."""
    if dist is None:
        return units / elapsed_s, elapsed_s
    import torch
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()) / float(t.item()), float(t.item())


def host_info():
    """Host core count and CPU model (recorded beside the CPU baseline)."""
    import platform
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":", 1)[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def cpu_baseline(A):
    """The oracle as it stands, on the machine's host cores: the C Moore refinement
    (oracle/moore.c) with OpenMP on all cores over the whole workload (the
    baseline proper), beside the same code on one thread (a 2^22-state sample of
    the recipe, scaled per transition) and one round of the numpy oracle."""
    import dfagen
    import oracle
    n, k = A.n, A.k
    cores = oracle.host_threads()
    t = time.perf_counter()
    r = oracle.moore_c(A.delta, A.accept, threads=0)
    dt = time.perf_counter() - t
    S = dfagen.random_dfa(1 << 22, k, WORKLOAD["p_accept"], WORKLOAD["seed"])
    t = time.perf_counter()
    rs = oracle.moore_c(S.delta, S.accept, threads=1)
    dt1 = time.perf_counter() - t
    block = oracle.initial_partition(A.accept)
    t = time.perf_counter()
    oracle.moore_round(A.delta, block)
    dtn = time.perf_counter() - t
    return {"value": n * k * r.rounds_executed / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "host": host_info(),
            "sample": f"oracle/moore.c with OpenMP on {cores} threads: the whole refinement of the {n}-state, "
                      f"{k}-letter workload ({r.rounds_executed} rounds, {dt:.2f} s)",
            "single_thread": {"value": S.n * k * rs.rounds_executed / dt1, "unit": UNIT, "cores": 1,
                              "sample": f"oracle/moore.c on one thread, the recipe at 2^22 states "
                                        f"({rs.rounds_executed} rounds, {dt1:.2f} s)"},
            "numpy_round": {"value": n * k / dtn, "unit": UNIT, "cores": 1,
                            "sample": f"one round of the numpy oracle on the full workload ({dtn:.1f} s)"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import dfagen
    import oracle
    A = dfagen.random_dfa(WORKLOAD["n"], WORKLOAD["k"], WORKLOAD["p_accept"], WORKLOAD["seed"])
    cores = oracle.host_threads()
    times, rounds = [], []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        r = oracle.moore_c(A.delta, A.accept, threads=0)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
            rounds.append(r.rounds_executed)
    tot = sum(times)
    value = A.n * A.k * sum(rounds) / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / len(times) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": dict(WORKLOAD, parallelism=f"cpu, {cores} threads", step="one whole oracle refinement"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "oracle/moore.c (OpenMP, all host cores): the whole refinement of the "
                                       "full workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _dev(A):
    import numpy as np
    import torch
    return (torch.from_numpy(np.ascontiguousarray(A.delta).view(np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(A.accept)).cuda())


def _time_calls(fn, reps):
    import torch
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t) / reps


def extras(g):
    """The other workloads of the hot path, measured after the headline (not part of it)."""
    import numpy as np
    import torch

    import dfagen
    out = {}
    import oracle
    cores = oracle.host_threads()
    # random DFA, n = 10,000, k = 2 (small: the cluster kernel), against the single-block and
    # cooperative kernels and the C oracle
    A = dfagen.random_dfa(10_000, 2, 0.5, 1)
    d, a = _dev(A)
    res = g.minimise(d, a)[1]
    dev, one, coop = [], [], []
    for _ in range(20):
        dev.append(g.minimise(d, a)[1].device_ns)
        one.append(g.minimise(d, a, flags=g.DFA_FLAG_ONE_BLOCK)[1].device_ns)   # forced single block
        coop.append(g.minimise(d, a, schedule=1)[1].device_ns)
    cpu1 = _best_of(lambda: oracle.moore_c(A.delta, A.accept, threads=1), 5)
    cpuN = _best_of(lambda: oracle.moore_c(A.delta, A.accept, threads=0), 5)
    out["random_n1e4_k2"] = {"device_us": statistics.median(dev) / 1e3, "rounds": res.rounds_executed,
                             "kernel": "one thread-block cluster (n <= 16,384)",
                             "single_block_kernel_device_us": statistics.median(one) / 1e3,
                             "cooperative_kernel_device_us": statistics.median(coop) / 1e3,
                             "transitions_per_s": A.n * A.k * res.rounds_executed / (statistics.median(dev) * 1e-9),
                             "cpu_oracle_us": {"1_core": cpu1 * 1e6, f"{cores}_cores": cpuN * 1e6}}
    # deep-round chain, n = 2^20: transPR in full; plain refinement over a bounded number of rounds
    C = dfagen.chain_dfa(1 << 20)
    d, a = _dev(C)
    g.minimise(d, a, algo="trans")
    tr = g.minimise(d, a, algo="trans")[1]
    bounded = 20_000
    mo = g.minimise(d, a, max_rounds=bounded, check=False)[1]
    us_round = mo.device_ns / 1e3 / mo.rounds_executed
    t = time.perf_counter()
    tref = oracle.trans_pr(C.delta, C.accept)
    trans_cpu = time.perf_counter() - t
    per_state_round = []
    for lg in (12, 13, 14):
        X = dfagen.chain_dfa(1 << lg)
        t = time.perf_counter()
        rx = oracle.moore_c(X.delta, X.accept, threads=1)
        per_state_round.append((time.perf_counter() - t) / rx.rounds_executed / X.n)
    ns_sr = statistics.median(per_state_round) * 1e9
    out["chain_n2p20"] = {
        "trans": {"rounds": tr.rounds_executed, "device_ms": tr.device_ns / 1e6, "blocks": tr.num_blocks,
                  "cpu_oracle_s": trans_cpu, "cpu_oracle_rounds": tref.rounds_executed,
                  "cpu_sample": "numpy oracle transPR (closure + naivePR) at the full 2^20 states, 1 core"},
        "moore": {"rounds_needed": C.n - 1, "rounds_timed": mo.rounds_executed, "us_per_round": us_round,
                  "projected_s_for_all_rounds": us_round * (C.n - 1) / 1e6,
                  "cpu_oracle_ns_per_state_round": ns_sr,
                  "cpu_oracle_projected_s_for_all_rounds": ns_sr * 1e-9 * C.n * (C.n - 1),
                  "cpu_sample": "oracle/moore.c on one core, whole refinement of the chains 2^12, 2^13, 2^14 "
                                "(n - 1 rounds each), cost per state and round extrapolated to 2^20"},
    }
    # the minimal DFA itself (reachability + quotient) of the 2^24-state workload, from its partition
    R = dfagen.random_dfa(WORKLOAD["n"], WORKLOAD["k"], WORKLOAD["p_accept"], WORKLOAD["seed"])
    rd, ra = _dev(R)
    blk, _ = g.minimise(rd, ra)
    g.quotient(rd, ra, R.start, blk)
    torch.cuda.synchronize()
    t = time.perf_counter()
    qd, qa, qs = g.quotient(rd, ra, R.start, blk)
    out["quotient_n2p24_k4"] = {"ms": (time.perf_counter() - t) * 1e3, "states_in": R.n, "states_out": int(qa.numel())}
    # the paper's renumbering (radix sort + adjacent difference + scan per round) against the hash
    g.minimise(rd, ra, algo="sort")
    so = g.minimise(rd, ra, algo="sort")[1]
    ha = g.minimise(rd, ra)[1]
    out["sort_vs_hash_n2p24_k4"] = {
        "sort": {"device_ms": so.device_ns / 1e6, "rounds": so.rounds_executed, "blocks": so.num_blocks},
        "hash": {"device_ms": ha.device_ns / 1e6, "rounds": ha.rounds_executed, "blocks": ha.num_blocks},
    }
    del rd, ra, blk, qd, qa
    # product exploration (Section 4's naive Hopcroft-Karp): the inclusion table's largest case, and a
    # million-state equivalent pair against refinement of the union
    for m in (15, 27):
        F, P = dfagen.memory_dfa(m, True), dfagen.memory_dfa(m, False)
        fd, pd_ = _dev(F) + (F.start,), _dev(P) + (P.start,)
        cap = 1 << 31 if m > 20 else None
        g.product_check(fd, pd_, inclusion=True, max_pairs=cap)
        torch.cuda.synchronize()
        t = time.perf_counter()
        holds, pairs, _ = g.product_check(fd, pd_, inclusion=True, max_pairs=cap)
        out[f"product_memory{m}_inclusion"] = {"ms": (time.perf_counter() - t) * 1e3, "holds": holds, "pairs": pairs}
        del fd, pd_
        torch.cuda.empty_cache()
    EA, EB, _ = dfagen.equivalence_pair(0, 17, n_lo=1_000_000, n_hi=1_000_001, force="equivalent")
    ea, eb = _dev(EA) + (EA.start,), _dev(EB) + (EB.start,)
    row = {}
    for name, call in (("product", lambda: g.product_check(ea, eb)), ("union_refinement", lambda: g.equivalent(ea, eb))):
        call()
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = call()
        row[name] = {"ms": (time.perf_counter() - t) * 1e3, "equivalent": bool(r[0])}
    row["states"] = [EA.n, EB.n]
    out["equivalence_1m_product_vs_union"] = row
    # trans (Algorithm 1): the table's largest Fibonacci DFA and two it could not run
    row = {}
    for N in (89, 144, 233):
        F = dfagen.fibonacci_dfa_with_states(N)
        fd, fa = _dev(F)
        g.trans(fd, fa)
        torch.cuda.synchronize()
        t = time.perf_counter()
        blk, it = g.trans(fd, fa)
        row[f"fibonacci_n{N}"] = {"ms": (time.perf_counter() - t) * 1e3, "iterations": it,
                                  "blocks": int(blk.max().item()) + 1, "pair_nodes": N * N}
    out["trans_fibonacci"] = row
    # signature refinement on the closure DFA against transPR (naivePR on the same closure)
    cm = {}
    for name, X in (("fibonacci_n121393", dfagen.fibonacci_dfa(25)), ("chain_n2p20", C)):
        d, a = _dev(X)
        row = {}
        for algo in ("closure_moore", "trans"):
            g.minimise(d, a, algo=algo)
            r = g.minimise(d, a, algo=algo)[1]
            row[algo] = {"device_ms": r.device_ns / 1e6, "rounds": r.rounds_executed, "blocks": r.num_blocks}
        cm[name] = row
    out["closure_moore_vs_trans"] = cm
    # batch of 4,096 DFAs: one launch vs one dfa_minimise per DFA; the autotuner
    # writes to a fresh cache file, so that its choice is measured in this run
    os.environ["DFA_AUTOTUNE_CACHE"] = os.path.join(tempfile.mkdtemp(prefix="dfa_tune_"), "autotune.json")
    dfas = dfagen.batch_dfas(4096, 64, 65_536, 2, 8, 0.3, 4)
    items = [_dev(X) for X in dfas]
    pn, pk, pd, pa = g.pack_batch([(X.delta, X.accept) for X in dfas])   # resident on the device, packed
    outb = torch.empty(sum(X.n for X in dfas), dtype=torch.int32, device="cuda")
    g.minimise_batch_packed(pn, pk, pd, pa, out=outb)   # autotune on first use
    tb = _time_calls(lambda: g.minimise_batch_packed(pn, pk, pd, pa, out=outb), 3)
    dev_ms = g.minimise_batch_packed(pn, pk, pd, pa, out=outb)[1][0].device_ns / 1e6
    tl = _time_calls(lambda: g.minimise_batch(items, out=outb), 3)
    singles = [(x[0], x[1], torch.empty(x[1].numel(), dtype=torch.int32, device="cuda")) for x in items]
    ts = _time_calls(lambda: [g.minimise(x[0], x[1], out=x[2]) for x in singles], 1)
    sample = dfas[:512]
    t = time.perf_counter()
    for X in sample:
        oracle.moore_c(X.delta, X.accept, threads=1)
    c1 = len(sample) / (time.perf_counter() - t)
    from concurrent.futures import ThreadPoolExecutor
    t = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(lambda X: oracle.moore_c(X.delta, X.accept, threads=1), sample))
    cN = len(sample) / (time.perf_counter() - t)
    out["batch_4096"] = {"states": int(sum(X.n for X in dfas)), "batched_dfas_per_s": 4096 / tb,
                         "single_launch_dfas_per_s": 4096 / ts, "speedup": ts / tb, "batched_ms": tb * 1e3,
                         "batched_device_ms": dev_ms, "list_form_ms": tl * 1e3,
                         "form": "packed (dfa_minimise_batch_packed); list_form_ms: one dfa_t per DFA",
                         "cpu_oracle_dfas_per_s": {"1_core": c1, f"{cores}_cores": cN},
                         "cpu_sample": "oracle/moore.c, one DFA per thread, the first 512 DFAs of the recipe",
                         "autotune": autotune_record(), "graph": dict(zip(("instantiations", "updates"),
                                                                          g.batch_graph_stats()))}
    out["serve_equiv"] = serve_study(g, pairs=1000, nreq=10_000)
    return out


def schedule_name(s):
    """The batch kernel's schedule s: states per lane, states per tile, and whether
    the DFAs that fit one thread block are refined one per block."""
    return f"{1 + (s & 1)} state(s) per lane, tile {256 >> ((s >> 1) % 3)}" + \
        (", block per DFA of up to 65,536 states" if s >= 6 else "")


def autotune_record():
    """The batch autotuner's entries in its cache file: the chosen schedule, every
    schedule's device time, and the margin of the choice over the runner-up."""
    path = os.environ.get("DFA_AUTOTUNE_CACHE")
    if not path or not os.path.exists(path):
        return None
    with open(path) as f:
        cache = json.load(f)
    rec = {}
    for key, entry in cache.items():
        choice, ns = entry[0], entry[1:]
        ranked = sorted(t for t in ns if t > 0)
        rec[key] = {"choice": schedule_name(choice),
                    "device_ms": {schedule_name(s): t / 1e6 for s, t in enumerate(ns)},
                    "margin_vs_runner_up": (ranked[1] / ranked[0] - 1.0) if len(ranked) > 1 else None}
    return rec


def _best_of(fn, reps):
    best = float("inf")
    for _ in range(reps):
        t = time.perf_counter()
        fn()
        best = min(best, time.perf_counter() - t)
    return best


def _gen_pair(i):
    import dfagen
    A, B, eq = dfagen.equivalence_pair(i, 5)
    return A.delta, A.accept, A.start, B.delta, B.accept, B.start, eq


def make_pair_pool(pairs: int):
    """`pairs` distinct requests of the served-equivalence recipe (seed 5), generated in a
    spawn process pool (no CUDA in the workers) before any arrival clock starts."""
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4),
                             mp_context=multiprocessing.get_context("spawn")) as ex:
        return list(ex.map(_gen_pair, range(pairs), chunksize=8))


def _union(dA, aA, dB, aB):
    """The disjoint union A ⊎ B as arrays (B's states after A's): the oracle's input for one request."""
    import numpy as np
    nA = aA.shape[0]
    return np.concatenate([dA, dB.astype(np.uint64) + nA], axis=1).astype(np.uint32), np.concatenate([aA, aB])


def serve_study(g, pairs: int, nreq: int, loads=(0.5, 0.8, 0.95), slots: int = 64, budget_gb: float = 24.0):
    """The served-equivalence stream: `nreq` requests drawn round robin from `pairs`
    distinct generated pairs whose arrays sit in pinned host memory (a server's receive
    buffers), first in a closed loop (capacity), then with Poisson arrivals at each load
    (a fraction of that capacity): p50/p99 latency and throughput, verdicts checked
    against the generator.  Beside it: the same requests through serial dfa_equivalent
    calls, and the CPU oracle (Moore on the union) per request."""
    import numpy as np
    import torch

    import oracle
    t = time.perf_counter()
    raw = make_pair_pool(pairs)
    gen_s = time.perf_counter() - t

    def _pinned(d, acc):
        return (torch.from_numpy(np.ascontiguousarray(d).view(np.int32)).pin_memory(),
                torch.from_numpy(np.ascontiguousarray(acc)).pin_memory())
    pool = [((*_pinned(dA, aA), sA), (*_pinned(dB, aB), sB), eq) for dA, aA, sA, dB, aB, sB, eq in raw]
    states = float(np.mean([r[1].shape[0] + r[4].shape[0] for r in raw]))
    with g.Server(int(budget_gb * (1 << 30)), max_slots=slots) as srv:
        t0 = time.perf_counter()
        tickets = [srv.submit_equivalent(A, B) for A, B, _ in (pool[i % len(pool)] for i in range(nreq))]
        wrong = 0
        for i, tk in enumerate(tickets):
            _, _, eq, _ = srv.wait(tk)
            wrong += int(bool(eq) != pool[i % len(pool)][2])
        cap = nreq / (time.perf_counter() - t0)
        counters = srv.counters()
    rng = np.random.default_rng(5)
    points = []
    for frac in loads:
        lam = frac * cap
        gaps = rng.exponential(1.0 / lam, nreq)
        with g.Server(int(budget_gb * (1 << 30)), max_slots=slots) as srv:
            tickets = []
            t_next = time.perf_counter()
            for i in range(nreq):
                t_next += gaps[i]
                while time.perf_counter() < t_next:
                    pass
                A, B, _ = pool[i % len(pool)]
                tickets.append(srv.submit_equivalent(A, B))
            bad = 0
            for i, tk in enumerate(tickets):
                _, _, eq, _ = srv.wait(tk)
                bad += int(bool(eq) != pool[i % len(pool)][2])
            st = srv.stats()
        wrong += bad
        points.append({"load": frac, "offered_rps": lam, "p50_us": st["p50_us"], "p99_us": st["p99_us"],
                       "throughput_rps": st["throughput_rps"], "wrong_verdicts": bad})
    sample = pool[:64]
    for A, B, _ in sample[:4]:
        g.equivalent(A, B)
    t0 = time.perf_counter()
    for A, B, _ in sample:
        g.equivalent(A, B)
    serial = len(sample) / (time.perf_counter() - t0)
    unions = [_union(r[0], r[1], r[3], r[4]) for r in raw[:64]]
    t0 = time.perf_counter()
    for d, acc in unions:
        oracle.moore_c(d, acc, threads=1)
    cpu1 = len(unions) / (time.perf_counter() - t0)
    from concurrent.futures import ThreadPoolExecutor
    cores = oracle.host_threads()
    t0 = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(lambda u: oracle.moore_c(u[0], u[1], threads=1), unions))
    cpuN = len(unions) / (time.perf_counter() - t0)
    ms = [counters["state_rounds_direct"], counters["state_rounds_filter"], counters["state_rounds_table"]]
    return {"requests": nreq, "distinct_pairs": len(pool), "mean_union_states": states,
            "pool_generation_s": gen_s, "closed_loop_rps": cap, "closed_loop_wrong_verdicts": wrong,
            "load_points": points, "serial_dfa_equivalent_rps": serial, "closed_loop_vs_serial": cap / serial,
            "closed_loop_counters": counters,
            "table_mode_share": ms[2] / max(1, sum(ms)),
            "cpu_oracle_rps": {"1_core": cpu1, f"{cores}_cores": cpuN},
            "cpu_sample": "oracle/moore.c on the union A ⊎ B of the first 64 pairs, one request per thread",
            "sample": f"Poisson arrivals at {', '.join(str(x) for x in loads)} x closed-loop capacity; "
                      f"{nreq} requests drawn round robin from {len(pool)} distinct pairs of the "
                      "served-equivalence recipe (A: n log-uniform in [1e3, 1e6], k in {2, 4}; seed 5), "
                      "inputs in pinned host memory"}


def run_batch_case(args, local):
    """The batched workload alone: one packed dfa_minimise_batch_packed call per
    step over --batch-dfas DFAs of the batch recipe (n log-uniform in [64, 65536],
    k in 2..8, acceptance 0.3, seed 4), inputs resident on the device."""
    import torch

    import dfagen
    import paper_2508_20735_gb300 as g
    torch.cuda.set_device(local)
    g.build()
    if args.schedule < 0:
        os.environ["DFA_AUTOTUNE_CACHE"] = os.path.join(tempfile.mkdtemp(prefix="dfa_tune_"), "autotune.json")
    dfas = dfagen.batch_dfas(args.batch_dfas, 64, 65_536, 2, 8, 0.3, 4)
    pn, pk, pd, pa = g.pack_batch([(X.delta, X.accept) for X in dfas])
    out = torch.empty(int(pn.sum()), dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        g.minimise_batch_packed(pn, pk, pd, pa, out=out, schedule=args.schedule)
    dev = []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(args.steps):
            dev.append(g.minimise_batch_packed(pn, pk, pd, pa, out=out, schedule=args.schedule)[1][0].device_ns)
        torch.cuda.synchronize()
        el = time.perf_counter() - t
    tune = autotune_record() if args.schedule < 0 else None
    chosen = next(iter(tune.values()))["choice"] if tune else schedule_name(args.schedule)
    # the cooperative kernel and/or the block-per-DFA kernel: with blocks, the cooperative
    # launch runs only for DFAs beyond 65,536 states
    if "block per DFA" in chosen:
        launches = 1 + (1 if int(pn.max()) > 65_536 else 0)
    else:
        launches = 1
    print(json.dumps({"metric": "DFAs minimised/sec (batched)", "value": args.batch_dfas * args.steps / el,
                      "unit": "DFAs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": el * 1e3 / args.steps, "device_ms": statistics.median(dev) / 1e6,
                      "higher_is_better": True, "dtype": "u32", "data": "synthetic",
                      "config": {"workload": f"batch_{args.batch_dfas}_dfas", "states": int(pn.sum()),
                                 "schedule": "autotuned" if args.schedule < 0 else schedule_name(args.schedule)},
                      "autotune": tune,
                      "graph": dict(zip(("instantiations", "updates"), g.batch_graph_stats())),
                      "clocks": clk.summary(), "gpu_launches": args.steps * launches}), flush=True)


def run_serve_case(args, local):
    """The served-equivalence workload alone: each step submits --serve-requests
    requests (drawn round robin from --serve-pairs distinct pairs of the
    served-equivalence recipe, seed 5, whose arrays sit in pinned host memory) to
    one server and waits for all of them (closed loop)."""
    import numpy as np
    import torch

    import paper_2508_20735_gb300 as g
    raw = make_pair_pool(args.serve_pairs)   # before any CUDA work (spawned workers)
    torch.cuda.set_device(local)
    g.build()

    def _pinned(d, acc):
        return (torch.from_numpy(np.ascontiguousarray(d).view(np.int32)).pin_memory(),
                torch.from_numpy(np.ascontiguousarray(acc)).pin_memory())
    pool = [((*_pinned(dA, aA), sA), (*_pinned(dB, aB), sB)) for dA, aA, sA, dB, aB, sB, _ in raw]
    nreq = args.serve_requests
    with g.Server(int(args.serve_budget_gb * (1 << 30)), max_slots=args.serve_slots) as srv:
        def step():
            tickets = [srv.submit_equivalent(*pool[i % len(pool)]) for i in range(nreq)]
            for t in tickets:
                srv.wait(t)
        for _ in range(args.warmup):
            step()
        c0 = srv.counters()
        with ClockSampler(local) as clk:
            t = time.perf_counter()
            for _ in range(args.steps):
                step()
            el = time.perf_counter() - t
        c1 = srv.counters()
    d = {k: c1[k] - c0[k] for k in c1}
    print(json.dumps({"metric": "equivalence requests/sec (served, closed loop)", "value": nreq * args.steps / el,
                      "unit": "requests/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True, "dtype": "u32",
                      "data": "synthetic", "config": {"workload": f"serve_equiv_{nreq}_requests",
                                                      "distinct_pairs": len(pool),
                                                      "max_slots": args.serve_slots,
                                                      "hbm_budget_gb": args.serve_budget_gb},
                      "counters": d, "clocks": clk.summary(), "gpu_launches": int(d["steps"])}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.case == "serve":
        if rank == 0:
            run_serve_case(args, local)
        return
    if args.case == "batch":
        if rank == 0:
            run_batch_case(args, local)
        return
    import numpy as np
    import torch

    import dfagen
    import paper_2508_20735_gb300 as g

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    g.build()

    A = dfagen.random_dfa(WORKLOAD["n"], WORKLOAD["k"], WORKLOAD["p_accept"], WORKLOAD["seed"])
    n, k = A.n, A.k
    d_delta = torch.from_numpy(A.delta.view(np.int32)).cuda()
    d_acc = torch.from_numpy(A.accept).cuda()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    dd, keep = g.make_dfa(d_delta, d_acc)
    opts = g.make_opts("moore", flags=(g.DFA_FLAG_STOP_DISCRETE if args.stop_discrete else 0) |
                       (g.DFA_FLAG_BUCKETED if args.bucketed else 0))
    ws_bytes = g.dfa_workspace_size(dd, opts)
    ws = g._workspace(ws_bytes)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream

    def step():
        st, res = g.dfa_minimise(dd, opts, out.data_ptr(), ws.data_ptr(), ws_bytes, sptr)
        if st != 0:
            raise RuntimeError(f"dfa_minimise failed: {st} {g.last_error()}")
        return res

    for _ in range(args.warmup):
        res = step()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    rounds = []
    dev_ns = []
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for i in range(args.steps):
            step_ev[i][0].record(stream)
            res = step()
            step_ev[i][1].record(stream)
            rounds.append(res.rounds_executed)
            dev_ns.append(res.device_ns)
        ev1.record(stream)
        barrier()
    # each launch's duration from CUDA events on its stream (the call's control-block reset and
    # read-back included), and from the kernel's own clock stamps
    launch_ms = [a.elapsed_time(b) for a, b in step_ev]
    elapsed_ms = ev0.elapsed_time(ev1)
    trans = n * k * sum(rounds)
    value, elapsed_s = whole_job(trans, elapsed_ms * 1e-3, dist, "cuda")
    elapsed_ms = elapsed_s * 1e3
    ms_per_step = elapsed_ms / args.steps

    # roofline of the refinement kernel: (4k+8)*n algorithmic bytes per round
    kernel_s = statistics.mean(launch_ms) * 1e-3
    algo_bytes = (4 * k + 8) * n * statistics.mean(rounds)
    peak, peak_kind = peaks()
    achieved = algo_bytes / kernel_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
                "traffic": None, "kernel": "dfa::moore_kernel",
                "algorithmic_bytes_per_launch": algo_bytes, "kernel_ms": kernel_s * 1e3,
                "kernel_ms_median": statistics.median(launch_ms), "kernel_ms_best": min(launch_ms),
                "kernel_ms_device_clock": statistics.mean(dev_ns) * 1e-6,
                "kernel_ms_source": "CUDA events around each launch on its stream"}
    prof = os.path.join(ROOT, "profiles", "moore_kernel_traffic_random_n2p24_k4.txt")
    if os.path.exists(prof) and args.lg == 24 and not args.stop_discrete and not args.bucketed:
        fields = {}
        with open(prof) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    key, val = line.split(":", 1)
                    fields[key.strip()] = val.strip()
        # the figure is null once the kernel sources have changed since it was measured
        if fields.get("kernel_source_hash") == kernel_source_hash():
            roofline["traffic"] = int(fields["dram_bytes_per_launch"])

    # the same workload stopping at n blocks (DFA_FLAG_STOP_DISCRETE): same partition, no confirming round
    stop_discrete = None
    if rank == 0 and world == 1 and not args.no_extras:
        sopts = g.make_opts("moore", flags=g.DFA_FLAG_STOP_DISCRETE)
        sdev = []
        for i in range(args.warmup + args.steps):
            st, sr = g.dfa_minimise(dd, sopts, out.data_ptr(), ws.data_ptr(), ws_bytes, sptr)
            if st != 0:
                raise RuntimeError(f"dfa_minimise (stop at n blocks) failed: {st} {g.last_error()}")
            if i >= args.warmup:
                sdev.append(sr.device_ns)
        sd_s = statistics.median(sdev) * 1e-9
        stop_discrete = {"device_ms": sd_s * 1e3, "rounds": sr.rounds_executed, "blocks": sr.num_blocks,
                         "transitions_per_s": n * k * sr.rounds_executed / sd_s,
                         "plain_device_ms": statistics.median(dev_ns) * 1e-6}

    # the ceiling of the label gathers: random 4-byte L2 reads, measured now on a 64 MiB (L2-resident) array;
    # each round issues (k + 1) n such requests (k label gathers, one renumbering atomic per state)
    l2 = None
    try:
        probe = torch.zeros(1 << 24, dtype=torch.int32, device="cuda")
        peak_l2 = l2probe_gather(probe, 1 << 28, stream=stream)
        del probe
        req = (k + 1) * n * statistics.mean(rounds)
        l2 = {"bound": "l2_random_requests", "achieved": req / kernel_s / 1e9, "peak": peak_l2 / 1e9,
              "unit": "G requests/s", "frac": req / kernel_s / peak_l2,
              "requests_per_launch": req, "peak_source": "bench_l2probe.cu, measured in this run (64 MiB array)"}
    except Exception as exc:   # a measurement aid: report why it is missing
        l2 = {"unavailable": str(exc)}

    # end to end through the public C calls with host buffers (pinned), copies inside the timed region:
    # every step stages its inputs host -> device, refines, and copies the partition device -> host.
    # Steps alternate between two streams (dfa_minimise_async, two workspaces), so one step's copies
    # overlap the previous step's refinement; each step's result is collected (dfa_minimise_result)
    # before its stream is reused.
    e2e = None
    if not args.no_e2e:
        h_delta = torch.from_numpy(A.delta.view(np.int32)).pin_memory()
        h_acc = torch.from_numpy(A.accept).pin_memory()
        h_out = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(2)]
        hd, hkeep = g.make_dfa(h_delta, h_acc)
        hws_bytes = g.dfa_workspace_size(hd, opts)
        hws = [g._workspace(hws_bytes) for _ in range(2)]
        hst = [torch.cuda.Stream(), torch.cuda.Stream()]

        def issue(i):
            s = i % 2
            st = g.minimise_async(hd, opts, h_out[s].data_ptr(), hws[s].data_ptr(), hws_bytes, hst[s].cuda_stream)
            if st != 0:
                raise RuntimeError(f"dfa_minimise_async (host buffers) failed: {st} {g.last_error()}")

        def collect(i):
            s = i % 2
            st, r = g.minimise_result(hws[s].data_ptr(), hst[s].cuda_stream)
            if st != 0:
                raise RuntimeError(f"dfa_minimise_result failed: {st} {g.last_error()}")
            return r.rounds_executed

        def run(count):
            rounds = []
            for i in range(count):
                if i >= 2:
                    rounds.append(collect(i - 2))
                issue(i)
            for i in range(max(0, count - 2), count):
                rounds.append(collect(i))
            return rounds

        run(max(2, args.warmup))
        barrier()
        t0 = time.perf_counter()
        er = run(args.steps)
        barrier()
        e2e_val, _ = whole_job(n * k * sum(er), time.perf_counter() - t0, dist, "cuda")
        e2e = {"value": e2e_val, "unit": UNIT,
               "h2d_bytes_per_step": int(h_delta.numel() * 4 + h_acc.numel()),
               "d2h_bytes_per_step": int(h_out[0].numel() * 4),
               "pipeline": "two streams, dfa_minimise_async + dfa_minimise_result"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(A)
    ex = None
    if rank == 0 and world == 1 and not args.no_extras:
        del ws
        torch.cuda.empty_cache()
        ex = extras(g)
        ex["random_n2p24_k4_stop_discrete"] = stop_discrete

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "u32", "data": "synthetic",
                "config": dict(WORKLOAD, algo="moore (signature refinement)", rounds=rounds[-1],
                               **({"flags": "DFA_FLAG_STOP_DISCRETE"} if args.stop_discrete else {}),
                               **({"gather": "bucketed (DFA_FLAG_BUCKETED)"} if args.bucketed else {}),
                               l2="inputs larger than L2 (delta 256 MiB)",
                               parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
                "clocks": clk.summary(), "e2e": e2e, "gpu_launches": args.steps,
                "roofline": roofline, "l2_roofline": l2, "cpu_baseline": cpu, "extras": ex}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ----------------------------------------------------------------- the L2 probe (a measurement aid)
L2PROBE_SRC = os.path.join(ROOT, "bench_l2probe.cu")
L2PROBE_LIB = os.path.join(ROOT, "_build", "libl2probe.so")


def build_l2probe() -> str:
    """Compiles bench_l2probe.cu (sm_103a) into _build/libl2probe.so when stale.
    The probe is kept out of the product library: it measures the GPU, not the method."""
    import shutil
    if os.path.exists(L2PROBE_LIB) and os.path.getmtime(L2PROBE_LIB) >= os.path.getmtime(L2PROBE_SRC):
        return L2PROBE_LIB
    os.makedirs(os.path.dirname(L2PROBE_LIB), exist_ok=True)
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = L2PROBE_LIB + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
                        "-Xcompiler", "-fPIC", "-shared", L2PROBE_SRC, "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on bench_l2probe.cu:\n{r.stderr}")
    os.replace(tmp, L2PROBE_LIB)
    return L2PROBE_LIB


def l2probe_gather(table, reads: int = 1 << 28, stream=None) -> float:
    """Random 4-byte reads per second from `table` (a CUDA tensor whose byte size
    is a power of two; 64 MiB stays in L2)."""
    import ctypes
    lib = ctypes.CDLL(build_l2probe())
    lib.l2probe_gather.restype = ctypes.c_int
    lib.l2probe_gather.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_double)]
    lib.l2probe_error.restype = ctypes.c_char_p
    rate = ctypes.c_double(0.0)
    st = lib.l2probe_gather(table.data_ptr(), table.numel() * table.element_size(), int(reads),
                            stream.cuda_stream if stream is not None else None, ctypes.byref(rate))
    if st != 0:
        raise ValueError(f"l2probe_gather: {lib.l2probe_error().decode()} ({st})")
    return rate.value


# the sources the signature-refinement kernel and its launch are compiled from
MOORE_SOURCES = ("api.cu", "api_util.h", "common.cuh", "internal.h", "moore.cu")


def kernel_source_hash() -> str:
    """Hash of the refinement kernel's sources, tying a committed ncu traffic figure to the code it measured."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2508_20735_gb300", "csrc")
    for f in MOORE_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
