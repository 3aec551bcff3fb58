/*
 * dfa.h -- C ABI of the GB300 DFA partition-refinement library (libdfa_gb300.so).
 *
 * Problem statement (Section 2 of the paper): a DFA A = (Q, Σ, δ, F, q0) with
 * states Q = {0..n-1} and letters Σ = {0..k-1}.  Minimisation identifies the
 * DFA with the fewest states and the same language; on the hot path it is the
 * coarsest partition of Q that respects F and is a congruence for δ ("the
 * coarsest set partition problem", Section 2).  Equivalence asks L(A) = L(B)
 * (Section 4).
 *
 * Representation (Section 2, "Representation"): δ is k arrays of length n,
 * letter-major, delta[a*n + q] = δ(q, a), as uint32.  accept[q] != 0 iff q ∈ F.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Memory: every array argument may be a device pointer or a host pointer
 *    (pageable or pinned); the library asks the CUDA runtime which it is.
 *    Host inputs are copied into the workspace and host outputs are copied
 *    back, all on `stream`.  The caller owns all inputs, outputs and the
 *    workspace; the library keeps no pointer after a call returns.
 *  - Workspace: the minimise, batch and equivalence calls never allocate
 *    device memory.  The caller passes `workspace` (device memory, 256-byte
 *    aligned) of at least the size the matching *_workspace_size call returns.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls are stream-ordered and synchronise `stream` once before
 *    returning, so `res`, verdicts and host outputs are valid on return.
 *  - Errors: calls return a dfa_status and never abort.  dfa_last_error()
 *    gives a thread-local message for the last failing call on this thread.
 *    DFA_EINVAL covers n = 0, start >= n, a transition target >= n (detected
 *    on the device), k_A != k_B for equivalence, and a workspace that is too
 *    small.
 *  - Limits: 1 <= n <= DFA_MAX_STATES; 0 <= k <= DFA_MAX_LETTERS (k = 0 gives
 *    the partition {F, Q\F}).  All arithmetic is exact integer.
 *  - Output: block_out[q] is q's block; blocks are numbered 0..B-1 in
 *    increasing order of their smallest state (canonical numbering), so two
 *    runs agree bit for bit whenever their partitions agree.
 */
#ifndef DFA_GB300_H
#define DFA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DFA_MAX_STATES 0x7FFFFFFFu
#define DFA_MAX_LETTERS 4096u

/* One DFA.  Pointers are device or host pointers (see conventions). */
typedef struct dfa_t {
  uint32_t n;              /* number of states */
  uint32_t k;              /* number of letters */
  const uint32_t *delta;   /* k*n targets, delta[a*n + q] = δ(q, a) */
  const uint8_t *accept;   /* n bytes, nonzero = accepting */
  uint32_t start;          /* initial state; used by equivalence, ignored by minimise */
} dfa_t;

typedef enum dfa_status {
  DFA_OK = 0,
  DFA_EINVAL = -1,        /* bad argument, bad transition target or workspace too small */
  DFA_ENOMEM = -2,        /* the server's HBM budget cannot hold a request */
  DFA_ECUDA = -3,         /* a CUDA runtime call failed (message in dfa_last_error) */
  DFA_ETIMEOUT = -4,      /* a device-side wait or the call's time limit ran out */
  DFA_EMAXROUNDS = -5,    /* opts.max_rounds rounds ran without reaching the fixpoint */
  DFA_EBUSY = -6,         /* server: request not finished yet (poll) */
  DFA_ECANCELLED = -7     /* server: request was cancelled */
} dfa_status;

typedef enum dfa_algo {
  DFA_ALGO_MOORE = 0,     /* signature refinement, Section 3.3 / Algorithm 4 (sortPR's result) */
  DFA_ALGO_NAIVE = 1,     /* leader-election refinement, Section 3.2 / Algorithm 2 */
  DFA_ALGO_TRANS = 2,     /* partial transitive closure + naivePR, Section 3.4 / Algorithm 5 */
  DFA_ALGO_CLOSURE_MOORE = 3  /* Algorithm 5's closure table feeding signature refinement (Algorithm 4)
                                 instead of naivePR: same partition (the extra letters are words over
                                 the alphabet); rounds are those of Algorithm 4 on the extended DFA,
                                 on the n-state chain max popcount(x), 1 <= x <= n - 2, of them.  An
                                 extension the paper leaves open (it asks for sublinear refinement). */,
  DFA_ALGO_SORT = 4       /* Algorithm 4 with the paper's own renumbering: each round radix-sorts the
                             states by signature, marks signature changes and scans the marks (the
                             count read back on the host every round).  Same partition and rounds as
                             DFA_ALGO_MOORE; kept as the sort-versus-hash comparison. */
} dfa_algo;

/* Flags for dfa_opts.flags */
#define DFA_FLAG_EARLY_EXIT 0x1u   /* equivalence: stop once the start states separate */
#define DFA_FLAG_TABLE_ONLY 0x2u   /* signature refinement: renumber through the exact hash table in
                                      every round (no direct or filter rounds); same results, for
                                      comparisons and tests */
#define DFA_FLAG_STOP_DISCRETE 0x4u  /* signature refinement: stop after the round that leaves n
                                      blocks.  A partition of singletons cannot split, so the
                                      confirming round of Algorithm 4's until-test is not run and
                                      rounds_executed == rounds_changed for such inputs.  This is
                                      how Table 2's iteration counts for B_n (n - 1) come out.
                                      Same partition as without the flag.  Honoured by
                                      dfa_minimise, dfa_minimise_noalloc, both batch calls and
                                      dfa_equivalent; ignored by naivePR, transPR and the
                                      server. */

#define DFA_FLAG_BUCKETED 0x8u   /* signature refinement: read each round's labels through the bucketed
                                      gather (1 <= k <= 16, at most 2^26 states).  Once per call the
                                      transitions are sorted by (source range, target range); every
                                      round then streams them, reads the labels of one target range
                                      at a time from shared memory, and rebuilds each source range's
                                      signatures in shared memory, instead of k random label reads
                                      per state.  Same results; more workspace (dfa_workspace_size
                                      accounts for it).  Off by default: the direct reads measured
                                      faster on GB300.  Honoured by dfa_minimise,
                                      dfa_minimise_async and dfa_equivalent. */
#define DFA_FLAG_GATHER 0x10u    /* signature refinement: never use the bucketed gather, even with
                                      DFA_FLAG_BUCKETED set; same results */
#define DFA_FLAG_ONE_BLOCK 0x20u /* signature refinement of a DFA (or union) of at most 16,384
                                      states: run it in one thread block where it fits (else the
                                      cooperative kernel); same results.  Honoured by dfa_minimise,
                                      dfa_minimise_async and dfa_equivalent. */
#define DFA_FLAG_CLUSTER 0x40u   /* the same on one thread-block cluster where the GPU can place it
                                      (else the cooperative kernel); without either flag the call
                                      picks the cluster from 6,144 states on, or where one block
                                      does not fit; same results. */

typedef struct dfa_opts {
  int32_t algo;            /* dfa_algo */
  uint32_t max_rounds;     /* 0 = no limit; otherwise DFA_EMAXROUNDS after this many rounds */
  uint64_t timeout_ns;     /* 0 = library default (600 s); limit on the whole call's device work */
  int32_t schedule;        /* -1 = autotune / default; >= 0 selects a kernel schedule.  Batch
                              calls: 0..11, 1 + (s & 1) states per lane, 256 >> ((s >> 1) % 3)
                              states per tile, and from 6 on every DFA of at most 65,536 states
                              refined alone by one thread block (DFA_EINVAL beyond 11; -1 lets
                              the autotuner time all twelve once per batch shape, see
                              dfa_minimise_batch).
                              dfa_minimise: 1, 2 or 4 forces the cooperative kernel with that
                              many states per thread (the default runs DFAs of at most 16,384
                              states in one thread block when they fit, see dfa_minimise) */
  uint32_t flags;          /* DFA_FLAG_* */
} dfa_opts;

/* Round counts follow Algorithm 4's loop: rounds_changed counts rounds whose
 * block count grew; rounds_executed also counts the final round that finds the
 * count unchanged (the fixpoint test), unless DFA_FLAG_STOP_DISCRETE ended the
 * loop at n blocks.  For naivePR/transPR a round is one
 * iteration of Algorithm 2's while-loop, the last one finding no split. */
typedef struct dfa_result {
  uint32_t num_blocks;
  uint32_t rounds_changed;
  uint32_t rounds_executed;
  int32_t status;          /* dfa_status of this DFA */
  uint64_t device_ns;      /* device time of the refinement kernel(s) */
} dfa_result;

/* ---------------------------------------------------------------- minimise */

/* Bytes of workspace dfa_minimise needs for this DFA and options (0 on bad arguments). */
size_t dfa_workspace_size(const dfa_t *dfa, const dfa_opts *opts);

/* Coarsest partition of all n states of `dfa` (unreachable states are kept;
 * Section 2 treats their removal as a separate pre-processing step).
 * block_out: n uint32 (device or host).  res: host struct.  opts may be NULL
 * (Moore, no round limit, default time limit).  Signature refinement of a DFA
 * of at most 16,384 states runs in one thread block with its labels, table
 * and (when they fit) transitions in shared memory, when its packed
 * signatures fit 63 bits or it has at most 4,096 states, up to 6,143 states;
 * from 6,144 states on, or where one block does not fit, on one thread-block
 * cluster (8 or 16 blocks; labels replicated and the renumbering table
 * distributed over the blocks' shared memory) where the GPU can place it
 * (DFA_FLAG_ONE_BLOCK and DFA_FLAG_CLUSTER force either); larger DFAs, DFA_FLAG_TABLE_ONLY,
 * DFA_FLAG_BUCKETED and an explicit schedule run the cooperative kernel over
 * the whole GPU.  The results are the same. */
int dfa_minimise(const dfa_t *dfa, const dfa_opts *opts, uint32_t *block_out, dfa_result *res,
                 void *workspace, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------- batch */

/* Workspace bytes for dfa_minimise_batch over `count` DFAs (host array of dfa_t). */
size_t dfa_batch_workspace_size(const dfa_t *dfas, uint32_t count, const dfa_opts *opts);

/* Refines `count` independent DFAs in one persistent launch.  block_out holds
 * sum(n_i) entries, DFA i's blocks at offset sum_{j<i} n_j, numbered within
 * DFA i.  res[i] (host array of count) equals what dfa_minimise reports for DFA
 * i alone (partition and round counts; device_ns is the whole batch's time).
 * The DFAs' arrays may live anywhere (host or device), independently.
 * Schedules (dfa_opts.schedule): with -1 the first call for a batch shape (GPU,
 * total states and batch size rounded up to powers of two, largest k) runs the
 * batch under all twelve schedules and keeps the fastest by device time; the
 * choice and every schedule's time are kept in memory and in the JSON file
 * $DFA_AUTOTUNE_CACHE (default ~/.cache/dfa_gb300_autotune.json), one line per
 * shape: "batch|<GPU>|states2^a|dfas2^b|kmaxc": [choice, ns_0, ..., ns_11].
 * The launch is a CUDA graph (control-block reset + the cooperative kernel,
 * then for schedules 6..11 the kernel that refines the DFAs of at most 65,536
 * states one per block, the cooperative kernel then refining only the larger
 * ones and left out when there are none), instantiated once per host thread,
 * device and graph shape and updated in place by later calls (dfa_batch_graph_stats
 * counts both). */
int dfa_minimise_batch(const dfa_t *dfas, uint32_t count, const dfa_opts *opts, uint32_t *block_out,
                       dfa_result *res, void *workspace, size_t ws_bytes, void *stream);

/* The same batch given as two packed buffers instead of one dfa_t per DFA
 * (the segment-offset form, no counterpart in the paper):
 *   n, k     host arrays of `count` entries: DFA i has n[i] >= 1 states and
 *            k[i] letters (start state 0);
 *   delta    sum_i k[i] n[i] uint32 targets: DFA i's letter-major k[i] x n[i]
 *            table starts at element sum_{j<i} k[j] n[j]; targets are local
 *            to DFA i (< n[i]); NULL only if every k[i] = 0;
 *   accept   sum_i n[i] bytes: DFA i's at offset sum_{j<i} n[j].
 * delta and accept may each be host or device memory (checked once per buffer;
 * host buffers are staged into the workspace with one copy each).  The caller
 * keeps ownership of every buffer.  block_out, res, the workspace, the stream
 * and every error (DFA_EINVAL for a bad size or target, DFA_EMAXROUNDS, ...)
 * behave as in dfa_minimise_batch, whose results these calls reproduce DFA by
 * DFA. */
size_t dfa_batch_packed_workspace_size(uint32_t count, const uint32_t *n, const uint32_t *k, const uint32_t *delta,
                                       const uint8_t *accept, const dfa_opts *opts);
int dfa_minimise_batch_packed(uint32_t count, const uint32_t *n, const uint32_t *k, const uint32_t *delta,
                              const uint8_t *accept, const dfa_opts *opts, uint32_t *block_out, dfa_result *res,
                              void *workspace, size_t ws_bytes, void *stream);

/* Process-wide counts of the batch calls' graph handling: instantiations of
 * the batch graph and calls that reused a kept instantiation through
 * cudaGraphExecUpdate.  Either pointer may be NULL.  Always DFA_OK. */
int dfa_batch_graph_stats(uint64_t *instantiations, uint64_t *updates);

/* ---------------------------------------------------------------- the minimal DFA */

/* Workspace bytes for dfa_quotient on these arrays (0 on bad arguments). */
size_t dfa_quotient_workspace_size(const dfa_t *d, const uint32_t *block, const uint32_t *delta_out,
                                   const uint8_t *accept_out);

/* The minimal DFA A' with L(A') = L(A) (the paper's problem statement), from a
 * coarsest partition `block` of d's states (n entries, ids < n, as
 * dfa_minimise writes it): A''s states are the blocks that hold a state
 * reachable from d->start, numbered in order of their smallest reachable
 * state; each takes the transitions and acceptance of that state.  Outputs,
 * caller-owned, host or device: delta_out (capacity k*n; A''s letter-major
 * table, row a at offset a*n'), accept_out (capacity n), *n_out = n' and
 * *start_out (host).  Reachability runs on the device (breadth-first, one
 * launch).  DFA_EINVAL for a target or block id >= n.  Synchronises the
 * stream. */
int dfa_quotient(const dfa_t *d, const uint32_t *block, uint32_t *delta_out, uint8_t *accept_out, uint32_t *n_out,
                 uint32_t *start_out, void *workspace, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------- equivalence */

/* Workspace bytes for dfa_equivalent on this pair. */
size_t dfa_equivalent_workspace_size(const dfa_t *a, const dfa_t *b, const dfa_opts *opts);

/* L(A) = L(B)?  Decided by refining the disjoint union A ⊎ B (B's states
 * offset by n_A) and comparing the blocks of the two start states (Section 4:
 * equivalence by minimisation).  Requires k_A = k_B.  *equivalent is set to 1
 * or 0.  res describes the union's refinement; with DFA_FLAG_EARLY_EXIT the
 * refinement stops at the first round that separates the start states, and
 * res->rounds_executed is then the length of a shortest word that A and B
 * disagree on.  A union of at most 16,384 states is refined by the same
 * small kernels as dfa_minimise (one thread block or one cluster; the
 * DFA_FLAG_ONE_BLOCK / DFA_FLAG_CLUSTER flags and an explicit schedule apply
 * as there), with the same results. */
int dfa_equivalent(const dfa_t *a, const dfa_t *b, const dfa_opts *opts, int *equivalent,
                   dfa_result *res, void *workspace, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------- stream-ordered minimisation */

/* dfa_minimise (signature refinement, DFA_ALGO_MOORE only) enqueued on `stream`
 * without waiting: the staging of host inputs, the refinement and the copy of
 * block_out (host or device) are stream-ordered, so several calls on different
 * streams overlap one call's copies with another's refinement.  The arrays and
 * the workspace must stay valid, and untouched by other work, until
 * dfa_minimise_result has returned.  Argument errors are returned at once;
 * errors found on the device (a target >= n, a timeout) by dfa_minimise_result. */
int dfa_minimise_async(const dfa_t *d, const dfa_opts *opts, uint32_t *block_out, void *workspace, size_t ws_bytes,
                       void *stream);

/* Waits for `stream` and returns the status of the dfa_minimise_async call that
 * used `workspace` on it; fills *res (host, may be NULL) as dfa_minimise does. */
int dfa_minimise_result(const void *workspace, dfa_result *res, void *stream);

/* ---------------------------------------------------------------- product exploration */

#define DFA_CHECK_EQUIVALENCE 0   /* L(A) = L(B) */
#define DFA_CHECK_INCLUSION 1     /* L(A) ⊆ L(B) */

/* Workspace bytes for dfa_product_check (0 on bad arguments). */
size_t dfa_product_workspace_size(const dfa_t *a, const dfa_t *b, uint64_t max_pairs);

/* Equivalence or inclusion by exploring the synchronous product from
 * <start_A, start_B> (Section 4: Algorithm 6 without R+, the "naive"
 * Hopcroft-Karp variant; inclusion keeps only the "A accepts, B rejects" half
 * of its acceptance test).  Requires k_A = k_B.  The search is breadth first on the device;
 * a violating pair ends it once its level is complete.  Outputs (host):
 *   *holds    1 if the condition holds, else 0;
 *   *pairs    pairs explored: all reachable pairs if it holds, else those of
 *             the levels up to the violating one (NULL to skip);
 *   *cex_len  that level, the length of a shortest word in L(A) \ L(B) (or in
 *             their symmetric difference), -1 if it holds (NULL to skip).
 * max_pairs bounds the explored pairs (capped at n_A n_B and 2^31) and sizes the
 * workspace (8 B per pair for each of two frontiers, 16 B per pair of set);
 * DFA_ENOMEM if the product has more reachable pairs.  Arrays may be host or
 * device memory.  Synchronises the stream. */
int dfa_product_check(const dfa_t *a, const dfa_t *b, int mode, uint64_t max_pairs, int *holds, uint64_t *pairs,
                      int64_t *cex_len, void *workspace, size_t ws_bytes, void *stream);

/* ---------------------------------------------------------------- trans (Algorithm 1) */

/* Largest n for dfa_trans: Reach has n^4 bits (two copies of 512 MiB at 256). */
#define DFA_TRANS_MAX_STATES 256u

/* Workspace bytes for dfa_trans (0 on bad arguments or n > DFA_TRANS_MAX_STATES). */
size_t dfa_trans_workspace_size(const dfa_t *d, const uint32_t *block_out);

/* Algorithm 1 (Section 3.1, "trans"): minimisation by the transitive closure
 * of the pair graph, whose nodes are the n^2 state pairs and whose edges are
 * (q, q') -> (δ(q,a), δ(q',a)).  Each iteration squares the boolean
 * reachability matrix (R := R | R R) and then labels Apart every pair with an
 * edge of R to an Apart pair; both steps read only the previous iteration's
 * values.  The loop stops after an iteration that labels nothing new.
 * Outputs: block_out[q] (n entries, host or device), the canonical partition
 * (q, q' in one block iff not Apart); *iterations (host), the loop's
 * executions including the last.  δ and accept may be host or device memory;
 * δ entries >= n give DFA_EINVAL.  Synchronises the stream once per
 * iteration (the loop test is read on the host). */
int dfa_trans(const dfa_t *d, uint32_t *block_out, uint32_t *iterations, void *workspace, size_t ws_bytes,
              void *stream);

/* ---------------------------------------------------------------- serving */

typedef struct dfa_server dfa_server;

#define DFA_REQ_MINIMISE 0
#define DFA_REQ_EQUIVALENT 1

/* A server owns one device arena of hbm_budget_bytes (allocated once here) and
 * a host thread that admits queued requests while arena space and one of
 * max_slots slots are free, and refines all admitted requests together, one
 * round at a time (continuous batching). */
int dfa_serve_create(dfa_server **out, size_t hbm_budget_bytes, uint32_t max_slots, int device);

/* Queues a request; the DFAs are copied in before this returns, so the caller
 * may free them.  `b` is NULL for DFA_REQ_MINIMISE.  *ticket identifies it.
 * DFA_ENOMEM if the request can never fit the budget. */
int dfa_serve_submit(dfa_server *s, int kind, const dfa_t *a, const dfa_t *b, const dfa_opts *opts,
                     uint64_t *ticket);

/* DFA_EBUSY while the request is queued or running; DFA_OK (or the request's
 * error) once finished, filling res, *equivalent (equivalence requests) and,
 * for a minimisation request with block_out non-NULL, its partition (host
 * memory, n entries, canonical numbering).  Results equal those of
 * dfa_minimise / dfa_equivalent on the same input.  A finished ticket is
 * released by the first poll/wait that returns it. */
int dfa_serve_poll(dfa_server *s, uint64_t ticket, dfa_result *res, int *equivalent, uint32_t *block_out);

/* As dfa_serve_poll, but blocks up to timeout_ns (0 = forever). */
int dfa_serve_wait(dfa_server *s, uint64_t ticket, uint64_t timeout_ns, dfa_result *res, int *equivalent,
                   uint32_t *block_out);

/* Latency percentiles (submit to completion) and throughput of finished requests. */
int dfa_serve_stats(dfa_server *s, double *p50_us, double *p99_us, double *throughput_rps);

/* Counters since creation: refinement steps run (one round of every admitted
 * request per step), requests and states advanced by a round (their sums over
 * the steps), the state sum split by the round's renumbering mode
 * (mode_state_rounds[3]: direct, filter, table), and host wall time spent in
 * steps (descriptor upload to results on the host), in microseconds.  Any
 * pointer may be NULL. */
int dfa_serve_counters(dfa_server *s, uint64_t *steps, uint64_t *request_rounds, uint64_t *state_rounds,
                       uint64_t *mode_state_rounds, double *step_us);

/* Cancels outstanding requests, joins the thread and frees the arena.  No other
 * call on `s` may run concurrently with or after this one. */
int dfa_serve_destroy(dfa_server *s);

/* ---------------------------------------------------------------- no-allocation variant */

/* The paper has no counterpart to this call.  It is dfa_minimise (signature
 * refinement only) for callers that cannot hand the library a workspace:
 * code inside a host framework that owns every device allocation, or
 * latency-critical paths where cudaMalloc is off-limits because it may
 * synchronise the device.  Its scratch is a fixed 8 MiB array compiled into
 * the library, held by every GPU that loads it until the process exits.
 *  - n <= DFA_NOALLOC_MAX_STATES, else DFA_EINVAL (use dfa_minimise).
 *  - delta, accept and block_out must be device pointers (else DFA_EINVAL).
 *  - The first call on a device looks the array's device address up.
 *  - Synchronous: the call waits for `stream` before it returns (it reads the
 *    round counts back).  On a stream that is being captured into a CUDA
 *    graph it enqueues nothing and returns DFA_EINVAL.
 *  - All calls on a device share the array, so a call holds a per-device lock
 *    until its stream has drained: calls from several host threads or on
 *    several streams run one after another.  Each call clears what it needs;
 *    nothing carries over.
 *  - Calls no cudaMalloc, cudaFree or allocating library routine. */
#define DFA_NOALLOC_MAX_STATES 65536u
int dfa_minimise_noalloc(const dfa_t *dfa, const dfa_opts *opts, uint32_t *block_out, dfa_result *res,
                         void *stream);

/* ---------------------------------------------------------------- misc */

/* Thread-local message describing the last failing call on this thread. */
const char *dfa_last_error(void);

/* Library version string. */
const char *dfa_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DFA_GB300_H */
