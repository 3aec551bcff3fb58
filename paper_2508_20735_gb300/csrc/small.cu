// Signature refinement of a DFA in one thread block: the single-DFA kernel for
// up to kSmallMaxStates states (everything in shared memory), and the batches'
// block-per-DFA kernel, which also refines DFAs of up to 65,536 states with
// only their labels in shared memory (medium_refine, further below).
//
// Algorithm 4 (Section 3.3) on a state space that fits in shared memory
// (n <= kSmallMaxStates): the labels of two consecutive rounds (16-bit), the
// transitions (16-bit targets, when they fit) and the renumbering table live
// in shared memory, and rounds are separated by __syncthreads instead of
// grid-wide barriers.  On a cooperative launch over the whole GPU the barriers
// dominate at this size (about 20 us a round for 10,000 states).
//
// Each round renumbers exactly, in one of three ways chosen alike by every
// thread from the width w of the labels it reads:
//  * direct  (k+1) w <= log2 T (at most 16): the packed signature is itself
//            the new label (so every label stays below T); each state sets the
//            flag of its signature in the table, and the flags set count the
//            blocks;
//  * packed  (k+1) w <= 63: the packed signature is the key of a shared-memory
//            table (one CAS per probe, on 32-bit slots while the key has at most
//            31 bits, else on 64-bit slots); the new label is its slot;
//  * compare otherwise: a table slot holds one representative state, and a
//            state joins a slot only if its full signature (own label and the
//            label of every successor) equals the representative's, so a hash
//            collision costs a probe, never a merge; the label is the slot.
// The final partition is numbered canonically (blocks in order of their
// smallest state) inside the block.
#include <algorithm>

#include "api_util.h"

namespace dfa {

static constexpr int kSmallThreads = 1024;
static constexpr size_t kSmallSmem = 220 * 1024;   // dynamic shared memory the kernel may take
static constexpr uint32_t kSmallDirectBits = 16;   // direct rounds: labels of at most 16 bits

struct SmallArgs {
  const uint32_t *delta;   // k*n, letter-major
  const uint8_t *accept;   // n
  uint32_t n, k;
  uint32_t *out;           // n: canonical block numbers
  Ctrl *ctrl;
  uint32_t log2T;          // table slots 2^log2T >= 1.5 n
  uint32_t wide_table;     // 1: the table has 64-bit slots (packed rounds possible)
  uint32_t staged;         // 1: δ is copied into shared memory as 16-bit targets (k n halfwords)
  uint32_t max_rounds;     // 0 = none
  uint32_t stop_discrete;  // 1: stop after a round that leaves n blocks
  unsigned long long timeout_ns;
  uint32_t track;          // equivalence by union: record the first round after which sa and sb are apart
  uint32_t sa, sb;
  uint32_t early_exit;     // with track: stop there (round 0: no round at all)
};

__device__ __forceinline__ uint32_t small_mix(uint32_t h, uint32_t v) {
  h ^= v + 0x9E3779B9u + (h << 6) + (h >> 2);
  return h * 0x85EBCA6Bu;
}

// What one refinement in a block produced.
struct SmallOut {
  uint32_t err, rounds_executed, rounds_changed, num_blocks, maxed;
  uint32_t sep_round;   // with A.track: first round that separated sa and sb (0: their acceptance), else ~0
};

// The refinement of one DFA by the calling block (every thread takes part),
// with the canonical numbering written to A.out.  sm: the block's dynamic
// shared memory; C: control block for the trace (thread 0), or null; t0: the
// start time the call's time limit counts from.
__device__ __forceinline__ SmallOut small_refine(const SmallArgs &A, uint32_t *sm, Ctrl *C, unsigned long long t0) {
  __shared__ uint32_t s_red[32];
  __shared__ uint32_t s_flag;   // ERR_BAD_DELTA seen by any thread (read after the round's last barrier)
  __shared__ uint32_t s_stop;   // the call's time limit ran out (thread 0 decides between rounds)
  const uint32_t n = A.n, k = A.k, tid = threadIdx.x, bd = blockDim.x;
  const uint32_t T = 1u << A.log2T, mask = T - 1u;
  const uint32_t twords = A.wide_table ? 2u * T : T;
  uint32_t *tbl = sm;                                             // table (also the direct rounds' flags)
  unsigned long long *tbl64 = reinterpret_cast<unsigned long long *>(sm);
  // label arrays of n rounded up to 8 halfwords, so that both and d16 start on 16 bytes
  uint16_t *const lab0 = reinterpret_cast<uint16_t *>(sm + twords), *const lab1 = lab0 + ((n + 7u) & ~7u);
  uint16_t *d16 = lab1 + ((n + 7u) & ~7u);                      // k n halfwords when staged
  volatile uint32_t *vtbl = tbl;
  if (tid == 0) s_flag = 0u;
  __syncthreads();   // s_flag is clear before any thread reports into it
  // the initial partition {F, Q \ F}: labels 0/1, B_0 = the classes present
  // (16-byte loads where the arrays allow, several in flight per thread: the
  // staging is latency-bound otherwise)
  uint32_t seen = 0, bad = 0;
  stage_accept(A.accept, n, lab0, &seen);
  if (A.staged) {   // δ into shared memory, validated once
    stage_delta(A.delta, (size_t)k * n, n, d16, &bad);
    if (bad) atomicOr(&s_flag, ERR_BAD_DELTA);
  }
  const uint32_t classes = block_sum(((seen & 1u) ? 1u : 0u) | ((seen & 2u) ? 0x10000u : 0u), s_red);
  const uint32_t any_acc = (classes & 0xFFFFu) != 0u, any_rej = (classes >> 16) != 0u;
  uint32_t B_prev = any_acc + any_rej, B_r = B_prev;
  uint32_t r = 0, changed = 0, cur = 0, maxed = 0, err = s_flag, w = 1, sep = 0xFFFFFFFFu;
  bool skip = false;
  if (A.track && (A.accept[A.sa] != 0) != (A.accept[A.sb] != 0)) {   // the empty word separates them
    sep = 0;
    skip = A.early_exit != 0;   // the answer needs no round: the initial partition is reported
  }
  uint32_t nt = 0;   // trace entries (thread 0)
  if (tid == 0 && C) trace_put(C, nt, t0, kTraceStart);
  // δ(q, a): the shared copy, or global memory (an invalid target reads as 0 and is reported)
  auto target = [&](uint32_t a, uint32_t q) -> uint32_t {
    if (A.staged) return d16[(size_t)a * n + q];
    uint32_t d = A.delta[(size_t)a * n + q];
    if (d >= n) {
      bad = 1u;
      d = 0u;
    }
    return d;
  };
  for (r = 1; !err && !skip; ++r) {
    const uint16_t *src = cur ? lab1 : lab0;
    uint16_t *dst = cur ? lab0 : lab1;
    const uint32_t K = (k + 1u) * w;
    const uint32_t mode = (K <= kSmallDirectBits && K <= A.log2T) ? 0u : K <= 31u ? 3u : (A.wide_table && K <= 63u) ? 1u : 2u;
    const uint32_t words = mode == 0u ? (1u << K) : (mode == 1u ? 2u * T : T);   // packed 32-bit keys (3): T words
    for (uint32_t i = tid; i < words; i += bd) tbl[i] = 0u;
    __syncthreads();
    uint32_t created = 0;
    bad = 0;
    if (mode == 0u) {   // direct: the signature is the label; a flag per signature present
      for (uint32_t q = tid; q < n; q += bd) {
        uint32_t key = src[q];
        uint32_t shift = w;
        for (uint32_t a = 0; a < k; ++a) {
          key |= (uint32_t)src[target(a, q)] << shift;
          shift += w;
        }
        dst[q] = (uint16_t)key;
        tbl[key] = 1u;   // every writer of a slot writes the same value
      }
      __syncthreads();
      for (uint32_t i = tid; i < (1u << K); i += bd) created += tbl[i];
    } else if (mode == 1u) {   // packed key, 64-bit slots
      for (uint32_t q = tid; q < n; q += bd) {
        unsigned long long key = src[q];
        uint32_t shift = w;
        for (uint32_t a = 0; a < k; ++a) {
          key |= (unsigned long long)src[target(a, q)] << shift;
          shift += w;
        }
        key |= 1ull << 63;   // never 0, the free marker
        uint32_t slot = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64u - A.log2T));
        for (uint32_t probe = 0; probe < T; ++probe) {
          const unsigned long long v = atomicCAS(&tbl64[slot], 0ull, key);
          if (v == 0ull) {   // q represents a new block
            ++created;
            break;
          }
          if (v == key) break;   // q joins that block
          slot = (slot + 1u) & mask;
        }
        dst[q] = (uint16_t)slot;
      }
    } else if (mode == 3u) {   // packed key of at most 31 bits, 32-bit slots
      for (uint32_t q = tid; q < n; q += bd) {
        uint32_t key = src[q];
        uint32_t shift = w;
        for (uint32_t a = 0; a < k; ++a) {
          key |= (uint32_t)src[target(a, q)] << shift;
          shift += w;
        }
        key |= 1u << 31;   // never 0, the free marker
        uint32_t slot = (key * 0x9E3779B1u) >> (32u - A.log2T);
        for (uint32_t probe = 0; probe < T; ++probe) {
          const uint32_t v = atomicCAS(&tbl[slot], 0u, key);
          if (v == 0u) {   // q represents a new block
            ++created;
            break;
          }
          if (v == key) break;   // q joins that block
          slot = (slot + 1u) & mask;
        }
        dst[q] = (uint16_t)slot;
      }
    } else {   // representative and full comparison
      for (uint32_t q = tid; q < n; q += bd) {
        uint32_t h = small_mix(0x3C6EF372u, src[q]);
        for (uint32_t a = 0; a < k; ++a) h = small_mix(h, src[target(a, q)]);
        h ^= h >> 15;
        uint32_t slot = (h * 0x2C1B3C6Du) >> (32u - A.log2T) & mask;
        for (uint32_t probe = 0; probe < T; ++probe) {
          uint32_t v = vtbl[slot];
          if (v == 0u) {
            v = atomicCAS(&tbl[slot], 0u, q + 1u);
            if (v == 0u) {   // q represents a new block
              ++created;
              break;
            }
          }
          const uint32_t p = v - 1u;
          bool same = src[q] == src[p];
          for (uint32_t a = 0; same && a < k; ++a) same = src[target(a, q)] == src[target(a, p)];
          if (same) break;   // q joins that block
          slot = (slot + 1u) & mask;
        }
        dst[q] = (uint16_t)slot;
      }
    }
    if (bad) atomicOr(&s_flag, ERR_BAD_DELTA);
    B_r = block_sum(created, s_red);   // includes the barriers that end the round
    if (tid == 0 && C) trace_put(C, nt, t0, kTraceRound | (mode << 4));
    cur ^= 1u;
    w = mode == 0u ? K : A.log2T;   // table rounds: labels are slots
    if (s_flag) {   // every thread reads it after the same barrier: a uniform decision
      err = s_flag;
      break;
    }
    const bool grew = B_r != B_prev;
    if (grew) ++changed;
    if (A.track && sep == 0xFFFFFFFFu) {   // the new labels, read after the round's barriers: uniform
      const uint16_t *nl = cur ? lab1 : lab0;
      if (nl[A.sa] != nl[A.sb]) {
        sep = r;
        if (A.early_exit) break;
      }
    }
    if (!grew) break;   // Algorithm 4's until-test: the round added no block
    if (A.stop_discrete && B_r == n) break;
    if (A.max_rounds != 0u && r >= A.max_rounds) {
      maxed = 1u;
      break;
    }
    // the call's time limit, every 16 rounds: thread 0 decides, every thread reads it after a barrier
    if ((r & 15u) == 0u) {
      if (tid == 0) s_stop = gtimer() - t0 > A.timeout_ns ? 1u : 0u;
      __syncthreads();
      if (s_stop) {
        err = ERR_TIMEOUT;
        break;
      }
    }
    B_prev = B_r;
  }
  if (skip) r = 0;
  if (err) return SmallOut{err, r, changed, 0u, maxed, sep};
  // canonical numbering: blocks in order of their smallest state (every label
  // is below T: a slot, or a direct signature of at most log2 T bits)
  const uint16_t *fin = cur ? lab1 : lab0;
  uint32_t blocks = B_r;
  if (B_r == n) {
    for (uint32_t q = tid; q < n; q += bd) A.out[q] = q;
  } else {
    uint16_t *rank = cur ? lab0 : lab1;   // free now: rank of each block's smallest state
    for (uint32_t i = tid; i < T; i += bd) tbl[i] = 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t q = tid; q < n; q += bd) atomicMin(&tbl[fin[q]], q);
    __syncthreads();
    const uint32_t per = (n + bd - 1) / bd;
    const uint32_t q0 = tid * per < n ? tid * per : n, q1 = q0 + per < n ? q0 + per : n;
    uint32_t c = 0;
    for (uint32_t q = q0; q < q1; ++q) c += tbl[fin[q]] == q;
    uint32_t total;
    uint32_t base = block_excl_scan(c, s_red, &total);
    for (uint32_t q = q0; q < q1; ++q)
      if (tbl[fin[q]] == q) rank[q] = (uint16_t)base++;
    __syncthreads();
    for (uint32_t q = tid; q < n; q += bd)
      if (tbl[fin[q]] == q) tbl[fin[q]] = 0x80000000u | rank[q];
    __syncthreads();
    for (uint32_t q = tid; q < n; q += bd) A.out[q] = tbl[fin[q]] & 0x7FFFFFFFu;
    blocks = total;
  }
  if (tid == 0 && C) trace_put(C, nt, t0, kTraceEnd);
  return SmallOut{0u, r, changed, blocks, maxed, sep};
}

// A DFA of at most 65,536 states refined by one block with its labels in
// shared memory and its renumbering table in global memory (the batch's
// block-per-DFA schedules, for DFAs the fully shared-memory refinement above
// cannot hold).  A label is the state number of its block's representative
// (so it fits 16 bits), one array of them in shared memory; a round writes the
// new labels to global memory (`newlab`) and copies them back after a block
// barrier.  Every round renumbers by representative comparison: a state hashes
// its signature, and a slot holds the representative that first claimed it; a
// state joins a slot's block only if its own label and every successor's label
// equal the representative's (so a hash collision costs a probe, never a
// merge).  Slots carry the round in their top 12 bits, so a slot of an earlier
// round reads as free and the table is cleared only once per 4,095 rounds.
struct MediumArgs {
  const uint32_t *delta;   // k*n, letter-major (global)
  const uint8_t *accept;   // n
  uint32_t n, k;
  uint32_t *out;           // n: canonical block numbers
  uint32_t *table;         // 2^log2T slots (global): round << 20 | (representative + 1)
  uint32_t log2T;
  uint32_t *newlab;        // n words of global scratch: a round's new labels, then the ranks
  uint32_t *minrep;        // n words of global scratch: each block's smallest state
  uint32_t max_rounds, stop_discrete;
  unsigned long long timeout_ns;
};
static constexpr uint32_t kMediumTagShift = 20;
static constexpr uint32_t kMediumTagMax = (1u << (32 - kMediumTagShift)) - 1u;   // 4,095

__device__ __forceinline__ SmallOut medium_refine(const MediumArgs &A, uint16_t *L, unsigned long long t0) {
  __shared__ uint32_t s_red[32];
  __shared__ uint32_t s_flag;
  __shared__ uint32_t s_stop;
  const uint32_t n = A.n, k = A.k, tid = threadIdx.x, bd = blockDim.x;
  const uint32_t T = 1u << A.log2T, mask = T - 1u;
  volatile uint32_t *vt = A.table;
  if (tid == 0) s_flag = 0u;
  for (uint32_t i = tid; i < T; i += bd) A.table[i] = 0u;   // no earlier round's slots
  // the initial partition {F, Q \ F}: labels 0/1
  uint32_t seen = 0, bad = 0;
  stage_accept(A.accept, n, L, &seen);
  const uint32_t classes = block_sum(((seen & 1u) ? 1u : 0u) | ((seen & 2u) ? 0x10000u : 0u), s_red);
  uint32_t B_prev = ((classes & 0xFFFFu) != 0u) + ((classes >> 16) != 0u), B_r = B_prev;
  uint32_t r = 0, changed = 0, maxed = 0, err = 0, tag = 0;
  auto target = [&](uint32_t a, uint32_t q) -> uint32_t {
    uint32_t d = A.delta[(size_t)a * n + q];
    if (d >= n) {
      bad |= 1u;
      d = 0u;
    }
    return d;
  };
  for (r = 1;; ++r) {
    if (++tag > kMediumTagMax) {   // the tags wrap: every slot is cleared
      tag = 1;
      for (uint32_t i = tid; i < T; i += bd) A.table[i] = 0u;
    }
    __syncthreads();   // the table (and last round's labels) ready
    uint32_t created = 0;
    bad = 0;
    for (uint32_t q = tid; q < n; q += bd) {
      const uint32_t lq = L[q];
      unsigned long long h = (0x243F6A8885A308D3ull ^ lq) * 0x9E3779B97F4A7C15ull;
      for (uint32_t a = 0; a < k; ++a) {
        h ^= L[target(a, q)];
        h *= 0x9E3779B97F4A7C15ull;
        h ^= h >> 29;
      }
      uint32_t slot = (uint32_t)(h >> (64u - A.log2T)), label = q;
      const uint32_t mine = (tag << kMediumTagShift) | (q + 1u);
      // at most T slots, each looked at at most twice (a failed claim re-reads it)
      bool placed = false;
      for (uint32_t step = 0; step < 2u * T && !placed; ++step) {
        uint32_t v = vt[slot];
        if ((v >> kMediumTagShift) != tag) {   // free in this round: claim it
          const uint32_t old = atomicCAS(&A.table[slot], v, mine);
          if (old == v) {   // q represents a new block
            ++created;
            placed = true;
            continue;
          }
          v = old;   // taken meanwhile (only by this round's claims): look at what took it
          if ((v >> kMediumTagShift) != tag) continue;
        }
        const uint32_t p = (v & ((1u << kMediumTagShift) - 1u)) - 1u;
        bool same = lq == L[p];
        for (uint32_t a = 0; same && a < k; ++a) same = L[target(a, q)] == L[target(a, p)];
        if (same) {   // q joins p's block
          label = p;
          placed = true;
          continue;
        }
        slot = (slot + 1u) & mask;
      }
      if (!placed) bad |= 2u;   // no slot (cannot happen at a load of at most 1/4)
      A.newlab[q] = label;
    }
    if (bad & 1u) atomicOr(&s_flag, ERR_BAD_DELTA);
    if (bad & 2u) atomicOr(&s_flag, ERR_TABLE_FULL);
    B_r = block_sum(created, s_red);   // its barriers also complete the round's new labels
    for (uint32_t q = tid; q < n; q += bd) L[q] = (uint16_t)A.newlab[q];
    if (s_flag) {   // read after the same barrier by every thread
      err = s_flag;
      break;
    }
    const bool grew = B_r != B_prev;
    if (grew) ++changed;
    if (!grew) break;   // Algorithm 4's until-test
    if (A.stop_discrete && B_r == n) break;
    if (A.max_rounds != 0u && r >= A.max_rounds) {
      maxed = 1u;
      break;
    }
    if ((r & 15u) == 0u) {
      if (tid == 0) s_stop = gtimer() - t0 > A.timeout_ns ? 1u : 0u;
      __syncthreads();
      if (s_stop) {
        err = ERR_TIMEOUT;
        break;
      }
    }
    B_prev = B_r;
  }
  if (err) return SmallOut{err, r, changed, 0u, maxed, 0xFFFFFFFFu};
  __syncthreads();   // the last labels are in shared memory
  // canonical numbering: blocks in order of their smallest state (labels are
  // representatives, so below n)
  uint32_t blocks = B_r;
  if (B_r == n) {
    for (uint32_t q = tid; q < n; q += bd) A.out[q] = q;
  } else {
    for (uint32_t q = tid; q < n; q += bd) A.minrep[q] = 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t q = tid; q < n; q += bd) atomicMin(&A.minrep[L[q]], q);
    __syncthreads();
    const uint32_t per = (n + bd - 1) / bd;
    const uint32_t q0 = tid * per < n ? tid * per : n, q1 = q0 + per < n ? q0 + per : n;
    uint32_t c = 0;
    for (uint32_t q = q0; q < q1; ++q) c += A.minrep[L[q]] == q;
    uint32_t total;
    uint32_t base = block_excl_scan(c, s_red, &total);
    for (uint32_t q = q0; q < q1; ++q)
      if (A.minrep[L[q]] == q) A.newlab[q] = base++;
    __syncthreads();
    for (uint32_t q = tid; q < n; q += bd)
      if (A.minrep[L[q]] == q) A.minrep[L[q]] = 0x80000000u | A.newlab[q];
    __syncthreads();
    for (uint32_t q = tid; q < n; q += bd) A.out[q] = A.minrep[L[q]] & 0x7FFFFFFFu;
    blocks = total;
  }
  return SmallOut{0u, r, changed, blocks, maxed, 0xFFFFFFFFu};
}

__global__ void __launch_bounds__(kSmallThreads, 1) moore_small_kernel(const __grid_constant__ SmallArgs A) {
  extern __shared__ __align__(16) uint32_t sm[];
  Ctrl *C = A.ctrl;
  const unsigned long long t0 = gtimer();
  if (threadIdx.x == 0) C->t_start = t0;
  const SmallOut o = small_refine(A, sm, C, t0);
  if (threadIdx.x == 0) {
    if (o.err) {
      C->err = o.err;
    } else {
      C->rounds_executed = o.rounds_executed;
      C->rounds_changed = o.rounds_changed;
      C->num_blocks = o.num_blocks;
      C->maxed = o.maxed;
    }
    C->sep_round = o.sep_round;
    C->t_end = gtimer();
  }
}

// Batches: the DFAs of items[0, count) refined one per block, each block
// taking the next DFA from *next (items sorted by decreasing size, so that the
// largest start first); each block writes its DFA's partition and round counts
// and adds its errors and its end time to the batch's control block.
struct BatchSmallArgs {
  const BatchSmallItem *items;
  uint32_t count;
  uint32_t *next;            // zeroed before the launch
  Ctrl *ctrl;
  BatchSmallWords words;     // where the results go in a DFA's bookkeeping row
  uint32_t max_rounds, stop_discrete;
  unsigned long long timeout_ns;
};

__global__ void __launch_bounds__(kSmallThreads, 1) batch_small_kernel(const __grid_constant__ BatchSmallArgs B) {
  extern __shared__ __align__(16) uint32_t sm[];
  __shared__ uint32_t s_i;
  if (threadIdx.x == 0) atomicCAS(&B.ctrl->t_start, 0ull, gtimer());   // when no cooperative launch set it
  for (;;) {
    if (threadIdx.x == 0) s_i = atomicAdd(B.next, 1u);
    __syncthreads();
    const uint32_t i = s_i;
    __syncthreads();   // every thread has read s_i before the next DFA's refinement reuses the block
    if (i >= B.count) break;
    const BatchSmallItem &it = B.items[i];
    SmallOut o;
    if ((it.plan >> 10) & 1u) {   // labels in shared memory, table in global memory
      MediumArgs m{};
      m.delta = it.delta;
      m.accept = it.accept;
      m.n = it.n;
      m.k = it.k;
      m.out = it.out;
      m.table = it.table;
      m.log2T = it.plan & 0xFFu;
      m.newlab = it.scratch0;
      m.minrep = it.scratch1;
      m.max_rounds = B.max_rounds;
      m.stop_discrete = B.stop_discrete;
      m.timeout_ns = B.timeout_ns;
      o = medium_refine(m, reinterpret_cast<uint16_t *>(sm), gtimer());
    } else {                      // everything in shared memory
      SmallArgs a{};
      a.delta = it.delta;
      a.accept = it.accept;
      a.n = it.n;
      a.k = it.k;
      a.out = it.out;
      a.ctrl = nullptr;
      a.log2T = it.plan & 0xFFu;
      a.wide_table = (it.plan >> 8) & 1u;
      a.staged = (it.plan >> 9) & 1u;
      a.max_rounds = B.max_rounds;
      a.stop_discrete = B.stop_discrete;
      a.timeout_ns = B.timeout_ns;
      o = small_refine(a, sm, nullptr, gtimer());
    }
    if (threadIdx.x == 0) {
      if (o.err) atomicOr(&B.ctrl->err, o.err);
      it.ss[B.words.b] = o.num_blocks;
      it.ss[B.words.changed] = o.rounds_changed;
      it.ss[B.words.executed] = o.rounds_executed;
      it.ss[B.words.maxed] = o.maxed;
    }
    __syncthreads();   // the refinement's last reads of shared memory are done
  }
  if (threadIdx.x == 0) atomicMax(&B.ctrl->t_end, gtimer());
}

// Shared memory of the kernel for n states and k letters (smem 0: no fit).
struct SmallPlan {
  uint32_t log2T, wide, staged;
  size_t smem;
};

static SmallPlan small_plan(uint32_t n, uint32_t k) {
  SmallPlan p{};
  p.log2T = ceil_log2(n + n / 2 < 64 ? 64 : n + n / 2);
  const size_t T = (size_t)1 << p.log2T;
  const size_t labels = 2 * (size_t)((n + 7u) & ~7u) * 2;
  p.wide = (uint64_t)(k + 1) * p.log2T <= 63 ? 1u : 0u;
  size_t table = T * (p.wide ? 8 : 4);   // also the direct rounds' flags (2^log2T words at most)
  if (table + labels > kSmallSmem && p.wide) {   // 64-bit slots do not fit: representatives
    p.wide = 0;
    table = T * 4;
  }
  p.smem = table + labels;
  if (p.smem > kSmallSmem) {
    p.smem = 0;
    return p;
  }
  if (p.smem + (size_t)k * n * 2 <= kSmallSmem) {
    p.staged = 1;
    p.smem += (size_t)k * n * 2;
  }
  return p;
}

// Which small kernel refines a DFA, if any.  Up to kSmallMaxStates states: the
// single block where it fits and measured faster than the cooperative kernel
// (packed keys fit 64-bit slots, or at most 4,096 states whatever the
// letters); the cluster kernel from kClusterMinStates states on, or where the
// single block does not fit, when the device can place its cluster.  The
// cluster's barrier and distributed-shared-memory traffic cost more than they
// save below about 6,000 states (4,096 states, 2 letters: 21 against 20 us;
// 10,000 states: 27 against 42 us).  DFA_FLAG_ONE_BLOCK and DFA_FLAG_CLUSTER
// force one of the two where it fits.  An explicit `schedule` (a width of the
// cooperative kernel), the table-only and bucketed flags keep the cooperative
// kernel.
enum SmallKernel { SK_NONE = 0, SK_ONE_BLOCK, SK_CLUSTER };
static constexpr uint32_t kClusterMinStates = 6144;

static SmallKernel pick_small(uint32_t n, uint32_t k, const dfa_opts &o) {
  if (o.algo != DFA_ALGO_MOORE) return SK_NONE;
  if (o.schedule >= 1) return SK_NONE;
  if (o.flags & (DFA_FLAG_BUCKETED | DFA_FLAG_TABLE_ONLY)) return SK_NONE;
  if (n < 1 || n > kSmallMaxStates) return SK_NONE;
  const SmallPlan p = small_plan(n, k);
  const bool one = p.smem != 0 && (p.wide || n <= 4096);
  if (o.flags & DFA_FLAG_ONE_BLOCK) return one ? SK_ONE_BLOCK : SK_NONE;
  const bool cl = cluster_fits(n, k);
  if (o.flags & DFA_FLAG_CLUSTER) return cl ? SK_CLUSTER : SK_NONE;
  if (one && n < kClusterMinStates) return SK_ONE_BLOCK;
  if (cl) return SK_CLUSTER;
  return one ? SK_ONE_BLOCK : SK_NONE;
}

bool small_fits(uint32_t n, uint32_t k, const dfa_opts &o) { return pick_small(n, k, o) != SK_NONE; }

int enqueue_small(const uint32_t *delta, const uint8_t *accept, uint32_t n, uint32_t k, uint32_t *out, Ctrl *ctrl,
                  const dfa_opts &o, cudaStream_t st, const PairTrack *track) {
  const SmallKernel which = pick_small(n, k, o);
  if (which == SK_CLUSTER) return enqueue_cluster(delta, accept, n, k, out, ctrl, o, st, track);
  const SmallPlan p = small_plan(n, k);
  if (p.smem == 0) return fail(DFA_EINVAL, "the single-block kernel does not fit %u states", n);
  SmallArgs a{};
  a.delta = delta;
  a.accept = accept;
  a.n = n;
  a.k = k;
  a.out = out;
  a.ctrl = ctrl;
  a.log2T = p.log2T;
  a.wide_table = p.wide;
  a.staged = p.staged;
  a.max_rounds = o.max_rounds;
  a.stop_discrete = (o.flags & DFA_FLAG_STOP_DISCRETE) ? 1u : 0u;
  a.timeout_ns = o.timeout_ns;
  if (track) {
    a.track = 1u;
    a.sa = track->a;
    a.sb = track->b;
    a.early_exit = track->early_exit;
  }
  cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(ctrl)");
  e = cudaFuncSetAttribute(moore_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
  if (e != cudaSuccess) return cuda_fail(e, "shared memory of the single-block kernel");
  moore_small_kernel<<<1, kSmallThreads, p.smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "launch of the single-block kernel");
  return DFA_OK;
}

bool medium_block_plan(uint32_t n, uint32_t log2S, uint32_t *plan, size_t *smem) {
  if (n < 1 || n > 65536u) return false;
  const uint32_t log2T = log2S + 1;   // slots at a load of at most 1/4, within the DFA's table region
  *plan = log2T | (1u << 10);
  *smem = (size_t)((n + 7u) & ~7u) * 2;
  return true;
}

bool small_block_plan(uint32_t n, uint32_t k, uint32_t *plan, size_t *smem) {
  if (n < 1 || n > kSmallMaxStates) return false;
  const SmallPlan p = small_plan(n, k);
  if (p.smem == 0) return false;
  *plan = p.log2T | (p.wide << 8) | (p.staged << 9);
  *smem = p.smem;
  return true;
}

cudaError_t enqueue_batch_small(const BatchSmallItem *items, uint32_t count, uint32_t *next, Ctrl *ctrl, size_t smem,
                                BatchSmallWords words, const dfa_opts &o, uint32_t grid, cudaStream_t st) {
  BatchSmallArgs b{};
  b.items = items;
  b.count = count;
  b.next = next;
  b.ctrl = ctrl;
  b.words = words;
  b.max_rounds = o.max_rounds;
  b.stop_discrete = (o.flags & DFA_FLAG_STOP_DISCRETE) ? 1u : 0u;
  b.timeout_ns = o.timeout_ns;
  batch_small_kernel<<<grid, kSmallThreads, smem, st>>>(b);
  return cudaGetLastError();
}

cudaError_t batch_small_setup() {
  return cudaFuncSetAttribute(batch_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmem);
}

}  // namespace dfa
