// Signature refinement of a small DFA on one thread-block cluster.
//
// Algorithm 4 (Section 3.3) for n <= kSmallMaxStates states, spread over the C
// thread blocks (CTAs) of one cluster (C = 16 where the GPU can place such a
// cluster, else 8) instead of the one SM that the single-block kernel
// (small.cu) issues from.  Per CTA, in shared memory:
//  * both label arrays of all n states (16-bit; every CTA holds a full copy);
//  * the transitions as 16-bit targets: only the rows of the CTA's own slice
//    when no round can compare representatives (packed keys of at most 63
//    bits), else all k n of them when they fit;
//  * its share of the renumbering table: the table has T = 2^log2T > n slots
//    of 64 bits, and CTA c owns slots [c T/C, (c+1) T/C).  Two tables alternate
//    by round parity, so that a CTA clears the one of the next round while the
//    others may still insert into the current one.
// CTA c refines the states of its own slice [c P, (c+1) P) (P a multiple of 8):
// it builds each state's signature from its local label copy, inserts it into
// the owner CTA's slot with a compare-and-swap on distributed shared memory,
// and writes the new label into its own slice.  Then it stores its slice of
// the new labels (16-byte stores) and one word holding its count of new blocks
// and its error bits into every other CTA's shared memory, and one cluster
// barrier ends the round: after it every CTA holds all new labels and all
// words, and nothing is read across CTAs.  Rounds renumber exactly, in one of
// three ways chosen alike by every CTA from the label width w:
//  * direct  (k+1) w <= log2 T: the packed signature is the new label and
//            its own slot (no probing); a slot set for the first time counts a
//            block;
//  * packed  (k+1) w <= 63: the packed signature is the key, probed linearly
//            from its hash across the whole distributed table; the slot is the
//            label;
//  * compare otherwise: a slot holds a representative state, and a state
//            joins it only if its own label and every successor's label equal
//            the representative's; the slot is the label.
// Every decision that ends the loop is taken from the same words, read after
// the same cluster barrier, so every CTA passes the same barriers.  The canonical
// numbering (blocks in order of their smallest state) needs all final labels,
// which every CTA holds after the last exchange: each CTA computes it for all
// n states and writes the numbers of its own slice, with no further exchange.
#include <cooperative_groups.h>

#include <mutex>

#include "api_util.h"

namespace cg = cooperative_groups;

namespace dfa {

static constexpr int kClusterThreads = 1024;
static constexpr size_t kClusterSmem = 220 * 1024;   // dynamic shared memory a CTA may take
static constexpr uint32_t kClusterMaxLog2T = 15;     // labels and slots stay below 2^15
static constexpr unsigned long long kUsed = 1ull << 63;   // set in every key: 0 marks a free slot

struct ClusterArgs {
  const uint32_t *delta;   // k*n, letter-major
  const uint8_t *accept;   // n
  uint32_t n, k;
  uint32_t *out;           // n: canonical block numbers
  Ctrl *ctrl;
  uint32_t log2T;          // table slots (all CTAs) 2^log2T > n; labels stay below 2^log2T
  uint32_t log2C;          // CTAs in the cluster: 2^log2C
  uint32_t per;            // states per CTA slice (a multiple of 8)
  uint32_t staged;         // 16-bit targets in shared memory: 0 none (global reads), 1 all of δ in every
                           // CTA, 2 the rows of the CTA's own slice only (k x per; possible whenever
                           // no round compares representatives, which need any state's successors)
  uint32_t max_rounds;     // 0 = none
  uint32_t stop_discrete;  // 1: stop after a round that leaves n blocks
  unsigned long long timeout_ns;
  uint32_t track;          // equivalence by union: record the first round after which sa and sb are apart
  uint32_t sa, sb;
  uint32_t early_exit;     // with track: stop there (round 0: no round at all)
};

// Shared memory of one CTA (bytes), for the layout the kernel uses:
// two label arrays of C*per halfwords, then a region holding the two table
// shares and the staged δ during the rounds, and the numbering table of T
// words after them.
__host__ __device__ inline size_t cluster_label_bytes(uint32_t per, uint32_t log2C) {
  return (size_t)per << log2C << 2;   // two arrays of C*per halfwords
}
__host__ __device__ inline size_t cluster_region_bytes(uint32_t n, uint32_t k, uint32_t log2T, uint32_t log2C,
                                                       uint32_t staged, uint32_t per) {
  const size_t shares = 2 * (((size_t)1 << log2T) >> log2C) * 8;
  const size_t rounds = shares + (staged == 1 ? (size_t)k * n * 2 : staged == 2 ? (size_t)k * per * 2 : 0);
  const size_t numbering = ((size_t)1 << log2T) * 4;
  return rounds > numbering ? rounds : numbering;
}

__device__ __forceinline__ unsigned long long cluster_mix(unsigned long long h, uint32_t v) {
  h = (h ^ v) * 0x9E3779B97F4A7C15ull;
  return h ^ (h >> 29);
}

__global__ void __launch_bounds__(kClusterThreads, 1) moore_cluster_kernel(const __grid_constant__ ClusterArgs A) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) uint16_t csm[];
  __shared__ uint32_t s_red[32];
  __shared__ uint32_t s_made[2];       // blocks this CTA created, by round parity
  __shared__ uint32_t s_word[2][16];   // round parity x CTA: blocks it created | its ERR_* bits << 24,
                                       // written into every CTA by the CTA that made them
  __shared__ uint32_t s_stop;          // CTA 0: the call's time limit ran out
  __shared__ uint32_t s_bad;           // this CTA saw an invalid target
  const uint32_t n = A.n, k = A.k, tid = threadIdx.x, bd = blockDim.x, lane = tid & 31u;
  const uint32_t me = cl.block_rank();
  const uint32_t T = 1u << A.log2T, log2S = A.log2T - A.log2C, S = 1u << log2S;   // S: slots per CTA
  const uint32_t np = A.per << A.log2C;                                           // label array length
  uint16_t *const lab0 = csm, *const lab1 = csm + np;
  unsigned long long *const share0 = reinterpret_cast<unsigned long long *>(csm + 2 * np), *const share1 = share0 + S;
  uint16_t *d16 = reinterpret_cast<uint16_t *>(share1 + S);   // k n (staged 1) or k per (staged 2) halfwords
  uint32_t *numtab = reinterpret_cast<uint32_t *>(csm + 2 * np);  // numbering: over the shares and δ
  Ctrl *Cc = A.ctrl;
  const unsigned long long t0 = gtimer();
  if (me == 0 && tid == 0) Cc->t_start = t0;
  if (tid == 0) {
    s_bad = 0u;
    s_stop = 0u;
    s_made[0] = s_made[1] = 0u;
  }
  __syncthreads();
  // every CTA: the initial partition {F, Q \ F} of all states (labels 0/1), δ, both table shares clear
  // (16-byte loads where the arrays allow, several in flight per thread: the
  // staging is latency-bound otherwise)
  uint32_t seen = 0, bad = 0;
  stage_accept(A.accept, n, lab0, &seen);
  const uint32_t q0 = me * A.per, q1 = q0 + A.per < n ? q0 + A.per : n;   // this CTA's slice
  if (A.staged == 1) {
    stage_delta(A.delta, (size_t)k * n, n, d16, &bad);
  } else if (A.staged == 2 && q0 < q1) {   // k rows of the slice, one batch of loads for all of them
    const uint32_t len = q1 - q0, tot = k * A.per;
    for (uint32_t base = 0; base < tot; base += 4u * bd) {
      uint32_t v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t i = base + j * bd + tid, a = i / A.per, x = i - a * A.per;
        v[j] = i < tot && x < len ? A.delta[(size_t)a * n + q0 + x] : 0u;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t i = base + j * bd + tid;
        if (i < tot) {
          bad |= v[j] >= n;
          d16[i] = (uint16_t)(v[j] < n ? v[j] : 0u);
        }
      }
    }
  }
  for (uint32_t i = tid; i < 2u * S; i += bd) share0[i] = 0ull;   // share1 follows share0
  if (bad) atomicOr(&s_bad, ERR_BAD_DELTA);
  const uint32_t classes = block_sum(((seen & 1u) ? 1u : 0u) | ((seen & 2u) ? 0x10000u : 0u), s_red);
  const uint32_t any_acc = (classes & 0xFFFFu) != 0u, any_rej = (classes >> 16) != 0u;
  __syncthreads();
  // with all of δ staged every CTA saw every target, so s_bad is the same
  // everywhere; otherwise it joins the first round's words (read alike by all)
  uint32_t err = A.staged == 1 ? s_bad : 0u;
  cl.sync();   // table shares clear before any remote insert
  uint32_t nt = 0;   // trace entries (CTA 0, thread 0)
  if (me == 0 && tid == 0) trace_put(Cc, nt, t0, kTraceStart);
  uint32_t B_prev = any_acc + any_rej, B_r = B_prev;
  uint32_t r = 0, changed = 0, cur = 0, maxed = 0, w = 1, sep = 0xFFFFFFFFu;
  bool skip = false;
  if (A.track && (A.accept[A.sa] != 0) != (A.accept[A.sb] != 0)) {   // the empty word separates them
    sep = 0;
    skip = A.early_exit != 0;   // the answer needs no round: the initial partition is reported
  }
  // δ(q, a): the shared copy, or global memory (an invalid target reads as 0 and is reported)
  auto target = [&](uint32_t a, uint32_t q) -> uint32_t {
    if (A.staged == 1) return d16[(size_t)a * n + q];
    if (A.staged == 2) return d16[(size_t)a * A.per + (q - q0)];   // q in this CTA's slice
    uint32_t d = A.delta[(size_t)a * n + q];
    if (d >= n) {
      bad = 1u;
      d = 0u;
    }
    return d;
  };
  // the owner's copy of global slot g of the current table
  auto slot_ptr = [&](unsigned long long *tab, uint32_t g) -> unsigned long long * {
    return cl.map_shared_rank(tab, g >> log2S) + (g & (S - 1u));
  };
  for (r = 1; !err && !skip; ++r) {
    const uint16_t *src = cur ? lab1 : lab0;
    uint16_t *dst = cur ? lab0 : lab1;
    const uint32_t K = (k + 1u) * w;
    const uint32_t mode = K <= A.log2T ? 0u : K <= 63u ? 1u : 2u;
    unsigned long long *tab = (r & 1u) ? share1 : share0;
    uint32_t created = 0;
    bad = 0;
    for (uint32_t base = q0; base < q1; base += bd) {   // the same trip count for every thread
      const uint32_t q = base + tid;
      const bool valid = q < q1;
      const uint32_t qq = valid ? q : q0;
      uint32_t label = 0;
      if (mode != 2u) {
        unsigned long long key = src[qq];
        uint32_t shift = w;
        for (uint32_t a = 0; a < k; ++a) {
          key |= (unsigned long long)src[target(a, qq)] << shift;
          shift += w;
        }
        key |= kUsed;
        // one lane per distinct key of the warp inserts it; the others take its slot
        const unsigned grp = __match_any_sync(0xFFFFFFFFu, valid ? key : 0ull);
        const uint32_t lead = __ffs(grp) - 1;
        uint32_t slot = 0;
        if (valid && lane == lead) {
          if (mode == 0u) {   // direct: the signature is the label, with a slot of its own
            slot = (uint32_t)key & (T - 1u);
            // signatures are small numbers: their low bits pick the CTA, so that
            // the slots of a round spread over the whole cluster
            const uint32_t g = ((slot & ((1u << A.log2C) - 1u)) << log2S) | (slot >> A.log2C);
            unsigned long long *p = slot_ptr(tab, g);
            if (*reinterpret_cast<volatile unsigned long long *>(p) == 0ull && atomicCAS(p, 0ull, key) == 0ull)
              ++created;
          } else {            // packed: linear probing from the key's hash
            slot = (uint32_t)((key * 0xD6E8FEB86659FD93ull) >> (64u - A.log2T));
            for (uint32_t probe = 0; probe < T; ++probe) {
              const unsigned long long v = atomicCAS(slot_ptr(tab, slot), 0ull, key);
              if (v == 0ull) {   // a new block
                ++created;
                break;
              }
              if (v == key) break;   // joins that block
              slot = (slot + 1u) & (T - 1u);
            }
          }
        }
        label = __shfl_sync(0xFFFFFFFFu, slot, lead);
      } else if (valid) {   // compare: a representative per slot, joined on a full comparison
        unsigned long long h = cluster_mix(0x243F6A8885A308D3ull, src[q]);
        for (uint32_t a = 0; a < k; ++a) h = cluster_mix(h, src[target(a, q)]);
        h ^= h >> 31;
        h *= 0xD6E8FEB86659FD93ull;
        uint32_t slot = (uint32_t)(h >> (64u - A.log2T));
        for (uint32_t probe = 0; probe < T; ++probe) {
          const unsigned long long v = atomicCAS(slot_ptr(tab, slot), 0ull, kUsed | (unsigned long long)(q + 1u));
          if (v == 0ull) {   // q represents a new block
            ++created;
            break;
          }
          const uint32_t rep = (uint32_t)v - 1u;
          bool same = src[q] == src[rep];
          for (uint32_t a = 0; same && a < k; ++a) same = src[target(a, q)] == src[target(a, rep)];
          if (same) break;
          slot = (slot + 1u) & (T - 1u);
        }
        label = slot;
      }
      if (valid) dst[q] = (uint16_t)label;
    }
    if (tid == 0 && me == 0 && (r & 15u) == 0u && gtimer() - t0 > A.timeout_ns) s_stop = 1u;
    if (bad) atomicOr(&s_bad, ERR_BAD_DELTA);
    {
      const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, created);
      if (lane == 0 && wsum) atomicAdd(&s_made[r & 1u], wsum);
      if (tid == 0) s_made[(r + 1u) & 1u] = 0u;   // read last round, before its cluster barrier
    }
    __syncthreads();   // this CTA's new labels, count and error bits are complete
    const uint32_t made = s_made[r & 1u];
    // this CTA's count and error bits, and its slice of the new labels, into every CTA
    const uint32_t C = 1u << A.log2C;
    if (tid < C)
      *cl.map_shared_rank(&s_word[r & 1u][me], tid) = made | ((s_bad | (s_stop ? ERR_TIMEOUT : 0u)) << 24);
    const uint32_t cper = A.per >> 3;   // 16-byte chunks of a slice
    const uint4 *mine = reinterpret_cast<const uint4 *>(dst) + me * cper;
    for (uint32_t i = tid; i < cper * (C - 1u); i += bd) {
      const uint32_t j = i / cper, c = j + (j >= me ? 1u : 0u), off = i - j * cper;
      reinterpret_cast<uint4 *>(cl.map_shared_rank(dst, c))[me * cper + off] = mine[off];
    }
    // the next round's table share starts clean (its inserts ended a round ago);
    // cleared before this CTA arrives at the barrier, since other CTAs insert
    // into it as soon as every thread has arrived
    unsigned long long *next = (r & 1u) ? share0 : share1;
    for (uint32_t i = tid; i < S; i += bd) next[i] = 0ull;
    cl.sync();   // every CTA's inserts, labels and words of the round are in place
    if (me == 0 && tid == 0) trace_put(Cc, nt, t0, kTraceRound | (mode << 4));
    B_r = 0;
    err = 0;
    for (uint32_t c = 0; c < C; ++c) {
      const uint32_t v = s_word[r & 1u][c];
      B_r += v & 0xFFFFFFu;
      err |= v >> 24;
    }
    cur ^= 1u;
    w = mode == 0u ? K : A.log2T;   // direct rounds: labels are signatures; else slots
    if (err) break;
    const bool grew = B_r != B_prev;
    if (grew) ++changed;
    if (A.track && sep == 0xFFFFFFFFu) {   // every CTA holds all new labels now: a uniform decision
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
    B_prev = B_r;
  }
  if (skip) r = 0;
  if (me == 0 && tid == 0) Cc->sep_round = sep;
  if (err) {
    if (me == 0 && tid == 0) {
      Cc->err = err;
      Cc->t_end = gtimer();
    }
    return;   // nothing crosses CTAs after the last cluster barrier
  }
  // canonical numbering of all n states in every CTA (every label is below T);
  // each CTA writes the numbers of its own slice
  const uint16_t *fin = cur ? lab1 : lab0;
  uint32_t blocks = B_r;
  if (B_r == n) {
    for (uint32_t q = q0 + tid; q < q1; q += bd) A.out[q] = q;
  } else {
    uint16_t *rank = cur ? lab0 : lab1;   // free now: rank of each block's smallest state
    for (uint32_t i = tid; i < T; i += bd) numtab[i] = 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t q = tid; q < n; q += bd) atomicMin(&numtab[fin[q]], q);
    __syncthreads();
    const uint32_t pt = (n + bd - 1) / bd;
    const uint32_t a0 = tid * pt < n ? tid * pt : n, a1 = a0 + pt < n ? a0 + pt : n;
    uint32_t c = 0;
    for (uint32_t q = a0; q < a1; ++q) c += numtab[fin[q]] == q;
    uint32_t total;
    uint32_t base = block_excl_scan(c, s_red, &total);
    for (uint32_t q = a0; q < a1; ++q)
      if (numtab[fin[q]] == q) rank[q] = (uint16_t)base++;
    __syncthreads();
    for (uint32_t q = tid; q < n; q += bd)
      if (numtab[fin[q]] == q) numtab[fin[q]] = 0x80000000u | rank[q];
    __syncthreads();
    for (uint32_t q = q0 + tid; q < q1; q += bd) A.out[q] = numtab[fin[q]] & 0x7FFFFFFFu;
    blocks = total;
  }
  if (me == 0 && tid == 0) {
    trace_put(Cc, nt, t0, kTraceEnd);
    Cc->rounds_executed = r;
    Cc->rounds_changed = changed;
    Cc->num_blocks = blocks;
    Cc->maxed = maxed;
    Cc->t_end = gtimer();
  }
  // nothing crosses CTAs after the last cluster barrier, so a CTA may leave
}

// ---------------------------------------------------------------- host side

struct ClusterPlan {
  uint32_t log2T, log2C, per, staged;
  size_t smem;
};

static bool cluster_plan(uint32_t n, uint32_t k, uint32_t log2C, ClusterPlan *p) {
  if (n < 1 || n > kSmallMaxStates) return false;
  const uint64_t want = (uint64_t)n * 3 < 64 ? 64 : (uint64_t)n * 3;   // load factor at most 1/3 where it fits
  p->log2T = ceil_log2(want) < kClusterMaxLog2T ? ceil_log2(want) : kClusterMaxLog2T;
  if (((uint64_t)1 << p->log2T) <= n || p->log2T < log2C) return false;
  p->log2C = log2C;
  const uint32_t C = 1u << log2C;
  p->per = ((n + C - 1) / C + 7) / 8 * 8;
  const size_t labels = cluster_label_bytes(p->per, log2C);
  // a round compares representatives when its packed keys exceed 63 bits:
  // then any state's successors are needed, else only the slice's own
  const bool compare = (uint64_t)(k + 1) * p->log2T > 63;
  for (uint32_t staged : {compare ? 1u : 2u, 0u}) {
    p->staged = staged;
    p->smem = labels + cluster_region_bytes(n, k, p->log2T, log2C, staged, p->per);
    if (p->smem <= kClusterSmem) return true;
  }
  return false;
}

// log2 of the cluster size this device runs (4: 16 CTAs, 3: 8), 0 when it
// cannot place a cluster of the kernel at its largest shared memory; looked
// up once per device.
static uint32_t cluster_log2_size() {
  static std::mutex mu;
  static int known[64];       // 0 = not looked up, else 1 + log2 size
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 0;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (known[dev]) return (uint32_t)(known[dev] - 1);
  uint32_t best = 0;
  if (cudaFuncSetAttribute(moore_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kClusterSmem) ==
          cudaSuccess &&
      cudaFuncSetAttribute(moore_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
    for (uint32_t l2 : {4u, 3u}) {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3(1u << l2);
      cfg.blockDim = dim3(kClusterThreads);
      cfg.dynamicSmemBytes = kClusterSmem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 1u << l2;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int clusters = 0;
      if (cudaOccupancyMaxActiveClusters(&clusters, moore_cluster_kernel, &cfg) == cudaSuccess && clusters >= 1) {
        best = l2;
        break;
      }
      cudaGetLastError();
    }
  }
  cudaGetLastError();
  known[dev] = (int)best + 1;
  return best;
}

bool cluster_fits(uint32_t n, uint32_t k) {
  const uint32_t l2 = cluster_log2_size();
  ClusterPlan p;
  return l2 != 0 && cluster_plan(n, k, l2, &p);
}

int enqueue_cluster(const uint32_t *delta, const uint8_t *accept, uint32_t n, uint32_t k, uint32_t *out, Ctrl *ctrl,
                    const dfa_opts &o, cudaStream_t st, const PairTrack *track) {
  const uint32_t l2 = cluster_log2_size();
  ClusterPlan p;
  if (l2 == 0 || !cluster_plan(n, k, l2, &p)) return fail(DFA_EINVAL, "the cluster kernel does not fit %u states", n);
  ClusterArgs a{};
  a.delta = delta;
  a.accept = accept;
  a.n = n;
  a.k = k;
  a.out = out;
  a.ctrl = ctrl;
  a.log2T = p.log2T;
  a.log2C = p.log2C;
  a.per = p.per;
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
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(1u << p.log2C);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1u << p.log2C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, moore_cluster_kernel, a);
  if (e != cudaSuccess) return cuda_fail(e, "launch of the cluster kernel");
  return DFA_OK;
}

}  // namespace dfa
