// Batched signature refinement: many independent DFAs in one persistent,
// segment-offset launch (a batching form the paper does not have; each DFA is
// refined exactly as dfa_minimise refines it alone, Section 3.3 / Algorithm 4).
//
// Layout.  All DFAs share one state space: DFA i owns states
// [state_off_i, state_off_i + n_i) of the label arrays and its own region of
// 2^ceil(log2(2 n_i)) slots of the renumbering table, so keys of different DFAs
// never meet and labels stay narrow (a DFA with 65,536 states packs 17-bit
// components).  Work is cut into tiles of at most `tile` states (64, 128 or
// 256, part of the schedule) that never cross a DFA boundary (listed on the
// device at the start of the launch from each DFA's first tile number); warps
// take tiles grid-stride and skip the tiles of DFAs that have already
// converged.
//
// Rounds.  Every pass packs each active state's signature into a key of its
// own DFA's width and inserts it into its DFA's table region; a new slot counts
// one new block for that DFA.  After the pass a grid-wide bookkeeping step
// compares each active DFA's count with its previous one: equal counts mean
// the DFA has reached its fixpoint, and it drops out with its round counts.
// The launch ends when no DFA is active; then the final labels are gathered,
// numbered canonically across the batch and rebased per DFA.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "api_util.h"

namespace dfa {

static constexpr int kBatchThreads = 512;
static constexpr size_t kMaxGridB = 8192;

// Schedules of the batch kernel, chosen per call (opts.schedule) or by the
// autotuner: states per lane within a tile pass (1, two blocks of 512 threads
// per SM; or 2, one block per SM with room for twice the keys), states per
// tile (256, 128 or 64: smaller tiles balance the passes between grid barriers
// better and cost more per-tile bookkeeping), and whether every DFA that fits
// one thread block's shared memory is refined alone by one block instead
// (after the cooperative launch, which then refines only the others; a block
// per DFA needs no grid barrier at all).  Schedule s (0..11) takes
// 1 + (s & 1) states per lane, 256 >> ((s >> 1) % 3) states per tile, and
// blocks per DFA from s = 6 on.
static constexpr int kBatchSchedules = 12;
struct BatchSchedule {
  uint32_t vec, tile;
  bool blocks;
};
static inline BatchSchedule batch_schedule(int s) {
  return BatchSchedule{1u + (uint32_t)(s & 1), 256u >> ((s >> 1) % 3), s >= 6};
}

struct SegInfo {
  const uint32_t *delta;   // device
  const uint8_t *accept;   // device
  uint32_t n, k;
  uint32_t state_off;      // first state in the batch's state space
  uint32_t log2S;          // table region of 2^log2S slots
  uint32_t wid;            // bits of a local state number (labels of filter rounds)
  uint64_t table_off;      // first slot of the region
  uint32_t small;          // 1: refined alone by one thread block after this kernel (skipped here)
  uint32_t pad_;
};

struct Tile {
  uint32_t seg, start, len;   // local states [start, start+len) of DFA seg
};

// Per-DFA bookkeeping words.
enum : uint32_t {
  SS_ACTIVE = 0, SS_PREV, SS_CHANGED, SS_EXECUTED, SS_FINAL, SS_B, SS_SEEN, SS_MAXED,
  SS_W,      // bits of the current labels
  SS_FOK,    // filter rounds allowed (cleared once one lists most of the DFA's states)
  SS_NDUP,   // states listed by the current filter round
  SS_WORDS
};

struct BatchArgs {
  const SegInfo *segs;
  uint32_t nsegs;
  const uint32_t *tile_off; // nsegs + 1: first tile of each DFA, then the tile count
  Tile *tiles;             // ntiles, filled by the kernel
  uint32_t ntiles;
  uint32_t total_states;
  uint64_t total_slots;
  uint32_t *lab[2];        // labels, local to each DFA (< 2^log2S)
  uint32_t *tmp;           // total_states (multi-stage plans)
  u128 *table;
  uint32_t *bm[2];         // direct rounds: one bit per table slot (ping-pong)
  uint32_t *seen1, *seen2; // filter rounds: 2-bit counters over 2^mbits buckets (all DFAs)
  uint32_t *seen3, *seen4; // second filter, 2^(mbits-1) buckets
  uint32_t *tmp2;          // total_states: second-filter bucket
  uint32_t mbits;
  unsigned long long *rep; // total_slots: filter rounds' (round, ~smallest local state) per slot
  uint32_t *dups, *dups2, *dups3;   // per-warp lists: global state, second bucket, DFA
  uint32_t *wcnt;          // per-warp list lengths
  uint32_t dup_cap;        // list capacity per block
  uint32_t *minrep;        // total_slots: smallest member per label (canonical numbering)
  uint32_t *tile_cnt;      // ntiles: first members per tile (canonical numbering)
  uint32_t *tile_pre;      // ntiles: their exclusive prefix sums
  uint32_t *partials;
  uint32_t *out;           // total_states
  uint32_t *cnt;           // nsegs x 3
  uint32_t *ss;            // nsegs x SS_WORDS
  Ctrl *ctrl;
  uint32_t ebits, max_stages, max_rounds;
  uint32_t stop_discrete;  // 1: a DFA whose round leaves n blocks stops (no confirming round)
  uint32_t vec;            // states per lane within a tile pass: 1 or 2
  uint32_t tile;           // states per tile: 64, 128 or 256
  unsigned long long timeout_ns, barrier_ns;
};

// Tiles of a pass are dealt per block: block b takes tiles b, b + grid, b +
// 2 grid, ... in order (so that the grid sweeps the batch front to back, with
// the tables of neighbouring DFAs in L2 together) and its warps take the next
// of them from a shared counter, so that costly tiles do not hold up a warp
// while its neighbours idle.  The counter is reset (start_tiles) after a
// barrier, before every pass.
__device__ __forceinline__ uint32_t next_tile(const BatchArgs &A, uint32_t *s_next) {
  uint32_t i = 0;
  if ((threadIdx.x & 31u) == 0) i = atomicAdd(s_next, 1u);
  i = __shfl_sync(0xFFFFFFFFu, i, 0);
  const uint64_t t = (uint64_t)blockIdx.x + (uint64_t)i * gridDim.x;
  return t < A.ntiles ? (uint32_t)t : A.ntiles;
}

__device__ __forceinline__ void start_tiles(uint32_t *s_next) {
  if (threadIdx.x == 0) *s_next = 0u;
  __syncthreads();
}

enum : uint32_t { BM_DIRECT = 0, BM_FILTER = 1, BM_TABLE = 2 };

// Mode of a DFA's round r (w = its words in the bookkeeping array, as they
// stand before the round): direct when the packed signature fits in log2S
// bits; filter when most signatures are likely unique: the previous round left
// at least n/64 blocks (most blocks small), or its B blocks allow B^(k+1) >= 64 n
// combinations (many letters: a signature then rarely repeats even while the
// blocks are large); otherwise table.  Filter rounds are exact either way; a
// filter round that lists most states hands the DFA's later rounds to the table.
__device__ __forceinline__ uint32_t batch_mode(const SegInfo &S, const uint32_t *w, uint32_t r) {
  const uint32_t wd = w[SS_W];
  if ((uint64_t)(S.k + 1) * wd <= S.log2S) return BM_DIRECT;
  if (r > 1 && w[SS_FOK]) {
    const uint32_t prev = w[SS_PREV];
    if ((uint64_t)prev * 64 >= S.n || signatures_sparse(S.k, prev, S.n)) return BM_FILTER;
  }
  return BM_TABLE;
}

// Filter round, pass A over one tile: hash every signature (the DFA's number
// mixed in, so that equal local signatures of different DFAs spread apart)
// into the 2-bit counters; keep the two buckets per state.
__device__ __forceinline__ void batch_filter_a(const BatchArgs &A, const SegInfo &S, const Tile &T,
                                              const uint32_t *__restrict__ src) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = S.n, k = S.k;
  const uint32_t *lsrc = src + S.state_off;
  const unsigned long long keep = policy_evict_last();
  for (uint32_t base = 0; base < T.len; base += 32) {
    if (base + lane >= T.len) continue;
    const uint32_t q = T.start + base + lane;
    unsigned long long h = hash_step(0x243F6A8885A308D3ull ^ ((unsigned long long)T.seg * 0xD6E8FEB86659FD93ull),
                                     lsrc[q]);
    for (uint32_t a = 0; a < k; ++a) h = hash_step(h, ld_u32_hint(lsrc + S.delta[(size_t)a * n + q], keep));
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    const uint32_t b = (uint32_t)(h >> (64 - A.mbits));
    const uint32_t bit = 1u << (b & 31u);
    if (atomicOr(&A.seen1[b >> 5], bit) & bit) atomicOr(&A.seen2[b >> 5], bit);
    A.tmp[S.state_off + q] = b;
    unsigned long long h2 = (h ^ 0x9E3779B97F4A7C15ull) * 0xc4ceb9fe1a85ec53ull;
    h2 ^= h2 >> 31;
    A.tmp2[S.state_off + q] = (uint32_t)(h2 >> (64 - (A.mbits - 1)));
  }
}

// Pass B over one tile: a state alone in its bucket keeps its local number as
// label (a new singleton block); the others are listed in the block's list
// (state, second bucket, DFA; slots taken from a shared cursor) and enter the
// second filter.
__device__ __forceinline__ void batch_filter_b(const BatchArgs &A, const SegInfo &S, const Tile &T,
                                              uint32_t *__restrict__ dst, uint32_t r, uint32_t *list,
                                              uint32_t *list2, uint32_t *list3, uint32_t *s_cursor) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t uniq = 0, listed = 0;
  for (uint32_t base = 0; base < T.len; base += 32) {
    const bool valid = base + lane < T.len;
    const uint32_t q = T.start + base + lane, gq = S.state_off + q;
    bool dup = false;
    uint32_t b2 = 0;
    if (valid) {
      const uint32_t b = A.tmp[gq];
      dup = (A.seen2[b >> 5] >> (b & 31u)) & 1u;
      if (!dup) {
        dst[gq] = q;
        ++uniq;
      } else {
        b2 = A.tmp2[gq];
        const uint32_t bit = 1u << (b2 & 31u);
        if (atomicOr(&A.seen3[b2 >> 5], bit) & bit) atomicOr(&A.seen4[b2 >> 5], bit);
      }
    }
    const unsigned dm = __ballot_sync(0xFFFFFFFFu, dup);
    if (dm) {
      uint32_t at = 0;
      if (lane == 0) at = atomicAdd(s_cursor, (uint32_t)__popc(dm));
      at = __shfl_sync(0xFFFFFFFFu, at, 0);
      if (dup) {
        const uint32_t p = at + __popc(dm & ((1u << lane) - 1u));
        list[p] = gq;
        list2[p] = b2;
        list3[p] = T.seg;
      }
    }
    listed += __popc(dm);
  }
  const uint32_t u = __reduce_add_sync(0xFFFFFFFFu, uniq);
  if (lane == 0) {
    if (u) atomicAdd(&A.cnt[T.seg * 3 + r % 3], u);
    if (listed) atomicAdd(&A.ss[T.seg * SS_WORDS + SS_NDUP], listed);
  }
}

// Adds one to DFA seg's count of new blocks for every lane with `hit`, one
// atomic per (warp, DFA).
__device__ __forceinline__ void count_per_dfa(const BatchArgs &A, bool valid, bool hit, uint32_t seg, uint32_t r) {
  const uint32_t lane = threadIdx.x & 31u;
  const unsigned hm = __ballot_sync(0xFFFFFFFFu, valid && hit);
  const unsigned grp = __match_any_sync(0xFFFFFFFFu, valid ? seg : 0xFFFFFFFFu) & __ballot_sync(0xFFFFFFFFu, valid);
  if (valid && lane == (uint32_t)(__ffs(grp) - 1) && (grp & hm)) atomicAdd(&A.cnt[seg * 3 + r % 3], __popc(grp & hm));
}

// Listed entries resolved by the second filter are marked in their DFA word.
static constexpr uint32_t kResolved = 0x80000000u;

// Pass F over the block's list (warps take 32-entry chunks): a listed state
// alone in its second bucket is unique too and is marked resolved.
__device__ __forceinline__ void batch_filter_f(const BatchArgs &A, uint32_t *__restrict__ dst, uint32_t r,
                                              const uint32_t *list, const uint32_t *list2, uint32_t *list3,
                                              uint32_t nd) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t base = warp * 32; base < nd; base += nw * 32) {
    const uint32_t i = base + lane;
    const bool valid = i < nd;
    uint32_t seg = 0;
    bool still = false;
    if (valid) {
      const uint32_t gq = list[i];
      seg = list3[i];
      const uint32_t b2 = list2[i];
      still = (A.seen4[b2 >> 5] >> (b2 & 31u)) & 1u;
      if (!still) {
        dst[gq] = gq - A.segs[seg].state_off;
        list3[i] = seg | kResolved;
      }
    }
    count_per_dfa(A, valid, !still, seg, r);
  }
}

// Pass D over the block's list: the listed states left insert their exact
// keys into their own DFA's table region, tagged with the round's stage-0
// epoch (lanes may hold different DFAs: each lane inserts alone); a signature
// wider than one key goes in as its hash, joined only on a full comparison.
// Each slot keeps its smallest member (atomicMax on (round, ~local state)).
__device__ __forceinline__ void batch_filter_d(const BatchArgs &A, const uint32_t *__restrict__ src, uint32_t r,
                                              uint32_t epoch0, const uint32_t *list, const uint32_t *list3,
                                              uint32_t nd) {
  const unsigned long long keep = policy_evict_last();
  for (uint32_t i = threadIdx.x; i < nd; i += blockDim.x) {
    if (list3[i] & kResolved) continue;
    const uint32_t gq = list[i];
    const SegInfo &S = A.segs[list3[i]];
    const uint32_t q = gq - S.state_off, w = A.ss[list3[i] * SS_WORDS + SS_W];
    const uint32_t *lsrc = src + S.state_off;
    const StagePlan P = make_plan(S.k, w, S.log2S);
    const uint32_t mask = table_mask(S.log2S);
    uint32_t slot[1] = {0u};
    if (P.stages == 1) {   // the whole signature is one exact key
      u128 key[1] = {u128{0ull, 0ull}};
      put_bits(key[0], lsrc[q], 0);
      for (uint32_t a = 0; a < S.k; ++a)
        put_bits(key[0], ld_u32_hint(lsrc + S.delta[(size_t)a * S.n + q], keep), (a + 1) * w);
      key[0].hi |= (unsigned long long)epoch0 << (64 - A.ebits);
      slot[0] = (uint32_t)(mix128(key[0]) >> 32) & mask;
      const bool want[1] = {true};
      bool is_new[1];
      table_insert_vec<1>(A.table + S.table_off, mask, key, A.ebits, epoch0, want, slot, is_new, &A.ctrl->err);
    } else {               // wider: signature hash plus full comparison with the slot's representative
      const SigEq eq{lsrc, S.delta, S.n, S.k};
      slot[0] = hashed_insert(A.table + S.table_off, mask, A.ebits, epoch0, eq.hash(q), q, eq, &A.ctrl->err);
    }
    A.tmp[gq] = slot[0];
    atomicMax(&A.rep[S.table_off + slot[0]], ((unsigned long long)r << 32) | (unsigned long long)(~q));
  }
}

// Pass C over the block's list: the listed states left take their slot's
// smallest member as label; a state that is its slot's smallest member counts
// a block.
__device__ __forceinline__ void batch_filter_c(const BatchArgs &A, uint32_t *__restrict__ dst, uint32_t r,
                                              const uint32_t *list, const uint32_t *list3, uint32_t nd) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t base = warp * 32; base < nd; base += nw * 32) {
    const uint32_t i = base + lane;
    const bool valid = i < nd && !(list3[i] & kResolved);
    uint32_t seg = 0;
    bool first = false;
    if (valid) {
      const uint32_t gq = list[i];
      seg = list3[i];
      const SegInfo &S = A.segs[seg];
      const uint32_t m = ~(uint32_t)A.rep[S.table_off + A.tmp[gq]];
      dst[gq] = m;
      first = m == gq - S.state_off;
    }
    count_per_dfa(A, valid, first, seg, r);
  }
}

// Direct round over one tile: new label = packed signature; a bitmap over the
// DFA's 2^log2S possible labels (bits [table_off, table_off + 2^log2S) of the
// batch bitmap; table_off is a multiple of 64) counts the labels that appear,
// one atomic per (warp, label).  Keys of at most kWarpBits bits are marked in
// the warp's own 32-word shared bitmap first and merged once per tile, so that
// the few words of such a DFA are not hit by every warp for every state.
static constexpr uint32_t kWarpBits = 10;
template <bool ROUND1>
__device__ __forceinline__ void batch_direct_tile(const BatchArgs &A, const SegInfo &S, const Tile &T, uint32_t w,
                                                 const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                                 uint32_t *bm, uint32_t *wbm, uint32_t r) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = S.n, k = S.k;
  const bool small = (k + 1) * w <= kWarpBits;
  if (small) {
    wbm[lane] = 0u;
    __syncwarp();
  }
  const uint32_t *lsrc = src + S.state_off;
  const unsigned long long keep = policy_evict_last();
  uint32_t seen = 0, created = 0;
  for (uint32_t base = 0; base < T.len; base += 32) {
    const bool valid = base + lane < T.len;
    const uint32_t q = T.start + (valid ? base + lane : 0u);
    uint32_t key;
    if (ROUND1) {
      key = S.accept[q] != 0;
      if (valid) seen |= key ? 1u : 2u;
    } else {
      key = lsrc[q];
    }
    uint32_t shift = w;
    for (uint32_t a = 0; a < k; ++a) {
      uint32_t d = S.delta[(size_t)a * n + q];
      if (ROUND1 && d >= n) {
        if (valid) atomicOr(&A.ctrl->err, ERR_BAD_DELTA);
        d = 0;
      }
      const uint32_t c = ROUND1 ? (uint32_t)(S.accept[d] != 0) : ld_u32_hint(lsrc + d, keep);
      key |= c << shift;
      shift += w;
    }
    if (valid) dst[S.state_off + q] = key;
    const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, valid ? key : 0xFFFFFFFFu) & vm;
    if (valid && lane == (uint32_t)(__ffs(grp) - 1)) {
      if (small) {
        atomicOr(&wbm[key >> 5], 1u << (key & 31u));
      } else {
        const uint64_t pos = S.table_off + key;
        const uint32_t bit = 1u << (pos & 31u);
        if (!(atomicOr(&bm[pos >> 5], bit) & bit)) ++created;
      }
    }
  }
  if (small) {
    __syncwarp();
    const uint32_t v = wbm[lane];
    if (v) created += __popc(v & ~atomicOr(&bm[(S.table_off >> 5) + lane], v));
    __syncwarp();
  }
  const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, created);
  if (lane == 0 && wsum) atomicAdd(&A.cnt[T.seg * 3 + r % 3], wsum);
  if (ROUND1) {
    const uint32_t wseen = __reduce_or_sync(0xFFFFFFFFu, seen);
    if (lane == 0 && wseen) atomicOr(&A.ss[T.seg * SS_WORDS + SS_SEEN], wseen);
  }
}

// Table round over one tile, stage `stage` of plan P: the signature's
// components [cbeg, cend) (after the previous stage's slot) form a key of the
// DFA's own table region; the slot is the new label.
template <int VEC, bool ROUND1>
__device__ __forceinline__ void batch_table_tile(const BatchArgs &A, const SegInfo &S, const Tile &T,
                                                const StagePlan &P, uint32_t stage, bool last, uint32_t epoch,
                                                const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                                CtaCache *cache, uint32_t r) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = S.n, total = S.k + 1, bits = P.bits;
  uint32_t cbeg, cend;
  bool has_prev;
  if (stage == 0) {
    cbeg = 0;
    cend = P.first < total ? P.first : total;
    has_prev = false;
  } else {
    cbeg = P.first + (stage - 1) * P.per;
    cend = cbeg + P.per < total ? cbeg + P.per : total;
    has_prev = true;
  }
  const unsigned long long etag = (unsigned long long)epoch << (64 - A.ebits);
  const unsigned long long keep = policy_evict_last();
  const uint32_t *lsrc = src + S.state_off;   // this DFA's labels (local numbers)
  u128 *table = A.table + S.table_off;
  uint32_t seen = 0, created_total = 0;
  for (uint32_t base = 0; base < T.len; base += 32u * VEC) {
    u128 key[VEC];
    bool valid = false;
    uint32_t qs[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const uint32_t off = base + lane * VEC + v;
      qs[v] = T.start + (off < T.len ? off : 0u);
      key[v] = u128{0ull, 0ull};
    }
    valid = base + lane * VEC < T.len;
    bool vv[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) vv[v] = base + lane * VEC + v < T.len;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const uint32_t q = qs[v];
      uint32_t shift = 0;
      if (has_prev) {
        put_bits(key[v], A.tmp[S.state_off + q], 0);
        shift = P.carry;
      }
      uint32_t j = cbeg;
      if (j == 0) {
        uint32_t c;
        if (ROUND1) {
          c = S.accept[q] != 0;
          if (vv[v]) seen |= c ? 1u : 2u;
        } else {
          c = lsrc[q];
        }
        put_bits(key[v], c, shift);
        shift += bits;
        j = 1;
      }
      for (; j < cend; ++j) {
        uint32_t d = S.delta[(size_t)(j - 1) * n + q];
        if (ROUND1 && d >= n) {
          if (vv[v]) atomicOr(&A.ctrl->err, ERR_BAD_DELTA);
          d = 0;
        }
        const uint32_t c = ROUND1 ? (uint32_t)(S.accept[d] != 0) : ld_u32_hint(lsrc + d, keep);
        put_bits(key[v], c, shift);
        shift += bits;
      }
      key[v].hi |= etag;
    }
    // Lanes whose states lie past the tile end insert nothing (their keys are
    // duplicates of the tile's first state).
    uint32_t lab[VEC];
    uint32_t created = 0;
    if constexpr (VEC == 1) {
      warp_insert<1>(table, S.log2S, key, valid, A.ebits, epoch, lab, created, &A.ctrl->err, cache, T.seg);
    } else {
      // second state of a pair may lie past the end: give it the first state's key
      if (!vv[1]) key[1] = key[0];
      warp_insert<VEC>(table, S.log2S, key, valid, A.ebits, epoch, lab, created, &A.ctrl->err, cache, T.seg);
    }
    if (last) created_total += created;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      if (!vv[v]) continue;
      const uint32_t gq = S.state_off + qs[v];
      if (last) dst[gq] = lab[v];
      else A.tmp[gq] = lab[v];
    }
  }
  // one atomic per warp and tile: every lane of the warp works on this DFA
  const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, created_total);
  if (lane == 0 && wsum) atomicAdd(&A.cnt[T.seg * 3 + r % 3], wsum);
  if (ROUND1) {
    const uint32_t wseen = __reduce_or_sync(0xFFFFFFFFu, seen);
    if (lane == 0 && wseen) atomicOr(&A.ss[T.seg * SS_WORDS + SS_SEEN], wseen);
  }
}

// Exclusive prefix sums of in[0, m) into out, by the whole grid: block b scans
// a contiguous range, then adds the totals of the blocks before it.  `partials`
// holds gridDim entries.  Returns false if a barrier failed.
__device__ bool grid_excl_scan(const uint32_t *in, uint32_t *out, uint32_t m, uint32_t *partials, Ctrl *C,
                               unsigned long long barrier_ns, uint32_t *s_red) {
  uint32_t chunk = (m + gridDim.x - 1) / gridDim.x;
  chunk = (chunk + blockDim.x - 1) / blockDim.x * blockDim.x;
  const uint64_t beg64 = (uint64_t)blockIdx.x * chunk;
  const uint32_t beg = beg64 < m ? (uint32_t)beg64 : m;
  const uint32_t end = (uint64_t)beg + chunk < m ? beg + chunk : m;
  uint32_t running = 0;
  for (uint32_t base = beg;; base += blockDim.x) {   // at least once: every thread takes part in the scan
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < end ? in[i] : 0u;
    uint32_t total;
    const uint32_t ex = block_excl_scan(v, s_red, &total);
    if (i < end) out[i] = running + ex;
    running += total;
    if (base + blockDim.x >= end) break;
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = running;
  if (!grid_sync(C, barrier_ns)) return false;
  uint32_t pre = 0;
  for (uint32_t b = threadIdx.x; b < blockIdx.x; b += blockDim.x) pre += partials[b];
  pre = block_sum(pre, s_red);
  for (uint32_t i = beg + threadIdx.x; i < end; i += blockDim.x) out[i] += pre;
  return true;
}

// One state per lane: two blocks per SM (at most 64 registers); two states per
// lane: one block per SM with room for the wider keys.
template <int VEC>
__global__ void __launch_bounds__(kBatchThreads, VEC == 1 ? 2 : 1) batch_kernel(BatchArgs A) {
  __shared__ uint32_t s_red[kBatchThreads / 32];
  __shared__ CtaCache cache;
  __shared__ uint32_t s_wbm[kBatchThreads / 32][32];
  __shared__ uint32_t s_next, s_cursor;   // next tile of the block; length of the block's list
  Ctrl *C = A.ctrl;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const uint32_t gwarp = tid >> 5, nwarps = stride >> 5, lane = threadIdx.x & 31u;
  if (leader) {
    const unsigned long long t = gtimer();
    C->t_start = t;
    C->deadline = t + A.timeout_ns;
  }
  const uint32_t emax = A.ebits >= 32 ? 0xFFFFFFFFu : ((1u << A.ebits) - 1u);
  const uint64_t bm_words = (A.total_slots + 31) / 32;
  // clear tables and round 1's bitmap; every DFA starts active with 1-bit labels
  for (uint64_t i = tid; i < A.total_slots; i += stride) reinterpret_cast<uint4 *>(A.table)[i] = make_uint4(0, 0, 0, 0);
  for (uint64_t i = tid; i < bm_words; i += stride) A.bm[1][i] = 0u;
  for (uint32_t i = tid; i < A.nsegs; i += stride) {
    A.ss[i * SS_WORDS + SS_ACTIVE] = A.segs[i].small ? 0u : 1u;
    A.ss[i * SS_WORDS + SS_FINAL] = 1u;
    A.ss[i * SS_WORDS + SS_W] = 1u;
    A.ss[i * SS_WORDS + SS_FOK] = 1u;
  }
  // filter counters and slot owners start clean
  for (uint64_t i = tid; i < ((uint64_t)1 << A.mbits) / 32; i += stride) {
    A.seen1[i] = 0u;
    A.seen2[i] = 0u;
  }
  for (uint64_t i = tid; i < ((uint64_t)1 << A.mbits) / 64; i += stride) {
    A.seen3[i] = 0u;
    A.seen4[i] = 0u;
  }
  for (uint64_t i = tid; i < A.total_slots; i += stride) A.rep[i] = 0ull;
  // tile list: DFA i's tiles are tile_off[i] .. tile_off[i + 1) - 1, one warp per DFA
  for (uint32_t i = gwarp; i < A.nsegs; i += nwarps) {
    const uint32_t t0 = A.tile_off[i], nt = A.tile_off[i + 1] - t0, n = A.segs[i].n;
    for (uint32_t j = lane; j < nt; j += 32) {
      const uint32_t start = j * A.tile;
      A.tiles[t0 + j] = Tile{i, start, n - start < A.tile ? n - start : A.tile};
    }
  }
  bool ok = grid_sync(C, A.barrier_ns);
  uint32_t epoch = 0, r;
  for (r = 1; ok; ++r) {
    const bool round1 = r == 1;
    const uint32_t *src = A.lab[(r - 1) & 1];
    uint32_t *dst = A.lab[r & 1];
    // some DFA takes a filter round (decided by the last bookkeeping)
    const bool any_filter = !round1 && ld_relaxed(&C->flag2[r % 3]) != 0u;
    if (leader) C->flag2[(r + 2) % 3] = 0u;
    // the bitmap of the next round starts clean (the one of the previous round is free now)
    for (uint64_t i = tid; i < bm_words; i += stride) A.bm[(r + 1) & 1][i] = 0u;
    uint32_t epoch0 = 0;
    for (uint32_t s = 0; ok && s < A.max_stages; ++s) {
      // a round's stages (and its filter inserts) take epochs epoch0 .. epoch0 + max_stages - 1:
      // wrap before stage 0 unless they all fit
      if (s == 0 ? (uint64_t)epoch + A.max_stages > emax : epoch == emax) {
        for (uint64_t i = tid; i < A.total_slots; i += stride)
          reinterpret_cast<uint4 *>(A.table)[i] = make_uint4(0, 0, 0, 0);
        ok = grid_sync(C, A.barrier_ns);
        epoch = 0;
        if (!ok) break;
      }
      ++epoch;
      if (s == 0) epoch0 = epoch;
      cta_cache_clear(&cache);
      start_tiles(&s_next);
      for (uint32_t t = next_tile(A, &s_next); t < A.ntiles; t = next_tile(A, &s_next)) {
        const Tile T = A.tiles[t];
        if (!ld_relaxed(&A.ss[T.seg * SS_WORDS + SS_ACTIVE])) continue;
        const SegInfo &S = A.segs[T.seg];
        const uint32_t w = A.ss[T.seg * SS_WORDS + SS_W];
        const uint32_t mode = batch_mode(S, A.ss + T.seg * SS_WORDS, r);
        if (mode == BM_FILTER) {
          if (s == 0) batch_filter_a(A, S, T, src);
          continue;
        }
        if (mode == BM_DIRECT) {
          if (s != 0) continue;
          uint32_t *wbm = s_wbm[threadIdx.x >> 5];
          if (round1) batch_direct_tile<true>(A, S, T, w, src, dst, A.bm[r & 1], wbm, r);
          else batch_direct_tile<false>(A, S, T, w, src, dst, A.bm[r & 1], wbm, r);
          continue;
        }
        const StagePlan P = make_plan(S.k, w, S.log2S);
        if (s >= P.stages) continue;
        const bool last = s + 1 == P.stages;
        if (round1) batch_table_tile<VEC, true>(A, S, T, P, s, last, epoch, src, dst, &cache, r);
        else batch_table_tile<VEC, false>(A, S, T, P, s, last, epoch, src, dst, &cache, r);
      }
      ok = grid_sync(C, A.barrier_ns);
      if (ok && s == 0 && any_filter) {
        // filter passes B, F, D, C over the block's own list
        const size_t at = (size_t)blockIdx.x * A.dup_cap;
        uint32_t *list = A.dups + at, *list2 = A.dups2 + at, *list3 = A.dups3 + at;
        if (threadIdx.x == 0) s_cursor = 0u;
        start_tiles(&s_next);
        for (uint32_t t = next_tile(A, &s_next); t < A.ntiles; t = next_tile(A, &s_next)) {
          const Tile T = A.tiles[t];
          if (!ld_relaxed(&A.ss[T.seg * SS_WORDS + SS_ACTIVE])) continue;
          const SegInfo &S = A.segs[T.seg];
          if (batch_mode(S, A.ss + T.seg * SS_WORDS, r) != BM_FILTER) continue;
          batch_filter_b(A, S, T, dst, r, list, list2, list3, &s_cursor);
        }
        ok = grid_sync(C, A.barrier_ns);
        const uint32_t nd = s_cursor;   // the block's list length (read after the barrier)
        if (ok) {
          batch_filter_f(A, dst, r, list, list2, list3, nd);
          ok = grid_sync(C, A.barrier_ns);
        }
        if (ok) {
          batch_filter_d(A, src, r, epoch0, list, list3, nd);
          ok = grid_sync(C, A.barrier_ns);
        }
        if (ok) {
          batch_filter_c(A, dst, r, list, list3, nd);
          for (uint64_t i = tid; i < ((uint64_t)1 << A.mbits) / 32; i += stride) {
            A.seen1[i] = 0u;
            A.seen2[i] = 0u;
          }
          for (uint64_t i = tid; i < ((uint64_t)1 << A.mbits) / 64; i += stride) {
            A.seen3[i] = 0u;
            A.seen4[i] = 0u;
          }
          ok = grid_sync(C, A.barrier_ns);
        }
      }
    }
    if (!ok) break;
    // bookkeeping: one thread per DFA
    uint32_t still = 0, next_filter = 0;
    for (uint32_t i = tid; i < A.nsegs; i += stride) {
      uint32_t *w = A.ss + i * SS_WORDS;
      A.cnt[i * 3 + (r + 2) % 3] = 0u;
      if (!w[SS_ACTIVE]) continue;
      const SegInfo &S = A.segs[i];
      const uint32_t mode = batch_mode(S, w, r);   // this round's mode (words not yet updated)
      const uint32_t B = A.cnt[i * 3 + r % 3];
      const uint32_t prev = round1 ? __popc(w[SS_SEEN]) : w[SS_PREV];
      w[SS_EXECUTED] = r;
      w[SS_FINAL] = r & 1;
      w[SS_B] = B;
      // width of this round's labels
      w[SS_W] = mode == BM_DIRECT ? (S.k + 1) * w[SS_W] : mode == BM_FILTER ? S.wid : S.log2S;
      // a filter round that listed most states (large blocks): later rounds use the table
      if (mode == BM_FILTER && (uint64_t)w[SS_NDUP] * 2 > S.n) w[SS_FOK] = 0u;
      w[SS_NDUP] = 0u;
      if (B == prev) {
        w[SS_ACTIVE] = 0u;               // fixpoint (Algorithm 4's until-test)
      } else {
        w[SS_CHANGED] += 1;
        w[SS_PREV] = B;
        if (A.stop_discrete && B == S.n) {
          w[SS_ACTIVE] = 0u;             // n singleton blocks cannot split any further
        } else if (A.max_rounds != 0u && r >= A.max_rounds) {
          w[SS_ACTIVE] = 0u;
          w[SS_MAXED] = 1u;
        } else {
          ++still;
          if (batch_mode(S, w, r + 1) == BM_FILTER) next_filter = 1u;
        }
      }
    }
    const uint32_t bs = block_sum(still, s_red);
    if (threadIdx.x == 0 && bs) atomicAdd(&C->cnt[r % 3], bs);
    const uint32_t bf = block_sum(next_filter, s_red);
    if (threadIdx.x == 0 && bf) atomicOr(&C->flag2[(r + 1) % 3], 1u);
    ok = grid_sync(C, A.barrier_ns);
    if (!ok) break;
    const uint32_t active = ld_relaxed(&C->cnt[r % 3]);
    if (leader) C->cnt[(r + 2) % 3] = 0u;
    if (active == 0u) break;
  }

  // Canonical numbering per DFA: block id = rank of its smallest state within
  // the DFA.  A DFA with n blocks is numbered by its states; the others find
  // each label's smallest state in their own slice of minrep (2^log2S entries
  // at table_off), count first members per tile, and rank them by a scan over
  // the tiles.
  if (ok) {
    start_tiles(&s_next);
    for (uint32_t t = next_tile(A, &s_next); t < A.ntiles; t = next_tile(A, &s_next)) {
      const Tile T = A.tiles[t];
      const SegInfo &S = A.segs[T.seg];
      if (S.small || A.ss[T.seg * SS_WORDS + SS_B] == S.n) continue;
      const uint64_t region = 1ull << S.log2S;
      const uint32_t nt = A.tile_off[T.seg + 1] - A.tile_off[T.seg], j = t - A.tile_off[T.seg];
      const uint64_t per = (region + nt - 1) / nt, lo = (uint64_t)j * per;
      const uint64_t hi = lo + per < region ? lo + per : region;
      for (uint64_t i = lo + lane; i < hi; i += 32) A.minrep[S.table_off + i] = 0xFFFFFFFFu;
    }
    ok = grid_sync(C, A.barrier_ns);
  }
  if (ok) {
    start_tiles(&s_next);
    for (uint32_t t = next_tile(A, &s_next); t < A.ntiles; t = next_tile(A, &s_next)) {
      const Tile T = A.tiles[t];
      const SegInfo &S = A.segs[T.seg];
      if (S.small || A.ss[T.seg * SS_WORDS + SS_B] == S.n) continue;
      const uint32_t *fl = A.lab[A.ss[T.seg * SS_WORDS + SS_FINAL]] + S.state_off;
      for (uint32_t base = 0; base < T.len; base += 32) {
        const bool valid = base + lane < T.len;
        const uint32_t q = T.start + base + lane;
        const uint32_t l = valid ? fl[q] : 0u;
        // lanes hold consecutive states: the lowest lane of a label group is its smallest state
        const unsigned grp = __match_any_sync(0xFFFFFFFFu, l) & __ballot_sync(0xFFFFFFFFu, valid);
        if (valid && lane == (uint32_t)(__ffs(grp) - 1)) atomicMin(&A.minrep[S.table_off + l], q);
      }
    }
    ok = grid_sync(C, A.barrier_ns);
  }
  if (ok) {
    start_tiles(&s_next);
    for (uint32_t t = next_tile(A, &s_next); t < A.ntiles; t = next_tile(A, &s_next)) {
      const Tile T = A.tiles[t];
      const SegInfo &S = A.segs[T.seg];
      uint32_t c = S.small ? 0u : T.len;
      if (!S.small && A.ss[T.seg * SS_WORDS + SS_B] != S.n) {
        const uint32_t *fl = A.lab[A.ss[T.seg * SS_WORDS + SS_FINAL]] + S.state_off;
        c = 0;
        for (uint32_t base = 0; base < T.len; base += 32) {
          const uint32_t q = T.start + base + lane;
          const bool first = base + lane < T.len && A.minrep[S.table_off + fl[q]] == q;
          c += __popc(__ballot_sync(0xFFFFFFFFu, first));
        }
      }
      if (lane == 0) A.tile_cnt[t] = c;
    }
    ok = grid_sync(C, A.barrier_ns);
  }
  if (ok) ok = grid_excl_scan(A.tile_cnt, A.tile_pre, A.ntiles, A.partials, C, A.barrier_ns, s_red);
  if (ok) ok = grid_sync(C, A.barrier_ns);
  if (ok) {
    start_tiles(&s_next);
    for (uint32_t t = next_tile(A, &s_next); t < A.ntiles; t = next_tile(A, &s_next)) {
      const Tile T = A.tiles[t];
      const SegInfo &S = A.segs[T.seg];
      uint32_t *o = A.out + S.state_off;
      if (S.small) continue;
      if (A.ss[T.seg * SS_WORDS + SS_B] == S.n) {
        for (uint32_t i = lane; i < T.len; i += 32) o[T.start + i] = T.start + i;
        continue;
      }
      const uint32_t *fl = A.lab[A.ss[T.seg * SS_WORDS + SS_FINAL]] + S.state_off;
      uint32_t rank = A.tile_pre[t] - A.tile_pre[A.tile_off[T.seg]];
      for (uint32_t base = 0; base < T.len; base += 32) {
        const uint32_t q = T.start + base + lane;
        const bool valid = base + lane < T.len;
        const uint32_t l = valid ? fl[q] : 0u;
        const bool first = valid && A.minrep[S.table_off + l] == q;
        const unsigned fm = __ballot_sync(0xFFFFFFFFu, first);
        // every lane has read minrep[l] above before any lane overwrites it
        __syncwarp();
        if (first) A.minrep[S.table_off + l] = 0x80000000u | (rank + __popc(fm & ((1u << lane) - 1u)));
        rank += __popc(fm);
      }
    }
    ok = grid_sync(C, A.barrier_ns);
  }
  if (ok) {
    start_tiles(&s_next);
    for (uint32_t t = next_tile(A, &s_next); t < A.ntiles; t = next_tile(A, &s_next)) {
      const Tile T = A.tiles[t];
      const SegInfo &S = A.segs[T.seg];
      if (S.small || A.ss[T.seg * SS_WORDS + SS_B] == S.n) continue;
      const uint32_t *fl = A.lab[A.ss[T.seg * SS_WORDS + SS_FINAL]] + S.state_off;
      for (uint32_t i = lane; i < T.len; i += 32) {
        const uint32_t q = T.start + i;
        A.out[S.state_off + q] = A.minrep[S.table_off + fl[q]] & 0x7FFFFFFFu;
      }
    }
  }
  if (leader) {
    C->rounds_executed = r;
    C->t_end = gtimer();
  }
}

// ------------------------------------------------------------------ host side

struct BatchLayout {
  size_t ctrl, segs, tile_off, tiles, lab0, lab1, tmp, tmp2, seen1, seen2, seen3, seen4, rep, dups, dups2, dups3, table,
      bm0, bm1, minrep, tile_cnt, tile_pre, partials, out, cnt, ss, items, small_next, stage, total;
  size_t list_entries;
  uint32_t mbits;
  uint64_t total_states, total_slots;
  uint32_t ntiles, max_stages, ebits;
  size_t stage_bytes;
  uint32_t ntiles_by[3];   // tiles of 256, 128 and 64 states (summed by the same pass)
};
static void batch_place(BatchLayout &L, uint32_t count, uint32_t tile, uint32_t ntiles);

// Warps of the batch kernel's cooperative grid (the larger of the two
// schedules' grids); without a visible device, the largest grid the launcher
// accepts.
static size_t batch_max_warps();

// Where the inputs of a batch live: host[2i] / host[2i + 1] tell whether DFA
// i's delta / accept are host memory, to be staged into the workspace.  With
// `packed`, the DFAs' arrays are consecutive pieces of one delta buffer and one
// accept buffer (in DFA order); host ones are staged as two copies, keeping
// that order.
struct BatchInputs {
  std::vector<uint8_t> host;
  bool packed = false;
};

static BatchInputs classify_inputs(const dfa_t *dfas, uint32_t count) {
  BatchInputs in;
  in.host.resize((size_t)count * 2);
  for (uint32_t i = 0; i < count; ++i) {
    in.host[2 * i] = dfas[i].k > 0 && !is_device_ptr(dfas[i].delta);
    in.host[2 * i + 1] = !is_device_ptr(dfas[i].accept);
  }
  return in;
}

static BatchLayout batch_layout(const dfa_t *dfas, uint32_t count, const BatchInputs &in, uint32_t tile,
                                std::vector<SegInfo> *segs_out, std::vector<uint32_t> *tile_off_out,
                                std::vector<size_t> *stage_off) {
  BatchLayout L{};
  uint64_t st = 0, sl = 0;
  uint32_t ntiles = 0, max_stages = 1, ebits = 32;
  size_t stage_bytes = 0;
  bool multi = false;
  size_t packed_delta_bytes = 0;
  if (in.packed)
    for (uint32_t i = 0; i < count; ++i)
      if (in.host[2 * i]) packed_delta_bytes += (size_t)dfas[i].k * dfas[i].n * 4;
  size_t pd = 0, pa = (packed_delta_bytes + 255) / 256 * 256;
  for (uint32_t i = 0; i < count; ++i) {
    const dfa_t &d = dfas[i];
    SegInfo s{};
    s.n = d.n;
    s.k = d.k;
    s.state_off = (uint32_t)st;
    s.log2S = ceil_log2((uint64_t)d.n * 2 < 64 ? 64 : (uint64_t)d.n * 2);
    s.wid = ceil_log2(d.n) > 0 ? ceil_log2(d.n) : 1;
    s.table_off = sl;
    // label widths a DFA goes through: 1 bit, then (k+1) times wider while the
    // rounds are direct; then log2S bits after a table round or wid bits after
    // a filter round.  The plans of the table and filter rounds decide the
    // stage count and the epoch bits left free.
    if (d.k > 0) {
      uint64_t w = 1;
      while ((uint64_t)(d.k + 1) * w <= s.log2S) w *= d.k + 1;   // direct rounds
      for (const uint64_t x : {w, (uint64_t)s.log2S, (uint64_t)s.wid}) {
        const StagePlan p = make_plan(d.k, (uint32_t)x, s.log2S);
        max_stages = std::max(max_stages, p.stages);
        ebits = std::min(ebits, p.ebits);
        multi |= p.stages > 1;
      }
    }
    if (tile_off_out) tile_off_out->push_back(ntiles);
    ntiles += (d.n + tile - 1) / tile;
    for (int t = 0; t < 3; ++t) L.ntiles_by[t] += (d.n + (256u >> t) - 1) >> (8 - t);
    // host-resident arrays are staged into the workspace
    const bool hd = in.host[2 * i], ha = in.host[2 * i + 1];
    const size_t db = (size_t)d.k * d.n * 4, ab = d.n;
    if (in.packed) {
      if (stage_off) {
        stage_off->push_back(hd ? pd : SIZE_MAX);
        stage_off->push_back(ha ? pa : SIZE_MAX);
      }
      if (hd) pd += db;
      if (ha) pa += ab;
      stage_bytes = pa;
    } else {
      if (stage_off) stage_off->push_back(hd ? stage_bytes : SIZE_MAX);
      if (hd) stage_bytes += (db + 255) / 256 * 256;
      if (stage_off) stage_off->push_back(ha ? stage_bytes : SIZE_MAX);
      if (ha) stage_bytes += (ab + 255) / 256 * 256;
    }
    st += d.n;
    sl += (uint64_t)1 << s.log2S;
    if (segs_out) segs_out->push_back(s);
  }
  if (tile_off_out) tile_off_out->push_back(ntiles);
  (void)multi;
  L.total_states = st;
  L.total_slots = sl;
  L.max_stages = max_stages;
  L.ebits = ebits;
  L.stage_bytes = stage_bytes;
  batch_place(L, count, tile, ntiles);
  return L;
}

// The workspace offsets of a batch whose totals the pass above has summed, for
// `tile` states per tile and `ntiles` tiles.
static void batch_place(BatchLayout &L, uint32_t count, uint32_t tile, uint32_t ntiles) {
  const uint64_t st = L.total_states, sl = L.total_slots;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  L.ntiles = ntiles;
  L.ctrl = take(sizeof(Ctrl));
  L.segs = take(sizeof(SegInfo) * count);
  L.tile_off = take(((size_t)count + 1) * 4);
  L.tiles = take((size_t)ntiles * sizeof(Tile));
  L.lab0 = take(st * 4);
  L.lab1 = take(st * 4);
  L.tmp = take(st * 4);   // multi-stage slots; filter buckets and slots
  L.tmp2 = take(st * 4);
  L.mbits = std::min<uint32_t>(31, std::max<uint32_t>(12, ceil_log2(st) + 2));
  L.seen1 = take(((size_t)1 << L.mbits) / 8);
  L.seen2 = take(((size_t)1 << L.mbits) / 8);
  L.seen3 = take(((size_t)1 << L.mbits) / 16);
  L.seen4 = take(((size_t)1 << L.mbits) / 16);
  L.rep = take(sl * 8);
  L.list_entries = ((size_t)ntiles + batch_max_warps() / (kBatchThreads / 32)) * tile;   // per block: its tiles
  L.dups = take(L.list_entries * 4);
  L.dups2 = take(L.list_entries * 4);
  L.dups3 = take(L.list_entries * 4);
  L.table = take(sl * 16);
  L.bm0 = take((sl + 31) / 32 * 4);
  L.bm1 = take((sl + 31) / 32 * 4);
  L.minrep = take(sl * 4);
  L.tile_cnt = take((size_t)ntiles * 4);
  L.tile_pre = take((size_t)ntiles * 4);
  L.partials = take(kMaxGridB * 4);
  L.out = take(st * 4);
  L.cnt = take((size_t)count * 3 * 4);
  L.ss = take((size_t)count * SS_WORDS * 4);
  L.items = take((size_t)count * sizeof(BatchSmallItem));
  L.small_next = take(4);
  L.stage = take(L.stage_bytes);
  L.total = off;
}

static const void *batch_kernel_for(uint32_t vec) {
  return vec == 2 ? (const void *)batch_kernel<2> : (const void *)batch_kernel<1>;
}

static size_t batch_max_warps() {
  const size_t fallback = kMaxGridB * (kBatchThreads / 32);
  static std::atomic<size_t> known[64];   // per device, 0 = not looked up yet
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fallback;
  }
  if (dev >= 0 && dev < 64) {
    const size_t k = known[dev].load(std::memory_order_relaxed);
    if (k) return k;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return fallback;
  }
  size_t best = 0;
  for (uint32_t v : {1u, 2u}) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_for(v), kBatchThreads, 0) != cudaSuccess) {
      cudaGetLastError();
      return fallback;
    }
    best = std::max(best, (size_t)sms * (size_t)(per_sm < 1 ? 1 : per_sm) * (kBatchThreads / 32));
  }
  if (dev >= 0 && dev < 64) known[dev].store(best, std::memory_order_relaxed);
  return best;
}

// The DFAs of a batch refined one per block after the cooperative launch.
struct SmallLaunch {
  const BatchSmallItem *items;   // device
  uint32_t count;
  uint32_t *next;                // device word, zeroed in the graph
  size_t smem;
  uint32_t grid;
  const dfa_opts *o;
};

struct GraphCache {
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec[6] = {};   // by graph shape: cooperative launch (lane width) or none, block kernel or none
  ~GraphCache() {   // at thread exit; errors are ignored (the runtime may be gone at process exit)
    for (cudaGraphExec_t &x : exec)
      if (x) cudaGraphExecDestroy(x);
    if (cap) cudaStreamDestroy(cap);
  }
};
static constexpr int kGraphDevices = 64;
static thread_local GraphCache g_graphs[kGraphDevices];   // per device: a capture stream belongs to one device
static std::atomic<uint64_t> g_graph_instantiations{0}, g_graph_updates{0};

// Launches the batch kernel as a CUDA graph: the control-block reset and the
// cooperative launch (left out when every DFA has a block of its own; then,
// with `sl`, the reset of the DFA counter and the block-per-DFA kernel) are
// captured on a library-owned stream (capture is not
// allowed on the legacy default stream) and the graph runs on `st`.  The
// instantiated graph is kept per host thread, per device and per graph shape: a later
// call captures its own nodes (new pointers, new grid) and moves them into the
// kept executable with cudaGraphExecUpdate, which costs a fraction of a new
// instantiation; only when the update is refused is the graph instantiated
// again.  An update affects later launches only, and launches of one
// executable run in order, so a call never changes a launch still in flight.
static cudaError_t launch_batch_graph(const BatchArgs &a, int grid, bool coop, const SmallLaunch *sl,
                                      cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kGraphDevices) return cudaErrorInvalidDevice;
  GraphCache &G = g_graphs[dev];
  if (!G.cap && (e = cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  BatchArgs copy = a;
  void *params[] = {&copy};
  cudaError_t le = cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl), G.cap);
  if (le == cudaSuccess && coop)
    le = cudaLaunchCooperativeKernel(batch_kernel_for(a.vec), dim3(grid), dim3(kBatchThreads), params, 0, G.cap);
  if (le == cudaSuccess && sl) {
    le = cudaMemsetAsync(sl->next, 0, 4, G.cap);
    const BatchSmallWords words{SS_B, SS_CHANGED, SS_EXECUTED, SS_MAXED};
    if (le == cudaSuccess)
      le = enqueue_batch_small(sl->items, sl->count, sl->next, a.ctrl, sl->smem, words, *sl->o, sl->grid, G.cap);
  }
  e = cudaStreamEndCapture(G.cap, &graph);
  if (le != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return le;
  }
  if (e != cudaSuccess) return e;
  cudaGraphExec_t &exec = G.exec[(coop ? (a.vec == 2 ? 1 : 0) : 2) + (sl ? 3 : 0)];
  bool updated = false;
  if (exec) {
    cudaGraphExecUpdateResultInfo info{};
    updated = cudaGraphExecUpdate(exec, graph, &info) == cudaSuccess;
    if (!updated) {
      cudaGetLastError();   // a refused update is not an error of this call
      cudaGraphExecDestroy(exec);
      exec = nullptr;
    }
  }
  if (!exec) {
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
      exec = nullptr;
      cudaGraphDestroy(graph);
      return e;
    }
    g_graph_instantiations.fetch_add(1, std::memory_order_relaxed);
  } else if (updated) {
    g_graph_updates.fetch_add(1, std::memory_order_relaxed);
  }
  cudaGraphDestroy(graph);
  return cudaGraphLaunch(exec, st);
}

// ------------------------------------------------------------------ autotuner
// With opts.schedule = -1 the first call for a (GPU, total-states bucket,
// batch-size bucket, largest k) key runs the batch once under every schedule,
// keeps the fastest by device time, and remembers the choice together with
// every schedule's time, in memory and in a JSON file ($DFA_AUTOTUNE_CACHE,
// default ~/.cache/dfa_gb300_autotune.json), one entry per line:
//   "batch|<GPU>|states2^a|dfas2^b|kmaxc": [choice, ns_0, ns_1, ..., ns_11]
// Later calls with the same key run the remembered schedule directly.
struct TuneEntry {
  int choice = -1;
  std::vector<uint64_t> ns;   // device time per schedule (0 = not measured)
};
static std::mutex g_tune_mu;
static std::map<std::string, TuneEntry> g_tune;
static bool g_tune_loaded = false;

static std::string tune_path() {
  const char *p = getenv("DFA_AUTOTUNE_CACHE");
  if (p && *p) return p;
  const char *h = getenv("HOME");
  return std::string(h ? h : "/tmp") + "/.cache/dfa_gb300_autotune.json";
}

static void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  FILE *f = fopen(tune_path().c_str(), "r");
  if (!f) return;
  char key[256];
  char line[1024];
  while (fgets(line, sizeof line, f)) {
    int used = 0;
    if (sscanf(line, " \"%255[^\"]\" : [%n", key, &used) != 1 || used == 0) continue;
    TuneEntry e;
    const char *c = line + used;
    char *end = nullptr;
    const long ch = strtol(c, &end, 10);
    if (end == c || ch < 0 || ch >= kBatchSchedules) continue;
    e.choice = (int)ch;
    c = end;
    while (*c == ',' || *c == ' ') {
      ++c;
      const unsigned long long v = strtoull(c, &end, 10);
      if (end == c) break;
      e.ns.push_back(v);
      c = end;
    }
    g_tune[key] = e;
  }
  fclose(f);
}

static void tune_save() {
  const std::string p = tune_path();
  const size_t slash = p.rfind('/');
  if (slash != std::string::npos) mkdir(p.substr(0, slash).c_str(), 0755);   // best effort
  FILE *f = fopen(p.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t i = 0;
  for (auto &kv : g_tune) {
    fprintf(f, "  \"%s\": [%d", kv.first.c_str(), kv.second.choice);
    for (uint64_t v : kv.second.ns) fprintf(f, ", %llu", (unsigned long long)v);
    fprintf(f, "]%s\n", ++i < g_tune.size() ? "," : "");
  }
  fprintf(f, "}\n");
  fclose(f);
}

// The device's name, looked up once per device (a full property query per
// batched call would add host time to every call).
static std::string device_name(int dev) {
  static std::mutex mu;
  static std::map<int, std::string> names;
  std::lock_guard<std::mutex> lock(mu);
  auto it = names.find(dev);
  if (it != names.end()) return it->second;
  cudaDeviceProp prop;
  std::string name = cudaGetDeviceProperties(&prop, dev) == cudaSuccess ? std::string(prop.name) : "unknown";
  names[dev] = name;
  return name;
}

static std::string tune_key(uint64_t states, uint32_t count, uint32_t kmax) {
  int dev = 0;
  cudaGetDevice(&dev);
  return "batch|" + device_name(dev) + "|states2^" + std::to_string(ceil_log2(states + 1)) + "|dfas2^" +
         std::to_string(ceil_log2((uint64_t)count + 1)) + "|kmax" + std::to_string(kmax);
}

}  // namespace dfa

using namespace dfa;

// Checks a batch and its sizes; fills total states and the largest k.
static int check_batch(const dfa_t *dfas, uint32_t count, uint64_t *total, uint32_t *kmax) {
  if (!dfas || count == 0) return fail(DFA_EINVAL, "empty batch");
  *total = 0;
  *kmax = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const int rc = check_dfa(&dfas[i], "dfas[i]");
    if (rc != DFA_OK) return fail(rc, "dfa %u: %s", i, dfa_last_error());
    *total += dfas[i].n;
    *kmax = std::max(*kmax, dfas[i].k);
  }
  if (*total > DFA_MAX_STATES)
    return fail(DFA_EINVAL, "batch of %llu states exceeds %u", (unsigned long long)*total, DFA_MAX_STATES);
  return DFA_OK;
}

static size_t batch_workspace_impl(const dfa_t *dfas, uint32_t count, const BatchInputs &in) {
  uint64_t total;
  uint32_t kmax;
  if (check_batch(dfas, count, &total, &kmax) != DFA_OK) return 0;
  // the workspace serves every schedule (they differ by tile): one pass over
  // the DFAs, then the placement for each tile size
  BatchLayout L = batch_layout(dfas, count, in, 256u, nullptr, nullptr, nullptr);
  if (L.total_slots > 0xFFFFFFFFull) return 0;
  size_t most = 0;
  for (int t = 0; t < 3; ++t) {
    batch_place(L, count, 256u >> t, L.ntiles_by[t]);
    most = std::max(most, L.total);
  }
  return most;
}

static int run_batch(const dfa_t *dfas, uint32_t count, const BatchInputs &in, const dfa_opts &o,
                     uint32_t *block_out, dfa_result *res, char *ws, size_t ws_bytes, cudaStream_t st, int schedule,
                     uint64_t *device_ns) {
  const uint32_t vec = batch_schedule(schedule).vec, tile = batch_schedule(schedule).tile;
  std::vector<SegInfo> segs;
  std::vector<uint32_t> tile_off;
  std::vector<size_t> stage_off;
  const BatchLayout L = batch_layout(dfas, count, in, tile, &segs, &tile_off, &stage_off);
  if (L.total_slots > 0xFFFFFFFFull) return fail(DFA_EINVAL, "batch too large for 32-bit labels");
  if (ws_bytes < L.total) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
  cudaError_t e;
  if (in.packed) {
    // one copy per host buffer: the pieces are consecutive in both places
    size_t db = 0, ab = 0;
    for (uint32_t i = 0; i < count; ++i) {
      if (in.host[2 * i]) db += (size_t)dfas[i].k * dfas[i].n * 4;
      if (in.host[2 * i + 1]) ab += dfas[i].n;
    }
    const uint32_t first_d = [&] {
      for (uint32_t i = 0; i < count; ++i)
        if (dfas[i].k > 0) return i;
      return count;
    }();
    if (db > 0) {
      e = cudaMemcpyAsync(ws + L.stage + stage_off[2 * first_d], dfas[first_d].delta, db, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "copy packed delta to device");
    }
    if (ab > 0) {
      e = cudaMemcpyAsync(ws + L.stage + stage_off[1], dfas[0].accept, ab, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "copy packed accept to device");
    }
  }
  for (uint32_t i = 0; i < count; ++i) {
    const dfa_t &d = dfas[i];
    segs[i].delta = d.delta;
    segs[i].accept = d.accept;
    if (stage_off[2 * i] != SIZE_MAX) {
      char *p = ws + L.stage + stage_off[2 * i];
      if (!in.packed) {
        e = cudaMemcpyAsync(p, d.delta, (size_t)d.k * d.n * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy delta to device");
      }
      segs[i].delta = reinterpret_cast<const uint32_t *>(p);
    }
    if (stage_off[2 * i + 1] != SIZE_MAX) {
      char *p = ws + L.stage + stage_off[2 * i + 1];
      if (!in.packed) {
        e = cudaMemcpyAsync(p, d.accept, d.n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy accept to device");
      }
      segs[i].accept = reinterpret_cast<const uint8_t *>(p);
    }
  }
  const bool ho = !is_device_ptr(block_out);
  uint32_t *out_dev = ho ? reinterpret_cast<uint32_t *>(ws + L.out) : block_out;
  // block per DFA: every DFA whose refinement one block can hold (all in
  // shared memory, or up to 65,536 states with the labels in shared memory and
  // the table in the DFA's own table region), largest first
  std::vector<BatchSmallItem> items;
  size_t small_smem = 0;
  uint32_t coop_dfas = count;
  if (batch_schedule(schedule).blocks) {
    for (uint32_t i = 0; i < count; ++i) {
      uint32_t plan;
      size_t sm;
      BatchSmallItem it{};
      if (small_block_plan(segs[i].n, segs[i].k, &plan, &sm)) {
      } else if (medium_block_plan(segs[i].n, segs[i].log2S, &plan, &sm)) {
        it.table = reinterpret_cast<uint32_t *>(ws + L.table) + segs[i].table_off * 4;   // 4 words a slot
        it.scratch0 = reinterpret_cast<uint32_t *>(ws + L.lab0) + segs[i].state_off;
        it.scratch1 = reinterpret_cast<uint32_t *>(ws + L.lab1) + segs[i].state_off;
      } else {
        continue;
      }
      segs[i].small = 1u;
      --coop_dfas;
      small_smem = std::max(small_smem, sm);
      it.delta = segs[i].delta;
      it.accept = segs[i].accept;
      it.n = segs[i].n;
      it.k = segs[i].k;
      it.out = out_dev + segs[i].state_off;
      it.ss = reinterpret_cast<uint32_t *>(ws + L.ss) + (size_t)i * SS_WORDS;
      it.plan = plan;
      items.push_back(it);
    }
    std::stable_sort(items.begin(), items.end(),
                     [](const BatchSmallItem &x, const BatchSmallItem &y) { return x.n > y.n; });
    if (!items.empty()) {
      e = cudaMemcpyAsync(ws + L.items, items.data(), sizeof(BatchSmallItem) * items.size(), cudaMemcpyHostToDevice,
                          st);
      if (e != cudaSuccess) return cuda_fail(e, "copy block-per-DFA items");
    }
  }
  e = cudaMemcpyAsync(ws + L.segs, segs.data(), sizeof(SegInfo) * count, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy segment table");
  e = cudaMemcpyAsync(ws + L.tile_off, tile_off.data(), tile_off.size() * 4, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy tile offsets");
  e = cudaMemsetAsync(ws + L.cnt, 0, (size_t)count * 3 * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.ss, 0, (size_t)count * SS_WORDS * 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "clear batch bookkeeping");
  BatchArgs a{};
  a.segs = reinterpret_cast<const SegInfo *>(ws + L.segs);
  a.nsegs = count;
  a.tile_off = reinterpret_cast<const uint32_t *>(ws + L.tile_off);
  a.tiles = reinterpret_cast<Tile *>(ws + L.tiles);
  a.ntiles = L.ntiles;
  a.total_states = (uint32_t)L.total_states;
  a.total_slots = L.total_slots;
  a.lab[0] = reinterpret_cast<uint32_t *>(ws + L.lab0);
  a.lab[1] = reinterpret_cast<uint32_t *>(ws + L.lab1);
  a.tmp = reinterpret_cast<uint32_t *>(ws + L.tmp);
  a.tmp2 = reinterpret_cast<uint32_t *>(ws + L.tmp2);
  a.mbits = L.mbits;
  a.seen1 = reinterpret_cast<uint32_t *>(ws + L.seen1);
  a.seen2 = reinterpret_cast<uint32_t *>(ws + L.seen2);
  a.seen3 = reinterpret_cast<uint32_t *>(ws + L.seen3);
  a.seen4 = reinterpret_cast<uint32_t *>(ws + L.seen4);
  a.rep = reinterpret_cast<unsigned long long *>(ws + L.rep);
  a.dups = reinterpret_cast<uint32_t *>(ws + L.dups);
  a.dups2 = reinterpret_cast<uint32_t *>(ws + L.dups2);
  a.dups3 = reinterpret_cast<uint32_t *>(ws + L.dups3);
  a.table = reinterpret_cast<u128 *>(ws + L.table);
  a.bm[0] = reinterpret_cast<uint32_t *>(ws + L.bm0);
  a.bm[1] = reinterpret_cast<uint32_t *>(ws + L.bm1);
  a.minrep = reinterpret_cast<uint32_t *>(ws + L.minrep);
  a.tile_cnt = reinterpret_cast<uint32_t *>(ws + L.tile_cnt);
  a.tile_pre = reinterpret_cast<uint32_t *>(ws + L.tile_pre);
  a.partials = reinterpret_cast<uint32_t *>(ws + L.partials);
  a.out = out_dev;
  a.cnt = reinterpret_cast<uint32_t *>(ws + L.cnt);
  a.ss = reinterpret_cast<uint32_t *>(ws + L.ss);
  a.ctrl = reinterpret_cast<Ctrl *>(ws + L.ctrl);
  a.ebits = L.ebits;
  a.max_stages = L.max_stages;
  a.max_rounds = o.max_rounds;
  a.stop_discrete = (o.flags & DFA_FLAG_STOP_DISCRETE) ? 1u : 0u;
  a.vec = vec;
  a.tile = tile;
  a.timeout_ns = o.timeout_ns;
  a.barrier_ns = o.timeout_ns < 5000000000ull ? o.timeout_ns : 5000000000ull;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(e, "device attribute");
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_for(vec), kBatchThreads, 0)) !=
      cudaSuccess)
    return cuda_fail(e, "occupancy");
  const int grid = sms * (per_sm < 1 ? 1 : per_sm);
  if ((size_t)grid > kMaxGridB) return fail(DFA_ECUDA, "grid too large");
  // list capacity per block: the states of the block's tiles (tiles t = block + j * grid)
  if ((size_t)grid * (kBatchThreads / 32) > batch_max_warps())
    return fail(DFA_ECUDA, "grid larger than the workspace was sized for");
  a.dup_cap = (uint32_t)(((size_t)L.ntiles + grid - 1) / grid * tile);
  SmallLaunch sl{};
  if (!items.empty()) {
    if ((e = batch_small_setup()) != cudaSuccess) return cuda_fail(e, "shared memory of the block-per-DFA kernel");
    sl.items = reinterpret_cast<const BatchSmallItem *>(ws + L.items);
    sl.count = (uint32_t)items.size();
    sl.next = reinterpret_cast<uint32_t *>(ws + L.small_next);
    sl.smem = small_smem;
    sl.grid = (uint32_t)std::min<size_t>((size_t)sms, items.size());
    sl.o = &o;
  }
  e = launch_batch_graph(a, grid, coop_dfas > 0, items.empty() ? nullptr : &sl, st);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch of the batch kernel");
  Ctrl c{};
  std::vector<uint32_t> ss((size_t)count * SS_WORDS);
  e = cudaMemcpyAsync(&c, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ss.data(), a.ss, ss.size() * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "batch kernel");
  const int status = status_from_ctrl(c);
  if (device_ns) *device_ns = c.t_end - c.t_start;
  if (status != DFA_OK) return status;
  int overall = DFA_OK;
  for (uint32_t i = 0; i < count; ++i) {
    const uint32_t *w = ss.data() + (size_t)i * SS_WORDS;
    if (res) {
      res[i].num_blocks = w[SS_B];
      res[i].rounds_changed = w[SS_CHANGED];
      res[i].rounds_executed = w[SS_EXECUTED];
      res[i].status = w[SS_MAXED] ? DFA_EMAXROUNDS : DFA_OK;
      res[i].device_ns = c.t_end - c.t_start;
    }
    if (w[SS_MAXED]) overall = DFA_EMAXROUNDS;
  }
  if (ho) {
    e = cudaMemcpyAsync(block_out, a.out, L.total_states * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "copy blocks to host");
  }
  if (overall != DFA_OK) fail(overall, "max_rounds reached before the fixpoint for some DFA");
  return overall;
}

static int minimise_batch_impl(const dfa_t *dfas, uint32_t count, const BatchInputs &in, const dfa_opts *opts,
                               uint32_t *block_out, dfa_result *res, void *workspace, size_t ws_bytes, void *stream) {
  uint64_t total;
  uint32_t kmax;
  const int rc0 = check_batch(dfas, count, &total, &kmax);
  if (rc0 != DFA_OK) return rc0;
  if (!block_out) return fail(DFA_EINVAL, "block_out is NULL");
  if (!workspace || !aligned(workspace, 256)) return fail(DFA_EINVAL, "workspace NULL or not 256-byte aligned");
  const dfa_opts o = default_opts(opts);
  if (o.algo != DFA_ALGO_MOORE) return fail(DFA_EINVAL, "batches use signature refinement (algo 0)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char *ws = static_cast<char *>(workspace);
  if (o.schedule >= kBatchSchedules) return fail(DFA_EINVAL, "batch schedule %d beyond %d", o.schedule, kBatchSchedules - 1);
  if (o.schedule >= 0) return run_batch(dfas, count, in, o, block_out, res, ws, ws_bytes, st, o.schedule, nullptr);
  // autotune
  const std::string key = tune_key(total, count, kmax);
  int choice = -1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) choice = it->second.choice;
  }
  if (choice < 0 || choice >= kBatchSchedules) {
    TuneEntry e;
    e.ns.assign(kBatchSchedules, 0);
    uint64_t best = ~0ull;
    for (int sc = 0; sc < kBatchSchedules; ++sc) {
      uint64_t ns = 0;
      const int rc = run_batch(dfas, count, in, o, block_out, res, ws, ws_bytes, st, sc, &ns);
      if (rc != DFA_OK && rc != DFA_EMAXROUNDS) return rc;
      e.ns[sc] = ns;
      if (ns < best) {
        best = ns;
        choice = sc;
      }
    }
    e.choice = choice;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = e;
    tune_save();
  }
  return run_batch(dfas, count, in, o, block_out, res, ws, ws_bytes, st, choice, nullptr);
}

// dfa_t entries of a packed batch (pieces of the two buffers, in DFA order).
static int packed_dfas(uint32_t count, const uint32_t *n, const uint32_t *k, const uint32_t *delta,
                       const uint8_t *accept, std::vector<dfa_t> *dfas, BatchInputs *in) {
  if (count == 0) return fail(DFA_EINVAL, "empty batch");
  if (!n || !k) return fail(DFA_EINVAL, "n or k is NULL");
  if (!accept) return fail(DFA_EINVAL, "accept is NULL");
  dfas->resize(count);
  size_t od = 0, oa = 0;
  bool any_letters = false;
  for (uint32_t i = 0; i < count; ++i) {
    dfa_t &d = (*dfas)[i];
    d.n = n[i];
    d.k = k[i];
    d.start = 0;
    any_letters |= k[i] > 0;
    d.delta = k[i] > 0 && delta ? delta + od : nullptr;
    d.accept = accept + oa;
    od += (size_t)k[i] * n[i];
    oa += n[i];
  }
  if (any_letters && !delta) return fail(DFA_EINVAL, "delta is NULL");
  in->packed = true;
  const bool hd = any_letters && !is_device_ptr(delta), ha = !is_device_ptr(accept);
  in->host.resize((size_t)count * 2);
  for (uint32_t i = 0; i < count; ++i) {
    in->host[2 * i] = hd && k[i] > 0;
    in->host[2 * i + 1] = ha;
  }
  return DFA_OK;
}

extern "C" {

int dfa_batch_graph_stats(uint64_t *instantiations, uint64_t *updates) {
  if (instantiations) *instantiations = g_graph_instantiations.load(std::memory_order_relaxed);
  if (updates) *updates = g_graph_updates.load(std::memory_order_relaxed);
  return DFA_OK;
}

size_t dfa_batch_workspace_size(const dfa_t *dfas, uint32_t count, const dfa_opts *opts) {
  (void)opts;
  if (!dfas || count == 0) return 0;
  return batch_workspace_impl(dfas, count, classify_inputs(dfas, count));
}

int dfa_minimise_batch(const dfa_t *dfas, uint32_t count, const dfa_opts *opts, uint32_t *block_out,
                       dfa_result *res, void *workspace, size_t ws_bytes, void *stream) {
  if (!dfas || count == 0) return fail(DFA_EINVAL, "empty batch");
  uint64_t total;
  uint32_t kmax;
  const int rc = check_batch(dfas, count, &total, &kmax);
  if (rc != DFA_OK) return rc;
  return minimise_batch_impl(dfas, count, classify_inputs(dfas, count), opts, block_out, res, workspace, ws_bytes,
                             stream);
}

size_t dfa_batch_packed_workspace_size(uint32_t count, const uint32_t *n, const uint32_t *k, const uint32_t *delta,
                                       const uint8_t *accept, const dfa_opts *opts) {
  (void)opts;
  std::vector<dfa_t> dfas;
  BatchInputs in;
  if (packed_dfas(count, n, k, delta, accept, &dfas, &in) != DFA_OK) return 0;
  return batch_workspace_impl(dfas.data(), count, in);
}

int dfa_minimise_batch_packed(uint32_t count, const uint32_t *n, const uint32_t *k, const uint32_t *delta,
                              const uint8_t *accept, const dfa_opts *opts, uint32_t *block_out, dfa_result *res,
                              void *workspace, size_t ws_bytes, void *stream) {
  std::vector<dfa_t> dfas;
  BatchInputs in;
  const int rc = packed_dfas(count, n, k, delta, accept, &dfas, &in);
  if (rc != DFA_OK) return rc;
  return minimise_batch_impl(dfas.data(), count, in, opts, block_out, res, workspace, ws_bytes, stream);
}

}  // extern "C"
