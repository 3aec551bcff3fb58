// Serving: continuous batching of minimisation and equivalence requests (a
// serving form the paper does not have; each request is answered exactly as
// dfa_minimise / dfa_equivalent answer it alone).
//
// A server owns one device arena (hbm_budget_bytes, allocated once at create)
// managed by a first-fit allocator, one CUDA stream and one worker thread.
// Requests are copied in at submit and queued.  The worker admits requests in
// arrival order while a slot and arena space are free, places each one's
// arrays in the arena (an equivalence request is laid out as the disjoint
// union A ⊎ B, Section 4), and then advances every admitted request by one
// refinement round per step: one cooperative kernel runs the signature pass
// (Section 3.3) over the tiles of all admitted requests, each with its own
// table region, round number and epoch.  After the step the worker reads each
// request's block count, retires requests at their fixpoint (or, for
// equivalence with early exit, when the start states separate), numbers the
// finished partitions canonically on the device, copies results out, frees
// their arena space and admits waiting requests before the next step.  New
// requests therefore join while others are mid-refinement, and their work
// shares every launch.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_util.h"

namespace dfa {

static constexpr int kServeThreads = 512;
static constexpr uint32_t kServeTile = 256;
static constexpr size_t kServeMaxGrid = 8192;

enum : uint32_t { SM_DIRECT = 0, SM_FILTER = 1, SM_TABLE = 2 };

// One admitted request as a step sees it.  The host picks the round's mode
// (as dfa_minimise does: direct while the packed signature fits in log2S
// bits, filter once the previous round left at least n/64 blocks, table
// otherwise) and the plan of its table or filter keys.
struct ServeSeg {
  const uint32_t *delta;
  const uint8_t *accept;
  uint32_t n, k;
  uint32_t *lab[2];
  uint32_t *tmp, *tmp2;          // multi-stage slots; filter buckets and slots
  uint32_t *list, *list2;        // filter: listed states and their second buckets, per tile slice
  u128 *table;
  unsigned long long *rep;       // filter: (round, ~smallest state) per slot
  uint32_t *bm[2];               // direct: one bit per possible label (ping-pong)
  uint32_t log2S, wid, ebits;
  uint32_t mode, w;              // this round's mode; bits of the labels it reads
  StagePlan plan;                // plan of the table or filter keys, (w, log2S)
  uint32_t round;                // round this step executes (1-based)
  uint32_t epoch0;               // epoch of stage 0 of this round
  uint32_t tile0, ntiles;        // this request's tiles in the step's tile list
  const uint32_t *err;           // nonzero if the request's targets failed validation: skip it
  uint32_t track, sa, sb;
};

struct ServeOut {
  uint32_t count, seen, sep, ndup, err, pad[3];
};

struct ServeTile {
  uint32_t seg, start, len;
};

struct StepArgs {
  const ServeSeg *segs;
  uint32_t nsegs;
  ServeTile *tiles;              // listed by the kernel from each request's tile0 and ntiles
  uint32_t ntiles;
  uint32_t *tile_cnt;            // per tile: states listed by the filter
  ServeOut *outs;
  uint32_t max_stages, any_filter;
  uint32_t *seen1, *seen2, *seen3, *seen4;   // filter counters shared by the step's requests
  uint32_t mbits;
  Ctrl *ctrl;
  unsigned long long barrier_ns;
};

// Tiles are dealt per block (block b: tiles b, b + grid, ... in order, its
// warps taking the next from a shared counter reset after each barrier).
__device__ __forceinline__ uint32_t serve_next_tile(const StepArgs &A, uint32_t *s_next) {
  uint32_t i = 0;
  if ((threadIdx.x & 31u) == 0) i = atomicAdd(s_next, 1u);
  i = __shfl_sync(0xFFFFFFFFu, i, 0);
  const uint64_t t = (uint64_t)blockIdx.x + (uint64_t)i * gridDim.x;
  return t < A.ntiles ? (uint32_t)t : A.ntiles;
}

__device__ __forceinline__ void serve_start_tiles(uint32_t *s_next) {
  if (threadIdx.x == 0) *s_next = 0u;
  __syncthreads();
}

// Table round (stage `stage` of the request's plan) over one tile.
template <bool ROUND1>
__device__ __forceinline__ void serve_tile(const StepArgs &A, const ServeSeg &S, const ServeTile &T, uint32_t stage,
                                          bool last, CtaCache *cache) {
  const StagePlan &P = S.plan;
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
  const uint32_t epoch = S.epoch0 + stage;
  const unsigned long long etag = (unsigned long long)epoch << (64 - S.ebits);
  const uint32_t *src = S.lab[(S.round - 1) & 1];
  uint32_t *dst = S.lab[S.round & 1];
  const unsigned long long keep = policy_evict_last();
  uint32_t seen = 0, created_total = 0;
  for (uint32_t base = 0; base < T.len; base += 32u) {
    const bool valid = base + lane < T.len;
    const uint32_t q = T.start + (valid ? base + lane : 0u);
    u128 key[1] = {u128{0ull, 0ull}};
    uint32_t shift = 0;
    if (has_prev) {
      put_bits(key[0], S.tmp[q], 0);
      shift = P.carry;
    }
    uint32_t j = cbeg;
    if (j == 0) {
      uint32_t c;
      if (ROUND1) {
        c = S.accept[q] != 0;
        if (valid) seen |= c ? 1u : 2u;
      } else {
        c = src[q];
      }
      put_bits(key[0], c, shift);
      shift += bits;
      j = 1;
    }
    for (; j < cend; ++j) {
      const uint32_t d = S.delta[(size_t)(j - 1) * n + q];   // validated at admission
      const uint32_t c = ROUND1 ? (uint32_t)(S.accept[d] != 0) : ld_u32_hint(src + d, keep);
      put_bits(key[0], c, shift);
      shift += bits;
    }
    key[0].hi |= etag;
    uint32_t lab[1];
    uint32_t created = 0;
    warp_insert<1>(S.table, S.log2S, key, valid, S.ebits, epoch, lab, created, &A.ctrl->err, cache, T.seg);
    if (last) created_total += created;
    if (valid) {
      if (last) dst[q] = lab[0];
      else S.tmp[q] = lab[0];
    }
  }
  const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, created_total);
  if (lane == 0 && wsum) atomicAdd(&A.outs[T.seg].count, wsum);
  if (ROUND1) {
    const uint32_t wseen = __reduce_or_sync(0xFFFFFFFFu, seen);
    if (lane == 0 && wseen) atomicOr(&A.outs[T.seg].seen, wseen);
  }
}

// Direct round over one tile: the packed signature is the new label, counted
// through the request's bitmap (keys of at most 10 bits first in the warp's
// shared bitmap).  The tile also clears its share of the other bitmap, which
// the next round will use.
static constexpr uint32_t kServeWarpBits = 10;
template <bool ROUND1>
__device__ __forceinline__ void serve_direct_tile(const StepArgs &A, const ServeSeg &S, const ServeTile &T, uint32_t t,
                                                 uint32_t *wbm) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = S.n, k = S.k, w = S.w;
  const uint32_t *src = S.lab[(S.round - 1) & 1];
  uint32_t *dst = S.lab[S.round & 1];
  uint32_t *bm = S.bm[S.round & 1];
  const unsigned long long keep = policy_evict_last();
  const bool small = (k + 1) * w <= kServeWarpBits;
  if (small) {
    wbm[lane] = 0u;
    __syncwarp();
  }
  uint32_t seen = 0, created = 0;
  for (uint32_t base = 0; base < T.len; base += 32) {
    const bool valid = base + lane < T.len;
    const uint32_t q = T.start + (valid ? base + lane : 0u);
    uint32_t key;
    if (ROUND1) {
      key = S.accept[q] != 0;
      if (valid) seen |= key ? 1u : 2u;
    } else {
      key = src[q];
    }
    uint32_t shift = w;
    for (uint32_t a = 0; a < k; ++a) {
      const uint32_t d = S.delta[(size_t)a * n + q];   // validated at admission
      const uint32_t c = ROUND1 ? (uint32_t)(S.accept[d] != 0) : ld_u32_hint(src + d, keep);
      key |= c << shift;
      shift += w;
    }
    if (valid) dst[q] = key;
    const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, valid ? key : 0xFFFFFFFFu) & vm;
    if (valid && lane == (uint32_t)(__ffs(grp) - 1)) {
      const uint32_t bit = 1u << (key & 31u);
      if (small) atomicOr(&wbm[key >> 5], bit);
      else if (!(atomicOr(&bm[key >> 5], bit) & bit)) ++created;
    }
  }
  if (small) {
    __syncwarp();
    const uint32_t v = wbm[lane];
    if (v) created += __popc(v & ~atomicOr(&bm[lane], v));
    __syncwarp();
  }
  // this tile's share of the next round's bitmap
  const uint64_t words = ((1ull << S.log2S) + 31) / 32;
  const uint64_t per = (words + S.ntiles - 1) / S.ntiles, lo = (uint64_t)(t - S.tile0) * per;
  const uint64_t hi = lo + per < words ? lo + per : words;
  uint32_t *nb = S.bm[(S.round + 1) & 1];
  for (uint64_t i = lo + lane; i < hi; i += 32) nb[i] = 0u;
  const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, created);
  if (lane == 0 && wsum) atomicAdd(&A.outs[T.seg].count, wsum);
  if (ROUND1) {
    const uint32_t wseen = __reduce_or_sync(0xFFFFFFFFu, seen);
    if (lane == 0 && wseen) atomicOr(&A.outs[T.seg].seen, wseen);
  }
}

// Filter round, pass A over one tile: signature hash (the request's slot mixed
// in) into the shared 2-bit counters; both buckets kept per state.
__device__ __forceinline__ void serve_filter_a(const StepArgs &A, const ServeSeg &S, const ServeTile &T) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t n = S.n, k = S.k;
  const uint32_t *src = S.lab[(S.round - 1) & 1];
  const unsigned long long keep = policy_evict_last();
  for (uint32_t base = 0; base < T.len; base += 32) {
    if (base + lane >= T.len) continue;
    const uint32_t q = T.start + base + lane;
    unsigned long long h = hash_step(0x243F6A8885A308D3ull ^ ((unsigned long long)T.seg * 0xD6E8FEB86659FD93ull),
                                     src[q]);
    for (uint32_t a = 0; a < k; ++a) h = hash_step(h, ld_u32_hint(src + S.delta[(size_t)a * n + q], keep));
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    const uint32_t b = (uint32_t)(h >> (64 - A.mbits));
    const uint32_t bit = 1u << (b & 31u);
    if (atomicOr(&A.seen1[b >> 5], bit) & bit) atomicOr(&A.seen2[b >> 5], bit);
    S.tmp[q] = b;
    unsigned long long h2 = (h ^ 0x9E3779B97F4A7C15ull) * 0xc4ceb9fe1a85ec53ull;
    h2 ^= h2 >> 31;
    S.tmp2[q] = (uint32_t)(h2 >> (64 - (A.mbits - 1)));
  }
}

// Pass B over one tile: unique states keep their number as label; the others
// are listed in the tile's own slice of the request's list and enter the
// second filter.
__device__ __forceinline__ void serve_filter_b(const StepArgs &A, const ServeSeg &S, const ServeTile &T, uint32_t t) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t *dst = S.lab[S.round & 1];
  uint32_t *list = S.list + T.start, *list2 = S.list2 + T.start;
  uint32_t cursor = 0, uniq = 0;
  for (uint32_t base = 0; base < T.len; base += 32) {
    const bool valid = base + lane < T.len;
    const uint32_t q = T.start + base + lane;
    bool dup = false;
    uint32_t b2 = 0;
    if (valid) {
      const uint32_t b = S.tmp[q];
      dup = (A.seen2[b >> 5] >> (b & 31u)) & 1u;
      if (!dup) {
        dst[q] = q;
        ++uniq;
      } else {
        b2 = S.tmp2[q];
        const uint32_t bit = 1u << (b2 & 31u);
        if (atomicOr(&A.seen3[b2 >> 5], bit) & bit) atomicOr(&A.seen4[b2 >> 5], bit);
      }
    }
    const unsigned dm = __ballot_sync(0xFFFFFFFFu, dup);
    if (dup) {
      const uint32_t p = cursor + __popc(dm & ((1u << lane) - 1u));
      list[p] = q;
      list2[p] = b2;
    }
    cursor += __popc(dm);
  }
  const uint32_t u = __reduce_add_sync(0xFFFFFFFFu, uniq);
  if (lane == 0) {
    A.tile_cnt[t] = cursor;
    if (u) atomicAdd(&A.outs[T.seg].count, u);
    if (cursor) atomicAdd(&A.outs[T.seg].ndup, cursor);
  }
}

static constexpr uint32_t kServeResolved = 0x80000000u;   // listed state labelled by the second filter

// Pass F over a tile's listed slice: a listed state alone in its second bucket
// is unique too (marked resolved).
__device__ __forceinline__ void serve_filter_f(const StepArgs &A, const ServeSeg &S, const ServeTile &T, uint32_t t) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t *dst = S.lab[S.round & 1];
  uint32_t *list = S.list + T.start;
  const uint32_t *list2 = S.list2 + T.start;
  const uint32_t nd = A.tile_cnt[t];
  uint32_t uniq = 0;
  for (uint32_t i = lane; i < nd; i += 32) {
    const uint32_t b2 = list2[i];
    if (!((A.seen4[b2 >> 5] >> (b2 & 31u)) & 1u)) {
      const uint32_t q = list[i];
      dst[q] = q;
      list[i] = q | kServeResolved;
      ++uniq;
    }
  }
  const uint32_t u = __reduce_add_sync(0xFFFFFFFFu, uniq);
  if (lane == 0 && u) atomicAdd(&A.outs[T.seg].count, u);
}

// Pass D over a tile's listed slice: the states left insert their exact keys
// (tagged with the round's epoch; a signature wider than one key as its hash,
// joined only on a full comparison) and each slot keeps its smallest member.
__device__ __forceinline__ void serve_filter_d(const StepArgs &A, const ServeSeg &S, const ServeTile &T, uint32_t t) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t *list = S.list + T.start;
  const uint32_t nd = A.tile_cnt[t];
  const uint32_t *src = S.lab[(S.round - 1) & 1];
  const unsigned long long keep = policy_evict_last();
  const StagePlan &P = S.plan;
  const uint32_t mask = table_mask(S.log2S), w = S.w;
  for (uint32_t i = lane; i < nd; i += 32) {
    const uint32_t q = list[i];
    if (q & kServeResolved) continue;
    uint32_t slot[1] = {0u};
    if (P.stages == 1) {   // the whole signature is one exact key
      u128 key[1] = {u128{0ull, 0ull}};
      put_bits(key[0], src[q], 0);
      for (uint32_t a = 0; a < S.k; ++a) put_bits(key[0], ld_u32_hint(src + S.delta[(size_t)a * S.n + q], keep), (a + 1) * w);
      key[0].hi |= (unsigned long long)S.epoch0 << (64 - S.ebits);
      slot[0] = (uint32_t)(mix128(key[0]) >> 32) & mask;
      const bool want[1] = {true};
      bool is_new[1];
      table_insert_vec<1>(S.table, mask, key, S.ebits, S.epoch0, want, slot, is_new, &A.ctrl->err);
    } else {               // wider: signature hash plus full comparison with the slot's representative
      const SigEq eq{src, S.delta, S.n, S.k};
      slot[0] = hashed_insert(S.table, mask, S.ebits, S.epoch0, eq.hash(q), q, eq, &A.ctrl->err);
    }
    S.tmp[q] = slot[0];
    atomicMax(&S.rep[slot[0]], ((unsigned long long)S.round << 32) | (unsigned long long)(~q));
  }
}

// Pass C over a tile's listed slice: the states left take their slot's
// smallest member as label; each slot's smallest member counts a block.
__device__ __forceinline__ void serve_filter_c(const StepArgs &A, const ServeSeg &S, const ServeTile &T, uint32_t t) {
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t *dst = S.lab[S.round & 1];
  const uint32_t *list = S.list + T.start;
  const uint32_t nd = A.tile_cnt[t];
  uint32_t first = 0;
  for (uint32_t i = lane; i < nd; i += 32) {
    const uint32_t q = list[i];
    if (q & kServeResolved) continue;
    const uint32_t m = ~(uint32_t)S.rep[S.tmp[q]];
    dst[q] = m;
    first += m == q;
  }
  const uint32_t u = __reduce_add_sync(0xFFFFFFFFu, first);
  if (lane == 0 && u) atomicAdd(&A.outs[T.seg].count, u);
}

// One refinement round for every admitted request.
__global__ void __launch_bounds__(kServeThreads, 2) serve_step_kernel(StepArgs A) {
  __shared__ CtaCache cache;
  __shared__ uint32_t s_wbm[kServeThreads / 32][32];
  __shared__ uint32_t s_next;
  Ctrl *C = A.ctrl;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const uint32_t lane = threadIdx.x & 31u, gwarp = tid >> 5, nwarps = stride >> 5;
  if (tid == 0) C->deadline = gtimer() + A.barrier_ns;
  // tile list: request i's tiles are tile0 .. tile0 + ntiles - 1, one warp per request
  for (uint32_t i = gwarp; i < A.nsegs; i += nwarps) {
    const ServeSeg &S = A.segs[i];
    for (uint32_t j = lane; j < S.ntiles; j += 32) {
      const uint32_t start = j * kServeTile;
      A.tiles[S.tile0 + j] = ServeTile{i, start, S.n - start < kServeTile ? S.n - start : kServeTile};
    }
  }
  if (!grid_sync(C, A.barrier_ns)) return;
  for (uint32_t s = 0; s < A.max_stages; ++s) {
    cta_cache_clear(&cache);
    serve_start_tiles(&s_next);
    for (uint32_t t = serve_next_tile(A, &s_next); t < A.ntiles; t = serve_next_tile(A, &s_next)) {
      const ServeTile T = A.tiles[t];
      const ServeSeg &S = A.segs[T.seg];
      if (ld_relaxed(S.err)) continue;   // invalid targets: never followed
      const bool round1 = S.round == 1;
      if (S.mode == SM_DIRECT) {
        if (s != 0) continue;
        uint32_t *wbm = s_wbm[threadIdx.x >> 5];
        if (round1) serve_direct_tile<true>(A, S, T, t, wbm);
        else serve_direct_tile<false>(A, S, T, t, wbm);
      } else if (S.mode == SM_FILTER) {
        if (s == 0) serve_filter_a(A, S, T);
      } else {
        if (s >= S.plan.stages) continue;
        const bool last = s + 1 == S.plan.stages;
        if (round1) serve_tile<true>(A, S, T, s, last, &cache);
        else serve_tile<false>(A, S, T, s, last, &cache);
      }
    }
    if (!grid_sync(C, A.barrier_ns)) return;
    if (s == 0 && A.any_filter) {
      // filter passes B, F, D, C over the tiles of the requests in filter rounds
      for (int pass = 0; pass < 4; ++pass) {
        serve_start_tiles(&s_next);
        for (uint32_t t = serve_next_tile(A, &s_next); t < A.ntiles; t = serve_next_tile(A, &s_next)) {
          const ServeTile T = A.tiles[t];
          const ServeSeg &S = A.segs[T.seg];
          if (S.mode != SM_FILTER || ld_relaxed(S.err)) continue;
          if (pass == 0) serve_filter_b(A, S, T, t);
          else if (pass == 1) serve_filter_f(A, S, T, t);
          else if (pass == 2) serve_filter_d(A, S, T, t);
          else serve_filter_c(A, S, T, t);
        }
        if (pass == 3) {   // the counters start clean for the next filter step
          for (uint64_t i = tid; i < ((uint64_t)1 << A.mbits) / 32; i += stride) {
            A.seen1[i] = 0u;
            A.seen2[i] = 0u;
          }
          for (uint64_t i = tid; i < ((uint64_t)1 << A.mbits) / 64; i += stride) {
            A.seen3[i] = 0u;
            A.seen4[i] = 0u;
          }
        }
        if (!grid_sync(C, A.barrier_ns)) return;
      }
    }
  }
  for (uint32_t i = tid; i < A.nsegs; i += stride) {
    const ServeSeg &S = A.segs[i];
    A.outs[i].err = ld_relaxed(S.err);
    if (S.track && !A.outs[i].err) {
      const uint32_t *dst = S.lab[S.round & 1];
      A.outs[i].sep = dst[S.sa] != dst[S.sb];
    }
  }
}

// Canonical numbering of one finished request.
__global__ void __launch_bounds__(kServeThreads) serve_canon_kernel(CanonArgs a, uint32_t B) {
  __shared__ uint32_t s_red[kServeThreads / 32];
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctrl->deadline = gtimer() + a.barrier_ns;
  canonicalise(a, B, s_red);
}

// Validates the targets of one DFA placed in a table of n_u states per row.
__global__ void serve_check_kernel(const uint32_t *delta_u, uint32_t n_u, uint32_t k, uint32_t first, uint32_t count,
                                   uint32_t *err) {
  const uint64_t total = (uint64_t)k * count;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const uint32_t a = (uint32_t)(i / count), q = (uint32_t)(i % count);
    if (delta_u[(size_t)a * n_u + first + q] >= count) atomicOr(err, ERR_BAD_DELTA);
  }
}

// ------------------------------------------------------------------ arena
// First-fit allocator over [0, size) with coalescing of free neighbours.
class Arena {
 public:
  explicit Arena(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t *off) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

// ------------------------------------------------------------------ requests
struct Req {
  uint64_t ticket = 0;
  int kind = DFA_REQ_MINIMISE;
  dfa_opts o{};
  uint32_t nA = 0, nB = 0, k = 0, sA = 0, sB = 0, n = 0;
  std::vector<uint32_t> dA, dB;
  std::vector<uint8_t> aA, aB;
  // placement
  size_t off = 0, bytes = 0;
  bool early = false;             // arena space taken and inputs copied in at submit
  size_t o_delta = 0, o_acc = 0, o_lab0 = 0, o_lab1 = 0, o_tmp = 0, o_tmp2 = 0, o_list = 0, o_list2 = 0, o_table = 0,
         o_rep = 0, o_bm0 = 0, o_bm1 = 0, o_minrep = 0, o_flag = 0, o_out = 0, o_err = 0;
  uint32_t log2S = 0, wid = 1, ebits = 32;
  // progress
  uint32_t round = 0, changed = 0, prevB = 0, epoch = 0, lastB = 0, sep_round = 0xFFFFFFFFu;
  uint32_t w = 1;                 // bits of the current labels
  uint32_t mode = SM_TABLE;       // mode of the round in flight (or the last one)
  bool fok = true;                // filter rounds allowed
  bool finished = false, converged = false;
  int status = DFA_OK;
  uint32_t ntiles = 0;            // tiles of kServeTile states
  std::chrono::steady_clock::time_point t_submit, t_done;
  std::vector<uint32_t> blocks;
  dfa_result res{};
  int equivalent = -1;
};

static size_t req_layout(Req &r) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  const uint64_t n = r.n;
  r.log2S = ceil_log2(n * 2 < 64 ? 64 : n * 2);
  r.wid = ceil_log2(n) > 0 ? ceil_log2(n) : 1;
  // the epoch bits left free by every table or filter plan the request can take
  // (label widths: 1 bit, (k+1)^j while direct, then log2S or wid bits)
  r.ebits = 32;
  if (r.k > 0) {
    uint64_t w = 1;
    while ((uint64_t)(r.k + 1) * w <= r.log2S) w *= r.k + 1;
    for (const uint64_t x : {w, (uint64_t)r.log2S, (uint64_t)r.wid})
      r.ebits = std::min(r.ebits, make_plan(r.k, (uint32_t)x, r.log2S).ebits);
  }
  const size_t S = (size_t)1 << r.log2S;
  r.o_err = take(4);
  r.o_delta = take((size_t)r.k * n * 4);
  r.o_acc = take(n);
  r.o_lab0 = take(n * 4);
  r.o_lab1 = take(n * 4);
  r.o_tmp = take(n * 4);
  r.o_tmp2 = take(n * 4);
  r.o_list = take(n * 4);
  r.o_list2 = take(n * 4);
  r.o_table = take(S * 16);
  r.o_rep = take(S * 8);
  r.o_bm0 = take(S / 8);
  r.o_bm1 = take(S / 8);
  r.o_minrep = take(((size_t)1 << r.log2S) * 4);
  r.o_flag = take(n);
  r.o_out = take(n * 4);
  return off;
}

// Serving scratch (allocated once): control block, scan partials, per-slot
// outputs and step descriptors, the step's tile list and per-tile listed
// counts, and the filter counters (2^kServeMaxMbits buckets at most).
static constexpr uint32_t kServeMaxMbits = 28;
struct ServeScratch {
  size_t ctrl, partials, outs, segs, tiles, tile_cnt, seen1, seen2, seen3, seen4, total;
  size_t max_tiles;
};

static ServeScratch serve_scratch_layout(uint32_t max_slots, size_t max_tiles) {
  ServeScratch L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  L.max_tiles = max_tiles;
  L.ctrl = take(sizeof(Ctrl));
  L.partials = take(kServeMaxGrid * 4);
  L.outs = take((size_t)max_slots * sizeof(ServeOut));
  L.segs = take((size_t)max_slots * sizeof(ServeSeg));
  L.tiles = take(max_tiles * sizeof(ServeTile));
  L.tile_cnt = take(max_tiles * 4);
  L.seen1 = take(((size_t)1 << kServeMaxMbits) / 8);
  L.seen2 = take(((size_t)1 << kServeMaxMbits) / 8);
  L.seen3 = take(((size_t)1 << kServeMaxMbits) / 16);
  L.seen4 = take(((size_t)1 << kServeMaxMbits) / 16);
  L.total = off;
  return L;
}

}  // namespace dfa

using namespace dfa;

struct dfa_server {
  int device = 0;
  size_t budget = 0;
  uint32_t max_slots = 0;
  char *arena_base = nullptr;
  std::unique_ptr<Arena> arena;
  cudaStream_t stream = nullptr;
  cudaStream_t in_stream = nullptr;   // submissions' copies into the arena
  // device scratch for steps and canonical numbering (allocated once)
  char *scratch = nullptr;
  ServeScratch sl{};
  ServeSeg *segs_pinned = nullptr;
  ServeOut *outs_pinned = nullptr;
  int grid_step = 0, grid_canon = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::vector<std::shared_ptr<Req>> active;
  std::unordered_map<uint64_t, std::shared_ptr<Req>> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  std::vector<double> latencies_us;
  std::chrono::steady_clock::time_point first_submit, last_done;
  bool any_submit = false;
  std::string worker_error;
  // counters (under mu): steps run, requests and states advanced by one round, host time in steps
  uint64_t steps = 0, request_rounds = 0, state_rounds = 0;
  bool front_blocked = false;   // a request held on the host waits for arena space (under mu)
  uint64_t mode_state_rounds[3] = {0, 0, 0};   // by round mode: direct, filter, table
  double step_us = 0.0;
};

namespace dfa {

static constexpr uint32_t kServeMaxSlots = 4096;

static void finish_req(dfa_server *s, const std::shared_ptr<Req> &r, int status) {
  r->status = status;
  r->finished = true;
  r->t_done = std::chrono::steady_clock::now();
  r->res.num_blocks = r->lastB;
  r->res.rounds_changed = r->changed;
  r->res.rounds_executed = r->round;
  r->res.status = status;
  if (r->kind == DFA_REQ_EQUIVALENT && status == DFA_OK) r->equivalent = r->sep_round == 0xFFFFFFFFu ? 1 : 0;
  r->dA.clear();
  r->dA.shrink_to_fit();
  r->dB.clear();
  r->dB.shrink_to_fit();
  r->aA.clear();
  r->aB.clear();
  s->arena->release(r->off, r->bytes);
  s->latencies_us.push_back(std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
  s->last_done = r->t_done;
}

// Places an admitted request in the arena and copies its data in.
static cudaError_t place_req(dfa_server *s, Req &r) {
  char *b = s->arena_base + r.off;
  cudaStream_t st = s->stream;
  cudaError_t e = cudaMemsetAsync(b + r.o_err, 0, 4, st);
  const uint32_t n = r.n;
  if (!r.early) {   // inputs held on the host since submit
    if (e == cudaSuccess && r.k > 0)
      e = cudaMemcpy2DAsync(b + r.o_delta, (size_t)n * 4, r.dA.data(), (size_t)r.nA * 4, (size_t)r.nA * 4, r.k,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && r.k > 0 && r.nB > 0)
      e = cudaMemcpy2DAsync(b + r.o_delta + (size_t)r.nA * 4, (size_t)n * 4, r.dB.data(), (size_t)r.nB * 4,
                            (size_t)r.nB * 4, r.k, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + r.o_acc, r.aA.data(), r.nA, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && r.nB > 0)
      e = cudaMemcpyAsync(b + r.o_acc + r.nA, r.aB.data(), r.nB, cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return e;
  uint32_t *du = reinterpret_cast<uint32_t *>(b + r.o_delta);
  uint32_t *err = reinterpret_cast<uint32_t *>(b + r.o_err);
  if (r.k > 0) {
    serve_check_kernel<<<1216, 256, 0, st>>>(du, n, r.k, 0, r.nA, err);
    if (r.nB > 0) {
      e = launch_offset_targets(du, n, r.k, r.nA, r.nB, r.nA, err, st);
      if (e != cudaSuccess) return e;
    }
  }
  const size_t S = (size_t)1 << r.log2S;
  e = cudaMemsetAsync(b + r.o_table, 0, S * 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + r.o_rep, 0, S * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + r.o_bm0, 0, S / 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + r.o_bm1, 0, S / 8, st);
  if (e != cudaSuccess) return e;
  r.ntiles = (n + kServeTile - 1) / kServeTile;
  r.round = 0;
  r.epoch = 0;
  r.w = 1;
  r.fok = true;
  return cudaGetLastError();
}

static void worker_main(dfa_server *s) {
  cudaSetDevice(s->device);
  char *sc = s->scratch;
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(sc + s->sl.ctrl);
  uint32_t *partials = reinterpret_cast<uint32_t *>(sc + s->sl.partials);
  ServeOut *outs = reinterpret_cast<ServeOut *>(sc + s->sl.outs);
  ServeSeg *segs_d = reinterpret_cast<ServeSeg *>(sc + s->sl.segs);
  ServeTile *tiles_d = reinterpret_cast<ServeTile *>(sc + s->sl.tiles);
  uint32_t *tile_cnt = reinterpret_cast<uint32_t *>(sc + s->sl.tile_cnt);
  const size_t max_tiles = s->sl.max_tiles;
  ServeSeg *segs_h = s->segs_pinned;   // pinned: the step's copies are truly asynchronous
  ServeOut *outs_h = s->outs_pinned;
  while (true) {
    std::vector<std::shared_ptr<Req>> admitted;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      if (s->active.empty())
        s->cv_work.wait_for(lock, std::chrono::milliseconds(50), [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) break;
      // admission in arrival order while a slot and arena space are free.  A
      // request held on the host that finds no arena space blocks the requests
      // held on the host behind it, but not those already placed in the arena
      // at submit (they need no space; were they to wait, the space they hold
      // could never come back and the front could wait forever); while the
      // front is blocked, submissions stop taking arena space early.
      size_t tiles_now = 0;
      for (auto &r : s->active) tiles_now += r->ntiles;
      bool blocked = false;
      for (auto it = s->queue.begin(); it != s->queue.end() && s->active.size() < s->max_slots;) {
        auto r = *it;
        const size_t want_tiles = (r->n + kServeTile - 1) / kServeTile;
        if (tiles_now + want_tiles > max_tiles) break;
        if (!r->early) {
          size_t off;
          if (blocked || !s->arena->alloc(r->bytes, &off)) {
            blocked = true;
            ++it;
            continue;
          }
          r->off = off;
        }
        it = s->queue.erase(it);
        s->active.push_back(r);
        admitted.push_back(r);
        tiles_now += want_tiles;
      }
      s->front_blocked = blocked;
    }
    for (auto &r : admitted) {
      const cudaError_t e = place_req(s, *r);
      if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->worker_error = cudaGetErrorString(e);
        finish_req(s, r, DFA_ECUDA);
      }
    }
    // (requests whose targets fail validation are skipped by the step kernel and
    // finish with DFA_EINVAL when the step's outputs come back)
    std::vector<std::shared_ptr<Req>> act;
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](auto &r) { return r->finished; }),
                      s->active.end());
      act = s->active;
      if (!act.empty() || !admitted.empty()) s->cv_done.notify_all();
    }
    if (act.empty()) continue;
    // ---- one round for every admitted request
    const auto t_step = std::chrono::steady_clock::now();
    uint32_t ntiles = 0;
    uint32_t max_stages = 1, any_filter = 0;
    uint64_t filter_states = 0;
    for (uint32_t i = 0; i < act.size(); ++i) {
      Req &r = *act[i];
      r.round += 1;
      // the round's mode, as dfa_minimise chooses it
      if ((uint64_t)(r.k + 1) * r.w <= r.log2S) r.mode = SM_DIRECT;
      else if (r.round > 1 && r.fok &&
               ((uint64_t)r.prevB * 64 >= r.n ||
                (r.kind == DFA_REQ_MINIMISE && signatures_sparse(r.k, r.prevB, r.n))))
        r.mode = SM_FILTER;   // most signatures unique (a union's states come in pairs: not predicted)
      else r.mode = SM_TABLE;
      const StagePlan P = make_plan(r.k, r.w, r.log2S);
      const uint32_t stages = r.mode == SM_DIRECT ? 0u : P.stages;
      const uint32_t emax = r.ebits >= 32 ? 0xFFFFFFFFu : ((1u << r.ebits) - 1u);
      if ((uint64_t)r.epoch + stages > emax) {   // epochs would wrap: clear this request's table
        cudaMemsetAsync(s->arena_base + r.off + r.o_table, 0, ((size_t)1 << r.log2S) * 16, s->stream);
        r.epoch = 0;
      }
      ServeSeg g{};
      char *b = s->arena_base + r.off;
      g.delta = reinterpret_cast<const uint32_t *>(b + r.o_delta);
      g.accept = reinterpret_cast<const uint8_t *>(b + r.o_acc);
      g.n = r.n;
      g.k = r.k;
      g.lab[0] = reinterpret_cast<uint32_t *>(b + r.o_lab0);
      g.lab[1] = reinterpret_cast<uint32_t *>(b + r.o_lab1);
      g.tmp = reinterpret_cast<uint32_t *>(b + r.o_tmp);
      g.tmp2 = reinterpret_cast<uint32_t *>(b + r.o_tmp2);
      g.list = reinterpret_cast<uint32_t *>(b + r.o_list);
      g.list2 = reinterpret_cast<uint32_t *>(b + r.o_list2);
      g.table = reinterpret_cast<u128 *>(b + r.o_table);
      g.rep = reinterpret_cast<unsigned long long *>(b + r.o_rep);
      g.bm[0] = reinterpret_cast<uint32_t *>(b + r.o_bm0);
      g.bm[1] = reinterpret_cast<uint32_t *>(b + r.o_bm1);
      g.log2S = r.log2S;
      g.wid = r.wid;
      g.ebits = r.ebits;
      g.mode = r.mode;
      g.w = r.w;
      g.plan = P;
      g.round = r.round;
      g.epoch0 = r.epoch + 1;
      g.tile0 = ntiles;
      g.ntiles = r.ntiles;
      g.err = reinterpret_cast<const uint32_t *>(b + r.o_err);
      g.track = r.kind == DFA_REQ_EQUIVALENT;
      g.sa = r.sA;
      g.sb = r.nA + r.sB;
      r.epoch += stages;
      if (r.mode == SM_TABLE) max_stages = std::max(max_stages, P.stages);
      if (r.mode == SM_FILTER) {
        any_filter = 1;
        filter_states += r.n;
      }
      segs_h[i] = g;
      ntiles += r.ntiles;
    }
    cudaMemcpyAsync(segs_d, segs_h, act.size() * sizeof(ServeSeg), cudaMemcpyHostToDevice, s->stream);
    cudaMemsetAsync(outs, 0, act.size() * sizeof(ServeOut), s->stream);
    cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s->stream);
    StepArgs a{};
    a.segs = segs_d;
    a.nsegs = (uint32_t)act.size();
    a.tiles = tiles_d;
    a.ntiles = ntiles;
    a.outs = outs;
    a.tile_cnt = tile_cnt;
    a.max_stages = max_stages;
    a.any_filter = any_filter;
    a.seen1 = reinterpret_cast<uint32_t *>(sc + s->sl.seen1);
    a.seen2 = reinterpret_cast<uint32_t *>(sc + s->sl.seen2);
    a.seen3 = reinterpret_cast<uint32_t *>(sc + s->sl.seen3);
    a.seen4 = reinterpret_cast<uint32_t *>(sc + s->sl.seen4);
    a.mbits = std::min<uint32_t>(kServeMaxMbits, std::max<uint32_t>(12, ceil_log2(filter_states + 1) + 2));
    a.ctrl = ctrl;
    a.barrier_ns = 5000000000ull;
    void *params[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)serve_step_kernel, dim3(s->grid_step),
                                                dim3(kServeThreads), params, 0, s->stream);
    Ctrl ch{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(outs_h, outs, act.size() * sizeof(ServeOut), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ch, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    {
      uint64_t states = 0, by_mode[3] = {0, 0, 0};
      for (auto &r : act) {
        states += r->n;
        by_mode[r->mode == SM_DIRECT ? 0 : r->mode == SM_FILTER ? 1 : 2] += r->n;
      }
      std::lock_guard<std::mutex> lock(s->mu);
      for (int m = 0; m < 3; ++m) s->mode_state_rounds[m] += by_mode[m];
      s->steps += 1;
      s->request_rounds += act.size();
      s->state_rounds += states;
      s->step_us += std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t_step).count();
    }
    if (e != cudaSuccess || ch.err) {
      std::lock_guard<std::mutex> lock(s->mu);
      s->worker_error = e != cudaSuccess ? cudaGetErrorString(e) : "device-side error in a serving step";
      for (auto &r : act)
        if (!r->finished) finish_req(s, r, e != cudaSuccess ? DFA_ECUDA : (ch.err & ERR_TIMEOUT ? DFA_ETIMEOUT : DFA_ECUDA));
      s->cv_done.notify_all();
      continue;
    }
    // ---- bookkeeping; finished requests are numbered canonically and copied out
    std::vector<std::shared_ptr<Req>> done;
    for (uint32_t i = 0; i < act.size(); ++i) {
      Req &r = *act[i];
      const ServeOut &o = outs_h[i];
      if (o.err) {   // targets out of range: the request never ran
        r.status = DFA_EINVAL;
        done.push_back(act[i]);
        continue;
      }
      const uint32_t prev = r.round == 1 ? (uint32_t)__builtin_popcount(o.seen) : r.prevB;
      const uint32_t B = o.count;
      r.lastB = B;
      // width of this round's labels; a filter round that listed most states
      // (large blocks) hands later rounds to the table
      r.w = r.mode == SM_DIRECT ? (r.k + 1) * r.w : r.mode == SM_FILTER ? r.wid : r.log2S;
      if (r.mode == SM_FILTER && (uint64_t)o.ndup * 2 > r.n) r.fok = false;
      const bool grew = B != prev;
      if (grew) r.changed += 1;
      bool fin = false;
      int st = DFA_OK;
      if (r.kind == DFA_REQ_EQUIVALENT && r.sep_round == 0xFFFFFFFFu) {
        if (o.sep) {
          r.sep_round = r.round;
          if (r.o.flags & DFA_FLAG_EARLY_EXIT) fin = true;
        }
      }
      if (!grew) {
        fin = true;
        r.converged = true;
      } else if (r.o.max_rounds != 0u && r.round >= r.o.max_rounds && !fin) {
        fin = true;
        st = DFA_EMAXROUNDS;
      }
      r.prevB = B;
      if (fin) {
        r.status = st;
        done.push_back(act[i]);
      }
    }
    for (auto &rp : done) {
      Req &r = *rp;
      if (r.kind == DFA_REQ_MINIMISE && (r.status == DFA_OK || r.status == DFA_EMAXROUNDS)) {   // labels valid
        char *b = s->arena_base + r.off;
        CanonArgs ca{r.n, reinterpret_cast<uint32_t *>(b + (r.round & 1 ? r.o_lab1 : r.o_lab0)),
                     (size_t)1 << r.log2S, reinterpret_cast<uint32_t *>(b + r.o_minrep),
                     reinterpret_cast<uint8_t *>(b + r.o_flag), partials, reinterpret_cast<uint32_t *>(b + r.o_out),
                     ctrl, 5000000000ull, r.mode == SM_FILTER ? 1u : 0u};   // filter labels: smallest members
        uint32_t B = r.lastB;
        cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s->stream);
        void *cp[] = {&ca, &B};
        e = cudaLaunchCooperativeKernel((const void *)serve_canon_kernel, dim3(s->grid_canon), dim3(kServeThreads), cp,
                                        0, s->stream);
        r.blocks.resize(r.n);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(r.blocks.data(), b + r.o_out, (size_t)r.n * 4, cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) r.status = DFA_ECUDA;
      }
    }
    {
      std::lock_guard<std::mutex> lock(s->mu);
      for (auto &rp : done) finish_req(s, rp, rp->status);
      s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](auto &r) { return r->finished; }),
                      s->active.end());
      if (!done.empty()) s->cv_done.notify_all();
    }
  }
}

// Copies a request's inputs straight into its arena region (A's columns
// first, then B's; B's targets are offset on the device at admission) on the
// server's input stream, and waits for the copies so the caller may free them.
static int copy_in_device(dfa_server *s, Req &r, const dfa_t *a, const dfa_t *b) {
  char *base = s->arena_base + r.off;
  cudaStream_t st = s->in_stream;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaError_t e = cudaSetDevice(s->device);
  if (r.k > 0)
    e = cudaMemcpy2DAsync(base + r.o_delta, (size_t)r.n * 4, a->delta, (size_t)r.nA * 4, (size_t)r.nA * 4, r.k,
                          cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(base + r.o_acc, a->accept, r.nA, cudaMemcpyDefault, st);
  if (b) {
    if (e == cudaSuccess && r.k > 0)
      e = cudaMemcpy2DAsync(base + r.o_delta + (size_t)r.nA * 4, (size_t)r.n * 4, b->delta, (size_t)r.nB * 4,
                            (size_t)r.nB * 4, r.k, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + r.o_acc + r.nA, b->accept, r.nB, cudaMemcpyDefault, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaSetDevice(prev);
  return e == cudaSuccess ? DFA_OK : cuda_fail(e, "copy request in");
}

// Copies a request's arrays to host vectors (it waits for arena space) on the
// server's input stream: a synchronous cudaMemcpy would run on the legacy
// default stream and wait behind unrelated work.
static int copy_dfa_in(dfa_server *s, const dfa_t *d, std::vector<uint32_t> &delta, std::vector<uint8_t> &acc) {
  delta.resize((size_t)d->k * d->n);
  acc.resize(d->n);
  cudaError_t e = cudaSuccess;
  if (d->k > 0) e = cudaMemcpyAsync(delta.data(), d->delta, delta.size() * 4, cudaMemcpyDefault, s->in_stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(acc.data(), d->accept, d->n, cudaMemcpyDefault, s->in_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->in_stream);
  return e == cudaSuccess ? DFA_OK : cuda_fail(e, "copy request in");
}

// One byte of a host or device array: host memory is read directly, device
// memory through the server's input stream.
static int read_byte(dfa_server *s, const uint8_t *p, uint8_t *out) {
  if (!is_device_ptr(p)) {
    *out = *p;
    return DFA_OK;
  }
  cudaError_t e = cudaMemcpyAsync(out, p, 1, cudaMemcpyDeviceToHost, s->in_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->in_stream);
  return e == cudaSuccess ? DFA_OK : cuda_fail(e, "read start acceptance");
}

}  // namespace dfa

extern "C" {

int dfa_serve_create(dfa_server **out, size_t hbm_budget_bytes, uint32_t max_slots, int device) {
  if (!out) return fail(DFA_EINVAL, "out is NULL");
  if (max_slots == 0 || max_slots > kServeMaxSlots) return fail(DFA_EINVAL, "max_slots must be 1..%u", kServeMaxSlots);
  if (hbm_budget_bytes < (1u << 20)) return fail(DFA_EINVAL, "HBM budget below 1 MiB");
  auto s = std::make_unique<dfa_server>();
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  const size_t max_tiles = hbm_budget_bytes / (kServeTile * 16) + max_slots + 1024;
  s->sl = serve_scratch_layout(max_slots, max_tiles);
  e = cudaMalloc(&s->arena_base, hbm_budget_bytes);
  if (e != cudaSuccess) return fail(DFA_ENOMEM, "cannot allocate the %zu-byte arena: %s", hbm_budget_bytes,
                                    cudaGetErrorString(e));
  e = cudaMalloc(&s->scratch, s->sl.total);
  if (e != cudaSuccess) {
    cudaFree(s->arena_base);
    return fail(DFA_ENOMEM, "cannot allocate serving scratch: %s", cudaGetErrorString(e));
  }
  e = cudaMallocHost(&s->segs_pinned, (size_t)max_slots * sizeof(ServeSeg));
  if (e == cudaSuccess) e = cudaMallocHost(&s->outs_pinned, (size_t)max_slots * sizeof(ServeOut));
  if (e != cudaSuccess) return fail(DFA_ENOMEM, "cannot allocate pinned step buffers: %s", cudaGetErrorString(e));
  // the filter counters start clean (each filter step clears what it used)
  e = cudaMemset(s->scratch + s->sl.seen1, 0, s->sl.total - s->sl.seen1);
  if (e != cudaSuccess) return cuda_fail(e, "clear serving scratch");
  s->arena = std::make_unique<Arena>(hbm_budget_bytes);
  e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->in_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, serve_step_kernel, kServeThreads, 0);
  s->grid_step = sms * std::max(per, 1);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, serve_canon_kernel, kServeThreads, 0);
  s->grid_canon = std::min<int>(sms * std::max(per, 1), (int)kServeMaxGrid);
  dfa_server *raw = s.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return DFA_OK;
}

int dfa_serve_submit(dfa_server *s, int kind, const dfa_t *a, const dfa_t *b, const dfa_opts *opts,
                     uint64_t *ticket) {
  if (!s || !ticket) return fail(DFA_EINVAL, "server or ticket is NULL");
  if (kind != DFA_REQ_MINIMISE && kind != DFA_REQ_EQUIVALENT) return fail(DFA_EINVAL, "unknown request kind %d", kind);
  int rc = check_dfa(a, "a");
  if (rc != DFA_OK) return rc;
  auto r = std::make_shared<Req>();
  r->kind = kind;
  r->o = default_opts(opts);
  if (r->o.algo != DFA_ALGO_MOORE) return fail(DFA_EINVAL, "serving uses signature refinement (algo 0)");
  r->nA = a->n;
  r->k = a->k;
  r->sA = a->start;
  if (kind == DFA_REQ_EQUIVALENT) {
    rc = check_dfa(b, "b");
    if (rc != DFA_OK) return rc;
    if (b->k != a->k) return fail(DFA_EINVAL, "alphabets differ: k_A = %u, k_B = %u", a->k, b->k);
    if ((uint64_t)a->n + b->n > DFA_MAX_STATES) return fail(DFA_EINVAL, "n_A + n_B too large");
    r->nB = b->n;
    r->sB = b->start;
  }
  r->n = r->nA + r->nB;
  r->bytes = req_layout(*r);
  if (r->bytes > s->budget) return fail(DFA_ENOMEM, "request needs %zu bytes, budget is %zu", r->bytes, s->budget);
  // round 0 of an equivalence request: the empty word already separates start
  // states of different acceptance; with early exit no round is needed
  uint8_t acc_a = 0, acc_b = 0;
  if (kind == DFA_REQ_EQUIVALENT) {
    const int e = read_byte(s, a->accept + a->start, &acc_a) != DFA_OK ? DFA_ECUDA
                                                                       : read_byte(s, b->accept + b->start, &acc_b);
    if (e != DFA_OK) return e;
  }
  const bool sep0 = kind == DFA_REQ_EQUIVALENT && ((acc_a != 0) != (acc_b != 0));
  const bool instant = sep0 && (r->o.flags & DFA_FLAG_EARLY_EXIT);
  if (!instant) {
    // inputs go straight into the request's arena region when it has room now;
    // otherwise they wait on the host until admission
    {
      std::lock_guard<std::mutex> lock(s->mu);
      size_t off;
      if (!s->front_blocked && s->arena->alloc(r->bytes, &off)) {   // the blocked front goes first
        r->off = off;
        r->early = true;
      }
    }
    if (r->early) {
      rc = copy_in_device(s, *r, a, kind == DFA_REQ_EQUIVALENT ? b : nullptr);
      if (rc != DFA_OK) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->arena->release(r->off, r->bytes);
        return rc;
      }
    } else {
      rc = copy_dfa_in(s, a, r->dA, r->aA);
      if (rc != DFA_OK) return rc;
      if (kind == DFA_REQ_EQUIVALENT) {
        rc = copy_dfa_in(s, b, r->dB, r->aB);
        if (rc != DFA_OK) return rc;
      }
    }
  }
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lock(s->mu);
    r->ticket = s->next_ticket++;
    if (!s->any_submit) {
      s->first_submit = r->t_submit;
      s->any_submit = true;
    }
    s->all[r->ticket] = r;
    if (sep0) r->sep_round = 0;
    if (instant) {
      r->finished = true;
      r->status = DFA_OK;
      r->equivalent = 0;
      r->t_done = std::chrono::steady_clock::now();
      r->res = dfa_result{2u, 0u, 0u, DFA_OK, 0ull};
      r->dA.clear();
      r->dB.clear();
      s->latencies_us.push_back(std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count());
      s->last_done = r->t_done;
      s->cv_done.notify_all();
    } else {
      s->queue.push_back(r);
    }
  }
  s->cv_work.notify_one();
  *ticket = r->ticket;
  return DFA_OK;
}

static int take_result(dfa_server *s, std::unordered_map<uint64_t, std::shared_ptr<Req>>::iterator it, dfa_result *res,
                       int *equivalent, uint32_t *block_out) {
  auto r = it->second;
  if (res) *res = r->res;
  if (equivalent) *equivalent = r->equivalent;
  if (block_out && !r->blocks.empty()) memcpy(block_out, r->blocks.data(), r->blocks.size() * 4);
  const int st = r->status;
  s->all.erase(it);
  if (st != DFA_OK) fail(st, "request finished with status %d", st);
  return st;
}

int dfa_serve_poll(dfa_server *s, uint64_t ticket, dfa_result *res, int *equivalent, uint32_t *block_out) {
  if (!s) return fail(DFA_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(DFA_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  if (!it->second->finished) return DFA_EBUSY;
  return take_result(s, it, res, equivalent, block_out);
}

int dfa_serve_wait(dfa_server *s, uint64_t ticket, uint64_t timeout_ns, dfa_result *res, int *equivalent,
                   uint32_t *block_out) {
  if (!s) return fail(DFA_EINVAL, "server is NULL");
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(DFA_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
  auto r = it->second;
  auto pred = [&] { return r->finished; };
  if (timeout_ns == 0) {
    s->cv_done.wait(lock, pred);
  } else if (!s->cv_done.wait_for(lock, std::chrono::nanoseconds(timeout_ns), pred)) {
    return fail(DFA_ETIMEOUT, "request %llu not finished within the wait limit", (unsigned long long)ticket);
  }
  it = s->all.find(ticket);
  return take_result(s, it, res, equivalent, block_out);
}

int dfa_serve_stats(dfa_server *s, double *p50_us, double *p99_us, double *throughput_rps) {
  if (!s) return fail(DFA_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  std::vector<double> v = s->latencies_us;
  if (v.empty()) {
    if (p50_us) *p50_us = 0;
    if (p99_us) *p99_us = 0;
    if (throughput_rps) *throughput_rps = 0;
    return DFA_OK;
  }
  std::sort(v.begin(), v.end());
  auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
  if (p50_us) *p50_us = pct(0.50);
  if (p99_us) *p99_us = pct(0.99);
  const double span = std::chrono::duration<double>(s->last_done - s->first_submit).count();
  if (throughput_rps) *throughput_rps = span > 0 ? v.size() / span : 0;
  return DFA_OK;
}

int dfa_serve_counters(dfa_server *s, uint64_t *steps, uint64_t *request_rounds, uint64_t *state_rounds,
                       uint64_t *mode_state_rounds, double *step_us) {
  if (!s) return fail(DFA_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lock(s->mu);
  if (steps) *steps = s->steps;
  if (request_rounds) *request_rounds = s->request_rounds;
  if (state_rounds) *state_rounds = s->state_rounds;
  if (mode_state_rounds)
    for (int m = 0; m < 3; ++m) mode_state_rounds[m] = s->mode_state_rounds[m];
  if (step_us) *step_us = s->step_us;
  return DFA_OK;
}

int dfa_serve_destroy(dfa_server *s) {
  if (!s) return DFA_OK;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    for (auto &r : s->queue) {
      r->finished = true;
      r->status = DFA_ECANCELLED;
    }
    s->queue.clear();
    for (auto &r : s->active) {
      r->finished = true;
      r->status = DFA_ECANCELLED;
    }
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  if (s->worker.joinable()) s->worker.join();
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->in_stream) cudaStreamDestroy(s->in_stream);
  if (s->arena_base) cudaFree(s->arena_base);
  if (s->scratch) cudaFree(s->scratch);
  if (s->segs_pinned) cudaFreeHost(s->segs_pinned);
  if (s->outs_pinned) cudaFreeHost(s->outs_pinned);
  delete s;
  return DFA_OK;
}

}  // extern "C"
