// Moore-style signature refinement as one persistent cooperative kernel.
//
// Section 3.3 (Algorithm 4, sortPR): every round builds, for each state q, the
// signature (block[q], block[δ(q,a_0)], ..., block[δ(q,a_{k-1})]) and gives
// states with equal signatures the same new block; it stops when a round does
// not increase the number of blocks.  The paper renumbers by sorting the
// signatures (Thrust sort + adjacent difference + inclusive scan).  Here the
// signature is packed exactly into a 128-bit key and renumbered by one insert
// into an open-addressing table (the hashing route of Tewari et al. that the
// paper cites): the key's slot index is the state's new label and a successful
// CAS counts one new block.  Labels are arbitrary until the fixpoint; then one
// canonicalisation pass numbers blocks 0..B-1 by their smallest state, using a
// warp-shuffle/block scan to compact.
//
// All rounds run inside one launch: a grid barrier separates rounds and a
// device-side counter decides convergence, so no round needs the host.
#include "common.cuh"
#include "internal.h"

namespace dfa {

static constexpr int kThreads = 1024;
static constexpr int kBucketThreads = 512;

// Vector loads/stores of VEC consecutive 32-bit values (VEC*4-byte aligned).
template <int VEC>
__device__ __forceinline__ void load_vec(const uint32_t *p, uint32_t (&x)[VEC]) {
  if constexpr (VEC == 4) {
    const uint4 t = *reinterpret_cast<const uint4 *>(p);
    x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
  } else if constexpr (VEC == 2) {
    const uint2 t = *reinterpret_cast<const uint2 *>(p);
    x[0] = t.x; x[1] = t.y;
  } else {
    x[0] = *p;
  }
}
template <int VEC>
__device__ __forceinline__ void load_vec_stream(const uint32_t *p, uint32_t (&x)[VEC], unsigned long long pol) {
  if constexpr (VEC == 4) {
    const uint4 t = ld_v4_stream(p, pol);
    x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
  } else {
#pragma unroll
    for (int v = 0; v < VEC; ++v) x[v] = ld_u32_stream(p + v, pol);
  }
}
template <int VEC>
__device__ __forceinline__ void load_acc(const uint8_t *p, uint32_t (&c)[VEC]) {
  if constexpr (VEC == 4) {
    const uchar4 t = *reinterpret_cast<const uchar4 *>(p);
    c[0] = t.x != 0; c[1] = t.y != 0; c[2] = t.z != 0; c[3] = t.w != 0;
  } else {
#pragma unroll
    for (int v = 0; v < VEC; ++v) c[v] = p[v] != 0;
  }
}
template <int VEC>
__device__ __forceinline__ void store_vec(uint32_t *p, const uint32_t (&x)[VEC], unsigned long long pol) {
  if constexpr (VEC == 4) {
    st_v4_hint(p, make_uint4(x[0], x[1], x[2], x[3]), pol);
  } else {
#pragma unroll
    for (int v = 0; v < VEC; ++v) st_u32_hint(p + v, x[v], pol);
  }
}

// One pass over all states for stage `s` of a round.  ROUND1: components are
// acceptance bits (the initial partition {F, Q\F}); otherwise labels in `src`.
// Warps walk the states in chunks of 32*VEC so that every lane of a warp is
// present for the warp-cooperative insert; lanes past the end compute on state
// 0 (in bounds) and neither insert nor store.
template <int VEC, bool ROUND1>
__device__ __forceinline__ void moore_pass(const MooreArgs &A, const StagePlan &P, uint32_t s,
                                           const uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                           bool last, uint32_t epoch, uint32_t &local_new, uint32_t &seen,
                                           CtaCache *cache) {
  cta_cache_clear(cache);
  const uint32_t n = A.n, k = A.k, bits = P.bits;
  const uint32_t total = k + 1;
  uint32_t cbeg, cend;
  bool has_prev;
  if (s == 0) {
    cbeg = 0;
    cend = P.first < total ? P.first : total;
    has_prev = false;
  } else {
    cbeg = P.first + (s - 1) * P.per;
    cend = cbeg + P.per < total ? cbeg + P.per : total;
    has_prev = true;
  }
  const unsigned long long etag = (unsigned long long)epoch << (64 - A.ebits);
  const uint32_t nv = n / VEC;
  const unsigned long long keep = policy_evict_last(), drop = policy_evict_first();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint64_t base = (uint64_t)gwarp * 32; base < nv; base += (uint64_t)nwarps * 32) {
    const uint32_t i = (uint32_t)base + lane;
    const bool valid = i < nv;
    const uint32_t q0 = valid ? i * VEC : 0u;
    u128 key[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) key[v] = u128{0ull, 0ull};
    uint32_t shift = 0;
    if (has_prev) {
      uint32_t t[VEC];
      load_vec<VEC>(A.tmp + q0, t);
#pragma unroll
      for (int v = 0; v < VEC; ++v) put_bits(key[v], t[v], 0);
      shift = P.carry;
    }
    uint32_t j = cbeg;
    if (j == 0) {
      uint32_t c[VEC];
      if constexpr (ROUND1) {
        load_acc<VEC>(A.accept + q0, c);
        if (valid) {
#pragma unroll
          for (int v = 0; v < VEC; ++v) seen |= c[v] ? 1u : 2u;
        }
      } else {
        load_vec<VEC>(src + q0, c);
      }
#pragma unroll
      for (int v = 0; v < VEC; ++v) put_bits(key[v], c[v], shift);
      shift += bits;
      j = 1;
    }
#pragma unroll 4
    for (; j < cend; ++j) {
      const uint32_t *row = A.delta + (size_t)(j - 1) * n + q0;
      uint32_t d[VEC];
      // large tables are streamed once per pass; small ones stay in L2 across rounds
      if (A.stream_delta) load_vec_stream<VEC>(row, d, drop);
      else load_vec<VEC>(row, d);
      if constexpr (ROUND1) {
#pragma unroll
        for (int v = 0; v < VEC; ++v)
          if (d[v] >= n) { atomicOr(&A.ctrl->err, ERR_BAD_DELTA); d[v] = 0; }
      }
      uint32_t c[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) c[v] = ROUND1 ? (uint32_t)(A.accept[d[v]] != 0) : ld_u32_hint(src + d[v], keep);
#pragma unroll
      for (int v = 0; v < VEC; ++v) put_bits(key[v], c[v], shift);
      shift += bits;
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) key[v].hi |= etag;
    uint32_t lab[VEC];
    uint32_t created = 0;
    warp_insert<VEC>(A.table, A.log2S, key, valid, A.ebits, epoch, lab, created, &A.ctrl->err, cache);
    if (last) local_new += created;
    if (valid) {
      uint32_t *out = last ? dst : A.tmp;
      store_vec<VEC>(out + q0, lab, drop);
    }
  }
}

__device__ __forceinline__ void clear_table(u128 *table, uint32_t log2S) {
  const size_t S = (size_t)1 << log2S;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < S; i += stride) {
    reinterpret_cast<uint4 *>(table)[i] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// ----------------------------------------------------------------- direct rounds
// When the whole signature fits in K <= log2 S bits, the packed signature is
// itself the new label: no table, no hash.  A bitmap over the 2^K possible
// signatures tells whether a signature is new (the first atomicOr to set its
// bit counts one block).  Signatures of at most 13 bits are first collected in
// a per-block bitmap in shared memory and merged once per block.
// Direct rounds with keys of at most kSmallK bits mark them in a shared-memory
// bitmap first; wider keys go straight to the global bitmap.
static constexpr uint32_t kSmallK = 13;

template <bool ROUND1>
__device__ __forceinline__ void direct_pass(const MooreArgs &A, uint32_t w, uint32_t K, const uint32_t *__restrict__ src,
                                            uint32_t *__restrict__ dst, uint32_t *bm, uint32_t &local_new,
                                            uint32_t &seen, uint32_t *sbm) {
  const uint32_t n = A.n, k = A.k;
  const bool small = K <= kSmallK;
  const uint32_t swords = small ? ((1u << K) + 31) / 32 : 0;
  if (small) {
    for (uint32_t i = threadIdx.x; i < swords; i += blockDim.x) sbm[i] = 0u;
    __syncthreads();
  }
  const unsigned long long keep = policy_evict_last(), drop = policy_evict_first();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  for (uint64_t base = (uint64_t)gwarp * 32; base < n; base += (uint64_t)nwarps * 32) {
    const uint32_t q0 = (uint32_t)base + lane;
    const bool valid = q0 < n;
    const uint32_t q = valid ? q0 : 0u;
    uint32_t key;
    if (ROUND1) {
      key = A.accept[q] != 0;
      if (valid) seen |= key ? 1u : 2u;
    } else {
      key = src[q];
    }
    uint32_t shift = w;
    for (uint32_t a = 0; a < k; ++a) {
      const uint32_t *row = A.delta + (size_t)a * n;
      uint32_t d = A.stream_delta ? ld_u32_stream(row + q, drop) : row[q];
      if (ROUND1 && d >= n) {
        if (valid) atomicOr(&A.ctrl->err, ERR_BAD_DELTA);
        d = 0;
      }
      const uint32_t c = ROUND1 ? (uint32_t)(A.accept[d] != 0) : ld_u32_hint(src + d, keep);
      key |= c << shift;
      shift += w;
    }
    if (valid) st_u32_hint(dst + q, key, drop);
    const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, valid ? key : 0xFFFFFFFFu) & vm;
    if (valid && lane == (uint32_t)(__ffs(grp) - 1)) {
      const uint32_t bit = 1u << (key & 31u);
      if (small) atomicOr(&sbm[key >> 5], bit);
      else red_or_hint(&bm[key >> 5], bit, keep);   // counted by popcount after the pass
    }
  }
  if (small) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < swords; i += blockDim.x) {
      const uint32_t v = sbm[i];
      if (v) {
        const uint32_t old = atomicOr(&bm[i], v);
        local_new += __popc(v & ~old);
      }
    }
  }
}

// ----------------------------------------------------------------- filter rounds
// Rounds in which most signatures are unique.  Pass A hashes every signature
// into an L2-resident array of 2-bit saturating counters (two bitmaps).  A
// signature alone in its bucket is unique, so its state forms a block by
// itself and is labelled with its own number (pass B).  Only signatures in
// shared buckets go through the exact table; each such block is labelled with
// its smallest member, kept per slot with a 64-bit atomicMax on
// (round << 32 | ~state) (pass B), and read back in pass C.  Labels of these
// rounds are state numbers, wid bits wide.
__device__ __forceinline__ u128 pack_key(const MooreArgs &A, uint32_t w, const uint32_t *__restrict__ src, uint32_t q,
                                         unsigned long long keep, unsigned long long drop) {
  const uint32_t n = A.n, k = A.k;
  u128 key{0ull, 0ull};
  put_bits(key, src[q], 0);
  uint32_t shift = w;
  for (uint32_t a = 0; a < k; ++a) {
    const uint32_t *row = A.delta + (size_t)a * n;
    const uint32_t d = A.stream_delta ? ld_u32_stream(row + q, drop) : row[q];
    put_bits(key, ld_u32_hint(src + d, keep), shift);
    shift += w;
  }
  return key;
}

// Pass A: hash every signature (a 64-bit hash built component by component;
// the packed key is not needed here) into the counters.  A bucket with count
// one proves its signature unique whatever the hash, since equal signatures
// hash alike; hash quality only affects how many unique signatures are sent
// on to the exact table.

__device__ __forceinline__ void filter_one(const MooreArgs &A, uint32_t q, unsigned long long h,
                                           unsigned long long keep, unsigned long long drop) {
  h ^= h >> 33;
  h *= 0xff51afd7ed558ccdull;
  h ^= h >> 33;
  const uint32_t b = (uint32_t)(h >> (64 - A.mbits));
  const uint32_t bit = 1u << (b & 31u);
  const uint32_t old = atom_or_hint(&A.seen1[b >> 5], bit, keep);
  if (old & bit) red_or_hint(&A.seen2[b >> 5], bit, keep);
  st_u32_hint(A.tmp + q, b, drop);
  unsigned long long h2 = (h ^ 0x9E3779B97F4A7C15ull) * 0xc4ceb9fe1a85ec53ull;
  h2 ^= h2 >> 31;
  st_u32_hint(A.tmp2 + q, (uint32_t)(h2 >> (64 - (A.mbits - 1))), drop);
}

__device__ __forceinline__ void filter_pass_a(const MooreArgs &A, const uint32_t *__restrict__ src) {
  const uint32_t n = A.n, k = A.k;
  const unsigned long long keep = policy_evict_last(), drop = policy_evict_first();
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  uint32_t q = tid;
  for (; (uint64_t)q + stride < n; q += 2 * stride) {
    const uint32_t q2 = q + stride;
    unsigned long long h = hash_step(0x243F6A8885A308D3ull, src[q]);
    unsigned long long g = hash_step(0x243F6A8885A308D3ull, src[q2]);
    for (uint32_t a = 0; a < k; ++a) {
      const uint32_t *row = A.delta + (size_t)a * n;
      const uint32_t d = A.stream_delta ? ld_u32_stream(row + q, drop) : row[q];
      const uint32_t d2 = A.stream_delta ? ld_u32_stream(row + q2, drop) : row[q2];
      const uint32_t c = ld_u32_hint(src + d, keep), c2 = ld_u32_hint(src + d2, keep);
      h = hash_step(h, c);
      g = hash_step(g, c2);
    }
    filter_one(A, q, h, keep, drop);
    filter_one(A, q2, g, keep, drop);
  }
  if (q < n) {
    unsigned long long h = hash_step(0x243F6A8885A308D3ull, src[q]);
    for (uint32_t a = 0; a < k; ++a) {
      const uint32_t *row = A.delta + (size_t)a * n;
      const uint32_t d = A.stream_delta ? ld_u32_stream(row + q, drop) : row[q];
      h = hash_step(h, ld_u32_hint(src + d, keep));
    }
    filter_one(A, q, h, keep, drop);
  }
}

// The listed states of a filter round live in per-warp slices of `dups`: warp
// g owns [g*cap, g*cap + count_g), cap = ceil(states per warp / 32) * 32, and
// appends with a register cursor (no global atomics).  `dups2` holds, at the
// same positions, each listed state's bucket in the second filter.  Passes G
// and C walk the same slices with the same warps.
__device__ __forceinline__ uint32_t dup_cap(uint32_t n, uint32_t nwarps) {
  const uint32_t chunks = (n + 31) / 32;
  return (chunks + nwarps - 1) / nwarps * 32;
}

// Pass B: a signature alone in its bucket is unique: its state becomes a
// singleton block labelled with its own number.  The others are listed and
// enter a second filter with an independent bucket of A.mbits - 1 bits (most
// listed signatures merely collided with another one in the first filter).
// Each warp takes its chunks (c = warp, warp + nwarps, ...) kB at a time, so
// that the loads of kB chunks are in flight together.
static constexpr int kB = 4;
__device__ __forceinline__ void filter_pass_b(const MooreArgs &A, uint32_t *__restrict__ dst, uint32_t &local_new) {
  const uint32_t n = A.n;
  const unsigned long long drop = policy_evict_first();
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t chunks = (n + 31) / 32;
  const size_t at = (size_t)gwarp * dup_cap(n, nwarps);
  uint32_t *list = A.dups + at, *list2 = A.dups2 + at;
  uint32_t cursor = 0;
  for (uint64_t c0 = gwarp; c0 < chunks; c0 += (uint64_t)kB * nwarps) {
    uint32_t q[kB], b[kB], wd[kB], b2[kB];
    bool valid[kB], dup[kB];
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const uint64_t qq = (c0 + (uint64_t)j * nwarps) * 32 + lane;
      valid[j] = qq < n;
      q[j] = valid[j] ? (uint32_t)qq : 0u;
      b[j] = valid[j] ? ld_u32_stream(A.tmp + q[j], drop) : 0u;
    }
#pragma unroll
    for (int j = 0; j < kB; ++j) wd[j] = valid[j] ? A.seen2[b[j] >> 5] : 0u;
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      dup[j] = valid[j] && ((wd[j] >> (b[j] & 31u)) & 1u);
      b2[j] = dup[j] ? ld_u32_stream(A.tmp2 + q[j], drop) : 0u;
    }
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      if (dup[j]) {
        const uint32_t bit = 1u << (b2[j] & 31u);
        const uint32_t old = atomicOr(&A.seen3[b2[j] >> 5], bit);
        if (old & bit) atomicOr(&A.seen4[b2[j] >> 5], bit);
      } else if (valid[j]) {
        st_u32_hint(dst + q[j], q[j], drop);
        ++local_new;
      }
    }
#pragma unroll
    for (int j = 0; j < kB; ++j) {
      const unsigned dm = __ballot_sync(0xFFFFFFFFu, dup[j]);
      if (dup[j]) {
        const uint32_t p = cursor + __popc(dm & ((1u << lane) - 1u));
        list[p] = q[j];
        list2[p] = b2[j];
      }
      cursor += __popc(dm);
    }
  }
  if (lane == 0) {
    A.wcnt[gwarp] = cursor;
    if (cursor) atomicAdd(&A.ctrl->ndup, cursor);
  }
}

// Pass F: a listed state alone in its second bucket is unique too: it is
// labelled with its own number.  The rest stay listed, compacted in place
// within the warp's slice, and are counted in ctrl->nstill.
__device__ __forceinline__ void filter_pass_f(const MooreArgs &A, uint32_t *__restrict__ dst, uint32_t &local_new) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  const size_t at = (size_t)gwarp * dup_cap(A.n, nwarps);
  uint32_t *list = A.dups + at;
  const uint32_t *list2 = A.dups2 + at;
  const uint32_t nd = A.wcnt[gwarp];
  uint32_t cursor = 0;
  for (uint32_t base = 0; base < nd; base += 32) {
    const uint32_t i = base + lane;
    const bool valid = i < nd;
    uint32_t q = 0;
    bool still = false;
    if (valid) {
      q = list[i];
      const uint32_t b2 = list2[i];
      still = (A.seen4[b2 >> 5] >> (b2 & 31u)) & 1u;
      if (!still) {
        dst[q] = q;
        ++local_new;
      }
    }
    // every lane read its entry above (q feeds the ballot): positions <= reads
    const unsigned sm = __ballot_sync(0xFFFFFFFFu, still);
    if (still) list[cursor + __popc(sm & ((1u << lane) - 1u))] = q;
    cursor += __popc(sm);
  }
  __syncwarp();
  if (lane == 0) {
    A.wcnt[gwarp] = cursor;
    if (cursor) atomicAdd(&A.ctrl->nstill, cursor);
  }
}

// Table size (log2 slots) of a filter round's exact insert: at least twice
// the listed states left (so that the region to clear stays small), at least
// 2^10 slots, never more than the table's 2^log2S.
__device__ __forceinline__ uint32_t filter_table_bits(uint32_t nstill, uint32_t log2S) {
  uint32_t m = log2S < 10 ? log2S : 10;
  while (m < log2S && ((uint64_t)1 << m) < 2ull * nstill) ++m;
  return m;
}

// Keys of filter rounds carry this tag; their region is cleared every round.
static constexpr uint32_t kFilterTag = 1;

// Pass D: the listed states left insert their exact keys into the region of
// 2^m slots cleared for this round; each slot keeps its smallest member via
// atomicMax on (round << 32 | ~state), one atomic per (warp, slot).
__device__ __forceinline__ void filter_pass_d(const MooreArgs &A, uint32_t w, const uint32_t *__restrict__ src,
                                              uint32_t m, uint32_t r, CtaCache *cache) {
  const unsigned long long keep = policy_evict_last(), drop = policy_evict_first();
  const unsigned long long etag = (unsigned long long)kFilterTag << (64 - A.ebits);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  const uint32_t *list = A.dups + (size_t)gwarp * dup_cap(A.n, nwarps);
  const uint32_t nd = A.wcnt[gwarp];
  if ((uint64_t)(A.k + 1) * w > 125) {
    // wide signatures: each lane inserts (signature hash, state) alone; equal
    // hashes join only if the full signatures are equal
    const SigEq eq{src, A.delta, A.n, A.k};
    const uint32_t mask = table_mask(m);
    for (uint32_t i = lane; i < nd; i += 32) {
      const uint32_t q = list[i];
      const uint32_t slot = hashed_insert(A.table, mask, A.ebits, kFilterTag, eq.hash(q), q, eq, &A.ctrl->err);
      A.tmp[q] = slot;
      atomicMax(&A.rep[slot], ((unsigned long long)r << 32) | (unsigned long long)(~q));
    }
    return;
  }
  for (uint32_t base = 0; base < nd; base += 32) {
    const uint32_t i = base + lane;
    const bool valid = i < nd;
    const uint32_t q = valid ? list[i] : 0u;
    u128 key[1];
    key[0] = pack_key(A, w, src, q, keep, drop);
    key[0].hi |= etag;
    uint32_t slot[1];
    uint32_t created = 0;
    warp_insert<1>(A.table, m, key, valid, A.ebits, kFilterTag, slot, created, &A.ctrl->err, cache);
    if (valid) A.tmp[q] = slot[0];
    // listed states are ascending within the slice, so the lowest lane of a
    // slot group holds the group's smallest state
    const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
    const unsigned sg = __match_any_sync(0xFFFFFFFFu, valid ? slot[0] : 0xFFFFFFFFu) & vm;
    if (valid && lane == (uint32_t)(__ffs(sg) - 1))
      atomicMax(&A.rep[slot[0]], ((unsigned long long)r << 32) | (unsigned long long)(~q));
  }
}

// Pass C: listed states read their block's smallest member; the counters are
// cleared for the next filter round.
__device__ __forceinline__ void filter_pass_c(const MooreArgs &A, uint32_t *__restrict__ dst, uint32_t &local_new) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t gwarp = tid >> 5, nwarps = stride >> 5;
  const uint32_t *list = A.dups + (size_t)gwarp * dup_cap(A.n, nwarps);
  const uint32_t nd = A.wcnt[gwarp];
  for (uint32_t i = lane; i < nd; i += 32) {
    const uint32_t q = list[i];
    const uint32_t rep = ~(uint32_t)A.rep[A.tmp[q]];
    dst[q] = rep;
    if (rep == q) ++local_new;
  }
  const size_t words = ((size_t)1 << A.mbits) / 32;
  for (size_t i = tid; i < words; i += stride) {
    A.seen1[i] = 0u;
    A.seen2[i] = 0u;
  }
  for (size_t i = tid; i < words / 2; i += stride) {
    A.seen3[i] = 0u;
    A.seen4[i] = 0u;
  }
}

// ----------------------------------------------------------------- bucketed gather
// Every round of Algorithm 4 reads block[δ(q,a)] for all n states and k
// letters.  Read straight from the label array these are k*n random 4-byte
// requests to L2 per round, and L2's random-request rate (not HBM bandwidth)
// then bounds the round.  δ is the same in every round, so the transitions are
// sorted once per call into segments by (source bucket, target bucket)
// (BucketArgs), and a round becomes two streaming passes plus shared-memory
// random access:
//   gather   (one block per target bucket T): load T's BT labels into shared
//            memory, stream the et entries of every segment (s, T), read the
//            labels from shared memory and write them to val;
//   assemble (one block per source bucket s): stream region s (es, val) into a
//            tile tile[a*BS + q - s*BS] = block[δ(q,a)] in shared memory, then
//            renumber the bucket's states from the tile.
// Filter rounds prove uniqueness without random atomics: each state's 32-bit
// signature hash goes to one of P partitions (sorted by partition in shared
// memory, written as runs); one block per partition then counts the hashes in
// a shared-memory hash set, and only states whose hash repeats are listed for
// the exact table.
static constexpr uint32_t kBucketPad = 0xFFFFu;
static constexpr uint32_t kDedupLog2 = 15;   // hash-set slots of one partition: 2^15 (pcap < 2^15 * 2/3)
static constexpr int kG = 4;                 // gather: 8-entry pieces per lane in flight
static constexpr int kRing = 4;              // assemble: stages of the region stream
static constexpr uint32_t kChunk = 2048;     // assemble: entries per stage (12 KB)
static constexpr int kP = 16;                // prep: transition loads per thread in flight

// floor(t / d) for t < 2^28 and 8 <= d < 2^20 with m = ceil(2^48 / d): the
// product overestimates t/d by less than t/2^48 < 2^-20 < 1/d, which never
// reaches the next integer.
__device__ __forceinline__ uint32_t div_by_magic(uint32_t t, unsigned long long m) {
  return (uint32_t)(((unsigned long long)t * m) >> 48);
}

// Appends q (for lanes with want) to the list; all 32 lanes must call.
__device__ __forceinline__ void list_append(uint32_t *list, uint32_t *count, bool want, uint32_t q) {
  const uint32_t lane = threadIdx.x & 31u;
  const unsigned m = __ballot_sync(0xFFFFFFFFu, want);
  if (m == 0u) return;
  const uint32_t leader = (uint32_t)(__ffs(m) - 1);
  uint32_t base = 0;
  if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(m));
  base = __shfl_sync(0xFFFFFFFFu, base, leader);
  if (want) list[base + __popc(m & ((1u << lane) - 1u))] = q;
}

// Once per call: segments of every source bucket (histogram of target
// buckets, padded offsets, then the entries), and δ validated.  A region is
// built in shared memory (stage: cap et entries, then cap es entries) and
// written out with contiguous vector stores.
__device__ __noinline__ void bucket_prep(const MooreArgs &A, uint32_t *smem, uint32_t *s_red) {
  const BucketArgs &B = A.B;
  const uint32_t n = A.n, k = A.k, NT = B.NT;
  uint32_t *hist = smem, *cur = smem + NT;
  uint16_t *set = reinterpret_cast<uint16_t *>(smem + 2 * ((NT + 3) & ~3u));   // 16-byte aligned
  uint16_t *ses = set + B.cap;
  const unsigned long long drop = policy_evict_first();
  const unsigned long long magic = ((1ull << 48) + B.BT - 1) / B.BT;
  for (uint32_t s = blockIdx.x; s < B.NS; s += gridDim.x) {
    const uint32_t q0 = s * B.BS;
    const uint32_t nq = B.BS < n - q0 ? B.BS : n - q0;
    const size_t base = (size_t)s * B.cap;
    for (uint32_t i = threadIdx.x; i < NT; i += blockDim.x) hist[i] = 0u;
    __syncthreads();
    for (uint32_t a = 0; a < k; ++a) {
      const uint32_t *row = A.delta + (size_t)a * n + q0;
      for (uint32_t i0 = threadIdx.x; i0 < nq; i0 += kP * blockDim.x) {
        uint32_t t[kP];
#pragma unroll
        for (int j = 0; j < kP; ++j) {
          const uint32_t i = i0 + j * blockDim.x;
          t[j] = i < nq ? row[i] : 0u;
        }
#pragma unroll
        for (int j = 0; j < kP; ++j) {
          if (i0 + j * blockDim.x < nq) {
            uint32_t tt = t[j];
            if (tt >= n) {
              atomicOr(&A.ctrl->err, ERR_BAD_DELTA);
              tt = 0;
            }
            atomicAdd(&hist[div_by_magic(tt, magic)], 1u);
          }
        }
      }
    }
    __syncthreads();
    // padded offsets: exclusive scan over the target buckets
    const uint32_t per = (NT + blockDim.x - 1) / blockDim.x;
    const uint32_t b0 = threadIdx.x * per < NT ? threadIdx.x * per : NT;
    const uint32_t b1 = b0 + per < NT ? b0 + per : NT;
    uint32_t sum = 0;
    for (uint32_t T = b0; T < b1; ++T) sum += (hist[T] + 7u) & ~7u;
    uint32_t total;
    uint32_t pre = block_excl_scan(sum, s_red, &total);
    for (uint32_t T = b0; T < b1; ++T) {
      B.seg[(size_t)T * B.NS + s] = make_uint2(pre, hist[T]);
      cur[T] = pre;
      pre += (hist[T] + 7u) & ~7u;
    }
    if (threadIdx.x == 0) B.used[s] = total;
    __syncthreads();
    for (uint32_t a = 0; a < k; ++a) {
      const uint32_t *row = A.delta + (size_t)a * n + q0;
      for (uint32_t i0 = threadIdx.x; i0 < nq; i0 += kP * blockDim.x) {
        uint32_t t[kP];
#pragma unroll
        for (int j = 0; j < kP; ++j) {
          const uint32_t i = i0 + j * blockDim.x;
          t[j] = i < nq ? ld_u32_stream(row + i, drop) : 0u;
        }
#pragma unroll
        for (int j = 0; j < kP; ++j) {
          const uint32_t i = i0 + j * blockDim.x;
          if (i >= nq) continue;
          const uint32_t tt = t[j] < n ? t[j] : 0u;
          const uint32_t T = div_by_magic(tt, magic);
          const uint32_t pos = atomicAdd(&cur[T], 1u);
          set[pos] = (uint16_t)(tt - T * B.BT);
          ses[pos] = (uint16_t)(a * B.BS + i);
        }
      }
    }
    __syncthreads();
    // padding entries: any in-range target, no tile position
    for (uint32_t T = threadIdx.x; T < NT; T += blockDim.x) {
      const uint32_t end = cur[T], pad = ((hist[T] + 7u) & ~7u) - hist[T];
      for (uint32_t j = 0; j < pad; ++j) {
        set[end + j] = 0;
        ses[end + j] = (uint16_t)kBucketPad;
      }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x * 8; i < total; i += blockDim.x * 8) {
      *reinterpret_cast<uint4 *>(B.et + base + i) = *reinterpret_cast<const uint4 *>(set + i);
      *reinterpret_cast<uint4 *>(B.es + base + i) = *reinterpret_cast<const uint4 *>(ses + i);
    }
    __syncthreads();
  }
}

// The block's bulk-copy barrier and the parity its next completion flips.
struct BulkBar {
  unsigned long long *bar;
  uint32_t phase;
};

// What a bucketed pass returns to the round loop (by value: the passes are
// separate functions, and a counter passed by reference would live in local
// memory): new blocks counted, acceptance classes seen, the barrier's parity.
struct PassOut {
  uint32_t fresh, seen, phase;
  uint32_t chunks;   // region-stream chunks consumed so far (the ring barriers' phases follow from it)
};

// Bulk copy of `count` 32-bit words (rounded up to whole 16-byte units: the
// source has at least that much readable memory) into shared memory, issued
// by thread 0 after every thread's earlier use of that memory.
__device__ __forceinline__ void bulk_words(uint32_t *dst, const uint32_t *src, uint32_t count, BulkBar &bb) {
  fence_proxy_async_smem();
  __syncthreads();
  if (threadIdx.x == 0) bulk_load(dst, src, (count * 4u + 15u) & ~15u, bb.bar);
}
__device__ __forceinline__ bool bulk_wait(const MooreArgs &A, BulkBar &bb) {
  const bool ok = mbar_wait(bb.bar, bb.phase, A.ctrl, A.barrier_ns);
  bb.phase ^= 1u;
  return ok;
}

// Segments per warp group: a warp deals the 8-entry pieces of G consecutive
// segments to its lanes; G is chosen so that every warp gets the same number
// of groups.
__device__ __forceinline__ uint32_t gather_group(uint32_t NS, uint32_t nw) {
  const uint32_t m = (NS + 32 * nw - 1) / (32 * nw);
  return (NS + m * nw - 1) / (m * nw);
}

// Gather pass of a round: val[e] = label of e's target, for every entry.
// ROUND1 reads acceptance bits (the initial partition) instead of labels.
// Shared memory: the bucket's labels (BT words), then its segment table (NS
// entries of 8 bytes).
template <bool ROUND1>
__device__ __noinline__ uint32_t bucket_gather(const MooreArgs &A, const uint32_t *__restrict__ src, uint32_t *dyn,
                                               unsigned long long *bar, uint32_t phase) {
  BulkBar bb{bar, phase};
  const BucketArgs &B = A.B;
  const uint32_t n = A.n;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t *lab = dyn;
  uint2 *sseg = reinterpret_cast<uint2 *>(dyn + B.BT);
  const unsigned long long drop = policy_evict_first();
  const uint32_t G = gather_group(B.NS, nw);
  const uint32_t ngroups = (B.NS + G - 1) / G;
  for (uint32_t T = blockIdx.x; T < B.NT; T += gridDim.x) {
    const uint32_t t0 = T * B.BT;
    const uint32_t nt = B.BT < n - t0 ? B.BT : n - t0;
    if (!ROUND1) bulk_words(lab, src + t0, nt, bb);   // t0 is a multiple of 8: 32-byte aligned
    else
      for (uint32_t i = threadIdx.x; i < nt; i += blockDim.x) lab[i] = A.accept[t0 + i] != 0;
    const uint2 *segT = B.seg + (size_t)T * B.NS;
    for (uint32_t i = threadIdx.x; i < B.NS; i += blockDim.x) sseg[i] = segT[i];
    __syncthreads();
    if (!ROUND1) bulk_wait(A, bb);
    for (uint32_t g = warp; g < ngroups; g += nw) {
      const uint32_t s0 = g * G;
      const uint2 sg = (lane < G && s0 + lane < B.NS) ? sseg[s0 + lane] : make_uint2(0u, 0u);
      const uint32_t pc = (sg.y + 7u) >> 3;
      const uint32_t incl = warp_incl_scan(pc);
      const uint32_t excl = incl - pc;
      const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
      for (uint32_t j0 = 0; j0 < tot; j0 += 32 * kG) {
        uint4 e[kG];
        uint32_t at[kG];   // entry index (NS * cap < 2^32)
#pragma unroll
        for (int u = 0; u < kG; ++u) {
          const uint32_t j = j0 + u * 32 + lane;
          uint32_t L = 0;   // the last lane whose first piece is <= j: j's segment
#pragma unroll
          for (uint32_t b = 16; b >= 1; b >>= 1) {
            const uint32_t c = L + b;
            const uint32_t ex = __shfl_sync(0xFFFFFFFFu, excl, c & 31u);
            if (ex <= j) L = c;
          }
          const uint32_t offL = __shfl_sync(0xFFFFFFFFu, sg.x, L);
          const uint32_t exL = __shfl_sync(0xFFFFFFFFu, excl, L);
          at[u] = (s0 + L) * B.cap + offL + 8 * (j - exL);
          if (j < tot) e[u] = ld_v4_stream(reinterpret_cast<const uint32_t *>(B.et + at[u]), drop);
        }
#pragma unroll
        for (int u = 0; u < kG; ++u) {
          if (j0 + u * 32 + lane >= tot) continue;
          uint4 o0, o1;
          o0.x = lab[e[u].x & 0xFFFFu];
          o0.y = lab[e[u].x >> 16];
          o0.z = lab[e[u].y & 0xFFFFu];
          o0.w = lab[e[u].y >> 16];
          o1.x = lab[e[u].z & 0xFFFFu];
          o1.y = lab[e[u].z >> 16];
          o1.z = lab[e[u].w & 0xFFFFu];
          o1.w = lab[e[u].w >> 16];
          uint4 *dv = reinterpret_cast<uint4 *>(B.val + at[u]);
          dv[0] = o0;
          dv[1] = o1;
        }
      }
    }
    __syncthreads();
  }
  return bb.phase;
}

// Assemble pass: the es and val entries of this block's source buckets flow
// through a ring of kRing shared-memory stages of kChunk entries (one bulk copy
// pair per stage, on the stage's own barrier).  Thread 0 refills a stage as
// soon as the block has consumed it, across bucket boundaries too, so that
// kRing copies stay in flight while the block scatters and renumbers.
struct RegionStream {
  unsigned long long *bars;   // kRing barriers
  uint16_t *ses;              // kRing * kChunk
  uint32_t *sval;             // kRing * kChunk
  uint32_t consumed;          // chunks consumed so far (every thread)
  uint32_t ps, pc, pused;     // producer (thread 0): bucket, chunk in it, its entries
  uint32_t issued;            // producer: chunks issued so far
};

__device__ __forceinline__ void stream_issue(const MooreArgs &A, RegionStream &rs) {
  const BucketArgs &B = A.B;
  while (rs.ps < B.NS && rs.pc * kChunk >= rs.pused) {
    rs.ps += gridDim.x;
    rs.pc = 0;
    rs.pused = rs.ps < B.NS ? B.used[rs.ps] : 0u;
  }
  if (rs.ps >= B.NS) return;
  const uint32_t stage = rs.issued % kRing;
  const uint32_t cnt = rs.pused - rs.pc * kChunk < kChunk ? rs.pused - rs.pc * kChunk : kChunk;   // a multiple of 8
  const size_t at = (size_t)rs.ps * B.cap + (size_t)rs.pc * kChunk;
  mbar_expect_tx(rs.bars + stage, cnt * 6u);
  bulk_copy(rs.ses + (size_t)stage * kChunk, B.es + at, cnt * 2u, rs.bars + stage);
  bulk_copy(rs.sval + (size_t)stage * kChunk, B.val + at, cnt * 4u, rs.bars + stage);
  ++rs.pc;
  ++rs.issued;
}

// Starts the stream at this block's first source bucket: kRing copies in
// flight.  `chunks` counts the chunks earlier passes streamed through the same
// ring (every issued chunk is consumed within its pass).
__device__ __forceinline__ RegionStream stream_begin(const MooreArgs &A, unsigned long long *bars, uint32_t *ring,
                                                     uint32_t chunks) {
  RegionStream rs;
  rs.bars = bars;
  rs.ses = reinterpret_cast<uint16_t *>(ring);
  rs.sval = ring + kRing * kChunk / 2;
  rs.consumed = chunks;
  rs.ps = blockIdx.x;
  rs.pc = 0;
  rs.pused = blockIdx.x < A.B.NS ? A.B.used[blockIdx.x] : 0u;
  rs.issued = chunks;
  if (threadIdx.x == 0)
    for (int i = 0; i < kRing; ++i) stream_issue(A, rs);
  return rs;
}

// Scatters source bucket s's entries (used of them) from the stream into the
// tile.  Returns false on a failed wait.
__device__ __forceinline__ bool stream_bucket(const MooreArgs &A, RegionStream &rs, uint32_t used, uint32_t *tile) {
  bool ok = true;
  for (uint32_t c0 = 0; c0 < used; c0 += kChunk) {
    const uint32_t stage = rs.consumed % kRing;
    ok &= mbar_wait(rs.bars + stage, (rs.consumed / kRing) & 1u, A.ctrl, A.barrier_ns);
    const uint32_t cnt = used - c0 < kChunk ? used - c0 : kChunk;
    const uint16_t *es = rs.ses + (size_t)stage * kChunk;
    const uint32_t *vs = rs.sval + (size_t)stage * kChunk;
    for (uint32_t i = threadIdx.x * 4; i < cnt; i += blockDim.x * 4) {
      const uint2 e = *reinterpret_cast<const uint2 *>(es + i);
      const uint4 v = *reinterpret_cast<const uint4 *>(vs + i);
      const uint32_t ix[4] = {e.x & 0xFFFFu, e.x >> 16, e.y & 0xFFFFu, e.y >> 16};
      const uint32_t vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (ix[j] != kBucketPad) tile[ix[j]] = vv[j];
    }
    fence_proxy_async_smem();   // this stage's reads before its refill
    __syncthreads();
    if (threadIdx.x == 0) stream_issue(A, rs);
    ++rs.consumed;
  }
  return ok;
}

// Assemble pass: source bucket s's own labels (own, BS words: a bulk copy on
// bb that overlaps the scatter; acceptance bits in round 1) and its tile
// (tile[a*BS + q - q0] = label of δ(q, a)).  Returns false on a failed wait.
template <bool ROUND1>
__device__ __forceinline__ bool bucket_unit(const MooreArgs &A, RegionStream &rs, uint32_t s, uint32_t q0,
                                            uint32_t nq, const uint32_t *__restrict__ src, uint32_t *tile,
                                            uint32_t *own, BulkBar &bb) {
  if (!ROUND1) {
    if (threadIdx.x == 0) bulk_load(own, src + q0, (nq * 4u + 15u) & ~15u, bb.bar);   // q0: a multiple of 8
  } else {
    for (uint32_t i = threadIdx.x; i < nq; i += blockDim.x) own[i] = A.accept[q0 + i] != 0;
  }
  bool ok = stream_bucket(A, rs, A.B.used[s], tile);
  if (!ROUND1) ok &= bulk_wait(A, bb);
  __syncthreads();
  return ok;
}

// Shared memory of the assemble pass: tile (max(k,2)*BS words, reused for the
// filter round's sort), own labels or hashes (BS words), the stream's ring
// (kRing*kChunk*6 bytes), then 2*P words for the filter round's partitions.
__device__ __forceinline__ uint32_t *bucket_own(const MooreArgs &A, uint32_t *dyn) {
  return dyn + (size_t)(A.k > 2 ? A.k : 2) * A.B.BS;
}
__device__ __forceinline__ uint32_t *bucket_ring(const MooreArgs &A, uint32_t *dyn) {
  return bucket_own(A, dyn) + A.B.BS;
}

// Direct round from the tiles: the packed signature is the new label; the
// signatures present are marked in a bitmap (see direct_pass).
template <bool ROUND1>
__device__ __noinline__ PassOut bucket_direct(const MooreArgs &A, uint32_t w, uint32_t K,
                                              const uint32_t *__restrict__ src, uint32_t *__restrict__ dst, uint32_t *bm,
                                              uint32_t *sbm, uint32_t *dyn, unsigned long long *bar, uint32_t phase,
                                              uint32_t chunks) {
  BulkBar bb{bar, phase};
  RegionStream rs = stream_begin(A, bar + 1, bucket_ring(A, dyn), chunks);
  uint32_t local_new = 0, seen = 0;
  const BucketArgs &B = A.B;
  const uint32_t n = A.n, k = A.k;
  const bool small = K <= kSmallK;
  const uint32_t swords = small ? ((1u << K) + 31) / 32 : 0;
  if (small) {
    for (uint32_t i = threadIdx.x; i < swords; i += blockDim.x) sbm[i] = 0u;
    __syncthreads();
  }
  uint32_t *tile = dyn, *own = bucket_own(A, dyn);
  const unsigned long long keep = policy_evict_last(), drop = policy_evict_first();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t s = blockIdx.x; s < B.NS; s += gridDim.x) {
    const uint32_t q0 = s * B.BS;
    const uint32_t nq = B.BS < n - q0 ? B.BS : n - q0;
    bucket_unit<ROUND1>(A, rs, s, q0, nq, src, tile, own, bb);
    for (uint32_t c = warp; c * 32 < nq; c += nw) {
      const uint32_t ql = c * 32 + lane;
      const bool valid = ql < nq;
      const uint32_t l = valid ? ql : 0u;
      uint32_t key = own[l];
      if (ROUND1 && valid) seen |= key ? 1u : 2u;
      uint32_t shift = w;
      for (uint32_t a = 0; a < k; ++a) {
        key |= tile[a * B.BS + l] << shift;
        shift += w;
      }
      if (valid) st_u32_hint(dst + q0 + ql, key, drop);
      const unsigned vm = __ballot_sync(0xFFFFFFFFu, valid);
      const unsigned grp = __match_any_sync(0xFFFFFFFFu, valid ? key : 0xFFFFFFFFu) & vm;
      if (valid && lane == (uint32_t)(__ffs(grp) - 1)) {
        const uint32_t bit = 1u << (key & 31u);
        if (small) atomicOr(&sbm[key >> 5], bit);
        else red_or_hint(&bm[key >> 5], bit, keep);
      }
    }
    __syncthreads();
  }
  if (small) {
    for (uint32_t i = threadIdx.x; i < swords; i += blockDim.x) {
      const uint32_t v = sbm[i];
      if (v) {
        const uint32_t old = atomicOr(&bm[i], v);
        local_new += __popc(v & ~old);
      }
    }
  }
  return PassOut{local_new, seen, bb.phase, rs.consumed};
}

// Exact-table round from the tiles (single-stage plans: (k+1)*bits <= 125).
template <bool ROUND1>
__device__ __noinline__ PassOut bucket_table(const MooreArgs &A, uint32_t bits, const uint32_t *__restrict__ src,
                                             uint32_t *__restrict__ dst, uint32_t epoch, CtaCache *cache, uint32_t *dyn,
                                             unsigned long long *bar, uint32_t phase, uint32_t chunks) {
  BulkBar bb{bar, phase};
  RegionStream rs = stream_begin(A, bar + 1, bucket_ring(A, dyn), chunks);
  uint32_t local_new = 0, seen = 0;
  const BucketArgs &B = A.B;
  const uint32_t n = A.n, k = A.k;
  cta_cache_clear(cache);
  uint32_t *tile = dyn, *own = bucket_own(A, dyn);
  const unsigned long long etag = (unsigned long long)epoch << (64 - A.ebits);
  const unsigned long long drop = policy_evict_first();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t s = blockIdx.x; s < B.NS; s += gridDim.x) {
    const uint32_t q0 = s * B.BS;
    const uint32_t nq = B.BS < n - q0 ? B.BS : n - q0;
    bucket_unit<ROUND1>(A, rs, s, q0, nq, src, tile, own, bb);
    for (uint32_t c = warp; c * 32 < nq; c += nw) {
      const uint32_t ql = c * 32 + lane;
      const bool valid = ql < nq;
      const uint32_t l = valid ? ql : 0u;
      u128 key[1] = {u128{0ull, 0ull}};
      const uint32_t own_l = own[l];
      if (ROUND1 && valid) seen |= own_l ? 1u : 2u;
      put_bits(key[0], own_l, 0);
      uint32_t shift = bits;
      for (uint32_t a = 0; a < k; ++a) {
        put_bits(key[0], tile[a * B.BS + l], shift);
        shift += bits;
      }
      key[0].hi |= etag;
      uint32_t lab[1];
      uint32_t created = 0;
      warp_insert<1>(A.table, A.log2S, key, valid, A.ebits, epoch, lab, created, &A.ctrl->err, cache);
      local_new += created;
      if (valid) st_u32_hint(dst + q0 + ql, lab[0], drop);
    }
    __syncthreads();
  }
  return PassOut{local_new, seen, bb.phase, rs.consumed};
}

// Filter round, assemble half: hash every signature (the high word of a
// 64-bit hash is kept; its top pbits choose the partition), label every state
// with its own number (listed states are corrected later) and send (hash word,
// state) to its partition, sorted by partition in shared memory so that each
// block writes runs.  Shared memory: the tile, hashes (where the own labels
// were), the stream's ring, then cursors and global bases (P words each).  The
// sort reuses the tile as BS 64-bit entries.
__device__ __noinline__ PassOut bucket_filter_assemble(const MooreArgs &A, const uint32_t *__restrict__ src,
                                                       uint32_t *__restrict__ dst, uint32_t *dyn, uint32_t *s_red,
                                                       unsigned long long *bar, uint32_t phase, uint32_t chunks) {
  BulkBar bb{bar, phase};
  RegionStream rs = stream_begin(A, bar + 1, bucket_ring(A, dyn), chunks);
  uint32_t local_new = 0;
  const BucketArgs &B = A.B;
  const uint32_t n = A.n, k = A.k, P = B.P;
  const uint32_t sh = 32u - B.pbits;   // partition = stored word >> sh (a 64-bit shift: sh may be 32)
  uint32_t *tile = dyn;
  uint32_t *hs = bucket_own(A, dyn);
  uint32_t *cur = bucket_ring(A, dyn) + kRing * kChunk * 6 / 4, *gbase = cur + P;
  unsigned long long *sorted = reinterpret_cast<unsigned long long *>(tile);
  const unsigned long long drop = policy_evict_first();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t s = blockIdx.x; s < B.NS; s += gridDim.x) {
    const uint32_t q0 = s * B.BS;
    const uint32_t nq = B.BS < n - q0 ? B.BS : n - q0;
    bucket_unit<false>(A, rs, s, q0, nq, src, tile, hs, bb);
    for (uint32_t ql = threadIdx.x; ql < nq; ql += blockDim.x) {
      unsigned long long h = hash_step(0x243F6A8885A308D3ull, hs[ql]);
      for (uint32_t a = 0; a < k; ++a) h = hash_step(h, tile[a * B.BS + ql]);
      h ^= h >> 33;
      h *= 0xff51afd7ed558ccdull;
      h ^= h >> 33;
      hs[ql] = (uint32_t)(h >> 32);
      st_u32_hint(dst + q0 + ql, q0 + ql, drop);
      ++local_new;
    }
    for (uint32_t p = threadIdx.x; p < P; p += blockDim.x) cur[p] = 0u;
    __syncthreads();   // tile reads done; hashes and zeroed counts visible
    for (uint32_t ql = threadIdx.x; ql < nq; ql += blockDim.x)
      atomicAdd(&cur[(uint32_t)((unsigned long long)hs[ql] >> sh)], 1u);
    __syncthreads();
    // local starts (exclusive scan) and each partition's global run
    const uint32_t per = (P + blockDim.x - 1) / blockDim.x;
    const uint32_t b0 = threadIdx.x * per < P ? threadIdx.x * per : P;
    const uint32_t b1 = b0 + per < P ? b0 + per : P;
    uint32_t sum = 0;
    for (uint32_t p = b0; p < b1; ++p) sum += cur[p];
    uint32_t total;
    uint32_t pre = block_excl_scan(sum, s_red, &total);
    for (uint32_t p = b0; p < b1; ++p) {
      const uint32_t c = cur[p];
      gbase[p] = c ? atomicAdd(&B.pcnt[p], c) : 0u;
      cur[p] = pre;
      pre += c;
    }
    __syncthreads();
    for (uint32_t ql = threadIdx.x; ql < nq; ql += blockDim.x) {
      const uint32_t h = hs[ql];
      const uint32_t r = atomicAdd(&cur[(uint32_t)((unsigned long long)h >> sh)], 1u);
      sorted[r] = ((unsigned long long)h << 32) | ql;
    }
    __syncthreads();   // cur[p] is now the end of partition p's run (= start of p + 1)
    for (uint32_t base = warp * 32; base < nq; base += nw * 32) {
      const uint32_t i = base + lane;
      bool over = false;
      uint32_t q = 0;
      if (i < nq) {
        const unsigned long long e = sorted[i];
        const uint32_t p = (uint32_t)((e >> 32) >> sh);
        q = q0 + (uint32_t)e;
        const uint32_t start = p ? cur[p - 1] : 0u;
        const uint32_t g = gbase[p] + (i - start);
        if (g < B.pcap) {
          const size_t at = (size_t)p * B.pcap + g;
          B.phash[at] = (uint32_t)(e >> 32);
          B.pq[at] = q;
        } else {   // partition full: not proved unique
          over = true;
        }
      }
      list_append(B.list, &A.ctrl->ndup, over, q);
      if (over) --local_new;
    }
    __syncthreads();
  }
  return PassOut{local_new, 0u, bb.phase, rs.consumed};
}

// Filter round, dedup half: one block per partition loads its hashes into
// shared memory (a bulk copy) and counts them in a shared-memory hash set;
// states whose hash occurs twice (true duplicates or collisions) are listed.
// A partition that overflowed lists all its entries.  Shared memory: hashes
// (pcap words), the set (2^kDedupLog2 words), duplicate bits.
__device__ __noinline__ PassOut bucket_dedup(const MooreArgs &A, uint32_t *dyn, unsigned long long *bar,
                                             uint32_t phase) {
  BulkBar bb{bar, phase};
  uint32_t local_new = 0;   // minus one per listed state (modulo 2^32)
  const BucketArgs &B = A.B;
  const uint32_t TS = 1u << kDedupLog2, mask = TS - 1u;
  uint32_t *hb = dyn, *tbl = dyn + B.pcap, *dupb = tbl + TS;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t p = blockIdx.x; p < B.P; p += gridDim.x) {
    const uint32_t cnt = ld_relaxed(&B.pcnt[p]);
    const uint32_t stored = cnt < B.pcap ? cnt : B.pcap;
    const size_t at = (size_t)p * B.pcap;
    if (cnt > B.pcap) {
      for (uint32_t base = warp * 32; base < stored; base += nw * 32) {
        const uint32_t i = base + lane;
        const bool valid = i < stored;
        const uint32_t q = valid ? B.pq[at + i] : 0u;
        list_append(B.list, &A.ctrl->ndup, valid, q);
        if (valid) --local_new;
      }
    } else if (stored > 1) {
      bulk_words(hb, B.phash + at, stored, bb);   // pcap is a multiple of 8: aligned, and room to round up
      for (uint32_t i = threadIdx.x; i < TS; i += blockDim.x) tbl[i] = 0u;
      for (uint32_t i = threadIdx.x; i < TS / 32; i += blockDim.x) dupb[i] = 0u;
      bulk_wait(A, bb);
      __syncthreads();
      for (uint32_t i = threadIdx.x; i < stored; i += blockDim.x) {
        const uint32_t key = hb[i] | 1u;   // nonzero: 0 marks a free slot
        uint32_t slot = (key >> 1) & mask;
        for (uint32_t it = 0; it < TS; ++it) {
          uint32_t cv = tbl[slot];
          if (cv == 0u) {
            cv = atomicCAS(&tbl[slot], 0u, key);
            if (cv == 0u) break;   // inserted
          }
          if (cv == key) {
            atomicOr(&dupb[slot >> 5], 1u << (slot & 31u));
            break;
          }
          slot = (slot + 1u) & mask;
        }
      }
      __syncthreads();
      for (uint32_t base = warp * 32; base < stored; base += nw * 32) {
        const uint32_t i = base + lane;
        bool dup = false;
        if (i < stored) {
          const uint32_t key = hb[i] | 1u;
          uint32_t slot = (key >> 1) & mask;
          for (uint32_t it = 0; it < TS && tbl[slot] != key; ++it) slot = (slot + 1u) & mask;
          dup = (dupb[slot >> 5] >> (slot & 31u)) & 1u;
        }
        const uint32_t q = dup ? B.pq[at + i] : 0u;
        list_append(B.list, &A.ctrl->ndup, dup, q);
        if (dup) --local_new;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) B.pcnt[p] = 0u;   // clean for the next filter round
  }
  return PassOut{local_new, 0u, bb.phase, 0u};
}

// Exact insert of the listed states of a bucketed filter round (the global
// list, in no particular order): as filter_pass_d, every listed lane records
// (round, ~state) in its slot so that the slot keeps its smallest member.
__device__ __noinline__ void filter_list_d(const MooreArgs &A, uint32_t w, const uint32_t *__restrict__ src, uint32_t m,
                              uint32_t r, uint32_t nlist, CtaCache *cache) {
  const unsigned long long keep = policy_evict_last(), drop = policy_evict_first();
  const unsigned long long etag = (unsigned long long)kFilterTag << (64 - A.ebits);
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const uint32_t gwarp = tid >> 5, nwarps = stride >> 5;
  const uint32_t *list = A.B.list;
  if ((uint64_t)(A.k + 1) * w > 125) {
    const SigEq eq{src, A.delta, A.n, A.k};
    const uint32_t mask = table_mask(m);
    for (uint32_t i = tid; i < nlist; i += stride) {
      const uint32_t q = list[i];
      const uint32_t slot = hashed_insert(A.table, mask, A.ebits, kFilterTag, eq.hash(q), q, eq, &A.ctrl->err);
      A.tmp[q] = slot;
      atomicMax(&A.rep[slot], ((unsigned long long)r << 32) | (unsigned long long)(~q));
    }
    return;
  }
  for (uint32_t base = gwarp * 32; base < nlist; base += nwarps * 32) {
    const uint32_t i = base + lane;
    const bool valid = i < nlist;
    const uint32_t q = valid ? list[i] : 0u;
    u128 key[1];
    key[0] = pack_key(A, w, src, q, keep, drop);
    key[0].hi |= etag;
    uint32_t slot[1];
    uint32_t created = 0;
    warp_insert<1>(A.table, m, key, valid, A.ebits, kFilterTag, slot, created, &A.ctrl->err, cache);
    if (valid) {
      A.tmp[q] = slot[0];
      atomicMax(&A.rep[slot[0]], ((unsigned long long)r << 32) | (unsigned long long)(~q));
    }
  }
}

// Listed states take their block's smallest member as label.
__device__ __forceinline__ void filter_list_c(const MooreArgs &A, uint32_t *__restrict__ dst, uint32_t nlist,
                                              uint32_t &local_new) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  for (uint32_t i = tid; i < nlist; i += stride) {
    const uint32_t q = A.B.list[i];
    const uint32_t rep = ~(uint32_t)A.rep[A.tmp[q]];
    dst[q] = rep;
    if (rep == q) ++local_new;
  }
}

enum : uint32_t { MODE_DIRECT = 0, MODE_TABLE = 1, MODE_FILTER = 2 };

// BUCKET: the bucketed gather (one 1024-thread block per SM with the shared
// memory of BucketPlan::smem); rounds whose exact key needs several stages
// keep the direct label reads.
template <int VEC, bool BUCKET>
__global__ void __launch_bounds__(BUCKET ? kBucketThreads : kThreads, 1)
    moore_kernel(const __grid_constant__ MooreArgs A) {
  __shared__ uint32_t s_red[32];
  __shared__ CtaCache cache;
  __shared__ uint32_t sbm[(1u << kSmallK) / 32];
  extern __shared__ __align__(16) uint32_t dyn[];
  __shared__ __align__(8) unsigned long long s_bars[1 + kRing];   // bulk copies of the bucketed kernel
  uint32_t bphase = 0;                                 // parity of s_bars[0] (single copies)
  uint32_t bchunks = 0;                                // chunks streamed through s_bars[1..kRing]
  if (BUCKET) {
    if (threadIdx.x == 0) {
      for (int i = 0; i <= kRing; ++i) mbar_init(&s_bars[i], 1u);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");   // visible to the bulk copies
    }
    __syncthreads();
  }
  Ctrl *C = A.ctrl;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  if (leader) {
    const unsigned long long t = gtimer();
    C->t_start = t;
    C->deadline = t + A.timeout_ns;
    C->sep_round = 0xFFFFFFFFu;
  }
  const uint32_t emax = A.ebits >= 32 ? 0xFFFFFFFFu : ((1u << A.ebits) - 1u);
  const size_t S = (size_t)1 << A.log2S;
  uint32_t epoch = 0, r = 0, changed = 0, B_prev = 0, final_buf = 0, B_final = 0xFFFFFFFFu;
  uint32_t w = 1;              // bits of the labels the next round reads (round 0: acceptance bits)
  uint32_t final_space = 2;    // label space of the final labels
  bool final_min = false;      // final labels are smallest members (filter rounds)
  bool ok = true, separated = false, skip = false, table_clean = false;
  bool filter_ok = true;       // cleared for good once a filter round lists most states

  // Equivalence by union: the empty word already separates start states that
  // differ in acceptance (round 0).
  if (A.track_pair && ((A.accept[A.sep_a] != 0) != (A.accept[A.sep_b] != 0))) {
    separated = true;
    if (leader) C->sep_round = 0;
    if (A.early_exit) {
      skip = true;   // the answer needs no round; report the initial partition
      for (uint32_t q = tid; q < A.n; q += stride) A.lab[0][q] = A.accept[q] != 0;
    }
  }
  // direct bitmap of round 1 and the filter counters start clean
  for (size_t i = tid; i < S / 32; i += stride) A.bm[1][i] = 0u;
  if constexpr (BUCKET) {
    for (uint32_t i = tid; i < A.B.P; i += stride) A.B.pcnt[i] = 0u;
    if (!skip) bucket_prep(A, dyn, s_red);
  } else {
    for (size_t i = tid; i < ((size_t)1 << A.mbits) / 32; i += stride) {
      A.seen1[i] = 0u;
      A.seen2[i] = 0u;
    }
    for (size_t i = tid; i < ((size_t)1 << A.mbits) / 64; i += stride) {
      A.seen3[i] = 0u;
      A.seen4[i] = 0u;
    }
  }
  ok = grid_sync(C, A.barrier_ns);
  if (leader) trace_mark(C, kTraceStart);
  for (r = 1; ok && !skip; ++r) {
    const bool round1 = r == 1;
    const uint32_t *src = A.lab[(r - 1) & 1];
    uint32_t *dst = A.lab[r & 1];
    const uint64_t K = (uint64_t)(A.k + 1) * w;
    uint32_t mode = MODE_TABLE;
    if ((A.modes & 1u) && K <= A.log2S && K <= 27) mode = MODE_DIRECT;
    else if ((A.modes & 2u) && filter_ok && !round1 &&
             ((uint64_t)B_prev * 64 >= A.n || (A.predict_sparse && signatures_sparse(A.k, B_prev, A.n))))
      mode = MODE_FILTER;   // most signatures unique
    if (mode == MODE_TABLE && !table_clean) {   // first table round: the table starts clean
      clear_table(A.table, A.log2S);
      ok = grid_sync(C, A.barrier_ns);
      if (!ok) break;
      table_clean = true;
    }
    // the bitmap the next round would use starts clean
    for (size_t i = tid; i < S / 32; i += stride) A.bm[(r + 1) & 1][i] = 0u;
    uint32_t local_new = 0, seen = 0;
    bool bucketed = false;   // this round reads its labels through the bucketed gather
    if constexpr (BUCKET) {
      bucketed = mode != MODE_TABLE || make_plan(A.k, w, A.log2S).stages == 1;
      if (bucketed) {
        bphase = round1 ? bucket_gather<true>(A, src, dyn, s_bars, bphase)
                        : bucket_gather<false>(A, src, dyn, s_bars, bphase);
        ok = grid_sync(C, A.barrier_ns);
        if (!ok) break;
        if (leader) trace_mark(C, kTraceGather);
      }
    }
    if (mode == MODE_DIRECT) {
      if (bucketed) {
        const PassOut o =
            round1 ? bucket_direct<true>(A, w, (uint32_t)K, src, dst, A.bm[r & 1], sbm, dyn, s_bars, bphase, bchunks)
                   : bucket_direct<false>(A, w, (uint32_t)K, src, dst, A.bm[r & 1], sbm, dyn, s_bars, bphase, bchunks);
        local_new += o.fresh;
        seen |= o.seen;
        bphase = o.phase;
        bchunks = o.chunks;
      } else if (round1) {
        direct_pass<true>(A, w, (uint32_t)K, src, dst, A.bm[r & 1], local_new, seen, sbm);
      } else {
        direct_pass<false>(A, w, (uint32_t)K, src, dst, A.bm[r & 1], local_new, seen, sbm);
      }
      if (K > kSmallK) {   // labels marked without return values: count the bitmap
        ok = grid_sync(C, A.barrier_ns);
        if (!ok) break;
        const uint32_t words = (uint32_t)(((1ull << K) + 31) / 32);
        for (uint32_t i = tid; i < words; i += stride) local_new += __popc(__ldcg(A.bm[r & 1] + i));
      }
      w = (uint32_t)K;
      final_space = 1u << K;
      final_min = false;
    } else if (mode == MODE_FILTER && bucketed) {
      PassOut o = bucket_filter_assemble(A, src, dst, dyn, s_red, s_bars, bphase, bchunks);
      local_new += o.fresh;
      bphase = o.phase;
      bchunks = o.chunks;
      ok = grid_sync(C, A.barrier_ns);
      if (!ok) break;
      if (leader) trace_mark(C, kTraceAssemble);
      o = bucket_dedup(A, dyn, s_bars, bphase);
      local_new += o.fresh;
      bphase = o.phase;
      ok = grid_sync(C, A.barrier_ns);
      if (!ok) break;
      if (leader) trace_mark(C, kTraceDedup);
      const uint32_t nlist = ld_relaxed(&C->ndup);
      if ((uint64_t)nlist * 2 > A.n) filter_ok = false;   // mostly true duplicates: later rounds use the table
      if (nlist != 0u) {
        const uint32_t m = filter_table_bits(nlist, A.log2S);
        clear_table(A.table, m);
        for (size_t i = tid; i < ((size_t)1 << m); i += stride) A.rep[i] = 0ull;
        table_clean = false;
        ok = grid_sync(C, A.barrier_ns);
        if (!ok) break;
        cta_cache_clear(&cache);
        filter_list_d(A, w, src, m, r, nlist, &cache);
        ok = grid_sync(C, A.barrier_ns);
        if (!ok) break;
        if (leader) trace_mark(C, kTraceExact);
        filter_list_c(A, dst, nlist, local_new);
      }
      w = A.wid;
      final_space = A.n;
      final_min = true;
    } else if (mode == MODE_FILTER) {
      filter_pass_a(A, src);
      ok = grid_sync(C, A.barrier_ns);
      if (!ok) break;
      filter_pass_b(A, dst, local_new);
      ok = grid_sync(C, A.barrier_ns);
      if (!ok) break;
      // mostly true duplicates (large blocks): later rounds use the table path
      if ((uint64_t)ld_relaxed(&C->ndup) * 2 > A.n) filter_ok = false;
      filter_pass_f(A, dst, local_new);
      ok = grid_sync(C, A.barrier_ns);
      if (!ok) break;
      const uint32_t m = filter_table_bits(ld_relaxed(&C->nstill), A.log2S);
      clear_table(A.table, m);
      for (size_t i = tid; i < ((size_t)1 << m); i += stride) A.rep[i] = 0ull;
      // the region now holds filter-tagged keys: a later table round starts from a full clear
      table_clean = false;
      ok = grid_sync(C, A.barrier_ns);
      if (!ok) break;
      cta_cache_clear(&cache);
      filter_pass_d(A, w, src, m, r, &cache);
      ok = grid_sync(C, A.barrier_ns);
      if (!ok) break;
      filter_pass_c(A, dst, local_new);
      w = A.wid;
      final_space = A.n;
      final_min = true;
    } else if (bucketed) {   // single-stage exact table
      if (epoch == emax) {
        clear_table(A.table, A.log2S);
        ok = grid_sync(C, A.barrier_ns);
        epoch = 0;
        if (!ok) break;
      }
      ++epoch;
      const PassOut o = round1 ? bucket_table<true>(A, w, src, dst, epoch, &cache, dyn, s_bars, bphase, bchunks)
                               : bucket_table<false>(A, w, src, dst, epoch, &cache, dyn, s_bars, bphase, bchunks);
      local_new += o.fresh;
      seen |= o.seen;
      bphase = o.phase;
      bchunks = o.chunks;
      w = A.log2S;
      final_space = (uint32_t)S;
      final_min = false;
    } else {
      const StagePlan P = make_plan(A.k, w, A.log2S);
      for (uint32_t s = 0; s < P.stages && ok; ++s) {
        if (epoch == emax) {
          clear_table(A.table, A.log2S);
          ok = grid_sync(C, A.barrier_ns);
          epoch = 0;
          if (!ok) break;
        }
        ++epoch;
        const bool last = s + 1 == P.stages;
        if (round1) moore_pass<VEC, true>(A, P, s, src, dst, last, epoch, local_new, seen, &cache);
        else moore_pass<VEC, false>(A, P, s, src, dst, last, epoch, local_new, seen, &cache);
        if (!last) ok = grid_sync(C, A.barrier_ns);
      }
      if (!ok) break;
      w = A.log2S;
      final_space = (uint32_t)S;
      final_min = false;
    }
    const uint32_t bnew = block_sum(local_new, s_red);
    if (threadIdx.x == 0 && bnew) atomicAdd(&C->cnt[r % 3], bnew);
    if (round1) {
      const uint32_t bseen = __reduce_or_sync(0xFFFFFFFFu, seen);
      if ((threadIdx.x & 31) == 0) {
        if (bseen & 1u) atomicOr(&C->seen_acc, 1u);
        if (bseen & 2u) atomicOr(&C->seen_rej, 1u);
      }
    }
    ok = grid_sync(C, A.barrier_ns);
    if (!ok) break;
    if (leader) trace_mark(C, kTraceRound | (mode << 4));
    const uint32_t B_r = ld_relaxed(&C->cnt[r % 3]);
    if (round1) B_prev = (ld_relaxed(&C->seen_acc) != 0u) + (ld_relaxed(&C->seen_rej) != 0u);
    if (leader) {
      C->cnt[(r + 2) % 3] = 0u;
      C->ndup = 0u;     // read only inside a filter round, after its pass B
      C->nstill = 0u;   // read only inside a filter round, after its pass F
    }
    final_buf = r & 1;
    B_final = B_r;
    const bool grew = B_r != B_prev;
    if (grew) ++changed;
    if (A.track_pair && !separated) {
      // every thread reads the same two labels after the barrier: a uniform decision
      if (ld_relaxed(dst + A.sep_a) != ld_relaxed(dst + A.sep_b)) {
        separated = true;
        if (leader) C->sep_round = r;
        if (A.early_exit) break;
      }
    }
    if (!grew) break;   // fixpoint: the round did not add a block (Algorithm 4's until-test)
    if (A.stop_discrete && B_r == A.n) break;   // n singleton blocks cannot split any further
    if (A.max_rounds != 0u && r >= A.max_rounds) {
      if (leader) C->maxed = 1u;
      break;
    }
    B_prev = B_r;
  }
  if (skip) r = 0;
  if (ok) {
    if (leader) {
      C->rounds_executed = r;
      C->rounds_changed = changed;
    }
    const size_t space = skip ? 2 : final_space;
    ok = canonicalise(CanonArgs{A.n, A.lab[final_buf], space < S ? space : S, A.minrep, A.flag, A.partials, A.out,
                                A.ctrl, A.barrier_ns, final_min ? 1u : 0u},
                      B_final, s_red);
  }
  if (leader) {
    trace_mark(C, kTraceEnd);
    C->t_end = gtimer();
  }
}

static const void *kernel_for(uint32_t vec, bool bucket) {
  if (bucket) return (const void *)moore_kernel<1, true>;
  return vec == 4 ? (const void *)moore_kernel<4, false>
                  : vec == 2 ? (const void *)moore_kernel<2, false> : (const void *)moore_kernel<1, false>;
}

cudaError_t moore_grid(uint32_t vec, LaunchInfo *info, size_t bucket_smem) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const bool bucket = bucket_smem > 0;
  const void *fn = kernel_for(vec, bucket);
  const int threads = bucket ? kBucketThreads : kThreads;
  if (bucket) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bucket_smem);
    if (e != cudaSuccess) return e;
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, bucket_smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  info->grid = sms * per_sm;
  info->block = threads;
  return cudaSuccess;
}

cudaError_t launch_moore(const MooreArgs &a, cudaStream_t stream, LaunchInfo *info) {
  const size_t smem = a.bucket ? a.B_smem : 0;
  LaunchInfo li{};
  cudaError_t e = moore_grid(a.vec, &li, smem);
  if (e != cudaSuccess) return e;
  if (info) *info = li;
  const void *fn = kernel_for(a.vec, a.bucket != 0);
  MooreArgs copy = a;
  void *params[] = {&copy};
  return cudaLaunchCooperativeKernel(fn, dim3(li.grid), dim3(li.block), params, smem, stream);
}

}  // namespace dfa
