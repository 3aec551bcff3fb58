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

static constexpr int kThreads = 512;

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

enum : uint32_t { MODE_DIRECT = 0, MODE_TABLE = 1, MODE_FILTER = 2 };

template <int VEC>
__global__ void __launch_bounds__(kThreads, 2) moore_kernel(MooreArgs A) {
  __shared__ uint32_t s_red[kThreads / 32];
  __shared__ CtaCache cache;
  __shared__ uint32_t sbm[(1u << kSmallK) / 32];
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
  for (size_t i = tid; i < ((size_t)1 << A.mbits) / 32; i += stride) {
    A.seen1[i] = 0u;
    A.seen2[i] = 0u;
  }
  for (size_t i = tid; i < ((size_t)1 << A.mbits) / 64; i += stride) {
    A.seen3[i] = 0u;
    A.seen4[i] = 0u;
  }
  ok = grid_sync(C, A.barrier_ns);
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
    if (mode == MODE_DIRECT) {
      if (round1) direct_pass<true>(A, w, (uint32_t)K, src, dst, A.bm[r & 1], local_new, seen, sbm);
      else direct_pass<false>(A, w, (uint32_t)K, src, dst, A.bm[r & 1], local_new, seen, sbm);
      if (K > kSmallK) {   // labels marked without return values: count the bitmap
        ok = grid_sync(C, A.barrier_ns);
        if (!ok) break;
        const uint32_t words = (uint32_t)(((1ull << K) + 31) / 32);
        for (uint32_t i = tid; i < words; i += stride) local_new += __popc(__ldcg(A.bm[r & 1] + i));
      }
      w = (uint32_t)K;
      final_space = 1u << K;
      final_min = false;
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
  if (leader) C->t_end = gtimer();
}

static const void *kernel_for(uint32_t vec) {
  return vec == 4 ? (const void *)moore_kernel<4> : vec == 2 ? (const void *)moore_kernel<2> : (const void *)moore_kernel<1>;
}

cudaError_t moore_grid(uint32_t vec, LaunchInfo *info) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const void *fn = kernel_for(vec);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  info->grid = sms * per_sm;
  info->block = kThreads;
  return cudaSuccess;
}

cudaError_t launch_moore(const MooreArgs &a, cudaStream_t stream, LaunchInfo *info) {
  LaunchInfo li{};
  cudaError_t e = moore_grid(a.vec, &li);
  if (e != cudaSuccess) return e;
  if (info) *info = li;
  const void *fn = kernel_for(a.vec);
  const int grid = li.grid;
  MooreArgs copy = a;
  void *params[] = {&copy};
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), params, 0, stream);
}

}  // namespace dfa
