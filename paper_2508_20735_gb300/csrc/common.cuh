// Device primitives shared by the refinement kernels (sm_103a).
//
//  * 128-bit keys and the exact open-addressing table used to renumber blocks
//    (Section 3.3 renumbers by sorting; the hashing alternative it cites is
//    used here, with exact keys so that no two signatures ever merge).
//  * A grid barrier for persistent cooperative kernels whose every wait is
//    bounded by %globaltimer, so a lost block turns into an error status, not
//    a hang.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dfa {

// ----------------------------------------------------------------- errors
enum : uint32_t {
  ERR_BAD_DELTA = 1u,      // a transition target >= n
  ERR_TIMEOUT = 2u,        // a barrier wait or the call's deadline ran out
  ERR_TABLE_FULL = 4u,     // no free slot (cannot happen with the sizing used)
};

static constexpr uint32_t kTraceLen = 96;

// Control block at the start of every workspace (zeroed by the host before launch).
struct Ctrl {
  uint32_t bar_count;      // grid barrier: arrivals in the current generation
  uint32_t bar_gen;        // grid barrier: generation
  uint32_t err;            // ERR_* bits
  uint32_t cnt[3];         // per-round new-block counts (ring of three)
  uint32_t seen_acc;       // some state accepting
  uint32_t seen_rej;       // some state rejecting
  uint32_t num_blocks;
  uint32_t rounds_changed;
  uint32_t rounds_executed;
  uint32_t flag;           // naivePR: some state split this round (ring use in kernels)
  uint32_t flag2[3];
  uint32_t sep_round;      // equivalence: round that separated the start states (or ~0)
  uint32_t verdict;        // equivalence: 1 = same block
  uint32_t maxed;          // stopped at opts.max_rounds (not an error for the barrier)
  uint32_t qf, qn;         // naivePR: initial leaders (min F, min Q\F)
  uint32_t ndup;           // filter rounds: states listed by the first filter
  uint32_t nstill;         // filter rounds: listed states left for the exact table
  unsigned long long t_start, t_end;
  unsigned long long deadline;  // absolute %globaltimer value
  uint32_t ntrace;         // entries of trace in use
  uint32_t pad_;
  unsigned long long trace[kTraceLen];  // (ns since t_start) << 8 | tag, at the phase ends of a launch
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Records the end of a phase (tag < 256) in the control block; called by one
// thread after a grid barrier, so entries are ordered in time.
// Trace tags (Ctrl::trace): the phase that ended at the recorded time.
enum : uint32_t {
  kTraceStart = 1,      // set-up (clearing, staging; the bucketed kernel's sorting of δ)
  kTraceGather = 2,     // bucketed gather of a round
  kTraceAssemble = 3,   // bucketed filter round: signatures hashed and partitioned
  kTraceDedup = 4,      // bucketed filter round: partitions deduplicated
  kTraceExact = 5,      // filter round: exact inserts of the listed states
  kTraceRound = 8,      // end of a round (| mode << 4)
  kTraceEnd = 0xFF,     // canonical numbering done
};

// The same with the entry count and the start time kept by the caller in
// registers (nothing loaded from memory: for kernels whose rounds last
// microseconds).  nt starts at 0; t_start is the value stored in c->t_start.
__device__ __forceinline__ void trace_put(Ctrl *c, uint32_t &nt, unsigned long long t_start, uint32_t tag) {
  if (nt < kTraceLen) {
    c->trace[nt] = ((gtimer() - t_start) << 8) | tag;
    c->ntrace = ++nt;
  }
}

__device__ __forceinline__ void trace_mark(Ctrl *c, uint32_t tag) {
  const uint32_t i = c->ntrace;
  if (i < kTraceLen) {
    c->trace[i] = ((gtimer() - c->t_start) << 8) | tag;
    c->ntrace = i + 1;
  }
}

// B^(k+1) >= 64 n: the previous round's B blocks allow far more signatures
// than there are states, so a signature rarely repeats even while the blocks
// are large (a DFA with many letters, early rounds).  Filter rounds suit that.
__host__ __device__ __forceinline__ bool signatures_sparse(uint32_t k, uint32_t B, uint32_t n) {
#ifdef __CUDA_ARCH__
  const uint32_t lg_b = B > 1u ? 31u - (uint32_t)__clz(B) : 0u;        // floor(log2 B)
  const uint32_t lg_n = n > 1u ? 32u - (uint32_t)__clz(n - 1u) : 0u;   // ceil(log2 n)
#else
  uint32_t lg_b = 0, lg_n = 0;
  while (lg_b < 31u && (B >> (lg_b + 1u)) != 0u) ++lg_b;
  while (lg_n < 32u && ((uint64_t)1 << lg_n) < n) ++lg_n;
#endif
  return (uint64_t)(k + 1u) * lg_b >= (uint64_t)lg_n + 6u;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t atom_add_acq_rel(uint32_t *p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Grid-wide barrier for a cooperative launch.  Returns false (in every thread of
// the block) if the error word is set or the wait exceeded `limit_ns`; the
// kernel must then stop.  The last block to arrive also checks the call's
// deadline, so the decision to stop is the same in every block.
__device__ __forceinline__ bool grid_sync(Ctrl *c, unsigned long long limit_ns) {
  __shared__ uint32_t s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t ok = 1;
    const uint32_t gen = ld_acquire(&c->bar_gen);
    const uint32_t arrived = atom_add_acq_rel(&c->bar_count, 1u);
    if (arrived == gridDim.x - 1) {
      if (gtimer() > c->deadline) atomicOr(&c->err, ERR_TIMEOUT);
      c->bar_count = 0;                       // nobody arrives again before gen moves on
      st_release(&c->bar_gen, gen + 1);
    } else {
      const unsigned long long t0 = gtimer();
      while (ld_acquire(&c->bar_gen) == gen) {
        if (ld_relaxed(&c->err) != 0u) { ok = 0; break; }
        if (gtimer() - t0 > limit_ns) { atomicOr(&c->err, ERR_TIMEOUT); ok = 0; break; }
        __nanosleep(64);
      }
    }
    if (ok && ld_acquire(&c->err) != 0u) ok = 0;
    // gpu-scope acquire by this thread also invalidates the SM's L1, so weak
    // loads issued by any thread of the block after the barrier see fresh data
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0u;
}

// ----------------------------------------------------------------- bulk copies (TMA) into shared memory
// One thread arms an mbarrier with the byte count and issues
// cp.async.bulk (global -> shared, 16-byte aligned addresses, size a multiple
// of 16); every thread waits on the barrier's phase.  Waits are bounded: a
// copy that does not land within limit_ns sets ERR_TIMEOUT (the next grid
// barrier then ends the launch).
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// orders this thread's earlier generic-proxy shared-memory accesses before
// later bulk copies into the same memory
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// The pieces of bulk_load for a barrier that several copies complete: one
// arrival announcing the bytes of all of them, then the copies.
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, uint32_t bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0u;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, Ctrl *c,
                                          unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = gtimer();
  while (!mbar_try_wait(bar, parity)) {
    if (gtimer() - t0 > limit_ns) {
      atomicOr(&c->err, ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}

// ----------------------------------------------------------------- L2 cache policies
// The label array gathered every round is kept in L2 (evict_last); streamed
// inputs, table probes and freshly written labels are evicted first, so the
// random traffic of a large renumbering table does not push the labels out.
__device__ __forceinline__ unsigned long long policy_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long policy_evict_normal() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long policy_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_u32_hint(const uint32_t *p, unsigned long long pol) {
  uint32_t v;
  asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint4 ld_v4_stream(const uint32_t *p, unsigned long long pol) {
  uint4 v;
  asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ld_u32_stream(const uint32_t *p, unsigned long long pol) {
  uint32_t v;
  asm volatile("ld.global.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_v4_hint(uint32_t *p, uint4 v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ uint32_t atom_or_hint(uint32_t *p, uint32_t v, unsigned long long pol) {
  uint32_t old;
  asm volatile("atom.global.L2::cache_hint.or.b32 %0, [%1], %2, %3;" : "=r"(old) : "l"(p), "r"(v), "l"(pol) : "memory");
  return old;
}
__device__ __forceinline__ void red_or_hint(uint32_t *p, uint32_t v, unsigned long long pol) {
  asm volatile("red.global.L2::cache_hint.or.b32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_u32_hint(uint32_t *p, uint32_t v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v), "l"(pol) : "memory");
}

// ----------------------------------------------------------------- 128-bit keys
struct __align__(16) u128 {
  unsigned long long lo, hi;
};

__device__ __forceinline__ bool eq128(u128 a, u128 b) { return a.lo == b.lo && a.hi == b.hi; }

// OR value v (< 2^bits, bits <= 32) into key at bit offset `shift` (shift + bits <= 128).
__device__ __forceinline__ void put_bits(u128 &k, uint32_t v, uint32_t shift) {
  const unsigned long long x = v;
  if (shift < 64) {
    k.lo |= x << shift;
    if (shift > 32) k.hi |= x >> (64 - shift);
  } else {
    k.hi |= x << (shift - 64);
  }
}

// Weak 16-byte load as one vector instruction.  Caches move whole 32-byte
// sectors, so the two halves come from the same write; the value may be stale.
__device__ __forceinline__ u128 ld_b128_weak(const u128 *p) {
  u128 r;
  asm volatile(
      "{\n\t.reg .b64 pol;\n\t"
      "createpolicy.fractional.L2::evict_first.b64 pol, 1.0;\n\t"
      "ld.global.L2::cache_hint.v2.u64 {%0, %1}, [%2], pol;\n\t}"
      : "=l"(r.lo), "=l"(r.hi)
      : "l"(p)
      : "memory");
  return r;
}

// 128-bit atomic load (single-copy atomic; never a torn mix of two writes).
__device__ __forceinline__ u128 ld_b128_relaxed(const u128 *p) {
  u128 r;
  asm volatile(
      "{\n\t.reg .b128 t;\n\t"
      "ld.relaxed.gpu.global.b128 t, [%2];\n\t"
      "mov.b128 {%0, %1}, t;\n\t}"
      : "=l"(r.lo), "=l"(r.hi)
      : "l"(p)
      : "memory");
  return r;
}

__device__ __forceinline__ u128 cas_b128(u128 *p, u128 cmp, u128 val) {
  u128 r;
  asm volatile(
      "{\n\t.reg .b128 c, v, d;\n\t"
      "mov.b128 c, {%2, %3};\n\t"
      "mov.b128 v, {%4, %5};\n\t"
      "atom.relaxed.gpu.global.cas.b128 d, [%6], c, v;\n\t"
      "mov.b128 {%0, %1}, d;\n\t}"
      : "=l"(r.lo), "=l"(r.hi)
      : "l"(cmp.lo), "l"(cmp.hi), "l"(val.lo), "l"(val.hi), "l"(p)
      : "memory");
  return r;
}

// Finaliser of MurmurHash3 (Appleby), applied to a fold of the two halves.
__device__ __forceinline__ unsigned long long mix128(u128 k) {
  unsigned long long h = k.lo ^ (k.hi * 0x9E3779B97F4A7C15ull) ^ (k.hi >> 29);
  h ^= h >> 33;
  h *= 0xff51afd7ed558ccdull;
  h ^= h >> 33;
  h *= 0xc4ceb9fe1a85ec53ull;
  h ^= h >> 33;
  return h;
}

// One step of the signature hash of filter rounds (a multiply-xorshift over
// the components; any hash will do: uniqueness is proved by counting).
__device__ __forceinline__ unsigned long long hash_step(unsigned long long h, uint32_t c) {
  h = (h ^ c) * 0x9E3779B97F4A7C15ull;
  return h ^ (h >> 29);
}

__device__ __forceinline__ uint32_t table_mask(uint32_t log2S) {
  return (log2S >= 32) ? 0xFFFFFFFFu : ((1u << log2S) - 1u);
}

// Exact inserts into an open-addressing table of 2^log2S 16-byte slots, for
// the VEC keys of one thread at once (their probes stay in flight together).
//
// A slot is current when its top `ebits` bits equal `epoch` (1..2^ebits-1);
// any other value (zero, or a key of an earlier pass) counts as free, so the
// table needs no clearing between passes.  Within a pass a slot changes at
// most once (free -> key).  That makes the weak first probe safe: a stale value
// only sends the thread to the CAS, which is atomic at L2, and a current value
// is final.  Linear probing; the table is sized to at least twice the number of
// distinct keys a pass can hold, so probe sequences are short.
//   want[v]  : insert key[v]
//   slot[v]  : in = home slot, out = the key's slot (its new label)
//   is_new[v]: this call created the entry
template <int VEC>
__device__ __forceinline__ void table_insert_vec(u128 *table, uint32_t mask, const u128 (&key)[VEC], uint32_t ebits,
                                                 uint32_t epoch, const bool (&want)[VEC], uint32_t (&slot)[VEC],
                                                 bool (&is_new)[VEC], uint32_t *err) {
  const uint32_t eshift = 64u - ebits;
  bool pending[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    pending[v] = want[v];
    is_new[v] = false;
  }
  for (uint64_t iter = 0; iter <= (uint64_t)mask + 1; ++iter) {
    bool any = false;
#pragma unroll
    for (int v = 0; v < VEC; ++v) any |= pending[v];
    if (!any) return;
    u128 cur[VEC], old[VEC];
    bool cas[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v)
      if (pending[v]) cur[v] = ld_b128_weak(table + slot[v]);
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      cas[v] = false;
      if (!pending[v]) continue;
      if ((uint32_t)(cur[v].hi >> eshift) == epoch) {
        if (eq128(cur[v], key[v])) pending[v] = false;   // found
        else slot[v] = (slot[v] + 1u) & mask;             // owned by another key
      } else {
        old[v] = cas_b128(table + slot[v], cur[v], key[v]);
        cas[v] = true;
      }
    }
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      if (!cas[v]) continue;
      if (eq128(old[v], cur[v])) {               // we wrote the key
        pending[v] = false;
        is_new[v] = true;
      } else if ((uint32_t)(old[v].hi >> eshift) == epoch) {
        if (eq128(old[v], key[v])) pending[v] = false;   // someone else wrote our key
        else slot[v] = (slot[v] + 1u) & mask;
      }
      // else: the slot held another stale value; retry it with that value
    }
  }
  atomicOr(err, ERR_TABLE_FULL);
}

// Per-block cache of (key -> slot) for the current pass, in shared memory.  A
// key that many states share (a large block that does not split) then reaches
// the global table once per thread block instead of once per warp.  Entries
// are claimed with a 32-bit tag; the claiming thread publishes the key and its
// slot before it waits on any other entry, so waits always end.
struct CtaCache {
  static constexpr uint32_t M = 256;
  uint32_t tag[M];
  uint32_t ready[M];
  uint32_t slot[M];
  uint32_t ns[M];          // key namespace (the DFA of a batch whose table the slot belongs to)
  u128 key[M];
};

__device__ __forceinline__ void cta_cache_clear(CtaCache *c) {
  for (uint32_t i = threadIdx.x; i < CtaCache::M; i += blockDim.x) {
    c->tag[i] = 0u;
    c->ready[i] = 0u;
  }
  __syncthreads();
}

// Warp-cooperative exact insert: lanes whose keys (for the same v) are equal
// send one insert and share its slot.  Grouping uses a 32-bit hash; a lane
// adopts its group leader's slot only after comparing the full 128-bit key, so
// a hash collision just costs that lane its own insert.  The group leader then
// consults the block's cache, and only misses reach the global table.  All 32
// lanes must call this; lanes with valid = false neither insert nor count.
// `ns` names the table the keys belong to (warps of one block may serve
// different tables); a cached slot is reused only for the same key and ns.
template <int VEC>
__device__ __forceinline__ void warp_insert(u128 *table, uint32_t log2S, const u128 (&key)[VEC], bool valid,
                                            uint32_t ebits, uint32_t epoch, uint32_t (&label)[VEC],
                                            uint32_t &created, uint32_t *err, CtaCache *cache, uint32_t ns = 0) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t mask = table_mask(log2S);
  const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid);
  uint32_t slot[VEC], leader[VEC], ci[VEC], tg[VEC];
  bool want[VEC], is_new[VEC], claimed[VEC], waiter[VEC];
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    const unsigned long long h = mix128(key[v]);
    slot[v] = (uint32_t)(h >> 32) & mask;
    const unsigned grp = __match_any_sync(0xFFFFFFFFu, (uint32_t)h) & vmask;
    uint32_t ld = valid ? (uint32_t)(__ffs(grp) - 1) : lane;
    const unsigned long long llo = __shfl_sync(0xFFFFFFFFu, key[v].lo, ld);
    const unsigned long long lhi = __shfl_sync(0xFFFFFFFFu, key[v].hi, ld);
    if (llo != key[v].lo || lhi != key[v].hi) ld = lane;   // same hash, different key
    leader[v] = ld;
    want[v] = valid && ld == lane;
    const uint32_t hn = (uint32_t)h ^ (ns * 0x9E3779B9u);
    tg[v] = hn | 1u;
    ci[v] = (hn >> 8) % CtaCache::M;
    claimed[v] = waiter[v] = false;
  }
  // 1. claim cache entries (or find them claimed by another warp of the block)
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    if (!want[v]) continue;
    const uint32_t old = atomicCAS(&cache->tag[ci[v]], 0u, tg[v]);
    if (old == 0u) {
      claimed[v] = true;
      cache->key[ci[v]] = key[v];
      cache->ns[ci[v]] = ns;
    } else if (old == tg[v]) {
      waiter[v] = true;
      want[v] = false;   // resolved through the cache below, if the key matches
    }
  }
  // 2. global inserts for claimed entries and cache misses, then publish
  table_insert_vec<VEC>(table, mask, key, ebits, epoch, want, slot, is_new, err);
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    if (!claimed[v]) continue;
    cache->slot[ci[v]] = slot[v];
    __threadfence_block();
    atomicExch(&cache->ready[ci[v]], 1u);
  }
  // 3. entries claimed by other threads: wait (bounded), compare the full key
  bool retry[VEC];
  bool any_retry = false;
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    retry[v] = false;
    if (!waiter[v]) continue;
    uint32_t spins = 0;
    while (atomicAdd(&cache->ready[ci[v]], 0u) == 0u && ++spins < (1u << 22)) {
    }
    __threadfence_block();
    const u128 ck = cache->key[ci[v]];
    if (spins < (1u << 22) && eq128(ck, key[v]) && cache->ns[ci[v]] == ns) {
      slot[v] = cache->slot[ci[v]];
    } else {
      retry[v] = true;
      any_retry = true;
    }
  }
  if (any_retry) {
    bool is_new2[VEC];
    table_insert_vec<VEC>(table, mask, key, ebits, epoch, retry, slot, is_new2, err);
#pragma unroll
    for (int v = 0; v < VEC; ++v)
      if (retry[v] && is_new2[v]) is_new[v] = true;
  }
#pragma unroll
  for (int v = 0; v < VEC; ++v) {
    label[v] = __shfl_sync(0xFFFFFFFFu, slot[v], leader[v]);
    if (is_new[v]) ++created;
  }
}

// Signature (src[q], src[δ(q,a)] for every letter a) of a wide-key insert:
// its 64-bit hash, and the exact comparison of two states' signatures.
struct SigEq {
  const uint32_t *src, *delta;
  uint32_t n, k;
  __device__ bool operator()(uint32_t q, uint32_t p) const {
    if (src[q] != src[p]) return false;
    for (uint32_t a = 0; a < k; ++a)
      if (src[delta[(size_t)a * n + q]] != src[delta[(size_t)a * n + p]]) return false;
    return true;
  }
  __device__ unsigned long long hash(uint32_t q) const {
    unsigned long long h = hash_step(0x452821E638D01377ull, src[q]);
    for (uint32_t a = 0; a < k; ++a) h = hash_step(h, src[delta[(size_t)a * n + q]]);
    h ^= h >> 31;
    h *= 0x94D049BB133111EBull;
    return h ^ (h >> 29);
  }
};

// Exact insert of a signature too wide for one key: the entry is (h, tag |
// representative state), h a 64-bit hash of the signature.  An entry with the
// same h joins q to its block only if eq(q, representative) finds the two full
// signatures equal; otherwise probing goes on, so a hash collision never
// merges blocks.  Entries whose tag (top tagbits bits of .hi) differs from
// `tag` are free.  Returns q's slot; on a full table sets ERR_TABLE_FULL.
template <class Eq>
__device__ uint32_t hashed_insert(u128 *table, uint32_t mask, uint32_t tagbits, uint32_t tag, unsigned long long h,
                                  uint32_t q, const Eq &eq, uint32_t *err) {
  const uint32_t eshift = 64u - tagbits;
  const u128 mine{h, ((unsigned long long)tag << eshift) | q};
  uint32_t slot = (uint32_t)(h >> 32) & mask;
  for (uint64_t iter = 0; iter <= 2ull * ((uint64_t)mask + 1); ++iter) {
    u128 cur = ld_b128_weak(table + slot);
    if ((uint32_t)(cur.hi >> eshift) != tag) {   // free: claim it
      const u128 old = cas_b128(table + slot, cur, mine);
      if (eq128(old, cur)) return slot;
      cur = old;
      if ((uint32_t)(cur.hi >> eshift) != tag) continue;   // replaced by another stale value: retry
    }
    if (cur.lo == h && eq(q, (uint32_t)cur.hi)) return slot;
    slot = (slot + 1u) & mask;
  }
  atomicOr(err, ERR_TABLE_FULL);
  return slot;
}

// ----------------------------------------------------------------- reductions / scans
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (uint32_t o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Block-wide exclusive scan of one value per thread; returns the prefix and
// writes the block total to *total.  `smem` holds blockDim.x/32 words.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *smem, uint32_t *total) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t incl = warp_incl_scan(v);
  if (lane == 31) smem[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = (lane < nw) ? smem[lane] : 0u;
    w = warp_incl_scan(w);
    if (lane < nw) smem[lane] = w;
  }
  __syncthreads();
  const uint32_t warp_prefix = (warp == 0) ? 0u : smem[warp - 1];
  *total = smem[nw - 1];
  __syncthreads();
  return warp_prefix + incl - v;
}

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t *smem) {
  uint32_t total;
  (void)block_excl_scan(v, smem, &total);
  return total;
}

// ----------------------------------------------------------------- staging into shared memory

// Initial labels 0/1 of all n states into lab (16-bit), and the classes seen
// (bit 0: accepting, bit 1: rejecting).  lab is 16-byte aligned.
__device__ __forceinline__ void stage_accept(const uint8_t *__restrict__ acc, uint32_t n, uint16_t *lab,
                                             uint32_t *seen) {
  const uint32_t tid = threadIdx.x, bd = blockDim.x;
  uint32_t head = 0;
  if ((reinterpret_cast<uintptr_t>(acc) & 15u) == 0) {
    const uint32_t n16 = n >> 4;   // 16 states per load
    const uint4 *a4 = reinterpret_cast<const uint4 *>(acc);
    for (uint32_t base = 0; base < n16; base += 4u * bd) {
      uint4 v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t i = base + j * bd + tid;
        v[j] = i < n16 ? a4[i] : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t i = base + j * bd + tid;
        if (i >= n16) continue;
        const uint32_t w[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
        uint32_t o[8];
#pragma unroll
        for (int b = 0; b < 8; ++b) {   // bytes 2b and 2b+1 -> two halfwords
          const uint32_t x = w[b >> 1] >> ((b & 1) * 16);
          const uint32_t lo = (x & 0xFFu) != 0, hi = (x & 0xFF00u) != 0;
          o[b] = lo | (hi << 16);
          *seen |= (lo | hi ? 1u : 0u) | (!lo || !hi ? 2u : 0u);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(lab + 16u * i);
        dst[0] = make_uint4(o[0], o[1], o[2], o[3]);
        dst[1] = make_uint4(o[4], o[5], o[6], o[7]);
      }
    }
    head = n16 << 4;
  }
  for (uint32_t q = head + tid; q < n; q += bd) {
    const uint32_t f = acc[q] != 0;
    lab[q] = (uint16_t)f;
    *seen |= f ? 1u : 2u;
  }
}

// δ (count = k n targets) into 16-bit targets d16 (8-byte aligned); a target
// >= n sets *bad and is stored as 0.
__device__ __forceinline__ void stage_delta(const uint32_t *__restrict__ delta, size_t count, uint32_t n,
                                            uint16_t *d16, uint32_t *bad) {
  const uint32_t tid = threadIdx.x, bd = blockDim.x;
  size_t head = 0;
  if ((reinterpret_cast<uintptr_t>(delta) & 15u) == 0) {
    const size_t c4 = count >> 2;   // 4 targets per load
    const uint4 *d4 = reinterpret_cast<const uint4 *>(delta);
    for (size_t base = 0; base < c4; base += 8u * bd) {
      uint4 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const size_t i = base + (size_t)j * bd + tid;
        v[j] = i < c4 ? d4[i] : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const size_t i = base + (size_t)j * bd + tid;
        if (i >= c4) continue;
        const uint32_t t[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
        uint32_t o[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          *bad |= t[b] >= n;
          o[b] = t[b] < n ? t[b] : 0u;
        }
        *reinterpret_cast<uint2 *>(d16 + 4 * i) = make_uint2(o[0] | (o[1] << 16), o[2] | (o[3] << 16));
      }
    }
    head = c4 << 2;
  }
  for (size_t i = head + tid; i < count; i += bd) {
    const uint32_t d = delta[i];
    *bad |= d >= n;
    d16[i] = (uint16_t)(d < n ? d : 0u);
  }
}

// Arguments of the canonical numbering that ends every refinement kernel.
struct CanonArgs {
  uint32_t n;
  const uint32_t *lab;     // final labels, < label_space
  size_t label_space;
  uint32_t *minrep;        // label_space entries of scratch
  uint8_t *flag;           // n bytes of scratch
  uint32_t *partials;      // gridDim entries
  uint32_t *out;           // n
  Ctrl *ctrl;
  unsigned long long barrier_ns;
  uint32_t min_labels;     // 1: every label already is its block's smallest state
};

// Canonical numbering of the final labels: block id = rank of its smallest
// state.  `B` is the number of blocks (0xFFFFFFFF if unknown).  Labels are
// < label_space.  Returns false if a barrier failed.
static __device__ __noinline__ bool canonicalise(const CanonArgs &A, uint32_t B, uint32_t *s_red) {
  Ctrl *C = A.ctrl;
  const uint32_t n = A.n;
  const uint32_t *__restrict__ lab = A.lab;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  if (B == n) {   // every block is a singleton {q}: its number is q
    for (uint32_t q = tid; q < n; q += stride) A.out[q] = q;
    if (blockIdx.x == 0 && threadIdx.x == 0) C->num_blocks = n;
    return true;
  }
  const size_t S = A.label_space;
  if (!A.min_labels) {   // smallest member per label
    for (size_t i = tid; i < S; i += stride) A.minrep[i] = 0xFFFFFFFFu;
    if (!grid_sync(C, A.barrier_ns)) return false;
    {
      // lanes hold consecutive states, so the lowest lane of a label group holds
      // the group's smallest state: one atomic per (warp, label)
      const uint32_t lane = threadIdx.x & 31u;
      const uint32_t gwarp = tid >> 5, nwarps = stride >> 5;
      for (uint64_t base = (uint64_t)gwarp * 32; base < n; base += (uint64_t)nwarps * 32) {
        const uint32_t q = (uint32_t)base + lane;
        const bool valid = q < n;
        const uint32_t l = valid ? lab[q] : 0u;
        const unsigned grp = __match_any_sync(0xFFFFFFFFu, l) & __ballot_sync(0xFFFFFFFFu, valid);
        if (valid && lane == (uint32_t)(__ffs(grp) - 1)) atomicMin(&A.minrep[l], q);
      }
    }
    if (!grid_sync(C, A.barrier_ns)) return false;
  }
  // contiguous chunk per block, a multiple of blockDim
  uint32_t chunk = (n + gridDim.x - 1) / gridDim.x;
  chunk = (chunk + blockDim.x - 1) / blockDim.x * blockDim.x;
  const uint64_t beg64 = (uint64_t)blockIdx.x * chunk;
  const uint32_t beg = beg64 < n ? (uint32_t)beg64 : n;
  const uint32_t end = (uint64_t)beg + chunk < n ? beg + chunk : n;
  uint32_t cnt = 0;
  for (uint32_t q = beg + threadIdx.x; q < end; q += blockDim.x) {
    const uint8_t f = A.min_labels ? (lab[q] == q) : (A.minrep[lab[q]] == q);
    A.flag[q] = f;
    cnt += f;
  }
  const uint32_t bsum = block_sum(cnt, s_red);
  if (threadIdx.x == 0) A.partials[blockIdx.x] = bsum;
  if (!grid_sync(C, A.barrier_ns)) return false;
  // offset of this block = sum of earlier blocks' counts; total = all
  uint32_t pre = 0, tot = 0;
  for (uint32_t b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const uint32_t v = A.partials[b];
    tot += v;
    if (b < blockIdx.x) pre += v;
  }
  pre = block_sum(pre, s_red);
  tot = block_sum(tot, s_red);
  uint32_t run = pre;
  for (uint32_t base = beg; base < end; base += blockDim.x) {
    const uint32_t q = base + threadIdx.x;
    const uint32_t f = (q < end) ? A.flag[q] : 0u;
    uint32_t tile_total;
    const uint32_t r = block_excl_scan(f, s_red, &tile_total);
    if (f) A.minrep[lab[q]] = run + r;
    run += tile_total;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) C->num_blocks = tot;
  if (!grid_sync(C, A.barrier_ns)) return false;
  for (uint32_t q = tid; q < n; q += stride) A.out[q] = A.minrep[lab[q]];
  return true;
}

}  // namespace dfa
