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

StagePlan make_plan(uint32_t k, uint32_t bits) {
  StagePlan p{};
  const uint32_t total = k + 1;     // own block + one per letter
  const uint32_t cap = 125;         // key bits; at least 3 bits remain for the epoch
  p.bits = bits;
  if ((uint64_t)total * bits <= cap) {
    p.first = total;
    p.per = 1;
    p.stages = 1;
    const uint32_t used = total * bits;
    p.ebits = (128 - used) > 32 ? 32 : (128 - used);
  } else {
    p.first = cap / bits;
    p.per = cap / bits - 1;
    p.stages = 1 + (total - p.first + p.per - 1) / p.per;
    const uint32_t used = p.first * bits;
    p.ebits = (128 - used) > 32 ? 32 : (128 - used);
  }
  return p;
}

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
      shift = bits;
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

template <int VEC>
__global__ void __launch_bounds__(kThreads) moore_kernel(MooreArgs A) {
  __shared__ uint32_t s_red[kThreads / 32];
  __shared__ CtaCache cache;
  Ctrl *C = A.ctrl;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  if (leader) {
    const unsigned long long t = gtimer();
    C->t_start = t;
    C->deadline = t + A.timeout_ns;
    C->sep_round = 0xFFFFFFFFu;
  }
  const uint32_t emax = A.ebits >= 32 ? 0xFFFFFFFFu : ((1u << A.ebits) - 1u);
  uint32_t epoch = 0, r = 0, changed = 0, B_prev = 0, final_buf = 0, B_final = 0xFFFFFFFFu;
  bool ok = true, separated = false, skip = false;

  // Equivalence by union: the empty word already separates start states that
  // differ in acceptance (round 0).
  if (A.track_pair && ((A.accept[A.sep_a] != 0) != (A.accept[A.sep_b] != 0))) {
    separated = true;
    if (leader) C->sep_round = 0;
    if (A.early_exit) {
      skip = true;   // the answer needs no round; report the initial partition
      const uint32_t stride = gridDim.x * blockDim.x;
      for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < A.n; q += stride)
        A.lab[0][q] = A.accept[q] != 0;
    }
  }
  if (!skip) clear_table(A.table, A.log2S);
  ok = grid_sync(C, A.barrier_ns);
  for (r = 1; ok && !skip; ++r) {
    const bool round1 = r == 1;
    const StagePlan &P = round1 ? A.plan1 : A.planr;
    const uint32_t *src = A.lab[(r - 1) & 1];
    uint32_t *dst = A.lab[r & 1];
    uint32_t local_new = 0, seen = 0;
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
    if (leader) C->cnt[(r + 2) % 3] = 0u;
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
    ok = canonicalise(CanonArgs{A.n, A.lab[final_buf], (size_t)1 << A.log2S, A.minrep, A.flag, A.partials, A.out,
                                A.ctrl, A.barrier_ns},
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
