// dfa_product_check: equivalence or inclusion by exploring the synchronous
// product of two DFAs (Section 4's naive Hopcroft-Karp variant, Algorithm 6
// without R+, which the paper runs on a GPU model checker; here as one
// cooperative kernel of this library).
//
// The explored set R of state pairs is a lock-free open-addressing set of
// 64-bit keys (p << 32) | q (all ones = empty: p, q < 2^31).  The search is breadth first, one
// grid barrier per level; while a level holds at most kPLocalMax pairs, block 0
// alone runs up to kPLocalLevels levels between grid barriers.  Every pair of a
// level is tested before the level's expansion counts: a pair with exactly one
// accepting state (equivalence) or with A accepting and B not (inclusion)
// ends the search once its level is complete, and that level is the length of
// a shortest counterexample.  The search state (frontier size and buffer, level,
// pairs so far) lives in a ring of three slots, as in the quotient kernel, so no
// block overwrites a value another has yet to read.
#include "api_util.h"

namespace dfa {

static constexpr int kPThreads = 512;
static constexpr size_t kMaxGridP = 8192;
static constexpr uint32_t kPLocalMax = 2 * kPThreads;
static constexpr uint32_t kPLocalLevels = 4096;

// Search state, one slot per iteration (ring of three): iteration it reads
// slot it % 3 and writes slot (it + 1) % 3; the third slot, last read in
// iteration it - 1, is cleared in iteration it.  Every in-kernel decision
// reads a slot no block writes during the iteration.
struct ProdRing {
  uint32_t size[3], buf[3], level[3];
  uint32_t vio[3];                // grid levels: a pair of the level read in the previous slot violates
  uint32_t stop[3];               // stop before this slot's iteration (violation found by a local run)
  unsigned long long pairs[3];    // pairs in the levels before this slot's level
  // results, read by the host only
  unsigned long long res_pairs;   // pairs explored
  uint32_t res_level;             // level of a first violation
  uint32_t violated, done;
};

struct ProdArgs {
  const uint32_t *dA, *dB;        // k*nA, k*nB letter-major
  const uint8_t *aA, *aB;
  uint32_t nA, nB, k, sA, sB, inclusion;
  unsigned long long *set;        // 2^log2set keys
  uint32_t log2set;
  unsigned long long *front[2];   // cap pairs each
  unsigned long long cap;         // max_pairs
  ProdRing *ring;
  Ctrl *ctrl;
  unsigned long long timeout_ns, barrier_ns;
};

static constexpr unsigned long long kEmptyKey = ~0ull;

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long pmix(unsigned long long x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  return x;
}

// Inserts key into the set; true if it was not there.  A full set raises
// ERR_TABLE_FULL (reported as DFA_ENOMEM) and returns false.  A slot changes
// once, from empty to a key, so a plain read that finds a key is final: only
// slots read as empty take an atomic (about half the successors of a level
// are already in the set, and atomics that miss L2 are the costly accesses).
__device__ __forceinline__ bool set_insert(const ProdArgs &A, unsigned long long key) {
  const unsigned long long mask = (1ull << A.log2set) - 1;
  unsigned long long slot = pmix(key) & mask;
  for (unsigned long long it = 0; it <= mask; ++it) {
    unsigned long long old = ld_relaxed_u64(&A.set[slot]);
    if (old == kEmptyKey) {
      old = atomicCAS(&A.set[slot], kEmptyKey, key);
      if (old == kEmptyKey) return true;
    }
    if (old == key) return false;
    slot = (slot + 1) & mask;
  }
  atomicOr(&A.ctrl->err, ERR_TABLE_FULL);
  return false;
}

__device__ __forceinline__ bool violates(const ProdArgs &A, uint32_t p, uint32_t q) {
  const bool a = A.aA[p] != 0, b = A.aB[q] != 0;
  return A.inclusion ? (a && !b) : (a != b);
}

// Tests and expands pairs [i0, size) (stride `step`) of frontier `cur` into
// `nxt`, counting new pairs in *next; sets *bad if a pair violates.  The lanes
// of a warp that found new pairs for the same letter take their frontier
// positions with one atomicAdd (a single counter taking one atomicAdd per new
// pair serialises the level).
__device__ __forceinline__ void expand_pairs(const ProdArgs &A, const unsigned long long *cur,
                                             unsigned long long *nxt, uint32_t size, uint32_t i0, uint32_t step,
                                             uint32_t *next, uint32_t *bad) {
  const uint32_t lane = threadIdx.x & 31u;
  for (uint32_t i = i0; i < size; i += step) {
    const uint32_t act = __activemask();
    const unsigned long long key = cur[i];
    const uint32_t p = (uint32_t)(key >> 32), q = (uint32_t)key;
    if (violates(A, p, q)) atomicOr(bad, 1u);
    for (uint32_t a = 0; a < A.k; ++a) {
      const uint32_t tp = A.dA[(size_t)a * A.nA + p], tq = A.dB[(size_t)a * A.nB + q];
      const unsigned long long nk = ((unsigned long long)tp << 32) | tq;
      const bool fresh = set_insert(A, nk);
      const uint32_t m = __ballot_sync(act, fresh);
      if (m == 0u) continue;
      const uint32_t first = __ffs(act) - 1;
      uint32_t base = 0;
      if (lane == first) base = atomicAdd(next, (uint32_t)__popc(m));
      base = __shfl_sync(act, base, first);
      if (fresh) {
        const uint32_t at = base + __popc(m & ((1u << lane) - 1u));
        if (at < A.cap) nxt[at] = nk;
        else atomicOr(&A.ctrl->err, ERR_TABLE_FULL);
      }
    }
  }
}

__global__ void __launch_bounds__(kPThreads) product_kernel(const __grid_constant__ ProdArgs A) {
  __shared__ uint32_t s_size[2], s_bad;
  Ctrl *C = A.ctrl;
  ProdRing *R = A.ring;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  if (leader) {
    const unsigned long long t = gtimer();
    C->t_start = t;
    C->deadline = t + A.timeout_ns;
  }
  // validate the targets; clear the set
  for (uint64_t i = tid; i < (uint64_t)A.k * A.nA; i += stride)
    if (A.dA[i] >= A.nA) atomicOr(&C->err, ERR_BAD_DELTA);
  for (uint64_t i = tid; i < (uint64_t)A.k * A.nB; i += stride)
    if (A.dB[i] >= A.nB) atomicOr(&C->err, ERR_BAD_DELTA);
  for (uint64_t i = tid; i < (1ull << A.log2set); i += stride) A.set[i] = kEmptyKey;
  bool ok = grid_sync(C, A.barrier_ns);
  if (ok && leader) {
    const unsigned long long k0 = ((unsigned long long)A.sA << 32) | A.sB;
    set_insert(A, k0);
    A.front[0][0] = k0;
    R->size[0] = 1u;   // slot 0: one pair, buffer 0, level 0, no pairs before it
  }
  if (ok) ok = grid_sync(C, A.barrier_ns);

  for (uint32_t it = 0; ok; ++it) {
    const uint32_t s0 = it % 3, s1 = (it + 1) % 3, s2 = (it + 2) % 3;
    const uint32_t size = ld_relaxed(&R->size[s0]), cur = ld_relaxed(&R->buf[s0]), lvl = ld_relaxed(&R->level[s0]);
    const unsigned long long before = R->pairs[s0];
    if (ld_relaxed(&R->stop[s0])) break;   // a local run found a violation (results written)
    if (size == 0u) {   // every reachable pair explored: the condition holds
      if (leader) {
        R->res_pairs = before;
        R->done = 1u;
      }
      break;
    }
    if (leader) {
      R->size[s2] = 0u;
      R->buf[s2] = 0u;
      R->level[s2] = 0u;
      R->vio[s2] = 0u;
      R->stop[s2] = 0u;
      R->pairs[s2] = 0ull;
    }
    if (size <= kPLocalMax) {
      // block 0 runs levels alone while they stay small
      if (blockIdx.x == 0) {
        uint32_t c = cur, sz = size, l = lvl, bad = 0;
        unsigned long long pb = before;
        // a level whose new pairs overflow the frontier (ERR_TABLE_FULL is set by
        // expand_pairs) ends the run: entries past `cap` were never written
        bool over = false;
        for (uint32_t n = 0; n < kPLocalLevels && sz > 0u && sz <= kPLocalMax && !bad && !over; ++n) {
          if (threadIdx.x == 0) {
            s_size[c ^ 1u] = 0u;
            s_bad = 0u;
          }
          __syncthreads();
          expand_pairs(A, A.front[c], A.front[c ^ 1u], sz, threadIdx.x, blockDim.x, &s_size[c ^ 1u], &s_bad);
          __syncthreads();
          bad = s_bad;
          const uint32_t next = s_size[c ^ 1u];
          __syncthreads();   // every thread has read s_bad before thread 0 resets it
          over = next > A.cap;
          if (!bad && !over) {   // the level is clean: move on
            pb += sz;
            sz = next;
            c ^= 1u;
            ++l;
          }
        }
        if (threadIdx.x == 0) {
          if (bad) {
            R->res_pairs = pb + sz;
            R->res_level = l;
            R->violated = 1u;
            R->done = 1u;
            R->stop[s1] = 1u;
          }
          R->size[s1] = sz;
          R->buf[s1] = c;
          R->level[s1] = l;
          R->pairs[s1] = pb;
        }
      }
    } else {
      // one level by the whole grid; slot s1 was cleared in the previous iteration
      expand_pairs(A, A.front[cur], A.front[cur ^ 1u], size, tid, stride, &R->size[s1], &R->vio[s1]);
      if (leader) {
        R->buf[s1] = cur ^ 1u;
        R->level[s1] = lvl + 1;
        R->pairs[s1] = before + size;
      }
    }
    ok = grid_sync(C, A.barrier_ns);
    if (!ok) break;
    if (size > kPLocalMax && ld_relaxed(&R->vio[s1])) {   // a pair of level lvl violated
      if (leader) {
        R->res_pairs = before + size;
        R->res_level = lvl;
        R->violated = 1u;
        R->done = 1u;
      }
      break;
    }
    if (R->pairs[s1] > A.cap) {   // more pairs than the caller allowed
      if (leader) atomicOr(&C->err, ERR_TABLE_FULL);
      break;
    }
  }
  if (leader) C->t_end = gtimer();
}

struct ProdLayout {
  uint32_t log2set;
  size_t ctrl, ring, set, f0, f1, dA, aA, dB, aB, total;
};

static ProdLayout prod_layout(const dfa_t *a, const dfa_t *b, uint64_t max_pairs, bool hdA, bool haA, bool hdB,
                              bool haB) {
  ProdLayout L{};
  L.log2set = ceil_log2(2 * (max_pairs < 16 ? 16 : max_pairs));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  L.ctrl = take(sizeof(Ctrl));
  L.ring = take(sizeof(ProdRing));
  L.set = take(((size_t)1 << L.log2set) * 8);
  L.f0 = take((size_t)max_pairs * 8);
  L.f1 = take((size_t)max_pairs * 8);
  L.dA = hdA ? take((size_t)a->k * a->n * 4) : SIZE_MAX;
  L.aA = haA ? take(a->n) : SIZE_MAX;
  L.dB = hdB ? take((size_t)b->k * b->n * 4) : SIZE_MAX;
  L.aB = haB ? take(b->n) : SIZE_MAX;
  L.total = off;
  return L;
}

// max_pairs never exceeds n_A n_B, nor kMaxPairs: frontier sizes and positions
// are 32-bit, and a grid-stride walk over a frontier must not wrap.
static constexpr uint64_t kMaxPairs = 1ull << 31;

static uint64_t clamp_pairs(const dfa_t *a, const dfa_t *b, uint64_t max_pairs) {
  const uint64_t all = (uint64_t)a->n * b->n;
  if (max_pairs > all) max_pairs = all;
  return max_pairs > kMaxPairs ? kMaxPairs : max_pairs;
}

}  // namespace dfa

using namespace dfa;

extern "C" {

size_t dfa_product_workspace_size(const dfa_t *a, const dfa_t *b, uint64_t max_pairs) {
  if (check_dfa(a, "a") != DFA_OK || check_dfa(b, "b") != DFA_OK || a->k != b->k || max_pairs == 0) return 0;
  max_pairs = clamp_pairs(a, b, max_pairs);
  return prod_layout(a, b, max_pairs, a->k > 0 && !is_device_ptr(a->delta), !is_device_ptr(a->accept),
                     b->k > 0 && !is_device_ptr(b->delta), !is_device_ptr(b->accept))
      .total;
}

int dfa_product_check(const dfa_t *a, const dfa_t *b, int mode, uint64_t max_pairs, int *holds, uint64_t *pairs,
                      int64_t *cex_len, void *workspace, size_t ws_bytes, void *stream) {
  int rc = check_dfa(a, "a");
  if (rc == DFA_OK) rc = check_dfa(b, "b");
  if (rc != DFA_OK) return rc;
  if (a->k != b->k) return fail(DFA_EINVAL, "alphabets differ: k_A = %u, k_B = %u", a->k, b->k);
  if (mode != DFA_CHECK_EQUIVALENCE && mode != DFA_CHECK_INCLUSION) return fail(DFA_EINVAL, "unknown mode %d", mode);
  if (max_pairs == 0) return fail(DFA_EINVAL, "max_pairs is 0");
  if (!holds) return fail(DFA_EINVAL, "holds is NULL");
  if (!workspace || !aligned(workspace, 256)) return fail(DFA_EINVAL, "workspace NULL or not 256-byte aligned");
  max_pairs = clamp_pairs(a, b, max_pairs);
  const bool hdA = a->k > 0 && !is_device_ptr(a->delta), haA = !is_device_ptr(a->accept);
  const bool hdB = b->k > 0 && !is_device_ptr(b->delta), haB = !is_device_ptr(b->accept);
  const ProdLayout L = prod_layout(a, b, max_pairs, hdA, haA, hdB, haB);
  if (ws_bytes < L.total) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
  char *ws = static_cast<char *>(workspace);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  ProdArgs p{};
  p.dA = a->delta;
  p.aA = a->accept;
  p.dB = b->delta;
  p.aB = b->accept;
  auto stage = [&](size_t at, const void *src, size_t bytes) -> const void * {
    if (e == cudaSuccess) e = cudaMemcpyAsync(ws + at, src, bytes, cudaMemcpyHostToDevice, st);
    return ws + at;
  };
  if (hdA) p.dA = static_cast<const uint32_t *>(stage(L.dA, a->delta, (size_t)a->k * a->n * 4));
  if (haA) p.aA = static_cast<const uint8_t *>(stage(L.aA, a->accept, a->n));
  if (hdB) p.dB = static_cast<const uint32_t *>(stage(L.dB, b->delta, (size_t)b->k * b->n * 4));
  if (haB) p.aB = static_cast<const uint8_t *>(stage(L.aB, b->accept, b->n));
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.ctrl, 0, sizeof(Ctrl), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.ring, 0, sizeof(ProdRing), st);
  if (e != cudaSuccess) return cuda_fail(e, "stage the product check");
  p.nA = a->n;
  p.nB = b->n;
  p.k = a->k;
  p.sA = a->start;
  p.sB = b->start;
  p.inclusion = mode == DFA_CHECK_INCLUSION;
  p.set = reinterpret_cast<unsigned long long *>(ws + L.set);
  p.log2set = L.log2set;
  p.front[0] = reinterpret_cast<unsigned long long *>(ws + L.f0);
  p.front[1] = reinterpret_cast<unsigned long long *>(ws + L.f1);
  p.cap = max_pairs;
  p.ring = reinterpret_cast<ProdRing *>(ws + L.ring);
  p.ctrl = reinterpret_cast<Ctrl *>(ws + L.ctrl);
  p.timeout_ns = default_opts(nullptr).timeout_ns;
  p.barrier_ns = 5000000000ull;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(e, "device attribute");
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, product_kernel, kPThreads, 0)) != cudaSuccess)
    return cuda_fail(e, "occupancy");
  const int grid = sms * (per_sm < 1 ? 1 : per_sm);
  if ((size_t)grid > kMaxGridP) return fail(DFA_ECUDA, "grid too large");
  void *params[] = {&p};
  e = cudaLaunchCooperativeKernel((const void *)product_kernel, dim3(grid), dim3(kPThreads), params, 0, st);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the product kernel");
  Ctrl c{};
  ProdRing r{};
  e = cudaMemcpyAsync(&c, p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&r, p.ring, sizeof(ProdRing), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "product kernel");
  if (c.err & ERR_BAD_DELTA) return fail(DFA_EINVAL, "a transition target is >= n");
  if (c.err & ERR_TABLE_FULL)
    return fail(DFA_ENOMEM, "the product has more than max_pairs = %llu reachable pairs", (unsigned long long)max_pairs);
  const int status = status_from_ctrl(c);
  if (status != DFA_OK) return status;
  if (!r.done) return fail(DFA_ECUDA, "product search ended without a result");
  *holds = r.violated ? 0 : 1;
  if (pairs) *pairs = r.res_pairs;
  if (cex_len) *cex_len = r.violated ? (int64_t)r.res_level : -1;
  return DFA_OK;
}

}  // extern "C"
