// dfa_quotient: the minimal DFA itself from the coarsest partition (the
// paper's problem statement asks for a minimal A' with L(A') = L(A); the
// partition of Section 3 is its state set once restricted to the states
// reachable from the start).
//
// One cooperative launch:
//  1. reachability from the start by level-synchronous search (a bitmap of
//     reached states, two frontier arrays, one grid barrier per level); while
//     the frontier is small, block 0 alone runs up to kLocalLevels levels
//     between grid barriers, so that deep unary DFAs do not pay a grid barrier
//     per level;
//  2. each block's smallest reachable state (atomicMin over reachable states);
//  3. the blocks with a reachable state, ranked by that state (a grid-wide
//     scan in state order): the quotient's state numbers;
//  4. the quotient's transitions and acceptance from each block's
//     representative, and its start state.
#include "api_util.h"

namespace dfa {

static constexpr int kQThreads = 512;
static constexpr size_t kMaxGridQ = 8192;
static constexpr uint32_t kLocalMax = 2 * kQThreads;   // frontier size handled by block 0 alone
static constexpr uint32_t kLocalLevels = 4096;         // levels per local run
static constexpr uint32_t kQNone = 0xFFFFFFFFu;

struct QuotArgs {
  const uint32_t *delta;   // k*n
  const uint8_t *accept;   // n
  const uint32_t *block;   // n: the partition (ids < n)
  uint32_t n, k, start;
  uint32_t *seen;          // ceil(n/32) words
  uint32_t *front[2];      // n each
  uint32_t *minr;          // n: smallest reachable state per block id
  uint32_t *newid;         // n: quotient state of a block id
  uint32_t *partials;      // gridDim
  uint32_t *delta_out;     // k*n capacity; row a of the quotient at a*n'
  uint8_t *accept_out;     // n capacity
  uint32_t *result;        // [n', start']
  Ctrl *ctrl;
  unsigned long long timeout_ns, barrier_ns;
};

// Expands frontier entries [i0, size) with stride `step` into the other
// frontier; new states counted in *next (atomic).
__device__ __forceinline__ void expand(const QuotArgs &A, const uint32_t *cur, uint32_t *nxt, uint32_t size,
                                       uint32_t i0, uint32_t step, uint32_t *next) {
  for (uint32_t i = i0; i < size; i += step) {
    const uint32_t q = cur[i];
    for (uint32_t a = 0; a < A.k; ++a) {
      const uint32_t t = A.delta[(size_t)a * A.n + q];
      const uint32_t bit = 1u << (t & 31u);
      if (!(atomicOr(&A.seen[t >> 5], bit) & bit)) nxt[atomicAdd(next, 1u)] = t;
    }
  }
}

__global__ void __launch_bounds__(kQThreads) quotient_kernel(QuotArgs A) {
  __shared__ uint32_t s_red[kQThreads / 32];
  __shared__ uint32_t s_size[2];
  Ctrl *C = A.ctrl;
  const uint32_t n = A.n;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const uint32_t lane = threadIdx.x & 31u, gwarp = tid >> 5, nwarps = stride >> 5;
  if (leader) {
    const unsigned long long t = gtimer();
    C->t_start = t;
    C->deadline = t + A.timeout_ns;
  }
  // validate the targets and the block ids; clear the search state
  const uint64_t kn = (uint64_t)A.k * n;
  for (uint64_t i = tid; i < kn; i += stride)
    if (A.delta[i] >= n) atomicOr(&C->err, ERR_BAD_DELTA);
  for (uint32_t q = tid; q < n; q += stride) {
    if (A.block[q] >= n) atomicOr(&C->err, ERR_BAD_DELTA);
    A.minr[q] = kQNone;
  }
  for (uint32_t i = tid; i < (n + 31) / 32; i += stride) A.seen[i] = 0u;
  bool ok = grid_sync(C, A.barrier_ns);
  // Search state of iteration it, in a ring of three slots: C->cnt[it % 3] =
  // frontier size, C->flag2[it % 3] = frontier buffer.  Iteration it reads its
  // slot and writes the next one; the slot after that was last read in
  // iteration it - 1 (before the barrier that ended it) and is cleared now, so
  // no block ever overwrites a value another block has yet to read.
  if (ok && leader) {
    A.seen[A.start >> 5] |= 1u << (A.start & 31u);
    A.front[0][0] = A.start;
    C->cnt[0] = 1u;   // slot 0: one state, buffer 0 (flag2[0] = 0, slots 1 and 2 zero)
  }
  if (ok) ok = grid_sync(C, A.barrier_ns);

  // 1. reachability
  for (uint32_t it = 0; ok; ++it) {
    const uint32_t s0 = it % 3, s1 = (it + 1) % 3, s2 = (it + 2) % 3;
    const uint32_t size = ld_relaxed(&C->cnt[s0]), cur = ld_relaxed(&C->flag2[s0]);
    if (size == 0u) break;
    if (leader) {
      C->cnt[s2] = 0u;
      C->flag2[s2] = 0u;
    }
    if (size <= kLocalMax) {
      // block 0 runs levels alone while the frontier stays small
      if (blockIdx.x == 0) {
        uint32_t c = cur, sz = size;
        for (uint32_t lvl = 0; lvl < kLocalLevels && sz > 0u && sz <= kLocalMax; ++lvl) {
          if (threadIdx.x == 0) s_size[c ^ 1u] = 0u;
          __syncthreads();
          expand(A, A.front[c], A.front[c ^ 1u], sz, threadIdx.x, blockDim.x, &s_size[c ^ 1u]);
          __syncthreads();
          sz = s_size[c ^ 1u];
          c ^= 1u;
        }
        if (threadIdx.x == 0) {
          C->cnt[s1] = sz;
          C->flag2[s1] = c;
        }
      }
    } else {
      // one level by the whole grid; slot s1 was cleared in the previous iteration
      expand(A, A.front[cur], A.front[cur ^ 1u], size, tid, stride, &C->cnt[s1]);
      if (leader) C->flag2[s1] = cur ^ 1u;
    }
    ok = grid_sync(C, A.barrier_ns);
  }

  // 2. smallest reachable state per block (one atomic per (warp, block))
  if (ok) {
    for (uint64_t base = (uint64_t)gwarp * 32; base < n; base += (uint64_t)nwarps * 32) {
      const uint32_t q = (uint32_t)base + lane;
      const bool r = q < n && ((A.seen[q >> 5] >> (q & 31u)) & 1u);
      const uint32_t b = r ? A.block[q] : kQNone;
      const unsigned grp = __match_any_sync(0xFFFFFFFFu, b) & __ballot_sync(0xFFFFFFFFu, r);
      if (r && lane == (uint32_t)(__ffs(grp) - 1)) atomicMin(&A.minr[b], q);
    }
    ok = grid_sync(C, A.barrier_ns);
  }
  // 3. representatives (reachable q with minr[block[q]] == q) ranked in state order
  uint32_t chunk = (n + gridDim.x - 1) / gridDim.x;
  chunk = (chunk + blockDim.x - 1) / blockDim.x * blockDim.x;
  const uint64_t beg64 = (uint64_t)blockIdx.x * chunk;
  const uint32_t beg = beg64 < n ? (uint32_t)beg64 : n;
  const uint32_t end = (uint64_t)beg + chunk < n ? beg + chunk : n;
  auto is_rep = [&](uint32_t q) {
    return ((A.seen[q >> 5] >> (q & 31u)) & 1u) && A.minr[A.block[q]] == q;
  };
  if (ok) {
    uint32_t cnt = 0;
    for (uint32_t q = beg + threadIdx.x; q < end; q += blockDim.x) cnt += is_rep(q);
    const uint32_t bsum = block_sum(cnt, s_red);
    if (threadIdx.x == 0) A.partials[blockIdx.x] = bsum;
    ok = grid_sync(C, A.barrier_ns);
  }
  uint32_t nq = 0;
  if (ok) {
    uint32_t pre = 0, tot = 0;
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
      const uint32_t v = A.partials[b];
      tot += v;
      if (b < blockIdx.x) pre += v;
    }
    pre = block_sum(pre, s_red);
    nq = block_sum(tot, s_red);
    uint32_t run = pre;
    for (uint32_t base = beg; base < end; base += blockDim.x) {
      const uint32_t q = base + threadIdx.x;
      const uint32_t f = q < end && is_rep(q);
      uint32_t total;
      const uint32_t ex = block_excl_scan(f, s_red, &total);
      if (f) A.newid[A.block[q]] = run + ex;
      run += total;
    }
    ok = grid_sync(C, A.barrier_ns);
  }
  // 4. the quotient's transitions and acceptance from the representatives
  if (ok) {
    for (uint32_t q = tid; q < n; q += stride) {
      if (!is_rep(q)) continue;
      const uint32_t b = A.newid[A.block[q]];
      A.accept_out[b] = A.accept[q];
      for (uint32_t a = 0; a < A.k; ++a) A.delta_out[(size_t)a * nq + b] = A.newid[A.block[A.delta[(size_t)a * n + q]]];
    }
    if (leader) {
      A.result[0] = nq;
      A.result[1] = A.newid[A.block[A.start]];
    }
  }
  if (leader) C->t_end = gtimer();
}

struct QuotLayout {
  size_t ctrl, seen, f0, f1, minr, newid, partials, result, delta, accept, block, dout, aout, total;
};

static QuotLayout quot_layout(uint64_t n, uint32_t k, bool hd, bool ha, bool hb, bool hdo, bool hao) {
  QuotLayout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  L.ctrl = take(sizeof(Ctrl));
  L.seen = take((n + 31) / 32 * 4);
  L.f0 = take(n * 4);
  L.f1 = take(n * 4);
  L.minr = take(n * 4);
  L.newid = take(n * 4);
  L.partials = take(kMaxGridQ * 4);
  L.result = take(8);
  L.delta = hd ? take((size_t)k * n * 4) : SIZE_MAX;
  L.accept = ha ? take(n) : SIZE_MAX;
  L.block = hb ? take(n * 4) : SIZE_MAX;
  L.dout = hdo ? take((size_t)k * n * 4) : SIZE_MAX;
  L.aout = hao ? take(n) : SIZE_MAX;
  L.total = off;
  return L;
}

}  // namespace dfa

using namespace dfa;

extern "C" {

size_t dfa_quotient_workspace_size(const dfa_t *d, const uint32_t *block, const uint32_t *delta_out,
                                   const uint8_t *accept_out) {
  if (check_dfa(d, "dfa") != DFA_OK || !block || (d->k > 0 && !delta_out) || !accept_out) return 0;
  return quot_layout(d->n, d->k, d->k > 0 && !is_device_ptr(d->delta), !is_device_ptr(d->accept),
                     !is_device_ptr(block), d->k > 0 && !is_device_ptr(delta_out), !is_device_ptr(accept_out))
      .total;
}

int dfa_quotient(const dfa_t *d, const uint32_t *block, uint32_t *delta_out, uint8_t *accept_out, uint32_t *n_out,
                 uint32_t *start_out, void *workspace, size_t ws_bytes, void *stream) {
  int rc = check_dfa(d, "dfa");
  if (rc != DFA_OK) return rc;
  if (!block) return fail(DFA_EINVAL, "block is NULL");
  if ((d->k > 0 && !delta_out) || !accept_out) return fail(DFA_EINVAL, "delta_out or accept_out is NULL");
  if (!n_out || !start_out) return fail(DFA_EINVAL, "n_out or start_out is NULL");
  if (!workspace || !aligned(workspace, 256)) return fail(DFA_EINVAL, "workspace NULL or not 256-byte aligned");
  const uint32_t n = d->n, k = d->k;
  const bool hd = k > 0 && !is_device_ptr(d->delta), ha = !is_device_ptr(d->accept), hb = !is_device_ptr(block);
  const bool hdo = k > 0 && !is_device_ptr(delta_out), hao = !is_device_ptr(accept_out);
  const QuotLayout L = quot_layout(n, k, hd, ha, hb, hdo, hao);
  if (ws_bytes < L.total) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
  char *ws = static_cast<char *>(workspace);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  QuotArgs a{};
  a.delta = d->delta;
  a.accept = d->accept;
  a.block = block;
  if (hd) {
    e = cudaMemcpyAsync(ws + L.delta, d->delta, (size_t)k * n * 4, cudaMemcpyHostToDevice, st);
    a.delta = reinterpret_cast<const uint32_t *>(ws + L.delta);
  }
  if (e == cudaSuccess && ha) {
    e = cudaMemcpyAsync(ws + L.accept, d->accept, n, cudaMemcpyHostToDevice, st);
    a.accept = reinterpret_cast<const uint8_t *>(ws + L.accept);
  }
  if (e == cudaSuccess && hb) {
    e = cudaMemcpyAsync(ws + L.block, block, (size_t)n * 4, cudaMemcpyHostToDevice, st);
    a.block = reinterpret_cast<const uint32_t *>(ws + L.block);
  }
  if (e != cudaSuccess) return cuda_fail(e, "copy inputs to device");
  a.n = n;
  a.k = k;
  a.start = d->start;
  a.seen = reinterpret_cast<uint32_t *>(ws + L.seen);
  a.front[0] = reinterpret_cast<uint32_t *>(ws + L.f0);
  a.front[1] = reinterpret_cast<uint32_t *>(ws + L.f1);
  a.minr = reinterpret_cast<uint32_t *>(ws + L.minr);
  a.newid = reinterpret_cast<uint32_t *>(ws + L.newid);
  a.partials = reinterpret_cast<uint32_t *>(ws + L.partials);
  a.delta_out = hdo ? reinterpret_cast<uint32_t *>(ws + L.dout) : delta_out;
  a.accept_out = hao ? reinterpret_cast<uint8_t *>(ws + L.aout) : accept_out;
  a.result = reinterpret_cast<uint32_t *>(ws + L.result);
  a.ctrl = reinterpret_cast<Ctrl *>(ws + L.ctrl);
  const dfa_opts o = default_opts(nullptr);
  a.timeout_ns = o.timeout_ns;
  a.barrier_ns = 5000000000ull;
  e = cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(ctrl)");
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(e, "device attribute");
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, quotient_kernel, kQThreads, 0)) != cudaSuccess)
    return cuda_fail(e, "occupancy");
  const int grid = sms * (per_sm < 1 ? 1 : per_sm);
  if ((size_t)grid > kMaxGridQ) return fail(DFA_ECUDA, "grid too large");
  void *params[] = {&a};
  e = cudaLaunchCooperativeKernel((const void *)quotient_kernel, dim3(grid), dim3(kQThreads), params, 0, st);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the quotient kernel");
  Ctrl c{};
  uint32_t res[2] = {0, 0};
  e = cudaMemcpyAsync(&c, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(res, a.result, 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "quotient kernel");
  if (c.err & ERR_BAD_DELTA) return fail(DFA_EINVAL, "a transition target or a block id is >= n");
  const int status = status_from_ctrl(c);
  if (status != DFA_OK) return status;
  *n_out = res[0];
  *start_out = res[1];
  if (hdo && k > 0) {
    e = cudaMemcpyAsync(delta_out, a.delta_out, (size_t)k * res[0] * 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy quotient to host");
  }
  if (hao) {
    e = cudaMemcpyAsync(accept_out, a.accept_out, res[0], cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy quotient to host");
  }
  if (hdo || hao) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "copy quotient to host");
  }
  return DFA_OK;
}

}  // extern "C"
