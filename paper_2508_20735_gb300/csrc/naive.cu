// naivePR (Section 3.2, Algorithm 2) and transPR (Section 3.4, Algorithm 5) as
// one persistent cooperative kernel.
//
// naivePR: block[q] is a leader state.  Each round, every state q compares,
// letter by letter, the block of δ(q,a) with the block of δ(block[q],a); states
// that differ elect a new leader for their block (the smallest of them: the
// paper's concurrent write made deterministic) and move to it.  Reads within a
// round see the previous round's blocks (double buffering), as in the PRAM
// lock-step model.  It stops after a round in which no state differs.
//
// transPR first extends the alphabet with the letters a^(2^i),
// i = 0..floor(log2 n), by pointer doubling:
//   δT(q, a^(2^i)) = δT(δT(q, a^(2^(i-1))), a^(2^(i-1))),
// one grid-wide step per level, then runs naivePR on the extended DFA.
// Row a*(L+1)+i of the closure table holds δ(., a^(2^i)).
#include "api_util.h"

namespace dfa {

static constexpr int kNaiveThreads = 512;
static constexpr uint32_t kNone = 0xFFFFFFFFu;

struct NaiveArgs {
  const uint32_t *delta;   // k*n, letter-major (validated by the kernel)
  const uint8_t *accept;   // n
  uint32_t n, k;
  uint32_t *dT;            // closure table, k*(L+1) rows of n (transPR); nullptr for naivePR
  uint32_t L;              // floor(log2 n)
  uint32_t *blk[2];        // leaders, ping-pong
  uint32_t *nl[2];         // new_leader per old leader, ping-pong
  uint8_t *diff;           // n: state differs from its leader this round
  uint32_t *minrep;        // n: canonical numbering scratch
  uint8_t *flag;           // n
  uint32_t *partials;      // gridDim
  uint32_t *out;           // n
  Ctrl *ctrl;
  uint32_t max_rounds;
  unsigned long long timeout_ns, barrier_ns;
};

// Validates δ (targets < n; a bad one sets ERR_BAD_DELTA and reads as 0) and,
// with a closure table, copies it to level 0: row a*(L+1) holds δ(., a).
__device__ __forceinline__ void validate_delta(const uint32_t *delta, uint32_t n, uint32_t k, uint32_t *dT,
                                               uint32_t L, Ctrl *C) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const uint64_t kn = (uint64_t)k * n;
  for (uint64_t i = tid; i < kn; i += stride) {
    uint32_t t = delta[i];
    if (t >= n) {
      atomicOr(&C->err, ERR_BAD_DELTA);
      t = 0;
    }
    if (dT) {
      const uint32_t a = (uint32_t)(i / n), q = (uint32_t)(i % n);
      dT[((size_t)a * (L + 1)) * n + q] = t;
    }
  }
}

// Closure levels 1..L by pointer doubling, one grid-wide step per level:
// δT(q, a^(2^i)) = δT(δT(q, a^(2^(i-1))), a^(2^(i-1))).  Level 0 must have been
// written by this launch; returns false if a barrier failed.
__device__ __forceinline__ bool closure_levels(uint32_t n, uint32_t k, uint32_t *dT, uint32_t L, Ctrl *C,
                                               unsigned long long barrier_ns) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const uint64_t kn = (uint64_t)k * n;
  for (uint32_t lvl = 1; lvl <= L; ++lvl) {
    // level lvl-1 (and the level-0 copy) must be complete everywhere
    if (!grid_sync(C, barrier_ns)) return false;
    for (uint64_t i = tid; i < kn; i += stride) {
      const uint32_t a = (uint32_t)(i / n), q = (uint32_t)(i % n);
      const uint32_t *prev = dT + ((size_t)a * (L + 1) + lvl - 1) * n;
      dT[((size_t)a * (L + 1) + lvl) * n + q] = prev[prev[q]];
    }
  }
  return true;
}

// The closure table alone (Algorithm 5's δT), for signature refinement on the
// extended DFA.
__global__ void __launch_bounds__(kNaiveThreads) closure_kernel(const uint32_t *delta, uint32_t n, uint32_t k,
                                                                uint32_t *dT, uint32_t L, Ctrl *C,
                                                                unsigned long long timeout_ns,
                                                                unsigned long long barrier_ns) {
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  if (leader) {
    const unsigned long long t = gtimer();
    C->t_start = t;
    C->deadline = t + timeout_ns;
  }
  validate_delta(delta, n, k, dT, L, C);
  if (closure_levels(n, k, dT, L, C, barrier_ns)) grid_sync(C, barrier_ns);
  if (leader) C->t_end = gtimer();
}

__global__ void __launch_bounds__(kNaiveThreads) naive_kernel(NaiveArgs A) {
  __shared__ uint32_t s_red[kNaiveThreads / 32];
  Ctrl *C = A.ctrl;
  const uint32_t n = A.n, k = A.k;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const uint32_t lane = threadIdx.x & 31u, gwarp = tid >> 5, nwarps = stride >> 5;
  if (leader) {
    const unsigned long long t = gtimer();
    C->t_start = t;
    C->deadline = t + A.timeout_ns;
    C->qf = kNone;
    C->qn = kNone;
  }
  // Transition rows of the DFA being refined: δ itself, or the closure table.
  const uint32_t kT = A.dT ? k * (A.L + 1) : k;
  const uint32_t *T = A.dT ? A.dT : A.delta;

  // --- validate δ (and copy it to closure level 0); reset new_leader
  validate_delta(A.delta, n, k, A.dT, A.L, C);
  for (uint32_t q = tid; q < n; q += stride) {
    A.nl[0][q] = kNone;
    A.nl[1][q] = kNone;
  }
  bool ok = grid_sync(C, A.barrier_ns);

  // --- initial leaders q_f = min F, q_n = min Q\F (one atomic per warp and class)
  if (ok) {
    for (uint64_t base = (uint64_t)gwarp * 32; base < n; base += (uint64_t)nwarps * 32) {
      const uint32_t q = (uint32_t)base + lane;
      const bool valid = q < n;
      const bool acc = valid && A.accept[q] != 0;
      const uint32_t mf = __reduce_min_sync(0xFFFFFFFFu, acc ? q : kNone);
      const uint32_t mn = __reduce_min_sync(0xFFFFFFFFu, (valid && !acc) ? q : kNone);
      if (lane == 0) {
        if (mf != kNone) atomicMin(&C->qf, mf);
        if (mn != kNone) atomicMin(&C->qn, mn);
      }
    }
  }
  // --- closure levels (transPR)
  if (ok && A.dT) ok = closure_levels(n, k, A.dT, A.L, C, A.barrier_ns);
  if (ok) ok = grid_sync(C, A.barrier_ns);
  if (ok) {
    const uint32_t qf = ld_relaxed(&C->qf), qn = ld_relaxed(&C->qn);
    for (uint32_t q = tid; q < n; q += stride) A.blk[0][q] = A.accept[q] != 0 ? qf : qn;
    ok = grid_sync(C, A.barrier_ns);
  }

  uint32_t r = 0, changed = 0, final_buf = 0;
  for (r = 1; ok; ++r) {
    const uint32_t *cur = A.blk[(r - 1) & 1];
    uint32_t *nxt = A.blk[r & 1];
    uint32_t *nlr = A.nl[r & 1];
    uint32_t *nlz = A.nl[(r + 1) & 1];
    uint32_t any = 0;
    // Phase A: compare with the leader; elect the smallest differing state per block.
    for (uint64_t base = (uint64_t)gwarp * 32; base < n; base += (uint64_t)nwarps * 32) {
      const uint32_t q = (uint32_t)base + lane;
      const bool valid = q < n;
      bool d = false;
      uint32_t l = kNone;
      if (valid) {
        l = cur[q];
        // entries of nlz were written (if at all) at leaders of round r-1, which
        // are still leaders now: reset them for round r+1
        if (l == q) nlz[q] = kNone;
        for (uint32_t a = 0; a < kT; ++a) {
          const uint32_t *row = T + (size_t)a * n;
          if (cur[row[q]] != cur[row[l]]) {
            d = true;
            break;
          }
        }
        A.diff[q] = d;
      }
      const unsigned dm = __ballot_sync(0xFFFFFFFFu, d);
      if (dm) {
        const unsigned grp = __match_any_sync(0xFFFFFFFFu, d ? l : kNone) & dm;
        // lanes hold consecutive states: the lowest lane of a group is its smallest state
        if (d && lane == (uint32_t)(__ffs(grp) - 1)) atomicMin(&nlr[l], q);
        any = 1;
      }
    }
    const uint32_t bany = block_sum(any, s_red);
    if (threadIdx.x == 0 && bany) atomicOr(&C->flag2[r % 3], 1u);
    ok = grid_sync(C, A.barrier_ns);
    if (!ok) break;
    const uint32_t split = ld_relaxed(&C->flag2[r % 3]);
    if (leader) C->flag2[(r + 2) % 3] = 0u;
    if (!split) {   // stable: no state differs from its leader
      final_buf = (r - 1) & 1;
      break;
    }
    ++changed;
    // Phase B: differing states move to their block's new leader.
    for (uint32_t q = tid; q < n; q += stride) {
      const uint32_t l = cur[q];
      nxt[q] = A.diff[q] ? nlr[l] : l;
    }
    ok = grid_sync(C, A.barrier_ns);
    if (!ok) break;
    final_buf = r & 1;
    if (A.max_rounds != 0u && r >= A.max_rounds) {
      if (leader) C->maxed = 1u;
      break;
    }
  }
  if (ok) {
    if (leader) {
      C->rounds_executed = r;
      C->rounds_changed = changed;
    }
    // leaders are the smallest members of their blocks (Algorithm 2 with min-leader election)
    ok = canonicalise(CanonArgs{n, A.blk[final_buf], (size_t)n, A.minrep, A.flag, A.partials, A.out, C,
                                A.barrier_ns, 1u},
                      0xFFFFFFFFu, s_red);
  }
  if (leader) C->t_end = gtimer();
}

static constexpr size_t kMaxGridN = 8192;

struct NaiveLayout {
  uint32_t L;
  size_t ctrl, blk0, blk1, nl0, nl1, diff, minrep, flag, partials, dT, delta, accept, out, total;
};

static NaiveLayout naive_layout(uint64_t n, uint32_t k, bool trans, bool stage_delta, bool stage_accept) {
  NaiveLayout Lo{};
  Lo.L = (uint32_t)(63 - __builtin_clzll(n));
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  Lo.ctrl = take(sizeof(Ctrl));
  Lo.blk0 = take(n * 4);
  Lo.blk1 = take(n * 4);
  Lo.nl0 = take(n * 4);
  Lo.nl1 = take(n * 4);
  Lo.diff = take(n);
  Lo.minrep = take(n * 4);
  Lo.flag = take(n);
  Lo.partials = take(kMaxGridN * 4);
  Lo.dT = trans ? take((size_t)k * (Lo.L + 1) * n * 4) : SIZE_MAX;
  Lo.delta = stage_delta ? take((size_t)k * n * 4) : SIZE_MAX;
  Lo.accept = stage_accept ? take(n) : SIZE_MAX;
  Lo.out = take(n * 4);
  Lo.total = off;
  return Lo;
}

size_t naive_workspace_size(const dfa_t *d, const dfa_opts &o) {
  const bool hd = d->k > 0 && !is_device_ptr(d->delta);
  const bool ha = !is_device_ptr(d->accept);
  return naive_layout(d->n, d->k, o.algo == DFA_ALGO_TRANS, hd, ha).total;
}

int run_naive_minimise(const dfa_t *d, const dfa_opts &o, uint32_t *block_out, dfa_result *res, void *workspace,
                       size_t ws_bytes, cudaStream_t st) {
  const bool trans = o.algo == DFA_ALGO_TRANS;
  const bool hd = d->k > 0 && !is_device_ptr(d->delta);
  const bool ha = !is_device_ptr(d->accept);
  const bool ho = !is_device_ptr(block_out);
  const NaiveLayout Lo = naive_layout(d->n, d->k, trans, hd, ha);
  if (ws_bytes < Lo.total) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, Lo.total);
  char *ws = static_cast<char *>(workspace);
  cudaError_t e;
  NaiveArgs a{};
  a.delta = d->delta;
  a.accept = d->accept;
  if (hd) {
    e = cudaMemcpyAsync(ws + Lo.delta, d->delta, (size_t)d->k * d->n * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy delta to device");
    a.delta = reinterpret_cast<const uint32_t *>(ws + Lo.delta);
  }
  if (ha) {
    e = cudaMemcpyAsync(ws + Lo.accept, d->accept, d->n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy accept to device");
    a.accept = reinterpret_cast<const uint8_t *>(ws + Lo.accept);
  }
  a.n = d->n;
  a.k = d->k;
  a.L = Lo.L;
  a.dT = trans ? reinterpret_cast<uint32_t *>(ws + Lo.dT) : nullptr;
  a.blk[0] = reinterpret_cast<uint32_t *>(ws + Lo.blk0);
  a.blk[1] = reinterpret_cast<uint32_t *>(ws + Lo.blk1);
  a.nl[0] = reinterpret_cast<uint32_t *>(ws + Lo.nl0);
  a.nl[1] = reinterpret_cast<uint32_t *>(ws + Lo.nl1);
  a.diff = reinterpret_cast<uint8_t *>(ws + Lo.diff);
  a.minrep = reinterpret_cast<uint32_t *>(ws + Lo.minrep);
  a.flag = reinterpret_cast<uint8_t *>(ws + Lo.flag);
  a.partials = reinterpret_cast<uint32_t *>(ws + Lo.partials);
  uint32_t *out = ho ? reinterpret_cast<uint32_t *>(ws + Lo.out) : block_out;
  a.out = out;
  a.ctrl = reinterpret_cast<Ctrl *>(ws + Lo.ctrl);
  a.max_rounds = o.max_rounds;
  a.timeout_ns = o.timeout_ns;
  a.barrier_ns = o.timeout_ns < 5000000000ull ? o.timeout_ns : 5000000000ull;
  e = cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(ctrl)");
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(e, "device attribute");
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, naive_kernel, kNaiveThreads, 0)) != cudaSuccess)
    return cuda_fail(e, "occupancy");
  const int grid = sms * (per_sm < 1 ? 1 : per_sm);
  if ((size_t)grid > kMaxGridN) return fail(DFA_ECUDA, "grid too large");
  void *params[] = {&a};
  e = cudaLaunchCooperativeKernel((const void *)naive_kernel, dim3(grid), dim3(kNaiveThreads), params, 0, st);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the naivePR kernel");
  Ctrl c{};
  e = cudaMemcpyAsync(&c, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(ctrl)");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "naivePR kernel");
  const int status = status_from_ctrl(c);
  if (res) {
    res->num_blocks = c.num_blocks;
    res->rounds_changed = c.rounds_changed;
    res->rounds_executed = c.rounds_executed;
    res->status = status;
    res->device_ns = c.t_end - c.t_start;
  }
  if (status != DFA_OK && status != DFA_EMAXROUNDS) return status;
  if (ho) {
    e = cudaMemcpyAsync(block_out, out, (size_t)d->n * 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy blocks to host");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "copy blocks to host");
  }
  return status;
}

// Builds the closure table of a device-resident DFA into dT (k * (L+1) rows of
// n, L = floor(log2 n)); fills *ctrl_host (ERR_BAD_DELTA for a target >= n).
int run_closure(const uint32_t *delta_dev, uint32_t n, uint32_t k, uint32_t *dT, Ctrl *ctrl_dev, const dfa_opts &o,
                cudaStream_t st, Ctrl *ctrl_host) {
  const uint32_t L = (uint32_t)(63 - __builtin_clzll((unsigned long long)n));
  cudaError_t e = cudaMemsetAsync(ctrl_dev, 0, sizeof(Ctrl), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(ctrl)");
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(e, "device attribute");
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, closure_kernel, kNaiveThreads, 0)) != cudaSuccess)
    return cuda_fail(e, "occupancy");
  const int grid = sms * (per_sm < 1 ? 1 : per_sm);
  if ((size_t)grid > kMaxGridN) return fail(DFA_ECUDA, "grid too large");
  unsigned long long timeout_ns = o.timeout_ns;
  unsigned long long barrier_ns = o.timeout_ns < 5000000000ull ? o.timeout_ns : 5000000000ull;
  void *params[] = {&delta_dev, &n, &k, &dT, const_cast<uint32_t *>(&L), &ctrl_dev, &timeout_ns, &barrier_ns};
  e = cudaLaunchCooperativeKernel((const void *)closure_kernel, dim3(grid), dim3(kNaiveThreads), params, 0, st);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the closure kernel");
  e = cudaMemcpyAsync(ctrl_host, ctrl_dev, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "closure kernel");
  return DFA_OK;
}

}  // namespace dfa
