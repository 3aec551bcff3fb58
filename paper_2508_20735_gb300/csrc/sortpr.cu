// sortPR (Section 3.3, Algorithm 4) with a hand-written LSD radix sort:
// every round sorts the states by their signature
//   (block[q], block[δ(q,a_0)], ..., block[δ(q,a_{k-1})]),
// marks each state whose signature differs from its predecessor's in sorted
// order, and numbers the blocks by an inclusive scan of the marks; the round
// loop stops when the count does not grow.  This is the paper's own
// renumbering (a sort, an adjacent difference and a scan per round, the count
// read back on the host each round), kept beside the hash renumbering of
// moore.cu as the A/B comparison.  Same partition and round counts.
//
// The sort runs over the k+1 signature components from the last letter to the
// own block, 8 bits of a component per pass (only as many bits as the previous
// count needs).  A pass is three steps: a digit histogram per chunk of 4,096
// positions (digits kept as bytes), one exclusive scan of the digit-major
// histogram (which gives every (digit, chunk) its output offset), and a stable
// scatter that ranks equal digits inside a chunk with warp match masks.
#include <chrono>

#include "api_util.h"

namespace dfa {

static constexpr int kSThreads = 256;
static constexpr int kSItems = 16;                         // positions per thread and chunk
static constexpr uint32_t kSChunk = kSThreads * kSItems;   // 4,096
static constexpr int kScanItems = 8;
static constexpr uint32_t kScanBlock = kSThreads * kScanItems;   // 2,048

struct SortCtrl {
  uint32_t err;       // bit 0: a transition target >= n
  uint32_t any_acc, any_rej;
};

__global__ void sort_validate_kernel(const uint32_t *__restrict__ delta, const uint8_t *__restrict__ accept, uint32_t n,
                                     uint32_t k, uint32_t *__restrict__ lab, SortCtrl *ctrl) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const size_t total = (size_t)k * n;
  bool bad = false, acc = false, rej = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) bad |= delta[i] >= n;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) {
    const uint32_t f = accept[q] != 0;
    lab[q] = f;
    acc |= f;
    rej |= !f;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctrl->err, 1u);
  if (__syncthreads_or(acc) && threadIdx.x == 0) atomicOr(&ctrl->any_acc, 1u);
  if (__syncthreads_or(rej) && threadIdx.x == 0) atomicOr(&ctrl->any_rej, 1u);
}

// Component c of state q's signature: its own block (c = 0) or the block of
// its a_{c-1}-successor.
__device__ __forceinline__ uint32_t sig_component(const uint32_t *__restrict__ delta, const uint32_t *__restrict__ lab,
                                                  uint32_t n, uint32_t c, uint32_t q) {
  return c == 0 ? lab[q] : lab[delta[(size_t)(c - 1) * n + q]];
}

__global__ void __launch_bounds__(kSThreads) sort_hist_kernel(const uint32_t *__restrict__ perm,
                                                              const uint32_t *__restrict__ delta,
                                                              const uint32_t *__restrict__ lab, uint32_t n, uint32_t c,
                                                              uint32_t shift, uint8_t *__restrict__ dig,
                                                              uint32_t *__restrict__ hist, uint32_t nb) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const size_t base = (size_t)blockIdx.x * kSChunk;
#pragma unroll 4
  for (int j = 0; j < kSItems; ++j) {
    const size_t i = base + (size_t)j * kSThreads + threadIdx.x;
    if (i < n) {
      const uint32_t d = (sig_component(delta, lab, n, c, perm[i]) >> shift) & 0xFFu;
      dig[i] = (uint8_t)d;
      atomicAdd(&h[d], 1u);
    }
  }
  __syncthreads();
  hist[(size_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one chunk: positions are taken 256 at a time in order;
// inside such a group, warp w's lanes come before warp w+1's.
__global__ void __launch_bounds__(kSThreads) sort_scatter_kernel(const uint32_t *__restrict__ perm,
                                                                 const uint8_t *__restrict__ dig,
                                                                 const uint32_t *__restrict__ offs, uint32_t n,
                                                                 uint32_t nb, uint32_t *__restrict__ perm_out) {
  constexpr int kWarps = kSThreads / 32;
  __shared__ uint32_t base[256];
  __shared__ uint32_t wc[kWarps][256];
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  base[threadIdx.x] = offs[(size_t)threadIdx.x * nb + blockIdx.x];
  const size_t chunk = (size_t)blockIdx.x * kSChunk;
  for (int j = 0; j < kSItems; ++j) {
#pragma unroll
    for (int x = 0; x < kWarps; ++x) wc[x][threadIdx.x] = 0;
    __syncthreads();
    const size_t i = chunk + (size_t)j * kSThreads + threadIdx.x;
    const bool valid = i < n;
    const uint32_t d = valid ? dig[i] : 0x100u;
    const uint32_t v = valid ? perm[i] : 0u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = __popc(peers & ((1u << lane) - 1u));
    if (valid && before == 0) wc[w][d] = __popc(peers);
    __syncthreads();
    {   // per digit: exclusive prefix over the warps, then advance the digit's base
      const uint32_t t = threadIdx.x;
      uint32_t s = base[t];
#pragma unroll
      for (int x = 0; x < kWarps; ++x) {
        const uint32_t cnt = wc[x][t];
        wc[x][t] = s;
        s += cnt;
      }
      base[t] = s;
    }
    __syncthreads();
    if (valid) perm_out[wc[w][d] + before] = v;
    __syncthreads();
  }
}

// flag[i] = 1 if the signature at sorted position i differs from the one at i-1.
__global__ void sort_mark_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ delta,
                                 const uint32_t *__restrict__ lab, uint32_t n, uint32_t k,
                                 uint32_t *__restrict__ flag) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint32_t f = 1;
    if (i > 0) {
      const uint32_t q = perm[i], p = perm[i - 1];
      f = 0;
      for (uint32_t c = 0; c <= k && !f; ++c)
        f = sig_component(delta, lab, n, c, q) != sig_component(delta, lab, n, c, p);
    }
    flag[i] = f;
  }
}

// Block-level scan of 2,048 values: each block scans its slice in place
// (exclusive or inclusive) and writes the slice's total to part[block].
__global__ void __launch_bounds__(kSThreads) scan_block_kernel(uint32_t *__restrict__ x, size_t m, int inclusive,
                                                               uint32_t *__restrict__ part) {
  __shared__ uint32_t warp_sum[kSThreads / 32];
  const size_t base = (size_t)blockIdx.x * kScanBlock + (size_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < m ? x[base + j] : 0u;
    s += v[j];
  }
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  uint32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) warp_sum[w] = incl;
  __syncthreads();
  uint32_t wbase = 0;
  for (uint32_t x2 = 0; x2 < w; ++x2) wbase += warp_sum[x2];
  uint32_t run = wbase + incl - s;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const uint32_t e = run;
    run += v[j];
    if (base + j < m) x[base + j] = inclusive ? run : e;
  }
  if (threadIdx.x == kSThreads - 1) part[blockIdx.x] = run;
}

// Exclusive scan of the block totals by one block (any count, in slices of
// blockDim.x with a carried sum); the grand total goes to *total.
__global__ void scan_parts_kernel(uint32_t *__restrict__ part, uint32_t m, uint32_t *__restrict__ total) {
  __shared__ uint32_t warp_sum[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (uint32_t b = 0; b < m; b += blockDim.x) {
    const uint32_t i = b + threadIdx.x;
    const uint32_t v = i < m ? part[i] : 0u;
    uint32_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) warp_sum[w] = incl;
    __syncthreads();
    uint32_t wbase = 0;
    for (uint32_t x = 0; x < w; ++x) wbase += warp_sum[x];
    const uint32_t c0 = carry;
    if (i < m) part[i] = c0 + wbase + incl - v;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (uint32_t x = 0; x < nw; ++x) t += warp_sum[x];
      carry = c0 + t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void scan_add_kernel(uint32_t *__restrict__ x, size_t m, const uint32_t *__restrict__ part) {
  const uint32_t add = part[blockIdx.x];
  const size_t base = (size_t)blockIdx.x * kScanBlock;
  for (uint32_t j = threadIdx.x; j < kScanBlock; j += blockDim.x)
    if (base + j < m) x[base + j] += add;
}

// new block of the state at sorted position i: the inclusive count of marks - 1.
__global__ void sort_label_kernel(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ flag, uint32_t n,
                                  uint32_t *__restrict__ lab_out) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) lab_out[perm[i]] = flag[i] - 1;
}

__global__ void sort_iota_kernel(uint32_t *__restrict__ perm, uint32_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) perm[i] = (uint32_t)i;
}

// Canonical numbering: minrep[label] = smallest state, then the rank of that
// state among all representatives.
__global__ void sort_minrep_kernel(const uint32_t *__restrict__ lab, uint32_t n, uint32_t *__restrict__ minrep) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride)
    atomicMin(&minrep[lab[q]], (uint32_t)q);
}

__global__ void sort_first_kernel(const uint32_t *__restrict__ lab, const uint32_t *__restrict__ minrep, uint32_t n,
                                  uint32_t *__restrict__ flag) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride)
    flag[q] = minrep[lab[q]] == (uint32_t)q;
}

__global__ void sort_canon_kernel(const uint32_t *__restrict__ lab, const uint32_t *__restrict__ minrep,
                                  const uint32_t *__restrict__ rank, uint32_t n, uint32_t *__restrict__ out) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += stride) out[q] = rank[minrep[lab[q]]];
}

struct SortLayout {
  uint32_t nb;      // sort chunks
  size_t hist_n;    // 256 * nb
  size_t lab0, lab1, perm0, perm1, dig, flag, hist, part, minrep, ctrl, total, delta, accept, out, bytes;
};

static size_t scan_parts(size_t m) { return (m + kScanBlock - 1) / kScanBlock; }

static SortLayout sort_layout(uint32_t n, uint32_t k, bool hd, bool ha, bool ho) {
  SortLayout L{};
  L.nb = (uint32_t)((n + kSChunk - 1) / kSChunk);
  L.hist_n = (size_t)256 * L.nb;
  size_t off = 0;
  auto take = [&](size_t b) {
    const size_t at = off;
    off += (b + 255) / 256 * 256;
    return at;
  };
  const size_t m = (size_t)n > L.hist_n ? (size_t)n : L.hist_n;
  L.lab0 = take((size_t)n * 4);
  L.lab1 = take((size_t)n * 4);
  L.perm0 = take((size_t)n * 4);
  L.perm1 = take((size_t)n * 4);
  L.dig = take(n);
  L.flag = take((size_t)n * 4);
  L.hist = take(L.hist_n * 4);
  L.part = take(scan_parts(m) * 4);
  L.minrep = take((size_t)n * 4);
  L.ctrl = take(sizeof(SortCtrl));
  L.total = take(4);
  L.delta = hd ? take((size_t)k * n * 4) : SIZE_MAX;
  L.accept = ha ? take(n) : SIZE_MAX;
  L.out = ho ? take((size_t)n * 4) : SIZE_MAX;
  L.bytes = off;
  return L;
}

size_t sort_workspace_size(const dfa_t *d, bool hd, bool ha, bool ho) {
  return sort_layout(d->n, d->k, hd, ha, ho).bytes;
}

static uint32_t grid_for(size_t items) {
  const size_t b = (items + kSThreads - 1) / kSThreads;
  return (uint32_t)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

// Scan of m values in place (exclusive or inclusive); *total_dev gets the sum.
static cudaError_t device_scan(uint32_t *x, size_t m, bool inclusive, uint32_t *part, uint32_t *total_dev,
                               cudaStream_t st) {
  const size_t nbk = scan_parts(m);
  scan_block_kernel<<<(unsigned)nbk, kSThreads, 0, st>>>(x, m, inclusive ? 1 : 0, part);
  scan_parts_kernel<<<1, 1024, 0, st>>>(part, (uint32_t)nbk, total_dev);
  scan_add_kernel<<<(unsigned)nbk, kSThreads, 0, st>>>(x, m, part);
  return cudaGetLastError();
}

static uint32_t bits_for(uint32_t max_label) {
  uint32_t b = 1;
  while (b < 32 && (max_label >> b) != 0) ++b;
  return b;
}

int run_sort_minimise(const dfa_t *d, const dfa_opts &o, uint32_t *block_out, dfa_result *res, void *workspace,
                      size_t ws_bytes, cudaStream_t st) {
  const uint32_t n = d->n, k = d->k;
  const bool hd = k > 0 && !is_device_ptr(d->delta), ha = !is_device_ptr(d->accept), ho = !is_device_ptr(block_out);
  const SortLayout L = sort_layout(n, k, hd, ha, ho);
  if (ws_bytes < L.bytes) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, L.bytes);
  char *ws = static_cast<char *>(workspace);
  const auto t0 = std::chrono::steady_clock::now();
  const uint32_t *delta = d->delta;
  const uint8_t *accept = d->accept;
  cudaError_t e = cudaSuccess;
  if (hd) {
    e = cudaMemcpyAsync(ws + L.delta, d->delta, (size_t)k * n * 4, cudaMemcpyHostToDevice, st);
    delta = reinterpret_cast<const uint32_t *>(ws + L.delta);
  }
  if (e == cudaSuccess && ha) {
    e = cudaMemcpyAsync(ws + L.accept, d->accept, n, cudaMemcpyHostToDevice, st);
    accept = reinterpret_cast<const uint8_t *>(ws + L.accept);
  }
  if (e != cudaSuccess) return cuda_fail(e, "copy inputs to device");
  uint32_t *lab[2] = {reinterpret_cast<uint32_t *>(ws + L.lab0), reinterpret_cast<uint32_t *>(ws + L.lab1)};
  uint32_t *perm[2] = {reinterpret_cast<uint32_t *>(ws + L.perm0), reinterpret_cast<uint32_t *>(ws + L.perm1)};
  uint8_t *dig = reinterpret_cast<uint8_t *>(ws + L.dig);
  uint32_t *flag = reinterpret_cast<uint32_t *>(ws + L.flag);
  uint32_t *hist = reinterpret_cast<uint32_t *>(ws + L.hist);
  uint32_t *part = reinterpret_cast<uint32_t *>(ws + L.part);
  uint32_t *minrep = reinterpret_cast<uint32_t *>(ws + L.minrep);
  uint32_t *total = reinterpret_cast<uint32_t *>(ws + L.total);
  SortCtrl *ctrl = reinterpret_cast<SortCtrl *>(ws + L.ctrl);
  uint32_t *out = ho ? reinterpret_cast<uint32_t *>(ws + L.out) : block_out;
  const uint32_t g = grid_for(n);

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if ((e = cudaEventCreate(&ev0)) != cudaSuccess || (e = cudaEventCreate(&ev1)) != cudaSuccess) {
    if (ev0) cudaEventDestroy(ev0);
    return cuda_fail(e, "cudaEventCreate");
  }
  struct EvGuard {
    cudaEvent_t a, b;
    ~EvGuard() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } guard{ev0, ev1};
  cudaEventRecord(ev0, st);
  e = cudaMemsetAsync(ctrl, 0, sizeof(SortCtrl), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const size_t vn = (size_t)k * n > n ? (size_t)k * n : n;
  sort_validate_kernel<<<grid_for(vn), kSThreads, 0, st>>>(delta, accept, n, k, lab[0], ctrl);
  SortCtrl c{};
  e = cudaMemcpyAsync(&c, ctrl, sizeof c, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "sortPR validation");
  if (c.err) return fail(DFA_EINVAL, "a transition target is >= n");

  uint32_t count = c.any_acc + c.any_rej, max_label = c.any_acc ? 1u : 0u;
  uint32_t cur = 0, rounds = 0, changed = 0;
  int status = DFA_OK;
  for (;;) {
    if (o.max_rounds && rounds == o.max_rounds) {
      status = fail(DFA_EMAXROUNDS, "max_rounds reached before the fixpoint");
      break;
    }
    if (o.timeout_ns && (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                            std::chrono::steady_clock::now() - t0).count() > o.timeout_ns)
      return fail(DFA_ETIMEOUT, "time limit exceeded after %u rounds", rounds);
    ++rounds;
    // sort the states by signature: components k, k-1, ..., 0; 8 bits a pass
    const uint32_t w = bits_for(max_label);
    sort_iota_kernel<<<g, kSThreads, 0, st>>>(perm[0], n);
    uint32_t pc = 0;
    for (uint32_t cc = k + 1; cc-- > 0;) {
      for (uint32_t sh = 0; sh < w; sh += 8) {
        sort_hist_kernel<<<L.nb, kSThreads, 0, st>>>(perm[pc], delta, lab[cur], n, cc, sh, dig, hist, L.nb);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "radix histogram");
        if ((e = device_scan(hist, L.hist_n, false, part, nullptr, st)) != cudaSuccess)
          return cuda_fail(e, "radix offsets");
        sort_scatter_kernel<<<L.nb, kSThreads, 0, st>>>(perm[pc], dig, hist, n, L.nb, perm[pc ^ 1]);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "radix scatter");
        pc ^= 1;
      }
    }
    // adjacent difference + inclusive scan = the new blocks
    sort_mark_kernel<<<g, kSThreads, 0, st>>>(perm[pc], delta, lab[cur], n, k, flag);
    if ((e = device_scan(flag, n, true, part, total, st)) != cudaSuccess) return cuda_fail(e, "block numbering");
    sort_label_kernel<<<g, kSThreads, 0, st>>>(perm[pc], flag, n, lab[cur ^ 1]);
    uint32_t next = 0;
    e = cudaMemcpyAsync(&next, total, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "sortPR round");
    cur ^= 1;
    max_label = next - 1;
    const bool grew = next > count;
    count = next;
    if (!grew) break;
    ++changed;
    if ((o.flags & DFA_FLAG_STOP_DISCRETE) && count == n) break;
  }
  // canonical numbering by smallest member
  e = cudaMemsetAsync(minrep, 0xFF, (size_t)n * 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(minrep)");
  sort_minrep_kernel<<<g, kSThreads, 0, st>>>(lab[cur], n, minrep);
  sort_first_kernel<<<g, kSThreads, 0, st>>>(lab[cur], minrep, n, flag);
  if ((e = device_scan(flag, n, false, part, nullptr, st)) != cudaSuccess) return cuda_fail(e, "canonical ranks");
  sort_canon_kernel<<<g, kSThreads, 0, st>>>(lab[cur], minrep, flag, n, out);
  cudaEventRecord(ev1, st);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "canonical numbering");
  if (ho) {
    e = cudaMemcpyAsync(block_out, out, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy blocks to host");
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "sortPR");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, ev0, ev1);
  if (res) {
    res->num_blocks = count;
    res->rounds_changed = changed;
    res->rounds_executed = rounds;
    res->status = status;
    res->device_ns = (uint64_t)((double)ms * 1e6);
  }
  return status;
}

}  // namespace dfa
