// C ABI (include/dfa.h): argument checks, workspace layout, host staging and
// launches.  Every step of the refinement runs in the kernels of this library.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/dfa.h"
#include "api_util.h"
#include "common.cuh"
#include "internal.h"

namespace dfa {

static thread_local std::string g_err;

int fail(int status, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return status;
}

int cuda_fail(cudaError_t e, const char *what) {
  return fail(DFA_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_device_ptr(const void *p) {
  if (p == nullptr) return true;
  cudaPointerAttributes at;
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

uint32_t ceil_log2(uint64_t x) {   // smallest b with 2^b >= x
  return x <= 1 ? 0u : 64u - (uint32_t)__builtin_clzll(x - 1);
}

dfa_opts default_opts(const dfa_opts *o) {
  dfa_opts d;
  memset(&d, 0, sizeof d);
  d.algo = DFA_ALGO_MOORE;
  d.schedule = -1;
  if (o) d = *o;
  if (d.timeout_ns == 0) d.timeout_ns = 600ull * 1000000000ull;
  return d;
}

int check_dfa(const dfa_t *d, const char *name) {
  if (!d) return fail(DFA_EINVAL, "%s is NULL", name);
  if (d->n == 0) return fail(DFA_EINVAL, "%s: n = 0", name);
  if (d->n > DFA_MAX_STATES) return fail(DFA_EINVAL, "%s: n = %u exceeds %u", name, d->n, DFA_MAX_STATES);
  if (d->k > DFA_MAX_LETTERS) return fail(DFA_EINVAL, "%s: k = %u exceeds %u", name, d->k, DFA_MAX_LETTERS);
  if (d->start >= d->n) return fail(DFA_EINVAL, "%s: start %u >= n %u", name, d->start, d->n);
  if (d->k > 0 && d->delta == nullptr) return fail(DFA_EINVAL, "%s: delta is NULL", name);
  if (d->accept == nullptr) return fail(DFA_EINVAL, "%s: accept is NULL", name);
  return DFA_OK;
}

// ------------------------------------------------------------------ Moore workspace
static constexpr size_t kMaxGrid = 8192;

// Per-device launch facts of the Moore kernels, looked up once per device
// (under a mutex: calls may come from several host threads).
struct DeviceFacts {
  bool known;
  int sms;                 // multiprocessors
  size_t warps;            // warps of the largest cooperative grid any Moore kernel uses
};
static constexpr int kMaxDevices = 64;
static std::mutex g_facts_mu;
static DeviceFacts g_facts[kMaxDevices];

// Without a visible device: the largest grid the launcher accepts, 148 SMs.
static DeviceFacts device_facts() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return DeviceFacts{false, 148, kMaxGrid * 16};
  }
  std::lock_guard<std::mutex> lock(g_facts_mu);
  if (g_facts[dev].known) return g_facts[dev];
  DeviceFacts f{false, 148, 0};
  if (cudaDeviceGetAttribute(&f.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return DeviceFacts{false, 148, kMaxGrid * 16};
  }
  for (uint32_t v : {1u, 2u, 4u}) {
    LaunchInfo li{};
    if (moore_grid(v, &li) != cudaSuccess) {
      cudaGetLastError();
      return DeviceFacts{false, f.sms, kMaxGrid * 16};
    }
    f.warps = std::max(f.warps, (size_t)li.grid * (li.block / 32));
  }
  // the bucketed kernel: one block of 1024 threads per SM
  f.warps = std::max(f.warps, (size_t)f.sms * 32);
  f.known = true;
  g_facts[dev] = f;
  return f;
}

static size_t moore_max_warps() { return device_facts().warps; }

// ------------------------------------------------------------------ bucketed gather plan
static constexpr size_t kBucketSmem = 200 * 1024;   // dynamic shared memory of the bucketed kernel
static constexpr uint64_t kBucketMaxStates = 1u << 26;
static constexpr uint32_t kBucketMaxLetters = 16;
static constexpr size_t kStreamRingBytes = 4 * 2048 * 6;   // assemble: 4 stages of 2048 (es, val) entries
static constexpr size_t kDedupBytes = ((1u << 15) + (1u << 15) / 32) * 4;   // dedup hash set + duplicate bits

// Bucket sizes for n states, k letters on a grid of `grid` blocks, within
// the shared memory of one block:
//   prep      2 counters per target bucket + the region being built (4 bytes an entry);
//   gather    BT labels + the bucket's segment table (8 bytes per source bucket);
//   assemble  per state of a source bucket max(4k, 8) bytes of tile (and sort)
//             and 4 of own label or hash; the region stream's ring; 8 bytes
//             per partition;
//   dedup     a partition's hashes (pcap words), 2^15 set slots, duplicate bits.
// Source buckets are as large as the assemble pass allows, target buckets as
// large as the gather pass then allows; both counts are rounded to a multiple
// of the grid so that every block gets the same number of buckets.  BS and BT
// are multiples of 8 (aligned bulk copies).  Partitions hold about 8 K hashes
// (a quarter more room, plus 256, before a partition overflows).
static bool bucket_plan(uint64_t n, uint32_t k, uint64_t grid, BucketPlan *bp) {
  if (k < 1 || k > kBucketMaxLetters || n < 1 || n > kBucketMaxStates || grid < 1) return false;
  BucketPlan b{};
  uint32_t pbits = 0;
  while (((n + (1ull << pbits) - 1) >> pbits) > 8192) ++pbits;
  b.pbits = pbits;
  b.P = 1u << pbits;
  const uint64_t per = (n + b.P - 1) / b.P;
  b.pcap = (uint32_t)((per + per / 4 + 256 + 7) / 8 * 8);
  const size_t dedup = (size_t)b.pcap * 4 + kDedupBytes;
  // source buckets
  const uint64_t tw = std::max<uint64_t>(4ull * k, 8) + 4;
  const uint64_t fixed = kStreamRingBytes + 8ull * b.P + 64;
  if (fixed >= kBucketSmem) return false;
  uint64_t bs_max = std::min<uint64_t>({(kBucketSmem - fixed) / tw, 65534 / k, 16384});
  bs_max = bs_max / 8 * 8;
  const uint64_t mS = (n + grid * bs_max - 1) / (grid * bs_max);
  uint64_t BS = (n + grid * mS - 1) / (grid * mS);
  BS = (BS + 7) / 8 * 8;
  b.BS = (uint32_t)BS;
  b.NS = (uint32_t)((n + BS - 1) / BS);
  // target buckets: labels beside the segment table
  if (8ull * b.NS + 64 >= kBucketSmem) return false;
  const uint64_t bt_max = std::min<uint64_t>(65528, (kBucketSmem - 8ull * b.NS - 64) / 4) / 8 * 8;
  if (bt_max < 8) return false;
  const uint64_t mT = (n + grid * bt_max - 1) / (grid * bt_max);
  uint64_t BT = (n + grid * mT - 1) / (grid * mT);
  BT = (BT + 7) / 8 * 8;
  b.BT = (uint32_t)BT;
  b.NT = (uint32_t)((n + BT - 1) / BT);
  b.cap = (uint32_t)(((uint64_t)k * BS + 7ull * b.NT + 7) / 8 * 8);
  const size_t prep = 8ull * ((b.NT + 3) / 4 * 4) + 4ull * b.cap;
  const size_t gather = (size_t)BT * 4 + 8ull * b.NS;
  const size_t assemble = (size_t)(std::max<uint64_t>(k, 2) * BS + BS + 2ull * b.P) * 4 + kStreamRingBytes;
  b.smem = std::max({prep, gather, assemble, dedup});
  // the device divides by BT with a 48-bit reciprocal: products stay below NT * 2^48 < 2^64
  if (b.smem > kBucketSmem || b.NT >= (1u << 15) || b.pcap >= (1u << 15) * 2 / 3) return false;
  if ((uint64_t)b.NS * b.cap >= (1ull << 32)) return false;   // entry indices are 32-bit
  *bp = b;
  return true;
}

// Opt-in: on GB300 the direct label reads (served by L2 at its random-request
// rate) measured faster than the bucketed passes at every size tried, 2^23 to
// 2^26 states with 4 letters.
bool choose_bucket(uint64_t n, uint32_t k, uint32_t flags, BucketPlan *bp) {
  if ((flags & DFA_FLAG_GATHER) || !(flags & DFA_FLAG_BUCKETED)) return false;
  (void)n;
  return bucket_plan(n, k, (uint64_t)device_facts().sms, bp);
}

MooreLayout moore_layout(uint64_t n, uint32_t k, bool stage_delta, bool stage_accept, bool stage_out,
                         const BucketPlan *bp) {
  MooreLayout L{};
  L.log2S = ceil_log2(n * 2 < 64 ? 64 : n * 2);
  L.mbits = L.log2S + 2 < 31 ? L.log2S + 2 : 31;
  L.wid = ceil_log2(n) > 0 ? ceil_log2(n) : 1;
  // every table key (exact-table or filter rounds) has at most
  // min(125, (k+1)*log2S) bits; the epoch tag takes the rest, at most 32
  const uint64_t keymax = (uint64_t)(k + 1) * L.log2S < 125 ? (uint64_t)(k + 1) * L.log2S : 125;
  L.ebits = 128 - keymax > 32 ? 32 : (uint32_t)(128 - keymax);
  const size_t S = (size_t)1 << L.log2S;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  L.ctrl = take(sizeof(Ctrl));
  L.table = take(S * 16);
  L.rep = take(S * 8);
  L.lab0 = take(n * 4);
  L.lab1 = take(n * 4);
  L.tmp = take(n * 4);
  const size_t warps = moore_max_warps();
  L.warps = warps;
  L.dups = take((n + (warps + 2) * 32) * 4);   // n plus one partial chunk per warp
  L.dups2 = take((n + (warps + 2) * 32) * 4);
  L.wcnt = take(warps * 4);
  L.minrep = take(S * 4);
  L.flag = take(n);
  L.partials = take(kMaxGrid * 4);
  L.bm0 = take(S / 8 > 4 ? S / 8 : 4);
  L.bm1 = take(S / 8 > 4 ? S / 8 : 4);
  L.seen1 = take(((size_t)1 << L.mbits) / 8);
  L.seen2 = take(((size_t)1 << L.mbits) / 8);
  L.seen3 = take(((size_t)1 << L.mbits) / 16);
  L.seen4 = take(((size_t)1 << L.mbits) / 16);
  L.tmp2 = take(n * 4);
  L.delta = stage_delta ? take((size_t)k * n * 4) : SIZE_MAX;
  L.accept = stage_accept ? take(n) : SIZE_MAX;
  L.out = stage_out ? take(n * 4) : SIZE_MAX;
  if (bp) {
    L.bucket = true;
    L.plan = *bp;
    const size_t entries = (size_t)bp->NS * bp->cap;
    L.et = take(entries * 2);
    L.es = take(entries * 2);
    L.val = take(entries * 4);
    L.seg = take((size_t)bp->NT * bp->NS * 8);
    L.used = take((size_t)bp->NS * 4);
    L.phash = take((size_t)bp->P * bp->pcap * 4);
    L.pq = take((size_t)bp->P * bp->pcap * 4);
    L.pcnt = take((size_t)bp->P * 4);
    L.list = take(n * 4);
  }
  L.total = off;
  return L;
}

// Runs the Moore kernel over a device-resident DFA (delta/accept are device
// pointers) writing canonical blocks to out_dev.  Fills *ctrl_host.
int enqueue_moore(const uint32_t *delta_dev, const uint8_t *accept_dev, uint32_t n, uint32_t k, uint32_t *out_dev,
                  const MooreLayout &L, char *ws, const dfa_opts &o, cudaStream_t st, const PairTrack *track,
                  uint32_t vec_ok, bool independent_letters) {
  MooreArgs a{};
  a.delta = delta_dev;
  a.accept = accept_dev;
  a.n = n;
  a.k = k;
  a.lab[0] = reinterpret_cast<uint32_t *>(ws + L.lab0);
  a.lab[1] = reinterpret_cast<uint32_t *>(ws + L.lab1);
  a.tmp = reinterpret_cast<uint32_t *>(ws + L.tmp);
  a.table = reinterpret_cast<u128 *>(ws + L.table);
  a.log2S = L.log2S;
  a.minrep = reinterpret_cast<uint32_t *>(ws + L.minrep);
  a.bm[0] = reinterpret_cast<uint32_t *>(ws + L.bm0);
  a.bm[1] = reinterpret_cast<uint32_t *>(ws + L.bm1);
  a.seen1 = reinterpret_cast<uint32_t *>(ws + L.seen1);
  a.seen2 = reinterpret_cast<uint32_t *>(ws + L.seen2);
  a.seen3 = reinterpret_cast<uint32_t *>(ws + L.seen3);
  a.seen4 = reinterpret_cast<uint32_t *>(ws + L.seen4);
  a.tmp2 = reinterpret_cast<uint32_t *>(ws + L.tmp2);
  a.mbits = L.mbits;
  a.rep = reinterpret_cast<unsigned long long *>(ws + L.rep);
  a.dups = reinterpret_cast<uint32_t *>(ws + L.dups);
  a.dups2 = reinterpret_cast<uint32_t *>(ws + L.dups2);
  a.wcnt = reinterpret_cast<uint32_t *>(ws + L.wcnt);
  a.wid = L.wid;
  a.modes = (o.flags & DFA_FLAG_TABLE_ONLY) ? 0u : 3u;
  a.stop_discrete = (o.flags & DFA_FLAG_STOP_DISCRETE) ? 1u : 0u;
  a.flag = reinterpret_cast<uint8_t *>(ws + L.flag);
  a.partials = reinterpret_cast<uint32_t *>(ws + L.partials);
  a.out = out_dev;
  a.ctrl = reinterpret_cast<Ctrl *>(ws + L.ctrl);
  a.ebits = L.ebits;
  a.max_rounds = o.max_rounds;
  a.timeout_ns = o.timeout_ns;
  a.barrier_ns = o.timeout_ns < 5000000000ull ? o.timeout_ns : 5000000000ull;
  a.vec = vec_ok;
  a.stream_delta = ((uint64_t)k * n * 4 > (64ull << 20)) ? 1u : 0u;
  // filter rounds from the sparse-signature estimate: only for a DFA's own letters (closure letters
  // are powers of one letter, far from independent), not for a union (its states come in pairs),
  // and only from 2^20 states on (below, a filter round's extra grid barriers cost more than the
  // table round's random inserts: 117 against 101 us at 10,000 states)
  a.predict_sparse = (independent_letters && !track && n >= (1u << 20)) ? 1u : 0u;
  if (track) {
    a.track_pair = 1;
    a.sep_a = track->a;
    a.sep_b = track->b;
    a.early_exit = track->early_exit;
  }
  if (L.bucket) {
    const BucketPlan &b = L.plan;
    a.bucket = 1;
    a.vec = 1;
    a.B_smem = b.smem;
    a.B.NT = b.NT;
    a.B.BT = b.BT;
    a.B.NS = b.NS;
    a.B.BS = b.BS;
    a.B.cap = b.cap;
    a.B.P = b.P;
    a.B.pbits = b.pbits;
    a.B.pcap = b.pcap;
    a.B.et = reinterpret_cast<uint16_t *>(ws + L.et);
    a.B.es = reinterpret_cast<uint16_t *>(ws + L.es);
    a.B.val = reinterpret_cast<uint32_t *>(ws + L.val);
    a.B.seg = reinterpret_cast<uint2 *>(ws + L.seg);
    a.B.used = reinterpret_cast<uint32_t *>(ws + L.used);
    a.B.phash = reinterpret_cast<uint32_t *>(ws + L.phash);
    a.B.pq = reinterpret_cast<uint32_t *>(ws + L.pq);
    a.B.pcnt = reinterpret_cast<uint32_t *>(ws + L.pcnt);
    a.B.list = reinterpret_cast<uint32_t *>(ws + L.list);
  }
  cudaError_t e = cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(ctrl)");
  LaunchInfo li{};
  e = moore_grid(a.vec, &li, a.bucket ? a.B_smem : 0);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  if ((size_t)li.grid > kMaxGrid) return fail(DFA_ECUDA, "grid of %d blocks exceeds %zu", li.grid, kMaxGrid);
  if ((size_t)li.grid * (li.block / 32) > L.warps)   // the per-warp lists would overrun
    return fail(DFA_ECUDA, "launch of %zu warps exceeds the %zu the workspace layout holds (internal error)",
                (size_t)li.grid * (li.block / 32), L.warps);
  e = launch_moore(a, st, &li);
  if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of the refinement kernel");
  return DFA_OK;
}

int run_moore(const uint32_t *delta_dev, const uint8_t *accept_dev, uint32_t n, uint32_t k, uint32_t *out_dev,
              const MooreLayout &L, char *ws, const dfa_opts &o, cudaStream_t st, const PairTrack *track,
              Ctrl *ctrl_host, uint32_t vec_ok, bool independent_letters) {
  const int rc = enqueue_moore(delta_dev, accept_dev, n, k, out_dev, L, ws, o, st, track, vec_ok, independent_letters);
  if (rc != DFA_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(ctrl_host, ws + L.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(ctrl)");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "refinement kernel");
  return DFA_OK;
}

int status_from_ctrl(const Ctrl &c) {
  if (c.err & ERR_BAD_DELTA) return fail(DFA_EINVAL, "a transition target is >= n");
  if (c.err & ERR_TIMEOUT) return fail(DFA_ETIMEOUT, "device-side wait or call time limit exceeded");
  if (c.err & ERR_TABLE_FULL) return fail(DFA_ECUDA, "renumbering table overflow (internal error)");
  if (c.maxed) return fail(DFA_EMAXROUNDS, "max_rounds reached before the fixpoint");
  return DFA_OK;
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// States per thread in the Moore kernel: `schedule` 1, 2 or 4 asks for that
// width; otherwise 1 (measured fastest on GB300 for both deep-round and
// bandwidth-bound inputs).  A width needs n divisible by it and aligned rows.
uint32_t pick_vec(uint32_t n, uint32_t k, const void *delta, const void *accept, int32_t schedule) {
  uint32_t want = (schedule == 1 || schedule == 2 || schedule == 4) ? (uint32_t)schedule : 1u;
  while (want > 1) {
    if (n % want == 0 && (k == 0 || aligned(delta, 4 * want)) && aligned(accept, want)) return want;
    want >>= 1;
  }
  return 1;
}

}  // namespace dfa

namespace dfa {

// Signature refinement on the closure DFA: [closure table | Moore workspace for
// (n, k (L+1)) letters | staged δ when the caller passes host memory].
struct ClosureMooreLayout {
  uint32_t L;
  size_t dT, moore, delta, total;
  MooreLayout m;
};

static ClosureMooreLayout closure_moore_layout(uint64_t n, uint32_t k, bool stage_delta, bool stage_accept) {
  ClosureMooreLayout C{};
  C.L = (uint32_t)(63 - __builtin_clzll((unsigned long long)n));
  const size_t rows = (size_t)k * (C.L + 1);
  C.dT = 0;
  C.moore = (rows * n * 4 + 255) / 256 * 256;
  C.m = moore_layout(n, (uint32_t)rows, false, stage_accept, true);
  C.delta = C.moore + (C.m.total + 255) / 256 * 256;
  C.total = C.delta + (stage_delta ? ((size_t)k * n * 4 + 255) / 256 * 256 : 0);
  return C;
}

static int run_closure_moore(const dfa_t *d, const dfa_opts &o, uint32_t *block_out, dfa_result *res,
                             void *workspace, size_t ws_bytes, cudaStream_t st) {
  const bool hd = d->k > 0 && !is_device_ptr(d->delta);
  const bool ha = !is_device_ptr(d->accept);
  const bool ho = !is_device_ptr(block_out);
  const ClosureMooreLayout C = closure_moore_layout(d->n, d->k, hd, ha);
  if (ws_bytes < C.total) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, C.total);
  char *ws = static_cast<char *>(workspace);
  char *wm = ws + C.moore;
  const uint32_t *delta = d->delta;
  const uint8_t *accept = d->accept;
  cudaError_t e;
  if (hd) {
    e = cudaMemcpyAsync(ws + C.delta, d->delta, (size_t)d->k * d->n * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy delta to device");
    delta = reinterpret_cast<const uint32_t *>(ws + C.delta);
  }
  if (ha) {
    e = cudaMemcpyAsync(wm + C.m.accept, d->accept, d->n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy accept to device");
    accept = reinterpret_cast<const uint8_t *>(wm + C.m.accept);
  }
  uint32_t *dT = reinterpret_cast<uint32_t *>(ws + C.dT);
  Ctrl cc{};
  int rc = run_closure(delta, d->n, d->k, dT, reinterpret_cast<Ctrl *>(wm + C.m.ctrl), o, st, &cc);
  if (rc != DFA_OK) return rc;
  rc = status_from_ctrl(cc);
  if (rc != DFA_OK) return rc;
  const uint32_t rows = d->k * (C.L + 1);
  uint32_t *out = ho ? reinterpret_cast<uint32_t *>(wm + C.m.out) : block_out;
  Ctrl c{};
  rc = run_moore(dT, accept, d->n, rows, out, C.m, wm, o, st, nullptr, &c, 1u, false);
  if (rc != DFA_OK) return rc;
  const int status = status_from_ctrl(c);
  if (res) {
    res->num_blocks = c.num_blocks;
    res->rounds_changed = c.rounds_changed;
    res->rounds_executed = c.rounds_executed;
    res->status = status;
    res->device_ns = (cc.t_end - cc.t_start) + (c.t_end - c.t_start);
  }
  if (status != DFA_OK && status != DFA_EMAXROUNDS) return status;
  if (ho) {
    e = cudaMemcpyAsync(block_out, out, (size_t)d->n * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "copy blocks to host");
  }
  return status;
}

}  // namespace dfa

using namespace dfa;

extern "C" {

const char *dfa_last_error(void) { return g_err.c_str(); }

const char *dfa_version(void) { return "dfa_gb300 0.1 (sm_103a)"; }

size_t dfa_workspace_size(const dfa_t *d, const dfa_opts *opts) {
  if (check_dfa(d, "dfa") != DFA_OK) return 0;
  const dfa_opts o = default_opts(opts);
  const bool hd = d->k > 0 && !is_device_ptr(d->delta);
  const bool ha = !is_device_ptr(d->accept);
  if (o.algo == DFA_ALGO_MOORE) {
    BucketPlan bp{};
    const bool bucket = choose_bucket(d->n, d->k, o.flags, &bp);
    return moore_layout(d->n, d->k, hd, ha, true, bucket ? &bp : nullptr).total;
  }
  if (o.algo == DFA_ALGO_CLOSURE_MOORE) return closure_moore_layout(d->n, d->k, hd, ha).total;
  if (o.algo == DFA_ALGO_SORT) return sort_workspace_size(d, hd, ha, true);
  return naive_workspace_size(d, o);
}

int dfa_minimise(const dfa_t *d, const dfa_opts *opts, uint32_t *block_out, dfa_result *res, void *workspace,
                 size_t ws_bytes, void *stream) {
  int rc = check_dfa(d, "dfa");
  if (rc != DFA_OK) return rc;
  if (!block_out) return fail(DFA_EINVAL, "block_out is NULL");
  if (!workspace) return fail(DFA_EINVAL, "workspace is NULL");
  if (!aligned(workspace, 256)) return fail(DFA_EINVAL, "workspace must be 256-byte aligned");
  const dfa_opts o = default_opts(opts);
  if (o.algo != DFA_ALGO_MOORE && o.algo != DFA_ALGO_NAIVE && o.algo != DFA_ALGO_TRANS &&
      o.algo != DFA_ALGO_CLOSURE_MOORE && o.algo != DFA_ALGO_SORT)
    return fail(DFA_EINVAL, "unknown algo %d", o.algo);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (o.algo == DFA_ALGO_CLOSURE_MOORE) return run_closure_moore(d, o, block_out, res, workspace, ws_bytes, st);
  if (o.algo == DFA_ALGO_SORT) return run_sort_minimise(d, o, block_out, res, workspace, ws_bytes, st);
  if (o.algo != DFA_ALGO_MOORE) return run_naive_minimise(d, o, block_out, res, workspace, ws_bytes, st);

  const bool hd = d->k > 0 && !is_device_ptr(d->delta);
  const bool ha = !is_device_ptr(d->accept);
  const bool ho = !is_device_ptr(block_out);
  BucketPlan bp{};
  const bool bucket = choose_bucket(d->n, d->k, o.flags, &bp);
  const MooreLayout L = moore_layout(d->n, d->k, hd, ha, true, bucket ? &bp : nullptr);
  if (ws_bytes < L.total) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
  char *ws = static_cast<char *>(workspace);
  const uint32_t *delta = d->delta;
  const uint8_t *accept = d->accept;
  cudaError_t e;
  if (hd) {
    e = cudaMemcpyAsync(ws + L.delta, d->delta, (size_t)d->k * d->n * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy delta to device");
    delta = reinterpret_cast<const uint32_t *>(ws + L.delta);
  }
  if (ha) {
    e = cudaMemcpyAsync(ws + L.accept, d->accept, d->n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy accept to device");
    accept = reinterpret_cast<const uint8_t *>(ws + L.accept);
  }
  uint32_t *out = ho ? reinterpret_cast<uint32_t *>(ws + L.out) : block_out;
  Ctrl c{};
  if (small_fits(d->n, d->k, o)) {   // one thread block, everything in shared memory
    Ctrl *cd = reinterpret_cast<Ctrl *>(ws + L.ctrl);
    rc = enqueue_small(delta, accept, d->n, d->k, out, cd, o, st);
    if (rc != DFA_OK) return rc;
    e = cudaMemcpyAsync(&c, cd, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "single-block refinement kernel");
  } else {
    const uint32_t vec_ok = pick_vec(d->n, d->k, delta, accept, o.schedule);
    rc = run_moore(delta, accept, d->n, d->k, out, L, ws, o, st, nullptr, &c, vec_ok);
    if (rc != DFA_OK) return rc;
  }
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

}  // extern "C"
