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

struct ServeSeg {
  const uint32_t *delta;
  const uint8_t *accept;
  uint32_t n, k;
  uint32_t *lab[2];
  uint32_t *tmp;
  u128 *table;
  uint32_t log2S;
  uint32_t ebits;
  StagePlan plan1, planr;
  uint32_t round;      // round this step executes (1-based)
  uint32_t epoch0;     // epoch of stage 0 of this round
  uint32_t track, sa, sb;
};

struct ServeOut {
  uint32_t count, seen, sep, pad;
};

struct ServeTile {
  uint32_t seg, start, len;
};

struct StepArgs {
  const ServeSeg *segs;
  uint32_t nsegs;
  const ServeTile *tiles;
  uint32_t ntiles;
  ServeOut *outs;
  uint32_t max_stages;
  Ctrl *ctrl;
  unsigned long long barrier_ns;
};

template <bool ROUND1>
__device__ __forceinline__ void serve_tile(const StepArgs &A, const ServeSeg &S, const ServeTile &T, uint32_t stage,
                                          bool last, CtaCache *cache) {
  const StagePlan &P = ROUND1 ? S.plan1 : S.planr;
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

// One refinement round for every admitted request.
__global__ void __launch_bounds__(kServeThreads) serve_step_kernel(StepArgs A) {
  __shared__ CtaCache cache;
  Ctrl *C = A.ctrl;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const uint32_t gwarp = tid >> 5, nwarps = stride >> 5;
  if (tid == 0) C->deadline = gtimer() + A.barrier_ns;
  for (uint32_t s = 0; s < A.max_stages; ++s) {
    cta_cache_clear(&cache);
    for (uint32_t t = gwarp; t < A.ntiles; t += nwarps) {
      const ServeTile T = A.tiles[t];
      const ServeSeg &S = A.segs[T.seg];
      const bool round1 = S.round == 1;
      const StagePlan &P = round1 ? S.plan1 : S.planr;
      if (s >= P.stages) continue;
      const bool last = s + 1 == P.stages;
      if (round1) serve_tile<true>(A, S, T, s, last, &cache);
      else serve_tile<false>(A, S, T, s, last, &cache);
    }
    if (!grid_sync(C, A.barrier_ns)) return;
  }
  for (uint32_t i = tid; i < A.nsegs; i += stride) {
    const ServeSeg &S = A.segs[i];
    if (S.track) {
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
  size_t o_delta = 0, o_acc = 0, o_lab0 = 0, o_lab1 = 0, o_tmp = SIZE_MAX, o_table = 0, o_minrep = 0, o_flag = 0,
         o_out = 0, o_err = 0;
  uint32_t log2S = 0, ebits = 32;
  StagePlan p1{}, pr{};
  // progress
  uint32_t round = 0, changed = 0, prevB = 0, epoch = 0, lastB = 0, sep_round = 0xFFFFFFFFu;
  bool finished = false, converged = false;
  int status = DFA_OK;
  std::vector<ServeTile> tiles;
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
  r.p1 = make_plan(r.k, 1, r.log2S);
  r.pr = make_plan(r.k, r.log2S, r.log2S);
  r.ebits = std::min(r.p1.ebits, r.pr.ebits);
  r.o_err = take(4);
  r.o_delta = take((size_t)r.k * n * 4);
  r.o_acc = take(n);
  r.o_lab0 = take(n * 4);
  r.o_lab1 = take(n * 4);
  r.o_tmp = (r.p1.stages > 1 || r.pr.stages > 1) ? take(n * 4) : SIZE_MAX;
  r.o_table = take(((size_t)1 << r.log2S) * 16);
  r.o_minrep = take(((size_t)1 << r.log2S) * 4);
  r.o_flag = take(n);
  r.o_out = take(n * 4);
  return off;
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
  // device scratch for steps and canonical numbering (allocated once)
  char *scratch = nullptr;
  size_t scratch_bytes = 0;
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
};

namespace dfa {

static constexpr uint32_t kServeMaxSlots = 4096;

// scratch: Ctrl (256) | partials (kServeMaxGrid*4) | outs (max_slots*16) | segs | tiles staging
static size_t serve_scratch_size(uint32_t max_slots, size_t max_tiles) {
  return 256 + kServeMaxGrid * 4 + (size_t)max_slots * sizeof(ServeOut) + (size_t)max_slots * sizeof(ServeSeg) +
         max_tiles * sizeof(ServeTile) + 4096;
}

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
  if (e == cudaSuccess && r.k > 0)
    e = cudaMemcpy2DAsync(b + r.o_delta, (size_t)n * 4, r.dA.data(), (size_t)r.nA * 4, (size_t)r.nA * 4, r.k,
                          cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && r.k > 0 && r.nB > 0)
    e = cudaMemcpy2DAsync(b + r.o_delta + (size_t)r.nA * 4, (size_t)n * 4, r.dB.data(), (size_t)r.nB * 4,
                          (size_t)r.nB * 4, r.k, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + r.o_acc, r.aA.data(), r.nA, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && r.nB > 0) e = cudaMemcpyAsync(b + r.o_acc + r.nA, r.aB.data(), r.nB, cudaMemcpyHostToDevice, st);
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
  e = cudaMemsetAsync(b + r.o_table, 0, ((size_t)1 << r.log2S) * 16, st);
  if (e != cudaSuccess) return e;
  r.tiles.clear();
  for (uint32_t t = 0; t * kServeTile < n; ++t) r.tiles.push_back(ServeTile{0, t * kServeTile, std::min(kServeTile, n - t * kServeTile)});
  r.round = 0;
  r.epoch = 0;
  return cudaGetLastError();
}

static void worker_main(dfa_server *s) {
  cudaSetDevice(s->device);
  char *sc = s->scratch;
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(sc);
  uint32_t *partials = reinterpret_cast<uint32_t *>(sc + 256);
  ServeOut *outs = reinterpret_cast<ServeOut *>(sc + 256 + kServeMaxGrid * 4);
  ServeSeg *segs_d = reinterpret_cast<ServeSeg *>(reinterpret_cast<char *>(outs) + (size_t)s->max_slots * sizeof(ServeOut));
  ServeTile *tiles_d = reinterpret_cast<ServeTile *>(reinterpret_cast<char *>(segs_d) + (size_t)s->max_slots * sizeof(ServeSeg));
  const size_t max_tiles = (s->scratch_bytes - (reinterpret_cast<char *>(tiles_d) - sc)) / sizeof(ServeTile);
  std::vector<ServeSeg> segs_h;
  std::vector<ServeTile> tiles_h;
  std::vector<ServeOut> outs_h;
  while (true) {
    std::vector<std::shared_ptr<Req>> admitted;
    {
      std::unique_lock<std::mutex> lock(s->mu);
      if (s->active.empty())
        s->cv_work.wait_for(lock, std::chrono::milliseconds(50), [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) break;
      // admission in arrival order while a slot and arena space are free
      size_t tiles_now = 0;
      for (auto &r : s->active) tiles_now += r->tiles.size();
      while (!s->queue.empty() && s->active.size() < s->max_slots) {
        auto r = s->queue.front();
        const size_t want_tiles = (r->n + kServeTile - 1) / kServeTile;
        if (tiles_now + want_tiles > max_tiles) break;
        size_t off;
        if (!s->arena->alloc(r->bytes, &off)) break;
        r->off = off;
        s->queue.pop_front();
        s->active.push_back(r);
        admitted.push_back(r);
        tiles_now += want_tiles;
      }
    }
    for (auto &r : admitted) {
      const cudaError_t e = place_req(s, *r);
      if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lock(s->mu);
        s->worker_error = cudaGetErrorString(e);
        finish_req(s, r, DFA_ECUDA);
      }
    }
    if (!admitted.empty()) {
      // requests whose targets were out of range finish with DFA_EINVAL
      std::vector<uint32_t> errs(admitted.size());
      for (size_t i = 0; i < admitted.size(); ++i)
        cudaMemcpyAsync(&errs[i], s->arena_base + admitted[i]->off + admitted[i]->o_err, 4, cudaMemcpyDeviceToHost,
                        s->stream);
      cudaStreamSynchronize(s->stream);
      std::lock_guard<std::mutex> lock(s->mu);
      for (size_t i = 0; i < admitted.size(); ++i)
        if (errs[i] && !admitted[i]->finished) finish_req(s, admitted[i], DFA_EINVAL);
    }
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
    segs_h.clear();
    tiles_h.clear();
    uint32_t max_stages = 1;
    for (uint32_t i = 0; i < act.size(); ++i) {
      Req &r = *act[i];
      r.round += 1;
      const StagePlan &P = r.round == 1 ? r.p1 : r.pr;
      const uint32_t emax = r.ebits >= 32 ? 0xFFFFFFFFu : ((1u << r.ebits) - 1u);
      if ((uint64_t)r.epoch + P.stages > emax) {   // epochs would wrap: clear this request's table
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
      g.tmp = r.o_tmp == SIZE_MAX ? nullptr : reinterpret_cast<uint32_t *>(b + r.o_tmp);
      g.table = reinterpret_cast<u128 *>(b + r.o_table);
      g.log2S = r.log2S;
      g.ebits = r.ebits;
      g.plan1 = r.p1;
      g.planr = r.pr;
      g.round = r.round;
      g.epoch0 = r.epoch + 1;
      g.track = r.kind == DFA_REQ_EQUIVALENT;
      g.sa = r.sA;
      g.sb = r.nA + r.sB;
      r.epoch += P.stages;
      max_stages = std::max(max_stages, P.stages);
      segs_h.push_back(g);
      for (ServeTile t : r.tiles) {
        t.seg = i;
        tiles_h.push_back(t);
      }
    }
    cudaMemcpyAsync(segs_d, segs_h.data(), segs_h.size() * sizeof(ServeSeg), cudaMemcpyHostToDevice, s->stream);
    cudaMemcpyAsync(tiles_d, tiles_h.data(), tiles_h.size() * sizeof(ServeTile), cudaMemcpyHostToDevice, s->stream);
    cudaMemsetAsync(outs, 0, act.size() * sizeof(ServeOut), s->stream);
    cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s->stream);
    StepArgs a{};
    a.segs = segs_d;
    a.nsegs = (uint32_t)act.size();
    a.tiles = tiles_d;
    a.ntiles = (uint32_t)tiles_h.size();
    a.outs = outs;
    a.max_stages = max_stages;
    a.ctrl = ctrl;
    a.barrier_ns = 5000000000ull;
    void *params[] = {&a};
    cudaError_t e = cudaLaunchCooperativeKernel((const void *)serve_step_kernel, dim3(s->grid_step),
                                                dim3(kServeThreads), params, 0, s->stream);
    outs_h.resize(act.size());
    Ctrl ch{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(outs_h.data(), outs, act.size() * sizeof(ServeOut), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ch, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
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
      const uint32_t prev = r.round == 1 ? (uint32_t)__builtin_popcount(o.seen) : r.prevB;
      const uint32_t B = o.count;
      r.lastB = B;
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
      if (r.kind == DFA_REQ_MINIMISE) {
        char *b = s->arena_base + r.off;
        CanonArgs ca{r.n, reinterpret_cast<uint32_t *>(b + (r.round & 1 ? r.o_lab1 : r.o_lab0)),
                     (size_t)1 << r.log2S, reinterpret_cast<uint32_t *>(b + r.o_minrep),
                     reinterpret_cast<uint8_t *>(b + r.o_flag), partials, reinterpret_cast<uint32_t *>(b + r.o_out),
                     ctrl, 5000000000ull, 0u};
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

static int copy_dfa_in(const dfa_t *d, std::vector<uint32_t> &delta, std::vector<uint8_t> &acc) {
  delta.resize((size_t)d->k * d->n);
  acc.resize(d->n);
  if (d->k > 0) {
    const cudaError_t e = cudaMemcpy(delta.data(), d->delta, delta.size() * 4, cudaMemcpyDefault);
    if (e != cudaSuccess) return cuda_fail(e, "copy request delta");
  }
  const cudaError_t e = cudaMemcpy(acc.data(), d->accept, d->n, cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(e, "copy request accept");
  return DFA_OK;
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
  s->scratch_bytes = serve_scratch_size(max_slots, max_tiles);
  e = cudaMalloc(&s->arena_base, hbm_budget_bytes);
  if (e != cudaSuccess) return fail(DFA_ENOMEM, "cannot allocate the %zu-byte arena: %s", hbm_budget_bytes,
                                    cudaGetErrorString(e));
  e = cudaMalloc(&s->scratch, s->scratch_bytes);
  if (e != cudaSuccess) {
    cudaFree(s->arena_base);
    return fail(DFA_ENOMEM, "cannot allocate serving scratch: %s", cudaGetErrorString(e));
  }
  s->arena = std::make_unique<Arena>(hbm_budget_bytes);
  e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
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
  rc = copy_dfa_in(a, r->dA, r->aA);
  if (rc != DFA_OK) return rc;
  if (kind == DFA_REQ_EQUIVALENT) {
    rc = copy_dfa_in(b, r->dB, r->aB);
    if (rc != DFA_OK) return rc;
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
    // round 0 of an equivalence request: the empty word already separates start
    // states of different acceptance; with early exit no round is needed
    const bool sep0 = kind == DFA_REQ_EQUIVALENT && ((r->aA[r->sA] != 0) != (r->aB[r->sB] != 0));
    if (sep0) r->sep_round = 0;
    if (sep0 && (r->o.flags & DFA_FLAG_EARLY_EXIT)) {
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
  if (s->arena_base) cudaFree(s->arena_base);
  if (s->scratch) cudaFree(s->scratch);
  delete s;
  return DFA_OK;
}

}  // extern "C"
