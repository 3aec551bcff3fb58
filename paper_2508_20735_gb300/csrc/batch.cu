// Batched signature refinement: many independent DFAs in one persistent,
// segment-offset launch (a batching form the paper does not have; each DFA is
// refined exactly as dfa_minimise refines it alone, Section 3.3 / Algorithm 4).
//
// Layout.  All DFAs share one state space: DFA i owns states
// [state_off_i, state_off_i + n_i) of the label arrays and its own region of
// 2^ceil(log2(2 n_i)) slots of the renumbering table, so keys of different DFAs
// never meet and labels stay narrow (a DFA with 65,536 states packs 17-bit
// components).  Work is cut into tiles of at most kTile states that never
// cross a DFA boundary; warps take tiles grid-stride and skip the tiles of
// DFAs that have already converged.
//
// Rounds.  Every pass packs each active state's signature into a key of its
// own DFA's width and inserts it into its DFA's table region; a new slot counts
// one new block for that DFA.  After the pass a grid-wide bookkeeping step
// compares each active DFA's count with its previous one: equal counts mean
// the DFA has reached its fixpoint, and it drops out with its round counts.
// The launch ends when no DFA is active; then the final labels are gathered,
// numbered canonically across the batch and rebased per DFA.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "api_util.h"

namespace dfa {

static constexpr int kBatchThreads = 512;
static constexpr uint32_t kTile = 256;
static constexpr size_t kMaxGridB = 8192;

struct SegInfo {
  const uint32_t *delta;   // device
  const uint8_t *accept;   // device
  uint32_t n, k;
  uint32_t state_off;      // first state in the batch's state space
  uint32_t log2S;          // table region of 2^log2S slots
  uint64_t table_off;      // first slot of the region
  StagePlan plan1, planr;
};

struct Tile {
  uint32_t seg, start, len;   // local states [start, start+len) of DFA seg
};

// Per-DFA bookkeeping words.
enum : uint32_t { SS_ACTIVE = 0, SS_PREV, SS_CHANGED, SS_EXECUTED, SS_FINAL, SS_B, SS_SEEN, SS_MAXED, SS_WORDS };

struct BatchArgs {
  const SegInfo *segs;
  uint32_t nsegs;
  const Tile *tiles;
  uint32_t ntiles;
  uint32_t total_states;
  uint64_t total_slots;
  uint32_t *lab[2];
  uint32_t *fin;           // total_states: final labels gathered from either buffer
  uint32_t *tmp;           // total_states (multi-stage plans)
  u128 *table;
  uint32_t *minrep;        // total_slots
  uint8_t *flag;           // total_states
  uint32_t *partials;
  uint32_t *out;           // total_states
  uint32_t *cnt;           // nsegs x 3
  uint32_t *ss;            // nsegs x SS_WORDS
  uint32_t *base;          // nsegs
  Ctrl *ctrl;
  uint32_t ebits, max_stages, max_rounds;
  uint32_t stop_discrete;  // 1: a DFA whose round leaves n blocks stops (no confirming round)
  uint32_t vec;            // states per lane within a tile pass: 1 or 2
  unsigned long long timeout_ns, barrier_ns;
};

template <int VEC, bool ROUND1>
__device__ __forceinline__ void batch_tile(const BatchArgs &A, const SegInfo &S, const Tile &T, uint32_t stage,
                                          bool last, uint32_t epoch, const uint32_t *__restrict__ src,
                                          uint32_t *__restrict__ dst, CtaCache *cache, uint32_t r) {
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
  const unsigned long long etag = (unsigned long long)epoch << (64 - A.ebits);
  const unsigned long long keep = policy_evict_last();
  const uint32_t *lsrc = src + S.state_off;   // this DFA's labels (global slot numbers)
  u128 *table = A.table + S.table_off;
  uint32_t seen = 0, created_total = 0;
  for (uint32_t base = 0; base < T.len; base += 32u * VEC) {
    u128 key[VEC];
    bool valid = false;
    uint32_t qs[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const uint32_t off = base + lane * VEC + v;
      qs[v] = T.start + (off < T.len ? off : 0u);
      key[v] = u128{0ull, 0ull};
    }
    valid = base + lane * VEC < T.len;
    bool vv[VEC];
#pragma unroll
    for (int v = 0; v < VEC; ++v) vv[v] = base + lane * VEC + v < T.len;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      const uint32_t q = qs[v];
      uint32_t shift = 0;
      if (has_prev) {
        put_bits(key[v], A.tmp[S.state_off + q], 0);
        shift = P.carry;
      }
      uint32_t j = cbeg;
      if (j == 0) {
        uint32_t c;
        if (ROUND1) {
          c = S.accept[q] != 0;
          if (vv[v]) seen |= c ? 1u : 2u;
        } else {
          c = lsrc[q] - (uint32_t)S.table_off;
        }
        put_bits(key[v], c, shift);
        shift += bits;
        j = 1;
      }
      for (; j < cend; ++j) {
        uint32_t d = S.delta[(size_t)(j - 1) * n + q];
        if (ROUND1 && d >= n) {
          if (vv[v]) atomicOr(&A.ctrl->err, ERR_BAD_DELTA);
          d = 0;
        }
        const uint32_t c = ROUND1 ? (uint32_t)(S.accept[d] != 0) : ld_u32_hint(lsrc + d, keep) - (uint32_t)S.table_off;
        put_bits(key[v], c, shift);
        shift += bits;
      }
      key[v].hi |= etag;
    }
    // Lanes whose states lie past the tile end insert nothing (their keys are
    // duplicates of the tile's first state).
    uint32_t lab[VEC];
    uint32_t created = 0;
    if constexpr (VEC == 1) {
      warp_insert<1>(table, S.log2S, key, valid, A.ebits, epoch, lab, created, &A.ctrl->err, cache, T.seg);
    } else {
      // second state of a pair may lie past the end: give it the first state's key
      if (!vv[1]) key[1] = key[0];
      warp_insert<VEC>(table, S.log2S, key, valid, A.ebits, epoch, lab, created, &A.ctrl->err, cache, T.seg);
    }
    if (last) created_total += created;
#pragma unroll
    for (int v = 0; v < VEC; ++v) {
      if (!vv[v]) continue;
      const uint32_t gq = S.state_off + qs[v];
      if (last) dst[gq] = (uint32_t)S.table_off + lab[v];
      else A.tmp[gq] = lab[v];
    }
  }
  // one atomic per warp and tile: every lane of the warp works on this DFA
  const uint32_t wsum = __reduce_add_sync(0xFFFFFFFFu, created_total);
  if (lane == 0 && wsum) atomicAdd(&A.cnt[T.seg * 3 + r % 3], wsum);
  if (ROUND1) {
    const uint32_t wseen = __reduce_or_sync(0xFFFFFFFFu, seen);
    if (lane == 0 && wseen) atomicOr(&A.ss[T.seg * SS_WORDS + SS_SEEN], wseen);
  }
}

template <int VEC>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(BatchArgs A) {
  __shared__ uint32_t s_red[kBatchThreads / 32];
  __shared__ CtaCache cache;
  Ctrl *C = A.ctrl;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  const uint32_t gwarp = tid >> 5, nwarps = stride >> 5;
  if (leader) {
    const unsigned long long t = gtimer();
    C->t_start = t;
    C->deadline = t + A.timeout_ns;
  }
  const uint32_t emax = A.ebits >= 32 ? 0xFFFFFFFFu : ((1u << A.ebits) - 1u);
  // clear tables; every DFA starts active
  for (uint64_t i = tid; i < A.total_slots; i += stride) reinterpret_cast<uint4 *>(A.table)[i] = make_uint4(0, 0, 0, 0);
  for (uint32_t i = tid; i < A.nsegs; i += stride) {
    A.ss[i * SS_WORDS + SS_ACTIVE] = 1u;
    A.ss[i * SS_WORDS + SS_FINAL] = 1u;
  }
  bool ok = grid_sync(C, A.barrier_ns);
  uint32_t epoch = 0, r;
  for (r = 1; ok; ++r) {
    const bool round1 = r == 1;
    const uint32_t *src = A.lab[(r - 1) & 1];
    uint32_t *dst = A.lab[r & 1];
    for (uint32_t s = 0; ok && s < A.max_stages; ++s) {
      if (epoch == emax) {
        for (uint64_t i = tid; i < A.total_slots; i += stride)
          reinterpret_cast<uint4 *>(A.table)[i] = make_uint4(0, 0, 0, 0);
        ok = grid_sync(C, A.barrier_ns);
        epoch = 0;
        if (!ok) break;
      }
      ++epoch;
      cta_cache_clear(&cache);
      for (uint32_t t = gwarp; t < A.ntiles; t += nwarps) {
        const Tile T = A.tiles[t];
        if (!ld_relaxed(&A.ss[T.seg * SS_WORDS + SS_ACTIVE])) continue;
        const SegInfo &S = A.segs[T.seg];
        const StagePlan &P = round1 ? S.plan1 : S.planr;
        if (s >= P.stages) continue;
        const bool last = s + 1 == P.stages;
        if (round1) batch_tile<VEC, true>(A, S, T, s, last, epoch, src, dst, &cache, r);
        else batch_tile<VEC, false>(A, S, T, s, last, epoch, src, dst, &cache, r);
      }
      ok = grid_sync(C, A.barrier_ns);
    }
    if (!ok) break;
    // bookkeeping: one thread per DFA
    uint32_t still = 0;
    for (uint32_t i = tid; i < A.nsegs; i += stride) {
      uint32_t *w = A.ss + i * SS_WORDS;
      A.cnt[i * 3 + (r + 2) % 3] = 0u;
      if (!w[SS_ACTIVE]) continue;
      const uint32_t B = A.cnt[i * 3 + r % 3];
      const uint32_t prev = round1 ? __popc(w[SS_SEEN]) : w[SS_PREV];
      w[SS_EXECUTED] = r;
      w[SS_FINAL] = r & 1;
      w[SS_B] = B;
      if (B == prev) {
        w[SS_ACTIVE] = 0u;               // fixpoint (Algorithm 4's until-test)
      } else {
        w[SS_CHANGED] += 1;
        w[SS_PREV] = B;
        if (A.stop_discrete && B == A.segs[i].n) {
          w[SS_ACTIVE] = 0u;             // n singleton blocks cannot split any further
        } else if (A.max_rounds != 0u && r >= A.max_rounds) {
          w[SS_ACTIVE] = 0u;
          w[SS_MAXED] = 1u;
        } else {
          ++still;
        }
      }
    }
    const uint32_t bs = block_sum(still, s_red);
    if (threadIdx.x == 0 && bs) atomicAdd(&C->cnt[r % 3], bs);
    ok = grid_sync(C, A.barrier_ns);
    if (!ok) break;
    const uint32_t active = ld_relaxed(&C->cnt[r % 3]);
    if (leader) C->cnt[(r + 2) % 3] = 0u;
    if (active == 0u) break;
  }
  if (ok) {
    // final labels of every DFA into one buffer
    for (uint32_t t = gwarp; t < A.ntiles; t += nwarps) {
      const Tile T = A.tiles[t];
      const SegInfo &S = A.segs[T.seg];
      const uint32_t *srcf = A.lab[A.ss[T.seg * SS_WORDS + SS_FINAL]];
      for (uint32_t i = threadIdx.x & 31u; i < T.len; i += 32) {
        const uint32_t gq = S.state_off + T.start + i;
        A.fin[gq] = srcf[gq];
      }
    }
    ok = grid_sync(C, A.barrier_ns);
  }
  if (ok) {
    ok = canonicalise(CanonArgs{A.total_states, A.fin, (size_t)A.total_slots, A.minrep, A.flag, A.partials, A.out,
                                C, A.barrier_ns, 0u},
                      0xFFFFFFFFu, s_red);
  }
  if (ok) ok = grid_sync(C, A.barrier_ns);
  if (ok) {
    // blocks of earlier DFAs precede DFA i's: its first state's number is its offset
    for (uint32_t i = tid; i < A.nsegs; i += stride) A.base[i] = A.out[A.segs[i].state_off];
    ok = grid_sync(C, A.barrier_ns);
  }
  if (ok) {
    for (uint32_t t = gwarp; t < A.ntiles; t += nwarps) {
      const Tile T = A.tiles[t];
      const uint32_t off = A.segs[T.seg].state_off + T.start, b = A.base[T.seg];
      for (uint32_t i = threadIdx.x & 31u; i < T.len; i += 32) A.out[off + i] -= b;
    }
  }
  if (leader) {
    C->rounds_executed = r;
    C->t_end = gtimer();
  }
}

// ------------------------------------------------------------------ host side

struct BatchLayout {
  size_t ctrl, segs, tiles, lab0, lab1, fin, tmp, table, minrep, flag, partials, out, cnt, ss, base, stage, total;
  uint64_t total_states, total_slots;
  uint32_t ntiles, max_stages, ebits;
  size_t stage_bytes;
};

static BatchLayout batch_layout(const dfa_t *dfas, uint32_t count, std::vector<SegInfo> *segs_out,
                                std::vector<Tile> *tiles_out, std::vector<size_t> *stage_off) {
  BatchLayout L{};
  uint64_t st = 0, sl = 0;
  uint32_t ntiles = 0, max_stages = 1, ebits = 32;
  size_t stage_bytes = 0;
  bool multi = false;
  for (uint32_t i = 0; i < count; ++i) {
    const dfa_t &d = dfas[i];
    SegInfo s{};
    s.n = d.n;
    s.k = d.k;
    s.state_off = (uint32_t)st;
    s.log2S = ceil_log2((uint64_t)d.n * 2 < 64 ? 64 : (uint64_t)d.n * 2);
    s.table_off = sl;
    s.plan1 = make_plan(d.k, 1, s.log2S);
    s.planr = make_plan(d.k, s.log2S, s.log2S);
    max_stages = std::max({max_stages, s.plan1.stages, s.planr.stages});
    ebits = std::min({ebits, s.plan1.ebits, s.planr.ebits});
    multi |= s.plan1.stages > 1 || s.planr.stages > 1;
    const uint32_t tiles_i = (d.n + kTile - 1) / kTile;
    if (tiles_out)
      for (uint32_t t = 0; t < tiles_i; ++t)
        tiles_out->push_back(Tile{i, t * kTile, std::min(kTile, d.n - t * kTile)});
    ntiles += tiles_i;
    // host-resident arrays are staged into the workspace
    const bool hd = d.k > 0 && !is_device_ptr(d.delta), ha = !is_device_ptr(d.accept);
    if (stage_off) {
      stage_off->push_back(hd ? stage_bytes : SIZE_MAX);
    }
    if (hd) stage_bytes += ((size_t)d.k * d.n * 4 + 255) / 256 * 256;
    if (stage_off) stage_off->push_back(ha ? stage_bytes : SIZE_MAX);
    if (ha) stage_bytes += ((size_t)d.n + 255) / 256 * 256;
    st += d.n;
    sl += (uint64_t)1 << s.log2S;
    if (segs_out) segs_out->push_back(s);
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  L.total_states = st;
  L.total_slots = sl;
  L.ntiles = ntiles;
  L.max_stages = max_stages;
  L.ebits = ebits;
  L.ctrl = take(sizeof(Ctrl));
  L.segs = take(sizeof(SegInfo) * count);
  L.tiles = take(sizeof(Tile) * ntiles);
  L.lab0 = take(st * 4);
  L.lab1 = take(st * 4);
  L.fin = take(st * 4);
  L.tmp = multi ? take(st * 4) : SIZE_MAX;
  L.table = take(sl * 16);
  L.minrep = take(sl * 4);
  L.flag = take(st);
  L.partials = take(kMaxGridB * 4);
  L.out = take(st * 4);
  L.cnt = take((size_t)count * 3 * 4);
  L.ss = take((size_t)count * SS_WORDS * 4);
  L.base = take((size_t)count * 4);
  L.stage_bytes = stage_bytes;
  L.stage = take(stage_bytes);
  L.total = off;
  return L;
}

static const void *batch_kernel_for(uint32_t vec) {
  return vec == 2 ? (const void *)batch_kernel<2> : (const void *)batch_kernel<1>;
}

// Launches the batch kernel as a CUDA graph: the control-block reset and the
// cooperative launch are captured on a library-owned stream (capture is not
// allowed on the legacy default stream) and the graph runs on `st`.
static cudaError_t launch_batch_graph(const BatchArgs &a, int grid, cudaStream_t st) {
  static thread_local cudaStream_t cap = nullptr;
  cudaError_t e;
  if (!cap && (e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  BatchArgs copy = a;
  void *params[] = {&copy};
  cudaError_t le = cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl), cap);
  if (le == cudaSuccess)
    le = cudaLaunchCooperativeKernel(batch_kernel_for(a.vec), dim3(grid), dim3(kBatchThreads), params, 0, cap);
  e = cudaStreamEndCapture(cap, &graph);
  if (le != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return le;
  }
  if (e != cudaSuccess) return e;
  e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
  if (exec) cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  return e;
}

// ------------------------------------------------------------------ autotuner
// Schedules: 0 = one state per lane, 1 = two states per lane.  With
// opts.schedule = -1 the first call for a (batch size bucket, letter bucket,
// GPU) key times both on the batch itself and remembers the faster, in memory
// and in a JSON file ($DFA_AUTOTUNE_CACHE, default ~/.cache/dfa_gb300_autotune.json).
static std::mutex g_tune_mu;
static std::map<std::string, int> g_tune;
static bool g_tune_loaded = false;

static std::string tune_path() {
  const char *p = getenv("DFA_AUTOTUNE_CACHE");
  if (p && *p) return p;
  const char *h = getenv("HOME");
  return std::string(h ? h : "/tmp") + "/.cache/dfa_gb300_autotune.json";
}

static void tune_load() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  FILE *f = fopen(tune_path().c_str(), "r");
  if (!f) return;
  char key[256];
  int val;
  // format: {"key": value, ...} one entry per line
  char line[512];
  while (fgets(line, sizeof line, f)) {
    if (sscanf(line, " \"%255[^\"]\" : %d", key, &val) == 2) g_tune[key] = val;
  }
  fclose(f);
}

static void tune_save() {
  const std::string p = tune_path();
  const size_t slash = p.rfind('/');
  if (slash != std::string::npos) mkdir(p.substr(0, slash).c_str(), 0755);   // best effort
  FILE *f = fopen(p.c_str(), "w");
  if (!f) return;
  fprintf(f, "{\n");
  size_t i = 0;
  for (auto &kv : g_tune) fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++i < g_tune.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
}

static std::string tune_key(uint64_t states, uint32_t count, uint32_t kmax) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev);
  char buf[256];
  snprintf(buf, sizeof buf, "batch|%s|states2^%u|dfas2^%u|kmax%u", prop.name, ceil_log2(states + 1),
           ceil_log2((uint64_t)count + 1), kmax);
  return buf;
}

}  // namespace dfa

using namespace dfa;

extern "C" {

size_t dfa_batch_workspace_size(const dfa_t *dfas, uint32_t count, const dfa_opts *opts) {
  (void)opts;
  if (!dfas || count == 0) return 0;
  uint64_t total = 0;
  for (uint32_t i = 0; i < count; ++i) {
    if (check_dfa(&dfas[i], "dfas[i]") != DFA_OK) return 0;
    total += dfas[i].n;
  }
  if (total > DFA_MAX_STATES) return 0;
  const BatchLayout L = batch_layout(dfas, count, nullptr, nullptr, nullptr);
  if (L.total_slots > 0xFFFFFFFFull) return 0;
  return L.total;
}

static int run_batch(const dfa_t *dfas, uint32_t count, const dfa_opts &o, uint32_t *block_out, dfa_result *res,
                     char *ws, size_t ws_bytes, cudaStream_t st, uint32_t vec, uint64_t *device_ns) {
  std::vector<SegInfo> segs;
  std::vector<Tile> tiles;
  std::vector<size_t> stage_off;
  const BatchLayout L = batch_layout(dfas, count, &segs, &tiles, &stage_off);
  if (L.total_slots > 0xFFFFFFFFull) return fail(DFA_EINVAL, "batch too large for 32-bit labels");
  if (ws_bytes < L.total) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
  cudaError_t e;
  for (uint32_t i = 0; i < count; ++i) {
    const dfa_t &d = dfas[i];
    segs[i].delta = d.delta;
    segs[i].accept = d.accept;
    if (stage_off[2 * i] != SIZE_MAX) {
      char *p = ws + L.stage + stage_off[2 * i];
      e = cudaMemcpyAsync(p, d.delta, (size_t)d.k * d.n * 4, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "copy delta to device");
      segs[i].delta = reinterpret_cast<const uint32_t *>(p);
    }
    if (stage_off[2 * i + 1] != SIZE_MAX) {
      char *p = ws + L.stage + stage_off[2 * i + 1];
      e = cudaMemcpyAsync(p, d.accept, d.n, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "copy accept to device");
      segs[i].accept = reinterpret_cast<const uint8_t *>(p);
    }
  }
  e = cudaMemcpyAsync(ws + L.segs, segs.data(), sizeof(SegInfo) * count, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy segment table");
  e = cudaMemcpyAsync(ws + L.tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy tile table");
  e = cudaMemsetAsync(ws + L.cnt, 0, (size_t)count * 3 * 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.ss, 0, (size_t)count * SS_WORDS * 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "clear batch bookkeeping");
  const bool ho = !is_device_ptr(block_out);
  BatchArgs a{};
  a.segs = reinterpret_cast<const SegInfo *>(ws + L.segs);
  a.nsegs = count;
  a.tiles = reinterpret_cast<const Tile *>(ws + L.tiles);
  a.ntiles = L.ntiles;
  a.total_states = (uint32_t)L.total_states;
  a.total_slots = L.total_slots;
  a.lab[0] = reinterpret_cast<uint32_t *>(ws + L.lab0);
  a.lab[1] = reinterpret_cast<uint32_t *>(ws + L.lab1);
  a.fin = reinterpret_cast<uint32_t *>(ws + L.fin);
  a.tmp = L.tmp == SIZE_MAX ? nullptr : reinterpret_cast<uint32_t *>(ws + L.tmp);
  a.table = reinterpret_cast<u128 *>(ws + L.table);
  a.minrep = reinterpret_cast<uint32_t *>(ws + L.minrep);
  a.flag = reinterpret_cast<uint8_t *>(ws + L.flag);
  a.partials = reinterpret_cast<uint32_t *>(ws + L.partials);
  a.out = ho ? reinterpret_cast<uint32_t *>(ws + L.out) : block_out;
  a.cnt = reinterpret_cast<uint32_t *>(ws + L.cnt);
  a.ss = reinterpret_cast<uint32_t *>(ws + L.ss);
  a.base = reinterpret_cast<uint32_t *>(ws + L.base);
  a.ctrl = reinterpret_cast<Ctrl *>(ws + L.ctrl);
  a.ebits = L.ebits;
  a.max_stages = L.max_stages;
  a.max_rounds = o.max_rounds;
  a.stop_discrete = (o.flags & DFA_FLAG_STOP_DISCRETE) ? 1u : 0u;
  a.vec = vec;
  a.timeout_ns = o.timeout_ns;
  a.barrier_ns = o.timeout_ns < 5000000000ull ? o.timeout_ns : 5000000000ull;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(e, "device attribute");
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel_for(vec), kBatchThreads, 0)) !=
      cudaSuccess)
    return cuda_fail(e, "occupancy");
  const int grid = sms * (per_sm < 1 ? 1 : per_sm);
  if ((size_t)grid > kMaxGridB) return fail(DFA_ECUDA, "grid too large");
  e = launch_batch_graph(a, grid, st);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch of the batch kernel");
  Ctrl c{};
  std::vector<uint32_t> ss((size_t)count * SS_WORDS);
  e = cudaMemcpyAsync(&c, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ss.data(), a.ss, ss.size() * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "batch kernel");
  const int status = status_from_ctrl(c);
  if (device_ns) *device_ns = c.t_end - c.t_start;
  if (status != DFA_OK) return status;
  int overall = DFA_OK;
  for (uint32_t i = 0; i < count; ++i) {
    const uint32_t *w = ss.data() + (size_t)i * SS_WORDS;
    if (res) {
      res[i].num_blocks = w[SS_B];
      res[i].rounds_changed = w[SS_CHANGED];
      res[i].rounds_executed = w[SS_EXECUTED];
      res[i].status = w[SS_MAXED] ? DFA_EMAXROUNDS : DFA_OK;
      res[i].device_ns = c.t_end - c.t_start;
    }
    if (w[SS_MAXED]) overall = DFA_EMAXROUNDS;
  }
  if (ho) {
    e = cudaMemcpyAsync(block_out, a.out, L.total_states * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "copy blocks to host");
  }
  if (overall != DFA_OK) fail(overall, "max_rounds reached before the fixpoint for some DFA");
  return overall;
}

int dfa_minimise_batch(const dfa_t *dfas, uint32_t count, const dfa_opts *opts, uint32_t *block_out,
                       dfa_result *res, void *workspace, size_t ws_bytes, void *stream) {
  if (!dfas || count == 0) return fail(DFA_EINVAL, "empty batch");
  uint64_t total = 0;
  uint32_t kmax = 0;
  for (uint32_t i = 0; i < count; ++i) {
    const int rc = check_dfa(&dfas[i], "dfas[i]");
    if (rc != DFA_OK) return fail(rc, "dfa %u: %s", i, dfa_last_error());
    total += dfas[i].n;
    kmax = std::max(kmax, dfas[i].k);
  }
  if (total > DFA_MAX_STATES) return fail(DFA_EINVAL, "batch of %llu states exceeds %u", (unsigned long long)total,
                                          DFA_MAX_STATES);
  if (!block_out) return fail(DFA_EINVAL, "block_out is NULL");
  if (!workspace || !aligned(workspace, 256)) return fail(DFA_EINVAL, "workspace NULL or not 256-byte aligned");
  const dfa_opts o = default_opts(opts);
  if (o.algo != DFA_ALGO_MOORE) return fail(DFA_EINVAL, "batches use signature refinement (algo 0)");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (o.schedule == 0 || o.schedule == 1)
    return run_batch(dfas, count, o, block_out, res, static_cast<char *>(workspace), ws_bytes, st,
                     o.schedule == 1 ? 2u : 1u, nullptr);
  // autotune
  const std::string key = tune_key(total, count, kmax);
  int choice = -1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) choice = it->second;
  }
  if (choice != 0 && choice != 1) {
    uint64_t best = ~0ull;
    for (int s = 0; s < 2; ++s) {
      uint64_t ns = 0;
      const int rc = run_batch(dfas, count, o, block_out, res, static_cast<char *>(workspace), ws_bytes, st,
                               s == 1 ? 2u : 1u, &ns);
      if (rc != DFA_OK && rc != DFA_EMAXROUNDS) return rc;
      if (ns < best) {
        best = ns;
        choice = s;
      }
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = choice;
    tune_save();
  }
  return run_batch(dfas, count, o, block_out, res, static_cast<char *>(workspace), ws_bytes, st,
                   choice == 1 ? 2u : 1u, nullptr);
}

}  // extern "C"
