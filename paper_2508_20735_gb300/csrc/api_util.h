// Host helpers shared by the C-ABI translation units.  Not part of the public ABI.
#pragma once
#include <cstdarg>
#include <cstddef>
#include <cstdint>

#include "../../include/dfa.h"
#include "common.cuh"
#include "internal.h"

namespace dfa {

// Byte offsets of the Moore kernel's buffers inside a caller's workspace
// (SIZE_MAX = absent).
struct MooreLayout {
  uint32_t log2S, mbits, wid, ebits;
  size_t ctrl, table, lab0, lab1, tmp, minrep, flag, partials, bm0, bm1, seen1, seen2, seen3, seen4, tmp2, rep, dups, dups2, wcnt, delta, accept, out,
      total;
  size_t warps;            // warps of the largest launch the per-warp lists (dups, dups2, wcnt) hold
  bool bucket;             // the bucketed gather runs (plan below); its buffers follow
  BucketPlan plan;
  size_t et, es, val, seg, used, phash, pq, pcnt, list;
};

// Equivalence by union: the two start states whose blocks are compared.
struct PairTrack {
  uint32_t a, b, early_exit;
};

int fail(int status, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);
bool is_device_ptr(const void *p);
uint32_t ceil_log2(uint64_t x);
dfa_opts default_opts(const dfa_opts *o);
int check_dfa(const dfa_t *d, const char *name);
bool aligned(const void *p, size_t a);
uint32_t pick_vec(uint32_t n, uint32_t k, const void *delta, const void *accept, int32_t schedule);
// bp: the bucketed gather's plan (its buffers are added), or NULL
MooreLayout moore_layout(uint64_t n, uint32_t k, bool stage_delta, bool stage_accept, bool stage_out,
                         const BucketPlan *bp = nullptr);
// Whether signature refinement of n states, k letters and these DFA_FLAG_*
// flags takes the bucketed gather on the current device, and its plan.
bool choose_bucket(uint64_t n, uint32_t k, uint32_t flags, BucketPlan *bp);
// independent_letters: the letters are the DFA's own (not closure letters, which are
// powers of the same letter), so the sparse-signature estimate may pick filter rounds
int run_moore(const uint32_t *delta_dev, const uint8_t *accept_dev, uint32_t n, uint32_t k, uint32_t *out_dev,
              const MooreLayout &L, char *ws, const dfa_opts &o, cudaStream_t st, const PairTrack *track,
              Ctrl *ctrl_host, uint32_t vec_ok, bool independent_letters = true);
// the refinement kernel's launch alone (no wait): control block at ws + L.ctrl
int enqueue_moore(const uint32_t *delta_dev, const uint8_t *accept_dev, uint32_t n, uint32_t k, uint32_t *out_dev,
                  const MooreLayout &L, char *ws, const dfa_opts &o, cudaStream_t st, const PairTrack *track,
                  uint32_t vec_ok, bool independent_letters = true);
int status_from_ctrl(const Ctrl &c);

// Signature refinement of a small DFA in one thread block (small.cu) or one
// thread-block cluster (cluster.cu): used by dfa_minimise and
// dfa_minimise_async when small_fits; results in *ctrl.
static constexpr uint32_t kSmallMaxStates = 16384;
bool small_fits(uint32_t n, uint32_t k, const dfa_opts &o);
// track (may be null): equivalence by union, the start pair whose separating
// round goes to ctrl->sep_round (~0: never apart), with early exit on request.
int enqueue_small(const uint32_t *delta, const uint8_t *accept, uint32_t n, uint32_t k, uint32_t *out, Ctrl *ctrl,
                  const dfa_opts &o, cudaStream_t st, const PairTrack *track = nullptr);
// Batches (batch.cu): a DFA refined alone by one thread block of small.cu's
// kernel; plan = log2 T | wide table << 8 | staged δ << 9 (small_block_plan:
// everything in shared memory), or log2 T | 1 << 10 (medium_block_plan: up to
// 65,536 states, labels in shared memory, the table at `table` in global
// memory, two n-word scratch arrays).
struct BatchSmallItem {
  const uint32_t *delta;   // device, k x n letter-major
  const uint8_t *accept;   // device, n
  uint32_t n, k;
  uint32_t *out;           // device, n canonical block numbers
  uint32_t *ss;            // device, the DFA's bookkeeping row
  uint32_t *table;         // medium plan: 2^log2T words of global memory
  uint32_t *scratch0, *scratch1;   // medium plan: n words each
  uint32_t plan, pad_;
};
// The medium plan of a DFA of n states whose table region has 2^log2S
// 16-byte slots (false beyond 65,536 states).
bool medium_block_plan(uint32_t n, uint32_t log2S, uint32_t *plan, size_t *smem);
// Indices, in a bookkeeping row, of the words the block writes.
struct BatchSmallWords {
  uint32_t b, changed, executed, maxed;
};
// Whether one block holds the DFA (shared memory), its plan and shared memory.
bool small_block_plan(uint32_t n, uint32_t k, uint32_t *plan, size_t *smem);
// One block per SM at most (grid), each refining the next item from *next (zeroed);
// batch_small_setup (outside any stream capture) allows the kernel its shared memory.
cudaError_t batch_small_setup();
cudaError_t enqueue_batch_small(const BatchSmallItem *items, uint32_t count, uint32_t *next, Ctrl *ctrl, size_t smem,
                                BatchSmallWords words, const dfa_opts &o, uint32_t grid, cudaStream_t st);

// The same on one thread-block cluster (cluster.cu), where the device can place
// one and the DFA fits; enqueue_small decides between the two.
bool cluster_fits(uint32_t n, uint32_t k);
int enqueue_cluster(const uint32_t *delta, const uint8_t *accept, uint32_t n, uint32_t k, uint32_t *out, Ctrl *ctrl,
                    const dfa_opts &o, cudaStream_t st, const PairTrack *track = nullptr);

// naivePR / transPR (naive.cu)
size_t naive_workspace_size(const dfa_t *d, const dfa_opts &o);
int run_closure(const uint32_t *delta_dev, uint32_t n, uint32_t k, uint32_t *dT, Ctrl *ctrl_dev, const dfa_opts &o,
                cudaStream_t st, Ctrl *ctrl_host);
int run_naive_minimise(const dfa_t *d, const dfa_opts &o, uint32_t *block_out, dfa_result *res, void *workspace,
                       size_t ws_bytes, cudaStream_t st);

// sortPR with radix-sort renumbering (sortpr.cu)
size_t sort_workspace_size(const dfa_t *d, bool stage_delta, bool stage_accept, bool stage_out);
int run_sort_minimise(const dfa_t *d, const dfa_opts &o, uint32_t *block_out, dfa_result *res, void *workspace,
                      size_t ws_bytes, cudaStream_t st);

// disjoint union helper (equiv.cu)
cudaError_t launch_offset_targets(uint32_t *delta_u, uint32_t n_u, uint32_t k, uint32_t first, uint32_t count,
                                  uint32_t offset, uint32_t *err, cudaStream_t st);

}  // namespace dfa
