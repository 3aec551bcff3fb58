// Internal interface between the C-ABI layer (api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace dfa {

struct Ctrl;
struct u128;

// Stage plan for packing a signature of (k+1) components of `bits` bits each
// into 128-bit keys: stage 0 takes components [0, first); every later stage
// takes the previous stage's label (a table slot, `carry` bits) plus `per`
// more components.
struct StagePlan {
  uint32_t bits;    // bits per component
  uint32_t carry;   // bits of the label carried from one stage to the next
  uint32_t first;   // components in stage 0
  uint32_t per;     // new components per later stage
  uint32_t stages;  // number of stages
  uint32_t ebits;   // epoch bits available in every stage of this plan
};

inline __host__ __device__ StagePlan make_plan(uint32_t k, uint32_t bits, uint32_t carry) {
  StagePlan p{};
  const uint32_t total = k + 1;     // own block + one per letter
  const uint32_t cap = 125;         // key bits; at least 3 bits remain for the epoch
  p.bits = bits;
  p.carry = carry;
  if ((uint64_t)total * bits <= cap) {
    p.first = total;
    p.per = 1;
    p.stages = 1;
    const uint32_t used = total * bits;
    p.ebits = (128 - used) > 32 ? 32 : (128 - used);
  } else {
    p.first = cap / bits;
    p.per = (cap - carry) / bits;
    p.stages = 1 + (total - p.first + p.per - 1) / p.per;
    const uint32_t used = p.first * bits > carry + p.per * bits ? p.first * bits : carry + p.per * bits;
    p.ebits = (128 - used) > 32 ? 32 : (128 - used);
  }
  return p;
}


// Bucketed signature gather (large state spaces).  δ is re-sorted once per
// call: states are cut into NS source buckets of BS states and NT target
// buckets of BT states; the transitions of source bucket s whose target lies
// in target bucket T form segment (s, T), stored inside region s (cap entries)
// at seg[T*NS + s].x with seg[T*NS + s].y transitions, padded to a multiple of
// 8 entries.  Per entry: et = target - T*BT, es = a*BS + (source - s*BS), or
// kBucketPad for padding.  Each round a pass per target bucket writes the
// target's label into val (same index); a pass per source bucket reads its
// region back into a signature tile in shared memory.
struct BucketArgs {
  uint32_t NT, BT, NS, BS, cap;
  uint16_t *et, *es;       // NS*cap
  uint32_t *val;           // NS*cap: gathered labels of the current round
  uint2 *seg;              // NT*NS: {offset in region s, transitions}
  uint32_t *used;          // NS: padded entries of region s
  // uniqueness test of filter rounds: signature hashes split into P = 2^pbits
  // partitions of at most pcap entries, each deduplicated in shared memory
  uint32_t P, pbits, pcap;
  uint32_t *phash, *pq;    // P*pcap entries: low word of the signature hash, state
  uint32_t *pcnt;          // P: entries sent to each partition this round
  uint32_t *list;          // n: states whose signature is not proved unique
};

// Sizes of the bucketed gather for one state space (host side).
struct BucketPlan {
  uint32_t NT, BT, NS, BS, cap, P, pbits, pcap;
  size_t smem;             // dynamic shared memory of the bucketed kernel
};

// Arguments of the Moore (signature refinement) persistent kernel.  One call
// refines one state space; a batch or a disjoint union is one state space whose
// per-state data are reached through the segment table.
struct MooreArgs {
  const uint32_t *delta;   // k*n, letter-major
  const uint8_t *accept;   // n
  uint32_t n, k;
  uint32_t *lab[2];        // label ping-pong buffers, n each
  uint32_t *tmp;           // n: intermediate labels of multi-stage plans
  u128 *table;             // 2^log2S slots
  uint32_t log2S;
  uint32_t *minrep;        // 2^log2S: canonicalisation scratch
  uint32_t *bm[2];         // direct-mode bitmaps, 2^log2S bits each (ping-pong)
  uint32_t *seen1, *seen2; // filter-mode 2-bit counters, 2^mbits bits each
  uint32_t *seen3, *seen4; // second filter over listed states, 2^(mbits-1) bits each
  uint32_t *tmp2;          // n: second-filter bucket per state
  uint32_t mbits;
  unsigned long long *rep; // 2^log2S: filter-mode smallest member per table slot
  uint32_t *dups;          // filter-mode per-warp lists of states in shared buckets
  uint32_t *dups2;         // second-filter bucket of each listed state (same positions)
  uint32_t *wcnt;          // per-warp list lengths
  uint32_t wid;            // bits of a state number (labels of filter rounds)
  uint8_t *flag;           // n: canonicalisation scratch
  uint32_t *partials;      // gridDim entries
  uint32_t *out;           // n: canonical block numbers
  Ctrl *ctrl;
  uint32_t ebits;          // epoch field width used by every table pass
  uint32_t max_rounds;     // 0 = none
  unsigned long long timeout_ns;  // limit on the whole launch
  unsigned long long barrier_ns;  // limit on one barrier wait
  uint32_t vec;            // states per lane in table rounds: 1, 2 or 4
  uint32_t modes;          // bit 0: allow direct rounds, bit 1: allow filter rounds
  uint32_t predict_sparse; // 1: filter rounds also when B^(k+1) >= 64 n predicts unique signatures
  uint32_t stream_delta;   // 1: load δ with evict-first hints (table larger than L2)
  // equivalence by union: stop when these two states separate (if early_exit)
  uint32_t sep_a, sep_b;
  uint32_t track_pair;     // 1: record the round separating sep_a and sep_b
  uint32_t early_exit;
  uint32_t stop_discrete;  // 1: stop after a round that leaves n blocks (no confirming round)
  uint32_t bucket;         // 1: bucketed gather (moore_kernel<1, true>; B describes it)
  BucketArgs B;
  size_t B_smem;           // its dynamic shared memory (BucketPlan::smem)
};

struct LaunchInfo {
  int grid;
  int block;
};

// Grid of the Moore kernel (one cooperative wave) and its launch.  The
// bucketed kernel (bucket_smem > 0) runs one 1024-thread block per SM with
// that much dynamic shared memory.
cudaError_t moore_grid(uint32_t vec, LaunchInfo *info, size_t bucket_smem = 0);
cudaError_t launch_moore(const MooreArgs &a, cudaStream_t stream, LaunchInfo *info);

}  // namespace dfa
