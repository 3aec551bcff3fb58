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
// takes the previous stage's label plus `per` more components.
struct StagePlan {
  uint32_t bits;    // bits per component
  uint32_t first;   // components in stage 0
  uint32_t per;     // new components per later stage
  uint32_t stages;  // number of stages
  uint32_t ebits;   // epoch bits available in every stage of this plan
};

StagePlan make_plan(uint32_t k, uint32_t bits);

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
  uint8_t *flag;           // n: canonicalisation scratch
  uint32_t *partials;      // gridDim entries
  uint32_t *out;           // n: canonical block numbers
  Ctrl *ctrl;
  StagePlan plan1;         // round 1 (components are acceptance bits)
  StagePlan planr;         // rounds >= 2 (components are labels < 2^log2S)
  uint32_t ebits;          // epoch field width used by every pass
  uint32_t max_rounds;     // 0 = none
  unsigned long long timeout_ns;  // limit on the whole launch
  unsigned long long barrier_ns;  // limit on one barrier wait
  uint32_t vec;            // 4: vectorised path (n % 4 == 0), else 1
  uint32_t stream_delta;   // 1: load δ with evict-first hints (table larger than L2)
  // equivalence by union: stop when these two states separate (if early_exit)
  uint32_t sep_a, sep_b;
  uint32_t track_pair;     // 1: record the round separating sep_a and sep_b
  uint32_t early_exit;
};

struct LaunchInfo {
  int grid;
  int block;
};

// Grid of the Moore kernel (one cooperative wave) and its launch.
cudaError_t moore_grid(uint32_t vec, LaunchInfo *info);
cudaError_t launch_moore(const MooreArgs &a, cudaStream_t stream, LaunchInfo *info);

}  // namespace dfa
