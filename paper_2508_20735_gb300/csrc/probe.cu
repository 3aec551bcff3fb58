// dfa_probe_l2_gather: the rate of random 4-byte reads from an L2-resident
// array on this GPU, the ceiling of the refinement rounds (a measurement aid;
// the paper has no counterpart).
//
// Every round of signature refinement reads block[δ(q,a)] for all n states
// and k letters: k·n reads at addresses that follow no pattern, served by L2
// (the block array is a few tens of MiB).  Each read costs one L2 request
// whatever its width, so the rate of such requests, not DRAM bandwidth, bounds
// a round.  This kernel issues only such reads (indices from a multiplicative
// hash of the thread's counter, eight independent reads in flight per
// thread), so its rate is the figure a round's gathers are compared with.
#include "api_util.h"

namespace dfa {

static constexpr int kProbeThreads = 512;
static constexpr int kProbeInflight = 8;
static __device__ uint32_t g_probe_sink;   // written only if a sum hits the sentinel

__global__ void __launch_bounds__(kProbeThreads) probe_gather_kernel(const uint32_t *__restrict__ table,
                                                                    uint32_t mask, uint64_t per_thread) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  uint64_t x = tid * 0x9E3779B97F4A7C15ull + 1;
  for (uint64_t i = 0; i < per_thread; i += kProbeInflight) {
    uint32_t v[kProbeInflight];
#pragma unroll
    for (int j = 0; j < kProbeInflight; ++j) {
      x = x * 6364136223846793005ull + 1442695040888963407ull;   // 64-bit LCG step
      v[j] = table[(uint32_t)(x >> 32) & mask];
    }
#pragma unroll
    for (int j = 0; j < kProbeInflight; ++j) acc += v[j];
  }
  if (acc == 0x9E3779B9u) g_probe_sink = acc;   // keeps the reads alive
}

}  // namespace dfa

using namespace dfa;

extern "C" int dfa_probe_l2_gather(void *table, size_t table_bytes, uint64_t reads, void *stream,
                                   double *reads_per_s) {
  if (!table || !reads_per_s) return fail(DFA_EINVAL, "table or reads_per_s is NULL");
  if (table_bytes < 8 || (table_bytes & (table_bytes - 1)) != 0)
    return fail(DFA_EINVAL, "table_bytes must be a power of two >= 8 (got %zu)", table_bytes);
  if (table_bytes / 4 > (1ull << 32)) return fail(DFA_EINVAL, "table larger than 2^32 words");
  if (!is_device_ptr(table)) return fail(DFA_EINVAL, "table must be device memory");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return cuda_fail(e, "device attribute");
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, probe_gather_kernel, kProbeThreads, 0)) !=
      cudaSuccess)
    return cuda_fail(e, "occupancy");
  const uint64_t threads = (uint64_t)sms * (per_sm < 2 ? per_sm : 2) * kProbeThreads;
  uint64_t per_thread = (reads + threads - 1) / threads;
  per_thread = (per_thread + kProbeInflight - 1) / kProbeInflight * kProbeInflight;
  if (per_thread == 0) per_thread = kProbeInflight;
  const dim3 grid((unsigned)(threads / kProbeThreads));
  const uint32_t mask = (uint32_t)(table_bytes / 4 - 1);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if ((e = cudaEventCreate(&ev[0])) != cudaSuccess || (e = cudaEventCreate(&ev[1])) != cudaSuccess)
    return cuda_fail(e, "cudaEventCreate");
  // one pass to bring the table into L2, then the timed pass
  probe_gather_kernel<<<grid, kProbeThreads, 0, st>>>(static_cast<const uint32_t *>(table), mask,
                                                      kProbeInflight);
  cudaEventRecord(ev[0], st);
  probe_gather_kernel<<<grid, kProbeThreads, 0, st>>>(static_cast<const uint32_t *>(table), mask, per_thread);
  cudaEventRecord(ev[1], st);
  e = cudaEventSynchronize(ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) return cuda_fail(e, "probe kernel");
  *reads_per_s = ms > 0.f ? (double)threads * (double)per_thread / (ms * 1e-3) : 0.0;
  return DFA_OK;
}
