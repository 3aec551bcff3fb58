// Measurement aid for bench.py, outside the product library: the rate of
// random 4-byte reads from an array small enough to stay in L2.
//
// Every round of signature refinement reads block[δ(q,a)] for all n states and
// k letters: k·n reads at addresses that follow no pattern, served by L2 (the
// label array is a few tens of MiB).  Each read costs one L2 request whatever
// its width, so the rate of such requests, not DRAM bandwidth, bounds a round
// of the refinement kernel.  This kernel issues only such reads (indices from
// a 64-bit linear congruential sequence per thread, eight independent reads
// in flight per thread), so its rate is the figure a round's gathers are
// compared with.  Built by bench.py (and __graft_entry__.build()) into
// _build/libl2probe.so.
//
//   int l2probe_gather(const void *table, size_t table_bytes, uint64_t reads,
//                      void *stream, double *reads_per_s);
//     table        device memory, table_bytes a power of two >= 8 (read only);
//     reads        reads to time (rounded up to a whole number per thread);
//     stream       cudaStream_t (NULL = legacy default stream);
//     reads_per_s  out: reads per second of the timed pass (one untimed pass
//                  first brings the table into L2).
//   Returns 0, -1 for bad arguments, -3 for a CUDA error (l2probe_error()
//   describes the last failure).  Synchronises the stream.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

namespace {

constexpr int kThreads = 512;
constexpr int kInflight = 8;
__device__ uint32_t g_sink;   // written only if a sum hits the sentinel
char g_err[256];

__global__ void __launch_bounds__(kThreads) gather_kernel(const uint32_t *__restrict__ table, uint32_t mask,
                                                         uint64_t per_thread) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t acc = 0;
  uint64_t x = tid * 0x9E3779B97F4A7C15ull + 1;
  for (uint64_t i = 0; i < per_thread; i += kInflight) {
    uint32_t v[kInflight];
#pragma unroll
    for (int j = 0; j < kInflight; ++j) {
      x = x * 6364136223846793005ull + 1442695040888963407ull;
      v[j] = table[(uint32_t)(x >> 32) & mask];
    }
#pragma unroll
    for (int j = 0; j < kInflight; ++j) acc += v[j];
  }
  if (acc == 0x9E3779B9u) g_sink = acc;   // keeps the reads alive
}

int fail(int code, const char *msg, cudaError_t e = cudaSuccess) {
  snprintf(g_err, sizeof g_err, "%s%s%s", msg, e != cudaSuccess ? ": " : "", e != cudaSuccess ? cudaGetErrorString(e) : "");
  return code;
}

}  // namespace

extern "C" const char *l2probe_error(void) { return g_err; }

extern "C" int l2probe_gather(const void *table, size_t table_bytes, uint64_t reads, void *stream,
                              double *reads_per_s) {
  if (!table || !reads_per_s) return fail(-1, "table or reads_per_s is NULL");
  if (table_bytes < 8 || (table_bytes & (table_bytes - 1)) != 0) return fail(-1, "table_bytes must be a power of two >= 8");
  if (table_bytes / 4 > (1ull << 32)) return fail(-1, "table larger than 2^32 words");
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, table) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
    cudaGetLastError();
    return fail(-1, "table must be device memory");
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return fail(-3, "cudaGetDevice", e);
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return fail(-3, "device attribute", e);
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gather_kernel, kThreads, 0)) != cudaSuccess)
    return fail(-3, "occupancy", e);
  const uint64_t threads = (uint64_t)sms * (per_sm < 2 ? per_sm : 2) * kThreads;
  uint64_t per_thread = (reads + threads - 1) / threads;
  per_thread = (per_thread + kInflight - 1) / kInflight * kInflight;
  if (per_thread == 0) per_thread = kInflight;
  const dim3 grid((unsigned)(threads / kThreads));
  const uint32_t mask = (uint32_t)(table_bytes / 4 - 1);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if ((e = cudaEventCreate(&ev[0])) != cudaSuccess || (e = cudaEventCreate(&ev[1])) != cudaSuccess)
    return fail(-3, "cudaEventCreate", e);
  gather_kernel<<<grid, kThreads, 0, st>>>(static_cast<const uint32_t *>(table), mask, kInflight);
  cudaEventRecord(ev[0], st);
  gather_kernel<<<grid, kThreads, 0, st>>>(static_cast<const uint32_t *>(table), mask, per_thread);
  cudaEventRecord(ev[1], st);
  e = cudaEventSynchronize(ev[1]);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  if (e != cudaSuccess) return fail(-3, "probe kernel", e);
  *reads_per_s = ms > 0.f ? (double)threads * (double)per_thread / (ms * 1e-3) : 0.0;
  return 0;
}
