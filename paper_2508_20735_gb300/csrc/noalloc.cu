// dfa_minimise_noalloc: signature refinement for callers that cannot give the
// library a workspace.
//
// Some callers have no way to obtain device memory for us: code embedded in a
// host framework that owns every device allocation and forbids outside ones,
// or latency-critical paths where cudaMalloc is off-limits because it may
// synchronise the device and take unbounded time.  This entry point uses a
// fixed scratch area compiled into the library instead.  The area is a
// file-scope __device__ array, so every GPU that loads the library holds it
// (kNoallocScratchBytes) until the process exits.
//
// The array's name, used in host code, is only a host-side handle, not a
// device address; passing it to a kernel would fault (or, where the GPU can
// reach host memory, silently touch the wrong memory).  The device address is
// looked up once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on it.  Every call waits for its stream (it
// reads the round counts back), so a call on a stream that is being captured
// is refused before anything is enqueued.  Calls on one device share the one
// array: each holds that device's lock from its launch until its stream has
// drained, so calls from several host threads or on several streams run one
// after another instead of racing.  Everything a call needs zeroed is cleared
// by the call itself.
#include <mutex>

#include "api_util.h"

namespace dfa {

// 8 MiB: the Moore kernel's scratch at DFA_NOALLOC_MAX_STATES states is about
// 6.6 MiB on a 152-SM GB300: table 2 MiB, slot owners 1 MiB, labels and
// filter buckets 4 x 256 KiB, canonical numbering 0.6 MiB, bitmaps 0.3 MiB,
// and the filter rounds' per-warp lists, 2 x 4 x (n + 32 x (warps + 2)) bytes
// with 32 warps per SM (1.7 MiB at 152 SMs).  The lists grow with the SM
// count; a layout that would not fit is rejected with DFA_EINVAL.
static constexpr size_t kNoallocScratchBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

static constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static char *g_noalloc_ptr[kMaxDevices];          // device address per device, filled on first use
static std::mutex g_noalloc_call_mu[kMaxDevices];   // held by a call for its whole run on that device

static int noalloc_scratch(int dev, char **out) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);   // with `dev` current
    if (e != cudaSuccess || p == nullptr) return cuda_fail(e, "cudaGetSymbolAddress(noalloc scratch)");
    g_noalloc_ptr[dev] = static_cast<char *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return DFA_OK;
}

}  // namespace dfa

using namespace dfa;

extern "C" int dfa_minimise_noalloc(const dfa_t *d, const dfa_opts *opts, uint32_t *block_out, dfa_result *res,
                                    void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int rc = check_dfa(d, "dfa");
  if (rc != DFA_OK) return rc;
  if (d->n > DFA_NOALLOC_MAX_STATES)
    return fail(DFA_EINVAL, "dfa_minimise_noalloc handles at most %u states (got %u); use dfa_minimise",
                DFA_NOALLOC_MAX_STATES, d->n);
  if (!block_out) return fail(DFA_EINVAL, "block_out is NULL");
  const dfa_opts o = default_opts(opts);
  if (o.algo != DFA_ALGO_MOORE) return fail(DFA_EINVAL, "dfa_minimise_noalloc supports signature refinement only");
  if ((d->k > 0 && !is_device_ptr(d->delta)) || !is_device_ptr(d->accept) || !is_device_ptr(block_out))
    return fail(DFA_EINVAL, "dfa_minimise_noalloc needs device pointers for delta, accept and block_out");
  const MooreLayout L = moore_layout(d->n, d->k, false, false, false);
  if (L.total > kNoallocScratchBytes)
    return fail(DFA_EINVAL, "scratch of %zu bytes exceeds the fixed %zu", L.total, kNoallocScratchBytes);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t ec = cudaStreamIsCapturing(st, &cs);
  if (ec != cudaSuccess) return cuda_fail(ec, "cudaStreamIsCapturing");
  if (cs != cudaStreamCaptureStatusNone)
    return fail(DFA_EINVAL, "dfa_minimise_noalloc waits for its stream and cannot be captured into a graph");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(DFA_EINVAL, "device %d beyond %d", dev, kMaxDevices);
  char *ws = nullptr;
  rc = noalloc_scratch(dev, &ws);
  if (rc != DFA_OK) return rc;
  std::lock_guard<std::mutex> busy(g_noalloc_call_mu[dev]);
  const uint32_t vec = pick_vec(d->n, d->k, d->delta, d->accept, o.schedule);
  Ctrl c{};
  // run_moore clears the control block; the kernel clears its table and scratch.
  rc = run_moore(d->delta, d->accept, d->n, d->k, block_out, L, ws, o, st, nullptr, &c, vec);
  if (rc != DFA_OK) return rc;
  const int status = status_from_ctrl(c);
  if (res) {
    res->num_blocks = c.num_blocks;
    res->rounds_changed = c.rounds_changed;
    res->rounds_executed = c.rounds_executed;
    res->status = status;
    res->device_ns = c.t_end - c.t_start;
  }
  return status;
}
