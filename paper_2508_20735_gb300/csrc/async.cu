// dfa_minimise_async / dfa_minimise_result: signature refinement enqueued on a
// stream without waiting for it, so that a caller can keep several
// minimisations in flight on different streams: the copies of one (inputs in,
// partition out) then overlap the refinement of another.  The enqueued work is
// exactly dfa_minimise's: staging of host inputs, the cooperative refinement
// kernel, the copy of the partition; the result (rounds, block count, status)
// is read from the workspace's control block once the stream has passed it.
#include "api_util.h"

using namespace dfa;

extern "C" {

int dfa_minimise_async(const dfa_t *d, const dfa_opts *opts, uint32_t *block_out, void *workspace, size_t ws_bytes,
                       void *stream) {
  int rc = check_dfa(d, "dfa");
  if (rc != DFA_OK) return rc;
  if (!block_out) return fail(DFA_EINVAL, "block_out is NULL");
  if (!workspace || !aligned(workspace, 256)) return fail(DFA_EINVAL, "workspace NULL or not 256-byte aligned");
  const dfa_opts o = default_opts(opts);
  if (o.algo != DFA_ALGO_MOORE) return fail(DFA_EINVAL, "the asynchronous call runs signature refinement (algo 0)");
  const bool hd = d->k > 0 && !is_device_ptr(d->delta);
  const bool ha = !is_device_ptr(d->accept);
  const bool ho = !is_device_ptr(block_out);
  BucketPlan bp{};
  const bool bucket = choose_bucket(d->n, d->k, o.flags, &bp);
  const MooreLayout L = moore_layout(d->n, d->k, hd, ha, true, bucket ? &bp : nullptr);
  if (ws_bytes < L.total) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
  if (L.ctrl != 0) return fail(DFA_ECUDA, "control block not at the workspace's start (internal error)");
  char *ws = static_cast<char *>(workspace);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t *delta = d->delta;
  const uint8_t *accept = d->accept;
  cudaError_t e = cudaSuccess;
  if (hd) {
    e = cudaMemcpyAsync(ws + L.delta, d->delta, (size_t)d->k * d->n * 4, cudaMemcpyHostToDevice, st);
    delta = reinterpret_cast<const uint32_t *>(ws + L.delta);
  }
  if (e == cudaSuccess && ha) {
    e = cudaMemcpyAsync(ws + L.accept, d->accept, d->n, cudaMemcpyHostToDevice, st);
    accept = reinterpret_cast<const uint8_t *>(ws + L.accept);
  }
  if (e != cudaSuccess) return cuda_fail(e, "copy inputs to device");
  uint32_t *out = ho ? reinterpret_cast<uint32_t *>(ws + L.out) : block_out;
  if (small_fits(d->n, d->k, o))
    rc = enqueue_small(delta, accept, d->n, d->k, out, reinterpret_cast<Ctrl *>(ws + L.ctrl), o, st);
  else
    rc = enqueue_moore(delta, accept, d->n, d->k, out, L, ws, o, st, nullptr,
                       pick_vec(d->n, d->k, delta, accept, o.schedule));
  if (rc != DFA_OK) return rc;
  if (ho) {
    e = cudaMemcpyAsync(block_out, out, (size_t)d->n * 4, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy blocks to host");
  }
  return DFA_OK;
}

int dfa_minimise_result(const void *workspace, dfa_result *res, void *stream) {
  if (!workspace) return fail(DFA_EINVAL, "workspace is NULL");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Ctrl c{};
  cudaError_t e = cudaMemcpyAsync(&c, workspace, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "refinement kernel");
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

}  // extern "C"
