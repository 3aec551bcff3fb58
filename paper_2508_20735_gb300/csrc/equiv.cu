// Language equivalence by refining the disjoint union (Section 4: equivalence
// can be decided via minimisation).  U = A ⊎ B has states 0..nA-1 from A and
// nA..nA+nB-1 from B; δ_U(nA+q, a) = nA + δ_B(q, a).  L(A) = L(B) iff the
// start states q0A and nA+q0B end in the same block of U's coarsest partition.
#include <cstring>

#include "api_util.h"

namespace dfa {

// Adds `offset` to the targets of states [first, first+count) of a letter-major
// table with n_u states per row, checking each original target < count.
__global__ void offset_targets_kernel(uint32_t *delta_u, uint32_t n_u, uint32_t k, uint32_t first, uint32_t count,
                                      uint32_t offset, uint32_t *err) {
  const uint64_t total = (uint64_t)k * count;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const uint32_t a = (uint32_t)(i / count), q = (uint32_t)(i % count);
    uint32_t *p = delta_u + (size_t)a * n_u + first + q;
    uint32_t t = *p;
    if (t >= count) {
      atomicOr(err, ERR_BAD_DELTA);
      t = 0;
    }
    *p = t + offset;
  }
}

__global__ void check_targets_kernel(const uint32_t *delta_u, uint32_t n_u, uint32_t k, uint32_t count,
                                     uint32_t *err) {
  const uint64_t total = (uint64_t)k * count;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const uint32_t a = (uint32_t)(i / count), q = (uint32_t)(i % count);
    if (delta_u[(size_t)a * n_u + q] >= count) atomicOr(err, ERR_BAD_DELTA);
  }
}

cudaError_t launch_offset_targets(uint32_t *delta_u, uint32_t n_u, uint32_t k, uint32_t first, uint32_t count,
                                  uint32_t offset, uint32_t *err, cudaStream_t st) {
  if (k == 0 || count == 0) return cudaSuccess;
  offset_targets_kernel<<<1216, 256, 0, st>>>(delta_u, n_u, k, first, count, offset, err);
  return cudaGetLastError();
}

static constexpr size_t kUnionExtra = 256;   // error word of the union build

}  // namespace dfa

using namespace dfa;

extern "C" {

size_t dfa_equivalent_workspace_size(const dfa_t *a, const dfa_t *b, const dfa_opts *opts) {
  if (check_dfa(a, "a") != DFA_OK || check_dfa(b, "b") != DFA_OK) return 0;
  if (a->k != b->k) return 0;
  const uint64_t n_u = (uint64_t)a->n + b->n;
  if (n_u > DFA_MAX_STATES) return 0;
  const dfa_opts o = default_opts(opts);
  BucketPlan bp{};
  const bool bucket = choose_bucket(n_u, a->k, o.flags, &bp);
  return moore_layout(n_u, a->k, true, true, true, bucket ? &bp : nullptr).total + kUnionExtra;
}

int dfa_equivalent(const dfa_t *a, const dfa_t *b, const dfa_opts *opts, int *equivalent, dfa_result *res,
                   void *workspace, size_t ws_bytes, void *stream) {
  int rc = check_dfa(a, "a");
  if (rc != DFA_OK) return rc;
  rc = check_dfa(b, "b");
  if (rc != DFA_OK) return rc;
  if (a->k != b->k) return fail(DFA_EINVAL, "alphabets differ: k_A = %u, k_B = %u", a->k, b->k);
  if (!equivalent) return fail(DFA_EINVAL, "equivalent is NULL");
  if (!workspace || !aligned(workspace, 256)) return fail(DFA_EINVAL, "workspace NULL or not 256-byte aligned");
  const uint64_t n_u64 = (uint64_t)a->n + b->n;
  if (n_u64 > DFA_MAX_STATES) return fail(DFA_EINVAL, "n_A + n_B exceeds %u", DFA_MAX_STATES);
  const uint32_t n_u = (uint32_t)n_u64, k = a->k;
  const dfa_opts o = default_opts(opts);
  if (o.algo != DFA_ALGO_MOORE) return fail(DFA_EINVAL, "equivalence uses signature refinement (algo 0)");
  BucketPlan bp{};
  const bool bucket = choose_bucket(n_u, k, o.flags, &bp);
  const MooreLayout L = moore_layout(n_u, k, true, true, true, bucket ? &bp : nullptr);
  const size_t need = L.total + kUnionExtra;
  if (ws_bytes < need) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, need);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char *ws = static_cast<char *>(workspace);
  uint32_t *du = reinterpret_cast<uint32_t *>(ws + L.delta);
  uint8_t *au = reinterpret_cast<uint8_t *>(ws + L.accept);
  uint32_t *err = reinterpret_cast<uint32_t *>(ws + L.total);
  cudaError_t e = cudaMemsetAsync(err, 0, 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "memset");
  if (k > 0) {
    e = cudaMemcpy2DAsync(du, (size_t)n_u * 4, a->delta, (size_t)a->n * 4, (size_t)a->n * 4, k, cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy delta of A");
    e = cudaMemcpy2DAsync(du + a->n, (size_t)n_u * 4, b->delta, (size_t)b->n * 4, (size_t)b->n * 4, k,
                          cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(e, "copy delta of B");
    check_targets_kernel<<<1216, 256, 0, st>>>(du, n_u, k, a->n, err);
    e = launch_offset_targets(du, n_u, k, a->n, b->n, a->n, err, st);
    if (e != cudaSuccess) return cuda_fail(e, "union kernel");
  }
  e = cudaMemcpyAsync(au, a->accept, a->n, cudaMemcpyDefault, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy accept of A");
  e = cudaMemcpyAsync(au + a->n, b->accept, b->n, cudaMemcpyDefault, st);
  if (e != cudaSuccess) return cuda_fail(e, "copy accept of B");
  uint32_t err_host = 0;
  e = cudaMemcpyAsync(&err_host, err, 4, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e, "read union status");
  PairTrack tr{a->start, a->n + b->start, (o.flags & DFA_FLAG_EARLY_EXIT) ? 1u : 0u};
  uint32_t *out = reinterpret_cast<uint32_t *>(ws + L.out);
  Ctrl c{};
  if (small_fits(n_u, k, o)) {   // a union of at most 16,384 states: one thread block or one cluster
    Ctrl *cd = reinterpret_cast<Ctrl *>(ws + L.ctrl);
    rc = enqueue_small(du, au, n_u, k, out, cd, o, st, &tr);
    if (rc != DFA_OK) return rc;
    e = cudaMemcpyAsync(&c, cd, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "refinement of the union");
  } else {
    const uint32_t vec_ok = pick_vec(n_u, k, du, au, o.schedule);
    rc = run_moore(du, au, n_u, k, out, L, ws, o, st, &tr, &c, vec_ok);
    if (rc != DFA_OK) return rc;
  }
  if (err_host & ERR_BAD_DELTA) return fail(DFA_EINVAL, "a transition target is >= n");
  const int status = status_from_ctrl(c);
  if (res) {
    res->num_blocks = c.num_blocks;
    res->rounds_changed = c.rounds_changed;
    res->rounds_executed = c.rounds_executed;
    res->status = status;
    res->device_ns = c.t_end - c.t_start;
  }
  if (status != DFA_OK) return status;
  *equivalent = (c.sep_round == 0xFFFFFFFFu) ? 1 : 0;
  return DFA_OK;
}

}  // extern "C"
