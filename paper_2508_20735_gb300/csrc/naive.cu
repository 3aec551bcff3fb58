// naivePR (Section 3.2, Algorithm 2) and transPR (Section 3.4, Algorithm 5).
#include "api_util.h"

namespace dfa {

size_t naive_workspace_size(const dfa_t *d, const dfa_opts &o) {
  (void)d;
  (void)o;
  return 256;
}

int run_naive_minimise(const dfa_t *d, const dfa_opts &o, uint32_t *block_out, dfa_result *res, void *workspace,
                       size_t ws_bytes, cudaStream_t st) {
  (void)d; (void)o; (void)block_out; (void)res; (void)workspace; (void)ws_bytes; (void)st;
  return fail(DFA_EINVAL, "naivePR/transPR path not built yet");
}

}  // namespace dfa
