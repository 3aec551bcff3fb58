// The serving loop.
#include "api_util.h"

using namespace dfa;

extern "C" {

int dfa_serve_create(dfa_server **out, size_t hbm_budget_bytes, uint32_t max_slots, int device) {
  (void)out; (void)hbm_budget_bytes; (void)max_slots; (void)device;
  return fail(DFA_EINVAL, "serving not built yet");
}
int dfa_serve_submit(dfa_server *s, int kind, const dfa_t *a, const dfa_t *b, const dfa_opts *opts,
                     uint64_t *ticket) {
  (void)s; (void)kind; (void)a; (void)b; (void)opts; (void)ticket;
  return fail(DFA_EINVAL, "serving not built yet");
}
int dfa_serve_poll(dfa_server *s, uint64_t ticket, dfa_result *res, int *equivalent, uint32_t *block_out) {
  (void)s; (void)ticket; (void)res; (void)equivalent; (void)block_out;
  return fail(DFA_EINVAL, "serving not built yet");
}
int dfa_serve_wait(dfa_server *s, uint64_t ticket, uint64_t timeout_ns, dfa_result *res, int *equivalent,
                   uint32_t *block_out) {
  (void)s; (void)ticket; (void)timeout_ns; (void)res; (void)equivalent; (void)block_out;
  return fail(DFA_EINVAL, "serving not built yet");
}
int dfa_serve_stats(dfa_server *s, double *p50_us, double *p99_us, double *throughput_rps) {
  (void)s; (void)p50_us; (void)p99_us; (void)throughput_rps;
  return fail(DFA_EINVAL, "serving not built yet");
}
int dfa_serve_destroy(dfa_server *s) {
  (void)s;
  return DFA_OK;
}

}  // extern "C"
