/*
 * CPU oracle, C part: Moore refinement (Algorithm 4's result) in plain C,
 * single-threaded or with OpenMP over all host cores.  TEST INFRASTRUCTURE
 * ONLY (the tests cross-check it against the numpy oracle and Hopcroft, and
 * bench.py times it as the CPU baseline); never part of the library's product
 * path.  It shares no code with the CUDA library.
 *
 * Each round computes, for every state q, the signature
 *   sig(q) = (L[q], L[δ(q,0)], ..., L[δ(q,k-1)])
 * and gives q the label of the smallest state with an equal signature (labels
 * are block representatives).  Equal signatures are found exactly: states are
 * grouped by a 64-bit hash of their signature into partitions (a counting sort
 * that keeps state order within a partition), and within a partition a state
 * joins the first earlier state whose full signature equals its own, compared
 * component by component; a hash collision never merges blocks.  The loop
 * stops after the first round whose block count equals the previous one (the
 * until-test of Algorithm 4).  The output numbers blocks 0..B-1 in order of
 * their smallest state.
 *
 *   threads  1: one thread; 0: OpenMP's default (all host cores); else that many.
 * Returns 0, -1 for a bad argument or transition target, -2 when memory runs out.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PBITS 10
#define NPART (1u << PBITS)

static uint64_t mix64(uint64_t h, uint32_t v) {
  h = (h ^ v) * 0x9E3779B97F4A7C15ull;
  return h ^ (h >> 31);
}

static int same_sig(uint32_t n, uint32_t k, const uint32_t *delta, const uint32_t *L, uint32_t q, uint32_t p) {
  if (L[q] != L[p]) return 0;
  for (uint32_t a = 0; a < k; ++a)
    if (L[delta[(size_t)a * n + q]] != L[delta[(size_t)a * n + p]]) return 0;
  return 1;
}

int oracle_moore_c(uint32_t n, uint32_t k, const uint32_t *delta, const uint8_t *accept, int threads,
                   uint32_t *block_out, uint32_t *rounds_changed, uint32_t *rounds_executed, uint32_t *num_blocks) {
  if (n == 0 || !accept || !block_out || (k > 0 && !delta)) return -1;
  for (size_t i = 0; i < (size_t)k * n; ++i)
    if (delta[i] >= n) return -1;
#ifdef _OPENMP
  const int nt = threads == 1 ? 1 : (threads > 0 ? threads : omp_get_max_threads());
#else
  const int nt = 1;
  (void)threads;
#endif
  uint32_t *L = (uint32_t *)malloc((size_t)n * 4), *N = (uint32_t *)malloc((size_t)n * 4);
  uint64_t *h = (uint64_t *)malloc((size_t)n * 8);
  uint32_t *perm = (uint32_t *)malloc((size_t)n * 4);
  uint64_t *hist = (uint64_t *)calloc((size_t)nt * NPART + 1, 8);
  uint64_t *start = (uint64_t *)malloc((NPART + 1) * 8);
  if (!L || !N || !h || !perm || !hist || !start) {
    free(L); free(N); free(h); free(perm); free(hist); free(start);
    return -2;
  }
  /* the initial partition {F, Q \ F}: representatives min F and min (Q \ F) */
  uint32_t qf = n, qn = n;
  for (uint32_t q = 0; q < n; ++q) {
    if (accept[q] && qf == n) qf = q;
    if (!accept[q] && qn == n) qn = q;
  }
  for (uint32_t q = 0; q < n; ++q) L[q] = accept[q] ? qf : qn;
  uint32_t B_prev = (qf < n) + (qn < n), B = B_prev, changed = 0, executed = 0;
  int rc = 0;
  for (;;) {
    ++executed;
    /* 1. signature hashes */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < (int64_t)n; ++i) {
      const uint32_t q = (uint32_t)i;
      uint64_t x = mix64(0x243F6A8885A308D3ull, L[q]);
      for (uint32_t a = 0; a < k; ++a) x = mix64(x, L[delta[(size_t)a * n + q]]);
      h[q] = x;
    }
    /* 2. counting sort by partition (top PBITS of the hash); each thread
          handles a contiguous range of states, so a partition lists its states
          in increasing order */
    memset(hist, 0, ((size_t)nt * NPART + 1) * 8);
#pragma omp parallel num_threads(nt)
    {
#ifdef _OPENMP
      const int t = omp_get_thread_num();
#else
      const int t = 0;
#endif
      const uint64_t lo = (uint64_t)n * t / nt, hi = (uint64_t)n * (t + 1) / nt;
      uint64_t *mine = hist + (size_t)t * NPART;
      for (uint64_t q = lo; q < hi; ++q) mine[h[q] >> (64 - PBITS)]++;
#pragma omp barrier
#pragma omp single
      {
        uint64_t run = 0;
        for (uint32_t p = 0; p < NPART; ++p) {
          start[p] = run;
          for (int u = 0; u < nt; ++u) {
            const uint64_t c = hist[(size_t)u * NPART + p];
            hist[(size_t)u * NPART + p] = run;
            run += c;
          }
        }
        start[NPART] = run;
      }
      for (uint64_t q = lo; q < hi; ++q) perm[mine[h[q] >> (64 - PBITS)]++] = (uint32_t)q;
    }
    /* 3. within each partition: the smallest state with an equal signature */
    uint32_t fresh = 0;
#pragma omp parallel num_threads(nt) reduction(+ : fresh)
    {
      uint32_t cap = 0;
      uint32_t *tab = NULL;   /* open addressing over the partition's positions: index + 1, 0 = free */
#pragma omp for schedule(dynamic, 4)
      for (int p = 0; p < (int)NPART; ++p) {
        const uint64_t b = start[p], e = start[p + 1];
        const uint32_t cnt = (uint32_t)(e - b);
        if (cnt == 0) continue;
        uint32_t size = 16;
        while (size < 2 * cnt) size <<= 1;
        if (size > cap) {
          free(tab);
          tab = (uint32_t *)malloc((size_t)size * 4);
          cap = size;
          if (!tab) {
            cap = 0;
#pragma omp atomic write
            rc = -2;
            continue;
          }
        }
        memset(tab, 0, (size_t)size * 4);
        for (uint64_t i = b; i < e; ++i) {
          const uint32_t q = perm[i];
          uint32_t s = (uint32_t)h[q] & (size - 1);
          for (;;) {
            const uint32_t v = tab[s];
            if (v == 0) {   /* q is the smallest state with its signature */
              tab[s] = (uint32_t)(i - b) + 1;
              N[q] = q;
              ++fresh;
              break;
            }
            const uint32_t p2 = perm[b + v - 1];
            if (h[p2] == h[q] && same_sig(n, k, delta, L, q, p2)) {
              N[q] = p2;
              break;
            }
            s = (s + 1) & (size - 1);
          }
        }
      }
      free(tab);
    }
    if (rc) break;
    uint32_t *t = L;
    L = N;
    N = t;
    B = fresh;
    if (B != B_prev) ++changed;
    if (B == B_prev) break;
    B_prev = B;
  }
  if (rc == 0) {
    /* canonical numbering: rank of each block's smallest state */
    uint32_t r = 0;
    for (uint32_t q = 0; q < n; ++q)
      if (L[q] == q) N[q] = r++;
    for (uint32_t q = 0; q < n; ++q) block_out[q] = N[L[q]];
    if (rounds_changed) *rounds_changed = changed;
    if (rounds_executed) *rounds_executed = executed;
    if (num_blocks) *num_blocks = r;
  }
  free(L); free(N); free(h); free(perm); free(hist); free(start);
  return rc;
}

/* Threads OpenMP would use by default (1 without OpenMP): the host cores. */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
