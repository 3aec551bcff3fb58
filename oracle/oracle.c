/*
 * CPU oracle, C part.  TEST INFRASTRUCTURE ONLY: it is called by the tests,
 * by __graft_entry__.smoke() and by bench.py's CPU-baseline leg, never by the
 * library's product path.  It shares no code with the CUDA library.
 *
 * Independent cross-checks for the partition-refinement oracle:
 *   oracle_hopcroft        Hopcroft's n log n coarsest-partition algorithm (the
 *                          classical sequential method the paper cites in
 *                          Section 1 as the best known bound), written from the
 *                          textbook formulation with a refinable partition.
 *   oracle_hk_equivalent   Hopcroft-Karp equivalence (Section 4, Algorithm 6)
 *                          with union-find for the closure R+.
 *   oracle_shortest_cex    Algorithm 6 without R+: breadth-first exploration of
 *                          the synchronous product (Section 4), returning the
 *                          length of a shortest word on which A and B disagree.
 *   oracle_pair_table      Section 3.1's characterisation (Algorithm 1): a pair
 *                          of states is inequivalent iff it is apart initially
 *                          or reaches an apart pair in the pair graph; computed
 *                          by backward search over pairs.  Tiny inputs only.
 *
 * All functions return 0 on success and a negative value on bad input or when
 * memory runs out.  Block numbers written to block_out are arbitrary labels.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------- inverse transitions: for letter a, the sources of each target ---------- */
typedef struct { uint64_t *off; uint32_t *src; } inverse_t;

static int build_inverse(uint32_t n, uint32_t k, const uint32_t *delta, inverse_t *inv) {
  inv->off = (uint64_t *)calloc((size_t)k * (n + 1) + 1, sizeof(uint64_t));
  inv->src = (uint32_t *)malloc(((size_t)k * n + 1) * sizeof(uint32_t));
  if (!inv->off || !inv->src) return -2;
  for (uint32_t a = 0; a < k; ++a) {
    uint64_t *o = inv->off + (size_t)a * (n + 1);
    const uint32_t *d = delta + (size_t)a * n;
    for (uint32_t q = 0; q < n; ++q) {
      if (d[q] >= n) return -1;
      o[d[q] + 1]++;
    }
    for (uint32_t t = 0; t < n; ++t) o[t + 1] += o[t];
    uint64_t *fill = (uint64_t *)malloc((size_t)(n + 1) * sizeof(uint64_t));
    if (!fill) return -2;
    memcpy(fill, o, (size_t)(n + 1) * sizeof(uint64_t));
    for (uint32_t q = 0; q < n; ++q) inv->src[(size_t)a * n + fill[d[q]]++] = q;
    free(fill);
  }
  return 0;
}

static void free_inverse(inverse_t *inv) { free(inv->off); free(inv->src); }

/* ---------- Hopcroft ---------- */
int oracle_hopcroft(uint32_t n, uint32_t k, const uint32_t *delta, const uint8_t *accept, uint32_t *block_out) {
  if (n == 0) return -1;
  inverse_t inv = {0, 0};
  int rc = build_inverse(n, k, delta, &inv);
  if (rc) { free_inverse(&inv); return rc; }

  uint32_t *elems = malloc((size_t)n * 4), *loc = malloc((size_t)n * 4), *blk = malloc((size_t)n * 4);
  uint32_t *first = malloc((size_t)n * 4), *end = malloc((size_t)n * 4), *mid = malloc((size_t)n * 4);
  uint32_t *touched = malloc((size_t)n * 4), *tmp = malloc((size_t)n * 4);
  uint8_t *inW = calloc((size_t)n * (k ? k : 1), 1);
  size_t wcap = 1024, wlen = 0;
  uint64_t *W = malloc(wcap * sizeof(uint64_t));
  if (!elems || !loc || !blk || !first || !end || !mid || !touched || !tmp || !inW || !W) { rc = -2; goto done; }

  /* initial partition {F, Q\F}: accepting states first */
  uint32_t nf = 0;
  for (uint32_t q = 0; q < n; ++q) if (accept[q]) elems[nf++] = q;
  uint32_t pos = nf;
  for (uint32_t q = 0; q < n; ++q) if (!accept[q]) elems[pos++] = q;
  uint32_t nb = 0;
  if (nf > 0) { first[nb] = 0; end[nb] = nf; mid[nb] = 0; nb++; }
  if (nf < n) { first[nb] = nf; end[nb] = n; mid[nb] = nf; nb++; }
  for (uint32_t b = 0; b < nb; ++b)
    for (uint32_t i = first[b]; i < end[b]; ++i) { blk[elems[i]] = b; loc[elems[i]] = i; }
  if (nb == 2) {
    uint32_t smaller = (end[0] - first[0] <= end[1] - first[1]) ? 0 : 1;
    for (uint32_t a = 0; a < k; ++a) { W[wlen++] = ((uint64_t)smaller << 32) | a; inW[(size_t)smaller * k + a] = 1; }
  }

  while (wlen > 0) {
    uint64_t w = W[--wlen];
    uint32_t A = (uint32_t)(w >> 32), a = (uint32_t)w;
    inW[(size_t)A * k + a] = 0;
    /* copy the splitter block: marking below may permute its elements */
    uint32_t na = end[A] - first[A];
    memcpy(tmp, elems + first[A], (size_t)na * 4);
    uint32_t ntouched = 0;
    const uint64_t *o = inv.off + (size_t)a * (n + 1);
    const uint32_t *src = inv.src + (size_t)a * n;
    for (uint32_t t = 0; t < na; ++t) {
      uint32_t s = tmp[t];
      for (uint64_t e = o[s]; e < o[s + 1]; ++e) {
        uint32_t p = src[e], b = blk[p], i = loc[p];
        if (i >= mid[b]) {           /* not yet marked: move to the marked prefix */
          if (mid[b] == first[b]) touched[ntouched++] = b;
          uint32_t j = mid[b], other = elems[j];
          elems[j] = p; loc[p] = j; elems[i] = other; loc[other] = i;
          mid[b]++;
        }
      }
    }
    for (uint32_t t = 0; t < ntouched; ++t) {
      uint32_t b = touched[t];
      if (mid[b] == end[b]) { mid[b] = first[b]; continue; }   /* every state marked: no split */
      uint32_t marked = mid[b] - first[b], unmarked = end[b] - mid[b];
      uint32_t nbk = nb++;
      if (marked <= unmarked) {          /* the new block takes the marked (smaller) part */
        first[nbk] = first[b]; end[nbk] = mid[b];
        first[b] = mid[b];
      } else {                           /* the new block takes the unmarked (smaller) part */
        first[nbk] = mid[b]; end[nbk] = end[b];
        end[b] = mid[b];
      }
      mid[b] = first[b]; mid[nbk] = first[nbk];
      for (uint32_t i = first[nbk]; i < end[nbk]; ++i) blk[elems[i]] = nbk;
      for (uint32_t c = 0; c < k; ++c) {
        uint32_t add;
        if (inW[(size_t)b * k + c]) add = nbk;
        else add = (end[nbk] - first[nbk] <= end[b] - first[b]) ? nbk : b;
        if (wlen == wcap) {
          wcap *= 2;
          uint64_t *W2 = realloc(W, wcap * sizeof(uint64_t));
          if (!W2) { rc = -2; goto done; }
          W = W2;
        }
        W[wlen++] = ((uint64_t)add << 32) | c;
        inW[(size_t)add * k + c] = 1;
      }
    }
  }
  for (uint32_t q = 0; q < n; ++q) block_out[q] = blk[q];
  rc = 0;
done:
  free(elems); free(loc); free(blk); free(first); free(end); free(mid); free(touched); free(tmp); free(inW); free(W);
  free_inverse(&inv);
  return rc;
}

/* ---------- Hopcroft-Karp with union-find (Algorithm 6) ---------- */
static uint32_t uf_find(uint32_t *parent, uint32_t x) {
  uint32_t r = x;
  while (parent[r] != r) r = parent[r];
  while (parent[x] != r) { uint32_t nx = parent[x]; parent[x] = r; x = nx; }
  return r;
}

int oracle_hk_equivalent(uint32_t nA, uint32_t k, const uint32_t *dA, const uint8_t *accA, uint32_t sA,
                         uint32_t nB, const uint32_t *dB, const uint8_t *accB, uint32_t sB) {
  if (nA == 0 || nB == 0 || sA >= nA || sB >= nB) return -1;
  uint32_t N = nA + nB;
  uint32_t *parent = malloc((size_t)N * 4);
  uint8_t *rank = calloc(N, 1);
  size_t cap = 1024, len = 0;
  uint64_t *S = malloc(cap * 8);
  int result = -2;
  if (!parent || !rank || !S) goto out;
  for (uint32_t i = 0; i < N; ++i) parent[i] = i;
  S[len++] = ((uint64_t)sA << 32) | sB;
  result = 1;
  while (len > 0) {
    uint64_t pr = S[--len];
    uint32_t p = (uint32_t)(pr >> 32), q = (uint32_t)pr;
    uint32_t rp = uf_find(parent, p), rq = uf_find(parent, nA + q);
    if (rp == rq) continue;                          /* already related by R+ */
    if ((accA[p] != 0) != (accB[q] != 0)) { result = 0; break; }
    for (uint32_t a = 0; a < k; ++a) {
      uint32_t p2 = dA[(size_t)a * nA + p], q2 = dB[(size_t)a * nB + q];
      if (p2 >= nA || q2 >= nB) { result = -1; goto out; }
      if (len == cap) {
        cap *= 2;
        uint64_t *S2 = realloc(S, cap * 8);
        if (!S2) { result = -2; goto out; }
        S = S2;
      }
      S[len++] = ((uint64_t)p2 << 32) | q2;
    }
    /* R := R ∪ {(p, q)}: union by rank */
    if (rank[rp] < rank[rq]) parent[rp] = rq;
    else if (rank[rp] > rank[rq]) parent[rq] = rp;
    else { parent[rq] = rp; rank[rp]++; }
  }
out:
  free(parent); free(rank); free(S);
  return result;
}

/* ---------- breadth-first product exploration: shortest distinguishing word ---------- */
static uint64_t mixkey(uint64_t x) {
  x ^= x >> 33; x *= 0xff51afd7ed558ccdULL; x ^= x >> 33; x *= 0xc4ceb9fe1a85ec53ULL; x ^= x >> 33;
  return x;
}

/* Returns the length of a shortest word w with δA*(sA,w) ∈ FA xor δB*(sB,w) ∈ FB,
 * or -1 when no such word exists (the DFAs are equivalent), or < -1 on error. */
int64_t oracle_shortest_cex(uint32_t nA, uint32_t k, const uint32_t *dA, const uint8_t *accA, uint32_t sA,
                            uint32_t nB, const uint32_t *dB, const uint8_t *accB, uint32_t sB) {
  if (nA == 0 || nB == 0 || sA >= nA || sB >= nB) return -2;
  size_t cap = 1024;
  while (cap < 4 * (size_t)(nA + nB)) cap <<= 1;
  uint64_t *table = malloc(cap * 8);
  size_t qcap = 1024, qhead = 0, qtail = 0, used = 0;
  uint64_t *queue = malloc(qcap * 8);
  int64_t result = -3;
  if (!table || !queue) goto out;
  memset(table, 0xff, cap * 8);
  const uint64_t EMPTY = ~0ULL;
#define INSERT(KEY, NEW)                                                   \
  do {                                                                     \
    uint64_t key_ = (KEY); size_t h_ = mixkey(key_) & (cap - 1);           \
    NEW = 0;                                                               \
    while (table[h_] != EMPTY && table[h_] != key_) h_ = (h_ + 1) & (cap - 1); \
    if (table[h_] == EMPTY) { table[h_] = key_; used++; NEW = 1; }         \
  } while (0)
  int isnew;
  INSERT(((uint64_t)sA << 32) | sB, isnew);
  queue[qtail++] = ((uint64_t)sA << 32) | sB;
  int64_t depth = 0;
  /* level-synchronous BFS: check a whole level, then expand it */
  result = -1;
  while (qhead < qtail) {
    size_t level_end = qtail;
    for (size_t i = qhead; i < level_end; ++i) {
      uint64_t pr = queue[i];
      uint32_t p = (uint32_t)(pr >> 32), q = (uint32_t)pr;
      if ((accA[p] != 0) != (accB[q] != 0)) { result = depth; goto out; }
    }
    for (size_t i = qhead; i < level_end; ++i) {
      uint64_t pr = queue[i];
      uint32_t p = (uint32_t)(pr >> 32), q = (uint32_t)pr;
      for (uint32_t a = 0; a < k; ++a) {
        uint32_t p2 = dA[(size_t)a * nA + p], q2 = dB[(size_t)a * nB + q];
        if (p2 >= nA || q2 >= nB) { result = -2; goto out; }
        uint64_t key = ((uint64_t)p2 << 32) | q2;
        if (2 * (used + 1) > cap) {            /* grow and rehash */
          size_t ncap = cap * 2;
          uint64_t *nt = malloc(ncap * 8);
          if (!nt) { result = -3; goto out; }
          memset(nt, 0xff, ncap * 8);
          for (size_t j = 0; j < cap; ++j) if (table[j] != EMPTY) {
            size_t h = mixkey(table[j]) & (ncap - 1);
            while (nt[h] != EMPTY) h = (h + 1) & (ncap - 1);
            nt[h] = table[j];
          }
          free(table); table = nt; cap = ncap;
        }
        INSERT(key, isnew);
        if (isnew) {
          if (qtail == qcap) {
            qcap *= 2;
            uint64_t *q2p = realloc(queue, qcap * 8);
            if (!q2p) { result = -3; goto out; }
            queue = q2p;
          }
          queue[qtail++] = key;
        }
      }
    }
    qhead = level_end;
    depth++;
  }
#undef INSERT
out:
  free(table); free(queue);
  return result;
}

/* ---------- pair table (Section 3.1 characterisation), tiny n ---------- */
int oracle_pair_table(uint32_t n, uint32_t k, const uint32_t *delta, const uint8_t *accept, uint32_t *block_out) {
  if (n == 0 || n > 4096) return -1;
  inverse_t inv = {0, 0};
  int rc = build_inverse(n, k, delta, &inv);
  if (rc) { free_inverse(&inv); return rc; }
  uint8_t *apart = calloc((size_t)n * n, 1);
  uint32_t *queue = malloc((size_t)n * n * 2 * sizeof(uint32_t));
  if (!apart || !queue) { rc = -2; goto done; }
  size_t qh = 0, qt = 0;
  for (uint32_t p = 0; p < n; ++p)
    for (uint32_t q = 0; q < n; ++q)
      if ((accept[p] != 0) != (accept[q] != 0)) {
        apart[(size_t)p * n + q] = 1;
        queue[2 * qt] = p; queue[2 * qt + 1] = q; qt++;
      }
  /* (p, q) -> (δ(p,a), δ(q,a)) is an edge of the pair graph; walk edges backwards */
  while (qh < qt) {
    uint32_t p2 = queue[2 * qh], q2 = queue[2 * qh + 1]; qh++;
    for (uint32_t a = 0; a < k; ++a) {
      const uint64_t *o = inv.off + (size_t)a * (n + 1);
      const uint32_t *src = inv.src + (size_t)a * n;
      for (uint64_t e = o[p2]; e < o[p2 + 1]; ++e)
        for (uint64_t f = o[q2]; f < o[q2 + 1]; ++f) {
          uint32_t p = src[e], q = src[f];
          if (!apart[(size_t)p * n + q]) {
            apart[(size_t)p * n + q] = 1;
            queue[2 * qt] = p; queue[2 * qt + 1] = q; qt++;
          }
        }
    }
  }
  for (uint32_t q = 0; q < n; ++q) {
    uint32_t p = 0;
    while (apart[(size_t)p * n + q]) p++;     /* smallest state not apart from q (q itself at worst) */
    block_out[q] = p;
  }
  rc = 0;
done:
  free(apart); free(queue); free_inverse(&inv);
  return rc;
}
