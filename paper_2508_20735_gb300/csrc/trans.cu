// dfa_trans: Algorithm 1 (trans, Section 3.1), the transitive closure of the
// pair graph, for small DFAs.
//
// The graph has one node per state pair s = q*n + q' (V = n^2 nodes) and an edge
// (q, q') -> (δ(q,a), δ(q',a)) per letter.  Reach is a dense V x V boolean
// matrix, bit-packed along rows (32 nodes per word); Apart is a V-bit vector.
// One iteration of the algorithm's loop is two launches:
//   trans_square_kernel  C = R | (R (x) R) over the boolean semiring, and
//   trans_label_kernel   Apart'[s] = Apart[s] | OR_t (C[s][t] & Apart[t]),
// each reading only the previous values (the synchronous reading of the
// parallel steps), and the loop stops after an iteration that labels nothing.
//
// The product is a dense contraction, but over (OR, AND) on bits: one 32-bit
// LOP3 performs 32 boolean multiply-adds, so the packed product on the integer
// pipe reaches about half the dense bf16 tensor-core multiply-add rate while
// keeping Reach at one bit per entry, needing no threshold between squarings,
// and skipping 32-column slabs that are zero in all of a tile's rows.
#include "api_util.h"

namespace dfa {

static constexpr int kSqThreads = 128;   // 8 row groups x 16 word groups
static constexpr int kSqRows = 64;       // rows of C per block (8 per thread)
static constexpr int kSqWords = 128;     // words of C per block (8 per thread)
static constexpr int kTransMaxIter = 40;

struct TransCtrl {
  uint32_t err;                    // bit 0: a transition target >= n
  uint32_t grew[kTransMaxIter + 1];  // pairs newly labelled Apart in iteration i
};

// Reach from the transitions, Apart from the acceptance bits.  R must be zero.
// Rows are stride `W` words; apart gets every one of the Vp/32 = W words.
__global__ void trans_init_kernel(const uint32_t *__restrict__ delta, const uint8_t *__restrict__ accept, uint32_t n,
                                  uint32_t k, uint32_t *__restrict__ R, uint32_t W, uint32_t *__restrict__ apart,
                                  TransCtrl *ctrl) {
  const uint32_t V = n * n, Vp = 32u * W;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t s0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); s0 < Vp; s0 += stride) {
    const uint32_t s = s0 + lane;
    bool ap = false;
    if (s < V) {
      const uint32_t q = s / n, qp = s - q * n;
      ap = (accept[q] != 0) != (accept[qp] != 0);
      for (uint32_t a = 0; a < k; ++a) {
        const uint32_t p = delta[(size_t)a * n + q], pp = delta[(size_t)a * n + qp];
        if (p >= n || pp >= n) {
          atomicOr(&ctrl->err, 1u);
          continue;
        }
        const uint32_t t = p * n + pp;
        atomicOr(&R[(size_t)s * W + (t >> 5)], 1u << (t & 31u));
      }
    }
    const uint32_t bits = __ballot_sync(0xffffffffu, ap);
    if (lane == 0) apart[s0 >> 5] = bits;
  }
}

// C = R | (R (x) R).  Block (bx, by) computes rows [64 by, 64 by + 64) and
// words [128 bx, 128 bx + 128) of C; thread (ty, tx) holds rows 8 ty .. 8 ty + 7
// and words 4 tx .. 4 tx + 3 and 64 + 4 tx .. 64 + 4 tx + 3 of that tile, so
// the shared-memory loads of a warp are contiguous.  The contraction index t
// runs one word (32 nodes) at a time: the tile's 64 row words of R at column
// word tw, expanded once into 32 x 64 all-ones/all-zeros row masks, and rows
// 32 tw .. 32 tw + 31 of R restricted to the tile's words, all in shared
// memory, so the inner step is one LOP3 per accumulator word.
// A column word that is zero in all 64 rows is skipped (R starts with k bits a
// row).  W is a multiple of 8 and the matrix has 32 W rows, so every uint4 is
// either wholly inside the row or wholly past its end.
__global__ void __launch_bounds__(kSqThreads, 3) trans_square_kernel(const uint32_t *__restrict__ R,
                                                                  uint32_t *__restrict__ C, uint32_t W) {
  __shared__ uint4 bs[32][32];           // 32 rows t x 128 words
  __shared__ uint4 ms[32][kSqRows / 4];  // ms[b] word r: all ones iff bit b of row r's column word
  __shared__ uint32_t as[kSqRows];       // the tile's rows, one column word
  const uint32_t tx = threadIdx.x & 15u, ty = threadIdx.x >> 4;
  const uint32_t row0 = blockIdx.y * kSqRows, w0 = blockIdx.x * kSqWords;
  uint32_t acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0;

  for (uint32_t tw = 0; tw < W; ++tw) {
    uint32_t mine = 0;
    if (threadIdx.x < kSqRows) {
      mine = R[(size_t)(row0 + threadIdx.x) * W + tw];
      as[threadIdx.x] = mine;
    }
    if (!__syncthreads_or(mine != 0)) continue;
    {   // row masks, computed once per column word instead of once per thread
      const uint32_t row = threadIdx.x & (kSqRows - 1), b0 = (threadIdx.x / kSqRows) * 16;
      const uint32_t w = as[row];
      uint32_t *mrow = reinterpret_cast<uint32_t *>(ms);
#pragma unroll
      for (uint32_t b = 0; b < 16; ++b) mrow[(b0 + b) * kSqRows + row] = 0u - ((w >> (b0 + b)) & 1u);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint32_t u = threadIdx.x + r * kSqThreads;   // uint4 index in the 32 x 32 tile
      const uint32_t j = u >> 5, c4 = u & 31u;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (w0 + 4 * c4 < W) v = *reinterpret_cast<const uint4 *>(&R[(size_t)(tw * 32 + j) * W + w0 + 4 * c4]);
      bs[j][c4] = v;
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 32; ++b) {
      const uint4 b0 = bs[b][tx], b1 = bs[b][16 + tx];
      const uint4 m0 = ms[b][2 * ty], m1 = ms[b][2 * ty + 1];
      const uint32_t mk[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const uint32_t m = mk[i];
        acc[i][0] |= m & b0.x;
        acc[i][1] |= m & b0.y;
        acc[i][2] |= m & b0.z;
        acc[i][3] |= m & b0.w;
        acc[i][4] |= m & b1.x;
        acc[i][5] |= m & b1.y;
        acc[i][6] |= m & b1.z;
        acc[i][7] |= m & b1.w;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const size_t row = (size_t)(row0 + ty * 8 + i) * W;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t w = w0 + 64u * h + 4u * tx;
      if (w < W) {
        const uint4 r = *reinterpret_cast<const uint4 *>(&R[row + w]);
        uint4 o;
        o.x = r.x | acc[i][4 * h + 0];
        o.y = r.y | acc[i][4 * h + 1];
        o.z = r.z | acc[i][4 * h + 2];
        o.w = r.w | acc[i][4 * h + 3];
        *reinterpret_cast<uint4 *>(&C[row + w]) = o;
      }
    }
  }
}

// Apart' = Apart | (C . Apart): one warp per output word (32 rows).
__global__ void trans_label_kernel(const uint32_t *__restrict__ C, const uint32_t *__restrict__ apart,
                                   uint32_t *__restrict__ apart_out, uint32_t W, uint32_t *grew) {
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = gridDim.x * blockDim.x / 32;
  for (uint32_t g = (blockIdx.x * blockDim.x + threadIdx.x) / 32; g < W; g += warps) {
    uint32_t word = 0;
    for (uint32_t r = 0; r < 32; ++r) {
      const uint32_t *row = C + (size_t)(g * 32 + r) * W;
      uint32_t hit = 0;
      for (uint32_t w = lane; w < W; w += 32) hit |= row[w] & apart[w];
      if (__any_sync(0xffffffffu, hit != 0)) word |= 1u << r;
    }
    if (lane == 0) {
      const uint32_t old = apart[g], now = old | word;
      apart_out[g] = now;
      if (now != old) atomicAdd(grew, __popc(now & ~old));
    }
  }
}

// Canonical partition: q's representative is the smallest q' not Apart from
// q; blocks are numbered by their representatives in increasing order.
// One block; n <= DFA_TRANS_MAX_STATES <= blockDim.x.
__global__ void trans_output_kernel(const uint32_t *__restrict__ apart, uint32_t n, uint32_t *__restrict__ out) {
  __shared__ uint32_t rep[DFA_TRANS_MAX_STATES], rank[DFA_TRANS_MAX_STATES];
  const uint32_t q = threadIdx.x;
  if (q < n) {
    uint32_t r = q;   // q is never Apart from itself
    for (uint32_t p = 0; p < q; ++p) {
      const uint32_t s = q * n + p;
      if (!((apart[s >> 5] >> (s & 31u)) & 1u)) {
        r = p;
        break;
      }
    }
    rep[q] = r;
  }
  __syncthreads();
  if (q == 0) {
    uint32_t c = 0;
    for (uint32_t p = 0; p < n; ++p) rank[p] = rep[p] == p ? c++ : 0u;
  }
  __syncthreads();
  if (q < n) out[q] = rank[rep[q]];
}

struct TransLayout {
  uint32_t W;   // words per row (multiple of 8); the matrix has 32 W rows
  size_t r0, r1, ap0, ap1, ctrl, delta, accept, out, total;
};

static TransLayout trans_layout(uint32_t n, uint32_t k, bool hd, bool ha, bool ho) {
  TransLayout L{};
  const uint64_t V = (uint64_t)n * n;
  L.W = (uint32_t)(((V + 31) / 32 + 7) / 8 * 8);
  const size_t mat = (size_t)L.W * 32 * L.W * 4;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  L.r0 = take(mat);
  L.r1 = take(mat);
  L.ap0 = take((size_t)L.W * 4);
  L.ap1 = take((size_t)L.W * 4);
  L.ctrl = take(sizeof(TransCtrl));
  L.delta = hd ? take((size_t)k * n * 4) : SIZE_MAX;
  L.accept = ha ? take(n) : SIZE_MAX;
  L.out = ho ? take((size_t)n * 4) : SIZE_MAX;
  L.total = off;
  return L;
}

static int check_trans(const dfa_t *d) {
  const int rc = check_dfa(d, "dfa");
  if (rc != DFA_OK) return rc;
  if (d->n > DFA_TRANS_MAX_STATES)
    return fail(DFA_EINVAL, "trans: n = %u exceeds %u (Reach has n^4 bits)", d->n, DFA_TRANS_MAX_STATES);
  return DFA_OK;
}

}  // namespace dfa

using namespace dfa;

extern "C" {

size_t dfa_trans_workspace_size(const dfa_t *d, const uint32_t *block_out) {
  if (check_trans(d) != DFA_OK || !block_out) return 0;
  return trans_layout(d->n, d->k, d->k > 0 && !is_device_ptr(d->delta), !is_device_ptr(d->accept),
                      !is_device_ptr(block_out))
      .total;
}

int dfa_trans(const dfa_t *d, uint32_t *block_out, uint32_t *iterations, void *workspace, size_t ws_bytes,
              void *stream) {
  int rc = check_trans(d);
  if (rc != DFA_OK) return rc;
  if (!block_out || !iterations) return fail(DFA_EINVAL, "block_out or iterations is NULL");
  if (!workspace || !aligned(workspace, 256)) return fail(DFA_EINVAL, "workspace NULL or not 256-byte aligned");
  const uint32_t n = d->n, k = d->k;
  const bool hd = k > 0 && !is_device_ptr(d->delta), ha = !is_device_ptr(d->accept), ho = !is_device_ptr(block_out);
  const TransLayout L = trans_layout(n, k, hd, ha, ho);
  if (ws_bytes < L.total) return fail(DFA_EINVAL, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
  char *ws = static_cast<char *>(workspace);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uint32_t *delta = d->delta;
  const uint8_t *accept = d->accept;
  cudaError_t e = cudaSuccess;
  if (hd) {
    e = cudaMemcpyAsync(ws + L.delta, d->delta, (size_t)k * n * 4, cudaMemcpyHostToDevice, st);
    delta = reinterpret_cast<const uint32_t *>(ws + L.delta);
  }
  if (e == cudaSuccess && ha) {
    e = cudaMemcpyAsync(ws + L.accept, d->accept, n, cudaMemcpyHostToDevice, st);
    accept = reinterpret_cast<const uint8_t *>(ws + L.accept);
  }
  if (e != cudaSuccess) return cuda_fail(e, "copy inputs to device");
  const uint32_t W = L.W;
  uint32_t *R[2] = {reinterpret_cast<uint32_t *>(ws + L.r0), reinterpret_cast<uint32_t *>(ws + L.r1)};
  uint32_t *ap[2] = {reinterpret_cast<uint32_t *>(ws + L.ap0), reinterpret_cast<uint32_t *>(ws + L.ap1)};
  TransCtrl *ctrl = reinterpret_cast<TransCtrl *>(ws + L.ctrl);
  uint32_t *out = ho ? reinterpret_cast<uint32_t *>(ws + L.out) : block_out;
  const size_t mat = (size_t)W * 32 * W * 4;
  e = cudaMemsetAsync(R[0], 0, mat, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctrl, 0, sizeof(TransCtrl), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  const uint32_t rows = 32 * W;
  trans_init_kernel<<<(rows + 255) / 256, 256, 0, st>>>(delta, accept, n, k, R[0], W, ap[0], ctrl);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "trans_init_kernel launch");
  uint32_t err = 0;
  e = cudaMemcpyAsync(&err, &ctrl->err, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "trans init");
  if (err) return fail(DFA_EINVAL, "dfa: a transition target is >= n");
  const dim3 sq_grid((W + kSqWords - 1) / kSqWords, rows / kSqRows);
  const uint32_t label_blocks = (W * 32 + 255) / 256;
  uint32_t cur = 0, it = 0;
  for (;;) {
    if (it == kTransMaxIter) return fail(DFA_EMAXROUNDS, "trans: no fixpoint after %d iterations", kTransMaxIter);
    ++it;
    trans_square_kernel<<<sq_grid, kSqThreads, 0, st>>>(R[cur], R[cur ^ 1], W);
    trans_label_kernel<<<label_blocks < 1024 ? label_blocks : 1024, 256, 0, st>>>(R[cur ^ 1], ap[cur], ap[cur ^ 1], W,
                                                                                  &ctrl->grew[it]);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "trans iteration launch");
    uint32_t grew = 0;
    e = cudaMemcpyAsync(&grew, &ctrl->grew[it], 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "trans iteration");
    cur ^= 1;
    if (grew == 0) break;
  }
  trans_output_kernel<<<1, DFA_TRANS_MAX_STATES, 0, st>>>(ap[cur], n, out);
  e = cudaGetLastError();
  if (e == cudaSuccess && ho) e = cudaMemcpyAsync(block_out, out, (size_t)n * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "trans output");
  *iterations = it;
  return DFA_OK;
}

}  // extern "C"
