// Per-query top-k selection (the paper's top-K phase, Sec. II.B.2: a
// selection per partition, a reduction, then a sort).  Here one CTA owns one
// query: every thread keeps the K best keys of its slice of the score row in
// registers (the per-partition selection), then the CTA merges the threads'
// sorted lists by k rounds of a block-wide maximum (reduction + sort).
//
// Order: score descending, then target id ascending -- packed into one
// 64-bit key (score with its sign bit flipped in the high word, the bitwise
// complement of the target id in the low word), so "larger key" = "better".
#include "dsa_internal.cuh"

namespace dsa {
namespace {

__device__ __forceinline__ uint64_t make_key(int32_t score, uint32_t tid) {
  return ((uint64_t)((uint32_t)score ^ 0x80000000u) << 32) | (uint64_t)(~tid);
}

template <int K, int TK_THREADS>
__global__ void __launch_bounds__(TK_THREADS) k_topk(const int32_t* __restrict__ score,
                                                     const int32_t* __restrict__ qend,
                                                     const int32_t* __restrict__ tend,
                                                     const uint8_t* __restrict__ flag,
                                                     uint32_t n_targets, uint32_t k,
                                                     dsa_hit* __restrict__ hits) {
  const uint32_t q = blockIdx.x;
  const int32_t* row = score + (uint64_t)q * n_targets;
  uint64_t L[K];
#pragma unroll
  for (int r = 0; r < K; ++r) L[r] = 0;   // 0 = empty (no real key is 0)
  for (uint32_t t = threadIdx.x; t < n_targets; t += TK_THREADS) {
    uint64_t x = make_key(row[t], t);
    if (x > L[K - 1]) {
#pragma unroll
      for (int r = 0; r < K; ++r) {
        if (x > L[r]) {
          const uint64_t tmp = L[r];
          L[r] = x;
          x = tmp;
        }
      }
    }
  }
  __shared__ uint64_t warp_best[TK_THREADS / 32];
  __shared__ uint64_t round_best;
  int pos = 0;
  const uint32_t kk = min(k, n_targets);
  for (uint32_t r = 0; r < kk; ++r) {
    uint64_t head = 0;
#pragma unroll
    for (int u = 0; u < K; ++u)
      if (u == pos) head = L[u];
    uint64_t m = head;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, m, off);
      m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0) warp_best[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint64_t v = threadIdx.x < TK_THREADS / 32 ? warp_best[threadIdx.x] : 0;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const uint64_t o = __shfl_xor_sync(0xFFFFFFFFu, v, off);
        v = o > v ? o : v;
      }
      if (threadIdx.x == 0) round_best = v;
    }
    __syncthreads();
    const uint64_t win = round_best;
    if (head == win && win != 0) {   // keys are unique: exactly one owner
      ++pos;
      const uint32_t t = ~(uint32_t)(win & 0xFFFFFFFFu);
      const uint64_t idx = (uint64_t)q * n_targets + t;
      dsa_hit h;
      h.score = (int32_t)((uint32_t)(win >> 32) ^ 0x80000000u);
      h.q_begin = -1; h.t_begin = -1;
      h.q_end = qend[idx]; h.t_end = tend[idx];
      h.query_id = q; h.target_id = t;
      h.flags = flag[idx] ? DSA_HIT_RERUN_INT32 : 0u;
      h.t_offset = 0; h.cigar_off = 0; h.cigar_len = 0; h.reserved = 0;
      hits[(uint64_t)q * kk + r] = h;
    }
    __syncthreads();
  }
}

__global__ void k_fill_hits(const int32_t* __restrict__ score, const int32_t* __restrict__ qend,
                            const int32_t* __restrict__ tend, const uint8_t* __restrict__ flag,
                            const dsa_pair* __restrict__ pairs, uint64_t n, uint32_t n_targets,
                            dsa_hit* __restrict__ hits) {
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    dsa_hit h;
    h.score = score[x]; h.q_end = qend[x]; h.t_end = tend[x];
    h.q_begin = -1; h.t_begin = -1;
    if (pairs) {
      const dsa_pair p = pairs[x];
      h.query_id = p.query_id; h.target_id = p.target_id; h.t_offset = p.t_offset;
    } else {
      h.query_id = (uint32_t)(x / n_targets); h.target_id = (uint32_t)(x % n_targets); h.t_offset = 0;
    }
    h.flags = flag[x] ? DSA_HIT_RERUN_INT32 : 0u;
    h.cigar_off = 0; h.cigar_len = 0; h.reserved = 0;
    hits[x] = h;
  }
}

}  // namespace

int launch_topk(dsa_ctx* ctx, const Scores& s, uint32_t n_queries, uint32_t n_targets, uint32_t k,
                dsa_hit* d_hits) {
  if (n_queries == 0 || k == 0) return DSA_OK;
  if (k <= 16) {
    k_topk<16, 512><<<n_queries, 512, 0, ctx->stream>>>(s.score, s.q_end, s.t_end, s.flag,
                                                          n_targets, k, d_hits);
  } else if (k <= 64) {
    k_topk<64, 128><<<n_queries, 128, 0, ctx->stream>>>(s.score, s.q_end, s.t_end, s.flag,
                                                          n_targets, k, d_hits);
  } else {
    set_error("top_k = %u is above the supported maximum of 64", k);
    return DSA_ERR_UNSUPPORTED;
  }
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_fill_hits(dsa_ctx* ctx, const Scores& s, const dsa_pair* d_pairs, uint64_t n,
                     uint32_t n_targets, dsa_hit* d_hits) {
  if (n == 0) return DSA_OK;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > (uint64_t)ctx->sm_count * 32) blocks = (uint64_t)ctx->sm_count * 32;
  k_fill_hits<<<(unsigned)blocks, 256, 0, ctx->stream>>>(s.score, s.q_end, s.t_end, s.flag,
                                                         d_pairs, n, n_targets, d_hits);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

}  // namespace dsa
