// dsa_score_pairs_noalloc: the exact int32 score pass over explicit pairs
// (the map phase's per-pair scores, Sec. II.B.1), for callers that cannot
// allocate device memory.
//
// Who needs it: code that must not call cudaMalloc or any allocating
// routine -- for example an embedding application that hands every byte of
// device memory to its own pool and forbids other allocations, a
// latency-critical serving thread that may not block on the device
// allocator, or a caller recording work while allocation is not permitted.
// Such callers pass every input and output as device memory they already
// own; the only other memory this path touches is the fixed scratch array
// below, which is part of the loaded library image.
//
// It computes the same scores and end cells as dsa_align on explicit pairs
// (one thread per pair, query strips of 8 rows in registers, target scanned
// column by column, the strip's last row handed to the next strip through a
// boundary row); the difference is where the boundary rows live and that
// the substitution matrix is read from shared memory instead of a profile.
#include "dsa_internal.cuh"

#include <algorithm>
#include <mutex>

namespace dsa {
namespace {

// Fixed scratch for the boundary rows of every call: 4 Mi int2 = 32 MiB.
// It exists once per device that loads the library and lives until exit.
constexpr uint64_t NOALLOC_SCRATCH_ELEMS = 4ull << 20;
constexpr uint32_t NOALLOC_MAX_T_LEN = 32768;   // 128 concurrent pairs at this length
constexpr int NOALLOC_STRIP = 8;
constexpr int NOALLOC_THREADS = 128;
static __device__ __align__(256) int2 g_noalloc_scratch[NOALLOC_SCRATCH_ELEMS];

__device__ __forceinline__ int32_t na_row0(int mode, uint32_t fe, int64_t j, int o, int e) {
  if (j == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_T_BEGIN))) return 0;
  return -(o + (int32_t)(j - 1) * e);
}
__device__ __forceinline__ int32_t na_col0(int mode, uint32_t fe, int64_t i, int o, int e) {
  if (i == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_Q_BEGIN))) return 0;
  return -(o + (int32_t)(i - 1) * e);
}

__global__ void __launch_bounds__(NOALLOC_THREADS) k_noalloc_pairs(
    const uint8_t* __restrict__ qcodes, const uint64_t* __restrict__ qoff, uint32_t nq,
    const uint8_t* __restrict__ tcodes, const uint64_t* __restrict__ toff, uint32_t nt,
    const dsa_pair* __restrict__ pairs, uint64_t n_pairs, int mode, uint32_t fe,
    const int8_t* __restrict__ Sg, int A, int o, int e, uint32_t slice, int64_t bound,
    int2* __restrict__ scratch, int32_t* __restrict__ o_score, int32_t* __restrict__ o_qend,
    int32_t* __restrict__ o_tend) {
  __shared__ int8_t S[32 * 32];
  for (int x = threadIdx.x; x < A * A; x += blockDim.x) S[x] = Sg[x];
  __syncthreads();
  const bool local = mode == DSA_LOCAL;
  const bool sg = mode == DSA_SEMIGLOBAL;
  const bool q_end_free = sg && (fe & DSA_FREE_Q_END);
  const bool t_end_free = sg && (fe & DSA_FREE_T_END);
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  int2* scr = scratch + tid * slice;   // this thread's boundary row
  for (uint64_t p = tid; p < n_pairs; p += (uint64_t)gridDim.x * blockDim.x) {
    const dsa_pair pr = pairs[p];
    // pairs that break a rule get score INT32_MIN and ends -2
    bool ok = pr.query_id < nq && pr.target_id < nt && pr.t_len >= 1 && pr.t_len <= slice;
    int32_t m = 0;
    if (ok) {
      m = (int32_t)(qoff[pr.query_id + 1] - qoff[pr.query_id]);
      const uint64_t tl = toff[pr.target_id + 1] - toff[pr.target_id];
      // window inside the target, tested without the sum t_offset + t_len (which
      // wraps for offsets near 2^64)
      ok = m >= 1 && pr.t_offset <= tl && pr.t_len <= tl - pr.t_offset &&
           ((int64_t)m + pr.t_len + 2) < bound;
    }
    if (ok) {   // every residue code must index the matrix
      const uint8_t* qq = qcodes + qoff[pr.query_id];
      const uint8_t* tt = tcodes + toff[pr.target_id] + pr.t_offset;
      for (int32_t i = 0; i < m && ok; ++i) ok = qq[i] < A;
      for (uint32_t j = 0; j < pr.t_len && ok; ++j) ok = tt[j] < A;
    }
    if (!ok) {
      o_score[p] = INT32_MIN; o_qend[p] = -2; o_tend[p] = -2;
      continue;
    }
    const int32_t n = (int32_t)pr.t_len;
    const uint8_t* q = qcodes + qoff[pr.query_id];
    const uint8_t* t = tcodes + toff[pr.target_id] + pr.t_offset;
    int32_t bs = 0, bi = -1, bj = -1;
    bool have = false;
    auto offer = [&](int32_t h, int32_t ii, int32_t jj) {
      if (!have || h > bs || (h == bs && (jj < bj || (jj == bj && ii < bi)))) {
        bs = h; bi = ii; bj = jj; have = true;
      }
    };
    if (q_end_free) offer(na_row0(mode, fe, n, o, e), 0, n);
    for (int32_t i0 = 0; i0 < m; i0 += NOALLOC_STRIP) {
      const int rows = min(NOALLOC_STRIP, m - i0);
      int32_t Hc[NOALLOC_STRIP], Ec[NOALLOC_STRIP];
      int qc[NOALLOC_STRIP];
#pragma unroll
      for (int r = 0; r < NOALLOC_STRIP; ++r) {
        Hc[r] = na_col0(mode, fe, i0 + r + 1, o, e);
        Ec[r] = NEG32;
        qc[r] = r < rows ? q[i0 + r] * A : 0;
      }
      if (t_end_free && i0 + rows == m) offer(Hc[rows - 1], m, 0);
      int32_t diag = na_col0(mode, fe, i0, o, e);
      for (int32_t j = 1; j <= n; ++j) {
        const int a = t[j - 1];
        int32_t Hup, Fup;
        if (i0 == 0) {
          Hup = na_row0(mode, fe, j, o, e);
          Fup = NEG32;
        } else {
          const int2 v = scr[j - 1];
          Hup = v.x;
          Fup = v.y;
        }
        int32_t d = diag;
        diag = Hup;
        int32_t F = Fup, Hprev = Hup;
#pragma unroll
        for (int r = 0; r < NOALLOC_STRIP; ++r) {
          if (r < rows) {
            F = max(F - e, Hprev - o);
            Ec[r] = max(Ec[r] - e, Hc[r] - o);
            int32_t h = max(d + S[qc[r] + a], max(Ec[r], F));
            if (local) h = max(h, 0);
            d = Hc[r];
            Hc[r] = h;
            Hprev = h;
            const int32_t i = i0 + r + 1;
            if (local) {
              if (h > 0) offer(h, i, j);
            } else {
              if (j == n && (q_end_free || i == m)) offer(h, i, j);
              if (t_end_free && i == m) offer(h, i, j);
            }
          }
        }
        scr[j - 1] = make_int2(Hprev, F);
      }
    }
    if (local && !have) {
      o_score[p] = 0; o_qend[p] = -1; o_tend[p] = -1;
    } else {
      o_score[p] = bs; o_qend[p] = bi - 1; o_tend[p] = bj - 1;
    }
  }
}

// Device address of g_noalloc_scratch per device, looked up once per device
// (with that device current) on the first call made on it.  The address
// belongs to the device's primary context: it does not survive a
// cudaDeviceReset of that device (the header says so).
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

}  // namespace
}  // namespace dsa

using namespace dsa;

extern "C" int dsa_score_pairs_noalloc(const uint8_t* d_q_codes, const uint64_t* d_q_offsets,
                                       uint32_t n_queries, const uint8_t* d_t_codes,
                                       const uint64_t* d_t_offsets, uint32_t n_targets,
                                       const dsa_pair* d_pairs, uint64_t n_pairs, int mode,
                                       uint32_t free_ends, const int8_t* d_matrix,
                                       int alphabet_size, int gap_open, int gap_extend,
                                       uint32_t max_t_len, int32_t* d_score, int32_t* d_q_end,
                                       int32_t* d_t_end, void* cuda_stream) {
  if (!d_q_codes || !d_q_offsets || !d_t_codes || !d_t_offsets || !d_pairs || !d_matrix ||
      !d_score || !d_q_end || !d_t_end) {
    set_error("dsa_score_pairs_noalloc: NULL pointer argument");
    return DSA_ERR_INVALID_ARG;
  }
  if (mode < DSA_LOCAL || mode > DSA_SEMIGLOBAL || free_ends > 15 || alphabet_size < 1 ||
      alphabet_size > MAX_ALPHABET || gap_extend < 0 || gap_extend > gap_open) {
    set_error("dsa_score_pairs_noalloc: bad mode, free_ends, alphabet_size or gap penalties");
    return DSA_ERR_INVALID_ARG;
  }
  if (max_t_len == 0 || max_t_len > NOALLOC_MAX_T_LEN) {
    set_error("dsa_score_pairs_noalloc: max_t_len %u outside 1..%u (the fixed scratch holds "
              "%llu boundary cells)", max_t_len, NOALLOC_MAX_T_LEN,
              (unsigned long long)NOALLOC_SCRATCH_ELEMS);
    return DSA_ERR_INVALID_ARG;
  }
  if (n_pairs == 0) return DSA_OK;
  int dev = 0;
  DSA_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) { set_error("device index %d unsupported", dev); return DSA_ERR_UNSUPPORTED; }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (err != cudaSuccess || !p) {
        set_error("cudaGetSymbolAddress(g_noalloc_scratch) failed: %s", cudaGetErrorString(err));
        return DSA_ERR_CUDA;
      }
      g_noalloc_ptr[dev] = p;
    }
    scratch = g_noalloc_ptr[dev];
  }
  // weight bound for int32 safety, as in dsa_align: (m + n) * max(|S|, o, e) < 2^29;
  // the matrix is on the device, so the bound uses the int8 range
  const int64_t w = std::max<int64_t>({128, gap_open, gap_extend});
  const int64_t bound = ((1ll << 29) / (w + 1));
  const uint32_t slice = max_t_len;
  const uint64_t max_threads = NOALLOC_SCRATCH_ELEMS / slice;
  uint64_t threads = std::min<uint64_t>(max_threads, n_pairs);
  uint64_t blocks = (threads + NOALLOC_THREADS - 1) / NOALLOC_THREADS;
  if (blocks * NOALLOC_THREADS > max_threads) blocks = max_threads / NOALLOC_THREADS;
  if (blocks == 0) blocks = 1;
  k_noalloc_pairs<<<(unsigned)blocks, NOALLOC_THREADS, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      d_q_codes, d_q_offsets, n_queries, d_t_codes, d_t_offsets, n_targets, d_pairs, n_pairs, mode,
      free_ends, d_matrix, alphabet_size, gap_open, gap_extend, slice, bound,
      static_cast<int2*>(scratch), d_score, d_q_end, d_t_end);
  DSA_CUDA_TRY(cudaGetLastError());
  return DSA_OK;
}
