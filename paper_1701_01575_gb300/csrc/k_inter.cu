// Inter-sequence local alignment kernel, packed int16x2 with DPX.
//
// Work decomposition (the paper's per-core SIMD alignment of one query against
// many references, Sec. II.B.1, re-laid out for a GB300 SM):
//   * the database is length-sorted and interleaved so that warp w of a CTA
//     owns 32 consecutive sorted targets, one per lane, and reads one 16-byte
//     word (16 residues) per lane per 16 columns, coalesced;
//   * two queries are packed into the two 16-bit halves of every DP register,
//     so one DPX instruction advances two cells;
//   * a query is processed in strips of 32 rows held in registers; the loop
//     runs over the target's residues; the strip's bottom row (H - o and the
//     next row's F) goes to a per-CTA boundary buffer and is read back by the
//     next strip;
//   * the query profile of each strip (R residue rows x 32 query rows of
//     int16x2 = R x 128 bytes) is staged into shared memory by TMA bulk copies,
//     double-buffered on two mbarriers, in 8 replicas whose start addresses
//     are rotated by 16 bytes so that the 8 lanes of each quarter-warp read
//     8 different bank groups whatever residues they hold;
//   * a persistent grid pops (query pair, block of 8 groups) items from a
//     work queue ordered longest-first.
//
// Cell update for one row (Gotoh, local), with Ho = H - o and profile S + o:
//   E  = max(E - e, Ho_left)            addmax2
//   t  = max(Ho_diag + (S + o), E)      addmax2
//   H  = max(t, F, 0)                   max2_relu
//   Ho = H - o                          add2
//   F' = max(F - e, Ho)                 addmax2   (F of the next row)
// and the column maximum of H (max3_2 every two rows) for the end cell.
//
// End cell (smallest target end j, then smallest query end i, among cells
// holding the best score): the column maximum is compared with the running
// best lowered by one while j is still below the best's column, so ties at an
// earlier column also trigger; the rare trigger scans the column for its
// first row.
//
// Saturation: in local mode no value falls below -(o + e), and a value can
// exceed the best seen so far by at most max(S), so if the best stays at or
// below 32767 - max(S) no lane wrapped.  Pairs above that are flagged for the
// exact int32 rerun.
#include "dsa_internal.cuh"
#include "dpx.cuh"

namespace dsa {
namespace {

constexpr int W = INTER_ROWS;    // query rows per strip
constexpr int NW = INTER_WARPS;  // warps per CTA
constexpr int NT = NW * 32;
constexpr int NCOPY = 8;         // profile replicas (one per lane of a quarter-warp)

struct InterArgs {
  const uint8_t* il;
  const uint64_t* gbase;
  const uint32_t* glen;
  const uint32_t* perm;
  uint32_t n_targets;
  uint32_t n_groups;
  const uint32_t* pprof;
  const uint64_t* pprof_off;
  const uint32_t* pair_q;
  const uint32_t* pair_ns;
  int R;
  uint32_t neg_o2, neg_e2;
  int o;
  int T;
  const uint32_t* items;
  uint32_t n_items;
  uint32_t* counter;
  uint2* scratch;
  uint64_t scratch_cols;
  int32_t* o_score;
  int32_t* o_qend;
  int32_t* o_tend;
  uint8_t* o_flag;
  uint32_t n_out_t;
  int32_t* status;
};

__device__ __forceinline__ void issue_strip(const InterArgs& A, uint8_t* buf, uint64_t* bar,
                                            const uint32_t* src, uint32_t cstride) {
  const uint32_t bytes = (uint32_t)A.R * 128u;
  mbar_arrive_expect_tx(bar, bytes * NCOPY);
#pragma unroll
  for (int c = 0; c < NCOPY; ++c) bulk_g2s(buf + c * cstride, src, bytes, bar);
}

__global__ void __launch_bounds__(NT, 2) k_inter_local16(const InterArgs A) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bars[2];
  __shared__ uint32_t s_item;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const uint32_t cstride = (uint32_t)A.R * 128u + 16u;
  const uint32_t bufbytes = NCOPY * cstride;
  const uint32_t strip_words = (uint32_t)A.R * 32u;
  const uint32_t neg_o2 = A.neg_o2, neg_e2 = A.neg_e2;
  const uint32_t NEG2 = pack2(NEG16, NEG16);

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t phase0 = 0, phase1 = 0;
  uint2* const scr_base = A.scratch + (uint64_t)blockIdx.x * A.scratch_cols * NT + tid;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(A.counter, 1u);
    __syncthreads();
    const uint32_t item = s_item;
    __syncthreads();
    if (item >= A.n_items) break;
    const uint32_t p = A.items[2 * item];
    const uint32_t g0 = A.items[2 * item + 1];
    const uint32_t ns = A.pair_ns[p];
    const uint32_t* psrc = A.pprof + A.pprof_off[p];
    if (tid == 0) {
      issue_strip(A, smem, &bars[0], psrc, cstride);
      if (ns > 1) issue_strip(A, smem + bufbytes, &bars[1], psrc + strip_words, cstride);
    }
    const uint32_t g = g0 + warp;
    const bool gvalid = g < A.n_groups;
    const uint32_t nlen = gvalid ? A.glen[g] : 0u;
    const uint32_t ncol = (nlen + 3u) & ~3u;
    const uint32_t st = g * 32u + lane;
    const bool tvalid = gvalid && st < A.n_targets;
    const uint4* res = reinterpret_cast<const uint4*>(A.il + (gvalid ? A.gbase[g] : 0)) + lane;

    int best_lo = 0, best_hi = 0, bj_lo = 0, bj_hi = 0, bi_lo = 0, bi_hi = 0;

    for (uint32_t s = 0; s < ns; ++s) {
      const int b = s & 1;
      const uint32_t par = b ? (phase1 & 1u) : (phase0 & 1u);
      const bool ok = mbar_wait_bounded(&bars[b], par, WAIT_LIMIT_NS);
      if (b) ++phase1; else ++phase0;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(A.status, DSA_ERR_DEVICE_TIMEOUT);
        // let any copy still in flight land before the CTA's shared memory is released
        mbar_wait_bounded(&bars[0], phase0 & 1u, WAIT_LIMIT_NS);
        mbar_wait_bounded(&bars[1], phase1 & 1u, WAIT_LIMIT_NS);
        return;
      }
      const uint8_t* pbuf = smem + b * bufbytes + (lane & 7) * cstride;
      const int i0 = (int)s * W;
      const bool first = s == 0;

      uint32_t Ho[W], E[W];
#pragma unroll
      for (int r = 0; r < W; ++r) {
        Ho[r] = neg_o2;
        E[r] = NEG2;
      }
      uint32_t diag = neg_o2;
      uint2* scr = scr_base;
      uint4 rv = make_uint4(0, 0, 0, 0);

      for (uint32_t c4 = 0; c4 < ncol; c4 += 4) {
        if ((c4 & 15u) == 0) rv = __ldg(res + (c4 >> 4) * 32u);
        const uint32_t sel = (c4 >> 2) & 3u;
        const uint32_t word = sel == 0 ? rv.x : sel == 1 ? rv.y : sel == 2 ? rv.z : rv.w;
        uint2 top[4];
        if (!first) {
#pragma unroll
          for (int k = 0; k < 4; ++k) top[k] = scr[(uint64_t)(c4 + k) * NT];
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) top[k] = make_uint2(neg_o2, neg_o2);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t a = (word >> (8 * k)) & 0xFFu;
          const uint4* prow = reinterpret_cast<const uint4*>(pbuf + a * 128u);
          uint32_t F = top[k].y;
          uint32_t d = diag;
          diag = top[k].x;
          uint32_t cm = 0, hprev = 0;
#pragma unroll
          for (int q4 = 0; q4 < W / 4; ++q4) {
            const uint4 pv = prow[q4];
            const uint32_t pr[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = q4 * 4 + u;
              const uint32_t old = Ho[r];
              E[r] = addmax2(E[r], neg_e2, old);
              const uint32_t t = addmax2(d, pr[u], E[r]);
              const uint32_t h = max2_relu(t, F);
              Ho[r] = add2(h, neg_o2);
              F = addmax2(F, neg_e2, Ho[r]);
              d = old;
              if (r & 1) cm = max3_2(cm, hprev, h);
              else hprev = h;
            }
          }
          scr[(uint64_t)(c4 + k) * NT] = make_uint2(Ho[W - 1], F);
          // end-cell tracking for column j
          const int j = (int)c4 + k + 1;
          const int cl = lo16(cm), ch = hi16(cm);
          const int thr_lo = best_lo - (j < bj_lo ? 1 : 0);
          const int thr_hi = best_hi - (j < bj_hi ? 1 : 0);
          if (cl > thr_lo || ch > thr_hi) {
            if (cl > thr_lo) {
              const int want = cl - A.o;
              int rr = 0;
#pragma unroll
              for (int r = W - 1; r >= 0; --r)
                if (lo16(Ho[r]) == want) rr = r;
              best_lo = cl; bj_lo = j; bi_lo = i0 + rr + 1;
            }
            if (ch > thr_hi) {
              const int want = ch - A.o;
              int rr = 0;
#pragma unroll
              for (int r = W - 1; r >= 0; --r)
                if (hi16(Ho[r]) == want) rr = r;
              best_hi = ch; bj_hi = j; bi_hi = i0 + rr + 1;
            }
          }
        }
      }
      __syncthreads();
      if (tid == 0 && s + 2 < ns) {
        fence_proxy_async_smem();
        issue_strip(A, smem + b * bufbytes, &bars[b], psrc + (s + 2) * strip_words, cstride);
      }
    }

    if (tvalid) {
      const uint32_t orig = A.perm[st];
      const uint32_t qa = A.pair_q[2 * p], qb = A.pair_q[2 * p + 1];
      if (qa != 0xFFFFFFFFu) {
        const uint64_t idx = (uint64_t)qa * A.n_out_t + orig;
        A.o_score[idx] = best_lo;
        A.o_qend[idx] = best_lo > 0 ? bi_lo - 1 : -1;
        A.o_tend[idx] = best_lo > 0 ? bj_lo - 1 : -1;
        A.o_flag[idx] = best_lo > A.T ? 1 : 0;
      }
      if (qb != 0xFFFFFFFFu) {
        const uint64_t idx = (uint64_t)qb * A.n_out_t + orig;
        A.o_score[idx] = best_hi;
        A.o_qend[idx] = best_hi > 0 ? bi_hi - 1 : -1;
        A.o_tend[idx] = best_hi > 0 ? bj_hi - 1 : -1;
        A.o_flag[idx] = best_hi > A.T ? 1 : 0;
      }
    }
  }
}

// Packed profile of query pair p: [strip][residue a][row r] int16x2 =
// (S[qa_i][a] + o, S[qb_i][a] + o) with i = 32*strip + r; padding rows and the
// padding residue a = A get NEG16.
__global__ void k_pair_profile(const uint8_t* __restrict__ qcodes,
                               const uint64_t* __restrict__ qoff, const uint32_t* __restrict__ qlen,
                               const uint32_t* __restrict__ pair_q,
                               const uint32_t* __restrict__ pair_ns,
                               const uint64_t* __restrict__ pprof_off, const int8_t* __restrict__ S,
                               int A, int R, int o, uint32_t* __restrict__ pprof) {
  const uint32_t p = blockIdx.y;
  const uint32_t qa = pair_q[2 * p], qb = pair_q[2 * p + 1];
  const uint32_t total = pair_ns[p] * (uint32_t)R * 32u;
  const int ma = qa != 0xFFFFFFFFu ? (int)qlen[qa] : 0;
  const int mb = qb != 0xFFFFFFFFu ? (int)qlen[qb] : 0;
  const uint8_t* qsa = ma ? qcodes + qoff[qa] : nullptr;
  const uint8_t* qsb = mb ? qcodes + qoff[qb] : nullptr;
  uint32_t* out = pprof + pprof_off[p];
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < total; x += gridDim.x * blockDim.x) {
    const uint32_t s = x / ((uint32_t)R * 32u);
    const int a = (int)((x / 32u) % (uint32_t)R);
    const int i = (int)(s * 32u + (x % 32u));
    const int lo = (a < A && i < ma) ? (int)S[qsa[i] * A + a] + o : NEG16;
    const int hi = (a < A && i < mb) ? (int)S[qsb[i] * A + a] + o : NEG16;
    out[x] = pack2(lo, hi);
  }
}

}  // namespace

int inter_blocks_per_sm() { return 2; }

int launch_pair_profile(dsa_ctx* ctx, const dsa_db* qs, const int8_t* d_matrix, int A, int o,
                        const InterPlan& plan) {
  if (plan.n_pairs == 0) return DSA_OK;
  dim3 grid(32, plan.n_pairs);
  k_pair_profile<<<grid, 256, 0, ctx->stream>>>(qs->d_codes, qs->d_off, qs->d_len, plan.d_pair_q,
                                                plan.d_pair_ns, plan.d_pprof_off, d_matrix, A,
                                                plan.R, o, plan.d_pprof);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_inter_local16(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const InterPlan& plan,
                         int o, int e, int smax, Scores out, uint32_t n_targets_out) {
  (void)qs;
  if (plan.n_items == 0) return DSA_OK;
  InterArgs A;
  A.il = db->d_il; A.gbase = db->d_gbase; A.glen = db->d_glen; A.perm = db->d_perm;
  A.n_targets = db->n; A.n_groups = db->n_groups;
  A.pprof = plan.d_pprof; A.pprof_off = plan.d_pprof_off; A.pair_q = plan.d_pair_q;
  A.pair_ns = plan.d_pair_ns; A.R = plan.R;
  A.neg_o2 = (uint32_t)((-o) & 0xFFFF) | ((uint32_t)((-o) & 0xFFFF) << 16);
  A.neg_e2 = (uint32_t)((-e) & 0xFFFF) | ((uint32_t)((-e) & 0xFFFF) << 16);
  A.o = o;
  A.T = 32767 - (smax > 0 ? smax : 0);
  A.items = plan.d_items; A.n_items = plan.n_items;
  A.counter = ctx->d_counters;
  const int grid = (int)std::min<uint64_t>(plan.n_items, (uint64_t)ctx->sm_count * inter_blocks_per_sm());
  const uint64_t cols = ((uint64_t)plan.max_glen + 3) & ~3ull;
  A.scratch_cols = cols;
  const size_t scr_bytes = (size_t)grid * cols * NT * sizeof(uint2);
  void* scr = nullptr;
  DSA_TRY(ctx->alloc(&scr, scr_bytes));
  A.scratch = static_cast<uint2*>(scr);
  A.o_score = out.score; A.o_qend = out.q_end; A.o_tend = out.t_end; A.o_flag = out.flag;
  A.n_out_t = n_targets_out;
  A.status = ctx->d_status;
  const size_t smem = 2ull * NCOPY * ((size_t)plan.R * 128 + 16);
  static bool attr_set = false;
  if (!attr_set) {
    DSA_CUDA_TRY(cudaFuncSetAttribute(k_inter_local16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      96 * 1024));
    attr_set = true;
  }
  DSA_CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, sizeof(uint32_t), ctx->stream));
  k_inter_local16<<<grid, NT, smem, ctx->stream>>>(A);
  ++ctx->launches;
  cudaError_t err = cudaGetLastError();
  ctx->release(scr, scr_bytes);
  if (err != cudaSuccess) {
    set_error("k_inter_local16 launch: %s", cudaGetErrorString(err));
    return DSA_ERR_CUDA;
  }
  return DSA_OK;
}

}  // namespace dsa
