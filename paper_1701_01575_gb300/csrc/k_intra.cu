// Intra-sequence local alignment kernel for long targets, packed int16x2 DPX
// (the local alignment of the map phase, Sec. II.B.1, for database targets
// too long for one thread).
//
// One warp aligns one long target against one packed query pair (the two
// 16-bit halves of every register hold two queries, as in the inter-sequence
// kernel).  The query rows are cut into bands of 32 x ROWS rows; in a band,
// lane k owns rows [band + ROWS*k, band + ROWS*(k+1)) in registers and
// processes target column j = step - k, so the warp sweeps an anti-diagonal
// wavefront: at every step lane k receives, by one warp shuffle each, the H-o
// and F of lane k-1's last row at its column and that column's residue.
// Lane 31 hands its last row to the next band through a boundary row in
// global memory; lane 0 of the next band reads it.  Persistent warps pop
// (target, query pair) items from a queue ordered longest-first.
//
// This splits one long alignment over 32 lanes, so a target of many thousand
// residues no longer keeps a single thread busy for the length of the whole
// search.  Cell update, end-cell rule and saturation test are those of the
// inter-sequence kernel; the per-lane bests are merged at the end under the
// same order (score desc, then smaller target end, then smaller query end).
#include "dsa_internal.cuh"
#include "dpx.cuh"

namespace dsa {
namespace {

constexpr int ROWS = 16;           // query rows per lane
constexpr int BAND = 32 * ROWS;    // rows per band
constexpr int WARPS = 4;           // warps per CTA

struct IntraArgs {
  const uint8_t* tcodes;
  const uint64_t* toff;
  const uint32_t* tlen;
  const uint32_t* long_ids;        // target ids of the long targets
    const uint32_t* prof;            // packed profiles, [strip][a][32 rows]
  const StripMeta* meta;
  const uint32_t* sbase;
  const uint32_t* nstrips;
  int R;
  uint32_t neg_o2, neg_e2;
  int o;
  int T;
  uint32_t* counter;
  const uint32_t* items;           // 2 words per item: long index, pair
  uint32_t n_items;
  uint2* scratch;                  // per warp slot: max_len boundary cells
  uint64_t scratch_cols;
  int32_t* o_score;
  int32_t* o_qend;
  int32_t* o_tend;
  uint8_t* o_flag;
  uint32_t n_out_t;
};

__device__ __forceinline__ void better(int& s, int& j, int& i, int s2, int j2, int i2) {
  if (s2 > s || (s2 == s && s2 > 0 && (j2 < j || (j2 == j && i2 < i)))) {
    s = s2; j = j2; i = i2;
  }
}

__global__ void __launch_bounds__(WARPS * 32) k_intra_local16(const IntraArgs A) {
  const int lane = threadIdx.x & 31;
  const uint32_t slot = blockIdx.x * WARPS + (threadIdx.x >> 5);
  uint2* const scr = A.scratch + (uint64_t)slot * A.scratch_cols;
  const uint32_t neg_o2 = A.neg_o2, neg_e2 = A.neg_e2;
  const uint32_t NEG2 = pack2(NEG16, NEG16);

  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(A.counter, 1u);
    item = __shfl_sync(0xFFFFFFFFu, item, 0);
    if (item >= A.n_items) break;
    const uint32_t li = A.items[2 * item], p = A.items[2 * item + 1];
    const uint32_t tid = A.long_ids[li];
    const int32_t n = (int32_t)A.tlen[tid];
    const uint8_t* t = A.tcodes + A.toff[tid];
    const uint32_t ns = A.nstrips[p];
    const int32_t mrows = (int32_t)ns * 32;
    const uint32_t* P = A.prof + (size_t)A.sbase[p] * A.R * 32;

    int best_lo = 0, best_hi = 0, bj_lo = 0, bj_hi = 0, bi_lo = 0, bi_hi = 0;

    for (int32_t b0 = 0; b0 < mrows; b0 += BAND) {
      const int32_t r0 = b0 + lane * ROWS;           // first row (0-based) of this lane
      const bool active = r0 < mrows;
      // profile rows of this lane: strip r0/32, half (r0/16)&1
      const uint32_t* prow = P + (size_t)(r0 >> 5) * A.R * 32 + (r0 & 16);
      uint32_t Ho[ROWS], E[ROWS];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        Ho[r] = neg_o2;
        E[r] = NEG2;
      }
      uint32_t diag = neg_o2;        // H - o of the row above at column j-1
      uint32_t sendHo = neg_o2, sendF = neg_o2;
      uint32_t sendA = 0;
      const int32_t steps = n + 31;
      for (int32_t s = 1; s <= steps; ++s) {
        const uint32_t upHo = __shfl_up_sync(0xFFFFFFFFu, sendHo, 1);
        const uint32_t upF = __shfl_up_sync(0xFFFFFFFFu, sendF, 1);
        const uint32_t upA = __shfl_up_sync(0xFFFFFFFFu, sendA, 1);
        const int32_t j = s - lane;
        if (j >= 1 && j <= n && active) {
          uint32_t topHo, F, a;
          if (lane == 0) {
            a = t[j - 1];
            if (b0 == 0) {
              topHo = neg_o2;
              F = neg_o2;
            } else {
              const uint2 v = scr[j - 1];
              topHo = v.x;
              F = v.y;
            }
          } else {
            topHo = upHo;
            F = upF;
            a = upA;
          }
          const uint4* pr4 = reinterpret_cast<const uint4*>(prow + a * 32u);
          uint32_t d = diag;
          diag = topHo;
          uint32_t cm = 0, hprev = 0;
#pragma unroll
          for (int q4 = 0; q4 < ROWS / 4; ++q4) {
            const uint4 pv = __ldg(pr4 + q4);
            const uint32_t pr[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = q4 * 4 + u;
              const uint32_t old = Ho[r];
              E[r] = addmax2(E[r], neg_e2, old);
              const uint32_t tt = addmax2(d, pr[u], E[r]);
              const uint32_t h = max2_relu(tt, F);
              Ho[r] = add2(h, neg_o2);
              F = addmax2(F, neg_e2, Ho[r]);
              d = old;
              if (r & 1) cm = max3_2(cm, hprev, h);
              else hprev = h;
            }
          }
          sendHo = Ho[ROWS - 1];
          sendF = F;
          sendA = a;
          if (lane == 31) scr[j - 1] = make_uint2(Ho[ROWS - 1], F);
          const int cl = lo16(cm), ch = hi16(cm);
          const int thr_lo = best_lo - (j < bj_lo ? 1 : 0);
          const int thr_hi = best_hi - (j < bj_hi ? 1 : 0);
          if (cl > thr_lo) {
            const int want = cl - A.o;
            int rr = 0;
#pragma unroll
            for (int r = ROWS - 1; r >= 0; --r)
              if (lo16(Ho[r]) == want) rr = r;
            best_lo = cl; bj_lo = j; bi_lo = r0 + rr + 1;
          }
          if (ch > thr_hi) {
            const int want = ch - A.o;
            int rr = 0;
#pragma unroll
            for (int r = ROWS - 1; r >= 0; --r)
              if (hi16(Ho[r]) == want) rr = r;
            best_hi = ch; bj_hi = j; bi_hi = r0 + rr + 1;
          }
        }
      }
      __syncwarp();
    }
    // merge the lanes' bests
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const int s2 = __shfl_xor_sync(0xFFFFFFFFu, best_lo, off);
      const int j2 = __shfl_xor_sync(0xFFFFFFFFu, bj_lo, off);
      const int i2 = __shfl_xor_sync(0xFFFFFFFFu, bi_lo, off);
      better(best_lo, bj_lo, bi_lo, s2, j2, i2);
      const int s3 = __shfl_xor_sync(0xFFFFFFFFu, best_hi, off);
      const int j3 = __shfl_xor_sync(0xFFFFFFFFu, bj_hi, off);
      const int i3 = __shfl_xor_sync(0xFFFFFFFFu, bi_hi, off);
      better(best_hi, bj_hi, bi_hi, s3, j3, i3);
    }
    if (lane == 0) {
      const StripMeta md = A.meta[A.sbase[p]];
      const uint32_t qa = md.qa, qb = md.qb;
      if (qa != 0xFFFFFFFFu) {
        const uint64_t idx = (uint64_t)qa * A.n_out_t + tid;
        A.o_score[idx] = best_lo;
        A.o_qend[idx] = best_lo > 0 ? bi_lo - 1 : -1;
        A.o_tend[idx] = best_lo > 0 ? bj_lo - 1 : -1;
        A.o_flag[idx] = best_lo > A.T ? 1 : 0;
      }
      if (qb != 0xFFFFFFFFu) {
        const uint64_t idx = (uint64_t)qb * A.n_out_t + tid;
        A.o_score[idx] = best_hi;
        A.o_qend[idx] = best_hi > 0 ? bi_hi - 1 : -1;
        A.o_tend[idx] = best_hi > 0 ? bj_hi - 1 : -1;
        A.o_flag[idx] = best_hi > A.T ? 1 : 0;
      }
    }
    __syncwarp();
  }
}

}  // namespace

int launch_intra_local16(dsa_ctx* ctx, cudaStream_t stream, const dsa_db* db,
                         const PackedPlan& plan, const IntraWork& work, int o, int e, int smax,
                         Scores out, uint32_t n_targets_out) {
  if (work.n_items == 0) return DSA_OK;
  IntraArgs A;
  A.tcodes = db->d_codes; A.toff = db->d_off; A.tlen = db->d_len;
  A.long_ids = work.d_long_ids;
  A.prof = plan.d_prof; A.meta = plan.d_meta; A.sbase = plan.d_sbase; A.nstrips = plan.d_ns;
  A.R = plan.R;
  A.neg_o2 = (uint32_t)((-o) & 0xFFFF) | ((uint32_t)((-o) & 0xFFFF) << 16);
  A.neg_e2 = (uint32_t)((-e) & 0xFFFF) | ((uint32_t)((-e) & 0xFFFF) << 16);
  A.o = o;
  A.T = 32767 - (smax > 0 ? smax : 0);
  A.counter = ctx->d_counters + 2;
  A.items = work.d_items;
  A.n_items = work.n_items;
  const uint64_t warps_total = std::min<uint64_t>(A.n_items, (uint64_t)ctx->sm_count * 16);
  const unsigned grid = (unsigned)((warps_total + WARPS - 1) / WARPS);
  A.scratch_cols = work.max_long_len;
  const size_t scr_bytes = (size_t)grid * WARPS * A.scratch_cols * sizeof(uint2);
  void* scr = nullptr;
  DSA_TRY(ctx->alloc(&scr, scr_bytes, stream));
  A.scratch = static_cast<uint2*>(scr);
  A.o_score = out.score; A.o_qend = out.q_end; A.o_tend = out.t_end; A.o_flag = out.flag;
  A.n_out_t = n_targets_out;
  DSA_CUDA_TRY(cudaMemsetAsync(A.counter, 0, sizeof(uint32_t), stream));
  k_intra_local16<<<grid, WARPS * 32, 0, stream>>>(A);
  ++ctx->launches;
  cudaError_t err = cudaGetLastError();
  ctx->release(scr, scr_bytes, stream);
  if (err != cudaSuccess) {
    set_error("k_intra_local16 launch: %s", cudaGetErrorString(err));
    return DSA_ERR_CUDA;
  }
  return DSA_OK;
}

}  // namespace dsa
