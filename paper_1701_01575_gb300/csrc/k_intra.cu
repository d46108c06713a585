// Intra-sequence alignment kernels for long targets, packed int16x2 DPX
// (the score pass of the map phase, Sec. II.B.1, for database targets too
// long for one thread): the local form, and below it the global /
// semi-global form on end-anchored strips.
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

// ---- global and semi-global form (Sec. II.C.2: DNW, DSG) ----
//
// The same wavefront for long targets in global and semi-global searches,
// with the end-anchored 32-row strips of the inter-sequence global kernel:
// a query of m rows starts (32 - m % 32) % 32 rows into its first strip, so
// row m is the last row (register 15) of one lane of one band, and each
// lane's 16 rows are, for each half, all at or above row m or all past it.
// Padding rows above a query reproduce row 0 (their S + o is 0 against the
// boundary -(o + (j-1)e), o against a free target begin), the real rows'
// column-0 values are set per lane, and lane 0 of the first band reads the
// row-0 boundary column by column.  Result cells: the lane holding row m
// keeps H[m][n] and, with a free target end, row m's best over j (smallest
// j); with a free query end every lane scans column n over its real rows
// (smallest i) and the warp reduces; candidates merge by (score desc, j asc,
// i asc).  Range: halves stay signed (halfword adds, no carry between
// them); pairs with 4o + (m + n + 2)e + |min S| + 64 >= 2^15 are flagged for
// the exact int32 rerun, and so is a pair whose column maximum of H over its
// real rows passes 32767 - max(S) (only the diagonal step raises a value).
struct IntraGlobArgs {
  int mode;
  uint32_t fe;
  int e;
  int smin;
  const uint32_t* qlen;
  uint32_t hmax2;   // 32767 - max(S) in both halves
};

template <bool TB, bool TE>
__global__ void __launch_bounds__(WARPS * 32) k_intra_glob16(const IntraArgs A, const IntraGlobArgs G) {
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const uint32_t slot = blockIdx.x * WARPS + (threadIdx.x >> 5);
  uint2* const scr = A.scratch + (uint64_t)slot * A.scratch_cols;
  const uint32_t neg_o2 = A.neg_o2, neg_e2 = A.neg_e2;
  const int o = A.o, e = G.e;
  const bool sg = G.mode == DSA_SEMIGLOBAL;
  const bool qb_free = sg && (G.fe & DSA_FREE_Q_BEGIN);
  const bool qe_free = sg && (G.fe & DSA_FREE_Q_END);
  const uint32_t NEGG2 = pack2(-32768 + e, -32768 + e);   // "-inf" whose - e does not wrap
  auto row0 = [&](int j) { return (j == 0 || TB) ? 0 : -(o + (j - 1) * e); };
  auto col0 = [&](int i) { return (i <= 0 || qb_free) ? 0 : -(o + (i - 1) * e); };

  for (;;) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(A.counter, 1u);
    item = __shfl_sync(FULL, item, 0);
    if (item >= A.n_items) break;
    const uint32_t li = A.items[2 * item], p = A.items[2 * item + 1];
    const uint32_t tid = A.long_ids[li];
    const int32_t n = (int32_t)A.tlen[tid];
    const uint8_t* t = A.tcodes + A.toff[tid];
    const uint32_t ns = A.nstrips[p];
    const int32_t mrows = (int32_t)ns * 32;
    const uint32_t* P = A.prof + (size_t)A.sbase[p] * A.R * 32;
    const StripMeta md = A.meta[A.sbase[p]];
    const int ma = md.qa != NONE ? (int)G.qlen[md.qa] : 0;
    const int mb = md.qb != NONE ? (int)G.qlen[md.qb] : 0;
    const int pa = (32 - ma % 32) % 32, pb = (32 - mb % 32) % 32;   // padding rows above
    const int gma = ma + pa - 1, gmb = mb + pb - 1;                 // row index of row m

    // per lane, over the bands: column n's best and its row (free query
    // end; from (0, n)), H[m][n] and row m's best (the lane holding row m),
    // the upward range bits
    int cb_lo = qe_free ? row0(n) : INT32_MIN, cb_hi = cb_lo, ci_lo = 0, ci_hi = 0;
    int hmn_lo = 0, hmn_hi = 0, rj_lo = 0, rj_hi = 0;
    uint32_t rthr = 0x7FFF7FFFu;   // row m's best H - o (a half not held: never passed)
    uint32_t sat = 0;

    for (int32_t b0 = 0; b0 < mrows; b0 += BAND) {
      const int32_t r0 = b0 + lane * ROWS;           // first row (0-based) of this lane
      const bool active = r0 < mrows;
      const uint32_t* prow = P + (size_t)(r0 >> 5) * A.R * 32 + (r0 & 16);
      const int ia = r0 - pa + 1, ib = r0 - pb + 1;  // 1-based query row of the lane's first row
      // halves whose query ended above this lane (a lane never holds both
      // sides of row m): left out of the range test and the result
      const uint32_t live = (ia > ma ? 0u : 0x0000FFFFu) | (ib > mb ? 0u : 0xFFFF0000u);
      const bool own_a = md.qa != NONE && r0 + ROWS - 1 == gma;
      const bool own_b = md.qb != NONE && r0 + ROWS - 1 == gmb;
      if (TE && own_a) rthr = (rthr & 0xFFFF0000u) | (pack2(col0(ma) - o, 0) & 0xFFFFu);
      if (TE && own_b) rthr = (rthr & 0x0000FFFFu) | (pack2(0, col0(mb) - o) & 0xFFFF0000u);
      uint32_t Ho[ROWS], E[ROWS];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        Ho[r] = pack2(col0(ia + r) - o, col0(ib + r) - o);
        E[r] = NEGG2;
      }
      uint32_t diag = pack2(col0(ia - 1) - o, col0(ib - 1) - o);   // H - o above-left
      uint32_t sendHo = neg_o2, sendF = neg_o2;
      uint32_t sendA = 0;
      const int32_t steps = n + 31;
      for (int32_t s = 1; s <= steps; ++s) {
        const uint32_t upHo = __shfl_up_sync(FULL, sendHo, 1);
        const uint32_t upF = __shfl_up_sync(FULL, sendF, 1);
        const uint32_t upA = __shfl_up_sync(FULL, sendA, 1);
        const int32_t j = s - lane;
        if (j >= 1 && j <= n && active) {
          uint32_t topHo, F, a;
          if (lane == 0) {
            a = t[j - 1];
            if (b0 == 0) {   // row 0: (B(j) - o, F of row 1 = B(j) - o)
              topHo = pack2(row0(j) - o, row0(j) - o);
              F = topHo;
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
          uint32_t cm = 0x80008000u, hprev = 0x80008000u;
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
              const uint32_t h = __vmaxs2(tt, F);
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
          // upward range test over the live halves (rare)
          const uint32_t cml = (cm & live) | (0x80008000u & ~live);
          if (__vmaxs2(cml, G.hmax2) != G.hmax2)
            sat |= (lo16(cml) > lo16(G.hmax2) ? 1u : 0u) | (hi16(cml) > hi16(G.hmax2) ? 2u : 0u);
          if (TE && (own_a || own_b)) {   // row m: strictly better, smallest j kept
            const uint32_t cur = Ho[ROWS - 1];
            if (__vmaxs2(cur, rthr) != rthr) {
              if (own_a && lo16(cur) > lo16(rthr)) { rthr = (rthr & 0xFFFF0000u) | (cur & 0xFFFFu); rj_lo = j; }
              if (own_b && hi16(cur) > hi16(rthr)) { rthr = (rthr & 0x0000FFFFu) | (cur & 0xFFFF0000u); rj_hi = j; }
            }
          }
          if (j == n) {   // column n
            if (own_a) hmn_lo = lo16(Ho[ROWS - 1]) + o;
            if (own_b) hmn_hi = hi16(Ho[ROWS - 1]) + o;
            if (qe_free) {
#pragma unroll
              for (int r = 0; r < ROWS; ++r) {
                const int va = lo16(Ho[r]) + o, vb = hi16(Ho[r]) + o;
                if (ia + r >= 1 && ia + r <= ma && va > cb_lo) { cb_lo = va; ci_lo = ia + r; }
                if (ib + r >= 1 && ib + r <= mb && vb > cb_hi) { cb_hi = vb; ci_hi = ib + r; }
              }
            }
          }
        }
      }
      __syncwarp();
    }
    // the lanes' column-n candidates (score desc, row asc), the held row's
    // values from its lane, the range bits of every lane
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const int s2 = __shfl_xor_sync(FULL, cb_lo, off), i2 = __shfl_xor_sync(FULL, ci_lo, off);
      if (s2 > cb_lo || (s2 == cb_lo && i2 < ci_lo)) { cb_lo = s2; ci_lo = i2; }
      const int s3 = __shfl_xor_sync(FULL, cb_hi, off), i3 = __shfl_xor_sync(FULL, ci_hi, off);
      if (s3 > cb_hi || (s3 == cb_hi && i3 < ci_hi)) { cb_hi = s3; ci_hi = i3; }
      sat |= __shfl_xor_sync(FULL, sat, off);
    }
    const int la = gma >= 0 ? (gma % BAND) / ROWS : 0, lb = gmb >= 0 ? (gmb % BAND) / ROWS : 0;
    const int hmn_a = __shfl_sync(FULL, hmn_lo, la), hmn_b = __shfl_sync(FULL, hmn_hi, lb);
    const uint32_t rt_a = __shfl_sync(FULL, rthr, la), rt_b = __shfl_sync(FULL, rthr, lb);
    const int rj_a = __shfl_sync(FULL, rj_lo, la), rj_b = __shfl_sync(FULL, rj_hi, lb);
    if (lane == 0) {
      auto finish = [&](uint32_t q, int m, int cb, int ci, int hmn, int rb, int rj, bool up) {
        int bs = qe_free ? cb : hmn, bi = qe_free ? ci : m, bj = n;   // column n, or (m, n)
        if (TE && (rb > bs || (rb == bs && rj < bj))) { bs = rb; bi = m; bj = rj; }
        const int64_t low = 4ll * o + (int64_t)(m + n + 2) * e + (G.smin < 0 ? -G.smin : 0) + 64;
        const uint64_t idx = (uint64_t)q * A.n_out_t + tid;
        A.o_score[idx] = bs;
        A.o_qend[idx] = bi - 1;
        A.o_tend[idx] = bj - 1;
        A.o_flag[idx] = (up || low >= 32768) ? 1 : 0;
      };
      if (md.qa != NONE) finish(md.qa, ma, cb_lo, ci_lo, hmn_a, lo16(rt_a) + o, rj_a, sat & 1u);
      if (md.qb != NONE) finish(md.qb, mb, cb_hi, ci_hi, hmn_b, hi16(rt_b) + o, rj_b, sat & 2u);
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

int launch_intra_glob16(dsa_ctx* ctx, cudaStream_t stream, const dsa_db* db, const dsa_db* qs,
                        const PackedPlan& plan, const IntraWork& work, int mode, uint32_t fe,
                        int o, int e, int smax, int smin, Scores out, uint32_t n_targets_out) {
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
  IntraGlobArgs G;
  G.mode = mode; G.fe = fe; G.e = e; G.smin = smin; G.qlen = qs->d_len;
  G.hmax2 = ((uint32_t)A.T << 16) | (uint32_t)A.T;
  const uint64_t warps_total = std::min<uint64_t>(A.n_items, (uint64_t)ctx->sm_count * 16);
  const unsigned grid = (unsigned)((warps_total + WARPS - 1) / WARPS);
  A.scratch_cols = work.max_long_len;
  const size_t scr_bytes = (size_t)grid * WARPS * A.scratch_cols * sizeof(uint2);
  void* scr = nullptr;
  DSA_TRY(ctx->alloc(&scr, scr_bytes, stream));
  A.scratch = static_cast<uint2*>(scr);
  A.o_score = out.score; A.o_qend = out.q_end; A.o_tend = out.t_end; A.o_flag = out.flag;
  A.n_out_t = n_targets_out;
  const bool sg = mode == DSA_SEMIGLOBAL;
  const bool tb = sg && (fe & DSA_FREE_T_BEGIN), te = sg && (fe & DSA_FREE_T_END);
  auto kern = tb ? (te ? k_intra_glob16<true, true> : k_intra_glob16<true, false>)
                 : (te ? k_intra_glob16<false, true> : k_intra_glob16<false, false>);
  DSA_CUDA_TRY(cudaMemsetAsync(A.counter, 0, sizeof(uint32_t), stream));
  kern<<<grid, WARPS * 32, 0, stream>>>(A, G);
  ++ctx->launches;
  cudaError_t err = cudaGetLastError();
  ctx->release(scr, scr_bytes, stream);
  if (err != cudaSuccess) {
    set_error("k_intra_glob16 launch: %s", cudaGetErrorString(err));
    return DSA_ERR_CUDA;
  }
  return DSA_OK;
}

}  // namespace dsa
