// Packed int16x2 kernel for explicit short pairs of the map phase (Sec. II.B.1,
// any of the three algorithms of Sec. II.C.2; e.g. reads against windows
// of a genome): one thread aligns two pairs at once, one in each 16-bit half
// of every DP register.  The two pairs of a thread have the same query length
// (pairs are sorted by query length, then window length), so the strips and
// the row of the query's last residue line up in both halves.
//
// Per thread: the query rows in strips of ROWS rows held in registers, the
// target windows scanned column by column, the strip's bottom row (H - o and
// the next row's F) handed to the next strip through a per-thread boundary
// row in global memory.  Substitution scores (S + o): for alphabets of at most
// four letters whose S + o fits a byte, each row keeps the four values of its
// query residue as bytes, one register per pair, and one byte permute per
// cell pair picks both and sign-extends them into the two halves (16-row
// strips); otherwise two lookups per cell pair in a shared-memory copy of
// S + o (int16, 16-row strips).
//
// Result cells (same rules as everywhere in the library): local = best cell
// with the smallest (j, i) -- a column-maximum trigger parks the column in
// shared memory and the first row is found at the end of the strip; global =
// (m, n); semi-global = best of row m (target end free, smallest j), column n
// (query end free, smallest i) and (m, n).
//
// Range: used only when (m + n) * max(|S|, o, e) + o stays far inside int16
// for non-local modes (every value is exact), and in local mode with the
// saturation flag of the inter-sequence kernel (best > 32767 - max S => the
// pair is rerun in int32).  Global / semi-global values are kept in offset
// binary (each half + 0x8000) so that H - o is one 32-bit subtract with no borrow between the
// halves: the pair with the longer window bounds every value of both halves
// over all columns to |v| < 12000, with o < 4096.  Local mode keeps signed
// halves (the ReLU maximum of DPX needs no constant register there).
#include "dsa_internal.cuh"
#include "dpx.cuh"

#include <type_traits>

namespace dsa {
namespace {

constexpr int NT = 128;
constexpr int BLOCKS_PER_SM = 4;
constexpr int ROWS_LDS = 16;     // strip rows, shared-memory substitution form
constexpr int ROWS_BYTES = 16;   // strip rows, byte-permute form (two table registers per row)
// the byte-permute form's wide variant: 20-row strips (the column overhead
// spread over more rows) at 3 blocks per SM (168 registers, 12 warps)
constexpr int ROWS_BYTES_WIDE = 20;
constexpr int BLOCKS_PER_SM_WIDE = 3;
constexpr int RING_SLOTS = 8;    // boundary-row ring: slots per thread (a power of two)
constexpr int AHEAD = RING_SLOTS - 1;   // columns copied ahead of the arithmetic

__device__ __forceinline__ int32_t h_row0(int mode, uint32_t fe, int64_t j, int o, int e) {
  if (j == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_T_BEGIN))) return 0;
  return -(o + (int32_t)(j - 1) * e);
}
__device__ __forceinline__ int32_t h_col0(int mode, uint32_t fe, int64_t i, int o, int e) {
  if (i == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_Q_BEGIN))) return 0;
  return -(o + (int32_t)(i - 1) * e);
}

template <bool LOCAL, int ROWS, bool BYTES, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_pairs16(
    const uint8_t* __restrict__ qcodes, const uint8_t* __restrict__ tcodes,
    const int8_t* __restrict__ Sg, int A, int o, int e, int mode, uint32_t fe, int T,
    const Pair16Job* __restrict__ jobs, uint32_t n_jobs, uint2* __restrict__ scratch,
    uint32_t scratch_cols, int32_t* __restrict__ o_score, int32_t* __restrict__ o_qend,
    int32_t* __restrict__ o_tend, uint8_t* __restrict__ o_flag) {
  __shared__ int16_t Sp[32 * 32];                       // S + o
  __shared__ uint32_t Sb[4];                            // BYTES: row q of S + o as 4 bytes
  __shared__ uint32_t park[2][ROWS][NT];                // parked columns (local mode)
  __shared__ uint2 ring[RING_SLOTS * NT];               // boundary-row columns in flight
  // global / semi-global result state per thread and half: column n's best
  // score and row, row m's best column
  __shared__ int s_cb[2][NT], s_ci[2][NT], s_rj[2][NT];
  for (int x = threadIdx.x; x < A * A; x += blockDim.x) Sp[x] = (int16_t)(Sg[x] + o);
  if (BYTES && threadIdx.x < 4) {
    uint32_t w = 0;
    for (int a = 0; a < A; ++a)
      if ((int)threadIdx.x < A) w |= (uint32_t)(uint8_t)(int8_t)(Sg[threadIdx.x * A + a] + o) << (8 * a);
    Sb[threadIdx.x] = w;
  }
  __syncthreads();
  const int tid = threadIdx.x;
  constexpr bool local = LOCAL;
  const bool sg = mode == DSA_SEMIGLOBAL;
  const bool q_end_free = sg && (fe & DSA_FREE_Q_END);
  const bool t_end_free = sg && (fe & DSA_FREE_T_END);
  // global / semi-global: values in offset binary (each half + 0x8000), as
  // in the inter-sequence kernels -- unsigned DPX maxima, constants added
  // mod 2^16, H - o one 32-bit subtract; local: signed halves, where the
  // ReLU maximum needs no constant register
  constexpr uint32_t BIAS2 = LOCAL ? 0u : 0x80008000u;
  const uint32_t neg_e2 = pack2(-e, -e);
  const uint32_t neg_o2 = pack2(-o, -o);
  const uint32_t o2 = ((uint32_t)o << 16) | (uint32_t)o;
  const uint32_t NEG2 = pack2(NEG16, NEG16) ^ BIAS2;
  const uint64_t gtid = blockIdx.x * (uint64_t)NT + tid;
  uint2* const scr = scratch + gtid;                   // column c at scr[c * stride]
  const uint64_t stride = (uint64_t)gridDim.x * NT;

  for (uint64_t k = gtid; k < n_jobs; k += stride) {
    const Pair16Job jb = jobs[k];
    const int32_t m = jb.m;
    const int32_t nlo = jb.n_lo, nhi = jb.n_hi;
    const int32_t nmax = max(nlo, nhi);
    const uint8_t* qlo = qcodes + jb.q_lo;
    const uint8_t* qhi = qcodes + jb.q_hi;
    // the windows as aligned words (see the column loop)
    // byte shifts of both windows in one register: the low half's in bits
    // 0-4 (a funnel shift reads only those), the high half's from bit 8
    const uint32_t sh2 = 8u * (uint32_t)(jb.t_lo & 3) | (8u * (uint32_t)(jb.t_hi & 3)) << 8;
    const uint32_t* wlo = reinterpret_cast<const uint32_t*>(tcodes + (jb.t_lo & ~3ull));
    const uint32_t* whi = reinterpret_cast<const uint32_t*>(tcodes + (jb.t_hi & ~3ull));
    // a window's last word index plus one (recomputed where used: registers)
    auto w_last = [](int32_t n) { return ((max(n, 1) - 1) >> 2) + 1; };

    // local: running best per half (registers); others: the result
    // candidates in shared memory (rarely touched) and a packed threshold
    int best_lo = 0, best_hi = 0, bj_lo = 0, bj_hi = 0, bi_lo = 0, bi_hi = 0;
    // row m (free target end): best H so far as an offset-binary threshold
    // (a half that is not tracked holds the largest value: never exceeded)
    uint32_t rthr = 0xFFFFFFFFu;
    if (!local) {
      const int32_t hm0 = h_col0(mode, fe, m, o, e);   // the candidate (m, 0)
      if (t_end_free) rthr = pack2(hm0, hm0) ^ BIAS2;
      s_rj[0][tid] = 0;
      s_rj[1][tid] = 0;
      // column n: the candidate (0, n) with a free query end, else none yet
      s_cb[0][tid] = q_end_free ? h_row0(mode, fe, nlo, o, e) : INT32_MIN;
      s_cb[1][tid] = q_end_free ? h_row0(mode, fe, nhi, o, e) : INT32_MIN;
      s_ci[0][tid] = 0;
      s_ci[1][tid] = 0;
    }

    for (int32_t i0 = 0; i0 < m; i0 += ROWS) {
      const int rows = min(ROWS, m - i0);
      const bool last = i0 + rows == m;
      // qa: LDS form, the two pairs' matrix row offsets; sb: BYTES form, the
      // two pairs' S + o rows as bytes
      uint32_t Ho[ROWS], E[ROWS], qa[ROWS], sb_lo[ROWS], sb_hi[ROWS];
#pragma unroll
      for (int r = 0; r < ROWS; ++r) {
        const int32_t i = i0 + r + 1;
        const int32_t hc = h_col0(mode, fe, i, o, e) - o;
        Ho[r] = pack2(hc, hc) ^ BIAS2;
        E[r] = NEG2;
        if (BYTES) {
          sb_lo[r] = r < rows ? Sb[qlo[i - 1]] : 0u;
          sb_hi[r] = r < rows ? Sb[qhi[i - 1]] : 0u;
        } else {
          qa[r] = r < rows ? ((uint32_t)qlo[i - 1] * A) | (((uint32_t)qhi[i - 1] * A) << 16) : 0u;
        }
      }
      const int32_t hd = h_col0(mode, fe, i0, o, e) - o;
      uint32_t diag = pack2(hd, hd) ^ BIAS2;
      int pend = 0;
      uint32_t thr2 = pack2(max(best_lo - 1, 0), max(best_hi - 1, 0)) ^ BIAS2;
      // The column loop in four forms (first strip: top row from the boundary
      // of the matrix; last strip: result candidates, no boundary row to hand
      // down), so that no per-column branch depends on the strip.
      auto columns = [&](auto first_c, auto last_c) {
        constexpr bool FIRST = decltype(first_c)::value;
        constexpr bool LAST = decltype(last_c)::value;
        const bool col_n = LAST || q_end_free;   // column-n candidates in this strip
        // the previous strip's boundary row arrives through a per-thread ring
        // of RING_SLOTS columns, copied AHEAD columns ahead by cp.async (one
        // commit group per column); the copy issued at column j refills the
        // slot read at column j - 1, and it reads a column this strip has not
        // yet overwritten (the strip writes column j - 1 at column j)
        uint2* const rt = ring + tid;
        if (!FIRST) {
#pragma unroll
          for (int c = 1; c <= AHEAD; ++c) {
            if (c <= nmax) cp_async8(rt + (c & (RING_SLOTS - 1)) * NT, scr + (uint64_t)(c - 1) * stride);
            cp_async_commit();
          }
        }
        // window residues by aligned 32-bit words: the residues of columns
        // 4g+1 .. 4g+4 are bytes s .. s+3 (s = the window's address mod 4)
        // of the word pair (g, g+1) counted from the aligned address below
        // the window; each group's second word is loaded one group (4
        // columns) ahead, and word indices stop at the window's last word
        // plus one, which stays inside the sequence buffer's padding
        uint32_t wa_lo = __ldg(wlo), wb_lo = __ldg(wlo + min(1, w_last(nlo)));
        uint32_t wa_hi = __ldg(whi), wb_hi = __ldg(whi + min(1, w_last(nhi)));
        uint32_t r4_lo = 0, r4_hi = 0;
        // column j = group start + kk + 1; IN: inside both windows (no
        // residue tests)
        auto column = [&](int32_t j, int kk, auto in_c) {
          constexpr bool IN = decltype(in_c)::value;
          const uint32_t kb = 8u * (uint32_t)kk;
          const uint32_t a_lo = (IN || j <= nlo) ? (r4_lo >> kb) & 0xFFu : 0u;
          const uint32_t a_hi = (IN || j <= nhi) ? (r4_hi >> kb) & 0xFFu : 0u;
          uint2 v = make_uint2(0u, 0u);
          if (!FIRST) {
            cp_async_wait<AHEAD - 1>();   // column j has landed
            v = rt[(j & (RING_SLOTS - 1)) * NT];
            const int32_t c = j + AHEAD;
            if (c <= nmax) cp_async8(rt + (c & (RING_SLOTS - 1)) * NT, scr + (uint64_t)(c - 1) * stride);
            cp_async_commit();
          }
          uint32_t topHo, F;
          if (FIRST) {
            const int32_t h0l = h_row0(mode, fe, min(j, nlo), o, e) - o;
            const int32_t h0h = h_row0(mode, fe, min(j, nhi), o, e) - o;
            topHo = pack2(h0l, h0h) ^ BIAS2;
            F = topHo;   // F of row 1 = H[0][j] - o
          } else {
            topHo = v.x;
            F = v.y;
          }
          uint32_t d = diag;
          diag = topHo;
          // BYTES: byte a_lo of the low row (sign-replicated into byte 1) and
          // byte 4 + a_hi of the high row (sign-replicated into byte 3)
          const uint32_t sel = (a_lo * 0x11u + 0x80u) | ((a_hi * 0x11u + 0xC4u) << 8);
          uint32_t cm = 0, hprev = 0, hlast = 0;
#pragma unroll
          for (int r = 0; r < ROWS; ++r) {
            if (LAST ? r < rows : true) {
              const uint32_t sp = BYTES ? prmt(sb_lo[r], sb_hi[r], sel)
                                        : (uint32_t)(uint16_t)Sp[(qa[r] & 0xFFFFu) + a_lo] |
                                              ((uint32_t)(uint16_t)Sp[(qa[r] >> 16) + a_hi] << 16);
              const uint32_t old = Ho[r];
              uint32_t h;
              if (local) {
                E[r] = addmax2(E[r], neg_e2, old);
                const uint32_t t = addmax2(d, sp, E[r]);
                h = max2_relu(t, F);
                Ho[r] = add2(h, neg_o2);
                F = addmax2(F, neg_e2, Ho[r]);
                if (r & 1) cm = max3_2(cm, hprev, h);
                else hprev = h;
              } else {
                E[r] = addmax2u(E[r], neg_e2, old);
                const uint32_t t = addmax2u(d, sp, E[r]);
                h = __vmaxu2(t, F);
                Ho[r] = h - o2;   // no borrow between the halves (see the header)
                F = addmax2u(F, neg_e2, Ho[r]);
              }
              d = old;
              hlast = h;
            }
          }
          if (local && LAST && (rows & 1)) cm = __vmaxs2(cm, hprev);
          if (!LAST) scr[(uint64_t)(j - 1) * stride] = make_uint2(Ho[ROWS - 1], F);
          if (local) {
            if (__vmaxs2(cm, thr2) != thr2) {
              const int cl = lo16(cm), ch = hi16(cm);
              const int thr_lo = best_lo - (j < bj_lo ? 1 : 0);
              const int thr_hi = best_hi - (j < bj_hi ? 1 : 0);
              if (cl > thr_lo && j <= nlo) {
#pragma unroll
                for (int r = 0; r < ROWS; ++r) park[0][r][tid] = Ho[r];
                best_lo = cl; bj_lo = j; pend |= 1;
              }
              if (ch > thr_hi && j <= nhi) {
#pragma unroll
                for (int r = 0; r < ROWS; ++r) park[1][r][tid] = Ho[r];
                best_hi = ch; bj_hi = j; pend |= 2;
              }
              thr2 = pack2(max(best_lo - 1, 0), max(best_hi - 1, 0)) ^ BIAS2;
            }
          } else {
            // row m (last strip, free target end): strictly better H, so the
            // smallest j of a tie stays
            if (LAST && __vmaxu2(hlast, rthr) != rthr) {
              if (j <= nlo && (hlast & 0xFFFFu) > (rthr & 0xFFFFu)) {
                rthr = (rthr & 0xFFFF0000u) | (hlast & 0xFFFFu);
                s_rj[0][tid] = j;
              }
              if (j <= nhi && (hlast >> 16) > (rthr >> 16)) {
                rthr = (rthr & 0x0000FFFFu) | (hlast & 0xFFFF0000u);
                s_rj[1][tid] = j;
              }
            }
            // column n: the first row of this strip holding its maximum,
            // strictly better than the earlier strips' (smaller i first)
            if (col_n && (j == nlo || j == nhi)) {
#pragma unroll
              for (int x = 0; x < 2; ++x) {
                if (j != (x ? nhi : nlo)) continue;
                int bs = -32768, br = 0;
#pragma unroll
                for (int r = ROWS - 1; r >= 0; --r) {
                  const int v16 = (x ? hi16(Ho[r] ^ BIAS2) : lo16(Ho[r] ^ BIAS2)) + o;
                  if (r < rows && (q_end_free || r == rows - 1) && v16 >= bs) { bs = v16; br = r; }
                }
                if (bs > s_cb[x][tid]) { s_cb[x][tid] = bs; s_ci[x][tid] = i0 + br + 1; }
              }
            }
          }
        };
        // columns in groups of 4 (one residue word): the group's body is
        // unrolled, so the residue's byte position is a constant and the
        // compiler can overlap the wavefronts of neighbouring columns
        const int32_t nmin = min(nlo, nhi);
        for (int32_t j0 = 0; j0 < nmax; j0 += 4) {
          const int32_t g = j0 >> 2;
          r4_lo = __funnelshift_r(wa_lo, wb_lo, sh2);
          r4_hi = __funnelshift_r(wa_hi, wb_hi, sh2 >> 8);
          wa_lo = wb_lo;
          wa_hi = wb_hi;
          wb_lo = __ldg(wlo + min(g + 2, w_last(nlo)));
          wb_hi = __ldg(whi + min(g + 2, w_last(nhi)));
          if (j0 + 4 <= nmin) {
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) column(j0 + 1 + kk, kk, std::true_type{});
          } else {
#pragma unroll 1
            for (int kk = 0; kk < 4 && j0 + 1 + kk <= nmax; ++kk) column(j0 + 1 + kk, kk, std::false_type{});
          }
        }
        if (!FIRST) cp_async_wait<0>();   // nothing in flight into the ring past the strip
      };
      using T_ = std::true_type;
      using F_ = std::false_type;
      if (i0 == 0) {
        if (last) columns(T_{}, T_{});
        else columns(T_{}, F_{});
      } else {
        if (last) columns(F_{}, T_{});
        else columns(F_{}, F_{});
      }
      if (pend & 1) {
        const int want = best_lo - o;
        int rr = ROWS - 1;
        for (int r = ROWS - 1; r >= 0; --r)
          if (lo16(park[0][r][tid] ^ BIAS2) == want) rr = r;
        bi_lo = i0 + rr + 1;
      }
      if (pend & 2) {
        const int want = best_hi - o;
        int rr = ROWS - 1;
        for (int r = ROWS - 1; r >= 0; --r)
          if (hi16(park[1][r][tid] ^ BIAS2) == want) rr = r;
        bi_hi = i0 + rr + 1;
      }
    }
    if (local) {
      o_score[jb.out_lo] = best_lo;
      o_qend[jb.out_lo] = best_lo > 0 ? bi_lo - 1 : -1;
      o_tend[jb.out_lo] = best_lo > 0 ? bj_lo - 1 : -1;
      o_flag[jb.out_lo] = best_lo > T ? 1 : 0;
      if (jb.out_hi != 0xFFFFFFFFu) {
        o_score[jb.out_hi] = best_hi;
        o_qend[jb.out_hi] = best_hi > 0 ? bi_hi - 1 : -1;
        o_tend[jb.out_hi] = best_hi > 0 ? bj_hi - 1 : -1;
        o_flag[jb.out_hi] = best_hi > T ? 1 : 0;
      }
    } else {
      // the better of row m's best (m, j) and column n's best (i, n) under
      // (score desc, j asc, i asc): row m wins a tie only at a smaller j
      for (int x = 0; x < 2; ++x) {
        const uint32_t out = x ? jb.out_hi : jb.out_lo;
        if (out == 0xFFFFFFFFu) continue;
        const int n = x ? nhi : nlo;
        int bs = s_cb[x][tid], bi = s_ci[x][tid], bj = n;
        if (t_end_free) {
          const int rb = (x ? hi16(rthr ^ BIAS2) : lo16(rthr ^ BIAS2));
          const int rj = s_rj[x][tid];
          if (rb > bs || (rb == bs && rj < n)) { bs = rb; bi = m; bj = rj; }
        }
        o_score[out] = bs; o_qend[out] = bi - 1; o_tend[out] = bj - 1;
        o_flag[out] = 0;
      }
    }
  }
}

}  // namespace

int pairs16_wide_rows() { return ROWS_BYTES_WIDE; }

int launch_pairs16(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int8_t* d_matrix, int A,
                   int o, int e, int mode, uint32_t fe, int smax, bool bytes, int rows,
                   const Pair16Job* d_jobs, uint32_t n_jobs, uint32_t max_n, Scores out) {
  if (n_jobs == 0) return DSA_OK;
  const bool wide = bytes && rows == ROWS_BYTES_WIDE;
  // persistent: every block resident at once, jobs taken in a grid stride
  const uint64_t blocks = std::min<uint64_t>(
      (n_jobs + NT - 1) / NT, (uint64_t)ctx->sm_count * (wide ? BLOCKS_PER_SM_WIDE : BLOCKS_PER_SM));
  const size_t scr_bytes = (size_t)blocks * NT * max_n * sizeof(uint2);
  void* scr = nullptr;
  DSA_TRY(ctx->alloc(&scr, scr_bytes));
  auto kern =
      mode == DSA_LOCAL
          ? (wide    ? k_pairs16<true, ROWS_BYTES_WIDE, true, BLOCKS_PER_SM_WIDE>
             : bytes ? k_pairs16<true, ROWS_BYTES, true, BLOCKS_PER_SM>
                     : k_pairs16<true, ROWS_LDS, false, BLOCKS_PER_SM>)
          : (wide    ? k_pairs16<false, ROWS_BYTES_WIDE, true, BLOCKS_PER_SM_WIDE>
             : bytes ? k_pairs16<false, ROWS_BYTES, true, BLOCKS_PER_SM>
                     : k_pairs16<false, ROWS_LDS, false, BLOCKS_PER_SM>);
  kern<<<(unsigned)blocks, NT, 0, ctx->stream>>>(
      qs->d_codes, db->d_codes, d_matrix, A, o, e, mode, fe, 32767 - std::max(0, smax), d_jobs,
      n_jobs, static_cast<uint2*>(scr), max_n, out.score, out.q_end, out.t_end, out.flag);
  ++ctx->launches;
  cudaError_t err = cudaGetLastError();
  ctx->release(scr, scr_bytes);
  if (err != cudaSuccess) {
    set_error("k_pairs16 launch: %s", cudaGetErrorString(err));
    return DSA_ERR_CUDA;
  }
  return DSA_OK;
}

}  // namespace dsa
