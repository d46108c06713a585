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
// pair is rerun in int32).
#include "dsa_internal.cuh"
#include "dpx.cuh"

#include <type_traits>

namespace dsa {
namespace {

constexpr int NT = 128;
constexpr int BLOCKS_PER_SM = 4;
constexpr int ROWS_LDS = 16;     // strip rows, shared-memory substitution form
constexpr int ROWS_BYTES = 16;   // strip rows, byte-permute form (two table registers per row)
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

// (score desc, j asc, i asc)
struct C16 {
  int s, i, j;
  bool has;
  __device__ __forceinline__ void offer(int s2, int i2, int j2) {
    if (!has || s2 > s || (s2 == s && (j2 < j || (j2 == j && i2 < i)))) {
      s = s2; i = i2; j = j2; has = true;
    }
  }
};

template <bool LOCAL, int ROWS, bool BYTES>
__global__ void __launch_bounds__(NT, BLOCKS_PER_SM) k_pairs16(
    const uint8_t* __restrict__ qcodes, const uint8_t* __restrict__ tcodes,
    const int8_t* __restrict__ Sg, int A, int o, int e, int mode, uint32_t fe, int T,
    const Pair16Job* __restrict__ jobs, uint32_t n_jobs, uint2* __restrict__ scratch,
    uint32_t scratch_cols, int32_t* __restrict__ o_score, int32_t* __restrict__ o_qend,
    int32_t* __restrict__ o_tend, uint8_t* __restrict__ o_flag) {
  __shared__ int16_t Sp[32 * 32];                       // S + o
  __shared__ uint32_t Sb[4];                            // BYTES: row q of S + o as 4 bytes
  __shared__ uint32_t park[2][ROWS][NT];                // parked columns (local mode)
  __shared__ uint2 ring[RING_SLOTS * NT];               // boundary-row columns in flight
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
  const uint32_t neg_o2 = pack2(-o, -o), neg_e2 = pack2(-e, -e);
  const uint32_t NEG2 = pack2(NEG16, NEG16);
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
    const uint8_t* tlo = tcodes + jb.t_lo;
    const uint8_t* thi = tcodes + jb.t_hi;

    // local: running best per half; others: candidates
    int best_lo = 0, best_hi = 0, bj_lo = 0, bj_hi = 0, bi_lo = 0, bi_hi = 0;
    C16 clo = {0, 0, 0, false}, chi = {0, 0, 0, false};
    if (!local) {
      const int32_t hm0 = h_col0(mode, fe, m, o, e);
      if (t_end_free) { clo.offer(hm0, m, 0); chi.offer(hm0, m, 0); }
      if (q_end_free) { clo.offer(h_row0(mode, fe, nlo, o, e), 0, nlo); chi.offer(h_row0(mode, fe, nhi, o, e), 0, nhi); }
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
        Ho[r] = pack2(hc, hc);
        E[r] = NEG2;
        if (BYTES) {
          sb_lo[r] = r < rows ? Sb[qlo[i - 1]] : 0u;
          sb_hi[r] = r < rows ? Sb[qhi[i - 1]] : 0u;
        } else {
          qa[r] = r < rows ? ((uint32_t)qlo[i - 1] * A) | (((uint32_t)qhi[i - 1] * A) << 16) : 0u;
        }
      }
      const int32_t hd = h_col0(mode, fe, i0, o, e) - o;
      uint32_t diag = pack2(hd, hd);
      int pend = 0;
      uint32_t thr2 = pack2(max(best_lo - 1, 0), max(best_hi - 1, 0));
      // The column loop in four forms (first strip: top row from the boundary
      // of the matrix; last strip: result candidates, no boundary row to hand
      // down), so that no per-column branch depends on the strip.
      auto columns = [&](auto first_c, auto last_c) {
        constexpr bool FIRST = decltype(first_c)::value;
        constexpr bool LAST = decltype(last_c)::value;
        const bool col_n = LAST || q_end_free;   // column-n candidates in this strip
        // loads run one column ahead of the arithmetic (target residues and
        // the boundary row handed down by the previous strip); the last
        // iteration re-reads a valid column instead of branching
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
        uint32_t n_alo = tlo[0], n_ahi = thi[0];
        for (int32_t j = 1; j <= nmax; ++j) {
          const uint32_t a_lo = j <= nlo ? n_alo : 0u;
          const uint32_t a_hi = j <= nhi ? n_ahi : 0u;
          uint2 v = make_uint2(0u, 0u);
          if (!FIRST) {
            cp_async_wait<AHEAD - 1>();   // column j has landed
            v = rt[(j & (RING_SLOTS - 1)) * NT];
            const int32_t c = j + AHEAD;
            if (c <= nmax) cp_async8(rt + (c & (RING_SLOTS - 1)) * NT, scr + (uint64_t)(c - 1) * stride);
            cp_async_commit();
          }
          const int32_t jn = min(j, nmax - 1);
          n_alo = tlo[min(jn, max(nlo - 1, 0))];
          n_ahi = thi[min(jn, max(nhi - 1, 0))];
          uint32_t topHo, F;
          if (FIRST) {
            const int32_t h0l = h_row0(mode, fe, min(j, nlo), o, e) - o;
            const int32_t h0h = h_row0(mode, fe, min(j, nhi), o, e) - o;
            topHo = pack2(h0l, h0h);
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
              E[r] = addmax2(E[r], neg_e2, old);
              const uint32_t t = addmax2(d, sp, E[r]);
              const uint32_t h = local ? max2_relu(t, F) : __vmaxs2(t, F);
              Ho[r] = add2(h, neg_o2);
              F = addmax2(F, neg_e2, Ho[r]);
              d = old;
              hlast = h;
              if (local) {
                if (r & 1) cm = max3_2(cm, hprev, h);
                else hprev = h;
              }
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
              thr2 = pack2(max(best_lo - 1, 0), max(best_hi - 1, 0));
            }
          } else {
            // row m (last strip) and column n
            if (LAST && t_end_free) {
              if (j <= nlo) clo.offer(lo16(hlast), m, j);
              if (j <= nhi) chi.offer(hi16(hlast), m, j);
            }
            if (col_n && j == nlo) {
              // column n of the low pair: first row of this strip holding its maximum
              int bs = -32768, br = 0;
#pragma unroll
              for (int r = ROWS - 1; r >= 0; --r)
                if (r < rows && (q_end_free || r == rows - 1) && lo16(Ho[r]) + o >= bs) { bs = lo16(Ho[r]) + o; br = r; }
              clo.offer(bs, i0 + br + 1, j);
            }
            if (col_n && j == nhi) {
              int bs = -32768, br = 0;
#pragma unroll
              for (int r = ROWS - 1; r >= 0; --r)
                if (r < rows && (q_end_free || r == rows - 1) && hi16(Ho[r]) + o >= bs) { bs = hi16(Ho[r]) + o; br = r; }
              chi.offer(bs, i0 + br + 1, j);
            }
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
          if (lo16(park[0][r][tid]) == want) rr = r;
        bi_lo = i0 + rr + 1;
      }
      if (pend & 2) {
        const int want = best_hi - o;
        int rr = ROWS - 1;
        for (int r = ROWS - 1; r >= 0; --r)
          if (hi16(park[1][r][tid]) == want) rr = r;
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
      o_score[jb.out_lo] = clo.s; o_qend[jb.out_lo] = clo.i - 1; o_tend[jb.out_lo] = clo.j - 1;
      o_flag[jb.out_lo] = 0;
      if (jb.out_hi != 0xFFFFFFFFu) {
        o_score[jb.out_hi] = chi.s; o_qend[jb.out_hi] = chi.i - 1; o_tend[jb.out_hi] = chi.j - 1;
        o_flag[jb.out_hi] = 0;
      }
    }
  }
}

}  // namespace

int launch_pairs16(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int8_t* d_matrix, int A,
                   int o, int e, int mode, uint32_t fe, int smax, bool bytes,
                   const Pair16Job* d_jobs, uint32_t n_jobs, uint32_t max_n, Scores out) {
  if (n_jobs == 0) return DSA_OK;
  // persistent: every block resident at once, jobs taken in a grid stride
  const uint64_t blocks =
      std::min<uint64_t>((n_jobs + NT - 1) / NT, (uint64_t)ctx->sm_count * BLOCKS_PER_SM);
  const size_t scr_bytes = (size_t)blocks * NT * max_n * sizeof(uint2);
  void* scr = nullptr;
  DSA_TRY(ctx->alloc(&scr, scr_bytes));
  auto kern = mode == DSA_LOCAL
                  ? (bytes ? k_pairs16<true, ROWS_BYTES, true> : k_pairs16<true, ROWS_LDS, false>)
                  : (bytes ? k_pairs16<false, ROWS_BYTES, true> : k_pairs16<false, ROWS_LDS, false>);
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
