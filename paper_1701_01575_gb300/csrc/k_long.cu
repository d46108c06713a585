// Long explicit pairs (e.g. genome fragments of 1e4-1e5 residues), exact
// int32, any mode (DSW / DNW / DSG, Sec. II.C.2): a band-pipelined wavefront
// for the score pass and a checkpointed traceback for the alignment object's
// location and CIGAR (Sec. II.B.1).
//
// Score pass.  The query rows of a pair are cut into bands of BAND = 32 x ROWS
// rows.  One warp computes one band as an anti-diagonal wavefront (lane k owns
// ROWS rows and processes column j = step - k; H and F of its last row go to
// lane k+1 by warp shuffle).  Band b reads the bottom row (H, F) of band b-1
// from a boundary row in global memory; band b-1 publishes how many columns
// of it are complete in a progress counter (after a memory fence), and band b
// waits on that counter with a bounded wait before it needs a column.  Work
// items (pair, band) are taken in order from one counter by persistent
// warps, so every band's predecessor was taken earlier by a warp that is
// already running: the pipeline always advances.  Checkpoint rows (H, F)
// for the traceback are kept every TB_BAND = BAND / 2 rows: a band's bottom
// row (also the next band's input) and its middle row.  Checkpoint c holds
// row (c + 1) TB_BAND.
//
// Result cell.  Inside a lane, cells are visited in increasing (j, i), so a
// lane keeps its first strictly better candidate; the lanes' and bands'
// candidates are merged under (score desc, j asc, i asc) by k_long_reduce.
//
// Traceback.  The checkpoints make every TB_BAND-row band independent: all
// bands of all hits are recomputed at once (one warp each, TB_ROWS rows per
// lane) over the rectangle up to the
// end cell, storing the 4-bit decision of every cell, then one warp per hit
// walks back through a shared-memory window of the decisions.  Decision
// memory is half a byte per cell of the rectangle (or of its diagonal band),
// handled in chunks of bounded size.  Each traceback band of a hit keeps its
// decisions as TB_BAND-row blocks of one word (8 columns) per row, the
// words of a column block consecutive by row: word w of row i0 + k of band b
// is at (b wpr + w) TB_BAND + k, so the 8 rows of a fill lane make whole
// sectors and the writes in flight stay within a few lines per band (row by
// row, a warp kept a partly written line per row, which at 2 bands per warp
// outgrew the L2).  A decision nibble here holds the H
// source in bits 0-1 (0 D, 1 M, 2 I, 3 stop: the empty local alignment),
// E opened here in bit 2 and F opened here in bit 3; the packed fill
// (k_long_tb16.cu) writes the same nibbles.
#include "dsa_internal.cuh"
#include "dpx.cuh"

#include <type_traits>

namespace dsa {
namespace {

constexpr int ROWS = 16;
constexpr int BAND = 32 * ROWS;
constexpr int TB_ROWS = 8;               // traceback fill: rows per lane
constexpr int TB_BAND = 32 * TB_ROWS;    // traceback bands (checkpoint spacing)
static_assert(BAND == 2 * TB_BAND, "a score band holds two traceback bands");
constexpr int WARPS = 4;
constexpr uint32_t PUBLISH = 32;   // columns between progress updates

__device__ __forceinline__ int32_t h_row0(int mode, uint32_t fe, int64_t j, int o, int e) {
  if (j == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_T_BEGIN))) return 0;
  return -(o + (int32_t)(j - 1) * e);
}
__device__ __forceinline__ int32_t h_col0(int mode, uint32_t fe, int64_t i, int o, int e) {
  if (i == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_Q_BEGIN))) return 0;
  return -(o + (int32_t)(i - 1) * e);
}

using Cand = LongCand;
__device__ __forceinline__ bool cand_better(const Cand& a, const Cand& b) {
  if (!a.has) return false;
  if (!b.has) return true;
  if (a.s != b.s) return a.s > b.s;
  if (a.j != b.j) return a.j < b.j;
  return a.i < b.i;
}


// Column inputs of the wavefront: lane 0 takes column j = s at step s; the
// boundary row of the band above and the target residues are fetched by the
// whole warp 32 columns at a time (lane k holds column blk + k + 1), one
// block ahead, and handed to lane 0 by shuffle; residues then travel lane to
// lane with H and F.  The wait on the band above is bounded and covers a
// whole block.
template <bool LOCAL, bool BYTES>
__global__ void __launch_bounds__(WARPS * 32, 4) k_long_score(
    const uint8_t* __restrict__ qcodes, const uint8_t* __restrict__ tcodes,
    const int8_t* __restrict__ Sg, int A, int o, int e, int mode, uint32_t fe,
    const LongJob* __restrict__ jobs, const uint32_t* __restrict__ items, uint32_t n_items,
    uint32_t* __restrict__ counter, int2* __restrict__ bnd, uint32_t* __restrict__ prog,
    Cand* __restrict__ cands, int32_t* __restrict__ status) {
  // substitution scores with o added: the diagonal term H[i-1][j-1] + S is
  // taken as (H[i-1][j-1] - o) + (S + o), from the stored H - o
  __shared__ int16_t So[32 * 32];
  __shared__ uint32_t Sb[4];   // BYTES: row q of S + o as 4 bytes (each fits int8)
  for (int x = threadIdx.x; x < A * A; x += blockDim.x) So[x] = (int16_t)(Sg[x] + o);
  if (BYTES && threadIdx.x < 4) {
    uint32_t w = 0;
    for (int a = 0; a < A; ++a)
      if ((int)threadIdx.x < A) w |= (uint32_t)(uint8_t)(int8_t)(Sg[threadIdx.x * A + a] + o) << (8 * a);
    Sb[threadIdx.x] = w;
  }
  __syncthreads();
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const bool sg = mode == DSA_SEMIGLOBAL;
  const bool q_end_free = sg && (fe & DSA_FREE_Q_END);
  const bool t_end_free = sg && (fe & DSA_FREE_T_END);
  for (;;) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(counter, 1u);
    it = __shfl_sync(FULL, it, 0);
    if (it >= n_items) break;
    const LongJob jb = jobs[items[2 * it]];
    const uint32_t b = items[2 * it + 1];
    const int32_t m = jb.m, n = jb.n;
    const uint8_t* q = qcodes + jb.q_start;
    const uint8_t* t = tcodes + jb.t_start;
    const int32_t i0 = (int32_t)b * BAND;
    const int32_t r0 = i0 + lane * ROWS;     // rows r0+1 .. r0+ROWS
    const int32_t nb = (m + BAND - 1) / BAND;
    const bool last_band = (int32_t)b == nb - 1;
    int2* my_bnd = bnd + jb.bnd_off + (uint64_t)(2 * b + 1) * n;  // checkpoint: bottom row
    int2* my_mid = bnd + jb.bnd_off + (uint64_t)(2 * b) * n;      // checkpoint: middle row
    const int2* up_bnd = bnd + jb.bnd_off + (uint64_t)(2 * b - 1) * n;
    uint32_t* my_prog = prog + jb.prog_off + b;
    const uint32_t* up_prog = prog + jb.prog_off + b - 1;
    // the lane that holds the band's bottom row publishes it
    const int32_t bottom = min(m, i0 + BAND);
    const int bot_lane = (bottom - 1 - i0) / ROWS;
    const bool owns_m = r0 < m && m <= r0 + ROWS;
    // lane 15 holds the middle row (a checkpoint when rows follow it), the
    // bottom lane the band's last row: one store instruction serves both
    const bool stores_mid = lane == TB_BAND / ROWS - 1 && m > i0 + TB_BAND;
    const bool stores_bot = !last_band && lane == bot_lane;
    const bool stores_ck = stores_mid || stores_bot;
    int2* const ck = stores_mid ? my_mid : my_bnd;

    // Ho = H - o of the lane's rows in the previous column (the operand both
    // gap recurrences extend), E of those rows
    int32_t Ho[ROWS], E[ROWS];
    uint32_t qv[ROWS];   // BYTES: S + o row of the query residue as bytes; else its matrix offset
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int32_t i = r0 + r + 1;
      Ho[r] = h_col0(mode, fe, i, o, e) - o;
      E[r] = NEG32;
      qv[r] = i <= m ? (BYTES ? Sb[q[i - 1]] : (uint32_t)q[i - 1] * A) : 0u;
    }
    Cand c = {0, 0, 0, 0};
    if (t_end_free && owns_m) {   // H[m][0] on row m
      c = {Ho[m - r0 - 1] + o, m, 0, 1};
    }
    int32_t diag = h_col0(mode, fe, r0, o, e) - o;   // H - o above-left of the lane's first row
    int32_t sendH = 0, sendF = NEG32;                  // H - o and F of the lane's last row
    int sendA = 0;
    bool timed_out = false;
    // bounded wait until the band above has published `need` columns
    auto wait_for = [&](uint32_t need) {
      bool late = false;
      if (!timed_out) {
        const uint64_t t0 = global_ns();
        uint32_t nap = 32;   // back off: a waiting warp leaves the issue slots to working ones
        for (;;) {
          if (ld_acquire_u32(up_prog) >= need) break;
          if (global_ns() - t0 > WAIT_LIMIT_NS) {
            late = true;
            break;
          }
          __nanosleep(nap);
          nap = min(nap * 2, 1024u);
        }
      }
      if (__any_sync(FULL, late)) {
        if (!timed_out && lane == 0) atomicExch(status, DSA_ERR_DEVICE_TIMEOUT);
        timed_out = true;
      }
    };
    // boundary row of the band above for columns blk+1 .. blk+32 (lane k: blk+k+1)
    auto fetch_bnd = [&](int32_t blk) -> int2 {
      if (b == 0 || blk >= n) return make_int2(NEG32, NEG32);
      wait_for((uint32_t)min(blk + 32, n));
      const int32_t jj = blk + lane + 1;
      return jj <= n ? up_bnd[jj - 1] : make_int2(NEG32, NEG32);
    };

    auto fetch_res = [&](int32_t blk) -> int {
      const int32_t jj = blk + lane;
      return jj < n ? (int)t[jj] : 0;
    };
    int2 bcur = fetch_bnd(0), bnxt = fetch_bnd(32);
    int tcur = fetch_res(0), tnxt = fetch_res(32);
    const int32_t steps = n + 31;
    // One step of the wavefront (k = (s - 1) mod 32).  CHECK = false: every
    // lane is on a real column of a band whose rows are all real rows and no
    // global / semi-global result cell lies in the block, so no bounds are
    // tested and no result tracked.
    auto step = [&](int32_t s, int k, auto check_c) {
      constexpr bool CHECK = decltype(check_c)::value;
      const int32_t bx = __shfl_sync(FULL, bcur.x, k);
      const int32_t by = __shfl_sync(FULL, bcur.y, k);
      const int ta = __shfl_sync(FULL, tcur, k);
      int32_t Hup = __shfl_up_sync(FULL, sendH, 1);   // H - o of the cell above the lane
      int32_t Fup = __shfl_up_sync(FULL, sendF, 1);
      int a = __shfl_up_sync(FULL, sendA, 1);
      // lane 0 reads the band above (or row 0): selects, not a branch
      const int32_t h0 = b == 0 ? h_row0(mode, fe, s, o, e) - o : bx - o;
      const int32_t f0 = b == 0 ? NEG32 : by;
      Hup = lane == 0 ? h0 : Hup;
      Fup = lane == 0 ? f0 : Fup;
      a = lane == 0 ? ta : a;
      sendA = a;
      const int32_t j = s - lane;
      if (!CHECK || (j >= 1 && j <= n && r0 < m)) {
        int32_t d = diag;   // H - o above-left
        diag = Hup;
        int32_t F = Fup, hoa = Hup;   // F and H - o of the cell above
        // BYTES: byte a of the row table, sign-replicated into bytes 1-3
        const uint32_t sel = (uint32_t)a + ((uint32_t)a | 8u) * 0x1110u;
        int32_t cm = 0;
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const int32_t i = r0 + r + 1;
          if (!CHECK || i <= m) {
            F = __viaddmax_s32(F, -e, hoa);                  // F = max(F - e, H_above - o)
            E[r] = __viaddmax_s32(E[r], -e, Ho[r]);          // E = max(E - e, H_left - o)
            const int32_t sv = BYTES ? (int32_t)prmt(qv[r], 0u, sel) : (int32_t)So[qv[r] + a];
            const int32_t t = __viaddmax_s32(d, sv, E[r]);   // max(H_diag + S, E)
            int32_t h;
            if (LOCAL) {
              h = __vimax_s32_relu(t, F);
              cm = max(cm, h);
            } else {
              h = max(t, F);
            }
            d = Ho[r];
            Ho[r] = h - o;
            hoa = Ho[r];
          }
        }
        if (LOCAL) {
          // first strictly better cell of this lane in (j, i) order
          if (cm > c.s) {
            int rr = 0;
#pragma unroll
            for (int r = ROWS - 1; r >= 0; --r)
              if (Ho[r] == cm - o) rr = r;
            c = {cm, r0 + rr + 1, j, 1};
          }
        } else if (CHECK) {
          if (j == n) {
            // column n (query end free) or the corner (m, n), rows in order
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
              const int32_t i = r0 + r + 1;
              if (i <= m && (q_end_free || i == m) && (!c.has || Ho[r] + o > c.s)) c = {Ho[r] + o, i, j, 1};
            }
          } else if (t_end_free && owns_m) {
            int32_t hm = Ho[0] + o;
#pragma unroll
            for (int r = 1; r < ROWS; ++r)
              if (r == m - r0 - 1) hm = Ho[r] + o;
            if (!c.has || hm > c.s) c = {hm, m, j, 1};
          }
        }
        sendH = hoa;
        sendF = F;
        if (stores_ck) ck[j - 1] = make_int2(hoa + o, F);
        // the release store orders this lane's own earlier row stores, the
        // only ones the band below reads
        if (stores_bot && ((uint32_t)j % PUBLISH == 0 || j == n)) st_release_u32(my_prog, (uint32_t)j);
      }
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    // Blocks of 32 steps; the steady-state body (every lane on a real
    // column of a full band, no global / semi-global result cell in the
    // block: the lanes' columns s0 - 30 .. s0 + 32 avoid n, and the band does
    // not hold row m with a free target end) is unrolled by 4 only, which
    // keeps it in the instruction cache with 16 warps per SM.
    const bool full = i0 + BAND <= m;
    const bool rowm = !LOCAL && t_end_free && m > i0 && m <= i0 + BAND;
    for (int32_t s0 = 0; s0 < steps; s0 += 32) {
      const int32_t jlo = s0 - 30, jhi = s0 + 32;
      const bool ev = !LOCAL && (rowm || (n >= jlo && n <= jhi));
      if (full && jlo >= 1 && jhi <= n && !ev) {
#pragma unroll 4
        for (int k = 0; k < 32; ++k) step(s0 + 1 + k, k, F_{});
      } else {
#pragma unroll 1
        for (int k = 0; k < 32 && s0 + 1 + k <= steps; ++k) step(s0 + 1 + k, k, T_{});
      }
      // block consumed: rotate, fetch the block after the next
      bcur = bnxt;
      tcur = tnxt;
      bnxt = fetch_bnd(s0 + 64);
      tnxt = fetch_res(s0 + 64);
    }
    // merge the lanes' candidates (each lane's is its first best in (j, i) order)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      Cand x;
      x.s = __shfl_xor_sync(FULL, c.s, off);
      x.i = __shfl_xor_sync(FULL, c.i, off);
      x.j = __shfl_xor_sync(FULL, c.j, off);
      x.has = __shfl_xor_sync(FULL, c.has, off);
      if (cand_better(x, c)) c = x;
    }
    if (lane == 0) cands[jb.cand_off + b] = c;
    __syncwarp();
  }
}

__global__ void k_long_reduce(const LongJob* __restrict__ jobs, uint32_t n_jobs,
                              const Cand* __restrict__ cands, int mode, uint32_t fe, int o, int e,
                              int32_t* __restrict__ o_score, int32_t* __restrict__ o_qend,
                              int32_t* __restrict__ o_tend, uint8_t* __restrict__ o_flag) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n_jobs; k += gridDim.x * blockDim.x) {
    const LongJob jb = jobs[k];
    const int32_t nb = (jb.m + BAND - 1) / BAND;
    Cand best = {0, 0, 0, 0};
    if (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_Q_END))
      best = {h_row0(mode, fe, jb.n, o, e), 0, jb.n, 1};   // H[0][n]
    for (int32_t b = 0; b < nb; ++b) {
      const Cand c = cands[jb.cand_off + b];
      if (cand_better(c, best)) best = c;
    }
    if (mode == DSA_LOCAL && !best.has) {
      o_score[jb.out] = 0; o_qend[jb.out] = -1; o_tend[jb.out] = -1;
    } else {
      o_score[jb.out] = best.s; o_qend[jb.out] = best.i - 1; o_tend[jb.out] = best.j - 1;
    }
    o_flag[jb.out] = 0;
  }
}

struct RevCigar {
  uint32_t* out;
  uint32_t n = 0;
  int op = -1;
  uint32_t run = 0;
  bool writer = true;   // a warp running one walk in every lane stores from one
  __device__ void emit(int o) {
    if (o == op) {
      ++run;
    } else {
      flush();
      op = o;
      run = 1;
    }
  }
  __device__ void emit_run(int o, uint32_t k) {   // k >= 1 ops `o`
    if (o == op) {
      run += k;
    } else {
      flush();
      op = o;
      run = k;
    }
  }
  __device__ void flush() {
    if (run) {
      if (writer) out[n] = (run << 4) | (uint32_t)op;
      ++n;
    }
    run = 0;
  }
};

// Checkpointed traceback, part 1: every band of every hit is recomputed at
// once (one warp per band, rows of the band x columns 1..je), starting from
// the checkpoint row above it, and the 4-bit decision of every cell of the
// rectangle up to the end cell is stored.
// First stored column of the rows of traceback band b (see LongTbJob).
__device__ __forceinline__ int32_t band_jlo(const LongTbJob& jb, int32_t b) {
  const int32_t want = b * TB_BAND + 1 + jb.dlo;
  return max(1, min(want, jb.je - jb.wc + 1));
}
// Band b's stored columns: the per-band window when there is one, else the
// job's diagonal window.
__device__ __forceinline__ void band_window(const LongTbJob& jb, const int2* win, int32_t b,
                                            int32_t& jlo, int32_t& wcb) {
  if (win) {
    const int2 w = win[jb.win_off + (uint32_t)b];
    jlo = w.x;
    wcb = w.y;
  } else {
    jlo = band_jlo(jb, b);
    wcb = jb.wc;
  }
}

template <bool BYTES>
__global__ void __launch_bounds__(WARPS * 32, 3) k_long_tb_fill(
    const uint8_t* __restrict__ qcodes, const uint8_t* __restrict__ tcodes,
    const int8_t* __restrict__ Sg, int A, int o, int e, int mode, uint32_t fe,
    const LongTbJob* __restrict__ jobs, const uint32_t* __restrict__ items, uint32_t n_items,
    const int2* __restrict__ bnd, uint32_t* __restrict__ dir, const int2* __restrict__ win) {
  __shared__ int8_t S[32 * 32];
  __shared__ uint32_t Sb[4];   // BYTES: row q of S as 4 bytes
  for (int x = threadIdx.x; x < A * A; x += blockDim.x) S[x] = Sg[x];
  if (BYTES && threadIdx.x < 4) {
    uint32_t w = 0;
    for (int a = 0; a < A; ++a)
      if ((int)threadIdx.x < A) w |= (uint32_t)(uint8_t)Sg[threadIdx.x * A + a] << (8 * a);
    Sb[threadIdx.x] = w;
  }
  __syncthreads();
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const bool local = mode == DSA_LOCAL;
  const uint32_t warps = gridDim.x * WARPS;
  for (uint32_t it = blockIdx.x * WARPS + (threadIdx.x >> 5); it < n_items; it += warps) {
    const LongTbJob jb = jobs[items[2 * it]];
    const int32_t b = (int32_t)items[2 * it + 1];
    const int32_t ie = jb.ie;
    const uint8_t* q = qcodes + jb.q_start;
    const uint8_t* t = tcodes + jb.t_start;
    uint32_t* D = dir + jb.dir_off;
    const uint32_t wpr = jb.wpr;
    const int32_t i0 = b * TB_BAND;
    const int32_t r0 = i0 + lane * TB_ROWS;
    const int2* up = bnd + jb.bnd_off + (uint64_t)(b - 1) * jb.n;
    // columns jlo .. jlo + wcb - 1 of this band; a wall (-inf) left of jlo > 1
    int32_t jlo, wcb;
    band_window(jb, win, b, jlo, wcb);
    const int32_t jhi = jlo + wcb - 1;
    const bool wall = jlo > 1;
    int32_t H[TB_ROWS], E[TB_ROWS];
    uint32_t nbw[TB_ROWS];
    uint32_t qv[TB_ROWS];   // BYTES: S row of the query residue as bytes; else its matrix offset
#pragma unroll
    for (int r = 0; r < TB_ROWS; ++r) {
      const int32_t ii = r0 + r + 1;
      H[r] = wall ? NEG32 : h_col0(mode, fe, ii, o, e);
      E[r] = NEG32;
      nbw[r] = 0;
      qv[r] = ii <= ie ? (BYTES ? Sb[q[ii - 1]] : (uint32_t)q[ii - 1] * A) : 0u;
    }
    // H[r0][jlo - 1]: for lane 0 the corner (i0, jlo - 1) lies on the window's
    // edge diagonal, inside the band -- the boundary row (band 0) or the
    // checkpoint row gives it; for the other lanes it lies left of the band
    int32_t diag;
    if (!wall) diag = h_col0(mode, fe, r0, o, e);
    else if (lane != 0) diag = NEG32;
    else if (b == 0) diag = h_row0(mode, fe, jlo - 1, o, e);
    else diag = up[jlo - 2].x;
    int32_t sendH = 0, sendF = NEG32;
    int sendA = 0;
    // checkpoint row above and target residues for columns jlo + blk .. + 31
    // (lane k: column jlo + blk + k), fetched by the warp one block ahead
    auto fetch_up = [&](int32_t blk) -> int2 {
      const int32_t jj = jlo + blk + lane;
      return (b > 0 && jj <= jhi) ? up[jj - 1] : make_int2(NEG32, NEG32);
    };
    auto fetch_res = [&](int32_t blk) -> int {
      const int32_t jj = jlo + blk + lane;
      return jj <= jhi ? (int)t[jj - 1] : 0;
    };
    int2 ucur = fetch_up(0), unxt = fetch_up(32);
    int tcur = fetch_res(0), tnxt = fetch_res(32);
    // One step (k = (s - 1) mod 32).  FAST: every lane on a stored column
    // of a band whose rows are all real, and no lane at the window's last
    // column: no bounds tests.
    auto step = [&](int32_t s, int k, auto fast_c) {
      constexpr bool FAST = decltype(fast_c)::value;
      const int32_t ux = __shfl_sync(FULL, ucur.x, k);
      const int32_t uy = __shfl_sync(FULL, ucur.y, k);
      const int ta = __shfl_sync(FULL, tcur, k);
      int32_t Hup = __shfl_up_sync(FULL, sendH, 1);
      int32_t Fup = __shfl_up_sync(FULL, sendF, 1);
      int a = __shfl_up_sync(FULL, sendA, 1);
      const int32_t jj = jlo - 1 + s - lane;
      // lane 0 reads the checkpoint row above (or row 0): selects, not a branch
      const int32_t h0 = b == 0 ? h_row0(mode, fe, jj, o, e) : ux;
      const int32_t f0 = b == 0 ? NEG32 : uy;
      Hup = lane == 0 ? h0 : Hup;
      Fup = lane == 0 ? f0 : Fup;
      a = lane == 0 ? ta : a;
      sendA = a;
      if (FAST || (jj >= jlo && jj <= jhi && r0 < ie)) {
        int32_t d = diag;
        diag = Hup;
        int32_t F = Fup, Hp = Hup;
        const uint32_t sel = (uint32_t)a + ((uint32_t)a | 8u) * 0x1110u;
        const int32_t jc = jj - jlo;   // stored column
        const int sh = 4 * (jc & 7);
        const bool flushw = ((jc & 7) == 7) || (!FAST && jj == jhi);
#pragma unroll
        for (int r = 0; r < TB_ROWS; ++r) {
          const int32_t ii = r0 + r + 1;
          if (FAST || ii <= ie) {
            // each maximum also yields its decision (first operand >= second,
            // one DPX instruction): a gap opens here on ties, M comes before
            // the gaps and I before D
            bool pf, pe, pg, pm;
            F = __vibmax_s32(Hp - o, F - e, &pf);
            E[r] = __vibmax_s32(H[r] - o, E[r] - e, &pe);
            const int32_t sv = BYTES ? (int32_t)prmt(qv[r], 0u, sel) : (int32_t)S[qv[r] + a];
            const int32_t mm = d + sv;
            const int32_t g = __vibmax_s32(F, E[r], &pg);
            int32_t v = __vibmax_s32(mm, g, &pm);
            uint32_t src = pm ? 1u : (pg ? 2u : 0u);
            if (local && v <= 0) {   // the empty alignment: stop
              v = 0;
              src = 3u;
            }
            nbw[r] |= (src | (pe ? 4u : 0u) | (pf ? 8u : 0u)) << sh;
            if (flushw) {
              D[((uint64_t)b * wpr + (uint32_t)jc / 8u) * TB_BAND + (uint32_t)(ii - 1 - i0)] = nbw[r];
              nbw[r] = 0;
            }
            d = H[r];
            H[r] = v;
            Hp = v;
          }
        }
        sendH = Hp;
        sendF = F;
      }
    };
    // Blocks of 32 steps; the steady-state body is unrolled by 4 only (the
    // instruction cache).  Lanes' stored columns in block s0: s0 - 31 ..
    // s0 + 31 (jc); steady when all lie in 0 .. wc - 2 and the band is full.
    const bool full = i0 + TB_BAND <= ie;
    const int32_t steps = wcb + 31;
    for (int32_t s0 = 0; s0 < steps; s0 += 32) {
      if (full && s0 >= 32 && s0 + 32 < wcb) {
#pragma unroll 4
        for (int k = 0; k < 32; ++k) step(s0 + 1 + k, k, std::true_type{});
      } else {
#pragma unroll 1
        for (int k = 0; k < 32 && s0 + 1 + k <= steps; ++k) step(s0 + 1 + k, k, std::false_type{});
      }
      // block consumed: rotate, fetch the block after the next
      ucur = unxt;
      tcur = tnxt;
      unxt = fetch_up(s0 + 64);
      tnxt = fetch_res(s0 + 64);
    }
    __syncwarp();
  }
}

// Checkpointed traceback, part 0: the window of each band from the
// checkpoint rows.  An optimal path to the hit (ie, je) with score `best`
// crosses row R at a column c only if H(R, c) plus the most any path from
// (R, c) to (ie, je) can still score reaches best; that most is
// max(S, 0) min(ie - R, je - c) minus e for each diagonal step between the
// two cells' diagonals (a gap cell costs at least e).  H at a checkpoint row
// is exact, so the columns passing this test at a band's top row bound the
// band's path from the left and those at its bottom row from the right (the
// path only moves down and right), within the job's diagonal window, which
// already contains every optimal path.  A path may also begin inside the
// band: local alignment (from any cell whose remaining reach covers best:
// the leftmost such column is largest-distance from the end, at the band's
// top row) and a free query begin (column 0); those bands widen to include
// them.  Every cell of every optimal path keeps its exact value in the
// narrowed band, so the decisions along them are the full matrix's.
__global__ void __launch_bounds__(128) k_long_tb_windows(
    const LongTbJob* __restrict__ jobs, const uint32_t* __restrict__ items, uint32_t n_items,
    const int2* __restrict__ bnd, const dsa_hit* __restrict__ hits, int mode, uint32_t fe,
    int o, int e, int smax_pos, int2* __restrict__ win, int32_t* __restrict__ maxw) {
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const uint32_t it = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (it >= n_items) return;
  const uint32_t job = items[2 * it];
  const LongTbJob jb = jobs[job];
  const int32_t b = (int32_t)items[2 * it + 1];
  const int64_t best = hits[jb.hit].score;
  const int64_t ie = jb.ie, je = jb.je;
  // the job's diagonal window for this band: no optimal path leaves it
  const int32_t olo = band_jlo(jb, b), ohi = olo + jb.wc - 1;
  auto reach = [&](int64_t R, int64_t c) -> int64_t {   // best score from (R, c) to the end
    const int64_t dr = ie - R, dc = je - c;
    const int64_t d = dr > dc ? dr - dc : dc - dr;
    return (int64_t)smax_pos * (dr < dc ? dr : dc) - d * e;
  };
  auto h_at = [&](int64_t R, int64_t c) -> int64_t {   // exact H on row R (0 or a checkpoint row)
    if (R == 0) return h_row0(mode, fe, c, o, e);
    if (c == 0) return h_col0(mode, fe, R, o, e);
    return bnd[jb.bnd_off + (uint64_t)(R / TB_BAND - 1) * (uint32_t)jb.n + (uint64_t)(c - 1)].x;
  };
  const int64_t Rt = (int64_t)b * TB_BAND, Rb = Rt + TB_BAND;
  // left bound: crossings of the top row
  int64_t lo = INT64_MAX;
  const int64_t c0 = olo > 1 ? (int64_t)olo - 1 : 0;
  for (int64_t c = c0 + lane; c <= ohi; c += 32)
    if (h_at(Rt, c) + reach(Rt, c) >= best) { lo = c; break; }
  // paths that begin inside the band
  if (e > 0 && mode == DSA_LOCAL) {
    const int64_t dr = ie - Rt;
    if ((int64_t)smax_pos * dr >= best) {
      const int64_t cs = je - dr - ((int64_t)smax_pos * dr - best) / e;
      lo = min(lo, cs > 0 ? cs : (int64_t)0);
    }
  } else if (e == 0 && mode == DSA_LOCAL) {
    lo = 0;
  }
  if (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_Q_BEGIN)) {
    const int64_t rm = min(max(ie - je, Rt), min(Rb, ie));   // the best row for a column-0 start
    if (reach(Rt, 0) >= best || reach(rm, 0) >= best) lo = 0;
  }
  // right bound: crossings of the bottom row (the end cell in the last band)
  int64_t hi = -1;
  if (Rb >= ie) {
    hi = je;
  } else {
    for (int64_t c = ohi - lane; c >= c0; c -= 32)
      if (h_at(Rb, c) + reach(Rb, c) >= best) { hi = c; break; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo = min(lo, (int64_t)__shfl_xor_sync(FULL, (long long)lo, off));
    hi = max(hi, (int64_t)__shfl_xor_sync(FULL, (long long)hi, off));
  }
  if (lane == 0) {
    int32_t jlo = (int32_t)max(max(lo, (int64_t)olo), (int64_t)1);
    int32_t jhi = (int32_t)min(hi, (int64_t)ohi);
    if (lo == INT64_MAX || hi < 0 || jhi < jlo) {   // no narrower window found
      jlo = olo;
      jhi = ohi;
    }
    win[jb.win_off + (uint32_t)b] = make_int2(jlo, jhi - jlo + 1);
    atomicMax(maxw + job, jhi - jlo + 1);
  }
}

// Checkpointed traceback, part 2: one warp per hit.  Every lane runs the
// same walk over the stored decisions from the end cell (stop > M > I > D,
// open preferred on ties), lane 0 storing the CIGAR; a match run is tested
// 32 diagonal cells at a time, lane k reading the k-th, by one ballot.  The
// warp keeps a window of them in shared memory -- up to WIN_ROWS rows of the
// current band ending at the walk's row, WIN_WORDS words (8 cells each)
// ending at the walk's column -- and reloads it with coalesced row loads
// whenever the walk leaves it (the walk only moves up and left), so each step
// reads shared memory instead of waiting on a global load.
constexpr int WIN_WORDS = 32;
constexpr int WIN_ROWS = 256;   // a window word's rows are consecutive (as in global memory)

__global__ void __launch_bounds__(32) k_long_tb_walk(const LongTbJob* __restrict__ jobs,
                                                     uint32_t n_jobs, int mode, uint32_t fe,
                                                     const uint32_t* __restrict__ dir,
                                                     uint32_t* __restrict__ cig_tmp,
                                                     dsa_hit* __restrict__ hits,
                                                     const int2* __restrict__ bwin) {
  __shared__ __align__(16) uint32_t win[WIN_WORDS * WIN_ROWS];
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x;
  const bool local = mode == DSA_LOCAL;
  const bool sg = mode == DSA_SEMIGLOBAL;
  for (uint32_t k = blockIdx.x; k < n_jobs; k += gridDim.x) {
    const LongTbJob jb = jobs[k];
    const uint32_t* D = dir + jb.dir_off;
    const uint32_t wpr = jb.wpr;
    int32_t wb = -1, wlo = 0, wr0 = 0, wr1 = 0;   // window: band, first word, rows [wr0, wr1)
    RevCigar c;
    c.out = cig_tmp + jb.cig_off;
    c.writer = lane == 0;
    int32_t i = jb.ie, j = jb.je;
    int st = 0;
    int64_t guard = 2 * ((int64_t)jb.ie + jb.je) + 2;
    // the walk's cell as (row in band wb, stored column of that band),
    // valid once a reload has placed the window around it.  The walk only
    // moves up and left, so only the window's lower bounds can be crossed;
    // crossing one (a new band included: its rows start at 0) reloads.
    int32_t rr = -1, jc = -1;
    for (;;) {
      int need = 2;   // 1: reload the window around (i, j); 2: finished
      {
        for (; guard > 0; --guard) {
          if (st == 0) {
            if (sg && ((i == 0 && (fe & DSA_FREE_T_BEGIN)) || (j == 0 && (fe & DSA_FREE_Q_BEGIN)))) break;
            if (i == 0 || j == 0) {
              if (!local) {
                while (j > 0) { c.emit(2); --j; }
                while (i > 0) { c.emit(1); --i; }
              }
              break;
            }
          } else if (i <= 0 || j <= 0) {
            break;
          }
          if (rr < wr0 || (jc >> 3) < wlo) { need = 1; break; }
          // Every step moves up, left or both by one, so the next `safe`
          // moves stay inside the window and off row 0 and column 0: take
          // them with no tests, stepping the window address and the
          // nibble's shift along.  A switch from H to a gap state reads the
          // same cell's open bit, so it is taken in the same step.
          const int32_t safe = min(min(rr - wr0, jc - 8 * wlo), min(i - 1, j - 1));
          const uint32_t* p = win + ((jc >> 3) - wlo) * WIN_ROWS + (rr - wr0);
          uint32_t sh = 4u * (uint32_t)(jc & 7);
          bool stop = false;
          int32_t q = 0;
          for (; q <= safe; ++q) {
            if (st == 0 && q + 31 <= safe) {
              // a match run: the next 32 cells along the diagonal lie in the
              // window; lane k reads the k-th, and the leading M steps are
              // taken together
              const int32_t jk = jc - lane;
              const uint32_t w = win[((jk >> 3) - wlo) * WIN_ROWS + (rr - lane - wr0)];
              const uint32_t notm = __ballot_sync(FULL, ((w >> (4 * (jk & 7))) & 3u) != 1u);
              const int32_t L = notm ? __ffs(notm) - 1 : 32;
              if (L > 0) {
                c.emit_run(0, (uint32_t)L);
                i -= L; j -= L; rr -= L; jc -= L;
                q += L - 1;
                p = win + ((jc >> 3) - wlo) * WIN_ROWS + (rr - wr0);
                sh = 4u * (uint32_t)(jc & 7);
                continue;
              }
            }
            const uint32_t nib = (*p >> sh) & 15u;
            if (st == 0) {
              const uint32_t src = nib & 3u;
              if (src == 3) { stop = true; break; }
              if (src == 1) {   // M: up and left
                c.emit(0);
                p -= 1 + (sh == 0 ? WIN_ROWS : 0);
                sh = (sh - 4u) & 31u;
                --i; --j; --rr; --jc;
                continue;
              }
              st = src == 2 ? 1 : 2;   // 1: I (F state), 2: D (E state)
            }
            if (st == 1) {   // I: up
              c.emit(1);
              if (nib & 8u) st = 0;
              p -= 1;
              --i; --rr;
            } else {         // D: left
              c.emit(2);
              if (nib & 4u) st = 0;
              p -= (sh == 0 ? WIN_ROWS : 0);
              sh = (sh - 4u) & 31u;
              --j; --jc;
            }
          }
          guard -= q;
          if (stop) break;
        }
      }
      if (need != 1) break;
      // reload: rows of (i, j)'s band ending at row i, words ending at j's word;
      // a cell left of the band's stored columns ends the walk (only a corrupt
      // decision leads there)
      const int32_t ci = __shfl_sync(FULL, i, 0), cj = __shfl_sync(FULL, j, 0);
      wb = (ci - 1) / TB_BAND;
      int32_t jlo, wcb;
      band_window(jb, bwin, wb, jlo, wcb);
      if (cj < jlo || cj >= jlo + wcb) break;
      const int32_t wi = (cj - jlo) >> 3;
      wlo = max(0, wi - (WIN_WORDS - 1));
      wr1 = ci - wb * TB_BAND;
      rr = wr1 - 1;
      // rows from a multiple of 4 (16-byte copies), ending at or after the
      // walk's row
      const int32_t wr1a = min((wr1 + 3) & ~3, TB_BAND);
      wr0 = max(0, wr1a - WIN_ROWS);
      jc = cj - jlo;
      __syncwarp();
      // words wlo .. wlo + 31 of rows wr0 .. wr1a - 1 of band wb: each
      // word's rows are consecutive in the decision layout and in the window,
      // so the warp copies 16-byte pieces (4 rows), every copy in flight at
      // once: a reload costs about one memory latency
      {
        const uint32_t* Db = D + (uint64_t)wb * wpr * TB_BAND;
        const int32_t n4 = (wr1a - wr0) >> 2;
#pragma unroll 4
        for (int k = 0; k < WIN_WORDS; ++k) {
          const int32_t w = wlo + k;
          for (int c = lane; c < n4; c += 32) {
            uint32_t* dst = win + k * WIN_ROWS + 4 * c;
            if (w < (int32_t)wpr) cp_async16(dst, Db + (uint64_t)w * TB_BAND + (uint32_t)(wr0 + 4 * c));
            else *reinterpret_cast<uint4*>(dst) = make_uint4(0u, 0u, 0u, 0u);
          }
        }
      }
      cp_async_commit();
      cp_async_wait<0>();
      __syncwarp();
    }
    if (lane == 0) {
      c.flush();
      dsa_hit* h = hits + jb.hit;
      h->q_begin = i;
      h->t_begin = j;
      h->cigar_len = c.n;
      h->flags |= DSA_HIT_HAS_TRACEBACK;
    }
    __syncwarp();
  }
}

}  // namespace

int launch_long_score(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int8_t* d_matrix,
                      int A, int o, int e, int mode, uint32_t fe, bool bytes_ok,
                      const LongJob* d_jobs, uint32_t n_jobs, const uint32_t* d_items,
                      uint32_t n_items, int2* d_bnd, uint32_t* d_prog, void* d_cands, Scores out,
                      int blocks_per_sm) {
  if (n_items == 0) return DSA_OK;
  // every warp must be resident at once (bands wait on their predecessors):
  // the grid never exceeds what the device holds simultaneously
  // alphabets of up to 4 letters with every S + o in int8: substitution
  // scores by byte permute
  const bool bytes = A <= 4 && bytes_ok;
  auto kern = mode == DSA_LOCAL ? (bytes ? k_long_score<true, true> : k_long_score<true, false>)
                                : (bytes ? k_long_score<false, true> : k_long_score<false, false>);
  int per_sm = 0;
  DSA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, 0));
  if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);
  const uint64_t resident = (uint64_t)std::max(1, per_sm) * ctx->sm_count;
  const unsigned grid = (unsigned)std::min<uint64_t>(resident, (n_items + WARPS - 1) / WARPS);
  uint32_t* counter = ctx->d_counters + 3;
  DSA_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(uint32_t), ctx->stream));
  kern<<<grid, WARPS * 32, 0, ctx->stream>>>(qs->d_codes, db->d_codes, d_matrix, A, o, e, mode, fe,
                                              d_jobs, d_items, n_items, counter, d_bnd, d_prog,
                                              static_cast<Cand*>(d_cands), ctx->d_status);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return launch_long_reduce(ctx, d_jobs, n_jobs, d_cands, mode, fe, o, e, out);
}

int launch_long_reduce(dsa_ctx* ctx, const LongJob* d_jobs, uint32_t n_jobs, const void* d_cands,
                       int mode, uint32_t fe, int o, int e, Scores out) {
  const unsigned rb = (unsigned)std::min<uint64_t>((n_jobs + 127) / 128, 1024);
  k_long_reduce<<<rb, 128, 0, ctx->stream>>>(d_jobs, n_jobs, static_cast<const Cand*>(d_cands),
                                              mode, fe, o, e, out.score, out.q_end, out.t_end,
                                              out.flag);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

size_t long_cand_size() { return sizeof(Cand); }
int long_band_rows() { return BAND; }
int long_ckpt_rows() { return TB_BAND; }

int launch_long_tb_fill(dsa_ctx* ctx, cudaStream_t stream, const dsa_db* db, const dsa_db* qs,
                        const int8_t* d_matrix, int A, int o, int e, int mode, uint32_t fe,
                        const LongTbJob* d_jobs, const uint32_t* d_items, uint32_t n_items,
                        const int2* d_bnd, uint32_t* d_dir, const int2* d_win) {
  if (n_items == 0) return DSA_OK;
  const unsigned grid = (unsigned)std::min<uint64_t>((n_items + WARPS - 1) / WARPS,
                                                     (uint64_t)ctx->sm_count * 16);
  auto fill = A <= 4 ? k_long_tb_fill<true> : k_long_tb_fill<false>;
  fill<<<grid, WARPS * 32, 0, stream>>>(qs->d_codes, db->d_codes, d_matrix, A, o, e, mode, fe,
                                        d_jobs, d_items, n_items, d_bnd, d_dir, d_win);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_long_tb_windows(dsa_ctx* ctx, cudaStream_t stream, const LongTbJob* d_jobs,
                           const uint32_t* d_items, uint32_t n_items, const int2* d_bnd,
                           const dsa_hit* d_hits, int mode, uint32_t fe, int o, int e,
                           int smax_pos, int2* d_win, int32_t* d_maxw) {
  if (n_items == 0) return DSA_OK;
  k_long_tb_windows<<<(n_items + 3) / 4, 128, 0, stream>>>(d_jobs, d_items, n_items, d_bnd, d_hits,
                                                           mode, fe, o, e, smax_pos, d_win, d_maxw);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_long_tb_walk(dsa_ctx* ctx, cudaStream_t stream, const LongTbJob* d_jobs,
                        uint32_t n_jobs, int mode, uint32_t fe, const uint32_t* d_dir,
                        uint32_t* d_cig_tmp, dsa_hit* d_hits, const int2* d_win) {
  if (n_jobs == 0) return DSA_OK;
  k_long_tb_walk<<<n_jobs, 32, 0, stream>>>(d_jobs, n_jobs, mode, fe, d_dir, d_cig_tmp, d_hits,
                                            d_win);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

}  // namespace dsa
