// Long explicit pairs, packed int16x2 score pass (DNW / DSG of Sec. II.C.2
// for pairs of 1e4-1e5 residues, the score pass of the map phase of
// Sec. II.B.1): the band pipeline of the int32 kernel with two pairs per
// warp, one in each 16-bit half of every register.
//
// Layout.  A unit is two long pairs (sorted neighbours by query length);
// band b of the unit covers rows 512b+1 .. 512b+512 of both, lane k owns 16
// of those rows and processes column j = step - k.  The unit runs max(nA,
// nB) columns and max(bands) bands; rows past a pair's end and columns past
// its window are computed in its half but never read for it (the half's
// results and checkpoints are taken from its own rows and columns only, and
// a real cell depends on no cell below or right of it).
//
// Values relative to a moving base.  Scores of a long pair reach far past
// int16, but neighbouring cells differ little: with D = o + max(S, 0),
// |H(i,j) - H(i,j-1)| <= D and |H(i,j) - H(i-1,j)| <= D (a gap of one costs
// o; a step that raises H is a diagonal or a gap from a neighbour that is at
// most D below), and E, F lie within o + D below H.  So every value a warp
// holds is kept as (value - base) with one absolute int32 base per half,
// common to all lanes.  Every 32 steps (while lane 0 is on a real column of
// the half) the base moves to the H of lane 0's first row; all cells a warp
// touches until the next move lie within 512 + 64 rows and columns of that
// cell (512 + 96 for the local locate pass below, which runs up to 64 steps
// past a block start without moving the base), so a relative value is
// bounded by 608 D + 2o + e + |min S| + 64, which long16_range_ok checks
// against 2^15 on the host (no rerun is ever needed).  Lane 0's input row
// (the band above, or row 0) is converted from absolute int32 once per 32
// columns; the checkpoint rows (the middle and
// the bottom row of the band, absolute int2 per pair, the same layout the
// int32 kernel writes and the traceback reads) collect in a shared-memory
// ring and are converted and stored by the whole warp every 32 steps, before
// the base moves, and the band below is told by a release store.
//
// Halves are offset binary (value + 2^15), so H - o is one 32-bit subtract
// without a borrow between the halves while both are in range; halves
// outside their pair are reset to the relative 0 every 32 steps to keep it
// so.  Cell update per register (2 cells): E = max(E - e, Ho_left),
// t = max(Ho_diag + (S + o), E), Ho = max(F - o, t - o) (= H - o with
// H = max(t, F)), and the next row's F = max(F - e, t - o) (equal to
// max(F - e, H - o) because e <= o), one operation per row on the F chain.
//
// Local (the DSW of Sec. II.C.2).  The floor 0 of local alignment enters as
// t - o = max(t - o, floor - o) with the relative floor per half (one addmax
// per register); a pair's local result is the first cell, in (column, row)
// order, holding the maximum of its matrix.  Tracking that cell on every improvement costs more than the
// packing gains (along a strong diagonal a lane's best rises on about a
// quarter of the steps), so the score pass keeps only a per-register
// running maximum over each 32-step block, reduced across the warp at the
// block end; when the block raises a band's best, the warp's state at the
// block start (saved in shared memory) goes to the band's slot in global
// memory.  A second kernel then takes, for every band whose best equals the
// pair's maximum, the saved state of the first block that reached it and
// reruns that block (and the next one, for lanes whose columns lag the
// block's steps) to find the first cell holding the maximum; the int32
// reduction then picks the first band's cell.
#include "dsa_internal.cuh"
#include "dpx.cuh"

#include <type_traits>

namespace dsa {
namespace {

constexpr int ROWS = 16;
constexpr int BAND = 32 * ROWS;
constexpr int TB_BAND = BAND / 2;   // checkpoint spacing
constexpr int WARPS = 4;
constexpr uint32_t JUNK_S = 0x80808080u;   // S + o = -128 for every residue: rows past a pair's end
// LOCAL: a lane's state at a block start (Ho, E of its rows, diag, and the H - o
// and F it hands down)
constexpr int SNAP_WORDS = 2 * ROWS + 3;

// LOCAL: a band's best cell value of one pair, and where to look for it:
// the start (step) of the first block in which the band's running maximum
// reached it, the relative base and the half of the packed state, whose
// snapshot at that block start is kept in the pair's band slot
struct LongBest {
  int32_t best;
  int32_t s0;
  int32_t base;
  int32_t half;
};

__device__ __forceinline__ int32_t h_row0(int mode, uint32_t fe, int64_t j, int o, int e) {
  if (j == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_T_BEGIN))) return 0;
  return -(o + (int32_t)(j - 1) * e);
}
__device__ __forceinline__ int32_t h_col0(int mode, uint32_t fe, int64_t i, int o, int e) {
  if (i == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_Q_BEGIN))) return 0;
  return -(o + (int32_t)(i - 1) * e);
}
__device__ __forceinline__ bool better(const LongCand& a, const LongCand& b) {
  if (!a.has) return false;
  if (!b.has) return true;
  if (a.s != b.s) return a.s > b.s;
  if (a.j != b.j) return a.j < b.j;
  return a.i < b.i;
}
constexpr uint32_t BIAS2 = 0x80008000u;   // offset binary: a half holds value + 2^15
__device__ __forceinline__ uint32_t bias2(int32_t lo, int32_t hi) { return pack2(lo, hi) ^ BIAS2; }
// the value of half `x` of an offset-binary register
__device__ __forceinline__ int32_t half(uint32_t v, int x) { return x ? hi16(v ^ BIAS2) : lo16(v ^ BIAS2); }

// MINB: the blocks per SM the build keeps resident.  The local form's
// running maxima and block-start state need more than the 128 registers of
// 4 blocks per SM (it spilled there); at 3 it takes 156.  The global form is
// built for 4 blocks (128 registers) and for 2 (198: the steady-state body
// scheduled with more registers ran 2% faster on the 64 long pairs), the
// local form for 3 and 2; the blocks-per-SM choice picks the build.
template <bool LOCAL, int MINB>
__global__ void __launch_bounds__(WARPS * 32, MINB) k_long_score16(
    const uint8_t* __restrict__ qcodes, const uint8_t* __restrict__ tcodes,
    const int8_t* __restrict__ Sg, int A, int o, int e, int mode, uint32_t fe,
    const LongJob* __restrict__ jobs, const LongPair16* __restrict__ pjobs,
    const uint32_t* __restrict__ items, uint32_t n_items, uint32_t* __restrict__ counter,
    int2* __restrict__ bnd, uint32_t* __restrict__ prog, LongCand* __restrict__ cands,
    int32_t* __restrict__ status, LongBest* __restrict__ lbest, uint32_t* __restrict__ lsnap) {
  __shared__ uint32_t Sb[4];                 // row q of S + o as 4 bytes
  __shared__ uint2 ring[WARPS][2][32];       // per warp: middle (lane 15) and bottom (lane 31) rows
  // LOCAL: the warp's state at the current block's start (word-major)
  __shared__ uint32_t snap[LOCAL ? WARPS : 1][LOCAL ? SNAP_WORDS : 1][32];
  // per thread and half: the lane's candidate (score, i, j, has)
  __shared__ int32_t c_s[2][WARPS * 32], c_i[2][WARPS * 32], c_j[2][WARPS * 32], c_h[2][WARPS * 32];
  const int tid = threadIdx.x;
  if (threadIdx.x < 4) {
    uint32_t w = 0;
    if ((int)threadIdx.x < A)
      for (int a = 0; a < A; ++a)
        w |= (uint32_t)(uint8_t)(int8_t)(Sg[threadIdx.x * A + a] + o) << (8 * a);
    Sb[threadIdx.x] = w;
  }
  __syncthreads();
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool sg = mode == DSA_SEMIGLOBAL;
  const bool q_end_free = sg && (fe & DSA_FREE_Q_END);
  const bool t_end_free = sg && (fe & DSA_FREE_T_END);
  const uint32_t neg_o2 = pack2(-o, -o), neg_e2 = pack2(-e, -e);
  const uint32_t o2 = ((uint32_t)o << 16) | (uint32_t)o;
  bool timed_out = false;

  for (;;) {
    uint32_t it = 0;
    if (lane == 0) it = atomicAdd(counter, 1u);
    it = __shfl_sync(FULL, it, 0);
    if (it >= n_items) break;
    const LongPair16 pj = pjobs[items[2 * it]];
    const uint32_t b = items[2 * it + 1];
    const bool hasB = pj.b != NONE;
    const LongJob JA = jobs[pj.a];
    const LongJob JB = jobs[hasB ? pj.b : pj.a];
    const int32_t mA = JA.m, nA = JA.n;
    const int32_t mB = hasB ? JB.m : 0, nB = hasB ? JB.n : 0;
    const int32_t n = max(nA, nB);
    const int32_t i0 = (int32_t)b * BAND;
    const int32_t r0 = i0 + lane * ROWS;   // rows r0+1 .. r0+16
    const bool inA = i0 < mA, inB = i0 < mB;   // the band holds rows of the pair
    const int32_t nbA = (mA + BAND - 1) / BAND, nbB = (mB + BAND - 1) / BAND;
    const uint8_t* qA = qcodes + JA.q_start;
    const uint8_t* qB = qcodes + JB.q_start;
    const uint8_t* tA = tcodes + JA.t_start;
    const uint8_t* tB = tcodes + JB.t_start;
    // checkpoint rows written by this band: middle (row i0 + 256) and bottom
    // (row i0 + 512, the next band's input)
    const bool midA = inA && mA > i0 + TB_BAND, midB = inB && mB > i0 + TB_BAND;
    const bool botA = inA && (int32_t)b < nbA - 1, botB = inB && (int32_t)b < nbB - 1;
    int2* const ckA = bnd + JA.bnd_off + (uint64_t)(2 * b) * (uint32_t)nA;   // + nA: bottom row
    int2* const ckB = bnd + JB.bnd_off + (uint64_t)(2 * b) * (uint32_t)nB;
    const int2* const upA = (b > 0 && inA) ? bnd + JA.bnd_off + (uint64_t)(2 * b - 1) * (uint32_t)nA : nullptr;
    const int2* const upB = (b > 0 && inB) ? bnd + JB.bnd_off + (uint64_t)(2 * b - 1) * (uint32_t)nB : nullptr;
    uint32_t* const my_prog = prog + pj.prog_off + b;
    const uint32_t* const up_prog = prog + pj.prog_off + b - 1;

    // bases and the lane's rows at column 0
    int32_t baseA = h_col0(mode, fe, i0 + 1, o, e), baseB = baseA;
    uint32_t Ho[ROWS], E[ROWS], sA[ROWS], sB[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int32_t i = r0 + r + 1;
      const int32_t hc = h_col0(mode, fe, i, o, e) - o - baseA;
      Ho[r] = bias2(hc, hc);
      E[r] = Ho[r];   // E(i, 0) = H(i, 0) - o leaves E(i, 1) unchanged
      sA[r] = i <= mA ? Sb[qA[i - 1]] : JUNK_S;
      sB[r] = i <= mB ? Sb[qB[i - 1]] : JUNK_S;
    }
    const int32_t hd = h_col0(mode, fe, r0, o, e) - o - baseA;
    uint32_t diag = bias2(hd, hd);
    uint32_t sendH = 0, sendF = 0, sendS = 0;
    const bool ownA = inA && r0 < mA && mA <= r0 + ROWS;   // the lane holds row mA
    const bool ownB = inB && r0 < mB && mB <= r0 + ROWS;
    auto cand_set = [&](int x, int32_t sc, int32_t i, int32_t j) {
      c_s[x][tid] = sc; c_i[x][tid] = i; c_j[x][tid] = j; c_h[x][tid] = 1;
    };
#pragma unroll
    for (int x = 0; x < 2; ++x) { c_s[x][tid] = 0; c_i[x][tid] = 0; c_j[x][tid] = 0; c_h[x][tid] = 0; }
    if (!LOCAL && t_end_free) {   // H[m][0] on row m
      if (ownA) cand_set(0, h_col0(mode, fe, mA, o, e), mA, 0);
      if (ownB) cand_set(1, h_col0(mode, fe, mB, o, e), mB, 0);
    }
    // LOCAL: the relative 0 as H - o per half (0: out of range, never the
    // maximum), the column maxima of the block, and each half's best so far
    // (absolute) with the block and base of its first appearance
    uint32_t z2o = 0, bmax2 = 0;
    int32_t bestA = 0, bestB = 0, bs0A = 0, bs0B = 0, bbaseA = 0, bbaseB = 0;
    auto set_floor = [&]() {
      const uint32_t zl = -baseA - o >= -32768 ? (uint32_t)(-baseA - o + 32768) & 0xFFFFu : 0u;
      const uint32_t zh = -baseB - o >= -32768 ? (uint32_t)(-baseB - o + 32768) & 0xFFFFu : 0u;
      z2o = zl | (zh << 16);
    };

    // bounded wait until the band above has published `need` columns
    auto wait_for = [&](uint32_t need) {
      bool late = false;
      if (!timed_out) {
        const uint64_t t0 = global_ns();
        uint32_t nap = 32;
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
    // lane 0's input row for columns blk+1 .. blk+32 (lane k: column blk+k+1),
    // (H - o, F) of the row above per half, relative to the current base
    // (the pending blocks move with the base): the band above, or row 0
    // (whose F is taken as H - o, so that row 1's F is H(0, j) - o)
    auto fetch_in = [&](int32_t blk) -> uint2 {
      const int32_t jj = blk + lane + 1;
      // a column outside a half's pair gets the relative 0 (see the reset)
      int32_t ha = o + baseA, fa = baseA, hb = o + baseB, fb = baseB;
      if (b == 0) {
        const int32_t h = h_row0(mode, fe, jj, o, e);
        if (inA && jj <= nA) { ha = h; fa = h - o; }
        if (inB && jj <= nB) { hb = h; fb = h - o; }
      } else {
        if (blk < n) wait_for((uint32_t)min(blk + 32, n));
        if (upA && jj <= nA) {
          const int2 x = upA[jj - 1];
          ha = x.x; fa = x.y;
        }
        if (upB && jj <= nB) {
          const int2 x = upB[jj - 1];
          hb = x.x; fb = x.y;
        }
      }
      return make_uint2(bias2(ha - o - baseA, hb - o - baseB), bias2(fa - baseA, fb - baseB));
    };
    // byte-permute selector of the column's two residues (bytes a_lo of the
    // low row table and 4 + a_hi of the high one, each sign-replicated)
    auto fetch_sel = [&](int32_t blk) -> uint32_t {
      const int32_t jj = blk + lane + 1;
      const uint32_t aa = jj <= nA ? tA[jj - 1] : 0u;
      const uint32_t ab = jj <= nB ? tB[jj - 1] : 0u;
      return (aa * 0x11u + 0x80u) | ((ab * 0x11u + 0xC4u) << 8);
    };
    uint2 incur = fetch_in(0), innxt = fetch_in(32);
    uint32_t selcur = fetch_sel(0), selnxt = fetch_sel(32);

    // checkpoint ring: columns (f31, ..] of lane 31 and (f15, ..] of lane 15
    // are pending; flushed with the base they were computed under
    int32_t f31 = 0, f15 = 0;
    auto flush = [&](int32_t upto31, int32_t upto15) {
      __syncwarp();
      const int32_t jb = f31 + 1 + lane;
      if (jb <= upto31) {
        const uint2 v = ring[wid][1][jb & 31];
        if (botA && jb <= nA)
          ckA[(uint32_t)nA + jb - 1] = make_int2(half(v.x, 0) + o + baseA, half(v.y, 0) + baseA);
        if (botB && jb <= nB)
          ckB[(uint32_t)nB + jb - 1] = make_int2(half(v.x, 1) + o + baseB, half(v.y, 1) + baseB);
      }
      const int32_t jm = f15 + 1 + lane;
      if (jm <= upto15) {
        const uint2 v = ring[wid][0][jm & 31];
        if (midA && jm <= nA) ckA[jm - 1] = make_int2(half(v.x, 0) + o + baseA, half(v.y, 0) + baseA);
        if (midB && jm <= nB) ckB[jm - 1] = make_int2(half(v.x, 1) + o + baseB, half(v.y, 1) + baseB);
      }
      __threadfence();
      __syncwarp();
      f31 = upto31;
      f15 = upto15;
      if (lane == 0 && (botA || botB)) st_release_u32(my_prog, (uint32_t)upto31);
    };

    // One step: column j = s - lane of the lane's rows.  FAST: every lane
    // is on a real column and no result cell lies in the block (no bounds
    // tests, no result tracking).
    auto step = [&](int32_t s, int k, auto fast_c) {
      constexpr bool FAST = decltype(fast_c)::value;
      const uint32_t inH = __shfl_sync(FULL, incur.x, k);
      const uint32_t inF = __shfl_sync(FULL, incur.y, k);
      const uint32_t inS = __shfl_sync(FULL, selcur, k);
      uint32_t Hup = __shfl_up_sync(FULL, sendH, 1);
      uint32_t Fup = __shfl_up_sync(FULL, sendF, 1);
      uint32_t sel = __shfl_up_sync(FULL, sendS, 1);
      Hup = lane == 0 ? inH : Hup;
      Fup = lane == 0 ? inF : Fup;
      sel = lane == 0 ? inS : sel;
      sendS = sel;
      const int32_t j = s - lane;
      if (FAST || (j >= 1 && j <= n)) {
        uint32_t d = diag;
        diag = Hup;
        // With H = max(t, F) and e <= o, the next row's F = max(F - e, H - o)
        // is max(F - e, t - o): the F recurrence takes one operation per
        // row, and H - o = max(F - o, t - o) is computed beside it.
        uint32_t F = addmax2u(Fup, neg_e2, Hup);   // F of the lane's first row
        uint32_t cm = 0, hprev = 0;   // LOCAL: the column maximum of H - o
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          E[r] = addmax2u(E[r], neg_e2, Ho[r]);
          const uint32_t t = addmax2u(d, prmt(sA[r], sB[r], sel), E[r]);
          d = Ho[r];
          // t - o, floored at the relative 0 in local alignment (no borrow
          // between the halves)
          const uint32_t tmo = LOCAL ? addmax2u(t, neg_o2, z2o) : t - o2;
          Ho[r] = addmax2u(F, neg_o2, tmo);
          if (r + 1 < ROWS) F = addmax2u(F, neg_e2, tmo);
          if (LOCAL) {
            if (r & 1) cm = max3_2u(cm, hprev, Ho[r]);
            else hprev = Ho[r];
          }
        }
        sendH = Ho[ROWS - 1];
        sendF = F;
        if (lane == 15 || lane == 31) ring[wid][lane >> 4][j & 31] = make_uint2(sendH, F);
        if (LOCAL) {
          // a half past its window holds no real cell in this column
          if (!FAST) cm &= (j <= nA ? 0x0000FFFFu : 0u) | (j <= nB ? 0xFFFF0000u : 0u);
          bmax2 = __vmaxu2(bmax2, cm);
        }
        if (!LOCAL && !FAST) {
#pragma unroll
          for (int x = 0; x < 2; ++x) {
            const int32_t mx = x ? mB : mA, nx = x ? nB : nA, base = x ? baseB : baseA;
            if (j == nx && r0 < mx && (x ? inB : inA)) {
              // column n (query end free) or the corner (m, n), rows in order
              int32_t cs = c_s[x][tid], ch = c_h[x][tid];
#pragma unroll
              for (int r = 0; r < ROWS; ++r) {
                const int32_t i = r0 + r + 1;
                const int32_t v = half(Ho[r], x) + o + base;
                if (i <= mx && (q_end_free || i == mx) && (!ch || v > cs)) {
                  cand_set(x, v, i, j);
                  cs = v;
                  ch = 1;
                }
              }
            } else if (t_end_free && (x ? ownB : ownA) && j < nx) {
              int32_t hm = half(Ho[0], x);
#pragma unroll
              for (int r = 1; r < ROWS; ++r)
                if (r == mx - r0 - 1) hm = half(Ho[r], x);
              hm += o + base;
              if (!c_h[x][tid] || hm > c_s[x][tid]) cand_set(x, hm, mx, j);
            }
          }
        }
      }
    };
    // Result cells of a half lie in a block when its column n falls in the
    // block's columns, or (free target end) when the band holds its row m.
    const bool rowmA = !LOCAL && t_end_free && inA && mA <= i0 + BAND;
    const bool rowmB = !LOCAL && t_end_free && inB && mB <= i0 + BAND;
    if (LOCAL) set_floor();
    const int32_t steps = n + 31;
    for (int32_t s0 = 0; s0 < steps; s0 += 32) {   // steps s0 + 1 .. s0 + 32
      if (s0 > 0) {
        // the completed checkpoint columns go out under the current base
        flush(min(s0 - 31, n), min(s0 - 15, n));
        // move the base to lane 0's first row while lane 0 is on a real
        // column of the half
        const uint32_t v = __shfl_sync(FULL, Ho[0], 0);
        const int32_t dA = (inA && s0 <= nA) ? half(v, 0) + o : 0;
        const int32_t dB = (inB && s0 <= nB) ? half(v, 1) + o : 0;
        const uint32_t nd2 = pack2(-dA, -dB);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          Ho[r] = add2(Ho[r], nd2);
          E[r] = add2(E[r], nd2);
        }
        diag = add2(diag, nd2);
        sendH = add2(sendH, nd2);
        sendF = add2(sendF, nd2);
        incur = make_uint2(add2(incur.x, nd2), add2(incur.y, nd2));
        innxt = make_uint2(add2(innxt.x, nd2), add2(innxt.y, nd2));
        baseA += dA;
        baseB += dB;
        // A half whose pair has no cell in the lane's current column (no
        // rows in this band, or the column is past its window) holds
        // values no result reads; they go back to the relative 0 here, so
        // that they never leave the int16 range either, and no 32-bit
        // subtract of H - o borrows from such a half into the other.
        const int32_t jl = s0 - lane;
        const uint32_t jm = ((!inA || jl > nA) ? 0x0000FFFFu : 0u) |
                            ((!inB || jl > nB) ? 0xFFFF0000u : 0u);
        if (__any_sync(FULL, jm != 0u)) {
          const uint32_t z = BIAS2 & jm, keep = ~jm;
#pragma unroll
          for (int r = 0; r < ROWS; ++r) {
            Ho[r] = (Ho[r] & keep) | z;
            E[r] = (E[r] & keep) | z;
          }
          diag = (diag & keep) | z;
          sendH = (sendH & keep) | z;
          sendF = (sendF & keep) | z;
        }
        if (LOCAL) set_floor();
      }
      if (LOCAL) {
        // the state at this block's start, kept until the block shows
        // whether the band's best rises in it
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          snap[wid][r][lane] = Ho[r];
          snap[wid][ROWS + r][lane] = E[r];
        }
        snap[wid][2 * ROWS][lane] = diag;
        snap[wid][2 * ROWS + 1][lane] = sendH;
        snap[wid][2 * ROWS + 2][lane] = sendF;
        bmax2 = 0;
      }
      // lanes' columns in this block: s0 + 1 - 31 .. s0 + 32
      const int32_t jlo = s0 - 30, jhi = s0 + 32;
      const bool evA = inA && (rowmA || (nA >= jlo && nA <= jhi));
      const bool evB = inB && (rowmB || (nB >= jlo && nB <= jhi));
      if (jlo >= 1 && jhi <= n && !evA && !evB) {
        // unrolled by 4 only: the loop body stays small enough for the
        // instruction cache with 16 warps per SM at different steps
#pragma unroll 4
        for (int k = 0; k < 32; ++k) step(s0 + 1 + k, k, std::true_type{});
      } else {
#pragma unroll 1
        for (int k = 0; k < 32 && s0 + 1 + k <= steps; ++k) step(s0 + 1 + k, k, std::false_type{});
      }
      if (LOCAL) {
        // the block's maximum of each half against the band's best: the
        // first block to raise it keeps its start state in the pair's slot
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) bmax2 = __vmaxu2(bmax2, __shfl_xor_sync(FULL, bmax2, off));
#pragma unroll
        for (int x = 0; x < 2; ++x) {
          const bool inx = x ? inB : inA;
          const int32_t nx = x ? nB : nA;
          if (!inx || s0 - 30 > nx) continue;   // no real cell of the half in the block
          const int32_t v = ((bmax2 >> (16 * x)) & 0xFFFFu) == 0u
                                ? 0 : half(bmax2, x) + o + (x ? baseB : baseA);
          if (v <= (x ? bestB : bestA)) continue;
          if (x) { bestB = v; bs0B = s0; bbaseB = baseB; }
          else { bestA = v; bs0A = s0; bbaseA = baseA; }
          uint32_t* slot = lsnap + (uint64_t)((x ? JB.cand_off : JA.cand_off) + b) * SNAP_WORDS * 32;
          __syncwarp();
#pragma unroll 5
          for (int w = 0; w < SNAP_WORDS; ++w) slot[w * 32 + lane] = snap[wid][w][lane];
        }
      }
      // block consumed: rotate, fetch the block after the next
      incur = innxt;
      selcur = selnxt;
      innxt = fetch_in(s0 + 64);
      selnxt = fetch_sel(s0 + 64);
    }
    flush(n, n);
    if (LOCAL) {
      if (lane == 0) {
        if (inA) lbest[JA.cand_off + b] = LongBest{bestA, bs0A, bbaseA, 0};
        if (inB) lbest[JB.cand_off + b] = LongBest{bestB, bs0B, bbaseB, 1};
      }
      __syncwarp();
      continue;
    }
    // merge the lanes' candidates of each half
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      LongCand c = {c_s[x][tid], c_i[x][tid], c_j[x][tid], c_h[x][tid]};
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        LongCand y;
        y.s = __shfl_xor_sync(FULL, c.s, off);
        y.i = __shfl_xor_sync(FULL, c.i, off);
        y.j = __shfl_xor_sync(FULL, c.j, off);
        y.has = __shfl_xor_sync(FULL, c.has, off);
        if (better(y, c)) c = y;
      }
      if (lane == 0 && (x ? inB : inA)) cands[(x ? JB.cand_off : JA.cand_off) + b] = c;
    }
    __syncwarp();
  }
}

// LOCAL, after the score pass: the first cell in (j, i) order holding the
// pair's best, in each band whose best it is.  One warp per (pair, band):
// the band's state at the start of the block in which its running maximum
// first reached the best is restored (the pair's half; the other half at the
// relative 0) and 64 steps are run again from it.  The first cell of the
// best in (j, i) order lies in those steps: the first cell to reach the best
// in step order is in the block's 32 steps, and a cell of the best at a
// smaller column j is processed at most 31 steps after its column's first
// step.  Candidates of all bands merge by (score desc, j asc, i asc).
__global__ void __launch_bounds__(WARPS * 32) k_long_locate16(
    const uint8_t* __restrict__ qcodes, const uint8_t* __restrict__ tcodes,
    const int8_t* __restrict__ Sg, int A, int o, int e, const LongJob* __restrict__ jobs,
    const uint32_t* __restrict__ items, uint32_t n_items, const int2* __restrict__ bnd,
    const LongBest* __restrict__ lbest, const uint32_t* __restrict__ lsnap,
    LongCand* __restrict__ cands) {
  __shared__ uint32_t Sb[4];
  if (threadIdx.x < 4) {
    uint32_t w = 0;
    if ((int)threadIdx.x < A)
      for (int a = 0; a < A; ++a)
        w |= (uint32_t)(uint8_t)(int8_t)(Sg[threadIdx.x * A + a] + o) << (8 * a);
    Sb[threadIdx.x] = w;
  }
  __syncthreads();
  constexpr unsigned FULL = 0xFFFFFFFFu;
  const int lane = threadIdx.x & 31;
  const uint32_t it = blockIdx.x * WARPS + (threadIdx.x >> 5);
  if (it >= n_items) return;
  const LongJob J = jobs[items[2 * it]];
  const int32_t b = (int32_t)items[2 * it + 1];
  const int32_t m = J.m, n = J.n;
  const int32_t nb = (m + BAND - 1) / BAND;
  int32_t V = 0;
  for (int32_t k = lane; k < nb; k += 32) V = max(V, lbest[J.cand_off + k].best);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) V = max(V, __shfl_xor_sync(FULL, V, off));
  const LongBest lb = lbest[J.cand_off + b];
  LongCand out = {0, 0, 0, 0};
  if (V > 0 && lb.best == V) {
    const int x = lb.half;
    const uint32_t keep = x ? 0xFFFF0000u : 0x0000FFFFu, z = BIAS2 & ~keep;
    const int32_t base = lb.base;
    const uint32_t* slot = lsnap + (uint64_t)(J.cand_off + b) * SNAP_WORDS * 32;
    const int32_t i0 = b * BAND, r0 = i0 + lane * ROWS;
    const uint8_t* q = qcodes + J.q_start;
    const uint8_t* t = tcodes + J.t_start;
    uint32_t Ho[ROWS], E[ROWS], sx[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      Ho[r] = (slot[r * 32 + lane] & keep) | z;
      E[r] = (slot[(ROWS + r) * 32 + lane] & keep) | z;
      sx[r] = r0 + r < m ? Sb[q[r0 + r]] : JUNK_S;
    }
    uint32_t diag = (slot[2 * ROWS * 32 + lane] & keep) | z;
    uint32_t sendH = (slot[(2 * ROWS + 1) * 32 + lane] & keep) | z;
    uint32_t sendF = (slot[(2 * ROWS + 2) * 32 + lane] & keep) | z;
    auto sel_of = [&](int32_t j) -> uint32_t {   // the byte-permute selector of column j
      const uint32_t a = (j >= 1 && j <= n) ? t[j - 1] : 0u;
      return x ? ((0x80u) | ((a * 0x11u + 0xC4u) << 8)) : (a * 0x11u + 0x80u) | (0xC4u << 8);
    };
    uint32_t sendS = sel_of(lb.s0 - lane);
    const uint32_t neg_o2 = pack2(-o, -o), neg_e2 = pack2(-e, -e);
    const uint32_t zh = -base - o >= -32768 ? (uint32_t)(-base - o + 32768) & 0xFFFFu : 0u;
    const uint32_t z2o = x ? (zh << 16) : zh;
    const int2* up = b > 0 ? bnd + J.bnd_off + (uint64_t)(2 * b - 1) * (uint32_t)n : nullptr;
    int32_t fj = INT32_MAX, fi = INT32_MAX;   // the lane's first cell of the best
    const int32_t s_end = min(lb.s0 + 64, n + 31);
    for (int32_t s = lb.s0 + 1; s <= s_end; ++s) {
      // lane 0's input: the row above at column s (row 0: H = 0, F = H - o)
      uint32_t inH = BIAS2, inF = BIAS2;
      if (lane == 0 && s <= n) {
        int32_t h = 0, f = -o;
        if (up) {
          const int2 v = up[s - 1];
          h = v.x;
          f = v.y;
        }
        const uint32_t hv = (uint32_t)(h - o - base + 32768) & 0xFFFFu;
        const uint32_t fv = (uint32_t)(f - base + 32768) & 0xFFFFu;
        inH = x ? (hv << 16) | 0x8000u : hv | 0x80000000u;
        inF = x ? (fv << 16) | 0x8000u : fv | 0x80000000u;
      }
      uint32_t Hup = __shfl_up_sync(FULL, sendH, 1);
      uint32_t Fup = __shfl_up_sync(FULL, sendF, 1);
      uint32_t sel = __shfl_up_sync(FULL, sendS, 1);
      if (lane == 0) {
        Hup = inH;
        Fup = inF;
        sel = sel_of(s);
      }
      sendS = sel;
      const int32_t j = s - lane;
      if (j >= 1 && j <= n) {
        uint32_t d = diag;
        diag = Hup;
        uint32_t F = addmax2u(Fup, neg_e2, Hup);
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          E[r] = addmax2u(E[r], neg_e2, Ho[r]);
          const uint32_t sp = x ? prmt(JUNK_S, sx[r], sel) : prmt(sx[r], JUNK_S, sel);
          const uint32_t tt = addmax2u(d, sp, E[r]);
          d = Ho[r];
          const uint32_t tmo = addmax2u(tt, neg_o2, z2o);
          Ho[r] = addmax2u(F, neg_o2, tmo);
          if (r + 1 < ROWS) F = addmax2u(F, neg_e2, tmo);
          if (fj == INT32_MAX && r0 + r < m && half(Ho[r], x) + o + base == V) {
            fj = j;
            fi = r0 + r + 1;
          }
        }
        sendH = Ho[ROWS - 1];
        sendF = F;
      }
    }
    // the warp's first cell in (j, i) order
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const int32_t oj = __shfl_xor_sync(FULL, fj, off), oi = __shfl_xor_sync(FULL, fi, off);
      if (oj < fj || (oj == fj && oi < fi)) { fj = oj; fi = oi; }
    }
    if (fj != INT32_MAX) out = {V, fi, fj, 1};
  }
  if (lane == 0) cands[J.cand_off + b] = out;
}

}  // namespace

bool long16_range_ok(int o, int e, int smax, int smin) {
  // relative values of the cells a warp touches before its next base move,
  // and of the 64 steps a local pair's best is looked up again in: within
  // 512 + 96 rows and columns of the base cell
  const int64_t D = (int64_t)o + std::max(smax, 0);
  return 608 * D + 2 * (int64_t)o + e + std::max(-smin, 0) + 64 < 32768;
}

int launch_long_score16(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int8_t* d_matrix,
                        int A, int o, int e, int mode, uint32_t fe, const LongJob* d_jobs,
                        uint32_t n_jobs, const LongPair16* d_pjobs, const uint32_t* d_items,
                        uint32_t n_items, int2* d_bnd, uint32_t* d_prog, void* d_cands,
                        Scores out, int blocks_per_sm, const uint32_t* d_litems,
                        uint32_t n_litems, uint64_t n_slots) {
  if (n_items == 0) return DSA_OK;
  const bool local = mode == DSA_LOCAL;
  const bool two = blocks_per_sm > 0 && blocks_per_sm <= 2;
  auto kern = local ? (two ? k_long_score16<true, 2> : k_long_score16<true, 3>)
                    : (two ? k_long_score16<false, 2> : k_long_score16<false, 4>);
  // every warp must be resident at once (bands wait on their predecessors)
  int per_sm = 0;
  DSA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, 0));
  if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);
  const uint64_t resident = (uint64_t)std::max(1, per_sm) * ctx->sm_count;
  const unsigned grid = (unsigned)std::min<uint64_t>(resident, (n_items + WARPS - 1) / WARPS);
  // local: each band's best per pair and its block-start snapshot
  void* pb = nullptr;
  void* ps = nullptr;
  const size_t b_bytes = (size_t)n_slots * sizeof(LongBest);
  const size_t s_bytes = (size_t)n_slots * SNAP_WORDS * 32 * sizeof(uint32_t);
  if (local) {
    DSA_TRY(ctx->alloc(&pb, b_bytes));
    DSA_TRY(ctx->alloc(&ps, s_bytes));
  }
  uint32_t* counter = ctx->d_counters + 3;
  DSA_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(uint32_t), ctx->stream));
  kern<<<grid, WARPS * 32, 0, ctx->stream>>>(qs->d_codes, db->d_codes, d_matrix, A, o, e, mode, fe,
                                              d_jobs, d_pjobs, d_items, n_items, counter, d_bnd,
                                              d_prog, static_cast<LongCand*>(d_cands),
                                              ctx->d_status, static_cast<LongBest*>(pb),
                                              static_cast<uint32_t*>(ps));
  cudaError_t err = cudaGetLastError();
  ++ctx->launches;
  if (err == cudaSuccess && local && n_litems) {
    k_long_locate16<<<(n_litems + WARPS - 1) / WARPS, WARPS * 32, 0, ctx->stream>>>(
        qs->d_codes, db->d_codes, d_matrix, A, o, e, d_jobs, d_litems, n_litems, d_bnd,
        static_cast<const LongBest*>(pb), static_cast<const uint32_t*>(ps),
        static_cast<LongCand*>(d_cands));
    err = cudaGetLastError();
    ++ctx->launches;
  }
  if (local) {
    ctx->release(pb, b_bytes);
    ctx->release(ps, s_bytes);
  }
  if (err != cudaSuccess) {
    set_error("k_long_score16: %s", cudaGetErrorString(err));
    return DSA_ERR_CUDA;
  }
  return launch_long_reduce(ctx, d_jobs, n_jobs, d_cands, mode, fe, o, e, out);
}

}  // namespace dsa
