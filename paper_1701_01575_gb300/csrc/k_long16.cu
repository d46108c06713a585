// Long explicit pairs, packed int16x2 score pass (DNW / DSG of Sec. II.C.2
// for pairs of 1e4-1e5 residues, the score pass of the map phase of
// Sec. II.B.1): the band pipeline of the int32 kernel with two pairs per
// warp, one in each 16-bit half of every register.  Local pairs stay on the
// int32 kernel: along a strong diagonal a lane's best improves on most
// steps, and the packed form's per-improvement work outweighs its gain.
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
// cell, so a relative value is bounded by 576 D + 2o + e + |min S| + 64,
// which long16_range_ok checks against 2^15 on the host (no rerun is ever
// needed).  Lane 0's input row (the band above, or row 0) is converted from
// absolute int32 once per 32 columns; the checkpoint rows (the middle and
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

__global__ void __launch_bounds__(WARPS * 32, 4) k_long_score16(
    const uint8_t* __restrict__ qcodes, const uint8_t* __restrict__ tcodes,
    const int8_t* __restrict__ Sg, int A, int o, int e, int mode, uint32_t fe,
    const LongJob* __restrict__ jobs, const LongPair16* __restrict__ pjobs,
    const uint32_t* __restrict__ items, uint32_t n_items, uint32_t* __restrict__ counter,
    int2* __restrict__ bnd, uint32_t* __restrict__ prog, LongCand* __restrict__ cands,
    int32_t* __restrict__ status) {
  __shared__ uint32_t Sb[4];                 // row q of S + o as 4 bytes
  __shared__ uint2 ring[WARPS][2][32];       // per warp: middle (lane 15) and bottom (lane 31) rows
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
    if (t_end_free) {   // H[m][0] on row m
      if (ownA) cand_set(0, h_col0(mode, fe, mA, o, e), mA, 0);
      if (ownB) cand_set(1, h_col0(mode, fe, mB, o, e), mB, 0);
    }

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
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          E[r] = addmax2u(E[r], neg_e2, Ho[r]);
          const uint32_t t = addmax2u(d, prmt(sA[r], sB[r], sel), E[r]);
          d = Ho[r];
          const uint32_t tmo = t - o2;   // no borrow between the halves
          Ho[r] = addmax2u(F, neg_o2, tmo);
          if (r + 1 < ROWS) F = addmax2u(F, neg_e2, tmo);
        }
        sendH = Ho[ROWS - 1];
        sendF = F;
        if (lane == 15 || lane == 31) ring[wid][lane >> 4][j & 31] = make_uint2(sendH, F);
        if (!FAST) {
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
    const bool rowmA = t_end_free && inA && mA <= i0 + BAND;
    const bool rowmB = t_end_free && inB && mB <= i0 + BAND;
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
      // block consumed: rotate, fetch the block after the next
      incur = innxt;
      selcur = selnxt;
      innxt = fetch_in(s0 + 64);
      selnxt = fetch_sel(s0 + 64);
    }
    flush(n, n);
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

}  // namespace

bool long16_range_ok(int o, int e, int smax, int smin) {
  const int64_t D = (int64_t)o + std::max(smax, 0);
  return 576 * D + 2 * (int64_t)o + e + std::max(-smin, 0) + 64 < 32768;
}

int launch_long_score16(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int8_t* d_matrix,
                        int A, int o, int e, int mode, uint32_t fe, const LongJob* d_jobs,
                        uint32_t n_jobs, const LongPair16* d_pjobs, const uint32_t* d_items,
                        uint32_t n_items, int2* d_bnd, uint32_t* d_prog, void* d_cands,
                        Scores out, int blocks_per_sm) {
  if (n_items == 0) return DSA_OK;
  if (mode == DSA_LOCAL) {
    set_error("the packed long-pair kernel takes global and semi-global pairs");
    return DSA_ERR_INVALID_ARG;
  }
  auto kern = k_long_score16;
  // every warp must be resident at once (bands wait on their predecessors)
  int per_sm = 0;
  DSA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, WARPS * 32, 0));
  if (blocks_per_sm > 0) per_sm = std::min(per_sm, blocks_per_sm);
  const uint64_t resident = (uint64_t)std::max(1, per_sm) * ctx->sm_count;
  const unsigned grid = (unsigned)std::min<uint64_t>(resident, (n_items + WARPS - 1) / WARPS);
  uint32_t* counter = ctx->d_counters + 3;
  DSA_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(uint32_t), ctx->stream));
  kern<<<grid, WARPS * 32, 0, ctx->stream>>>(qs->d_codes, db->d_codes, d_matrix, A, o, e, mode, fe,
                                              d_jobs, d_pjobs, d_items, n_items, counter, d_bnd,
                                              d_prog, static_cast<LongCand*>(d_cands),
                                              ctx->d_status);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return launch_long_reduce(ctx, d_jobs, n_jobs, d_cands, mode, fe, o, e, out);
}

}  // namespace dsa
