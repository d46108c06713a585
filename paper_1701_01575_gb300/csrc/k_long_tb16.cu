// Checkpointed traceback of long pairs, part 1 in packed int16x2 form (the
// traceback of Sec. II.B.1 for pairs of 1e4-1e5 residues): two traceback
// bands per warp, one in each 16-bit half of every register, for alphabets
// of up to 4 letters with every S + o in int8.
//
// Layout.  A unit is two traceback bands (of any jobs; the host pairs bands
// of similar window width).  Lane k owns rows i0 + 8k + 1 .. i0 + 8k + 8 of
// its half's band and, at step s, the half's stored column jc = s - 1 - k
// (absolute column jlo + jc): the stored column, the decision word and the
// nibble position are the same in both halves, only the windows' lengths
// differ.  A half past its window or its pair's last row computes values no
// decision is stored for.
//
// Values.  As in the packed score pass, H - o, E and F are kept relative to
// one absolute int32 base per half, in offset binary (value + 2^15 per
// half); every 32 steps the base moves to the H of lane 0's first row (while
// lane 0 is on a stored column of the half), and halves past their window
// return to the relative 0.  All cells a warp touches between two moves lie
// within 256 + 96 rows and columns of the base cell, so with
// D = o + max(S, 0) a relative value is bounded by 352 D + 2o + e +
// |min S| + 64; long_tb16_range_ok keeps that below 15360, so the value
// standing for minus infinity (the wall left of a window, row 0's F) can be
// -16000 and every difference of two values stays inside int16.
//
// Cell update per register (2 cells), with Ho = H - o of the row above
// (hoa), of the column to the left (Ho), and of the diagonal (d):
//   F = max(F - e, hoa),  E = max(E - e, Ho),  g = max(F, E),
//   H = max(d + (S + o), g) [local: and 0],  Ho' = H - o.
// Each decision is the sign of a borrow-free difference of two offset-binary
// registers (a - b + 0x80008000: bits 15 and 31 are a >= b for the two
// halves): F opened here (hoa >= F - e), E opened here (Ho >= E - e), I
// before D (F >= E), M (d + S + o >= g, from max(d + S + o, g - 1) in one
// add-max) and, in local mode, stop (0 >= the maximum).  Two sign-replicating
// byte permutes turn the four flags of both halves into bytes of 0 / 0xFF,
// two masks and a fold place them as the nibble of each cell (bits 0-1 the
// H source: 0 D, 1 M, 2 I, 3 stop; bit 2 E opened; bit 3 F opened), and
// bit-field inserts collect eight columns of them in one word per half, each
// stored by its lane at the word's last column (the stores per cell of the
// int32 fill: 16-bit stores of every 4 columns measured 2.6 times slower).
#include "dsa_internal.cuh"
#include "dpx.cuh"

#include <type_traits>

namespace dsa {
namespace {

constexpr int TB_ROWS = 8;
constexpr int TB_BAND = 32 * TB_ROWS;
constexpr int WARPS = 4;
// blocks per SM the build keeps resident: 4 (124 registers, no spills) ran
// the 64 long pairs' traceback 0.25 ms faster than 3; 2 was no faster than 3
constexpr int FILL_BLOCKS = 4;
constexpr uint32_t BIAS2 = 0x80008000u;
constexpr int32_t WALL = -16000;             // stands for minus infinity
// local floor when the absolute 0 is out of range: below every real value
// (|v| < 15360) and within 2^15 of all of them
constexpr int32_t FLOOR_MIN = -16384;
constexpr uint32_t JUNK_S = 0x80808080u;     // S + o = -128: rows past a pair's end

__device__ __forceinline__ uint32_t bias2(int32_t lo, int32_t hi) { return pack2(lo, hi) ^ BIAS2; }
__device__ __forceinline__ int32_t half(uint32_t v, int x) {
  return x ? hi16(v ^ BIAS2) : lo16(v ^ BIAS2);
}
__device__ __forceinline__ int32_t h_row0(int mode, uint32_t fe, int64_t j, int o, int e) {
  if (j == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_T_BEGIN))) return 0;
  return -(o + (int32_t)(j - 1) * e);
}
__device__ __forceinline__ int32_t h_col0(int mode, uint32_t fe, int64_t i, int o, int e) {
  if (i == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_Q_BEGIN))) return 0;
  return -(o + (int32_t)(i - 1) * e);
}
// a - b per half, offset so that bit 15 / 31 is (a >= b); no borrow crosses
// the halves while |a - b| < 2^15 in each
__device__ __forceinline__ uint32_t ge_flags(uint32_t a, uint32_t b) { return a - b + BIAS2; }
// the low 4 bits of `field` written into `base` at bit `pos`
__device__ __forceinline__ uint32_t bfi4(uint32_t field, uint32_t base, uint32_t pos) {
  uint32_t r;
  asm("bfi.b32 %0, %1, %2, %3, 4;" : "=r"(r) : "r"(field), "r"(base), "r"(pos));
  return r;
}

// one traceback band as one half of a unit
struct TbHalf {
  const uint8_t* q;
  const uint8_t* t;
  uint32_t* D;        // the job's decisions (bands x TB_BAND x wpr words)
  const int2* up;     // checkpoint row above the band (band 0: none)
  int32_t b, i0, ie, jlo, wcb;
  uint32_t wpr;       // decision words per row
  int32_t base0;      // H of (i0, jlo): the first base
};

__device__ __forceinline__ TbHalf tb_half(const LongTbJob& jb, int32_t b, const int2* win,
                                          const uint8_t* qcodes, const uint8_t* tcodes,
                                          uint32_t* dir, const int2* bnd, int mode, uint32_t fe,
                                          int o, int e) {
  TbHalf h;
  const int2 w = win[jb.win_off + (uint32_t)b];
  h.q = qcodes + jb.q_start;
  h.t = tcodes + jb.t_start;
  h.D = dir + jb.dir_off;
  h.up = b > 0 ? bnd + jb.bnd_off + (uint64_t)(b - 1) * (uint32_t)jb.n : nullptr;
  h.b = b;
  h.i0 = b * TB_BAND;
  h.ie = jb.ie;
  h.jlo = w.x;
  h.wcb = w.y;
  h.wpr = jb.wpr;
  h.base0 = b > 0 ? h.up[h.jlo - 1].x : h_row0(mode, fe, h.jlo, o, e);
  return h;
}

template <bool LOCAL>
__global__ void __launch_bounds__(WARPS * 32, FILL_BLOCKS) k_long_tb_fill16(
    const uint8_t* __restrict__ qcodes, const uint8_t* __restrict__ tcodes,
    const int8_t* __restrict__ Sg, int A, int o, int e, int mode, uint32_t fe,
    const LongTbJob* __restrict__ jobs, const uint32_t* __restrict__ units, uint32_t n_units,
    const int2* __restrict__ bnd, uint32_t* __restrict__ dir, const int2* __restrict__ win) {
  __shared__ uint32_t Sb[4];   // row q of S + o as 4 bytes
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
  const uint32_t e2 = pack2(e, e), o2 = pack2(o, o);
  const uint32_t wall2 = bias2(WALL, WALL);
  const uint32_t warps = gridDim.x * WARPS;
  for (uint32_t it = blockIdx.x * WARPS + (threadIdx.x >> 5); it < n_units; it += warps) {
    const uint32_t* u = units + 4 * (uint64_t)it;
    const bool hasB = u[2] != NONE;
    // an empty high half repeats the low one and stores nothing
    const TbHalf HA = tb_half(jobs[u[0]], (int32_t)u[1], win, qcodes, tcodes, dir, bnd, mode, fe, o, e);
    const TbHalf HB = hasB ? tb_half(jobs[u[2]], (int32_t)u[3], win, qcodes, tcodes, dir, bnd, mode,
                                     fe, o, e)
                           : HA;
    const int32_t r0A = HA.i0 + lane * TB_ROWS, r0B = HB.i0 + lane * TB_ROWS;
    // what the steps read, held as plain values: the windows' lengths, the
    // rows' limits and this lane's first decision row of each half
    const int32_t wcbA = HA.wcb, wcbB = HB.wcb, ieA = HA.ie, ieB = HB.ie;
    // decision word w of the lane's row r: DA[w TB_BAND + r] (the band's
    // column blocks, rows consecutive)
    uint32_t* const DA = HA.D + (uint64_t)HA.b * HA.wpr * TB_BAND + (uint32_t)(r0A - HA.i0);
    uint32_t* const DB = HB.D + (uint64_t)HB.b * HB.wpr * TB_BAND + (uint32_t)(r0B - HB.i0);
    int32_t baseA = HA.base0, baseB = HB.base0;
    const bool wallA = HA.jlo > 1, wallB = HB.jlo > 1;
    // nbA / nbB: each half's decision word of the current 8 columns
    uint32_t Ho[TB_ROWS], E[TB_ROWS], nbA[TB_ROWS], nbB[TB_ROWS], sA[TB_ROWS], sB[TB_ROWS];
#pragma unroll
    for (int r = 0; r < TB_ROWS; ++r) {
      const int32_t iA = r0A + r + 1, iB = r0B + r + 1;
      const int32_t ha = wallA ? WALL : h_col0(mode, fe, iA, o, e) - o - baseA;
      const int32_t hb = wallB ? WALL : h_col0(mode, fe, iB, o, e) - o - baseB;
      Ho[r] = bias2(ha, hb);
      E[r] = wall2;
      nbA[r] = 0;
      nbB[r] = 0;
      sA[r] = iA <= HA.ie ? Sb[HA.q[iA - 1]] : JUNK_S;
      sB[r] = iB <= HB.ie ? Sb[HB.q[iB - 1]] : JUNK_S;
    }
    // H - o of (r0, jlo - 1): column 0, or (lane 0) the checkpoint row's
    // cell on the window's edge, or the wall
    auto diag0 = [&](const TbHalf& h, int32_t r0, bool wall, int32_t base) -> int32_t {
      if (!wall) return h_col0(mode, fe, r0, o, e) - o - base;
      if (lane != 0) return WALL;
      const int32_t v = h.b == 0 ? h_row0(mode, fe, h.jlo - 1, o, e) : h.up[h.jlo - 2].x;
      return v - o - base;
    };
    uint32_t diag = bias2(diag0(HA, r0A, wallA, baseA), diag0(HB, r0B, wallB, baseB));
    uint32_t sendH = BIAS2, sendF = wall2, sendS = 0;
    // local: the relative 0 per half (clamped far below every real value
    // when the absolute 0 is out of range)
    uint32_t z2 = 0;
    auto set_floor = [&]() {
      z2 = bias2(max(-baseA, FLOOR_MIN), max(-baseB, FLOOR_MIN));
    };
    if (LOCAL) set_floor();
    // lane 0's inputs for steps blk + 1 .. blk + 32 (lane k: step blk + k +
    // 1, column jlo + blk + k of each half): (H - o, F) of the row above,
    // relative to the current base; columns past a window get the relative 0
    auto in_half = [&](const TbHalf& h, int32_t blk, int32_t base, int32_t& hr, int32_t& fr) {
      const int32_t jc = blk + lane;
      hr = 0;
      fr = 0;
      if (jc < h.wcb) {
        const int32_t jj = h.jlo + jc;
        if (h.b == 0) {
          hr = h_row0(mode, fe, jj, o, e) - o - base;
          fr = WALL;
        } else {
          const int2 v = h.up[jj - 1];
          hr = v.x - o - base;
          fr = v.y - base;
        }
      }
    };
    auto fetch_in = [&](int32_t blk) -> uint2 {
      int32_t ha, fa, hb, fb;
      in_half(HA, blk, baseA, ha, fa);
      in_half(HB, blk, baseB, hb, fb);
      return make_uint2(bias2(ha, hb), bias2(fa, fb));
    };
    // byte-permute selector of the two residues (byte a_lo of the low row
    // table, byte 4 + a_hi of the high one, each sign-replicated)
    auto fetch_sel = [&](int32_t blk) -> uint32_t {
      const int32_t jc = blk + lane;
      const uint32_t aa = jc < HA.wcb ? HA.t[HA.jlo + jc - 1] : 0u;
      const uint32_t ab = jc < HB.wcb ? HB.t[HB.jlo + jc - 1] : 0u;
      return (aa * 0x11u + 0x80u) | ((ab * 0x11u + 0xC4u) << 8);
    };
    uint2 incur = fetch_in(0), innxt = fetch_in(32);
    uint32_t selcur = fetch_sel(0), selnxt = fetch_sel(32);

    // One step.  FAST: both bands full (no row past a pair's end), every
    // lane inside both windows, no window's last column.
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
      const int32_t jc = s - 1 - lane;
      const bool liveA = jc >= 0 && jc < wcbA, liveB = jc >= 0 && jc < wcbB;
      if (FAST || liveA || liveB) {
        uint32_t d = diag;
        diag = Hup;
        uint32_t F = Fup, hoa = Hup;
        const uint32_t sh = 4u * (uint32_t)(jc & 7);
        // a word ends at its eighth column or at the window's last column
        const bool wendA = FAST ? (jc & 7) == 7 : liveA && ((jc & 7) == 7 || jc == wcbA - 1);
        const bool wendB = hasB && (FAST ? (jc & 7) == 7 : liveB && ((jc & 7) == 7 || jc == wcbB - 1));
        const uint32_t w = (uint32_t)(jc >> 3);
#pragma unroll
        for (int r = 0; r < TB_ROWS; ++r) {
          const uint32_t fx = F - e2;
          const uint32_t tF = ge_flags(hoa, fx);   // F opened here
          F = __vmaxu2(hoa, fx);
          const uint32_t ex = E[r] - e2;
          const uint32_t tE = ge_flags(Ho[r], ex);   // E opened here
          E[r] = __vmaxu2(Ho[r], ex);
          const uint32_t g = __vmaxu2(F, E[r]);
          uint32_t tG = ge_flags(F, E[r]);   // I before D
          const uint32_t v2 = addmax2u(d, prmt(sA[r], sB[r], sel), g - 0x00010001u);
          uint32_t v = __vmaxu2(v2, g);
          uint32_t tM = ge_flags(v2, g);   // M: d + S + o >= g
          if (LOCAL) {
            const uint32_t tS = ge_flags(z2, v);   // the empty alignment: stop
            v = __vmaxu2(v, z2);
            tG = (tG & ~tM) | tS;
            tM |= tS;
          } else {
            tG &= ~tM;
          }
          d = Ho[r];
          Ho[r] = v - o2;
          hoa = Ho[r];
          // bytes [M, I, M, I] and [E, F, E, F] of the two cells as 0 / 0xFF,
          // masked to their nibble bits, then folded to one nibble per half
          // (bits 0-3: A, 16-19: B)
          const uint32_t pMI = prmt(tM, tG, 0xFBD9u);
          const uint32_t pEF = prmt(tE, tF, 0xFBD9u);
          const uint32_t x = (pMI & 0x02010201u) | (pEF & 0x08040804u);
          const uint32_t y = x | (x >> 8);
          nbA[r] = bfi4(y, nbA[r], sh);
          nbB[r] = bfi4(y >> 16, nbB[r], sh);
          if (wendA) {
            if (FAST || r0A + r + 1 <= ieA) DA[w * TB_BAND + r] = nbA[r];
            nbA[r] = 0;
          }
          if (wendB) {
            if (FAST || r0B + r + 1 <= ieB) DB[w * TB_BAND + r] = nbB[r];
            nbB[r] = 0;
          }
        }
        sendH = hoa;
        sendF = F;
      }
    };

    const bool full = HA.i0 + TB_BAND <= ieA && HB.i0 + TB_BAND <= ieB;
    const int32_t wmin = min(wcbA, wcbB);
    const int32_t steps = max(wcbA, wcbB) + 31;
    for (int32_t s0 = 0; s0 < steps; s0 += 32) {
      if (s0 > 0) {
        // move each base to lane 0's first row while lane 0 is on a stored
        // column of the half (lane 0's last column: s0 - 1)
        const uint32_t v0 = __shfl_sync(FULL, Ho[0], 0);
        const int32_t dA = s0 - 1 < wcbA ? half(v0, 0) + o : 0;
        const int32_t dB = s0 - 1 < wcbB ? half(v0, 1) + o : 0;
        const uint32_t nd2 = pack2(-dA, -dB);
#pragma unroll
        for (int r = 0; r < TB_ROWS; ++r) {
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
        // halves past their window go back to the relative 0
        const int32_t jl = s0 - 1 - lane;
        const uint32_t jm = (jl >= wcbA ? 0x0000FFFFu : 0u) | (jl >= wcbB ? 0xFFFF0000u : 0u);
        if (__any_sync(FULL, jm != 0u)) {
          const uint32_t z = BIAS2 & jm, keep = ~jm;
#pragma unroll
          for (int r = 0; r < TB_ROWS; ++r) {
            Ho[r] = (Ho[r] & keep) | z;
            E[r] = (E[r] & keep) | z;
          }
          diag = (diag & keep) | z;
          sendH = (sendH & keep) | z;
          sendF = (sendF & keep) | z;
        }
        if (LOCAL) set_floor();
      }
      if (full && s0 >= 32 && s0 + 32 < wmin) {
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
    __syncwarp();
  }
}

}  // namespace

bool long_tb16_range_ok(int o, int e, int smax, int smin) {
  const int64_t D = (int64_t)o + std::max(smax, 0);
  return 352 * D + 2 * (int64_t)o + e + std::max(-smin, 0) + 64 < 15360;
}

int launch_long_tb_fill16(dsa_ctx* ctx, cudaStream_t stream, const dsa_db* db, const dsa_db* qs,
                          const int8_t* d_matrix, int A, int o, int e, int mode, uint32_t fe,
                          const LongTbJob* d_jobs, const uint32_t* d_units, uint32_t n_units,
                          const int2* d_bnd, uint32_t* d_dir, const int2* d_win) {
  if (n_units == 0) return DSA_OK;
  const unsigned grid = (unsigned)std::min<uint64_t>((n_units + WARPS - 1) / WARPS,
                                                     (uint64_t)ctx->sm_count * 16);
  auto fill = mode == DSA_LOCAL ? k_long_tb_fill16<true> : k_long_tb_fill16<false>;
  fill<<<grid, WARPS * 32, 0, stream>>>(qs->d_codes, db->d_codes, d_matrix, A, o, e, mode, fe,
                                        d_jobs, d_units, n_units, d_bnd, d_dir, d_win);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

}  // namespace dsa
