// Start coordinates and CIGAR for reported hits (the paper's "location and
// traceback", Sec. I and the alignment object of Sec. II.B.1).
//
// One warp per hit recomputes the exact int32 DP over the rectangle from
// (0, 0) to the hit's end cell as an anti-diagonal wavefront: lane k owns
// ROWS consecutive query rows of a band of 32*ROWS rows, processes column
// j = step - k, and hands its last row's H and F to lane k+1 through a warp
// shuffle; bands are chained through a boundary row in global memory.  For
// every cell it stores a 4-bit decision word:
//   bits 0-1  source of H: 0 = diagonal (M), 1 = F (I), 2 = E (D), 3 = stop
//             (local cell equal to 0); tested in the order stop, M, F, E;
//   bit 2     E opened here: H[i][j-1] - o >= E[i][j-1] - e;
//   bit 3     F opened here: H[i-1][j] - o >= F[i-1][j] - e;
// eight cells per 32-bit word along the row.  Lane 0 then walks back from the
// end cell (priority stop > M > I > D, opening preferred on ties) and writes
// run-length CIGAR words in reverse order; a second kernel packs them
// forward into the result's CIGAR array.
#include "dsa_internal.cuh"
#include "dpx.cuh"

#include <type_traits>

namespace dsa {
namespace {

constexpr int ROWS = 8;
constexpr int BAND = 32 * ROWS;

__device__ __forceinline__ int32_t h_row0(int mode, uint32_t fe, int64_t j, int o, int e) {
  if (j == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_T_BEGIN))) return 0;
  return -(o + (int32_t)(j - 1) * e);
}
__device__ __forceinline__ int32_t h_col0(int mode, uint32_t fe, int64_t i, int o, int e) {
  if (i == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_Q_BEGIN))) return 0;
  return -(o + (int32_t)(i - 1) * e);
}

struct RevCigar {
  uint32_t* out;
  uint32_t n = 0;
  int op = -1;
  uint32_t run = 0;
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
    if (run) out[n++] = (run << 4) | (uint32_t)op;
    run = 0;
  }
};

__global__ void __launch_bounds__(128) k_traceback(
    const uint8_t* __restrict__ qcodes, const uint8_t* __restrict__ tcodes,
    const int8_t* __restrict__ Sg, int A, int o, int e, int mode, uint32_t fe,
    const TbJob* __restrict__ jobs, uint32_t n_jobs, uint32_t* __restrict__ dir,
    uint32_t* __restrict__ cig_tmp, int2* __restrict__ scratch, dsa_hit* __restrict__ hits) {
  __shared__ int8_t S[32 * 32];
  for (int x = threadIdx.x; x < A * A; x += blockDim.x) S[x] = Sg[x];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  const bool local = mode == DSA_LOCAL;
  for (uint32_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w < n_jobs; w += warps) {
    const TbJob jb = jobs[w];
    const int32_t ie = jb.ie, je = jb.je;
    const uint8_t* q = qcodes + jb.q_start;
    const uint8_t* t = tcodes + jb.t_start;
    uint32_t* D = dir + jb.dir_off;
    int2* scr = scratch + jb.scr_off;
    const uint32_t wpr = jb.wpr;

    if (ie > 0 && je > 0) {
      for (int32_t i0 = 0; i0 < ie; i0 += BAND) {
        const int32_t r0 = i0 + lane * ROWS;   // rows r0+1 .. r0+ROWS
        int32_t H[ROWS], E[ROWS];
        uint32_t nb[ROWS];
        int qc[ROWS];
#pragma unroll
        for (int r = 0; r < ROWS; ++r) {
          const int32_t i = r0 + r + 1;
          H[r] = jb.jlo > 0 ? NEG32 : h_col0(mode, fe, i, o, e);
          E[r] = NEG32;
          nb[r] = 0;
          qc[r] = i <= ie ? q[i - 1] : 0;
        }
        int32_t diag = (jb.jlo > 0 && r0 > 0) ? NEG32 : h_col0(mode, fe, r0, o, e);
        int32_t sendH = 0, sendF = NEG32;
        const int32_t steps = je + 31;
        for (int32_t s = 1; s <= steps; ++s) {
          const int32_t upH = __shfl_up_sync(0xFFFFFFFFu, sendH, 1);
          const int32_t upF = __shfl_up_sync(0xFFFFFFFFu, sendF, 1);
          const int32_t j = s - lane;
          if (j >= 1 && j <= je && r0 < ie) {
            int32_t Hup, Fup;
            if (lane == 0) {
              if (i0 == 0) {
                Hup = h_row0(mode, fe, j, o, e);
                Fup = NEG32;
              } else {
                const int2 v = scr[j - 1];
                Hup = v.x;
                Fup = v.y;
              }
            } else {
              Hup = upH;
              Fup = upF;
            }
            const int a = t[j - 1];
            int32_t d = diag;
            diag = Hup;
            int32_t F = Fup, Hp = Hup;
            const int sh = 4 * ((j - 1) & 7);
            const bool flushw = ((j & 7) == 0) || j == je;
#pragma unroll
            for (int r = 0; r < ROWS; ++r) {
              const int32_t i = r0 + r + 1;
              if (i <= ie) {
                const int32_t fo = Hp - o, fx = F - e;
                F = max(fx, fo);
                const int32_t eo = H[r] - o, ex = E[r] - e;
                E[r] = max(ex, eo);
                const int32_t m = d + S[qc[r] * A + a];
                int32_t v = max(m, max(E[r], F));
                if (local) v = max(v, 0);
                uint32_t src;
                if (local && v == 0) src = 3;
                else if (v == m) src = 0;
                else if (v == F) src = 1;
                else src = 2;
                const uint32_t nib = src | ((eo >= ex) ? 4u : 0u) | ((fo >= fx) ? 8u : 0u);
                nb[r] |= nib << sh;
                if (flushw) {
                  D[(uint64_t)(i - 1) * wpr + (uint32_t)(j - 1) / 8u] = nb[r];
                  nb[r] = 0;
                }
                d = H[r];
                H[r] = v;
                Hp = v;
              }
            }
            sendH = Hp;
            sendF = F;
            if (lane == 31) scr[j - 1] = make_int2(Hp, F);
          }
        }
        __syncwarp();
      }
    }
    __syncwarp();
    if (lane == 0) {
      RevCigar c;
      c.out = cig_tmp + jb.cig_off;
      int32_t i = ie, j = je;
      int st = 0;  // 0 = H, 1 = F, 2 = E
      const bool sg = mode == DSA_SEMIGLOBAL;
      // every residue is consumed by at most two iterations (a change of
      // state, then the move), so 2 (ie + je) + 2 iterations always suffice;
      // the guards below keep a corrupt decision word from indexing outside
      // the rectangle
      for (int64_t guard = 2 * ((int64_t)ie + je) + 2; guard > 0; --guard) {
        if (st == 0) {
          if (sg && ((i == 0 && (fe & DSA_FREE_T_BEGIN)) || (j == 0 && (fe & DSA_FREE_Q_BEGIN))))
            break;
          if (i == 0 || j == 0) {
            if (local) break;
            while (j > 0) { c.emit(2); --j; }
            while (i > 0) { c.emit(1); --i; }
            break;
          }
          const uint32_t nib = (D[(uint64_t)(i - 1) * wpr + (uint32_t)(j - 1) / 8u] >> (4 * ((j - 1) & 7))) & 15u;
          const uint32_t src = nib & 3u;
          if (src == 3) break;
          if (src == 0) { c.emit(0); --i; --j; }
          else st = src == 1 ? 1 : 2;
        } else if (st == 1) {
          if (i <= 0 || j <= 0) break;
          const uint32_t nib = (D[(uint64_t)(i - 1) * wpr + (uint32_t)(j - 1) / 8u] >> (4 * ((j - 1) & 7))) & 15u;
          c.emit(1);
          if (nib & 8u) st = 0;
          --i;
        } else {
          if (i <= 0 || j <= 0) break;
          const uint32_t nib = (D[(uint64_t)(i - 1) * wpr + (uint32_t)(j - 1) / 8u] >> (4 * ((j - 1) & 7))) & 15u;
          c.emit(2);
          if (nib & 4u) st = 0;
          --j;
        }
      }
      c.flush();
      dsa_hit* h = hits + jb.hit;
      h->q_begin = i;
      h->t_begin = j + jb.jlo;
      h->cigar_len = c.n;
      h->flags |= DSA_HIT_HAS_TRACEBACK;
    }
  }
}

// Band (both kernels): with a free target begin, a hit's score bounds the
// deletions of any path that reaches it (each M scores at most max S, a run
// of k deletions costs at least o + (k-1)e), so every optimal path starts at
// a column >= jlo = je - ie - kmax.  The DP restricted to columns jlo..je with
// a wall at column jlo has the same values on every cell of an optimal path
// and the same ties, hence the same decisions along the walk; the host then
// passes t_start + jlo and je - jlo, and t_begin is shifted back by jlo.
//
// Thread-per-hit variant for large batches of small rectangles (reads in
// windows): one thread recomputes its hit's rectangle in strips of TROWS
// query rows held in registers, column by column, with the same 4-bit
// decisions as above.  The decisions of a strip column (TROWS nibbles, NW =
// TROWS / 8 words) go to a layout interleaved over the 32 hits of a warp,
//   word (strip s, stored column c, part h) of lane l at
//   dir_off + ((s * cols + c) * NW + h) * 32       (dir_off = group base + l),
// so every store of the warp is one 128-byte line; the strip's bottom row
// (H, F) is handed to the next strip through an interleaved scratch row
// indexed by target column.  Each thread then walks its own hit back, so the
// 32 walks of a warp run side by side instead of one after another.
//
// Diagonal window: the host bounds the diagonals j - i of every optimal path
// to dlo .. dlo + wc - TROWS (from the score: deletions, insertions or total
// gaps are bounded as for the column band), so strip s keeps only the wc
// columns from jlo_s = clamp(i0 + 1 + dlo, 1, je - wc + 1).  Cells left of
// jlo_s and above-right of the previous strip's columns lie outside the
// band and enter as -inf; a recomputed value is then at most the full DP's
// and at least the band-restricted DP's, which agree on every cell of an
// optimal path and on every candidate that ties there.
constexpr int TROWS = TB_STRIP;
constexpr int NW = TB_STRIP_WORDS;

// 7 blocks per SM (72 registers): the kernel waits mostly on global loads,
// and 28 warps per SM hide more of them than 24 (8 blocks spilled at 64).
template <bool LOCAL, bool BYTES>
__global__ void __launch_bounds__(128, TROWS <= 8 ? 7 : 4) k_traceback_thread(
    const uint8_t* __restrict__ qcodes, const uint8_t* __restrict__ tcodes,
    const int8_t* __restrict__ Sg, int A, int o, int e, int mode, uint32_t fe,
    const TbJob* __restrict__ jobs, uint32_t n_jobs, uint32_t* __restrict__ dir,
    uint32_t* __restrict__ cig_tmp, int2* __restrict__ scratch, dsa_hit* __restrict__ hits) {
  // substitution scores with o added: the diagonal term H + S is taken as
  // (H - o) + (S + o) from the stored H - o
  __shared__ int32_t So[32 * 32];
  __shared__ uint32_t Sb[4];   // BYTES: row q of S + o as 4 bytes (each fits int8)
  for (int x = threadIdx.x; x < A * A; x += blockDim.x) So[x] = Sg[x] + o;
  if (BYTES && threadIdx.x < 4) {
    uint32_t w = 0;
    for (int a = 0; a < A; ++a)
      if ((int)threadIdx.x < A) w |= (uint32_t)(uint8_t)(int8_t)(Sg[threadIdx.x * A + a] + o) << (8 * a);
    Sb[threadIdx.x] = w;
  }
  __syncthreads();
  const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_jobs) return;
  constexpr bool local = LOCAL;
  const TbJob jb = jobs[k];
  const int32_t ie = jb.ie, je = jb.je;
  const uint8_t* q = qcodes + jb.q_start;
  const uint8_t* t = tcodes + jb.t_start;
  uint32_t* D = dir + jb.dir_off;
  int2* scr = scratch + jb.scr_off;
  const uint64_t cols = jb.wpr;   // stored columns per strip in the group's layout (>= wc)
  const int32_t wc = jb.wc;       // this hit's stored columns per strip (<= je)
  auto strip_jlo = [&](int32_t i0) { return max(1, min(i0 + 1 + jb.dlo, je - wc + 1)); };
  const int2 NEGP = make_int2(NEG32, NEG32);

  if (ie > 0 && je > 0) {
    int32_t plo = 1, phi = je;   // columns the previous strip computed
    for (int32_t i0 = 0, s = 0; i0 < ie; i0 += TROWS, ++s) {
      const int rows = min(TROWS, ie - i0);
      const bool last = i0 + rows == ie;
      const int32_t jlo = strip_jlo(i0), jhi = jlo + wc - 1;
      const bool wall = jlo > 1 || jb.jlo > 0;   // column jlo - 1 is -inf below row 0
      // Ho = H - o of the strip's rows in the previous column, E of those rows
      int32_t Ho[TROWS], E[TROWS];
      uint32_t qv[TROWS];   // BYTES: S + o row of the query residue as bytes; else its matrix offset
#pragma unroll
      for (int r = 0; r < TROWS; ++r) {
        Ho[r] = (wall ? NEG32 : h_col0(mode, fe, i0 + r + 1, o, e)) - o;
        E[r] = NEG32;
        qv[r] = r < rows ? (BYTES ? Sb[q[i0 + r]] : (uint32_t)q[i0 + r] * A) : 0u;
      }
      // H[i0][jlo - 1] - o
      int32_t diag;
      if (i0 == 0) diag = h_row0(mode, fe, jlo - 1, o, e);
      else if (jlo == 1) diag = jb.jlo > 0 ? NEG32 : h_col0(mode, fe, i0, o, e);
      else diag = (jlo - 1 >= plo && jlo - 1 <= phi) ? scr[(uint64_t)(jlo - 2) * 32].x : NEG32;
      diag -= o;
      uint32_t* Ds = D + (uint64_t)s * cols * (32 * NW);
      // the column loop in four forms (first strip: top row from the boundary
      // of the matrix; last strip: nothing to hand down), with no per-column
      // branch that depends on the strip
      auto columns = [&](auto first_c, auto last_c) {
        constexpr bool FIRST = decltype(first_c)::value;
        constexpr bool LAST = decltype(last_c)::value;
        // loads run one column ahead of the arithmetic; the last iteration
        // re-reads a valid column instead of branching
        int n_a = t[jlo - 1];
        int2 n_v = (!FIRST && jlo <= phi) ? scr[(uint64_t)(jlo - 1) * 32] : NEGP;
        for (int32_t j = jlo; j <= jhi; ++j) {
          const int a = n_a;
          const int2 v = n_v;
          n_a = t[min(j, jhi - 1)];
          if (!FIRST) {
            const int2 nv = scr[(uint64_t)min(j, phi - 1) * 32];
            n_v = j + 1 <= phi ? nv : NEGP;
          }
          int32_t hoa, F;   // H - o and F of the cell above
          if (FIRST) {
            hoa = h_row0(mode, fe, j, o, e) - o;
            F = NEG32;
          } else {
            hoa = v.x - o;
            F = v.y;
          }
          int32_t d = diag;   // H - o above-left
          diag = hoa;
          // BYTES: byte a of the row table, sign-replicated into bytes 1-3
          const uint32_t sel = (uint32_t)a + ((uint32_t)a | 8u) * 0x1110u;
          uint32_t w[NW];
#pragma unroll
          for (int h = 0; h < NW; ++h) w[h] = 0;
#pragma unroll
          for (int r = 0; r < TROWS; ++r) {
            if (LAST ? r < rows : true) {
              // a gap is opened here exactly when the opening term wins or ties:
              // max(F - e, H_above - o) == H_above - o  <=>  H_above - o >= F - e
              F = __viaddmax_s32(F, -e, hoa);
              const uint32_t fbit = F == hoa ? 8u : 0u;
              E[r] = __viaddmax_s32(E[r], -e, Ho[r]);
              const uint32_t ebit = E[r] == Ho[r] ? 4u : 0u;
              const int32_t sv = BYTES ? (int32_t)prmt(qv[r], 0u, sel) : So[qv[r] + a];
              const int32_t m = d + sv;   // H_diag + S
              const int32_t v = local ? __vimax_s32_relu(m, max(E[r], F)) : __vimax3_s32(m, E[r], F);
              uint32_t src;
              if (local && v == 0) src = 3;
              else if (v == m) src = 0;
              else if (v == F) src = 1;
              else src = 2;
              const uint32_t nib = src | ebit | fbit;
              w[r >> 3] |= nib << (4 * (r & 7));
              d = Ho[r];
              Ho[r] = v - o;
              hoa = Ho[r];
            }
          }
          const uint64_t c = (uint64_t)(j - jlo);
#pragma unroll
          for (int h = 0; h < NW; ++h)
            if (!LAST || rows > 8 * h) Ds[(c * NW + h) * 32] = w[h];
          if (!LAST) scr[(uint64_t)(j - 1) * 32] = make_int2(hoa + o, F);
        }
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
      plo = jlo;
      phi = jhi;
    }
  }
  // decision nibble of (i, j); false outside the stored window (only a
  // corrupt decision could lead there)
  auto nibble = [&](int32_t i, int32_t j, uint32_t& nib) -> bool {
    const uint32_t r = (uint32_t)(i - 1) % TROWS, s = (uint32_t)(i - 1) / TROWS;
    const int32_t c = j - strip_jlo((int32_t)s * TROWS);
    if (c < 0 || c >= wc) return false;
    const uint32_t w = D[(((uint64_t)s * cols + (uint32_t)c) * NW + (r >> 3)) * 32];
    nib = (w >> (4 * (r & 7))) & 15u;
    return true;
  };
  RevCigar c;
  c.out = cig_tmp + jb.cig_off;
  int32_t i = ie, j = je;
  int st = 0;  // 0 = H, 1 = F, 2 = E
  const bool sg = mode == DSA_SEMIGLOBAL;
  for (int64_t guard = 2 * ((int64_t)ie + je) + 2; guard > 0; --guard) {
    if (st == 0 && i > 8 && j > 8) {
      // a match run: the next 8 cells along the diagonal (all off row 0 and
      // column 0) are read at once -- independent loads, one latency -- and
      // the leading M steps taken together; a cell outside the window counts
      // as the end of the run
      uint32_t notm = 0;
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        uint32_t nib = 0;
        const bool in = nibble(i - kk, j - kk, nib);
        notm |= ((!in || (nib & 3u) != 0u) ? 1u : 0u) << kk;
      }
      const int32_t L = notm ? __ffs(notm) - 1 : 8;
      if (L > 0) {
        c.emit_run(0, (uint32_t)L);
        i -= L;
        j -= L;
        guard -= L - 1;
        continue;
      }
    }
    if (st == 0) {
      if (sg && ((i == 0 && (fe & DSA_FREE_T_BEGIN)) || (j == 0 && (fe & DSA_FREE_Q_BEGIN)))) break;
      if (i == 0 || j == 0) {
        if (local) break;
        while (j > 0) { c.emit(2); --j; }
        while (i > 0) { c.emit(1); --i; }
        break;
      }
      uint32_t nib;
      if (!nibble(i, j, nib)) break;
      const uint32_t src = nib & 3u;
      if (src == 3) break;
      if (src == 0) { c.emit(0); --i; --j; }
      else st = src == 1 ? 1 : 2;
    } else if (st == 1) {
      uint32_t nib;
      if (i <= 0 || j <= 0 || !nibble(i, j, nib)) break;
      c.emit(1);
      if (nib & 8u) st = 0;
      --i;
    } else {
      uint32_t nib;
      if (i <= 0 || j <= 0 || !nibble(i, j, nib)) break;
      c.emit(2);
      if (nib & 4u) st = 0;
      --j;
    }
  }
  c.flush();
  dsa_hit* h = hits + jb.hit;
  h->q_begin = i;
  h->t_begin = j + jb.jlo;
  h->cigar_len = c.n;
  h->flags |= DSA_HIT_HAS_TRACEBACK;
}

// Exclusive scan of the jobs' CIGAR word counts (single CTA), then a reversed copy.
__global__ void __launch_bounds__(1024) k_cigar_offsets(dsa_hit* __restrict__ hits,
                                                        const TbJob* __restrict__ jobs,
                                                        uint32_t n, uint64_t base,
                                                        uint64_t* __restrict__ total) {
  __shared__ uint64_t part[1024];
  const uint32_t per = (n + 1023) / 1024;
  const uint32_t lo = threadIdx.x * per, hi = min(n, lo + per);
  uint64_t sum = 0;
  for (uint32_t x = lo; x < hi; ++x) sum += hits[jobs[x].hit].cigar_len;
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const uint64_t v = threadIdx.x >= (unsigned)off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  uint64_t run = base + part[threadIdx.x] - sum;
  for (uint32_t x = lo; x < hi; ++x) {
    dsa_hit* h = hits + jobs[x].hit;
    h->cigar_off = run;
    run += h->cigar_len;
  }
  if (threadIdx.x == 1023) *total += part[1023];
}

__global__ void k_cigar_copy(const dsa_hit* __restrict__ hits, const TbJob* __restrict__ jobs,
                             uint32_t n, const uint32_t* __restrict__ tmp,
                             uint32_t* __restrict__ out) {
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  const int lane = threadIdx.x & 31;
  for (uint32_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w < n; w += warps) {
    const dsa_hit h = hits[jobs[w].hit];
    const uint32_t* src = tmp + jobs[w].cig_off;
    for (uint32_t k = lane; k < h.cigar_len; k += 32) out[h.cigar_off + k] = src[h.cigar_len - 1 - k];
  }
}

}  // namespace

int launch_traceback(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int8_t* d_matrix,
                     int A, int o, int e, int mode, uint32_t fe, const TbJob* d_jobs,
                     uint32_t n_jobs, uint32_t* d_dir, uint32_t* d_cig_tmp, int2* d_scr,
                     dsa_hit* d_hits) {
  if (n_jobs == 0) return DSA_OK;
  const int threads = 128;
  uint64_t blocks = ((uint64_t)n_jobs * 32 + threads - 1) / threads;
  if (blocks > (uint64_t)ctx->sm_count * 16) blocks = (uint64_t)ctx->sm_count * 16;
  k_traceback<<<(unsigned)blocks, threads, 0, ctx->stream>>>(qs->d_codes, db->d_codes, d_matrix,
                                                             A, o, e, mode, fe, d_jobs, n_jobs,
                                                             d_dir, d_cig_tmp, d_scr, d_hits);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_traceback_thread(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs,
                            const int8_t* d_matrix, int A, int o, int e, int mode, uint32_t fe,
                            bool bytes_ok, const TbJob* d_jobs, uint32_t n_jobs, uint32_t* d_dir,
                            uint32_t* d_cig_tmp, int2* d_scr, dsa_hit* d_hits) {
  if (n_jobs == 0) return DSA_OK;
  const unsigned blocks = (n_jobs + 127) / 128;
  // substitution scores (S + o) by byte permute
  const bool bytes = A <= 4 && bytes_ok;
  auto kern = mode == DSA_LOCAL
                  ? (bytes ? k_traceback_thread<true, true> : k_traceback_thread<true, false>)
                  : (bytes ? k_traceback_thread<false, true> : k_traceback_thread<false, false>);
  kern<<<blocks, 128, 0, ctx->stream>>>(qs->d_codes, db->d_codes, d_matrix, A, o, e, mode, fe, d_jobs,
                                        n_jobs, d_dir, d_cig_tmp, d_scr, d_hits);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_cigar_compact(dsa_ctx* ctx, dsa_hit* d_hits, const TbJob* d_jobs, uint32_t n_jobs,
                         const uint32_t* d_cig_tmp, uint32_t* d_cigar, uint64_t base,
                         uint64_t* d_total) {
  if (n_jobs == 0) return DSA_OK;
  if (n_jobs >= 8192) {
    // many jobs: offsets from a device scan (the base is *d_total, which equals `base`)
    DSA_TRY(launch_cigar_offsets_scan(ctx, d_hits, d_jobs, n_jobs, d_total));
  } else {
    k_cigar_offsets<<<1, 1024, 0, ctx->stream>>>(d_hits, d_jobs, n_jobs, base, d_total);
    DSA_CUDA_TRY(cudaGetLastError());
    ++ctx->launches;
  }
  uint64_t blocks = ((uint64_t)n_jobs * 32 + 255) / 256;
  if (blocks > (uint64_t)ctx->sm_count * 16) blocks = (uint64_t)ctx->sm_count * 16;
  k_cigar_copy<<<(unsigned)blocks, 256, 0, ctx->stream>>>(d_hits, d_jobs, n_jobs, d_cig_tmp,
                                                          d_cigar);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

}  // namespace dsa
