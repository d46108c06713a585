// Inter-sequence local alignment kernel, packed int16x2 with DPX.
//
// Work decomposition (the paper's per-core SIMD alignment of one query against
// many references, Sec. II.B.1, re-laid out for a GB300 SM):
//   * the database is length-sorted and interleaved so that warp w of a CTA
//     owns 32 consecutive sorted targets, one per lane, and reads one 16-byte
//     word (16 residues) per lane per 16 columns, coalesced;
//   * the two 16-bit halves of every DP register follow two query streams
//     (queries concatenated strip by strip, balanced in length), so one DPX
//     instruction advances two cells; per-strip metadata says when a half
//     starts a new query (its best and its top boundary restart) or ends one
//     (its result is written);
//   * a query is processed in strips of W = INTER_ROWS (28) rows held in registers; the loop
//     runs over the target's residues; the strip's bottom row (H - o and the
//     next row's F) goes to a per-CTA boundary buffer and is read back by the
//     next strip through a small shared-memory ring that per-thread
//     asynchronous copies fill two 4-column blocks ahead of the arithmetic;
//   * the query profile of each strip (R residue rows x W query rows of
//     int16x2 = R x 4W bytes) is staged into shared memory by TMA bulk copies,
//     double-buffered on two mbarriers, in 8 replicas whose start addresses
//     are rotated by 16 bytes so that the 8 lanes of each quarter-warp read
//     8 different bank groups whatever residues they hold;
//   * a persistent grid pops (stream pair, block of 8 groups) items from a
//     work queue ordered longest-first.
//
// Cell update for one row (Gotoh, local), with Ho = H - o and profile S + o:
//   E  = max(E - e, Ho_left)            addmax2u
//   t  = max(Ho_diag + (S + o), E)      addmax2u
//   H  = max(t, F, 0)                   max3_2u
//   Ho = H - o                          32-bit subtract
//   F' = max(F - e, Ho)                 addmax2u  (F of the next row)
// and the column maximum of H (max3_2u every two rows) for the end cell.
// Values are kept in offset binary (each half + 0x8000): the maxima are the
// unsigned DPX forms, additions of constants wrap identically, and since
// H >= 0, the low half of H + 0x8000 is at least 0x8000 > o, so H - o is a
// plain 32-bit subtraction with no borrow between the halves -- an integer
// add the compiler may issue outside the ALU pipe that carries the maxima.
//
// End cell (smallest target end j, then smallest query end i, among cells
// holding the best score): the column maximum is compared with the running
// best lowered by one while j is still below the best's column, so ties at an
// earlier column also trigger.  A (rare) trigger only parks the column in its
// half's area of shared memory; at the end of the strip the last parked
// column of each improved half is scanned for its first row holding the
// maximum.  No scan runs inside the column loop.
//
// Saturation: in local mode no value falls below -(o + e), and a value can
// exceed the best seen so far by at most max(S), so if the best stays at or
// below 32767 - max(S) no lane wrapped.  Pairs above that are flagged for the
// exact int32 rerun.
#include "dsa_internal.cuh"
#include "dpx.cuh"

#include <type_traits>

namespace dsa {
namespace {

// query rows per strip: a template parameter of both kernels (INTER_ROWS,
// or the shorter INTER_ROWS_SHORT that wastes fewer padding rows on short
// queries); the autotuner picks one per workload shape
constexpr int NW = INTER_WARPS;  // warps per CTA
constexpr int NT = NW * 32;
constexpr int NCOPY = 8;         // profile replicas (one per lane of a quarter-warp)
constexpr uint32_t RING = 3;     // boundary-row ring slots (blocks of 4 columns)

struct InterArgs {
  const uint8_t* il;
  const uint64_t* gbase;
  const uint32_t* glen;
  const uint32_t* perm;
  uint32_t n_targets;
  uint32_t n_groups;
  const uint32_t* prof;            // [strip][a][32] int16x2
  const StripMeta* meta;
  const uint32_t* sbase;
  const uint32_t* nstrips;
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

// Profile rows are padded to 128 bytes (PITCH words): with 8 replicas whose
// starts are 16 bytes apart mod 128, the 16-byte word k of row a in replica c
// then sits in bank group (c + k) mod 8 whatever a is, so the 8 lanes of a
// quarter-warp never share a bank group.
constexpr int PITCH = 32;
static_assert(INTER_ROWS <= PITCH && INTER_ROWS_SHORT <= PITCH,
              "strip rows must fit one padded profile row");

// Bytes between profile replicas: at least one strip profile (R x PITCH x 4 B),
// a multiple of 16, and 16 (mod 128) so replica c starts in bank group c.
__host__ __device__ __forceinline__ uint32_t replica_stride(int R) {
  const uint32_t units = ((uint32_t)R * PITCH * 4u + 15u) / 16u;
  return ((units + 6u) / 8u * 8u + 1u) * 16u;
}

__device__ __forceinline__ void issue_strip(const InterArgs& A, uint8_t* buf, uint64_t* bar,
                                            const uint32_t* src, uint32_t cstride) {
  const uint32_t bytes = (uint32_t)A.R * PITCH * 4u;
  mbar_arrive_expect_tx(bar, bytes * NCOPY);
#pragma unroll
  for (int c = 0; c < NCOPY; ++c) bulk_g2s(buf + c * cstride, src, bytes, bar);
}

template <int W>
__global__ void __launch_bounds__(NT, 2) k_inter_local16(const InterArgs A) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bars[2];
  __shared__ uint32_t s_item;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const uint32_t cstride = replica_stride(A.R);
  const uint32_t bufbytes = NCOPY * cstride;
  // column parking areas for the end-cell search, one 16-bit half each: [row][thread]
  volatile int16_t* const park_lo = reinterpret_cast<volatile int16_t*>(smem + 2 * bufbytes);
  volatile int16_t* const park_hi = park_lo + W * NT;
  // boundary-row ring: RING blocks of 4 columns, [slot][k][thread], filled by
  // per-thread asynchronous copies two blocks ahead of the arithmetic
  uint2* const ring = reinterpret_cast<uint2*>(smem + 2 * bufbytes + 2 * W * NT * sizeof(int16_t)) + tid;
  const uint32_t strip_words = (uint32_t)A.R * PITCH;
  constexpr uint32_t BIAS2 = 0x80008000u;                  // offset-binary 0 in both halves
  const uint32_t neg_e2 = A.neg_e2;                         // -e, added mod 2^16
  const uint32_t mo2 = A.neg_o2 ^ BIAS2;                    // -o (offset binary)
  const uint32_t o2 = ((uint32_t)A.o << 16) | (uint32_t)A.o;
  const uint32_t NEG2 = pack2(NEG16, NEG16) ^ BIAS2;

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
    const uint32_t ns = A.nstrips[p];
    const uint32_t sb = A.sbase[p];
    const uint32_t* psrc = A.prof + (size_t)sb * strip_words;
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
      const StripMeta md = A.meta[sb + s];
      const uint32_t ka = md.ka & ~LAST, kb = md.kb & ~LAST;
      // a half whose query starts here restarts its best and takes the
      // row-0 boundary (H = 0) instead of the previous strip's bottom row
      if (ka == 0) { best_lo = 0; bj_lo = 0; bi_lo = 0; }
      if (kb == 0) { best_hi = 0; bj_hi = 0; bi_hi = 0; }
      const uint32_t keep = (ka == 0 ? 0u : 0x0000FFFFu) | (kb == 0 ? 0u : 0xFFFF0000u);
      const bool first = keep == 0;
      const int ia = (int)ka * W, ib = (int)kb * W;   // first row of the strip inside each query

      uint32_t Ho[W], E[W];
#pragma unroll
      for (int r = 0; r < W; ++r) {
        Ho[r] = mo2;
        E[r] = NEG2;
      }
      uint32_t diag = mo2;
      uint2* scr = scr_base;
      uint4 rv = make_uint4(0, 0, 0, 0);
      // Packed trigger threshold per half, tested as cm > thr with
      // thr = max(best - 1, 0): every column whose maximum reaches the best
      // (or is the first positive one) triggers; the exact rule (strictly
      // better, or equal at a smaller column) is applied in the trigger path.
      uint32_t thr2 = 0;
      auto set_thr = [&]() { thr2 = pack2(max(best_lo - 1, 0), max(best_hi - 1, 0)) ^ BIAS2; };
      set_thr();
      int pend = 0;   // bit 0 / 1: low / high half improved in this strip

      // the previous strip's bottom row, block c4x of 4 columns, into ring slot
      auto fetch = [&](uint32_t c4x, uint32_t slot) {
        if (c4x < ncol) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            cp_async8(ring + (slot * 4 + k) * NT, scr + (uint64_t)(c4x + k) * NT);
        }
        cp_async_commit();
      };
      if (!first) {
        fetch(0, 0);
        fetch(4, 1);
      }
      uint32_t slot = 0;
      for (uint32_t c4 = 0; c4 < ncol; c4 += 4, slot = slot == RING - 1 ? 0 : slot + 1) {
        if ((c4 & 15u) == 0) rv = __ldg(res + (c4 >> 4) * 32u);
        const uint32_t sel = (c4 >> 2) & 3u;
        const uint32_t word = sel == 0 ? rv.x : sel == 1 ? rv.y : sel == 2 ? rv.z : rv.w;
        uint2 top[4];
        if (!first) {
          fetch(c4 + 8, slot == 0 ? RING - 1 : slot - 1);   // slot (slot + 2) mod 3
          cp_async_wait<2>();                               // block c4 has landed
#pragma unroll
          for (int k = 0; k < 4; ++k) top[k] = ring[(slot * 4 + k) * NT];
          if (keep != 0xFFFFFFFFu) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              top[k].x = (top[k].x & keep) | (mo2 & ~keep);
              top[k].y = (top[k].y & keep) | (mo2 & ~keep);
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) top[k] = make_uint2(mo2, mo2);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t a = (word >> (8 * k)) & 0xFFu;
          const uint4* prow = reinterpret_cast<const uint4*>(pbuf + a * (PITCH * 4u));
          uint32_t F = top[k].y;
          uint32_t d = diag;
          diag = top[k].x;
          uint32_t cm = BIAS2, hprev = BIAS2;
#pragma unroll
          for (int q4 = 0; q4 < W / 4; ++q4) {
            const uint4 pv = prow[q4];
            const uint32_t pr[4] = {pv.x, pv.y, pv.z, pv.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = q4 * 4 + u;
              const uint32_t old = Ho[r];
              E[r] = addmax2u(E[r], neg_e2, old);
              const uint32_t t = addmax2u(d, pr[u], E[r]);
              const uint32_t h = max3_2u(t, F, BIAS2);
              Ho[r] = h - o2;
              F = addmax2u(F, neg_e2, Ho[r]);
              d = old;
              if (r & 1) cm = max3_2u(cm, hprev, h);
              else hprev = h;
            }
          }
          scr[(uint64_t)(c4 + k) * NT] = make_uint2(Ho[W - 1], F);
          // end-cell tracking for column j: trigger when cm > thr (per half)
          const int j = (int)c4 + k + 1;
          if (__vmaxu2(cm, thr2) != thr2) {   // some half has cm > thr
            const int cl = lo16(cm ^ BIAS2), ch = hi16(cm ^ BIAS2);
            const int thr_lo = best_lo - (j < bj_lo ? 1 : 0);
            const int thr_hi = best_hi - (j < bj_hi ? 1 : 0);
            // rare: a half improved.  Park the column in that half's area of
            // shared memory; its first row holding the maximum is looked up
            // once, at the end of the strip (a later trigger of the same half
            // supersedes this one)
            if (cl > thr_lo) {
#pragma unroll
              for (int r = 0; r < W; ++r) park_lo[r * NT + tid] = (int16_t)lo16(Ho[r] ^ BIAS2);
              best_lo = cl; bj_lo = j; pend |= 1;
            }
            if (ch > thr_hi) {
#pragma unroll
              for (int r = 0; r < W; ++r) park_hi[r * NT + tid] = (int16_t)hi16(Ho[r] ^ BIAS2);
              best_hi = ch; bj_hi = j; pend |= 2;
            }
            set_thr();
          }
        }
      }
      cp_async_wait<0>();   // nothing in flight into the ring past the strip
      if (pend & 1) {   // first row of the last improving column, low half
        const int want = best_lo - A.o;
        int rr = W - 1;
        for (int r = W - 1; r >= 0; --r)
          if (park_lo[r * NT + tid] == want) rr = r;
        bi_lo = ia + rr + 1;
      }
      if (pend & 2) {
        const int want = best_hi - A.o;
        int rr = W - 1;
        for (int r = W - 1; r >= 0; --r)
          if (park_hi[r * NT + tid] == want) rr = r;
        bi_hi = ib + rr + 1;
      }
      if (tvalid) {   // queries that end in this strip: write their results
        const uint32_t orig = A.perm[st];
        if ((md.ka & LAST) && md.qa != NONE) {
          const uint64_t idx = (uint64_t)md.qa * A.n_out_t + orig;
          A.o_score[idx] = best_lo;
          A.o_qend[idx] = best_lo > 0 ? bi_lo - 1 : -1;
          A.o_tend[idx] = best_lo > 0 ? bj_lo - 1 : -1;
          A.o_flag[idx] = best_lo > A.T ? 1 : 0;
        }
        if ((md.kb & LAST) && md.qb != NONE) {
          const uint64_t idx = (uint64_t)md.qb * A.n_out_t + orig;
          A.o_score[idx] = best_hi;
          A.o_qend[idx] = best_hi > 0 ? bi_hi - 1 : -1;
          A.o_tend[idx] = best_hi > 0 ? bj_hi - 1 : -1;
          A.o_flag[idx] = best_hi > A.T ? 1 : 0;
        }
      }
      __syncthreads();
      if (tid == 0 && s + 2 < ns) {
        fence_proxy_async_smem();
        issue_strip(A, smem + b * bufbytes, &bars[b], psrc + (s + 2) * strip_words, cstride);
      }
    }

  }
}

// ---- global and semi-global form (Sec. II.C.2: DNW, DSG) ----
//
// Same work decomposition, staging and cell update as k_inter_local16, with
// three differences:
//   * no floor at 0: H = max(t, F) (max3_2u(t, F, t));
//   * end-anchored strips: a query of m rows starts (W - m % W) % W rows into
//     its first strip, so row m is the bottom register of its last strip.
//     The padding rows above the query reproduce the row-0 boundary exactly
//     (their S + o is 0 for a boundary -(o + (j-1)e), o for a free target
//     begin), and the real rows' column-0 values are set per row;
//   * result cells: the column at the lane's own target end n is parked in
//     shared memory when the loop reaches it (its bottom row is H[m][n]; with
//     a free query end its rows are scanned after the strip, smallest i
//     first), and with a free target end the bottom row of the last strip is
//     tracked column by column (smallest j first).  The candidates are merged
//     by (score desc, j asc, i asc).
// Range: every value of a real cell is at least -(3o + (m + n)e) (the path
// along the boundaries), so pairs with 4o + (m + n + 2)e + |min S| + 64 below
// 2^15 never wrap downward, and H - o never borrows between the halves; the
// "-inf" of E and F is -2^15 + e, whose - e does not wrap.  Upward, as in
// local mode, only the diagonal step raises a value, by at most max(S), so if
// no column maximum of H passes 32767 - max(S), no cell wrapped.
// Pairs outside either bound are flagged for the exact int32 rerun.  Columns
// past a lane's own target end (its group's longer targets) are computed
// with a profile value of 0 for the padding residue; they feed no real cell,
// and the running maximum leaves them out.
struct GlobArgs {
  int mode;
  uint32_t fe;
  int e;
  int smin;
  uint32_t hmax2;         // 32767 - max(S) in both halves, offset binary
  const uint32_t* qlen;   // query lengths
  const uint32_t* slen;   // target lengths in the length-sorted order
};

// TB: free target begin (row 0 is 0), TE: free target end (row m is
// tracked): compile-time, so each form carries only the state it uses.
template <int W, bool TB, bool TE>
__global__ void __launch_bounds__(NT, 2) k_inter_glob16(const InterArgs A, const GlobArgs G) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bars[2];
  __shared__ uint32_t s_item;
  // per thread and half, kept out of registers (read once per strip): best
  // of column n so far and its row (free query end; starts at (0, n)), and
  // the column of row m's best (free target end)
  __shared__ int s_cb[2][NT], s_ci[2][NT], s_rj[2][NT];
  // per thread: bit h set when half h of the current query passed 32767 - max S
  __shared__ uint32_t s_sat[NT];
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const uint32_t cstride = replica_stride(A.R);
  const uint32_t bufbytes = NCOPY * cstride;
  // the column at the lane's own target end, parked for the result: [row][thread]
  volatile uint32_t* const park = reinterpret_cast<volatile uint32_t*>(smem + 2 * bufbytes);
  uint2* const ring = reinterpret_cast<uint2*>(smem + 2 * bufbytes + W * NT * sizeof(uint32_t)) + tid;
  const uint32_t strip_words = (uint32_t)A.R * PITCH;
  constexpr uint32_t BIAS2 = 0x80008000u;
  const uint32_t neg_e2 = A.neg_e2;
  const uint32_t o2 = ((uint32_t)A.o << 16) | (uint32_t)A.o;
  const int o = A.o, e = G.e;
  const uint32_t NEGG2 = ((uint32_t)e << 16) | (uint32_t)e;   // -2^15 + e in both halves
  const uint32_t neg_e4 = pack2(-4 * e, -4 * e);              // four columns of the boundary
  const bool sg = G.mode == DSA_SEMIGLOBAL;
  constexpr bool tb_free = TB;
  constexpr bool te_free = TE;
  const bool qb_free = sg && (G.fe & DSA_FREE_Q_BEGIN);
  const bool qe_free = sg && (G.fe & DSA_FREE_Q_END);
  // boundary values of H: row 0 at column j, column 0 at row i (rows <= 0:
  // row 0 itself or the padding rows above a query)
  auto row0 = [&](int j) { return (j == 0 || tb_free) ? 0 : -(o + (j - 1) * e); };
  auto col0 = [&](int i) { return (i <= 0 || qb_free) ? 0 : -(o + (i - 1) * e); };
  auto off2 = [](int lo, int hi) { return pack2(lo, hi) ^ BIAS2; };

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
    const uint32_t ns = A.nstrips[p];
    const uint32_t sb = A.sbase[p];
    const uint32_t* psrc = A.prof + (size_t)sb * strip_words;
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
    const int nl = tvalid ? (int)G.slen[st] : -1;   // this lane's target length
    const uint4* res = reinterpret_cast<const uint4*>(A.il + (gvalid ? A.gbase[g] : 0)) + lane;

    s_sat[tid] = 0;

    for (uint32_t s = 0; s < ns; ++s) {
      const int b = s & 1;
      const uint32_t par = b ? (phase1 & 1u) : (phase0 & 1u);
      const bool ok = mbar_wait_bounded(&bars[b], par, WAIT_LIMIT_NS);
      if (b) ++phase1; else ++phase0;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicExch(A.status, DSA_ERR_DEVICE_TIMEOUT);
        mbar_wait_bounded(&bars[0], phase0 & 1u, WAIT_LIMIT_NS);
        mbar_wait_bounded(&bars[1], phase1 & 1u, WAIT_LIMIT_NS);
        return;
      }
      const uint8_t* pbuf = smem + b * bufbytes + (lane & 7) * cstride;
      const StripMeta md = A.meta[sb + s];
      const uint32_t ka = md.ka & ~LAST, kb = md.kb & ~LAST;
      // the query rows of each half in this strip: m, the 0-based row of the
      // strip's first row (negative: padding rows), whether row m is here
      auto geom = [&](uint32_t q, uint32_t kq, int& m, int& i0, bool& last) {
        m = q != NONE ? (int)G.qlen[q] : 0;
        i0 = (int)(kq & ~LAST) * W - (W - m % W) % W;
        last = (kq & LAST) && q != NONE;
      };
      int ma, mb, ia0, ib0;
      bool last_a, last_b;
      geom(md.qa, md.ka, ma, ia0, last_a);
      geom(md.qb, md.kb, mb, ib0, last_b);
      if (ka == 0) { s_cb[0][tid] = row0(nl); s_ci[0][tid] = 0; s_sat[tid] &= ~1u; }
      if (kb == 0) { s_cb[1][tid] = row0(nl); s_ci[1][tid] = 0; s_sat[tid] &= ~2u; }
      const uint32_t keep = (ka == 0 ? 0u : 0x0000FFFFu) | (kb == 0 ? 0u : 0xFFFF0000u);
      const bool first = keep == 0;

      uint32_t Ho[W], E[W];
#pragma unroll
      for (int r = 0; r < W; ++r) {
        Ho[r] = off2(col0(ia0 + r + 1) - o, col0(ib0 + r + 1) - o);
        E[r] = NEGG2;
      }
      uint32_t diag = off2(col0(ia0) - o, col0(ib0) - o);
      // row-0 boundary as (H - o, F of row 1) = (B(j) - o, B(j) - o) at the
      // first column of the current block of 4 (only read where a half starts
      // a query)
      uint32_t bt = off2(row0(1) - o, row0(1) - o);
      // bottom row of a last strip (row m), free target end: best H - o over
      // j <= n, smallest j first, from the candidate (m, 0); a half that does
      // not end here holds the largest value, which nothing exceeds
      uint32_t rthr = 0xFFFFFFFFu;
      s_rj[0][tid] = 0;
      s_rj[1][tid] = 0;
      if (te_free) {
        if (last_a) rthr = (rthr & 0xFFFF0000u) | (off2(col0(ma) - o, 0) & 0xFFFFu);
        if (last_b) rthr = (rthr & 0x0000FFFFu) | (off2(0, col0(mb) - o) & 0xFFFF0000u);
      }
      uint2* scr = scr_base;
      uint4 rv = make_uint4(0, 0, 0, 0);

      auto fetch = [&](uint32_t c4x, uint32_t slot) {
        if (c4x < ncol) {
#pragma unroll
          for (int k = 0; k < 4; ++k)
            cp_async8(ring + (slot * 4 + k) * NT, scr + (uint64_t)(c4x + k) * NT);
        }
        cp_async_commit();
      };
      if (!first) {
        fetch(0, 0);
        fetch(4, 1);
      }
      uint32_t slot = 0;
      for (uint32_t c4 = 0; c4 < ncol; c4 += 4, slot = slot == RING - 1 ? 0 : slot + 1) {
        if ((c4 & 15u) == 0) rv = __ldg(res + (c4 >> 4) * 32u);
        const uint32_t sel = (c4 >> 2) & 3u;
        const uint32_t word = sel == 0 ? rv.x : sel == 1 ? rv.y : sel == 2 ? rv.z : rv.w;
        uint2 top[4];
        if (!first) {
          fetch(c4 + 8, slot == 0 ? RING - 1 : slot - 1);
          cp_async_wait<2>();
#pragma unroll
          for (int k = 0; k < 4; ++k) top[k] = ring[(slot * 4 + k) * NT];
          if (keep != 0xFFFFFFFFu) {
            uint32_t bk = bt;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              top[k].x = (top[k].x & keep) | (bk & ~keep);
              top[k].y = (top[k].y & keep) | (bk & ~keep);
              if (!tb_free) bk = __vadd2(bk, neg_e2);
            }
          }
        } else {
          uint32_t bk = bt;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            top[k] = make_uint2(bk, bk);
            if (!tb_free) bk = __vadd2(bk, neg_e2);
          }
        }
        if (keep != 0xFFFFFFFFu && !tb_free) bt = __vadd2(bt, neg_e4);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint32_t a = (word >> (8 * k)) & 0xFFu;
          const uint4* prow = reinterpret_cast<const uint4*>(pbuf + a * (PITCH * 4u));
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
              E[r] = addmax2u(E[r], neg_e2, old);
              const uint32_t t = addmax2u(d, pr[u], E[r]);
              const uint32_t h = max3_2u(t, F, t);
              Ho[r] = h - o2;
              F = addmax2u(F, neg_e2, Ho[r]);
              d = old;
              if (r & 1) cm = max3_2u(cm, hprev, h);
              else hprev = h;
            }
          }
          scr[(uint64_t)(c4 + k) * NT] = make_uint2(Ho[W - 1], F);
          const int j = (int)c4 + k + 1;
          // upward range test of the column (rare); columns past the lane's
          // target end feed no real cell (values only move right and down)
          // and may wrap in a long group: left out
          if (__vmaxu2(cm, G.hmax2) != G.hmax2 && j <= nl)
            s_sat[tid] |= ((cm & 0xFFFFu) > (G.hmax2 & 0xFFFFu) ? 1u : 0u) |
                          ((cm >> 16) > (G.hmax2 >> 16) ? 2u : 0u);
          if (j == nl) {   // the lane's own target end: park the column
#pragma unroll
            for (int r = 0; r < W; ++r) park[r * NT + tid] = Ho[r];
          }
          if (te_free) {
            const uint32_t cur = Ho[W - 1];
            if (__vmaxu2(cur, rthr) != rthr && j <= nl) {
              if ((cur & 0xFFFFu) > (rthr & 0xFFFFu)) {
                rthr = (rthr & 0xFFFF0000u) | (cur & 0xFFFFu);
                s_rj[0][tid] = j;
              }
              if ((cur >> 16) > (rthr >> 16)) {
                rthr = (rthr & 0x0000FFFFu) | (cur & 0xFFFF0000u);
                s_rj[1][tid] = j;
              }
            }
          }
        }
      }
      cp_async_wait<0>();
      if (tvalid) {
        // H of half `sh` (0 / 16) from a packed H - o in offset binary
        auto hval = [&](uint32_t w, int sh) { return (int)((w >> sh) & 0xFFFFu) - 0x8000 + o; };
        auto finish = [&](int h, uint32_t q, uint32_t kq) {
          const int sh = 16 * h;
          int m, i0;
          bool last;
          geom(q, kq, m, i0, last);
          int cb = s_cb[h][tid], ci = s_ci[h][tid];
          const int rj = s_rj[h][tid];
          if (qe_free) {   // column n of this strip's real rows, smallest i first
            for (int r = 0; r < W; ++r) {
              const int i = i0 + r + 1;
              const int v = hval(park[r * NT + tid], sh);
              if (i >= 1 && v > cb) { cb = v; ci = i; }
            }
          }
          s_cb[h][tid] = cb;
          s_ci[h][tid] = ci;
          if (!last) return;
          int bs = hval(park[(W - 1) * NT + tid], sh), bi = m, bj = nl;   // (m, n)
          if (qe_free && (cb > bs || (cb == bs && ci < bi))) { bs = cb; bi = ci; }
          if (te_free) {
            const int rvv = hval(rthr, sh);
            if (rvv > bs || (rvv == bs && rj < bj)) { bs = rvv; bi = m; bj = rj; }
          }
          const bool up = (s_sat[tid] >> h) & 1u;
          const int64_t low = 4ll * o + (int64_t)(m + nl + 2) * e + (G.smin < 0 ? -G.smin : 0) + 64;
          const uint64_t idx = (uint64_t)q * A.n_out_t + A.perm[st];
          A.o_score[idx] = bs;
          A.o_qend[idx] = bi - 1;
          A.o_tend[idx] = bj - 1;
          A.o_flag[idx] = (up || low >= 32768) ? 1 : 0;
        };
        const StripMeta mr = A.meta[sb + s];   // reloaded: not kept live over the column loop
        if (mr.qa != NONE) finish(0, mr.qa, mr.ka);
        if (mr.qb != NONE) finish(1, mr.qb, mr.kb);
      }
      __syncthreads();
      if (tid == 0 && s + 2 < ns) {
        fence_proxy_async_smem();
        issue_strip(A, smem + b * bufbytes, &bars[b], psrc + (s + 2) * strip_words, cstride);
      }
    }
  }
}

// Packed profile of every strip: [strip][residue a][row r] int16x2 =
// (S[qa_i][a] + o, S[qb_i][a] + o) with i = rows * (strip index in the query) + r;
// rows past a query's end, absent queries and the padding residue a = A get
// NEG16.  With a position-specific profile P (row per query residue of the
// set, Sec. II.C.2's user-defined scoring) the score is P[qoff + i][a].
//
// End-anchored form (anchored = 1, the global / semi-global kernels): a query
// of m rows starts (rows - m % rows) % rows rows into its first strip, so its
// last row is the bottom row of its last strip.  The padding rows above it,
// rows past its end, absent queries and the padding residue get values that
// keep every cell inside the int16 range: `tpad` (S + o) for padding rows and
// absent queries, 0 for the padding residue of a real row.
__global__ void k_strip_profile(const uint8_t* __restrict__ qcodes,
                                const uint64_t* __restrict__ qoff, const uint32_t* __restrict__ qlen,
                                const StripMeta* __restrict__ meta, uint32_t n_strips,
                                const int8_t* __restrict__ S, const int8_t* __restrict__ P, int A,
                                int R, int rows, int pitch, int o, int anchored, int tpad,
                                uint32_t* __restrict__ prof) {
  auto sub = [&](uint32_t q, int i, int a) -> int {
    const uint64_t k = qoff[q] + (uint64_t)i;
    return P ? (int)P[k * A + a] : (int)S[qcodes[k] * A + a];
  };
  auto anchored_val = [&](uint32_t q, uint32_t kq, int r, int a) -> int {
    if (q == NONE) return tpad;
    const int m = (int)qlen[q];
    const int i = (int)(kq & ~LAST) * rows + r - (rows - m % rows) % rows;
    // rows above the query, and (in a unit of the wavefront kernel, whose
    // halves can differ in strips) rows past its end
    if (i < 0 || i >= m) return tpad;
    if (a >= A) return 0;
    return sub(q, i, a) + o;
  };
  const uint64_t total = (uint64_t)n_strips * R * pitch;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < total;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t s = (uint32_t)(x / ((uint64_t)R * pitch));
    const int a = (int)((x / pitch) % (uint64_t)R);
    const int r = (int)(x % pitch);
    const StripMeta md = meta[s];
    int lo = NEG16, hi = NEG16;
    if (r >= rows) {
      // row padding, never read
    } else if (anchored) {
      lo = anchored_val(md.qa, md.ka, r, a);
      hi = anchored_val(md.qb, md.kb, r, a);
    } else if (a < A && md.qa != NONE) {
      const int i = (int)(md.ka & ~LAST) * rows + r;
      if (i < (int)qlen[md.qa]) lo = sub(md.qa, i, a) + o;
    }
    if (!anchored && r < rows && a < A && md.qb != NONE) {
      const int i = (int)(md.kb & ~LAST) * rows + r;
      if (i < (int)qlen[md.qb]) hi = sub(md.qb, i, a) + o;
    }
    prof[x] = pack2(lo, hi);
  }
}

}  // namespace

int inter_blocks_per_sm() { return 2; }

int launch_strip_profile(dsa_ctx* ctx, const dsa_db* qs, const int8_t* d_matrix,
                         const int8_t* d_pssm, int A, int o, const PackedPlan& plan,
                         bool anchored, int tpad) {
  if (plan.n_strips == 0) return DSA_OK;
  const uint64_t total = (uint64_t)plan.n_strips * plan.R * plan.pitch;
  uint64_t blocks = std::min<uint64_t>((total + 255) / 256, (uint64_t)ctx->sm_count * 8);
  k_strip_profile<<<(unsigned)blocks, 256, 0, ctx->stream>>>(qs->d_codes, qs->d_off, qs->d_len,
                                                            plan.d_meta, plan.n_strips, d_matrix,
                                                            d_pssm, A, plan.R, plan.rows,
                                                            plan.pitch, o, anchored ? 1 : 0, tpad,
                                                            plan.d_prof);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_inter_local16(dsa_ctx* ctx, const dsa_db* db, const PackedPlan& plan,
                         const InterWork& work, int o, int e, int smax, Scores out,
                         uint32_t n_targets_out) {
  if (work.n_items == 0) return DSA_OK;
  InterArgs A;
  A.il = db->d_il; A.gbase = db->d_gbase; A.glen = db->d_glen; A.perm = db->d_perm;
  A.n_targets = db->n; A.n_groups = db->n_groups;
  A.prof = plan.d_prof; A.meta = plan.d_meta; A.sbase = plan.d_sbase; A.nstrips = plan.d_ns;
  A.R = plan.R;
  A.neg_o2 = (uint32_t)((-o) & 0xFFFF) | ((uint32_t)((-o) & 0xFFFF) << 16);
  A.neg_e2 = (uint32_t)((-e) & 0xFFFF) | ((uint32_t)((-e) & 0xFFFF) << 16);
  A.o = o;
  A.T = 32767 - (smax > 0 ? smax : 0);
  A.items = work.d_items; A.n_items = work.n_items;
  A.counter = ctx->d_counters;
  const int grid = (int)std::min<uint64_t>(work.n_items, (uint64_t)ctx->sm_count * inter_blocks_per_sm());
  const uint64_t cols = ((uint64_t)work.max_glen + 3) & ~3ull;
  A.scratch_cols = cols;
  const size_t scr_bytes = (size_t)grid * cols * NT * sizeof(uint2);
  void* scr = nullptr;
  DSA_TRY(ctx->alloc(&scr, scr_bytes));
  A.scratch = static_cast<uint2*>(scr);
  A.o_score = out.score; A.o_qend = out.q_end; A.o_tend = out.t_end; A.o_flag = out.flag;
  A.n_out_t = n_targets_out;
  A.status = ctx->d_status;
  const size_t smem = 2ull * NCOPY * replica_stride(plan.R) + 2ull * plan.rows * NT * sizeof(int16_t) +
                      (size_t)RING * 4 * NT * sizeof(uint2);
  auto kern = plan.rows == INTER_ROWS_SHORT ? k_inter_local16<INTER_ROWS_SHORT>
                                            : k_inter_local16<INTER_ROWS>;
  if (plan.rows != INTER_ROWS && plan.rows != INTER_ROWS_SHORT) {
    ctx->release(scr, scr_bytes);
    set_error("strip height %d has no kernel", plan.rows);
    return DSA_ERR_INVALID_ARG;
  }
  // the attribute belongs to the current device: set it on every launch (cheap)
  DSA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DSA_CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, sizeof(uint32_t), ctx->stream));
  kern<<<grid, NT, smem, ctx->stream>>>(A);
  ++ctx->launches;
  cudaError_t err = cudaGetLastError();
  ctx->release(scr, scr_bytes);
  if (err != cudaSuccess) {
    set_error("k_inter_local16 launch: %s", cudaGetErrorString(err));
    return DSA_ERR_CUDA;
  }
  return DSA_OK;
}

int launch_inter_glob16(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const PackedPlan& plan,
                        const InterWork& work, int mode, uint32_t fe, int o, int e, int smax,
                        int smin, Scores out, uint32_t n_targets_out) {
  if (work.n_items == 0) return DSA_OK;
  InterArgs A;
  A.il = db->d_il; A.gbase = db->d_gbase; A.glen = db->d_glen; A.perm = db->d_perm;
  A.n_targets = db->n; A.n_groups = db->n_groups;
  A.prof = plan.d_prof; A.meta = plan.d_meta; A.sbase = plan.d_sbase; A.nstrips = plan.d_ns;
  A.R = plan.R;
  A.neg_o2 = (uint32_t)((-o) & 0xFFFF) | ((uint32_t)((-o) & 0xFFFF) << 16);
  A.neg_e2 = (uint32_t)((-e) & 0xFFFF) | ((uint32_t)((-e) & 0xFFFF) << 16);
  A.o = o;
  A.T = 32767 - (smax > 0 ? smax : 0);
  A.items = work.d_items; A.n_items = work.n_items;
  A.counter = ctx->d_counters;
  GlobArgs G;
  G.mode = mode; G.fe = fe; G.e = e; G.smin = smin;
  G.qlen = qs->d_len; G.slen = db->d_slen;
  G.hmax2 = ((uint32_t)(A.T + 0x8000) << 16) | (uint32_t)(A.T + 0x8000);
  const int grid = (int)std::min<uint64_t>(work.n_items, (uint64_t)ctx->sm_count * inter_blocks_per_sm());
  const uint64_t cols = ((uint64_t)work.max_glen + 3) & ~3ull;
  A.scratch_cols = cols;
  const size_t scr_bytes = (size_t)grid * cols * NT * sizeof(uint2);
  void* scr = nullptr;
  DSA_TRY(ctx->alloc(&scr, scr_bytes));
  A.scratch = static_cast<uint2*>(scr);
  A.o_score = out.score; A.o_qend = out.q_end; A.o_tend = out.t_end; A.o_flag = out.flag;
  A.n_out_t = n_targets_out;
  A.status = ctx->d_status;
  const size_t smem = 2ull * NCOPY * replica_stride(plan.R) + (size_t)plan.rows * NT * sizeof(uint32_t) +
                      (size_t)RING * 4 * NT * sizeof(uint2);
  const bool sg = mode == DSA_SEMIGLOBAL;
  const bool tb = sg && (fe & DSA_FREE_T_BEGIN), te = sg && (fe & DSA_FREE_T_END);
  auto pick = [&](auto w) {
    constexpr int Wc = decltype(w)::value;
    return tb ? (te ? k_inter_glob16<Wc, true, true> : k_inter_glob16<Wc, true, false>)
              : (te ? k_inter_glob16<Wc, false, true> : k_inter_glob16<Wc, false, false>);
  };
  auto kern = plan.rows == INTER_ROWS_SHORT ? pick(std::integral_constant<int, INTER_ROWS_SHORT>{})
                                            : pick(std::integral_constant<int, INTER_ROWS>{});
  if (plan.rows != INTER_ROWS && plan.rows != INTER_ROWS_SHORT) {
    ctx->release(scr, scr_bytes);
    set_error("strip height %d has no kernel", plan.rows);
    return DSA_ERR_INVALID_ARG;
  }
  DSA_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  DSA_CUDA_TRY(cudaMemsetAsync(ctx->d_counters, 0, sizeof(uint32_t), ctx->stream));
  kern<<<grid, NT, smem, ctx->stream>>>(A, G);
  ++ctx->launches;
  cudaError_t err = cudaGetLastError();
  ctx->release(scr, scr_bytes);
  if (err != cudaSuccess) {
    set_error("k_inter_glob16 launch: %s", cudaGetErrorString(err));
    return DSA_ERR_CUDA;
  }
  return DSA_OK;
}

}  // namespace dsa
