// Internal declarations shared by the libdsa translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/dsa.h"

namespace dsa {

// -inf sentinels.  int32: far below any reachable score, so that adding a
// few hundred thousand gap penalties never wraps.  int16 packed lanes: the
// lower half of the int16 range; the packed kernels only run when every real
// value stays above it (local mode: values never fall below -(o + e)).
constexpr int32_t NEG32 = INT32_MIN / 4;
constexpr int32_t NEG16 = -16384;

// Launch / layout constants.
constexpr int GROUP = 32;          // targets per interleaved group (one warp)
constexpr int CHUNK = 16;          // residues per 16-byte interleaved word
constexpr int MAX_ALPHABET = 31;   // code 31 is reserved for padding

void set_error(const char* fmt, ...);

#define DSA_CUDA_TRY(expr)                                                        \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      dsa::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_),      \
                     __FILE__, __LINE__);                                         \
      return e_ == cudaErrorMemoryAllocation ? DSA_ERR_OOM : DSA_ERR_CUDA;         \
    }                                                                             \
  } while (0)

#define DSA_TRY(expr)            \
  do {                           \
    int rc_ = (expr);            \
    if (rc_ != DSA_OK) return rc_; \
  } while (0)

struct TbJob;

}  // namespace dsa

struct dsa_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;     // 0 = unlimited
  size_t in_use = 0;
  int sm_count = 0;
  cudaStream_t side = nullptr;   // second stream for work that overlaps the main kernels
  cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
  int32_t* d_status = nullptr;   // device status word written by kernels
  uint32_t* d_counters = nullptr;  // work-queue counters (reset per launch)
  uint64_t launches = 0;         // kernels launched through this context
  bool tune = true;              // may spend calls on autotuning (off for serving workers)
  // the context's own stream-ordered memory pool; it keeps freed memory
  // mapped (up to the budget) instead of returning it at every synchronize
  cudaMemPool_t pool = nullptr;
  // host staging reused across calls (large fresh vectors cost page faults)
  std::vector<dsa::TbJob> h_tb, h_tb2;
  std::mutex mu;

  int alloc(void** p, size_t bytes, cudaStream_t on = nullptr);
  void release(void* p, size_t bytes, cudaStream_t on = nullptr);
};

// A device-resident sequence set (database or queries).
struct dsa_db {
  dsa_ctx* ctx = nullptr;
  uint32_t n = 0;
  uint64_t n_res = 0;
  int A = 0;
  // input order
  uint8_t* d_codes = nullptr;     // n_res (+16 pad) bytes
  uint64_t* d_off = nullptr;      // n + 1
  uint32_t* d_len = nullptr;      // n
  std::vector<uint64_t> h_off;
  std::vector<uint32_t> h_len;
  uint32_t max_len = 0;
  // length-sorted (descending, ties by id), lane-interleaved copy; built on
  // first use by an all-vs-all search (ensure_interleaved), not at load
  std::mutex il_mu;
  bool il_ready = false;
  uint32_t* d_perm = nullptr;     // sorted position -> id
  uint32_t* d_slen = nullptr;     // sorted position -> length
  std::vector<uint32_t> h_perm;
  uint32_t n_groups = 0;
  uint8_t* d_il = nullptr;        // [group][chunk][lane][16 B]
  uint64_t* d_gbase = nullptr;    // byte offset of each group in d_il
  uint32_t* d_glen = nullptr;     // longest length in each group
  std::vector<uint64_t> h_gbase;
  std::vector<uint32_t> h_glen;
  uint64_t il_bytes = 0;
  size_t bytes_held = 0;
};

namespace dsa {
// Stream-ordered device buffer charged against the context's budget.
struct DevBuf {
  dsa_ctx* ctx = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { reset(); }
  int alloc(dsa_ctx* c, size_t n) {
    reset();
    ctx = c;
    bytes = n ? n : 16;
    return ctx->alloc(&p, bytes);
  }
  void reset() {
    if (p && ctx) ctx->release(p, bytes);
    p = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Builds the length-sorted, lane-interleaved copy of db (once; thread-safe),
// on ctx's stream, and waits for it.
int ensure_interleaved(dsa_ctx* ctx, const dsa_db* db);
}  // namespace dsa

struct dsa_res {
  dsa_ctx* ctx = nullptr;
  const dsa_db* db = nullptr;
  const dsa_db* queries = nullptr;
  dsa_db* owned_queries = nullptr;   // set when dsa_align_batch uploaded them
  int mode = 0;
  uint32_t free_ends = 15;
  int A = 0, gap_open = 0, gap_extend = 0;
  std::vector<int8_t> matrix;
  bool pssm = false;   // scored with position-specific profiles: no traceback
  uint32_t flags = 0;
  uint64_t n_hits = 0;
  dsa_hit* d_hits = nullptr;
  uint32_t* d_cigar = nullptr;
  uint64_t n_cigar = 0;
  uint64_t cigar_bytes = 0;
  std::vector<dsa_hit> h_hits;
  std::vector<uint32_t> h_cigar;
  bool host_valid = false;
  uint64_t cells = 0;
  uint64_t n_rerun = 0;
  // DSA_TIMING: one begin/end event pair per phase
  static constexpr int NPHASE = 5;
  cudaEvent_t ev[2 * NPHASE] = {};
  bool used[NPHASE] = {};
  uint64_t phase_cells[NPHASE] = {};
  // checkpoints of long explicit pairs (band boundary rows), kept for traceback
  int2* d_bnd = nullptr;
  size_t bnd_bytes = 0;
  std::vector<uint64_t> long_bnd_off;   // per hit: boundary offset, or UINT64_MAX
  std::vector<int32_t> long_n;          // per hit: window length of a long pair
};

namespace dsa {
// Phase timer over a result's events (no-op unless the result has DSA_TIMING).
enum Phase { PH_INTER = 0, PH_INTRA = 1, PH_INT32 = 2, PH_HITS = 3, PH_TRACE = 4 };
void phase_begin(dsa_res* res, Phase p, cudaStream_t on = nullptr);
void phase_end(dsa_res* res, Phase p, cudaStream_t on = nullptr);
}  // namespace dsa

namespace dsa {

// ---- kernels' host-side launchers (one translation unit each) ----

// Work item of the generic int32 kernel: one (query, target window) pair.
struct PairJob {
  uint64_t t_start;   // absolute residue offset of the target window in the DB codes
  uint64_t scratch;   // offset (in int2 elements) of this job's boundary row
  uint32_t q;         // query index
  uint32_t n;         // target window length
  uint32_t out;       // output slot
  uint32_t pad;       // 1: rerun of a saturated packed result (sets the hit's rerun flag)
};

struct Scores {      // structure-of-arrays output of the score pass
  int32_t* score = nullptr;
  int32_t* q_end = nullptr;
  int32_t* t_end = nullptr;
  uint8_t* flag = nullptr;
};

// Plain / generic exact int32 kernel: any mode, any pair list.  With
// d_jobs == nullptr the jobs are every DB target (input order) against query
// `fixed_q`, boundary rows at the targets' residue offsets.
int launch_generic_int32(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int32_t* d_prof,
                         const uint64_t* d_prof_off, const PairJob* d_jobs, uint64_t n_jobs,
                         uint32_t fixed_q, int2* d_scratch, int mode, uint32_t fe, int o, int e,
                         uint8_t flag_value, Scores out);

// Per-query int32 profile P[a][i] = S[q_i][a] (rows a = 0..A-1, row stride = m),
// or the position-specific row d_pssm[q_off + i][a] when d_pssm is given.
int launch_profile_int32(dsa_ctx* ctx, const dsa_db* qs, const int8_t* d_matrix,
                         const int8_t* d_pssm, int A, int32_t* d_prof, const uint64_t* d_prof_off);

// Interleaved DB build (dsa_db_load).
int launch_interleave(dsa_ctx* ctx, dsa_db* db);

// Packed 16-bit local kernels (all queries x all targets).
//
// A plan is a list of units; each unit is a run of strips (`rows` query rows)
// whose low 16-bit half follows one stream of queries and whose high half
// another.  Per strip, a StripMeta record names the query of each half and
// the strip's index inside that query; the packed profile holds, per strip,
// R residue rows x `rows` query rows of int16x2 (S + o, padding = -16384).
struct StripMeta {
  uint32_t qa, ka;   // low half: query id (NONE = no query), strip index in it | LAST bit
  uint32_t qb, kb;   // high half
};
constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr uint32_t LAST = 0x80000000u;   // in ka / kb: the query ends in this strip

struct PackedPlan {
  uint32_t n_units = 0;
  uint32_t n_strips = 0;
  StripMeta* d_meta = nullptr;     // n_strips
  uint32_t* d_sbase = nullptr;     // first strip of each unit
  uint32_t* d_ns = nullptr;        // strips of each unit
  uint32_t* d_prof = nullptr;      // n_strips x R x pitch words
  int R = 0;                       // profile rows = A + 1 (last = padding)
  int rows = 32;                   // query rows per strip
  int pitch = 32;                  // words per profile row (rows padded to 128 bytes)
};

// Inter-sequence kernel work: items = (unit, first group of a block of 8).
struct InterWork {
  uint32_t* d_items = nullptr;     // 2 words per item
  uint32_t n_items = 0;
  uint32_t max_glen = 0;           // longest group it touches (boundary-row length)
};
// Wavefront kernel work: items = (long target index, unit).
struct IntraWork {
  const uint32_t* d_long_ids = nullptr;
  uint32_t* d_items = nullptr;     // 2 words per item
  uint32_t n_items = 0;
  uint32_t max_long_len = 0;
};

// d_pssm: position-specific rows (one per query residue of the set) or NULL.
// anchored: strips end at each query's last row (global / semi-global kernel),
// with `tpad` as the S + o of padding rows and absent queries.
int launch_strip_profile(dsa_ctx* ctx, const dsa_db* qs, const int8_t* d_matrix,
                         const int8_t* d_pssm, int A, int o, const PackedPlan& plan,
                         bool anchored = false, int tpad = 0);
int launch_inter_local16(dsa_ctx* ctx, const dsa_db* db, const PackedPlan& plan,
                         const InterWork& work, int o, int e, int smax, Scores out,
                         uint32_t n_targets_out);
// Global / semi-global form of the inter-sequence kernel (end-anchored
// strips); every target of the database, mode DSA_GLOBAL or DSA_SEMIGLOBAL.
int launch_inter_glob16(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const PackedPlan& plan,
                        const InterWork& work, int mode, uint32_t fe, int o, int e, int smax,
                        int smin, Scores out, uint32_t n_targets_out);
int inter_blocks_per_sm();
constexpr int INTER_WARPS = 8;
constexpr int INTER_ROWS = 28;         // strip rows of the packed inter-sequence kernels
constexpr int INTER_ROWS_SHORT = 20;   // their short-strip variant (short queries)

// Long-target intra-sequence (wavefront) kernel; each unit of `plan` must
// hold one query per half (no stream switches).  Runs on `stream`
// (allocation and release of its scratch are ordered there).
int launch_intra_local16(dsa_ctx* ctx, cudaStream_t stream, const dsa_db* db,
                         const PackedPlan& plan, const IntraWork& work, int o, int e, int smax,
                         Scores out, uint32_t n_targets_out);
// Its global / semi-global form: `plan` built with end-anchored 32-row strips.
int launch_intra_glob16(dsa_ctx* ctx, cudaStream_t stream, const dsa_db* db, const dsa_db* qs,
                        const PackedPlan& plan, const IntraWork& work, int mode, uint32_t fe,
                        int o, int e, int smax, int smin, Scores out, uint32_t n_targets_out);

// Top-k per query over a dense [n_queries][n_targets] score matrix.
int launch_topk(dsa_ctx* ctx, const Scores& s, uint32_t n_queries, uint32_t n_targets,
                uint32_t k, dsa_hit* d_hits);
// Dense pair results -> hit array.
// d_pairs: the explicit pairs (device), or nullptr for an all-vs-all matrix.
int launch_fill_hits(dsa_ctx* ctx, const Scores& s, const dsa_pair* d_pairs, uint64_t n,
                     uint32_t n_targets, dsa_hit* d_hits);

// Traceback of hits.
// Thread-per-hit traceback: query rows per strip (a multiple of 8; each strip
// column keeps TB_STRIP / 8 words of 4-bit decisions per hit).
constexpr int TB_STRIP = 8;
constexpr int TB_STRIP_WORDS = TB_STRIP / 8;
struct TbJob {
  uint64_t q_start;   // absolute offset of the query in the query codes
  uint64_t t_start;   // absolute offset of the target window in the DB codes
  uint64_t dir_off;   // word offset of this job's direction matrix
  uint64_t cig_off;   // word offset of this job's CIGAR capacity (reverse-order scratch)
  uint64_t scr_off;   // int2 offset of this job's band-boundary row
  int32_t ie, je;     // 1-based result cell (rectangle to recompute)
  uint32_t hit;       // hit index
  uint32_t wpr;       // direction words per row
  int32_t jlo;        // first target column of the recomputed band (0 = whole rectangle);
                      // > 0: column jlo is a wall (H = -inf below row 0)
  // thread-per-hit kernel: diagonal window of each TB_STRIP-row strip (relative to
  // the band): wc stored columns from clamp(i0 + 1 + dlo, 1, je - wc + 1)
  int32_t dlo;
  int32_t wc;
  // index of band 0's entry in the per-band window table (int2: first
  // stored column, stored columns) when the traceback narrows each band from
  // the checkpoint rows; the table's widths are at most wc
  uint32_t win_off;
};
// Score-derived traceback windows, shared by the host staging and the
// device staging of the traceback (see k_traceback.cu for the argument).
struct TbBounds {
  int mode;
  uint32_t fe;
  int o, e;
  int smax_pos;      // max(S, 0)
  bool band_ok;      // semi-global with a free target begin and e > 0: column band
  bool diag_ok;      // max(S, 0) + 2e > 0: total-gap bound
  bool from_origin;  // paths start at (0, 0): two-sided diagonal window
};

// Diagonals dlo..dhi of every optimal path reaching (ie, je); false: none narrower.
__host__ __device__ inline bool tb_diag_window(const TbBounds& B, int32_t ie, int32_t je,
                                               int32_t score, int64_t& dlo, int64_t& dhi) {
  if (!B.diag_ok) return false;
  // at most (ie + je - g) / 2 M columns, each scoring at most max(S, 0), and
  // gap runs costing at least g e + (o - e) when g > 0
  const int64_t num = (int64_t)B.smax_pos * ((int64_t)ie + je) - 2 * (int64_t)score -
                      2 * ((int64_t)B.o - B.e);
  const int64_t gmax = num < 0 ? 0 : num / ((int64_t)B.smax_pos + 2 * (int64_t)B.e);
  const int64_t dn = (int64_t)je - ie;
  if (!B.from_origin) {   // gaps after the cell only
    dlo = dn - gmax;
    dhi = dn + gmax;
    return true;
  }
  const int64_t adn = dn < 0 ? -dn : dn;
  if (gmax < adn) return false;
  const int64_t half = (gmax - adn) / 2;
  dlo = (dn < 0 ? dn : 0) - half;
  dhi = (dn > 0 ? dn : 0) + half;
  return true;
}

// The thread-per-hit job of a hit with end cell (ie, je) (1-based) and score:
// column band (free target begin) and the diagonal window of its TB_STRIP-row strips.
__host__ __device__ inline void tb_short_job(const TbBounds& B, int32_t ie, int32_t je,
                                             int32_t score, uint64_t q_start, uint64_t t_start,
                                             uint32_t hit, TbJob& j) {
  j = TbJob{};
  j.ie = ie;
  j.je = je;
  j.hit = hit;
  j.q_start = q_start;
  j.t_start = t_start;
  int64_t dlo = -(int64_t)ie, dhi = je;   // default: whole rows
  if (B.band_ok) {
    // deletions on any path reaching the hit: score <= ie max(S, 0) - (o + (k - 1) e)
    const int64_t o = B.o, e = B.e;
    const int64_t slack = (int64_t)ie * B.smax_pos - score;
    const int64_t kmax = slack < o ? 0 : (slack - o) / e + 1;
    const int64_t jlo = (int64_t)je - ie - kmax;
    if (jlo > 0) {
      j.jlo = (int32_t)jlo;
      j.t_start += (uint64_t)jlo;
      j.je -= (int32_t)jlo;
    }
    // insertions: each one removes an M (at most max S) and costs at least e
    // (the first o): score <= max(S, 0)(ie - k) - (o + (k - 1) e)
    const int64_t imax = slack < o ? 0 : (slack - o + e) / (B.smax_pos + e);
    // a cell (i, j) on the path: (je - j) - (ie - i) = D after - I after
    const int64_t dn = (int64_t)j.je - ie;
    dlo = dn - kmax;
    dhi = dn + imax;
  } else {
    int64_t a, b;
    if (tb_diag_window(B, ie, je, score, a, b)) {
      dlo = a;
      dhi = b;
    }
  }
  j.dlo = (int32_t)(dlo > -(int64_t)ie ? dlo : -(int64_t)ie);
  const int64_t wc = TB_STRIP + dhi - j.dlo;
  j.wc = (int32_t)(wc < j.je ? wc : j.je);
  j.wpr = (uint32_t)((j.je + 7) / 8);
}

// Device-side staging kernels (k_tbstage.cu).
int launch_scan_u64(dsa_ctx* ctx, uint64_t* d_data, uint64_t n, uint64_t* d_total);
// d_out = the jobs of d_in stably ordered by (rows, stored columns).
int launch_tb_order(dsa_ctx* ctx, const TbJob* d_in, uint64_t n, TbJob* d_out);
int launch_tb_stage(dsa_ctx* ctx, const dsa_hit* d_hits, uint64_t n, const uint64_t* d_q_off,
                    const uint64_t* d_t_off, const TbBounds& B, TbJob* d_full, uint64_t* d_valid,
                    uint32_t* d_not_small);
int launch_tb_compact(dsa_ctx* ctx, const TbJob* d_full, const uint64_t* d_pos,
                      const uint64_t* d_total, uint64_t n, TbJob* d_jobs);
int launch_tb_layout(dsa_ctx* ctx, TbJob* d_jobs, uint64_t n, uint64_t* d_gdir, uint64_t* d_gscr,
                     uint64_t* d_jcig, uint64_t* d_totals);
int launch_cigar_offsets_scan(dsa_ctx* ctx, dsa_hit* d_hits, const TbJob* d_jobs, uint64_t n,
                              uint64_t* d_base);

// Device staging of the traceback of every hit of a result on the thread path
// (jobs built, compacted and laid out on the device).  Returns DSA_OK, or
// TB_STAGE_FALLBACK when some hit needs another path or the decisions would
// take more than `dir_limit` words in one launch (nothing was changed).
constexpr int TB_STAGE_FALLBACK = 1;
int traceback_device_staged(dsa_ctx* ctx, dsa_res* res, const TbBounds& B, uint64_t dir_limit);

int launch_traceback(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int8_t* d_matrix,
                     int A, int o, int e, int mode, uint32_t fe, const TbJob* d_jobs,
                     uint32_t n_jobs, uint32_t* d_dir, uint32_t* d_cig_tmp, int2* d_scr,
                     dsa_hit* d_hits);
// Reverse each job's CIGAR words into `d_cigar` starting at `base`, packed in
// job order; total words written are added to *d_total.
// One thread per hit; TbJob.dir_off = group base + lane, .wpr = the group's
// column count, .scr_off = group scratch base + lane (layouts interleaved by 32).
// bytes_ok: every S + o fits int8 (with A <= 4 the byte-permute form is used)
int launch_traceback_thread(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs,
                            const int8_t* d_matrix, int A, int o, int e, int mode, uint32_t fe,
                            bool bytes_ok, const TbJob* d_jobs, uint32_t n_jobs, uint32_t* d_dir,
                            uint32_t* d_cig_tmp, int2* d_scr, dsa_hit* d_hits);
int launch_cigar_compact(dsa_ctx* ctx, dsa_hit* d_hits, const TbJob* d_jobs, uint32_t n_jobs,
                         const uint32_t* d_cig_tmp, uint32_t* d_cigar, uint64_t base,
                         uint64_t* d_total);

// Long explicit pairs: band-pipelined score pass and checkpointed traceback.
struct LongJob {
  uint64_t q_start, t_start;   // absolute offsets of query and target window
  uint64_t bnd_off;            // int2 offset of the job's band boundary rows (bands x n)
  uint64_t prog_off;           // offset of the job's per-band progress counters
  uint64_t cand_off;           // offset of the job's per-band candidates
  int32_t m, n;
  uint32_t out;                // output slot (pair index)
  uint32_t pad;
};
struct LongTbJob {
  uint64_t q_start, t_start;
  uint64_t bnd_off;            // checkpoints of the score pass
  uint64_t dir_off;            // word offset of the decisions (bands x TB_BAND x wpr words)
  uint64_t cig_off;
  int32_t n;                   // boundary row length (the pair's window length)
  int32_t ie, je;
  uint32_t hit;
  uint32_t wpr;                // decision words per row: ceil(wc / 8)
  // Diagonal band: rows of band b (BAND rows from i0 = b * BAND) keep the wc
  // columns from jlo_b = clamp(i0 + 1 + dlo, 1, je - wc + 1); wc = je and
  // dlo = 0 recompute whole rows.
  int32_t dlo;
  int32_t wc;
  // index of band 0's entry in the per-band window table (int2: first
  // stored column, stored columns) when the traceback narrows each band from
  // the checkpoint rows; the table's widths are at most wc
  uint32_t win_off;
};
// bytes_ok: every S + o fits int8 (with A <= 4 the byte-permute form is used).
// blocks_per_sm > 0 caps the resident blocks per SM (fewer warps per SM run
// the bands' chains faster; the autotuner chooses).
int launch_long_score(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int8_t* d_matrix,
                      int A, int o, int e, int mode, uint32_t fe, bool bytes_ok,
                      const LongJob* d_jobs, uint32_t n_jobs, const uint32_t* d_items,
                      uint32_t n_items, int2* d_bnd, uint32_t* d_prog, void* d_cands, Scores out,
                      int blocks_per_sm = 0);
// Checkpointed traceback of long pairs, part 0: each band's window of the
// bands named by `items` (2 words (job, band) each) from the checkpoint rows:
// the columns where an optimal path to the hit can cross the band's top and
// bottom rows (H there plus the best score still reachable from the cell
// reaches the hit's score), within the job's diagonal window; writes
// d_win[win_off + band] and the widest band of each job into d_maxw (zeroed
// before).  smax_pos: max(S, 0).
int launch_long_tb_windows(dsa_ctx* ctx, cudaStream_t stream, const LongTbJob* d_jobs,
                           const uint32_t* d_items, uint32_t n_items, const int2* d_bnd,
                           const dsa_hit* d_hits, int mode, uint32_t fe, int o, int e,
                           int smax_pos, int2* d_win, int32_t* d_maxw);
// Part 1: the decisions of the bands named by `items`; d_win: the per-band
// windows (nullptr: every band takes the job's diagonal window).
int launch_long_tb_fill(dsa_ctx* ctx, cudaStream_t stream, const dsa_db* db, const dsa_db* qs,
                        const int8_t* d_matrix, int A, int o, int e, int mode, uint32_t fe,
                        const LongTbJob* d_jobs, const uint32_t* d_items, uint32_t n_items,
                        const int2* d_bnd, uint32_t* d_dir, const int2* d_win = nullptr);
// Part 1, packed (k_long_tb16.cu): two traceback bands per warp, one per
// 16-bit half, for alphabets of up to 4 letters with every S + o in int8 and
// scores within long_tb16_range_ok; d_units holds 4 words per unit (job,
// band, job, band; the second job NONE for an empty half), d_win the
// per-band windows.  Writes the same decisions as launch_long_tb_fill.
bool long_tb16_range_ok(int o, int e, int smax, int smin);
int launch_long_tb_fill16(dsa_ctx* ctx, cudaStream_t stream, const dsa_db* db, const dsa_db* qs,
                          const int8_t* d_matrix, int A, int o, int e, int mode, uint32_t fe,
                          const LongTbJob* d_jobs, const uint32_t* d_units, uint32_t n_units,
                          const int2* d_bnd, uint32_t* d_dir, const int2* d_win);
// Part 2: one warp per job walks its decisions back from the end cell
// (every band of those jobs filled before, in stream order).
int launch_long_tb_walk(dsa_ctx* ctx, cudaStream_t stream, const LongTbJob* d_jobs,
                        uint32_t n_jobs, int mode, uint32_t fe, const uint32_t* d_dir,
                        uint32_t* d_cig_tmp, dsa_hit* d_hits, const int2* d_win = nullptr);
// Per-band end-cell candidate of a long pair, ordered (score desc, j asc,
// i asc); has = 0: none.
struct LongCand {
  int32_t s, i, j;
  int32_t has;
};
// Two long pairs aligned together by the packed band pipeline, one in each
// 16-bit half (indices into the LongJob array; b = NONE: the high half is
// empty); the unit has its own per-band progress counters.
struct LongPair16 {
  uint32_t a, b;
  uint64_t prog_off;
};
// Packed (int16x2) form of the long-pair score pass for alphabets of up to 4
// letters with every S + o in int8 and scores whose range passes
// long16_range_ok; writes the same boundary rows, checkpoints and per-band
// candidates as launch_long_score and reduces them into `out`.  Local mode
// also takes d_litems (2 words (pair, band) for every band of every pair,
// n_litems of them) and n_slots (the candidate slots, one per pair band):
// the score pass keeps each band's best and a snapshot of the block where it
// first appeared, and a second kernel locates the first cell of the pair's
// best from those.
bool long16_range_ok(int o, int e, int smax, int smin);
int launch_long_score16(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int8_t* d_matrix,
                        int A, int o, int e, int mode, uint32_t fe, const LongJob* d_jobs,
                        uint32_t n_jobs, const LongPair16* d_pjobs, const uint32_t* d_items,
                        uint32_t n_items, int2* d_bnd, uint32_t* d_prog, void* d_cands,
                        Scores out, int blocks_per_sm = 0, const uint32_t* d_litems = nullptr,
                        uint32_t n_litems = 0, uint64_t n_slots = 0);
int launch_long_reduce(dsa_ctx* ctx, const LongJob* d_jobs, uint32_t n_jobs, const void* d_cands,
                       int mode, uint32_t fe, int o, int e, Scores out);
size_t long_cand_size();
int long_band_rows();   // rows of a score-pass band
int long_ckpt_rows();   // rows between traceback checkpoints (a traceback band)
constexpr uint64_t LONG_PAIR_CELLS = 1ull << 22;   // explicit pairs at least this big run banded

// Packed int16x2 kernel for explicit short pairs: two pairs of equal query
// length per thread.  q_* / t_* are absolute offsets of the query and of the
// target window; out_hi = NONE when the high half is empty.
struct Pair16Job {
  uint64_t q_lo, q_hi, t_lo, t_hi;
  int32_t m, n_lo, n_hi;
  uint32_t out_lo, out_hi;
  uint32_t pad;
};
// bytes: A <= 4 and every S + o in [-128, 127] (byte-permute substitution
// form); rows: strip rows of the byte form, 16 or pairs16_wide_rows() (the
// wide variant); the shared-memory form always uses 16
int launch_pairs16(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int8_t* d_matrix, int A,
                   int o, int e, int mode, uint32_t fe, int smax, bool bytes, int rows,
                   const Pair16Job* d_jobs, uint32_t n_jobs, uint32_t max_n, Scores out);
int pairs16_wide_rows();

// Device planning of explicit pairs (k_pairplan.cu).
struct PairPlanParams {
  uint32_t n_queries, n_targets;
  int64_t w16;          // largest |S|, o, e: int16 range bound (m + n) * w16 + o
  int32_t o, e;
  bool local16;         // local mode with the saturation flag: every size fits
  bool packed_ok;       // the packed int16 form is allowed
};
struct PairPlanStats {   // field order is used by the kernels' atomics
  uint64_t cells;        // cells of all valid pairs
  uint64_t cells16;      // cells of the packed pairs
  uint64_t n_other;      // valid pairs for the long or int32 paths
  uint64_t first_bad;    // smallest index of an out-of-range pair, or UINT64_MAX
  uint64_t n_jobs;       // packed jobs (two pairs of equal query length each)
  uint32_t max_t_len;    // longest window of a valid pair
  uint32_t pad;
};
// Range check, class, sort key ((m << 32) | t_len) and value (pair index) of
// every packed pair; hist[m] = packed pairs of query length m, jcnt[m] = their
// jobs; L = longest query + 2 entries (the last stays 0).
int launch_pair_classify(dsa_ctx* ctx, const dsa_pair* d_pairs, uint64_t n, const dsa_db* qs,
                         const dsa_db* db, const PairPlanParams& P, uint64_t* d_key,
                         uint32_t* d_idx, uint64_t* d_hist, uint64_t L, uint64_t* d_jcnt,
                         PairPlanStats* d_stats);
// Stable sort of (key, value) by key; d_key / d_val are set to the buffer
// pair that holds the result (the input pair or the *2 pair).
int launch_pair_sort(dsa_ctx* ctx, uint64_t*& d_key, uint32_t*& d_val, uint64_t* d_key2,
                     uint32_t* d_val2, uint64_t n, uint32_t max_m, uint32_t max_t);
// Job list from the sorted packed pairs (hist and jcnt are scanned in place).
int launch_pair_build_jobs(dsa_ctx* ctx, const uint64_t* d_key, const uint32_t* d_val, uint64_t n,
                           uint64_t* d_hist, uint64_t* d_jcnt, uint64_t L, const dsa_pair* d_pairs,
                           const dsa_db* qs, const dsa_db* db, Pair16Job* d_jobs);

// Issue-rate probe; bounded-wait self-test.
int run_issue_probe(dsa_ctx* ctx, int form, double* rate);
int run_selftest_wait(dsa_ctx* ctx, int kind, uint64_t limit_ns);

}  // namespace dsa
