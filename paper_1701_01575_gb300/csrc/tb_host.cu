// Traceback of reported hits (the alignment object's location and CIGAR,
// Sec. II.B.1): host staging of the jobs, the device-staged path for large
// batches, chunking by decision memory, and the checkpointed band traceback
// of long pairs and big hits.  The arithmetic runs in k_traceback.cu,
// k_tbstage.cu and k_long.cu.
#include "host_util.cuh"

#include <algorithm>
#include <cstdlib>
#include <numeric>
#include <string>

namespace dsa {

int fetch_hits(dsa_res* res) {
  dsa_ctx* ctx = res->ctx;
  if (res->host_valid) return DSA_OK;
  res->h_hits.resize(res->n_hits);
  if (res->n_hits)
    DSA_CUDA_TRY(cudaMemcpyAsync(res->h_hits.data(), res->d_hits, res->n_hits * sizeof(dsa_hit),
                                 cudaMemcpyDeviceToHost, ctx->stream));
  res->h_cigar.resize(res->n_cigar);
  if (res->n_cigar)
    DSA_CUDA_TRY(cudaMemcpyAsync(res->h_cigar.data(), res->d_cigar, res->n_cigar * 4,
                                 cudaMemcpyDeviceToHost, ctx->stream));
  DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  res->host_valid = true;
  return DSA_OK;
}

int traceback_device_staged(dsa_ctx* ctx, dsa_res* res, const TbBounds& B, uint64_t dir_limit) {
  const uint64_t n = res->n_hits;
  const dsa_db* db = res->db;
  const dsa_db* qs = res->queries;
  DevBuf d_full, d_valid, d_cnt;
  DSA_TRY(d_full.alloc(ctx, n * sizeof(TbJob)));
  DSA_TRY(d_valid.alloc(ctx, n * sizeof(uint64_t)));
  DSA_TRY(d_cnt.alloc(ctx, 8 * sizeof(uint64_t)));
  uint64_t* cnt = d_cnt.as<uint64_t>();   // [0] valid jobs, [1..3] layout totals, [4] not small
  DSA_CUDA_TRY(cudaMemsetAsync(cnt, 0, 8 * sizeof(uint64_t), ctx->stream));
  phase_begin(res, PH_TRACE);   // the phase includes the staging
  DSA_TRY(launch_tb_stage(ctx, res->d_hits, n, qs->d_off, db->d_off, B, d_full.as<TbJob>(),
                          d_valid.as<uint64_t>(), reinterpret_cast<uint32_t*>(cnt + 4)));
  DSA_TRY(launch_scan_u64(ctx, d_valid.as<uint64_t>(), n, cnt + 0));
  uint64_t h_cnt[8];
  DSA_CUDA_TRY(cudaMemcpyAsync(h_cnt, cnt, sizeof h_cnt, cudaMemcpyDeviceToHost, ctx->stream));
  DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if ((uint32_t)h_cnt[4] != 0) return TB_STAGE_FALLBACK;   // a hit needs another path
  const uint64_t nv = h_cnt[0];
  if (nv == 0) return DSA_OK;
  DevBuf d_jobs, d_gdir, d_gscr, d_jcig;
  const uint64_t n_groups = (nv + 31) / 32;
  DSA_TRY(d_jobs.alloc(ctx, nv * sizeof(TbJob)));
  DSA_TRY(launch_tb_compact(ctx, d_full.as<TbJob>(), d_valid.as<uint64_t>(), cnt + 0, n,
                            d_jobs.as<TbJob>()));
  d_full.reset();
  d_valid.reset();
  {
    // a warp of the thread kernel runs as long as its longest hit: order the
    // jobs by (rows, stored columns) so each group of 32 does similar work
    DevBuf d_sorted;
    DSA_TRY(d_sorted.alloc(ctx, nv * sizeof(TbJob)));
    DSA_TRY(launch_tb_order(ctx, d_jobs.as<TbJob>(), nv, d_sorted.as<TbJob>()));
    std::swap(d_jobs.p, d_sorted.p);
    std::swap(d_jobs.bytes, d_sorted.bytes);
  }
  DSA_TRY(d_gdir.alloc(ctx, n_groups * sizeof(uint64_t)));
  DSA_TRY(d_gscr.alloc(ctx, n_groups * sizeof(uint64_t)));
  DSA_TRY(d_jcig.alloc(ctx, nv * sizeof(uint64_t)));
  DSA_TRY(launch_tb_layout(ctx, d_jobs.as<TbJob>(), nv, d_gdir.as<uint64_t>(), d_gscr.as<uint64_t>(),
                           d_jcig.as<uint64_t>(), cnt + 1));
  DSA_CUDA_TRY(cudaMemcpyAsync(h_cnt, cnt, sizeof h_cnt, cudaMemcpyDeviceToHost, ctx->stream));
  DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  const uint64_t dir = h_cnt[1], scr = h_cnt[2], cap = h_cnt[3];
  if (dir > dir_limit) return TB_STAGE_FALLBACK;   // the host staging splits it into chunks
  d_gdir.reset();
  d_gscr.reset();
  d_jcig.reset();
  // grow the result's CIGAR array by the capacity bound
  const uint64_t old_n = res->n_cigar;
  void* newp = nullptr;
  DSA_TRY(ctx->alloc(&newp, (old_n + cap) * sizeof(uint32_t)));
  if (old_n)
    DSA_CUDA_TRY(cudaMemcpyAsync(newp, res->d_cigar, old_n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (res->d_cigar) ctx->release(res->d_cigar, res->cigar_bytes);
  res->d_cigar = (uint32_t*)newp;
  res->cigar_bytes = (old_n + cap) * sizeof(uint32_t);
  DevBuf d_mat, d_dir, d_cig, d_scr;
  DSA_TRY(d_mat.alloc(ctx, res->A * res->A));
  DSA_CUDA_TRY(cudaMemcpyAsync(d_mat.p, res->matrix.data(), res->A * res->A, cudaMemcpyHostToDevice,
                               ctx->stream));
  DSA_TRY(d_dir.alloc(ctx, dir * 4));
  DSA_TRY(d_cig.alloc(ctx, cap * 4));
  DSA_TRY(d_scr.alloc(ctx, scr * sizeof(int2)));
  DSA_CUDA_TRY(cudaMemcpyAsync(cnt, &old_n, sizeof(uint64_t), cudaMemcpyHostToDevice, ctx->stream));
  DSA_TRY(launch_traceback_thread(ctx, db, qs, d_mat.as<int8_t>(), res->A, res->gap_open,
                                  res->gap_extend, res->mode, res->free_ends,
                                  s_plus_o_fits_int8(res->matrix.data(), res->A, res->gap_open),
                                  d_jobs.as<TbJob>(),
                                  (uint32_t)nv, d_dir.as<uint32_t>(), d_cig.as<uint32_t>(),
                                  d_scr.as<int2>(), res->d_hits));
  DSA_TRY(launch_cigar_compact(ctx, res->d_hits, d_jobs.as<TbJob>(), (uint32_t)nv,
                               d_cig.as<uint32_t>(), res->d_cigar, old_n, cnt));
  phase_end(res, PH_TRACE);
  uint64_t total = 0;
  DSA_CUDA_TRY(cudaMemcpyAsync(&total, cnt, sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
  DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  res->n_cigar = total;
  res->host_valid = false;
  return DSA_OK;
}

namespace {

// Decision memory of one traceback launch, in 32-bit words: `dflt`, or the
// smaller DSA_TB_CHUNK_WORDS (a test hook that makes a batch span several
// chunks).
uint64_t tb_chunk_words(uint64_t dflt) {
  if (const char* env = getenv("DSA_TB_CHUNK_WORDS")) {
    const uint64_t w = strtoull(env, nullptr, 10);
    if (w > 0 && w < dflt) return w;
  }
  return dflt;
}

constexpr uint64_t TB_SHORT_CHUNK_WORDS = 1ull << 30;   // 4 GiB of decisions
constexpr uint64_t TB_LONG_CHUNK_WORDS = 8ull << 30;    // 32 GiB of decisions

// The jobs of one traceback call, by path.
struct TbPlan {
  std::vector<TbJob>* tjobs = nullptr;   // thread per hit (the context's reused buffer)
  std::vector<TbJob> jobs;               // warp per hit
  std::vector<LongTbJob> ljobs;          // long pairs (checkpoint rows of the score pass)
  std::vector<LongJob> bscore;           // big hits: a checkpointed score pass ...
  std::vector<LongTbJob> bjobs;          // ... then the long-pair traceback
  uint64_t b_bnd = 0, b_bands = 0;       // checkpoint words and bands of the big hits
  uint64_t cap_total = 0;                // CIGAR capacity bound
};

// Device state shared by the chunks of one call.
struct TbRun {
  dsa_ctx* ctx;
  dsa_res* res;
  DevBuf d_mat, d_total;
  uint64_t total = 0;   // CIGAR words written so far
  int smax_pos = 0;     // max(S, 0)
};

// Traceback band window of a long job from the diagonal bound of its score.
void long_window(const TbBounds& B, LongTbJob& lj, int32_t score) {
  lj.dlo = 0;
  lj.wc = lj.je;
  int64_t dlo, dhi;
  if (lj.ie > 0 && lj.je > 0 && tb_diag_window(B, lj.ie, lj.je, score, dlo, dhi)) {
    const int64_t wc = (int64_t)long_ckpt_rows() + dhi - dlo;   // a traceback band's window
    if (wc < lj.je) {
      lj.dlo = (int32_t)std::max<int64_t>(dlo, -(int64_t)lj.ie);
      lj.wc = (int32_t)wc;
    }
  }
  lj.wpr = (uint32_t)((lj.wc + 7) / 8);
}

// Sort the selected hits into the paths: long pairs, thread per hit, warp
// per hit, and big hits without checkpoints.
void tb_collect(dsa_res* res, const TbBounds& bounds, const std::vector<uint64_t>& sel,
                uint64_t thread_min, TbPlan& P) {
  const dsa_db* db = res->db;
  const dsa_db* qs = res->queries;
  auto small = [](const TbJob& j) { return j.ie <= 4096 && (uint64_t)j.ie * j.je <= (1u << 20); };
  std::vector<TbJob>& tjobs = *P.tjobs;
  tjobs.clear();
  const int band = long_band_rows(), ckpt = long_ckpt_rows();
  // hit h -> short job (false: the hit is skipped or is a long pair)
  auto make_short = [&](uint64_t h, TbJob& j) -> bool {
    const dsa_hit& hit = res->h_hits[h];
    if (hit.flags & DSA_HIT_HAS_TRACEBACK) return false;
    if (res->mode == DSA_LOCAL && (hit.q_end < 0 || hit.t_end < 0)) return false;
    if (!res->long_bnd_off.empty() && res->long_bnd_off[h] != UINT64_MAX) return false;
    tb_short_job(bounds, hit.q_end + 1, hit.t_end + 1, hit.score, qs->h_off[hit.query_id],
                 db->h_off[hit.target_id] + hit.t_offset, (uint32_t)h, j);
    return true;
  };
  // long pairs (few): serial
  if (!res->long_bnd_off.empty()) for (uint64_t h : sel) {
    const dsa_hit& hit = res->h_hits[h];
    if (hit.flags & DSA_HIT_HAS_TRACEBACK) continue;
    if (res->mode == DSA_LOCAL && (hit.q_end < 0 || hit.t_end < 0)) continue;
    if (res->long_bnd_off[h] == UINT64_MAX) continue;
    LongTbJob lj{};
    lj.q_start = qs->h_off[hit.query_id];
    lj.t_start = db->h_off[hit.target_id] + hit.t_offset;
    lj.bnd_off = res->long_bnd_off[h];
    lj.n = res->long_n[h];
    lj.ie = hit.q_end + 1;
    lj.je = hit.t_end + 1;
    lj.hit = (uint32_t)h;
    long_window(bounds, lj, hit.score);
    P.ljobs.push_back(lj);
    P.cap_total += (uint64_t)lj.ie + lj.je + 1;
  }
  // short jobs: count per host thread, then fill in place (hit order kept)
  {
    const unsigned T = host_threads(sel.size(), 1u << 16);
    std::vector<uint64_t> n_small(T + 1, 0), n_large(T + 1, 0), cap(T, 0);
    parallel_for(sel.size(), T, [&](unsigned t, size_t b, size_t e) {
      TbJob j;
      uint64_t ns = 0, nl = 0, cp = 0;   // thread-local: no shared cache lines in the loop
      for (size_t x = b; x < e; ++x)
        if (make_short(sel[x], j)) {
          ++(small(j) ? ns : nl);
          cp += (uint64_t)j.ie + j.je + 1;
        }
      n_small[t + 1] = ns;
      n_large[t + 1] = nl;
      cap[t] = cp;
    });
    for (unsigned t = 0; t < T; ++t) {
      n_small[t + 1] += n_small[t];
      n_large[t + 1] += n_large[t];
      P.cap_total += cap[t];
    }
    tjobs.resize(n_small[T]);
    P.jobs.resize(n_large[T]);
    parallel_for(sel.size(), T, [&](unsigned t, size_t b, size_t e) {
      uint64_t ks = n_small[t], kl = n_large[t];
      TbJob j;
      for (size_t x = b; x < e; ++x)
        if (make_short(sel[x], j)) {
          if (small(j)) tjobs[ks++] = j;
          else P.jobs[kl++] = j;
        }
    });
  }
  if (tjobs.size() < std::max<uint64_t>(thread_min, 1)) {
    P.jobs.insert(P.jobs.end(), tjobs.begin(), tjobs.end());
    tjobs.clear();
  }
  // Big rectangles of hits without score-pass checkpoints (256 k cells or
  // more over at least two 512-row bands): a checkpointed score pass over the
  // hit's rectangle (the band pipeline of the long pairs), then the long-pair
  // traceback (parallel band fill, windowed walk) instead of one warp working
  // through the bands one after another.
  std::vector<TbJob> keep;
  for (const TbJob& j : P.jobs) {
    const dsa_hit& hit = res->h_hits[j.hit];
    const int32_t ie = hit.q_end + 1, je = hit.t_end + 1;   // the whole rectangle
    if ((uint64_t)ie * (uint64_t)je < (1u << 18) || ie <= band) {
      keep.push_back(j);
      continue;
    }
    const uint64_t nb = ((uint64_t)ie + band - 1) / band;
    const uint64_t q0 = qs->h_off[hit.query_id], t0 = db->h_off[hit.target_id] + hit.t_offset;
    P.bscore.push_back({q0, t0, P.b_bnd, P.b_bands, P.b_bands, ie, je, (uint32_t)P.bscore.size(), 0});
    LongTbJob lj{};
    lj.q_start = q0;
    lj.t_start = t0;
    lj.bnd_off = P.b_bnd;
    lj.n = je;
    lj.ie = ie;
    lj.je = je;
    lj.hit = j.hit;
    long_window(bounds, lj, hit.score);
    P.bjobs.push_back(lj);
    P.cap_total += (uint64_t)je - j.je;   // CIGAR capacity of the whole rectangle
    P.b_bnd += ((uint64_t)ie + ckpt - 1) / ckpt * (uint64_t)je;   // checkpoint rows
    P.b_bands += nb;
  }
  P.jobs.swap(keep);
}

// Groups of 32 thread-per-hit jobs share a layout padded to their largest
// (ie, je): keep the given order unless it would double the work, else order
// by (ie, wc) descending.
void tb_order_thread_jobs(dsa_ctx* ctx, std::vector<TbJob>& tjobs) {
  const size_t n_groups = (tjobs.size() + 31) / 32;
  const unsigned T = host_threads(tjobs.size(), 1u << 16);
  std::vector<uint64_t> cells_t(T, 0), padded_t(T, 0);
  parallel_for(n_groups, T, [&](unsigned t, size_t gb, size_t ge) {
    uint64_t cl = 0, pd = 0;
    for (size_t g = gb; g < ge; ++g) {
      int32_t im = 0, jm = 0;
      const size_t x1 = std::min(tjobs.size(), 32 * g + 32);
      for (size_t x = 32 * g; x < x1; ++x) {
        im = std::max(im, tjobs[x].ie);
        jm = std::max(jm, tjobs[x].wc);
        cl += (uint64_t)tjobs[x].ie * tjobs[x].wc;
      }
      pd += (uint64_t)im * jm * (x1 - 32 * g);
    }
    cells_t[t] = cl;
    padded_t[t] = pd;
  });
  uint64_t cells = 0, padded = 0;
  for (unsigned t = 0; t < T; ++t) {
    cells += cells_t[t];
    padded += padded_t[t];
  }
  if (padded <= 2 * cells) return;
  std::vector<uint64_t> key(tjobs.size());
  parallel_for(tjobs.size(), T, [&](unsigned, size_t b, size_t e) {
    for (size_t x = b; x < e; ++x)
      key[x] = ~(((uint64_t)(uint32_t)tjobs[x].ie << 32) | (uint32_t)tjobs[x].wc);
  });
  const std::vector<uint32_t> ord = radix_order(key);
  std::vector<TbJob>& sorted = ctx->h_tb2;
  sorted.resize(tjobs.size());
  parallel_for(ord.size(), host_threads(ord.size(), 1u << 16), [&](unsigned, size_t b, size_t e) {
    for (size_t x = b; x < e; ++x) sorted[x] = tjobs[ord[x]];
  });
  tjobs.swap(sorted);
}

// After a chunk's kernels: the CIGAR words it appended.
int tb_read_total(TbRun& R) {
  DSA_CUDA_TRY(cudaMemcpyAsync(&R.total, R.d_total.p, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                               R.ctx->stream));
  DSA_CUDA_TRY(cudaStreamSynchronize(R.ctx->stream));
  return DSA_OK;
}

// Thread per hit, in chunks of whole groups of 32 under `limit` words.
int tb_run_thread(TbRun& R, std::vector<TbJob>& tjobs, uint64_t limit) {
  dsa_ctx* ctx = R.ctx;
  dsa_res* res = R.res;
  size_t k0 = 0;
  while (k0 < tjobs.size()) {
    uint64_t dir = 0, cig = 0, scr = 0;
    size_t k1 = k0;
    while (k1 < tjobs.size()) {
      const size_t g1 = std::min(tjobs.size(), k1 + 32);
      int32_t ie_max = 1, je_max = 1, wc_max = 1;
      for (size_t x = k1; x < g1; ++x) {
        ie_max = std::max(ie_max, tjobs[x].ie);
        je_max = std::max(je_max, tjobs[x].je);
        wc_max = std::max(wc_max, tjobs[x].wc);
      }
      const uint64_t strips = ((uint64_t)ie_max + TB_STRIP - 1) / TB_STRIP;
      const uint64_t w = strips * (uint64_t)wc_max * (32 * TB_STRIP_WORDS);
      if (k1 > k0 && dir + w > limit) break;
      for (size_t x = k1; x < g1; ++x) {
        const uint32_t lane = (uint32_t)(x - k1);
        tjobs[x].dir_off = dir + lane;
        tjobs[x].wpr = (uint32_t)wc_max;
        tjobs[x].scr_off = scr + lane;
        tjobs[x].cig_off = cig;
        cig += (uint64_t)tjobs[x].ie + tjobs[x].je + 1;
      }
      dir += w;
      scr += (uint64_t)je_max * 32;
      k1 = g1;
    }
    const size_t n_chunk = k1 - k0;
    DevBuf d_jobs, d_dir, d_cig, d_scr;
    DSA_TRY(upload(ctx, d_jobs, tjobs.data() + k0, n_chunk));
    DSA_TRY(d_dir.alloc(ctx, dir * 4));
    DSA_TRY(d_cig.alloc(ctx, cig * 4));
    DSA_TRY(d_scr.alloc(ctx, scr * sizeof(int2)));
    DSA_TRY(launch_traceback_thread(ctx, res->db, res->queries, R.d_mat.as<int8_t>(), res->A,
                                    res->gap_open, res->gap_extend, res->mode, res->free_ends,
                                    s_plus_o_fits_int8(res->matrix.data(), res->A, res->gap_open),
                                    d_jobs.as<TbJob>(), (uint32_t)n_chunk, d_dir.as<uint32_t>(),
                                    d_cig.as<uint32_t>(), d_scr.as<int2>(), res->d_hits));
    DSA_TRY(launch_cigar_compact(ctx, res->d_hits, d_jobs.as<TbJob>(), (uint32_t)n_chunk,
                                 d_cig.as<uint32_t>(), res->d_cigar, R.total,
                                 R.d_total.as<uint64_t>()));
    DSA_TRY(tb_read_total(R));
    k0 = k1;
  }
  return DSA_OK;
}

// Warp per hit, in chunks under `limit` words.
int tb_run_warp(TbRun& R, std::vector<TbJob>& jobs, uint64_t limit) {
  dsa_ctx* ctx = R.ctx;
  dsa_res* res = R.res;
  size_t k0 = 0;
  while (k0 < jobs.size()) {
    uint64_t dir = 0, cig = 0, scr = 0;
    size_t k1 = k0;
    while (k1 < jobs.size()) {
      const uint64_t w = (uint64_t)jobs[k1].ie * jobs[k1].wpr;
      if (k1 > k0 && dir + w > limit) break;
      jobs[k1].dir_off = dir;
      jobs[k1].cig_off = cig;
      jobs[k1].scr_off = scr;
      dir += w;
      cig += (uint64_t)jobs[k1].ie + jobs[k1].je + 1;
      scr += (uint64_t)jobs[k1].je;
      ++k1;
    }
    std::vector<TbJob> chunk(jobs.begin() + k0, jobs.begin() + k1);
    DevBuf d_jobs, d_dir, d_cig, d_scr;
    DSA_TRY(upload(ctx, d_jobs, chunk));
    DSA_TRY(d_dir.alloc(ctx, dir * 4));
    DSA_TRY(d_cig.alloc(ctx, cig * 4));
    DSA_TRY(d_scr.alloc(ctx, scr * sizeof(int2)));
    DSA_TRY(launch_traceback(ctx, res->db, res->queries, R.d_mat.as<int8_t>(), res->A,
                             res->gap_open, res->gap_extend, res->mode, res->free_ends,
                             d_jobs.as<TbJob>(), (uint32_t)chunk.size(), d_dir.as<uint32_t>(),
                             d_cig.as<uint32_t>(), d_scr.as<int2>(), res->d_hits));
    DSA_TRY(launch_cigar_compact(ctx, res->d_hits, d_jobs.as<TbJob>(), (uint32_t)chunk.size(),
                                 d_cig.as<uint32_t>(), res->d_cigar, R.total,
                                 R.d_total.as<uint64_t>()));
    DSA_TRY(tb_read_total(R));
    k0 = k1;
  }
  return DSA_OK;
}

// Decision matrices of long rectangles (or their diagonal bands), in chunks
// under `limit` words; bnd_rows: the score pass's checkpoint rows.
int tb_run_long(TbRun& R, std::vector<LongTbJob>& list, const int2* bnd_rows, uint64_t limit) {
  dsa_ctx* ctx = R.ctx;
  dsa_res* res = R.res;
  const int ckpt = long_ckpt_rows();
  // The packed fill takes alphabets of up to 4 letters whose S + o fit a
  // byte and scores whose relative values fit its range, and runs when a
  // chunk's bands fill the device twice over (it runs one warp per two
  // bands: with fewer, the int32 fill's warps hide latency better);
  // DSA_TB_FILL=int32 | packed fixes the choice.
  int smin = 0;
  for (int8_t v : res->matrix) smin = std::min<int>(smin, v);
  const char* fill_env = getenv("DSA_TB_FILL");
  const std::string fill_pick = fill_env ? fill_env : "";
  const bool packed_ok = res->A <= 4 &&
                         s_plus_o_fits_int8(res->matrix.data(), res->A, res->gap_open) &&
                         long_tb16_range_ok(res->gap_open, res->gap_extend, R.smax_pos, smin) &&
                         fill_pick != "int32";
  // (4 blocks of 4 warps per SM: 16 warps, one per two bands)
  const uint64_t packed_min_bands = 2ull * 16 * (uint64_t)ctx->sm_count;
  size_t k0 = 0;
  while (k0 < list.size()) {
    uint64_t dir = 0, cig = 0;
    size_t k1 = k0;
    std::vector<uint32_t> items;
    while (k1 < list.size()) {
      LongTbJob& lj = list[k1];
      const uint64_t w = (uint64_t)((lj.ie + ckpt - 1) / ckpt) * ckpt * lj.wpr;
      if (k1 > k0 && dir + w > limit) break;
      lj.dir_off = dir;
      lj.cig_off = cig;
      dir += w;
      cig += (uint64_t)lj.ie + lj.je + 1;
      const uint32_t nb = (uint32_t)((lj.ie + ckpt - 1) / ckpt);   // traceback bands
      for (uint32_t b = 0; b < nb; ++b) { items.push_back((uint32_t)(k1 - k0)); items.push_back(b); }
      ++k1;
    }
    std::vector<LongTbJob> chunk(list.begin() + k0, list.begin() + k1);
    // per-band windows from the checkpoint rows (each within the job's
    // diagonal window); the decision rows take the widest band's words
    uint32_t n_bands = 0;
    for (LongTbJob& lj : chunk) {
      lj.win_off = n_bands;
      n_bands += (uint32_t)((lj.ie + ckpt - 1) / ckpt);
    }
    const bool packed = packed_ok && (fill_pick == "packed" || n_bands >= packed_min_bands);
    DevBuf d_lj, d_items, d_dir, d_cig, d_shim, d_win, d_maxw;
    DSA_TRY(upload(ctx, d_lj, chunk));
    DSA_TRY(upload(ctx, d_items, items));
    DSA_TRY(d_win.alloc(ctx, (size_t)std::max<uint32_t>(n_bands, 1) * sizeof(int2)));
    DSA_TRY(d_maxw.alloc(ctx, chunk.size() * sizeof(int32_t)));
    DSA_CUDA_TRY(cudaMemsetAsync(d_maxw.p, 0, chunk.size() * sizeof(int32_t), ctx->stream));
    DSA_TRY(launch_long_tb_windows(ctx, ctx->stream, d_lj.as<LongTbJob>(), d_items.as<uint32_t>(),
                                   (uint32_t)(items.size() / 2), bnd_rows, res->d_hits, res->mode,
                                   res->free_ends, res->gap_open, res->gap_extend,
                                   R.smax_pos, d_win.as<int2>(),
                                   d_maxw.as<int32_t>()));
    std::vector<int32_t> maxw(chunk.size());
    std::vector<int2> bwin(packed ? n_bands : 0);
    DSA_CUDA_TRY(cudaMemcpyAsync(maxw.data(), d_maxw.p, chunk.size() * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, ctx->stream));
    if (packed)
      DSA_CUDA_TRY(cudaMemcpyAsync(bwin.data(), d_win.p, n_bands * sizeof(int2),
                                   cudaMemcpyDeviceToHost, ctx->stream));
    DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    dir = 0;
    for (size_t k = 0; k < chunk.size(); ++k) {
      LongTbJob& lj = chunk[k];
      lj.wpr = (uint32_t)((std::max(maxw[k], 1) + 7) / 8);
      lj.dir_off = dir;
      dir += (uint64_t)((lj.ie + ckpt - 1) / ckpt) * ckpt * lj.wpr;
    }
    DSA_CUDA_TRY(cudaMemcpyAsync(d_lj.p, chunk.data(), chunk.size() * sizeof(LongTbJob),
                                 cudaMemcpyHostToDevice, ctx->stream));
    std::vector<TbJob> shim(chunk.size());   // the CIGAR packer reads hit and cig_off
    for (size_t k = 0; k < chunk.size(); ++k) {
      shim[k].hit = chunk[k].hit;
      shim[k].cig_off = chunk[k].cig_off;
    }
    DSA_TRY(upload(ctx, d_shim, shim));
    DSA_TRY(d_dir.alloc(ctx, dir * 4));
    DSA_TRY(d_cig.alloc(ctx, cig * 4));
    // every band of every hit of the chunk in one launch, then one warp per hit
    if (packed) {
      // bands paired by window width (widest first), two per warp
      std::vector<uint32_t> ord(items.size() / 2);
      std::iota(ord.begin(), ord.end(), 0u);
      auto width = [&](uint32_t x) {
        return bwin[chunk[items[2 * x]].win_off + items[2 * x + 1]].y;
      };
      std::stable_sort(ord.begin(), ord.end(),
                       [&](uint32_t x, uint32_t y) { return width(x) > width(y); });
      std::vector<uint32_t> units;
      units.reserve(2 * items.size());
      for (size_t k = 0; k < ord.size(); k += 2) {
        units.push_back(items[2 * ord[k]]);
        units.push_back(items[2 * ord[k] + 1]);
        units.push_back(k + 1 < ord.size() ? items[2 * ord[k + 1]] : NONE);
        units.push_back(k + 1 < ord.size() ? items[2 * ord[k + 1] + 1] : 0u);
      }
      DevBuf d_units;
      DSA_TRY(upload(ctx, d_units, units));
      DSA_TRY(launch_long_tb_fill16(ctx, ctx->stream, res->db, res->queries,
                                    R.d_mat.as<int8_t>(), res->A, res->gap_open, res->gap_extend,
                                    res->mode, res->free_ends, d_lj.as<LongTbJob>(),
                                    d_units.as<uint32_t>(), (uint32_t)(units.size() / 4),
                                    bnd_rows, d_dir.as<uint32_t>(), d_win.as<int2>()));
    } else {
      DSA_TRY(launch_long_tb_fill(ctx, ctx->stream, res->db, res->queries, R.d_mat.as<int8_t>(),
                                  res->A, res->gap_open, res->gap_extend, res->mode,
                                  res->free_ends, d_lj.as<LongTbJob>(), d_items.as<uint32_t>(),
                                  (uint32_t)(items.size() / 2), bnd_rows, d_dir.as<uint32_t>(),
                                  d_win.as<int2>()));
    }
    DSA_TRY(launch_long_tb_walk(ctx, ctx->stream, d_lj.as<LongTbJob>(), (uint32_t)chunk.size(),
                                res->mode, res->free_ends, d_dir.as<uint32_t>(),
                                d_cig.as<uint32_t>(), res->d_hits, d_win.as<int2>()));
    DSA_TRY(launch_cigar_compact(ctx, res->d_hits, d_shim.as<TbJob>(), (uint32_t)shim.size(),
                                 d_cig.as<uint32_t>(), res->d_cigar, R.total,
                                 R.d_total.as<uint64_t>()));
    DSA_TRY(tb_read_total(R));
    k0 = k1;
  }
  return DSA_OK;
}

// Big hits: checkpointed score pass over their rectangles (bands in
// latest-start order), then the long-pair traceback from those checkpoints.
int tb_run_big(TbRun& R, TbPlan& P, uint64_t limit) {
  dsa_ctx* ctx = R.ctx;
  dsa_res* res = R.res;
  std::vector<std::pair<uint32_t, uint32_t>> mn(P.bscore.size());
  for (size_t k = 0; k < P.bscore.size(); ++k)
    mn[k] = {(uint32_t)P.bscore[k].m, (uint32_t)P.bscore[k].n};
  const std::vector<uint32_t> items = band_items(mn, long_band_rows());
  const size_t nj = P.bscore.size();
  DevBuf d_bs, d_bitems, d_bbnd, d_bprog, d_bcand, d_bout;
  DSA_TRY(upload(ctx, d_bs, P.bscore));
  DSA_TRY(upload(ctx, d_bitems, items));
  DSA_TRY(d_bbnd.alloc(ctx, P.b_bnd * sizeof(int2)));
  DSA_TRY(d_bprog.alloc(ctx, P.b_bands * sizeof(uint32_t)));
  DSA_TRY(d_bcand.alloc(ctx, P.b_bands * long_cand_size()));
  DSA_TRY(d_bout.alloc(ctx, nj * 13));
  DSA_CUDA_TRY(cudaMemsetAsync(d_bprog.p, 0, P.b_bands * sizeof(uint32_t), ctx->stream));
  Scores bsc;   // the rerun's scores are not needed: only its checkpoint rows
  bsc.score = d_bout.as<int32_t>();
  bsc.q_end = bsc.score + nj;
  bsc.t_end = bsc.q_end + nj;
  bsc.flag = reinterpret_cast<uint8_t*>(bsc.t_end + nj);
  DSA_TRY(launch_long_score(ctx, res->db, res->queries, R.d_mat.as<int8_t>(), res->A,
                            res->gap_open, res->gap_extend, res->mode, res->free_ends,
                            s_plus_o_fits_int8(res->matrix.data(), res->A, res->gap_open),
                            d_bs.as<LongJob>(), (uint32_t)nj, d_bitems.as<uint32_t>(),
                            (uint32_t)(items.size() / 2), d_bbnd.as<int2>(),
                            d_bprog.as<uint32_t>(), d_bcand.p, bsc));
  return tb_run_long(R, P.bjobs, d_bbnd.as<int2>(), limit);
}

}  // namespace
}  // namespace dsa

using namespace dsa;

extern "C" int dsa_traceback(dsa_ctx* ctx, dsa_res* res, const uint64_t* which, uint64_t n) {
  if (!ctx || !res || res->ctx != ctx) {
    set_error("bad ctx / res (results handed out by a server are host-only)");
    return DSA_ERR_INVALID_ARG;
  }
  if (res->pssm) {
    set_error("results scored with position-specific profiles carry scores and ends only");
    return DSA_ERR_UNSUPPORTED;
  }
  DSA_TRY(set_device(ctx));
  // Many small rectangles: one thread per hit (groups of 32 hits of similar
  // size share an interleaved decision layout).  Few or large ones: one warp
  // per hit.
  uint64_t thread_min = 16384;
  if (const char* env = getenv("DSA_TB_THREAD_MIN")) thread_min = strtoull(env, nullptr, 10);
  // exact column band for a free target begin (see k_traceback.cu); needs e > 0
  int smax_pos = 0;
  for (int8_t v : res->matrix) smax_pos = std::max<int>(smax_pos, v);
  const bool band_ok = res->mode == DSA_SEMIGLOBAL && (res->free_ends & DSA_FREE_T_BEGIN) &&
                       res->gap_extend > 0;
  // Diagonal bands from the total gap length g of a path reaching (ie, je)
  // (tb_diag_window): it has at most (ie + je - g) / 2 M columns whatever its
  // start, so 2 score <= max(S, 0)(ie + je) - g (max(S, 0) + 2e) - 2 (o - e);
  // a cell (i, j) on it has |dn - d| <= g (gaps after it; d = j - i,
  // dn = je - ie) and, for paths from (0, 0), |d| <= g as well (gaps before).
  const bool diag_ok = smax_pos + 2 * res->gap_extend > 0;
  const bool from_origin = res->mode == DSA_GLOBAL ||
                           (res->mode == DSA_SEMIGLOBAL &&
                            !(res->free_ends & (DSA_FREE_Q_BEGIN | DSA_FREE_T_BEGIN)));
  const TbBounds bounds{res->mode, res->free_ends, res->gap_open, res->gap_extend, smax_pos,
                        band_ok, diag_ok, from_origin};
  const uint64_t short_limit = tb_chunk_words(TB_SHORT_CHUNK_WORDS);
  // every hit of a large result on the thread path: staged on the device
  // (DSA_TB_HOST_STAGING=1 keeps the host staging below)
  const char* host_staging = getenv("DSA_TB_HOST_STAGING");
  if (!which && res->long_bnd_off.empty() && res->n_hits >= std::max<uint64_t>(thread_min, 1) &&
      !(host_staging && host_staging[0] == '1')) {
    const int rc = traceback_device_staged(ctx, res, bounds, short_limit);
    if (rc != TB_STAGE_FALLBACK) return rc;
  }
  DSA_TRY(fetch_hits(res));
  std::vector<uint64_t> sel;
  if (which) {
    for (uint64_t k = 0; k < n; ++k) {
      if (which[k] >= res->n_hits) { set_error("hit index out of range"); return DSA_ERR_INVALID_ARG; }
      sel.push_back(which[k]);
    }
  } else {
    sel.resize(res->n_hits);
    std::iota(sel.begin(), sel.end(), 0ull);
  }
  TbPlan P;
  P.tjobs = &ctx->h_tb;
  tb_collect(res, bounds, sel, thread_min, P);
  std::vector<TbJob>& tjobs = *P.tjobs;
  if (P.jobs.empty() && tjobs.empty() && P.ljobs.empty() && P.bjobs.empty()) return DSA_OK;

  // grow the result's CIGAR array by the capacity bound
  const uint64_t old_n = res->n_cigar;
  void* newp = nullptr;
  DSA_TRY(ctx->alloc(&newp, (old_n + P.cap_total) * sizeof(uint32_t)));
  if (old_n)
    DSA_CUDA_TRY(cudaMemcpyAsync(newp, res->d_cigar, old_n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (res->d_cigar) ctx->release(res->d_cigar, res->cigar_bytes);
  res->d_cigar = (uint32_t*)newp;
  res->cigar_bytes = (old_n + P.cap_total) * sizeof(uint32_t);

  TbRun R{ctx, res};
  R.smax_pos = smax_pos;
  DSA_TRY(R.d_mat.alloc(ctx, res->A * res->A));
  DSA_CUDA_TRY(cudaMemcpyAsync(R.d_mat.p, res->matrix.data(), res->A * res->A,
                               cudaMemcpyHostToDevice, ctx->stream));
  DSA_TRY(R.d_total.alloc(ctx, sizeof(uint64_t)));
  DSA_CUDA_TRY(cudaMemcpyAsync(R.d_total.p, &old_n, sizeof(uint64_t), cudaMemcpyHostToDevice,
                               ctx->stream));
  R.total = old_n;

  phase_begin(res, PH_TRACE);
  if (!tjobs.empty()) {
    tb_order_thread_jobs(ctx, tjobs);
    DSA_TRY(tb_run_thread(R, tjobs, short_limit));
  }
  DSA_TRY(tb_run_warp(R, P.jobs, short_limit));
  const uint64_t long_limit = tb_chunk_words(TB_LONG_CHUNK_WORDS);
  if (!P.ljobs.empty()) DSA_TRY(tb_run_long(R, P.ljobs, res->d_bnd, long_limit));
  if (!P.bscore.empty()) DSA_TRY(tb_run_big(R, P, long_limit));
  phase_end(res, PH_TRACE);
  res->n_cigar = R.total;
  res->host_valid = false;
  return DSA_OK;
}
