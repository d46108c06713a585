// Score pass of explicit (query, target window) pairs -- the read-vs-window
// and long-pair alignments of the map phase (Sec. II.B.1) in any of the three
// algorithms (Sec. II.C.2).  Pairs are checked and classified on the device;
// when every pair takes the packed int16x2 kernel the device also plans the
// jobs (stable radix order by query and window length), otherwise the host
// planner classifies on host threads.  Long pairs run on the band pipeline,
// the rest on the exact int32 kernel, and local packed pairs that saturate
// are rerun exactly in int32.
#include "host_util.cuh"

#include <algorithm>
#include <numeric>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

namespace dsa {

int PairPass::need_hp(dsa_ctx* ctx) {
  if (hp_ready) return DSA_OK;
  hp.resize(n_pairs);
  if (flags & DSA_PAIRS_ON_DEVICE) {
    if (n_pairs)
      DSA_CUDA_TRY(cudaMemcpyAsync(hp.data(), pairs, n_pairs * sizeof(dsa_pair),
                                   cudaMemcpyDeviceToHost, ctx->stream));
    DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  } else if (n_pairs) {
    memcpy(hp.data(), pairs, n_pairs * sizeof(dsa_pair));
  }
  hp_ready = true;
  return DSA_OK;
}

int pairs_classify(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const PairPlanParams& P,
                   PairPass& pp) {
  const uint64_t n_pairs = pp.n_pairs;
  pp.L = (uint64_t)qs->max_len + 2;
  const uint64_t L = pp.L;
  if (pp.flags & DSA_PAIRS_ON_DEVICE) {
    pp.d_pairs = pp.pairs;
  } else {
    DSA_TRY(upload(ctx, pp.d_pairs_buf, pp.pairs, n_pairs));
    pp.d_pairs = pp.d_pairs_buf.as<dsa_pair>();
  }
  DSA_TRY(pp.d_key.alloc(ctx, n_pairs * sizeof(uint64_t)));
  DSA_TRY(pp.d_idx.alloc(ctx, n_pairs * sizeof(uint32_t)));
  DSA_TRY(pp.d_hist.alloc(ctx, L * sizeof(uint64_t)));
  DSA_TRY(pp.d_jcnt.alloc(ctx, L * sizeof(uint64_t)));
  DSA_TRY(pp.d_stats.alloc(ctx, sizeof(PairPlanStats)));
  PairPlanStats* st = pp.d_stats.as<PairPlanStats>();
  DSA_CUDA_TRY(cudaMemsetAsync(pp.d_hist.p, 0, L * sizeof(uint64_t), ctx->stream));
  DSA_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(PairPlanStats), ctx->stream));
  DSA_CUDA_TRY(cudaMemsetAsync(&st->first_bad, 0xFF, sizeof(uint64_t), ctx->stream));
  DSA_TRY(launch_pair_classify(ctx, pp.d_pairs, n_pairs, qs, db, P, pp.d_key.as<uint64_t>(),
                               pp.d_idx.as<uint32_t>(), pp.d_hist.as<uint64_t>(), L,
                               pp.d_jcnt.as<uint64_t>(), st));
  DSA_CUDA_TRY(cudaMemcpyAsync(&pp.pst, st, sizeof pp.pst, cudaMemcpyDeviceToHost, ctx->stream));
  DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  if (pp.pst.first_bad != UINT64_MAX) {
    set_error("pair %llu is out of range", (unsigned long long)pp.pst.first_bad);
    return DSA_ERR_INVALID_ARG;
  }
  return DSA_OK;
}

int score_pairs(dsa_ctx* ctx, dsa_res* res, const dsa_db* db, const dsa_db* qs, PairPass& pp,
                int mode, uint32_t fe, const int8_t* matrix, const int8_t* d_mat, int A, int o,
                int e, const Validated& v, bool local16, bool packed_ok, int64_t w16, Scores sc) {
  const uint64_t n_pairs = pp.n_pairs;
  const dsa_pair* d_pairs = pp.d_pairs;
  int rc = DSA_OK;
  std::vector<PairJob> jobs;
  std::vector<LongJob> ljobs;
  std::vector<uint64_t> p16;   // pairs for the packed int16 kernel
  uint64_t scr = 0, cells = 0, lcells = 0, p16cells = 0;
  uint64_t bnd = 0, prog = 0, cand = 0;
  const int band = long_band_rows(), ckpt = long_ckpt_rows();
  // every pair packed: the device planner lays out the jobs
  const bool dev_plan = n_pairs > 0 && pp.pst.n_other == 0;
  // host planner: classify on host threads: packed pairs (filled in place,
  // pair order kept); long and int32 pairs are few and follow serially
  enum : uint8_t { C_P16, C_LONG, C_INT32 };
  std::vector<uint8_t> cls;
  if (dev_plan) {
    cells = pp.pst.cells;
    p16cells = pp.pst.cells16;
  } else {
    if ((rc = pp.need_hp(ctx))) return (rc);
    cls.resize(n_pairs);
    const unsigned T = host_threads(n_pairs, 1u << 16);
    std::vector<uint64_t> n16(T + 1, 0), cells_t(T, 0), c16_t(T, 0);
    parallel_for(n_pairs, T, [&](unsigned t, size_t b, size_t x1) {
      uint64_t n = 0, cl = 0, c16 = 0;   // thread-local: no shared cache lines in the loop
      for (size_t k = b; k < x1; ++k) {
        const dsa_pair& p = pp.hp[k];
        const uint64_t m = qs->h_len[p.query_id];
        const uint64_t c = m * p.t_len;
        cl += c;
        const bool fits16 = local16 || ((int64_t)(m + p.t_len) * w16 + o < 12000 && o + e < 4096);
        if (packed_ok && fits16 && m >= 1 && p.t_len >= 1 && c < LONG_PAIR_CELLS) {
          cls[k] = C_P16;
          ++n;
          c16 += c;
        } else {
          cls[k] = c >= LONG_PAIR_CELLS ? C_LONG : C_INT32;
        }
      }
      n16[t + 1] = n;
      cells_t[t] = cl;
      c16_t[t] = c16;
    });
    for (unsigned t = 0; t < T; ++t) {
      n16[t + 1] += n16[t];
      cells += cells_t[t];
      p16cells += c16_t[t];
    }
    p16.resize(n16[T]);
    parallel_for(n_pairs, T, [&](unsigned t, size_t b, size_t x1) {
      uint64_t pos = n16[t];
      for (size_t k = b; k < x1; ++k)
        if (cls[k] == C_P16) p16[pos++] = k;
    });
  }
  for (uint64_t k = 0; k < cls.size(); ++k) {
    if (cls[k] == C_P16) continue;
    const dsa_pair& p = pp.hp[k];
    const uint64_t m = qs->h_len[p.query_id];
    if (cls[k] == C_LONG) {
      const uint64_t nb = (m + band - 1) / band;
      const uint64_t nck = (m + ckpt - 1) / ckpt;   // checkpoint rows
      LongJob lj{qs->h_off[p.query_id], db->h_off[p.target_id] + p.t_offset, bnd, prog, cand,
                 (int32_t)m, (int32_t)p.t_len, (uint32_t)k, 0};
      ljobs.push_back(lj);
      bnd += nck * p.t_len;
      prog += nb;
      cand += nb;
      lcells += m * p.t_len;
    } else {
      jobs.push_back({db->h_off[p.target_id] + p.t_offset, scr, p.query_id, p.t_len, (uint32_t)k, 0});
      scr += p.t_len;
    }
  }
  res->cells = cells;
  res->phase_cells[PH_INT32] = cells;
  if (!ljobs.empty()) {
    // The packed form takes two pairs per warp (sorted neighbours by query
    // and window length) when the alphabet, the byte tables and the range
    // bound allow it; DSA_LONG_INT32=1 keeps every pair on the int32 kernel.
    const char* force32 = getenv("DSA_LONG_INT32");
    const bool l16 = A <= 4 && s_plus_o_fits_int8(matrix, A, o) &&
                     long16_range_ok(o, e, v.smax, v.smin) && !(force32 && atoi(force32));
    std::vector<LongPair16> units;
    std::vector<std::pair<uint32_t, uint32_t>> mn;
    if (l16) {
      std::vector<uint32_t> ord(ljobs.size());
      std::iota(ord.begin(), ord.end(), 0u);
      std::stable_sort(ord.begin(), ord.end(), [&](uint32_t x, uint32_t y) {
        return ljobs[x].m != ljobs[y].m ? ljobs[x].m > ljobs[y].m : ljobs[x].n > ljobs[y].n;
      });
      prog = 0;
      for (size_t k = 0; k < ord.size(); k += 2) {
        const uint32_t a = ord[k], b = k + 1 < ord.size() ? ord[k + 1] : NONE;
        const uint32_t m = (uint32_t)std::max(ljobs[a].m, b != NONE ? ljobs[b].m : 0);
        const uint32_t n = (uint32_t)std::max(ljobs[a].n, b != NONE ? ljobs[b].n : 0);
        units.push_back({a, b, prog});
        prog += (m + band - 1) / band;
        mn.push_back({m, n});
      }
    } else {
      mn.resize(ljobs.size());
      for (size_t k = 0; k < ljobs.size(); ++k) mn[k] = {(uint32_t)ljobs[k].m, (uint32_t)ljobs[k].n};
    }
    // band items in latest-start order (bands in order inside a pair or unit)
    const std::vector<uint32_t> items = band_items(mn, band);
    // local, packed: every band of every pair, for locating the best cell
    std::vector<uint32_t> litems;
    if (l16 && mode == DSA_LOCAL)
      for (size_t k = 0; k < ljobs.size(); ++k)
        for (uint32_t b = 0; b < (uint32_t)((ljobs[k].m + band - 1) / band); ++b) {
          litems.push_back((uint32_t)k);
          litems.push_back(b);
        }
    DevBuf d_ljobs, d_items, d_prog, d_cands, d_units, d_litems;
    void* pb = nullptr;
    if ((rc = upload(ctx, d_ljobs, ljobs)) || (rc = upload(ctx, d_items, items)) ||
        (l16 && (rc = upload(ctx, d_units, units))) ||
        (!litems.empty() && (rc = upload(ctx, d_litems, litems))) ||
        (rc = d_prog.alloc(ctx, prog * sizeof(uint32_t))) ||
        (rc = d_cands.alloc(ctx, cand * long_cand_size())) ||
        (rc = ctx->alloc(&pb, bnd * sizeof(int2))))
      return (rc);
    res->d_bnd = static_cast<int2*>(pb);
    res->bnd_bytes = bnd * sizeof(int2);
    res->long_bnd_off.assign(n_pairs, UINT64_MAX);
    res->long_n.assign(n_pairs, 0);
    for (const LongJob& lj : ljobs) {
      res->long_bnd_off[lj.out] = lj.bnd_off;
      res->long_n[lj.out] = lj.n;
    }
    // one score pass with at most `bps` blocks per SM (0: as many as fit),
    // from zeroed progress counters
    auto run_long = [&](int bps) -> int {
      if (cudaMemsetAsync(d_prog.p, 0, prog * sizeof(uint32_t), ctx->stream) != cudaSuccess) {
        set_error("memset failed");
        return DSA_ERR_CUDA;
      }
      if (l16)
        return launch_long_score16(ctx, db, qs, d_mat, A, o, e, mode, fe, d_ljobs.as<LongJob>(),
                                   (uint32_t)ljobs.size(), d_units.as<LongPair16>(),
                                   d_items.as<uint32_t>(), (uint32_t)(items.size() / 2),
                                   res->d_bnd, d_prog.as<uint32_t>(), d_cands.p, sc, bps,
                                   d_litems.as<uint32_t>(), (uint32_t)(litems.size() / 2), cand);
      return launch_long_score(ctx, db, qs, d_mat, A, o, e, mode, fe,
                               s_plus_o_fits_int8(matrix, A, o), d_ljobs.as<LongJob>(),
                               (uint32_t)ljobs.size(), d_items.as<uint32_t>(),
                               (uint32_t)(items.size() / 2), res->d_bnd, d_prog.as<uint32_t>(),
                               d_cands.p, sc, bps);
    };
    // Blocks per SM: every block fits 4 per SM; with 2, each band's warp
    // shares its SM sub-partition with fewer others, and the bands' chains
    // (a band waits on the band above) run faster, which wins when the
    // longest pairs' chains bound the pass.  DSA_LONG_BLOCKS (2 | 4) fixes
    // it, else the autotuner times both on the first call of a shape
    // (kernel, mode, and log2 bins of the pair count, the longest query and
    // the longest window) and keeps the faster (a switch needs 3%).
    int bps = 4;
    const char* bps_env = getenv("DSA_LONG_BLOCKS");
    const char* tune_env = getenv("DSA_AUTOTUNE");
    if (bps_env) {
      bps = std::min(4, std::max(1, atoi(bps_env)));
    } else if (ctx->tune && !(tune_env && std::string(tune_env) == "off")) {
      uint32_t mmax = 0, nmax = 0;
      for (const LongJob& lj : ljobs) {
        mmax = std::max(mmax, (uint32_t)lj.m);
        nmax = std::max(nmax, (uint32_t)lj.n);
      }
      char k[160];
      snprintf(k, sizeof k, "|long|%s|%s|p%d|m%d|n%d|bps", l16 ? "p16" : "i32",
               mode == DSA_LOCAL ? "local" : (mode == DSA_GLOBAL ? "global" : "semi"),
               tuner_bin(ljobs.size()), tuner_bin(mmax), tuner_bin(nmax));
      const std::string key = tuner_shape_prefix(ctx) + k;
      uint32_t cached = 0;
      if (tuner_get(key, &cached)) {
        bps = cached == 2 ? 2 : 4;
      } else {
        cudaEvent_t ev[3];
        for (auto& x : ev) DSA_CUDA_TRY(cudaEventCreate(&x));
        int trc = DSA_OK;
        if (cudaEventRecord(ev[0], ctx->stream) != cudaSuccess || (trc = run_long(4)) ||
            cudaEventRecord(ev[1], ctx->stream) != cudaSuccess || (trc = run_long(2)) ||
            cudaEventRecord(ev[2], ctx->stream) != cudaSuccess ||
            cudaEventSynchronize(ev[2]) != cudaSuccess)
          trc = trc ? trc : DSA_ERR_CUDA;
        float t4 = 0.f, t2 = 0.f;
        if (!trc) {
          cudaEventElapsedTime(&t4, ev[0], ev[1]);
          cudaEventElapsedTime(&t2, ev[1], ev[2]);
        }
        for (auto& x : ev) cudaEventDestroy(x);
        if (trc) {
          set_error("long-pair autotune: %s", cudaGetErrorString(cudaGetLastError()));
          return trc;
        }
        bps = t2 < 0.97f * t4 ? 2 : 4;
        tuner_put(key, (uint32_t)bps);
      }
    }
    phase_begin(res, PH_INTRA);
    if ((rc = run_long(bps))) return (rc);
    phase_end(res, PH_INTRA);
    res->phase_cells[PH_INTRA] = lcells;
    res->phase_cells[PH_INT32] = cells - lcells;
  }
  if (dev_plan || !p16.empty()) {
    DevBuf d_pj;
    uint32_t n_pj = 0, max_n = 1;
    if (dev_plan) {
      // device planner: stable sort by (query length, window length), jobs
      // from the runs of equal query length
      DevBuf d_key2, d_idx2;
      if ((rc = d_key2.alloc(ctx, n_pairs * sizeof(uint64_t))) ||
          (rc = d_idx2.alloc(ctx, n_pairs * sizeof(uint32_t))) ||
          (rc = d_pj.alloc(ctx, pp.pst.n_jobs * sizeof(Pair16Job))))
        return (rc);
      uint64_t* kk = pp.d_key.as<uint64_t>();
      uint32_t* vv = pp.d_idx.as<uint32_t>();
      if ((rc = launch_pair_sort(ctx, kk, vv, d_key2.as<uint64_t>(), d_idx2.as<uint32_t>(), n_pairs,
                                 qs->max_len, pp.pst.max_t_len)) ||
          (rc = launch_pair_build_jobs(ctx, kk, vv, n_pairs, pp.d_hist.as<uint64_t>(),
                                       pp.d_jcnt.as<uint64_t>(), pp.L, d_pairs, qs, db,
                                       d_pj.as<Pair16Job>())))
        return (rc);
      n_pj = (uint32_t)pp.pst.n_jobs;
      max_n = std::max<uint32_t>(1, pp.pst.max_t_len);
    } else {
      // order by (query length, window length); two pairs of equal query length per thread
      const unsigned T = host_threads(p16.size(), 1u << 16);
      std::vector<uint64_t> key(p16.size());
      parallel_for(p16.size(), T, [&](unsigned, size_t b, size_t x1) {
        for (size_t x = b; x < x1; ++x) {
          const dsa_pair& px = pp.hp[p16[x]];
          key[x] = ((uint64_t)qs->h_len[px.query_id] << 32) | px.t_len;
        }
      });
      {
        const std::vector<uint32_t> ord = radix_order(key);
        std::vector<uint64_t> sorted(p16.size()), skey(p16.size());
        parallel_for(ord.size(), T, [&](unsigned, size_t b, size_t x1) {
          for (size_t x = b; x < x1; ++x) {
            sorted[x] = p16[ord[x]];
            skey[x] = key[ord[x]];
          }
        });
        p16.swap(sorted);
        key.swap(skey);
      }
      // a job starts at every even offset inside a run of equal query length
      std::vector<uint32_t> starts;
      starts.reserve(p16.size() / 2 + 1);
      uint32_t max_n16 = 1;
      for (size_t x = 0, run = 0; x < p16.size(); ++x) {
        if (x > 0 && (key[x] >> 32) != (key[x - 1] >> 32)) run = x;
        if (((x - run) & 1) == 0) starts.push_back((uint32_t)x);
        max_n16 = std::max<uint32_t>(max_n16, (uint32_t)key[x]);
      }
      std::vector<Pair16Job> pj(starts.size());
      parallel_for(starts.size(), T, [&](unsigned, size_t b, size_t x1) {
        for (size_t k = b; k < x1; ++k) {
          const size_t x = starts[k];
          const dsa_pair& a = pp.hp[p16[x]];
          Pair16Job j{};
          j.m = (int32_t)(key[x] >> 32);
          j.q_lo = qs->h_off[a.query_id];
          j.t_lo = db->h_off[a.target_id] + a.t_offset;
          j.n_lo = (int32_t)a.t_len;
          j.out_lo = (uint32_t)p16[x];
          if (x + 1 < p16.size() && (key[x + 1] >> 32) == (key[x] >> 32)) {
            const dsa_pair& bb = pp.hp[p16[x + 1]];
            j.q_hi = qs->h_off[bb.query_id];
            j.t_hi = db->h_off[bb.target_id] + bb.t_offset;
            j.n_hi = (int32_t)bb.t_len;
            j.out_hi = (uint32_t)p16[x + 1];
          } else {
            j.q_hi = j.q_lo;
            j.t_hi = j.t_lo;
            j.n_hi = 0;
            j.out_hi = NONE;
          }
          pj[k] = j;
        }
      });
      if ((rc = upload(ctx, d_pj, pj))) return (rc);
      n_pj = (uint32_t)pj.size();
      max_n = max_n16;
    }
    bool bytes = A <= 4;   // byte-permute substitution form
    for (int x = 0; x < A * A; ++x) bytes = bytes && matrix[x] + o >= -128 && matrix[x] + o <= 127;
    auto launch = [&](int rows) {
      return launch_pairs16(ctx, db, qs, d_mat, A, o, e, mode, fe, v.smax, bytes, rows,
                            d_pj.as<Pair16Job>(), n_pj, max_n, sc);
    };
    // kernel variant of the byte form (16-row strips at 4 blocks per SM, or
    // the wide 20-row strips at 3): DSA_PAIRS_ROWS, else the autotuner, per
    // workload shape (mode, alphabet, and log2 bins of the job count, the
    // longest query and the longest window), timing both on the first call
    int rows = 16;
    const int wide = pairs16_wide_rows();
    const char* rows_env = getenv("DSA_PAIRS_ROWS");
    const char* tune_env = getenv("DSA_AUTOTUNE");
    if (rows_env) {
      rows = bytes && atoi(rows_env) == wide ? wide : 16;
    } else if (bytes && ctx->tune && !(tune_env && std::string(tune_env) == "off")) {
      char k[160];
      snprintf(k, sizeof k, "|pairs|%s|A%d|j%d|m%d|n%d|rows",
               mode == DSA_LOCAL ? "local" : (mode == DSA_GLOBAL ? "global" : "semi"), A,
               tuner_bin(n_pj), tuner_bin(qs->max_len), tuner_bin(max_n));
      const std::string key = tuner_shape_prefix(ctx) + k;
      uint32_t cached = 0;
      if (tuner_get(key, &cached)) {
        rows = (int)cached == wide ? wide : 16;
      } else {
        cudaEvent_t ev[3];
        for (auto& x : ev) DSA_CUDA_TRY(cudaEventCreate(&x));
        int trc = DSA_OK;
        if (cudaEventRecord(ev[0], ctx->stream) != cudaSuccess || (trc = launch(16)) ||
            cudaEventRecord(ev[1], ctx->stream) != cudaSuccess || (trc = launch(wide)) ||
            cudaEventRecord(ev[2], ctx->stream) != cudaSuccess ||
            cudaEventSynchronize(ev[2]) != cudaSuccess)
          trc = trc ? trc : DSA_ERR_CUDA;
        float t16 = 0.f, tw = 0.f;
        if (!trc) {
          cudaEventElapsedTime(&t16, ev[0], ev[1]);
          cudaEventElapsedTime(&tw, ev[1], ev[2]);
        }
        for (auto& x : ev) cudaEventDestroy(x);
        if (trc) {
          set_error("pairs autotune: %s", cudaGetErrorString(cudaGetLastError()));
          return trc;
        }
        rows = tw < 0.97f * t16 ? wide : 16;   // a switch needs a 3% gain
        tuner_put(key, (uint32_t)rows);
      }
    }
    phase_begin(res, PH_INTER);
    if ((rc = launch(rows))) return (rc);
    phase_end(res, PH_INTER);
    res->phase_cells[PH_INTER] = p16cells;
    res->phase_cells[PH_INT32] -= p16cells;
    if (mode == DSA_LOCAL) {
      // exact int32 rerun of pairs whose packed pass saturated
      const uint32_t cap = (uint32_t)std::min<uint64_t>(n_pairs, 1u << 22);
      DevBuf d_list;
      if ((rc = d_list.alloc(ctx, (size_t)cap * sizeof(uint32_t)))) return (rc);
      uint32_t* d_count = ctx->d_counters + 1;
      if (cudaMemsetAsync(d_count, 0, sizeof(uint32_t), ctx->stream) != cudaSuccess) return (DSA_ERR_CUDA);
      if ((rc = launch_collect_flags(ctx, sc.flag, n_pairs, d_list.as<uint32_t>(), cap, d_count)))
        return rc;
      uint32_t count = 0;
      if (cudaMemcpyAsync(&count, d_count, sizeof(count), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
          cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        set_error("rerun count: %s", cudaGetErrorString(cudaGetLastError()));
        return (DSA_ERR_CUDA);
      }
      res->n_rerun = count;
      if (count > cap) { set_error("too many saturated pairs (%u)", count); return (DSA_ERR_UNSUPPORTED); }
      if (count) {
        if ((rc = pp.need_hp(ctx))) return (rc);
        std::vector<uint32_t> list(count);
        if (cudaMemcpy(list.data(), d_list.p, count * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
          return (DSA_ERR_CUDA);
        for (uint32_t k : list) {
          const dsa_pair& p = pp.hp[k];
          jobs.push_back({db->h_off[p.target_id] + p.t_offset, scr, p.query_id, p.t_len, k, 1});
          scr += p.t_len;
        }
      }
    }
  }
  const uint64_t n_short = jobs.size();
  if (n_short > 0) {   // pairs left for the int32 kernel
    std::vector<uint64_t> poff(qs->n);
    uint64_t pw = 0;
    for (uint32_t q = 0; q < qs->n; ++q) {
      poff[q] = pw;
      pw += (uint64_t)A * ((qs->h_len[q] + 7u) & ~7u);
    }
    DevBuf d_prof, d_poff, d_jobs, d_scr;
    if ((rc = d_prof.alloc(ctx, pw * 4)) || (rc = upload(ctx, d_poff, poff)) ||
        (rc = upload(ctx, d_jobs, jobs)) || (rc = d_scr.alloc(ctx, scr * sizeof(int2))))
      return (rc);
    if ((rc = launch_profile_int32(ctx, qs, d_mat, nullptr, A, d_prof.as<int32_t>(),
                                   d_poff.as<uint64_t>())))
      return (rc);
    phase_begin(res, PH_INT32);
    if ((rc = launch_generic_int32(ctx, db, qs, d_prof.as<int32_t>(), d_poff.as<uint64_t>(),
                                   d_jobs.as<PairJob>(), n_short, 0, d_scr.as<int2>(), mode, fe, o,
                                   e, 0, sc)))
      return (rc);
    phase_end(res, PH_INT32);
  }
  return DSA_OK;
}

}  // namespace dsa
