// All-vs-all score pass (the map phase's per-pair scores of every query
// against every database sequence, Sec. II.B.1; DSW / DNW / DSG of
// Sec. II.C.2): the packed int16x2 path (inter-sequence kernel for most
// targets, wavefront kernel for the longest, with the autotuned split between
// them), the exact int32 rerun of saturated pairs, and the exact int32 kernel
// for searches the packed path cannot take.
#include "host_util.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <sys/stat.h>
#include <unistd.h>

namespace dsa {
namespace {


// ---- autotuner: kernel variant and long-target threshold of the packed path ----
//
// Two speed choices of the packed path (every choice gives the same exact
// results): the strip height of the inter-sequence kernel (28 rows, or 20
// rows, which wastes fewer padding rows on short queries), and which
// targets go to the wavefront kernel (long) and which to the inter-sequence
// kernel.  For a workload shape (GPU, driver, mode, alphabet,
// and log2 bins of the query count, query residues, longest query, target
// count, database residues and longest target) the first call times each
// strip height at the default threshold (a switch needs a 3% gain), then a
// local search of thresholds -- starting at 4096, then lower or higher by
// factors of 4 while it keeps improving by 3% or more -- and keeps both in a
// JSON cache file.  DSA_AUTOTUNE=off (28 rows, 4096) | cache (default: tune
// on a miss) | retune (always tune); DSA_AUTOTUNE_CACHE names the file
// (default $XDG_CACHE_HOME/dsa/autotune.json or ~/.cache/dsa/autotune.json);
// DSA_INTER_ROWS (28 | 20) and DSA_LONG_THRESHOLD fix their choice.
struct Tuner {
  std::mutex mu;
  bool loaded = false;
  std::string path;
  std::map<std::string, uint32_t> cache;
};
Tuner& tuner() {
  static Tuner t;
  return t;
}

std::string tune_cache_path() {
  if (const char* p = getenv("DSA_AUTOTUNE_CACHE")) return p;
  std::string dir;
  if (const char* x = getenv("XDG_CACHE_HOME")) dir = x;
  else if (const char* h = getenv("HOME")) dir = std::string(h) + "/.cache";
  else return "";
  return dir + "/dsa/autotune.json";
}

// flat JSON object of "key": unsigned integer
void tune_load(Tuner& t, const std::string& path) {
  t.loaded = true;
  t.path = path;
  t.cache.clear();
  if (t.path.empty()) return;
  FILE* f = fopen(t.path.c_str(), "rb");
  if (!f) return;
  std::string txt;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof buf, f)) > 0) txt.append(buf, n);
  fclose(f);
  size_t pos = 0;
  for (;;) {
    const size_t k0 = txt.find('"', pos);
    if (k0 == std::string::npos) break;
    const size_t k1 = txt.find('"', k0 + 1);
    if (k1 == std::string::npos) break;
    const size_t c = txt.find(':', k1);
    if (c == std::string::npos) break;
    char* endp = nullptr;
    const unsigned long long val = strtoull(txt.c_str() + c + 1, &endp, 10);
    if (endp == txt.c_str() + c + 1) break;
    t.cache[txt.substr(k0 + 1, k1 - k0 - 1)] =
        (uint32_t)std::min<unsigned long long>(val, UINT32_MAX);
    pos = (size_t)(endp - txt.c_str());
  }
}

void tune_store(Tuner& t) {
  if (t.path.empty()) return;
  const size_t slash = t.path.rfind('/');
  if (slash != std::string::npos) {
    // create the directory chain (failures are ignored: the cache is optional)
    const std::string d = t.path.substr(0, slash);
    for (size_t k = 1; k <= d.size(); ++k)
      if (k == d.size() || d[k] == '/') mkdir(d.substr(0, k).c_str(), 0755);
  }
  const std::string tmp = t.path + ".tmp" + std::to_string((long long)getpid());
  FILE* f = fopen(tmp.c_str(), "wb");
  if (!f) return;
  fputs("{\n", f);
  size_t k = 0;
  for (const auto& kv : t.cache)
    fprintf(f, "  \"%s\": %u%s\n", kv.first.c_str(), kv.second, ++k < t.cache.size() ? "," : "");
  fputs("}\n", f);
  fclose(f);
  rename(tmp.c_str(), t.path.c_str());
}

int ilog2_bin(uint64_t x) {
  int b = 0;
  while (x > 1) { x >>= 1; ++b; }
  return b;
}

// Packed score pass (int16x2).  Targets of groups longer than `long_thr` go
// to the wavefront kernel on the side stream, the rest to the
// inter-sequence kernel; the results do not depend on long_thr, only the
// time.  Global / semi-global use the end-anchored forms of both kernels.
int packed_score(dsa_ctx* ctx, dsa_res* res, const dsa_db* db, const dsa_db* qs,
                 const int8_t* d_mat, const int8_t* d_pssm, int A, int o, int e, const Validated& v, Scores out,
                 uint32_t long_thr, int rows, int mode = DSA_LOCAL, uint32_t fe = 15) {
  const bool local = mode == DSA_LOCAL;
  const uint32_t W = (uint32_t)rows;   // strip rows of the inter-sequence kernel
  const uint32_t nq = qs->n, nt = db->n;
  const int R = A + 1;
  std::vector<uint32_t> qorder(nq);
  std::iota(qorder.begin(), qorder.end(), 0u);
  std::stable_sort(qorder.begin(), qorder.end(),
                   [&](uint32_t a, uint32_t b) { return qs->h_len[a] > qs->h_len[b]; });
  auto strips_of = [&](uint32_t q) { return (qs->h_len[q] + W - 1) / W; };

  // groups whose longest target exceeds the threshold go to the wavefront kernel
  uint32_t g_long = 0;
  while (g_long < db->n_groups && db->h_glen[g_long] > long_thr) ++g_long;
  const uint32_t n_long = std::min<uint32_t>(nt, g_long * GROUP);

  // Stream plan for the inter-sequence kernel: queries are dealt, longest
  // first, to the currently shortest of K lanes (K about total / longest, so a
  // lane is about as long as the longest query); lanes are then paired by
  // length into units, low half = first lane, high half = second.
  uint64_t tot = 0, maxq = 1;
  for (uint32_t q = 0; q < nq; ++q) {
    tot += strips_of(q);
    maxq = std::max<uint64_t>(maxq, strips_of(q));
  }
  uint32_t K = (uint32_t)std::max<uint64_t>(1, (tot + maxq - 1) / maxq);
  K = std::min<uint32_t>(K, nq);
  K = (K + 1) & ~1u;   // even: lanes come in pairs
  std::vector<std::vector<uint32_t>> lanes(K);
  std::vector<uint64_t> load(K, 0);
  for (uint32_t q : qorder) {
    const uint32_t l = (uint32_t)(std::min_element(load.begin(), load.end()) - load.begin());
    lanes[l].push_back(q);
    load[l] += strips_of(q);
  }
  std::vector<uint32_t> lorder(K);
  std::iota(lorder.begin(), lorder.end(), 0u);
  std::stable_sort(lorder.begin(), lorder.end(), [&](uint32_t a, uint32_t b) { return load[a] > load[b]; });
  std::vector<StripMeta> smeta;
  std::vector<uint32_t> s_sbase, s_ns;
  auto lane_meta = [&](const std::vector<uint32_t>& lane, uint64_t s, uint32_t* q, uint32_t* k) {
    uint64_t start = 0;
    for (uint32_t x : lane) {
      const uint32_t ns_q = strips_of(x);
      if (s < start + ns_q) {
        *q = x;
        *k = (uint32_t)(s - start) | (s - start == ns_q - 1 ? LAST : 0u);
        return;
      }
      start += ns_q;
    }
    *q = NONE;
    *k = 0;
  };
  for (uint32_t u = 0; u < K / 2; ++u) {
    const auto& la = lanes[lorder[2 * u]];
    const auto& lb = lanes[lorder[2 * u + 1]];
    const uint64_t ns_u = std::max(load[lorder[2 * u]], load[lorder[2 * u + 1]]);
    if (ns_u == 0) continue;
    s_sbase.push_back((uint32_t)smeta.size());
    s_ns.push_back((uint32_t)ns_u);
    for (uint64_t st = 0; st < ns_u; ++st) {
      StripMeta m;
      lane_meta(la, st, &m.qa, &m.ka);
      lane_meta(lb, st, &m.qb, &m.kb);
      smeta.push_back(m);
    }
  }
  PackedPlan spl;
  spl.R = R;
  spl.rows = rows;
  spl.n_units = (uint32_t)s_ns.size();
  spl.n_strips = (uint32_t)smeta.size();

  const uint32_t blocks = (db->n_groups - g_long + INTER_WARPS - 1) / INTER_WARPS;
  struct Item { uint64_t cost; uint32_t p, g0; };
  std::vector<Item> items;
  items.reserve((size_t)spl.n_units * blocks);
  for (uint32_t u = 0; u < spl.n_units; ++u)
    for (uint32_t b = 0; b < blocks; ++b) {
      const uint32_t g0 = g_long + b * INTER_WARPS;
      items.push_back({(uint64_t)db->h_glen[g0] * s_ns[u], u, g0});
    }
  std::stable_sort(items.begin(), items.end(),
                   [](const Item& a, const Item& b) { return a.cost > b.cost; });
  std::vector<uint32_t> item_words(2 * items.size());
  for (size_t k = 0; k < items.size(); ++k) {
    item_words[2 * k] = items[k].p;
    item_words[2 * k + 1] = items[k].g0;
  }
  InterWork iw;
  iw.n_items = (uint32_t)items.size();
  iw.max_glen = g_long < db->n_groups ? db->h_glen[g_long] : 0;

  // Pair plan for the wavefront kernel: one query per half (sorted neighbours).
  PackedPlan ppl;
  IntraWork xw;
  std::vector<StripMeta> pmeta;
  std::vector<uint32_t> p_sbase, p_ns, long_ids, litem_words;
  uint64_t long_res = 0;
  if (n_long) {
    ppl.R = R;
    ppl.rows = 32;   // the wavefront kernel's lanes take half-strips of 16 rows
    auto strips32 = [&](uint32_t q) { return (qs->h_len[q] + 31u) / 32u; };
    for (uint32_t u = 0; 2 * u < nq; ++u) {
      const uint32_t qa = qorder[2 * u];
      const uint32_t qb = 2 * u + 1 < nq ? qorder[2 * u + 1] : NONE;
      const uint32_t ns_u = std::max(strips32(qa), qb != NONE ? strips32(qb) : 0u);
      p_sbase.push_back((uint32_t)pmeta.size());
      p_ns.push_back(ns_u);
      for (uint32_t st = 0; st < ns_u; ++st)
        pmeta.push_back({qa, st | (st == ns_u - 1 ? LAST : 0u), qb, st | (st == ns_u - 1 ? LAST : 0u)});
    }
    ppl.n_units = (uint32_t)p_ns.size();
    ppl.n_strips = (uint32_t)pmeta.size();
    long_ids.assign(db->h_perm.begin(), db->h_perm.begin() + n_long);
    struct LItem { uint64_t cost; uint32_t li, p; };
    std::vector<LItem> litems;
    litems.reserve((size_t)n_long * ppl.n_units);
    for (uint32_t li = 0; li < n_long; ++li) {
      const uint32_t L = db->h_len[long_ids[li]];
      long_res += L;
      xw.max_long_len = std::max(xw.max_long_len, L);
      for (uint32_t u = 0; u < ppl.n_units; ++u) litems.push_back({(uint64_t)L * p_ns[u], li, u});
    }
    std::stable_sort(litems.begin(), litems.end(),
                     [](const LItem& a, const LItem& b) { return a.cost > b.cost; });
    litem_words.resize(2 * litems.size());
    for (size_t k = 0; k < litems.size(); ++k) {
      litem_words[2 * k] = litems[k].li;
      litem_words[2 * k + 1] = litems[k].p;
    }
    xw.n_items = (uint32_t)litems.size();
  }
  uint64_t qsum = 0;
  for (uint32_t x : qs->h_len) qsum += x;
  if (res) {
    res->phase_cells[PH_INTRA] = qsum * long_res;
    res->phase_cells[PH_INTER] = qsum * (db->n_res - long_res);
  }

  DevBuf d_smeta, d_sbase, d_sns, d_sprof, d_items, d_pmeta, d_pbase, d_pns, d_pprof, d_long, d_litems;
  DSA_TRY(upload(ctx, d_smeta, smeta));
  DSA_TRY(upload(ctx, d_sbase, s_sbase));
  DSA_TRY(upload(ctx, d_sns, s_ns));
  DSA_TRY(upload(ctx, d_items, item_words));
  DSA_TRY(d_sprof.alloc(ctx, (size_t)spl.n_strips * R * spl.pitch * sizeof(uint32_t)));
  spl.d_meta = d_smeta.as<StripMeta>();
  spl.d_sbase = d_sbase.as<uint32_t>();
  spl.d_ns = d_sns.as<uint32_t>();
  spl.d_prof = d_sprof.as<uint32_t>();
  iw.d_items = d_items.as<uint32_t>();
  // end-anchored strips: the padding rows above a query reproduce row 0
  // (S + o = 0 against the boundary -(o + (j-1)e), o against a free begin)
  const int tpad = (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_T_BEGIN)) ? o : 0;
  DSA_TRY(launch_strip_profile(ctx, qs, d_mat, d_pssm, A, o, spl, !local, tpad));
  if (n_long) {
    DSA_TRY(upload(ctx, d_pmeta, pmeta));
    DSA_TRY(upload(ctx, d_pbase, p_sbase));
    DSA_TRY(upload(ctx, d_pns, p_ns));
    DSA_TRY(upload(ctx, d_long, long_ids));
    DSA_TRY(upload(ctx, d_litems, litem_words));
    DSA_TRY(d_pprof.alloc(ctx, (size_t)ppl.n_strips * R * ppl.pitch * sizeof(uint32_t)));
    ppl.d_meta = d_pmeta.as<StripMeta>();
    ppl.d_sbase = d_pbase.as<uint32_t>();
    ppl.d_ns = d_pns.as<uint32_t>();
    ppl.d_prof = d_pprof.as<uint32_t>();
    xw.d_long_ids = d_long.as<uint32_t>();
    xw.d_items = d_litems.as<uint32_t>();
    DSA_TRY(launch_strip_profile(ctx, qs, d_mat, d_pssm, A, o, ppl, !local, tpad));
    // long targets on the side stream, overlapping the inter-sequence kernel:
    // the two kernels write disjoint targets' results
    DSA_CUDA_TRY(cudaEventRecord(ctx->fork_ev, ctx->stream));
    DSA_CUDA_TRY(cudaStreamWaitEvent(ctx->side, ctx->fork_ev, 0));
    phase_begin(res, PH_INTRA, ctx->side);
    if (local)
      DSA_TRY(launch_intra_local16(ctx, ctx->side, db, ppl, xw, o, e, v.smax, out, nt));
    else
      DSA_TRY(launch_intra_glob16(ctx, ctx->side, db, qs, ppl, xw, mode, fe, o, e, v.smax, v.smin,
                                  out, nt));
    phase_end(res, PH_INTRA, ctx->side);
    DSA_CUDA_TRY(cudaEventRecord(ctx->join_ev, ctx->side));
  }
  phase_begin(res, PH_INTER);
  if (local)
    DSA_TRY(launch_inter_local16(ctx, db, spl, iw, o, e, v.smax, out, nt));
  else
    DSA_TRY(launch_inter_glob16(ctx, db, qs, spl, iw, mode, fe, o, e, v.smax, v.smin, out, nt));
  phase_end(res, PH_INTER);
  if (n_long) DSA_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->join_ev, 0));
  return DSA_OK;
}

// Strip rows forced by DSA_INTER_ROWS (0: let the tuner choose).
int forced_rows() {
  if (const char* env = getenv("DSA_INTER_ROWS")) {
    const int r = atoi(env);
    if (r == INTER_ROWS || r == INTER_ROWS_SHORT) return r;
  }
  return 0;
}

// The packed pass with the autotuned kernel variant (strip rows) and
// long-target threshold.
int run_packed_tuned(dsa_ctx* ctx, dsa_res* res, const dsa_db* db, const dsa_db* qs,
                     const int8_t* d_mat, const int8_t* d_pssm, int A, int o, int e,
                     const Validated& v, Scores out, int mode, uint32_t fe) {
  const bool local = mode == DSA_LOCAL;
  constexpr uint32_t DEFAULT_THR = 4096;
  const int rows_forced = forced_rows();
  const char* thr_env = getenv("DSA_LONG_THRESHOLD");
  const uint32_t thr_forced = thr_env ? (uint32_t)strtoul(thr_env, nullptr, 10) : 0;
  auto run = [&](dsa_res* r, uint32_t thr, int rows) {
    return packed_score(ctx, r, db, qs, d_mat, d_pssm, A, o, e, v, out, thr, rows, mode, fe);
  };
  const char* mode_env = getenv("DSA_AUTOTUNE");
  const std::string tmode = mode_env ? mode_env : "cache";
  const int rows_default = rows_forced ? rows_forced : INTER_ROWS;
  const uint32_t thr_default = thr_env ? thr_forced : DEFAULT_THR;
  if (tmode == "off" || (rows_forced && thr_env))
    return run(res, thr_default, rows_default);
  // workload shape key: GPU, driver, mode, alphabet, and log2 bins of the
  // query count, query residues, longest query, target count, database
  // residues and longest target
  uint64_t qres = 0;
  uint32_t qmax = 0;
  for (uint32_t x : qs->h_len) { qres += x; qmax = std::max(qmax, x); }
  cudaDeviceProp prop;
  DSA_CUDA_TRY(cudaGetDeviceProperties(&prop, ctx->device));
  int drv = 0;
  cudaDriverGetVersion(&drv);
  char key[512];
  snprintf(key, sizeof key, "%s|sm%d|drv%d|%s|A%d|q%d|qr%d|qm%d|t%d|tr%d|L%d", prop.name,
           ctx->sm_count, drv, local ? "local" : (mode == DSA_GLOBAL ? "global" : "semi"), A,
           ilog2_bin(qs->n), ilog2_bin(qres), ilog2_bin(qmax), ilog2_bin(db->n),
           ilog2_bin(db->n_res), ilog2_bin(db->max_len));
  const std::string key_thr = std::string(key) + "|thr", key_rows = std::string(key) + "|rows";
  Tuner& t = tuner();
  {
    std::lock_guard<std::mutex> lk(t.mu);
    const std::string path = tune_cache_path();
    if (!t.loaded || path != t.path) tune_load(t, path);   // first use, or another file
    auto it_r = t.cache.find(key_rows);
    auto it_t = t.cache.find(key_thr);
    if (tmode != "retune" && it_r != t.cache.end() && it_t != t.cache.end())
      return run(res, thr_env ? thr_forced : it_t->second,
                 rows_forced ? rows_forced : (int)it_r->second);
  }
  if (!ctx->tune)   // contexts that must not spend calls on tuning (serving workers)
    return run(res, thr_default, rows_default);
  std::map<std::pair<uint32_t, int>, double> timed;   // (long groups, rows) -> ms
  auto groups_over = [&](uint32_t thr) {
    uint32_t g = 0;
    while (g < db->n_groups && db->h_glen[g] > thr) ++g;
    return g;
  };
  cudaEvent_t ev0, ev1;
  DSA_CUDA_TRY(cudaEventCreate(&ev0));
  DSA_CUDA_TRY(cudaEventCreate(&ev1));
  int rc = DSA_OK;
  auto measure = [&](uint32_t thr, int rows) -> double {
    const auto k = std::make_pair(groups_over(thr), rows);
    auto it = timed.find(k);
    if (it != timed.end()) return it->second;
    float ms = 0.f;
    if (rc == DSA_OK && cudaEventRecord(ev0, ctx->stream) != cudaSuccess) rc = DSA_ERR_CUDA;
    if (rc == DSA_OK) rc = run(nullptr, thr, rows);
    if (rc == DSA_OK && cudaEventRecord(ev1, ctx->stream) != cudaSuccess) rc = DSA_ERR_CUDA;
    if (rc == DSA_OK && cudaEventSynchronize(ev1) != cudaSuccess) rc = DSA_ERR_CUDA;
    if (rc == DSA_OK) cudaEventElapsedTime(&ms, ev0, ev1);
    timed[k] = ms;
    return ms;
  };
  // 1. the kernel variant (strip rows) at the default threshold; a switch
  //    from the default needs a gain of at least 3% (single timings)
  int best_rows = rows_default;
  double best_ms = measure(thr_default, best_rows);
  if (!rows_forced)
    for (int rows : {INTER_ROWS_SHORT}) {
      const double ms = measure(thr_default, rows);
      if (ms < 0.97 * best_ms) { best_ms = ms; best_rows = rows; }
    }
  // 2. the long-target threshold, a local search from the
  //    default by factors of 4 in each direction while it improves;
  //    thresholds that move the same groups as the last one are skipped
  uint32_t best = thr_default;
  if (!thr_env)
    for (int dir = -1; dir <= 1 && rc == DSA_OK; dir += 2) {
      uint64_t cur = DEFAULT_THR;
      uint32_t last_g = groups_over(DEFAULT_THR);
      for (int step = 0; step < 12 && rc == DSA_OK; ++step) {
        const uint64_t nx = dir < 0 ? cur / 4 : cur * 4;
        const uint32_t thr = (dir > 0 && nx >= db->max_len) ? UINT32_MAX : (uint32_t)nx;
        cur = nx;
        const uint32_t g = groups_over(thr);
        if (g == last_g) {
          if (thr == 0 || thr == UINT32_MAX) break;
          continue;
        }
        last_g = g;
        const double ms = measure(thr, best_rows);
        if (ms < 0.97 * best_ms) {
          best_ms = ms;
          best = thr;
        } else {
          break;
        }
        if (thr == 0 || thr == UINT32_MAX) break;
      }
    }
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  if (rc) {
    set_error("autotune: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  {
    std::lock_guard<std::mutex> lk(t.mu);
    if (!rows_forced) t.cache[key_rows] = (uint32_t)best_rows;
    if (!thr_env) t.cache[key_thr] = best;
    tune_store(t);
  }
  // the final pass with the chosen variant records the phase timings and cells
  return run(res, best, best_rows);
}

}  // namespace

bool tuner_get(const std::string& key, uint32_t* val) {
  Tuner& t = tuner();
  std::lock_guard<std::mutex> lk(t.mu);
  const std::string path = tune_cache_path();
  if (!t.loaded || path != t.path) tune_load(t, path);
  const char* mode_env = getenv("DSA_AUTOTUNE");
  if (mode_env && std::string(mode_env) == "retune") return false;
  auto it = t.cache.find(key);
  if (it == t.cache.end()) return false;
  *val = it->second;
  return true;
}

void tuner_put(const std::string& key, uint32_t val) {
  Tuner& t = tuner();
  std::lock_guard<std::mutex> lk(t.mu);
  t.cache[key] = val;
  tune_store(t);
}

std::string tuner_shape_prefix(dsa_ctx* ctx) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess) {
    cudaGetLastError();
    return "?";
  }
  int drv = 0;
  cudaDriverGetVersion(&drv);
  char key[320];
  snprintf(key, sizeof key, "%s|sm%d|drv%d", prop.name, ctx->sm_count, drv);
  return key;
}

int tuner_bin(uint64_t x) { return ilog2_bin(x); }

// Score pass for all queries x all targets.
int score_all_vs_all(dsa_ctx* ctx, dsa_res* res, const dsa_db* db, const dsa_db* qs, int mode,
                     uint32_t fe, const int8_t* d_mat, const int8_t* d_pssm, int A, int o, int e, const Validated& v,
                     uint32_t flags, Scores out, uint64_t* n_rerun) {
  const uint32_t nq = qs->n, nt = db->n;
  // int16x2 lanes: local with the saturation flag; global and semi-global
  // with the range flags of the end-anchored kernel (both reruns exact)
  const bool packed = !(flags & (DSA_FORCE_INT32 | DSA_PLAIN_FORM)) &&
                      (mode == DSA_LOCAL ? o >= 1 : true) && o + e <= 4096 &&
                      v.smax + o < 8192 && v.smin > -8192;
  *n_rerun = 0;
  if (!packed) {
    // exact int32: one launch per query over every target (input order)
    std::vector<uint64_t> poff(nq);
    uint64_t words = 0;
    for (uint32_t q = 0; q < nq; ++q) {
      poff[q] = words;
      words += (uint64_t)A * ((qs->h_len[q] + 7u) & ~7u);
    }
    DevBuf d_prof, d_poff, d_scr;
    DSA_TRY(d_prof.alloc(ctx, words * sizeof(int32_t)));
    DSA_TRY(upload(ctx, d_poff, poff));
    DSA_TRY(launch_profile_int32(ctx, qs, d_mat, d_pssm, A, d_prof.as<int32_t>(), d_poff.as<uint64_t>()));
    DSA_TRY(d_scr.alloc(ctx, db->n_res * sizeof(int2)));
    if (res) {
      uint64_t qsum = 0;
      for (uint32_t x : qs->h_len) qsum += x;
      res->phase_cells[PH_INT32] += qsum * db->n_res;
    }
    phase_begin(res, PH_INT32);
    for (uint32_t q = 0; q < nq; ++q)
      DSA_TRY(launch_generic_int32(ctx, db, qs, d_prof.as<int32_t>(), d_poff.as<uint64_t>(),
                                   nullptr, nt, q, d_scr.as<int2>(), mode, fe, o, e, 0, out));
    phase_end(res, PH_INT32);
    return DSA_OK;
  }

  // ---- packed path ----
  DSA_TRY(ensure_interleaved(ctx, db));
  DSA_TRY(run_packed_tuned(ctx, res, db, qs, d_mat, d_pssm, A, o, e, v, out, mode, fe));

  // ---- exact int32 rerun of saturated pairs ----
  const uint64_t n_out = (uint64_t)nq * nt;
  const uint32_t cap = (uint32_t)std::min<uint64_t>(n_out, 1u << 22);
  DevBuf d_list;
  DSA_TRY(d_list.alloc(ctx, (size_t)cap * sizeof(uint32_t)));
  uint32_t* d_count = ctx->d_counters + 1;
  DSA_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(uint32_t), ctx->stream));
  DSA_TRY(launch_collect_flags(ctx, out.flag, n_out, d_list.as<uint32_t>(), cap, d_count));
  uint32_t count = 0;
  DSA_CUDA_TRY(cudaMemcpyAsync(&count, d_count, sizeof(count), cudaMemcpyDeviceToHost, ctx->stream));
  DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  *n_rerun = count;
  if (count == 0) return DSA_OK;
  std::vector<PairJob> jobs;
  if (count > cap) {
    // too many to list: rerun everything in int32
    return score_all_vs_all(ctx, res, db, qs, mode, fe, d_mat, d_pssm, A, o, e, v, flags | DSA_FORCE_INT32,
                            out, n_rerun);
  }
  std::vector<uint32_t> list(count);
  DSA_CUDA_TRY(cudaMemcpyAsync(list.data(), d_list.p, count * sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, ctx->stream));
  DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  std::sort(list.begin(), list.end());
  jobs.resize(count);
  uint64_t scr = 0;
  for (uint32_t k = 0; k < count; ++k) {
    const uint32_t q = list[k] / nt, t = list[k] % nt;
    jobs[k] = {db->h_off[t], scr, q, db->h_len[t], list[k], 0};
    scr += db->h_len[t];
  }
  std::vector<uint64_t> poff(nq);
  uint64_t pw = 0;
  for (uint32_t q = 0; q < nq; ++q) {
    poff[q] = pw;
    pw += (uint64_t)A * ((qs->h_len[q] + 7u) & ~7u);
  }
  DevBuf d_prof32, d_poff32, d_jobs, d_scr;
  DSA_TRY(d_prof32.alloc(ctx, pw * sizeof(int32_t)));
  DSA_TRY(upload(ctx, d_poff32, poff));
  DSA_TRY(launch_profile_int32(ctx, qs, d_mat, d_pssm, A, d_prof32.as<int32_t>(), d_poff32.as<uint64_t>()));
  DSA_TRY(upload(ctx, d_jobs, jobs));
  DSA_TRY(d_scr.alloc(ctx, scr * sizeof(int2)));
  phase_begin(res, PH_INT32);
  DSA_TRY(launch_generic_int32(ctx, db, qs, d_prof32.as<int32_t>(), d_poff32.as<uint64_t>(),
                               d_jobs.as<PairJob>(), count, 0, d_scr.as<int2>(), mode, fe, o, e, 1,
                               out));
  phase_end(res, PH_INT32);
  return DSA_OK;
}

}  // namespace dsa
