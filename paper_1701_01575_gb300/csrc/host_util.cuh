// Host-side helpers shared by the planning, traceback and entry-point
// translation units: loops over host threads, a stable radix order, device
// uploads, argument checks, and the score-pass and traceback drivers each
// file exports to the others.
#pragma once

#include "dsa_internal.cuh"

#include <string>
#include <thread>
#include <utility>
#include <vector>

namespace dsa {

// Host threads for a loop of n items, at least `per` items each (1 .. 16).
unsigned host_threads(size_t n, size_t per);

// fn(t, begin, end) over T contiguous ranges of [0, n), on T host threads.
template <class F>
void parallel_for(size_t n, unsigned T, F&& fn) {
  if (T <= 1) {
    fn(0u, (size_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(T);
  for (unsigned t = 0; t < T; ++t) th.emplace_back([&, t]() { fn(t, n * t / T, n * (t + 1) / T); });
  for (std::thread& x : th) x.join();
}

// Stable ascending order of 64-bit keys (an LSD radix sort on host threads).
std::vector<uint32_t> radix_order(const std::vector<uint64_t>& key);

template <class T>
int upload(dsa_ctx* ctx, DevBuf& buf, const T* p, size_t n) {
  DSA_TRY(buf.alloc(ctx, n * sizeof(T)));
  if (n) DSA_CUDA_TRY(cudaMemcpyAsync(buf.p, p, n * sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
  return DSA_OK;
}

template <class T>
int upload(dsa_ctx* ctx, DevBuf& buf, const std::vector<T>& v) {
  DSA_TRY(buf.alloc(ctx, v.size() * sizeof(T)));
  if (!v.empty())
    DSA_CUDA_TRY(cudaMemcpyAsync(buf.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice,
                                 ctx->stream));
  return DSA_OK;
}

int set_device(dsa_ctx* ctx);

struct Validated {
  int smax = 0, smin = 0;
  uint32_t max_m = 0, max_n = 0;
};

int check_matrix(const int8_t* matrix, int A, int o, int e, Validated* v);
// Position-specific profile: the value range of its `n` entries.
int check_pssm(const int8_t* pssm, uint64_t n, int o, int e, Validated* v);
// Band items (pair, band) of a band-pipelined score pass, in latest-start order.
std::vector<uint32_t> band_items(const std::vector<std::pair<uint32_t, uint32_t>>& mn, int band);
// Every S + o of the matrix fits int8 (the byte-permute substitution tables).
bool s_plus_o_fits_int8(const int8_t* matrix, int A, int o);

// Indices of the set flags among n (pairs whose packed pass saturated),
// gathered on the device into list (at most cap; *count gets the total).
int launch_collect_flags(dsa_ctx* ctx, const uint8_t* flag, uint64_t n, uint32_t* list,
                         uint32_t cap, uint32_t* count);

// Score pass for all queries x all targets (plan_all.cu).
int score_all_vs_all(dsa_ctx* ctx, dsa_res* res, const dsa_db* db, const dsa_db* qs, int mode,
                     uint32_t fe, const int8_t* d_mat, const int8_t* d_pssm, int A, int o, int e,
                     const Validated& v, uint32_t flags, Scores out, uint64_t* n_rerun);

// An explicit-pair score pass as dsa_align sets it up (plan_pairs.cu): the
// caller's pair array, its device copy, and the device classification.
struct PairPass {
  const dsa_pair* pairs = nullptr;    // the caller's array (device with DSA_PAIRS_ON_DEVICE)
  uint64_t n_pairs = 0;
  uint32_t flags = 0;
  const dsa_pair* d_pairs = nullptr;  // device copy (the caller's own when on the device)
  DevBuf d_pairs_buf, d_key, d_idx, d_hist, d_jcnt, d_stats;
  PairPlanStats pst{};
  uint64_t L = 0;                     // query lengths 0 .. L-1 are counted
  std::vector<dsa_pair> hp;           // host copy, made only when the host planner needs it
  bool hp_ready = false;
  int need_hp(dsa_ctx* ctx);
};
// Upload (unless on the device), range-check and classify the pairs.
int pairs_classify(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const PairPlanParams& P,
                   PairPass& pp);
// Score pass of classified pairs: packed int16x2 pairs (device or host
// planned) with the local saturation rerun, band-pipelined long pairs, and the
// exact int32 kernel for the rest.
int score_pairs(dsa_ctx* ctx, dsa_res* res, const dsa_db* db, const dsa_db* qs, PairPass& pp,
                int mode, uint32_t fe, const int8_t* matrix, const int8_t* d_mat, int A, int o,
                int e, const Validated& v, bool local16, bool packed_ok, int64_t w16, Scores sc);

// The autotuner's cache (a JSON file shared by the planners, plan_all.cu):
// tuner_get fails on a miss and under DSA_AUTOTUNE=retune; tuner_put records
// and writes the file.  tuner_shape_prefix: GPU name, SM count, driver.
bool tuner_get(const std::string& key, uint32_t* val);
void tuner_put(const std::string& key, uint32_t val);
std::string tuner_shape_prefix(dsa_ctx* ctx);
int tuner_bin(uint64_t x);   // floor(log2 x)

// Result hits (and CIGAR words) copied to the host arrays of the result.
int fetch_hits(dsa_res* res);

}  // namespace dsa
