// Device planning of an explicit pair list for the map phase's alignments
// (Sec. II.B.1; e.g. a million reads, each against
// its candidate window): validation, classification, the (query length,
// window length) ordering and the two-pairs-per-thread job layout of the
// packed int16 pairs kernel are all computed on the device, so the host
// touches no per-pair data.  The host planner in api.cu stays the path for
// calls that hold long or int32 pairs; both produce the same job list.
#include "dsa_internal.cuh"

namespace dsa {
namespace {

constexpr int PLAN_T = 256;
constexpr int RS_T = 256;       // radix sort: threads per tile (one per digit value)
constexpr int RS_ROUNDS = 8;    // items per thread; tile = RS_T * RS_ROUNDS
constexpr int RS_TILE = RS_T * RS_ROUNDS;
constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ uint64_t warp_sum(uint64_t v) {
  for (int s = 16; s > 0; s >>= 1) v += __shfl_xor_sync(FULL, v, s);
  return v;
}
__device__ __forceinline__ uint32_t warp_max(uint32_t v) {
  for (int s = 16; s > 0; s >>= 1) v = max(v, __shfl_xor_sync(FULL, v, s));
  return v;
}

// One pass over the pairs: range check (smallest bad index), the class of
// every pair, the sort key (m << 32 | t_len) of every packed pair, the number
// of packed pairs of every query length, and the call's totals.
__global__ void __launch_bounds__(PLAN_T) k_pair_classify(
    const dsa_pair* __restrict__ pairs, uint64_t n, const uint32_t* __restrict__ q_len,
    const uint32_t* __restrict__ db_len, PairPlanParams P, uint64_t* __restrict__ key,
    uint32_t* __restrict__ idx, uint64_t* __restrict__ hist, PairPlanStats* __restrict__ st) {
  __shared__ uint64_t red[4][PLAN_T / 32];
  __shared__ uint32_t redm[PLAN_T / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint64_t cells = 0, c16 = 0, n_other = 0, bad = UINT64_MAX;
  uint32_t max_t = 0;
  const uint64_t stride = (uint64_t)gridDim.x * PLAN_T;
  // whole warps iterate together (warp-aggregated histogram updates)
  for (uint64_t base = blockIdx.x * (uint64_t)PLAN_T + (threadIdx.x & ~31u); base < n; base += stride) {
    const uint64_t k = base + lane;
    uint32_t hm = UINT32_MAX;   // query length to count, or none
    if (k < n) {
      const dsa_pair p = pairs[k];
      const bool ok = p.query_id < P.n_queries && p.target_id < P.n_targets && p.t_len != 0 &&
                      p.t_offset <= db_len[p.target_id] &&
                      p.t_len <= db_len[p.target_id] - p.t_offset;
      if (!ok) {
        bad = min(bad, k);
      } else {
        const uint64_t m = q_len[p.query_id];
        const uint64_t c = m * p.t_len;
        cells += c;
        max_t = max(max_t, p.t_len);
        const bool fits16 =
            P.local16 || ((int64_t)(m + p.t_len) * P.w16 + P.o < 12000 && P.o + P.e < 4096);
        if (P.packed_ok && fits16 && m >= 1 && c < LONG_PAIR_CELLS) {
          key[k] = (m << 32) | p.t_len;
          idx[k] = (uint32_t)k;
          c16 += c;
          hm = (uint32_t)m;
        } else {
          ++n_other;
        }
      }
    }
    const unsigned peers = __match_any_sync(FULL, hm);
    if (hm != UINT32_MAX && (peers & ((1u << lane) - 1)) == 0)
      atomicAdd(reinterpret_cast<unsigned long long*>(hist + hm), (unsigned long long)__popc(peers));
  }
  cells = warp_sum(cells);
  c16 = warp_sum(c16);
  n_other = warp_sum(n_other);
  max_t = warp_max(max_t);
  for (int s = 16; s > 0; s >>= 1) bad = min(bad, __shfl_xor_sync(FULL, bad, s));
  if (lane == 0) {
    red[0][w] = cells; red[1][w] = c16; red[2][w] = n_other; red[3][w] = bad; redm[w] = max_t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int x = 1; x < PLAN_T / 32; ++x) {
      red[0][0] += red[0][x]; red[1][0] += red[1][x]; red[2][0] += red[2][x];
      red[3][0] = min(red[3][0], red[3][x]);
      redm[0] = max(redm[0], redm[x]);
    }
    auto* s = reinterpret_cast<unsigned long long*>(st);
    if (red[0][0]) atomicAdd(s + 0, (unsigned long long)red[0][0]);
    if (red[1][0]) atomicAdd(s + 1, (unsigned long long)red[1][0]);
    if (red[2][0]) atomicAdd(s + 2, (unsigned long long)red[2][0]);
    if (red[3][0] != UINT64_MAX) atomicMin(s + 3, (unsigned long long)red[3][0]);
    if (redm[0]) atomicMax(&st->max_t_len, redm[0]);
  }
}

// jobs of every query length: two pairs per job, the last one alone when the
// run is odd; their total goes to the stats
__global__ void __launch_bounds__(PLAN_T) k_pair_jobs_per_len(const uint64_t* __restrict__ hist,
                                                               uint64_t L, uint64_t* __restrict__ jcnt,
                                                               PairPlanStats* __restrict__ st) {
  uint64_t t = 0;
  for (uint64_t m = blockIdx.x * (uint64_t)PLAN_T + threadIdx.x; m < L;
       m += (uint64_t)gridDim.x * PLAN_T) {
    jcnt[m] = (hist[m] + 1) / 2;
    t += jcnt[m];
  }
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0 && t)
    atomicAdd(reinterpret_cast<unsigned long long*>(&st->n_jobs), (unsigned long long)t);
}

// Stable LSD radix sort of (key, value), one 8-bit digit per pass.  Pass part
// 1: digit counts of every tile, digit-major (the exclusive scan of this
// array is the first output position of every (digit, tile)).
__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint64_t* __restrict__ kin, uint64_t n,
                                                  int shift, uint64_t* __restrict__ counts,
                                                  uint32_t n_tiles) {
  __shared__ uint32_t h[256];
  const int lane = threadIdx.x & 31;
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t t0 = blockIdx.x * (uint64_t)RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const uint64_t x = t0 + (uint64_t)r * RS_T + threadIdx.x;
    const uint32_t d = x < n ? (uint32_t)(kin[x] >> shift) & 255u : 256u;
    const unsigned peers = __match_any_sync(FULL, d);
    if (d < 256 && (peers & ((1u << lane) - 1)) == 0) atomicAdd(&h[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  counts[(uint64_t)threadIdx.x * n_tiles + blockIdx.x] = h[threadIdx.x];
}

// Pass part 2: every item goes to its digit's position for this tile plus the
// number of equal digits before it in the tile (earlier rounds, earlier
// warps of its round, earlier lanes of its warp): input order is kept.
__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                     const uint32_t* __restrict__ vin, uint64_t n,
                                                     int shift, const uint64_t* __restrict__ off,
                                                     uint32_t n_tiles, uint64_t* __restrict__ kout,
                                                     uint32_t* __restrict__ vout) {
  __shared__ uint64_t base[256];
  __shared__ uint32_t wcnt[RS_T / 32][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  base[threadIdx.x] = off[(uint64_t)threadIdx.x * n_tiles + blockIdx.x];
#pragma unroll
  for (int x = 0; x < RS_T / 32; ++x) wcnt[x][threadIdx.x] = 0;
  __syncthreads();
  const uint64_t t0 = blockIdx.x * (uint64_t)RS_TILE;
  for (int r = 0; r < RS_ROUNDS; ++r) {
    const uint64_t x = t0 + (uint64_t)r * RS_T + threadIdx.x;
    const bool valid = x < n;
    const uint64_t k = valid ? kin[x] : 0;
    const uint32_t v = valid ? vin[x] : 0;
    const uint32_t d = valid ? (uint32_t)(k >> shift) & 255u : 256u;
    const unsigned peers = __match_any_sync(FULL, d);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1));
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      uint64_t pos = base[d] + rank;
      for (int y = 0; y < w; ++y) pos += wcnt[y][d];
      kout[pos] = k;
      vout[pos] = v;
    }
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int y = 0; y < RS_T / 32; ++y) {
      s += wcnt[y][threadIdx.x];
      wcnt[y][threadIdx.x] = 0;
    }
    base[threadIdx.x] += s;
    __syncthreads();
  }
}

// Jobs from the sorted pairs: a job starts at every even offset inside the
// run of a query length (run_start / job_off: exclusive scans of the run
// lengths and of the jobs per length; run m ends where run m + 1 starts).
__global__ void __launch_bounds__(PLAN_T) k_pair_build_jobs(
    const uint64_t* __restrict__ key, const uint32_t* __restrict__ val, uint64_t n,
    const uint64_t* __restrict__ run_start, const uint64_t* __restrict__ job_off,
    const dsa_pair* __restrict__ pairs, const uint64_t* __restrict__ q_off,
    const uint64_t* __restrict__ db_off, Pair16Job* __restrict__ jobs) {
  for (uint64_t x = blockIdx.x * (uint64_t)PLAN_T + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * PLAN_T) {
    const uint32_t m = (uint32_t)(key[x] >> 32);
    const uint64_t r = x - run_start[m];
    if (r & 1) continue;
    const dsa_pair a = pairs[val[x]];
    Pair16Job j{};
    j.m = (int32_t)m;
    j.q_lo = q_off[a.query_id];
    j.t_lo = db_off[a.target_id] + a.t_offset;
    j.n_lo = (int32_t)a.t_len;
    j.out_lo = val[x];
    if (x + 1 < run_start[m + 1]) {
      const dsa_pair b = pairs[val[x + 1]];
      j.q_hi = q_off[b.query_id];
      j.t_hi = db_off[b.target_id] + b.t_offset;
      j.n_hi = (int32_t)b.t_len;
      j.out_hi = val[x + 1];
    } else {
      j.q_hi = j.q_lo;
      j.t_hi = j.t_lo;
      j.n_hi = 0;
      j.out_hi = UINT32_MAX;
    }
    jobs[job_off[m] + r / 2] = j;
  }
}

unsigned plan_grid(dsa_ctx* ctx, uint64_t n) {
  const uint64_t b = (n + PLAN_T - 1) / PLAN_T;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, (uint64_t)ctx->sm_count * 8));
}

int launched(dsa_ctx* ctx, const char* what) {
  ++ctx->launches;
  if (cudaGetLastError() != cudaSuccess) {
    set_error("%s launch failed", what);
    return DSA_ERR_CUDA;
  }
  return DSA_OK;
}

int bits_of(uint64_t v) {
  int b = 0;
  while (v) { ++b; v >>= 1; }
  return b;
}

}  // namespace

int launch_pair_classify(dsa_ctx* ctx, const dsa_pair* d_pairs, uint64_t n, const dsa_db* qs,
                         const dsa_db* db, const PairPlanParams& P, uint64_t* d_key,
                         uint32_t* d_idx, uint64_t* d_hist, uint64_t L, uint64_t* d_jcnt,
                         PairPlanStats* d_stats) {
  if (n) {
    k_pair_classify<<<plan_grid(ctx, n), PLAN_T, 0, ctx->stream>>>(d_pairs, n, qs->d_len, db->d_len,
                                                                   P, d_key, d_idx, d_hist, d_stats);
    DSA_TRY(launched(ctx, "pair classify"));
  }
  k_pair_jobs_per_len<<<plan_grid(ctx, L), PLAN_T, 0, ctx->stream>>>(d_hist, L, d_jcnt, d_stats);
  return launched(ctx, "pair jobs per length");
}

int launch_pair_sort(dsa_ctx* ctx, uint64_t*& d_key, uint32_t*& d_val, uint64_t* d_key2,
                     uint32_t* d_val2, uint64_t n, uint32_t max_m, uint32_t max_t) {
  if (n == 0) return DSA_OK;
  const uint64_t tiles = (n + RS_TILE - 1) / RS_TILE;
  if (tiles > UINT32_MAX / 256) {
    set_error("too many pairs to sort (%llu)", (unsigned long long)n);
    return DSA_ERR_UNSUPPORTED;
  }
  DevBuf d_counts, d_total;
  DSA_TRY(d_counts.alloc(ctx, 256 * tiles * sizeof(uint64_t)));
  DSA_TRY(d_total.alloc(ctx, sizeof(uint64_t)));
  // window length digits first, then query length digits (LSD)
  std::vector<int> shifts;
  for (int s = 0; s < bits_of(max_t); s += 8) shifts.push_back(s);
  for (int s = 0; s < bits_of(max_m); s += 8) shifts.push_back(32 + s);
  uint64_t* kin = d_key; uint32_t* vin = d_val;
  uint64_t* kout = d_key2; uint32_t* vout = d_val2;
  for (int s : shifts) {
    k_rs_hist<<<(unsigned)tiles, RS_T, 0, ctx->stream>>>(kin, n, s, d_counts.as<uint64_t>(),
                                                         (uint32_t)tiles);
    DSA_TRY(launched(ctx, "radix histogram"));
    DSA_TRY(launch_scan_u64(ctx, d_counts.as<uint64_t>(), 256 * tiles, d_total.as<uint64_t>()));
    k_rs_scatter<<<(unsigned)tiles, RS_T, 0, ctx->stream>>>(kin, vin, n, s, d_counts.as<uint64_t>(),
                                                            (uint32_t)tiles, kout, vout);
    DSA_TRY(launched(ctx, "radix scatter"));
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  d_key = kin;
  d_val = vin;
  return DSA_OK;
}

int launch_pair_build_jobs(dsa_ctx* ctx, const uint64_t* d_key, const uint32_t* d_val, uint64_t n,
                           uint64_t* d_hist, uint64_t* d_jcnt, uint64_t L, const dsa_pair* d_pairs,
                           const dsa_db* qs, const dsa_db* db, Pair16Job* d_jobs) {
  if (n == 0) return DSA_OK;
  DevBuf d_total;
  DSA_TRY(d_total.alloc(ctx, sizeof(uint64_t)));
  DSA_TRY(launch_scan_u64(ctx, d_hist, L, d_total.as<uint64_t>()));
  DSA_TRY(launch_scan_u64(ctx, d_jcnt, L, d_total.as<uint64_t>()));
  k_pair_build_jobs<<<plan_grid(ctx, n), PLAN_T, 0, ctx->stream>>>(d_key, d_val, n, d_hist, d_jcnt,
                                                                   d_pairs, qs->d_off, db->d_off,
                                                                   d_jobs);
  return launched(ctx, "pair job build");
}

}  // namespace dsa
