// Device staging of the thread-per-hit traceback (location and CIGAR of the
// alignment object, Sec. II.B.1) for large hit batches (e.g. every read of
// a reads-in-windows search): the jobs are built from the
// device-resident hits, compacted, and laid out in groups of 32 on the
// device, so the host touches no per-hit data.  The job of a hit and its
// score-derived windows come from tb_short_job, the same function the host
// staging uses.
#include "dsa_internal.cuh"

namespace dsa {
namespace {

constexpr int SCAN_T = 256;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;
constexpr int STAGE_T = 256;
constexpr int TB_ORDER_WC_CAP = 65535;   // ordering key: wider windows sort together

// exclusive scan of one tile per block; the tile's sum goes to sums[block]
__global__ void __launch_bounds__(SCAN_T) k_scan_tile(uint64_t* __restrict__ data, uint64_t n,
                                                       uint64_t* __restrict__ sums) {
  __shared__ uint64_t part[SCAN_T];
  const int tid = threadIdx.x;
  const uint64_t base = blockIdx.x * (uint64_t)SCAN_TILE + (uint64_t)tid * SCAN_ITEMS;
  uint64_t v[SCAN_ITEMS];
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = base + k < n ? data[base + k] : 0;
    acc += v[k];
  }
  part[tid] = acc;
  __syncthreads();
  for (int off = 1; off < SCAN_T; off <<= 1) {
    const uint64_t x = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += x;
    __syncthreads();
  }
  uint64_t run = part[tid] - acc;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) data[base + k] = run;
    run += v[k];
  }
  if (tid == SCAN_T - 1) sums[blockIdx.x] = part[tid];
}

__global__ void __launch_bounds__(SCAN_T) k_scan_add(uint64_t* __restrict__ data, uint64_t n,
                                                      const uint64_t* __restrict__ sums) {
  const uint64_t base = blockIdx.x * (uint64_t)SCAN_TILE;
  const uint64_t add = sums[blockIdx.x];
  for (uint64_t x = threadIdx.x; x < SCAN_TILE; x += SCAN_T)
    if (base + x < n) data[base + x] += add;
}

// job of every hit (valid[k] = 1) or a skip (already traced, or local score 0)
__global__ void __launch_bounds__(STAGE_T) k_tb_stage(
    const dsa_hit* __restrict__ hits, uint64_t n, const uint64_t* __restrict__ q_off,
    const uint64_t* __restrict__ t_off, TbBounds B, TbJob* __restrict__ full,
    uint64_t* __restrict__ valid, uint32_t* __restrict__ not_small) {
  for (uint64_t k = blockIdx.x * (uint64_t)STAGE_T + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * STAGE_T) {
    const dsa_hit h = hits[k];
    const bool skip = (h.flags & DSA_HIT_HAS_TRACEBACK) ||
                      (B.mode == DSA_LOCAL && (h.q_end < 0 || h.t_end < 0));
    valid[k] = skip ? 0u : 1u;
    if (skip) continue;
    TbJob j;
    tb_short_job(B, h.q_end + 1, h.t_end + 1, h.score, q_off[h.query_id],
                 t_off[h.target_id] + h.t_offset, (uint32_t)k, j);
    if (!(j.ie <= 4096 && (uint64_t)j.ie * (uint64_t)j.je <= (1u << 20))) atomicAdd(not_small, 1u);
    full[k] = j;
  }
}

// valid jobs in hit order (pos = exclusive scan of valid, total = their count)
__global__ void __launch_bounds__(STAGE_T) k_tb_compact(const TbJob* __restrict__ full,
                                                         const uint64_t* __restrict__ pos,
                                                         const uint64_t* __restrict__ total,
                                                         uint64_t n, TbJob* __restrict__ jobs) {
  for (uint64_t k = blockIdx.x * (uint64_t)STAGE_T + threadIdx.x; k < n;
       k += (uint64_t)gridDim.x * STAGE_T) {
    const uint64_t next = k + 1 < n ? pos[k + 1] : *total;
    if (next > pos[k]) jobs[pos[k]] = full[k];
  }
}

// per group of 32 jobs: its layout sizes (decision words, scratch columns);
// per job its CIGAR capacity; the group's column stride goes to every member
__global__ void __launch_bounds__(STAGE_T) k_tb_groups(TbJob* __restrict__ jobs, uint64_t n,
                                                        uint64_t* __restrict__ gdir,
                                                        uint64_t* __restrict__ gscr,
                                                        uint64_t* __restrict__ jcig) {
  const uint64_t n_groups = (n + 31) / 32;
  for (uint64_t g = blockIdx.x * (uint64_t)STAGE_T + threadIdx.x; g < n_groups;
       g += (uint64_t)gridDim.x * STAGE_T) {
    const uint64_t x0 = 32 * g, x1 = x0 + 32 < n ? x0 + 32 : n;
    int32_t ie_max = 1, je_max = 1, wc_max = 1;
    for (uint64_t x = x0; x < x1; ++x) {
      const TbJob& j = jobs[x];
      ie_max = max(ie_max, j.ie);
      je_max = max(je_max, j.je);
      wc_max = max(wc_max, j.wc);
      jcig[x] = (uint64_t)j.ie + j.je + 1;
    }
    for (uint64_t x = x0; x < x1; ++x) jobs[x].wpr = (uint32_t)wc_max;
    gdir[g] = ((uint64_t)ie_max + TB_STRIP - 1) / TB_STRIP * (uint64_t)wc_max * (32 * TB_STRIP_WORDS);
    gscr[g] = (uint64_t)je_max * 32;
  }
}

__global__ void __launch_bounds__(STAGE_T) k_tb_assign(TbJob* __restrict__ jobs, uint64_t n,
                                                        const uint64_t* __restrict__ gdir,
                                                        const uint64_t* __restrict__ gscr,
                                                        const uint64_t* __restrict__ jcig) {
  for (uint64_t x = blockIdx.x * (uint64_t)STAGE_T + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * STAGE_T) {
    const uint64_t g = x / 32, lane = x % 32;
    jobs[x].dir_off = gdir[g] + lane;
    jobs[x].scr_off = gscr[g] + lane;
    jobs[x].cig_off = jcig[x];
  }
}

// sort key of a job: (rows, stored columns), the work of its thread
__global__ void __launch_bounds__(STAGE_T) k_tb_keys(const TbJob* __restrict__ jobs, uint64_t n,
                                                      uint64_t* __restrict__ key,
                                                      uint32_t* __restrict__ idx) {
  for (uint64_t x = blockIdx.x * (uint64_t)STAGE_T + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * STAGE_T) {
    const TbJob& j = jobs[x];
    key[x] = ((uint64_t)(uint32_t)j.ie << 32) | (uint32_t)min(j.wc, TB_ORDER_WC_CAP);
    idx[x] = (uint32_t)x;
  }
}

__global__ void __launch_bounds__(STAGE_T) k_tb_gather(const TbJob* __restrict__ in,
                                                        const uint32_t* __restrict__ idx,
                                                        uint64_t n, TbJob* __restrict__ out) {
  for (uint64_t x = blockIdx.x * (uint64_t)STAGE_T + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * STAGE_T)
    out[x] = in[idx[x]];
}

unsigned stage_grid(dsa_ctx* ctx, uint64_t n) {
  const uint64_t b = (n + STAGE_T - 1) / STAGE_T;
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, (uint64_t)ctx->sm_count * 16));
}

}  // namespace

int launch_scan_u64(dsa_ctx* ctx, uint64_t* d_data, uint64_t n, uint64_t* d_total) {
  if (n == 0) {
    DSA_CUDA_TRY(cudaMemsetAsync(d_total, 0, sizeof(uint64_t), ctx->stream));
    return DSA_OK;
  }
  const uint64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  void* sums = nullptr;
  DSA_TRY(ctx->alloc(&sums, tiles * sizeof(uint64_t)));
  uint64_t* s = static_cast<uint64_t*>(sums);
  k_scan_tile<<<(unsigned)tiles, SCAN_T, 0, ctx->stream>>>(d_data, n, s);
  ++ctx->launches;
  int rc = DSA_OK;
  if (cudaGetLastError() != cudaSuccess) {
    set_error("scan launch failed");
    rc = DSA_ERR_CUDA;
  } else if (tiles > 1) {
    rc = launch_scan_u64(ctx, s, tiles, d_total);
    if (rc == DSA_OK) {
      k_scan_add<<<(unsigned)tiles, SCAN_T, 0, ctx->stream>>>(d_data, n, s);
      ++ctx->launches;
      if (cudaGetLastError() != cudaSuccess) {
        set_error("scan launch failed");
        rc = DSA_ERR_CUDA;
      }
    }
  } else if (cudaMemcpyAsync(d_total, s, sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                             ctx->stream) != cudaSuccess) {
    set_error("scan total copy failed");
    rc = DSA_ERR_CUDA;
  }
  ctx->release(sums, tiles * sizeof(uint64_t));
  return rc;
}

int launch_tb_stage(dsa_ctx* ctx, const dsa_hit* d_hits, uint64_t n, const uint64_t* d_q_off,
                    const uint64_t* d_t_off, const TbBounds& B, TbJob* d_full, uint64_t* d_valid,
                    uint32_t* d_not_small) {
  k_tb_stage<<<stage_grid(ctx, n), STAGE_T, 0, ctx->stream>>>(d_hits, n, d_q_off, d_t_off, B,
                                                             d_full, d_valid, d_not_small);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_tb_compact(dsa_ctx* ctx, const TbJob* d_full, const uint64_t* d_pos,
                      const uint64_t* d_total, uint64_t n, TbJob* d_jobs) {
  k_tb_compact<<<stage_grid(ctx, n), STAGE_T, 0, ctx->stream>>>(d_full, d_pos, d_total, n, d_jobs);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_tb_layout(dsa_ctx* ctx, TbJob* d_jobs, uint64_t n, uint64_t* d_gdir, uint64_t* d_gscr,
                     uint64_t* d_jcig, uint64_t* d_totals) {
  const uint64_t n_groups = (n + 31) / 32;
  k_tb_groups<<<stage_grid(ctx, n_groups), STAGE_T, 0, ctx->stream>>>(d_jobs, n, d_gdir, d_gscr,
                                                                       d_jcig);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  DSA_TRY(launch_scan_u64(ctx, d_gdir, n_groups, d_totals + 0));
  DSA_TRY(launch_scan_u64(ctx, d_gscr, n_groups, d_totals + 1));
  DSA_TRY(launch_scan_u64(ctx, d_jcig, n, d_totals + 2));
  k_tb_assign<<<stage_grid(ctx, n), STAGE_T, 0, ctx->stream>>>(d_jobs, n, d_gdir, d_gscr, d_jcig);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

}  // namespace dsa

namespace dsa {
namespace {

__global__ void __launch_bounds__(STAGE_T) k_cig_lens(const dsa_hit* __restrict__ hits,
                                                      const TbJob* __restrict__ jobs, uint64_t n,
                                                      uint64_t* __restrict__ lens) {
  for (uint64_t x = blockIdx.x * (uint64_t)STAGE_T + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * STAGE_T)
    lens[x] = hits[jobs[x].hit].cigar_len;
}

__global__ void __launch_bounds__(STAGE_T) k_cig_place(dsa_hit* __restrict__ hits,
                                                       const TbJob* __restrict__ jobs, uint64_t n,
                                                       const uint64_t* __restrict__ pos,
                                                       const uint64_t* __restrict__ base) {
  for (uint64_t x = blockIdx.x * (uint64_t)STAGE_T + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * STAGE_T)
    hits[jobs[x].hit].cigar_off = *base + pos[x];
}

__global__ void k_add_u64(uint64_t* __restrict__ a, const uint64_t* __restrict__ b) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *a += *b;
}

}  // namespace

// Jobs in (rows, stored columns) order, stable: consecutive groups of 32 --
// one warp of the thread kernel, which runs as long as its longest hit --
// then hold hits of about the same work.
int launch_tb_order(dsa_ctx* ctx, const TbJob* d_in, uint64_t n, TbJob* d_out) {
  if (n == 0) return DSA_OK;
  DevBuf key, idx, key2, idx2;
  DSA_TRY(key.alloc(ctx, n * sizeof(uint64_t)));
  DSA_TRY(idx.alloc(ctx, n * sizeof(uint32_t)));
  DSA_TRY(key2.alloc(ctx, n * sizeof(uint64_t)));
  DSA_TRY(idx2.alloc(ctx, n * sizeof(uint32_t)));
  k_tb_keys<<<stage_grid(ctx, n), STAGE_T, 0, ctx->stream>>>(d_in, n, key.as<uint64_t>(),
                                                              idx.as<uint32_t>());
  ++ctx->launches;
  if (cudaGetLastError() != cudaSuccess) {
    set_error("traceback job order launch failed");
    return DSA_ERR_CUDA;
  }
  uint64_t* kk = key.as<uint64_t>();
  uint32_t* vv = idx.as<uint32_t>();
  // thread-path jobs have at most 4096 rows
  DSA_TRY(launch_pair_sort(ctx, kk, vv, key2.as<uint64_t>(), idx2.as<uint32_t>(), n, 4096u,
                           (uint32_t)TB_ORDER_WC_CAP));
  k_tb_gather<<<stage_grid(ctx, n), STAGE_T, 0, ctx->stream>>>(d_in, vv, n, d_out);
  ++ctx->launches;
  if (cudaGetLastError() != cudaSuccess) {
    set_error("traceback job order launch failed");
    return DSA_ERR_CUDA;
  }
  return DSA_OK;
}

// CIGAR offsets of the jobs' hits from a device scan of their lengths: hit of
// job x gets *d_base + (words of jobs before x); *d_base grows by the total.
int launch_cigar_offsets_scan(dsa_ctx* ctx, dsa_hit* d_hits, const TbJob* d_jobs, uint64_t n,
                              uint64_t* d_base) {
  if (n == 0) return DSA_OK;
  void* p = nullptr;
  DSA_TRY(ctx->alloc(&p, (n + 1) * sizeof(uint64_t)));
  uint64_t* lens = static_cast<uint64_t*>(p);
  uint64_t* total = lens + n;
  int rc = DSA_OK;
  k_cig_lens<<<stage_grid(ctx, n), STAGE_T, 0, ctx->stream>>>(d_hits, d_jobs, n, lens);
  ++ctx->launches;
  if (cudaGetLastError() != cudaSuccess) rc = DSA_ERR_CUDA;
  if (rc == DSA_OK) rc = launch_scan_u64(ctx, lens, n, total);
  if (rc == DSA_OK) {
    k_cig_place<<<stage_grid(ctx, n), STAGE_T, 0, ctx->stream>>>(d_hits, d_jobs, n, lens, d_base);
    k_add_u64<<<1, 32, 0, ctx->stream>>>(d_base, total);
    ctx->launches += 2;
    if (cudaGetLastError() != cudaSuccess) rc = DSA_ERR_CUDA;
  }
  if (rc == DSA_ERR_CUDA) set_error("cigar offset launch failed");
  ctx->release(p, (n + 1) * sizeof(uint64_t));
  return rc;
}

}  // namespace dsa
