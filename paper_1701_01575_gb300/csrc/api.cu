// Host side of the libdsa C ABI (the per-core alignment of the map phase,
// Sec. II.B.1, with its three algorithms, Sec. II.C.2, and the top K of
// Sec. II.B.2): contexts, device-resident sequence sets,
// planning of the score pass (packed inter-sequence kernel, long-target
// wavefront kernel, exact int32 kernel), saturation reruns, top-k and
// traceback orchestration.  Every arithmetic step runs in the kernels of the
// other translation units.
#include "dsa_internal.cuh"

#include <algorithm>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <unistd.h>
#include <sys/stat.h>
#include <map>
#include <thread>

namespace dsa {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

namespace {

// Host threads for a loop of n items, at least `per` items each (1 .. 16).
unsigned host_threads(size_t n, size_t per) {
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  return (unsigned)std::max<size_t>(1, std::min<size_t>(hw, n / std::max<size_t>(per, 1)));
}

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

// Stable ascending order of 64-bit keys: identity when they already are in
// order, else an LSD radix sort on 11-bit digits (digits shared by every key
// are skipped); each pass counts per host thread, then scatters in parallel
// (thread t's items of a digit follow those of threads < t: stable).
std::vector<uint32_t> radix_order(const std::vector<uint64_t>& key) {
  const size_t n = key.size();
  std::vector<uint32_t> idx(n);
  std::iota(idx.begin(), idx.end(), 0u);
  if (std::is_sorted(key.begin(), key.end())) return idx;
  uint64_t all_or = 0, all_and = ~0ull;
  for (uint64_t k : key) { all_or |= k; all_and &= k; }
  const uint64_t varying = all_or ^ all_and;
  const unsigned T = host_threads(n, 1u << 16);
  constexpr size_t B = 2048;
  std::vector<uint32_t> tmp(n);
  std::vector<uint64_t> cur(n), nxt(n);   // keys in the current order
  for (size_t x = 0; x < n; ++x) cur[x] = key[x];
  std::vector<size_t> cnt((size_t)T * B);
  for (int shift = 0; shift < 64; shift += 11) {
    if (((varying >> shift) & 0x7FFull) == 0) continue;
    std::fill(cnt.begin(), cnt.end(), 0);
    parallel_for(n, T, [&](unsigned t, size_t b, size_t e) {
      size_t* c = cnt.data() + (size_t)t * B;
      for (size_t x = b; x < e; ++x) ++c[(cur[x] >> shift) & 0x7FF];
    });
    size_t run = 0;   // exclusive offsets in (digit, thread) order
    for (size_t d = 0; d < B; ++d)
      for (unsigned t = 0; t < T; ++t) {
        const size_t c = cnt[(size_t)t * B + d];
        cnt[(size_t)t * B + d] = run;
        run += c;
      }
    parallel_for(n, T, [&](unsigned t, size_t b, size_t e) {
      size_t* c = cnt.data() + (size_t)t * B;
      for (size_t x = b; x < e; ++x) {
        const size_t dst = c[(cur[x] >> shift) & 0x7FF]++;
        tmp[dst] = idx[x];
        nxt[dst] = cur[x];
      }
    });
    idx.swap(tmp);
    cur.swap(nxt);
  }
  return idx;
}


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

int set_device(dsa_ctx* ctx) {
  DSA_CUDA_TRY(cudaSetDevice(ctx->device));
  return DSA_OK;
}

// Pairs whose packed pass saturated: indices gathered on the device.
__global__ void k_collect_flags(const uint8_t* __restrict__ flag, uint64_t n,
                                uint32_t* __restrict__ list, uint32_t cap,
                                uint32_t* __restrict__ count) {
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    if (flag[x]) {
      const uint32_t k = atomicAdd(count, 1u);
      if (k < cap) list[k] = (uint32_t)x;
    }
  }
}

struct Validated {
  int smax = 0, smin = 0;
  uint32_t max_m = 0, max_n = 0;
};

int check_matrix(const int8_t* matrix, int A, int o, int e, Validated* v) {
  if (!matrix) { set_error("matrix is NULL"); return DSA_ERR_INVALID_ARG; }
  if (o < 0 || e < 0 || e > o) {
    set_error("gap penalties must satisfy 0 <= gap_extend <= gap_open (got %d, %d)", o, e);
    return DSA_ERR_INVALID_ARG;
  }
  int smax = -128, smin = 127;
  for (int k = 0; k < A * A; ++k) {
    smax = std::max<int>(smax, matrix[k]);
    smin = std::min<int>(smin, matrix[k]);
  }
  v->smax = smax;
  v->smin = smin;
  return DSA_OK;
}

// Band items (pair, band) of a band-pipelined score pass, in latest-start
// order.  Band b of a pair trails its predecessor, so it can start about
// b * LAG steps after the pair's first band, and the pair needs about
// n + bands * LAG steps in all; sorting the items by b * LAG - (n + bands *
// LAG) starts the longest chains first without parking warps on bands that
// are far behind their predecessors.  Inside a pair the key grows with b, so
// a band's predecessor is always taken earlier (the bounded waits rely on
// that: a warp waits only on a band some running warp holds).
std::vector<uint32_t> band_items(const std::vector<std::pair<uint32_t, uint32_t>>& mn, int band) {
  constexpr int64_t LAG = 128;
  struct It { int64_t key; uint32_t p, b; };
  std::vector<It> its;
  for (uint32_t p = 0; p < mn.size(); ++p) {
    const uint32_t nb = (mn[p].first + band - 1) / band;
    const int64_t cp = (int64_t)mn[p].second + (int64_t)nb * LAG;
    for (uint32_t b = 0; b < nb; ++b) its.push_back({(int64_t)b * LAG - cp, p, b});
  }
  std::stable_sort(its.begin(), its.end(), [](const It& x, const It& y) { return x.key < y.key; });
  std::vector<uint32_t> items;
  items.reserve(2 * its.size());
  for (const It& it : its) { items.push_back(it.p); items.push_back(it.b); }
  return items;
}

// Every S + o of the matrix fits int8 (the byte-permute substitution tables).
bool s_plus_o_fits_int8(const int8_t* matrix, int A, int o) {
  for (int x = 0; x < A * A; ++x)
    if (matrix[x] + o < -128 || matrix[x] + o > 127) return false;
  return true;
}

// Position-specific profile: the value range of its `n` entries.
int check_pssm(const int8_t* pssm, uint64_t n, int o, int e, Validated* v) {
  if (!pssm) { set_error("pssm is NULL"); return DSA_ERR_INVALID_ARG; }
  if (o < 0 || e < 0 || e > o) {
    set_error("gap penalties must satisfy 0 <= gap_extend <= gap_open (got %d, %d)", o, e);
    return DSA_ERR_INVALID_ARG;
  }
  int smax = -128, smin = 127;
  for (uint64_t k = 0; k < n; ++k) {
    smax = std::max<int>(smax, pssm[k]);
    smin = std::min<int>(smin, pssm[k]);
  }
  v->smax = smax;
  v->smin = smin;
  return DSA_OK;
}

}  // namespace

void phase_begin(dsa_res* res, Phase p, cudaStream_t on) {
  if (!res || !(res->flags & DSA_TIMING)) return;
  if (!res->ev[2 * p]) {
    cudaEventCreate(&res->ev[2 * p]);
    cudaEventCreate(&res->ev[2 * p + 1]);
  }
  if (!res->used[p]) cudaEventRecord(res->ev[2 * p], on ? on : res->ctx->stream);
}

void phase_end(dsa_res* res, Phase p, cudaStream_t on) {
  if (!res || !(res->flags & DSA_TIMING) || !res->ev[2 * p + 1]) return;
  cudaEventRecord(res->ev[2 * p + 1], on ? on : res->ctx->stream);
  res->used[p] = true;
}

}  // namespace dsa

using namespace dsa;

// ---------------------------------------------------------------- context --

int dsa_ctx::alloc(void** p, size_t bytes, cudaStream_t on) {
  *p = nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (budget && in_use + bytes > budget) {
    set_error("request of %zu bytes exceeds the memory budget (%zu of %zu in use)", bytes, in_use,
              budget);
    return DSA_ERR_OVER_BUDGET;
  }
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, on ? on : stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return DSA_ERR_OOM;
  }
  in_use += bytes;
  return DSA_OK;
}

void dsa_ctx::release(void* p, size_t bytes, cudaStream_t on) {
  if (!p) return;
  cudaFreeAsync(p, on ? on : stream);
  std::lock_guard<std::mutex> lk(mu);
  in_use -= bytes;
}

extern "C" const char* dsa_last_error(void) { return g_err.c_str(); }

extern "C" int dsa_create(dsa_ctx** out, int device, size_t mem_budget_bytes, void* cuda_stream) {
  if (!out) { set_error("out is NULL"); return DSA_ERR_INVALID_ARG; }
  *out = nullptr;
  int n_dev = 0;
  DSA_CUDA_TRY(cudaGetDeviceCount(&n_dev));
  if (device < 0 || device >= n_dev) {
    set_error("device %d out of range (%d devices)", device, n_dev);
    return DSA_ERR_INVALID_ARG;
  }
  DSA_CUDA_TRY(cudaSetDevice(device));
  int major = 0, minor = 0;
  DSA_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device));
  DSA_CUDA_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device));
  if (major != 10 || minor != 3) {
    set_error("libdsa is built for sm_103a; device %d is sm_%d%d", device, major, minor);
    return DSA_ERR_UNSUPPORTED;
  }
  dsa_ctx* c = new (std::nothrow) dsa_ctx;
  if (!c) { set_error("host allocation failed"); return DSA_ERR_OOM; }
  c->device = device;
  c->budget = mem_budget_bytes;
  cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      set_error("cudaStreamCreate failed");
      return DSA_ERR_CUDA;
    }
    c->own_stream = true;
  }
  {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    uint64_t keep = mem_budget_bytes ? (uint64_t)mem_budget_bytes : UINT64_MAX;
    if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess ||
        cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
      cudaGetLastError();
      if (c->pool) cudaMemPoolDestroy(c->pool);
      if (c->own_stream) cudaStreamDestroy(c->stream);
      delete c;
      set_error("memory pool creation failed");
      return DSA_ERR_CUDA;
    }
  }
  if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(&c->d_status, 256) != cudaSuccess || cudaMalloc(&c->d_counters, 256) != cudaSuccess ||
      cudaMemset(c->d_status, 0, 256) != cudaSuccess || cudaMemset(c->d_counters, 0, 256) != cudaSuccess) {
    cudaGetLastError();
    if (c->d_status) cudaFree(c->d_status);
    if (c->d_counters) cudaFree(c->d_counters);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    cudaMemPoolDestroy(c->pool);
    delete c;
    set_error("context allocation failed");
    return DSA_ERR_OOM;
  }
  *out = c;
  return DSA_OK;
}

extern "C" int dsa_destroy(dsa_ctx* ctx) {
  if (!ctx) return DSA_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaStreamSynchronize(ctx->side);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_counters);
  cudaEventDestroy(ctx->fork_ev);
  cudaEventDestroy(ctx->join_ev);
  cudaStreamDestroy(ctx->side);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  // allocations still outstanding (none when every db / result was freed
  // first) keep the pool alive until they are freed
  cudaMemPoolDestroy(ctx->pool);
  delete ctx;
  return DSA_OK;
}

extern "C" size_t dsa_mem_in_use(const dsa_ctx* ctx) { return ctx ? ctx->in_use : 0; }

extern "C" uint64_t dsa_kernel_launches(const dsa_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" int dsa_sync(dsa_ctx* ctx) {
  if (!ctx) { set_error("ctx is NULL"); return DSA_ERR_INVALID_ARG; }
  DSA_TRY(set_device(ctx));
  DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  int32_t st = 0;
  DSA_CUDA_TRY(cudaMemcpy(&st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st != 0) {
    DSA_CUDA_TRY(cudaMemset(ctx->d_status, 0, sizeof(st)));
    set_error("a kernel reported device status %d", st);
    return st;
  }
  return DSA_OK;
}

// ---------------------------------------------------------------- databases --

static void db_release(dsa_db* db) {
  dsa_ctx* c = db->ctx;
  auto rel = [&](void* p, size_t n) { if (p) c->release(p, n); };
  rel(db->d_codes, db->n_res + 64);
  rel(db->d_off, (db->n + 1) * sizeof(uint64_t));
  rel(db->d_len, db->n * sizeof(uint32_t));
  // the interleaved copy, when an all-vs-all search built it
  rel(db->d_perm, db->n * sizeof(uint32_t));
  rel(db->d_slen, db->n * sizeof(uint32_t));
  rel(db->d_gbase, db->n_groups * sizeof(uint64_t));
  rel(db->d_glen, db->n_groups * sizeof(uint32_t));
  rel(db->d_il, db->il_bytes ? db->il_bytes : 16);
}

extern "C" int dsa_db_load(dsa_ctx* ctx, const uint8_t* codes, const uint64_t* offsets,
                           uint32_t n_seqs, int alphabet_size, dsa_db** out) {
  if (!ctx || !out || !offsets || n_seqs == 0) {
    set_error("dsa_db_load: NULL argument or empty set");
    return DSA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (alphabet_size < 1 || alphabet_size > MAX_ALPHABET) {
    set_error("alphabet_size %d outside 1..%d", alphabet_size, MAX_ALPHABET);
    return DSA_ERR_INVALID_ARG;
  }
  DSA_TRY(set_device(ctx));
  const uint64_t base = offsets[0];
  std::vector<uint64_t> off(n_seqs + 1);
  std::vector<uint32_t> len(n_seqs);
  for (uint32_t k = 0; k < n_seqs; ++k) {
    if (offsets[k + 1] <= offsets[k]) {
      set_error("sequence %u is empty or offsets decrease", k);
      return DSA_ERR_INVALID_ARG;
    }
    const uint64_t L = offsets[k + 1] - offsets[k];
    if (L > (1ull << 30)) { set_error("sequence %u longer than 2^30", k); return DSA_ERR_INVALID_ARG; }
    off[k] = offsets[k] - base;
    len[k] = (uint32_t)L;
  }
  off[n_seqs] = offsets[n_seqs] - base;
  const uint64_t n_res = off[n_seqs];
  if (!codes) { set_error("codes is NULL"); return DSA_ERR_INVALID_ARG; }
  const uint8_t* src = codes + base;
  {
    // every code below the alphabet size (host threads; first offender reported)
    const unsigned T = host_threads(n_res, 1u << 20);
    std::vector<uint64_t> bad(T, UINT64_MAX);
    parallel_for(n_res, T, [&](unsigned t, size_t b, size_t e) {
      for (size_t x = b; x < e; ++x)
        if (src[x] >= (uint8_t)alphabet_size) {
          bad[t] = x;
          return;
        }
    });
    for (unsigned t = 0; t < T; ++t)
      if (bad[t] != UINT64_MAX) {
        set_error("residue code %u at position %llu is not below alphabet_size %d", src[bad[t]],
                  (unsigned long long)bad[t], alphabet_size);
        return DSA_ERR_INVALID_ARG;
      }
  }
  dsa_db* db = new (std::nothrow) dsa_db;
  if (!db) { set_error("host allocation failed"); return DSA_ERR_OOM; }
  db->ctx = ctx;
  db->n = n_seqs;
  db->n_res = n_res;
  db->A = alphabet_size;
  db->h_off = off;
  db->h_len = len;
  for (uint32_t L : len) db->max_len = std::max(db->max_len, L);
  db->n_groups = (n_seqs + GROUP - 1) / GROUP;

  int rc = DSA_OK;
  auto fail = [&](int r) { db_release(db); delete db; return r; };
  void* p;
  if ((rc = ctx->alloc(&p, n_res + 64))) return fail(rc);
  db->d_codes = (uint8_t*)p;
  if ((rc = ctx->alloc(&p, (n_seqs + 1) * sizeof(uint64_t)))) return fail(rc);
  db->d_off = (uint64_t*)p;
  if ((rc = ctx->alloc(&p, n_seqs * sizeof(uint32_t)))) return fail(rc);
  db->d_len = (uint32_t*)p;

  cudaStream_t s = ctx->stream;
  if (cudaMemcpyAsync(db->d_codes, src, n_res, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(db->d_codes + n_res, 0, 64, s) != cudaSuccess ||
      cudaMemcpyAsync(db->d_off, off.data(), off.size() * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(db->d_len, len.data(), len.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    set_error("dsa_db_load: copy to device failed: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(DSA_ERR_CUDA);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    set_error("dsa_db_load: %s", cudaGetErrorString(cudaGetLastError()));
    return fail(DSA_ERR_CUDA);
  }
  *out = db;
  return DSA_OK;
}

namespace dsa {

int ensure_interleaved(dsa_ctx* ctx, const dsa_db* cdb) {
  dsa_db* db = const_cast<dsa_db*>(cdb);
  std::lock_guard<std::mutex> lk(db->il_mu);
  if (db->il_ready) return DSA_OK;
  const uint32_t n_seqs = db->n;
  // length-sorted order: longest first, ties by id
  std::vector<uint32_t> perm(n_seqs);
  {
    std::vector<uint64_t> key(n_seqs);
    for (uint32_t k = 0; k < n_seqs; ++k) key[k] = ~(uint64_t)db->h_len[k] << 32 | k;
    const std::vector<uint32_t> ord = radix_order(key);
    for (uint32_t k = 0; k < n_seqs; ++k) perm[k] = ord[k];
  }
  std::vector<uint32_t> slen(n_seqs);
  for (uint32_t k = 0; k < n_seqs; ++k) slen[k] = db->h_len[perm[k]];
  std::vector<uint32_t> glen(db->n_groups);
  std::vector<uint64_t> gbase(db->n_groups);
  uint64_t il = 0;
  for (uint32_t g = 0; g < db->n_groups; ++g) {
    glen[g] = slen[(size_t)g * GROUP];
    gbase[g] = il;
    il += (uint64_t)((glen[g] + CHUNK - 1) / CHUNK) * CHUNK * GROUP;
  }
  // device arrays come from the owner's pool, ordered on the caller's stream
  dsa_ctx* own = db->ctx;
  cudaStream_t s = ctx->stream;
  void* p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  const size_t sz[5] = {n_seqs * sizeof(uint32_t), n_seqs * sizeof(uint32_t),
                        db->n_groups * sizeof(uint64_t), db->n_groups * sizeof(uint32_t),
                        il ? il : 16};
  for (int k = 0; k < 5; ++k) {
    int rc = own->alloc(&p[k], sz[k], s);
    if (rc) {
      for (int x = 0; x < k; ++x) own->release(p[x], sz[x], s);
      return rc;
    }
  }
  db->d_perm = (uint32_t*)p[0];
  db->d_slen = (uint32_t*)p[1];
  db->d_gbase = (uint64_t*)p[2];
  db->d_glen = (uint32_t*)p[3];
  db->d_il = (uint8_t*)p[4];
  db->il_bytes = il;
  db->h_perm.swap(perm);
  db->h_glen.swap(glen);
  db->h_gbase.swap(gbase);
  if (cudaMemcpyAsync(db->d_perm, db->h_perm.data(), n_seqs * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(db->d_slen, slen.data(), n_seqs * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(db->d_gbase, db->h_gbase.data(), db->n_groups * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(db->d_glen, db->h_glen.data(), db->n_groups * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    set_error("interleave: copy to device failed: %s", cudaGetErrorString(cudaGetLastError()));
    return DSA_ERR_CUDA;
  }
  DSA_TRY(launch_interleave(ctx, db));
  DSA_CUDA_TRY(cudaStreamSynchronize(s));   // usable from any stream from here on
  db->il_ready = true;
  return DSA_OK;
}

}  // namespace dsa

extern "C" int dsa_db_free(dsa_db* db) {
  if (!db) return DSA_OK;
  cudaSetDevice(db->ctx->device);
  db_release(db);
  delete db;
  return DSA_OK;
}

extern "C" int dsa_db_info(const dsa_db* db, uint32_t* n_seqs, uint64_t* n_residues,
                           int* alphabet_size) {
  if (!db) { set_error("db is NULL"); return DSA_ERR_INVALID_ARG; }
  if (n_seqs) *n_seqs = db->n;
  if (n_residues) *n_residues = db->n_res;
  if (alphabet_size) *alphabet_size = db->A;
  return DSA_OK;
}

// ---------------------------------------------------------------- align --

namespace {

// ---- autotuner: the long-target threshold of the packed path ----
//
// Which targets go to the wavefront kernel (long) and which to the
// inter-sequence kernel is a speed choice only (both are exact).  For a
// workload shape (GPU, alphabet, and log2 bins of the query count, query
// residues, target count, database residues and longest target) the first
// call times a small local search of thresholds -- starting at 4096, then
// lower or higher by factors of 4 while it keeps improving by 3% or more --
// and keeps the best in a JSON cache file.  DSA_AUTOTUNE=off (fixed 4096) | cache (default:
// tune on a miss) | retune (always tune); DSA_AUTOTUNE_CACHE names the file
// (default $XDG_CACHE_HOME/dsa/autotune.json or ~/.cache/dsa/autotune.json);
// DSA_LONG_THRESHOLD overrides everything.
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

// Packed score pass (local, int16x2): targets of groups longer than
// `long_thr` go to the wavefront kernel on the side stream, the rest to the
// inter-sequence kernel.  The results do not depend on long_thr, only the time.
int packed_score(dsa_ctx* ctx, dsa_res* res, const dsa_db* db, const dsa_db* qs,
                 const int8_t* d_mat, const int8_t* d_pssm, int A, int o, int e, const Validated& v, Scores out,
                 uint32_t long_thr) {
  const uint32_t nq = qs->n, nt = db->n;
  const int R = A + 1;
  std::vector<uint32_t> qorder(nq);
  std::iota(qorder.begin(), qorder.end(), 0u);
  std::stable_sort(qorder.begin(), qorder.end(),
                   [&](uint32_t a, uint32_t b) { return qs->h_len[a] > qs->h_len[b]; });
  auto strips_of = [&](uint32_t q) { return (qs->h_len[q] + INTER_ROWS - 1) / INTER_ROWS; };

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
  spl.rows = INTER_ROWS;
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
  DSA_TRY(launch_strip_profile(ctx, qs, d_mat, d_pssm, A, o, spl));
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
    DSA_TRY(launch_strip_profile(ctx, qs, d_mat, d_pssm, A, o, ppl));
    // long targets on the side stream, overlapping the inter-sequence kernel:
    // the two kernels write disjoint targets' results
    DSA_CUDA_TRY(cudaEventRecord(ctx->fork_ev, ctx->stream));
    DSA_CUDA_TRY(cudaStreamWaitEvent(ctx->side, ctx->fork_ev, 0));
    phase_begin(res, PH_INTRA, ctx->side);
    DSA_TRY(launch_intra_local16(ctx, ctx->side, db, ppl, xw, o, e, v.smax, out, nt));
    phase_end(res, PH_INTRA, ctx->side);
    DSA_CUDA_TRY(cudaEventRecord(ctx->join_ev, ctx->side));
  }
  phase_begin(res, PH_INTER);
  DSA_TRY(launch_inter_local16(ctx, db, spl, iw, o, e, v.smax, out, nt));
  phase_end(res, PH_INTER);
  if (n_long) DSA_CUDA_TRY(cudaStreamWaitEvent(ctx->stream, ctx->join_ev, 0));
  return DSA_OK;
}

// The packed pass with the autotuned long-target threshold.
int run_packed_tuned(dsa_ctx* ctx, dsa_res* res, const dsa_db* db, const dsa_db* qs,
                     const int8_t* d_mat, const int8_t* d_pssm, int A, int o, int e, const Validated& v, Scores out) {
  if (const char* env = getenv("DSA_LONG_THRESHOLD"))
    return packed_score(ctx, res, db, qs, d_mat, d_pssm, A, o, e, v, out,
                        (uint32_t)strtoul(env, nullptr, 10));
  const char* mode_env = getenv("DSA_AUTOTUNE");
  const std::string mode = mode_env ? mode_env : "cache";
  constexpr uint32_t DEFAULT_THR = 4096;
  if (mode == "off") return packed_score(ctx, res, db, qs, d_mat, d_pssm, A, o, e, v, out, DEFAULT_THR);
  // workload shape key
  uint64_t qres = 0;
  for (uint32_t x : qs->h_len) qres += x;
  cudaDeviceProp prop;
  DSA_CUDA_TRY(cudaGetDeviceProperties(&prop, ctx->device));
  int drv = 0;
  cudaDriverGetVersion(&drv);
  char key[512];
  snprintf(key, sizeof key, "%s|sm%d|drv%d|A%d|q%d|qr%d|t%d|tr%d|L%d", prop.name, ctx->sm_count,
           drv, A, ilog2_bin(qs->n), ilog2_bin(qres), ilog2_bin(db->n), ilog2_bin(db->n_res),
           ilog2_bin(db->max_len));
  Tuner& t = tuner();
  {
    std::lock_guard<std::mutex> lk(t.mu);
    const std::string path = tune_cache_path();
    if (!t.loaded || path != t.path) tune_load(t, path);   // first use, or another file
    auto it = t.cache.find(key);
    if (mode != "retune" && it != t.cache.end())
      return packed_score(ctx, res, db, qs, d_mat, d_pssm, A, o, e, v, out, it->second);
  }
  if (!ctx->tune)   // contexts that must not spend calls on tuning (serving workers)
    return packed_score(ctx, res, db, qs, d_mat, d_pssm, A, o, e, v, out, DEFAULT_THR);
  // thresholds are compared by the number of target groups they move
  auto groups_over = [&](uint32_t thr) {
    uint32_t g = 0;
    while (g < db->n_groups && db->h_glen[g] > thr) ++g;
    return g;
  };
  std::map<uint32_t, double> timed;   // long groups -> ms
  cudaEvent_t ev0, ev1;
  DSA_CUDA_TRY(cudaEventCreate(&ev0));
  DSA_CUDA_TRY(cudaEventCreate(&ev1));
  int rc = DSA_OK;
  auto measure = [&](uint32_t thr) -> double {
    const uint32_t g = groups_over(thr);
    auto it = timed.find(g);
    if (it != timed.end()) return it->second;
    float ms = 0.f;
    if (rc == DSA_OK && cudaEventRecord(ev0, ctx->stream) != cudaSuccess) rc = DSA_ERR_CUDA;
    if (rc == DSA_OK) rc = packed_score(ctx, nullptr, db, qs, d_mat, d_pssm, A, o, e, v, out, thr);
    if (rc == DSA_OK && cudaEventRecord(ev1, ctx->stream) != cudaSuccess) rc = DSA_ERR_CUDA;
    if (rc == DSA_OK && cudaEventSynchronize(ev1) != cudaSuccess) rc = DSA_ERR_CUDA;
    if (rc == DSA_OK) cudaEventElapsedTime(&ms, ev0, ev1);
    timed[g] = ms;
    return ms;
  };
  // local search from the default by factors of 4, in each direction while it
  // improves; thresholds that move the same groups as the last one are
  // skipped, and a switch needs a gain of at least 3% (single timings)
  uint32_t best = DEFAULT_THR;
  double best_ms = measure(best);
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
      const double ms = measure(thr);
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
    t.cache[key] = best;
    tune_store(t);
  }
  // the final pass with the chosen threshold records the phase timings and cells
  return packed_score(ctx, res, db, qs, d_mat, d_pssm, A, o, e, v, out, best);
}

// Score pass for all queries x all targets.
int score_all_vs_all(dsa_ctx* ctx, dsa_res* res, const dsa_db* db, const dsa_db* qs, int mode,
                     uint32_t fe, const int8_t* d_mat, const int8_t* d_pssm, int A, int o, int e, const Validated& v,
                     uint32_t flags, Scores out, uint64_t* n_rerun) {
  const uint32_t nq = qs->n, nt = db->n;
  const bool packed = mode == DSA_LOCAL && !(flags & (DSA_FORCE_INT32 | DSA_PLAIN_FORM)) &&
                      o >= 1 && o + e <= 4096 && v.smax + o < 8192 && v.smin > -8192;
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
  DSA_TRY(run_packed_tuned(ctx, res, db, qs, d_mat, d_pssm, A, o, e, v, out));

  // ---- exact int32 rerun of saturated pairs ----
  const uint64_t n_out = (uint64_t)nq * nt;
  const uint32_t cap = (uint32_t)std::min<uint64_t>(n_out, 1u << 22);
  DevBuf d_list;
  DSA_TRY(d_list.alloc(ctx, (size_t)cap * sizeof(uint32_t)));
  uint32_t* d_count = ctx->d_counters + 1;
  DSA_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(uint32_t), ctx->stream));
  {
    uint64_t blk = std::min<uint64_t>((n_out + 255) / 256, (uint64_t)ctx->sm_count * 16);
    k_collect_flags<<<(unsigned)blk, 256, 0, ctx->stream>>>(out.flag, n_out, d_list.as<uint32_t>(),
                                                             cap, d_count);
    DSA_CUDA_TRY(cudaGetLastError());
    ++ctx->launches;
  }
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

// pssm (host, optional): position-specific rows, one per query residue of
// the set (qs->n_res x A), used instead of `matrix` by an all-vs-all search.
int align_impl(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const dsa_pair* pairs,
               uint64_t n_pairs, int mode, uint32_t fe, const int8_t* matrix, int A, int o, int e,
               uint32_t top_k, uint32_t flags, dsa_res** out, const int8_t* pssm = nullptr) {
  if (!ctx || !db || !qs || !out) { set_error("NULL argument"); return DSA_ERR_INVALID_ARG; }
  *out = nullptr;
  if (mode < DSA_LOCAL || mode > DSA_SEMIGLOBAL) { set_error("bad mode %d", mode); return DSA_ERR_INVALID_ARG; }
  if (fe > 15) { set_error("bad free_ends %u", fe); return DSA_ERR_INVALID_ARG; }
  if (A != db->A || A != qs->A) {
    set_error("alphabet_size %d does not match the sequence sets (%d, %d)", A, db->A, qs->A);
    return DSA_ERR_INVALID_ARG;
  }
  Validated v;
  if (pssm) {
    if (pairs) {
      set_error("position-specific profiles apply to all-vs-all searches only");
      return DSA_ERR_UNSUPPORTED;
    }
    DSA_TRY(check_pssm(pssm, qs->n_res * (uint64_t)A, o, e, &v));
  } else {
    DSA_TRY(check_matrix(matrix, A, o, e, &v));
  }
  DSA_TRY(set_device(ctx));
  const bool all = pairs == nullptr;
  if (!all && top_k) {
    set_error("top_k applies to all-vs-all searches only");
    return DSA_ERR_UNSUPPORTED;
  }
  // int16 eligibility: local with the saturation flag, or any mode whose
  // scores provably stay inside int16: (m + n) * w + o well below 2^14
  const int64_t w16 = std::max<int64_t>({(int64_t)std::abs(v.smax), (int64_t)std::abs(v.smin), o, e});
  const bool local16 = mode == DSA_LOCAL && o >= 1 && o + e <= 4096 && v.smax + o < 8192 && v.smin > -8192;
  const bool packed_ok = !(flags & (DSA_FORCE_INT32 | DSA_PLAIN_FORM));
  // explicit pairs: a device copy (the caller's own when they are on the
  // device), checked and classified there; the host sees only the totals
  DevBuf d_pairs_buf, d_key, d_idx, d_hist, d_jcnt, d_stats;
  const dsa_pair* d_pairs = nullptr;
  PairPlanStats pst{};
  const uint64_t L = (uint64_t)qs->max_len + 2;
  if (!all) {
    if (flags & DSA_PAIRS_ON_DEVICE) {
      d_pairs = pairs;
    } else {
      DSA_TRY(upload(ctx, d_pairs_buf, pairs, n_pairs));
      d_pairs = d_pairs_buf.as<dsa_pair>();
    }
    DSA_TRY(d_key.alloc(ctx, n_pairs * sizeof(uint64_t)));
    DSA_TRY(d_idx.alloc(ctx, n_pairs * sizeof(uint32_t)));
    DSA_TRY(d_hist.alloc(ctx, L * sizeof(uint64_t)));
    DSA_TRY(d_jcnt.alloc(ctx, L * sizeof(uint64_t)));
    DSA_TRY(d_stats.alloc(ctx, sizeof(PairPlanStats)));
    PairPlanStats* st = d_stats.as<PairPlanStats>();
    DSA_CUDA_TRY(cudaMemsetAsync(d_hist.p, 0, L * sizeof(uint64_t), ctx->stream));
    DSA_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(PairPlanStats), ctx->stream));
    DSA_CUDA_TRY(cudaMemsetAsync(&st->first_bad, 0xFF, sizeof(uint64_t), ctx->stream));
    const PairPlanParams P{qs->n, db->n, w16, o, e, local16, packed_ok};
    DSA_TRY(launch_pair_classify(ctx, d_pairs, n_pairs, qs, db, P, d_key.as<uint64_t>(),
                                 d_idx.as<uint32_t>(), d_hist.as<uint64_t>(), L,
                                 d_jcnt.as<uint64_t>(), st));
    DSA_CUDA_TRY(cudaMemcpyAsync(&pst, st, sizeof pst, cudaMemcpyDeviceToHost, ctx->stream));
    DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    if (pst.first_bad != UINT64_MAX) {
      set_error("pair %llu is out of range", (unsigned long long)pst.first_bad);
      return DSA_ERR_INVALID_ARG;
    }
  }
  // host copy of the pairs, made only when the host planner needs it
  std::vector<dsa_pair> hp;
  bool hp_ready = all;
  auto need_hp = [&]() -> int {
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
  };
  // int32 range: (m + n) * max|value step| must stay far from 2^31
  const uint32_t max_m = qs->max_len;
  const uint32_t max_n = all ? db->max_len : pst.max_t_len;
  if (((int64_t)max_m + max_n + 2) * (w16 + 1) >= (1ll << 29)) {
    set_error("scores could leave the int32 range (lengths %u + %u, weight %lld)", max_m, max_n,
              (long long)w16);
    return DSA_ERR_UNSUPPORTED;
  }

  dsa_res* res = new (std::nothrow) dsa_res;
  if (!res) { set_error("host allocation failed"); return DSA_ERR_OOM; }
  res->ctx = ctx; res->db = db; res->queries = qs; res->mode = mode; res->free_ends = fe;
  res->A = A; res->gap_open = o; res->gap_extend = e;
  if (matrix) res->matrix.assign(matrix, matrix + A * A);
  res->pssm = pssm != nullptr;
  res->flags = flags;
  auto fail = [&](int rc) {
    if (res->d_hits) ctx->release(res->d_hits, std::max<uint64_t>(1, res->n_hits) * sizeof(dsa_hit));
    if (res->d_bnd) ctx->release(res->d_bnd, res->bnd_bytes);
    delete res;
    return rc;
  };

  DevBuf d_mat, d_pssm;
  if (matrix) {
    if (int rc = d_mat.alloc(ctx, A * A)) return fail(rc);
    if (cudaMemcpyAsync(d_mat.p, matrix, A * A, cudaMemcpyHostToDevice, ctx->stream) != cudaSuccess) {
      set_error("matrix upload failed");
      return fail(DSA_ERR_CUDA);
    }
  }
  if (pssm) {
    if (int rc = upload(ctx, d_pssm, pssm, qs->n_res * (uint64_t)A)) return fail(rc);
  }

  const uint64_t n_out = all ? (uint64_t)qs->n * db->n : n_pairs;
  DevBuf s_score, s_qend, s_tend, s_flag;
  int rc;
  if ((rc = s_score.alloc(ctx, n_out * 4)) || (rc = s_qend.alloc(ctx, n_out * 4)) ||
      (rc = s_tend.alloc(ctx, n_out * 4)) || (rc = s_flag.alloc(ctx, n_out)))
    return fail(rc);
  Scores sc{s_score.as<int32_t>(), s_qend.as<int32_t>(), s_tend.as<int32_t>(), s_flag.as<uint8_t>()};

  if (all) {
    uint64_t sq = 0;
    for (uint32_t x : qs->h_len) sq += x;
    res->cells = sq * db->n_res;
    if ((rc = score_all_vs_all(ctx, res, db, qs, mode, fe, d_mat.as<int8_t>(), d_pssm.as<int8_t>(),
                               A, o, e, v, flags,
                               sc, &res->n_rerun)))
      return fail(rc);
  } else {
    std::vector<PairJob> jobs;
    std::vector<LongJob> ljobs;
    std::vector<uint64_t> p16;   // pairs for the packed int16 kernel
    uint64_t scr = 0, cells = 0, lcells = 0, p16cells = 0;
    uint64_t bnd = 0, prog = 0, cand = 0;
    const int band = long_band_rows(), ckpt = long_ckpt_rows();
    // every pair packed: the device planner lays out the jobs
    const bool dev_plan = n_pairs > 0 && pst.n_other == 0;
    // host planner: classify on host threads: packed pairs (filled in place,
    // pair order kept); long and int32 pairs are few and follow serially
    enum : uint8_t { C_P16, C_LONG, C_INT32 };
    std::vector<uint8_t> cls;
    if (dev_plan) {
      cells = pst.cells;
      p16cells = pst.cells16;
    } else {
      if ((rc = need_hp())) return fail(rc);
      cls.resize(n_pairs);
      const unsigned T = host_threads(n_pairs, 1u << 16);
      std::vector<uint64_t> n16(T + 1, 0), cells_t(T, 0), c16_t(T, 0);
      parallel_for(n_pairs, T, [&](unsigned t, size_t b, size_t x1) {
        uint64_t n = 0, cl = 0, c16 = 0;   // thread-local: no shared cache lines in the loop
        for (size_t k = b; k < x1; ++k) {
          const dsa_pair& p = hp[k];
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
      const dsa_pair& p = hp[k];
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
      // band items in latest-start order (bands in order inside a pair)
      std::vector<std::pair<uint32_t, uint32_t>> mn(ljobs.size());
      for (size_t k = 0; k < ljobs.size(); ++k) mn[k] = {(uint32_t)ljobs[k].m, (uint32_t)ljobs[k].n};
      const std::vector<uint32_t> items = band_items(mn, band);
      DevBuf d_ljobs, d_items, d_prog, d_cands;
      void* pb = nullptr;
      if ((rc = upload(ctx, d_ljobs, ljobs)) || (rc = upload(ctx, d_items, items)) ||
          (rc = d_prog.alloc(ctx, prog * sizeof(uint32_t))) ||
          (rc = d_cands.alloc(ctx, cand * long_cand_size())) ||
          (rc = ctx->alloc(&pb, bnd * sizeof(int2))))
        return fail(rc);
      res->d_bnd = static_cast<int2*>(pb);
      res->bnd_bytes = bnd * sizeof(int2);
      res->long_bnd_off.assign(n_pairs, UINT64_MAX);
      res->long_n.assign(n_pairs, 0);
      for (const LongJob& lj : ljobs) {
        res->long_bnd_off[lj.out] = lj.bnd_off;
        res->long_n[lj.out] = lj.n;
      }
      if (cudaMemsetAsync(d_prog.p, 0, prog * sizeof(uint32_t), ctx->stream) != cudaSuccess) {
        set_error("memset failed");
        return fail(DSA_ERR_CUDA);
      }
      phase_begin(res, PH_INTRA);
      if ((rc = launch_long_score(ctx, db, qs, d_mat.as<int8_t>(), A, o, e, mode, fe,
                                  s_plus_o_fits_int8(matrix, A, o), d_ljobs.as<LongJob>(), (uint32_t)ljobs.size(), d_items.as<uint32_t>(),
                                  (uint32_t)(items.size() / 2), res->d_bnd, d_prog.as<uint32_t>(),
                                  d_cands.p, sc)))
        return fail(rc);
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
            (rc = d_pj.alloc(ctx, pst.n_jobs * sizeof(Pair16Job))))
          return fail(rc);
        uint64_t* kk = d_key.as<uint64_t>();
        uint32_t* vv = d_idx.as<uint32_t>();
        if ((rc = launch_pair_sort(ctx, kk, vv, d_key2.as<uint64_t>(), d_idx2.as<uint32_t>(), n_pairs,
                                   qs->max_len, pst.max_t_len)) ||
            (rc = launch_pair_build_jobs(ctx, kk, vv, n_pairs, d_hist.as<uint64_t>(),
                                         d_jcnt.as<uint64_t>(), L, d_pairs, qs, db,
                                         d_pj.as<Pair16Job>())))
          return fail(rc);
        n_pj = (uint32_t)pst.n_jobs;
        max_n = std::max<uint32_t>(1, pst.max_t_len);
      } else {
        // order by (query length, window length); two pairs of equal query length per thread
        const unsigned T = host_threads(p16.size(), 1u << 16);
        std::vector<uint64_t> key(p16.size());
        parallel_for(p16.size(), T, [&](unsigned, size_t b, size_t x1) {
          for (size_t x = b; x < x1; ++x) {
            const dsa_pair& pp = hp[p16[x]];
            key[x] = ((uint64_t)qs->h_len[pp.query_id] << 32) | pp.t_len;
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
            const dsa_pair& a = hp[p16[x]];
            Pair16Job j{};
            j.m = (int32_t)(key[x] >> 32);
            j.q_lo = qs->h_off[a.query_id];
            j.t_lo = db->h_off[a.target_id] + a.t_offset;
            j.n_lo = (int32_t)a.t_len;
            j.out_lo = (uint32_t)p16[x];
            if (x + 1 < p16.size() && (key[x + 1] >> 32) == (key[x] >> 32)) {
              const dsa_pair& bb = hp[p16[x + 1]];
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
        if ((rc = upload(ctx, d_pj, pj))) return fail(rc);
        n_pj = (uint32_t)pj.size();
        max_n = max_n16;
      }
      bool bytes = A <= 4;   // byte-permute substitution form
      for (int x = 0; x < A * A; ++x) bytes = bytes && matrix[x] + o >= -128 && matrix[x] + o <= 127;
      phase_begin(res, PH_INTER);
      if ((rc = launch_pairs16(ctx, db, qs, d_mat.as<int8_t>(), A, o, e, mode, fe, v.smax, bytes,
                               d_pj.as<Pair16Job>(), n_pj, max_n, sc)))
        return fail(rc);
      phase_end(res, PH_INTER);
      res->phase_cells[PH_INTER] = p16cells;
      res->phase_cells[PH_INT32] -= p16cells;
      if (mode == DSA_LOCAL) {
        // exact int32 rerun of pairs whose packed pass saturated
        const uint32_t cap = (uint32_t)std::min<uint64_t>(n_pairs, 1u << 22);
        DevBuf d_list;
        if ((rc = d_list.alloc(ctx, (size_t)cap * sizeof(uint32_t)))) return fail(rc);
        uint32_t* d_count = ctx->d_counters + 1;
        if (cudaMemsetAsync(d_count, 0, sizeof(uint32_t), ctx->stream) != cudaSuccess) return fail(DSA_ERR_CUDA);
        const uint64_t blk = std::min<uint64_t>((n_pairs + 255) / 256, (uint64_t)ctx->sm_count * 16);
        k_collect_flags<<<(unsigned)blk, 256, 0, ctx->stream>>>(sc.flag, n_pairs, d_list.as<uint32_t>(),
                                                                 cap, d_count);
        ++ctx->launches;
        uint32_t count = 0;
        if (cudaMemcpyAsync(&count, d_count, sizeof(count), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
          set_error("rerun count: %s", cudaGetErrorString(cudaGetLastError()));
          return fail(DSA_ERR_CUDA);
        }
        res->n_rerun = count;
        if (count > cap) { set_error("too many saturated pairs (%u)", count); return fail(DSA_ERR_UNSUPPORTED); }
        if (count) {
          if ((rc = need_hp())) return fail(rc);
          std::vector<uint32_t> list(count);
          if (cudaMemcpy(list.data(), d_list.p, count * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(DSA_ERR_CUDA);
          for (uint32_t k : list) {
            const dsa_pair& p = hp[k];
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
        return fail(rc);
      if ((rc = launch_profile_int32(ctx, qs, d_mat.as<int8_t>(), nullptr, A, d_prof.as<int32_t>(),
                                     d_poff.as<uint64_t>())))
        return fail(rc);
      phase_begin(res, PH_INT32);
      if ((rc = launch_generic_int32(ctx, db, qs, d_prof.as<int32_t>(), d_poff.as<uint64_t>(),
                                     d_jobs.as<PairJob>(), n_short, 0, d_scr.as<int2>(), mode, fe, o,
                                     e, 0, sc)))
        return fail(rc);
      phase_end(res, PH_INT32);
    }
  }

  // hits
  phase_begin(res, PH_HITS);
  if (all && top_k) {
    const uint32_t k = std::min<uint32_t>(top_k, db->n);
    res->n_hits = (uint64_t)qs->n * k;
    void* p;
    if ((rc = ctx->alloc(&p, res->n_hits * sizeof(dsa_hit)))) return fail(rc);
    res->d_hits = (dsa_hit*)p;
    if ((rc = launch_topk(ctx, sc, qs->n, db->n, top_k, res->d_hits))) return fail(rc);
  } else {
    res->n_hits = n_out;
    void* p;
    if ((rc = ctx->alloc(&p, std::max<uint64_t>(1, res->n_hits) * sizeof(dsa_hit)))) return fail(rc);
    res->d_hits = (dsa_hit*)p;
    if ((rc = launch_fill_hits(ctx, sc, all ? nullptr : d_pairs, n_out, db->n, res->d_hits)))
      return fail(rc);
  }
  phase_end(res, PH_HITS);
  if (cudaGetLastError() != cudaSuccess) { set_error("kernel launch failed"); return fail(DSA_ERR_CUDA); }
  *out = res;
  return DSA_OK;
}

}  // namespace

extern "C" int dsa_align(dsa_ctx* ctx, const dsa_db* db, const dsa_db* queries,
                         const dsa_pair* pairs, uint64_t n_pairs, int mode, uint32_t free_ends,
                         const int8_t* matrix, int alphabet_size, int gap_open, int gap_extend,
                         uint32_t top_k, uint32_t flags, dsa_res** out) {
  return align_impl(ctx, db, queries, pairs, n_pairs, mode, free_ends, matrix, alphabet_size,
                    gap_open, gap_extend, top_k, flags, out);
}

extern "C" int dsa_align_batch(dsa_ctx* ctx, const dsa_db* db, const uint8_t* q_codes,
                               const uint64_t* q_offsets, uint32_t n_queries, const dsa_pair* pairs,
                               uint64_t n_pairs, int mode, uint32_t free_ends, const int8_t* matrix,
                               int alphabet_size, int gap_open, int gap_extend, uint32_t top_k,
                               uint32_t flags, dsa_res** out) {
  if (!ctx || !out) { set_error("NULL argument"); return DSA_ERR_INVALID_ARG; }
  dsa_db* qs = nullptr;
  DSA_TRY(dsa_db_load(ctx, q_codes, q_offsets, n_queries, alphabet_size, &qs));
  int rc = align_impl(ctx, db, qs, pairs, n_pairs, mode, free_ends, matrix, alphabet_size,
                      gap_open, gap_extend, top_k, flags, out);
  if (rc) { dsa_db_free(qs); return rc; }
  (*out)->owned_queries = qs;
  return DSA_OK;
}

extern "C" int dsa_align_pssm(dsa_ctx* ctx, const dsa_db* db, const dsa_db* queries,
                              const int8_t* pssm, int alphabet_size, int mode, uint32_t free_ends,
                              int gap_open, int gap_extend, uint32_t top_k, uint32_t flags,
                              dsa_res** out) {
  if (!pssm) { set_error("pssm is NULL"); return DSA_ERR_INVALID_ARG; }
  if (flags & DSA_PAIRS_ON_DEVICE) {
    set_error("position-specific profiles apply to all-vs-all searches only");
    return DSA_ERR_UNSUPPORTED;
  }
  return align_impl(ctx, db, queries, nullptr, 0, mode, free_ends, nullptr, alphabet_size,
                    gap_open, gap_extend, top_k, flags, out, pssm);
}

// ---------------------------------------------------------------- traceback --

static int fetch_hits(dsa_res* res) {
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

namespace dsa {

int traceback_device_staged(dsa_ctx* ctx, dsa_res* res, const TbBounds& B) {
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

}  // namespace dsa

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
  // every hit of a large result on the thread path: staged on the device
  // (DSA_TB_HOST_STAGING=1 keeps the host staging below)
  const char* host_staging = getenv("DSA_TB_HOST_STAGING");
  if (!which && res->long_bnd_off.empty() && res->n_hits >= std::max<uint64_t>(thread_min, 1) &&
      !(host_staging && host_staging[0] == '1')) {
    const int rc = traceback_device_staged(ctx, res, bounds);
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
  const dsa_db* db = res->db;
  const dsa_db* qs = res->queries;
  auto small = [](const TbJob& j) { return j.ie <= 4096 && (uint64_t)j.ie * j.je <= (1u << 20); };
  std::vector<TbJob>& tjobs = ctx->h_tb;   // thread-per-hit candidates
  tjobs.clear();
  std::vector<TbJob> jobs;                 // warp-per-hit
  std::vector<LongTbJob> ljobs;
  uint64_t cap_total = 0;
  const int band = long_band_rows(), ckpt = long_ckpt_rows();
  auto diag_window = [&](int32_t ie, int32_t je, int32_t score, int64_t& dlo, int64_t& dhi) {
    return tb_diag_window(bounds, ie, je, score, dlo, dhi);
  };
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
    if (!res->long_bnd_off.empty() && res->long_bnd_off[h] != UINT64_MAX) {
      LongTbJob lj{};
      lj.q_start = qs->h_off[hit.query_id];
      lj.t_start = db->h_off[hit.target_id] + hit.t_offset;
      lj.bnd_off = res->long_bnd_off[h];
      lj.n = res->long_n[h];
      lj.ie = hit.q_end + 1;
      lj.je = hit.t_end + 1;
      lj.hit = (uint32_t)h;
      lj.dlo = 0;
      lj.wc = lj.je;
      int64_t dlo, dhi;
      if (lj.ie > 0 && lj.je > 0 && diag_window(lj.ie, lj.je, hit.score, dlo, dhi)) {
        const int64_t wc = (int64_t)ckpt + dhi - dlo;   // a traceback band's window
        if (wc < lj.je) {
          lj.dlo = (int32_t)std::max<int64_t>(dlo, -(int64_t)lj.ie);
          lj.wc = (int32_t)wc;
        }
      }
      lj.wpr = (uint32_t)((lj.wc + 7) / 8);
      ljobs.push_back(lj);
      cap_total += (uint64_t)lj.ie + lj.je + 1;
    }
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
      cap_total += cap[t];
    }
    tjobs.resize(n_small[T]);
    jobs.resize(n_large[T]);
    parallel_for(sel.size(), T, [&](unsigned t, size_t b, size_t e) {
      uint64_t ks = n_small[t], kl = n_large[t];
      TbJob j;
      for (size_t x = b; x < e; ++x)
        if (make_short(sel[x], j)) {
          if (small(j)) tjobs[ks++] = j;
          else jobs[kl++] = j;
        }
    });
  }
  if (tjobs.size() < std::max<uint64_t>(thread_min, 1)) {
    jobs.insert(jobs.end(), tjobs.begin(), tjobs.end());
    tjobs.clear();
  }
  // Big rectangles of hits without score-pass checkpoints (1 M cells or more
  // over at least two 256-row bands): a checkpointed score pass over the
  // hit's rectangle (the band pipeline of the long pairs), then the long-pair
  // traceback (parallel band fill, windowed walk) instead of one warp working
  // through the bands one after another.
  std::vector<LongJob> bscore;
  std::vector<LongTbJob> bjobs;
  uint64_t b_bnd = 0, b_bands = 0;
  {
    std::vector<TbJob> keep;
    for (const TbJob& j : jobs) {
      const dsa_hit& hit = res->h_hits[j.hit];
      const int32_t ie = hit.q_end + 1, je = hit.t_end + 1;   // the whole rectangle
      if ((uint64_t)ie * (uint64_t)je < (1u << 18) || ie <= band) {
        keep.push_back(j);
        continue;
      }
      const uint64_t nb = ((uint64_t)ie + band - 1) / band;
      const uint64_t q0 = qs->h_off[hit.query_id], t0 = db->h_off[hit.target_id] + hit.t_offset;
      bscore.push_back({q0, t0, b_bnd, b_bands, b_bands, ie, je, (uint32_t)bscore.size(), 0});
      LongTbJob lj{};
      lj.q_start = q0;
      lj.t_start = t0;
      lj.bnd_off = b_bnd;
      lj.n = je;
      lj.ie = ie;
      lj.je = je;
      lj.hit = j.hit;
      lj.dlo = 0;
      lj.wc = je;
      int64_t dlo, dhi;
      if (diag_window(ie, je, hit.score, dlo, dhi)) {
        const int64_t wc = (int64_t)ckpt + dhi - dlo;   // a traceback band's window
        if (wc < je) {
          lj.dlo = (int32_t)std::max<int64_t>(dlo, -(int64_t)ie);
          lj.wc = (int32_t)wc;
        }
      }
      lj.wpr = (uint32_t)((lj.wc + 7) / 8);
      bjobs.push_back(lj);
      cap_total += (uint64_t)je - j.je;   // CIGAR capacity of the whole rectangle
      b_bnd += ((uint64_t)ie + ckpt - 1) / ckpt * (uint64_t)je;   // checkpoint rows
      b_bands += nb;
    }
    jobs.swap(keep);
  }
  if (jobs.empty() && tjobs.empty() && ljobs.empty() && bjobs.empty()) return DSA_OK;

  // grow the result's CIGAR array by the capacity bound
  const uint64_t old_n = res->n_cigar;
  void* newp = nullptr;
  DSA_TRY(ctx->alloc(&newp, (old_n + cap_total) * sizeof(uint32_t)));
  if (old_n)
    DSA_CUDA_TRY(cudaMemcpyAsync(newp, res->d_cigar, old_n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
  if (res->d_cigar) ctx->release(res->d_cigar, res->cigar_bytes);
  res->d_cigar = (uint32_t*)newp;
  res->cigar_bytes = (old_n + cap_total) * sizeof(uint32_t);

  DevBuf d_mat, d_total;
  DSA_TRY(d_mat.alloc(ctx, res->A * res->A));
  DSA_CUDA_TRY(cudaMemcpyAsync(d_mat.p, res->matrix.data(), res->A * res->A, cudaMemcpyHostToDevice,
                               ctx->stream));
  DSA_TRY(d_total.alloc(ctx, sizeof(uint64_t)));
  DSA_CUDA_TRY(cudaMemcpyAsync(d_total.p, &old_n, sizeof(uint64_t), cudaMemcpyHostToDevice, ctx->stream));
  uint64_t total = old_n;

  // chunks bounded by direction-matrix memory
  const uint64_t dir_limit = 1ull << 30;   // words (4 GiB)
  phase_begin(res, PH_TRACE);

  {
    if (!tjobs.empty()) {
      // groups of 32 hits share a layout padded to their largest (ie, je):
      // keep the given order unless it would double the work, else order by (ie, wc)
      // descending
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
      if (padded > 2 * cells) {
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
    }
  }
  if (!tjobs.empty()) {
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
        if (k1 > k0 && dir + w > dir_limit) break;
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
      DSA_TRY(launch_traceback_thread(ctx, db, qs, d_mat.as<int8_t>(), res->A, res->gap_open,
                                      res->gap_extend, res->mode, res->free_ends,
                                      s_plus_o_fits_int8(res->matrix.data(), res->A, res->gap_open),
                                      d_jobs.as<TbJob>(), (uint32_t)n_chunk,
                                      d_dir.as<uint32_t>(), d_cig.as<uint32_t>(), d_scr.as<int2>(),
                                      res->d_hits));
      DSA_TRY(launch_cigar_compact(ctx, res->d_hits, d_jobs.as<TbJob>(), (uint32_t)n_chunk,
                                   d_cig.as<uint32_t>(), res->d_cigar, total,
                                   d_total.as<uint64_t>()));
      DSA_CUDA_TRY(cudaMemcpyAsync(&total, d_total.p, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                   ctx->stream));
      DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      k0 = k1;
    }
  }

  size_t k0 = 0;
  while (k0 < jobs.size()) {
    uint64_t dir = 0, cig = 0, scr = 0;
    size_t k1 = k0;
    while (k1 < jobs.size()) {
      const uint64_t w = (uint64_t)jobs[k1].ie * jobs[k1].wpr;
      if (k1 > k0 && dir + w > dir_limit) break;
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
    DSA_TRY(launch_traceback(ctx, db, qs, d_mat.as<int8_t>(), res->A, res->gap_open,
                             res->gap_extend, res->mode, res->free_ends, d_jobs.as<TbJob>(),
                             (uint32_t)chunk.size(), d_dir.as<uint32_t>(), d_cig.as<uint32_t>(),
                             d_scr.as<int2>(), res->d_hits));
    DSA_TRY(launch_cigar_compact(ctx, res->d_hits, d_jobs.as<TbJob>(), (uint32_t)chunk.size(),
                                 d_cig.as<uint32_t>(), res->d_cigar, total, d_total.as<uint64_t>()));
    DSA_CUDA_TRY(cudaMemcpyAsync(&total, d_total.p, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    k0 = k1;
  }
  // decision matrices of the rectangles (or their diagonal bands), in chunks
  // of at most 32 GiB; bnd_rows: the score pass's checkpoint rows
  auto run_long = [&](std::vector<LongTbJob>& list, const int2* bnd_rows) -> int {
    const uint64_t limit = 8ull << 30;   // words
    size_t k0 = 0;
    while (k0 < list.size()) {
      uint64_t dir = 0, cig = 0;
      size_t k1 = k0;
      std::vector<uint32_t> items;
      while (k1 < list.size()) {
        LongTbJob& lj = list[k1];
        const uint64_t w = (uint64_t)lj.ie * lj.wpr;
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
      std::vector<TbJob> shim(chunk.size());   // the CIGAR packer reads hit and cig_off
      for (size_t k = 0; k < chunk.size(); ++k) {
        shim[k].hit = chunk[k].hit;
        shim[k].cig_off = chunk[k].cig_off;
      }
      DevBuf d_lj, d_items, d_dir, d_cig, d_shim;
      DSA_TRY(upload(ctx, d_lj, chunk));
      DSA_TRY(upload(ctx, d_items, items));
      DSA_TRY(upload(ctx, d_shim, shim));
      DSA_TRY(d_dir.alloc(ctx, dir * 4));
      DSA_TRY(d_cig.alloc(ctx, cig * 4));
      DSA_TRY(launch_long_traceback(ctx, db, qs, d_mat.as<int8_t>(), res->A, res->gap_open,
                                    res->gap_extend, res->mode, res->free_ends,
                                    d_lj.as<LongTbJob>(), (uint32_t)chunk.size(),
                                    d_items.as<uint32_t>(), (uint32_t)(items.size() / 2),
                                    bnd_rows, d_dir.as<uint32_t>(), d_cig.as<uint32_t>(),
                                    res->d_hits));
      DSA_TRY(launch_cigar_compact(ctx, res->d_hits, d_shim.as<TbJob>(), (uint32_t)shim.size(),
                                   d_cig.as<uint32_t>(), res->d_cigar, total,
                                   d_total.as<uint64_t>()));
      DSA_CUDA_TRY(cudaMemcpyAsync(&total, d_total.p, sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                   ctx->stream));
      DSA_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      k0 = k1;
    }
    return DSA_OK;
  };
  if (!ljobs.empty()) DSA_TRY(run_long(ljobs, res->d_bnd));
  if (!bscore.empty()) {
    // checkpointed score pass over the big rectangles, bands in latest-start order
    std::vector<std::pair<uint32_t, uint32_t>> mn(bscore.size());
    for (size_t k = 0; k < bscore.size(); ++k) mn[k] = {(uint32_t)bscore[k].m, (uint32_t)bscore[k].n};
    const std::vector<uint32_t> items = band_items(mn, band);
    const size_t nj = bscore.size();
    DevBuf d_bs, d_bitems, d_bbnd, d_bprog, d_bcand, d_bout;
    DSA_TRY(upload(ctx, d_bs, bscore));
    DSA_TRY(upload(ctx, d_bitems, items));
    DSA_TRY(d_bbnd.alloc(ctx, b_bnd * sizeof(int2)));
    DSA_TRY(d_bprog.alloc(ctx, b_bands * sizeof(uint32_t)));
    DSA_TRY(d_bcand.alloc(ctx, b_bands * long_cand_size()));
    DSA_TRY(d_bout.alloc(ctx, nj * 13));
    DSA_CUDA_TRY(cudaMemsetAsync(d_bprog.p, 0, b_bands * sizeof(uint32_t), ctx->stream));
    Scores bsc;   // the rerun's scores are not needed: only its checkpoint rows
    bsc.score = d_bout.as<int32_t>();
    bsc.q_end = bsc.score + nj;
    bsc.t_end = bsc.q_end + nj;
    bsc.flag = reinterpret_cast<uint8_t*>(bsc.t_end + nj);
    DSA_TRY(launch_long_score(ctx, db, qs, d_mat.as<int8_t>(), res->A, res->gap_open,
                              res->gap_extend, res->mode, res->free_ends,
                              s_plus_o_fits_int8(res->matrix.data(), res->A, res->gap_open),
                              d_bs.as<LongJob>(),
                              (uint32_t)nj, d_bitems.as<uint32_t>(), (uint32_t)(items.size() / 2),
                              d_bbnd.as<int2>(), d_bprog.as<uint32_t>(), d_bcand.p, bsc));
    DSA_TRY(run_long(bjobs, d_bbnd.as<int2>()));
  }
  phase_end(res, PH_TRACE);
  res->n_cigar = total;
  res->host_valid = false;
  return DSA_OK;
}

extern "C" int dsa_res_get(dsa_res* res, const dsa_hit** hits, uint64_t* n_hits,
                           const uint32_t** cigar, uint64_t* n_cigar_words) {
  if (!res) { set_error("res is NULL"); return DSA_ERR_INVALID_ARG; }
  if (res->ctx) DSA_TRY(set_device(res->ctx));
  if (res->flags & DSA_RESULTS_ON_DEVICE) {
    if (hits) *hits = res->d_hits;
    if (cigar) *cigar = res->d_cigar;
  } else {
    DSA_TRY(fetch_hits(res));
    if (hits) *hits = res->h_hits.data();
    if (cigar) *cigar = res->h_cigar.data();
  }
  if (n_hits) *n_hits = res->n_hits;
  if (n_cigar_words) *n_cigar_words = res->n_cigar;
  return DSA_OK;
}

extern "C" int dsa_res_stats(const dsa_res* res, uint64_t* cells, uint64_t* n_rerun) {
  if (!res) { set_error("res is NULL"); return DSA_ERR_INVALID_ARG; }
  if (cells) *cells = res->cells;
  if (n_rerun) *n_rerun = res->n_rerun;
  return DSA_OK;
}

extern "C" int dsa_res_timing(const dsa_res* res, double* ms, int n) {
  if (!res || !ms || n < 0) { set_error("bad argument"); return DSA_ERR_INVALID_ARG; }
  for (int p = 0; p < n && p < dsa_res::NPHASE; ++p) {
    ms[p] = -1.0;
    if (!res->used[p]) continue;
    float t = 0.f;
    if (cudaEventSynchronize(res->ev[2 * p + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, res->ev[2 * p], res->ev[2 * p + 1]) != cudaSuccess) {
      set_error("event timing failed: %s", cudaGetErrorString(cudaGetLastError()));
      return DSA_ERR_CUDA;
    }
    ms[p] = t;
  }
  return DSA_OK;
}

extern "C" int dsa_res_phase_cells(const dsa_res* res, uint64_t* cells, int n) {
  if (!res || !cells || n < 0) { set_error("bad argument"); return DSA_ERR_INVALID_ARG; }
  for (int p = 0; p < n && p < dsa_res::NPHASE; ++p) cells[p] = res->phase_cells[p];
  return DSA_OK;
}

extern "C" int dsa_res_free(dsa_res* res) {
  if (!res) return DSA_OK;
  dsa_ctx* ctx = res->ctx;
  if (!ctx) {   // host-only result (serving): nothing on the device
    delete res;
    return DSA_OK;
  }
  cudaSetDevice(ctx->device);
  for (int k = 0; k < 2 * dsa_res::NPHASE; ++k)
    if (res->ev[k]) cudaEventDestroy(res->ev[k]);
  if (res->d_hits) ctx->release(res->d_hits, std::max<uint64_t>(1, res->n_hits) * sizeof(dsa_hit));
  if (res->d_cigar) ctx->release(res->d_cigar, res->cigar_bytes);
  if (res->d_bnd) ctx->release(res->d_bnd, res->bnd_bytes);
  if (res->owned_queries) dsa_db_free(res->owned_queries);
  delete res;
  return DSA_OK;
}

extern "C" int dsa_selftest_wait_timeout(dsa_ctx* ctx, int kind, uint64_t limit_ns) {
  if (!ctx) { set_error("NULL argument"); return DSA_ERR_INVALID_ARG; }
  DSA_TRY(set_device(ctx));
  return run_selftest_wait(ctx, kind, limit_ns);
}

extern "C" int dsa_probe_issue_rate(dsa_ctx* ctx, int form, double* rate) {
  if (!ctx || !rate) { set_error("NULL argument"); return DSA_ERR_INVALID_ARG; }
  DSA_TRY(set_device(ctx));
  return run_issue_probe(ctx, form, rate);
}
