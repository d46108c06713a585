// Host side of the libdsa C ABI (the per-core alignment of the map phase,
// Sec. II.B.1, with its three algorithms, Sec. II.C.2, and the top K of
// Sec. II.B.2): contexts, device-resident sequence sets, argument checks and
// the result object of dsa_align.  The score passes are planned in
// plan_all.cu (all-vs-all) and plan_pairs.cu (explicit pairs), the traceback
// in tb_host.cu; every arithmetic step runs in the kernels of the other
// translation units.
#include "host_util.cuh"

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
  PairPass pp;
  pp.pairs = pairs;
  pp.n_pairs = n_pairs;
  pp.flags = flags;
  pp.hp_ready = all;
  if (!all) {
    const PairPlanParams P{qs->n, db->n, w16, o, e, local16, packed_ok};
    DSA_TRY(pairs_classify(ctx, db, qs, P, pp));
  }
  // int32 range: (m + n) * max|value step| must stay far from 2^31
  const uint32_t max_m = qs->max_len;
  const uint32_t max_n = all ? db->max_len : pp.pst.max_t_len;
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
    if ((rc = score_pairs(ctx, res, db, qs, pp, mode, fe, matrix, d_mat.as<int8_t>(), A, o, e, v,
                          local16, packed_ok, w16, sc)))
      return fail(rc);
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
    if ((rc = launch_fill_hits(ctx, sc, all ? nullptr : pp.d_pairs, n_out, db->n, res->d_hits)))
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
