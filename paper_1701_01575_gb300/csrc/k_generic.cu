// Exact int32 Gotoh kernel for any mode and any list of (query, target window)
// pairs: one thread per pair, the query processed in strips of STRIP rows held
// in registers, the target scanned column by column, the strip's last row
// (H and F) handed to the next strip through a per-pair boundary row in
// global memory.
//
// Used as (1) the plain per-query form (one launch per query over the DB in
// input order, profile read from global memory), (2) the exact rerun of pairs
// whose packed 16-bit pass saturated, and (3) the path for modes and score
// ranges the packed kernels do not cover.
//
// Recurrences (Gotoh; the paper delegates the arithmetic to SSW and Parasail,
// Sec. II.B.1):
//   E[i][j] = max(E[i][j-1] - e, H[i][j-1] - o)
//   F[i][j] = max(F[i-1][j] - e, H[i-1][j] - o)
//   H[i][j] = max(H[i-1][j-1] + S[q_i][t_j], E[i][j], F[i][j] [, 0 local])
#include "dsa_internal.cuh"

namespace dsa {
namespace {

constexpr int STRIP = 8;

__device__ __forceinline__ int32_t h_row0(int mode, uint32_t fe, int64_t j, int o, int e) {
  if (j == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_T_BEGIN))) return 0;
  return -(o + (int32_t)(j - 1) * e);
}
__device__ __forceinline__ int32_t h_col0(int mode, uint32_t fe, int64_t i, int o, int e) {
  if (i == 0 || mode == DSA_LOCAL || (mode == DSA_SEMIGLOBAL && (fe & DSA_FREE_Q_BEGIN))) return 0;
  return -(o + (int32_t)(i - 1) * e);
}

// Result-cell order: higher score, then smaller j, then smaller i.
struct Best {
  int32_t s;
  int32_t i, j;
  bool have;
  __device__ __forceinline__ void offer(int32_t h, int32_t ii, int32_t jj) {
    if (!have || h > s || (h == s && (jj < j || (jj == j && ii < i)))) {
      s = h; i = ii; j = jj; have = true;
    }
  }
};

__global__ void __launch_bounds__(128) k_generic_int32(
    const uint8_t* __restrict__ tcodes, const uint8_t* __restrict__ qcodes,
    const uint64_t* __restrict__ qoff, const uint32_t* __restrict__ qlen,
    const int32_t* __restrict__ prof, const uint64_t* __restrict__ prof_off,
    const PairJob* __restrict__ jobs, uint64_t n_jobs, uint32_t fixed_q,
    const uint64_t* __restrict__ t_off, const uint32_t* __restrict__ t_len, uint32_t n_t,
    int2* __restrict__ scratch, int mode, uint32_t fe, int o, int e, uint8_t flag_value,
    int32_t* __restrict__ o_score, int32_t* __restrict__ o_qend, int32_t* __restrict__ o_tend,
    uint8_t* __restrict__ o_flag) {
  const bool local = mode == DSA_LOCAL;
  const bool sg = mode == DSA_SEMIGLOBAL;
  const bool q_end_free = sg && (fe & DSA_FREE_Q_END);
  const bool t_end_free = sg && (fe & DSA_FREE_T_END);
  for (uint64_t jid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; jid < n_jobs;
       jid += (uint64_t)gridDim.x * blockDim.x) {
    PairJob job;
    if (jobs) {
      job = jobs[jid];
    } else {   // every target of query fixed_q, in input order
      job.t_start = t_off[jid];
      job.scratch = t_off[jid];
      job.q = fixed_q;
      job.n = t_len[jid];
      job.out = (uint32_t)((uint64_t)fixed_q * n_t + jid);
      job.pad = 0;
    }
    const int32_t m = (int32_t)qlen[job.q];
    const int32_t n = (int32_t)job.n;
    const int32_t mpad = (m + 7) & ~7;
    const int32_t* P = prof + prof_off[job.q];
    const uint8_t* t = tcodes + job.t_start;
    int2* scr = scratch + job.scratch;

    Best b;
    b.s = 0; b.i = -1; b.j = -1; b.have = false;
    if (q_end_free) b.offer(h_row0(mode, fe, n, o, e), 0, n);

    for (int32_t i0 = 0; i0 < m; i0 += STRIP) {
      const int rows = min(STRIP, m - i0);
      int32_t Hc[STRIP], Ec[STRIP];
#pragma unroll
      for (int r = 0; r < STRIP; ++r) {
        Hc[r] = h_col0(mode, fe, i0 + r + 1, o, e);
        Ec[r] = NEG32;
      }
      if (t_end_free && i0 + rows == m) b.offer(Hc[rows - 1], m, 0);
      int32_t diag = h_col0(mode, fe, i0, o, e);   // H[i0][0]
      for (int32_t j = 1; j <= n; ++j) {
        const int a = t[j - 1];
        int32_t Hup, Fup;
        if (i0 == 0) {
          Hup = h_row0(mode, fe, j, o, e);
          Fup = NEG32;
        } else {
          const int2 v = scr[j - 1];
          Hup = v.x;
          Fup = v.y;
        }
        const int4* prow = reinterpret_cast<const int4*>(P + (size_t)a * mpad + i0);
        const int4 p0 = __ldg(prow);
        const int4 p1 = __ldg(prow + 1);
        const int32_t sv[STRIP] = {p0.x, p0.y, p0.z, p0.w, p1.x, p1.y, p1.z, p1.w};
        int32_t d = diag;
        diag = Hup;
        int32_t F = Fup, Hprev = Hup;
#pragma unroll
        for (int r = 0; r < STRIP; ++r) {
          if (r < rows) {
            F = max(F - e, Hprev - o);
            Ec[r] = max(Ec[r] - e, Hc[r] - o);
            int32_t h = max(d + sv[r], max(Ec[r], F));
            if (local) h = max(h, 0);
            d = Hc[r];
            Hc[r] = h;
            Hprev = h;
            const int32_t i = i0 + r + 1;
            if (local) {
              if (h > 0) b.offer(h, i, j);
            } else {
              if (j == n && (q_end_free || i == m)) b.offer(h, i, j);
              if (t_end_free && i == m) b.offer(h, i, j);
            }
          }
        }
        scr[j - 1] = make_int2(Hprev, F);
      }
    }
    const uint32_t out = job.out;
    if (local && !b.have) {
      o_score[out] = 0; o_qend[out] = -1; o_tend[out] = -1;
    } else {
      o_score[out] = b.s; o_qend[out] = b.i - 1; o_tend[out] = b.j - 1;
    }
    o_flag[out] = flag_value | (uint8_t)job.pad;   // pad = 1 marks a saturation rerun
  }
}

// P[q][a][i] = S[q_i][a] for a < A, rows padded to a multiple of 8 with 0;
// with a position-specific profile Pq (one row per query residue of the set)
// P[q][a][i] = Pq[qoff[q] + i][a].
__global__ void k_profile_int32(const uint8_t* __restrict__ qcodes, const uint64_t* __restrict__ qoff,
                                const uint32_t* __restrict__ qlen, uint32_t nq,
                                const int8_t* __restrict__ S, const int8_t* __restrict__ Pq, int A,
                                int32_t* __restrict__ prof, const uint64_t* __restrict__ prof_off) {
  for (uint32_t q = blockIdx.y; q < nq; q += gridDim.y) {
    const int32_t m = (int32_t)qlen[q];
    const int32_t mpad = (m + 7) & ~7;
    const uint8_t* qs = qcodes + qoff[q];
    int32_t* P = prof + prof_off[q];
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < (int64_t)A * mpad;
         x += (int64_t)gridDim.x * blockDim.x) {
      const int a = (int)(x / mpad);
      const int i = (int)(x % mpad);
      P[x] = i >= m ? 0
             : Pq   ? (int32_t)Pq[(qoff[q] + (uint64_t)i) * A + a]
                    : (int32_t)S[qs[i] * A + a];
    }
  }
}

// Interleaved copy: group g (sorted targets 32g..32g+31), chunk c, lane l ->
// 16 residues c*16.. of target 32g+l, padding code beyond its length.
__global__ void k_interleave(const uint8_t* __restrict__ codes, const uint64_t* __restrict__ off,
                             const uint32_t* __restrict__ perm, const uint32_t* __restrict__ slen,
                             uint32_t n, const uint64_t* __restrict__ gbase,
                             const uint32_t* __restrict__ glen, uint32_t n_groups, uint8_t pad,
                             uint8_t* __restrict__ il) {
  const uint32_t g = blockIdx.x;
  if (g >= n_groups) return;
  const uint32_t chunks = (glen[g] + CHUNK - 1) / CHUNK;
  const uint32_t total = chunks * GROUP;   // 16-byte words in this group
  for (uint32_t w = threadIdx.x; w < total; w += blockDim.x) {
    const uint32_t c = w / GROUP, lane = w % GROUP;
    const uint32_t st = g * GROUP + lane;
    uint8_t buf[CHUNK];
    uint32_t len = 0;
    const uint8_t* src = nullptr;
    if (st < n) {
      len = slen[st];
      src = codes + off[perm[st]];
    }
#pragma unroll
    for (int b = 0; b < CHUNK; ++b) {
      const uint32_t p = c * CHUNK + b;
      buf[b] = p < len ? src[p] : pad;
    }
    uint4 v;
    memcpy(&v, buf, 16);
    reinterpret_cast<uint4*>(il + gbase[g])[c * GROUP + lane] = v;
  }
}

}  // namespace

int launch_generic_int32(dsa_ctx* ctx, const dsa_db* db, const dsa_db* qs, const int32_t* d_prof,
                         const uint64_t* d_prof_off, const PairJob* d_jobs, uint64_t n_jobs,
                         uint32_t fixed_q, int2* d_scratch, int mode, uint32_t fe, int o, int e,
                         uint8_t flag_value, Scores out) {
  if (n_jobs == 0) return DSA_OK;
  const int threads = 128;
  uint64_t blocks = (n_jobs + threads - 1) / threads;
  const uint64_t cap = (uint64_t)ctx->sm_count * 64;
  if (blocks > cap) blocks = cap;
  k_generic_int32<<<(unsigned)blocks, threads, 0, ctx->stream>>>(
      db->d_codes, qs->d_codes, qs->d_off, qs->d_len, d_prof, d_prof_off, d_jobs, n_jobs, fixed_q,
      db->d_off, db->d_len, db->n, d_scratch, mode, fe, o, e, flag_value, out.score, out.q_end,
      out.t_end, out.flag);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_profile_int32(dsa_ctx* ctx, const dsa_db* qs, const int8_t* d_matrix,
                         const int8_t* d_pssm, int A, int32_t* d_prof, const uint64_t* d_prof_off) {
  if (qs->n == 0) return DSA_OK;
  dim3 grid(qs->n > 4096 ? 1 : 64, std::min<uint32_t>(qs->n, 65535));
  k_profile_int32<<<grid, 256, 0, ctx->stream>>>(qs->d_codes, qs->d_off, qs->d_len, qs->n,
                                                 d_matrix, d_pssm, A, d_prof, d_prof_off);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

int launch_interleave(dsa_ctx* ctx, dsa_db* db) {
  if (db->n_groups == 0) return DSA_OK;
  k_interleave<<<db->n_groups, 256, 0, ctx->stream>>>(db->d_codes, db->d_off, db->d_perm,
                                                       db->d_slen, db->n, db->d_gbase, db->d_glen,
                                                       db->n_groups, (uint8_t)db->A, db->d_il);
  DSA_CUDA_TRY(cudaGetLastError());
  ++ctx->launches;
  return DSA_OK;
}

}  // namespace dsa
