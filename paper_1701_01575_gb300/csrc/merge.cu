// Partition + reduce (Sec. II.B.2): every partition of the database keeps the
// top K of each query, and a reduce keeps the top K of those.  Under the
// total order (score descending, then global target id ascending) the reduce
// of exact per-partition lists equals one search of the whole database, so a
// database larger than the device (or the context's budget) can be searched
// one partition at a time on one GPU, and the per-device lists of a sharded
// database reduce the same way.
#include "dsa_internal.cuh"

#include <algorithm>
#include <vector>

namespace {

// a before b in the top-K order
inline bool ranks_before(const dsa_hit& a, uint64_t ga, const dsa_hit& b, uint64_t gb) {
  return a.score != b.score ? a.score > b.score : ga < gb;
}

}  // namespace

extern "C" int dsa_merge_topk(const dsa_hit* const* part_hits, const uint64_t* part_n_hits,
                              const uint32_t* const* part_cigar, const uint32_t* target_base,
                              uint32_t n_parts, uint32_t n_queries, uint32_t k, dsa_hit* out_hits,
                              uint64_t* out_n_hits, uint32_t* out_cigar, uint64_t* out_n_cigar) {
  if (!part_n_hits || !target_base || !out_hits || !out_n_hits || (n_parts && !part_hits) ||
      n_queries == 0 || k == 0) {
    dsa::set_error("dsa_merge_topk: NULL argument, no queries or k = 0");
    return DSA_ERR_INVALID_ARG;
  }
  std::vector<uint64_t> kp(n_parts);
  for (uint32_t p = 0; p < n_parts; ++p) {
    if (part_n_hits[p] % n_queries) {
      dsa::set_error("partition %u: %llu hits is not a multiple of %u queries", p,
                     (unsigned long long)part_n_hits[p], n_queries);
      return DSA_ERR_INVALID_ARG;
    }
    kp[p] = part_n_hits[p] / n_queries;
    if (kp[p] && !part_hits[p]) {
      dsa::set_error("partition %u: NULL hit list", p);
      return DSA_ERR_INVALID_ARG;
    }
    // every list must be in rank order, of the right query, and carry a
    // CIGAR array when it has traced hits
    for (uint32_t q = 0; q < n_queries; ++q) {
      const dsa_hit* h = part_hits[p] + (uint64_t)q * kp[p];
      for (uint64_t x = 0; x < kp[p]; ++x) {
        if (h[x].query_id != q) {
          dsa::set_error("partition %u: hit %llu belongs to query %u, not %u", p,
                         (unsigned long long)((uint64_t)q * kp[p] + x), h[x].query_id, q);
          return DSA_ERR_INVALID_ARG;
        }
        if (x && !ranks_before(h[x - 1], h[x - 1].target_id, h[x], h[x].target_id)) {
          dsa::set_error("partition %u: the list of query %u is not in top-K order", p, q);
          return DSA_ERR_INVALID_ARG;
        }
        if ((h[x].flags & DSA_HIT_HAS_TRACEBACK) && h[x].cigar_len &&
            (!part_cigar || !part_cigar[p] || !out_cigar)) {
          dsa::set_error("partition %u: traced hits need the partition's CIGAR words and out_cigar", p);
          return DSA_ERR_INVALID_ARG;
        }
      }
    }
  }
  uint64_t total_k = 0;
  for (uint64_t x : kp) total_k += x;
  const uint64_t kk = std::min<uint64_t>(k, total_k);
  uint64_t n_out = 0, n_cig = 0;
  std::vector<uint64_t> pos(n_parts);
  for (uint32_t q = 0; q < n_queries; ++q) {
    std::fill(pos.begin(), pos.end(), 0);
    for (uint64_t r = 0; r < kk; ++r) {
      // the best head among the partitions' lists (few partitions: a scan)
      int best = -1;
      uint64_t best_g = 0;
      for (uint32_t p = 0; p < n_parts; ++p) {
        if (pos[p] == kp[p]) continue;
        const dsa_hit& h = part_hits[p][(uint64_t)q * kp[p] + pos[p]];
        const uint64_t g = (uint64_t)target_base[p] + h.target_id;
        if (best < 0 || ranks_before(h, g, part_hits[best][(uint64_t)q * kp[best] + pos[best]], best_g)) {
          best = (int)p;
          best_g = g;
        }
      }
      dsa_hit h = part_hits[best][(uint64_t)q * kp[best] + pos[best]];
      ++pos[best];
      if (best_g > UINT32_MAX) {
        dsa::set_error("global target id %llu does not fit 32 bits", (unsigned long long)best_g);
        return DSA_ERR_INVALID_ARG;
      }
      h.target_id = (uint32_t)best_g;
      if (out_cigar && h.cigar_len) {
        std::copy(part_cigar[best] + h.cigar_off, part_cigar[best] + h.cigar_off + h.cigar_len,
                  out_cigar + n_cig);
        h.cigar_off = n_cig;
        n_cig += h.cigar_len;
      } else {
        h.cigar_off = 0;
      }
      out_hits[n_out++] = h;
    }
  }
  *out_n_hits = n_out;
  if (out_n_cigar) *out_n_cigar = n_cig;
  return DSA_OK;
}

extern "C" int dsa_search_partitioned(dsa_ctx* ctx, const uint8_t* codes, const uint64_t* offsets,
                                      uint32_t n_seqs, int alphabet_size,
                                      uint64_t partition_residues, const dsa_db* queries, int mode,
                                      uint32_t free_ends, const int8_t* matrix, int gap_open,
                                      int gap_extend, uint32_t top_k, int traceback,
                                      dsa_res** out) {
  if (!ctx || !codes || !offsets || !queries || !matrix || !out || n_seqs == 0 || top_k == 0) {
    dsa::set_error("dsa_search_partitioned: NULL argument, empty database or top_k = 0");
    return DSA_ERR_INVALID_ARG;
  }
  *out = nullptr;
  uint32_t nq = 0;
  DSA_TRY(dsa_db_info(queries, &nq, nullptr, nullptr));
  // consecutive targets while the partition holds at most partition_residues
  // (at least one target per partition)
  std::vector<uint32_t> cut{0};
  for (uint32_t t = 1; t < n_seqs; ++t)
    if (partition_residues && offsets[t + 1] - offsets[cut.back()] > partition_residues) cut.push_back(t);
  cut.push_back(n_seqs);
  const uint32_t n_parts = (uint32_t)cut.size() - 1;
  std::vector<std::vector<dsa_hit>> hits(n_parts);
  std::vector<std::vector<uint32_t>> cigs(n_parts);
  uint64_t cells = 0, rerun = 0, cig_total = 0;
  for (uint32_t p = 0; p < n_parts; ++p) {
    const uint32_t b = cut[p], e = cut[p + 1];
    std::vector<uint64_t> loc(e - b + 1);
    for (uint32_t t = b; t <= e; ++t) loc[t - b] = offsets[t] - offsets[b];
    dsa_db* pdb = nullptr;
    DSA_TRY(dsa_db_load(ctx, codes + offsets[b], loc.data(), e - b, alphabet_size, &pdb));
    dsa_res* res = nullptr;
    int rc = dsa_align(ctx, pdb, queries, nullptr, 0, mode, free_ends, matrix, alphabet_size,
                       gap_open, gap_extend, top_k, 0, &res);
    if (rc == DSA_OK && traceback) rc = dsa_traceback(ctx, res, nullptr, 0);
    const dsa_hit* h = nullptr;
    const uint32_t* c = nullptr;
    uint64_t nh = 0, nc = 0;
    if (rc == DSA_OK) rc = dsa_res_get(res, &h, &nh, &c, &nc);
    if (rc == DSA_OK) {
      hits[p].assign(h, h + nh);
      cigs[p].assign(c, c + nc);
      cig_total += nc;
      uint64_t cl = 0, rr = 0;
      dsa_res_stats(res, &cl, &rr);
      cells += cl;
      rerun += rr;
    }
    if (res) dsa_res_free(res);
    dsa_db_free(pdb);
    if (rc) return rc;
  }
  dsa_res* m = new (std::nothrow) dsa_res;
  if (!m) { dsa::set_error("host allocation failed"); return DSA_ERR_OOM; }
  std::vector<const dsa_hit*> ph(n_parts);
  std::vector<const uint32_t*> pc(n_parts);
  std::vector<uint64_t> pn(n_parts);
  std::vector<uint32_t> base(n_parts);
  for (uint32_t p = 0; p < n_parts; ++p) {
    ph[p] = hits[p].data();
    pc[p] = cigs[p].data();
    pn[p] = hits[p].size();
    base[p] = cut[p];
  }
  try {
    m->h_hits.resize((uint64_t)nq * top_k);
    m->h_cigar.resize(std::max<uint64_t>(cig_total, 1));
  } catch (...) {
    delete m;
    dsa::set_error("host allocation failed");
    return DSA_ERR_OOM;
  }
  uint64_t n_out = 0, n_cig = 0;
  const int rc = dsa_merge_topk(ph.data(), pn.data(), pc.data(), base.data(), n_parts, nq, top_k,
                                m->h_hits.data(), &n_out, m->h_cigar.data(), &n_cig);
  if (rc) { delete m; return rc; }
  m->h_hits.resize(n_out);
  m->h_cigar.resize(n_cig);
  m->n_hits = n_out;
  m->n_cigar = n_cig;
  m->host_valid = true;   // host-only: ctx stays NULL
  m->mode = mode;
  m->free_ends = free_ends;
  m->cells = cells;
  m->n_rerun = rerun;
  *out = m;
  return DSA_OK;
}
