// Serving loop: continuous batching of alignment requests against
// device-resident databases.
//
// The paper's system answers alignment jobs submitted to a Spark cluster,
// one job at a time (Sec. II.B).  A serving process on one GPU instead keeps
// the database resident and admits requests as they arrive: worker slots
// (each a context with its own stream) repeatedly take the oldest pending
// request plus every later compatible one (same database, kind and scoring)
// up to the batch limits, provided the batch's estimated device footprint
// fits the memory not reserved by running batches, and run them as one
// alignment call.  Batching matters most for single-query protein requests:
// two queries share each packed 16-bit register pair, so a lone query would
// leave half of every DP instruction idle.  Batches of different slots
// overlap on the device.  A request's results do not depend on its batch:
// scores are exact and the top-k order is total.
#include "dsa_internal.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <new>
#include <unordered_map>

namespace {

struct Req {
  uint64_t ticket = 0;
  dsa_request r{};
  std::vector<uint8_t> q_codes;
  std::vector<uint64_t> q_off;
  std::vector<dsa_pair> pairs;
  std::vector<int8_t> matrix;
  double arrive = 0, admit = 0, finish = 0;
  uint32_t batch_requests = 0;
  int status = DSA_OK;
  bool done = false;
  dsa_res* result = nullptr;
};

bool compatible(const Req& a, const Req& b) {
  return a.r.kind == b.r.kind && a.r.db == b.r.db && a.r.mode == b.r.mode &&
         a.r.free_ends == b.r.free_ends && a.r.alphabet_size == b.r.alphabet_size &&
         a.r.gap_open == b.r.gap_open && a.r.gap_extend == b.r.gap_extend &&
         a.r.top_k == b.r.top_k && (a.r.traceback != 0) == (b.r.traceback != 0) &&
         a.matrix == b.matrix;
}

}  // namespace

struct dsa_server {
  int device = 0;
  dsa_server_config cfg{};
  size_t capacity = 0;     // bytes batches may reserve in total
  std::vector<dsa_ctx*> slots;
  std::vector<std::thread> workers;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::unordered_map<uint64_t, Req*> reqs;
  uint64_t next_ticket = 1;
  size_t reserved = 0;
  uint32_t running = 0;
  bool stop = false;
  std::chrono::steady_clock::time_point t0;
  int sm_count = 0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  size_t estimate(const std::vector<Req*>& batch) const;
  void worker(int slot);
  void run_batch(dsa_ctx* ctx, std::vector<Req*>& batch);
};

size_t dsa_server::estimate(const std::vector<Req*>& batch) const {
  const dsa_db* db = batch[0]->r.db;
  uint64_t nq = 0, np = 0, tlen = 0, mmax = 0;
  uint64_t dirs = 0;
  for (const Req* q : batch) {
    nq += q->r.n_queries;
    for (uint32_t k = 0; k < q->r.n_queries; ++k)
      mmax = std::max<uint64_t>(mmax, q->q_off[k + 1] - q->q_off[k]);
    if (q->r.kind == DSA_REQ_PAIRS) {
      np += q->pairs.size();
      for (const dsa_pair& p : q->pairs) {
        tlen += p.t_len;
        const uint64_t m = q->q_off[p.query_id + 1] - q->q_off[p.query_id];
        if (q->r.traceback) dirs += (m + 1) * ((p.t_len + 8) / 8) * 4;
      }
    }
  }
  uint64_t bytes = 64ull << 20;   // profiles, job lists, small buffers
  if (batch[0]->r.kind == DSA_REQ_SEARCH) {
    const uint64_t nt = db->n;
    const uint64_t glen = db->max_len;
    bytes += nq * nt * 13;                                           // dense scores
    // boundary rows of the packed kernel: grid = min(items, 2 CTAs per SM),
    // items = units (<= query pairs) x blocks of 8 groups
    const uint64_t blocks = (db->n_groups + dsa::INTER_WARPS - 1) / dsa::INTER_WARPS;
    const uint64_t grid = std::min<uint64_t>((nq + 1) / 2 * blocks, (uint64_t)sm_count * 2);
    bytes += grid * dsa::INTER_WARPS * 32 * glen * 8;
    const uint64_t k = std::min<uint64_t>(batch[0]->r.top_k ? batch[0]->r.top_k : nt, nt);
    bytes += nq * k * sizeof(dsa_hit);
    if (batch[0]->r.traceback) bytes += nq * k * (mmax + 1) * ((glen + 8) / 8) * 4;
  } else {
    bytes += np * (13 + sizeof(dsa_hit) + sizeof(dsa::PairJob)) + tlen * 8;
    bytes += std::min<uint64_t>(dirs, 4ull << 30);
  }
  return (size_t)bytes;
}

void dsa_server::run_batch(dsa_ctx* ctx, std::vector<Req*>& batch) {
  const Req& h = *batch[0];
  // concatenate the queries of the batch
  std::vector<uint8_t> codes;
  std::vector<uint64_t> off{0};
  std::vector<uint32_t> qbase(batch.size());
  std::vector<dsa_pair> pairs;
  std::vector<uint64_t> pbase(batch.size());
  for (size_t b = 0; b < batch.size(); ++b) {
    const Req& q = *batch[b];
    qbase[b] = (uint32_t)(off.size() - 1);
    codes.insert(codes.end(), q.q_codes.begin(), q.q_codes.end());
    const uint64_t base = off.back();
    for (uint32_t k = 0; k < q.r.n_queries; ++k) off.push_back(base + q.q_off[k + 1]);
    pbase[b] = pairs.size();
    for (dsa_pair p : q.pairs) {
      p.query_id += qbase[b];
      pairs.push_back(p);
    }
  }
  int rc = DSA_OK;
  dsa_db* qs = nullptr;
  dsa_res* res = nullptr;
  rc = dsa_db_load(ctx, codes.data(), off.data(), (uint32_t)(off.size() - 1), h.r.alphabet_size, &qs);
  if (rc == DSA_OK) {
    rc = dsa_align(ctx, h.r.db, qs, h.r.kind == DSA_REQ_PAIRS ? pairs.data() : nullptr,
                   pairs.size(), h.r.mode, h.r.free_ends, h.matrix.data(), h.r.alphabet_size,
                   h.r.gap_open, h.r.gap_extend, h.r.kind == DSA_REQ_SEARCH ? h.r.top_k : 0, 0,
                   &res);
  }
  if (rc == DSA_OK && h.r.traceback) rc = dsa_traceback(ctx, res, nullptr, 0);
  const dsa_hit* hits = nullptr;
  const uint32_t* cig = nullptr;
  uint64_t n_hits = 0, n_cig = 0;
  if (rc == DSA_OK) rc = dsa_res_get(res, &hits, &n_hits, &cig, &n_cig);
  if (rc == DSA_OK) rc = dsa_sync(ctx);
  // split per request
  const uint64_t nt = h.r.db->n;
  const uint64_t per_q = h.r.kind == DSA_REQ_SEARCH
                             ? (h.r.top_k ? std::min<uint64_t>(h.r.top_k, nt) : nt)
                             : 0;
  for (size_t b = 0; b < batch.size(); ++b) {
    Req& q = *batch[b];
    q.status = rc;
    if (rc != DSA_OK) continue;
    uint64_t h0, h1;
    if (h.r.kind == DSA_REQ_SEARCH) {
      h0 = (uint64_t)qbase[b] * per_q;
      h1 = h0 + (uint64_t)q.r.n_queries * per_q;
    } else {
      h0 = pbase[b];
      h1 = h0 + q.pairs.size();
    }
    dsa_res* out = new dsa_res;
    out->ctx = nullptr;
    out->mode = h.r.mode;
    out->free_ends = h.r.free_ends;
    out->A = h.r.alphabet_size;
    out->gap_open = h.r.gap_open;
    out->gap_extend = h.r.gap_extend;
    out->matrix = q.matrix;
    out->n_hits = h1 - h0;
    out->h_hits.assign(hits + h0, hits + h1);
    for (dsa_hit& x : out->h_hits) {
      x.query_id -= qbase[b];
      const uint64_t src = x.cigar_off;
      x.cigar_off = out->h_cigar.size();
      out->h_cigar.insert(out->h_cigar.end(), cig + src, cig + src + x.cigar_len);
    }
    out->n_cigar = out->h_cigar.size();
    out->host_valid = true;
    q.result = out;
  }
  if (res) dsa_res_free(res);
  if (qs) dsa_db_free(qs);
}

void dsa_server::worker(int slot) {
  dsa_ctx* ctx = slots[slot];
  cudaSetDevice(device);
  for (;;) {
    std::vector<Req*> batch;
    size_t est = 0;
    {
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        if (stop) return;
        if (!pending.empty()) {
          // the oldest request and the later compatible ones, within the limits
          Req* head = pending.front();
          batch.assign(1, head);
          uint64_t nq = head->r.n_queries, np = head->pairs.size();
          for (size_t k = 1; k < pending.size(); ++k) {
            Req* c = pending[k];
            if (!compatible(*head, *c)) continue;
            if (head->r.kind == DSA_REQ_SEARCH && nq + c->r.n_queries > cfg.max_batch_queries) break;
            if (head->r.kind == DSA_REQ_PAIRS && np + c->pairs.size() > cfg.max_batch_pairs) break;
            batch.push_back(c);
            nq += c->r.n_queries;
            np += c->pairs.size();
          }
          // shrink until it fits next to the running batches
          while (true) {
            est = estimate(batch);
            if (reserved + est <= capacity || batch.size() == 1) break;
            batch.pop_back();
          }
          if (reserved + est <= capacity) break;
          if (running == 0) {   // cannot fit even alone: fail the head request
            head->status = DSA_ERR_OVER_BUDGET;
            head->done = true;
            head->admit = head->finish = now();
            pending.pop_front();
            cv_done.notify_all();
            continue;
          }
        }
        cv_work.wait(lk);
      }
      for (Req* q : batch) pending.erase(std::find(pending.begin(), pending.end(), q));
      reserved += est;
      ++running;
      const double t = now();
      for (Req* q : batch) {
        q->admit = t;
        q->batch_requests = (uint32_t)batch.size();
      }
    }
    run_batch(ctx, batch);
    {
      std::lock_guard<std::mutex> lk(mu);
      reserved -= est;
      --running;
      const double t = now();
      for (Req* q : batch) {
        q->finish = t;
        q->done = true;
      }
    }
    cv_done.notify_all();
    cv_work.notify_all();
  }
}

using namespace dsa;

extern "C" int dsa_server_create(int device, const dsa_server_config* cfg, dsa_server** out) {
  if (!out) { set_error("out is NULL"); return DSA_ERR_INVALID_ARG; }
  *out = nullptr;
  dsa_server* s = new (std::nothrow) dsa_server;
  if (!s) { set_error("host allocation failed"); return DSA_ERR_OOM; }
  s->device = device;
  s->cfg.n_slots = 2;
  s->cfg.max_batch_queries = 64;
  s->cfg.max_batch_pairs = 2000000;
  s->cfg.mem_reserve = 4ull << 30;
  s->cfg.mem_budget = 0;
  s->cfg.max_pending = 100000;
  if (cfg) {
    if (cfg->n_slots) s->cfg.n_slots = cfg->n_slots;
    if (cfg->max_batch_queries) s->cfg.max_batch_queries = cfg->max_batch_queries;
    if (cfg->max_batch_pairs) s->cfg.max_batch_pairs = cfg->max_batch_pairs;
    if (cfg->mem_reserve) s->cfg.mem_reserve = cfg->mem_reserve;
    s->cfg.mem_budget = cfg->mem_budget;
    if (cfg->max_pending) s->cfg.max_pending = cfg->max_pending;
  }
  if (s->cfg.n_slots > 16) s->cfg.n_slots = 16;
  for (uint32_t k = 0; k < s->cfg.n_slots; ++k) {
    dsa_ctx* c = nullptr;
    int rc = dsa_create(&c, device, 0, nullptr);
    if (rc) {
      for (dsa_ctx* x : s->slots) dsa_destroy(x);
      delete s;
      return rc;
    }
    c->tune = false;   // requests use cached tuning decisions only: no tuning passes in a request
    s->slots.push_back(c);
  }
  s->sm_count = s->slots[0]->sm_count;
  size_t free_b = 0, total_b = 0;
  cudaSetDevice(device);
  cudaMemGetInfo(&free_b, &total_b);
  s->capacity = s->cfg.mem_budget ? s->cfg.mem_budget
                                  : (free_b > s->cfg.mem_reserve ? free_b - s->cfg.mem_reserve : 0);
  s->t0 = std::chrono::steady_clock::now();
  for (uint32_t k = 0; k < s->cfg.n_slots; ++k) s->workers.emplace_back(&dsa_server::worker, s, (int)k);
  *out = s;
  return DSA_OK;
}

extern "C" int dsa_submit(dsa_server* srv, const dsa_request* req, uint64_t* ticket) {
  if (!srv || !req || !ticket || !req->db || !req->q_codes || !req->q_offsets ||
      req->n_queries == 0 || !req->matrix) {
    set_error("dsa_submit: NULL argument or empty request");
    return DSA_ERR_INVALID_ARG;
  }
  if (req->kind != DSA_REQ_SEARCH && req->kind != DSA_REQ_PAIRS) {
    set_error("dsa_submit: unknown request kind %d", req->kind);
    return DSA_ERR_INVALID_ARG;
  }
  if (req->kind == DSA_REQ_PAIRS && (!req->pairs || req->n_pairs == 0)) {
    set_error("dsa_submit: a pairs request needs pairs");
    return DSA_ERR_INVALID_ARG;
  }
  Req* q = new (std::nothrow) Req;
  if (!q) { set_error("host allocation failed"); return DSA_ERR_OOM; }
  q->r = *req;
  const uint64_t base = req->q_offsets[0];
  const uint64_t total = req->q_offsets[req->n_queries] - base;
  q->q_codes.assign(req->q_codes + base, req->q_codes + base + total);
  q->q_off.resize(req->n_queries + 1);
  for (uint32_t k = 0; k <= req->n_queries; ++k) q->q_off[k] = req->q_offsets[k] - base;
  if (req->kind == DSA_REQ_PAIRS) {
    q->pairs.assign(req->pairs, req->pairs + req->n_pairs);
    for (const dsa_pair& p : q->pairs)
      if (p.query_id >= req->n_queries) {
        delete q;
        set_error("dsa_submit: pair query_id out of range");
        return DSA_ERR_INVALID_ARG;
      }
  }
  q->matrix.assign(req->matrix, req->matrix + req->alphabet_size * req->alphabet_size);
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->pending.size() >= srv->cfg.max_pending) {
      delete q;
      set_error("dsa_submit: %u requests pending", srv->cfg.max_pending);
      return DSA_ERR_BUSY;
    }
    q->ticket = srv->next_ticket++;
    q->arrive = srv->now();
    srv->pending.push_back(q);
    srv->reqs[q->ticket] = q;
    *ticket = q->ticket;
  }
  srv->cv_work.notify_one();
  return DSA_OK;
}

extern "C" int dsa_poll(dsa_server* srv, uint64_t ticket, dsa_res** out, dsa_request_times* times) {
  if (!srv || !out) { set_error("NULL argument"); return DSA_ERR_INVALID_ARG; }
  *out = nullptr;
  std::lock_guard<std::mutex> lk(srv->mu);
  auto it = srv->reqs.find(ticket);
  if (it == srv->reqs.end()) { set_error("unknown ticket %llu", (unsigned long long)ticket); return DSA_ERR_INVALID_ARG; }
  Req* q = it->second;
  if (!q->done) return DSA_ERR_BUSY;
  if (times) {
    times->arrive = q->arrive;
    times->admit = q->admit;
    times->finish = q->finish;
    times->batch_requests = q->batch_requests;
    times->status = q->status;
  }
  const int st = q->status;
  *out = q->result;
  srv->reqs.erase(it);
  delete q;
  if (st != DSA_OK) set_error("request failed with status %d", st);
  return st;
}

extern "C" int dsa_server_drain(dsa_server* srv) {
  if (!srv) { set_error("NULL argument"); return DSA_ERR_INVALID_ARG; }
  std::unique_lock<std::mutex> lk(srv->mu);
  srv->cv_done.wait(lk, [&] { return srv->pending.empty() && srv->running == 0; });
  return DSA_OK;
}

extern "C" double dsa_server_now(const dsa_server* srv) { return srv ? srv->now() : 0.0; }

extern "C" int dsa_server_destroy(dsa_server* srv) {
  if (!srv) return DSA_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  for (std::thread& t : srv->workers) t.join();
  for (auto& kv : srv->reqs) {
    if (kv.second->result) dsa_res_free(kv.second->result);
    delete kv.second;
  }
  for (dsa_ctx* c : srv->slots) dsa_destroy(c);
  delete srv;
  return DSA_OK;
}
