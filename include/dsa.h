/*
 * dsa.h -- C ABI of libdsa: exact Gotoh affine-gap alignment of query
 * sequences against a device-resident sequence database on one GB300 GPU.
 *
 * The paper (Xu et al., "DSA: Scalable Distributed Sequence Alignment System
 * Using SIMD Instructions") aligns query sequences against reference
 * sequences with a score matrix (Sec. II.B.1), with three algorithms --
 * distributed Smith-Waterman, Needleman-Wunsch and semi-global (Sec. II.C.2)
 * -- returns for each alignment the maximum score, the reference name, the
 * location and the CIGAR (Sec. II.B.1), and reduces the per-partition results
 * to the top K by score (Sec. II.B.2).  This header is that computation as a
 * plain C interface; every step runs in CUDA kernels of this library.
 *
 * Conventions (the paper prints no recurrence; these are the library's
 * definitions, identical to the CPU oracle used to test it):
 *   - residues are small integer codes 0..A-1; S is an A x A int8 matrix,
 *     row-major, rows = query residue, columns = target residue;
 *   - a run of k gap columns costs gap_open + (k-1)*gap_extend, and
 *     0 <= gap_extend <= gap_open (BLAST-style "open o / extend e" with cost
 *     o + k*e is obtained by passing gap_open = o + e);
 *   - H/E/F Gotoh recurrences, local scores floored at 0;
 *   - global boundary H[i][0] = -(o+(i-1)e), H[0][j] = -(o+(j-1)e); in
 *     semi-global mode a free query (target) begin sets H[i][0] (H[0][j]) to 0;
 *   - result cell: local = best cell; global = (m, n); semi-global = best of
 *     row m (target end free), column n (query end free) and (m, n);
 *   - ties between optimal result cells: the smallest target end, then the
 *     smallest query end;
 *   - traceback starts at the result cell; priority stop > M > I > D; a gap
 *     is taken as opened at a cell whenever opening ties extending;
 *   - coordinates are 0-based and inclusive; begin = residues skipped before
 *     the aligned region; a local alignment with score 0 reports -1 for all
 *     coordinates and an empty CIGAR;
 *   - CIGAR words are (run_length << 4) | op with op M = 0, I = 1 (query
 *     residue against a gap), D = 2 (target residue against a gap), in
 *     alignment order; overhangs on free ends are not part of the CIGAR.
 *
 * Ownership: host arrays passed in are copied before the call returns.
 * dsa_db and dsa_res objects own device memory until freed.  All work is
 * ordered on the context's CUDA stream.  No function aborts or throws; each
 * returns DSA_OK (0) or a negative error code, and dsa_last_error() gives the
 * calling thread's last message.
 */
#ifndef DSA_H
#define DSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define DSA_OK 0
#define DSA_ERR_INVALID_ARG (-1)   /* an argument breaks a documented rule */
#define DSA_ERR_OOM (-2)           /* device allocation failed */
#define DSA_ERR_OVER_BUDGET (-3)   /* request exceeds the context's memory budget */
#define DSA_ERR_CUDA (-4)          /* a CUDA runtime call failed */
#define DSA_ERR_DEVICE_TIMEOUT (-5)/* a bounded device-side wait gave up */
#define DSA_ERR_BUSY (-6)          /* serving queue full */
#define DSA_ERR_UNSUPPORTED (-7)   /* valid request this build does not handle */

/* ---- alignment modes (Sec. II.C.2: DSW, DNW, DSG) ---- */
#define DSA_LOCAL 0
#define DSA_GLOBAL 1
#define DSA_SEMIGLOBAL 2

/* ---- semi-global free ends (bit set = that end's overhang is free) ---- */
#define DSA_FREE_Q_BEGIN 1u
#define DSA_FREE_Q_END 2u
#define DSA_FREE_T_BEGIN 4u
#define DSA_FREE_T_END 8u

/* ---- dsa_align_* flags ---- */
#define DSA_RESULTS_ON_DEVICE 1u  /* dsa_res_get returns device pointers */
#define DSA_FORCE_INT32 2u        /* skip the packed 16-bit pass; every pair runs in int32 */
#define DSA_PLAIN_FORM 4u         /* one unbatched int32 launch per query, DB in input order */
#define DSA_PAIRS_ON_DEVICE 8u    /* `pairs` is a device pointer */
#define DSA_TIMING 16u            /* record CUDA events around each phase (dsa_res_timing) */

/* ---- hit flags ---- */
#define DSA_HIT_RERUN_INT32 1u    /* the packed pass saturated; result is from the int32 rerun */
#define DSA_HIT_HAS_TRACEBACK 2u  /* begin coordinates and CIGAR are filled in */

typedef struct dsa_ctx dsa_ctx;
typedef struct dsa_db dsa_db;
typedef struct dsa_res dsa_res;

/* One explicit alignment: query `query_id` against `t_len` residues of
 * sequence `target_id` starting at residue `t_offset` (a window). */
typedef struct {
  uint32_t query_id;
  uint32_t target_id;
  uint64_t t_offset;
  uint32_t t_len;
  uint32_t reserved; /* set to 0; kept for later use, no call reads it */
} dsa_pair;

/* One alignment result (the paper's alignment object, Sec. II.B.1: score,
 * reference name -> target_id, location -> begin/end, CIGAR). */
typedef struct {
  int32_t score;
  int32_t q_begin, q_end;   /* 0-based, inclusive; -1 if none / not traced */
  int32_t t_begin, t_end;   /* relative to the pair's window (t_offset) */
  uint32_t query_id;
  uint32_t target_id;
  uint32_t flags;           /* DSA_HIT_* */
  uint64_t t_offset;        /* window offset of the pair (0 for whole targets) */
  uint64_t cigar_off;       /* index of the first CIGAR word in the result's CIGAR array */
  uint32_t cigar_len;       /* number of CIGAR words */
  uint32_t reserved;
} dsa_hit;

/* Create a context on CUDA device `device`.  `mem_budget_bytes` caps the
 * device memory this context may hold (0 = no cap).  `cuda_stream` is a
 * cudaStream_t to order all work on (NULL = a stream the context creates). */
int dsa_create(dsa_ctx** out, int device, size_t mem_budget_bytes, void* cuda_stream);
int dsa_destroy(dsa_ctx* ctx);

/* Message describing the calling thread's most recent error ("" if none). */
const char* dsa_last_error(void);

/* Bytes of device memory the context currently holds. */
size_t dsa_mem_in_use(const dsa_ctx* ctx);

/* Number of CUDA kernels this context has launched so far. */
uint64_t dsa_kernel_launches(const dsa_ctx* ctx);

/* Load `n_seqs` sequences to the device (the paper's map phase reading the
 * reference set, Sec. II.B.1).  `codes` holds all residues concatenated;
 * sequence k is codes[offsets[k] .. offsets[k+1]).  Every code must be below
 * `alphabet_size` (1..31); every sequence must be non-empty.  The same call
 * loads query sets.  The length-sorted, lane-interleaved copy that the
 * batched all-vs-all kernels read is built on the set's first all-vs-all use
 * (charged to the loading context), so query sets and pair windows never pay
 * for it.  The codes are copied; the caller keeps its arrays. */
int dsa_db_load(dsa_ctx* ctx, const uint8_t* codes, const uint64_t* offsets, uint32_t n_seqs,
                int alphabet_size, dsa_db** out);
int dsa_db_free(dsa_db* db);
int dsa_db_info(const dsa_db* db, uint32_t* n_seqs, uint64_t* n_residues, int* alphabet_size);

/* Align queries against the database (Sec. II.B.1 map phase + Sec. II.B.2 top K).
 *
 * queries: a dsa_db loaded with dsa_db_load (device resident).
 * pairs:   NULL = every query against every target; otherwise `n_pairs`
 *          explicit (query, target window) pairs (host pointer, or device
 *          pointer with DSA_PAIRS_ON_DEVICE).
 * mode / free_ends: DSA_LOCAL, DSA_GLOBAL or DSA_SEMIGLOBAL (+ DSA_FREE_* bits).
 * matrix:  host int8 A x A substitution matrix, A = alphabet_size of both sets.
 * top_k:   0 = one hit per pair (all x all: query-major, target-minor order;
 *          explicit pairs: pair order).  k > 0 = per query the k best targets
 *          ordered by (score desc, target_id asc) -- all x all only.
 * The result holds scores and end coordinates; begin coordinates and CIGARs
 * are filled in by dsa_traceback. */
int dsa_align(dsa_ctx* ctx, const dsa_db* db, const dsa_db* queries, const dsa_pair* pairs,
              uint64_t n_pairs, int mode, uint32_t free_ends, const int8_t* matrix,
              int alphabet_size, int gap_open, int gap_extend, uint32_t top_k, uint32_t flags,
              dsa_res** out);

/* Same as dsa_align with queries given as host arrays (copied to the device
 * inside the call). */
int dsa_align_batch(dsa_ctx* ctx, const dsa_db* db, const uint8_t* q_codes,
                    const uint64_t* q_offsets, uint32_t n_queries, const dsa_pair* pairs,
                    uint64_t n_pairs, int mode, uint32_t free_ends, const int8_t* matrix,
                    int alphabet_size, int gap_open, int gap_extend, uint32_t top_k,
                    uint32_t flags, dsa_res** out);

/* All-vs-all search with position-specific scores (the user-defined scoring
 * extension of Sec. II.C.2, e.g. a PSSM built from a query family): query
 * residue i of query q scores against target residue a with
 * pssm[(o_q + i) * alphabet_size + a], where o_q is the query's offset in
 * the set `queries` was loaded from (so the rows follow the query codes;
 * the codes themselves are not read).  `pssm` is host memory of
 * n_residues(queries) x alphabet_size int8 values, copied during the call.
 * Everything else is as for dsa_align without pairs (modes, free ends, top
 * K, flags; local mode runs the packed int16 kernels with the exact int32
 * rerun, whose range check uses the profile's extreme values).  The result
 * holds scores and end cells only: dsa_traceback on it returns
 * DSA_ERR_UNSUPPORTED. */
int dsa_align_pssm(dsa_ctx* ctx, const dsa_db* db, const dsa_db* queries, const int8_t* pssm,
                   int alphabet_size, int mode, uint32_t free_ends, int gap_open, int gap_extend,
                   uint32_t top_k, uint32_t flags, dsa_res** out);

/* Begin coordinates and CIGAR for hits of `res` (the paper's location +
 * CIGAR, Sec. I and II.B.1).  `which` lists hit indices (host array), NULL =
 * every hit.  Hits with a local score of 0 get no CIGAR.  The DP of each hit
 * is recomputed over the part of its rectangle that every optimal path must
 * cross (bounded from the hit's score), storing 4-bit decisions, and walked
 * back with the tie rules stop > M > I > D, gap opening preferred; results
 * are identical to a walk over the full rectangle. */
int dsa_traceback(dsa_ctx* ctx, dsa_res* res, const uint64_t* which, uint64_t n);

/* Access results.  Without DSA_RESULTS_ON_DEVICE the arrays are host copies
 * owned by `res` (the call synchronizes the stream); with it they are device
 * pointers.  `cigar` holds all CIGAR words; hit.cigar_off indexes it.  A
 * hit's words are contiguous; the order of different hits' words in the
 * array is unspecified (large batches are laid out in work order). */
int dsa_res_get(dsa_res* res, const dsa_hit** hits, uint64_t* n_hits, const uint32_t** cigar,
                uint64_t* n_cigar_words);
/* DP cells of the score pass (sum over pairs of m*n) and the number of pairs
 * whose packed 16-bit pass saturated and were rerun in int32. */
int dsa_res_stats(const dsa_res* res, uint64_t* cells, uint64_t* n_rerun);
/* Device time in milliseconds of each phase of a result made with DSA_TIMING,
 * measured with CUDA events on the context's stream (call after dsa_sync):
 * ms[0] packed inter-sequence kernel, ms[1] long-target wavefront kernel,
 * ms[2] exact int32 kernels (int32 path or saturation rerun), ms[3] top-k /
 * hit assembly, ms[4] traceback (all dsa_traceback calls).  Phases that did
 * not run report -1.  `n` is the length of `ms` (at most 5 are written). */
int dsa_res_timing(const dsa_res* res, double* ms, int n);
/* DP cells computed in each of the phases above (same order; 0 if none). */
int dsa_res_phase_cells(const dsa_res* res, uint64_t* cells, int n);
int dsa_res_free(dsa_res* res);

/* Wait for all queued work of the context; returns a device-side status if
 * a kernel reported one (e.g. DSA_ERR_DEVICE_TIMEOUT). */
int dsa_sync(dsa_ctx* ctx);

/* Issue-rate probe used for the roofline denominator: runs a throughput
 * microbenchmark of one instruction form on the context's device and
 * returns warp-instructions per SM per clock.  form: 0 = s16x2 add-max
 * (DPX), 1 = s16x2 max with ReLU (DPX), 2 = s16x2 three-way max (DPX),
 * 3 = int32 add, 4 = int32 max, 5 = s16x2 add (SIMD video), 6 = int32
 * add-max (DPX), 7 = the packed local cell update mix (5 instructions per
 * two cells), 8 = u8x4 max, 9 = u8x4 saturating add, 10 = u8x4 saturating
 * subtract (the packed-byte SIMD intrinsics), 11 = an 8-bit biased unsigned
 * local cell update (10 intrinsics per four cells), counted per intrinsic
 * call.  Returns DSA_ERR_INVALID_ARG for another form. */
int dsa_probe_issue_rate(dsa_ctx* ctx, int form, double* warp_instr_per_sm_per_clk);

/* Self-test of the device-side failure path (no fault is raised): enqueues a
 * kernel whose wait can never be satisfied -- kind 0 an mbarrier whose
 * transaction bytes never arrive, kind 1 a progress flag nobody publishes --
 * with a wait limit of `limit_ns` nanoseconds (at most 10 s).  The kernel
 * gives up, records DSA_ERR_DEVICE_TIMEOUT in the context's status word and
 * returns; the next dsa_sync reports that status and clears it, and the
 * context stays usable.  These are the waits the kernels use for their TMA
 * profile copies and for the long-pair band pipeline. */
int dsa_selftest_wait_timeout(dsa_ctx* ctx, int kind, uint64_t limit_ns);

/* ---- serving: continuous batching of alignment requests ----
 *
 * A server owns `n_slots` worker slots, each with its own stream.  Submitted
 * requests wait in a FIFO; a free slot takes the oldest pending request and
 * every later pending request compatible with it (same database, kind and
 * scoring) up to the batch limits, provided the batch's estimated device
 * footprint fits in the free memory (cudaMemGetInfo minus `mem_reserve`, or
 * `mem_budget` if non-zero) next to what running batches reserved; it then
 * runs them as one dsa_align (+ dsa_traceback) call.  Batches of different
 * slots overlap on the device.  Each request's results are identical to
 * those it gets alone: scores are exact and top-k uses a total order. */
typedef struct dsa_server dsa_server;

#define DSA_REQ_SEARCH 0   /* queries vs every target of `db`, top_k hits per query */
#define DSA_REQ_PAIRS 1    /* explicit (query, target window) pairs, one hit per pair */

typedef struct {
  int kind;                       /* DSA_REQ_SEARCH or DSA_REQ_PAIRS */
  const dsa_db* db;
  const uint8_t* q_codes;         /* host; copied by dsa_submit */
  const uint64_t* q_offsets;
  uint32_t n_queries;
  const dsa_pair* pairs;          /* host, DSA_REQ_PAIRS; query_id is request-local */
  uint64_t n_pairs;
  int mode;
  uint32_t free_ends;
  const int8_t* matrix;           /* host, alphabet_size^2; copied */
  int alphabet_size;
  int gap_open, gap_extend;
  uint32_t top_k;                 /* DSA_REQ_SEARCH */
  int traceback;                  /* non-zero: begin coordinates and CIGARs */
} dsa_request;

typedef struct {
  uint32_t n_slots;               /* concurrent batches (default 2) */
  uint32_t max_batch_queries;     /* DSA_REQ_SEARCH batch limit (default 64) */
  uint64_t max_batch_pairs;       /* DSA_REQ_PAIRS batch limit (default 2,000,000) */
  size_t mem_reserve;             /* bytes kept free (default 4 GiB) */
  size_t mem_budget;              /* if non-zero: total bytes batches may reserve */
  uint32_t max_pending;           /* dsa_submit returns DSA_ERR_BUSY beyond this (default 100000) */
} dsa_server_config;

/* Times of one request, in seconds on the server's clock: arrival (submit),
 * admission (its batch started) and finish (results on the host). */
typedef struct {
  double arrive, admit, finish;
  uint32_t batch_requests;        /* requests in its batch */
  int status;                     /* DSA_OK or the batch's error */
} dsa_request_times;

int dsa_server_create(int device, const dsa_server_config* cfg, dsa_server** out);
int dsa_submit(dsa_server* srv, const dsa_request* req, uint64_t* ticket);
/* DSA_OK and *out = the request's result (host arrays, request-local query
 * ids; free with dsa_res_free) once it is done; DSA_ERR_BUSY while it is not.
 * A finished request is handed out once. */
int dsa_poll(dsa_server* srv, uint64_t ticket, dsa_res** out, dsa_request_times* times);
/* Block until every submitted request has finished. */
int dsa_server_drain(dsa_server* srv);
/* Seconds on the server's clock (the clock of dsa_request_times). */
double dsa_server_now(const dsa_server* srv);
int dsa_server_destroy(dsa_server* srv);

/* Exact int32 scores and end cells of explicit pairs, allocating nothing.
 *
 * The paper has no counterpart to this entry point: it exists for callers
 * that cannot allocate device memory -- an application that gives every byte
 * of device memory to its own pool, a latency-critical serving thread that
 * may not block on the device allocator, or code recording work while
 * allocation is not permitted.  Every input and output is device memory the
 * caller owns: query and target codes with their uint64 offsets (sequence k
 * = codes[offsets[k] .. offsets[k+1])), `n_pairs` dsa_pair records, the
 * A x A int8 matrix, and three int32 output arrays of `n_pairs` entries
 * (score, q_end, t_end, as dsa_align reports them for explicit pairs).  The
 * call works on the current CUDA device and enqueues one kernel on
 * `cuda_stream` (NULL = the legacy default stream); it does not synchronize.
 *
 * Scratch: the query strips' boundary rows live in a fixed 32 MiB array
 * inside the library (one per device that loads the library, held until the
 * process exits).  `max_t_len`, an upper bound on every pair's t_len, must
 * be at most 32768; larger values return DSA_ERR_INVALID_ARG.  The first
 * call on each device looks up that array's device address (with the device
 * current); make that first call before any stream capture.  Every call
 * shares the array and no part of it needs to start at zero (each pair
 * writes its boundary row before reading it), so calls whose kernels overlap
 * on the GPU race on it: order them on one stream or synchronize between
 * them.  The looked-up address belongs to the device's primary context and
 * is kept for the life of the process: after a cudaDeviceReset of a device
 * this entry point must not be called on that device again.  A pair whose
 * ids, window, lengths or codes are out of range gets score INT32_MIN and
 * ends -2 instead of a result; its `reserved` field is not read. */
int dsa_score_pairs_noalloc(const uint8_t* d_q_codes, const uint64_t* d_q_offsets,
                            uint32_t n_queries, const uint8_t* d_t_codes,
                            const uint64_t* d_t_offsets, uint32_t n_targets,
                            const dsa_pair* d_pairs, uint64_t n_pairs, int mode,
                            uint32_t free_ends, const int8_t* d_matrix, int alphabet_size,
                            int gap_open, int gap_extend, uint32_t max_t_len, int32_t* d_score,
                            int32_t* d_q_end, int32_t* d_t_end, void* cuda_stream);

/* ---- partition + reduce of top-K searches (Sec. II.B.2) ----
 *
 * The paper keeps the top K of every database partition and reduces those
 * lists to the top K of the whole database.  Under the library's total order
 * (score descending, then target id ascending) the reduce of exact
 * per-partition lists equals one search of the whole database, so a
 * database larger than the device or the context's budget can be searched
 * one partition at a time, and lists from several devices merge the same
 * way. */

/* Merge `n_parts` top-K hit lists (host arrays) of the same `n_queries`
 * queries against consecutive partitions of one database.  part_hits[p]
 * holds part_n_hits[p] hits, query-major, part_n_hits[p] / n_queries per
 * query in rank order (the layout dsa_res_get gives for a top-K search);
 * their target ids are partition-local and target_base[p], the global id of
 * the partition's first target, is added.  part_cigar[p] holds the
 * partition's CIGAR words (may be NULL when no hit of it is traced).
 * Output: out_hits (caller-allocated, n_queries * k entries) receives per
 * query the best min(k, sum of the per-query list lengths) hits in rank
 * order with global target ids; out_cigar (caller-allocated, at least the
 * sum of the inputs' cigar_len, or NULL when nothing is traced) receives
 * their CIGAR words, re-indexed by cigar_off.  Lists out of order, hits of
 * the wrong query, or traced hits without CIGAR arrays are
 * DSA_ERR_INVALID_ARG. */
int dsa_merge_topk(const dsa_hit* const* part_hits, const uint64_t* part_n_hits,
                   const uint32_t* const* part_cigar, const uint32_t* target_base,
                   uint32_t n_parts, uint32_t n_queries, uint32_t k, dsa_hit* out_hits,
                   uint64_t* out_n_hits, uint32_t* out_cigar, uint64_t* out_n_cigar);

/* Top-K search of device-resident `queries` against a host database
 * (`codes`, `offsets`, `n_seqs` sequences as for dsa_db_load) too large to
 * hold at once: consecutive targets are loaded `partition_residues` residues
 * at a time (at least one target per partition; 0 = one partition), each
 * partition is searched (and, if `traceback` is non-zero, traced) on the
 * context's stream and freed, and the lists are merged with dsa_merge_topk.
 * The result is host-only (dsa_res_get gives host arrays; it cannot be
 * traced further) and holds the same hits and CIGARs as one dsa_align +
 * dsa_traceback over the whole database; dsa_res_stats gives the summed
 * cells and reruns. */
int dsa_search_partitioned(dsa_ctx* ctx, const uint8_t* codes, const uint64_t* offsets,
                           uint32_t n_seqs, int alphabet_size, uint64_t partition_residues,
                           const dsa_db* queries, int mode, uint32_t free_ends,
                           const int8_t* matrix, int gap_open, int gap_extend, uint32_t top_k,
                           int traceback, dsa_res** out);

/* ---- sequence ingest: FASTA / FASTQ text to residue codes (host) ----
 *
 * The paper's data-format API converts the common sequence file formats to
 * its internal representation before alignment (Sec. II.C.1); these calls do
 * that for FASTA and FASTQ (the paper's third format, ADAM, belongs to its
 * JVM ecosystem and is not read), streaming, on the host, and produce exactly the
 * (codes, offsets) arrays dsa_db_load and dsa_align_batch take.
 *
 * Format: each record starts at a line whose first character is '>' (FASTA)
 * or '@' (FASTQ); the rest of that line is the record's name.  FASTA
 * sequence lines run to the next '>' line; FASTQ sequence lines run to a
 * line starting with '+', followed by quality lines of exactly as many
 * characters as the sequence (so a quality line may itself start with '@'
 * or '+'); qualities are checked for length only and not kept.  Lines end
 * in "\n" or "\r\n"; blank lines between records and spaces or tabs inside
 * sequence lines are ignored; residues are case-insensitive.
 *
 * Alphabets (code = position in the string):
 *   DSA_ALPHABET_DNA4    "ACGT"   (U reads as T)
 *   DSA_ALPHABET_DNA5    "ACGTN"  (U reads as T; the IUPAC ambiguity codes
 *                                  R Y S W K M B D H V read as N)
 *   DSA_ALPHABET_PROTEIN "ARNDCQEGHILKMFPSTWYVBZX*" (the NCBI BLOSUM62
 *                                  order; U, O and J read as X)
 * Any other character in a sequence line is an error (DSA_ERR_INVALID_ARG,
 * message with the line number) unless DSA_READ_MAP_UNKNOWN is given, which
 * reads it as the alphabet's catch-all code: N for DNA5, X for protein, and
 * A (code 0) for DNA4, which has none.
 * A record with no residues is kept as an empty sequence (dsa_db_load
 * refuses empty sequences) unless DSA_READ_SKIP_EMPTY is given. */
#define DSA_ALPHABET_DNA4 1
#define DSA_ALPHABET_DNA5 2
#define DSA_ALPHABET_PROTEIN 3
#define DSA_READ_MAP_UNKNOWN 1u
#define DSA_READ_SKIP_EMPTY 2u

typedef struct dsa_reader dsa_reader;
typedef struct dsa_seqs dsa_seqs;

/* Open a reader over the file at `path` (read in chunks of `chunk_bytes`,
 * 0 = 4 MiB) or over `len` bytes of text at `data` (not copied: the buffer
 * must stay valid until dsa_reader_close).  `alphabet` is a
 * DSA_ALPHABET_* value, `flags` DSA_READ_* bits. */
int dsa_reader_open(const char* path, int alphabet, uint32_t flags, uint64_t chunk_bytes,
                    dsa_reader** out);
int dsa_reader_open_mem(const char* data, uint64_t len, int alphabet, uint32_t flags,
                        dsa_reader** out);
/* Parse the next batch of whole records: records are added while the batch
 * holds at most `max_residues` residues and `max_seqs` records (0 = no
 * limit), and a batch holds at least one record even if that record alone
 * is larger.  *out = NULL at the end of the input.  After an error the
 * reader stays at the failing record and every later call returns the same
 * error. */
int dsa_reader_next(dsa_reader* r, uint64_t max_residues, uint32_t max_seqs, dsa_seqs** out);
int dsa_reader_close(dsa_reader* r);

/* The arrays of a parsed batch, owned by it: `codes` (offsets[n_seqs]
 * residues), `offsets` (n_seqs + 1 entries, record k = codes[offsets[k] ..
 * offsets[k+1])), the names concatenated in `names` with `name_offsets`
 * (n_seqs + 1 entries; names are not NUL-terminated), and the 1-based line
 * number of each record's header in `lines` (n_seqs entries).  Any output
 * pointer may be NULL. */
int dsa_seqs_get(const dsa_seqs* s, const uint8_t** codes, const uint64_t** offsets,
                 uint32_t* n_seqs, const char** names, const uint64_t** name_offsets,
                 const uint64_t** lines);
int dsa_seqs_free(dsa_seqs* s);

#ifdef __cplusplus
}
#endif
#endif /* DSA_H */
