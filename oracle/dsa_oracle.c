/*
 * CPU oracle for Gotoh affine-gap alignment -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  The product path (the CUDA library) never calls it and
 * shares no code, header, table or helper with it.
 *
 * What it computes.  The paper (Sec. II.B.1) aligns every query against every
 * reference sequence with local (SSW), global and semi-global (Parasail)
 * dynamic programming and returns, per alignment, the maximum score, the
 * location and the CIGAR (Sec. II.B.1, alignment object; Sec. II.C.2: DSW,
 * DNW, DSG).  It prints no recurrence, so this file is the textbook Gotoh DP
 * under the following readings (the library's documented conventions):
 *
 *   gap cost   a run of k gap columns costs  o + (k-1)*e,  0 <= e <= o
 *   E[i][j] = max(E[i][j-1] - e, H[i][j-1] - o)       gap in query  (CIGAR D)
 *   F[i][j] = max(F[i-1][j] - e, H[i-1][j] - o)       gap in target (CIGAR I)
 *   H[i][j] = max(H[i-1][j-1] + S[q_i][t_j], E[i][j], F[i][j] [, 0 if local])
 *   E[i][0] = F[0][j] = -inf;  H[0][0] = 0
 *   local:       H[i][0] = H[0][j] = 0
 *   global:      H[i][0] = -(o+(i-1)e), H[0][j] = -(o+(j-1)e)
 *   semi-global: as global, but H[0][j] = 0 if the target begin is free and
 *                H[i][0] = 0 if the query begin is free.
 *   result cell: local: max over all cells (0 if none is positive);
 *                global: (m, n);
 *                semi-global: max over row m if the target end is free, over
 *                column n if the query end is free, and (m, n) always.
 *   tie-break:   among optimal result cells, the smallest (j, i).
 *   traceback:   from the result cell in state H; stop > M > I > D; a gap is
 *                taken as "opened here" whenever opening ties extending.
 *
 * Arithmetic is plain int32 with -inf = INT32_MIN/4; arguments are rejected
 * when (m+n)*max(|S|, o, e) could reach 2^29.
 *
 * Rows of S are query residues, columns target residues: S[q*A + t].
 *
 * Position-specific form (the user-defined scoring of Sec. II.C.2): a query
 * may instead be given as a profile P of m rows of A scores, and the
 * substitution term of cell (i, j) is P[i-1][t_j] in place of S[q_i][t_j];
 * everything else is unchanged (oracle_score_pssm, oracle_score_pairs_pssm).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORC_NEG_INF (INT32_MIN / 4)

enum { ORC_LOCAL = 0, ORC_GLOBAL = 1, ORC_SEMIGLOBAL = 2 };
enum { ORC_FREE_Q_BEGIN = 1, ORC_FREE_Q_END = 2, ORC_FREE_T_BEGIN = 4, ORC_FREE_T_END = 8 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };
enum { OP_M = 0, OP_I = 1, OP_D = 2 };

static int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }

static int is_free(int mode, uint32_t fe, uint32_t bit) {
  return mode == ORC_SEMIGLOBAL && (fe & bit);
}

/* H in row 0 (no query residue consumed) at column j. */
static int32_t h_row0(int mode, uint32_t fe, int64_t j, int32_t o, int32_t e) {
  if (j == 0 || mode == ORC_LOCAL || is_free(mode, fe, ORC_FREE_T_BEGIN)) return 0;
  return -(o + (int32_t)(j - 1) * e);
}

/* H in column 0 (no target residue consumed) at row i. */
static int32_t h_col0(int mode, uint32_t fe, int64_t i, int32_t o, int32_t e) {
  if (i == 0 || mode == ORC_LOCAL || is_free(mode, fe, ORC_FREE_Q_BEGIN)) return 0;
  return -(o + (int32_t)(i - 1) * e);
}

static int check_args(int64_t m, int64_t n, const int8_t* S, int A, int32_t o, int32_t e,
                      int mode) {
  if (m < 1 || n < 1 || A < 1 || A > 256 || o < 0 || e < 0 || e > o) return ORC_EINVAL;
  if (mode < 0 || mode > 2) return ORC_EINVAL;
  int32_t smax = 0;
  for (int k = 0; k < A * A; ++k) {
    int32_t v = S[k] < 0 ? -S[k] : S[k];
    if (v > smax) smax = v;
  }
  int64_t w = smax > o ? smax : o;
  if (e > w) w = e;
  if ((m + n + 2) * (w + 1) >= ((int64_t)1 << 29)) return ORC_EINVAL;
  return ORC_OK;
}

/* Candidate update with the (score desc, j asc, i asc) order. */
static void offer(int32_t h, int64_t i, int64_t j, int32_t* best, int64_t* bi, int64_t* bj,
                  int* have) {
  if (!*have || h > *best || (h == *best && (j < *bj || (j == *bj && i < *bi)))) {
    *best = h; *bi = i; *bj = j; *have = 1;
  }
}

/* Largest |value| of a position-specific score profile (m rows of A). */
static int check_pssm(int64_t m, int64_t n, const int8_t* P, int A, int32_t o, int32_t e,
                      int mode) {
  if (m < 1 || n < 1 || A < 1 || A > 256 || o < 0 || e < 0 || e > o) return ORC_EINVAL;
  if (mode < 0 || mode > 2) return ORC_EINVAL;
  int32_t smax = 0;
  for (int64_t k = 0; k < m * A; ++k) {
    int32_t v = P[k] < 0 ? -P[k] : P[k];
    if (v > smax) smax = v;
  }
  int64_t w = smax > o ? smax : o;
  if (e > w) w = e;
  if ((m + n + 2) * (w + 1) >= ((int64_t)1 << 29)) return ORC_EINVAL;
  return ORC_OK;
}

/*
 * Score pass of one pair, the DP shared by the matrix and the profile forms:
 * the substitution row of query position i is S[q_i] (P == NULL) or the
 * profile's row i, P[i] (the position-specific scores of the user-defined
 * scoring extension, Sec. II.C.2).
 */
static int score_core(const uint8_t* q, const int8_t* S, const int8_t* P, int64_t m,
                      const uint8_t* t, int64_t n, int A, int32_t o, int32_t e, int mode,
                      uint32_t fe, int32_t* score, int32_t* q_end, int32_t* t_end) {
  int32_t* H = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
  int32_t* F = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
  if (!H || !F) { free(H); free(F); return ORC_ENOMEM; }

  int32_t best = 0; int64_t bi = -1, bj = -1; int have = 0;
  int t_end_free = is_free(mode, fe, ORC_FREE_T_END);
  int q_end_free = is_free(mode, fe, ORC_FREE_Q_END);

  for (int64_t j = 0; j <= n; ++j) { H[j] = h_row0(mode, fe, j, o, e); F[j] = ORC_NEG_INF; }
  if (mode == ORC_SEMIGLOBAL && q_end_free) offer(H[n], 0, n, &best, &bi, &bj, &have);

  for (int64_t i = 1; i <= m; ++i) {
    int32_t diag = H[0];                 /* H[i-1][0] */
    H[0] = h_col0(mode, fe, i, o, e);    /* H[i][0]   */
    int32_t E = ORC_NEG_INF;             /* E[i][0]   */
    const int8_t* Srow = P ? P + (size_t)(i - 1) * A : S + (size_t)q[i - 1] * A;
    for (int64_t j = 1; j <= n; ++j) {
      E = imax(E - e, H[j - 1] - o);              /* H[j-1] holds H[i][j-1] */
      int32_t f = imax(F[j] - e, H[j] - o);       /* H[j] still holds H[i-1][j] */
      int32_t h = imax(diag + Srow[t[j - 1]], imax(E, f));
      if (mode == ORC_LOCAL && h < 0) h = 0;
      diag = H[j];
      H[j] = h;
      F[j] = f;
      if (mode == ORC_LOCAL && h > 0) offer(h, i, j, &best, &bi, &bj, &have);
    }
    if (mode == ORC_SEMIGLOBAL && q_end_free) offer(H[n], i, n, &best, &bi, &bj, &have);
    if (i == m) {
      if (mode == ORC_GLOBAL) offer(H[n], m, n, &best, &bi, &bj, &have);
      if (mode == ORC_SEMIGLOBAL) {
        offer(H[n], m, n, &best, &bi, &bj, &have);
        if (t_end_free)
          for (int64_t j = 0; j <= n; ++j) offer(H[j], m, j, &best, &bi, &bj, &have);
      }
    }
  }
  free(H); free(F);
  if (mode == ORC_LOCAL && !have) { *score = 0; *q_end = -1; *t_end = -1; return ORC_OK; }
  *score = best; *q_end = (int32_t)(bi - 1); *t_end = (int32_t)(bj - 1);
  return ORC_OK;
}

/*
 * Score pass: optimal score and result cell of one pair.
 * Outputs 0-based inclusive ends (q_end = i-1, t_end = j-1 of the 1-based
 * result cell); local alignments with score 0 report ends -1.
 */
int oracle_score(const uint8_t* q, int64_t m, const uint8_t* t, int64_t n,
                 const int8_t* S, int A, int32_t o, int32_t e, int mode, uint32_t fe,
                 int32_t* score, int32_t* q_end, int32_t* t_end) {
  int rc = check_args(m, n, S, A, o, e, mode);
  if (rc) return rc;
  return score_core(q, S, NULL, m, t, n, A, o, e, mode, fe, score, q_end, t_end);
}

/*
 * Score pass of a query given as a position-specific profile: P holds m rows
 * of A int8 scores, P[i * A + a] for query position i against target residue
 * a.  Same outputs as oracle_score.
 */
int oracle_score_pssm(const int8_t* P, int64_t m, const uint8_t* t, int64_t n, int A,
                      int32_t o, int32_t e, int mode, uint32_t fe, int32_t* score,
                      int32_t* q_end, int32_t* t_end) {
  int rc = check_pssm(m, n, P, A, o, e, mode);
  if (rc) return rc;
  return score_core(NULL, NULL, P, m, t, n, A, o, e, mode, fe, score, q_end, t_end);
}

/*
 * Traceback from a result cell (q_end, t_end as returned by oracle_score):
 * fills the 0-based begin (number of query/target residues before the aligned
 * region) and the CIGAR as (len << 4 | op) words, op M=0, I=1, D=2, in
 * forward order.  Stores H, E and F for the whole rectangle up to the result
 * cell (12 bytes per cell) and replays the decisions from the values.
 */
int oracle_traceback(const uint8_t* q, int64_t m, const uint8_t* t, int64_t n,
                     const int8_t* S, int A, int32_t o, int32_t e, int mode, uint32_t fe,
                     int32_t q_end, int32_t t_end,
                     int32_t* q_begin, int32_t* t_begin,
                     uint32_t* cigar, int64_t cigar_cap, int64_t* n_ops) {
  int rc = check_args(m, n, S, A, o, e, mode);
  if (rc) return rc;
  *n_ops = 0;
  if (mode == ORC_LOCAL && (q_end < 0 || t_end < 0)) { *q_begin = -1; *t_begin = -1; return ORC_OK; }
  int64_t ie = (int64_t)q_end + 1, je = (int64_t)t_end + 1;   /* 1-based result cell */
  if (ie < 0 || je < 0 || ie > m || je > n) return ORC_EINVAL;
  int64_t W = je + 1;
  size_t cells = (size_t)(ie + 1) * (size_t)W;
  int32_t* H = (int32_t*)malloc(cells * sizeof(int32_t));
  int32_t* Em = (int32_t*)malloc(cells * sizeof(int32_t));
  int32_t* Fm = (int32_t*)malloc(cells * sizeof(int32_t));
  char* ops = (char*)malloc((size_t)(ie + je + 2));
  if (!H || !Em || !Fm || !ops) { free(H); free(Em); free(Fm); free(ops); return ORC_ENOMEM; }
#define AT(M_, i_, j_) M_[(size_t)(i_) * W + (size_t)(j_)]
  for (int64_t j = 0; j <= je; ++j) {
    AT(H, 0, j) = h_row0(mode, fe, j, o, e); AT(Em, 0, j) = ORC_NEG_INF; AT(Fm, 0, j) = ORC_NEG_INF;
  }
  for (int64_t i = 1; i <= ie; ++i) {
    AT(H, i, 0) = h_col0(mode, fe, i, o, e); AT(Em, i, 0) = ORC_NEG_INF; AT(Fm, i, 0) = ORC_NEG_INF;
    for (int64_t j = 1; j <= je; ++j) {
      int32_t E = imax(AT(Em, i, j - 1) - e, AT(H, i, j - 1) - o);
      int32_t F = imax(AT(Fm, i - 1, j) - e, AT(H, i - 1, j) - o);
      int32_t h = imax(AT(H, i - 1, j - 1) + S[(size_t)q[i - 1] * A + t[j - 1]], imax(E, F));
      if (mode == ORC_LOCAL && h < 0) h = 0;
      AT(H, i, j) = h; AT(Em, i, j) = E; AT(Fm, i, j) = F;
    }
  }
  /* Walk back. */
  int64_t i = ie, j = je, k = 0;
  int state = 0; /* 0 = H, 1 = F, 2 = E */
  for (;;) {
    if (state == 0) {
      int32_t v = AT(H, i, j);
      if (mode == ORC_LOCAL && v == 0) break;
      if ((i == 0 && is_free(mode, fe, ORC_FREE_T_BEGIN)) ||
          (j == 0 && is_free(mode, fe, ORC_FREE_Q_BEGIN))) break;
      if (i == 0 || j == 0) {      /* global / semi-global edge: remaining gap run */
        while (j > 0) { ops[k++] = OP_D; --j; }
        while (i > 0) { ops[k++] = OP_I; --i; }
        break;
      }
      if (v == AT(H, i - 1, j - 1) + S[(size_t)q[i - 1] * A + t[j - 1]]) {
        ops[k++] = OP_M; --i; --j;
      } else if (v == AT(Fm, i, j)) {
        state = 1;
      } else {
        state = 2;
      }
    } else if (state == 1) {
      ops[k++] = OP_I;
      if (AT(Fm, i, j) == AT(H, i - 1, j) - o) state = 0;
      --i;
    } else {
      ops[k++] = OP_D;
      if (AT(Em, i, j) == AT(H, i, j - 1) - o) state = 0;
      --j;
    }
  }
#undef AT
  *q_begin = (int32_t)i; *t_begin = (int32_t)j;
  /* reverse and run-length encode */
  int64_t n_out = 0;
  for (int64_t p = k - 1; p >= 0;) {
    char op = ops[p];
    int64_t len = 0;
    while (p >= 0 && ops[p] == op) { ++len; --p; }
    if (n_out < cigar_cap) cigar[n_out] = (uint32_t)(len << 4) | (uint32_t)op;
    ++n_out;
  }
  *n_ops = n_out;
  free(H); free(Em); free(Fm); free(ops);
  return n_out > cigar_cap ? ORC_EINVAL : ORC_OK;
}

/* ---------------- multithreaded batch over explicit pairs ---------------- */

typedef struct {
  const uint8_t* q_codes; const uint64_t* q_off;
  const uint8_t* t_codes; const uint64_t* t_off;
  const uint32_t* pair_q; const uint32_t* pair_t;
  const uint64_t* pair_toff;   /* NULL: whole target sequence */
  const uint32_t* pair_tlen;
  int64_t n_pairs;
  const int8_t* S; int A; int32_t o, e; int mode; uint32_t fe;
  const int8_t* pssm;          /* NULL: matrix S; else rows of every query residue */
  int32_t* score; int32_t* q_end; int32_t* t_end;
  int64_t next; pthread_mutex_t mu; int rc;
} batch_job;

static void* batch_worker(void* arg) {
  batch_job* J = (batch_job*)arg;
  for (;;) {
    pthread_mutex_lock(&J->mu);
    int64_t p = J->next++;
    pthread_mutex_unlock(&J->mu);
    if (p >= J->n_pairs) break;
    uint32_t qi = J->pair_q[p], ti = J->pair_t[p];
    const uint8_t* qs = J->q_codes + J->q_off[qi];
    int64_t m = (int64_t)(J->q_off[qi + 1] - J->q_off[qi]);
    const uint8_t* ts = J->t_codes + J->t_off[ti];
    int64_t n = (int64_t)(J->t_off[ti + 1] - J->t_off[ti]);
    if (J->pair_toff) { ts += J->pair_toff[p]; n = J->pair_tlen[p]; }
    int rc = J->pssm
                 ? oracle_score_pssm(J->pssm + J->q_off[qi] * (uint64_t)J->A, m, ts, n, J->A,
                                     J->o, J->e, J->mode, J->fe, &J->score[p], &J->q_end[p],
                                     &J->t_end[p])
                 : oracle_score(qs, m, ts, n, J->S, J->A, J->o, J->e, J->mode, J->fe,
                                &J->score[p], &J->q_end[p], &J->t_end[p]);
    if (rc) { pthread_mutex_lock(&J->mu); J->rc = rc; pthread_mutex_unlock(&J->mu); }
  }
  return NULL;
}

static int run_batch(batch_job* J, int n_threads);
int oracle_score_pairs_pssm(const uint8_t* q_codes, const uint64_t* q_off,
                            const uint8_t* t_codes, const uint64_t* t_off,
                            const uint32_t* pair_q, const uint32_t* pair_t,
                            const uint64_t* pair_toff, const uint32_t* pair_tlen,
                            int64_t n_pairs, const int8_t* S, const int8_t* pssm, int A,
                            int32_t o, int32_t e, int mode, uint32_t fe, int n_threads,
                            int32_t* score, int32_t* q_end, int32_t* t_end);

int oracle_score_pairs(const uint8_t* q_codes, const uint64_t* q_off,
                       const uint8_t* t_codes, const uint64_t* t_off,
                       const uint32_t* pair_q, const uint32_t* pair_t,
                       const uint64_t* pair_toff, const uint32_t* pair_tlen, int64_t n_pairs,
                       const int8_t* S, int A, int32_t o, int32_t e, int mode, uint32_t fe,
                       int n_threads, int32_t* score, int32_t* q_end, int32_t* t_end) {
  return oracle_score_pairs_pssm(q_codes, q_off, t_codes, t_off, pair_q, pair_t, pair_toff,
                                 pair_tlen, n_pairs, S, NULL, A, o, e, mode, fe, n_threads,
                                 score, q_end, t_end);
}

/* As oracle_score_pairs; with pssm != NULL the queries are position-specific
 * profiles: query residue k of the query set (offsets q_off) has the score
 * row pssm[k * A .. k * A + A - 1], and q_codes is not read. */
int oracle_score_pairs_pssm(const uint8_t* q_codes, const uint64_t* q_off,
                            const uint8_t* t_codes, const uint64_t* t_off,
                            const uint32_t* pair_q, const uint32_t* pair_t,
                            const uint64_t* pair_toff, const uint32_t* pair_tlen,
                            int64_t n_pairs, const int8_t* S, const int8_t* pssm, int A,
                            int32_t o, int32_t e, int mode, uint32_t fe, int n_threads,
                            int32_t* score, int32_t* q_end, int32_t* t_end) {
  batch_job J;
  memset(&J, 0, sizeof(J));
  J.pssm = pssm;
  J.q_codes = q_codes; J.q_off = q_off; J.t_codes = t_codes; J.t_off = t_off;
  J.pair_q = pair_q; J.pair_t = pair_t; J.pair_toff = pair_toff; J.pair_tlen = pair_tlen;
  J.n_pairs = n_pairs; J.S = S; J.A = A; J.o = o; J.e = e; J.mode = mode; J.fe = fe;
  J.score = score; J.q_end = q_end; J.t_end = t_end;
  return run_batch(&J, n_threads);
}

static int run_batch(batch_job* Jp, int n_threads) {
  batch_job J = *Jp;
  pthread_mutex_init(&J.mu, NULL);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 512) n_threads = 512;
  pthread_t th[512];
  for (int k = 0; k < n_threads; ++k) pthread_create(&th[k], NULL, batch_worker, &J);
  for (int k = 0; k < n_threads; ++k) pthread_join(th[k], NULL);
  pthread_mutex_destroy(&J.mu);
  return J.rc;
}
