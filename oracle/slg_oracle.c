/*
 * CPU oracle for s-overlaps and s-line graphs.  TEST INFRASTRUCTURE ONLY:
 * it is called by the tests, by the harness smoke check and by the
 * benchmark's CPU-baseline leg, never by the library's product path.  It
 * shares no code with the CUDA library.
 *
 * What it computes (Section III, definition of the s-line graph): for the
 * hyperedges e_0..e_{m-1} of H (rows of the CSR incidence), every pair (i, j)
 * with i < j and w_ij = |e_i ∩ e_j| >= s, listed in ascending (i, j) order.
 *
 * How (Section IV-B, Algorithm 2 restricted to the strictly upper triangle as
 * in Algorithm 3): for each hyperedge e, visit every wedge e -> v -> f with
 * v in e and f in N(v), f > e, and add one to a count kept for f.  Because
 * each row lists a vertex at most once, the count of f after the walk is
 * exactly |e ∩ f|.  No pruning heuristic is applied (no size filter, no
 * early stop), so the oracle checks those heuristics rather than relying on
 * them.  The vertex -> hyperedge lists N(v) are rebuilt here from the CSR by
 * a counting transpose, independently of any CSC a caller may hold.
 *
 * Parallel form (Section IV-F): rows are split into contiguous chunks handed
 * to threads; each chunk keeps its own output, and the chunks are
 * concatenated in row order.  Each thread owns its count array (the paper's
 * thread-local "visited" array, holding counts instead of flags).
 */
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t *i, *j, *w;
  int64_t n, cap;
  int failed;
} triples;

static int push(triples *t, int32_t i, int32_t j, int32_t w) {
  if (t->n == t->cap) {
    int64_t cap = t->cap ? 2 * t->cap : 1024;
    int32_t *a = realloc(t->i, (size_t)cap * sizeof(int32_t));
    if (!a) return -1;
    t->i = a;
    a = realloc(t->j, (size_t)cap * sizeof(int32_t));
    if (!a) return -1;
    t->j = a;
    a = realloc(t->w, (size_t)cap * sizeof(int32_t));
    if (!a) return -1;
    t->w = a;
    t->cap = cap;
  }
  t->i[t->n] = i;
  t->j[t->n] = j;
  t->w[t->n] = w;
  t->n++;
  return 0;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

typedef struct {
  /* hypergraph */
  int32_t m, n;
  const int32_t *e_off, *e_idx;
  int32_t *v_off, *v_idx; /* the oracle's own transpose */
  int32_t s;
  /* rows to process: rows[0..n_rows) or 0..m-1 when rows == NULL */
  const int32_t *rows;
  int64_t n_rows;
  /* chunking */
  int64_t chunk;
  int64_t n_chunks;
  atomic_llong next_chunk;
  triples *out; /* one per chunk */
  int64_t wedges; /* total wedges visited (f > e), summed at the end */
  atomic_llong wedges_acc;
  int failed;
} job;

/* One hyperedge e: count every wedge e -> v -> f (f > e), then report the f
 * whose count reached s, in ascending f. */
static int64_t overlap_row(const job *J, int32_t e, int32_t *cnt,
                           int32_t *touched, triples *out) {
  int64_t n_touched = 0, wedges = 0;
  for (int32_t k = J->e_off[e]; k < J->e_off[e + 1]; ++k) {
    int32_t v = J->e_idx[k];
    for (int32_t q = J->v_off[v]; q < J->v_off[v + 1]; ++q) {
      int32_t f = J->v_idx[q];
      if (f <= e) continue; /* strictly upper triangle, no self-loop */
      ++wedges;
      if (cnt[f]++ == 0) touched[n_touched++] = f;
    }
  }
  qsort(touched, (size_t)n_touched, sizeof(int32_t), cmp_i32);
  for (int64_t t = 0; t < n_touched; ++t) {
    int32_t f = touched[t];
    if (cnt[f] >= J->s && push(out, e, f, cnt[f]) != 0) out->failed = 1;
    cnt[f] = 0;
  }
  return wedges;
}

static void *worker(void *arg) {
  job *J = (job *)arg;
  int32_t *cnt = calloc((size_t)J->m + 1, sizeof(int32_t));
  int32_t *touched = malloc(((size_t)J->m + 1) * sizeof(int32_t));
  if (!cnt || !touched) {
    J->failed = 1;
    free(cnt);
    free(touched);
    return NULL;
  }
  int64_t wedges = 0;
  for (;;) {
    int64_t c = atomic_fetch_add(&J->next_chunk, 1);
    if (c >= J->n_chunks) break;
    int64_t lo = c * J->chunk, hi = lo + J->chunk;
    if (hi > J->n_rows) hi = J->n_rows;
    for (int64_t r = lo; r < hi; ++r) {
      int32_t e = J->rows ? J->rows[r] : (int32_t)r;
      wedges += overlap_row(J, e, cnt, touched, &J->out[c]);
    }
  }
  atomic_fetch_add(&J->wedges_acc, wedges);
  free(cnt);
  free(touched);
  return NULL;
}

/* Counting transpose of the CSR: N(v) ascending for every vertex v. */
static int transpose(job *J, int64_t nnz) {
  J->v_off = calloc((size_t)J->n + 1, sizeof(int32_t));
  J->v_idx = malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
  int32_t *fill = malloc(((size_t)J->n + 1) * sizeof(int32_t));
  if (!J->v_off || !J->v_idx || !fill) {
    free(fill);
    return -1;
  }
  for (int64_t k = 0; k < nnz; ++k) J->v_off[J->e_idx[k] + 1]++;
  for (int32_t v = 0; v < J->n; ++v) J->v_off[v + 1] += J->v_off[v];
  memcpy(fill, J->v_off, ((size_t)J->n + 1) * sizeof(int32_t));
  for (int32_t e = 0; e < J->m; ++e)
    for (int32_t k = J->e_off[e]; k < J->e_off[e + 1]; ++k)
      J->v_idx[fill[J->e_idx[k]]++] = e; /* rows visited in ascending e */
  free(fill);
  return 0;
}

/*
 * Exported entry point.
 *   m, n, e_off[m+1], e_idx[nnz]: CSR of the side to compute (H, or H* when
 *     the caller passes the dual's CSR).
 *   s >= 1: threshold.
 *   rows / n_rows: ascending list of rows to report (NULL: all m rows).
 *   threads >= 1.
 * On success returns the number of pairs and hands out malloc'd arrays in
 * *out_i, *out_j, *out_w (free with slg_oracle_free); *wedges receives the
 * number of upper-triangle wedges visited.  Returns -1 on allocation failure
 * or invalid arguments.
 */
int64_t slg_oracle_line_graph(int32_t m, int32_t n, const int32_t *e_off,
                              const int32_t *e_idx, int32_t s,
                              const int32_t *rows, int64_t n_rows,
                              int32_t threads, int32_t **out_i,
                              int32_t **out_j, int32_t **out_w,
                              int64_t *wedges) {
  if (m < 0 || n < 0 || s < 1 || threads < 1 || !e_off) return -1;
  job J;
  memset(&J, 0, sizeof J);
  J.m = m;
  J.n = n;
  J.e_off = e_off;
  J.e_idx = e_idx;
  J.s = s;
  J.rows = rows;
  J.n_rows = rows ? n_rows : m;
  if (transpose(&J, (int64_t)e_off[m]) != 0) goto fail;
  J.chunk = 64;
  if (J.n_rows / (J.chunk * 8 * threads) > 0) J.chunk *= J.n_rows / (J.chunk * 8 * threads);
  J.n_chunks = (J.n_rows + J.chunk - 1) / J.chunk;
  J.out = calloc((size_t)(J.n_chunks > 0 ? J.n_chunks : 1), sizeof(triples));
  if (!J.out) goto fail;
  atomic_init(&J.next_chunk, 0);
  atomic_init(&J.wedges_acc, 0);

  pthread_t *tid = malloc(sizeof(pthread_t) * (size_t)threads);
  if (!tid) goto fail;
  int started = 0;
  for (int t = 1; t < threads; ++t)
    if (pthread_create(&tid[t], NULL, worker, &J) == 0) ++started;
    else break;
  worker(&J);
  for (int t = 1; t <= started; ++t) pthread_join(tid[t], NULL);
  free(tid);

  int64_t total = 0;
  for (int64_t c = 0; c < J.n_chunks; ++c) {
    if (J.out[c].failed) J.failed = 1;
    total += J.out[c].n;
  }
  if (J.failed) goto fail;
  *out_i = malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  *out_j = malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  *out_w = malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  if (!*out_i || !*out_j || !*out_w) goto fail;
  int64_t at = 0;
  for (int64_t c = 0; c < J.n_chunks; ++c) {
    triples *t = &J.out[c];
    if (t->n) {
      memcpy(*out_i + at, t->i, (size_t)t->n * sizeof(int32_t));
      memcpy(*out_j + at, t->j, (size_t)t->n * sizeof(int32_t));
      memcpy(*out_w + at, t->w, (size_t)t->n * sizeof(int32_t));
    }
    at += t->n;
    free(t->i);
    free(t->j);
    free(t->w);
  }
  free(J.out);
  free(J.v_off);
  free(J.v_idx);
  if (wedges) *wedges = (int64_t)atomic_load(&J.wedges_acc);
  return total;

fail:
  if (J.out)
    for (int64_t c = 0; c < J.n_chunks; ++c) {
      free(J.out[c].i);
      free(J.out[c].j);
      free(J.out[c].w);
    }
  free(J.out);
  free(J.v_off);
  free(J.v_idx);
  return -1;
}

void slg_oracle_free(void *p) { free(p); }
