/*
 * CPU oracle for exact batched sparse scoring (TEST INFRASTRUCTURE ONLY).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library.  It shares no code with the GPU library: it builds its own
 * term -> postings lists, walks them term by term into a dense FP64 score row
 * and fully sorts the row.
 *
 * Definition followed (Sec. 4.1, Eq. 4): for a query q = {(t_i, w_i)} and a
 * document d,   score(q, d) = sum_i w_i * s_d(t_i),
 * where s_d(t) is the impact the index stores for (d, t), 0 when d is not in
 * the posting list of t.  Eq. 5 is the same sum written as one scatter-add per
 * query term, which is the order this oracle adds in.  Every posting of every
 * query term is processed (Sec. 4.3), padding never contributes (Sec. 3.2).
 * All N documents are eligible; the result is the first k of the order
 * (score descending, document id ascending).
 *
 * Stored impacts (the index's precision):
 *   F32  : the document weight itself;
 *   F16  : the weight rounded to IEEE binary16, nearest-even;
 *   BF16 : the weight rounded to bfloat16 (8-bit exponent, 7-bit fraction),
 *          nearest-even;
 *   U8   : round(w * 255 / 5) = nearest-even integer of 51 * w, in [0, 255];
 *          query weights are quantised by the same rule and scores are the
 *          exact integer sums.
 * Float paths accumulate in FP64; f32 x f32 products are exact in FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_F32 = 0, OR_F16 = 1, OR_BF16 = 2, OR_U8 = 3 };
enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_NOMEM = 2, OR_ERR_DATA = 3 };

/* ---- stored-impact rounding, written from the format definitions ---- */

/* nearest-even integer of 51 * w (= w * 255 / 5), clamped to [0, 255] */
int32_t oracle_quant_u8(float w) {
  double v = rint(51.0 * (double)w); /* exact product: 24-bit x 6-bit */
  if (!(v >= 0.0)) v = 0.0;
  if (v > 255.0) v = 255.0;
  return (int32_t)v;
}

/* f32 -> IEEE binary16 (1/5/10, bias 15), nearest-even, returned as a double */
double oracle_round_f16(float f) {
  double x = (double)f;
  if (!isfinite(x) || x == 0.0) return x;
  double ax = fabs(x);
  double ulp;
  if (ax < 6.103515625e-05) { /* below 2^-14: binary16 subnormal spacing 2^-24 */
    ulp = ldexp(1.0, -24);
  } else {
    int e;
    frexp(ax, &e); /* ax = m * 2^e, m in [0.5, 1): floor(log2 ax) = e - 1 */
    ulp = ldexp(1.0, (e - 1) - 10);
  }
  double r = rint(x / ulp) * ulp;
  if (fabs(r) > 65504.0) r = copysign(INFINITY, x);
  return r;
}

/* f32 -> bfloat16 (1/8/7), nearest-even, returned as a double */
double oracle_round_bf16(float f) {
  double x = (double)f;
  if (!isfinite(x) || x == 0.0) return x;
  double ax = fabs(x);
  double ulp;
  if (ax < ldexp(1.0, -126)) { /* subnormal: spacing 2^-133 */
    ulp = ldexp(1.0, -133);
  } else {
    int e;
    frexp(ax, &e);
    ulp = ldexp(1.0, (e - 1) - 7);
  }
  double r = rint(x / ulp) * ulp;
  /* largest finite bfloat16 is (2 - 2^-7) * 2^127 */
  if (fabs(r) > ldexp(2.0 - ldexp(1.0, -7), 127)) r = copysign(INFINITY, x);
  return r;
}

static double stored_impact(int impact, float w) {
  switch (impact) {
    case OR_F16: return oracle_round_f16(w);
    case OR_BF16: return oracle_round_bf16(w);
    case OR_U8: return (double)oracle_quant_u8(w);
    default: return (double)w;
  }
}

static double query_weight(int impact, float w) {
  return impact == OR_U8 ? (double)oracle_quant_u8(w) : (double)w;
}

/* ---- the oracle's own inverted index (Sec. 3.2, without padding) ---- */

typedef struct {
  int64_t N;
  int32_t V;
  int impact;
  int64_t* ptr; /* V + 1 */
  int32_t* doc; /* postings, doc-sorted within each term */
  double* x;    /* stored impact of each posting */
  int64_t* xi;  /* integer impact (U8 only) */
} or_index;

void oracle_index_free(or_index* ix) {
  if (!ix) return;
  free(ix->ptr);
  free(ix->doc);
  free(ix->x);
  free(ix->xi);
  free(ix);
}

/* Returns OR_ERR_DATA for a term id outside [0, V), a non-finite weight, a
 * term repeated inside one document, a U8 weight outside [0, 5] or an F16
 * weight beyond the binary16 range. */
int oracle_index_build(int64_t N, int32_t V, const int64_t* indptr, const int32_t* terms, const float* w,
                       int impact, or_index** out) {
  if (N < 1 || V < 1 || !indptr || !out || impact < OR_F32 || impact > OR_U8) return OR_ERR_ARG;
  *out = NULL;
  if (indptr[0] != 0) return OR_ERR_ARG;
  for (int64_t d = 0; d < N; ++d)
    if (indptr[d + 1] < indptr[d]) return OR_ERR_ARG;
  int64_t nnz = indptr[N];
  for (int64_t p = 0; p < nnz; ++p) {
    if (terms[p] < 0 || terms[p] >= V) return OR_ERR_DATA;
    if (!isfinite(w[p])) return OR_ERR_DATA;
    if (impact == OR_U8 && (w[p] < 0.0f || w[p] > 5.0f)) return OR_ERR_DATA;
    if (impact == OR_F16 && isinf(oracle_round_f16(w[p]))) return OR_ERR_DATA;
  }
  or_index* ix = (or_index*)calloc(1, sizeof(or_index));
  if (!ix) return OR_ERR_NOMEM;
  ix->N = N;
  ix->V = V;
  ix->impact = impact;
  ix->ptr = (int64_t*)calloc((size_t)V + 1, sizeof(int64_t));
  ix->doc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  ix->x = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (impact == OR_U8) ix->xi = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  if (!ix->ptr || !ix->doc || !ix->x || !fill || (impact == OR_U8 && !ix->xi)) {
    free(fill);
    oracle_index_free(ix);
    return OR_ERR_NOMEM;
  }
  /* counting sort by term; documents visited in increasing id keep each list
   * sorted by document id */
  for (int64_t p = 0; p < nnz; ++p) ix->ptr[terms[p] + 1]++;
  for (int32_t t = 0; t < V; ++t) ix->ptr[t + 1] += ix->ptr[t];
  for (int32_t t = 0; t < V; ++t) fill[t] = ix->ptr[t];
  int err = OR_OK;
  for (int64_t d = 0; d < N && err == OR_OK; ++d) {
    for (int64_t p = indptr[d]; p < indptr[d + 1]; ++p) {
      int32_t t = terms[p];
      int64_t slot = fill[t]++;
      if (slot > ix->ptr[t] && ix->doc[slot - 1] == (int32_t)d) { /* repeated term in d */
        err = OR_ERR_DATA;
        break;
      }
      ix->doc[slot] = (int32_t)d;
      ix->x[slot] = stored_impact(impact, w[p]);
      if (impact == OR_U8) ix->xi[slot] = oracle_quant_u8(w[p]);
    }
  }
  free(fill);
  if (err != OR_OK) {
    oracle_index_free(ix);
    return err;
  }
  *out = ix;
  return OR_OK;
}

int64_t oracle_index_postings(const or_index* ix) { return ix ? ix->ptr[ix->V] : -1; }

/* copy of one posting list (for layout tests): returns its length; writes at
 * most cap entries */
int64_t oracle_index_list(const or_index* ix, int32_t t, int64_t cap, int32_t* docs, double* x) {
  if (!ix || t < 0 || t >= ix->V) return -1;
  int64_t a = ix->ptr[t], b = ix->ptr[t + 1];
  for (int64_t p = a; p < b && p - a < cap; ++p) {
    if (docs) docs[p - a] = ix->doc[p];
    if (x) x[p - a] = ix->x[p];
  }
  return b - a;
}

/* ---- scoring ---- */

/* Fills row[0..N) with score(q, d) for one query, walking the query terms in
 * the given order (Eq. 5).  A term id outside [0, V) or a non-finite weight is
 * skipped and reported through *bad. */
static void score_row(const or_index* ix, const int32_t* qt, const float* qw, int64_t nq, double* row,
                      int64_t* irow, int* bad) {
  if (ix->impact == OR_U8) {
    memset(irow, 0, sizeof(int64_t) * (size_t)ix->N);
  } else {
    memset(row, 0, sizeof(double) * (size_t)ix->N);
  }
  for (int64_t i = 0; i < nq; ++i) {
    int32_t t = qt[i];
    float wf = qw[i];
    if (t < 0 || t >= ix->V || !isfinite(wf)) {
      *bad = 1;
      continue;
    }
    int64_t a = ix->ptr[t], b = ix->ptr[t + 1];
    if (ix->impact == OR_U8) {
      int64_t wq = oracle_quant_u8(wf);
      for (int64_t p = a; p < b; ++p) irow[ix->doc[p]] += wq * ix->xi[p];
    } else {
      double wq = query_weight(ix->impact, wf);
      for (int64_t p = a; p < b; ++p) row[ix->doc[p]] += wq * ix->x[p];
    }
  }
  if (ix->impact == OR_U8)
    for (int64_t d = 0; d < ix->N; ++d) row[d] = (double)irow[d];
}

typedef struct {
  double s;
  int32_t id;
} scored;

/* score descending, then document id ascending */
static int cmp_scored(const void* a, const void* b) {
  const scored* x = (const scored*)a;
  const scored* y = (const scored*)b;
  if (x->s > y->s) return -1;
  if (x->s < y->s) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}

/* Exact top-k of B queries.  q_indptr has B + 1 entries.  Outputs are B x k:
 * ids (int32) and scores (double; exact integers on the U8 path).
 * *data_error is set to 1 when some query term was skipped. */
int oracle_topk(const or_index* ix, int32_t B, const int64_t* q_indptr, const int32_t* q_terms,
                const float* q_w, int32_t k, int32_t* out_ids, double* out_scores, int* data_error,
                int nthreads) {
  if (!ix || B < 0 || k < 1 || (int64_t)k > ix->N || !q_indptr || !out_ids || !out_scores) return OR_ERR_ARG;
  int err = OR_OK, bad_any = 0;
  set_threads(nthreads);
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    double* row = (double*)malloc(sizeof(double) * (size_t)ix->N);
    int64_t* irow = ix->impact == OR_U8 ? (int64_t*)malloc(sizeof(int64_t) * (size_t)ix->N) : NULL;
    scored* all = (scored*)malloc(sizeof(scored) * (size_t)ix->N);
    int ok = row && all && (ix->impact != OR_U8 || irow);
    if (!ok) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      err = OR_ERR_NOMEM;
    }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int32_t q = 0; q < B; ++q) {
      if (!ok) continue;
      int bad = 0;
      score_row(ix, q_terms + q_indptr[q], q_w + q_indptr[q], q_indptr[q + 1] - q_indptr[q], row, irow, &bad);
      if (bad) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
        bad_any = 1;
      }
      for (int64_t d = 0; d < ix->N; ++d) {
        all[d].s = row[d] == 0.0 ? 0.0 : row[d]; /* -0 -> +0 */
        all[d].id = (int32_t)d;
      }
      qsort(all, (size_t)ix->N, sizeof(scored), cmp_scored);
      for (int32_t j = 0; j < k; ++j) {
        out_ids[(int64_t)q * k + j] = all[j].id;
        out_scores[(int64_t)q * k + j] = all[j].s;
      }
    }
    free(row);
    free(irow);
    free(all);
  }
  if (data_error) *data_error = bad_any;
  return err;
}

/* Full B x N score rows (small collections only). */
int oracle_rows(const or_index* ix, int32_t B, const int64_t* q_indptr, const int32_t* q_terms,
                const float* q_w, double* rows, int* data_error, int nthreads) {
  if (!ix || B < 0 || !q_indptr || !rows) return OR_ERR_ARG;
  int err = OR_OK, bad_any = 0;
  set_threads(nthreads);
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    int64_t* irow = ix->impact == OR_U8 ? (int64_t*)malloc(sizeof(int64_t) * (size_t)ix->N) : NULL;
    int ok = (ix->impact != OR_U8 || irow);
    if (!ok) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      err = OR_ERR_NOMEM;
    }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int32_t q = 0; q < B; ++q) {
      if (!ok) continue;
      int bad = 0;
      score_row(ix, q_terms + q_indptr[q], q_w + q_indptr[q], q_indptr[q + 1] - q_indptr[q],
                rows + (int64_t)q * ix->N, irow, &bad);
      if (bad) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
        bad_any = 1;
      }
    }
    free(irow);
  }
  if (data_error) *data_error = bad_any;
  return err;
}

/* Doc-major recomputation of score(q, d) and of A(q, d) = sum_i |w_i x_d(t_i)|
 * for m given documents per query (ids B x m, -1 = skip), straight from the
 * document vectors.  This traversal is independent of the term-major walk
 * above and serves the tolerance checks. */
int oracle_doc_scores(int64_t N, int32_t V, const int64_t* indptr, const int32_t* terms, const float* w,
                      int impact, int32_t B, const int64_t* q_indptr, const int32_t* q_terms,
                      const float* q_w, int32_t m, const int32_t* docs, double* s_out, double* a_out,
                      int nthreads) {
  if (N < 1 || V < 1 || B < 0 || m < 0 || !indptr || !docs || !s_out) return OR_ERR_ARG;
  int err = OR_OK;
  set_threads(nthreads);
#ifdef _OPENMP
#pragma omp parallel
#endif
  {
    double* qv = (double*)calloc((size_t)V, sizeof(double));
    double* qa = (double*)calloc((size_t)V, sizeof(double));
    if (!qv || !qa) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      err = OR_ERR_NOMEM;
    }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int32_t q = 0; q < B; ++q) {
      if (!qv || !qa) continue;
      for (int64_t i = q_indptr[q]; i < q_indptr[q + 1]; ++i) {
        int32_t t = q_terms[i];
        if (t < 0 || t >= V || !isfinite(q_w[i])) continue;
        double wq = query_weight(impact, q_w[i]);
        qv[t] += wq;
        qa[t] += fabs(wq);
      }
      for (int32_t j = 0; j < m; ++j) {
        int32_t d = docs[(int64_t)q * m + j];
        double s = 0.0, a = 0.0;
        if (d >= 0 && d < N) {
          for (int64_t p = indptr[d]; p < indptr[d + 1]; ++p) {
            int32_t t = terms[p];
            if (t < 0 || t >= V) continue;
            double x = stored_impact(impact, w[p]);
            s += qv[t] * x;
            a += qa[t] * fabs(x);
          }
        }
        s_out[(int64_t)q * m + j] = s;
        if (a_out) a_out[(int64_t)q * m + j] = a;
      }
      for (int64_t i = q_indptr[q]; i < q_indptr[q + 1]; ++i) {
        int32_t t = q_terms[i];
        if (t >= 0 && t < V) {
          qv[t] = 0.0;
          qa[t] = 0.0;
        }
      }
    }
    free(qv);
    free(qa);
  }
  return err;
}

/* stored impacts of n weights (vectorised helper for tests) */
int oracle_stored_array(int impact, int64_t n, const float* w, double* out) {
  if (n < 0 || !w || !out || impact < OR_F32 || impact > OR_U8) return OR_ERR_ARG;
  for (int64_t i = 0; i < n; ++i) out[i] = stored_impact(impact, w[i]);
  return OR_OK;
}

/* query weights as the scoring uses them (U8: quantised) */
int oracle_query_array(int impact, int64_t n, const float* w, double* out) {
  if (n < 0 || !w || !out || impact < OR_F32 || impact > OR_U8) return OR_ERR_ARG;
  for (int64_t i = 0; i < n; ++i) out[i] = query_weight(impact, w[i]);
  return OR_OK;
}
