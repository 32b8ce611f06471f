/*
 * Seeded synthetic sparse vectors for the exact sparse-scoring workloads.
 *
 * This module holds no scoring arithmetic: it only draws inputs (document and
 * query sparse vectors over a fixed vocabulary).  Both the CPU oracle and the
 * GPU library consume its output; neither is used here.
 *
 * The vocabulary permutation has its own seed (perm_seed): documents and
 * queries drawn with different stream seeds share one rank -> term map, so
 * frequent query terms are frequent document terms.
 *
 * Laws (the paper's SPLADE statistics, Sec. 6.1, replaced by synthetic laws):
 *   - number of non-zeros per vector: a mixture of up to 4 components
 *     (Poisson(lambda) or uniform integer [a, b]), clamped to [lo, hi];
 *   - term ranks ~ Zipf(s) truncated to 1..V, mapped to term ids through a
 *     seeded permutation of the vocabulary, drawn one by one with repeats
 *     rejected (weighted sampling without replacement);
 *   - weights ~ lognormal(mu, sigma) clipped to (0, wmax], stored as float32.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014) used as a counter-based stream: every item
 * (document or query) owns an independent stream keyed by (seed, stream, item),
 * so the output does not depend on the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SYN_OK 0
#define SYN_ERR_ARG 1
#define SYN_ERR_NOMEM 2

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

typedef struct {
  uint64_t s;
} rng_t;

static inline uint64_t rng_next(rng_t* r) {
  r->s += 0x9E3779B97F4A7C15ULL;
  return mix64(r->s);
}

/* uniform double in [0, 1) with 53 random bits */
static inline double rng_u01(rng_t* r) { return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0); }

static inline rng_t rng_for(uint64_t seed, uint64_t stream, uint64_t item) {
  rng_t r;
  uint64_t k = mix64(seed * 0xD1B54A32D192ED03ULL + mix64(stream + 0x632BE59BD9B4E019ULL));
  r.s = mix64(k ^ mix64(item * 0x9E3779B97F4A7C15ULL + 0x2545F4914F6CDD1DULL));
  return r;
}

/* Poisson(lambda) by inversion with sequential search (exact up to double
 * rounding; lambda <= 700 keeps exp(-lambda) a normal double). */
static int poisson_draw(rng_t* r, double lambda) {
  double u = rng_u01(r);
  double p = exp(-lambda);
  double F = p;
  int k = 0;
  while (u > F && k < 100000) {
    ++k;
    p *= lambda / (double)k;
    F += p;
    if (p == 0.0 && (double)k > lambda) break;
  }
  return k;
}

/* standard normal by Box-Muller (one value per two uniforms) */
static double normal_draw(rng_t* r) {
  double u1 = 1.0 - rng_u01(r); /* (0, 1] */
  double u2 = rng_u01(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

/* nnz law: ncomp components, each (weight, kind, a, b); kind 0 = Poisson(a),
 * kind 1 = uniform integer in [a, b]; result clamped to [lo, hi]. */
typedef struct {
  int ncomp;
  double weight[4];
  int kind[4];
  double a[4];
  double b[4];
  int lo, hi;
} nnz_law;

static int nnz_draw(rng_t* r, const nnz_law* L) {
  double u = rng_u01(r);
  int c = L->ncomp - 1;
  double acc = 0.0;
  for (int i = 0; i < L->ncomp; ++i) {
    acc += L->weight[i];
    if (u < acc) {
      c = i;
      break;
    }
  }
  int n;
  if (L->kind[c] == 0) {
    n = poisson_draw(r, L->a[c]);
  } else {
    int a = (int)L->a[c], b = (int)L->b[c];
    n = a + (int)(rng_u01(r) * (double)(b - a + 1));
    if (n > b) n = b;
  }
  if (n < L->lo) n = L->lo;
  if (n > L->hi) n = L->hi;
  return n;
}

/* Vose alias table for the truncated Zipf(s) pmf over ranks 1..V. */
typedef struct {
  int V;
  double* prob;
  int32_t* alias;
  int32_t* perm; /* rank-1 -> term id */
} zipf_table;

static int zipf_init(zipf_table* z, int V, double s, uint64_t seed) {
  z->V = V;
  z->prob = (double*)malloc(sizeof(double) * (size_t)V);
  z->alias = (int32_t*)malloc(sizeof(int32_t) * (size_t)V);
  z->perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)V);
  double* q = (double*)malloc(sizeof(double) * (size_t)V);
  int32_t* small = (int32_t*)malloc(sizeof(int32_t) * (size_t)V);
  int32_t* large = (int32_t*)malloc(sizeof(int32_t) * (size_t)V);
  if (!z->prob || !z->alias || !z->perm || !q || !small || !large) {
    free(q); free(small); free(large);
    return SYN_ERR_NOMEM;
  }
  double H = 0.0;
  for (int r = V; r >= 1; --r) H += pow((double)r, -s);
  int ns = 0, nl = 0;
  for (int i = 0; i < V; ++i) {
    q[i] = pow((double)(i + 1), -s) / H * (double)V;
    if (q[i] < 1.0) small[ns++] = i; else large[nl++] = i;
  }
  while (ns > 0 && nl > 0) {
    int sm = small[--ns];
    int lg = large[--nl];
    z->prob[sm] = q[sm];
    z->alias[sm] = lg;
    q[lg] = (q[lg] + q[sm]) - 1.0;
    if (q[lg] < 1.0) small[ns++] = lg; else large[nl++] = lg;
  }
  while (nl > 0) { int i = large[--nl]; z->prob[i] = 1.0; z->alias[i] = i; }
  while (ns > 0) { int i = small[--ns]; z->prob[i] = 1.0; z->alias[i] = i; }
  /* seeded vocabulary permutation (Fisher-Yates) */
  rng_t pr = rng_for(seed, 0x7065726DULL /* "perm" */, 0);
  for (int i = 0; i < V; ++i) z->perm[i] = i;
  for (int i = V - 1; i > 0; --i) {
    int j = (int)(rng_u01(&pr) * (double)(i + 1));
    if (j > i) j = i;
    int32_t t = z->perm[i]; z->perm[i] = z->perm[j]; z->perm[j] = t;
  }
  free(q); free(small); free(large);
  return SYN_OK;
}

static void zipf_free(zipf_table* z) {
  free(z->prob); free(z->alias); free(z->perm);
}

static inline int32_t zipf_term(const zipf_table* z, rng_t* r) {
  double u = rng_u01(r) * (double)z->V;
  int i = (int)u;
  if (i >= z->V) i = z->V - 1;
  double f = u - (double)i;
  int rank0 = (f < z->prob[i]) ? i : z->alias[i];
  return z->perm[rank0];
}

static int cmp_pair(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

static void fill_law(nnz_law* L, int ncomp, const double* comp, int lo, int hi) {
  memset(L, 0, sizeof(*L));
  L->ncomp = ncomp;
  for (int i = 0; i < ncomp; ++i) {
    L->weight[i] = comp[4 * i + 0];
    L->kind[i] = (int)comp[4 * i + 1];
    L->a[i] = comp[4 * i + 2];
    L->b[i] = comp[4 * i + 3];
  }
  L->lo = lo;
  L->hi = hi;
}

/* Number of non-zeros of items [0, n) of a stream.
 * comp: ncomp x (weight, kind, a, b). */
int synth_counts(int64_t n, uint64_t seed, uint64_t stream, int ncomp, const double* comp, int lo, int hi,
                 int32_t* out_nnz, int nthreads) {
  if (n < 0 || ncomp < 1 || ncomp > 4 || lo < 0 || hi < lo || !out_nnz) return SYN_ERR_ARG;
  for (int i = 0; i < ncomp; ++i) {
    if (comp[4 * i + 1] == 0.0 && (comp[4 * i + 2] < 0.0 || comp[4 * i + 2] > 700.0)) return SYN_ERR_ARG;
  }
  nnz_law L;
  fill_law(&L, ncomp, comp, lo, hi);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static, 4096)
#endif
  for (int64_t i = 0; i < n; ++i) {
    rng_t r = rng_for(seed, stream * 2 + 0, (uint64_t)i);
    out_nnz[i] = nnz_draw(&r, &L);
  }
  (void)nthreads;
  return SYN_OK;
}

/* Terms and weights of items [0, n) given the CSR row pointer built from
 * synth_counts.  sort_terms != 0 sorts each row by term id (documents);
 * rows of queries keep their draw order. */
int synth_fill(int64_t n, int32_t V, double zipf_s, double mu, double sigma, double wmax, uint64_t seed,
               uint64_t perm_seed, uint64_t stream, const int64_t* indptr, int sort_terms, int32_t* out_terms,
               float* out_w, int nthreads) {
  if (n < 0 || V < 2 || !indptr || !out_terms || !out_w || !(wmax > 0.0)) return SYN_ERR_ARG;
  for (int64_t i = 0; i < n; ++i) {
    int64_t len = indptr[i + 1] - indptr[i];
    if (len < 0 || len > V / 2) return SYN_ERR_ARG;
  }
  zipf_table z;
  if (zipf_init(&z, V, zipf_s, perm_seed) != SYN_OK) return SYN_ERR_NOMEM;
  int err = SYN_OK;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
  {
    uint32_t* mark = (uint32_t*)calloc((size_t)V, sizeof(uint32_t));
    uint64_t* pairs = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(V / 2 + 1));
    uint32_t stamp = 0;
    if (!mark || !pairs) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      err = SYN_ERR_NOMEM;
    }
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1024)
#endif
    for (int64_t i = 0; i < n; ++i) {
      if (!mark || !pairs) continue;
      int64_t base = indptr[i];
      int len = (int)(indptr[i + 1] - base);
      rng_t r = rng_for(seed, stream * 2 + 1, (uint64_t)i);
      if (++stamp == 0) {
        memset(mark, 0, sizeof(uint32_t) * (size_t)V);
        stamp = 1;
      }
      int cnt = 0;
      while (cnt < len) {
        int32_t t = zipf_term(&z, &r);
        if (mark[t] != stamp) {
          mark[t] = stamp;
          out_terms[base + cnt] = t;
          ++cnt;
        }
      }
      for (int j = 0; j < len; ++j) {
        double w = exp(mu + sigma * normal_draw(&r));
        if (w > wmax) w = wmax;
        float wf = (float)w;
        if (!(wf > 0.0f)) wf = 1.401298464324817e-45f;
        out_w[base + j] = wf;
      }
      if (sort_terms && len > 1) {
        for (int j = 0; j < len; ++j) {
          uint32_t wb;
          memcpy(&wb, &out_w[base + j], 4);
          pairs[j] = ((uint64_t)(uint32_t)out_terms[base + j] << 32) | wb;
        }
        qsort(pairs, (size_t)len, sizeof(uint64_t), cmp_pair);
        for (int j = 0; j < len; ++j) {
          uint32_t wb = (uint32_t)(pairs[j] & 0xFFFFFFFFu);
          out_terms[base + j] = (int32_t)(pairs[j] >> 32);
          memcpy(&out_w[base + j], &wb, 4);
        }
      }
    }
    free(mark);
    free(pairs);
  }
  zipf_free(&z);
  return err;
}

/* The vocabulary permutation used by synth_fill (rank r -> term id), for tests. */
int synth_vocab_perm(int32_t V, uint64_t seed, int32_t* out_perm) {
  if (V < 2 || !out_perm) return SYN_ERR_ARG;
  zipf_table z;
  if (zipf_init(&z, V, 1.0, seed) != SYN_OK) return SYN_ERR_NOMEM;
  memcpy(out_perm, z.perm, sizeof(int32_t) * (size_t)V);
  zipf_free(&z);
  return SYN_OK;
}
