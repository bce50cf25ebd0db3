/*
 * simpfer_cpu.c -- CPU Simpfer (Algorithms 1-3 of the paper) in float64 with
 * OpenMP over blocks: the CPU baseline of the reverse k-MIPS path, and an
 * independent exact method for checking full result sets at sizes the brute
 * force cannot reach.  Test infrastructure: only tests/, the smoke check and
 * bench.py's CPU-baseline legs load it.  It shares no code with the CUDA
 * library.
 *
 * Problem (Definition 2) under the strict tie rule: u is in the result iff
 * fewer than k items p have u.p > u.q, inner products taken exactly on the
 * float32 inputs.
 *
 * Algorithm 1 (pre-processing, Section 4.1): norms, both sets sorted by
 * descending norm (ties by ascending id), P' = the first p_prime sorted items,
 * L_i^j = the j-th largest u_i.p over P' (with the item that attains it),
 * blocks of b consecutive sorted users with L^j(B) = min_i L_i^j (Equation 1)
 * and the first user's norm as the block's norm bound.
 *
 * Algorithm 3 (Section 4.3), per block in parallel:
 *   Lemma 3: prune B when ||u_first|| ||q|| < L^k(B);
 *   Lemma 1: u is a no when u.q < L_i^k (L_i^k is u.p for a known item p, so
 *            this is an exact comparison of two inner products);
 *   Lemma 2: u is a yes when u.q >= ||u|| ||p_k|| (p_k: the item with the
 *            k-th largest norm);
 *   Algorithm 2 for the rest: items in descending norm; Corollary 1 stops
 *            with yes once ||u|| ||p_j|| <= u.q, Corollary 2 with no once k
 *            items are strictly above u.q; the end of P means yes.
 * Under the strict tie rule Lemmas 1 and 3 prune only on strict inequality,
 * the scan's threshold starts at minus infinity and falling off the end of P
 * is a yes (the printed algorithm leaves both open).
 *
 * Arithmetic: float64.  A test that compares two inner products is exact:
 * when the float64 difference is within its rounding bound (Higham, Accuracy
 * and Stability of Numerical Algorithms, Sec. 3.1: gamma_d sum |u_i x_i| per
 * dot product), the sign of u.(a - b) is found exactly by summing the exact
 * products u_i a_i and -u_i b_i as a floating-point expansion (Shewchuk,
 * "Adaptive precision floating-point arithmetic and fast robust geometric
 * predicates", 1997: Two-Sum and Grow-Expansion).  A test against a product
 * of norms (Lemmas 2 and 3, Corollary 1) only acts when it holds with a
 * relative margin larger than every rounding error involved, so it can only
 * send a user on to the exact steps, never decide one wrongly.
 *
 * Build: cc -O2 -fopenmp -ffp-contract=off -shared -fPIC (fused multiply-add
 * contraction would break Two-Sum).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define U64 (1.0 / 9007199254740992.0) /* 2^-53 */

typedef struct {
  int64_t n, m, pp;
  int d, k_max, bs;
  int64_t nb;
  float* Qs;       /* [n][d] users, descending norm */
  float* Ps;       /* [m][d] items, descending norm */
  double* nQ;      /* [n] user norms */
  double* nP;      /* [m] item norms */
  int64_t* permQ;  /* sorted position -> caller's id */
  double* L;       /* [n][k_max] j-th largest u.p over P' (-inf past |P'|) */
  double* Labs;    /* [n][k_max] sum |u_i p_i| of that product (its error scale) */
  int64_t* Lit;    /* [n][k_max] sorted item position attaining it (-1) */
  double* LB;      /* [nb][k_max] block minima */
  double* hdr;     /* [nb] first user's norm */
  double pabs;     /* largest item norm */
} simpfer_index;

/* ------------------------------------------------------------------------ */
/* exact sign of u.a - u.b: Shewchuk expansion of the exact float64 products */
/* ------------------------------------------------------------------------ */
static void two_sum(double a, double b, double* x, double* y) {
  volatile double s = a + b;
  double bv = s - a;
  double av = s - bv;
  double br = b - bv;
  double ar = a - av;
  *x = s;
  *y = ar + br;
}

/* e (len terms, increasing magnitude, non-overlapping) + b -> h; returns the
   new length (zero terms dropped). */
static int grow_expansion(const double* e, int len, double b, double* h) {
  double q = b, hh;
  int out = 0;
  for (int i = 0; i < len; ++i) {
    two_sum(q, e[i], &q, &hh);
    if (hh != 0.0) h[out++] = hh;
  }
  if (q != 0.0) h[out++] = q;
  return out;
}

static int exact_sign_diff(const float* u, const float* a, const float* b, int d) {
  double e[520], h[520];
  int len = 0;
  for (int i = 0; i < d; ++i) {
    const double pa = (double)u[i] * (double)a[i];  /* exact: 24 + 24 bits */
    const double pb = -((double)u[i] * (double)b[i]);
    len = grow_expansion(e, len, pa, h);
    memcpy(e, h, (size_t)len * sizeof(double));
    len = grow_expansion(e, len, pb, h);
    memcpy(e, h, (size_t)len * sizeof(double));
  }
  if (len == 0) return 0;
  return e[len - 1] > 0.0 ? 1 : -1;                 /* the largest term decides */
}

static double dot64(const float* a, const float* b, int d, double* abs_sum) {
  double s = 0.0, t = 0.0;
  for (int i = 0; i < d; ++i) {
    const double p = (double)a[i] * (double)b[i];
    s += p;
    t += fabs(p);
  }
  if (abs_sum) *abs_sum = t;
  return s;
}

/* bound on |computed - exact| of a float64 dot product, per unit of sum |u_i x_i| */
static double gamma_d(int d) { return (d + 2) * U64 / (1.0 - (d + 2) * U64); }

/* sign of u.a - u.b, exact, given their float64 values and absolute sums */
static int cmp_known(const float* u, const float* a, double sa, double sa_abs, const float* b, double sb,
                     double sb_abs, int d) {
  const double bound = 2.0 * gamma_d(d) * (sa_abs + sb_abs) * (1.0 + 4 * U64);
  const double diff = sa - sb;
  if (diff > bound) return 1;
  if (diff < -bound) return -1;
  if (memcmp(a, b, (size_t)d * sizeof(float)) == 0) return 0;   /* identical vectors tie */
  return exact_sign_diff(u, a, b, d);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  double norm;
  int64_t id;
} keyed;

static int by_norm_desc(const void* x, const void* y) {
  const keyed* a = (const keyed*)x;
  const keyed* b = (const keyed*)y;
  if (a->norm > b->norm) return -1;
  if (a->norm < b->norm) return 1;
  return (a->id > b->id) - (a->id < b->id);
}

static double norm64(const float* x, int d) {
  double s = 0.0;
  for (int i = 0; i < d; ++i) s += (double)x[i] * (double)x[i];
  return sqrt(s);
}

static void sort_rows(const float* X, int64_t rows, int d, float* Xs, double* nrm, int64_t* perm) {
  keyed* k = (keyed*)malloc((size_t)rows * sizeof(keyed));
  for (int64_t i = 0; i < rows; ++i) {
    k[i].norm = norm64(X + i * d, d);
    k[i].id = i;
  }
  qsort(k, (size_t)rows, sizeof(keyed), by_norm_desc);
  for (int64_t i = 0; i < rows; ++i) {
    memcpy(Xs + i * d, X + k[i].id * d, (size_t)d * sizeof(float));
    nrm[i] = k[i].norm;
    if (perm) perm[i] = k[i].id;
  }
  free(k);
}

void simpfer_free(simpfer_index* x) {
  if (!x) return;
  free(x->Qs); free(x->Ps); free(x->nQ); free(x->nP); free(x->permQ);
  free(x->L); free(x->Labs); free(x->Lit); free(x->LB); free(x->hdr);
  free(x);
}

int simpfer_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int simpfer_openmp(void) {
#ifdef _OPENMP
  return 1;
#else
  return 0;
#endif
}

static void set_threads(int threads) {
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
}

simpfer_index* simpfer_build(const float* Q, int64_t n, const float* P, int64_t m, int d, int k_max,
                             int64_t p_prime, int block_size, int threads) {
  if (n < 1 || m < 1 || d < 1 || d > 256 || k_max < 1 || block_size < 1) return NULL;
  set_threads(threads);
  simpfer_index* x = (simpfer_index*)calloc(1, sizeof(simpfer_index));
  x->n = n; x->m = m; x->d = d; x->k_max = k_max; x->bs = block_size;
  x->pp = (p_prime <= 0 || p_prime > m) ? m : p_prime;
  x->nb = (n + block_size - 1) / block_size;
  x->Qs = (float*)malloc((size_t)n * d * sizeof(float));
  x->Ps = (float*)malloc((size_t)m * d * sizeof(float));
  x->nQ = (double*)malloc((size_t)n * sizeof(double));
  x->nP = (double*)malloc((size_t)m * sizeof(double));
  x->permQ = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  x->L = (double*)malloc((size_t)n * k_max * sizeof(double));
  x->Labs = (double*)malloc((size_t)n * k_max * sizeof(double));
  x->Lit = (int64_t*)malloc((size_t)n * k_max * sizeof(int64_t));
  x->LB = (double*)malloc((size_t)x->nb * k_max * sizeof(double));
  x->hdr = (double*)malloc((size_t)x->nb * sizeof(double));
  sort_rows(Q, n, d, x->Qs, x->nQ, x->permQ);
  sort_rows(P, m, d, x->Ps, x->nP, NULL);
  x->pabs = x->nP[0];
  const int64_t pp = x->pp;
  /* L_i^j: the k_max largest u_i.p over P' kept sorted by insertion (exact
     comparisons, so equal products keep the earlier item first) */
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    const float* u = x->Qs + i * d;
    double* Li = x->L + i * k_max;
    double* Ai = x->Labs + i * k_max;
    int64_t* Ii = x->Lit + i * k_max;
    int cnt = 0;
    for (int64_t j = 0; j < pp; ++j) {
      const float* p = x->Ps + j * d;
      double va;
      const double v = dot64(u, p, d, &va);
      if (cnt == k_max) {
        const float* w = x->Ps + Ii[cnt - 1] * d;
        if (cmp_known(u, p, v, va, w, Li[cnt - 1], Ai[cnt - 1], d) <= 0) continue;
        --cnt;
      }
      int at = cnt;
      while (at > 0 && cmp_known(u, p, v, va, x->Ps + Ii[at - 1] * d, Li[at - 1], Ai[at - 1], d) > 0) {
        Li[at] = Li[at - 1];
        Ai[at] = Ai[at - 1];
        Ii[at] = Ii[at - 1];
        --at;
      }
      Li[at] = v;
      Ai[at] = va;
      Ii[at] = j;
      ++cnt;
    }
    for (int j = cnt; j < k_max; ++j) {
      Li[j] = -INFINITY;
      Ai[j] = 0.0;
      Ii[j] = -1;
    }
  }
  for (int64_t b = 0; b < x->nb; ++b) {
    const int64_t lo = b * block_size, hi = (lo + block_size < n) ? lo + block_size : n;
    x->hdr[b] = x->nQ[lo];
    for (int j = 0; j < k_max; ++j) {
      double mn = INFINITY;
      for (int64_t i = lo; i < hi; ++i) mn = x->L[i * k_max + j] < mn ? x->L[i * k_max + j] : mn;
      x->LB[b * k_max + j] = mn;
    }
  }
  return x;
}

/* ------------------------------------------------------------------------ */
/* Algorithms 2 and 3                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  int64_t pruned_blocks, lemma1_no, lemma2_yes, scanned, scanned_items;
} simpfer_stats;

/* Algorithm 2 for sorted user i: 1 = yes, 0 = no. */
static int linear_scan(const simpfer_index* x, int64_t i, const float* q, double g, double g_abs, double g_err,
                       int k, int64_t* items) {
  const int d = x->d;
  const float* u = x->Qs + i * d;
  const double marg = 1.0 + 16.0 * (d + 4) * U64;
  int above = 0;
  for (int64_t j = 0; j < x->m; ++j) {
    if (g - g_err >= x->nQ[i] * x->nP[j] * marg) return 1;        /* Corollary 1 */
    ++*items;
    const float* p = x->Ps + j * d;
    double pa;
    const double pv = dot64(u, p, d, &pa);
    if (cmp_known(u, p, pv, pa, q, g, g_abs, d) > 0 && ++above >= k) return 0;   /* Corollary 2 */
  }
  return 1;                                                        /* end of P */
}

/* Returns the result size (ids written ascending, up to cap); -1 on bad k. */
int64_t simpfer_query(const simpfer_index* x, const float* q, int k, int64_t* out, int64_t cap, int threads,
                      simpfer_stats* stats) {
  if (!x || k < 1 || k > x->k_max) return -1;
  set_threads(threads);
  const int d = x->d, km = x->k_max;
  const double qn = norm64(q, d);
  const double gd = gamma_d(d);
  const double marg = 1.0 + 16.0 * (d + 4) * U64;
  /* Lemma 2's p_k: the k-th largest item norm */
  const double pk = k <= x->m ? x->nP[k - 1] : 0.0;
  char* yes = (char*)calloc((size_t)x->n, 1);
  int64_t pruned = 0, l1 = 0, l2 = 0, sc = 0, items = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : pruned, l1, l2, sc, items)
  for (int64_t b = 0; b < x->nb; ++b) {
    /* Lemma 3, with a margin covering the rounding of the norms and of L */
    const double lb = x->LB[b * km + (k - 1)];
    if (x->hdr[b] * qn * marg + gd * x->hdr[b] * x->pabs * marg < lb) {
      ++pruned;
      continue;
    }
    const int64_t lo = b * x->bs, hi = (lo + x->bs < x->n) ? lo + x->bs : x->n;
    for (int64_t i = lo; i < hi; ++i) {
      const float* u = x->Qs + i * d;
      const int64_t it = x->Lit[i * km + (k - 1)];
      double gabs;
      const double g = dot64(u, q, d, &gabs);
      if (it >= 0 && cmp_known(u, q, g, gabs, x->Ps + it * d, x->L[i * km + (k - 1)], x->Labs[i * km + (k - 1)],
                               d) < 0) {                          /* Lemma 1, exact */
        ++l1;
        continue;
      }
      const double g_err = gd * gabs * (1.0 + 4 * U64);
      if (g - g_err >= x->nQ[i] * pk * marg && pk > 0.0) {        /* Lemma 2 */
        ++l2;
        yes[i] = 1;
        continue;
      }
      ++sc;
      yes[i] = (char)linear_scan(x, i, q, g, gabs, g_err, k, &items);
    }
  }
  int64_t cnt = 0;
  /* sorted positions -> ids, ascending */
  for (int64_t i = 0; i < x->n; ++i) cnt += yes[i];
  int64_t* ids = (int64_t*)malloc((size_t)(cnt > 0 ? cnt : 1) * sizeof(int64_t));
  int64_t w = 0;
  for (int64_t i = 0; i < x->n; ++i)
    if (yes[i]) ids[w++] = x->permQ[i];
  free(yes);
  /* ascending ids: counting through a bitmap of the id space */
  unsigned char* mark = (unsigned char*)calloc((size_t)x->n, 1);
  for (int64_t t = 0; t < cnt; ++t) mark[ids[t]] = 1;
  w = 0;
  for (int64_t id = 0; id < x->n; ++id)
    if (mark[id]) {
      if (w < cap) out[w] = id;
      ++w;
    }
  free(mark);
  free(ids);
  if (stats) {
    stats->pruned_blocks = pruned;
    stats->lemma1_no = l1;
    stats->lemma2_yes = l2;
    stats->scanned = sc;
    stats->scanned_items = items;
  }
  return cnt;
}

/* Exact sign of u.a - u.b (for tests of the expansion arithmetic). */
int simpfer_exact_sign(const float* u, const float* a, const float* b, int d) {
  if (d < 1 || d > 256) return 0;
  return exact_sign_diff(u, a, b, d);
}

int64_t simpfer_blocks(const simpfer_index* x) { return x ? x->nb : 0; }
