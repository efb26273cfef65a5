/*
 * CPU oracle for exact batch top-K maximum inner product search.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the tests, the smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or constant with
 * the CUDA library.
 *
 * Everything here is the plain definition, written for a reader to check
 * against the paper by eye:
 *   - the problem (Sec. II-B "Problem Statement: Batch Exact MIPS"): for
 *     every user u, the K items i maximising u^T i;
 *   - brute force (Sec. II-C): one inner product per (u, i) pair, then a
 *     selection of the K best;
 *   - the Maximus index (Sec. III, Algorithm 1): k-means user clusters,
 *     theta_b = max angle between a cluster's users and its centroid, the
 *     CBound of Eq. (appx_bound), per-cluster lists sorted by CBound, and
 *     QueryIndex's walk that stops once the bound falls below the K-th
 *     best score seen so far.
 *
 * Arithmetic: FP32 inputs are widened to double (exact); every inner
 * product is the sequential sum over k = 0..f-1 in double.  Since a
 * product of two FP32 numbers is exact in double, contraction into FMA
 * would not change any result; the build still passes -ffp-contract=off.
 *
 * Ranking rule: item a ranks above item b when s_a > s_b, or s_a == s_b
 * and a < b (the smaller index wins a tie).  The brute force applies it
 * through a full sort of all items per user.
 *
 * Readings of the paper taken here (each is also listed in the design
 * notes):
 *   1. Algorithm 1 compares CBound, a bound on u^T i / ||u|| (Eq. max and
 *      Lemma "upper bound in index lists"), with heap weights u^T i.  The
 *      walk here stops when ||u|| * CBound < (K-th best score).
 *   2. Strictness: the walk stops only on a strictly smaller bound, and a
 *      visited item replaces the heap's worst entry only if it ranks above
 *      it under the rule above, so ties resolve exactly as in the brute
 *      force.
 *   3. acos/cos are evaluated in double; the stop test uses the bound
 *      scaled by (1 + 2^-40) plus 2^-40 ||u|| ||i|| so that rounding in
 *      the bound can never stop a walk early.
 *   4. Zero vectors: a zero user has all scores 0 and is left out of
 *      theta_b; a zero centroid gives theta_b = pi (no pruning); a zero
 *      item has CBound 0; an empty cluster keeps theta_b = 0.
 *   5. k-means: initial centroids are the users whose ids the caller
 *      passes (a seeded draw), exactly `iters` Lloyd iterations
 *      (assign, then update), L2 distance, ties to the smaller centroid
 *      index, an empty cluster keeps its previous centroid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double s;
  int32_t idx;
} scored_t;

/* a ranks before b: higher score, then smaller index */
static int ranks_before(double sa, int32_t ia, double sb, int32_t ib) {
  return sa > sb || (sa == sb && ia < ib);
}

static int cmp_rank(const void* pa, const void* pb) {
  const scored_t* a = (const scored_t*)pa;
  const scored_t* b = (const scored_t*)pb;
  if (ranks_before(a->s, a->idx, b->s, b->idx)) return -1;
  if (ranks_before(b->s, b->idx, a->s, a->idx)) return 1;
  return 0;
}

/* u^T i: sequential double sum over k = 0..f-1 (Sec. II-B). */
double oracle_dot(const float* u, const float* i, int f) {
  double s = 0.0;
  for (int k = 0; k < f; ++k) s += (double)u[k] * (double)i[k];
  return s;
}

static double norm_f(const float* x, int f) { return sqrt(oracle_dot(x, x, f)); }

static double norm_d(const double* x, int f) {
  double s = 0.0;
  for (int k = 0; k < f; ++k) s += x[k] * x[k];
  return sqrt(s);
}

static double dot_fd(const float* u, const double* c, int f) {
  double s = 0.0;
  for (int k = 0; k < f; ++k) s += (double)u[k] * c[k];
  return s;
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
  return nthreads;
#else
  (void)nthreads;
  return 1;
#endif
}

/*
 * Brute force (Sec. II-C): score every item, sort all of them by the
 * ranking rule, keep the first K.  Outputs are row-major [n_users][K].
 * Returns the number of threads used.
 */
int oracle_topk(const float* U, int64_t n_users, const float* I, int64_t n_items, int f, int K,
                int nthreads, int32_t* out_idx, double* out_score) {
  int nt = set_threads(nthreads);
#pragma omp parallel num_threads(nt)
  {
    scored_t* row = (scored_t*)malloc(sizeof(scored_t) * (size_t)n_items);
#pragma omp for schedule(dynamic, 16)
    for (int64_t u = 0; u < n_users; ++u) {
      const float* uv = U + (size_t)u * f;
      for (int64_t j = 0; j < n_items; ++j) {
        row[j].s = oracle_dot(uv, I + (size_t)j * f, f);
        row[j].idx = (int32_t)j;
      }
      qsort(row, (size_t)n_items, sizeof(scored_t), cmp_rank);
      for (int k = 0; k < K; ++k) {
        out_idx[(size_t)u * K + k] = row[k].idx;
        out_score[(size_t)u * K + k] = row[k].s;
      }
    }
    free(row);
  }
  return nt;
}

/* ---------------------------------------------------------------------
 * k-means (Sec. III-A "Clustering Users"; Algorithm 1, ConstructIndex).
 * ------------------------------------------------------------------- */
static double sqdist_fd(const float* u, const double* c, int f) {
  double s = 0.0;
  for (int k = 0; k < f; ++k) {
    double d = (double)u[k] - c[k];
    s += d * d;
  }
  return s;
}

static int32_t nearest_centroid(const float* u, const double* cent, int C, int f) {
  int32_t best = 0;
  double bd = sqdist_fd(u, cent, f);
  for (int j = 1; j < C; ++j) {
    double d = sqdist_fd(u, cent + (size_t)j * f, f);
    if (d < bd) {
      bd = d;
      best = j;
    }
  }
  return best;
}

/* sum over users of the squared distance to the assigned centroid */
double oracle_kmeans_objective(const float* U, int64_t n_users, int f, const double* cent,
                               const int32_t* assign) {
  double s = 0.0;
  for (int64_t u = 0; u < n_users; ++u)
    s += sqdist_fd(U + (size_t)u * f, cent + (size_t)assign[u] * f, f);
  return s;
}

/*
 * Lloyd's k-means: centroids start at the users listed in init_ids;
 * each of `iters` iterations assigns every user to its nearest centroid
 * and then moves each centroid to the mean of its members.  On return
 * `assign` is the last assignment and `cent` holds the updated means.
 * objective_trace (optional, length iters) receives the objective of
 * each assignment step against the centroids it was assigned to.
 */
void oracle_kmeans(const float* U, int64_t n_users, int f, int C, int iters,
                   const int64_t* init_ids, int nthreads, double* cent, int32_t* assign,
                   double* objective_trace) {
  int nt = set_threads(nthreads);
  for (int j = 0; j < C; ++j)
    for (int k = 0; k < f; ++k) cent[(size_t)j * f + k] = (double)U[(size_t)init_ids[j] * f + k];
  double* sums = (double*)malloc(sizeof(double) * (size_t)C * f);
  int64_t* cnt = (int64_t*)malloc(sizeof(int64_t) * (size_t)C);
  for (int it = 0; it < iters; ++it) {
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t u = 0; u < n_users; ++u) assign[u] = nearest_centroid(U + (size_t)u * f, cent, C, f);
    if (objective_trace) objective_trace[it] = oracle_kmeans_objective(U, n_users, f, cent, assign);
    memset(sums, 0, sizeof(double) * (size_t)C * f);
    memset(cnt, 0, sizeof(int64_t) * (size_t)C);
    for (int64_t u = 0; u < n_users; ++u) {
      int32_t j = assign[u];
      cnt[j] += 1;
      for (int k = 0; k < f; ++k) sums[(size_t)j * f + k] += (double)U[(size_t)u * f + k];
    }
    for (int j = 0; j < C; ++j) {
      if (cnt[j] == 0) continue; /* empty cluster keeps its centroid */
      for (int k = 0; k < f; ++k) cent[(size_t)j * f + k] = sums[(size_t)j * f + k] / (double)cnt[j];
    }
  }
  free(sums);
  free(cnt);
}

/* ---------------------------------------------------------------------
 * Bounds (Eq. max, Eq. upper_bound, Eq. appx_bound; Algorithm 1).
 * ------------------------------------------------------------------- */
static double clamp_cos(double x) { return x > 1.0 ? 1.0 : (x < -1.0 ? -1.0 : x); }

/*
 * theta_b[j] = max over users u assigned to cluster j of the angle
 * acos(u^T c_j / (||u|| ||c_j||))  (Algorithm 1, ConstructIndex).
 */
void oracle_theta_b(const float* U, int64_t n_users, int f, int C, const double* cent,
                    const int32_t* assign, double* theta_b) {
  for (int j = 0; j < C; ++j) theta_b[j] = 0.0;
  for (int64_t u = 0; u < n_users; ++u) {
    const float* uv = U + (size_t)u * f;
    int32_t j = assign[u];
    const double* c = cent + (size_t)j * f;
    double nu = norm_f(uv, f), nc = norm_d(c, f);
    double th;
    if (nu == 0.0) continue;
    if (nc == 0.0)
      th = M_PI;
    else
      th = acos(clamp_cos(dot_fd(uv, c, f) / (nu * nc)));
    if (th > theta_b[j]) theta_b[j] = th;
  }
}

/*
 * CBound(c, i, theta_b) of Eq. (appx_bound): ||i|| cos(theta_ic - theta_b)
 * when theta_b < theta_ic, else ||i||.  It bounds u^T i / ||u|| for every
 * user u of the cluster (Lemma "upper bound in index lists").
 */
double oracle_cbound(const double* c, const float* i, int f, double theta_b) {
  double ni = norm_f(i, f), nc = norm_d(c, f);
  if (ni == 0.0) return 0.0;
  if (nc == 0.0) return ni;
  double theta_ic = acos(clamp_cos(dot_fd(i, c, f) / (ni * nc)));
  return theta_b < theta_ic ? ni * cos(theta_ic - theta_b) : ni;
}

/* CBound for every (cluster, item): out is [C][n_items]. */
void oracle_cbound_all(const double* cent, int C, const float* I, int64_t n_items, int f,
                       const double* theta_b, int nthreads, double* out) {
  int nt = set_threads(nthreads);
#pragma omp parallel for num_threads(nt) schedule(static) collapse(2)
  for (int j = 0; j < C; ++j)
    for (int64_t t = 0; t < n_items; ++t)
      out[(size_t)j * n_items + t] = oracle_cbound(cent + (size_t)j * f, I + (size_t)t * f, f, theta_b[j]);
}

typedef struct {
  double b;
  int32_t idx;
} bound_t;

static int cmp_bound_desc(const void* pa, const void* pb) {
  const bound_t* a = (const bound_t*)pa;
  const bound_t* b = (const bound_t*)pb;
  if (a->b > b->b) return -1;
  if (a->b < b->b) return 1;
  return a->idx < b->idx ? -1 : (a->idx > b->idx);
}

/*
 * Maximus (Algorithm 1).  ConstructIndex: k-means over the users, theta_b
 * per cluster, and for each cluster the item list sorted by CBound
 * (descending; equal bounds by item index).  QueryIndex for every user:
 * score the first K items of its cluster's list, then walk the rest,
 * stopping at the first item whose ||u|| * CBound (with the rounding
 * margin of reading 3) is below the current K-th best score, otherwise
 * scoring the item and keeping it if it ranks above the current K-th.
 *
 * Outputs: top-K per user (sorted by the ranking rule), the number of
 * items each user scored (visited), and the clustering it used.
 * Returns the number of threads used.
 */
int oracle_maximus(const float* U, int64_t n_users, const float* I, int64_t n_items, int f, int K,
                   int C, int iters, const int64_t* init_ids, int nthreads, int32_t* out_idx,
                   double* out_score, int64_t* visited, double* cent_out, int32_t* assign_out,
                   double* theta_b_out) {
  int nt = set_threads(nthreads);
  oracle_kmeans(U, n_users, f, C, iters, init_ids, nt, cent_out, assign_out, NULL);
  oracle_theta_b(U, n_users, f, C, cent_out, assign_out, theta_b_out);

  /* L[C_j]: items sorted by CBound, descending */
  bound_t* lists = (bound_t*)malloc(sizeof(bound_t) * (size_t)C * n_items);
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
  for (int j = 0; j < C; ++j) {
    bound_t* L = lists + (size_t)j * n_items;
    for (int64_t t = 0; t < n_items; ++t) {
      L[t].b = oracle_cbound(cent_out + (size_t)j * f, I + (size_t)t * f, f, theta_b_out[j]);
      L[t].idx = (int32_t)t;
    }
    qsort(L, (size_t)n_items, sizeof(bound_t), cmp_bound_desc);
  }

  double* item_norm = (double*)malloc(sizeof(double) * (size_t)n_items);
  for (int64_t t = 0; t < n_items; ++t) item_norm[t] = norm_f(I + (size_t)t * f, f);
  const double margin = 9.094947017729282e-13; /* 2^-40 */

#pragma omp parallel num_threads(nt)
  {
    scored_t* H = (scored_t*)malloc(sizeof(scored_t) * (size_t)K);
#pragma omp for schedule(dynamic, 16)
    for (int64_t u = 0; u < n_users; ++u) {
      const float* uv = U + (size_t)u * f;
      const bound_t* L = lists + (size_t)assign_out[u] * n_items;
      double nu = norm_f(uv, f);
      /* heap seeded with the first K list items, weighted by u^T i */
      for (int k = 0; k < K; ++k) {
        H[k].idx = L[k].idx;
        H[k].s = oracle_dot(uv, I + (size_t)L[k].idx * f, f);
      }
      int worst = 0;
      for (int k = 1; k < K; ++k)
        if (ranks_before(H[worst].s, H[worst].idx, H[k].s, H[k].idx)) worst = k;
      int64_t seen = K;
      for (int64_t t = K; t < n_items; ++t) {
        const int32_t it = L[t].idx;
        double bound = nu * L[t].b * (1.0 + margin) + margin * nu * item_norm[it];
        if (bound < H[worst].s) break;
        double s = oracle_dot(uv, I + (size_t)it * f, f);
        ++seen;
        if (ranks_before(s, it, H[worst].s, H[worst].idx)) {
          H[worst].s = s;
          H[worst].idx = it;
          worst = 0;
          for (int k = 1; k < K; ++k)
            if (ranks_before(H[worst].s, H[worst].idx, H[k].s, H[k].idx)) worst = k;
        }
      }
      qsort(H, (size_t)K, sizeof(scored_t), cmp_rank);
      for (int k = 0; k < K; ++k) {
        out_idx[(size_t)u * K + k] = H[k].idx;
        out_score[(size_t)u * K + k] = H[k].s;
      }
      visited[u] = seen;
    }
    free(H);
  }
  free(item_norm);
  free(lists);
  return nt;
}
