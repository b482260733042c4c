/*
 * exact_pairs.c - TEST INFRASTRUCTURE ONLY (part of the CPU oracle).
 *
 * Every non-trivial pair of length-w windows of a D-dimensional series
 * whose d-dimensional distance dist_d is at most tau, in float64, by the
 * textbook matrix-profile recurrence along diagonals.  It shares no code
 * with the CUDA library and nothing on the product path may call it; the
 * tests, the golden-value script and the benchmark's CPU baseline do.
 *
 * What it computes (Section 3.1 of the paper; readings stated in the
 * oracle's Python header):
 *   - each dimension less its overall mean (a shift: z-normalised windows
 *     are unchanged), then per dimension f and window a: mean mu and
 *     population sigma (two passes over the window);
 *   - for every pair a < b with b - a > excl, per dimension, the raw dot
 *     product QT of the two windows, slid along the diagonal
 *     (QT(a+1, b+1) = QT(a, b) - x_a x_b + x_{a+w} x_{b+w}) and recomputed
 *     directly every 1024 steps;
 *   - the z-normalised Euclidean distance (Eq. zned) in its Pearson form,
 *     dist^2 = 2 w (1 - (QT - w mu_a mu_b) / (w sigma_a sigma_b)), clamped
 *     at 0; a flat window (sigma <= flat_rel (1 + |mu|)) z-normalises to the
 *     zero vector: distance 0 to another flat window, sqrt(w) to any other;
 *   - dist_d = the sum of the d smallest per-dimension distances
 *     (Definition distdims), dims_d those d dimensions (ties to the lower
 *     index), dist_d^max the largest of them (Eq. distdmax).
 * Blocks of 32 diagonals are shared among threads (OpenMP) and advance row
 * by row; the output order is not specified (the caller sorts).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef struct {
  int64_t a, b;
  double dist_d, dist_max;
  uint64_t dims;
} oracle_pair;

static void window_stats(const double* x, int64_t M, int w, double* mu, double* sg) {
  for (int64_t a = 0; a < M; ++a) {
    double s = 0.0;
    for (int t = 0; t < w; ++t) s += x[a + t];
    const double m = s / w;
    double v = 0.0;
    for (int t = 0; t < w; ++t) v += (x[a + t] - m) * (x[a + t] - m);
    mu[a] = m;
    sg[a] = sqrt(v / w);
  }
}

static double dot(const double* x, int64_t a, int64_t b, int w) {
  double s = 0.0;
  for (int t = 0; t < w; ++t) s += x[a + t] * x[b + t];
  return s;
}

/* Pairs with dist_d <= tau into out (at most cap of them); returns how many
 * there are in all (may exceed cap), or -1 if memory runs out. */
int64_t oracle_pairs_below(const double* T, int D, int64_t n, int w, int d, int64_t excl,
                           double tau, double flat_rel, oracle_pair* out, int64_t cap) {
  const int64_t M = n - w + 1;
  if (M < 1 || D < 1 || D > 64 || d < 1 || d > D) return 0;
  /* per dimension: the series less its overall mean (a shift: z-normalised
     windows do not change, and the raw dot products of the Pearson form
     lose less to cancellation), then every window's mean and population
     sigma by two passes; stored point-major ([t][f], [a][f]) so that the
     D values of a step are contiguous */
  double* X = malloc(sizeof(double) * (size_t)(D * n));
  double* mu = malloc(sizeof(double) * (size_t)(D * M));
  double* wmu = malloc(sizeof(double) * (size_t)(D * M));
  double* isw = malloc(sizeof(double) * (size_t)(D * M));      /* 1 / (w sigma), 0 if flat */
  unsigned char* flat = malloc((size_t)(D * M));
  double* xf = malloc(sizeof(double) * (size_t)n);
  double* mf = malloc(sizeof(double) * (size_t)M);
  double* sf = malloc(sizeof(double) * (size_t)M);
  if (!X || !mu || !wmu || !isw || !flat || !xf || !mf || !sf) {
    free(X); free(mu); free(wmu); free(isw); free(flat); free(xf); free(mf); free(sf);
    return -1;
  }
  for (int f = 0; f < D; ++f) {
    double s = 0.0;
    for (int64_t t = 0; t < n; ++t) s += T[(int64_t)f * n + t];
    const double c = s / (double)n;
    for (int64_t t = 0; t < n; ++t) xf[t] = T[(int64_t)f * n + t] - c;
    window_stats(xf, M, w, mf, sf);
    for (int64_t t = 0; t < n; ++t) X[t * D + f] = xf[t];
    for (int64_t q = 0; q < M; ++q) {
      const int64_t o = q * D + f;
      /* flat relative to the window's own level (before the shift) */
      flat[o] = sf[q] <= flat_rel * (1.0 + fabs(mf[q] + c));
      mu[o] = mf[q];
      wmu[o] = w * mf[q];
      isw[o] = flat[o] ? 0.0 : 1.0 / (w * sf[q]);
    }
  }
  free(xf); free(mf); free(sf);
  int64_t found = 0;
  const double tau2 = tau * tau;
#pragma omp parallel
  {
    /* diagonals advance in blocks of DB, row by row, so that the rows a
       and a + delta of consecutive steps stay in cache; each diagonal's
       recurrence runs in the same order as one diagonal at a time */
    enum { DB = 32 };
    static double qts[DB][64];
#pragma omp threadprivate(qts)
    double dist[64];
    int ord[64];
#pragma omp for schedule(dynamic, 1)
    for (int64_t d0 = excl + 1; d0 < M; d0 += DB) {
      const int nb = (int)((M - d0) < DB ? (M - d0) : DB);
      for (int64_t a = 0; a + d0 < M; ++a) {
        for (int j = 0; j < nb; ++j) {
          const int64_t delta = d0 + j;
          const int64_t b = a + delta;
          if (b >= M) break;                        /* longer diagonals first */
          double* qt = qts[j];
          const double* xa0 = X + (a - 1) * D;      /* point a - 1 (not read at a = 0) */
          const double* xb0 = X + (b - 1) * D;
          const double* xa1 = X + (a + w - 1) * D;  /* point a + w - 1 */
          const double* xb1 = X + (b + w - 1) * D;
          const int64_t oa = a * D, ob = b * D;
          int near = 0;
          for (int f = 0; f < D; ++f) {
            if (a % 1024 == 0) {
              double s = 0.0;
              for (int t = 0; t < w; ++t) s += X[(a + t) * D + f] * X[(b + t) * D + f];
              qt[f] = s;
            } else {
              qt[f] = qt[f] - xa0[f] * xb0[f] + xa1[f] * xb1[f];
            }
            double sq;
            if (flat[oa + f] || flat[ob + f]) {
              sq = (flat[oa + f] && flat[ob + f]) ? 0.0 : (double)w;
            } else {
              /* corr = (QT - w mu_a mu_b) / (w sigma_a sigma_b) */
              const double corr = (qt[f] - wmu[oa + f] * mu[ob + f]) * isw[oa + f] * isw[ob + f] * w;
              sq = 2.0 * w * (1.0 - corr);
              if (sq < 0.0) sq = 0.0;
            }
            dist[f] = sq;                        /* squared for now */
            near += sq <= tau2;
          }
          /* fewer than d dims within tau: one of the d smallest exceeds
             tau, so dist_d > tau (distances are >= 0) */
          if (near < d) continue;
          for (int f = 0; f < D; ++f) dist[f] = sqrt(dist[f]);
          /* the d smallest, ties to the lower dimension: insertion into an
             ordered list of dimension indices */
          int m = 0;
          for (int f = 0; f < D; ++f) {
            int p = m < d ? m : d;
            while (p > 0 && dist[ord[p - 1]] > dist[f]) --p;
            if (p >= d) continue;
            const int last = m < d ? m : d - 1;
            for (int q = last; q > p; --q) ord[q] = ord[q - 1];
            ord[p] = f;
            if (m < d) ++m;
          }
          double sum = 0.0, mx = 0.0;
          uint64_t dims = 0;
          for (int q = 0; q < d; ++q) {
            sum += dist[ord[q]];
            if (dist[ord[q]] > mx) mx = dist[ord[q]];
            dims |= (uint64_t)1 << ord[q];
          }
          if (sum <= tau) {
            int64_t slot;
#pragma omp atomic capture
            slot = found++;
            if (slot < cap) {
              out[slot].a = a;
              out[slot].b = b;
              out[slot].dist_d = sum;
              out[slot].dist_max = mx;
              out[slot].dims = dims;
            }
          }
        }
      }
    }
  }
  free(X);
  free(mu);
  free(wmu);
  free(isw);
  free(flat);
  return found;
}
