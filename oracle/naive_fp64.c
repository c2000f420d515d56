/*
 * Oracle for NaivePT (test infrastructure only).
 *
 * Plain FP64 CPU statement of what the exhaustive permutation test computes:
 *   - Alg. 1 (NaivePT): for every relabelling i, the first n1 entries of the
 *     permuted index list form group 1, the rest group 2; compute the
 *     voxel-wise statistic for every voxel and take the column maximum m_i.
 *   - Eq. (5), read as the pooled-variance two-sample t (Sec. 3.2 calls the
 *     normaliser "pooled variances"):
 *         t = (mean1 - mean2) / sqrt( sp2 * (1/n1 + 1/n2) ),
 *         sp2 = ( sum_{G1} (x - mean1)^2 + sum_{G2} (x - mean2)^2 ) / (n - 2).
 *   - Max statistic / max-null (Sec. 2, "The case for strong null"): the
 *     histogram of the per-relabelling maxima m_i over all voxels.
 *   - Per-voxel uncorrected exceedance count: #{i : t_ij >= t_obs_j}, with
 *     t_obs the statistic of the observed (identity) labelling.
 *
 * Group sums are taken in subject order 0..n-1 (membership tested from a
 * label vector), so two relabellings with the same group-1 set produce
 * bit-identical statistics. Voxels whose values are all equal (zero total
 * sum of squares) have no defined t; they are excluded from the maxima and
 * their counts are 0.
 *
 * Only tests, the smoke check and the CPU-baseline leg of the benchmark use
 * this file. It shares no code with the CUDA path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Returns 0 if row is a permutation of 0..n-1, else 1. Fills g1[s] = 1 for
 * subjects in the first n1 positions. */
static int labels_from_perm(const int32_t* row, int n, int n1, unsigned char* g1,
                            unsigned char* seen) {
  memset(g1, 0, (size_t)n);
  memset(seen, 0, (size_t)n);
  for (int q = 0; q < n; ++q) {
    int32_t s = row[q];
    if (s < 0 || s >= n || seen[s]) return 1;
    seen[s] = 1;
    if (q < n1) g1[s] = 1;
  }
  return 0;
}

/* Pooled-variance two-sample t of one voxel (x has n entries), Eq. (5). */
static double t_two_sample(const double* x, const unsigned char* g1, int n, int n1) {
  const int n2 = n - n1;
  double sum1 = 0.0, sum2 = 0.0;
  for (int s = 0; s < n; ++s) {
    if (g1[s]) sum1 += x[s];
    else sum2 += x[s];
  }
  const double mean1 = sum1 / n1, mean2 = sum2 / n2;
  double ss = 0.0;
  for (int s = 0; s < n; ++s) {
    const double d = x[s] - (g1[s] ? mean1 : mean2);
    ss += d * d;
  }
  const double sp2 = ss / (double)(n - 2);
  return (mean1 - mean2) / sqrt(sp2 * (1.0 / n1 + 1.0 / n2));
}

/* Voxel j is degenerate when all n values are equal. */
static int voxel_degenerate(const double* x, int n) {
  for (int s = 1; s < n; ++s)
    if (x[s] != x[0]) return 0;
  return 1;
}

static double stat_of(double t, int two_sided) { return two_sided ? fabs(t) : t; }

/* The statistic as the group-1 share of the unit-norm centred voxel:
 * u = t / sqrt(k (n-2) + k t^2), k = 1/n1 + 1/n2. It is the exact inverse of
 * t = sqrt(k(n-2)) u / sqrt(1 - k u^2), strictly increasing, and well
 * conditioned for every t; near-ties are judged on this scale. */
static double u_of(double t, int n, int n1) {
  const double k = 1.0 / n1 + 1.0 / (n - n1);
  if (isinf(t)) return t > 0 ? 1.0 / sqrt(k) : -1.0 / sqrt(k);
  return t / sqrt(k * (n - 2) + k * t * t);
}

/* sum_s |x_s - mean| / sqrt(sum_s (x_s - mean)^2): the l1 norm of the
 * unit-norm centred voxel (scale of the rounding error of a group sum). */
static double l1_unit(const double* x, int n) {
  double m = 0.0;
  for (int s = 0; s < n; ++s) m += x[s];
  m /= n;
  double ss = 0.0, a = 0.0;
  for (int s = 0; s < n; ++s) {
    ss += (x[s] - m) * (x[s] - m);
    a += fabs(x[s] - m);
  }
  return ss > 0.0 ? a / sqrt(ss) : 0.0;
}

/*
 * Full NaivePT over P relabellings.
 *   Xt      : v x n, voxel-major FP64 data (row j = the n subjects of voxel j)
 *   perms   : P x n int32, each row a permutation of 0..n-1
 *   outputs : maxnull[P], argmax[P] (smallest voxel index on ties; -1 if no
 *             valid voxel), second[P] (largest statistic over the other
 *             voxels, -inf if none), counts[v], t_obs[v] (NAN if degenerate),
 *             tau[v] = tie_rel * (l1 norm of the unit-norm centred voxel),
 *             near[v] = #{i : |u(stat_ij) - u(stat_obs_j)| <= tau_j}, with u()
 *             the monotone rescaling above (near-ties with the observed value)
 *   two_sided: 0 -> statistic t, 1 -> |t|
 * Returns 0 on success, 1 + (first invalid row) if a row is not a permutation,
 * -1 on bad sizes or allocation failure.
 */
int64_t oracle_naive(const double* Xt, int n, int64_t v, int n1, const int32_t* perms,
                     int64_t P, int two_sided, int nthreads, double tie_rel,
                     double* maxnull, int64_t* argmax, double* second, uint32_t* counts,
                     double* t_obs, uint32_t* near, double* tau) {
  if (n < 3 || n1 < 1 || n1 > n - 1 || v < 0 || P < 0) return -1;
  unsigned char* degen = (unsigned char*)malloc((size_t)(v > 0 ? v : 1));
  unsigned char* g1 = (unsigned char*)malloc((size_t)n);
  unsigned char* seen = (unsigned char*)malloc((size_t)n);
  int32_t* ident = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  if (!degen || !g1 || !seen || !ident) return -1;
  for (int s = 0; s < n; ++s) ident[s] = s;
  labels_from_perm(ident, n, n1, g1, seen);
  for (int64_t j = 0; j < v; ++j) {
    const double* x = Xt + (size_t)j * n;
    degen[j] = (unsigned char)voxel_degenerate(x, n);
    t_obs[j] = degen[j] ? NAN : t_two_sample(x, g1, n, n1);
    tau[j] = tie_rel * l1_unit(x, n);
  }
  int64_t bad_row = -1;
  for (int64_t i = 0; i < P; ++i) {
    if (labels_from_perm(perms + (size_t)i * n, n, n1, g1, seen)) {
      bad_row = i;
      break;
    }
  }
  free(g1);
  free(seen);
  free(ident);
  if (bad_row >= 0) {
    free(degen);
    return 1 + bad_row;
  }
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  memset(counts, 0, sizeof(uint32_t) * (size_t)v);
  memset(near, 0, sizeof(uint32_t) * (size_t)v);
  int failed = 0;
#pragma omp parallel
  {
    uint32_t* cnt = (uint32_t*)calloc((size_t)(v > 0 ? v : 1), sizeof(uint32_t));
    uint32_t* nr = (uint32_t*)calloc((size_t)(v > 0 ? v : 1), sizeof(uint32_t));
    unsigned char* lab = (unsigned char*)malloc((size_t)n);
    unsigned char* sn = (unsigned char*)malloc((size_t)n);
    if (!cnt || !nr || !lab || !sn) {
#pragma omp atomic write
      failed = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t i = 0; i < P; ++i) {
        labels_from_perm(perms + (size_t)i * n, n, n1, lab, sn);
        double best = -INFINITY, second_best = -INFINITY;
        int64_t best_j = -1;
        for (int64_t j = 0; j < v; ++j) {
          if (degen[j]) continue;
          const double st = stat_of(t_two_sample(Xt + (size_t)j * n, lab, n, n1), two_sided);
          const double so = stat_of(t_obs[j], two_sided);
          if (st >= so) cnt[j] += 1;
          if (fabs(u_of(st, n, n1) - u_of(so, n, n1)) <= tau[j]) nr[j] += 1;
          if (best_j < 0 || st > best) {
            if (best_j >= 0) second_best = fmax(second_best, best);
            best = st;
            best_j = j;
          } else {
            second_best = fmax(second_best, st);
          }
        }
        maxnull[i] = best;
        argmax[i] = best_j;
        second[i] = second_best;
      }
#pragma omp critical
      {
        for (int64_t j = 0; j < v; ++j) {
          counts[j] += cnt[j];
          near[j] += nr[j];
        }
      }
    }
    free(cnt);
    free(nr);
    free(lab);
    free(sn);
  }
  free(degen);
  return failed ? -1 : 0;
}

/*
 * Rows of the permutation testing matrix T (Sec. 2.1), P x v, FP64:
 * T[i][j] = t of voxel j under relabelling i (NAN for degenerate voxels).
 * Same return convention as oracle_naive.
 */
int64_t oracle_t_rows(const double* Xt, int n, int64_t v, int n1, const int32_t* perms,
                      int64_t P, int nthreads, double* T) {
  if (n < 3 || n1 < 1 || n1 > n - 1 || v < 0 || P < 0) return -1;
  unsigned char* g1 = (unsigned char*)malloc((size_t)n);
  unsigned char* seen = (unsigned char*)malloc((size_t)n);
  if (!g1 || !seen) return -1;
  for (int64_t i = 0; i < P; ++i) {
    if (labels_from_perm(perms + (size_t)i * n, n, n1, g1, seen)) {
      free(g1);
      free(seen);
      return 1 + i;
    }
  }
  free(g1);
  free(seen);
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
#pragma omp parallel
  {
    unsigned char* lab = (unsigned char*)malloc((size_t)n);
    unsigned char* sn = (unsigned char*)malloc((size_t)n);
#pragma omp for schedule(dynamic, 1)
    for (int64_t i = 0; i < P; ++i) {
      labels_from_perm(perms + (size_t)i * n, n, n1, lab, sn);
      for (int64_t j = 0; j < v; ++j) {
        const double* x = Xt + (size_t)j * n;
        T[(size_t)i * v + j] = voxel_degenerate(x, n) ? NAN : t_two_sample(x, lab, n, n1);
      }
    }
    free(lab);
    free(sn);
  }
  return 0;
}

/*
 * Statistic at selected entries: out[q] = t of voxel idx[q] under
 * relabelling rows[q] of perms (used for the sampled entries of the
 * recovery phase, Alg. 2). Degenerate voxels give NAN.
 */
int64_t oracle_t_entries(const double* Xt, int n, int64_t v, int n1, const int32_t* perms,
                         const int64_t* rows, const int64_t* idx, int64_t Q, double* out) {
  if (n < 3 || n1 < 1 || n1 > n - 1) return -1;
  unsigned char* g1 = (unsigned char*)malloc((size_t)n);
  unsigned char* seen = (unsigned char*)malloc((size_t)n);
  if (!g1 || !seen) return -1;
  int64_t last = -1;
  int64_t rc = 0;
  for (int64_t q = 0; q < Q; ++q) {
    if (idx[q] < 0 || idx[q] >= v) {
      rc = -1;
      break;
    }
    if (rows[q] != last) {
      if (labels_from_perm(perms + (size_t)rows[q] * n, n, n1, g1, seen)) {
        rc = 1 + rows[q];
        break;
      }
      last = rows[q];
    }
    const double* x = Xt + (size_t)idx[q] * n;
    out[q] = voxel_degenerate(x, n) ? NAN : t_two_sample(x, g1, n, n1);
  }
  free(g1);
  free(seen);
  return rc;
}
