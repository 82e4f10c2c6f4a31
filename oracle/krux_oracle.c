/*
 * krux_oracle.c -- FP64 CPU oracle for the Kruskal-Wallis SNP x trait scan.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline / reference leg may load this library.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * What it computes (Qi et al., "kruX: Matrix-based non-parametric eQTL
 * discovery", arXiv:1307.3519): for every (trait n, SNP m) pair the
 * tie-corrected Kruskal-Wallis statistic and its chi-square p-value, taken
 * straight from the definition, one pair at a time -- the "one-by-one" check the
 * paper validates its matrix method against (section "kruX is exact and fast").
 * Per pair:
 *   1. the sample set U = samples whose genotype is not missing (-1) and whose
 *      expression is not NaN (section "Handling missing values": ranks are over
 *      the observed samples only), K = |U|;
 *   2. sort the expression values of U and give each run of equal values the
 *      average of the 1-based positions it occupies (section "Input data":
 *      ranks per trait; ties get average ranks); accumulate sum(t^3 - t) over
 *      the runs (section "Handling tied data");
 *   3. rank sums S_i and counts N_i of each genotype group i = 0..l (Eq. 4;
 *      section "Input data": markers take values 0..l, l = 2 for biallelic
 *      markers, and any number of alleles is allowed);
 *   4. S = 12/(K(K+1)) * sum_{i: N_i>0} S_i^2/N_i - 3(K+1) (Eq. 2; empty groups
 *      contribute nothing, the paper's NaN -> 0 rule);
 *   5. divide by 1 - sum(t^3-t)/(K^3-K) (section "Handling tied data");
 *   6. df = (number of non-empty groups) - 1; p = upper chi-square tail with df
 *      degrees of freedom (section "P-value calculation"), from the closed
 *      forms of the regularised upper incomplete gamma function Q(df/2, H/2)
 *      for integer and half-integer shapes (df = 1: erfc(sqrt(H/2)); df = 2:
 *      exp(-H/2));
 *   7. the pair is a hit iff p < P_c.
 * Degenerate pairs (df = 0, K < 2, or all values tied so the tie factor is 0)
 * get H = 0, p = 1 and are never hits.
 *
 * Parity pins for every function here live in tests/test_oracle.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  double H;        /* tie-corrected statistic                                  */
  double H_alt;    /* same statistic from the variance-ratio textbook form    */
  double p;        /* chi-square upper tail                                    */
  double tie;      /* sum over tie runs of t^3 - t                             */
  int64_t rank2[5];/* twice the rank sum of each genotype group: 2*S_i        */
  int64_t d[5];    /* centred sums 2*S_i - N_i*(K+1)                           */
  int32_t n[5];    /* group sizes N_i                                          */
  int32_t K;       /* samples used                                            */
  int32_t df;      /* degrees of freedom                                      */
  int32_t hit;     /* p < P_c                                                 */
} oracle_pair_t;

typedef struct {
  float v;
  int32_t k;
} keyed_t;

static int cmp_keyed(const void *a, const void *b) {
  const keyed_t *x = (const keyed_t *)a, *y = (const keyed_t *)b;
  if (x->v < y->v) return -1;
  if (x->v > y->v) return 1;
  return (x->k > y->k) - (x->k < y->k);
}

/* Average ranks (as 2*rank, an integer) of the present values of one row, in the
 * original sample order; absent samples (mask 0) get 0.  Returns K and the tie
 * sum sum(t^3 - t).  work must hold n entries. */
static int32_t rank_row(const float *x, const unsigned char *use, int n,
                        int64_t *rank2, double *tie, keyed_t *work) {
  int32_t K = 0;
  for (int k = 0; k < n; ++k) {
    rank2[k] = 0;
    if (use[k]) {
      work[K].v = x[k];
      work[K].k = k;
      ++K;
    }
  }
  qsort(work, (size_t)K, sizeof(keyed_t), cmp_keyed);
  double ts = 0.0;
  int i = 0;
  while (i < K) {
    int j = i;
    while (j + 1 < K && work[j + 1].v == work[i].v) ++j;
    /* positions i..j (0-based) share the average of 1-based ranks i+1..j+1,
     * i.e. (i + j + 2) / 2; store twice that */
    for (int q = i; q <= j; ++q) rank2[work[q].k] = (int64_t)(i + j + 2);
    double t = (double)(j - i + 1);
    ts += t * t * t - t;
    i = j + 1;
  }
  *tie = ts;
  return K;
}

/* Upper tail of the chi-square law with df degrees of freedom at H:
 * Q(df/2, x), x = H/2, the regularised upper incomplete gamma function.  For an
 * integer shape m (df = 2m):      Q(m, x)     = e^-x sum_{k<m} x^k / k!;
 * for a half-integer shape (df = 2m+1): Q(m+1/2, x) = erfc(sqrt x)
 *                                     + e^-x sum_{k=1..m} x^(k-1/2) / Gamma(k+1/2),
 * with Gamma(k+1/2) = Gamma(k-1/2) * (k-1/2) and Gamma(1/2) = sqrt(pi). */
static double chi2_upper(double H, int df) {
  if (df <= 0) return 1.0;
  const double x = 0.5 * H;
  if (df % 2 == 0) {
    double term = 1.0, sum = 0.0;
    for (int k = 0; k < df / 2; ++k) {
      if (k > 0) term *= x / (double)k;
      sum += term;
    }
    return exp(-x) * sum;
  }
  if (!(x > 0.0)) return 1.0;
  double q = erfc(sqrt(x));
  double g = sqrt(3.14159265358979323846); /* Gamma(1/2) = sqrt(pi) */
  double xp = 1.0 / sqrt(x);   /* x^(-1/2) */
  for (int k = 1; k <= df / 2; ++k) {
    g *= (double)k - 0.5;           /* Gamma(k + 1/2) */
    xp *= x;                         /* x^(k - 1/2) */
    q += exp(-x) * xp / g;
  }
  return q;
}

/* One (trait, SNP) pair.  x: expression of the trait over n samples (NaN =
 * missing); g: genotype codes of the SNP (0..lmax; -1 = missing), lmax <= 4.
 * Returns 0, or -1 if a genotype code is outside {-1, 0..lmax}. */
int oracle_pair_l(const float *x, const int8_t *g, int n, int lmax, double pthresh,
                  oracle_pair_t *out) {
  memset(out, 0, sizeof(*out));
  unsigned char *use = (unsigned char *)malloc((size_t)n + 1);
  int64_t *r2 = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
  keyed_t *work = (keyed_t *)malloc(sizeof(keyed_t) * ((size_t)n + 1));
  int rc = 0;
  if (lmax < 1 || lmax > 4) rc = -1;
  for (int k = 0; k < n; ++k) {
    if (g[k] < -1 || g[k] > lmax) rc = -1;
    use[k] = (g[k] >= 0 && g[k] <= lmax && !isnan(x[k])) ? 1 : 0;
  }
  if (rc != 0) goto done;

  double tie = 0.0;
  int32_t K = rank_row(x, use, n, r2, &tie, work);
  out->K = K;
  out->tie = tie;
  for (int k = 0; k < n; ++k) {
    if (!use[k]) continue;
    out->rank2[g[k]] += r2[k];
    out->n[g[k]] += 1;
  }
  int groups = 0;
  for (int i = 0; i <= lmax; ++i) {
    out->d[i] = out->rank2[i] - (int64_t)out->n[i] * (int64_t)(K + 1);
    if (out->n[i] > 0) ++groups;
  }
  out->df = groups > 0 ? groups - 1 : 0;

  double Kd = (double)K;
  double corr = (K >= 2) ? 1.0 - tie / (Kd * Kd * Kd - Kd) : 0.0;
  if (out->df == 0 || K < 2 || !(corr > 0.0)) {
    out->H = 0.0;
    out->H_alt = 0.0;
    out->p = 1.0;
    out->hit = 0;
    goto done;
  }
  /* Eq. 2 with rank sums S_i = rank2_i / 2, empty groups skipped */
  double acc = 0.0;
  for (int i = 0; i <= lmax; ++i) {
    if (out->n[i] == 0) continue;
    double Si = 0.5 * (double)out->rank2[i];
    acc += Si * Si / (double)out->n[i];
  }
  double H = 12.0 / (Kd * (Kd + 1.0)) * acc - 3.0 * (Kd + 1.0);
  H /= corr;
  if (H < 0.0) H = 0.0; /* rounding below an exact zero */

  /* Variance-ratio form: (K-1) * sum_i N_i (mean_i - mean)^2 / sum_k (r_k - mean)^2,
   * which includes the tie correction by construction. */
  double mean = 0.5 * (Kd + 1.0);
  double num = 0.0, den = 0.0;
  for (int i = 0; i <= lmax; ++i) {
    if (out->n[i] == 0) continue;
    double mi = 0.5 * (double)out->rank2[i] / (double)out->n[i];
    num += (double)out->n[i] * (mi - mean) * (mi - mean);
  }
  for (int k = 0; k < n; ++k) {
    if (!use[k]) continue;
    double r = 0.5 * (double)r2[k];
    den += (r - mean) * (r - mean);
  }
  out->H_alt = (Kd - 1.0) * num / den;

  out->H = H;
  out->p = chi2_upper(H, out->df);
  out->hit = out->p < pthresh ? 1 : 0;
done:
  free(use);
  free(r2);
  free(work);
  return rc;
}

/* Biallelic form (codes 0, 1, 2). */
int oracle_pair(const float *x, const int8_t *g, int n, double pthresh, oracle_pair_t *out) {
  return oracle_pair_l(x, g, n, 2, pthresh, out);
}

/* Upper chi-square tail, exported for the pins. */
double oracle_chi2_upper(double H, int df) { return chi2_upper(H, df); }

/* Ranks of one expression row over its non-NaN samples: 2*average rank (0 for
 * NaN), the tie sum and K (section "Input data", "Handling missing values",
 * "Handling tied data"). */
int32_t oracle_rank_row(const float *x, int n, int64_t *rank2, double *tie) {
  unsigned char *use = (unsigned char *)malloc((size_t)n + 1);
  keyed_t *work = (keyed_t *)malloc(sizeof(keyed_t) * ((size_t)n + 1));
  for (int k = 0; k < n; ++k) use[k] = isnan(x[k]) ? 0 : 1;
  int32_t K = rank_row(x, use, n, rank2, tie, work);
  free(use);
  free(work);
  return K;
}

/* Dense scan over a trait subset x SNP subset.  expr: T rows of ldx floats;
 * geno: rows of ldg int8.  traits[nt], snps[ns] select the pairs; outputs are
 * nt x ns row-major (any output pointer may be NULL).  perm, if not NULL, is a
 * permutation of 0..N-1 applied to the expression columns: sample k of the
 * pair takes expression value x[perm[k]] (section "P-value calculation and
 * empirical FDR correction": the columns of the expression ranks are
 * permuted).  Returns 0 or -1 (bad genotype code). */
int oracle_scan_l(const float *expr, int64_t ldx, const int8_t *geno, int64_t ldg,
                  int N, int lmax, const int64_t *traits, int64_t nt, const int64_t *snps,
                  int64_t ns, const int32_t *perm, double pthresh, double *H,
                  double *p, int32_t *df, int64_t *d, int32_t *nk, int32_t *K,
                  uint8_t *hit, double *H_alt) {
  const int ng = lmax + 1;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
  for (int64_t a = 0; a < nt; ++a) {
    float *x = (float *)malloc(sizeof(float) * (size_t)N);
    const float *row = expr + traits[a] * ldx;
    for (int k = 0; k < N; ++k) x[k] = perm ? row[perm[k]] : row[k];
    for (int64_t b = 0; b < ns; ++b) {
      oracle_pair_t r;
      if (oracle_pair_l(x, geno + snps[b] * ldg, N, lmax, pthresh, &r) != 0) bad |= 1;
      int64_t o = a * ns + b;
      if (H) H[o] = r.H;
      if (p) p[o] = r.p;
      if (df) df[o] = r.df;
      if (d) for (int i = 0; i < ng; ++i) d[ng * o + i] = r.d[i];
      if (nk) for (int i = 0; i < ng; ++i) nk[ng * o + i] = r.n[i];
      if (K) K[o] = r.K;
      if (hit) hit[o] = (uint8_t)r.hit;
      if (H_alt) H_alt[o] = r.H_alt;
    }
    free(x);
  }
  return bad ? -1 : 0;
}

/* Biallelic dense scan (codes 0, 1, 2). */
int oracle_scan(const float *expr, int64_t ldx, const int8_t *geno, int64_t ldg,
                int N, const int64_t *traits, int64_t nt, const int64_t *snps,
                int64_t ns, const int32_t *perm, double pthresh, double *H,
                double *p, int32_t *df, int64_t *d, int32_t *nk, int32_t *K,
                uint8_t *hit, double *H_alt) {
  return oracle_scan_l(expr, ldx, geno, ldg, N, 2, traits, nt, snps, ns, perm, pthresh, H, p, df,
                       d, nk, K, hit, H_alt);
}

/* Permutation null: for each permutation q and trait a, the minimum p over
 * all selected SNPs of the scan with expression columns permuted by
 * perms[q] (section "P-value calculation and empirical FDR correction").
 * minp is P x nt row-major. */
int oracle_perm_minp(const float *expr, int64_t ldx, const int8_t *geno,
                     int64_t ldg, int N, const int64_t *traits, int64_t nt,
                     const int64_t *snps, int64_t ns, const int32_t *perms,
                     int P, double *minp) {
  int bad = 0;
#pragma omp parallel for collapse(2) schedule(dynamic, 1) reduction(| : bad)
  for (int q = 0; q < P; ++q) {
    for (int64_t a = 0; a < nt; ++a) {
      float *x = (float *)malloc(sizeof(float) * (size_t)N);
      const float *row = expr + traits[a] * ldx;
      const int32_t *pi = perms + (int64_t)q * N;
      for (int k = 0; k < N; ++k) x[k] = row[pi[k]];
      double best = 1.0;
      for (int64_t b = 0; b < ns; ++b) {
        oracle_pair_t r;
        if (oracle_pair(x, geno + snps[b] * ldg, N, 1.0, &r) != 0) bad |= 1;
        if (r.p < best) best = r.p;
      }
      minp[(int64_t)q * nt + a] = best;
      free(x);
    }
  }
  return bad ? -1 : 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
