/*
 * oracle.c -- plain, slow, CPU reference for the Monte Carlo simulation of
 * Kolmogorov-Smirnov cutoffs for the discrete power law (Zipf / zeta law)
 * with a maximum-likelihood exponent, after Rappos & Robert,
 * "Using GPU Simulation to Accurately Fit to the Power-Law Distribution"
 * (2013).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the
 * CUDA library: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * Everything is IEEE binary64 (double), no fast-math, no blocking or fusion
 * beyond what the definitions below state.  Each function names the passage
 * of the paper it follows; where the paper is silent the reading adopted is
 * stated in the comment.
 *
 * Notation: the paper writes the exponent gamma and the sample size N; here
 * they are alpha and n.  xmin is the lower end of the support (the paper has
 * xmin = 1; the Hurwitz generalisation p(k) = k^-alpha / zeta(alpha, xmin),
 * k >= xmin, reduces to Eq. 1 at xmin = 1).
 *
 * Parity status (pins live in tests/):
 *   or_philox4x32_10 ..... pinned (cuRAND host Philox4_32_10 generator)
 *   or_hurwitz3 .......... pinned (pi^2/6, pi^4/90, mpmath/scipy values,
 *                          shift identity)
 *   or_survival/or_invert  pinned (pmf sums to 1, chi-square of draws,
 *                          brute-force inverse CDF on small cases)
 *   or_mle ............... pinned (log-likelihood grid argmax, mpmath root,
 *                          Table 1 all-ones atoms)
 *   or_ks / or_ks_brute .. pinned (brute force over every integer, Table 1
 *                          atoms, exact enumeration for n <= 4)
 *   or_quantile .......... pinned (integer index rule, Table 1 cells)
 *   or_bootstrap_pvalue .. pinned (uniformity of p under the null, power
 *                          against lognormal data)
 *   or_tz_* (truncated) .. pinned (zeta_K closed forms and mpmath,
 *                          linear-search inverse CDF, chi-square of draws,
 *                          log-likelihood argmax, uniform data -> 0,
 *                          D by definition, Tables 2-6 cells, K=20 atom)
 *   or_estimate_xmin ..... pinned (planted lower ends, pure power law,
 *                          candidates against the brute-force KS)
 *   or_binomial/or_mn_* .. pinned (pmf against SciPy, chi-square of the
 *                          binomial and of the bin counts, D distribution
 *                          against the inverse-CDF sampler's)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_ENOCONV 3

/* Samples saturate here: the paper's support is bounded (K < 32,766) so it
 * never meets the issue; for the untruncated law at alpha <= 2 the inverse
 * CDF can exceed any integer type, so values are capped at 2^62. */
#define OR_XCAP ((uint64_t)1 << 62)

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11).  The paper draws
 * from cuRAND's default generator (Section 4); a counter-based generator is
 * substituted so that every draw is a pure function of
 * (seed, cell, replicate, purpose, index).                                  */

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                      uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
    uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(prod_b >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)prod_b;
    uint32_t y2 = (uint32_t)(prod_a >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)prod_a;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Draw i of stream (seed, cell, rep, purpose), key (seed_lo, seed_hi): its
 * high word h is word j = i mod 4 of the Philox block with counter
 * (floor(i/4), rep, cell, purpose), its low word l word j of the block with
 * counter (floor(i/4), rep, cell, purpose + 2^31) (purposes are below 2^31).
 * m = h 2^21 + floor(l / 2^11) + 1 lies in [1, 2^53] (53 random bits) and the
 * uniform is v = m 2^-53 in (0, 1], the same half-open interval as the
 * double-precision uniform the paper's sampler consumes. */
#define OR_LOW_STREAM 0x80000000u
uint64_t or_draw_m(uint64_t seed, uint32_t cell, uint32_t rep,
                   uint32_t purpose, uint64_t i) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t ctr_hi[4] = {(uint32_t)(i >> 2), rep, cell, purpose};
  uint32_t ctr_lo[4] = {(uint32_t)(i >> 2), rep, cell, purpose | OR_LOW_STREAM};
  uint32_t wh[4], wl[4];
  or_philox4x32_10(ctr_hi, key, wh);
  or_philox4x32_10(ctr_lo, key, wl);
  int j = (int)(i & 3);
  return (((uint64_t)wh[j] << 21) | (uint64_t)(wl[j] >> 11)) + 1;
}

/* ------------------------------------------------------------------------ */
/* Hurwitz zeta zeta(s, a) = sum_{k>=0} (a+k)^-s and its first two
 * derivatives in s, by Euler-Maclaurin summation (DLMF 2.10.1, 25.11):
 *   zeta(s,a) = sum_{k<M} (a+k)^-s + N^(1-s)/(s-1) + N^-s/2
 *             + sum_{j=1..J} B_2j/(2j)! * s(s+1)...(s+2j-2) * N^(-s-2j+1),
 * N = a + M.  The paper sums the (finite) normaliser term by term (Section 4
 * and Eq. 2); for the untruncated law Euler-Maclaurin replaces the infinite
 * sum.  Derivatives are taken term by term; the rising factorial P_j(s) and
 * its derivatives follow the product rule.  Oracle parameters: J = 10
 * Bernoulli terms and N >= max(24, s + 24); the first omitted term is then
 * below (2 pi)^-22 ~ 3e-18 of the integral term for every s > 1 (the series
 * is asymptotic: with N much smaller than s it diverges before it helps).  */

static const double OR_BERNOULLI_2J[10] = {
    1.0 / 6.0,         -1.0 / 30.0,      1.0 / 42.0,     -1.0 / 30.0,
    5.0 / 66.0,        -691.0 / 2730.0,  7.0 / 6.0,      -3617.0 / 510.0,
    43867.0 / 798.0,   -174611.0 / 330.0};

void or_hurwitz3(double s, double a, double out[3]) {
  const double n_floor = ceil(s) + 24.0;
  double z0 = 0.0, z1 = 0.0, z2 = 0.0;
  int M = 0;
  if (a < n_floor) M = (int)ceil(n_floor - a);
  for (int k = 0; k < M; ++k) {
    double x = a + (double)k;
    double lx = log(x);
    double t = pow(x, -s);
    z0 += t;
    z1 -= lx * t;
    z2 += lx * lx * t;
  }
  double N = a + (double)M;
  double L = log(N);
  double Ns = pow(N, -s);            /* N^-s */
  double u = 1.0 / (s - 1.0);
  /* integral term N^(1-s)/(s-1) */
  double N1s = N * Ns;
  z0 += N1s * u;
  z1 += -N1s * (L * u + u * u);
  z2 += N1s * (L * L * u + 2.0 * L * u * u + 2.0 * u * u * u);
  /* end-point term N^-s / 2 */
  z0 += 0.5 * Ns;
  z1 += -0.5 * L * Ns;
  z2 += 0.5 * L * L * Ns;
  /* Bernoulli terms */
  double P = s, dP = 1.0, d2P = 0.0; /* P_1(s) = s */
  double Npow = Ns / N;              /* N^(-s-1) */
  double fact = 2.0;                 /* (2j)! */
  for (int j = 1; j <= 10; ++j) {
    double c = OR_BERNOULLI_2J[j - 1] / fact;
    z0 += c * Npow * P;
    z1 += c * Npow * (dP - L * P);
    z2 += c * Npow * (d2P - 2.0 * L * dP + L * L * P);
    for (int f = 2 * j - 1; f <= 2 * j; ++f) {
      double g = s + (double)f;
      d2P = d2P * g + 2.0 * dP;
      dP = dP * g + P;
      P = P * g;
    }
    Npow /= N * N;
    fact *= (double)(2 * j + 1) * (double)(2 * j + 2);
  }
  out[0] = z0;
  out[1] = z1;
  out[2] = z2;
}

double or_hurwitz(double s, double a) {
  double z[3];
  or_hurwitz3(s, a, z);
  return z[0];
}

/* ------------------------------------------------------------------------ */
/* The law (Eq. 1, generalised to a lower end xmin):
 *   p(k) = k^-alpha / zeta(alpha, xmin),  k >= xmin,
 * with survival function Q(k) = P(X > k) = zeta(alpha, k+1) / zeta(alpha,
 * xmin); Q(xmin - 1) = 1.  Z is zeta(alpha, xmin).                          */

double or_pmf(double alpha, uint64_t xmin, uint64_t k) {
  if (k < xmin) return 0.0;
  return pow((double)k, -alpha) / or_hurwitz(alpha, (double)xmin);
}

double or_survival(double alpha, double Z, uint64_t xmin, uint64_t k) {
  if (k < xmin) return 1.0;
  return or_hurwitz(alpha, (double)k + 1.0) / Z;
}

/* Inverse-CDF sampling (the paper's sampler, Section 4: the smallest value
 * whose cumulative probability reaches the uniform).  Reading: with v in
 * (0,1], X = min{k >= xmin : Q(k) < v}, which has P(X = k) = p(k) and uses
 * the survival function so that tail values keep full relative accuracy.
 * Plain exponential search then bisection on k.  The result is
 * min(OR_XCAP, that k): values beyond the cap saturate at OR_XCAP. */
uint64_t or_invert(double alpha, double Z, uint64_t xmin, uint64_t m) {
  double v = ldexp((double)m, -53);
  uint64_t lo = xmin; /* answer >= lo: Q(lo - 1) >= v */
  uint64_t span = 1, hi;
  if (lo >= OR_XCAP) return OR_XCAP;
  for (;;) {
    hi = lo + span - 1;
    if (hi >= OR_XCAP) hi = OR_XCAP;
    if (or_survival(alpha, Z, xmin, hi) < v) break;
    if (hi == OR_XCAP) return OR_XCAP; /* answer beyond the cap */
    lo = hi + 1;
    span *= 2;
  }
  while (lo < hi) {
    uint64_t mid = lo + (hi - lo) / 2;
    if (or_survival(alpha, Z, xmin, mid) < v)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

/* n draws of replicate rep (stream tag purpose) of cell `cell`. */
void or_sample(double alpha, uint64_t xmin, uint64_t seed, uint32_t cell,
               uint32_t rep, uint32_t purpose, int64_t n, uint64_t *out) {
  double Z = or_hurwitz(alpha, (double)xmin);
  for (int64_t i = 0; i < n; ++i)
    out[i] = or_invert(alpha, Z, xmin, or_draw_m(seed, cell, rep, purpose,
                                                  (uint64_t)i));
}

/* ------------------------------------------------------------------------ */
/* Maximum-likelihood exponent (Eq. 2 generalised to xmin):
 *   zeta'(alpha, xmin) / zeta(alpha, xmin) = -(1/n) sum_i ln x_i.
 * f(alpha) = zeta'/zeta + mbar is increasing in alpha (its derivative is
 * the variance of ln X), so the root is unique.  Newton-Raphson (as the
 * paper prescribes, Section 2) safeguarded by bisection on the bracket
 * (1 + 2^-40, 64], started at the continuous-law estimate
 * 1 + 1/(mbar - ln(xmin - 1/2)), stopped when a step is within 4 ulp.
 * Reading: the paper's absolute 1e-5 step tolerance is replaced by
 * convergence to the FP64 root.
 * All-equal rule (Section 4's code comment: "as if one point was 2"): when
 * every x_i equals xmin the root is at infinity; L is then increased by
 * ln((xmin+1)/xmin), i.e. one point is treated as xmin+1 in the log-sum.   */

static void or_neumaier_add(double *sum, double *comp, double x) {
  double t = *sum + x;
  if (fabs(*sum) >= fabs(x))
    *comp += (*sum - t) + x;
  else
    *comp += (x - t) + *sum;
  *sum = t;
}

/* Sum of ln x_i with the all-equal rule applied.  Returns L. */
double or_log_sum(const uint64_t *x, int64_t n, uint64_t xmin) {
  double s = 0.0, c = 0.0;
  int all_min = 1;
  for (int64_t i = 0; i < n; ++i) {
    or_neumaier_add(&s, &c, log((double)x[i]));
    if (x[i] != xmin) all_min = 0;
  }
  if (all_min) or_neumaier_add(&s, &c, log1p(1.0 / (double)xmin));
  return s + c;
}

int or_mle_from_logsum(double L, int64_t n, uint64_t xmin, double *alpha_hat,
                       int *iterations) {
  if (n < 1 || xmin < 1) return OR_EINVAL;
  double mbar = L / (double)n;
  double lo = 1.0 + ldexp(1.0, -40), hi = 64.0;
  double a = 1.0 + 1.0 / (mbar - log((double)xmin - 0.5));
  if (!(a > lo && a < hi)) a = 0.5 * (lo + hi);
  int it;
  for (it = 1; it <= 200; ++it) {
    double z[3];
    or_hurwitz3(a, (double)xmin, z);
    double g = z[1] / z[0];
    double f = g + mbar;
    double fp = z[2] / z[0] - g * g;
    if (f > 0.0)
      hi = a;
    else
      lo = a;
    double next = a - f / fp;
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    double step = fabs(next - a);
    a = next;
    if (step <= 4.0 * ldexp(1.0, ilogb(a) - 52) || hi - lo <= 4.0 * ldexp(1.0, ilogb(a) - 52)) {
      if (iterations) *iterations = it;
      *alpha_hat = a;
      return OR_OK;
    }
  }
  if (iterations) *iterations = it;
  *alpha_hat = a;
  return OR_ENOCONV;
}

int or_mle(const uint64_t *x, int64_t n, uint64_t xmin, double *alpha_hat) {
  if (n < 1 || xmin < 1) return OR_EINVAL;
  for (int64_t i = 0; i < n; ++i)
    if (x[i] < xmin) return OR_EINVAL;
  return or_mle_from_logsum(or_log_sum(x, n, xmin), n, xmin, alpha_hat, 0);
}

/* ------------------------------------------------------------------------ */
/* Kolmogorov-Smirnov distance (Eq. 3): D = sup_x |F(x) - S(x)|, F the law
 * at the fitted exponent, S the empirical CDF.  Both are right-continuous
 * step functions with jumps only at integers, so the supremum over the reals
 * equals the maximum over integers t >= xmin (and for t < xmin both are 0).
 * F(t) = 1 - Q(t) with Q from the Hurwitz zeta.                            */

static int or_cmp_u64(const void *pa, const void *pb) {
  uint64_t a = *(const uint64_t *)pa, b = *(const uint64_t *)pb;
  return (a > b) - (a < b);
}

/* Brute force: every integer t from xmin to the sample maximum (beyond it
 * S = 1 and |F - 1| = Q(t) only decreases).  Cost grows with max x. */
int or_ks_brute(const uint64_t *x, int64_t n, uint64_t xmin, double alpha,
                double *D) {
  if (n < 1) return OR_EINVAL;
  uint64_t *s = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  if (!s) return OR_ENOMEM;
  memcpy(s, x, (size_t)n * sizeof(uint64_t));
  qsort(s, (size_t)n, sizeof(uint64_t), or_cmp_u64);
  double Z = or_hurwitz(alpha, (double)xmin);
  double best = 0.0;
  int64_t below = 0; /* number of samples <= t */
  for (uint64_t t = xmin; t <= s[n - 1]; ++t) {
    while (below < n && s[below] <= t) ++below;
    double F = 1.0 - or_survival(alpha, Z, xmin, t);
    double d = fabs(F - (double)below / (double)n);
    if (d > best) best = d;
  }
  free(s);
  *D = best;
  return OR_OK;
}

/* Same maximum, evaluated only where it can be attained: on each maximal
 * run of integers where S is constant, F is increasing, so |F - S| peaks at
 * one of the run's two ends.  The runs end at the distinct sample values v
 * and at v - 1, so D = max over distinct v of
 *   max(|F(v) - C(v)/n|, |F(v-1) - C(v-1)/n|),  C(t) = #{x_i <= t}. */
int or_ks(const uint64_t *x, int64_t n, uint64_t xmin, double alpha,
          double *D) {
  if (n < 1) return OR_EINVAL;
  uint64_t *s = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  if (!s) return OR_ENOMEM;
  memcpy(s, x, (size_t)n * sizeof(uint64_t));
  qsort(s, (size_t)n, sizeof(uint64_t), or_cmp_u64);
  double Z = or_hurwitz(alpha, (double)xmin);
  double best = 0.0;
  int64_t i = 0;
  while (i < n) {
    uint64_t v = s[i];
    int64_t j = i;
    while (j < n && s[j] == v) ++j;
    double F_v = 1.0 - or_survival(alpha, Z, xmin, v);
    double F_before = (v == xmin) ? 0.0 : 1.0 - or_survival(alpha, Z, xmin, v - 1);
    double d1 = fabs(F_v - (double)j / (double)n);
    double d0 = fabs(F_before - (double)i / (double)n);
    if (d1 > best) best = d1;
    if (d0 > best) best = d0;
    i = j;
  }
  free(s);
  *D = best;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* One Monte Carlo replicate (Section 4): draw n values at the true
 * exponent, fit alpha-hat by maximum likelihood, return the KS distance at
 * the fitted exponent (the paper evaluates the statistic at the estimate,
 * which is why generic KS tables do not apply, Section 3).                 */

int or_replicate(double alpha, uint64_t xmin, int64_t n, uint64_t seed,
                 uint32_t cell, uint32_t rep, uint32_t purpose,
                 double *alpha_hat, double *D) {
  uint64_t *x = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  if (!x) return OR_ENOMEM;
  or_sample(alpha, xmin, seed, cell, rep, purpose, n, x);
  int st = or_mle(x, n, xmin, alpha_hat);
  if (st == OR_OK || st == OR_ENOCONV) {
    int st2 = or_ks(x, n, xmin, *alpha_hat, D);
    if (st2 != OR_OK) st = st2;
  }
  free(x);
  return st;
}

/* Replicates rep0 .. rep0+R-1 of one cell; D[r], alpha_hat[r] for each.
 * Threads split the replicate range (OpenMP); results do not depend on
 * the thread count.  Returns the number of replicates whose Newton solve
 * did not converge via *nonconv. */
int or_cell(double alpha, uint64_t xmin, int64_t n, uint64_t seed,
            uint32_t cell, uint32_t purpose, uint32_t rep0, int64_t R,
            int nthreads, double *D, double *alpha_hat, int64_t *nonconv) {
  if (n < 1 || R < 1 || xmin < 1 || !(alpha > 1.0)) return OR_EINVAL;
  int64_t bad = 0, fails = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(+ : bad, fails)
#endif
  for (int64_t r = 0; r < R; ++r) {
    double ah = 0.0, d = 0.0;
    int st = or_replicate(alpha, xmin, n, seed, cell, rep0 + (uint32_t)r,
                          purpose, &ah, &d);
    if (st == OR_ENOCONV) bad += 1;
    else if (st != OR_OK) fails += 1;
    D[r] = d;
    if (alpha_hat) alpha_hat[r] = ah;
  }
  if (nonconv) *nonconv = bad;
  (void)nthreads;
  return fails ? OR_ENOMEM : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Cutoff = order statistic of the simulated D values (Section 4's code:
 * sort, then read the entry at 0-based index R*q).  Reading: the index is
 * floor(R*q) evaluated in binary64, no interpolation, clamped to R-1.      */

static int or_cmp_f64(const void *pa, const void *pb) {
  double a = *(const double *)pa, b = *(const double *)pb;
  return (a > b) - (a < b);
}

int64_t or_quantile_index(int64_t R, double q) {
  int64_t i = (int64_t)floor((double)R * q);
  if (i < 0) i = 0;
  if (i > R - 1) i = R - 1;
  return i;
}

int or_quantiles(const double *D, int64_t R, const double *q, int nq,
                 double *out) {
  if (R < 1) return OR_EINVAL;
  double *s = (double *)malloc((size_t)R * sizeof(double));
  if (!s) return OR_ENOMEM;
  memcpy(s, D, (size_t)R * sizeof(double));
  qsort(s, (size_t)R, sizeof(double), or_cmp_f64);
  for (int j = 0; j < nq; ++j) out[j] = s[or_quantile_index(R, q[j])];
  free(s);
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Using the cutoffs on observed data (Section 4, last paragraphs): fit
 * alpha-hat, compute D, compare with simulations at the same n and
 * alpha-hat.  Reading of the bespoke simulation as a parametric-bootstrap
 * p-value (the paper defers the procedure to its references): simulate B
 * datasets of the same n at alpha-hat (stream tag 1, cell = request id),
 * refit each, p = #{D_b >= D_obs} / B.                                     */

int or_fit(const int32_t *data, int64_t n, uint64_t xmin, double *alpha_hat,
           double *D) {
  if (n < 1 || xmin < 1) return OR_EINVAL;
  uint64_t *x = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  if (!x) return OR_ENOMEM;
  for (int64_t i = 0; i < n; ++i) {
    if (data[i] < 1 || (uint64_t)data[i] < xmin) {
      free(x);
      return OR_EINVAL;
    }
    x[i] = (uint64_t)data[i];
  }
  int st = or_mle(x, n, xmin, alpha_hat);
  if (st == OR_OK || st == OR_ENOCONV) {
    int st2 = or_ks(x, n, xmin, *alpha_hat, D);
    if (st2 != OR_OK) st = st2;
  }
  free(x);
  return st;
}

int or_bootstrap_pvalue(const int32_t *data, int64_t n, uint64_t xmin,
                        int64_t B, uint64_t seed, uint32_t request_id,
                        int nthreads, double *alpha_hat, double *D,
                        double *p, double *D_boot) {
  if (B < 1) return OR_EINVAL;
  int st = or_fit(data, n, xmin, alpha_hat, D);
  if (st != OR_OK && st != OR_ENOCONV) return st;
  double *Db = D_boot ? D_boot : (double *)malloc((size_t)B * sizeof(double));
  if (!Db) return OR_ENOMEM;
  int64_t nonconv = 0;
  st = or_cell(*alpha_hat, xmin, n, seed, request_id, 1u, 0u, B, nthreads,
               Db, 0, &nonconv);
  int64_t ge = 0;
  for (int64_t b = 0; b < B; ++b)
    if (Db[b] >= *D) ++ge;
  *p = (double)ge / (double)B;
  if (!D_boot) free(Db);
  return st;
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ======================================================================== */
/* Truncated Zipf law (Section 1's second version): support k = 1 .. K,
 * p(k) = k^-gamma / zeta_K(gamma), zeta_K(gamma) = sum_{k=1}^{K} k^-gamma,
 * any gamma > 0 (the MLE itself may fall anywhere on the real line).  The
 * same method: inverse-CDF draws, the MLE of Eq. 2 with the finite scaling
 * factor, and D of Eq. 3 against the fitted truncated law.
 * Sums run from k = K down to the smallest index (small terms first).     */

/* Survival Q(k) = P(X > k) = sum_{j=k+1}^{K} j^-gamma / zeta_K for k = 0..K
 * into Q[0..K] (Q[0] = 1 up to rounding, Q[K] = 0); returns zeta_K. */
double or_tz_survival_table(double gamma, int64_t K, double *Q) {
  double s = 0.0;
  Q[K] = 0.0;
  for (int64_t k = K; k >= 1; --k) {
    s += pow((double)k, -gamma);
    Q[k - 1] = s;
  }
  for (int64_t k = 0; k < K; ++k) Q[k] /= s;
  return s;
}

/* Inverse CDF on the finite support: X = min{k in 1..K : Q(k) < v},
 * v = m 2^-53, by bisection on the table (Q(K) = 0 < v always). */
int64_t or_tz_invert(const double *Q, int64_t K, uint64_t m) {
  const double v = ldexp((double)m, -53);
  int64_t lo = 1, hi = K; /* answer in [lo, hi] */
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (Q[mid] < v)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

void or_tz_sample(double gamma, int64_t K, uint64_t seed, uint32_t cell, uint32_t rep,
                  uint32_t purpose, int64_t n, uint64_t *out) {
  double *Q = (double *)malloc((size_t)(K + 1) * sizeof(double));
  if (!Q) return;
  or_tz_survival_table(gamma, K, Q);
  for (int64_t i = 0; i < n; ++i) out[i] = (uint64_t)or_tz_invert(Q, K, or_draw_m(seed, cell, rep, purpose, (uint64_t)i));
  free(Q);
}

/* zeta_K and its first two gamma-derivatives: sums of k^-g, -ln k k^-g,
 * ln^2 k k^-g (small terms first). */
static void or_tz_sums(double g, int64_t K, double z[3]) {
  double z0 = 0.0, z1 = 0.0, z2 = 0.0;
  for (int64_t k = K; k >= 1; --k) {
    double l = log((double)k), t = pow((double)k, -g);
    z0 += t;
    z1 -= l * t;
    z2 += l * l * t;
  }
  z[0] = z0;
  z[1] = z1;
  z[2] = z2;
}

/* MLE (Eq. 2 with the finite scaling factor): the root of
 * h(g) = zeta_K'(g)/zeta_K(g) + mbar, decreasing in g (h' = Var(ln X) > 0
 * with the sign convention z1 = zeta_K'), i.e. E_g[ln X] = mbar.  The root
 * exists for 0 < mbar < ln K; it is searched on [-64, 64] by
 * bisection-safeguarded Newton from g = 1 and clamped to that interval
 * (reading: the paper states gamma > 0 for the law; the estimate is the
 * unconstrained root, bounded for the rare samples whose mean log reaches
 * an end of the range).  The all-equal rule as in the untruncated case: a
 * sample of only ones gets ln 2 added to its log-sum.                      */
int or_tz_mle_from_logsum(double L, int64_t n, int64_t K, double *gamma_hat) {
  if (n < 1 || K < 2) return OR_EINVAL;
  const double mbar = L / (double)n;
  double lo = -64.0, hi = 64.0, g = 1.0;
  for (int it = 1; it <= 400; ++it) {
    double z[3];
    or_tz_sums(g, K, z);
    double e = -z[1] / z[0];                  /* E_g[ln X] */
    double var = z[2] / z[0] - e * e;         /* Var_g[ln X] */
    double f = e - mbar;                      /* decreasing in g */
    if (f > 0.0)
      lo = g;
    else
      hi = g;
    double next = g + f / var;
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    double step = fabs(next - g);
    g = next;
    double tol = 4.0 * ldexp(1.0, ilogb(fabs(g) > 1.0 ? g : 1.0) - 52);
    if (step <= tol || hi - lo <= tol) {
      *gamma_hat = g;
      return OR_OK;
    }
  }
  *gamma_hat = g;
  return OR_ENOCONV;
}

/* D (Eq. 3) against the truncated law at gamma: every t in 1..K. */
int or_tz_ks(const uint64_t *x, int64_t n, int64_t K, double gamma, double *D) {
  if (n < 1 || K < 2) return OR_EINVAL;
  double *Q = (double *)malloc((size_t)(K + 1) * sizeof(double));
  int64_t *cnt = (int64_t *)calloc((size_t)(K + 1), sizeof(int64_t));
  if (!Q || !cnt) {
    free(Q);
    free(cnt);
    return OR_ENOMEM;
  }
  or_tz_survival_table(gamma, K, Q);
  for (int64_t i = 0; i < n; ++i) {
    if (x[i] < 1 || (int64_t)x[i] > K) {
      free(Q);
      free(cnt);
      return OR_EINVAL;
    }
    cnt[x[i]] += 1;
  }
  double best = 0.0;
  int64_t below = 0;
  for (int64_t t = 1; t <= K; ++t) {
    below += cnt[t];
    double d = fabs((1.0 - Q[t]) - (double)below / (double)n);
    if (d > best) best = d;
  }
  free(Q);
  free(cnt);
  *D = best;
  return OR_OK;
}

int or_tz_replicate(double gamma, int64_t K, int64_t n, uint64_t seed, uint32_t cell, uint32_t rep,
                    uint32_t purpose, double *gamma_hat, double *D) {
  uint64_t *x = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  if (!x) return OR_ENOMEM;
  or_tz_sample(gamma, K, seed, cell, rep, purpose, n, x);
  int st = or_tz_mle_from_logsum(or_log_sum(x, n, 1), n, K, gamma_hat);
  if (st == OR_OK || st == OR_ENOCONV) {
    int st2 = or_tz_ks(x, n, K, *gamma_hat, D);
    if (st2 != OR_OK) st = st2;
  }
  free(x);
  return st;
}

int or_tz_cell(double gamma, int64_t K, int64_t n, uint64_t seed, uint32_t cell, uint32_t purpose,
               uint32_t rep0, int64_t R, int nthreads, double *D, double *gamma_hat, int64_t *nonconv) {
  /* the law on a finite support is normalisable for every real exponent;
   * the cells of the tables have gamma > 0, bespoke cutoffs simulate at the
   * fitted exponent, which may be negative */
  if (n < 1 || R < 1 || K < 2 || !(gamma >= -64.0 && gamma <= 64.0)) return OR_EINVAL;
  int64_t bad = 0, fails = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(+ : bad, fails)
#endif
  for (int64_t r = 0; r < R; ++r) {
    double gh = 0.0, d = 0.0;
    int st = or_tz_replicate(gamma, K, n, seed, cell, rep0 + (uint32_t)r, purpose, &gh, &d);
    if (st == OR_ENOCONV) bad += 1;
    else if (st != OR_OK) fails += 1;
    D[r] = d;
    if (gamma_hat) gamma_hat[r] = gh;
  }
  if (nonconv) *nonconv = bad;
  (void)nthreads;
  return fails ? OR_ENOMEM : OR_OK;
}

/* ======================================================================== */
/* Lower end by KS minimisation (the procedure of Clauset, Shalizi & Newman,
 * which the paper's tables are used with, Section 3): for every candidate
 * x_min among the sample's distinct values (the smallest max_candidates of
 * them), fit alpha-hat on the tail {x >= x_min} (Eq. 2 with the Hurwitz
 * normaliser) and compute D of the tail at its fit (Eq. 3); the estimate is
 * the candidate of smallest D (the first on ties).  Candidates whose tail
 * has fewer than min_tail values get D = NaN and are not chosen.
 * Outputs per candidate (arrays of max_candidates): xmin, alpha-hat, D, tail
 * size; *ncand the number of candidates, *best the chosen one (-1 if none). */
int or_estimate_xmin(const uint64_t *x, int64_t n, int64_t max_candidates, int64_t min_tail, int nthreads,
                     uint64_t *cand_xmin, double *cand_alpha, double *cand_D, int64_t *cand_ntail,
                     int64_t *ncand, int64_t *best) {
  if (n < 1 || max_candidates < 1 || min_tail < 1) return OR_EINVAL;
  uint64_t *s = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
  int64_t *first = (int64_t *)malloc((size_t)max_candidates * sizeof(int64_t));
  if (!s || !first) {
    free(s);
    free(first);
    return OR_ENOMEM;
  }
  memcpy(s, x, (size_t)n * sizeof(uint64_t));
  qsort(s, (size_t)n, sizeof(uint64_t), or_cmp_u64);
  int64_t m = 0;
  for (int64_t i = 0; i < n && m < max_candidates; ++i)
    if (i == 0 || s[i] != s[i - 1]) first[m++] = i;
  int fails = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(+ : fails)
#endif
  for (int64_t j = 0; j < m; ++j) {
    const uint64_t xm = s[first[j]];
    const int64_t nt = n - first[j];
    cand_xmin[j] = xm;
    cand_ntail[j] = nt;
    cand_alpha[j] = NAN;
    cand_D[j] = NAN;
    if (nt < min_tail) continue;
    double a = 0.0, d = 0.0;
    int st = or_mle(s + first[j], nt, xm, &a);
    if (st != OR_OK && st != OR_ENOCONV) {
      fails += 1;
      continue;
    }
    if (or_ks(s + first[j], nt, xm, a, &d) != OR_OK) {
      fails += 1;
      continue;
    }
    cand_alpha[j] = a;
    cand_D[j] = d;
  }
  (void)nthreads;
  int64_t b = -1;
  for (int64_t j = 0; j < m; ++j)
    if (!isnan(cand_D[j]) && (b < 0 || cand_D[j] < cand_D[b])) b = j;
  *ncand = m;
  *best = b;
  free(s);
  free(first);
  return fails ? OR_ENOMEM : OR_OK;
}

/* ======================================================================== */
/* Multinomial histogram sampler (a large-n variant of the sampler, not in
 * the paper): the histogram of a replicate drawn bin by bin by conditional
 * binomials instead of one draw per value.  Same law as the inverse-CDF
 * sampler (its integer thresholds), a different random stream.            */

/* Word i of 64 bits of stream (seed, cell, rep, purpose), the multinomial
 * sampler's random numbers: the words (w[2j], w[2j+1]), j = i mod 2, of the
 * Philox block with counter (floor(i/2), rep, cell, purpose) as the low and
 * high halves. */
uint64_t or_draw_bits64(uint64_t seed, uint32_t cell, uint32_t rep, uint32_t purpose, uint64_t i) {
  uint32_t ctr[4] = {(uint32_t)(i >> 1), rep, cell, purpose};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  or_philox4x32_10(ctr, key, w);
  int j = (int)(i & 1);
  return ((uint64_t)w[2 * j + 1] << 32) | (uint64_t)w[2 * j];
}

/* ln k! minus Stirling's formula (k + 1/2) ln k - k + ln sqrt(2 pi): for
 * k > 15 the asymptotic series 1/(12k) - 1/(360k^3) + 1/(1260k^5)
 * - 1/(1680k^7) + 1/(1188k^9) (Bernoulli numbers B_2j / (2j (2j-1))), next
 * term below 1e-16; for smaller k the sum of logs. */
static double or_stirling_err(double k) {
  if (k > 15.0) {
    const double r = 1.0 / (k * k);
    return (1.0 / 12.0 - r * (1.0 / 360.0 - r * (1.0 / 1260.0 - r * (1.0 / 1680.0 - r / 1188.0)))) / k;
  }
  double lf = 0.0;
  for (int i = 2; i <= (int)k; ++i) lf += log((double)i);
  return lf - ((k + 0.5) * log(k) - k + 0.918938533204672741780329736406);
}

/* x ln(x / M) + M - x without cancellation: near x = M the series
 * (x - M) v + 2x (v^3/3 + v^5/5 + ...), v = (x - M) / (x + M). */
static double or_deviance(double x, double M) {
  if (fabs(x - M) < 0.1 * (x + M)) {
    double v = (x - M) / (x + M);
    double s = (x - M) * v, e = 2.0 * x * v;
    const double v2 = v * v;
    for (int j = 1; j < 1000; ++j) {
      e *= v2;
      const double s1 = s + e / (double)(2 * j + 1);
      if (s1 == s) return s1;
      s = s1;
    }
    return s;
  }
  return x * log(x / M) + M - x;
}

/* P(Bin(n, p) = x), q = 1 - p given separately: the saddle-point form
 * (Loader, "Fast and accurate computation of binomial probabilities", 2000)
 *   exp(sterr(n) - sterr(x) - sterr(n-x) - dev(x, np) - dev(n-x, nq))
 *   * sqrt(n / (2 pi x (n - x))),  0 < x < n. */
double or_binom_pmf(int64_t x, int64_t n, double p, double q) {
  if (x < 0 || x > n) return 0.0;
  if (x == 0) return exp((double)n * (p < 0.5 ? log1p(-p) : log(q)));
  if (x == n) return exp((double)n * (q < 0.5 ? log1p(-q) : log(p)));
  const double dn = (double)n, dx = (double)x, dy = (double)(n - x);
  const double lc = or_stirling_err(dn) - or_stirling_err(dx) - or_stirling_err(dy) - or_deviance(dx, dn * p) -
                    or_deviance(dy, dn * q);
  return exp(lc) * sqrt(dn / (6.283185307179586476925286766559 * dx * dy));
}

/* Bin(n, p), p = num / den (integers, num <= den), from one uniform u in
 * (0, 1] by inversion along a fixed order of the outcomes (any order that
 * lists every outcome once gives the law): for a mean n p below 30 the order
 * 0, 1, 2, ... from P(0) = q^n; otherwise from M = floor((n+1) p) (the mode,
 * to within a part in 2^24 of p) outward, M+1, M-1, M+2, M-2, ... (one side
 * alone once the other is exhausted or its probabilities have underflowed).
 * The branch and M come from integer arithmetic on num and den cut to their
 * top 24 bits, so the order depends neither on rounding nor on the last
 * units of the thresholds.  Probabilities by the ratio P(k+1)/P(k) = (n-k)/(k+1) p/q. */
int64_t or_binomial(int64_t n, uint64_t num, uint64_t den, double u) {
  if (n <= 0 || num == 0) return 0;
  if (num >= den) return n;
  const double p = (double)num / (double)den, q = (double)(den - num) / (double)den;
  const double r = p / q;
  /* the branch and the mode from num and den cut to their top 24 bits: the
   * thresholds behind num and den are computed independently by each
   * implementation and may differ in their last units, and p is often an
   * exact ratio for which (n+1) p is an integer */
  const int sh = 64 - __builtin_clzll(den) > 24 ? 64 - __builtin_clzll(den) - 24 : 0;
  const uint64_t nc = num >> sh, dc = den >> sh;
  if ((uint64_t)n * nc < 30ull * dc) {
    double f = or_binom_pmf(0, n, p, q), c = f;
    int64_t k = 0;
    while (c < u && k < n) {
      f *= (double)(n - k) / (double)(k + 1) * r;
      ++k;
      c += f;
      if (f == 0.0 && (double)k > (double)n * p) break;
    }
    return k;
  }
  int64_t M = (int64_t)(((uint64_t)(n + 1) * nc) / dc);
  if (M > n) M = n;
  const double fM = or_binom_pmf(M, n, p, q);
  double rest = u - fM;
  if (rest <= 0.0) return M;
  int64_t lo = M - 1, hi = M + 1, last = M;
  double flo = lo >= 0 ? fM * (double)M / ((double)(n - M + 1) * r) : 0.0;
  double fhi = hi <= n ? fM * (double)(n - M) / (double)(M + 1) * r : 0.0;
  int up = 1;
  while (flo > 0.0 || fhi > 0.0) {
    if (up ? fhi > 0.0 : !(flo > 0.0)) {
      rest -= fhi;
      last = hi;
      if (rest <= 0.0) return hi;
      fhi = hi < n ? fhi * (double)(n - hi) / (double)(hi + 1) * r : 0.0;
      ++hi;
    } else {
      rest -= flo;
      last = lo;
      if (rest <= 0.0) return lo;
      flo = lo > 0 ? flo * (double)lo / ((double)(n - lo + 1) * r) : 0.0;
      --lo;
    }
    up = !up;
  }
  return last;
}

/* Integer thresholds of the law for i = 0..len-1: T[i] = floor(Q(xmin+i)
 * 2^53) + 1 (the inverse-CDF test Q(k) < m 2^-53 is T[k] <= m). */
void or_thresholds(double alpha, uint64_t xmin, int64_t len, uint64_t *T) {
  const double Z = or_hurwitz(alpha, (double)xmin);
  for (int64_t i = 0; i < len; ++i)
    T[i] = (uint64_t)floor(ldexp(or_survival(alpha, Z, xmin, xmin + (uint64_t)i), 53)) + 1;
}

/* One replicate by conditional binomials on a binary tree of the first
 * OR_MN_BINS values.  With T[-1] = 2^53 + 1 the inverse-CDF law gives the
 * index range [l, r) the mass (T[l-1] - T[r-1]) 2^-53.  First the count
 * beyond the tree, Bin(n, (T[B-1] - 1) / 2^53) (B = OR_MN_BINS); then node 1
 * (the range [0, B)) holds the rest, and node k of range [l, r) passes
 * Bin(c_k, (T[l-1] - T[mid-1]) / (T[l-1] - T[r-1])) of its count to its
 * left child 2k ([l, mid), mid = (l + r) / 2) and the others to its right
 * child 2k+1; the leaves B..2B-1 are the values xmin .. xmin + B - 1.  The
 * values beyond are drawn one by one conditional on X >= xmin + B: m' uniform
 * on [1, T[B-1] - 1] (the multiply-high of a 64-bit random word by
 * T[B-1] - 1, plus one) and X = min{k : Q(k) < m' 2^-53}.  Random words: draw
 * index 0 for the count beyond, k for node k's binomial (u = m 2^-53), and
 * 2B + t for the t-th value beyond (all 64 bits).  T: the thresholds of the
 * first B values.  Writes the n values, the tree's first. */
#define OR_MN_BINS 2048
static uint64_t or_mn_tm1(const uint64_t *T, int64_t i) { return i == 0 ? (1ull << 53) + 1 : T[i - 1]; }

void or_mn_sample(double alpha, uint64_t xmin, const uint64_t *T, uint64_t seed, uint32_t cell, uint32_t rep,
                  uint32_t purpose, int64_t n, uint64_t *out) {
  const int64_t B = OR_MN_BINS;
  const double Z = or_hurwitz(alpha, (double)xmin);
  const uint64_t TB = T[B - 1];
  const uint64_t m0 = (or_draw_bits64(seed, cell, rep, purpose, 0) >> 11) + 1;
  const int64_t beyond = or_binomial(n, TB - 1, 1ull << 53, ldexp((double)m0, -53));
  int64_t *cnt = (int64_t *)calloc((size_t)(2 * B), sizeof(int64_t));
  if (!cnt) return;
  cnt[1] = n - beyond;
  for (int64_t k = 1; k < B; ++k) {
    const int64_t c = cnt[k];
    if (c == 0) continue;
    int level = 0;
    while ((2ll << level) <= k) ++level;
    const int64_t width = B >> level, l = (k - (1ll << level)) * width, r = l + width, mid = l + width / 2;
    const uint64_t a = or_mn_tm1(T, l), b = or_mn_tm1(T, mid), e = or_mn_tm1(T, r);
    int64_t cl = 0;
    if (a > e) {
      const uint64_t m = (or_draw_bits64(seed, cell, rep, purpose, (uint64_t)k) >> 11) + 1;
      cl = or_binomial(c, a - b, a - e, ldexp((double)m, -53));
    }
    cnt[2 * k] = cl;
    cnt[2 * k + 1] = c - cl;
  }
  int64_t w = 0;
  for (int64_t i = 0; i < B; ++i)
    for (int64_t t = 0; t < cnt[B + i]; ++t) out[w++] = xmin + (uint64_t)i;
  free(cnt);
  for (int64_t t = 0; t < beyond; ++t) {
    const uint64_t bits = or_draw_bits64(seed, cell, rep, purpose, (uint64_t)(2 * B + t));
    const uint64_t mp = (uint64_t)(((unsigned __int128)bits * (unsigned __int128)(TB - 1)) >> 64) + 1;
    out[w++] = or_invert(alpha, Z, xmin, mp);
  }
}

int or_mn_cell(double alpha, uint64_t xmin, int64_t n, uint64_t seed, uint32_t cell, uint32_t purpose,
               uint32_t rep0, int64_t R, int nthreads, double *D, double *alpha_hat, int64_t *nonconv) {
  if (n < 1 || R < 1 || !(alpha > 1.0) || xmin < 1) return OR_EINVAL;
  uint64_t *T = (uint64_t *)malloc(OR_MN_BINS * sizeof(uint64_t));
  if (!T) return OR_ENOMEM;
  or_thresholds(alpha, xmin, OR_MN_BINS, T);
  int64_t bad = 0, fails = 0;
#ifdef _OPENMP
  if (nthreads < 1) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) reduction(+ : bad, fails)
#endif
  for (int64_t r = 0; r < R; ++r) {
    uint64_t *x = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    if (!x) {
      fails += 1;
      continue;
    }
    or_mn_sample(alpha, xmin, T, seed, cell, rep0 + (uint32_t)r, purpose, n, x);
    double a = 0.0, d = 0.0;
    int st = or_mle(x, n, xmin, &a);
    if (st == OR_ENOCONV) bad += 1;
    else if (st != OR_OK) fails += 1;
    if (or_ks(x, n, xmin, a, &d) != OR_OK) fails += 1;
    D[r] = d;
    if (alpha_hat) alpha_hat[r] = a;
    free(x);
  }
  free(T);
  if (nonconv) *nonconv = bad;
  (void)nthreads;
  return fails ? OR_ENOMEM : OR_OK;
}
