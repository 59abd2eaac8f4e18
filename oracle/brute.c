/* Brute-force tensor-product quadrature (oracle, test infrastructure only).
 *
 * Computes the tensor-product rule of Sec. 4.1, Eq. (5),
 *     I = sum_{i_1..i_d} w_{i_1} ... w_{i_d} g(t_{i_1}, ..., t_{i_d}),
 * by enumerating every multi-index, with Neumaier-compensated summation
 * (Neumaier 1974: running sum plus a correction term that collects the
 * low-order bits lost in each addition).  The caller multiplies by the
 * family constant.
 *
 * Integrands g (Sec. 5.1, Eqs. 9-11, and the s-in-R^n form):
 *   family 0 = C, 1 = D, 2 = E, 3 = TEST;  form 0 = R^n (d = n), 1 = unit cube (d = n-1).
 *
 * ttq_oracle_brute_sym: for C/D in the R^n form with the same rule in every
 * mode, g is symmetric in its arguments, so the sum runs over sorted tuples
 * i_1 <= ... <= i_d weighted by the multinomial count d!/prod(m_v!).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double s, c; } neu_t;

static void neu_add(neu_t *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else                      a->c += (x - t) + a->s;
  a->s = t;
}

static double g_eval(int family, int form, int n, int d, const double *x) {
  if (family == 3) {                       /* TEST: sum_t exp(-t mean(x)) */
    double S = 0.0, out = 0.0;
    for (int k = 0; k < d; ++k) S += x[k];
    for (int t = 1; t <= n; ++t) out += exp(-(double)t * S / (double)d);
    return out;
  }
  if (form == 0) {                         /* s in R^n */
    double ssum = 0.0;
    for (int j = 0; j < d; ++j) ssum += 2.0 * cosh(x[j]);
    double val = 1.0 / (ssum * ssum);
    if (family == 1) {
      for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j) {
          double th = tanh((x[i] - x[j]) / 2.0);
          val *= th * th;
        }
    }
    return val;
  }
  /* unit cube: x[q] = x_{q+2}, q = 0..n-2 */
  double Bv = 1.0, Av = 1.0;
  if (family == 0 || family == 1) {
    double left = 1.0, right = 1.0, p = 1.0;
    for (int k = 2; k <= n; ++k) { p *= x[k - 2]; left += p; }
    p = 1.0;
    for (int k = n; k >= 2; --k) { p *= x[k - 2]; right += p; }
    Bv = 1.0 / (left * right);
  }
  if (family == 1 || family == 2) {
    for (int i = 1; i <= n; ++i) {
      double p = 1.0;
      for (int j = i + 1; j <= n; ++j) {
        p *= x[j - 2];
        double q = (1.0 - p) / (1.0 + p);
        Av *= q * q;
      }
    }
  }
  if (family == 0) return Bv;
  if (family == 1) return Av * Bv;
  return Av;
}

/* nodes/weights: concatenated per mode, mode k starts at off[k] = sum_{m<k} N[m]. */
double ttq_oracle_brute(int family, int form, int n, int d, const int *N,
                        const double *nodes, const double *weights) {
  int off[64], idx[64];
  double x[64];
  if (d < 1 || d > 64) return NAN;
  off[0] = 0;
  for (int k = 1; k < d; ++k) off[k] = off[k - 1] + N[k - 1];
  int64_t outer = N[0];
  neu_t *part = (neu_t *)calloc((size_t)outer, sizeof(neu_t));
#pragma omp parallel for schedule(dynamic, 1) private(idx, x)
  for (int64_t i0 = 0; i0 < outer; ++i0) {
    neu_t acc = {0.0, 0.0};
    for (int k = 0; k < d; ++k) idx[k] = 0;
    idx[0] = (int)i0;
    for (;;) {
      double w = 1.0;
      for (int k = 0; k < d; ++k) {
        x[k] = nodes[off[k] + idx[k]];
        w *= weights[off[k] + idx[k]];
      }
      neu_add(&acc, w * g_eval(family, form, n, d, x));
      int k = d - 1;                       /* odometer over modes 1..d-1 */
      while (k >= 1) {
        if (++idx[k] < N[k]) break;
        idx[k] = 0;
        --k;
      }
      if (k < 1) break;
    }
    part[i0] = acc;
  }
  neu_t tot = {0.0, 0.0};
  for (int64_t i0 = 0; i0 < outer; ++i0) { neu_add(&tot, part[i0].s); neu_add(&tot, part[i0].c); }
  free(part);
  return tot.s + tot.c;
}

double ttq_oracle_brute_sym(int family, int n, int d, int N, const double *nodes,
                            const double *weights) {
  int idx[64];
  double x[64], fact[65];
  if (d < 1 || d > 64 || (family != 0 && family != 1)) return NAN;
  fact[0] = 1.0;
  for (int m = 1; m <= 64; ++m) fact[m] = fact[m - 1] * m;
  neu_t *part = (neu_t *)calloc((size_t)N, sizeof(neu_t));
#pragma omp parallel for schedule(dynamic, 1) private(idx, x)
  for (int i0 = 0; i0 < N; ++i0) {
    neu_t acc = {0.0, 0.0};
    for (int k = 0; k < d; ++k) idx[k] = i0;
    for (;;) {
      double w = 1.0, mult = fact[d];
      int run = 1;
      for (int k = 0; k < d; ++k) {
        x[k] = nodes[idx[k]];
        w *= weights[idx[k]];
        if (k > 0) {
          if (idx[k] == idx[k - 1]) ++run;
          else { mult /= fact[run]; run = 1; }
        }
      }
      mult /= fact[run];
      neu_add(&acc, mult * w * g_eval(family, 0, n, d, x));
      int k = d - 1;                       /* next non-decreasing tuple with idx[0] fixed */
      while (k >= 1) {
        if (++idx[k] < N) break;
        --k;
      }
      if (k < 1) break;
      for (int m = k + 1; m < d; ++m) idx[m] = idx[k];
    }
    part[i0] = acc;
  }
  neu_t tot = {0.0, 0.0};
  for (int i0 = 0; i0 < N; ++i0) { neu_add(&tot, part[i0].s); neu_add(&tot, part[i0].c); }
  free(part);
  return tot.s + tot.c;
}

/* g at npts points (row-major npts x d): lets tests compare this C restatement
 * with the numpy one in integrands.py. */
void ttq_oracle_g(int family, int form, int n, int d, int64_t npts, const double *X, double *out) {
  for (int64_t p = 0; p < npts; ++p) out[p] = g_eval(family, form, n, d, X + p * d);
}
