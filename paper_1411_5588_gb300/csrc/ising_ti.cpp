// Host FP64 arithmetic that turns the integer records into the paper's
// thermodynamic integrations (Eq. 9 over H1, Eq. 19 over beta or T).
#include <cmath>
#include <cstdint>
#include <vector>

#include "ising_host.h"

using namespace isg;

namespace {

// Legendre P_n(x) and its derivative by the three-term recurrence.
void legendre(int n, double x, double* p, double* dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { *p = 1.0; *dp = 0.0; return; }
  for (int k = 2; k <= n; k++) {
    const double pk = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = pk;
  }
  *p = p1;
  *dp = n * (x * p1 - p0) / (x * x - 1.0);
}

}  // namespace

extern "C" {

int ising_gauss_legendre(int n, double a, double b, double* x, double* w) {
  clear_error();
  if (n < 1 || n > 4096 || !x || !w) return fail(ISING_EINVAL, "gauss_legendre: bad arguments");
  const double half = 0.5 * (b - a), mid = 0.5 * (b + a);
  for (int i = 0; i < n; i++) {
    // i-th root from the top, Newton from the asymptotic guess
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double p = 0, dp = 1;
    for (int it = 0; it < 100; it++) {
      legendre(n, t, &p, &dp);
      const double dt = p / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    legendre(n, t, &p, &dp);
    // ascending order on [a, b]
    x[n - 1 - i] = mid + half * t;
    w[n - 1 - i] = half * 2.0 / ((1.0 - t * t) * dp * dp);
  }
  return ISING_OK;
}

int ising_series_mean(const int64_t* records, size_t n, size_t stride, size_t col, size_t first, double* mean) {
  clear_error();
  if (!records || !mean || first >= n || col >= stride) return fail(ISING_EINVAL, "series_mean: bad arguments");
  __int128 s = 0;
  for (size_t k = first; k < n; k++) s += records[k * stride + col];
  *mean = (double)s / (double)(n - first);
  return ISING_OK;
}

int ising_series_energy(const int64_t* records, size_t n, int Lx, double J, double H, double H1, double* E,
                        size_t first, double* mean) {
  clear_error();
  if (!records || Lx < 1 || (!E && !mean) || (mean && first >= n)) return fail(ISING_EINVAL, "series_energy: bad arguments");
  const size_t stride = 5 + (size_t)Lx;
  // Eq. 1 with Hn = -H1, term by term from the record's integers
  if (E)
    for (size_t k = 0; k < n; k++) {
      const int64_t* r = records + k * stride;
      E[k] = -J * (double)r[1] - H * (double)r[2] - H1 * (double)r[3] + H1 * (double)r[4];
    }
  if (mean) {
    __int128 sB = 0, sM = 0, s1 = 0, sn = 0;
    for (size_t k = first; k < n; k++) {
      const int64_t* r = records + k * stride;
      sB += r[1];
      sM += r[2];
      s1 += r[3];
      sn += r[4];
    }
    const double c = (double)(n - first);
    *mean = -J * ((double)sB / c) - H * ((double)sM / c) - H1 * ((double)s1 / c) + H1 * ((double)sn / c);
  }
  return ISING_OK;
}

int ising_ti_surface_field(int n, double H1, const double* m1, const double* mn, double* delta_f1) {
  clear_error();
  if (n < 1 || !m1 || !mn || !delta_f1) return fail(ISING_EINVAL, "ti_surface_field: bad arguments");
  std::vector<double> x(n), w(n);
  int rc = ising_gauss_legendre(n, 0.0, H1, x.data(), w.data());
  if (rc) return rc;
  double s = 0.0;
  for (int i = 0; i < n; i++) s += w[i] * (m1[i] - mn[i]);
  *delta_f1 = -s;
  return ISING_OK;
}

int ising_ti_beta_trapezoid(int n, const double* beta, const double* U, double* out) {
  clear_error();
  if (n < 2 || !beta || !U || !out) return fail(ISING_EINVAL, "ti_beta_trapezoid: bad arguments");
  double s = 0.0;
  for (int i = 0; i + 1 < n; i++) s += 0.5 * (beta[i + 1] - beta[i]) * (U[i] + U[i + 1]);
  *out = s;
  return ISING_OK;
}

int ising_ti_temperature_trapezoid(int n, const double* T, const double* U, double* out) {
  clear_error();
  if (n < 2 || !T || !U || !out) return fail(ISING_EINVAL, "ti_temperature_trapezoid: bad arguments");
  double s = 0.0;
  for (int i = 0; i + 1 < n; i++)
    s += 0.5 * (T[i + 1] - T[i]) * (U[i] / (T[i] * T[i]) + U[i + 1] / (T[i + 1] * T[i + 1]));
  *out = -s;
  return ISING_OK;
}

}  // extern "C"
