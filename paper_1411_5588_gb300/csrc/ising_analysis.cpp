// Host FP64 analysis of the paper's Secs. II B-IV on top of the records:
// layer profiles and the contact angle (Eqs. 12, 17-18), the Young difference
// (Eq. 9) and Young's angle (Eq. 8), the angle-dependent interface tension
// from the modified Young equation (Eq. 16), free energies by integration
// over beta (Eq. 19) and the fit of Eq. 20, the line tension (Eqs. 21-22),
// stiffness (Eqs. 23-25), step free energy (Eqs. 26-27) and the single-step
// model (Eqs. 28-32).
#include <cmath>
#include <cstdint>
#include <vector>

#include "ising_host.h"

using namespace isg;

namespace {

// Least squares y = a + b x over n points, centred sums.
bool line_fit(int n, const double* x, const double* y, double* a, double* b) {
  double sx = 0, sy = 0;
  for (int i = 0; i < n; i++) {
    sx += x[i];
    sy += y[i];
  }
  const double mx = sx / n, my = sy / n;
  double sxx = 0, sxy = 0;
  for (int i = 0; i < n; i++) {
    sxx += (x[i] - mx) * (x[i] - mx);
    sxy += (x[i] - mx) * (y[i] - my);
  }
  if (!(sxx > 0)) return false;
  *b = sxy / sxx;
  *a = my - *b * mx;
  return true;
}

// Least squares y = b x through the origin.
bool origin_fit(int n, const double* x, const double* y, double* b) {
  double sxx = 0, sxy = 0;
  for (int i = 0; i < n; i++) {
    sxx += x[i] * x[i];
    sxy += x[i] * y[i];
  }
  if (!(sxx > 0)) return false;
  *b = sxy / sxx;
  return true;
}

}  // namespace

extern "C" {

int ising_layer_profile(const int64_t* records, size_t n, int Lx, int Ly, int Lz, size_t first, double* mbar) {
  clear_error();
  if (!records || !mbar || Lx < 1 || Ly < 1 || Lz < 1 || first >= n)
    return fail(ISING_EINVAL, "layer_profile: bad arguments");
  const size_t stride = 5 + (size_t)Lx;
  const double per = (double)(n - first) * (double)Ly * (double)Lz;
  for (int k = 0; k < Lx; k++) {
    __int128 s = 0;
    for (size_t r = first; r < n; r++) s += records[r * stride + 5 + k];
    mbar[k] = (double)s / per;
  }
  return ISING_OK;
}

int ising_mirror_profile(int Lx, const double* m_plus, double* m_minus) {
  clear_error();
  if (Lx < 1 || !m_plus || !m_minus || m_plus == m_minus) return fail(ISING_EINVAL, "mirror_profile: bad arguments");
  for (int k = 0; k < Lx; k++) m_minus[k] = -m_plus[Lx - 1 - k];
  return ISING_OK;
}

int ising_contact_angle(int Lx, int Ly, const double* mbar, const double* m_plus, const double* m_minus, int k_lo,
                        int k_hi, double* y_plus, double* theta) {
  clear_error();
  if (Lx < 2 || Ly < 1 || !mbar || !m_plus || !m_minus || !y_plus || !theta)
    return fail(ISING_EINVAL, "contact_angle: bad arguments");
  if (k_lo < 1 || k_hi > Lx || k_hi <= k_lo) return fail(ISING_EINVAL, "contact_angle: need 1 <= k_lo < k_hi <= Lx");
  // Eq. 18 with y+ + y- = Ly: Ly mbar = y+ m+ + (Ly - y+) m-
  for (int k = 0; k < Lx; k++) {
    const double den = m_plus[k] - m_minus[k];
    if (!(std::fabs(den) > 0)) return fail(ISING_EINVAL, "contact_angle: m+ = m- in layer %d", k + 1);
    y_plus[k] = Ly * (mbar[k] - m_minus[k]) / den;
  }
  // the dividing surface is a plane through the layers k_lo..k_hi: y+ is
  // linear in kx and the acute angle with the walls has cot(theta) = |slope|
  const int n = k_hi - k_lo + 1;
  std::vector<double> x(n);
  for (int i = 0; i < n; i++) x[i] = k_lo + i;
  double a, b;
  if (!line_fit(n, x.data(), y_plus + (k_lo - 1), &a, &b)) return fail(ISING_EINVAL, "contact_angle: degenerate fit");
  *theta = std::atan2(1.0, std::fabs(b));
  return ISING_OK;
}

int ising_ti_young_difference(int n, double H1, const double* m1, const double* mn, double* delta_f1) {
  clear_error();
  if (n < 1 || !m1 || !mn || !delta_f1) return fail(ISING_EINVAL, "ti_young_difference: bad arguments");
  // Eq. 9: each wall's own Eq. 7, the wall n field being -H1
  std::vector<double> x(n), w(n);
  const int rc = ising_gauss_legendre(n, 0.0, H1, x.data(), w.data());
  if (rc) return rc;
  double s = 0.0;
  for (int i = 0; i < n; i++) s += w[i] * (m1[i] + mn[i]);
  *delta_f1 = -s;
  return ISING_OK;
}

int ising_young_angle(double delta_f1, double gamma_pi2, double* theta) {
  clear_error();
  if (!theta || !(gamma_pi2 > 0)) return fail(ISING_EINVAL, "young_angle: bad arguments");
  // Eq. 8 for the acute angle: cos(theta) = |delta_f1| / f_int
  const double c = std::fabs(delta_f1) / gamma_pi2;
  if (c > 1.0) return fail(ISING_EINVAL, "young_angle: |delta_f1| > f_int (wet wall)");
  *theta = std::acos(c);
  return ISING_OK;
}

int ising_gamma_of_theta(int n, const double* theta, const double* delta_f1, double gamma0, double* gamma) {
  clear_error();
  if (n < 1 || !theta || !delta_f1 || !gamma) return fail(ISING_EINVAL, "gamma_of_theta: bad arguments");
  for (int i = 0; i < n; i++)
    if (!(theta[i] > 0 && theta[i] < M_PI)) return fail(ISING_EINVAL, "gamma_of_theta: theta outside (0, pi)");
  // Eq. 16, gamma cos - gamma' sin = delta_f1, is
  // d(gamma / sin)/dtheta = -delta_f1 / sin^2: trapezoid over the points
  // from gamma(theta[0]) = gamma0
  double g = gamma0 / std::sin(theta[0]);
  gamma[0] = gamma0;
  for (int i = 1; i < n; i++) {
    const double s0 = std::sin(theta[i - 1]), s1 = std::sin(theta[i]);
    const double f0 = -delta_f1[i - 1] / (s0 * s0), f1 = -delta_f1[i] / (s1 * s1);
    g += 0.5 * (theta[i] - theta[i - 1]) * (f0 + f1);
    gamma[i] = g * s1;
  }
  return ISING_OK;
}

int ising_ti_free_energy_beta(int n, const double* beta, const double* U, double F0, double* F) {
  clear_error();
  if (n < 1 || !beta || !U || !F) return fail(ISING_EINVAL, "ti_free_energy_beta: bad arguments");
  for (int i = 0; i < n; i++)
    if (!(beta[i] > 0)) return fail(ISING_EINVAL, "ti_free_energy_beta: beta must be > 0");
  // Eq. 19: beta F(beta) = beta0 F(beta0) + integral_{beta0}^{beta} U, trapezoid
  double I = beta[0] * F0;
  F[0] = F0;
  for (int i = 1; i < n; i++) {
    I += 0.5 * (beta[i] - beta[i - 1]) * (U[i] + U[i - 1]);
    F[i] = I / beta[i];
  }
  return ISING_OK;
}

int ising_fit_gamma_tau(int n, const double* Lx, const double* Lz, const double* dF, double* gamma_pi2, double* tau0) {
  clear_error();
  if (n < 2 || !Lx || !Lz || !dF || !gamma_pi2 || !tau0) return fail(ISING_EINVAL, "fit_gamma_tau: bad arguments");
  // Eq. 20: dF / (Lz Lx) = gamma(pi/2) + (2 / Lx) tau(0, pi/2)
  std::vector<double> x(n), y(n);
  for (int i = 0; i < n; i++) {
    if (!(Lx[i] > 0 && Lz[i] > 0)) return fail(ISING_EINVAL, "fit_gamma_tau: sizes must be > 0");
    x[i] = 2.0 / Lx[i];
    y[i] = dF[i] / (Lz[i] * Lx[i]);
  }
  double a, b;
  if (!line_fit(n, x.data(), y.data(), &a, &b)) return fail(ISING_EINVAL, "fit_gamma_tau: all Lx equal");
  *gamma_pi2 = a;
  *tau0 = b;
  return ISING_OK;
}

int ising_line_tension_residual(double dF_film, double Lx, double Ly, double Lz, double theta, double gamma_theta,
                                double gamma_pi2, double s_wall, double delta_f1, double* R) {
  clear_error();
  if (!R || !(Lx > 0 && Ly > 0 && Lz > 0) || !(theta > 0 && theta < M_PI))
    return fail(ISING_EINVAL, "line_tension_residual: bad arguments");
  // Eq. 21 solved for 2 Lz [tau(H1, theta) - tau(0, pi/2)]; s_wall is the
  // per-site wall term gamma+(|H1|) + gamma+(-|H1|) - 2 gamma+(0) and
  // delta_f1 = gamma+(|H1|) - gamma+(-|H1|) (Eq. 9)
  *R = dF_film - Lx * Lz * (gamma_theta / std::sin(theta) - gamma_pi2) - Lz * Ly * s_wall -
       Lz * Lx * delta_f1 / std::tan(theta);
  return ISING_OK;
}

int ising_line_tension_lz_scan(int n, const double* Lz, const double* R, double* dtau, double* intercept) {
  clear_error();
  if (n < 2 || !Lz || !R || !dtau || !intercept) return fail(ISING_EINVAL, "line_tension_lz_scan: bad arguments");
  // at fixed Lx Lz and Ly Lz the residual varies as 2 Lz dtau (Sec. II C)
  double a, b;
  if (!line_fit(n, Lz, R, &a, &b)) return fail(ISING_EINVAL, "line_tension_lz_scan: all Lz equal");
  *dtau = 0.5 * b;
  *intercept = a;
  return ISING_OK;
}

int ising_stiffness(int n, const double* theta, const double* gamma, double gamma_pi2, double* c, double* kappa) {
  clear_error();
  if (n < 1 || !theta || !gamma || !c || !kappa || !(gamma_pi2 != 0.0))
    return fail(ISING_EINVAL, "stiffness: bad arguments");
  // Eq. 23: gamma / gamma(pi/2) - 1 = c (pi/2 - theta)^2, fit through the origin
  std::vector<double> x(n), y(n);
  for (int i = 0; i < n; i++) {
    const double d = 0.5 * M_PI - theta[i];
    x[i] = d * d;
    y[i] = gamma[i] / gamma_pi2 - 1.0;
  }
  if (!origin_fit(n, x.data(), y.data(), c)) return fail(ISING_EINVAL, "stiffness: all angles at pi/2");
  *kappa = gamma_pi2 * (1.0 + 2.0 * *c);  // Eq. 24
  return ISING_OK;
}

int ising_roughening_kappa_fit(int n, const double* T, const double* kappa, double T_R, double T_c, double* C) {
  clear_error();
  if (n < 1 || !T || !kappa || !C || !(T_c > 0)) return fail(ISING_EINVAL, "roughening_kappa_fit: bad arguments");
  // Eq. 25: 1 - 2 kappa beta / pi = C ((T - T_R) / T_c)^(1/2), through the origin
  std::vector<double> x(n), y(n);
  for (int i = 0; i < n; i++) {
    if (!(T[i] > T_R)) return fail(ISING_EINVAL, "roughening_kappa_fit: needs T > T_R");
    x[i] = std::sqrt((T[i] - T_R) / T_c);
    y[i] = 1.0 - 2.0 * kappa[i] / (M_PI * T[i]);
  }
  if (!origin_fit(n, x.data(), y.data(), C)) return fail(ISING_EINVAL, "roughening_kappa_fit: degenerate fit");
  return ISING_OK;
}

int ising_step_free_energy(int n, const double* theta, const double* gamma, double* f_s, double* gamma_flat) {
  clear_error();
  if (n < 2 || !theta || !gamma || !f_s || !gamma_flat) return fail(ISING_EINVAL, "step_free_energy: bad arguments");
  // Eq. 26 below roughening: gamma = gamma(pi/2) + f_s |pi/2 - theta| near pi/2
  std::vector<double> x(n);
  for (int i = 0; i < n; i++) x[i] = std::fabs(0.5 * M_PI - theta[i]);
  double a, b;
  if (!line_fit(n, x.data(), gamma, &a, &b)) return fail(ISING_EINVAL, "step_free_energy: degenerate fit");
  *f_s = std::fabs(b);
  *gamma_flat = a;
  return ISING_OK;
}

int ising_roughening_fs_fit(int n, const double* T, const double* f_s, double T_R, double* A, double* log_amp) {
  clear_error();
  if (n < 2 || !T || !f_s || !A || !log_amp || !(T_R > 0)) return fail(ISING_EINVAL, "roughening_fs_fit: bad arguments");
  // Eq. 27 with f_s proportional to 1 / xi_R: ln f_s = ln a - A (1 - T/T_R)^(-1/2)
  std::vector<double> x(n), y(n);
  for (int i = 0; i < n; i++) {
    if (!(T[i] < T_R) || !(f_s[i] > 0)) return fail(ISING_EINVAL, "roughening_fs_fit: needs T < T_R and f_s > 0");
    x[i] = 1.0 / std::sqrt(1.0 - T[i] / T_R);
    y[i] = std::log(f_s[i]);
  }
  double a, b;
  if (!line_fit(n, x.data(), y.data(), &a, &b)) return fail(ISING_EINVAL, "roughening_fs_fit: degenerate fit");
  *A = -b;
  *log_amp = a;
  return ISING_OK;
}

int ising_step_model(double H1, double f_s, double T, double Lx, double Lz, double* phi, double* h1_star) {
  clear_error();
  if (!(T > 0) || !(Lx > 0) || !(Lz > 0) || !phi || !h1_star) return fail(ISING_EINVAL, "step_model: bad arguments");
  // Eqs. 28-31 with every weight taken relative to the largest, so that
  // large Lz / T cannot overflow
  const double l0 = 0.0;
  const double lp = std::log(Lx) - f_s * Lz / T + 2.0 * H1 * Lz / T;
  const double lm = std::log(Lx) - f_s * Lz / T - 2.0 * H1 * Lz / T;
  const double top = std::fmax(l0, std::fmax(lp, lm));
  const double w0 = std::exp(l0 - top), wp = std::exp(lp - top), wm = std::exp(lm - top);
  *phi = (wp - wm) / (w0 + wp + wm) / Lx;
  *h1_star = 0.5 * f_s - T * std::log(Lx) / (2.0 * Lz);  // Eq. 32
  return ISING_OK;
}

int ising_critical_field(int n, const double* H1, const double* theta, double tol, double T, double Lx, double Lz,
                         double* h1_star, double* f_s) {
  clear_error();
  if (n < 2 || !H1 || !theta || !h1_star || !f_s || !(tol > 0) || !(T > 0) || !(Lx > 0) || !(Lz > 0))
    return fail(ISING_EINVAL, "critical_field: bad arguments");
  for (int i = 1; i < n; i++)
    if (!(H1[i] > H1[i - 1])) return fail(ISING_EINVAL, "critical_field: H1 must increase");
  // Sec. III C: the first point whose tilt pi/2 - theta exceeds tol; H1* is
  // where the straight line through it and the point before crosses tol
  const double half_pi = 0.5 * M_PI;
  int i = 0;
  while (i < n && half_pi - theta[i] <= tol) i++;
  if (i == 0 || i == n) return fail(ISING_EINVAL, "critical_field: the tilt does not cross tol inside the scan");
  const double p0 = half_pi - theta[i - 1], p1 = half_pi - theta[i];
  *h1_star = H1[i - 1] + (tol - p0) * (H1[i] - H1[i - 1]) / (p1 - p0);
  *f_s = 2.0 * *h1_star + T * std::log(Lx) / Lz;  // Eq. 32 solved for f_s
  return ISING_OK;
}

}  // extern "C"
