// Host construction of the tau / omega grids and of the tau -> i omega transform matrix
// (Sec. 2, cosine transform: non-uniform grids, coefficients from an L2 minimisation).
//
// The paper takes its grids from GreenX, whose tables are not available here; the
// construction below is stated in librpa_gpu.h (librpa_gpu_build_grid):
//   * omega_k, W_k: n-point Gauss-Legendre rule mapped to (0, inf) by
//     omega = w0 (1 + t) / (1 - t), w0 = sqrt(dmin dmax), W = w0 2 w / (1 - t)^2;
//   * tau_j: the same rule mapped with 1 / w0;
//   * Gamma_kj: relative least-squares fit of 2D / (D^2 + omega_k^2) by
//     sum_j Gamma_kj exp(-D tau_j) on 1000 log-spaced D in [dmin, dmax], solved through
//     a one-sided Jacobi SVD with singular values below 1e-12 s_max dropped.
#include <cmath>
#include <vector>

#include "internal.h"

namespace librpa {
namespace {

// Nodes (ascending) and weights of the n-point Gauss-Legendre rule: Newton iteration on
// the three-term recurrence of the Legendre polynomials.
void gauss_legendre(int n, std::vector<double> &t, std::vector<double> &w) {
  t.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double x = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = n == 1 ? x : p1, pm = n == 1 ? 1.0 : p0;
      dp = n * (x * pn - pm) / (x * x - 1.0);
      double dx = pn / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    // recompute the derivative at the converged node
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double pn = n == 1 ? x : p1, pm = n == 1 ? 1.0 : p0;
    dp = n * (x * pn - pm) / (x * x - 1.0);
    t[n - 1 - i] = x;
    w[n - 1 - i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// Minimum-norm least-squares solution of A x = b (A: m x n row-major, m >= n) through a
// one-sided (Hestenes) Jacobi SVD, dropping singular values below rcond * s_max.
std::vector<double> lsq_svd(std::vector<double> A, int m, int n, const std::vector<double> &b,
                            double rcond) {
  std::vector<double> V(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  for (int sweep = 0; sweep < 80; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double a = 0, bb = 0, g = 0;
        for (int r = 0; r < m; ++r) {
          double x = A[r * n + p], y = A[r * n + q];
          a += x * x;
          bb += y * y;
          g += x * y;
        }
        if (g == 0.0) continue;
        double rel = std::fabs(g) / std::sqrt(a * bb);
        if (rel > off) off = rel;
        if (rel < 1e-15) continue;
        double zeta = (bb - a) / (2.0 * g);
        double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int r = 0; r < m; ++r) {
          double x = A[r * n + p], y = A[r * n + q];
          A[r * n + p] = c * x - s * y;
          A[r * n + q] = s * x + c * y;
        }
        for (int r = 0; r < n; ++r) {
          double x = V[r * n + p], y = V[r * n + q];
          V[r * n + p] = c * x - s * y;
          V[r * n + q] = s * x + c * y;
        }
      }
    if (off < 1e-15) break;
  }
  std::vector<double> sig(n);
  double smax = 0;
  for (int j = 0; j < n; ++j) {
    double s = 0;
    for (int r = 0; r < m; ++r) s += A[r * n + j] * A[r * n + j];
    sig[j] = std::sqrt(s);
    if (sig[j] > smax) smax = sig[j];
  }
  std::vector<double> x(n, 0.0);
  for (int j = 0; j < n; ++j) {
    if (!(sig[j] > rcond * smax)) continue;
    double ub = 0;  // (A V)_j . b = sigma_j u_j . b
    for (int r = 0; r < m; ++r) ub += A[r * n + j] * b[r];
    double coef = ub / (sig[j] * sig[j]);
    for (int i = 0; i < n; ++i) x[i] += V[i * n + j] * coef;
  }
  return x;
}

}  // namespace

int build_grid(int n, double dmin, double dmax, double *tau, double *omega, double *w_omega,
               double *gamma) {
  if (n < 1 || n > 64 || !(dmin > 0) || !(dmax >= dmin) || !tau || !omega || !w_omega || !gamma)
    return LIBRPA_E_ARG;
  std::vector<double> t, w;
  gauss_legendre(n, t, w);
  const double w0 = std::sqrt(dmin * dmax);
  for (int k = 0; k < n; ++k) {
    omega[k] = w0 * (1.0 + t[k]) / (1.0 - t[k]);
    w_omega[k] = w0 * 2.0 * w[k] / ((1.0 - t[k]) * (1.0 - t[k]));
    tau[k] = (1.0 / w0) * (1.0 + t[k]) / (1.0 - t[k]);
  }
  fit_gamma(n, tau, omega, dmin, dmax, gamma);
  return LIBRPA_OK;
}

void fit_gamma(int n, const double *tau, const double *omega, double dmin, double dmax, double *gamma) {
  const int m = 1000;
  std::vector<double> d(m);
  const double lr = std::log(dmax / dmin);
  for (int i = 0; i < m; ++i) d[i] = dmax > dmin ? dmin * std::exp(lr * i / (m - 1)) : dmin;
  std::vector<double> A(m * n), ones(m, 1.0);
  for (int k = 0; k < n; ++k) {
    for (int i = 0; i < m; ++i) {
      double f = 2.0 * d[i] / (d[i] * d[i] + omega[k] * omega[k]);
      for (int j = 0; j < n; ++j) A[i * n + j] = std::exp(-d[i] * tau[j]) / f;
    }
    std::vector<double> g = lsq_svd(A, m, n, ones, 1e-12);
    for (int j = 0; j < n; ++j) gamma[k * n + j] = g[j];
  }
}

}  // namespace librpa
