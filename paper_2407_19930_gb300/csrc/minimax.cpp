// Minimax tau / omega grids (Sec. 2: the non-uniform tau_j, omega_k grids the paper takes from
// GreenX), built on the host by the Remez exchange in double-double arithmetic.
//
// Scaled units x = D / dmin on [1, R] (R is the range ratio the grid is built for, below):
//   time grid:      the n-term exponential sum closest to 1/x in the maximum norm,
//                   min max_x |1/x - sum_j a_j exp(-t_j x)|   (1/x = int_0^inf exp(-x tau) d tau);
//   frequency grid: the n-term sum closest to 1/x in the maximum norm among
//                   sum_k c_k 4x^2 / (x^2 + o_k^2)^2, W_k = pi c_k   (pi/x = int_0^inf
//                   (2x / (x^2 + w^2))^2 dw: weights of int_0^inf d omega for the squared
//                   Lorentzian of each transition).
// Both optima equioscillate: the error reaches its largest modulus with alternating signs at
// 2n + 1 points.  Remez exchange: Newton on r(x_i) = (-1)^i E for the 2n parameters
// (logarithms of a, t) and E, then the x_i move to the extrema of the new error curve, until
// those are level to 1e-13.  Terms are added one at a time; each new term starts from a
// Levenberg-Marquardt least-squares fit reweighted towards the largest errors (double).
//
// Range: R_b = 2^{ceil(8 log2 R_eff) / 8}, R_eff = max(dmax / dmin, R_floor(n)),
// R_floor(n) = exp(n pi^2 / ln 1e9) / 8: ranges where n terms would fit below ~1e-9 are
// degenerate (parameters fixed only by rounding), and the 1/8-octave buckets let grids be
// cached.  The grid covers [dmin, R_b dmin] and hence [dmin, dmax].  Gamma: the L2 fit of the
// Gauss-Legendre route on [1, R_b].  Physical units: tau = t / dmin, omega = o dmin,
// W = pi c dmin, Gamma = Gamma^ / dmin.
#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

namespace librpa {
namespace {

// ------------------------------------------------------------------ double-double arithmetic
struct dd {
  double hi = 0, lo = 0;
  dd() = default;
  dd(double h) : hi(h), lo(0) {}
  dd(double h, double l) : hi(h), lo(l) {}
};
inline dd two_sum(double a, double b) {
  const double s = a + b, bb = s - a;
  return dd(s, (a - (s - bb)) + (b - bb));
}
inline dd quick_two_sum(double a, double b) {
  const double s = a + b;
  return dd(s, b - (s - a));
}
inline dd operator+(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi), t = two_sum(a.lo, b.lo);
  s.lo += t.hi;
  s = quick_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return quick_two_sum(s.hi, s.lo);
}
inline dd operator-(dd a) { return dd(-a.hi, -a.lo); }
inline dd operator-(dd a, dd b) { return a + (-b); }
inline dd operator*(dd a, dd b) {
  const double p = a.hi * b.hi;
  const double e = std::fma(a.hi, b.hi, -p);
  return quick_two_sum(p, e + (a.hi * b.lo + a.lo * b.hi));
}
inline dd operator/(dd a, dd b) {
  const double q1 = a.hi / b.hi;
  dd r = a - b * dd(q1);
  const double q2 = r.hi / b.hi;
  r = r - b * dd(q2);
  const double q3 = r.hi / b.hi;
  return dd(q1) + dd(q2) + dd(q3);
}
inline dd ldexp_dd(dd a, int k) { return dd(std::ldexp(a.hi, k), std::ldexp(a.lo, k)); }
inline bool lt(dd a, dd b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
inline dd fabs_dd(dd a) { return a.hi < 0 ? -a : a; }

// ln 2 = sum_k 1 / (k 2^k), summed in double-double once
dd ln2_dd() {
  static const dd v = [] {
    dd s(0.0);
    for (int k = 110; k >= 1; --k) s = s + dd(1.0) / dd(std::ldexp((double)k, k));
    return s;
  }();
  return v;
}

// exp(x): x = k ln 2 + r, exp(r 2^-6) by its Taylor series (Horner, 1/i! precomputed), squared
// 6 times, times 2^k
dd exp_dd(dd x) {
  static const std::vector<dd> inv_fact = [] {
    std::vector<dd> c(13);
    c[0] = dd(1.0);
    for (int i = 1; i < 13; ++i) c[i] = c[i - 1] / dd((double)i);
    return c;
  }();
  if (x.hi < -700) return dd(0.0);
  const double k = std::nearbyint(x.hi / ln2_dd().hi);
  const dd r = ldexp_dd(x - ln2_dd() * dd(k), -6);
  dd s = inv_fact[12];
  for (int i = 11; i >= 0; --i) s = s * r + inv_fact[i];
  for (int i = 0; i < 6; ++i) s = s * s;
  return ldexp_dd(s, (int)k);
}

// ------------------------------------------------------------------ the two families
// Evaluated in double (the growth of the sums) or double-double (the final levelling).
inline double exp_t(double x) { return std::exp(x); }
inline dd exp_t(const dd &x) { return exp_dd(x); }
inline double hi_t(double v) { return v; }
inline double hi_t(const dd &v) { return v.hi; }
inline bool lt(double a, double b) { return a < b; }
inline double fabs_t(double a) { return std::fabs(a); }
inline dd fabs_t(const dd &a) { return fabs_dd(a); }

// p = (log a_1..n, log t_1..n); kind 0 = time (a exp(-t x)), 1 = frequency (c 4x^2/(x^2+o^2)^2)
template <class T>
struct Terms {
  std::vector<T> a, t;
};
template <class T>
Terms<T> terms(const std::vector<T> &p) {
  const int n = (int)p.size() / 2;
  Terms<T> S;
  for (int j = 0; j < n; ++j) {
    S.a.push_back(exp_t(p[j]));
    S.t.push_back(exp_t(p[n + j]));
  }
  return S;
}

// r(x) = 1/x - phi(x) and, when wanted, r'(x), r''(x)
template <class T>
void eval(int kind, const Terms<T> &S, T x, T *r, T *r1, T *r2) {
  const int n = (int)S.a.size();
  const T ix = T(1.0) / x;
  T f(0.0), f1(0.0), f2(0.0);
  for (int j = 0; j < n; ++j) {
    if (kind == 0) {
      const T e = S.a[j] * exp_t(-(S.t[j] * x));
      f = f + e;
      if (r1) f1 = f1 - S.t[j] * e;
      if (r2) f2 = f2 + S.t[j] * S.t[j] * e;
    } else {
      const T u = x * x, v = S.t[j] * S.t[j], s = u + v, s2 = s * s;
      f = f + S.a[j] * T(4.0) * u / s2;
      if (r1) f1 = f1 + S.a[j] * T(8.0) * x * (v - u) / (s2 * s);
      if (r2) f2 = f2 + S.a[j] * (T(8.0) * v * v - T(64.0) * u * v + T(24.0) * u * u) / (s2 * s2);
    }
  }
  *r = ix - f;
  if (r1) *r1 = -(ix * ix) - f1;
  if (r2) *r2 = T(2.0) * ix * ix * ix - f2;
}

// d r / d p at x (the gradient of -phi)
template <class T>
void grad(int kind, const Terms<T> &S, T x, std::vector<T> &g) {
  const int n = (int)S.a.size();
  g.assign(2 * n, T(0.0));
  for (int j = 0; j < n; ++j) {
    if (kind == 0) {
      const T e = S.a[j] * exp_t(-(S.t[j] * x));
      g[j] = -e;
      g[n + j] = S.t[j] * x * e;
    } else {
      const T u = x * x, v = S.t[j] * S.t[j], s = u + v;
      const T L = T(4.0) * u / (s * s);
      g[j] = -(S.a[j] * L);
      g[n + j] = S.a[j] * T(16.0) * u * v / (s * s * s);
    }
  }
}

// ------------------------------------------------------------------ least-squares starts (double)
// sample points x = R^{u^2}, u uniform on [0, 1]: the error lobes are narrowest near x = 1
inline double sample_x(double R, int i, int m) {
  const double u = (double)i / (m - 1);
  return i == m - 1 ? R : std::exp(std::log(R) * u * u);
}

void family_d(int kind, const std::vector<double> &p, const std::vector<double> &xs, std::vector<double> &f,
              std::vector<double> &J) {
  const int n = (int)p.size() / 2, m = (int)xs.size();
  f.assign(m, 0.0);
  J.assign((size_t)m * 2 * n, 0.0);
  for (int j = 0; j < n; ++j) {
    const double a = std::exp(p[j]), t = std::exp(p[n + j]);
    for (int i = 0; i < m; ++i) {
      const double x = xs[i];
      if (kind == 0) {
        const double e = a * std::exp(-t * x);
        f[i] += e;
        J[(size_t)i * 2 * n + j] = e;
        J[(size_t)i * 2 * n + n + j] = -e * t * x;
      } else {
        const double s = x * x + t * t, L = 4 * x * x / (s * s);
        f[i] += a * L;
        J[(size_t)i * 2 * n + j] = a * L;
        J[(size_t)i * 2 * n + n + j] = -a * 16 * x * x * t * t / (s * s * s);
      }
    }
  }
}

// solves A x = b (n x n, row-major) by Gaussian elimination with partial pivoting; false if singular
inline double mag(double v) { return std::fabs(v); }
inline double mag(const dd &v) { return std::fabs(v.hi); }
template <class T>
bool solve(std::vector<T> A, std::vector<T> b, int n, std::vector<T> &x) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (mag(A[(size_t)r * n + c]) > mag(A[(size_t)piv * n + c])) piv = r;
    if (!(mag(A[(size_t)piv * n + c]) > 0)) return false;
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      const T f = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      for (int k = c; k < n; ++k) A[(size_t)r * n + k] = A[(size_t)r * n + k] - f * A[(size_t)c * n + k];
      b[r] = b[r] - f * b[c];
    }
  }
  x.assign(n, T(0.0));
  for (int r = n - 1; r >= 0; --r) {
    T s = b[r];
    for (int k = r + 1; k < n; ++k) s = s - A[(size_t)r * n + k] * x[k];
    x[r] = s / A[(size_t)r * n + r];
  }
  return true;
}

// weighted Levenberg-Marquardt fit of 1/x on the sample points
void least_squares(int kind, std::vector<double> &p, const std::vector<double> &xs, const std::vector<double> &w) {
  const int np = (int)p.size(), m = (int)xs.size();
  std::vector<double> f, J, fn, Jn;
  family_d(kind, p, xs, f, J);
  auto cost_of = [&](const std::vector<double> &ff) {
    double c = 0;
    for (int i = 0; i < m; ++i) {
      const double r = (1.0 / xs[i] - ff[i]) * w[i];
      c += r * r;
    }
    return c;
  };
  double cost = cost_of(f), lam = 1e-3;
  for (int it = 0; it < 100; ++it) {
    std::vector<double> A((size_t)np * np, 0.0), g(np, 0.0);
    for (int i = 0; i < m; ++i) {
      const double r = (1.0 / xs[i] - f[i]) * w[i] * w[i];
      const double *Ji = &J[(size_t)i * np];
      for (int a = 0; a < np; ++a) {
        g[a] += Ji[a] * r;
        for (int b = 0; b <= a; ++b) A[(size_t)a * np + b] += Ji[a] * Ji[b] * w[i] * w[i];
      }
    }
    double dmax = 0;
    for (int a = 0; a < np; ++a) {
      for (int b = a + 1; b < np; ++b) A[(size_t)a * np + b] = A[(size_t)b * np + a];
      dmax = std::max(dmax, A[(size_t)a * np + a]);
    }
    bool improved = false, done = false;
    while (lam < 1e14) {
      std::vector<double> M = A, d;
      for (int a = 0; a < np; ++a) M[(size_t)a * np + a] += lam * (A[(size_t)a * np + a] + 1e-12 * dmax);
      if (!solve<double>(M, g, np, d)) {
        lam *= 10;
        continue;
      }
      double mx = 0;
      for (double v : d) mx = std::max(mx, std::fabs(v));
      if (mx > 0.5)
        for (double &v : d) v *= 0.5 / mx;
      std::vector<double> pn = p;
      for (int a = 0; a < np; ++a) pn[a] += d[a];
      family_d(kind, pn, xs, fn, Jn);
      const double cn = cost_of(fn);
      if (std::isfinite(cn) && cn < cost) {
        done = cost - cn < 1e-13 * cost;
        p = pn;
        f.swap(fn);
        J.swap(Jn);
        cost = cn;
        lam = std::max(lam / 3, 1e-12);
        improved = true;
        break;
      }
      lam *= 4;
    }
    if (!improved || done) break;
  }
}

// Start for n + 1 terms from the n-term solution prev (empty: one term).  variant 0: the new term
// beyond the largest parameter (spacing extrapolated, the set then narrowed); 1: below the
// smallest; v >= 2: in the middle of the (v - 1)-th widest gap between neighbouring parameters.
// Returns an empty vector when the variant does not exist.
std::vector<double> start_point(int kind, const std::vector<double> &prev, double R, int variant) {
  std::vector<double> p;
  if (prev.empty()) {
    if (variant > 0) return p;
    p = kind == 0 ? std::vector<double>{0.0, 0.0} : std::vector<double>{0.0, std::log(std::sqrt(R))};
  } else {
    const int n = (int)prev.size() / 2;
    std::vector<std::pair<double, double>> tl(n);   // (log t, log a) ascending in t
    for (int j = 0; j < n; ++j) tl[j] = {prev[n + j], prev[j]};
    std::sort(tl.begin(), tl.end());
    std::vector<double> la, lt;
    for (int j = 0; j < n; ++j) {
      lt.push_back(tl[j].first);
      la.push_back(tl[j].second);
    }
    if (n == 1) {
      if (variant > 1) return p;
      const double d = variant == 0 ? 1.0 : -1.0;
      lt = {tl[0].first - 1.5 * d, tl[0].first + d};
      la = {tl[0].second - 1.0, tl[0].second};
    } else if (variant <= 1) {
      if (variant == 0) {
        lt.push_back(lt[n - 1] + (lt[n - 1] - lt[n - 2]));
        la.push_back(la[n - 1] + (la[n - 1] - la[n - 2]));
      } else {
        lt.insert(lt.begin(), lt[0] - (lt[1] - lt[0]));
        la.insert(la.begin(), la[0] - (la[1] - la[0]));
      }
      double c = 0;
      for (double v : lt) c += v;
      c /= n + 1;
      const double sh = std::sqrt((double)n / (n + 1.0));
      for (double &v : lt) v = c + (v - c) * sh;
    } else {
      std::vector<std::pair<double, int>> gaps;
      for (int j = 0; j + 1 < n; ++j) gaps.push_back({lt[j + 1] - lt[j], j});
      std::sort(gaps.rbegin(), gaps.rend());
      if (variant - 2 >= (int)gaps.size()) return p;
      const int j = gaps[variant - 2].second;
      lt.insert(lt.begin() + j + 1, 0.5 * (lt[j] + lt[j + 1]));
      la.insert(la.begin() + j + 1, 0.5 * (la[j] + la[j + 1]) - std::log(2.0));
    }
    p = la;
    p.insert(p.end(), lt.begin(), lt.end());
  }
  const int m = 400;
  std::vector<double> xs(m), w(m, 1.0), f, J;
  for (int i = 0; i < m; ++i) xs[i] = sample_x(R, i, m);
  for (int round = 0; round < 6; ++round) {   // least squares reweighted towards the largest errors
    least_squares(kind, p, xs, w);
    family_d(kind, p, xs, f, J);
    double emax = 0;
    std::vector<double> e(m);
    for (int i = 0; i < m; ++i) emax = std::max(emax, e[i] = std::fabs(1.0 / xs[i] - f[i]));
    double wmax = 0;
    for (int i = 0; i < m; ++i) wmax = std::max(wmax, w[i] = w[i] * std::sqrt(e[i] / emax) + 1e-3);
    for (double &v : w) v /= wmax;
  }
  return p;
}

// ------------------------------------------------------------------ Remez exchange
template <class T>
struct Ext {
  T x, r;
};

// r'(x) and r''(x) in double (parameters p: double parts)
std::pair<double, double> drv_d(int kind, const std::vector<double> &p, double x) {
  const int n = (int)p.size() / 2;
  double f1 = 0, f2 = 0;
  for (int j = 0; j < n; ++j) {
    const double a = std::exp(p[j]), t = std::exp(p[n + j]);
    if (kind == 0) {
      const double e = a * std::exp(-t * x);
      f1 -= t * e;
      f2 += t * t * e;
    } else {
      const double u = x * x, v = t * t, s = u + v, s2 = s * s;
      f1 += a * 8 * x * (v - u) / (s2 * s);
      f2 += a * (8 * v * v - 64 * u * v + 24 * u * u) / (s2 * s2);
    }
  }
  return {-1.0 / (x * x) - f1, 2.0 / (x * x * x) - f2};
}

// alternating extrema of r on [1, R]: the endpoints and the interior maxima of |r|, located on a
// sample (double) and refined by bracketed Newton on r' (double, then three steps in T)
template <class T>
std::vector<Ext<T>> extrema(int kind, const std::vector<T> &p, double R, int m) {
  const Terms<T> S = terms(p);
  std::vector<double> pd(p.size()), xs(m), e(m), f, J;
  for (size_t i = 0; i < p.size(); ++i) pd[i] = hi_t(p[i]);
  for (int i = 0; i < m; ++i) xs[i] = sample_x(R, i, m);
  family_d(kind, pd, xs, f, J);
  for (int i = 0; i < m; ++i) e[i] = 1.0 / xs[i] - f[i];
  auto sgn = [](double v) { return (v > 0) - (v < 0); };
  std::vector<Ext<T>> pts;
  for (int i = 0; i < m; ++i) {
    T x, r;
    if (i == 0 || i == m - 1) {
      x = i == 0 ? T(1.0) : T(R);
    } else {
      if (!(std::fabs(e[i]) >= std::fabs(e[i - 1]) && std::fabs(e[i]) >= std::fabs(e[i + 1]) &&
            sgn(e[i - 1]) == sgn(e[i]) && sgn(e[i]) == sgn(e[i + 1])))
        continue;
      // the root of r' in [x_{i-1}, x_{i+1}] (r' changes sign across the maximum of |r|)
      double lo = xs[i - 1], hi = xs[i + 1], xd = xs[i];
      const bool slo = drv_d(kind, pd, lo).first > 0;
      for (int it = 0; it < 60; ++it) {
        const std::pair<double, double> d12 = drv_d(kind, pd, xd);
        if ((d12.first > 0) == slo)
          lo = xd;
        else
          hi = xd;
        double xn = xd - d12.first / d12.second;
        if (!(d12.second != 0) || !(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        const double step = std::fabs(xn - xd);
        xd = xn;
        if (step < 1e-13 * xd || hi - lo < 1e-13 * xd) break;
      }
      x = T(xd);
      for (int it = 0; it < 3; ++it) {
        T r1, r2;
        eval(kind, S, x, &r, &r1, &r2);
        if (!(hi_t(r2) != 0)) break;
        const T xn = x - r1 / r2;
        if (!(hi_t(xn) > lo && hi_t(xn) < hi)) break;
        x = xn;
      }
    }
    eval(kind, S, x, &r, (T *)nullptr, (T *)nullptr);
    pts.push_back({x, r});
  }
  std::vector<Ext<T>> alt;
  for (const Ext<T> &q : pts) {
    if (!alt.empty() && (hi_t(q.r) > 0) == (hi_t(alt.back().r) > 0)) {
      if (lt(fabs_t(alt.back().r), fabs_t(q.r))) alt.back() = q;
    } else {
      alt.push_back(q);
    }
  }
  return alt;
}

// Newton on r(x_i; p) - (-1)^i E = 0 (2n + 1 equations and unknowns)
template <class T>
bool level(int kind, std::vector<T> &p, const std::vector<T> &xs, T E) {
  const int n2 = (int)p.size(), N = n2 + 1;
  const double stop = sizeof(T) == sizeof(double) ? 1e-13 : 1e-28;
  std::vector<T> g;
  for (int it = 0; it < 60; ++it) {
    const Terms<T> S = terms(p);
    std::vector<T> J((size_t)N * N), F(N), d;
    for (int i = 0; i < N; ++i) {
      const T s(i % 2 == 0 ? 1.0 : -1.0);
      T r;
      eval(kind, S, xs[i], &r, (T *)nullptr, (T *)nullptr);
      F[i] = -(r - s * E);
      grad(kind, S, xs[i], g);
      for (int j = 0; j < n2; ++j) J[(size_t)i * N + j] = g[j];
      J[(size_t)i * N + n2] = -s;
    }
    if (!solve<T>(J, F, N, d)) return false;
    double mx = 0;
    for (int j = 0; j < n2; ++j) mx = std::max(mx, std::fabs(hi_t(d[j])));
    if (!std::isfinite(mx)) return false;
    const T step(mx > 0.5 ? 0.5 / mx : 1.0);
    for (int j = 0; j < n2; ++j) p[j] = p[j] + step * d[j];
    E = E + step * d[n2];
    if (mx <= 0.5 && mx < stop) break;
  }
  return true;
}

// Levels the error curve from p on [1, R] until the 2n + 1 extrema agree to tol.  ref (optional,
// 2n + 1 points): a reference set to level on first (a previous range's extrema mapped onto this
// range); on success it receives the extrema of the levelled curve.
template <class T>
bool remez(int kind, std::vector<T> &p, double R, double tol, double &emax_out, std::vector<T> *ref = nullptr) {
  const int n2 = (int)p.size();
  const int m = std::max(400, 60 * n2);
  if (ref && (int)ref->size() == n2 + 1) {
    const Terms<T> S = terms(p);
    T E(0.0);
    for (int i = 0; i <= n2; ++i) {
      T r;
      eval(kind, S, (*ref)[i], &r, (T *)nullptr, (T *)nullptr);
      E = i % 2 == 0 ? E + r : E - r;
    }
    if (!level(kind, p, *ref, E / T((double)(n2 + 1)))) return false;
  }
  for (int it = 0; it < 40; ++it) {
    std::vector<Ext<T>> alt = extrema(kind, p, R, m);
    if ((int)alt.size() < n2 + 1) return false;
    int big = 0;
    for (int i = 1; i < (int)alt.size(); ++i)
      if (lt(fabs_t(alt[big].r), fabs_t(alt[i].r))) big = i;
    const int s0 = std::min(std::max(0, big - n2 / 2), (int)alt.size() - n2 - 1);
    const double emax = std::fabs(hi_t(alt[big].r));
    double emin = emax;
    T esum(0.0);
    std::vector<T> xs;
    for (int i = s0; i < s0 + n2 + 1; ++i) {
      emin = std::min(emin, std::fabs(hi_t(alt[i].r)));
      esum = esum + fabs_t(alt[i].r);
      xs.push_back(alt[i].x);
    }
    if ((emax - emin) / emax < tol) {   // level, and no other extremum above the level
      emax_out = emax;
      if (ref) *ref = xs;
      return true;
    }
    T E = esum / T((double)(n2 + 1));
    if (hi_t(alt[s0].r) < 0) E = -E;
    if (!level(kind, p, xs, E)) return false;
  }
  return false;
}

struct Scaled {
  std::vector<double> t, o, c, gamma;   // ascending t, ascending o; gamma [n][n] in scaled units
  double err_t = 0, err_o = 0;
};

// n-term minimax parameters on [1, R], ascending in t; false if the exchange did not level.
// Terms are added at a range Rg >= R wide enough that n terms stay above ~1e-6 (the least-squares
// starts resolve every alternation there), in double; the solution is carried to R by
// continuation (each step's exchange starts from the previous range's solution and extrema,
// mapped onto the new range), in double to a level of 1e-6, and levelled to 1e-13 in
// double-double at R.
bool minimax_scaled(int kind, int n, double R, std::vector<double> &a, std::vector<double> &t, double &err) {
  const double Rg = std::max(R, std::exp(n * M_PI * M_PI / std::log(1e6)) / 8.0);
  std::vector<double> p, ref;
  for (int k = 1; k <= n; ++k) {
    bool ok = false;
    const std::vector<double> prev = p;
    for (int variant = 0; variant < 8 && !ok; ++variant) {
      p = start_point(kind, prev, Rg, variant);
      if (p.empty()) break;
      ref.clear();
      ok = remez(kind, p, Rg, 1e-6, err, &ref);
    }
    if (!ok) return false;
  }
  auto mapped = [](const std::vector<double> &r, double Rc, double Rn) {
    std::vector<double> q(r.size());
    const double sc = std::log(Rn) / std::log(Rc);
    for (size_t i = 0; i < r.size(); ++i)
      q[i] = i == 0 ? 1.0 : i + 1 == r.size() ? Rn : std::exp(std::log(r[i]) * sc);
    return q;
  };
  double Rc = Rg, f = 1.25;
  bool in_dd = false;   // double until a step fails or the level drops below 1e-8
  std::vector<dd> pd, rd;
  while (Rc > R) {
    const double Rn = std::max(R, Rc / f);
    if (!in_dd && err < 1e-8) {
      in_dd = true;
      pd.assign(p.begin(), p.end());
      rd.assign(ref.begin(), ref.end());
    }
    bool ok;
    std::vector<double> rq = mapped(in_dd ? std::vector<double>() : ref, Rc, Rn);
    if (!in_dd) {
      std::vector<double> q = p;
      ok = remez(kind, q, Rn, 1e-6, err, &rq);
      if (ok) {
        p.swap(q);
        ref.swap(rq);
      } else {
        in_dd = true;   // retry the step in double-double
        pd.assign(p.begin(), p.end());
        rd.assign(ref.begin(), ref.end());
        continue;
      }
    } else {
      std::vector<double> rh(rd.size());
      for (size_t i = 0; i < rd.size(); ++i) rh[i] = rd[i].hi;
      rh = mapped(rh, Rc, Rn);
      std::vector<dd> q = pd, rqd(rh.begin(), rh.end());
      ok = remez(kind, q, Rn, 1e-10, err, &rqd);
      if (ok) {
        pd.swap(q);
        rd.swap(rqd);
      }
    }
    if (ok) {
      Rc = Rn;
      f = std::min(2.0, f * 1.5);
    } else {
      f = std::sqrt(f);
      if (f < 1.01) return false;
    }
  }
  if (!in_dd) {
    pd.assign(p.begin(), p.end());
    rd.assign(ref.begin(), ref.end());
  }
  if (!remez(kind, pd, R, 1e-13, err, &rd)) return false;
  std::vector<std::pair<double, double>> ta(n);
  for (int j = 0; j < n; ++j) {
    const dd av = exp_dd(pd[j]), tv = exp_dd(pd[n + j]);
    ta[j] = {tv.hi + tv.lo, av.hi + av.lo};
  }
  std::sort(ta.begin(), ta.end());
  a.resize(n);
  t.resize(n);
  for (int j = 0; j < n; ++j) {
    t[j] = ta[j].first;
    a[j] = ta[j].second;
  }
  return true;
}

std::mutex g_mm_mutex;
std::map<std::pair<int, int>, Scaled> g_mm_cache;

}  // namespace

double minimax_range(int n, double dmin, double dmax) {
  const double R = std::max({dmax / dmin, std::exp(n * M_PI * M_PI / std::log(1e9)) / 8.0, 1.0});
  return std::exp2(std::ceil(8.0 * std::log2(R)) / 8.0);
}

int build_grid_minimax(int n, double dmin, double dmax, double *tau, double *omega, double *w_omega, double *gamma,
                       double *info) {
  if (n < 1 || n > kMinimaxMaxN || !(dmin > 0) || !(dmax >= dmin) || !std::isfinite(dmax) || !tau || !omega || !w_omega ||
      !gamma)
    return LIBRPA_E_ARG;
  const double Rb = minimax_range(n, dmin, dmax);
  const int bucket = (int)std::lround(8.0 * std::log2(Rb));
  Scaled S;
  {
    std::lock_guard<std::mutex> lk(g_mm_mutex);
    auto it = g_mm_cache.find({n, bucket});
    if (it != g_mm_cache.end()) S = it->second;
  }
  if (S.t.empty()) {
    std::vector<double> a;
    if (!minimax_scaled(0, n, Rb, a, S.t, S.err_t)) return LIBRPA_E_NUMERIC;
    if (!minimax_scaled(1, n, Rb, S.c, S.o, S.err_o)) return LIBRPA_E_NUMERIC;
    S.gamma.resize((size_t)n * n);
    fit_gamma(n, S.t.data(), S.o.data(), 1.0, Rb, S.gamma.data());
    std::lock_guard<std::mutex> lk(g_mm_mutex);
    g_mm_cache[{n, bucket}] = S;
  }
  for (int j = 0; j < n; ++j) tau[j] = S.t[j] / dmin;
  for (int k = 0; k < n; ++k) {
    omega[k] = S.o[k] * dmin;
    w_omega[k] = M_PI * S.c[k] * dmin;
  }
  for (int i = 0; i < n * n; ++i) gamma[i] = S.gamma[i] / dmin;
  if (info) {
    info[0] = Rb;
    info[1] = S.err_t;
    info[2] = S.err_o;
  }
  return LIBRPA_OK;
}

}  // namespace librpa
