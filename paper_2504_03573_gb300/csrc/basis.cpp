// Host 1D point sets and Lagrange tables (Sec. 2.1: Gauss-Lobatto-Legendre
// nodes for the Lagrange basis of Table 1; Gauss-Legendre or Gauss-Lobatto-
// Legendre points for volume and trace quadrature, Eq. iproduct, Fig. 1).
// FP64, computed once per process and rule and copied to __constant__ memory of
// the kernel translation units of that rule.
#include <cmath>
#include <vector>

#include "sip_internal.h"

namespace sip {

// P_n(x) and P_n'(x) by the Bonnet recurrence.
static void legendre_pd(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x, d0 = 0.0, d1 = 1.0;
  if (n == 0) { p = 1.0; dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    double d2 = d0 + (2.0 * k - 1.0) * p1;  // P_k' = P_{k-2}' + (2k-1) P_{k-1}
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  p = p1; dp = d1;
}

static void symmetrise(std::vector<double>& x, std::vector<double>& w) {
  const int n = (int)x.size();
  for (int i = 0; i < n / 2; ++i) {
    double a = 0.5 * (x[n - 1 - i] - x[i]);
    x[i] = -a; x[n - 1 - i] = a;
    double b = 0.5 * (w[i] + w[n - 1 - i]);
    w[i] = b; w[n - 1 - i] = b;
  }
  if (n % 2) x[n / 2] = 0.0;
}

void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0); w.assign(q, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < q; ++i) {
    double z = -std::cos(pi * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre_pd(q, z, p, dp);
      double dz = p / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p, dp;
    legendre_pd(q, z, p, dp);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
  symmetrise(x, w);
}

// Interior GLL nodes are the interior roots of P_n - P_{n-2} (n = number of
// points), a multiple of (1 - x^2) P_{n-1}'.
void gauss_lobatto(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0); w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  x[0] = -1.0; x[n - 1] = 1.0;
  for (int i = 1; i < n - 1; ++i) {
    double z = -std::cos(pi * i / (n - 1));
    for (int it = 0; it < 100; ++it) {
      double pa, da, pb, db;
      legendre_pd(n, z, pa, da);
      legendre_pd(n - 2, z, pb, db);
      double dz = (pa - pb) / (da - db);
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
  }
  for (int i = 0; i < n; ++i) {
    double p, dp;
    legendre_pd(n - 1, x[i], p, dp);
    w[i] = 2.0 / (n * (n - 1.0) * p * p);
  }
  symmetrise(x, w);
}

double lagrange(const std::vector<double>& nodes, int j, double x) {
  double v = 1.0;
  for (int m = 0; m < (int)nodes.size(); ++m)
    if (m != j) v *= (x - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

double lagrange_deriv(const std::vector<double>& nodes, int j, double x) {
  const int n = (int)nodes.size();
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    if (k == j) continue;
    double t = 1.0 / (nodes[j] - nodes[k]);
    for (int m = 0; m < n; ++m)
      if (m != j && m != k) t *= (x - nodes[m]) / (nodes[j] - nodes[m]);
    s += t;
  }
  return s;
}

void point_rule(int rule, int q, std::vector<double>& x, std::vector<double>& w) {
  if (rule == SIP_RULE_GLL) gauss_lobatto(q, x, w);
  else gauss_legendre(q, x, w);
}

void fill_tables(int rule, std::vector<double>& tab) {
  tab.assign(kTabSize, 0.0);
  std::vector<double> xg, wg, xl, wl, xf, wf;
  auto fill_b = [&](int N, int Q) {
    gauss_lobatto(N, xl, wl);
    point_rule(rule, Q, xg, wg);
    for (int q = 0; q < Q; ++q)
      for (int i = 0; i < N; ++i) tab[tab_B(N, Q) + q * N + i] = lagrange(xl, i, xg[q]);
  };
  for (int N = kNMin; N <= kNMax; ++N) fill_b(N, N + 1);
  for (int i = 0; i < kNumExtra; ++i) fill_b(kExtraPairs[i].n, kExtraPairs[i].q);
  for (int Q = kQMin; Q <= kQMax; ++Q) {
    point_rule(rule, Q, xg, wg);
    for (int q = 0; q < Q; ++q)
      for (int r = 0; r < Q; ++r) tab[tab_D(Q) + q * Q + r] = lagrange_deriv(xg, r, xg[q]);
    for (int r = 0; r < Q; ++r) {
      tab[tab_L(Q) + 0 * Q + r] = lagrange(xg, r, -1.0);
      tab[tab_L(Q) + 1 * Q + r] = lagrange(xg, r, 1.0);
      tab[tab_L(Q) + 2 * Q + r] = lagrange_deriv(xg, r, -1.0);
      tab[tab_L(Q) + 3 * Q + r] = lagrange_deriv(xg, r, 1.0);
    }
    for (int F = Q; F <= kQMax; ++F) {
      point_rule(rule, F, xf, wf);
      for (int z = 0; z < F; ++z)
        for (int r = 0; r < Q; ++r) tab[tab_I(Q, F) + z * Q + r] = lagrange(xg, r, xf[z]);
    }
  }
}

}  // namespace sip
