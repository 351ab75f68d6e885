// Reference-element mathematics of libdg in FP64 (see dg_reference.h).
//
// Quadrature (the paper leaves N^s and N^t of Eq. "2nd term" open): collapsed
// Gauss-Jacobi rules with N+1 nodes per direction on the tetrahedron and the
// triangle, N+1 Gauss-Legendre nodes in time; all exact to degree 2N+1.
// Basis: orthonormal Dubiner polynomials (Sec. 2.2, Eq. "modal dg space") in
// the scaled-Jacobi form y^n P_n(x/y), which has no division and is regular on
// the element boundary.
#include "dg_reference.h"

#include <cmath>

namespace dg {
namespace ref {

namespace {

// P_n^{(a,0)}(x) and its derivative by the three-term recurrence.
void jacobi_eval(int n, double a, double x, double* p_out, double* dp_out) {
  double p0 = 1.0, d0 = 0.0;
  if (n == 0) { *p_out = p0; *dp_out = d0; return; }
  double p1 = 0.5 * ((a + 2.0) * x + a), d1 = 0.5 * (a + 2.0);
  for (int k = 1; k < n; ++k) {
    const double s = 2.0 * k + a;
    const double den = 2.0 * (k + 1) * (k + a + 1) * s;
    const double A = (s + 1) * (s + 2) * s / den;
    const double B = (s + 1) * a * a / den;
    const double C = 2.0 * (k + a) * k * (s + 2) / den;
    const double p2 = (A * x + B) * p1 - C * p0;
    const double d2 = A * p1 + (A * x + B) * d1 - C * d0;
    p0 = p1; d0 = d1; p1 = p2; d1 = d2;
  }
  *p_out = p1;
  *dp_out = d1;
}

// Scaled Jacobi Q_n(x,y) = y^n P_n^{(a,0)}(x/y), n = 0..nmax, with partials.
void scaled_jacobi(int nmax, double a, double x, double y, double* Q, double* Qx, double* Qy) {
  Q[0] = 1.0; Qx[0] = 0.0; Qy[0] = 0.0;
  if (nmax < 1) return;
  Q[1] = 0.5 * ((a + 2.0) * x + a * y);
  Qx[1] = 0.5 * (a + 2.0);
  Qy[1] = 0.5 * a;
  for (int k = 1; k < nmax; ++k) {
    const double s = 2.0 * k + a;
    const double den = 2.0 * (k + 1) * (k + a + 1) * s;
    const double A = (s + 1) * (s + 2) * s / den;
    const double B = (s + 1) * a * a / den;
    const double C = 2.0 * (k + a) * k * (s + 2) / den;
    const double lin = A * x + B * y;
    Q[k + 1] = lin * Q[k] - C * y * y * Q[k - 1];
    Qx[k + 1] = A * Q[k] + lin * Qx[k] - C * y * y * Qx[k - 1];
    Qy[k + 1] = B * Q[k] + lin * Qy[k] - 2.0 * C * y * Q[k - 1] - C * y * y * Qy[k - 1];
  }
}

}  // namespace

void gauss_jacobi(int n, double alpha, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < n; ++k) {
    // Chebyshev-like start, then Newton with deflation of the roots found so far
    double r = -std::cos((2.0 * k + 1.0) * pi / (2.0 * n));
    if (k > 0 && r <= x[k - 1]) r = x[k - 1] + 1e-3;
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      jacobi_eval(n, alpha, r, &p, &dp);
      double sum = 0.0;
      for (int j = 0; j < k; ++j) sum += 1.0 / (r - x[j]);
      const double delta = p / (dp - p * sum);
      r -= delta;
      if (std::fabs(delta) < 1e-16) break;
    }
    x[k] = r;
  }
  for (int k = 0; k < n; ++k) {
    double p, dp;
    jacobi_eval(n, alpha, x[k], &p, &dp);
    w[k] = std::pow(2.0, alpha + 1.0) / ((1.0 - x[k] * x[k]) * dp * dp);
  }
}

Rule3 volume_rule(int n) {
  std::vector<double> a, wa, b, wb, c, wc;
  gauss_jacobi(n, 0.0, a, wa);
  gauss_jacobi(n, 1.0, b, wb);
  gauss_jacobi(n, 2.0, c, wc);
  Rule3 r;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        r.xi.push_back((1 + a[i]) * (1 - b[j]) * (1 - c[k]) / 8.0);
        r.eta.push_back((1 + b[j]) * (1 - c[k]) / 4.0);
        r.zeta.push_back((1 + c[k]) / 2.0);
        r.w.push_back(wa[i] * wb[j] * wc[k] / 64.0);
      }
  return r;
}

Rule2 face_rule(int n) {
  std::vector<double> a, wa, b, wb;
  gauss_jacobi(n, 0.0, a, wa);
  gauss_jacobi(n, 1.0, b, wb);
  Rule2 r;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      r.s.push_back((1 + a[i]) * (1 - b[j]) / 4.0);
      r.t.push_back((1 + b[j]) / 2.0);
      r.w.push_back(wa[i] * wb[j] / 4.0);   // /8 for the area 1/2, x2 to normalise to 1
    }
  return r;
}

Rule1 time_rule(int n) {
  std::vector<double> a, wa;
  gauss_jacobi(n, 0.0, a, wa);
  Rule1 r;
  for (int i = 0; i < n; ++i) {
    r.x.push_back(0.5 * (a[i] + 1.0));
    r.w.push_back(0.5 * wa[i]);
  }
  return r;
}

void dubiner(int N, double xi, double eta, double zeta, double* values, double* grads) {
  const double u = 1.0 - eta - zeta, w = 1.0 - zeta;
  const double x1 = 2.0 * xi - u, y1 = u;           // d/d(xi,eta,zeta): x1 (2,1,1), y1 (0,-1,-1)
  const double x2 = 2.0 * eta - w, y2 = w;          // x2 (0,2,1), y2 (0,0,-1)
  const double x3 = 2.0 * zeta - 1.0;               // x3 (0,0,2)
  double QA[8], QAx[8], QAy[8], QB[8], QBx[8], QBy[8], QC[8], QCx[8], QCy[8];
  scaled_jacobi(N, 0.0, x1, y1, QA, QAx, QAy);
  int m = 0;
  for (int d = 0; d <= N; ++d)
    for (int i = 0; i <= d; ++i) {
      scaled_jacobi(N, 2.0 * i + 1.0, x2, y2, QB, QBx, QBy);
      for (int j = 0; j <= d - i; ++j, ++m) {
        const int k = d - i - j;
        scaled_jacobi(N, 2.0 * i + 2.0 * j + 2.0, x3, 1.0, QC, QCx, QCy);
        const double c = std::sqrt((2.0 * i + 1) * (2.0 * i + 2 * j + 2) * (2.0 * i + 2 * j + 2 * k + 3));
        const double A = QA[i], B = QB[j], C = QC[k];
        values[m] = c * A * B * C;
        if (grads) {
          const double dA[3] = {2.0 * QAx[i], QAx[i] - QAy[i], QAx[i] - QAy[i]};
          const double dB[3] = {0.0, 2.0 * QBx[j], QBx[j] - QBy[j]};
          const double dC[3] = {0.0, 0.0, 2.0 * QCx[k]};
          for (int e = 0; e < 3; ++e)
            grads[3 * m + e] = c * (dA[e] * B * C + A * dB[e] * C + A * B * dC[e]);
        }
      }
    }
}

}  // namespace ref
}  // namespace dg
