// Host-side reference-element mathematics of libdg (FP64): Gauss-Jacobi nodes
// by Newton iteration, collapsed volume/face rules, Gauss-Legendre time rule,
// and the orthonormal Dubiner basis with gradients.
#pragma once

#include <vector>

namespace dg {
namespace ref {

// n-point Gauss rule for int_{-1}^{1} (1-x)^alpha f(x) dx (beta = 0).
void gauss_jacobi(int n, double alpha, std::vector<double>& x, std::vector<double>& w);

struct Rule3 { std::vector<double> xi, eta, zeta, w; };   // weights sum to 1/6
struct Rule2 { std::vector<double> s, t, w; };            // weights sum to 1
struct Rule1 { std::vector<double> x, w; };               // on [0,1], weights sum to 1

Rule3 volume_rule(int n);
Rule2 face_rule(int n);
Rule1 time_rule(int n);

// Dubiner basis of degree N at (xi, eta, zeta): values[L], grads[L][3] (may be null).
void dubiner(int N, double xi, double eta, double zeta, double* values, double* grads);

}  // namespace ref
}  // namespace dg
