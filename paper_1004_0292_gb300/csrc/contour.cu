// Quadrature points and weights (host).  Section 2.1 (circle C) and
// Section 3 (line pair L+-) of the paper.
//
// Weights solve sum_j w_j zeta_j^(k-1) = delta_{k0}, k = 0..N-1
// (zeta_j = (z_j - gamma)/rho).  The system is Vandermonde-like and its
// condition number grows past 1e18 at N = 64, so it is not solved
// numerically: its unique solution is w_j = -P(0)/P'(zeta_j) with
// P(zeta) = prod_k (zeta - zeta_k), evaluated as
// zeta_j * prod_{k != j} (-zeta_k)/(zeta_j - zeta_k) (every factor O(1)).
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace ssqcd {

using cd = std::complex<double>;

int contour_nodes(int path, double gamma, double rho, double beta, int N, std::vector<double2>& z,
                  std::vector<double2>& w) {
  if (!(rho > 0.0) || !std::isfinite(rho) || !std::isfinite(gamma))
    return fail(SSQCD_ERR_ARG, "contour: rho must be > 0 and gamma finite");
  std::vector<cd> zeta(N);
  if (path == SSQCD_PATH_LINES) {
    if (N < 4 || N % 2) return fail(SSQCD_ERR_ARG, "contour: lines need an even N >= 4");
    if (!(beta > 0.0) || !std::isfinite(beta)) return fail(SSQCD_ERR_ARG, "contour: beta must be > 0");
    const int h = N / 2;
    for (int i = 0; i < h; ++i) {
      const double x = -1.0 + 2.0 * i / (h - 1);
      zeta[2 * i] = cd(x, beta);
      zeta[2 * i + 1] = cd(x, -beta);
    }
  } else if (path == SSQCD_PATH_CIRCLE) {
    if (N < 1) return fail(SSQCD_ERR_ARG, "contour: N must be >= 1");
    const double two_pi = 6.283185307179586476925286766559;
    for (int j = 0; j < N; ++j) {
      const double th = two_pi * (j + 0.5) / N;
      zeta[j] = cd(std::cos(th), std::sin(th));
    }
  } else {
    return fail(SSQCD_ERR_ARG, "contour: unknown path");
  }
  z.resize(N);
  w.resize(N);
  for (int j = 0; j < N; ++j) {
    cd prod = zeta[j];
    for (int k = 0; k < N; ++k) {
      if (k == j) continue;
      prod *= -zeta[k] / (zeta[j] - zeta[k]);
    }
    const cd zj = gamma + rho * zeta[j];
    z[j] = make_double2(zj.real(), zj.imag());
    w[j] = make_double2(prod.real(), prod.imag());
  }
  return SSQCD_OK;
}

}  // namespace ssqcd

extern "C" int ssqcd_contour(int path, double gamma, double rho, double beta, int N, double* z, double* w) {
  if (z == nullptr || w == nullptr) return ssqcd::fail(SSQCD_ERR_ARG, "ssqcd_contour: NULL output");
  std::vector<double2> zz, ww;
  SS_TRY(ssqcd::contour_nodes(path, gamma, rho, beta, N, zz, ww));
  for (int j = 0; j < N; ++j) {
    z[2 * j] = zz[j].x;
    z[2 * j + 1] = zz[j].y;
    w[2 * j] = ww[j].x;
    w[2 * j + 1] = ww[j].y;
  }
  return SSQCD_OK;
}
