// Small dense complex Hermitian eigenproblem (host) for the Rayleigh-Ritz
// step (Section 2.1): the m x m projected matrix Q^H A Q and the Gram
// matrices of the basis, m = rank <= M L.
//
// Method: Householder reflections reduce A to a Hermitian tridiagonal T
// (A = Q T Q^H); a diagonal unitary D makes T real (T' = D^H T D with
// off-diagonals |e_k|); implicit symmetric QR steps with Wilkinson shifts
// diagonalise T' = Z Lambda Z^T with plane rotations; the eigenvectors of A
// are Q D Z.  O(m^3); m <= 256 here.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <complex>
#include <numeric>
#include <vector>

#include "internal.h"

namespace ssqcd {
namespace {

using cd = std::complex<double>;

// Implicit symmetric QR with Wilkinson shifts on a real symmetric
// tridiagonal matrix (the textbook "implicit shifted QR step", Golub & Van
// Loan, Matrix Computations, Sec. 8.3): d[0..n) diagonal, e[i] couples i and
// i + 1.  Each step works on the lowest block [lo, hi] that is still
// coupled: the shift mu is the eigenvalue of its trailing 2x2 block nearer
// its last diagonal entry; a plane rotation of rows/columns lo, lo + 1 is
// chosen from (d[lo] - mu, e[lo]), and the bulge it creates below the
// sub-diagonal is chased down the block by rotations of (k, k + 1).  The
// columns of Z (n x n, row-major) receive every rotation, so Z T_final Z^T
// stays equal to the input.  Couplings below eps (|d_i| + |d_i+1|) are set
// to zero.
int tridiagonal_qr(int n, std::vector<double>& d, std::vector<double>& e, std::vector<double>& Z) {
  auto rotate_cols = [&](int k, double c, double s) {
    for (int r = 0; r < n; ++r) {
      double* zr = &Z[(size_t)r * n];
      const double a = zr[k], b = zr[k + 1];
      zr[k] = c * a + s * b;
      zr[k + 1] = c * b - s * a;
    }
  };
  int steps = 0;
  int hi = n - 1;
  while (hi > 0) {
    // deflate converged couplings at the bottom
    if (std::fabs(e[hi - 1]) <= DBL_EPSILON * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    // top of the coupled block ending at hi
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > DBL_EPSILON * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    if (lo > 0) e[lo - 1] = 0.0;
    if (++steps > 60 * n) return -1;
    // Wilkinson shift from the trailing 2x2 block [[d[hi-1], b], [b, d[hi]]]
    const double b = e[hi - 1];
    const double half = 0.5 * (d[hi - 1] - d[hi]);
    const double root = std::hypot(half, b);
    const double mu = d[hi] - b * b / (half + (half >= 0.0 ? root : -root));
    // first rotation from the shifted leading column, then chase the bulge
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = std::hypot(x, z);
      const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? z / r : 0.0;
      if (k > lo) e[k - 1] = r;  // the bulge (k + 1, k - 1) is annihilated
      // rotate the 2x2 block of rows/columns k, k + 1
      const double a = d[k], f = e[k], g = d[k + 1];
      const double cs = c * s, c2 = c * c, s2 = s * s;
      d[k] = c2 * a + 2.0 * cs * f + s2 * g;
      d[k + 1] = s2 * a - 2.0 * cs * f + c2 * g;
      e[k] = cs * (g - a) + (c2 - s2) * f;
      rotate_cols(k, c, s);
      if (k + 1 < hi) {
        // coupling (k + 2, k + 1) splits into a new bulge (k + 2, k)
        x = e[k];
        z = s * e[k + 1];
        e[k + 1] = c * e[k + 1];
      }
    }
  }
  return 0;
}

}  // namespace

int small_eigh(int m, const double2* a_in, double* evals, double2* evecs) {
  if (m <= 0) return fail(SSQCD_ERR_ARG, "small_eigh: m must be > 0");
  // full Hermitian copy from the lower triangle
  std::vector<cd> A((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j <= i; ++j) {
      const cd v(a_in[(size_t)i * m + j].x, a_in[(size_t)i * m + j].y);
      A[(size_t)i * m + j] = (i == j) ? cd(v.real(), 0.0) : v;
      A[(size_t)j * m + i] = std::conj(A[(size_t)i * m + j]);
    }
  std::vector<cd> Q((size_t)m * m, cd(0.0, 0.0));
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  std::vector<double> d(m), e(m, 0.0);
  std::vector<cd> sub(m, cd(0.0, 0.0));  // complex sub-diagonal T[k+1][k]
  std::vector<cd> v(m), p(m), w(m), qv(m);
  for (int k = 0; k + 2 < m; ++k) {
    const int len = m - k - 1;
    double xnorm2 = 0.0;
    for (int i = 0; i < len; ++i) xnorm2 += std::norm(A[(size_t)(k + 1 + i) * m + k]);
    const double xnorm = std::sqrt(xnorm2);
    const cd x0 = A[(size_t)(k + 1) * m + k];
    double tail2 = xnorm2 - std::norm(x0);
    if (xnorm == 0.0 || tail2 <= 0.0) continue;  // column already reduced
    const cd phase = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cd(1.0, 0.0);
    for (int i = 0; i < len; ++i) v[i] = A[(size_t)(k + 1 + i) * m + k];
    v[0] += phase * xnorm;
    double vv = 0.0;
    for (int i = 0; i < len; ++i) vv += std::norm(v[i]);
    const double tau = 2.0 / vv;
    // p = tau A22 v
    for (int i = 0; i < len; ++i) {
      cd acc(0.0, 0.0);
      const cd* row = &A[(size_t)(k + 1 + i) * m + (k + 1)];
      for (int j = 0; j < len; ++j) acc += row[j] * v[j];
      p[i] = tau * acc;
    }
    cd vp(0.0, 0.0);
    for (int i = 0; i < len; ++i) vp += std::conj(v[i]) * p[i];
    const double K = 0.5 * tau * vp.real();
    for (int i = 0; i < len; ++i) w[i] = p[i] - K * v[i];
    // A22 -= v w^H + w v^H
    for (int i = 0; i < len; ++i) {
      cd* row = &A[(size_t)(k + 1 + i) * m + (k + 1)];
      for (int j = 0; j < len; ++j) row[j] -= v[i] * std::conj(w[j]) + w[i] * std::conj(v[j]);
    }
    // column k below the diagonal becomes (-phase * |x|, 0, ..., 0)
    A[(size_t)(k + 1) * m + k] = -phase * xnorm;
    A[(size_t)k * m + (k + 1)] = std::conj(-phase * xnorm);
    for (int i = 1; i < len; ++i) {
      A[(size_t)(k + 1 + i) * m + k] = 0.0;
      A[(size_t)k * m + (k + 1 + i)] = 0.0;
    }
    // Q[:, k+1:] -= tau (Q[:, k+1:] v) v^H
    for (int r = 0; r < m; ++r) {
      cd acc(0.0, 0.0);
      const cd* row = &Q[(size_t)r * m + (k + 1)];
      for (int j = 0; j < len; ++j) acc += row[j] * v[j];
      acc *= tau;
      cd* roww = &Q[(size_t)r * m + (k + 1)];
      for (int j = 0; j < len; ++j) roww[j] -= acc * std::conj(v[j]);
    }
  }
  for (int i = 0; i < m; ++i) d[i] = A[(size_t)i * m + i].real();
  for (int i = 0; i + 1 < m; ++i) sub[i] = A[(size_t)(i + 1) * m + i];
  // D: delta_0 = 1, delta_{k+1} = delta_k e_k/|e_k|  -> real off-diagonals |e_k|
  std::vector<cd> delta(m, cd(1.0, 0.0));
  for (int i = 0; i + 1 < m; ++i) {
    const double ae = std::abs(sub[i]);
    delta[i + 1] = ae > 0.0 ? delta[i] * (sub[i] / ae) : delta[i];
    e[i] = ae;
  }
  std::vector<double> Z((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Z[(size_t)i * m + i] = 1.0;
  if (tridiagonal_qr(m, d, e, Z) != 0) return fail(SSQCD_ERR_NOCONV, "small_eigh: QR did not converge");
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return d[a] < d[b]; });
  for (int c = 0; c < m; ++c) evals[c] = d[order[c]];
  if (evecs != nullptr) {
    // V = Q D Z
    for (int r = 0; r < m; ++r)
      for (int c = 0; c < m; ++c) {
        const int oc = order[c];
        cd acc(0.0, 0.0);
        for (int k = 0; k < m; ++k) acc += Q[(size_t)r * m + k] * delta[k] * Z[(size_t)k * m + oc];
        evecs[(size_t)r * m + c] = make_double2(acc.real(), acc.imag());
      }
  }
  return SSQCD_OK;
}

// Left singular vectors of a small complex m x m matrix by one-sided
// (Hestenes) Jacobi: columns b_p, b_q are rotated until pairwise orthogonal,
// B J = U Sigma; singular values are the final column norms.  Small singular
// values keep high relative accuracy, which the rank decision of the
// Rayleigh-Ritz basis relies on.
int small_svd_left(int m, const double2* a_in, double* sigma, double2* U) {
  if (m <= 0) return fail(SSQCD_ERR_ARG, "small_svd_left: m must be > 0");
  // columns as separate real and imaginary arrays, column-major (Bre[c m + r]);
  // the complex products are written out in real arithmetic (no library
  // complex multiplication with its special-value handling in the inner loops)
  std::vector<double> Bre((size_t)m * m), Bim((size_t)m * m);
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < m; ++c) {
      Bre[(size_t)c * m + r] = a_in[(size_t)r * m + c].x;
      Bim[(size_t)c * m + r] = a_in[(size_t)r * m + c].y;
    }
  bool rotated = true;
  for (int sweep = 0; sweep < 60 && rotated; ++sweep) {
    rotated = false;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        double* pr = &Bre[(size_t)p * m];
        double* pi = &Bim[(size_t)p * m];
        double* qr = &Bre[(size_t)q * m];
        double* qi = &Bim[(size_t)q * m];
        double alpha = 0.0, beta = 0.0, gr = 0.0, gi = 0.0;  // |b_p|^2, |b_q|^2, b_p^H b_q
        for (int r = 0; r < m; ++r) {
          alpha += pr[r] * pr[r] + pi[r] * pi[r];
          beta += qr[r] * qr[r] + qi[r] * qi[r];
          gr += pr[r] * qr[r] + pi[r] * qi[r];
          gi += pr[r] * qi[r] - pi[r] * qr[r];
        }
        const double ag = std::sqrt(gr * gr + gi * gi);
        if (ag == 0.0 || ag <= DBL_EPSILON * std::sqrt(alpha * beta)) continue;
        rotated = true;
        const double phr = gr / ag, phi = -gi / ag;  // conj(g) / |g|: b_q e^{-i phi} makes the coupling real
        const double zeta = (beta - alpha) / (2.0 * ag);
        const double t = std::copysign(1.0, zeta) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int r = 0; r < m; ++r) {
          const double xr = pr[r], xi = pi[r];
          const double yr = qr[r] * phr - qi[r] * phi, yi = qr[r] * phi + qi[r] * phr;
          pr[r] = c * xr - s * yr;
          pi[r] = c * xi - s * yi;
          qr[r] = s * xr + c * yr;
          qi[r] = s * xi + c * yi;
        }
      }
  }
  std::vector<double> nrm(m);
  for (int c = 0; c < m; ++c) {
    double s2 = 0.0;
    for (int r = 0; r < m; ++r) s2 += Bre[(size_t)c * m + r] * Bre[(size_t)c * m + r] + Bim[(size_t)c * m + r] * Bim[(size_t)c * m + r];
    nrm[c] = std::sqrt(s2);
  }
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return nrm[x] > nrm[y]; });
  for (int k = 0; k < m; ++k) {
    const int c = order[k];
    sigma[k] = nrm[c];
    const double inv = nrm[c] > 0.0 ? 1.0 / nrm[c] : 0.0;
    for (int r = 0; r < m; ++r)
      U[(size_t)r * m + k] = make_double2(Bre[(size_t)c * m + r] * inv, Bim[(size_t)c * m + r] * inv);
  }
  return SSQCD_OK;
}

// Right singular vector of the smallest singular value of a small complex
// rows x cols matrix (rows >= cols, row-major) by one-sided Jacobi on its
// columns, accumulating the rotations: M J = U Sigma, so the columns of J
// are the right singular vectors.  Returns sigma_min in *smin and the vector
// in v[cols].
int small_svd_min_right(int rows, int cols, const double2* a_in, double* smin, double2* v) {
  if (rows < cols || cols <= 0) return fail(SSQCD_ERR_ARG, "small_svd_min_right: need rows >= cols > 0");
  std::vector<cd> B((size_t)cols * rows);  // column-major
  for (int r = 0; r < rows; ++r)
    for (int c = 0; c < cols; ++c) B[(size_t)c * rows + r] = cd(a_in[(size_t)r * cols + c].x, a_in[(size_t)r * cols + c].y);
  std::vector<cd> J((size_t)cols * cols, cd(0.0, 0.0));  // column-major
  for (int c = 0; c < cols; ++c) J[(size_t)c * cols + c] = 1.0;
  bool rotated = true;
  for (int sweep = 0; sweep < 60 && rotated; ++sweep) {
    rotated = false;
    for (int p = 0; p < cols - 1; ++p)
      for (int q = p + 1; q < cols; ++q) {
        cd* bp = &B[(size_t)p * rows];
        cd* bq = &B[(size_t)q * rows];
        double alpha = 0.0, beta = 0.0;
        cd g(0.0, 0.0);
        for (int r = 0; r < rows; ++r) {
          alpha += std::norm(bp[r]);
          beta += std::norm(bq[r]);
          g += std::conj(bp[r]) * bq[r];
        }
        const double ag = std::abs(g);
        if (ag == 0.0 || ag <= DBL_EPSILON * std::sqrt(alpha * beta)) continue;
        rotated = true;
        const cd ph = g / ag;
        const double zeta = (beta - alpha) / (2.0 * ag);
        const double t = std::copysign(1.0, zeta) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int r = 0; r < rows; ++r) {
          const cd x = bp[r], y = bq[r] * std::conj(ph);
          bp[r] = c * x - s * y;
          bq[r] = s * x + c * y;
        }
        cd* jp = &J[(size_t)p * cols];
        cd* jq = &J[(size_t)q * cols];
        for (int r = 0; r < cols; ++r) {
          const cd x = jp[r], y = jq[r] * std::conj(ph);
          jp[r] = c * x - s * y;
          jq[r] = s * x + c * y;
        }
      }
  }
  int cmin = 0;
  double nmin = 0.0;
  for (int c = 0; c < cols; ++c) {
    double s2 = 0.0;
    for (int r = 0; r < rows; ++r) s2 += std::norm(B[(size_t)c * rows + r]);
    if (c == 0 || s2 < nmin) {
      nmin = s2;
      cmin = c;
    }
  }
  *smin = std::sqrt(nmin);
  for (int r = 0; r < cols; ++r) {
    const cd x = J[(size_t)cmin * cols + r];
    v[r] = make_double2(x.real(), x.imag());
  }
  return SSQCD_OK;
}

}  // namespace ssqcd

extern "C" int ssqcd_small_eigh(int m, const double* a, double* evals, double* evecs) {
  if (a == nullptr || evals == nullptr) return ssqcd::fail(SSQCD_ERR_ARG, "ssqcd_small_eigh: NULL argument");
  return ssqcd::small_eigh(m, reinterpret_cast<const double2*>(a), evals, reinterpret_cast<double2*>(evecs));
}
