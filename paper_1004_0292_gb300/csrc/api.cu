// C-ABI entry points: lattice handles, gauge upload, operator application,
// shifted CG, moments and the Sakurai-Sugiura / Rayleigh-Ritz solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "internal.h"

using namespace ssqcd;

struct ssqcd_result_s {
  cudaStream_t stream = nullptr;
  long long n = 0;
  int V = 0;
  std::vector<double> evals;
  std::vector<double> residuals;
  DevBuf evecs;  // [count][12][V] device layout
  ssqcd_stats stats{};
};

namespace {

// A solve with its host-side setup done (plan_solve).
struct SolvePlan {
  ssqcd_opts o{};
  int N = 0, M = 0, L = 0, K = 1, MM = 0, NU = 0;
  bool hankel = false;
  double a = 0.0, b = 0.0, core = 0.0, gamma0 = 0.0, rho = 0.0;
  // per window: centre, radius, accepted interval [lo, hi] (hi_open: the
  // upper end belongs to the next window)
  std::vector<double> gam, rad, lo, hi;
  std::vector<char> hi_open;
  std::vector<double2> zu;                   // union of the windows' points
  std::vector<std::vector<double2>> coefk;   // per window: [NU][MM] moment coefficients
  // every point's conjugate is a point, with conjugate coefficients in every
  // window: the moments are real combinations of the seed residuals
  bool real_moments = false;
};

}  // namespace

namespace {

int check_lattice(ssqcd_lattice lat, bool need_gauge) {
  if (lat == nullptr) return fail(SSQCD_ERR_ARG, "NULL lattice");
  if (need_gauge && !lat->has_gauge) return fail(SSQCD_ERR_ARG, "no gauge field uploaded");
  return SSQCD_OK;
}

// Bring a user-layout block of nf spinor fields (host or device) to the device
// layout in `dst` (resized).
int to_device_layout(ssqcd_lattice lat, const double* src, int nf, int on_device, DevBuf& dst) {
  const int V = lat->g.V;
  const size_t bytes = sizeof(double2) * 12 * (size_t)V * nf;
  SS_TRY(dst.alloc(bytes));
  const double2* user = reinterpret_cast<const double2*>(src);
  if (!on_device) {
    SS_TRY(lat->stage.alloc(bytes));
    SS_CUDA(cudaMemcpyAsync(lat->stage.p, src, bytes, cudaMemcpyHostToDevice, lat->stream));
    user = lat->stage.as<double2>();
  }
  return pack_spinors(user, dst.as<double2>(), nf, V, lat->stream);
}

// Write nf device-layout fields to a user-layout buffer (host or device).
int from_device_layout(ssqcd_lattice lat, const double2* src, int nf, int on_device, double* dst) {
  const int V = lat->g.V;
  const size_t bytes = sizeof(double2) * 12 * (size_t)V * nf;
  if (on_device) return unpack_spinors(src, reinterpret_cast<double2*>(dst), nf, V, lat->stream);
  SS_TRY(lat->stage.alloc(bytes));
  SS_TRY(unpack_spinors(src, lat->stage.as<double2>(), nf, V, lat->stream));
  SS_CUDA(cudaMemcpyAsync(dst, lat->stage.p, bytes, cudaMemcpyDeviceToHost, lat->stream));
  SS_CUDA(cudaStreamSynchronize(lat->stream));
  return SSQCD_OK;
}

}  // namespace

// --------------------------------------------------------------------------------------------
extern "C" int ssqcd_create_lattice(const int dims[4], double kappa, int bc_t, int precision, void* cuda_stream,
                                    ssqcd_lattice* out) {
  if (out == nullptr || dims == nullptr) return fail(SSQCD_ERR_ARG, "ssqcd_create_lattice: NULL argument");
  *out = nullptr;
  long long V = 1;
  for (int i = 0; i < 4; ++i) {
    if (dims[i] < 1) return fail(SSQCD_ERR_ARG, "lattice extents must be >= 1");
    V *= dims[i];
  }
  if (V > (1LL << 27)) return fail(SSQCD_ERR_ARG, "lattice volume above 2^27 sites");
  if (bc_t != 1 && bc_t != -1) return fail(SSQCD_ERR_ARG, "bc_t must be +1 or -1");
  if (!valid_precision(precision)) return fail(SSQCD_ERR_ARG, "unknown precision");
  if (!std::isfinite(kappa)) return fail(SSQCD_ERR_ARG, "kappa must be finite");
  int dev = 0;
  SS_CUDA(cudaGetDevice(&dev));
  auto* lat = new (std::nothrow) ssqcd_lattice_s();
  if (!lat) return fail(SSQCD_ERR_OOM, "host allocation failed");
  lat->g = Geometry{dims[0], dims[1], dims[2], dims[3], (int)V, kappa, (double)bc_t};
  lat->precision = precision;
  lat->stream = static_cast<cudaStream_t>(cuda_stream);
  *out = lat;
  return SSQCD_OK;
}

extern "C" void ssqcd_lattice_destroy(ssqcd_lattice lat) {
  if (!lat) return;
  cudaStreamSynchronize(lat->stream);
  delete lat;
}

extern "C" int ssqcd_upload_gauge(ssqcd_lattice lat, const double* links, int on_device) {
  SS_TRY(check_lattice(lat, false));
  if (links == nullptr) return fail(SSQCD_ERR_ARG, "NULL links");
  const int V = lat->g.V;
  const size_t bytes = sizeof(double2) * 36 * (size_t)V;
  SS_TRY(lat->u64.alloc(bytes));
  const double2* user = reinterpret_cast<const double2*>(links);
  if (!on_device) {
    SS_TRY(lat->stage.alloc(bytes));
    SS_CUDA(cudaMemcpyAsync(lat->stage.p, links, bytes, cudaMemcpyHostToDevice, lat->stream));
    user = lat->stage.as<double2>();
  }
  SS_TRY(pack_gauge64(user, lat->u64.as<double2>(), V, lat->stream));
  if (lat->precision == SSQCD_MIXED) {
    SS_TRY(lat->u16.alloc(sizeof(uint2) * 12 * (size_t)V));
    SS_TRY(pack_gauge16(lat->u64.as<double2>(), lat->u16.p, V, lat->stream));
  } else if (lat->precision == SSQCD_MIXED_F32LINKS) {
    SS_TRY(lat->u32.alloc(sizeof(float4) * 12 * (size_t)V));
    SS_TRY(pack_gauge32(lat->u64.as<double2>(), lat->u32.p, V, lat->stream));
  }
  lat->gauge_version++;
  if (lat->precision == SSQCD_DF) SS_TRY(ensure_df_links(lat));
  SS_CUDA(cudaStreamSynchronize(lat->stream));
  lat->has_gauge = true;
  return SSQCD_OK;
}

int ssqcd::ensure_df_links(ssqcd_lattice lat) {
  if (lat->udf.p != nullptr && lat->udf_version == lat->gauge_version) return SSQCD_OK;
  SS_TRY(lat->udf.alloc(sizeof(float4) * 36 * (size_t)lat->g.V));
  SS_TRY(pack_gauge_df(lat->u64.as<double2>(), lat->udf.as<float4>(), lat->g.V, lat->stream));
  // ready for work on any stream (the request scheduler uses its own)
  SS_CUDA(cudaStreamSynchronize(lat->stream));
  lat->udf_version = lat->gauge_version;
  return SSQCD_OK;
}

extern "C" int ssqcd_apply_H(ssqcd_lattice lat, const double* in, double* out, int nrhs, int on_device) {
  SS_TRY(check_lattice(lat, true));
  if (nrhs < 0 || (nrhs > 0 && (in == nullptr || out == nullptr))) return fail(SSQCD_ERR_ARG, "bad apply_H arguments");
  if (nrhs == 0) return SSQCD_OK;
  DevBuf a, b;
  SS_TRY(to_device_layout(lat, in, nrhs, on_device, a));
  SS_TRY(b.alloc(a.bytes));
  SS_TRY(wilson64(lat->g, lat->u64.as<double2>(), a.as<double2>(), b.as<double2>(), nrhs, 0.0, 1.0, nullptr,
                  nullptr, lat->stream));
  SS_TRY(from_device_layout(lat, b.as<double2>(), nrhs, on_device, out));
  SS_CUDA(cudaStreamSynchronize(lat->stream));
  return SSQCD_OK;
}

extern "C" int ssqcd_apply_H_mixed(ssqcd_lattice lat, const double* in, double* out, int nrhs, int on_device) {
  SS_TRY(check_lattice(lat, true));
  if (!is_mixed(lat->precision) && lat->precision != SSQCD_DF)
    return fail(SSQCD_ERR_ARG, "apply_H_mixed needs a mixed-precision or SSQCD_DF lattice");
  if (nrhs < 0 || (nrhs > 0 && (in == nullptr || out == nullptr))) return fail(SSQCD_ERR_ARG, "bad apply_H arguments");
  if (nrhs == 0) return SSQCD_OK;
  const long long n = 12LL * lat->g.V * nrhs;
  DevBuf a, a32, b32;
  SS_TRY(to_device_layout(lat, in, nrhs, on_device, a));
  if (lat->precision == SSQCD_DF) {
    SS_TRY(ensure_df_links(lat));
    SS_TRY(a32.alloc(sizeof(float4) * n));
    SS_TRY(b32.alloc(sizeof(float4) * n));
    SS_TRY(convert_f64_to_df(a.as<double2>(), a32.as<float4>(), n, lat->stream));
    SS_TRY(wilson_df(lat->g, lat->udf.as<float4>(), a32.as<float4>(), b32.as<float4>(), nrhs, 0.0, 1.0,
                     lat->stream));
    SS_TRY(convert_df_to_f64(b32.as<float4>(), a.as<double2>(), n, lat->stream));
    SS_TRY(from_device_layout(lat, a.as<double2>(), nrhs, on_device, out));
    SS_CUDA(cudaStreamSynchronize(lat->stream));
    return SSQCD_OK;
  }
  SS_TRY(a32.alloc(sizeof(float2) * n));
  SS_TRY(b32.alloc(sizeof(float2) * n));
  SS_TRY(convert_f64_to_f32(a.as<double2>(), a32.as<float2>(), n, lat->stream));
  const bool f16 = lat->precision == SSQCD_MIXED;
  SS_TRY(wilson32(lat->g, f16 ? lat->u16.p : lat->u32.p, f16 ? 16 : 32, a32.as<float2>(), b32.as<float2>(), nrhs,
                  0.f, 1.f, nullptr, nullptr, lat->stream));
  SS_TRY(convert_f32_to_f64(b32.as<float2>(), a.as<double2>(), n, lat->stream));
  SS_TRY(from_device_layout(lat, a.as<double2>(), nrhs, on_device, out));
  SS_CUDA(cudaStreamSynchronize(lat->stream));
  return SSQCD_OK;
}

extern "C" int ssqcd_shifted_cg(ssqcd_lattice lat, int N, const double* z, int L, const double* v, int on_device,
                                double sigma, double tol, int max_iter, int precision, int reliable_every,
                                double* y, int* iters, double* xi, int* seed_iters) {
  SS_TRY(check_lattice(lat, true));
  if (z == nullptr || v == nullptr) return fail(SSQCD_ERR_ARG, "NULL z or v");
  if (N < 1 || L < 1 || !(tol > 0.0) || max_iter < 1 || !std::isfinite(sigma))
    return fail(SSQCD_ERR_ARG, "bad shifted_cg arguments");
  if (is_mixed(precision) && precision != lat->precision)
    return fail(SSQCD_ERR_ARG, "a mixed-precision solve needs a lattice created with that precision");
  DevBuf vd, yd;
  SS_TRY(to_device_layout(lat, v, L, on_device, vd));
  std::vector<int> it(iters ? (size_t)L * N : 0);
  std::vector<double2> xx(xi ? (size_t)L * N : 0);
  ShiftedCGOut o;
  const int st = shifted_cg_device(lat, N, reinterpret_cast<const double2*>(z), L, vd.as<double2>(), sigma, tol,
                                   max_iter, precision, reliable_every, yd, iters ? it.data() : nullptr,
                                   xi ? xx.data() : nullptr, &o);
  if (st != SSQCD_OK && st != SSQCD_ERR_BREAKDOWN && st != SSQCD_ERR_NOCONV) return st;
  if (y != nullptr) SS_TRY(from_device_layout(lat, yd.as<double2>(), L * N, on_device, y));
  if (iters != nullptr) {
    if (on_device) SS_CUDA(cudaMemcpy(iters, it.data(), sizeof(int) * it.size(), cudaMemcpyHostToDevice));
    else std::memcpy(iters, it.data(), sizeof(int) * it.size());
  }
  if (xi != nullptr) {
    if (on_device) SS_CUDA(cudaMemcpy(xi, xx.data(), sizeof(double2) * xx.size(), cudaMemcpyHostToDevice));
    else std::memcpy(xi, xx.data(), sizeof(double2) * xx.size());
  }
  if (seed_iters) *seed_iters = o.seed_iters;
  SS_CUDA(cudaStreamSynchronize(lat->stream));
  return st;
}

extern "C" int ssqcd_moments(ssqcd_lattice lat, int N, int M, int L, const double* w, const double* zeta,
                             const double* y, double* s_hat, int on_device) {
  SS_TRY(check_lattice(lat, false));
  if (N < 1 || M < 1 || L < 1 || !w || !zeta || !y || !s_hat) return fail(SSQCD_ERR_ARG, "bad moments arguments");
  std::vector<double2> coef((size_t)N * M);
  for (int j = 0; j < N; ++j) {
    double zr = 1.0, zi = 0.0;  // zeta_j^k
    for (int k = 0; k < M; ++k) {
      const double wr = w[2 * j], wi = w[2 * j + 1];
      coef[(size_t)j * M + k] = make_double2(wr * zr - wi * zi, wr * zi + wi * zr);
      const double ar = zeta[2 * j], ai = zeta[2 * j + 1];
      const double nr = zr * ar - zi * ai, ni = zr * ai + zi * ar;
      zr = nr;
      zi = ni;
    }
  }
  DevBuf yd, sd, scratch;
  SS_TRY(to_device_layout(lat, y, L * N, on_device, yd));
  const long long n = 12LL * lat->g.V;
  SS_TRY(sd.alloc(sizeof(double2) * n * M * L));
  SS_TRY(moments_device(yd.as<double2>(), N, M, L, n, coef.data(), sd.as<double2>(), scratch, lat->stream));
  SS_TRY(from_device_layout(lat, sd.as<double2>(), L * M, on_device, s_hat));
  SS_CUDA(cudaStreamSynchronize(lat->stream));
  return SSQCD_OK;
}

namespace ssqcd {

int moments_device(const double2* y, int N, int M, int L, long long n, const double2* coef_host, double2* s_hat,
                   DevBuf& scratch, cudaStream_t s) {
  SS_TRY(scratch.alloc(sizeof(double2) * (size_t)N * M));
  SS_CUDA(cudaMemcpyAsync(scratch.p, coef_host, sizeof(double2) * (size_t)N * M, cudaMemcpyHostToDevice, s));
  for (int l = 0; l < L; ++l)
    SS_TRY(combine(y + (long long)l * N * n, N, n, scratch.as<double2>(), M, s_hat + (long long)l * M * n, s));
  // the coefficient upload must finish before `scratch` can be reused by the caller
  SS_CUDA(cudaStreamSynchronize(s));
  return SSQCD_OK;
}

}  // namespace ssqcd

// --------------------------------------------------------------------------------------------
extern "C" void ssqcd_default_opts(ssqcd_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->path = SSQCD_PATH_LINES;
  o->beta = 0.3;
  o->nprime = 0;
  o->tol = 1e-12;
  o->sigma = 0.0;
  o->max_iter = 100000;
  o->rank_tol = 1e-14;
  o->reliable_every = 0;
  o->windows = 1;
  o->extract = SSQCD_EXTRACT_RR;
  o->hankel_tol = 1e-12;
  o->refine = 0;
  o->basis = 1;
  o->basis_max_bytes = 0.0;
  o->source_block = 0;
  o->converged_tol = 1e-8;
  o->block_streams = 1;
}

namespace {

// Orthonormal basis of span(S) (m vectors of length n, device): CGS2 QR on
// the device, S = Q0 R, then the SVD of the small R on the host,
// R = U Sigma W^H, so that S = (Q0 U) Sigma W^H.  The basis is Q0 U_r, the
// left singular vectors of S whose singular value exceeds rank_tol times the
// largest (the paper leaves the orthogonalisation open).  Returns r, Q [r][n].
int orthonormalise(const double2* S, int m, long long n, double rank_tol, DevBuf& Q, int& r, DevBuf& tmp,
                   DevBuf& scratch, cudaStream_t st, const cudaEvent_t* ready = nullptr, int group = 0) {
  DevBuf Rd, Cd;
  SS_TRY(Rd.alloc(sizeof(double2) * m * m));
  SS_TRY(tmp.alloc(sizeof(double2) * n * m));
  SS_TRY(cgs2(S, m, n, tmp.as<double2>(), Rd.as<double2>(), scratch, st, ready, group));
  std::vector<double2> R((size_t)m * m), U((size_t)m * m);
  std::vector<double> sig(m);
  SS_CUDA(cudaMemcpyAsync(R.data(), Rd.p, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  SS_TRY(small_svd_left(m, R.data(), sig.data(), U.data()));
  if (!(sig[0] > 0.0)) return fail(SSQCD_ERR_ARG, "moment block is zero");
  int r1 = 0;
  while (r1 < m && sig[r1] > rank_tol * sig[0]) ++r1;
  std::vector<double2> C((size_t)m * r1);
  for (int a = 0; a < m; ++a)
    for (int c = 0; c < r1; ++c) C[(size_t)a * r1 + c] = U[(size_t)a * m + c];
  SS_TRY(Cd.alloc(sizeof(double2) * m * r1));
  SS_CUDA(cudaMemcpyAsync(Cd.p, C.data(), sizeof(double2) * m * r1, cudaMemcpyHostToDevice, st));
  SS_TRY(Q.alloc(sizeof(double2) * n * r1));
  SS_TRY(combine(tmp.as<double2>(), m, n, Cd.as<double2>(), r1, Q.as<double2>(), st));
  SS_CUDA(cudaStreamSynchronize(st));
  r = r1;
  return SSQCD_OK;
}

}  // namespace

namespace {

// Ritz values in [lo, hi] (hi_open: the upper end belongs to the next
// window) out of theta.
std::vector<int> accepted(const std::vector<double>& theta, double lo, double hi, bool hi_open) {
  std::vector<int> acc;
  for (int c = 0; c < (int)theta.size(); ++c)
    if (theta[c] >= lo && (hi_open ? theta[c] < hi : theta[c] <= hi)) acc.push_back(c);
  return acc;
}

// A X and ||A x - theta x|| for the accepted pairs, X (cnt vectors of n,
// device, FP64) formed by the caller; appends the eigenvalues and residuals.
int finish_ritz(ssqcd_lattice lat, const DevBuf& X, const std::vector<double>& ev, std::vector<double>& evals,
                std::vector<double>& resid, DevBuf& scratch, cudaStream_t st) {
  const long long n = 12LL * lat->g.V;
  const int cnt = (int)ev.size();
  std::vector<double> rs(cnt);
  DevBuf AX, th, rn;
  SS_TRY(AX.alloc(sizeof(double2) * n * cnt));
  SS_TRY(wilson64(lat->g, lat->u64.as<double2>(), X.as<double2>(), AX.as<double2>(), cnt, 0.0, 1.0, nullptr,
                  nullptr, st));
  SS_TRY(th.alloc(sizeof(double) * cnt));
  SS_TRY(rn.alloc(sizeof(double) * cnt));
  SS_CUDA(cudaMemcpyAsync(th.p, ev.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
  SS_TRY(col_residual_norms(AX.as<double2>(), X.as<double2>(), th.as<double>(), cnt, n, rn.as<double>(), scratch,
                            st));
  SS_CUDA(cudaMemcpyAsync(rs.data(), rn.p, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  evals.insert(evals.end(), ev.begin(), ev.end());
  resid.insert(resid.end(), rs.begin(), rs.end());
  return SSQCD_OK;
}

// Rayleigh-Ritz for one window with the projection kept implicit: the CGS2
// basis T of S (m columns, orthonormal or zero, S = T R) is used as it is,
// and the rank cut of the SVD R = U Sigma V^H enters only the small
// matrices: with U_r the left singular vectors above rank_tol, the
// orthonormal basis is T U_r, so (T U_r)^H A (T U_r) = U_r^H (T^H A T) U_r
// and a Ritz vector is T U_r w.  The same Ritz pairs as forming T U_r first,
// without that n x m x r combination; T^H A T is Hermitian, so only its
// upper tiles are formed.
int rayleigh_ritz_projected(ssqcd_lattice lat, const double2* S, int m, double rank_tol, double lo, double hi,
                            bool hi_open, std::vector<double>& evals, std::vector<double>& resid, DevBuf& X,
                            int& cnt, int& rank, DevBuf& scratch, cudaStream_t st, const cudaEvent_t* ready,
                            int group) {
  const long long n = 12LL * lat->g.V;
  // SSQCD_DF solves: the basis, A T and the products in float-float on the
  // FP32 pipes (blas_df.cu); the eigenvectors and their residuals in FP64
  const bool df = lat->precision == SSQCD_DF;
  DevBuf T, AT, Gd, Rd, gs;
  SS_TRY(T.alloc(sizeof(double2) * n * m));  // a float-float element takes 16 B too
  SS_TRY(Rd.alloc(sizeof(double2) * m * m));
  if (df) {
    if (ready != nullptr && group > 0)  // the conversion reads every column
      for (int g = 0; g * group < m; ++g)
        if (ready[g] != nullptr) SS_CUDA(cudaStreamWaitEvent(st, ready[g], 0));
    DevBuf Sdf;
    SS_TRY(Sdf.alloc(sizeof(float4) * n * m));
    SS_TRY(convert_f64_to_df(S, Sdf.as<float4>(), n * m, st));
    SS_TRY(cgs2_df(Sdf.as<float4>(), m, n, T.as<float4>(), Rd.as<double2>(), scratch, st));
  } else {
    SS_TRY(cgs2(S, m, n, T.as<double2>(), Rd.as<double2>(), scratch, st, ready, group));
  }
  std::vector<double2> R((size_t)m * m), U((size_t)m * m), G((size_t)m * m);
  SS_CUDA(cudaMemcpyAsync(R.data(), Rd.p, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, st));
  // A T and T^H A T do not depend on the rank cut: they run on the device
  // while the host takes the SVD of R
  SS_TRY(AT.alloc(sizeof(double2) * n * m));
  SS_TRY(Gd.alloc(sizeof(double2) * m * m));
  if (df) {
    SS_TRY(ensure_df_links(lat));
    SS_TRY(wilson_df(lat->g, lat->udf.as<float4>(), T.as<float4>(), AT.as<float4>(), m, 0.0, 1.0, st));
    SS_TRY(gram_df(T.as<float4>(), m, AT.as<float4>(), m, n, Gd.as<double2>(), gs, st, true));
  } else {
    SS_TRY(wilson64(lat->g, lat->u64.as<double2>(), T.as<double2>(), AT.as<double2>(), m, 0.0, 1.0, nullptr,
                    nullptr, st));
    SS_TRY(gram(T.as<double2>(), m, AT.as<double2>(), m, n, Gd.as<double2>(), gs, st, true));
  }
  // (a copy to pageable host memory returns when it is complete: R is
  // here, and G is read after the SVD)
  std::vector<double> sig(m);
  SS_TRY(small_svd_left(m, R.data(), sig.data(), U.data()));
  if (!(sig[0] > 0.0)) return fail(SSQCD_ERR_ARG, "moment block is zero");
  int r = 0;
  while (r < m && sig[r] > rank_tol * sig[0]) ++r;
  rank = r;
  SS_CUDA(cudaMemcpyAsync(G.data(), Gd.p, sizeof(double2) * m * m, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  AT.release();
  auto g_full = [&](int i, int j) {  // Hermitian T^H A T from its upper triangle
    return i <= j ? G[(size_t)i * m + j] : make_double2(G[(size_t)j * m + i].x, -G[(size_t)j * m + i].y);
  };
  // GU = G U_r (m x r), then At = U_r^H GU (r x r; small_eigh reads the lower triangle)
  std::vector<double2> GU((size_t)m * r), At((size_t)r * r), W((size_t)r * r);
  for (int i = 0; i < m; ++i)
    for (int c = 0; c < r; ++c) {
      double re = 0.0, im = 0.0;
      for (int j = 0; j < m; ++j) {
        const double2 g = g_full(i, j), u = U[(size_t)j * m + c];
        re += g.x * u.x - g.y * u.y;
        im += g.x * u.y + g.y * u.x;
      }
      GU[(size_t)i * r + c] = make_double2(re, im);
    }
  for (int a = 0; a < r; ++a)
    for (int c = 0; c <= a; ++c) {
      double re = 0.0, im = 0.0;
      for (int i = 0; i < m; ++i) {
        const double2 u = U[(size_t)i * m + a], g = GU[(size_t)i * r + c];  // conj(u) g
        re += u.x * g.x + u.y * g.y;
        im += u.x * g.y - u.y * g.x;
      }
      At[(size_t)a * r + c] = make_double2(re, im);
    }
  std::vector<double> theta(r);
  SS_TRY(small_eigh(r, At.data(), theta.data(), W.data()));
  const std::vector<int> acc = accepted(theta, lo, hi, hi_open);
  cnt = (int)acc.size();
  if (cnt == 0) return SSQCD_OK;
  // Ritz vectors T (U_r w): coefficients Cx = U_r W_acc (m x cnt)
  std::vector<double2> Cx((size_t)m * cnt);
  std::vector<double> ev(cnt);
  for (int c = 0; c < cnt; ++c) ev[c] = theta[acc[c]];
  for (int i = 0; i < m; ++i)
    for (int c = 0; c < cnt; ++c) {
      double re = 0.0, im = 0.0;
      for (int k = 0; k < r; ++k) {
        const double2 u = U[(size_t)i * m + k], w = W[(size_t)k * r + acc[c]];
        re += u.x * w.x - u.y * w.y;
        im += u.x * w.y + u.y * w.x;
      }
      Cx[(size_t)i * cnt + c] = make_double2(re, im);
    }
  DevBuf Wd;
  SS_TRY(Wd.alloc(sizeof(double2) * m * cnt));
  SS_CUDA(cudaMemcpyAsync(Wd.p, Cx.data(), sizeof(double2) * m * cnt, cudaMemcpyHostToDevice, st));
  SS_TRY(X.alloc(sizeof(double2) * n * cnt));
  if (df)
    SS_TRY(combine_df(T.as<float4>(), m, n, Wd.as<double2>(), cnt, X.as<double2>(), st));
  else
    SS_TRY(combine(T.as<double2>(), m, n, Wd.as<double2>(), cnt, X.as<double2>(), st));
  return finish_ritz(lat, X, ev, evals, resid, scratch, st);
}

// Rayleigh-Ritz for one window: orthonormal basis of S (m vectors), Ritz
// pairs of A on it, acceptance of the Ritz values in [lo, hi] (hi_open: the
// upper end belongs to the next window), eigenvectors X (device, [cnt][n]),
// residuals.  Appends to evals / resid and returns X in `X`.
int rayleigh_ritz_window(ssqcd_lattice lat, const double2* S, int m, double rank_tol, bool refine, double lo,
                         double hi, bool hi_open, std::vector<double>& evals, std::vector<double>& resid, DevBuf& X,
                         int& cnt, int& rank, DevBuf& scratch, cudaStream_t st, const cudaEvent_t* ready = nullptr,
                         int group = 0) {
  const long long n = 12LL * lat->g.V;
  if (!refine)
    return rayleigh_ritz_projected(lat, S, m, rank_tol, lo, hi, hi_open, evals, resid, X, cnt, rank, scratch, st,
                                   ready, group);
  DevBuf Q, tmp, AQ, Gd;
  int r = 0;
  SS_TRY(orthonormalise(S, m, n, rank_tol, Q, r, tmp, scratch, st, ready, group));
  tmp.release();
  rank = r;
  SS_TRY(AQ.alloc(sizeof(double2) * n * r));
  SS_TRY(wilson64(lat->g, lat->u64.as<double2>(), Q.as<double2>(), AQ.as<double2>(), r, 0.0, 1.0, nullptr, nullptr,
                  st));
  SS_TRY(Gd.alloc(sizeof(double2) * r * r));
  SS_TRY(gram(Q.as<double2>(), r, AQ.as<double2>(), r, n, Gd.as<double2>(), scratch, st));
  std::vector<double2> At((size_t)r * r), W((size_t)r * r);
  std::vector<double> theta(r);
  SS_CUDA(cudaMemcpyAsync(At.data(), Gd.p, sizeof(double2) * r * r, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  // Hermitian part (small_eigh reads the lower triangle)
  for (int i = 0; i < r; ++i)
    for (int j = 0; j <= i; ++j) {
      const double2 x = At[(size_t)i * r + j], y = At[(size_t)j * r + i];
      At[(size_t)i * r + j] = make_double2(0.5 * (x.x + y.x), 0.5 * (x.y - y.y));
    }
  SS_TRY(small_eigh(r, At.data(), theta.data(), W.data()));
  std::vector<int> acc;
  for (int c = 0; c < r; ++c)
    if (theta[c] >= lo && (hi_open ? theta[c] < hi : theta[c] <= hi)) acc.push_back(c);
  cnt = (int)acc.size();
  if (cnt == 0) return SSQCD_OK;
  std::vector<double2> Wacc((size_t)r * cnt);
  for (int i = 0; i < r; ++i)
    for (int c = 0; c < cnt; ++c) Wacc[(size_t)i * cnt + c] = W[(size_t)i * r + acc[c]];
  std::vector<double> ev(cnt), rs(cnt);
  for (int c = 0; c < cnt; ++c) ev[c] = theta[acc[c]];
  if (refine) {
    // Refined Ritz vectors: [Q, AQ] = W2 R2 (CGS2 on the device), so that
    // (A - theta) Q w = W2 R2 [-theta w; w]; w minimises the norm of the
    // small 2r x r matrix R2 [-theta I; I] times w (one-sided Jacobi, host)
    DevBuf QA, W2, R2d;
    SS_TRY(QA.alloc(sizeof(double2) * n * 2 * r));
    SS_CUDA(cudaMemcpyAsync(QA.p, Q.p, sizeof(double2) * n * r, cudaMemcpyDeviceToDevice, st));
    SS_CUDA(cudaMemcpyAsync(QA.as<double2>() + (size_t)n * r, AQ.p, sizeof(double2) * n * r,
                            cudaMemcpyDeviceToDevice, st));
    SS_TRY(W2.alloc(sizeof(double2) * n * 2 * r));
    SS_TRY(R2d.alloc(sizeof(double2) * 4 * r * r));
    SS_TRY(cgs2(QA.as<double2>(), 2 * r, n, W2.as<double2>(), R2d.as<double2>(), scratch, st));
    const int r2 = 2 * r;
    std::vector<double2> R2((size_t)r2 * r2), Mt((size_t)r2 * r), w(r);
    SS_CUDA(cudaMemcpyAsync(R2.data(), R2d.p, sizeof(double2) * R2.size(), cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaStreamSynchronize(st));
    auto a_full = [&](int i, int j) {  // Hermitian part of Q^H A Q from its lower triangle
      return i >= j ? At[(size_t)i * r + j] : make_double2(At[(size_t)j * r + i].x, -At[(size_t)j * r + i].y);
    };
    std::vector<double> sminv(cnt);
    for (int c = 0; c < cnt; ++c) {
      const double th = ev[c];
      for (int i = 0; i < r2; ++i)
        for (int j = 0; j < r; ++j) {
          const double2 a0 = R2[(size_t)i * r2 + j], a1 = R2[(size_t)i * r2 + r + j];
          Mt[(size_t)i * r + j] = make_double2(a1.x - th * a0.x, a1.y - th * a0.y);
        }
      double smin = 0.0;
      SS_TRY(small_svd_min_right(r2, r, Mt.data(), &smin, w.data()));
      sminv[c] = smin;
      double rq = 0.0;  // Rayleigh quotient w^H (Q^H A Q) w (|w| = 1)
      for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) {
          const double2 a = a_full(i, j), wi = w[i], wj = w[j];
          // Re(conj(wi) a wj)
          const double tr = a.x * wj.x - a.y * wj.y, ti = a.x * wj.y + a.y * wj.x;
          rq += wi.x * tr + wi.y * ti;
        }
      ev[c] = rq;
      for (int i = 0; i < r; ++i) Wacc[(size_t)i * cnt + c] = w[i];
    }
    // A Ritz value with no eigenvalue next to it (spurious) gets the refined
    // vector of the nearest eigenvalue, a duplicate of that pair: of two
    // refined vectors with overlap |x_i^H x_j| > 1/sqrt(2) (X = Q W, Q
    // orthonormal: the overlap is w_i^H w_j) keep the one with the smaller
    // ||(A - theta) x||.
    std::vector<char> keep(cnt, 1);
    for (int i = 0; i < cnt; ++i)
      for (int j = i + 1; j < cnt; ++j) {
        if (!keep[i] || !keep[j]) continue;
        double or_ = 0.0, oi = 0.0;
        for (int a = 0; a < r; ++a) {
          const double2 x = Wacc[(size_t)a * cnt + i], y = Wacc[(size_t)a * cnt + j];
          or_ += x.x * y.x + x.y * y.y;
          oi += x.x * y.y - x.y * y.x;
        }
        if (or_ * or_ + oi * oi > 0.5) keep[sminv[i] <= sminv[j] ? j : i] = 0;
      }
    int kept = 0;
    for (int c = 0; c < cnt; ++c) kept += keep[c];
    if (kept < cnt) {
      std::vector<double2> W2acc((size_t)r * kept);
      std::vector<double> ev2;
      for (int c = 0, o = 0; c < cnt; ++c) {
        if (!keep[c]) continue;
        for (int i = 0; i < r; ++i) W2acc[(size_t)i * kept + o] = Wacc[(size_t)i * cnt + c];
        ev2.push_back(ev[c]);
        ++o;
      }
      Wacc.swap(W2acc);
      ev.swap(ev2);
      cnt = kept;
      rs.resize(cnt);
    }
  }
  DevBuf Wd, AX, th, rn;
  SS_TRY(Wd.alloc(sizeof(double2) * r * cnt));
  SS_CUDA(cudaMemcpyAsync(Wd.p, Wacc.data(), sizeof(double2) * r * cnt, cudaMemcpyHostToDevice, st));
  SS_TRY(X.alloc(sizeof(double2) * n * cnt));
  SS_TRY(combine(Q.as<double2>(), r, n, Wd.as<double2>(), cnt, X.as<double2>(), st));
  SS_TRY(AX.alloc(sizeof(double2) * n * cnt));
  SS_TRY(wilson64(lat->g, lat->u64.as<double2>(), X.as<double2>(), AX.as<double2>(), cnt, 0.0, 1.0, nullptr,
                  nullptr, st));
  SS_TRY(th.alloc(sizeof(double) * cnt));
  SS_TRY(rn.alloc(sizeof(double) * cnt));
  SS_CUDA(cudaMemcpyAsync(th.p, ev.data(), sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
  SS_TRY(col_residual_norms(AX.as<double2>(), X.as<double2>(), th.as<double>(), cnt, n, rn.as<double>(), scratch,
                            st));
  SS_CUDA(cudaMemcpyAsync(rs.data(), rn.p, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  evals.insert(evals.end(), ev.begin(), ev.end());
  resid.insert(resid.end(), rs.begin(), rs.end());
  return SSQCD_OK;
}

// Block Hankel extraction for one window (Section 2.1): mu_k = V^H s_hat_k
// (L x L, k < 2M), H = [mu_{i+j}], H< = [mu_{i+j+1}] (ML x ML); the
// eigenvalues of the pencil (H<, H) are eta = (lambda - gamma) / rho.  With a
// contour symmetric under conjugation (both line pairs and the circle are)
// and Hermitian A, every mu_k is Hermitian and H = W^H f_0(Lambda) W with
// the filter f_0 > 0 on the real axis, so H is Hermitian positive
// semidefinite: H = Q diag(h) Q^H truncated to h_i > tol h_max reduces the
// pencil to the Hermitian matrix h^-1/2 Q^H H< Q h^-1/2, whose eigenvalues
// are those of the pencil (the same reduction as through the SVD of H,
// which equals this eigendecomposition).  Both small problems use the host
// Hermitian eigensolver.  S = [L][2M][n], V = [L][n] (device).
int hankel_window(const double2* V, int L, const double2* S, int M, long long n, double tol, double gamma,
                  double rho, double lo, double hi, bool hi_open, std::vector<double>& evals,
                  std::vector<double>& resid, int& rank, DevBuf& scratch, cudaStream_t st) {
  const int M2 = 2 * M, m = M * L;
  DevBuf Gd;
  SS_TRY(Gd.alloc(sizeof(double2) * L * L * M2));
  SS_TRY(gram(V, L, S, L * M2, n, Gd.as<double2>(), scratch, st));
  std::vector<double2> G((size_t)L * L * M2);
  SS_CUDA(cudaMemcpyAsync(G.data(), Gd.p, sizeof(double2) * G.size(), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  // mu_k[l][l'] = v_l^H s_hat_{k, l'} = G[l][l' 2M + k]
  auto mu = [&](int k, int l, int lp) { return G[(size_t)l * L * M2 + (size_t)lp * M2 + k]; };
  // Hermitian parts of H and H< (lower triangles suffice for small_eigh)
  std::vector<double2> H((size_t)m * m), Hs((size_t)m * m);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < M; ++j)
      for (int l = 0; l < L; ++l)
        for (int lp = 0; lp < L; ++lp) {
          const size_t r = (size_t)i * L + l, c = (size_t)j * L + lp;
          const double2 a0 = mu(i + j, l, lp), b0 = mu(i + j, lp, l);
          const double2 a1 = mu(i + j + 1, l, lp), b1 = mu(i + j + 1, lp, l);
          H[r * m + c] = make_double2(0.5 * (a0.x + b0.x), 0.5 * (a0.y - b0.y));
          Hs[r * m + c] = make_double2(0.5 * (a1.x + b1.x), 0.5 * (a1.y - b1.y));
        }
  std::vector<double> h(m);
  std::vector<double2> Q((size_t)m * m);
  SS_TRY(small_eigh(m, H.data(), h.data(), Q.data()));
  const double hmax = h[m - 1];
  if (!(hmax > 0.0)) return fail(SSQCD_ERR_ARG, "Hankel matrix of the moments is zero");
  std::vector<int> keep;
  for (int c = m - 1; c >= 0; --c)
    if (h[c] > tol * hmax) keep.push_back(c);
  const int r = (int)keep.size();
  rank = r;
  // C = h^-1/2 Q_r^H H< Q_r h^-1/2
  std::vector<double2> T((size_t)m * r), C((size_t)r * r);
  for (int a = 0; a < m; ++a)
    for (int q = 0; q < r; ++q) {  // T = H< Q_r (full H< from its Hermitian lower part)
      double sr = 0.0, si = 0.0;
      for (int b = 0; b < m; ++b) {
        const double2 x = a >= b ? Hs[(size_t)a * m + b] : make_double2(Hs[(size_t)b * m + a].x, -Hs[(size_t)b * m + a].y);
        const double2 y = Q[(size_t)b * m + keep[q]];
        sr += x.x * y.x - x.y * y.y;
        si += x.x * y.y + x.y * y.x;
      }
      T[(size_t)a * r + q] = make_double2(sr, si);
    }
  for (int p = 0; p < r; ++p)
    for (int q = 0; q < r; ++q) {
      double sr = 0.0, si = 0.0;
      for (int a = 0; a < m; ++a) {
        const double2 x = Q[(size_t)a * m + keep[p]], y = T[(size_t)a * r + q];
        sr += x.x * y.x + x.y * y.y;  // conj(x) y
        si += x.x * y.y - x.y * y.x;
      }
      const double sc = 1.0 / std::sqrt(h[keep[p]] * h[keep[q]]);
      C[(size_t)p * r + q] = make_double2(sr * sc, si * sc);
    }
  std::vector<double> eta(r);
  SS_TRY(small_eigh(r, C.data(), eta.data(), nullptr));
  for (int c = 0; c < r; ++c) {
    const double lam = gamma + rho * eta[c];
    if (lam >= lo && (hi_open ? lam < hi : lam <= hi)) {
      evals.push_back(lam);
      resid.push_back(std::nan(""));
    }
  }
  return SSQCD_OK;
}

}  // namespace

namespace {

// Everything of a solve that does not touch the device: windows, nodes,
// the union of the windows' points and the moment coefficients.
// True when the union of the points is closed under conjugation (exactly:
// the line pairs of a real centre are built that way) and every window's
// coefficient of the conjugate point is the conjugate of the point's own, to
// within 1e-12 of the largest coefficient of that moment.  The moment
// sum_j c_j x_j over such a set then has real coefficients in the Krylov
// basis of the seed residuals (x of conj z has the conjugate coefficients).
bool conjugate_closed(const std::vector<double2>& zu, const std::vector<std::vector<double2>>& coefk, int MM) {
  const int NU = (int)zu.size();
  std::vector<int> partner(NU, -1);
  for (int u = 0; u < NU; ++u) {
    for (int q = 0; q < NU; ++q)
      if (zu[q].x == zu[u].x && zu[q].y == -zu[u].y) {
        partner[u] = q;
        break;
      }
    if (partner[u] < 0) return false;
  }
  for (const auto& c : coefk)
    for (int m = 0; m < MM; ++m) {
      double big = 0.0;
      for (int u = 0; u < NU; ++u) big = std::max(big, std::hypot(c[(size_t)u * MM + m].x, c[(size_t)u * MM + m].y));
      for (int u = 0; u < NU; ++u) {
        const double2 a = c[(size_t)u * MM + m], b = c[(size_t)partner[u] * MM + m];
        if (std::hypot(a.x - b.x, a.y + b.y) > 1e-12 * big) return false;
      }
    }
  return true;
}

int plan_solve(const double interval[2], int N, int M, int L, const ssqcd_opts* opts_in, SolvePlan* P) {
  if (interval == nullptr || !(interval[1] > interval[0])) return fail(SSQCD_ERR_ARG, "interval must have b > a");
  if (N < 1 || M < 1 || L < 1) return fail(SSQCD_ERR_ARG, "N, M, L must be >= 1");
  ssqcd_opts o;
  ssqcd_default_opts(&o);
  if (opts_in) o = *opts_in;
  if (o.sources == nullptr) return fail(SSQCD_ERR_ARG, "opts.sources is required");
  if (o.extract != SSQCD_EXTRACT_RR && o.extract != SSQCD_EXTRACT_HANKEL)
    return fail(SSQCD_ERR_ARG, "unknown extraction");
  const bool hankel = o.extract == SSQCD_EXTRACT_HANKEL;
  if (hankel && !(o.hankel_tol > 0.0 && o.hankel_tol < 1.0)) return fail(SSQCD_ERR_ARG, "hankel_tol must be in (0, 1)");
  // Hankel needs the moments up to k = 2M - 1 (filter identity: 2M <= N)
  const int MM = hankel ? 2 * M : M;
  if (hankel && MM > N) return fail(SSQCD_ERR_ARG, "Hankel extraction needs 2M <= N");
  const int K = o.windows < 1 ? 1 : o.windows;
  if (K > 1 && o.path != SSQCD_PATH_LINES) return fail(SSQCD_ERR_ARG, "several windows need the line contour");
  const double a = interval[0], b = interval[1];
  const double core = (b - a) / K;  // accepted width of each window
  double gamma0 = a + 0.5 * core, rho = 0.5 * core;
  int np = 0, step = 0, half = N / 2;
  if (o.path == SSQCD_PATH_LINES) {
    np = o.nprime == 0 ? N / 2 : o.nprime;
    if (N < 4 || N % 2 || np < 4 || np % 2 || np > N)
      return fail(SSQCD_ERR_ARG, "lines need even N >= 4 and even 4 <= N' <= N");
    rho = 0.5 * core * (half - 1) / (double)(np / 2 - 1);
    step = np / 2 - 1;  // grid points per line between neighbouring windows (Section 3)
  } else if (o.path != SSQCD_PATH_CIRCLE) {
    return fail(SSQCD_ERR_ARG, "unknown path");
  }
  // nodes and weights of one window (the same in every window's own zeta)
  std::vector<double2> z, w;
  SS_TRY(contour_nodes(o.path, gamma0, rho, o.beta, N, z, w));
  // the union of the windows' nodes: windows k and k+1 share N - (N' - 2)
  // points; point j of window k is union point 2 (k step + j/2) + j%2
  const int NU = (K == 1) ? N : 2 * (half + (K - 1) * step);
  std::vector<double2> zu(NU);
  if (K == 1) {
    zu = z;
  } else {
    for (int gi = 0; gi < NU / 2; ++gi) {
      const double x = -1.0 + 2.0 * gi / (half - 1);
      zu[2 * gi] = make_double2(gamma0 + rho * x, rho * o.beta);
      zu[2 * gi + 1] = make_double2(gamma0 + rho * x, -rho * o.beta);
    }
  }
  // moment coefficients over the union for each window: c_k[u][m] = w_j zeta_j^m
  // for the window's points u = u(k, j), zero elsewhere
  std::vector<std::vector<double2>> coefk(K, std::vector<double2>((size_t)NU * MM, make_double2(0.0, 0.0)));
  for (int j = 0; j < N; ++j) {
    const double zr0 = (z[j].x - gamma0) / rho, zi0 = z[j].y / rho;
    double zr = 1.0, zi = 0.0;
    for (int m = 0; m < MM; ++m) {
      const double2 cv = make_double2(w[j].x * zr - w[j].y * zi, w[j].x * zi + w[j].y * zr);
      for (int k = 0; k < K; ++k) {
        const int u = (K == 1) ? j : 2 * (k * step + j / 2) + j % 2;
        coefk[k][(size_t)u * MM + m] = cv;
      }
      const double nr = zr * zr0 - zi * zi0, ni = zr * zi0 + zi * zr0;
      zr = nr;
      zi = ni;
    }
  }
  P->o = o;
  P->N = N;
  P->M = M;
  P->L = L;
  P->K = K;
  P->MM = MM;
  P->NU = NU;
  P->hankel = hankel;
  P->a = a;
  P->b = b;
  P->core = core;
  P->gamma0 = gamma0;
  P->rho = rho;
  P->zu.swap(zu);
  P->coefk.swap(coefk);
  P->real_moments = conjugate_closed(P->zu, P->coefk, MM);
  P->gam.resize(K);
  P->rad.assign(K, rho);
  P->lo.resize(K);
  P->hi.resize(K);
  P->hi_open.resize(K);
  for (int k = 0; k < K; ++k) {
    P->gam[k] = gamma0 + k * core;
    P->lo[k] = (K == 1) ? a : a + k * core;
    P->hi[k] = (K == 1) ? b : (k == K - 1 ? b : a + (k + 1) * core);
    P->hi_open[k] = k < K - 1;
  }
  return SSQCD_OK;
}

// A list of K windows [a_k, b_k] (any positions, the same N, N', beta and
// path): each window gets its own centre and radius as in plan_solve with
// one window; the union of the points is the concatenation of the windows'
// points with exact duplicates merged (windows laid out on a common grid
// share them, as in Section 3), and every window's moment coefficients sit
// at its own points of the union.  One shifted-CG run then serves all
// windows; each window accepts the Ritz values in its own [a_k, b_k].
int plan_windows(int K, const double* iv, int N, int M, int L, const ssqcd_opts* opts_in, SolvePlan* P) {
  if (K < 1 || iv == nullptr) return fail(SSQCD_ERR_ARG, "need K >= 1 windows");
  std::vector<std::vector<double2>> zk(K), wk(K);
  std::vector<double> gam(K), rad(K);
  SolvePlan one;
  for (int k = 0; k < K; ++k) {
    ssqcd_opts o;
    ssqcd_default_opts(&o);
    if (opts_in) o = *opts_in;
    o.windows = 1;
    SS_TRY(plan_solve(iv + 2 * k, N, M, L, &o, &one));
    gam[k] = one.gamma0;
    rad[k] = one.rho;
    zk[k] = one.zu;
    wk[k].resize(N);
    // the window's own coefficients: column m of point j is w_j zeta_j^m
    for (int j = 0; j < N; ++j) wk[k][j] = one.coefk[0][(size_t)j * one.MM];
  }
  P->o = one.o;
  P->N = N;
  P->M = M;
  P->L = L;
  P->K = K;
  P->MM = one.MM;
  P->hankel = one.hankel;
  P->a = iv[0];
  P->b = iv[1];
  P->core = iv[1] - iv[0];
  P->gamma0 = gam[0];
  P->rho = rad[0];
  P->gam = gam;
  P->rad = rad;
  P->lo.resize(K);
  P->hi.resize(K);
  P->hi_open.assign(K, 0);
  for (int k = 0; k < K; ++k) {
    P->lo[k] = iv[2 * k];
    P->hi[k] = iv[2 * k + 1];
  }
  // union with exact duplicates merged
  std::vector<double2> zu;
  std::vector<std::vector<int>> at(K, std::vector<int>(N));
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < N; ++j) {
      const double2 z = zk[k][j];
      int u = -1;
      for (int q = 0; q < (int)zu.size(); ++q)
        if (zu[q].x == z.x && zu[q].y == z.y) {
          u = q;
          break;
        }
      if (u < 0) {
        u = (int)zu.size();
        zu.push_back(z);
      }
      at[k][j] = u;
    }
  const int NU = (int)zu.size(), MM = P->MM;
  std::vector<std::vector<double2>> coefk(K, std::vector<double2>((size_t)NU * MM, make_double2(0.0, 0.0)));
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < N; ++j) {
      const double zr0 = (zk[k][j].x - gam[k]) / rad[k], zi0 = zk[k][j].y / rad[k];
      const double2 w = wk[k][j];
      double zr = 1.0, zi = 0.0;
      for (int m = 0; m < MM; ++m) {
        coefk[k][(size_t)at[k][j] * MM + m] = make_double2(w.x * zr - w.y * zi, w.x * zi + w.y * zr);
        const double nr = zr * zr0 - zi * zi0, ni = zr * zi0 + zi * zr0;
        zr = nr;
        zi = ni;
      }
    }
  P->NU = NU;
  P->zu.swap(zu);
  P->coefk.swap(coefk);
  P->real_moments = conjugate_closed(P->zu, P->coefk, MM);
  return SSQCD_OK;
}

// plan_real: the plan's points are conjugate-closed (SolvePlan::real_moments)
void fill_cg_stats(const ShiftedCGOut& cg, const std::vector<int>& iters, ssqcd_stats* st, bool plan_real = false) {
  st->iterations = cg.seed_iters;
  st->reliable_updates = cg.reliable_updates;
  st->ms_cg = cg.ms;
  st->max_shift_iters = iters.empty() ? 0 : *std::max_element(iters.begin(), iters.end());
  st->shift_updates = cg.shift_updates;
  st->timed = cg.timed ? 1 : 0;
  st->launches_update = cg.launches_update;
  st->ms_k_stencil = cg.ms_k[0];
  st->ms_k_seed = cg.ms_k[1];
  st->ms_k_scalars = cg.ms_k[2];
  st->ms_k_update = cg.ms_k[3];
  st->timed_shift_updates = cg.timed_units;
  st->basis = cg.basis;
  st->basis_bytes = cg.basis_bytes;
  st->real_moments = (plan_real && real_moments_enabled() && cg.basis == 1) ? 1 : 0;
}

// After the shifted CG: per window the moments (Eq. 2) and Rayleigh-Ritz (or
// the Hankel pencil) with acceptance in the window's core; then the
// eigenpairs of all windows sorted by eigenvalue.  yd: [L][NU][n] FP64
// solutions, or kb: the stored residuals of a Krylov-basis run (whichever
// is filled; released once the last window's moments exist); vd: the
// sources [L][n].  All device work on st.
int extract_eigenpairs(ssqcd_lattice lat, const SolvePlan& P, DevBuf& yd, KrylovBasis& kb, DevBuf& vd,
                       ssqcd_result_s* res, cudaStream_t st, std::vector<DevBuf>* Spre = nullptr) {
  const long long n = 12LL * lat->g.V;
  const int K = P.K, L = P.L, MM = P.MM, M = P.M, NU = P.NU;
  res->stats.gamma = P.gamma0;
  res->stats.rho = P.rho;
  res->stats.points = NU;
  DevBuf S, scratch;
  cudaEvent_t e0, e1, e2;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventCreate(&e2);
  struct Ev {
    cudaEvent_t* e[3];
    ~Ev() {
      for (auto x : e) cudaEventDestroy(*x);
    }
  } evs{{&e0, &e1, &e2}};
  cudaEventRecord(e0, st);
  const int m = MM * L;
  std::vector<DevBuf> Xk(K);
  std::vector<int> cntk(K, 0);
  // Moments from the stored residuals and Rayleigh-Ritz overlap: the last
  // source's moments form on a side stream, and the CGS2 of the basis waits
  // per source, so it orthogonalises the other sources' moments meanwhile.  The moment
  // scratch stays alive, and st waits for every side event, until the end.
  struct Overlap {
    cudaStream_t side = nullptr;
    std::vector<cudaEvent_t> ev;
    cudaStream_t st = nullptr;
    ~Overlap() {
      if (st != nullptr && !ev.empty()) cudaStreamWaitEvent(st, ev.back(), 0);  // error paths: st after the side work
      for (auto e : ev) cudaEventDestroy(e);
      if (side) cudaStreamDestroy(side);
    }
  } ov;
  DevBuf mscratch;
  const bool overlap = Spre == nullptr && kb.S > 0 && !P.hankel && L > 1;
  if (overlap) {
    SS_CUDA(cudaStreamCreateWithFlags(&ov.side, cudaStreamNonBlocking));
    ov.ev.resize(L);
    for (auto& e : ov.ev) SS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ov.st = st;
  }
  cudaEvent_t e_mom = nullptr;  // the end of the last window's moments (side stream when overlapped)
  struct EvOne {
    cudaEvent_t* e;
    ~EvOne() {
      if (*e) cudaEventDestroy(*e);
    }
  } ev_mom{&e_mom};
  for (int k = 0; k < K; ++k) {
    // moments of window k (Eq. 2), S = [L][MM][n] (formed here, or given)
    if (Spre != nullptr) {
      S.release();
      S.swap((*Spre)[k]);  // window k's moments, freed with S
      // every window's moments are formed already: the extraction of all
      // of them is Rayleigh-Ritz time
      if (k == 0) cudaEventRecord(e1, st);
    } else {
    SS_TRY(S.alloc(sizeof(double2) * n * m));
    if (overlap)
      SS_TRY(basis_moments(kb, P.coefk[k].data(), MM, S.as<double2>(), mscratch, st, ov.side, ov.ev.data(),
                           P.real_moments));
    else if (kb.S > 0)
      SS_TRY(basis_moments(kb, P.coefk[k].data(), MM, S.as<double2>(), scratch, st, nullptr, nullptr, P.real_moments));
    else
      SS_TRY(moments_device(yd.as<double2>(), NU, MM, L, n, P.coefk[k].data(), S.as<double2>(), scratch, st));
    if (k == K - 1) {
      if (overlap) {
        SS_CUDA(cudaEventCreate(&e_mom));
        SS_CUDA(cudaEventRecord(e_mom, ov.side));
      } else {
        cudaEventRecord(e1, st);
        yd.release();
        kb.release();
      }
    }
    }
    // Rayleigh-Ritz (or the Hankel pencil) and acceptance in the window's core
    const double lo = P.lo[k], hi = P.hi[k];
    const bool hi_open = P.hi_open[k] != 0;
    int rank = 0;
    if (P.hankel) {
      const size_t before = res->evals.size();
      SS_TRY(hankel_window(vd.as<double2>(), L, S.as<double2>(), M, n, P.o.hankel_tol, P.gam[k], P.rad[k], lo,
                           hi, hi_open, res->evals, res->residuals, rank, scratch, st));
      cntk[k] = (int)(res->evals.size() - before);
      res->stats.rank += rank;
      res->stats.n_ritz += rank;
      continue;
    }
    SS_TRY(rayleigh_ritz_window(lat, S.as<double2>(), m, P.o.rank_tol, P.o.refine != 0, lo, hi, hi_open,
                                res->evals, res->residuals, Xk[k], cntk[k], rank, scratch, st,
                                overlap ? ov.ev.data() : nullptr, MM));
    if (k == K - 1 && overlap) kb.release();  // st has waited for every source's moments
    res->stats.rank += rank;
    res->stats.n_ritz += rank;
    res->stats.matvecs_rr += rank + cntk[k];
  }
  // gather the windows' eigenvectors, then sort everything by eigenvalue
  int cnt = 0;
  for (int k = 0; k < K; ++k) cnt += cntk[k];
  res->stats.n_accepted = cnt;
  res->stats.n_converged = 0;
  for (double r : res->residuals)
    if (r <= P.o.converged_tol) ++res->stats.n_converged;
  if (P.hankel) {  // eigenvalues only: sort them
    std::sort(res->evals.begin(), res->evals.end());
  } else if (cnt > 0) {
    DevBuf all;
    SS_TRY(all.alloc(sizeof(double2) * n * cnt));
    int off = 0;
    for (int k = 0; k < K; ++k) {
      if (cntk[k] == 0) continue;
      cudaMemcpyAsync(all.as<double2>() + (size_t)off * n, Xk[k].p, sizeof(double2) * n * cntk[k],
                      cudaMemcpyDeviceToDevice, st);
      off += cntk[k];
    }
    std::vector<int> order(cnt);
    for (int i = 0; i < cnt; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return res->evals[x] < res->evals[y]; });
    {
      AllocStream plain(nullptr, false);  // the result outlives the caller's streams
      SS_TRY(res->evecs.alloc(sizeof(double2) * n * cnt));
    }
    std::vector<double> ev(cnt), rs(cnt);
    for (int i = 0; i < cnt; ++i) {
      ev[i] = res->evals[order[i]];
      rs[i] = res->residuals[order[i]];
      cudaMemcpyAsync(res->evecs.as<double2>() + (size_t)i * n, all.as<double2>() + (size_t)order[i] * n,
                      sizeof(double2) * n, cudaMemcpyDeviceToDevice, st);
    }
    res->evals = ev;
    res->residuals = rs;
    if (cudaStreamSynchronize(st) != cudaSuccess)
      return cuda_fail(cudaGetLastError(), "gathering eigenvectors", __FILE__, __LINE__);
  }
  cudaEventRecord(e2, st);
  cudaEventSynchronize(e2);
  // overlapped: moments up to the last source's combination (side stream),
  // Rayleigh-Ritz from there on (its start ran beside the moments)
  const cudaEvent_t e_mid = e_mom != nullptr ? e_mom : e1;
  float ms1 = 0.f, ms2 = 0.f;
  cudaEventElapsedTime(&ms1, e0, e_mid);
  cudaEventElapsedTime(&ms2, e_mid, e2);
  res->stats.ms_moments = ms1;
  res->stats.ms_rr = ms2;
  return SSQCD_OK;
}

}  // namespace

namespace {

void add_cg_stats(const ShiftedCGOut& b, ShiftedCGOut* acc) {
  acc->seed_iters = std::max(acc->seed_iters, b.seed_iters);
  acc->reliable_updates += b.reliable_updates;
  acc->ms += b.ms;
  acc->shift_updates += b.shift_updates;
  acc->timed = acc->timed || b.timed;
  acc->launches_update += b.launches_update;
  acc->timed_units += b.timed_units;
  for (int i = 0; i < 4; ++i) acc->ms_k[i] += b.ms_k[i];
  acc->basis = std::max(acc->basis, b.basis);
  acc->basis_bytes = std::max(acc->basis_bytes, b.basis_bytes);
}

// A planned solve: shifted CG over the union of the windows' points, the
// moments and the extraction.  With opts.source_block = B (0 < B < L) the
// sources run in blocks of B, one shifted-CG run per block (the seed
// recurrences of different sources never interact), and each block's
// moments of every window are formed before the next block starts, so the
// stored seed residuals of only B sources are held at a time.
// Drive several shifted-CG runs (each on its own stream) to the end
// together: two chunks in flight per run, the runs polled in turn.  Returns
// the first status other than OK (a run that breaks down or does not
// converge ends; the others go on).
int drive_runs(const std::vector<CgRunBase*>& runs) {
  const int nr = (int)runs.size();
  std::vector<char> done(nr, 0);
  int first = SSQCD_OK, live = nr;
  auto end_run = [&](int i, int status) {
    done[i] = 1;
    --live;
    if (first == SSQCD_OK) first = status;
  };
  for (int i = 0; i < nr; ++i) {
    int status = runs[i]->launch();
    if (status == SSQCD_OK) status = runs[i]->launch();
    if (status != SSQCD_OK) end_run(i, status);
  }
  while (live > 0) {
    for (int i = 0; i < nr; ++i) {
      if (done[i]) continue;
      int state = 0;
      int status = runs[i]->poll(true, &state);
      if (status == SSQCD_OK && state == CgRunBase::kPollDone) {
        end_run(i, SSQCD_OK);
        continue;
      }
      if (status == SSQCD_OK) status = runs[i]->launch();
      if (status != SSQCD_OK) end_run(i, status);
    }
  }
  return first;
}

int run_solve(ssqcd_lattice lat, const SolvePlan& P, ssqcd_result* out) {
  const int L = P.L, NU = P.NU, K = P.K, MM = P.MM;
  const long long n = 12LL * lat->g.V;
  auto* res = new (std::nothrow) ssqcd_result_s();
  if (!res) return fail(SSQCD_ERR_OOM, "host allocation failed");
  res->stream = lat->stream;
  res->V = lat->g.V;
  res->n = n;
  res->stats.gamma = P.gamma0;
  res->stats.rho = P.rho;
  res->stats.points = NU;
  cudaStream_t st = lat->stream;
  // sources -> device layout
  DevBuf vd, yd;
  KrylovBasis kb;
  int s1 = to_device_layout(lat, P.o.sources, L, P.o.sources_on_device, vd);
  if (s1 != SSQCD_OK) {
    delete res;
    return s1;
  }
  const int B = (P.o.source_block > 0 && P.o.source_block < L) ? P.o.source_block : L;
  std::vector<int> iters((size_t)NU * L);
  if (B == L) {
    // shifted CG over the union of the quadrature points (one seed recurrence per source)
    ShiftedCGOut cg;
    s1 = shifted_cg_solve(lat, NU, P.zu.data(), L, vd.as<double2>(), P.o.sigma, P.o.tol, P.o.max_iter,
                          lat->precision, P.o.reliable_every,
                          basis_cap_for(lat->precision, P.o.basis, P.o.basis_max_bytes, n, NU, L), yd, &kb,
                          iters.data(), &cg);
    fill_cg_stats(cg, iters, &res->stats, P.real_moments);
    *out = res;  // a result handle even on failure, so its stats can be read
    if (s1 != SSQCD_OK) return s1;
    if (!P.hankel) vd.release();
    return extract_eigenpairs(lat, P, yd, kb, vd, res, st);
  }
  // source blocks: every window's moments [L][MM][n], filled block by block
  std::vector<DevBuf> Sk(K);
  *out = res;
  for (int k = 0; k < K; ++k) SS_TRY(Sk[k].alloc(sizeof(double2) * n * MM * L));
  ShiftedCGOut cg;
  cudaEvent_t m0 = nullptr, m1 = nullptr;
  struct Evs {
    cudaEvent_t* a;
    cudaEvent_t* b;
    ~Evs() {
      if (*a) cudaEventDestroy(*a);
      if (*b) cudaEventDestroy(*b);
    }
  } evs{&m0, &m1};
  SS_CUDA(cudaEventCreate(&m0));
  SS_CUDA(cudaEventCreate(&m1));
  float ms_mom = 0.f;
  // G blocks at a time (opts.block_streams), each shifted-CG run on its own
  // stream: the runs share nothing but the links, so while one run's stencil
  // fills the GPU the other's latency-bound seed kernels and grid reductions
  // run beside it.  The stored residuals of all G runs are held at once
  // (basis_max_bytes is split between them).
  const int nblocks = (L + B - 1) / B;
  const int G = std::max(1, std::min(P.o.block_streams, nblocks));
  std::vector<cudaStream_t> streams(G, st);
  std::vector<cudaEvent_t> evj(G, nullptr);
  cudaEvent_t fork = nullptr, c0 = nullptr, c1 = nullptr;
  struct StreamsEvs {
    std::vector<cudaStream_t>* s;
    std::vector<cudaEvent_t>* e;
    cudaEvent_t* f[3];
    ~StreamsEvs() {
      for (size_t i = 1; i < s->size(); ++i)
        if ((*s)[i]) cudaStreamDestroy((*s)[i]);
      for (auto ev : *e)
        if (ev) cudaEventDestroy(ev);
      for (auto* ev : f)
        if (*ev) cudaEventDestroy(*ev);
    }
  } sev{&streams, &evj, {&fork, &c0, &c1}};
  for (int g = 1; g < G; ++g) {
    streams[g] = nullptr;
    SS_CUDA(cudaStreamCreateWithFlags(&streams[g], cudaStreamNonBlocking));
  }
  for (int g = 0; g < G; ++g) SS_CUDA(cudaEventCreateWithFlags(&evj[g], cudaEventDisableTiming));
  SS_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  SS_CUDA(cudaEventCreate(&c0));
  SS_CUDA(cudaEventCreate(&c1));
  for (int b0 = 0; b0 < nblocks; b0 += G) {
    const int gn = std::min(G, nblocks - b0);
    std::vector<std::unique_ptr<CgRunBase>> runs(gn);
    std::vector<DevBuf> ys(gn);
    std::vector<KrylovBasis> kbs(gn);
    SS_CUDA(cudaEventRecord(c0, st));
    SS_CUDA(cudaEventRecord(fork, st));  // the sources are on st
    for (int g = 0; g < gn; ++g) {
      const int l0 = (b0 + g) * B, Lb = std::min(B, L - l0);
      if (streams[g] != st) SS_CUDA(cudaStreamWaitEvent(streams[g], fork, 0));
      const double cap = basis_cap_for(lat->precision, P.o.basis, P.o.basis_max_bytes, n, NU, Lb) / gn;
      SS_TRY(make_cg_run(lat, NU, P.zu.data(), Lb, vd.as<double2>() + (size_t)l0 * n, P.o.sigma, P.o.tol,
                         P.o.max_iter, lat->precision, P.o.reliable_every, cap, streams[g], &runs[g]));
    }
    std::vector<CgRunBase*> rp(gn);
    for (int g = 0; g < gn; ++g) rp[g] = runs[g].get();
    s1 = drive_runs(rp);
    if (s1 != SSQCD_OK && s1 != SSQCD_ERR_BREAKDOWN && s1 != SSQCD_ERR_NOCONV) return s1;
    const double ms_before = cg.ms;
    for (int g = 0; g < gn; ++g) {
      const int l0 = (b0 + g) * B;
      ShiftedCGOut cgb;
      SS_TRY(runs[g]->finish(ys[g], iters.data() + (size_t)l0 * NU, nullptr, &cgb));
      runs[g]->take_basis(&kbs[g]);
      add_cg_stats(cgb, &cg);
      SS_CUDA(cudaEventRecord(evj[g], streams[g]));
      SS_CUDA(cudaStreamWaitEvent(st, evj[g], 0));
    }
    SS_CUDA(cudaEventRecord(c1, st));
    SS_CUDA(cudaEventSynchronize(c1));
    if (gn > 1) {  // the runs overlap: the group's span, not the sum of the runs' times
      float ms = 0.f;
      cudaEventElapsedTime(&ms, c0, c1);
      cg.ms = ms_before + ms;
    }
    fill_cg_stats(cg, iters, &res->stats, P.real_moments);
    if (s1 != SSQCD_OK) return s1;
    runs.clear();
    DevBuf scratch;
    SS_CUDA(cudaEventRecord(m0, st));
    for (int g = 0; g < gn; ++g) {
      const int l0 = (b0 + g) * B, Lb = std::min(B, L - l0);
      for (int k = 0; k < K; ++k) {
        double2* dst = Sk[k].as<double2>() + (size_t)l0 * MM * n;
        if (kbs[g].S > 0)
          SS_TRY(basis_moments(kbs[g], P.coefk[k].data(), MM, dst, scratch, st, nullptr, nullptr, P.real_moments));
        else
          SS_TRY(moments_device(ys[g].as<double2>(), NU, MM, Lb, n, P.coefk[k].data(), dst, scratch, st));
      }
    }
    SS_CUDA(cudaEventRecord(m1, st));
    SS_CUDA(cudaEventSynchronize(m1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, m0, m1);
    ms_mom += ms;
  }
  if (!P.hankel) vd.release();
  s1 = extract_eigenpairs(lat, P, yd, kb, vd, res, st, &Sk);
  res->stats.ms_moments += ms_mom;
  return s1;
}

}  // namespace

extern "C" int ssqcd_ss_solve(ssqcd_lattice lat, const double interval[2], int N, int M, int L,
                              const ssqcd_opts* opts_in, ssqcd_result* out) {
  if (out == nullptr) return fail(SSQCD_ERR_ARG, "NULL result pointer");
  *out = nullptr;
  SS_TRY(check_lattice(lat, true));
  SolvePlan P;
  SS_TRY(plan_solve(interval, N, M, L, opts_in, &P));
  return run_solve(lat, P, out);
}

extern "C" int ssqcd_ss_solve_windows(ssqcd_lattice lat, int K, const double* intervals, int N, int M, int L,
                                      const ssqcd_opts* opts_in, ssqcd_result* out) {
  if (out == nullptr) return fail(SSQCD_ERR_ARG, "NULL result pointer");
  *out = nullptr;
  SS_TRY(check_lattice(lat, true));
  if (opts_in != nullptr && opts_in->windows > 1)
    return fail(SSQCD_ERR_ARG, "ssqcd_ss_solve_windows: opts.windows must be 0 or 1 (the list gives the windows)");
  if (K < 1 || intervals == nullptr) return fail(SSQCD_ERR_ARG, "ssqcd_ss_solve_windows: need K >= 1 intervals");
  for (int k = 0; k < K; ++k)
    if (!(intervals[2 * k + 1] > intervals[2 * k]))
      return fail(SSQCD_ERR_ARG, "ssqcd_ss_solve_windows: every interval needs b > a");
  SolvePlan P;
  SS_TRY(plan_windows(K, intervals, N, M, L, opts_in, &P));
  return run_solve(lat, P, out);
}

extern "C" int ssqcd_ss_moments(ssqcd_lattice lat, const double interval[2], int N, int M, int L,
                                const ssqcd_opts* opts_in, double* s_hat, int s_hat_on_device, ssqcd_stats* stats) {
  SS_TRY(check_lattice(lat, true));
  if (s_hat == nullptr) return fail(SSQCD_ERR_ARG, "NULL s_hat");
  SolvePlan P;
  SS_TRY(plan_solve(interval, N, M, L, opts_in, &P));
  const long long n = 12LL * lat->g.V;
  cudaStream_t st = lat->stream;
  DevBuf vd, yd, S, scratch;
  KrylovBasis kb;
  SS_TRY(to_device_layout(lat, P.o.sources, L, P.o.sources_on_device, vd));
  ShiftedCGOut cg;
  std::vector<int> iters((size_t)P.NU * L);
  SS_TRY(shifted_cg_solve(lat, P.NU, P.zu.data(), L, vd.as<double2>(), P.o.sigma, P.o.tol, P.o.max_iter,
                          lat->precision, P.o.reliable_every,
                          basis_cap_for(lat->precision, P.o.basis, P.o.basis_max_bytes, 12LL * lat->g.V, P.NU, L), yd, &kb,
                        iters.data(), &cg));
  SS_TRY(S.alloc(sizeof(double2) * n * P.MM * L));
  if (kb.S > 0)
    SS_TRY(basis_moments(kb, P.coefk[0].data(), P.MM, S.as<double2>(), scratch, st, nullptr, nullptr,
                         P.real_moments));
  else
    SS_TRY(moments_device(yd.as<double2>(), P.NU, P.MM, L, n, P.coefk[0].data(), S.as<double2>(), scratch, st));
  // the first M of the MM moments of each source
  SS_TRY(vd.alloc(sizeof(double2) * n * M * L));
  for (int l = 0; l < L; ++l)
    SS_CUDA(cudaMemcpyAsync(vd.as<double2>() + (size_t)l * M * n, S.as<double2>() + (size_t)l * P.MM * n,
                            sizeof(double2) * n * M, cudaMemcpyDeviceToDevice, st));
  SS_TRY(from_device_layout(lat, vd.as<double2>(), M * L, s_hat_on_device, s_hat));
  SS_CUDA(cudaStreamSynchronize(st));
  if (stats) {
    *stats = ssqcd_stats{};
    fill_cg_stats(cg, iters, stats, P.real_moments);
  }
  return SSQCD_OK;
}

// --------------------------------------------------------------------------------------------
// Request scheduler: continuous batching of independent solves on one GPU.
//
// A request is one ss_solve.  Submitted requests wait in a FIFO; each call
// of ssqcd_server_progress admits from its head while the estimated device
// memory of the running requests (shift vectors y and p-hat of every
// quadrature point and source dominate) stays within the budget, gives every
// admitted request its own stream, and keeps up to two 16-iteration chunks of
// its shifted CG enqueued there, so the kernels of all running requests
// interleave on the device.  A request whose shifts have all frozen gets its
// moments and Rayleigh-Ritz on its stream and frees its memory; its latency
// runs from submission to that point.  Arithmetic and reduction order of a
// request do not depend on the others: results are the same alone and in
// the mix.  One host thread drives a server.

struct ServerRequest {
  long long id = 0;
  ssqcd_lattice lat = nullptr;
  SolvePlan P;
  std::vector<double> src;  // user layout, copied at submission
  size_t est_bytes = 0;
  int state = SSQCD_REQ_QUEUED;
  int status = SSQCD_OK;
  bool waited_on_memory = false;
  std::string error;
  std::chrono::steady_clock::time_point t_submit, t_done;
  cudaStream_t stream = nullptr;
  DevBuf vd;
  double basis_cap = 0.0;  // bytes its stored residuals may take (in est_bytes)
  std::unique_ptr<CgRunBase> run;
  KrylovBasis basis;
  ssqcd_result_s* res = nullptr;
  // source blocks (opts.source_block): the first source of the running
  // block, the block size, every window's moments [L][MM][n] filled block by
  // block, and the shifted-CG counters so far
  int blk0 = 0, B = 0;
  std::vector<DevBuf> Sk;
  ShiftedCGOut cg_acc;
  std::vector<int> iters;
  float ms_mom = 0.f;

  ~ServerRequest() {
    run.reset();
    basis.release();
    vd.release();
    if (stream) {
      cudaStreamSynchronize(stream);
      cudaStreamDestroy(stream);
    }
    delete res;
  }
};

struct ssqcd_server_s {
  size_t budget = 0;
  size_t running_bytes = 0;
  int running = 0;
  long long deferred = 0;  // requests that waited at the head of the queue for memory
  long long next_id = 1;
  std::deque<long long> queue;
  std::map<long long, std::unique_ptr<ServerRequest>> reqs;
};

namespace {

constexpr int kServerChunksAhead = 2;

// Device memory of one request at its peak: shift vectors (or the stored
// residuals up to their cap), seed vectors and sources during the CG;
// moments and the Rayleigh-Ritz basis afterwards.
size_t estimate_request_bytes(ssqcd_lattice lat, const SolvePlan& P, double basis_cap) {
  const size_t n = 12ull * lat->g.V;
  const int prec = lat->precision;
  const size_t sh = (prec == SSQCD_FP64_SHIFT32 || is_mixed(prec)) ? 8 : 16;
  const size_t sd = is_mixed(prec) ? 8 : 16;
  const size_t NL = (size_t)P.NU * P.L;
  size_t cg = 2 * sh * n * NL + 4 * sd * n * P.L + 16 * n * P.L;
  if (sh == 8) cg += 16 * n * NL;  // FP64 copy of the solutions at the end
  // at the cap the run forms y and p-hat while the residuals are still held
  if (basis_cap > 0.0) cg = std::max(cg, (size_t)basis_cap + 2 * sh * n * NL + 4 * sd * n * P.L + 16 * n * P.L);
  const size_t ex = 16 * n * NL + 4 * 16 * n * (size_t)P.MM * P.L;
  return std::max(cg, ex) + (64u << 20);
}

// Stored-residual cap of a request: the one ss_solve would use (so that the
// result is the same as solved alone); if the request does not fit the
// budget with it, the update form (cap 0) when that fits.
double request_basis_cap(ssqcd_lattice lat, const SolvePlan& P, size_t budget) {
  const double cap = basis_cap_for(lat->precision, P.o.basis, P.o.basis_max_bytes, 12LL * lat->g.V, P.NU, P.L);
  if (cap > 0.0 && estimate_request_bytes(lat, P, cap) > budget) return 0.0;
  return cap;
}

void request_fail(ssqcd_server_s* srv, ServerRequest& r, int status) {
  r.status = status;
  r.error = ssqcd_last_error();
  r.state = SSQCD_REQ_FAILED;
  r.t_done = std::chrono::steady_clock::now();
  if (r.run) {
    r.run.reset();
    srv->running_bytes -= r.est_bytes;
    srv->running -= 1;
  }
  r.basis.release();
  r.vd.release();
}

int request_start(ssqcd_server_s* srv, ServerRequest& r) {
  ssqcd_lattice lat = r.lat;
  SS_CUDA(cudaStreamCreateWithFlags(&r.stream, cudaStreamNonBlocking));
  {
    AllocStream scope(r.stream);
    const int V = lat->g.V, L = r.P.L;
    const size_t bytes = sizeof(double2) * 12 * (size_t)V * L;
    DevBuf stage;
    SS_TRY(stage.alloc(bytes));
    SS_TRY(r.vd.alloc(bytes));
    SS_CUDA(cudaMemcpyAsync(stage.p, r.src.data(), bytes, cudaMemcpyHostToDevice, r.stream));
    SS_TRY(pack_spinors(stage.as<double2>(), r.vd.as<double2>(), L, V, r.stream));
  }
  r.iters.assign((size_t)r.P.NU * r.P.L, 0);
  if (r.B < r.P.L) {
    AllocStream scope(r.stream);
    std::vector<DevBuf> sk(r.P.K);
    r.Sk.swap(sk);
    for (auto& b : r.Sk) SS_TRY(b.alloc(sizeof(double2) * 12 * (size_t)lat->g.V * r.P.MM * r.P.L));
  }
  std::unique_ptr<CgRunBase> run;
  SS_TRY(make_cg_run(lat, r.P.NU, r.P.zu.data(), std::min(r.B, r.P.L), r.vd.as<double2>(), r.P.o.sigma, r.P.o.tol,
                     r.P.o.max_iter, lat->precision, r.P.o.reliable_every, r.basis_cap, r.stream, &run));
  r.run = std::move(run);
  srv->running_bytes += r.est_bytes;
  srv->running += 1;
  r.state = SSQCD_REQ_RUNNING;
  for (int i = 0; i < kServerChunksAhead; ++i) SS_TRY(r.run->launch());
  return SSQCD_OK;
}

// A source block's run has ended: its moments of every window into r.Sk,
// then the next block's run (returns with *more = true) or, after the last
// block, nothing (*more = false; the caller extracts).
int request_next_block(ServerRequest& r, bool* more) {
  ssqcd_lattice lat = r.lat;
  const long long n = 12LL * lat->g.V;
  const int Lb = std::min(r.B, r.P.L - r.blk0);
  DevBuf yd;
  ShiftedCGOut cg;
  SS_TRY(r.run->finish(yd, r.iters.data() + (size_t)r.blk0 * r.P.NU, nullptr, &cg));
  r.run->take_basis(&r.basis);
  r.run.reset();
  add_cg_stats(cg, &r.cg_acc);
  {
    AllocStream scope(r.stream);
    DevBuf scratch;
    cudaEvent_t m0 = nullptr, m1 = nullptr;
    SS_CUDA(cudaEventCreate(&m0));
    SS_CUDA(cudaEventCreate(&m1));
    cudaEventRecord(m0, r.stream);
    int st1 = SSQCD_OK;
    for (int k = 0; k < r.P.K && st1 == SSQCD_OK; ++k) {
      double2* dst = r.Sk[k].as<double2>() + (size_t)r.blk0 * r.P.MM * n;
      st1 = r.basis.S > 0 ? basis_moments(r.basis, r.P.coefk[k].data(), r.P.MM, dst, scratch, r.stream, nullptr,
                                            nullptr, r.P.real_moments)
                          : moments_device(yd.as<double2>(), r.P.NU, r.P.MM, Lb, n, r.P.coefk[k].data(), dst, scratch,
                                           r.stream);
    }
    cudaEventRecord(m1, r.stream);
    cudaEventSynchronize(m1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, m0, m1);
    r.ms_mom += ms;
    cudaEventDestroy(m0);
    cudaEventDestroy(m1);
    SS_TRY(st1);
    yd.release();
    r.basis.release();
  }
  r.blk0 += Lb;
  *more = r.blk0 < r.P.L;
  if (!*more) return SSQCD_OK;
  std::unique_ptr<CgRunBase> run;
  SS_TRY(make_cg_run(lat, r.P.NU, r.P.zu.data(), std::min(r.B, r.P.L - r.blk0), r.vd.as<double2>() + (size_t)r.blk0 * n,
                     r.P.o.sigma, r.P.o.tol, r.P.o.max_iter, lat->precision, r.P.o.reliable_every, r.basis_cap,
                     r.stream, &run));
  r.run = std::move(run);
  for (int i = 0; i < kServerChunksAhead; ++i) SS_TRY(r.run->launch());
  return SSQCD_OK;
}

// A request whose (last) shifted-CG run has ended: moments, extraction,
// memory freed.  With source blocks left, starts the next block instead and
// sets *still_running.
int request_complete(ssqcd_server_s* srv, ServerRequest& r, bool* still_running = nullptr) {
  ssqcd_lattice lat = r.lat;
  if (still_running) *still_running = false;
  if (r.B < r.P.L) {
    bool more = false;
    SS_TRY(request_next_block(r, &more));
    if (more) {
      if (still_running) *still_running = true;
      return SSQCD_OK;
    }
    auto* res = new (std::nothrow) ssqcd_result_s();
    if (!res) return fail(SSQCD_ERR_OOM, "host allocation failed");
    r.res = res;
    res->V = lat->g.V;
    res->n = 12LL * lat->g.V;
    fill_cg_stats(r.cg_acc, r.iters, &res->stats, r.P.real_moments);
    if (!r.P.hankel) r.vd.release();
    DevBuf yd;
    {
      AllocStream scope(r.stream);
      SS_TRY(extract_eigenpairs(lat, r.P, yd, r.basis, r.vd, res, r.stream, &r.Sk));
    }
    res->stats.ms_moments += r.ms_mom;
    r.vd.release();
    r.Sk.clear();
    SS_CUDA(cudaStreamSynchronize(r.stream));
    res->stream = lat->stream;
    srv->running_bytes -= r.est_bytes;
    srv->running -= 1;
    r.state = SSQCD_REQ_DONE;
    r.t_done = std::chrono::steady_clock::now();
    return SSQCD_OK;
  }
  auto* res = new (std::nothrow) ssqcd_result_s();
  if (!res) return fail(SSQCD_ERR_OOM, "host allocation failed");
  r.res = res;
  res->V = lat->g.V;
  res->n = 12LL * lat->g.V;
  DevBuf yd;
  ShiftedCGOut cg;
  std::vector<int> iters((size_t)r.P.NU * r.P.L);
  SS_TRY(r.run->finish(yd, iters.data(), nullptr, &cg));
  r.run->take_basis(&r.basis);
  fill_cg_stats(cg, iters, &res->stats, r.P.real_moments);
  r.run.reset();
  if (!r.P.hankel) r.vd.release();
  {
    AllocStream scope(r.stream);  // no device-wide synchronisation on frees
    SS_TRY(extract_eigenpairs(lat, r.P, yd, r.basis, r.vd, res, r.stream));
  }
  yd.release();
  r.basis.release();
  r.vd.release();
  SS_CUDA(cudaStreamSynchronize(r.stream));
  res->stream = lat->stream;  // later reads of the result run on the lattice stream
  srv->running_bytes -= r.est_bytes;
  srv->running -= 1;
  r.state = SSQCD_REQ_DONE;
  r.t_done = std::chrono::steady_clock::now();
  return SSQCD_OK;
}

}  // namespace

extern "C" int ssqcd_server_create(size_t memory_budget, ssqcd_server* out) {
  if (out == nullptr) return fail(SSQCD_ERR_ARG, "NULL server pointer");
  *out = nullptr;
  if (memory_budget == 0) {
    size_t fr = 0, tot = 0;
    SS_CUDA(cudaMemGetInfo(&fr, &tot));
    memory_budget = fr / 10 * 8;  // 80% of the free device memory
  }
  auto* srv = new (std::nothrow) ssqcd_server_s();
  if (!srv) return fail(SSQCD_ERR_OOM, "host allocation failed");
  srv->budget = memory_budget;
  *out = srv;
  return SSQCD_OK;
}

namespace {

int server_enqueue(ssqcd_server srv, ssqcd_lattice lat, std::unique_ptr<ServerRequest> r, int L, long long* id) {
  r->lat = lat;
  r->B = (r->P.o.source_block > 0 && r->P.o.source_block < L) ? r->P.o.source_block : L;
  // a source block holds the shift vectors / stored residuals of B sources
  // and the moments of all L
  SolvePlan Pb = r->P;
  Pb.L = r->B;
  r->basis_cap = request_basis_cap(lat, Pb, srv->budget);
  r->est_bytes = estimate_request_bytes(lat, Pb, r->basis_cap);
  if (r->B < L) r->est_bytes += sizeof(double2) * 12 * (size_t)lat->g.V * r->P.MM * L * r->P.K;
  if (r->est_bytes > srv->budget)
    return fail(SSQCD_ERR_OOM, "request needs more device memory than the server budget");
  const size_t nd = 2ull * 12 * lat->g.V * L;  // doubles
  r->src.resize(nd);
  if (r->P.o.sources_on_device)
    SS_CUDA(cudaMemcpy(r->src.data(), r->P.o.sources, sizeof(double) * nd, cudaMemcpyDeviceToHost));
  else
    std::memcpy(r->src.data(), r->P.o.sources, sizeof(double) * nd);
  r->P.o.sources = nullptr;
  r->id = srv->next_id++;
  r->t_submit = std::chrono::steady_clock::now();
  *id = r->id;
  srv->queue.push_back(r->id);
  srv->reqs[r->id] = std::move(r);
  return SSQCD_OK;
}

}  // namespace

extern "C" int ssqcd_server_submit(ssqcd_server srv, ssqcd_lattice lat, const double interval[2], int N, int M,
                                   int L, const ssqcd_opts* opts, long long* id) {
  if (srv == nullptr || id == nullptr) return fail(SSQCD_ERR_ARG, "NULL server or id");
  SS_TRY(check_lattice(lat, true));
  auto r = std::make_unique<ServerRequest>();
  SS_TRY(plan_solve(interval, N, M, L, opts, &r->P));
  return server_enqueue(srv, lat, std::move(r), L, id);
}

extern "C" int ssqcd_server_submit_windows(ssqcd_server srv, ssqcd_lattice lat, int K, const double* intervals, int N,
                                           int M, int L, const ssqcd_opts* opts, long long* id) {
  if (srv == nullptr || id == nullptr) return fail(SSQCD_ERR_ARG, "NULL server or id");
  SS_TRY(check_lattice(lat, true));
  if (opts != nullptr && opts->windows > 1)
    return fail(SSQCD_ERR_ARG, "ssqcd_server_submit_windows: opts.windows must be 0 or 1");
  if (K < 1 || intervals == nullptr) return fail(SSQCD_ERR_ARG, "ssqcd_server_submit_windows: need K >= 1 intervals");
  for (int k = 0; k < K; ++k)
    if (!(intervals[2 * k + 1] > intervals[2 * k]))
      return fail(SSQCD_ERR_ARG, "ssqcd_server_submit_windows: every interval needs b > a");
  auto r = std::make_unique<ServerRequest>();
  SS_TRY(plan_windows(K, intervals, N, M, L, opts, &r->P));
  return server_enqueue(srv, lat, std::move(r), L, id);
}

extern "C" int ssqcd_server_progress(ssqcd_server srv, int wait, int* completed) {
  if (srv == nullptr) return fail(SSQCD_ERR_ARG, "NULL server");
  int done = 0;
  // admission from the head of the queue
  while (!srv->queue.empty()) {
    auto it = srv->reqs.find(srv->queue.front());
    if (it == srv->reqs.end()) {
      srv->queue.pop_front();
      continue;
    }
    ServerRequest& r = *it->second;
    if (srv->running > 0 && srv->running_bytes + r.est_bytes > srv->budget) {
      if (!r.waited_on_memory) {
        r.waited_on_memory = true;
        ++srv->deferred;
      }
      break;
    }
    srv->queue.pop_front();
    const int s1 = request_start(srv, r);
    if (s1 != SSQCD_OK) {
      request_fail(srv, r, s1);
      ++done;
    }
  }
  // advance every running request; with wait, block on the first one whose
  // oldest chunk is still on the device if no request moved
  bool moved = false;
  ServerRequest* first_busy = nullptr;
  for (auto& kv : srv->reqs) {
    ServerRequest& r = *kv.second;
    if (r.state != SSQCD_REQ_RUNNING) continue;
    for (;;) {
      int state = 0;
      int s1 = r.run->poll(false, &state);
      if (s1 != SSQCD_OK) {
        request_fail(srv, r, s1);
        ++done;
        moved = true;
        break;
      }
      if (state == CgRunBase::kPollBusy) {
        if (!first_busy) first_busy = &r;
        break;
      }
      moved = true;
      if (state == CgRunBase::kPollDone) {
        bool again = false;
        s1 = request_complete(srv, r, &again);
        if (s1 != SSQCD_OK) {
          request_fail(srv, r, s1);
          ++done;
          break;
        }
        if (again) continue;  // the next source block is running
        ++done;
        break;
      }
      while (r.run->in_flight() < kServerChunksAhead) {
        s1 = r.run->launch();
        if (s1 != SSQCD_OK) break;
      }
      if (s1 != SSQCD_OK) {
        request_fail(srv, r, s1);
        ++done;
        break;
      }
    }
  }
  if (wait && !moved && done == 0 && first_busy != nullptr) {
    int state = 0;
    ServerRequest& r = *first_busy;
    int s1 = r.run->poll(true, &state);
    if (s1 != SSQCD_OK) {
      request_fail(srv, r, s1);
      ++done;
    } else if (state == CgRunBase::kPollDone) {
      bool again = false;
      s1 = request_complete(srv, r, &again);
      if (s1 != SSQCD_OK) {
        request_fail(srv, r, s1);
        ++done;
      } else if (!again) {
        ++done;
      }
    } else {
      while (r.run->in_flight() < kServerChunksAhead)
        if ((s1 = r.run->launch()) != SSQCD_OK) {
          request_fail(srv, r, s1);
          ++done;
          break;
        }
    }
  }
  if (completed) *completed = done;
  return SSQCD_OK;
}

extern "C" int ssqcd_server_deferred(ssqcd_server srv, long long* requests) {
  if (srv == nullptr || requests == nullptr) return fail(SSQCD_ERR_ARG, "NULL server or output");
  *requests = srv->deferred;
  return SSQCD_OK;
}

extern "C" int ssqcd_server_status(ssqcd_server srv, long long id, int* state, double* latency_ms) {
  if (srv == nullptr || state == nullptr) return fail(SSQCD_ERR_ARG, "NULL server or state");
  auto it = srv->reqs.find(id);
  if (it == srv->reqs.end()) return fail(SSQCD_ERR_ARG, "unknown request id");
  const ServerRequest& r = *it->second;
  *state = r.state;
  if (latency_ms) {
    const bool fin = r.state == SSQCD_REQ_DONE || r.state == SSQCD_REQ_FAILED;
    const auto t1 = fin ? r.t_done : std::chrono::steady_clock::now();
    *latency_ms = std::chrono::duration<double, std::milli>(t1 - r.t_submit).count();
  }
  return SSQCD_OK;
}

extern "C" int ssqcd_server_take(ssqcd_server srv, long long id, ssqcd_result* out) {
  if (srv == nullptr || out == nullptr) return fail(SSQCD_ERR_ARG, "NULL server or result pointer");
  *out = nullptr;
  auto it = srv->reqs.find(id);
  if (it == srv->reqs.end()) return fail(SSQCD_ERR_ARG, "unknown request id");
  ServerRequest& r = *it->second;
  if (r.state == SSQCD_REQ_QUEUED || r.state == SSQCD_REQ_RUNNING)
    return fail(SSQCD_ERR_ARG, "request not finished");
  const int status = r.status;
  const std::string err = r.error;
  *out = r.res;
  r.res = nullptr;
  srv->reqs.erase(it);
  if (status != SSQCD_OK) return fail(status, err);
  return SSQCD_OK;
}

extern "C" int ssqcd_server_request_bytes(ssqcd_server srv, long long id, size_t* bytes) {
  if (srv == nullptr || bytes == nullptr) return fail(SSQCD_ERR_ARG, "NULL server or bytes");
  auto it = srv->reqs.find(id);
  if (it == srv->reqs.end()) return fail(SSQCD_ERR_ARG, "unknown request id");
  *bytes = it->second->est_bytes;
  return SSQCD_OK;
}

extern "C" int ssqcd_server_counts(ssqcd_server srv, int* queued, int* running, int* finished) {
  if (srv == nullptr) return fail(SSQCD_ERR_ARG, "NULL server");
  int q = 0, ru = 0, f = 0;
  for (auto& kv : srv->reqs) {
    const int st = kv.second->state;
    q += st == SSQCD_REQ_QUEUED;
    ru += st == SSQCD_REQ_RUNNING;
    f += st == SSQCD_REQ_DONE || st == SSQCD_REQ_FAILED;
  }
  if (queued) *queued = q;
  if (running) *running = ru;
  if (finished) *finished = f;
  return SSQCD_OK;
}

extern "C" void ssqcd_server_destroy(ssqcd_server srv) {
  if (!srv) return;
  delete srv;  // requests finish their device work and free their memory
}

extern "C" int ssqcd_set_stencil_variant(int variant) { return set_fp32_stencil_variant(variant); }

extern "C" int ssqcd_stencil_tuning(ssqcd_lattice lat, int nrhs, int* variant, double* us) {
  SS_TRY(check_lattice(lat, false));
  if (!is_mixed(lat->precision)) return fail(SSQCD_ERR_ARG, "ssqcd_stencil_tuning: the lattice has no FP32 stencil");
  if (variant == nullptr || nrhs < 1) return fail(SSQCD_ERR_ARG, "ssqcd_stencil_tuning: bad arguments");
  float t[8];
  SS_TRY(fp32_stencil_tuning(lat->g.V, nrhs, lat->precision == SSQCD_MIXED ? 16 : 32, variant, t));
  if (us != nullptr)
    for (int v = 0; v < 8; ++v) us[v] = t[v];
  return SSQCD_OK;
}

extern "C" int ssqcd_time_stencil(ssqcd_lattice lat, int nrhs, int reps, double* ms_per_call) {
  SS_TRY(check_lattice(lat, true));
  if (nrhs < 1 || reps < 1 || ms_per_call == nullptr) return fail(SSQCD_ERR_ARG, "bad ssqcd_time_stencil arguments");
  cudaStream_t st = lat->stream;
  const long long n = 12LL * lat->g.V * nrhs;
  const bool mixed = is_mixed(lat->precision), df = lat->precision == SSQCD_DF;
  if (df) SS_TRY(ensure_df_links(lat));
  const size_t elem = mixed ? sizeof(float2) : sizeof(double2);
  DevBuf a, b;
  SS_TRY(a.alloc(elem * n));
  SS_TRY(b.alloc(elem * n));
  SS_CUDA(cudaMemsetAsync(a.p, 0, elem * n, st));
  auto once = [&]() -> int {
    if (mixed) {
      const bool f16 = lat->precision == SSQCD_MIXED;
      return wilson32_kernel_only(lat->g, f16 ? lat->u16.p : lat->u32.p, f16 ? 16 : 32, a.as<float2>(),
                                  b.as<float2>(), nrhs, 0.f, 1.f, st);
    }
    if (df) return wilson_df(lat->g, lat->udf.as<float4>(), a.as<float4>(), b.as<float4>(), nrhs, 0.0, 1.0, st);
    return wilson64(lat->g, lat->u64.as<double2>(), a.as<double2>(), b.as<double2>(), nrhs, 0.0, 1.0, nullptr,
                    nullptr, st);
  };
  for (int i = 0; i < 2; ++i) SS_TRY(once());
  cudaEvent_t e0, e1;
  SS_CUDA(cudaEventCreate(&e0));
  SS_CUDA(cudaEventCreate(&e1));
  cudaEventRecord(e0, st);
  int s1 = SSQCD_OK;
  for (int i = 0; i < reps && s1 == SSQCD_OK; ++i) s1 = once();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SS_TRY(s1);
  *ms_per_call = ms / reps;
  return SSQCD_OK;
}

extern "C" int ssqcd_ss_eigpairs(ssqcd_result res, int* count, double* evals, double* evecs, double* residuals,
                                 ssqcd_stats* stats) {
  if (res == nullptr || count == nullptr) return fail(SSQCD_ERR_ARG, "NULL result or count");
  const int cnt = (int)res->evals.size();
  *count = cnt;
  if (stats) *stats = res->stats;
  if (evals == nullptr) return SSQCD_OK;
  std::memcpy(evals, res->evals.data(), sizeof(double) * cnt);
  if (residuals) std::memcpy(residuals, res->residuals.data(), sizeof(double) * cnt);
  if (evecs && cnt > 0 && res->evecs.p == nullptr)
    return fail(SSQCD_ERR_ARG, "no eigenvectors: the solve used the Hankel extraction");
  if (evecs && cnt > 0) {
    DevBuf stage;
    SS_TRY(stage.alloc(sizeof(double2) * res->n * cnt));
    SS_TRY(unpack_spinors(res->evecs.as<double2>(), stage.as<double2>(), cnt, res->V, res->stream));
    SS_CUDA(cudaMemcpyAsync(evecs, stage.p, sizeof(double2) * res->n * cnt, cudaMemcpyDeviceToHost, res->stream));
    SS_CUDA(cudaStreamSynchronize(res->stream));
  }
  return SSQCD_OK;
}

extern "C" void ssqcd_result_destroy(ssqcd_result res) {
  if (!res) return;
  cudaStreamSynchronize(res->stream);
  delete res;
}
