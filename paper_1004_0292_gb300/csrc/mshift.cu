// Shifted CG (Section 2.2 of the paper): all quadrature-point systems
// (z_j I - A) y_j = v from one CG recurrence on the Hermitian seed matrix
// K = sigma I - A (sigma real), per source v_l.
//
// With s_j = z_j - sigma, z_j I - A = K + s_j I and the shifted residuals stay
// collinear with the seed residual, r^j_k = xi^j_k r_k (Eq. 5 and the text
// after it).  The recurrences (standard multi-shift CG):
//
//   alpha_k = (r_k, r_k) / (p_k, K p_k),  r_{k+1} = r_k - alpha_k K p_k,
//   beta_k = (r_{k+1}, r_{k+1}) / (r_k, r_k),  p_{k+1} = r_{k+1} + beta_k p_k,
//   xi_{k+1} = xi_k xi_{k-1} alpha_{k-1} /
//              [alpha_k beta_{k-1} (xi_{k-1} - xi_k) + xi_{k-1} alpha_{k-1} (1 + s alpha_k)],
//   y += alpha_k (xi_{k+1}/xi_k) p^j,  p^j = xi_{k+1} r_{k+1} + (xi_{k+1}/xi_k)^2 beta_k p^j.
//
// The device keeps p-hat_j = p^j / xi^j_k instead of p^j, which turns the
// per-shift vector work into two complex AXPYs (8 FP64 FMA per element):
//   y_j += a_j p-hat_j,  p-hat_j = r_{k+1} + b_j p-hat_j,
//   a_j = alpha_k xi_{k+1},  b_j = beta_k xi_{k+1} / xi_k.
// A shift stops ("freezes") once |xi_{k+1}| ||r_{k+1}|| <= tol ||v|| (the
// paper's stopping rule ||r_j|| / ||v|| <= tol, Section 3 and Section 4).
//
// One iteration = four kernels, all issued asynchronously; the host only
// polls a counter every few iterations:
//   1. stencil q = K p with per-block partials of (p, q)            (wilson.cu)
//   2. seed update: alpha, r -= alpha q, partials of ||r||^2
//   3. shift scalars: one thread per (source, shift) -> xi, a_j, b_j, freeze
//   4. fused multi-shift update: y_j, p-hat_j for every live shift, seed p
// Iteration control without host round trips: counters of live shifts are
// double-buffered by iteration parity P.  Kernels of iteration k skip their
// work when cnt[1-P] (the count left by iteration k-1) is zero; kernel 3
// accumulates cnt[P]; kernel 4 clears cnt[1-P] for iteration k+1 (every reader
// of cnt[1-P] in iteration k ran before it).  Seed scalars (rr, alpha,
// beta) are double-buffered the same way; per-shift state is owned by a
// single thread of kernel 3 and needs no buffering.
//
// The reductions are fixed-order, so every run gives bit-identical results.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "internal.h"

namespace ssqcd {
namespace {

struct SeedScalars {
  double rr;          // (r_k, r_k)
  double alpha_prev;  // alpha_{k-1}
  double beta_prev;   // beta_{k-1}
  double pad;
};

struct ShiftCoef {
  double2 a;  // y += a * p-hat
  double2 b;  // p-hat = r + b * p-hat
};

// Device-side control block of one solve (all sized for L sources, N shifts).
struct Control {
  SeedScalars* seed;   // [2][L]
  double* alpha_cur;   // [L]
  double* vnorm2;      // [L]
  int* cnt;            // [2]
  int* cnt_src;        // [2][L]
  int* err;            // [1]
  int* seed_iters;     // [1]
  double2* shift_s;    // [L*N]  s_j = z_j - sigma
  double2* xi_cur;     // [L*N]
  double2* xi_prev;    // [L*N]
  int* active;         // [L*N]
  int* upd;            // [L*N]
  int* iters;          // [L*N]
  ShiftCoef* coef;     // [L*N]
};

constexpr int kBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of partial[0..nb) with a fixed order; result valid in every thread.
__device__ double block_sum_fixed(const double* __restrict__ partial, int nb, double* sh) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
  acc = warp_sum(acc);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = acc;
  __syncthreads();
  double r = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) r += sh[i];
  return r;
}

__device__ double block_reduce(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  const int nw = blockDim.x >> 5;
  for (int i = 0; i < nw; ++i) r += sh[i];
  return r;
}

// ---- initialisation: r = p = v, p-hat_j = v, y_j = 0 ------------------------
__global__ void init_vectors_kernel(const double2* __restrict__ v, double2* __restrict__ r, double2* __restrict__ p,
                                    double2* __restrict__ y, double2* __restrict__ ph, int N, long long n) {
  const int l = blockIdx.y;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double2 x = v[l * n + e];
    r[l * n + e] = x;
    p[l * n + e] = x;
    for (int j = 0; j < N; ++j) {
      y[((long long)l * N + j) * n + e] = make_double2(0.0, 0.0);
      ph[((long long)l * N + j) * n + e] = x;
    }
  }
}

// One block: seed scalars, per-shift state and the live counts.  A source with
// ||v|| = 0 has the exact solution y = 0 and starts frozen.
__global__ void init_control_kernel(Control c, const double* __restrict__ vn2, int L, int N) {
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    c.seed[t] = SeedScalars{vn2[t], 1.0, 0.0, 0.0};
    c.seed[L + t] = SeedScalars{0.0, 0.0, 0.0, 0.0};
    c.vnorm2[t] = vn2[t];
    c.alpha_cur[t] = 0.0;
    c.cnt_src[t] = 0;                          // parity 0
    c.cnt_src[L + t] = vn2[t] > 0.0 ? N : 0;   // parity 1 = "previous iteration"
  }
  for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
    c.xi_cur[t] = make_double2(1.0, 0.0);
    c.xi_prev[t] = make_double2(1.0, 0.0);
    c.active[t] = vn2[t / N] > 0.0 ? 1 : 0;
    c.upd[t] = 0;
    c.iters[t] = 0;
  }
  if (threadIdx.x == 0) {
    int live = 0;
    for (int l = 0; l < L; ++l) live += vn2[l] > 0.0 ? N : 0;
    c.cnt[0] = 0;
    c.cnt[1] = live;
    *c.err = 0;
    *c.seed_iters = 0;
  }
}

// ---- 2. seed update -----------------------------------------------------------
// grid (nb, L).  alpha_l = rr_l / pq_l (pq from the stencil partials), r -= alpha q,
// partials of ||r||^2 into rr_part[l * nb + block].
__global__ void __launch_bounds__(kBlock)
seed_update_kernel(Control c, int P, double2* __restrict__ r, const double2* __restrict__ q,
                   const double* __restrict__ pq_part, int nbw, double* __restrict__ rr_part, long long n) {
  const int l = blockIdx.y;
  const int L = gridDim.y;
  if (c.cnt[1 - P] == 0 || c.cnt_src[(1 - P) * L + l] == 0) return;
  __shared__ double sh[kBlock / 32];
  const double pq = block_sum_fixed(pq_part + (long long)l * nbw, nbw, sh);
  const double rr = c.seed[P * L + l].rr;
  double alpha = rr / pq;
  if (!(fabs(pq) >= 1e-30 * rr)) {  // breakdown (also catches NaN)
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(c.err, 1);
    alpha = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) c.alpha_cur[l] = alpha;
  double acc = 0.0;
  double2* rl = r + (long long)l * n;
  const double2* ql = q + (long long)l * n;
  for (long long e = blockIdx.x * (long long)kBlock + threadIdx.x; e < n; e += (long long)gridDim.x * kBlock) {
    double2 x = rl[e];
    const double2 y = ql[e];
    x.x = fma(-alpha, y.x, x.x);
    x.y = fma(-alpha, y.y, x.y);
    rl[e] = x;
    acc = fma(x.x, x.x, fma(x.y, x.y, acc));
  }
  const double b = block_reduce(acc, sh);
  if (threadIdx.x == 0) rr_part[(long long)l * gridDim.x + blockIdx.x] = b;
}

// ---- 3. shift scalars -----------------------------------------------------------
// one thread per (l, j), 32 per block.
__global__ void __launch_bounds__(32)
shift_scalars_kernel(Control c, int P, int L, int N, const double* __restrict__ rr_part, int nbr, double tol2) {
  const int q = blockIdx.x * 32 + threadIdx.x;
  const bool valid = q < L * N;
  const int l = valid ? q / N : L - 1;
  const bool run = c.cnt[1 - P] != 0 && *c.err == 0;
  // rr_{k+1} for every source present in this warp (warp-cooperative, fixed order)
  double rr_new = 0.0;
  const int l_first = (blockIdx.x * 32) / N;
  const int l_last = min(L - 1, (blockIdx.x * 32 + 31) / N);
  if (run) {
    for (int ls = l_first; ls <= l_last; ++ls) {
      double acc = 0.0;
      for (int i = threadIdx.x; i < nbr; i += 32) acc += rr_part[(long long)ls * nbr + i];
      acc = warp_sum(acc);
      if (ls == l) rr_new = acc;
    }
  }
  if (!valid) return;
  if (!run || c.cnt_src[(1 - P) * L + l] == 0) {
    c.upd[q] = 0;
    return;
  }
  const SeedScalars sd = c.seed[P * L + l];
  const double alpha = c.alpha_cur[l];
  const double beta = rr_new / sd.rr;
  const int j = q - l * N;
  if (j == 0) c.seed[(1 - P) * L + l] = SeedScalars{rr_new, alpha, beta, 0.0};
  if (q == 0) atomicAdd(c.seed_iters, 1);  // an iteration in which some source was live
  int live = 0;
  if (c.active[q]) {
    const double2 xc = c.xi_cur[q], xp = c.xi_prev[q], s = c.shift_s[q];
    const double ap = sd.alpha_prev, bp = sd.beta_prev;
    // numerator xi_k xi_{k-1} alpha_{k-1}
    double2 num;
    num.x = (xc.x * xp.x - xc.y * xp.y) * ap;
    num.y = (xc.x * xp.y + xc.y * xp.x) * ap;
    // alpha_k beta_{k-1} (xi_{k-1} - xi_k) + xi_{k-1} alpha_{k-1} (1 + s alpha_k)
    const double ab = alpha * bp;
    const double2 t1 = make_double2(ab * (xp.x - xc.x), ab * (xp.y - xc.y));
    const double2 u = make_double2(1.0 + s.x * alpha, s.y * alpha);
    double2 t2;
    t2.x = (xp.x * u.x - xp.y * u.y) * ap;
    t2.y = (xp.x * u.y + xp.y * u.x) * ap;
    const double2 den = make_double2(t1.x + t2.x, t1.y + t2.y);
    const double dd = den.x * den.x + den.y * den.y;
    double2 xn;
    xn.x = (num.x * den.x + num.y * den.y) / dd;
    xn.y = (num.y * den.x - num.x * den.y) / dd;
    // b = beta xi_{k+1} / xi_k
    const double cc = xc.x * xc.x + xc.y * xc.y;
    double2 ratio;
    ratio.x = (xn.x * xc.x + xn.y * xc.y) / cc;
    ratio.y = (xn.y * xc.x - xn.x * xc.y) / cc;
    ShiftCoef cf;
    cf.a = make_double2(alpha * xn.x, alpha * xn.y);
    cf.b = make_double2(beta * ratio.x, beta * ratio.y);
    c.coef[q] = cf;
    c.upd[q] = 1;
    c.xi_prev[q] = xc;
    c.xi_cur[q] = xn;
    c.iters[q] += 1;
    const double xn2 = xn.x * xn.x + xn.y * xn.y;
    if (xn2 * rr_new <= tol2 * c.vnorm2[l]) {
      c.active[q] = 0;
    } else {
      live = 1;
    }
  } else {
    c.upd[q] = 0;
  }
  // count live shifts, per source and in total
  if (live) {
    atomicAdd(&c.cnt[P], 1);
    atomicAdd(&c.cnt_src[P * L + l], 1);
  }
}

// ---- 4. fused multi-shift update --------------------------------------------------
// grid (nb, L).  Per element: r once; for every shift of source l marked in upd:
// y += a p-hat; p-hat = r + b p-hat; then p = r + beta p while the source lives.
constexpr int kMaxShifts = 128;

__global__ void __launch_bounds__(kBlock)
shift_update_kernel(Control c, int P, int L, int N, const double2* __restrict__ r, double2* __restrict__ p,
                    double2* __restrict__ y, double2* __restrict__ ph, long long n) {
  const int l = blockIdx.y;
  if (blockIdx.x == 0 && l == 0 && threadIdx.x == 0) {
    c.cnt[1 - P] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) c.cnt_src[(1 - P) * L + l] = 0;
  __shared__ int s_j[kMaxShifts];
  __shared__ double2 s_a[kMaxShifts];
  __shared__ double2 s_b[kMaxShifts];
  __shared__ int s_n;
  if (threadIdx.x == 0) {
    int m = 0;
    for (int j = 0; j < N; ++j) {
      const int q = l * N + j;
      if (c.upd[q]) {
        s_j[m] = j;
        s_a[m] = c.coef[q].a;
        s_b[m] = c.coef[q].b;
        ++m;
      }
    }
    s_n = m;
  }
  __syncthreads();
  const int m = s_n;
  const bool seed_live = c.cnt_src[P * L + l] != 0;
  if (m == 0 && !seed_live) return;
  const double beta = c.seed[(1 - P) * L + l].beta_prev;
  const double2* rl = r + (long long)l * n;
  double2* pl = p + (long long)l * n;
  for (long long e = blockIdx.x * (long long)kBlock + threadIdx.x; e < n; e += (long long)gridDim.x * kBlock) {
    const double2 re = rl[e];
    int t = 0;
    for (; t + 2 <= m; t += 2) {
      double2* y0 = y + ((long long)l * N + s_j[t]) * n + e;
      double2* p0 = ph + ((long long)l * N + s_j[t]) * n + e;
      double2* y1 = y + ((long long)l * N + s_j[t + 1]) * n + e;
      double2* p1 = ph + ((long long)l * N + s_j[t + 1]) * n + e;
      double2 yv0 = *y0, pv0 = *p0, yv1 = *y1, pv1 = *p1;
      const double2 a0 = s_a[t], b0 = s_b[t], a1 = s_a[t + 1], b1 = s_b[t + 1];
      yv0.x = fma(a0.x, pv0.x, fma(-a0.y, pv0.y, yv0.x));
      yv0.y = fma(a0.x, pv0.y, fma(a0.y, pv0.x, yv0.y));
      yv1.x = fma(a1.x, pv1.x, fma(-a1.y, pv1.y, yv1.x));
      yv1.y = fma(a1.x, pv1.y, fma(a1.y, pv1.x, yv1.y));
      double2 n0, n1;
      n0.x = fma(b0.x, pv0.x, fma(-b0.y, pv0.y, re.x));
      n0.y = fma(b0.x, pv0.y, fma(b0.y, pv0.x, re.y));
      n1.x = fma(b1.x, pv1.x, fma(-b1.y, pv1.y, re.x));
      n1.y = fma(b1.x, pv1.y, fma(b1.y, pv1.x, re.y));
      *y0 = yv0;
      *p0 = n0;
      *y1 = yv1;
      *p1 = n1;
    }
    if (t < m) {
      double2* y0 = y + ((long long)l * N + s_j[t]) * n + e;
      double2* p0 = ph + ((long long)l * N + s_j[t]) * n + e;
      double2 yv0 = *y0, pv0 = *p0;
      const double2 a0 = s_a[t], b0 = s_b[t];
      yv0.x = fma(a0.x, pv0.x, fma(-a0.y, pv0.y, yv0.x));
      yv0.y = fma(a0.x, pv0.y, fma(a0.y, pv0.x, yv0.y));
      double2 n0;
      n0.x = fma(b0.x, pv0.x, fma(-b0.y, pv0.y, re.x));
      n0.y = fma(b0.x, pv0.y, fma(b0.y, pv0.x, re.y));
      *y0 = yv0;
      *p0 = n0;
    }
    if (seed_live) {
      double2 pv = pl[e];
      pv.x = fma(beta, pv.x, re.x);
      pv.y = fma(beta, pv.y, re.y);
      pl[e] = pv;
    }
  }
}

int update_blocks(long long n) {
  long long b = (n + kBlock - 1) / kBlock;
  if (b > 152 * 8) b = 152 * 8;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

int shifted_cg_device(ssqcd_lattice lat, int N, const double2* z_host, int L, const double2* v, double sigma,
                      double tol, int max_iter, int precision, int reliable_every, DevBuf& y, int* iters_host,
                      double2* xi_host, ShiftedCGOut* out) {
  (void)reliable_every;
  if (precision != SSQCD_FP64) return fail(SSQCD_ERR_ARG, "shifted_cg_device: only SSQCD_FP64 here");
  if (N < 1 || N > kMaxShifts) return fail(SSQCD_ERR_ARG, "N must be in [1, 128]");
  if (L < 1) return fail(SSQCD_ERR_ARG, "L must be >= 1");
  cudaStream_t st = lat->stream;
  const Geometry& g = lat->g;
  const long long n = 12LL * g.V;
  const int NL = N * L;
  const int nbw = wilson_blocks(g);
  const int nbu = update_blocks(n);

  // vectors
  DevBuf r, p, q, ph;
  SS_TRY(r.alloc(sizeof(double2) * n * L));
  SS_TRY(p.alloc(sizeof(double2) * n * L));
  SS_TRY(q.alloc(sizeof(double2) * n * L));
  SS_TRY(y.alloc(sizeof(double2) * n * NL));
  SS_TRY(ph.alloc(sizeof(double2) * n * NL));
  // control block + partials in one allocation
  DevBuf ctl;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t o_seed = take(sizeof(SeedScalars) * 2 * L), o_alpha = take(sizeof(double) * L),
               o_vn = take(sizeof(double) * L), o_cnt = take(sizeof(int) * 2), o_cnts = take(sizeof(int) * 2 * L),
               o_err = take(sizeof(int)), o_si = take(sizeof(int)), o_s = take(sizeof(double2) * NL),
               o_xc = take(sizeof(double2) * NL), o_xp = take(sizeof(double2) * NL), o_act = take(sizeof(int) * NL),
               o_upd = take(sizeof(int) * NL), o_it = take(sizeof(int) * NL), o_coef = take(sizeof(ShiftCoef) * NL),
               o_pq = take(sizeof(double) * (size_t)nbw * L), o_rr = take(sizeof(double) * (size_t)nbu * L),
               o_vp = take(sizeof(double) * (size_t)nbu * L), o_vn2 = take(sizeof(double) * L);
  SS_TRY(ctl.alloc(off));
  char* base = ctl.as<char>();
  Control c;
  c.seed = reinterpret_cast<SeedScalars*>(base + o_seed);
  c.alpha_cur = reinterpret_cast<double*>(base + o_alpha);
  c.vnorm2 = reinterpret_cast<double*>(base + o_vn);
  c.cnt = reinterpret_cast<int*>(base + o_cnt);
  c.cnt_src = reinterpret_cast<int*>(base + o_cnts);
  c.err = reinterpret_cast<int*>(base + o_err);
  c.seed_iters = reinterpret_cast<int*>(base + o_si);
  c.shift_s = reinterpret_cast<double2*>(base + o_s);
  c.xi_cur = reinterpret_cast<double2*>(base + o_xc);
  c.xi_prev = reinterpret_cast<double2*>(base + o_xp);
  c.active = reinterpret_cast<int*>(base + o_act);
  c.upd = reinterpret_cast<int*>(base + o_upd);
  c.iters = reinterpret_cast<int*>(base + o_it);
  c.coef = reinterpret_cast<ShiftCoef*>(base + o_coef);
  double* pq_part = reinterpret_cast<double*>(base + o_pq);
  double* rr_part = reinterpret_cast<double*>(base + o_rr);
  double* vn_part = reinterpret_cast<double*>(base + o_vp);
  double* vn2 = reinterpret_cast<double*>(base + o_vn2);

  // shifts s_j = z_j - sigma, repeated per source
  std::vector<double2> sh(NL);
  for (int l = 0; l < L; ++l)
    for (int j = 0; j < N; ++j) sh[l * N + j] = make_double2(z_host[j].x - sigma, z_host[j].y);
  SS_CUDA(cudaMemcpyAsync(c.shift_s, sh.data(), sizeof(double2) * NL, cudaMemcpyHostToDevice, st));

  SS_TRY(norm2_partials(v, L, n, vn_part, nbu, st));
  SS_TRY(sum_partials(vn_part, L, nbu, vn2, st));
  init_vectors_kernel<<<dim3(nbu, L), kBlock, 0, st>>>(v, r.as<double2>(), p.as<double2>(), y.as<double2>(),
                                                         ph.as<double2>(), N, n);
  SS_CHECK_LAUNCH();
  init_control_kernel<<<1, 256, 0, st>>>(c, vn2, L, N);
  SS_CHECK_LAUNCH();
  count_launches(2);

  cudaEvent_t e0, e1;
  SS_CUDA(cudaEventCreate(&e0));
  SS_CUDA(cudaEventCreate(&e1));
  SS_CUDA(cudaEventRecord(e0, st));

  int* h_poll = nullptr;
  SS_CUDA(cudaMallocHost(&h_poll, sizeof(int) * 4));
  const double tol2 = tol * tol;
  int status = SSQCD_OK;
  int k = 0;
  const int nbs = (NL + 31) / 32;
  // optional per-kernel timing: events around the four kernels of every
  // iteration of a chunk, read back at the chunk's poll
  constexpr int kChunk = 16;
  const bool timing = kernel_timing_enabled();
  std::vector<cudaEvent_t> tev;
  std::vector<double> t_iter[4];
  if (timing) {
    tev.resize(kChunk * 8);
    for (auto& e : tev) SS_CUDA(cudaEventCreate(&e));
  }
  auto mark = [&](int it, int slot) {
    if (timing) cudaEventRecord(tev[it * 8 + slot], st);
  };
  while (true) {
    const int chunk = std::min(kChunk, max_iter - k);  // iterations between polls
    int done_in_chunk = 0;
    for (int it = 0; it < chunk; ++it, ++k) {
      const int P = k & 1;
      mark(it, 0);
      int s1 = wilson64(g, lat->u64.as<double2>(), p.as<double2>(), q.as<double2>(), L, sigma, -1.0, pq_part,
                        c.cnt + (1 - P), st);
      if (s1 != SSQCD_OK) { status = s1; break; }
      mark(it, 1);
      mark(it, 2);
      seed_update_kernel<<<dim3(nbu, L), kBlock, 0, st>>>(c, P, r.as<double2>(), q.as<double2>(), pq_part, nbw,
                                                          rr_part, n);
      mark(it, 3);
      mark(it, 4);
      shift_scalars_kernel<<<nbs, 32, 0, st>>>(c, P, L, N, rr_part, nbu, tol2);
      mark(it, 5);
      mark(it, 6);
      shift_update_kernel<<<dim3(nbu, L), kBlock, 0, st>>>(c, P, L, N, r.as<double2>(), p.as<double2>(),
                                                           y.as<double2>(), ph.as<double2>(), n);
      mark(it, 7);
      count_launches(3);
      ++done_in_chunk;
      cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) { status = cuda_fail(le, "shifted CG launch", __FILE__, __LINE__); break; }
    }
    if (status != SSQCD_OK) break;
    // live-shift count left by the last iteration (parity (k-1) & 1)
    cudaError_t ce = cudaMemcpyAsync(h_poll, c.cnt + ((k - 1) & 1), sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_poll + 1, c.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { status = cuda_fail(ce, "shifted CG poll", __FILE__, __LINE__); break; }
    if (timing) {
      for (int it = 0; it < done_in_chunk; ++it)
        for (int cls = 0; cls < 4; ++cls) {
          float ms = 0.f;
          cudaEventElapsedTime(&ms, tev[it * 8 + 2 * cls], tev[it * 8 + 2 * cls + 1]);
          t_iter[cls].push_back(ms);
        }
    }
    if (h_poll[1] != 0) { status = fail(SSQCD_ERR_BREAKDOWN, "seed CG breakdown: |(p, K p)| < 1e-30 (r, r)"); break; }
    if (h_poll[0] == 0) break;
    if (k >= max_iter) {
      char buf[128];
      std::snprintf(buf, sizeof(buf), "shifted CG: %d shifts still above tol after %d iterations", h_poll[0], k);
      status = fail(SSQCD_ERR_NOCONV, buf);
      break;
    }
  }
  if (status == SSQCD_OK || status == SSQCD_ERR_BREAKDOWN || status == SSQCD_ERR_NOCONV) {
    SS_CUDA(cudaEventRecord(e1, st));
    int seed_iters = 0;
    std::vector<int> it_all(NL);
    SS_CUDA(cudaMemcpyAsync(&seed_iters, c.seed_iters, sizeof(int), cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaMemcpyAsync(it_all.data(), c.iters, sizeof(int) * NL, cudaMemcpyDeviceToHost, st));
    if (xi_host) SS_CUDA(cudaMemcpyAsync(xi_host, c.xi_cur, sizeof(double2) * NL, cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaStreamSynchronize(st));
    if (iters_host) std::copy(it_all.begin(), it_all.end(), iters_host);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (out) {
      out->seed_iters = seed_iters;
      out->ms = ms;
      out->shift_updates = 0;
      for (int v2 : it_all) out->shift_updates += v2;
      out->timed = timing;
      out->launches_update = timing ? std::min<int>(seed_iters, (int)t_iter[3].size()) : 0;
      for (int cls = 0; cls < 4; ++cls) {
        double acc = 0.0;
        // iterations after the last live one only skip their work: not counted
        for (int i = 0; i < (int)t_iter[cls].size() && i < seed_iters; ++i) acc += t_iter[cls][i];
        out->ms_k[cls] = acc;
      }
    }
  }
  for (auto& e : tev) cudaEventDestroy(e);
  cudaFreeHost(h_poll);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return status;
}

}  // namespace ssqcd
