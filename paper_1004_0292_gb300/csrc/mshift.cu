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
// One iteration = three kernels, each finishing its reduction in its last
// block (fixed summation order, no host round trip):
//   A. stencil q = K p for every source with block partials of (p, q); the
//      last block forms alpha_k = (r, r) / (p, q) (breakdown check);
//   B. seed update r -= alpha q with partials of ||r||^2; the last block
//      forms (r_{k+1}, r_{k+1}) and beta_k;
//   C. fused update: every block recomputes the xi recurrence of its
//      source's shifts (a few dozen FP64 operations per shift, spread over all
//      SMs instead of serialised in one), then for every live shift
//      y_j += a_j p-hat_j, p-hat_j = r + b_j p-hat_j, and p = r + beta p.
// (A two-kernel form that obtains ||r_{k+1}||^2 from (r, r) - 2 alpha (r, q)
// + alpha^2 (q, q) was tried and rejected: on the indefinite seed the
// residual can drop by many orders in one step, the three terms cancel, and
// shifts froze on a wrong residual estimate.)
// Block 0 of each source also stores xi_{k+1}, the freeze flags and the
// per-shift iteration counts.  xi lives in a ring of three slots indexed by
// k mod 3, the other state in two slots indexed by the parity P = k mod 2, so
// readers and the single writer of an iteration never touch the same slot.
// Kernel A of iteration k skips when no shift was live after iteration k-1;
// the host polls the live count every 16 iterations.  All reductions have a
// fixed order, so runs are bit-reproducible.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "wilson_core.cuh"

namespace ssqcd {
namespace {

using namespace wcore;

struct SeedIter {
  double alpha;  // alpha_k
  double beta;   // beta_k
  double rr;     // (r_{k+1}, r_{k+1})
  double pad;
};

// Device-side control block of one solve (L sources, N shifts).
struct Control {
  SeedIter* seed;      // [2][L]   slot k&1 written by kernel A of iteration k
  double* vnorm2;      // [L]
  int* src_live;       // [2][L]   live shifts at the start of iteration k: slot k&1
  int* live_total;     // [2]
  int* ran;            // [2]      kernel A of iteration k did its work
  int* err;            // [1]
  int* seed_iters;     // [1]
  unsigned* done;      // [2]      last-block tickets of kernels A and B
  double2* shift_s;    // [L*N]    s_j = z_j - sigma
  double2* xi;         // [3][L*N] ring: slot k%3 = xi_k
  int* act;            // [2][L*N] active at the start of iteration k: slot k&1
  int* iters;          // [L*N]
  double* partial;     // [L][nbw]  (p, q) partials of kernel A
  double* partial_rr;  // [L][nbu]  ||r||^2 partials of kernel B
};

constexpr int kUpdBlock = 256;
constexpr int kMaxShifts = 256;
constexpr int kMaxSources = 64;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- initialisation ---------------------------------------------------------------
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

// A source with ||v|| = 0 has the exact solution y = 0 and starts frozen.
__global__ void init_control_kernel(Control c, const double* __restrict__ vn2, int L, int N) {
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    c.seed[L + t] = SeedIter{1.0, 0.0, vn2[t], 0.0};  // "iteration -1": alpha_{-1} = 1, beta_{-1} = 0, rr_0
    c.seed[t] = SeedIter{0.0, 0.0, 0.0, 0.0};
    c.vnorm2[t] = vn2[t];
    c.src_live[t] = vn2[t] > 0.0 ? N : 0;
    c.src_live[L + t] = 0;
  }
  for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
    c.xi[t] = make_double2(1.0, 0.0);              // xi_0
    c.xi[2 * L * N + t] = make_double2(1.0, 0.0);  // xi_{-1} (slot 2 = -1 mod 3)
    c.act[t] = vn2[t / N] > 0.0 ? 1 : 0;
    c.act[L * N + t] = 0;
    c.iters[t] = 0;
  }
  if (threadIdx.x == 0) {
    int live = 0;
    for (int l = 0; l < L; ++l) live += vn2[l] > 0.0 ? N : 0;
    c.live_total[0] = live;
    c.live_total[1] = 0;
    c.ran[0] = c.ran[1] = 0;
    *c.err = 0;
    *c.seed_iters = 0;
    c.done[0] = c.done[1] = 0u;
  }
}

// ---- A. stencil q = K p + (p, q) partials; last block: alpha_k ---------------------
__global__ void __launch_bounds__(kStencilThreads)
cg_stencil_kernel(Control c, int P, int L, Geometry g, const double2* __restrict__ u, double sigma,
                  const double2* __restrict__ p_all, double2* __restrict__ q_all) {
  if (*c.err != 0 || c.live_total[P] == 0) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
      c.ran[P] = 0;
      c.live_total[1 - P] = 0;
      for (int l = 0; l < L; ++l) c.src_live[(1 - P) * L + l] = 0;
    }
    return;
  }
  __shared__ double2 sh[12 * 4 * 32];
  __shared__ double sred[kStencilThreads / 32];
  __shared__ double sums[kMaxSources];
  __shared__ bool s_last;
  const int l = blockIdx.y;
  const int V = g.V;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double d_pq = 0.0;
  if (c.src_live[P * L + l] != 0) {
    const double2* p = p_all + (size_t)l * 12 * V;
    double2* q = q_all + (size_t)l * 12 * V;
    const int s = blockIdx.x * kSitesPerBlock + lane;
    double2 acc[3];
    block_hops64(Links64{u, V}, p, s, g, sh, acc);
    if (s < V) {
      // q = sigma p - gamma5 (p - kappa D p); components 3w..3w+2 are spin w
      const double sg = w < 2 ? -1.0 : 1.0;
      const double mk = -g.kappa;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int i = 3 * w + k;
        const double2 pv = p[i * V + s];
        double2 o;
        o.x = fma(sg, fma(mk, acc[k].x, pv.x), sigma * pv.x);
        o.y = fma(sg, fma(mk, acc[k].y, pv.y), sigma * pv.y);
        q[i * V + s] = o;
        d_pq = fma(pv.x, o.x, fma(pv.y, o.y, d_pq));
      }
    }
  }
  d_pq = warp_sum(d_pq);
  if (lane == 0) sred[w] = d_pq;
  __syncthreads();
  const int nbw = gridDim.x;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kStencilThreads / 32; ++i) t += sred[i];
    c.partial[(size_t)l * nbw + blockIdx.x] = t;
    __threadfence();
    const unsigned ticket = atomicAdd(&c.done[0], 1u);
    s_last = ticket == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // warp w sums the partials of sources w, w+4, ... in a fixed order
  for (int ls = w; ls < L; ls += kStencilThreads / 32) {
    double a = 0.0;
    for (int b = lane; b < nbw; b += 32) a += __ldcg(c.partial + (size_t)ls * nbw + b);
    a = warp_sum(a);
    if (lane == 0) sums[ls] = a;
  }
  __syncthreads();
  for (int ls = threadIdx.x; ls < L; ls += blockDim.x) {
    if (c.src_live[P * L + ls] == 0) {
      c.seed[P * L + ls] = SeedIter{0.0, 0.0, 0.0, 0.0};
      continue;
    }
    const double pq = sums[ls];
    const double rr = c.seed[(1 - P) * L + ls].rr;
    if (!(fabs(pq) >= 1e-30 * rr)) {  // breakdown (also catches NaN)
      atomicExch(c.err, 1);
      continue;
    }
    c.seed[P * L + ls] = SeedIter{rr / pq, 0.0, 0.0, 0.0};
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = *((volatile int*)c.err) == 0;
    c.ran[P] = ok ? 1 : 0;
    c.live_total[1 - P] = 0;
    if (ok) atomicAdd(c.seed_iters, 1);
    c.done[0] = 0u;
  }
  for (int ls = threadIdx.x; ls < L; ls += blockDim.x) c.src_live[(1 - P) * L + ls] = 0;
}

// ---- B. seed update r -= alpha q, ||r||^2 partials; last block: rr_{k+1}, beta_k -----
__global__ void __launch_bounds__(kUpdBlock)
cg_seed_kernel(Control c, int P, int L, double2* __restrict__ r, const double2* __restrict__ q, long long n) {
  if (c.ran[P] == 0) return;
  __shared__ double sred[kUpdBlock / 32];
  __shared__ double sums[kMaxSources];
  __shared__ bool s_last;
  const int l = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double acc = 0.0;
  if (c.src_live[P * L + l] != 0) {
    const double alpha = c.seed[P * L + l].alpha;
    double2* rl = r + (long long)l * n;
    const double2* ql = q + (long long)l * n;
    for (long long e = blockIdx.x * (long long)kUpdBlock + threadIdx.x; e < n;
         e += (long long)gridDim.x * kUpdBlock) {
      double2 x = rl[e];
      const double2 y = ql[e];
      x.x = fma(-alpha, y.x, x.x);
      x.y = fma(-alpha, y.y, x.y);
      rl[e] = x;
      acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) sred[w] = acc;
  __syncthreads();
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kUpdBlock / 32; ++i) t += sred[i];
    c.partial_rr[(size_t)l * nb + blockIdx.x] = t;
    __threadfence();
    const unsigned ticket = atomicAdd(&c.done[1], 1u);
    s_last = ticket == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int ls = w; ls < L; ls += kUpdBlock / 32) {
    double a = 0.0;
    for (int b = lane; b < nb; b += 32) a += __ldcg(c.partial_rr + (size_t)ls * nb + b);
    a = warp_sum(a);
    if (lane == 0) sums[ls] = a;
  }
  __syncthreads();
  for (int ls = threadIdx.x; ls < L; ls += blockDim.x) {
    if (c.src_live[P * L + ls] == 0) continue;
    SeedIter sd = c.seed[P * L + ls];
    const double rr = c.seed[(1 - P) * L + ls].rr;
    sd.rr = sums[ls];
    sd.beta = sums[ls] / rr;
    c.seed[P * L + ls] = sd;
  }
  if (threadIdx.x == 0) c.done[1] = 0u;
}

// ---- C. fused update ------------------------------------------------------------------
__global__ void __launch_bounds__(kUpdBlock)
cg_update_kernel(Control c, int k, int L, int N, double tol2, const double2* __restrict__ r,
                 double2* __restrict__ p, double2* __restrict__ y, double2* __restrict__ ph, long long n) {
  const int P = k & 1;
  const int l = blockIdx.y;
  if (c.ran[P] == 0 || c.src_live[P * L + l] == 0) return;
  __shared__ int s_j[kMaxShifts];
  __shared__ double2 s_a[kMaxShifts];
  __shared__ double2 s_b[kMaxShifts];
  __shared__ int s_flag[kMaxShifts];  // 1: update this iteration; 2: and stays live
  __shared__ int s_n, s_live;
  const SeedIter cur = c.seed[P * L + l];
  const SeedIter prev = c.seed[(1 - P) * L + l];
  const int slot_k = k % 3, slot_km1 = (k + 2) % 3, slot_kp1 = (k + 1) % 3;
  const int NL = N * L;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    const int qi = l * N + j;
    int flag = 0;
    if (c.act[P * NL + qi]) {
      const double2 xc = c.xi[slot_k * NL + qi], xp = c.xi[slot_km1 * NL + qi], s = c.shift_s[qi];
      const double alpha = cur.alpha, ap = prev.alpha, bp = prev.beta;
      // xi_{k+1} = xi_k xi_{k-1} alpha_{k-1} /
      //            [alpha_k beta_{k-1} (xi_{k-1} - xi_k) + xi_{k-1} alpha_{k-1} (1 + s alpha_k)]
      double2 num;
      num.x = (xc.x * xp.x - xc.y * xp.y) * ap;
      num.y = (xc.x * xp.y + xc.y * xp.x) * ap;
      const double ab = alpha * bp;
      const double ux = 1.0 + s.x * alpha, uy = s.y * alpha;
      double2 den;
      den.x = ab * (xp.x - xc.x) + (xp.x * ux - xp.y * uy) * ap;
      den.y = ab * (xp.y - xc.y) + (xp.x * uy + xp.y * ux) * ap;
      const double inv_d = 1.0 / (den.x * den.x + den.y * den.y);
      double2 xn;
      xn.x = (num.x * den.x + num.y * den.y) * inv_d;
      xn.y = (num.y * den.x - num.x * den.y) * inv_d;
      // b = beta xi_{k+1} / xi_k = beta xi_{k+1} conj(xi_k) / |xi_k|^2
      const double bc = cur.beta / (xc.x * xc.x + xc.y * xc.y);
      s_a[j] = make_double2(alpha * xn.x, alpha * xn.y);
      s_b[j] = make_double2(bc * (xn.x * xc.x + xn.y * xc.y), bc * (xn.y * xc.x - xn.x * xc.y));
      const bool live = (xn.x * xn.x + xn.y * xn.y) * cur.rr > tol2 * c.vnorm2[l];
      flag = live ? 2 : 1;
      if (blockIdx.x == 0) {
        c.xi[slot_kp1 * NL + qi] = xn;
        c.act[(1 - P) * NL + qi] = live ? 1 : 0;
        c.iters[qi] += 1;
      }
    } else if (blockIdx.x == 0) {
      c.act[(1 - P) * NL + qi] = 0;
    }
    s_flag[j] = flag;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int m = 0, live = 0;
    for (int j = 0; j < N; ++j) {
      if (s_flag[j]) {
        s_j[m] = j;
        s_a[m] = s_a[j];  // m <= j: in-place compaction keeps the order
        s_b[m] = s_b[j];
        ++m;
      }
      live += s_flag[j] == 2;
    }
    s_n = m;
    s_live = live;
    if (blockIdx.x == 0) {
      c.src_live[(1 - P) * L + l] = live;
      atomicAdd(&c.live_total[1 - P], live);
    }
  }
  __syncthreads();
  const int m = s_n;
  const bool seed_continues = s_live > 0;
  const double alpha = cur.alpha, beta = cur.beta;
  (void)alpha;
  const double2* rl = r + (long long)l * n;
  double2* pl = p + (long long)l * n;
  for (long long e = blockIdx.x * (long long)kUpdBlock + threadIdx.x; e < n; e += (long long)gridDim.x * kUpdBlock) {
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
    if (seed_continues) {
      double2 pv = pl[e];
      pv.x = fma(beta, pv.x, re.x);
      pv.y = fma(beta, pv.y, re.y);
      pl[e] = pv;
    }
  }
}

int update_blocks(long long n, int L) {
  long long b = (n + kUpdBlock - 1) / kUpdBlock;
  const long long cap = (152LL * 8 + L - 1) / L;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

int shifted_cg_device(ssqcd_lattice lat, int N, const double2* z_host, int L, const double2* v, double sigma,
                      double tol, int max_iter, int precision, int reliable_every, DevBuf& y, int* iters_host,
                      double2* xi_host, ShiftedCGOut* out) {
  (void)reliable_every;
  if (precision != SSQCD_FP64) return fail(SSQCD_ERR_ARG, "shifted_cg_device: only SSQCD_FP64 here");
  if (N < 1 || N > kMaxShifts) return fail(SSQCD_ERR_ARG, "N must be in [1, 256]");
  if (L < 1 || L > kMaxSources) return fail(SSQCD_ERR_ARG, "L must be in [1, 64]");
  cudaStream_t st = lat->stream;
  const Geometry& g = lat->g;
  const long long n = 12LL * g.V;
  const int NL = N * L;
  const int nbw = wilson_blocks(g);
  const int nbu = update_blocks(n, L);

  DevBuf r, p, q, ph;
  SS_TRY(r.alloc(sizeof(double2) * n * L));
  SS_TRY(p.alloc(sizeof(double2) * n * L));
  SS_TRY(q.alloc(sizeof(double2) * n * L));
  SS_TRY(y.alloc(sizeof(double2) * n * NL));
  SS_TRY(ph.alloc(sizeof(double2) * n * NL));
  DevBuf ctl;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) / 256 * 256;
    return o;
  };
  const size_t o_seed = take(sizeof(SeedIter) * 2 * L), o_vn = take(sizeof(double) * L),
               o_live = take(sizeof(int) * 2 * L), o_tot = take(sizeof(int) * 2), o_ran = take(sizeof(int) * 2),
               o_err = take(sizeof(int)), o_si = take(sizeof(int)), o_done = take(sizeof(unsigned) * 2),
               o_s = take(sizeof(double2) * NL), o_xi = take(sizeof(double2) * 3 * NL),
               o_act = take(sizeof(int) * 2 * NL), o_it = take(sizeof(int) * NL),
               o_part = take(sizeof(double) * (size_t)nbw * L), o_prr = take(sizeof(double) * (size_t)nbu * L),
               o_vp = take(sizeof(double) * (size_t)nbu * L),
               o_vn2 = take(sizeof(double) * L);
  SS_TRY(ctl.alloc(off));
  char* base = ctl.as<char>();
  Control c;
  c.seed = reinterpret_cast<SeedIter*>(base + o_seed);
  c.vnorm2 = reinterpret_cast<double*>(base + o_vn);
  c.src_live = reinterpret_cast<int*>(base + o_live);
  c.live_total = reinterpret_cast<int*>(base + o_tot);
  c.ran = reinterpret_cast<int*>(base + o_ran);
  c.err = reinterpret_cast<int*>(base + o_err);
  c.seed_iters = reinterpret_cast<int*>(base + o_si);
  c.done = reinterpret_cast<unsigned*>(base + o_done);
  c.shift_s = reinterpret_cast<double2*>(base + o_s);
  c.xi = reinterpret_cast<double2*>(base + o_xi);
  c.act = reinterpret_cast<int*>(base + o_act);
  c.iters = reinterpret_cast<int*>(base + o_it);
  c.partial = reinterpret_cast<double*>(base + o_part);
  c.partial_rr = reinterpret_cast<double*>(base + o_prr);
  double* vn_part = reinterpret_cast<double*>(base + o_vp);
  double* vn2 = reinterpret_cast<double*>(base + o_vn2);

  std::vector<double2> sh(NL);
  for (int l = 0; l < L; ++l)
    for (int j = 0; j < N; ++j) sh[l * N + j] = make_double2(z_host[j].x - sigma, z_host[j].y);
  SS_CUDA(cudaMemcpyAsync(c.shift_s, sh.data(), sizeof(double2) * NL, cudaMemcpyHostToDevice, st));

  SS_TRY(norm2_partials(v, L, n, vn_part, nbu, st));
  SS_TRY(sum_partials(vn_part, L, nbu, vn2, st));
  init_vectors_kernel<<<dim3(nbu, L), kUpdBlock, 0, st>>>(v, r.as<double2>(), p.as<double2>(), y.as<double2>(),
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
  constexpr int kChunk = 16;
  const bool timing = kernel_timing_enabled();
  std::vector<cudaEvent_t> tev;
  std::vector<double> t_iter[3];
  if (timing) {
    tev.resize(kChunk * 6);
    for (auto& e : tev) SS_CUDA(cudaEventCreate(&e));
  }
  auto mark = [&](int it, int slot) {
    if (timing) cudaEventRecord(tev[it * 6 + slot], st);
  };
  const dim3 grid_a(nbw, L), grid_b(nbu, L);
  while (true) {
    const int chunk = std::min(kChunk, max_iter - k);
    int launched = 0;
    for (int it = 0; it < chunk; ++it, ++k) {
      const int P = k & 1;
      mark(it, 0);
      cg_stencil_kernel<<<grid_a, kStencilThreads, 0, st>>>(c, P, L, g, lat->u64.as<double2>(), sigma,
                                                             p.as<double2>(), q.as<double2>());
      mark(it, 1);
      mark(it, 2);
      cg_seed_kernel<<<grid_b, kUpdBlock, 0, st>>>(c, P, L, r.as<double2>(), q.as<double2>(), n);
      mark(it, 3);
      mark(it, 4);
      cg_update_kernel<<<grid_b, kUpdBlock, 0, st>>>(c, k, L, N, tol2, r.as<double2>(), p.as<double2>(),
                                                     y.as<double2>(), ph.as<double2>(), n);
      mark(it, 5);
      count_launches(3);
      ++launched;
      cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) { status = cuda_fail(le, "shifted CG launch", __FILE__, __LINE__); break; }
    }
    if (status != SSQCD_OK) break;
    // live-shift count at the start of the next iteration, and the error flag
    cudaError_t ce = cudaMemcpyAsync(h_poll, c.live_total + (k & 1), sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_poll + 1, c.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) { status = cuda_fail(ce, "shifted CG poll", __FILE__, __LINE__); break; }
    if (timing) {
      for (int it = 0; it < launched; ++it)
        for (int cls = 0; cls < 3; ++cls) {
          float ms = 0.f;
          cudaEventElapsedTime(&ms, tev[it * 6 + 2 * cls], tev[it * 6 + 2 * cls + 1]);
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
    std::vector<double2> xi_all(3 * (size_t)NL);
    SS_CUDA(cudaMemcpyAsync(&seed_iters, c.seed_iters, sizeof(int), cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaMemcpyAsync(it_all.data(), c.iters, sizeof(int) * NL, cudaMemcpyDeviceToHost, st));
    if (xi_host) SS_CUDA(cudaMemcpyAsync(xi_all.data(), c.xi, sizeof(double2) * 3 * NL, cudaMemcpyDeviceToHost, st));
    SS_CUDA(cudaStreamSynchronize(st));
    if (iters_host) std::copy(it_all.begin(), it_all.end(), iters_host);
    if (xi_host)  // a shift's last xi sits in slot (its iteration count) mod 3
      for (int qi = 0; qi < NL; ++qi) xi_host[qi] = xi_all[(size_t)(it_all[qi] % 3) * NL + qi];
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (out) {
      out->seed_iters = seed_iters;
      out->ms = ms;
      out->shift_updates = 0;
      for (int v2 : it_all) out->shift_updates += v2;
      out->timed = timing;
      out->launches_update = timing ? std::min<int>(seed_iters, (int)t_iter[2].size()) : 0;
      for (int cls = 0; cls < 4; ++cls) out->ms_k[cls] = 0.0;
      const int slot_of[3] = {0, 1, 3};  // stencil, seed update, shift update
      for (int cls = 0; cls < 3; ++cls) {
        double acc = 0.0;
        // iterations after the last live one skip their work: not counted
        for (int i = 0; i < (int)t_iter[cls].size() && i < seed_iters; ++i) acc += t_iter[cls][i];
        out->ms_k[slot_of[cls]] = acc;
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
