// Wilson-Dirac stencil: the Hermitian fermion matrix A = gamma5 (I - kappa D)
// of the paper's Section 4, applied matrix-free on the GPU.
//
//   (D psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x + mu)
//                     + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu)
//
// DeGrand-Rossi basis: gamma_mu = [[0, B_mu], [B_mu^H, 0]] in 2x2 spin
// blocks and gamma5 = diag(1, 1, -1, -1).  Because (1 -+ gamma_mu)/2 are rank-2
// projectors, each hop multiplies only a two-spin "half spinor" by the link:
//   forward : h = psi_u - B psi_l,  lower part of (1 - gamma) psi = -B^H h
//   backward: h = psi_u + B psi_l,  lower part of (1 + gamma) psi = +B^H h
// B_mu and B_mu^H are signed permutations with entries in {+-1, +-i}, so the
// projections and reconstructions are additions only.
//
// One thread per (site, right-hand side).  Spinors are [rhs][12][V]
// (component-major, site fastest); neighbours of consecutive sites are
// consecutive, so every component load of a warp is one coalesced segment.
//
// FP64 kernel: on GB300 FP64 runs at 1/64 of the FP32 rate (about 1.2 TFLOP/s
// measured), so this kernel is bound by the FP64 pipe, not by HBM: per site
// and right-hand side it issues 8 x (12 adds projection + 6 x 12 FMA/MUL link
// product + 24 adds reconstruction) + 24 FMA = 888 FP64 instructions against
// 192 B (spinor) + 576 B (links) of compulsory traffic.
//
// FP32 kernel (mixed path): links stored as FP16 first two rows (12 reals);
// the third row is rebuilt as the complex conjugate of the cross product of
// the first two (exact for SU(3)); spinors FP32.  HBM-bound: 96 B spinor in,
// 96 B out, 96 B links per site.
#include "internal.h"

namespace ssqcd {
namespace {

// multiplication of a complex number by one of {+1, -1, +i, -i}
enum : int { P1 = 0, M1 = 1, PI = 2, MI = 3 };

template <typename C>
__device__ __forceinline__ C unit_mul(int code, C z) {
  switch (code) {
    case P1: return z;
    case M1: return C{-z.x, -z.y};
    case PI: return C{-z.y, z.x};
    default: return C{z.y, -z.x};
  }
}

// Spin tables: row r of B_mu has its single nonzero in column bcol_r with
// value bcode_r; likewise for B_mu^H (hcol_r / hcode_r).
template <int MU>
struct Spin {
  static constexpr int bcol0 = (MU == 0 || MU == 1) ? 1 : 0;
  static constexpr int bcol1 = (MU == 0 || MU == 1) ? 0 : 1;
  static constexpr int bcode0 = MU == 0 ? PI : MU == 1 ? M1 : MU == 2 ? PI : P1;
  static constexpr int bcode1 = MU == 0 ? PI : MU == 1 ? P1 : MU == 2 ? MI : P1;
  static constexpr int hcol0 = bcol0;
  static constexpr int hcol1 = bcol1;
  static constexpr int hcode0 = MU == 0 ? MI : MU == 1 ? P1 : MU == 2 ? MI : P1;
  static constexpr int hcode1 = MU == 0 ? MI : MU == 1 ? M1 : MU == 2 ? PI : P1;
};

__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 fadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 fsub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// acc += u * h   (complex)
__device__ __forceinline__ void cmac(double2& acc, double2 u, double2 h) {
  acc.x = fma(u.x, h.x, acc.x);
  acc.x = fma(-u.y, h.y, acc.x);
  acc.y = fma(u.x, h.y, acc.y);
  acc.y = fma(u.y, h.x, acc.y);
}
// acc += conj(u) * h
__device__ __forceinline__ void cmac_conj(double2& acc, double2 u, double2 h) {
  acc.x = fma(u.x, h.x, acc.x);
  acc.x = fma(u.y, h.y, acc.x);
  acc.y = fma(u.x, h.y, acc.y);
  acc.y = fma(-u.y, h.x, acc.y);
}
__device__ __forceinline__ double2 cmul(double2 u, double2 h) {
  return make_double2(fma(u.x, h.x, -u.y * h.y), fma(u.x, h.y, u.y * h.x));
}
__device__ __forceinline__ double2 cmul_conj(double2 u, double2 h) {
  return make_double2(fma(u.x, h.x, u.y * h.y), fma(u.x, h.y, -u.y * h.x));
}

__device__ __forceinline__ void fcmac(float2& acc, float2 u, float2 h) {
  acc.x = fmaf(u.x, h.x, acc.x);
  acc.x = fmaf(-u.y, h.y, acc.x);
  acc.y = fmaf(u.x, h.y, acc.y);
  acc.y = fmaf(u.y, h.x, acc.y);
}
__device__ __forceinline__ void fcmac_conj(float2& acc, float2 u, float2 h) {
  acc.x = fmaf(u.x, h.x, acc.x);
  acc.x = fmaf(u.y, h.y, acc.x);
  acc.y = fmaf(u.x, h.y, acc.y);
  acc.y = fmaf(-u.y, h.x, acc.y);
}

struct Coords {
  int x, y, z, t;
};

__device__ __forceinline__ Coords site_coords(int s, const Geometry& g) {
  Coords c;
  c.x = s % g.X;
  int r = s / g.X;
  c.y = r % g.Y;
  r /= g.Y;
  c.z = r % g.Z;
  c.t = r / g.Z;
  return c;
}

// neighbour site index in direction MU, forward (+1) or backward (-1), and
// whether the hop wraps the t boundary
template <int MU, int DIR>
__device__ __forceinline__ int neighbour(int s, const Coords& c, const Geometry& g, bool& twrap) {
  twrap = false;
  if (MU == 0) {
    if (DIR > 0) return c.x == g.X - 1 ? s - (g.X - 1) : s + 1;
    return c.x == 0 ? s + (g.X - 1) : s - 1;
  } else if (MU == 1) {
    const int st = g.X;
    if (DIR > 0) return c.y == g.Y - 1 ? s - (g.Y - 1) * st : s + st;
    return c.y == 0 ? s + (g.Y - 1) * st : s - st;
  } else if (MU == 2) {
    const int st = g.X * g.Y;
    if (DIR > 0) return c.z == g.Z - 1 ? s - (g.Z - 1) * st : s + st;
    return c.z == 0 ? s + (g.Z - 1) * st : s - st;
  } else {
    const int st = g.X * g.Y * g.Z;
    if (DIR > 0) {
      twrap = c.t == g.T - 1;
      return twrap ? s - (g.T - 1) * st : s + st;
    }
    twrap = c.t == 0;
    return twrap ? s + (g.T - 1) * st : s - st;
  }
}

// ---------------------------------------------------------------- FP64 ----

template <int MU>
__device__ __forceinline__ void hop64(const double2* __restrict__ u, const double2* __restrict__ in,
                                      int s, const Coords& c, const Geometry& g, double2 (&acc)[12]) {
  using S = Spin<MU>;
  const int V = g.V;
  // ---- forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
  {
    bool w;
    const int nb = neighbour<MU, +1>(s, c, g, w);
    double2 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 u0 = __ldg(in + (0 * 3 + a) * V + nb);
      const double2 u1 = __ldg(in + (1 * 3 + a) * V + nb);
      const double2 l0 = __ldg(in + ((2 + S::bcol0) * 3 + a) * V + nb);
      const double2 l1 = __ldg(in + ((2 + S::bcol1) * 3 + a) * V + nb);
      h[0][a] = dsub(u0, unit_mul(S::bcode0, l0));
      h[1][a] = dsub(u1, unit_mul(S::bcode1, l1));
    }
    if (MU == 3 && w && g.bc_t < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h[0][a] = make_double2(-h[0][a].x, -h[0][a].y);
        h[1][a] = make_double2(-h[1][a].x, -h[1][a].y);
      }
    }
    double2 wv[2][3];
    const double2* um = u + (size_t)(MU * 9) * V + s;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 ua0 = __ldg(um + (3 * a + 0) * V);
      const double2 ua1 = __ldg(um + (3 * a + 1) * V);
      const double2 ua2 = __ldg(um + (3 * a + 2) * V);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        double2 t = cmul(ua0, h[r][0]);
        cmac(t, ua1, h[r][1]);
        cmac(t, ua2, h[r][2]);
        wv[r][a] = t;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[0 * 3 + a] = dadd(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = dadd(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = dsub(acc[2 * 3 + a], unit_mul(S::hcode0, wv[S::hcol0][a]));
      acc[3 * 3 + a] = dsub(acc[3 * 3 + a], unit_mul(S::hcode1, wv[S::hcol1][a]));
    }
  }
  // ---- backward: (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu)
  {
    bool w;
    const int nb = neighbour<MU, -1>(s, c, g, w);
    double2 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 u0 = __ldg(in + (0 * 3 + a) * V + nb);
      const double2 u1 = __ldg(in + (1 * 3 + a) * V + nb);
      const double2 l0 = __ldg(in + ((2 + S::bcol0) * 3 + a) * V + nb);
      const double2 l1 = __ldg(in + ((2 + S::bcol1) * 3 + a) * V + nb);
      h[0][a] = dadd(u0, unit_mul(S::bcode0, l0));
      h[1][a] = dadd(u1, unit_mul(S::bcode1, l1));
    }
    if (MU == 3 && w && g.bc_t < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h[0][a] = make_double2(-h[0][a].x, -h[0][a].y);
        h[1][a] = make_double2(-h[1][a].x, -h[1][a].y);
      }
    }
    double2 wv[2][3];
    const double2* um = u + (size_t)(MU * 9) * V + nb;
    // (U^H h)_a = sum_b conj(U_ba) h_b
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 u0a = __ldg(um + (0 * 3 + a) * V);
      const double2 u1a = __ldg(um + (1 * 3 + a) * V);
      const double2 u2a = __ldg(um + (2 * 3 + a) * V);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        double2 t = cmul_conj(u0a, h[r][0]);
        cmac_conj(t, u1a, h[r][1]);
        cmac_conj(t, u2a, h[r][2]);
        wv[r][a] = t;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[0 * 3 + a] = dadd(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = dadd(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = dadd(acc[2 * 3 + a], unit_mul(S::hcode0, wv[S::hcol0][a]));
      acc[3 * 3 + a] = dadd(acc[3 * 3 + a], unit_mul(S::hcode1, wv[S::hcol1][a]));
    }
  }
}

template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < BLOCK / 32; ++i) r += sh[i];
  }
  return r;
}

template <int BLOCK>
__device__ __forceinline__ float block_sumf(float v, float* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  float r = 0.f;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < BLOCK / 32; ++i) r += sh[i];
  }
  return r;
}

constexpr int kWilsonBlock = 128;

__global__ void __launch_bounds__(kWilsonBlock)
wilson64_kernel(Geometry g, const double2* __restrict__ u, const double2* __restrict__ in_all,
                double2* __restrict__ out_all, double c0, double c1, double* __restrict__ dot_partial,
                const int* __restrict__ skip_if_zero) {
  if (skip_if_zero != nullptr && *skip_if_zero == 0) return;
  __shared__ double sh[kWilsonBlock / 32];
  const int rhs = blockIdx.y;
  const int V = g.V;
  const double2* in = in_all + (size_t)rhs * 12 * V;
  double2* out = out_all + (size_t)rhs * 12 * V;
  const int s = blockIdx.x * kWilsonBlock + threadIdx.x;
  double dot = 0.0;
  if (s < V) {
    const Coords c = site_coords(s, g);
    double2 acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = make_double2(0.0, 0.0);
    hop64<0>(u, in, s, c, g, acc);
    hop64<1>(u, in, s, c, g, acc);
    hop64<2>(u, in, s, c, g, acc);
    hop64<3>(u, in, s, c, g, acc);
    // out = c0 psi + c1 gamma5 (psi - kappa D psi)
    const double mk = -g.kappa;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const double2 p = in[i * V + s];
      const double sg = i < 6 ? c1 : -c1;
      double2 m;
      m.x = fma(mk, acc[i].x, p.x);
      m.y = fma(mk, acc[i].y, p.y);
      double2 o;
      o.x = fma(sg, m.x, c0 * p.x);
      o.y = fma(sg, m.y, c0 * p.y);
      out[i * V + s] = o;
      if (dot_partial != nullptr) dot = fma(p.x, o.x, fma(p.y, o.y, dot));
    }
  }
  if (dot_partial != nullptr) {
    const double b = block_sum<kWilsonBlock>(dot, sh);
    if (threadIdx.x == 0) dot_partial[(size_t)rhs * gridDim.x + blockIdx.x] = b;
  }
}

// ---------------------------------------------------------------- FP32 ----
// FP16 12-parameter links: for each mu and site, rows 0 and 1 of U (6 complex)
// as 6 __half2 (re, im), stored [mu][3][V] x uint2 (two __half2 per uint2).

struct Link32 {
  float2 e[3][3];
};

__device__ __forceinline__ float2 h2f(unsigned int v) {
  __half2 h = *reinterpret_cast<__half2*>(&v);
  return __half22float2(h);
}

__device__ __forceinline__ void load_link16(const uint2* __restrict__ u16, int mu, int s, int V, Link32& L) {
  const uint2 q0 = __ldg(u16 + (size_t)(mu * 3 + 0) * V + s);
  const uint2 q1 = __ldg(u16 + (size_t)(mu * 3 + 1) * V + s);
  const uint2 q2 = __ldg(u16 + (size_t)(mu * 3 + 2) * V + s);
  L.e[0][0] = h2f(q0.x);
  L.e[0][1] = h2f(q0.y);
  L.e[0][2] = h2f(q1.x);
  L.e[1][0] = h2f(q1.y);
  L.e[1][1] = h2f(q2.x);
  L.e[1][2] = h2f(q2.y);
  // row 2 = conj(row0 x row1)
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
    const float2 a1 = L.e[0][b1], a2 = L.e[0][b2], c1 = L.e[1][b1], c2 = L.e[1][b2];
    float re = a1.x * c2.x - a1.y * c2.y - (a2.x * c1.x - a2.y * c1.y);
    float im = a1.x * c2.y + a1.y * c2.x - (a2.x * c1.y + a2.y * c1.x);
    L.e[2][b] = make_float2(re, -im);
  }
}

template <int MU>
__device__ __forceinline__ void hop32(const uint2* __restrict__ u16, const float2* __restrict__ in, int s,
                                      const Coords& c, const Geometry& g, float2 (&acc)[12]) {
  using S = Spin<MU>;
  const int V = g.V;
  {
    bool w;
    const int nb = neighbour<MU, +1>(s, c, g, w);
    float2 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float2 u0 = __ldg(in + (0 * 3 + a) * V + nb);
      const float2 u1 = __ldg(in + (1 * 3 + a) * V + nb);
      const float2 l0 = __ldg(in + ((2 + S::bcol0) * 3 + a) * V + nb);
      const float2 l1 = __ldg(in + ((2 + S::bcol1) * 3 + a) * V + nb);
      h[0][a] = fsub(u0, unit_mul(S::bcode0, l0));
      h[1][a] = fsub(u1, unit_mul(S::bcode1, l1));
    }
    if (MU == 3 && w && g.bc_t < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h[0][a] = make_float2(-h[0][a].x, -h[0][a].y);
        h[1][a] = make_float2(-h[1][a].x, -h[1][a].y);
      }
    }
    Link32 L;
    load_link16(u16, MU, s, V, L);
    float2 wv[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float2 t = make_float2(0.f, 0.f);
        fcmac(t, L.e[a][0], h[r][0]);
        fcmac(t, L.e[a][1], h[r][1]);
        fcmac(t, L.e[a][2], h[r][2]);
        wv[r][a] = t;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[0 * 3 + a] = fadd(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = fadd(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = fsub(acc[2 * 3 + a], unit_mul(S::hcode0, wv[S::hcol0][a]));
      acc[3 * 3 + a] = fsub(acc[3 * 3 + a], unit_mul(S::hcode1, wv[S::hcol1][a]));
    }
  }
  {
    bool w;
    const int nb = neighbour<MU, -1>(s, c, g, w);
    float2 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float2 u0 = __ldg(in + (0 * 3 + a) * V + nb);
      const float2 u1 = __ldg(in + (1 * 3 + a) * V + nb);
      const float2 l0 = __ldg(in + ((2 + S::bcol0) * 3 + a) * V + nb);
      const float2 l1 = __ldg(in + ((2 + S::bcol1) * 3 + a) * V + nb);
      h[0][a] = fadd(u0, unit_mul(S::bcode0, l0));
      h[1][a] = fadd(u1, unit_mul(S::bcode1, l1));
    }
    if (MU == 3 && w && g.bc_t < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h[0][a] = make_float2(-h[0][a].x, -h[0][a].y);
        h[1][a] = make_float2(-h[1][a].x, -h[1][a].y);
      }
    }
    Link32 L;
    load_link16(u16, MU, nb, V, L);
    float2 wv[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float2 t = make_float2(0.f, 0.f);
        fcmac_conj(t, L.e[0][a], h[r][0]);
        fcmac_conj(t, L.e[1][a], h[r][1]);
        fcmac_conj(t, L.e[2][a], h[r][2]);
        wv[r][a] = t;
      }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[0 * 3 + a] = fadd(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = fadd(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = fadd(acc[2 * 3 + a], unit_mul(S::hcode0, wv[S::hcol0][a]));
      acc[3 * 3 + a] = fadd(acc[3 * 3 + a], unit_mul(S::hcode1, wv[S::hcol1][a]));
    }
  }
}

__global__ void __launch_bounds__(kWilsonBlock)
wilson32_kernel(Geometry g, const uint2* __restrict__ u16, const float2* __restrict__ in_all,
                float2* __restrict__ out_all, float c0, float c1, float* __restrict__ dot_partial,
                const int* __restrict__ skip_if_zero) {
  if (skip_if_zero != nullptr && *skip_if_zero == 0) return;
  __shared__ float sh[kWilsonBlock / 32];
  const int rhs = blockIdx.y;
  const int V = g.V;
  const float2* in = in_all + (size_t)rhs * 12 * V;
  float2* out = out_all + (size_t)rhs * 12 * V;
  const int s = blockIdx.x * kWilsonBlock + threadIdx.x;
  float dot = 0.f;
  if (s < V) {
    const Coords c = site_coords(s, g);
    float2 acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = make_float2(0.f, 0.f);
    hop32<0>(u16, in, s, c, g, acc);
    hop32<1>(u16, in, s, c, g, acc);
    hop32<2>(u16, in, s, c, g, acc);
    hop32<3>(u16, in, s, c, g, acc);
    const float mk = -(float)g.kappa;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const float2 p = in[i * V + s];
      const float sg = i < 6 ? c1 : -c1;
      float2 m;
      m.x = fmaf(mk, acc[i].x, p.x);
      m.y = fmaf(mk, acc[i].y, p.y);
      float2 o;
      o.x = fmaf(sg, m.x, c0 * p.x);
      o.y = fmaf(sg, m.y, c0 * p.y);
      out[i * V + s] = o;
      if (dot_partial != nullptr) dot = fmaf(p.x, o.x, fmaf(p.y, o.y, dot));
    }
  }
  if (dot_partial != nullptr) {
    const float b = block_sumf<kWilsonBlock>(dot, sh);
    if (threadIdx.x == 0) dot_partial[(size_t)rhs * gridDim.x + blockIdx.x] = b;
  }
}

// FP64 links [4][9][V] -> FP16 rows 0,1 [4][3][V] uint2
__global__ void pack_gauge16_kernel(const double2* __restrict__ u, uint2* __restrict__ u16, int V) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 4LL * V) return;
  const int mu = (int)(i / V), s = (int)(i % V);
  unsigned int h[6];
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const double2 z = u[(size_t)(mu * 9 + e) * V + s];
    __half2 hv = __halves2half2(__double2half(z.x), __double2half(z.y));  // rounded once
    h[e] = *reinterpret_cast<unsigned int*>(&hv);
  }
  u16[(size_t)(mu * 3 + 0) * V + s] = make_uint2(h[0], h[1]);
  u16[(size_t)(mu * 3 + 1) * V + s] = make_uint2(h[2], h[3]);
  u16[(size_t)(mu * 3 + 2) * V + s] = make_uint2(h[4], h[5]);
}

}  // namespace

int wilson_blocks(const Geometry& g) { return (g.V + kWilsonBlock - 1) / kWilsonBlock; }

int wilson64(const Geometry& g, const double2* u, const double2* in, double2* out, int nrhs, double c0,
             double c1, double* dot_partial, const int* skip_if_zero, cudaStream_t s) {
  if (nrhs <= 0) return SSQCD_OK;
  dim3 grid(wilson_blocks(g), nrhs);
  wilson64_kernel<<<grid, kWilsonBlock, 0, s>>>(g, u, in, out, c0, c1, dot_partial, skip_if_zero);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int wilson32(const Geometry& g, const void* u16, const float2* in, float2* out, int nrhs, float c0,
             float c1, float* dot_partial, const int* skip_if_zero, cudaStream_t s) {
  if (nrhs <= 0) return SSQCD_OK;
  dim3 grid(wilson_blocks(g), nrhs);
  wilson32_kernel<<<grid, kWilsonBlock, 0, s>>>(g, static_cast<const uint2*>(u16), in, out, c0, c1,
                                                dot_partial, skip_if_zero);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int pack_gauge16(const double2* u64dev, void* u16, int V, cudaStream_t s) {
  pack_gauge16_kernel<<<grid_for(4LL * V, 256), 256, 0, s>>>(u64dev, static_cast<uint2*>(u16), V);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

}  // namespace ssqcd
