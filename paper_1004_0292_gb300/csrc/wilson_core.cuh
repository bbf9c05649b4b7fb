// Device building blocks of the Wilson-Dirac stencil (A = gamma5 (I - kappa D),
// Section 4 of the paper), shared by the stand-alone operator kernels
// (wilson.cu) and the fused shifted-CG kernels (mshift.cu).
//
//   (D psi)(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x + mu)
//                     + (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu)
//
// DeGrand-Rossi basis: gamma_mu = [[0, B_mu], [B_mu^H, 0]] in 2x2 spin blocks,
// gamma5 = diag(1, 1, -1, -1).  (1 -+ gamma_mu)/2 are rank-2 projectors, so a
// hop multiplies only a two-spin half spinor by the link:
//   forward : h = psi_u - B psi_l, lower part of (1 - gamma) psi = -B^H h,
//   backward: h = psi_u + B psi_l, lower part of (1 + gamma) psi = +B^H h.
// B_mu, B_mu^H are signed permutations with entries in {+-1, +-i}: the
// projection and reconstruction are additions only.
//
// Work split: a block covers 32 consecutive sites of one right-hand side;
// warp w (0..3) applies the forward and backward hop in direction mu = w for
// those 32 sites, so every warp is branch-uniform and every component load
// of a warp is one coalesced segment (neighbours of consecutive sites are
// consecutive except at wraps).  The four partial sums meet in shared
// memory; warp w then finishes spinor components 3w..3w+2 of the 32 sites.
// Spinor layout [rhs][12][V] (component-major, site fastest).
#pragma once

#include "internal.h"
#include "pair32.cuh"

namespace ssqcd {
namespace wcore {

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

// Row r of B_mu has its single nonzero in column bcol_r with value bcode_r;
// likewise for B_mu^H (hcol_r / hcode_r).
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

template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C>
__device__ __forceinline__ C cneg(C a) { return C{-a.x, -a.y}; }

// acc += u h,  acc += conj(u) h
template <typename C>
__device__ __forceinline__ void cmac(C& acc, C u, C h) {
  acc.x = fma(u.x, h.x, acc.x);
  acc.x = fma(-u.y, h.y, acc.x);
  acc.y = fma(u.x, h.y, acc.y);
  acc.y = fma(u.y, h.x, acc.y);
}
template <typename C>
__device__ __forceinline__ void cmac_conj(C& acc, C u, C h) {
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
__device__ __forceinline__ float2 cmul(float2 u, float2 h) {
  return make_float2(fmaf(u.x, h.x, -u.y * h.y), fmaf(u.x, h.y, u.y * h.x));
}
__device__ __forceinline__ float2 cmul_conj(float2 u, float2 h) {
  return make_float2(fmaf(u.x, h.x, u.y * h.y), fmaf(u.x, h.y, -u.y * h.x));
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

// neighbour in direction MU, forward (DIR > 0) or backward; wraps
// periodically, twrap tells whether the hop crossed the t boundary
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

// ---- link access ----------------------------------------------------------------
// FP64: [4][9][V] double2, row-major 3x3.
struct Links64 {
  const double2* __restrict__ u;
  int V;
  __device__ __forceinline__ double2 get(int mu, int a, int b, int s) const {
    return __ldg(u + (size_t)(mu * 9 + 3 * a + b) * V + s);
  }
};

// Reduced-precision links keep rows 0 and 1 (12 reals); row 2 is rebuilt as
// conj(row0 x row1), exact for SU(3).
__device__ __forceinline__ float2 h2f(unsigned int v) {
  __half2 h = *reinterpret_cast<__half2*>(&v);
  return __half22float2(h);
}

struct Link32 {
  float2 e[3][3];
};

// row 2 of an SU(3) matrix = complex conjugate of (row 0 x row 1)
__device__ __forceinline__ void reconstruct_row2(Link32& L) {
#pragma unroll
  for (int b = 0; b < 3; ++b) {
    const int b1 = (b + 1) % 3, b2 = (b + 2) % 3;
    const float2 a1 = L.e[0][b1], a2 = L.e[0][b2], c1 = L.e[1][b1], c2 = L.e[1][b2];
    const float re = a1.x * c2.x - a1.y * c2.y - (a2.x * c1.x - a2.y * c1.y);
    const float im = a1.x * c2.y + a1.y * c2.x - (a2.x * c1.y + a2.y * c1.x);
    L.e[2][b] = make_float2(re, -im);
  }
}

// FP16 12-parameter links: rows 0 and 1 as six __half2 in [4][3][V] uint2
struct LinksF16 {
  const uint2* __restrict__ u;
  int V;
  __device__ __forceinline__ void load(int mu, int s, Link32& L) const {
    const uint2 q0 = __ldg(u + (size_t)(mu * 3 + 0) * V + s);
    const uint2 q1 = __ldg(u + (size_t)(mu * 3 + 1) * V + s);
    const uint2 q2 = __ldg(u + (size_t)(mu * 3 + 2) * V + s);
    L.e[0][0] = h2f(q0.x);
    L.e[0][1] = h2f(q0.y);
    L.e[0][2] = h2f(q1.x);
    L.e[1][0] = h2f(q1.y);
    L.e[1][1] = h2f(q2.x);
    L.e[1][2] = h2f(q2.y);
    reconstruct_row2(L);
  }
};

// FP32 12-parameter links: rows 0 and 1 as six float2 in [4][3][V] float4
struct LinksF32 {
  const float4* __restrict__ u;
  int V;
  __device__ __forceinline__ void load(int mu, int s, Link32& L) const {
    const float4 q0 = __ldg(u + (size_t)(mu * 3 + 0) * V + s);
    const float4 q1 = __ldg(u + (size_t)(mu * 3 + 1) * V + s);
    const float4 q2 = __ldg(u + (size_t)(mu * 3 + 2) * V + s);
    L.e[0][0] = make_float2(q0.x, q0.y);
    L.e[0][1] = make_float2(q0.z, q0.w);
    L.e[0][2] = make_float2(q1.x, q1.y);
    L.e[1][0] = make_float2(q1.z, q1.w);
    L.e[1][1] = make_float2(q2.x, q2.y);
    L.e[1][2] = make_float2(q2.z, q2.w);
    reconstruct_row2(L);
  }
};

// ---- one direction: forward + backward hop, accumulated into acc[12] --------------
template <int MU>
__device__ __forceinline__ void hop_dir64(const Links64& lk, const double2* __restrict__ in, int s, const Coords& c,
                                          const Geometry& g, double2 (&acc)[12]) {
  using S = Spin<MU>;
  const int V = g.V;
  {  // forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
    bool w;
    const int nb = neighbour<MU, +1>(s, c, g, w);
    double2 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 u0 = __ldg(in + (0 * 3 + a) * V + nb);
      const double2 u1 = __ldg(in + (1 * 3 + a) * V + nb);
      const double2 l0 = __ldg(in + ((2 + S::bcol0) * 3 + a) * V + nb);
      const double2 l1 = __ldg(in + ((2 + S::bcol1) * 3 + a) * V + nb);
      h[0][a] = csub(u0, unit_mul(S::bcode0, l0));
      h[1][a] = csub(u1, unit_mul(S::bcode1, l1));
    }
    if (MU == 3 && w && g.bc_t < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h[0][a] = cneg(h[0][a]);
        h[1][a] = cneg(h[1][a]);
      }
    }
    double2 wv[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 ua0 = lk.get(MU, a, 0, s), ua1 = lk.get(MU, a, 1, s), ua2 = lk.get(MU, a, 2, s);
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
      acc[0 * 3 + a] = cadd(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = cadd(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = csub(acc[2 * 3 + a], unit_mul(S::hcode0, wv[S::hcol0][a]));
      acc[3 * 3 + a] = csub(acc[3 * 3 + a], unit_mul(S::hcode1, wv[S::hcol1][a]));
    }
  }
  {  // backward: (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu)
    bool w;
    const int nb = neighbour<MU, -1>(s, c, g, w);
    double2 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 u0 = __ldg(in + (0 * 3 + a) * V + nb);
      const double2 u1 = __ldg(in + (1 * 3 + a) * V + nb);
      const double2 l0 = __ldg(in + ((2 + S::bcol0) * 3 + a) * V + nb);
      const double2 l1 = __ldg(in + ((2 + S::bcol1) * 3 + a) * V + nb);
      h[0][a] = cadd(u0, unit_mul(S::bcode0, l0));
      h[1][a] = cadd(u1, unit_mul(S::bcode1, l1));
    }
    if (MU == 3 && w && g.bc_t < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h[0][a] = cneg(h[0][a]);
        h[1][a] = cneg(h[1][a]);
      }
    }
    double2 wv[2][3];
    // (U^H h)_a = sum_b conj(U_ba) h_b
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double2 u0a = lk.get(MU, 0, a, nb), u1a = lk.get(MU, 1, a, nb), u2a = lk.get(MU, 2, a, nb);
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
      acc[0 * 3 + a] = cadd(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = cadd(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = cadd(acc[2 * 3 + a], unit_mul(S::hcode0, wv[S::hcol0][a]));
      acc[3 * 3 + a] = cadd(acc[3 * 3 + a], unit_mul(S::hcode1, wv[S::hcol1][a]));
    }
  }
}

template <int MU, typename LK>
__device__ __forceinline__ void hop_dir32(const LK& lk, const float2* __restrict__ in, int s,
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
      h[0][a] = csub(u0, unit_mul(S::bcode0, l0));
      h[1][a] = csub(u1, unit_mul(S::bcode1, l1));
    }
    if (MU == 3 && w && g.bc_t < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h[0][a] = cneg(h[0][a]);
        h[1][a] = cneg(h[1][a]);
      }
    }
    Link32 L;
    lk.load(MU, s, L);
    float2 wv[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float2 t = cmul(L.e[a][0], h[r][0]);
        cmac(t, L.e[a][1], h[r][1]);
        cmac(t, L.e[a][2], h[r][2]);
        wv[r][a] = t;
      }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[0 * 3 + a] = cadd(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = cadd(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = csub(acc[2 * 3 + a], unit_mul(S::hcode0, wv[S::hcol0][a]));
      acc[3 * 3 + a] = csub(acc[3 * 3 + a], unit_mul(S::hcode1, wv[S::hcol1][a]));
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
      h[0][a] = cadd(u0, unit_mul(S::bcode0, l0));
      h[1][a] = cadd(u1, unit_mul(S::bcode1, l1));
    }
    if (MU == 3 && w && g.bc_t < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h[0][a] = cneg(h[0][a]);
        h[1][a] = cneg(h[1][a]);
      }
    }
    Link32 L;
    lk.load(MU, nb, L);
    float2 wv[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float2 t = cmul_conj(L.e[0][a], h[r][0]);
        cmac_conj(t, L.e[1][a], h[r][1]);
        cmac_conj(t, L.e[2][a], h[r][2]);
        wv[r][a] = t;
      }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[0 * 3 + a] = cadd(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = cadd(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = cadd(acc[2 * 3 + a], unit_mul(S::hcode0, wv[S::hcol0][a]));
      acc[3 * 3 + a] = cadd(acc[3 * 3 + a], unit_mul(S::hcode1, wv[S::hcol1][a]));
    }
  }
}

// ---- block-level stencil ------------------------------------------------------------
// A block of 128 threads = 4 warps covers sites s0 .. s0+31 of one rhs.  On
// return, thread (w, lane) holds hop sums acc_out[0..2] = (D psi) components
// 3w..3w+2 of site s0 + lane (zero beyond V).  sh: 32 x 12 x 4 complex
// shared-memory scratch.
constexpr int kSitesPerBlock = 32;
constexpr int kStencilThreads = 128;

template <typename C>
__device__ __forceinline__ void reduce_dirs(C (&acc)[12], C* sh, C (&acc_out)[3]) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // sh layout [comp 12][dir 4][site 32]
#pragma unroll
  for (int i = 0; i < 12; ++i) sh[(i * 4 + w) * 32 + lane] = acc[i];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int comp = 3 * w + k;
    C v = sh[(comp * 4 + 0) * 32 + lane];
    v = cadd(v, sh[(comp * 4 + 1) * 32 + lane]);
    v = cadd(v, sh[(comp * 4 + 2) * 32 + lane]);
    v = cadd(v, sh[(comp * 4 + 3) * 32 + lane]);
    acc_out[k] = v;
  }
}

__device__ __forceinline__ void block_hops64(const Links64& lk, const double2* __restrict__ in, int s,
                                             const Geometry& g, double2* sh, double2 (&acc_out)[3]) {
  double2 acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = make_double2(0.0, 0.0);
  if (s < g.V) {
    const Coords c = site_coords(s, g);
    switch (threadIdx.x >> 5) {
      case 0: hop_dir64<0>(lk, in, s, c, g, acc); break;
      case 1: hop_dir64<1>(lk, in, s, c, g, acc); break;
      case 2: hop_dir64<2>(lk, in, s, c, g, acc); break;
      default: hop_dir64<3>(lk, in, s, c, g, acc); break;
    }
  }
  reduce_dirs(acc, sh, acc_out);
}

// ---- FP64, balanced form: 16 sites per block, spin halves split ---------------------
// The FP64 stencil is bound by the FP64 pipe.  With 32 sites per block
// (above) an 8^4 lattice with four right-hand sides is 512 blocks, 3.4 per
// SM: the SMs holding four blocks set the time and the others idle ~25% of
// it.  Here a block covers 16 sites with 4 warps (warp w: direction w, both
// hops); the half-warp h = lane / 16 computes spin row h of the projected
// half spinor (h_r = psi_r -+ (B psi_l)_r) and its link product wv_r, which
// feeds upper output spin r and one lower output spin 2 + t(r) (B^H is a
// signed permutation).  No FP64 work is duplicated: the two halves share
// only the link loads (same addresses in one warp instruction), and each
// thread keeps 6 complex accumulators instead of 12, so the block fits 64
// registers a thread and 8 blocks an SM: 1024 blocks in one wave, 6.7 per SM.
// The per-lane differences (which spin components, which unit +-1, +-i of
// B and B^H) are applied with selects and sign-bit flips on the integer
// pipes, so the warp never diverges and the FP64 instruction count per
// site is the same as above.
constexpr int kSitesPerBlockH = 16;
constexpr unsigned long long kSignBit = 0x8000000000000000ull;

// multiplication by the unit `code` (+1, -1, +i, -i) with an extra sign flip
// of both parts (neg): selects and integer xors only
__device__ __forceinline__ double2 unit_apply(double2 z, int code, unsigned long long neg) {
  const bool swap = code >= PI;
  const unsigned long long mx = ((code == M1 || code == PI) ? kSignBit : 0ull) ^ neg;
  const unsigned long long my = ((code == M1 || code == MI) ? kSignBit : 0ull) ^ neg;
  const double a = swap ? z.y : z.x, b = swap ? z.x : z.y;
  return make_double2(__longlong_as_double(__double_as_longlong(a) ^ mx),
                      __longlong_as_double(__double_as_longlong(b) ^ my));
}
__device__ __forceinline__ double2 flip(double2 z, unsigned long long neg) {
  return make_double2(__longlong_as_double(__double_as_longlong(z.x) ^ neg),
                      __longlong_as_double(__double_as_longlong(z.y) ^ neg));
}

// One hop (forward: DIR = +1, U_mu(x) psi(x + mu), h = psi_u - B psi_l;
// backward: U_mu(x - mu)^H psi(x - mu), h = psi_u + B psi_l) for spin row r
// of site s.  The forward hop (first) sets up[] = lo[] = its product wf (no
// additions to zero, which IEEE arithmetic cannot drop by itself because of
// -0); the backward hop accumulates its product wb into up[] by FMA chains
// (up = wf + wb) and forms the lower row from the same sum: the lower spin
// t gets hcode (wb - wf) = hcode (up - 2 wf), one FMA a real part instead of
// a product and two additions.
template <int MU, int DIR>
__device__ __forceinline__ void hop_half64(const Links64& lk, const double2* __restrict__ in, int s, const Coords& c,
                                           const Geometry& g, int r, double2 (&up)[3], double2 (&lo)[3]) {
  using S = Spin<MU>;
  const int V = g.V;
  bool w;
  const int nb = neighbour<MU, DIR>(s, c, g, w);
  const int bcol = r ? S::bcol1 : S::bcol0;
  const int bcode = r ? S::bcode1 : S::bcode0;
  const int t = (r == S::hcol0) ? 0 : 1;
  const int hcode = t ? S::hcode1 : S::hcode0;
  // forward subtracts B psi_l and B^H wv; antiperiodic wrap negates h
  const unsigned long long nproj = DIR > 0 ? kSignBit : 0ull;
  const unsigned long long nwrap = (MU == 3 && w && g.bc_t < 0) ? kSignBit : 0ull;
  const unsigned long long nrec = DIR > 0 ? kSignBit : 0ull;
  double2 h[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double2 u = __ldg(in + (r * 3 + a) * V + nb);
    const double2 l = unit_apply(__ldg(in + ((2 + bcol) * 3 + a) * V + nb), bcode, nproj);
    h[a] = flip(make_double2(u.x + l.x, u.y + l.y), nwrap);
  }
  (void)nrec;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (DIR > 0) {
      const double2 u0 = lk.get(MU, a, 0, s), u1 = lk.get(MU, a, 1, s), u2 = lk.get(MU, a, 2, s);
      double2 tv = cmul(u0, h[0]);
      cmac(tv, u1, h[1]);
      cmac(tv, u2, h[2]);
      up[a] = tv;
      lo[a] = tv;
    } else {
      const double2 u0 = lk.get(MU, 0, a, nb), u1 = lk.get(MU, 1, a, nb), u2 = lk.get(MU, 2, a, nb);
      double2 tv = up[a];
      cmac_conj(tv, u0, h[0]);
      cmac_conj(tv, u1, h[1]);
      cmac_conj(tv, u2, h[2]);
      up[a] = tv;
      lo[a] = unit_apply(make_double2(fma(-2.0, lo[a].x, tv.x), fma(-2.0, lo[a].y, tv.y)), hcode, 0ull);
    }
  }
}

template <int MU>
__device__ __forceinline__ void hop_dir_half64(const Links64& lk, const double2* __restrict__ in, int s,
                                               const Geometry& g, int r, double2* sh, int i) {
  double2 up[3], lo[3];
  if (s < g.V) {
    const Coords c = site_coords(s, g);
    hop_half64<MU, +1>(lk, in, s, c, g, r, up, lo);
    hop_half64<MU, -1>(lk, in, s, c, g, r, up, lo);
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) up[a] = lo[a] = make_double2(0.0, 0.0);
  }
  using S = Spin<MU>;
  const int t = (r == S::hcol0) ? 0 : 1;
  // sh layout [comp 12][dir 4][site 16]
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    sh[((r * 3 + a) * 4 + MU) * kSitesPerBlockH + i] = up[a];
    sh[(((2 + t) * 3 + a) * 4 + MU) * kSitesPerBlockH + i] = lo[a];
  }
}

// Block of 128 threads: sites s0 .. s0 + 15 of one rhs; on return (after the
// barrier) sh holds the four directions' sums of every component.
__device__ __forceinline__ void block_hops64h(const Links64& lk, const double2* __restrict__ in, int s0,
                                              const Geometry& g, double2* sh) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = lane & (kSitesPerBlockH - 1), r = lane >> 4;
  const int s = s0 + i;
  switch (w) {
    case 0: hop_dir_half64<0>(lk, in, s, g, r, sh, i); break;
    case 1: hop_dir_half64<1>(lk, in, s, g, r, sh, i); break;
    case 2: hop_dir_half64<2>(lk, in, s, g, r, sh, i); break;
    default: hop_dir_half64<3>(lk, in, s, g, r, sh, i); break;
  }
  __syncthreads();
}

// ---- FP32: one thread per site ------------------------------------------------------
// For the memory-bound FP32 stencil a thread applies all eight hops of its
// site and keeps the twelve output components in registers: no cross-warp
// reduction, no barrier, and the coordinates are computed once per site.  A
// block of kSiteThreads threads covers kSiteThreads consecutive sites.
constexpr int kSiteThreads = 128;

template <typename LK>
__device__ __forceinline__ void site_hops32(const LK& lk, const float2* __restrict__ in, int s, const Geometry& g,
                                            float2 (&acc)[12]) {
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = make_float2(0.f, 0.f);
  const Coords c = site_coords(s, g);
  hop_dir32<0>(lk, in, s, c, g, acc);
  hop_dir32<1>(lk, in, s, c, g, acc);
  hop_dir32<2>(lk, in, s, c, g, acc);
  hop_dir32<3>(lk, in, s, c, g, acc);
}

template <typename LK>
__device__ __forceinline__ void block_hops32(const LK& lk, const float2* __restrict__ in, int s,
                                             const Geometry& g, float2* sh, float2 (&acc_out)[3]) {
  float2 acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = make_float2(0.f, 0.f);
  if (s < g.V) {
    const Coords c = site_coords(s, g);
    switch (threadIdx.x >> 5) {
      case 0: hop_dir32<0>(lk, in, s, c, g, acc); break;
      case 1: hop_dir32<1>(lk, in, s, c, g, acc); break;
      case 2: hop_dir32<2>(lk, in, s, c, g, acc); break;
      default: hop_dir32<3>(lk, in, s, c, g, acc); break;
    }
  }
  reduce_dirs(acc, sh, acc_out);
}

// ---- FP32, many right-hand sides a block ----------------------------------------------
// The FP32 stencil with 12-parameter links is bound by HBM only if its
// instruction count per site and rhs stays below ~1100 (the issue rate of
// 152 SMs against the 1632 compulsory bytes of a site with eight rhs).  The
// one-thread-per-site form above spends ~3000: every rhs rebuilds the third
// link row and recomputes the neighbour addresses.  Here a block covers 32
// sites for every rhs: warp w takes direction mu = w (forward and backward
// hop) for the 32 sites, loads and rebuilds its two links once, keeps them
// in registers pre-packed for paired FP32 arithmetic, and then loops over
// the rhs.  Per rhs the four directions' sums meet in shared memory and warp
// w finishes spinor components 3w..3w+2.
//
// Paired arithmetic: Blackwell executes fma/add/sub.rn.f32x2 on a register
// pair as one instruction (two lanes of FP32).  A complex multiply-add
// acc += u h is then two paired FMAs,
//   acc += (u.x, u.x) (h.x, h.y) + (-u.y, u.y) (h.y, h.x),
// with the link pairs (u.x, u.x), (-u.y, u.y) formed once per thread (they
// serve every rhs) and the swapped half-spinor (h.y, h.x) once per hop; the
// 72 FP32 FMAs of a hop's link product become 36 paired ones.
// unit (+1, -1, +i, -i) times z, as a pair
__device__ __forceinline__ f32x2_t unit2(int code, f32x2_t z) {
  const float2 v = upk2(z);
  switch (code) {
    case P1: return z;
    case M1: return pk2(-v.x, -v.y);
    case PI: return pk2(-v.y, v.x);
    default: return pk2(v.y, -v.x);
  }
}

// A link rebuilt from its 12 parameters, packed for the paired products:
// a[e] = (u.x, u.x), b[e] = (-u.y, u.y) for element e = 3 row + column of U
// (forward hop, U h) or of U^H (backward hop, U^H h: element (a, b) of U^H
// is conj(U_ba), so b holds (u.y, -u.y) of U_ba).
struct PackedLink {
  f32x2_t a[9], b[9];
};

template <typename LK>
__device__ __forceinline__ void load_packed(const LK& lk, int mu, int site, bool dagger, PackedLink& P) {
  Link32 L;
  lk.load(mu, site, L);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 u = dagger ? L.e[c][r] : L.e[r][c];
      const float uy = dagger ? -u.y : u.y;
      P.a[3 * r + c] = pk2(u.x, u.x);
      P.b[3 * r + c] = pk2(-uy, uy);
    }
}

// wv[a] = sum_b M_ab h_b for the packed link M, with hs[b] = (h_b.y, h_b.x)
__device__ __forceinline__ void link_mul2(const PackedLink& P, const f32x2_t (&h)[3], const f32x2_t (&hs)[3],
                                          f32x2_t (&wv)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    f32x2_t t = mul2(P.a[3 * a], h[0]);
    t = fma2(P.b[3 * a], hs[0], t);
    t = fma2(P.a[3 * a + 1], h[1], t);
    t = fma2(P.b[3 * a + 1], hs[1], t);
    t = fma2(P.a[3 * a + 2], h[2], t);
    t = fma2(P.b[3 * a + 2], hs[2], t);
    wv[a] = t;
  }
}

// One hop of direction MU (DIR = +1 forward, -1 backward) for right-hand
// side `in`, neighbour nb, accumulated into acc[12] (FIRST: set instead of
// add).  Forward: h = psi_u - B psi_l, lower part -B^H wv; backward:
// h = psi_u + B psi_l, lower part +B^H wv; an antiperiodic t wrap negates h.
template <int MU, int DIR, bool FIRST>
__device__ __forceinline__ void hop_mrhs(const PackedLink& P, const float2* __restrict__ in, int nb, int V,
                                         bool negate, f32x2_t (&acc)[12]) {
  using S = Spin<MU>;
  f32x2_t h[2][3], hs[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float2 u0 = __ldg(in + (0 * 3 + a) * V + nb);
    const float2 u1 = __ldg(in + (1 * 3 + a) * V + nb);
    const float2 l0 = __ldg(in + ((2 + S::bcol0) * 3 + a) * V + nb);
    const float2 l1 = __ldg(in + ((2 + S::bcol1) * 3 + a) * V + nb);
    const f32x2_t bl0 = unit2(S::bcode0, pk2(l0.x, l0.y)), bl1 = unit2(S::bcode1, pk2(l1.x, l1.y));
    f32x2_t h0 = DIR > 0 ? sub2(pk2(u0.x, u0.y), bl0) : add2(pk2(u0.x, u0.y), bl0);
    f32x2_t h1 = DIR > 0 ? sub2(pk2(u1.x, u1.y), bl1) : add2(pk2(u1.x, u1.y), bl1);
    if (MU == 3 && negate) {
      h0 = unit2(M1, h0);
      h1 = unit2(M1, h1);
    }
    h[0][a] = h0;
    h[1][a] = h1;
    hs[0][a] = swap2(h0);
    hs[1][a] = swap2(h1);
  }
  f32x2_t wv[2][3];
  link_mul2(P, h[0], hs[0], wv[0]);
  link_mul2(P, h[1], hs[1], wv[1]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const f32x2_t lo0 = unit2(S::hcode0, wv[S::hcol0][a]), lo1 = unit2(S::hcode1, wv[S::hcol1][a]);
    if (FIRST) {
      acc[0 * 3 + a] = wv[0][a];
      acc[1 * 3 + a] = wv[1][a];
      acc[2 * 3 + a] = DIR > 0 ? unit2(M1, lo0) : lo0;
      acc[3 * 3 + a] = DIR > 0 ? unit2(M1, lo1) : lo1;
    } else {
      acc[0 * 3 + a] = add2(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = add2(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = DIR > 0 ? sub2(acc[2 * 3 + a], lo0) : add2(acc[2 * 3 + a], lo0);
      acc[3 * 3 + a] = DIR > 0 ? sub2(acc[3 * 3 + a], lo1) : add2(acc[3 * 3 + a], lo1);
    }
  }
}

// out_r = c0 in_r + c1 A in_r for the rhs r = 0..nrhs-1 of 32 sites
// (block of 128 threads, warp w = direction MU = w); dot_partial (optional):
// per rhs the block's share of Re <in_r, out_r> at dot_partial[r * gridDim.x
// + blockIdx.x].  sh: 2 x 12 x 4 x 32 float2 and shred: 2 x 4 floats, double
// buffered by rhs parity, so one barrier per rhs separates the four
// directions' partial sums from their combination (a buffer is rewritten two
// rhs later, after the next barrier, by which every warp has finished
// reading it).
template <int MU, typename LK>
__device__ __forceinline__ void mrhs_block(const Geometry& g, const LK& lk, const float2* __restrict__ in_all,
                                           float2* __restrict__ out_all, int nrhs, float c0, float c1,
                                           float2* sh2, float* shred2, float* __restrict__ dot_partial) {
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x * 32 + lane;
  const int V = g.V;
  const bool act = s < V;
  PackedLink Pf, Pb;
  int nbf = 0, nbb = 0;
  bool wf = false, wb = false;
  if (act) {
    const Coords c = site_coords(s, g);
    nbf = neighbour<MU, +1>(s, c, g, wf);
    nbb = neighbour<MU, -1>(s, c, g, wb);
    load_packed(lk, MU, s, false, Pf);
    load_packed(lk, MU, nbb, true, Pb);
  }
  const bool negf = wf && g.bc_t < 0, negb = wb && g.bc_t < 0;
  const float mk = -(float)g.kappa;
  const float sg = MU < 2 ? c1 : -c1;  // gamma5 on spin MU of components 3 MU .. 3 MU + 2
  for (int r = 0; r < nrhs; ++r) {
    float2* sh = sh2 + (r & 1) * (12 * 4 * 32);
    float* shred = shred2 + (r & 1) * 4;
    const float2* in = in_all + (size_t)r * 12 * V;
    f32x2_t acc[12];
    if (act) {
      hop_mrhs<MU, +1, true>(Pf, in, nbf, V, negf, acc);
      hop_mrhs<MU, -1, false>(Pb, in, nbb, V, negb, acc);
    } else {
#pragma unroll
      for (int i = 0; i < 12; ++i) acc[i] = 0ull;
    }
#pragma unroll
    for (int i = 0; i < 12; ++i) sh[(i * 4 + MU) * 32 + lane] = upk2(acc[i]);
    __syncthreads();
    if (dot_partial != nullptr && r > 0 && threadIdx.x == 0) {
      const float* pr = shred2 + ((r - 1) & 1) * 4;
      dot_partial[(size_t)(r - 1) * gridDim.x + blockIdx.x] = (pr[0] + pr[1]) + (pr[2] + pr[3]);
    }
    float dot = 0.f;
    if (act) {
      float2* out = out_all + (size_t)r * 12 * V;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int i = 3 * MU + k;
        const float2 e0 = sh[(i * 4 + 0) * 32 + lane], e1 = sh[(i * 4 + 1) * 32 + lane];
        const float2 e2 = sh[(i * 4 + 2) * 32 + lane], e3 = sh[(i * 4 + 3) * 32 + lane];
        const float2 dv = upk2(add2(add2(pk2(e0.x, e0.y), pk2(e1.x, e1.y)), add2(pk2(e2.x, e2.y), pk2(e3.x, e3.y))));
        const float2 p = __ldg(in + i * V + s);
        float2 o;
        o.x = fmaf(sg, fmaf(mk, dv.x, p.x), c0 * p.x);
        o.y = fmaf(sg, fmaf(mk, dv.y, p.y), c0 * p.y);
        out[i * V + s] = o;
        dot = fmaf(p.x, o.x, fmaf(p.y, o.y, dot));
      }
    }
    if (dot_partial != nullptr) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) dot += __shfl_down_sync(0xffffffffu, dot, o);
      if (lane == 0) shred[MU] = dot;
    }
  }
  if (dot_partial != nullptr) {
    __syncthreads();
    if (threadIdx.x == 0 && nrhs > 0) {
      const float* pr = shred2 + ((nrhs - 1) & 1) * 4;
      dot_partial[(size_t)(nrhs - 1) * gridDim.x + blockIdx.x] = (pr[0] + pr[1]) + (pr[2] + pr[3]);
    }
  }
}

// ---- FP32, one thread per site and rhs pair ------------------------------------------
// Without the block's cross-warp sum: a thread applies all eight hops of its
// site to two rhs at once, so every link is loaded and rebuilt once for two
// rhs, the neighbour indices once for both, and there is no barrier.  The
// 2 x 12 accumulators and the hop's packed link stay in registers.
template <int MU, int DIR, typename LK>
__device__ __forceinline__ void hop_pair(const LK& lk, const float2* __restrict__ in0,
                                         const float2* __restrict__ in1, int s, const Coords& c, const Geometry& g,
                                         bool first, f32x2_t (&acc0)[12], f32x2_t (&acc1)[12]) {
  bool w;
  const int nb = neighbour<MU, DIR>(s, c, g, w);
  PackedLink P;
  load_packed(lk, MU, DIR > 0 ? s : nb, DIR < 0, P);
  const bool neg = MU == 3 && w && g.bc_t < 0;
  if (first) {
    hop_mrhs<MU, DIR, true>(P, in0, nb, g.V, neg, acc0);
    hop_mrhs<MU, DIR, true>(P, in1, nb, g.V, neg, acc1);
  } else {
    hop_mrhs<MU, DIR, false>(P, in0, nb, g.V, neg, acc0);
    hop_mrhs<MU, DIR, false>(P, in1, nb, g.V, neg, acc1);
  }
}

template <typename LK>
__device__ __forceinline__ void site_hops_pair(const LK& lk, const float2* __restrict__ in0,
                                               const float2* __restrict__ in1, int s, const Geometry& g,
                                               f32x2_t (&acc0)[12], f32x2_t (&acc1)[12]) {
  const Coords c = site_coords(s, g);
  hop_pair<0, +1>(lk, in0, in1, s, c, g, true, acc0, acc1);
  hop_pair<0, -1>(lk, in0, in1, s, c, g, false, acc0, acc1);
  hop_pair<1, +1>(lk, in0, in1, s, c, g, false, acc0, acc1);
  hop_pair<1, -1>(lk, in0, in1, s, c, g, false, acc0, acc1);
  hop_pair<2, +1>(lk, in0, in1, s, c, g, false, acc0, acc1);
  hop_pair<2, -1>(lk, in0, in1, s, c, g, false, acc0, acc1);
  hop_pair<3, +1>(lk, in0, in1, s, c, g, false, acc0, acc1);
  hop_pair<3, -1>(lk, in0, in1, s, c, g, false, acc0, acc1);
}

// ---- FP32, two rhs in the lanes of the paired instructions ------------------------------
// Layout "rhs pairs": rhs 2q and 2q + 1 interleaved, [npair][12][V] float4
// = (re_{2q}, re_{2q+1}, im_{2q}, im_{2q+1}), so the real parts of the two
// rhs form one register pair and the imaginary parts another.  A complex
// number times a link element u is then four paired FMAs for two rhs with
// the broadcast pairs (u.x, u.x), (u.y, u.y), (-u.y, -u.y), and a factor
// +-1 or +-i (the spin projection and reconstruction) only chooses which
// pair and which sign: no lane swaps.  A thread covers one site and one rhs
// pair: 12 16-byte loads per neighbour, 72 paired FMAs per hop for two rhs.
struct C2 {
  f32x2_t re, im;
};

__device__ __forceinline__ C2 c2_load(const float4* __restrict__ p) {
  const float4 v = __ldg(p);
  return C2{pk2(v.x, v.y), pk2(v.z, v.w)};
}
// z + code * w (code +1, -1, +i, -i)
__device__ __forceinline__ C2 c2_add_unit(const C2& z, int code, const C2& w) {
  switch (code) {
    case P1: return C2{add2(z.re, w.re), add2(z.im, w.im)};
    case M1: return C2{sub2(z.re, w.re), sub2(z.im, w.im)};
    case PI: return C2{sub2(z.re, w.im), add2(z.im, w.re)};  // + i w = (-w.im, w.re)
    default: return C2{add2(z.re, w.im), sub2(z.im, w.re)};  // - i w = (w.im, -w.re)
  }
}
__device__ __forceinline__ C2 c2_neg(const C2& z) { return C2{neg2(z.re), neg2(z.im)}; }

// A link rebuilt from its 12 parameters as broadcast pairs: x[e] = (u.x,
// u.x), y[e] = (u.y, u.y), ny[e] = (-u.y, -u.y) for element e = 3 row +
// column of U (dagger = false) or of U^H (true; conj folds into the signs).
struct BcastLink {
  f32x2_t x[9], y[9], ny[9];
};
template <typename LK>
__device__ __forceinline__ void load_bcast(const LK& lk, int mu, int site, bool dagger, BcastLink& B) {
  Link32 L;
  lk.load(mu, site, L);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float2 u = dagger ? L.e[c][r] : L.e[r][c];
      const float uy = dagger ? -u.y : u.y;
      B.x[3 * r + c] = pk2(u.x, u.x);
      B.y[3 * r + c] = pk2(uy, uy);
      B.ny[3 * r + c] = pk2(-uy, -uy);
    }
}
// row a of the link times h: sum_b M_ab h_b for both rhs
__device__ __forceinline__ C2 c2_row(const BcastLink& B, int a, const C2 (&h)[3]) {
  f32x2_t re = mul2(B.x[3 * a], h[0].re), im = mul2(B.x[3 * a], h[0].im);
  re = fma2(B.ny[3 * a], h[0].im, re);
  im = fma2(B.y[3 * a], h[0].re, im);
#pragma unroll
  for (int b = 1; b < 3; ++b) {
    re = fma2(B.x[3 * a + b], h[b].re, re);
    im = fma2(B.x[3 * a + b], h[b].im, im);
    re = fma2(B.ny[3 * a + b], h[b].im, re);
    im = fma2(B.y[3 * a + b], h[b].re, im);
  }
  return C2{re, im};
}

// Where a hop reads its neighbour's components: global memory (component
// comp of site nb at in + comp V + nb) or a shared-memory tile (sh + comp
// stride + idx).
struct SrcGlobal {
  const float4* __restrict__ in;
  int V, nb;
  __device__ __forceinline__ C2 operator()(int comp) const { return c2_load(in + comp * V + nb); }
};
struct SrcShared {
  const float4* sh;
  int stride, idx;
  __device__ __forceinline__ C2 operator()(int comp) const {
    const float4 v = sh[comp * stride + idx];
    return C2{pk2(v.x, v.y), pk2(v.z, v.w)};
  }
};

// One hop (DIR +1: U_mu(x) psi(x + mu), h = psi_u - B psi_l, lower -B^H wv;
// DIR -1: U_mu(x - mu)^H psi(x - mu), h = psi_u + B psi_l, lower +B^H wv)
// of one rhs pair into acc[12] (FIRST: set instead of add).
template <int MU, int DIR, bool FIRST, typename SRC>
__device__ __forceinline__ void hop_rp(const BcastLink& B, const SRC& src, bool negate, C2 (&acc)[12]) {
  using S = Spin<MU>;
  C2 h[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const C2 u0 = src(0 * 3 + a);
    const C2 u1 = src(1 * 3 + a);
    const C2 l0 = src((2 + S::bcol0) * 3 + a);
    const C2 l1 = src((2 + S::bcol1) * 3 + a);
    // forward subtracts B psi_l: the code with its sign flipped (P1 <-> M1, PI <-> MI)
    h[0][a] = c2_add_unit(u0, DIR > 0 ? (S::bcode0 ^ 1) : S::bcode0, l0);
    h[1][a] = c2_add_unit(u1, DIR > 0 ? (S::bcode1 ^ 1) : S::bcode1, l1);
    if (MU == 3 && negate) {
      h[0][a] = c2_neg(h[0][a]);
      h[1][a] = c2_neg(h[1][a]);
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const C2 w0 = c2_row(B, a, h[0]), w1 = c2_row(B, a, h[1]);
    const C2 wt0 = S::hcol0 == 0 ? w0 : w1, wt1 = S::hcol1 == 0 ? w0 : w1;
    const int c0 = DIR > 0 ? (S::hcode0 ^ 1) : S::hcode0, c1 = DIR > 0 ? (S::hcode1 ^ 1) : S::hcode1;
    if (FIRST) {
      acc[0 * 3 + a] = w0;
      acc[1 * 3 + a] = w1;
      const C2 zero{0ull, 0ull};
      acc[2 * 3 + a] = c2_add_unit(zero, c0, wt0);
      acc[3 * 3 + a] = c2_add_unit(zero, c1, wt1);
    } else {
      acc[0 * 3 + a] = c2_add_unit(acc[0 * 3 + a], P1, w0);
      acc[1 * 3 + a] = c2_add_unit(acc[1 * 3 + a], P1, w1);
      acc[2 * 3 + a] = c2_add_unit(acc[2 * 3 + a], c0, wt0);
      acc[3 * 3 + a] = c2_add_unit(acc[3 * 3 + a], c1, wt1);
    }
  }
}

template <int MU, int DIR, typename LK>
__device__ __forceinline__ void hop_rp_site(const LK& lk, const float4* __restrict__ in, int s, const Coords& c,
                                            const Geometry& g, bool first, C2 (&acc)[12]) {
  bool w;
  const int nb = neighbour<MU, DIR>(s, c, g, w);
  BcastLink B;
  load_bcast(lk, MU, DIR > 0 ? s : nb, DIR < 0, B);
  const bool neg = MU == 3 && w && g.bc_t < 0;
  const SrcGlobal src{in, g.V, nb};
  if (first)
    hop_rp<MU, DIR, true>(B, src, neg, acc);
  else
    hop_rp<MU, DIR, false>(B, src, neg, acc);
}

// The same hop with the neighbour's spinor read from a shared-memory tile
// (directions x and y only: no boundary sign).
template <int MU, int DIR, typename LK>
__device__ __forceinline__ void hop_rp_tile(const LK& lk, const float4* sh, int stride, int idx, int s,
                                            const Coords& c, const Geometry& g, bool first, C2 (&acc)[12]) {
  static_assert(MU < 2, "tile hops are the x and y directions");
  bool w;
  const int nb = neighbour<MU, DIR>(s, c, g, w);
  BcastLink B;
  load_bcast(lk, MU, DIR > 0 ? s : nb, DIR < 0, B);
  const SrcShared src{sh, stride, idx};
  if (first)
    hop_rp<MU, DIR, true>(B, src, false, acc);
  else
    hop_rp<MU, DIR, false>(B, src, false, acc);
}

}  // namespace wcore
}  // namespace ssqcd
