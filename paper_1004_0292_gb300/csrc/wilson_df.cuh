// Float-float form of the Wilson-Dirac stencil (A = gamma5 (I - kappa D),
// Section 4 of the paper) for the SSQCD_DF solve precision: spinors and
// links are complex float-float (float4 {re.hi, im.hi, re.lo, im.lo}, see
// floatfloat.cuh), so every operation runs on the FP32 pipes with a 48-bit
// significand.  Same work split, spin projection and data layout as the FP64
// stencil in wilson_core.cuh: a block covers 32 sites of one rhs, warp mu
// applies the forward and backward hop in direction mu, and the four partial
// sums meet in shared memory.
#pragma once

#include "floatfloat.cuh"
#include "wilson_core.cuh"

namespace ssqcd {
namespace wcore {

// float-float links [4][9][V] float4, row-major 3x3 (same order as Links64)
struct LinksDF {
  const float4* __restrict__ u;
  int V;
  __device__ __forceinline__ float4 get(int mu, int a, int b, int s) const {
    return __ldg(u + (size_t)(mu * 9 + 3 * a + b) * V + s);
  }
};

template <int MU>
__device__ __forceinline__ void hop_dir_df(const LinksDF& lk, const float4* __restrict__ in, int s, const Coords& c,
                                           const Geometry& g, float4 (&acc)[12]) {
  using S = Spin<MU>;
  const int V = g.V;
  {  // forward: (1 - gamma_mu) U_mu(x) psi(x + mu)
    bool w;
    const int nb = neighbour<MU, +1>(s, c, g, w);
    float4 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float4 u0 = __ldg(in + (0 * 3 + a) * V + nb);
      const float4 u1 = __ldg(in + (1 * 3 + a) * V + nb);
      const float4 l0 = __ldg(in + ((2 + S::bcol0) * 3 + a) * V + nb);
      const float4 l1 = __ldg(in + ((2 + S::bcol1) * 3 + a) * V + nb);
      h[0][a] = ff::csub(u0, ff::unit_mul(S::bcode0, l0));
      h[1][a] = ff::csub(u1, ff::unit_mul(S::bcode1, l1));
    }
    if (MU == 3 && w && g.bc_t < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h[0][a] = ff::cneg(h[0][a]);
        h[1][a] = ff::cneg(h[1][a]);
      }
    }
    float4 wv[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float4 ua0 = lk.get(MU, a, 0, s), ua1 = lk.get(MU, a, 1, s), ua2 = lk.get(MU, a, 2, s);
#pragma unroll
      for (int r = 0; r < 2; ++r) wv[r][a] = ff::cdot3(ua0, ua1, ua2, h[r][0], h[r][1], h[r][2]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[0 * 3 + a] = ff::cadd(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = ff::cadd(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = ff::csub(acc[2 * 3 + a], ff::unit_mul(S::hcode0, wv[S::hcol0][a]));
      acc[3 * 3 + a] = ff::csub(acc[3 * 3 + a], ff::unit_mul(S::hcode1, wv[S::hcol1][a]));
    }
  }
  {  // backward: (1 + gamma_mu) U_mu(x - mu)^H psi(x - mu)
    bool w;
    const int nb = neighbour<MU, -1>(s, c, g, w);
    float4 h[2][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float4 u0 = __ldg(in + (0 * 3 + a) * V + nb);
      const float4 u1 = __ldg(in + (1 * 3 + a) * V + nb);
      const float4 l0 = __ldg(in + ((2 + S::bcol0) * 3 + a) * V + nb);
      const float4 l1 = __ldg(in + ((2 + S::bcol1) * 3 + a) * V + nb);
      h[0][a] = ff::cadd(u0, ff::unit_mul(S::bcode0, l0));
      h[1][a] = ff::cadd(u1, ff::unit_mul(S::bcode1, l1));
    }
    if (MU == 3 && w && g.bc_t < 0) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        h[0][a] = ff::cneg(h[0][a]);
        h[1][a] = ff::cneg(h[1][a]);
      }
    }
    float4 wv[2][3];
    // (U^H h)_a = sum_b conj(U_ba) h_b
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float4 u0a = lk.get(MU, 0, a, nb), u1a = lk.get(MU, 1, a, nb), u2a = lk.get(MU, 2, a, nb);
#pragma unroll
      for (int r = 0; r < 2; ++r) wv[r][a] = ff::cdot3_conj(u0a, u1a, u2a, h[r][0], h[r][1], h[r][2]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[0 * 3 + a] = ff::cadd(acc[0 * 3 + a], wv[0][a]);
      acc[1 * 3 + a] = ff::cadd(acc[1 * 3 + a], wv[1][a]);
      acc[2 * 3 + a] = ff::cadd(acc[2 * 3 + a], ff::unit_mul(S::hcode0, wv[S::hcol0][a]));
      acc[3 * 3 + a] = ff::cadd(acc[3 * 3 + a], ff::unit_mul(S::hcode1, wv[S::hcol1][a]));
    }
  }
}

// On return, thread (w, lane) holds the hop sums acc_out[0..2] = (D psi)
// components 3w..3w+2 of site s0 + lane; sh: 12 x 4 x 32 float4 scratch.
__device__ __forceinline__ void block_hops_df(const LinksDF& lk, const float4* __restrict__ in, int s,
                                              const Geometry& g, float4* sh, float4 (&acc_out)[3]) {
  float4 acc[12];
#pragma unroll
  for (int i = 0; i < 12; ++i) acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (s < g.V) {
    const Coords c = site_coords(s, g);
    switch (threadIdx.x >> 5) {
      case 0: hop_dir_df<0>(lk, in, s, c, g, acc); break;
      case 1: hop_dir_df<1>(lk, in, s, c, g, acc); break;
      case 2: hop_dir_df<2>(lk, in, s, c, g, acc); break;
      default: hop_dir_df<3>(lk, in, s, c, g, acc); break;
    }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < 12; ++i) sh[(i * 4 + w) * 32 + lane] = acc[i];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int comp = 3 * w + k;
    float4 v = sh[(comp * 4 + 0) * 32 + lane];
    v = ff::cadd(v, sh[(comp * 4 + 1) * 32 + lane]);
    v = ff::cadd(v, sh[(comp * 4 + 2) * 32 + lane]);
    v = ff::cadd(v, sh[(comp * 4 + 3) * 32 + lane]);
    acc_out[k] = v;
  }
}

// q = c0 p + c1 gamma5 (p - kappa D p) at the three components of spin w of
// site s (s < V), from the hop sums acc; returns this thread's float-float
// share of (p, q).
__device__ __forceinline__ float2 finish_df(const Geometry& g, const float4* __restrict__ p, float4* __restrict__ q,
                                            float2 c0, float2 c1, int s, int w, const float4 (&acc)[3]) {
  const float2 mk = ff::split(-g.kappa);
  const float2 sg = w < 2 ? c1 : ff::neg(c1);
  float2 a[6], b[6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int i = 3 * w + k;
    const float4 pv = p[i * g.V + s];
    const float4 t = ff::caxpy(pv, mk, acc[k]);  // p - kappa D p
    const float2 cs[2] = {c0, sg};
    const float2 br[2] = {ff::re(pv), ff::re(t)}, bi[2] = {ff::im(pv), ff::im(t)};
    const float4 o = ff::make(ff::dot<2>(cs, br), ff::dot<2>(cs, bi));
    q[i * g.V + s] = o;
    a[2 * k] = ff::re(pv);
    b[2 * k] = ff::re(o);
    a[2 * k + 1] = ff::im(pv);
    b[2 * k + 1] = ff::im(o);
  }
  return ff::dot<6>(a, b);
}

}  // namespace wcore
}  // namespace ssqcd
