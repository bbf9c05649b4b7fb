// Float-float form of the Wilson-Dirac stencil (A = gamma5 (I - kappa D),
// Section 4 of the paper) for the SSQCD_DF solve precision: spinors and
// links are complex float-float (float4 {re.hi, im.hi, re.lo, im.lo}, see
// floatfloat.cuh), so every operation runs on the FP32 pipes with a 48-bit
// significand.  Same spin projection and data layout as the FP64 stencil in
// wilson_core.cuh; the work split differs (one hop per warp, below).
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

// ---- one hop per warp ----------------------------------------------------------------
// A block of 256 threads = 8 warps covers 32 sites: warp 2 mu + d applies the
// forward (d = 0) or backward (d = 1) hop in direction mu and stores the
// link-multiplied half spinor wv[2][3] of each site to shared memory; after
// a barrier, the eight hops are summed per spinor component, components w
// and w + 8 by warp w (the lower spins through the signed permutations
// B_mu^H).  Against two hops per warp with a 12-component accumulator this
// holds half the registers per thread, so more warps hide the latency of
// the float-float chains, and stays balanced next to the concurrent
// shift-update kernel.  The complex float-float operations run on register
// pairs (real and imaginary part in the two lanes of one paired
// instruction, floatfloat.cuh), bit-identical to the scalar form.
constexpr int kStencilThreadsDF = 256;

// One hop of warp 2 mu + d at site s: h = (1 -/+ gamma_mu) psi(x +/- mu) in
// the two-spinor form h_r = psi_r + c_r psi_{bcol_r} (c_r the unit factor
// of B_mu's row r, negated on the forward hop: exact), then U_mu(x) h by
// rows (forward) or U_mu(x - mu)^H h by conjugated columns (backward).  The
// direction is a run-time value, so the eight warps of a block share one
// instruction stream: with a compile-time copy per direction the kernel's
// code outgrew the instruction cache and warps waited on instruction fetch
// ("no instruction" the first stall reason in ncu, 6.4 cycles per issue at
// one rhs).
__device__ __forceinline__ void hop_one_df_rt(const LinksDF& lk, const float4* __restrict__ in, int s,
                                              const Coords& c, const Geometry& g, int mu, bool fwd,
                                              float4* __restrict__ out) {
  const int V = g.V;
  const int coord = mu == 0 ? c.x : mu == 1 ? c.y : mu == 2 ? c.z : c.t;
  const int ext = mu == 0 ? g.X : mu == 1 ? g.Y : mu == 2 ? g.Z : g.T;
  const int st = mu == 0 ? 1 : mu == 1 ? g.X : mu == 2 ? g.X * g.Y : g.X * g.Y * g.Z;
  const bool wrap = fwd ? coord == ext - 1 : coord == 0;
  const int nb = fwd ? (wrap ? s - (ext - 1) * st : s + st) : (wrap ? s + (ext - 1) * st : s - st);
  // Spin<mu>: lower-spin column and unit factor of B_mu's two rows
  constexpr int bcol[4] = {Spin<0>::bcol0, Spin<1>::bcol0, Spin<2>::bcol0, Spin<3>::bcol0};
  constexpr int bcode[2][4] = {{Spin<0>::bcode0, Spin<1>::bcode0, Spin<2>::bcode0, Spin<3>::bcode0},
                               {Spin<0>::bcode1, Spin<1>::bcode1, Spin<2>::bcode1, Spin<3>::bcode1}};
  const int bcol0 = bcol[mu], bcol1 = 1 - bcol0;
  const int bc0 = bcode[0][mu], bc1 = bcode[1][mu];
  // (1 - gamma_mu): h = psi_u - B psi_l, the unit factor's sign flipped
  const int code0 = fwd ? (bc0 ^ 1) : bc0, code1 = fwd ? (bc1 ^ 1) : bc1;
  const bool negate = mu == 3 && wrap && g.bc_t < 0;
  float4 h[2][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float4 u0 = __ldg(in + (0 * 3 + a) * V + nb);
    const float4 u1 = __ldg(in + (1 * 3 + a) * V + nb);
    const float4 l0 = __ldg(in + ((2 + bcol0) * 3 + a) * V + nb);
    const float4 l1 = __ldg(in + ((2 + bcol1) * 3 + a) * V + nb);
    h[0][a] = ff::p_cadd(u0, ff::unit_mul(code0, l0));
    h[1][a] = ff::p_cadd(u1, ff::unit_mul(code1, l1));
    if (negate) {
      h[0][a] = ff::cneg(h[0][a]);
      h[1][a] = ff::cneg(h[1][a]);
    }
  }
  const float sg = fwd ? -1.f : 1.f;  // conjugated link columns on the backward hop
  const int ls = fwd ? s : nb;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float4 w0 = lk.get(mu, fwd ? a : 0, fwd ? 0 : a, ls);
    const float4 w1 = lk.get(mu, fwd ? a : 1, fwd ? 1 : a, ls);
    const float4 w2 = lk.get(mu, fwd ? a : 2, fwd ? 2 : a, ls);
    out[(0 * 3 + a) * 32] = ff::p_cdot3_sg(w0, w1, w2, h[0][0], h[0][1], h[0][2], sg);
    out[(1 * 3 + a) * 32] = ff::p_cdot3_sg(w0, w1, w2, h[1][0], h[1][1], h[1][2], sg);
  }
}

// Hop sum of spinor component i (spin i / 3, colour i % 3) of site s0 + lane
// from the eight stored hops (sh: 8 x 6 x 32 float4).
__device__ __forceinline__ float4 hop_sum_df(const float4* __restrict__ sh, int i, int lane) {
  // lower spins: (1 -+ gamma) puts -+ B^H wv in spins 2, 3; spin 2 reads wv[hcol0] with hcode0, spin 3 wv[hcol1]
  constexpr int hcol[2][4] = {{Spin<0>::hcol0, Spin<1>::hcol0, Spin<2>::hcol0, Spin<3>::hcol0},
                              {Spin<0>::hcol1, Spin<1>::hcol1, Spin<2>::hcol1, Spin<3>::hcol1}};
  constexpr int hcode[2][4] = {{Spin<0>::hcode0, Spin<1>::hcode0, Spin<2>::hcode0, Spin<3>::hcode0},
                               {Spin<0>::hcode1, Spin<1>::hcode1, Spin<2>::hcode1, Spin<3>::hcode1}};
  const int sp = i / 3, a = i - 3 * sp;
  const float4* base = sh + lane;
  float4 acc;
  if (sp < 2) {
    acc = base[(0 * 6 + sp * 3 + a) * 32];
#pragma unroll
    for (int hp = 1; hp < 8; ++hp) acc = ff::p_cadd(acc, base[(hp * 6 + sp * 3 + a) * 32]);
  } else {
    const int rr = sp - 2;
#pragma unroll
    for (int hp = 0; hp < 8; ++hp) {
      const int mu = hp >> 1;
      const bool fwd = (hp & 1) == 0;
      const int col = rr == 0 ? hcol[0][mu] : hcol[1][mu];
      const int code = rr == 0 ? hcode[0][mu] : hcode[1][mu];
      const float4 t = ff::unit_mul(fwd ? (code ^ 1) : code, base[(hp * 6 + col * 3 + a) * 32]);
      acc = hp == 0 ? t : ff::p_cadd(acc, t);
    }
  }
  return acc;
}

// All eight hops of the block's 32 sites into sh (zeros beyond V), then a
// block barrier; the caller sums with hop_sum_df.
__device__ __forceinline__ void block_hops_df8(const LinksDF& lk, const float4* __restrict__ in, int s,
                                               const Geometry& g, float4* sh) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4* out = sh + (size_t)w * 6 * 32 + lane;
  if (s < g.V) {
    const Coords c = site_coords(s, g);
    hop_one_df_rt(lk, in, s, c, g, w >> 1, (w & 1) == 0, out);  // warp 2 mu + d: direction mu, d = 0 forward
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) out[k * 32] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  __syncthreads();
}

// q_i = c0 p_i + c1 g5_i (p_i - kappa (D p)_i) for one spinor component i of
// site s from its hop sum; returns the float-float share p_i^* q_i of (p, q)
// (real part).
__device__ __forceinline__ float2 finish_df1(const Geometry& g, const float4* __restrict__ p,
                                             float4* __restrict__ q, float2 c0, float2 c1, int s, int i, float4 acc) {
  const float2 mk = ff::split(-g.kappa);
  const float2 sg = i < 6 ? c1 : ff::neg(c1);
  const float4 pv = p[i * g.V + s];
  const float4 t = ff::caxpy(pv, mk, acc);  // p - kappa D p
  const float2 cs[2] = {c0, sg};
  const float2 br[2] = {ff::re(pv), ff::re(t)}, bi[2] = {ff::im(pv), ff::im(t)};
  const float4 o = ff::make(ff::dot<2>(cs, br), ff::dot<2>(cs, bi));
  q[i * g.V + s] = o;
  const float2 a2[2] = {ff::re(pv), ff::im(pv)}, b2[2] = {ff::re(o), ff::im(o)};
  return ff::dot<2>(a2, b2);
}

}  // namespace wcore
}  // namespace ssqcd
