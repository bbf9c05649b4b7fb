// Stand-alone application of the Hermitian fermion matrix A = gamma5 (I - kappa D)
// (Section 4 of the paper): out = c0 in + c1 A in for a block of right-hand
// sides, in FP64 (FP64 links) or FP32 (FP16 12-parameter links).  The device
// building blocks and the work split are described in wilson_core.cuh.
//
// FP64: on GB300 FP64 runs at 1/64 of the FP32 rate (~1.2 TFLOP/s measured),
// so this kernel is bound by the FP64 pipe, not by HBM: per site and rhs
// 8 x (12 projection adds + 72 link FMA/MUL + 24 reconstruction adds) + 18
// combine adds + 24 FMA ~ 906 FP64 instructions against 192 B (spinor in) +
// 192 B (out) + 576 B (links, shared by the rhs) of compulsory traffic.
// FP32 spinors with FP16 (or FP32) 12-parameter links: HBM-bound; 96 B in,
// 96 B out, 96 (192) B links per site.
#include <atomic>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "wilson_core.cuh"
#include "wilson_df.cuh"

namespace ssqcd {
namespace {

using namespace wcore;

// ---- the FP32 stencil variants and their autotuner ----------------------------------
// (see fp32_variant below)

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

__global__ void __launch_bounds__(kStencilThreads)
wilson64_kernel(Geometry g, const double2* __restrict__ u, const double2* __restrict__ in_all,
                double2* __restrict__ out_all, double c0, double c1, double* __restrict__ dot_partial,
                const int* __restrict__ skip_if_zero) {
  if (skip_if_zero != nullptr && *skip_if_zero == 0) return;
  __shared__ double2 sh[12 * 4 * 32];
  __shared__ double shd[kStencilThreads / 32];
  const int rhs = blockIdx.y;
  const int V = g.V;
  const double2* in = in_all + (size_t)rhs * 12 * V;
  double2* out = out_all + (size_t)rhs * 12 * V;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int s = blockIdx.x * kSitesPerBlock + lane;
  double2 acc[3];
  block_hops64(Links64{u, V}, in, s, g, sh, acc);
  double dot = 0.0;
  if (s < V) {
    // out = c0 psi + c1 gamma5 (psi - kappa D psi); components 3w..3w+2 = spin w
    const double sg = w < 2 ? c1 : -c1;
    const double mk = -g.kappa;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int i = 3 * w + k;
      const double2 p = in[i * V + s];
      double2 o;
      o.x = fma(sg, fma(mk, acc[k].x, p.x), c0 * p.x);
      o.y = fma(sg, fma(mk, acc[k].y, p.y), c0 * p.y);
      out[i * V + s] = o;
      dot = fma(p.x, o.x, fma(p.y, o.y, dot));
    }
  }
  if (dot_partial != nullptr) {
    const double b = block_sum<kStencilThreads>(dot, shd);
    if (threadIdx.x == 0) dot_partial[(size_t)rhs * gridDim.x + blockIdx.x] = b;
  }
}

// FP32 spinors, one thread per site (see site_hops32).
template <typename LK>
__global__ void __launch_bounds__(kSiteThreads)
wilson32_kernel(Geometry g, LK lk, const float2* __restrict__ in_all,
                float2* __restrict__ out_all, float c0, float c1, float* __restrict__ dot_partial,
                const int* __restrict__ skip_if_zero) {
  if (skip_if_zero != nullptr && *skip_if_zero == 0) return;
  __shared__ double shd[kSiteThreads / 32];
  const int rhs = blockIdx.y;
  const int V = g.V;
  const float2* in = in_all + (size_t)rhs * 12 * V;
  float2* out = out_all + (size_t)rhs * 12 * V;
  const int s = blockIdx.x * kSiteThreads + threadIdx.x;
  double dot = 0.0;
  if (s < V) {
    float2 acc[12];
    site_hops32(lk, in, s, g, acc);
    const float mk = -(float)g.kappa;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const float sg = i < 6 ? c1 : -c1;
      const float2 p = in[i * V + s];
      float2 o;
      o.x = fmaf(sg, fmaf(mk, acc[i].x, p.x), c0 * p.x);
      o.y = fmaf(sg, fmaf(mk, acc[i].y, p.y), c0 * p.y);
      out[i * V + s] = o;
      dot += (double)p.x * o.x + (double)p.y * o.y;
    }
  }
  if (dot_partial != nullptr) {
    const double b = block_sum<kSiteThreads>(dot, shd);
    if (threadIdx.x == 0) dot_partial[(size_t)rhs * gridDim.x + blockIdx.x] = (float)b;
  }
}

// FP32 spinors, all rhs of 32 sites a block (see mrhs_block): warp w takes
// direction w, its links are loaded once for every rhs.  MinB blocks an SM.
template <typename LK, int MinB>
__global__ void __launch_bounds__(128, MinB)
wilson32m_kernel(Geometry g, LK lk, const float2* __restrict__ in_all, float2* __restrict__ out_all, int nrhs,
                 float c0, float c1, float* __restrict__ dot_partial) {
  __shared__ float2 sh[2 * 12 * 4 * 32];
  __shared__ float shred[2 * 4];
  switch (threadIdx.x >> 5) {
    case 0: mrhs_block<0>(g, lk, in_all, out_all, nrhs, c0, c1, sh, shred, dot_partial); break;
    case 1: mrhs_block<1>(g, lk, in_all, out_all, nrhs, c0, c1, sh, shred, dot_partial); break;
    case 2: mrhs_block<2>(g, lk, in_all, out_all, nrhs, c0, c1, sh, shred, dot_partial); break;
    default: mrhs_block<3>(g, lk, in_all, out_all, nrhs, c0, c1, sh, shred, dot_partial); break;
  }
}

// FP32 spinors, one thread per site and pair of rhs (see site_hops_pair);
// blockIdx.y = rhs pair; an odd last rhs is computed twice, stored once.
template <typename LK, int MinB>
__global__ void __launch_bounds__(128, MinB)
wilson32p_kernel(Geometry g, LK lk, const float2* __restrict__ in_all, float2* __restrict__ out_all, int nrhs,
                 float c0, float c1) {
  const int s = blockIdx.x * 128 + threadIdx.x;
  const int V = g.V;
  if (s >= V) return;
  const int r0 = 2 * blockIdx.y, r1 = min(r0 + 1, nrhs - 1);
  const float2* in0 = in_all + (size_t)r0 * 12 * V;
  const float2* in1 = in_all + (size_t)r1 * 12 * V;
  f32x2_t acc0[12], acc1[12];
  site_hops_pair(lk, in0, in1, s, g, acc0, acc1);
  const float mk = -(float)g.kappa;
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (q == 1 && r1 == r0) break;
    const float2* in = q ? in1 : in0;
    float2* out = out_all + (size_t)(q ? r1 : r0) * 12 * V;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      const float sg = i < 6 ? c1 : -c1;
      const float2 p = __ldg(in + i * V + s);
      const float2 d = upk2(q ? acc1[i] : acc0[i]);
      float2 o;
      o.x = fmaf(sg, fmaf(mk, d.x, p.x), c0 * p.x);
      o.y = fmaf(sg, fmaf(mk, d.y, p.y), c0 * p.y);
      out[i * V + s] = o;
    }
  }
}

// FP32 spinors in the rhs-pair layout [npair][12][V] float4 (see hop_rp):
// one thread per site and rhs pair (blockIdx.y).
template <typename LK, int MinB>
__global__ void __launch_bounds__(128, MinB)
wilson32rp_kernel(Geometry g, LK lk, const float4* __restrict__ in_all, float4* __restrict__ out_all, float c0,
                  float c1) {
  const int s = blockIdx.x * 128 + threadIdx.x;
  const int V = g.V;
  if (s >= V) return;
  const float4* in = in_all + (size_t)blockIdx.y * 12 * V;
  float4* out = out_all + (size_t)blockIdx.y * 12 * V;
  C2 acc[12];
  const Coords c = site_coords(s, g);
  hop_rp_site<0, +1>(lk, in, s, c, g, true, acc);
  hop_rp_site<0, -1>(lk, in, s, c, g, false, acc);
  hop_rp_site<1, +1>(lk, in, s, c, g, false, acc);
  hop_rp_site<1, -1>(lk, in, s, c, g, false, acc);
  hop_rp_site<2, +1>(lk, in, s, c, g, false, acc);
  hop_rp_site<2, -1>(lk, in, s, c, g, false, acc);
  hop_rp_site<3, +1>(lk, in, s, c, g, false, acc);
  hop_rp_site<3, -1>(lk, in, s, c, g, false, acc);
  const f32x2_t mk = pk2(-(float)g.kappa, -(float)g.kappa), cc0 = pk2(c0, c0);
  const f32x2_t sgu = pk2(c1, c1), sgl = pk2(-c1, -c1);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const C2 p = c2_load(in + i * V + s);
    // out = c0 p + c1 gamma5 (p - kappa D p)
    const f32x2_t sg = i < 6 ? sgu : sgl;
    const f32x2_t tre = fma2(mk, acc[i].re, p.re), tim = fma2(mk, acc[i].im, p.im);
    const float2 ore = upk2(fma2(sg, tre, mul2(cc0, p.re))), oim = upk2(fma2(sg, tim, mul2(cc0, p.im)));
    out[i * V + s] = make_float4(ore.x, ore.y, oim.x, oim.y);
  }
}

// The rhs-pair kernel with its x-y plane staged in shared memory: a block of
// 128 threads covers 128 consecutive sites, i.e. 128 / X full x-lines of one
// (z, t) plane (applicable when X divides 128 and 128 / X divides Y); the
// block's own spinors and the two neighbouring y-rows are copied into a
// shared tile first, so the x and y hops read their neighbours there (~30
// cycles instead of a global load each) and only the z and t hops go to
// global memory -- first, so that their loads overlap the staging.
// Tile rows r = 0 .. R + 1: row 0 is y0 - 1, rows 1..R the block's own,
// row R + 1 is y0 + R (periodic in y); element (r, x) at r X + x.
template <typename LK, int MinB>
__global__ void __launch_bounds__(128, MinB)
wilson32rs_kernel(Geometry g, LK lk, const float4* __restrict__ in_all, float4* __restrict__ out_all, float c0,
                  float c1) {
  extern __shared__ float4 tile[];
  const int X = g.X, Y = g.Y, V = g.V;
  const int R = 128 / X, stride = (R + 2) * X;
  const int s0 = blockIdx.x * 128, s = s0 + threadIdx.x;
  const float4* in = in_all + (size_t)blockIdx.y * 12 * V;
  float4* out = out_all + (size_t)blockIdx.y * 12 * V;
  const int plane = s0 / (X * Y), y0 = (s0 / X) % Y;  // the block's (z, t) plane and first row
#pragma unroll
  for (int comp = 0; comp < 12; ++comp) tile[comp * stride + X + threadIdx.x] = __ldg(in + comp * V + s);
  if ((int)threadIdx.x < 2 * X) {
    const bool lo = (int)threadIdx.x < X;
    const int xx = (int)threadIdx.x - (lo ? 0 : X);
    const int yy = lo ? (y0 + Y - 1) % Y : (y0 + R) % Y;
    const int site = xx + X * (yy + Y * plane);
    const int r = lo ? 0 : R + 1;
#pragma unroll
    for (int comp = 0; comp < 12; ++comp) tile[comp * stride + r * X + xx] = __ldg(in + comp * V + site);
  }
  C2 acc[12];
  const Coords c = site_coords(s, g);
  // z and t hops from global memory while the tile fills
  hop_rp_site<2, +1>(lk, in, s, c, g, true, acc);
  hop_rp_site<2, -1>(lk, in, s, c, g, false, acc);
  hop_rp_site<3, +1>(lk, in, s, c, g, false, acc);
  hop_rp_site<3, -1>(lk, in, s, c, g, false, acc);
  __syncthreads();
  const int r = 1 + (c.y - y0);
  const int xp = c.x + 1 == X ? 0 : c.x + 1, xm = c.x == 0 ? X - 1 : c.x - 1;
  hop_rp_tile<0, +1>(lk, tile, stride, r * X + xp, s, c, g, false, acc);
  hop_rp_tile<0, -1>(lk, tile, stride, r * X + xm, s, c, g, false, acc);
  hop_rp_tile<1, +1>(lk, tile, stride, (r + 1) * X + c.x, s, c, g, false, acc);
  hop_rp_tile<1, -1>(lk, tile, stride, (r - 1) * X + c.x, s, c, g, false, acc);
  const f32x2_t mk = pk2(-(float)g.kappa, -(float)g.kappa), cc0 = pk2(c0, c0);
  const f32x2_t sgu = pk2(c1, c1), sgl = pk2(-c1, -c1);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    const float4 pv = tile[i * stride + X + threadIdx.x];
    const C2 p{pk2(pv.x, pv.y), pk2(pv.z, pv.w)};
    const f32x2_t sg = i < 6 ? sgu : sgl;
    const f32x2_t tre = fma2(mk, acc[i].re, p.re), tim = fma2(mk, acc[i].im, p.im);
    const float2 ore = upk2(fma2(sg, tre, mul2(cc0, p.re))), oim = upk2(fma2(sg, tim, mul2(cc0, p.im)));
    out[i * V + s] = make_float4(ore.x, ore.y, oim.x, oim.y);
  }
}

// the staged kernel applies: X divides 128 and 128 / X divides Y
bool rs_applicable(const Geometry& g) { return g.X >= 1 && 128 % g.X == 0 && g.Y % (128 / g.X) == 0; }
size_t rs_smem(const Geometry& g) { return sizeof(float4) * 12 * (128 + 2 * g.X); }

// FP32 [nrhs][12][V] float2 <-> rhs pairs [npair][12][V] float4 (a missing
// second rhs of the last pair reads as zero and is not written back)
__global__ void to_rhs_pairs_kernel(const float2* __restrict__ a, float4* __restrict__ b, int nrhs, long long n12) {
  const long long npn = (long long)((nrhs + 1) / 2) * n12;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < npn; e += (long long)gridDim.x * blockDim.x) {
    const long long q = e / n12, k = e % n12;
    const float2 x = a[(2 * q) * n12 + k];
    const float2 y = (2 * q + 1 < nrhs) ? a[(2 * q + 1) * n12 + k] : make_float2(0.f, 0.f);
    b[e] = make_float4(x.x, y.x, x.y, y.y);
  }
}
__global__ void from_rhs_pairs_kernel(const float4* __restrict__ b, float2* __restrict__ a, int nrhs, long long n12) {
  const long long npn = (long long)((nrhs + 1) / 2) * n12;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < npn; e += (long long)gridDim.x * blockDim.x) {
    const long long q = e / n12, k = e % n12;
    const float4 v = b[e];
    a[(2 * q) * n12 + k] = make_float2(v.x, v.z);
    if (2 * q + 1 < nrhs) a[(2 * q + 1) * n12 + k] = make_float2(v.y, v.w);
  }
}

// Float-float stencil (SSQCD_DF): out = c0 in + c1 A in with float-float
// spinors and links; see wilson_df.cuh.
__global__ void __launch_bounds__(kStencilThreadsDF)
wilson_df_kernel(Geometry g, const float4* __restrict__ u, const float4* __restrict__ in_all,
                 float4* __restrict__ out_all, float2 c0, float2 c1) {
  __shared__ float4 sh[8 * 6 * 32];
  const int rhs = blockIdx.y;
  const int V = g.V;
  const float4* in = in_all + (size_t)rhs * 12 * V;
  float4* out = out_all + (size_t)rhs * 12 * V;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int s = blockIdx.x * kSitesPerBlock + lane;
  block_hops_df8(LinksDF{u, V}, in, s, g, sh);
  if (s < V) {
    (void)finish_df1(g, in, out, c0, c1, s, w, hop_sum_df(sh, w, lane));
    if (w < 4) (void)finish_df1(g, in, out, c0, c1, s, w + 8, hop_sum_df(sh, w + 8, lane));
  }
}

// FP64 <-> float-float complex arrays (same element size)
__global__ void f64_to_df_kernel(const double2* __restrict__ a, float4* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = ff::from_double2(a[i]);
}
__global__ void df_to_f64_kernel(const float4* __restrict__ a, double2* __restrict__ b, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = ff::to_double2(a[i]);
}

// FP64 links [4][9][V] -> FP32 rows 0 and 1, [4][3][V] float4
__global__ void pack_gauge32_kernel(const double2* __restrict__ u, float4* __restrict__ u32, int V) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 4LL * V) return;
  const int mu = (int)(i / V), s = (int)(i % V);
  float2 e[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const double2 z = u[(size_t)(mu * 9 + k) * V + s];
    e[k] = make_float2((float)z.x, (float)z.y);
  }
  u32[(size_t)(mu * 3 + 0) * V + s] = make_float4(e[0].x, e[0].y, e[1].x, e[1].y);
  u32[(size_t)(mu * 3 + 1) * V + s] = make_float4(e[2].x, e[2].y, e[3].x, e[3].y);
  u32[(size_t)(mu * 3 + 2) * V + s] = make_float4(e[4].x, e[4].y, e[5].x, e[5].y);
}

// FP64 links [4][9][V] -> FP16 rows 0 and 1, [4][3][V] uint2, each value
// rounded once from double
__global__ void pack_gauge16_kernel(const double2* __restrict__ u, uint2* __restrict__ u16, int V) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 4LL * V) return;
  const int mu = (int)(i / V), s = (int)(i % V);
  unsigned int h[6];
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const double2 z = u[(size_t)(mu * 9 + e) * V + s];
    __half2 hv = __halves2half2(__double2half(z.x), __double2half(z.y));
    h[e] = *reinterpret_cast<unsigned int*>(&hv);
  }
  u16[(size_t)(mu * 3 + 0) * V + s] = make_uint2(h[0], h[1]);
  u16[(size_t)(mu * 3 + 1) * V + s] = make_uint2(h[2], h[3]);
  u16[(size_t)(mu * 3 + 2) * V + s] = make_uint2(h[4], h[5]);
}

}  // namespace

int wilson_blocks(const Geometry& g) { return (g.V + kSitesPerBlock - 1) / kSitesPerBlock; }

int wilson64(const Geometry& g, const double2* u, const double2* in, double2* out, int nrhs, double c0,
             double c1, double* dot_partial, const int* skip_if_zero, cudaStream_t s) {
  if (nrhs <= 0) return SSQCD_OK;
  dim3 grid(wilson_blocks(g), nrhs);
  wilson64_kernel<<<grid, kStencilThreads, 0, s>>>(g, u, in, out, c0, c1, dot_partial, skip_if_zero);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

namespace {
using namespace wcore;

// Six variants of the FP32 stencil with 12-parameter links (kernels above):
//   0: all rhs of 32 sites a block (wilson32m), 4 blocks an SM (128 registers)
//   1: the same at 3 blocks an SM (170 registers)
//   2: one thread per site and rhs pair (wilson32p), 4 blocks an SM
//   3: the same at 3 blocks an SM
//   4: one thread per site and rhs pair, the two rhs in the lanes of the
//      paired instructions (wilson32rp, rhs-pair layout), 4 blocks an SM
//   5: the same at 3 blocks an SM
//   6: variant 4 with the block's x-y plane and its y-halo staged in shared
//      memory (wilson32rs: the x and y hops read the tile), 4 blocks an SM;
//      only where X divides 128 and 128 / X divides Y
//   7: the same at 3 blocks an SM
// Which is fastest depends on the lattice volume, the number of rhs and the
// link storage, so the first application for a (V, nrhs, link bits) key
// times each variant (three launches each, CUDA events on the caller's
// stream; variants 4-7 only for an even nrhs, on the same buffers, which
// then have the same size in the rhs-pair layout) and records the fastest;
// later applications with that key use it (variants 4-7 convert to and from
// the rhs-pair layout around the kernel).  Variants 2-7 give no (in, out)
// partials, so callers that want them tune among 0-1 only.
// ssqcd_set_stencil_variant forces one variant (tests, measurements),
// ssqcd_stencil_tuning reports the choice of a key.
constexpr int kFp32Variants = 8;

struct TuneEntry {
  int variant;
  float us[kFp32Variants];
};
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int>, TuneEntry> g_tune;
std::atomic<int> g_variant_override{-1};

template <typename LK>
void launch_fp32_variant(int v, const Geometry& g, const LK& lk, const float2* in, float2* out, int nrhs, float c0,
                         float c1, float* dot_partial, cudaStream_t s) {
  if (v <= 1) {
    const int nb = (g.V + 31) / 32;
    if (v == 0)
      wilson32m_kernel<LK, 4><<<nb, 128, 0, s>>>(g, lk, in, out, nrhs, c0, c1, dot_partial);
    else
      wilson32m_kernel<LK, 3><<<nb, 128, 0, s>>>(g, lk, in, out, nrhs, c0, c1, dot_partial);
  } else if (v <= 3) {
    const dim3 grid((g.V + 127) / 128, (nrhs + 1) / 2);
    if (v == 2)
      wilson32p_kernel<LK, 4><<<grid, 128, 0, s>>>(g, lk, in, out, nrhs, c0, c1);
    else
      wilson32p_kernel<LK, 3><<<grid, 128, 0, s>>>(g, lk, in, out, nrhs, c0, c1);
  } else {  // in, out in the rhs-pair layout
    const dim3 grid((g.V + 127) / 128, (nrhs + 1) / 2);
    const float4* a = reinterpret_cast<const float4*>(in);
    float4* b = reinterpret_cast<float4*>(out);
    if (v == 4)
      wilson32rp_kernel<LK, 4><<<grid, 128, 0, s>>>(g, lk, a, b, c0, c1);
    else if (v == 5)
      wilson32rp_kernel<LK, 3><<<grid, 128, 0, s>>>(g, lk, a, b, c0, c1);
    else if (v == 6)
      wilson32rs_kernel<LK, 4><<<grid, 128, rs_smem(g), s>>>(g, lk, a, b, c0, c1);
    else
      wilson32rs_kernel<LK, 3><<<grid, 128, rs_smem(g), s>>>(g, lk, a, b, c0, c1);
  }
}

// a forced variant where it applies: 4-7 need an even nrhs (else 2-3), 6-7
// the tile geometry (else 4-5)
int applicable_variant(int v, const Geometry& g, int nrhs) {
  if (v >= 6 && !rs_applicable(g)) v -= 2;
  if (v >= 4 && nrhs % 2 != 0) v = 2 + (v % 2);
  return v;
}

// the variant for this key: forced, recorded, or tuned now (when the
// stream is not being captured; a capturing caller gets variant 0 untimed)
template <typename LK>
int fp32_variant(const Geometry& g, const LK& lk, int bits, const float2* in, float2* out, int nrhs, float c0,
                 float c1, float* dot_partial, cudaStream_t s) {
  const int forced = g_variant_override.load();
  if (forced >= 0) {
    if (dot_partial != nullptr && forced >= 2) return 0;
    return applicable_variant(forced, g, nrhs);
  }
  const auto key = std::make_tuple(g.V, nrhs, bits, dot_partial != nullptr ? 1 : 0);
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second.variant;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return 0;
  }
  TuneEntry t{0, {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}};
  const int nv = dot_partial != nullptr ? 2 : (nrhs % 2 == 0 ? (rs_applicable(g) ? kFp32Variants : 6) : 4);
  float best = 0.f;
  for (int v = 0; v < nv; ++v) {
    launch_fp32_variant(v, g, lk, in, out, nrhs, c0, c1, dot_partial, s);  // warm-up
    cudaEventRecord(e0, s);
    for (int k = 0; k < 3; ++k) launch_fp32_variant(v, g, lk, in, out, nrhs, c0, c1, dot_partial, s);
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    t.us[v] = 1e3f * ms / 3.f;
    if (v == 0 || t.us[v] < best) {
      best = t.us[v];
      t.variant = v;
    }
  }
  count_launches(4LL * nv);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (cudaGetLastError() != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_tune[key] = t;
  return t.variant;
}

}  // namespace

int wilson32_blocks(const Geometry& g) { return (g.V + 31) / 32; }

int set_fp32_stencil_variant(int v) {
  if (v < -1 || v >= kFp32Variants) return fail(SSQCD_ERR_ARG, "stencil variant must be -1 (tuned) or 0..7");
  g_variant_override.store(v);
  return SSQCD_OK;
}

// The tuned variant's kernel alone on in, out (std layout buffers; an
// rhs-pair variant runs on them as rhs-pair buffers of the same size), for
// kernel timing.
int wilson32_kernel_only(const Geometry& g, const void* links, int link_bits, const float2* in, float2* out, int nrhs,
                         float c0, float c1, cudaStream_t s) {
  if (nrhs <= 0) return SSQCD_OK;
  const LinksF16 l16{static_cast<const uint2*>(links), g.V};
  const LinksF32 l32{static_cast<const float4*>(links), g.V};
  const int v = link_bits == 16 ? fp32_variant(g, l16, 16, in, out, nrhs, c0, c1, nullptr, s)
                                : fp32_variant(g, l32, 32, in, out, nrhs, c0, c1, nullptr, s);
  if (link_bits == 16)
    launch_fp32_variant(v, g, l16, in, out, nrhs, c0, c1, nullptr, s);
  else
    launch_fp32_variant(v, g, l32, in, out, nrhs, c0, c1, nullptr, s);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int fp32_stencil_tuning(int V, int nrhs, int link_bits, int* variant, float* us) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tune.find(std::make_tuple(V, nrhs, link_bits, 0));
  if (it == g_tune.end()) return fail(SSQCD_ERR_ARG, "no tuning recorded for this lattice size, rhs count and links");
  *variant = it->second.variant;
  for (int v = 0; v < kFp32Variants; ++v) us[v] = it->second.us[v];
  return SSQCD_OK;
}

int wilson32(const Geometry& g, const void* links, int link_bits, const float2* in, float2* out, int nrhs, float c0,
             float c1, float* dot_partial, const int* skip_if_zero, cudaStream_t s) {
  if (nrhs <= 0) return SSQCD_OK;
  if (skip_if_zero == nullptr) {
    // the tuned all-rhs variants: links loaded once for several rhs
    const LinksF16 l16{static_cast<const uint2*>(links), g.V};
    const LinksF32 l32{static_cast<const float4*>(links), g.V};
    const int v = link_bits == 16 ? fp32_variant(g, l16, 16, in, out, nrhs, c0, c1, dot_partial, s)
                                  : fp32_variant(g, l32, 32, in, out, nrhs, c0, c1, dot_partial, s);
    if (v >= 4) {
      // the rhs-pair kernel between two layout conversions
      const long long n12 = 12LL * g.V, np = (long long)((nrhs + 1) / 2) * n12;
      DevBuf ta, tb;
      SS_TRY(ta.alloc(sizeof(float4) * np));
      SS_TRY(tb.alloc(sizeof(float4) * np));
      to_rhs_pairs_kernel<<<grid_for(np, 256), 256, 0, s>>>(in, ta.as<float4>(), nrhs, n12);
      const float2* a = reinterpret_cast<const float2*>(ta.p);
      float2* b = reinterpret_cast<float2*>(tb.p);
      if (link_bits == 16)
        launch_fp32_variant(v, g, l16, a, b, nrhs, c0, c1, nullptr, s);
      else
        launch_fp32_variant(v, g, l32, a, b, nrhs, c0, c1, nullptr, s);
      from_rhs_pairs_kernel<<<grid_for(np, 256), 256, 0, s>>>(tb.as<float4>(), out, nrhs, n12);
      count_launches(3);
      SS_CHECK_LAUNCH();
      return SSQCD_OK;
    }
    if (link_bits == 16)
      launch_fp32_variant(v, g, l16, in, out, nrhs, c0, c1, dot_partial, s);
    else
      launch_fp32_variant(v, g, l32, in, out, nrhs, c0, c1, dot_partial, s);
    count_launches(1);
    SS_CHECK_LAUNCH();
    return SSQCD_OK;
  }
  dim3 grid((g.V + kSiteThreads - 1) / kSiteThreads, nrhs);
  if (link_bits == 16)
    wilson32_kernel<<<grid, kSiteThreads, 0, s>>>(g, LinksF16{static_cast<const uint2*>(links), g.V}, in, out, c0, c1,
                                                  dot_partial, skip_if_zero);
  else
    wilson32_kernel<<<grid, kSiteThreads, 0, s>>>(g, LinksF32{static_cast<const float4*>(links), g.V}, in, out, c0,
                                                  c1, dot_partial, skip_if_zero);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int wilson_df(const Geometry& g, const float4* u, const float4* in, float4* out, int nrhs, double c0, double c1,
              cudaStream_t s) {
  if (nrhs <= 0) return SSQCD_OK;
  dim3 grid(wilson_blocks(g), nrhs);
  auto split = [](double x) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
  };
  wilson_df_kernel<<<grid, kStencilThreadsDF, 0, s>>>(g, u, in, out, split(c0), split(c1));
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int convert_f64_to_df(const double2* a, float4* b, long long n, cudaStream_t s) {
  if (n <= 0) return SSQCD_OK;
  f64_to_df_kernel<<<grid_for(n, 256), 256, 0, s>>>(a, b, n);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int convert_df_to_f64(const float4* a, double2* b, long long n, cudaStream_t s) {
  if (n <= 0) return SSQCD_OK;
  df_to_f64_kernel<<<grid_for(n, 256), 256, 0, s>>>(a, b, n);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

// float-float links: the FP64 [4][9][V] array element by element
int pack_gauge_df(const double2* u64dev, float4* udf, int V, cudaStream_t s) {
  return convert_f64_to_df(u64dev, udf, 36LL * V, s);
}

int pack_gauge32(const double2* u64dev, void* u32, int V, cudaStream_t s) {
  pack_gauge32_kernel<<<grid_for(4LL * V, 256), 256, 0, s>>>(u64dev, static_cast<float4*>(u32), V);
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
