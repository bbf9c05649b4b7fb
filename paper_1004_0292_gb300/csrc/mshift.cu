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
// Two forms of the loop; every kernel finishes its reduction in its last
// block (fixed summation order, no host round trip).
//
// Update form (opts.basis = 0; the path of ssqcd_shifted_cg): per iteration
//   A. stencil q = K p for every source with block partials of (p, q); the
//      last block forms alpha_k = (r, r) / (p, q) (breakdown check);
//   B. seed update r -= alpha q with partials of ||r||^2; meanwhile the
//      blocks also form xi_{k+1} (it needs only alpha_k and older scalars),
//      one shift per block, so the FP64 divisions run on many SMs; the last
//      block forms (r_{k+1}, r_{k+1}), beta_k, the coefficients a_j, b_j and
//      the freeze test, and writes per source the ordered list of shifts to
//      update;
//   P. seed direction p = r + beta p;
//   C. fused update, on a side stream beside A, B, P of the next iteration:
//      for every listed shift y_j += a_j p-hat_j, p-hat_j = r + b_j p-hat_j.
// Krylov-basis form (default for FP64 and float-float solves): A, B, P as
// above, B writing r_{k+1} into a stored slot, and S (the shift scalars:
// xi_{k+1}, a_j, b_j into per-iteration records, the freeze test) on the
// side stream; the shift vectors are never formed -- see "Krylov-basis form"
// below.
// (A two-kernel form that obtains ||r_{k+1}||^2 from (r, r) - 2 alpha (r, q)
// + alpha^2 (q, q) was tried and rejected: on the indefinite seed the
// residual can drop by many orders in one step, the three terms cancel, and
// shifts froze on a wrong residual estimate.)
// Every piece of state has a single writer per iteration; what a side-stream
// kernel reads is double buffered by iteration parity.  Kernel A skips when
// no shift is live; the host replays a CUDA graph of 16 iterations and polls
// the live count between replays.  All reductions have a fixed order: runs
// are bit-reproducible.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <mutex>
#include <new>
#include <type_traits>
#include <utility>
#include <vector>

#include "floatfloat.cuh"
#include "wilson_core.cuh"
#include "wilson_df.cuh"

namespace ssqcd {
namespace {

using namespace wcore;

// Per-source seed state; single writer: the last block of kernel B.
struct SeedState {
  double rr;          // (r_k, r_k)
  double alpha_prev;  // alpha_{k-1}
  double beta_prev;   // beta_{k-1}
  double beta;        // beta_k (valid after kernel B of iteration k)
  double scale;       // power of two applied to p by kernel C of this iteration and to r
                      // by kernel B of the next (C reads r scaled in registers)
  double pad[3];      // pad[0] = 1 / rr, pad[1] = S = product of all scales so far
};

// Device-side control block of one solve (L sources, N shifts).  Every field
// has one writer per iteration: the last block of kernel A (alpha, ran, err,
// seed_iters) or of kernel B (everything per shift, the coefficient lists,
// the live counts); the other kernels only read.
struct Control {
  SeedState* seed;     // [L]
  double* alpha;       // [L]     alpha_k
  double* vnorm2;      // [L]
  int* live;           // [L]     shifts still iterating
  int* live_total;     // [1]
  int* ran;            // [1]     kernel A of this iteration did its work (read by B and P)
  int* rec_ran;        // [2]     the same per iteration parity (read by C, which may run
                       //         while the next iteration's A rewrites ran)
  int* err;            // [1]
  int* seed_iters;     // [2]     seed iterations, reliable updates applied
  unsigned* done;      // [2]     last-block tickets of kernels A and B
  unsigned* task_ctr;  // [2]     per parity: next task of the TMA-fed update (reset by B)
  double2* shift_s;    // [L*N]   s_j = z_j - sigma
  double2* xi_cur;     // [L*N]   xi_k
  double2* xi_prev;    // [L*N]   xi_{k-1}
  double2* xi_next;    // [L*N]   xi_{k+1}, from the blocks of kernel B
  double2* ratio;      // [L*N]   xi_{k+1} / xi_k
  int* act;            // [L*N]
  int* iters;          // [L*N]
  // the record kernel C reads, double-buffered by iteration parity: C of
  // iteration k runs beside A, B, P of iteration k + 1
  int* list_n;         // [2][L]     shifts updated in this iteration
  int* list_j;         // [2][L*N]   their indices, ascending
  double2* list_a;     // [2][L*N]   y += a p-hat
  double2* list_b;     // [2][L*N]   p-hat = r + b p-hat
  double* list_sc;     // [2][L]     scale of r (power of two) for C
  double* partial;     // [L][nbw]  (p, q) partials of kernel A
  double* partial_rr;  // [L][nbs]  ||r||^2 partials of kernel B
  double2* x;          // [L][n]    FP64 seed solution (mixed precision only, else null)
  // Krylov-basis form (null otherwise): table of the blocks that hold the
  // stored residuals and coefficient records, and the bytes of a block's
  // residual slots
  char* const* tab;
  size_t blk_vec;
  char** rptr;         // [2] slots r_k, r_{k+1} of the coming iteration (written by the last block of B)
  // Krylov-basis loop: the per-shift scalar work runs in kernel S on a side
  // stream (split = 1) from these per-parity records
  int split;
  double* alpha_rec;   // [2][L]    alpha_k (last block of A)
  double* srec;        // [2][L][4] rr_{k+1}, beta_k, scale s_k, product of the earlier scales (last block of B)
  int* srec_k;         // [2]       iteration index k
  double* sprev;       // [L][2]    alpha_{k-1}, beta_{k-1} (kernel S's own state)
};

constexpr int kUpdBlock = 256;
constexpr int kSeedBlock = 256;

// ---- Krylov-basis form ------------------------------------------------------------------
// Instead of updating y_j and p-hat_j for every live shift in every iteration
// (kernel C), the run keeps every seed residual and the coefficients a_j, b_j
// and scale of every iteration; since
//   p-hat_j(k+1) = u_k + b_j(k) p-hat_j(k),  y_j += a_j(k) p-hat_j(k),
//   p-hat_j(0) = v,  u_k = sc_k r_{k+1}  (r_{k+1} as kernel B stores it),
// the solution is a fixed combination of the stored vectors r_0 = v, r_1, ...:
//   y_j = sum_s g_j(s) scs(s) r_s,  g_j(s) = a_j(s) + b_j(s) g_j(s+1)
// for s = K_j .. 0 with g_j(K_j + 1) = 0 (K_j: the last iteration that
// updated shift j), scs(0) = 1 and scs(s) = sc_{s-1}.  The moments (Eq. 2)
// are then one combination of the stored residuals per source, formed once
// after the loop, and the loop itself is the seed recurrence alone.  The
// residuals live in blocks of kBasisBlock slots (one chunk of iterations):
//   [kBasisBlock][L][n] residuals | a [kBasisBlock][L N] | b [kBasisBlock][L N]
//   | scale [kBasisBlock][L],
// slot s in block s / kBasisBlock; the coefficient records of iteration k in
// block k / kBasisBlock.  Kernel B of iteration k reads slot k and writes slot
// k + 1, with k from the device iteration counter, so the captured chunk
// graph stays valid as the blocks grow.
constexpr int kBasisLog = 4;
constexpr int kBasisBlock = 1 << kBasisLog;

template <typename VR>
__device__ __forceinline__ VR* basis_slot(const Control& c, int s, long long Ln) {
  return reinterpret_cast<VR*>(c.tab[s >> kBasisLog]) + (long long)(s & (kBasisBlock - 1)) * Ln;
}
// which 0: a_j, 1: b_j of iteration k
__device__ __forceinline__ double2* basis_coef(const Control& c, int k, int NL, int which) {
  return reinterpret_cast<double2*>(c.tab[k >> kBasisLog] + c.blk_vec) +
         ((size_t)which * kBasisBlock + (k & (kBasisBlock - 1))) * NL;
}
__device__ __forceinline__ double* basis_scale(const Control& c, int k, int NL, int L) {
  return reinterpret_cast<double*>(c.tab[k >> kBasisLog] + c.blk_vec + (size_t)2 * kBasisBlock * NL * sizeof(double2)) +
         (size_t)(k & (kBasisBlock - 1)) * L;
}
size_t basis_block_bytes(size_t vec_bytes, int NL, int L) {
  return vec_bytes + (size_t)2 * kBasisBlock * NL * sizeof(double2) + (size_t)kBasisBlock * L * sizeof(double);
}
constexpr int kMaxShifts = 512;   // quadrature points per source
constexpr int kMaxTotal = 1024;   // (source, point) pairs in one solve
constexpr int kMaxSources = 64;

// Programmatic dependent launch (Blackwell/Hopper griddepcontrol): the chain
// kernels of the Krylov-basis loop are launched with programmatic stream
// serialisation, so a kernel's launch and block scheduling overlap the tail
// of its predecessor.  Every kernel waits for its predecessor grid to
// complete (and its writes to be visible) before it reads anything the
// predecessor wrote; a kernel launched without the attribute returns from
// the wait at once.  A block signals its dependents once its main work is
// done (a dependent grid starts only when every block has signalled or
// exited, so it never takes the place of an unscheduled block).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// The seed system usually converges far faster than the shifted ones (its
// shift sigma lies in a gap of the spectrum while the quadrature points sit
// close to eigenvalues), so ||r|| keeps shrinking -- 1e-100 and below --
// while xi grows to compensate.  Before (r, r) leaves the floating-point
// range (FP64: below 2^-400 ||v||^2; FP32 vectors: below 2^-40), r and p are
// multiplied by an exact power of two s and every xi is divided by s; y is
// unchanged and p-hat absorbs s through b (see kernels B and C).  This also
// keeps |xi|^2 and the other products of the recurrences far inside the FP64
// range, so they need no overflow guards.

// ---- initialisation ---------------------------------------------------------------
// A shift vector element from an FP64 complex: FP64, FP32 (rounded) or
// float-float (hi + lo).
__device__ __forceinline__ void put_shift(double2& d, double2 x) { d = x; }
__device__ __forceinline__ void put_shift(float2& d, double2 x) {
  d = make_float2(__double2float_rn(x.x), __double2float_rn(x.y));
}
__device__ __forceinline__ void put_shift(float4& d, double2 x) { d = ff::from_double2(x); }

template <typename VR, typename V2>
__global__ void init_vectors_kernel(const double2* __restrict__ v, VR* __restrict__ r, VR* __restrict__ p,
                                    V2* __restrict__ y, V2* __restrict__ ph, int N, long long n) {
  const int l = blockIdx.y;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double2 xd = v[l * n + e];
    VR xr;
    put_shift(xr, xd);
    V2 x;
    put_shift(x, xd);
    r[l * n + e] = xr;
    p[l * n + e] = xr;
    for (int j = 0; j < N; ++j) {
      y[((long long)l * N + j) * n + e] = V2{};
      ph[((long long)l * N + j) * n + e] = x;
    }
  }
}

// A source with ||v|| = 0 has the exact solution y = 0 and starts frozen.
__global__ void init_control_kernel(Control c, const double* __restrict__ vn2, int L, int N) {
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    // rr_0, alpha_{-1} = 1, beta_{-1} = 0, scale 1, 1 / rr_0
    c.seed[t] = SeedState{vn2[t], 1.0, 0.0, 0.0, 1.0, {vn2[t] > 0.0 ? 1.0 / vn2[t] : 0.0, 1.0, 0.0}};
    c.alpha[t] = 0.0;
    c.vnorm2[t] = vn2[t];
    c.live[t] = vn2[t] > 0.0 ? N : 0;
    c.list_n[t] = c.list_n[L + t] = 0;
    if (c.sprev != nullptr) {
      c.sprev[2 * t] = 1.0;  // alpha_{-1}
      c.sprev[2 * t + 1] = 0.0;  // beta_{-1}
    }
  }
  for (int t = threadIdx.x; t < L * N; t += blockDim.x) {
    c.xi_cur[t] = make_double2(1.0, 0.0);
    c.xi_prev[t] = make_double2(1.0, 0.0);
    c.act[t] = vn2[t / N] > 0.0 ? 1 : 0;
    c.iters[t] = 0;
  }
  if (threadIdx.x == 0) {
    int live = 0;
    for (int l = 0; l < L; ++l) live += vn2[l] > 0.0 ? N : 0;
    *c.live_total = live;
    *c.ran = 0;
    c.rec_ran[0] = c.rec_ran[1] = 0;
    *c.err = 0;
    c.seed_iters[0] = c.seed_iters[1] = 0;
    c.done[0] = c.done[1] = 0u;
    c.task_ctr[0] = c.task_ctr[1] = 0u;
  }
}

// ---- A. stencil q = K p + (p, q) partials; last block: alpha_k ---------------------
// Stencil of one block for one source: q = sigma p - gamma5 (p - kappa D p) at
// spin w's three components of site s; returns this thread's share of (p, q).
struct Stencil64 {
  static constexpr bool kThreadPerSite = false;
  static constexpr int kThreads = kStencilThreads;
  static constexpr int kSites = kSitesPerBlock;
  static constexpr int kShElems = 12 * 4 * kSitesPerBlock;
  static constexpr int kMinBlocks = 4;  // <= 128 registers (four 128-thread blocks per SM)
  const double2* __restrict__ u;
  __device__ __forceinline__ double run(const Geometry& g, const double2* __restrict__ p, double2* __restrict__ q,
                                        double sigma, int s, int w, void* shm) const {
    double2 acc[3];
    block_hops64(Links64{u, g.V}, p, s, g, static_cast<double2*>(shm), acc);
    double d = 0.0;
    if (s < g.V) {
      const double sg = w < 2 ? -1.0 : 1.0;
      const double mk = -g.kappa;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int i = 3 * w + k;
        const double2 pv = p[i * g.V + s];
        double2 o;
        o.x = fma(sg, fma(mk, acc[k].x, pv.x), sigma * pv.x);
        o.y = fma(sg, fma(mk, acc[k].y, pv.y), sigma * pv.y);
        q[i * g.V + s] = o;
        d = fma(pv.x, o.x, fma(pv.y, o.y, d));
      }
    }
    return d;
  }
};

// FP64, balanced form (16 sites per block, spin halves in half-warps); used
// by the solve loop
// MinB blocks an SM: 7 (<= 72 registers; 1064 resident blocks >= the 1024 of
// 8^4 x 4 rhs) by default, 8 (64 registers, a few spilled) for comparison
template <int MinB>
struct Stencil64h {
  static constexpr bool kThreadPerSite = false;
  static constexpr int kThreads = kStencilThreads;
  static constexpr int kSites = kSitesPerBlockH;
  static constexpr int kShElems = 12 * 4 * kSitesPerBlockH;
  static constexpr int kMinBlocks = MinB;
  const double2* __restrict__ u;
  __device__ __forceinline__ double run(const Geometry& g, const double2* __restrict__ p, double2* __restrict__ q,
                                        double sigma, int, int, void* shm) const {
    double2* sh = static_cast<double2*>(shm);
    const int s0 = blockIdx.x * kSitesPerBlockH;
    block_hops64h(Links64{u, g.V}, p, s0, g, sh);
    // finish: 16 sites x 12 components, component-major so that a warp's
    // stores are two 256-byte segments
    double d = 0.0;
    const double mk = -g.kappa;
    for (int idx = threadIdx.x; idx < 12 * kSitesPerBlockH; idx += kThreads) {
      const int comp = idx / kSitesPerBlockH, i = idx % kSitesPerBlockH;
      const int s = s0 + i;
      if (s >= g.V) continue;
      const double2* e = sh + comp * 4 * kSitesPerBlockH + i;
      double2 acc = cadd(cadd(e[0], e[kSitesPerBlockH]), cadd(e[2 * kSitesPerBlockH], e[3 * kSitesPerBlockH]));
      const double sg = comp < 6 ? -1.0 : 1.0;
      const double2 pv = p[comp * g.V + s];
      double2 o;
      if (sigma == 0.0) {  // the paper's seed shift: no sigma p term; the gamma5 sign as a negation
        const double tx = fma(mk, acc.x, pv.x), ty = fma(mk, acc.y, pv.y);
        o.x = comp < 6 ? -tx : tx;
        o.y = comp < 6 ? -ty : ty;
      } else {
        o.x = fma(sg, fma(mk, acc.x, pv.x), sigma * pv.x);
        o.y = fma(sg, fma(mk, acc.y, pv.y), sigma * pv.y);
      }
      q[comp * g.V + s] = o;
      d = fma(pv.x, o.x, fma(pv.y, o.y, d));
    }
    return d;
  }
};

// FP32 spinors (mixed precisions): one thread per site (memory-bound form)
template <typename LK>
struct Stencil32 {
  static constexpr int kThreads = kSiteThreads;
  static constexpr int kMinBlocks = 1;
  static constexpr bool kThreadPerSite = true;
  static constexpr int kSites = kSiteThreads;
  static constexpr int kShElems = 1;
  LK lk;
  __device__ __forceinline__ double run(const Geometry& g, const float2* __restrict__ p, float2* __restrict__ q,
                                        double sigma, int s, int, void*) const {
    double d = 0.0;
    if (s < g.V) {
      float2 acc[12];
      site_hops32(lk, p, s, g, acc);
      const float mk = -(float)g.kappa, sf = (float)sigma;
      float dp = 0.f;
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        const float sg = i < 6 ? -1.f : 1.f;
        const float2 pv = p[i * g.V + s];
        float2 o;
        o.x = fmaf(sg, fmaf(mk, acc[i].x, pv.x), sf * pv.x);
        o.y = fmaf(sg, fmaf(mk, acc[i].y, pv.y), sf * pv.y);
        q[i * g.V + s] = o;
        dp = fmaf(pv.x, o.x, fmaf(pv.y, o.y, dp));
      }
      d = (double)dp;
    }
    return d;
  }
};

// float-float stencil (SSQCD_DF): q = sigma p - A p, float-float share of
// (p, q); one hop per warp, 8 warps per block (wilson_df.cuh)
// MinB blocks an SM: 4 (64 registers, a few spilled) by default, which puts
// the 512 blocks of 8^4 x 4 rhs in one wave (CG iteration 45.0 us against
// 57.2 us at 3 blocks an SM, <= 85 registers, 1.12 waves); 3 for comparison
template <int MinB>
struct StencilDF {
  static constexpr bool kThreadPerSite = false;
  static constexpr int kThreads = kStencilThreadsDF;
  static constexpr int kSites = kSitesPerBlock;
  static constexpr int kShElems = 12 * 4 * kSitesPerBlock;  // 8 x 6 x 32 float4
  static constexpr int kMinBlocks = MinB;
  const float4* __restrict__ u;
  __device__ __forceinline__ double run(const Geometry& g, const float4* __restrict__ p, float4* __restrict__ q,
                                        double sigma, int s, int w, void* shm) const {
    float4* sh = static_cast<float4*>(shm);
    const int lane = threadIdx.x & 31;
    block_hops_df8(LinksDF{u, g.V}, p, s, g, sh);
    double d = 0.0;
    if (s < g.V) {
      const float2 c0 = ff::split(sigma), c1 = make_float2(-1.f, 0.f);
      float2 t = finish_df1(g, p, q, c0, c1, s, w, hop_sum_df(sh, w, lane));
      d = (double)t.x + (double)t.y;
      if (w < 4) {
        t = finish_df1(g, p, q, c0, c1, s, w + 8, hop_sum_df(sh, w + 8, lane));
        d += (double)t.x + (double)t.y;
      }
    }
    return d;
  }
};

template <typename Op, typename V2>
__global__ void __launch_bounds__(Op::kThreads, Op::kMinBlocks)
cg_stencil_kernel(Control c, int L, int par, Geometry g, Op op, double sigma, const V2* __restrict__ p_all,
                  V2* __restrict__ q_all) {
  pdl_wait();
  if (*c.err != 0 || *c.live_total == 0) {
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *c.ran = c.rec_ran[par] = 0;
    return;
  }
  constexpr int kWarps = Op::kThreads / 32;
  __shared__ double2 sh[Op::kShElems];  // the op's reduction scratch
  __shared__ double sred[kWarps];
  __shared__ double sums[kMaxSources];
  __shared__ bool s_last;
  const int l = blockIdx.y;
  const int V = g.V;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double d_pq = 0.0;
  if (c.live[l] != 0) {
    const int s = Op::kThreadPerSite ? blockIdx.x * Op::kThreads + (int)threadIdx.x
                                     : blockIdx.x * Op::kSites + lane;
    d_pq = op.run(g, p_all + (size_t)l * 12 * V, q_all + (size_t)l * 12 * V, sigma, s, w, sh);
  }
  d_pq = warp_sum(d_pq);
  if (lane == 0) sred[w] = d_pq;
  __syncthreads();
  const int nbw = gridDim.x;
  if (threadIdx.x == 0) {
    // pairwise sum of the warp partials (fixed order)
    double t = (sred[0] + sred[1]) + (sred[2] + sred[3]);
    if constexpr (kWarps == 8) t += (sred[4] + sred[5]) + (sred[6] + sred[7]);
    static_assert(kWarps == 4 || kWarps == 8, "four or eight warps");
    c.partial[(size_t)l * nbw + blockIdx.x] = t;
    pdl_trigger();
    __threadfence();
    const unsigned ticket = atomicAdd(&c.done[0], 1u);
    s_last = ticket == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // warp w sums the partials of sources w, w + kWarps, ... in a fixed order,
  // eight loads in flight a lane (this tail runs on one SM while the rest
  // of the GPU waits for alpha)
  for (int ls = w; ls < L; ls += kWarps) {
    double a = 0.0;
    for (int b0 = lane; b0 < nbw; b0 += 32 * 8) {
      double t[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int b = b0 + 32 * i;
        t[i] = b < nbw ? __ldcg(c.partial + (size_t)ls * nbw + b) : 0.0;
      }
      a += ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
    }
    a = warp_sum(a);
    if (lane == 0) sums[ls] = a;
  }
  __syncthreads();
  for (int ls = threadIdx.x; ls < L; ls += blockDim.x) {
    if (c.live[ls] == 0) continue;
    const double pq = sums[ls];
    const double rr = c.seed[ls].rr;
    if (!(fabs(pq) >= 1e-30 * rr)) {  // breakdown (also catches NaN)
      atomicExch(c.err, 1);
      continue;
    }
    c.alpha[ls] = rr / pq;
    if (c.split) c.alpha_rec[par * L + ls] = rr / pq;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool ok = *((volatile int*)c.err) == 0;
    *c.ran = c.rec_ran[par] = ok ? 1 : 0;
    if (ok) atomicAdd(c.seed_iters, 1);
    c.done[0] = 0u;
  }
}

// ---- B. seed update + all scalar recurrences -----------------------------------------
// FP64 on GB300 has a dependent-operation latency of ~64 cycles (a division
// ~630), so this kernel is written to keep FP64 dependency chains short:
//  * the blocks do r -= alpha q with two independent accumulators of ||r||^2;
//  * meanwhile lane i of the last warp of block b forms xi_{k+1} and
//    xi_{k+1}/xi_k for shifts b + i nblocks, b + (i + 32) nblocks, ... (they
//    need only alpha_k and older scalars): the divisions of different
//    shifts run in parallel lanes and SMs;
//  * the last block sums the partials, forms beta_k = rr_{k+1} / rr_k with the
//    stored reciprocal of rr_k, the coefficients a_j = alpha_k xi_{k+1} and
//    b_j = s beta_k xi_{k+1}/xi_k and the freeze test |xi|^2 rr <= tol^2 ||v||^2
//    (products only), and builds each source's ordered list of shifts with
//    warp ballots.
template <typename V2>
__global__ void __launch_bounds__(kSeedBlock)
cg_seed_kernel(Control c, int L, int N, int par, double tol2, const V2* __restrict__ r_in, V2* __restrict__ r_out,
               const V2* __restrict__ q, const V2* __restrict__ p, long long n, double rescale_below,
               double rescale_by) {
  pdl_wait();
  // the control words this block needs, loaded together (one round trip)
  const int l = blockIdx.y;
  const int ran = *c.ran, live_l = c.live[l];
  const double alpha_l = c.alpha[l], scale_l = c.seed[l].scale, spad1_l = c.seed[l].pad[1];
  if (c.tab != nullptr) {  // Krylov-basis form: this iteration's slots
    r_in = reinterpret_cast<const V2*>(c.rptr[0]);
    r_out = reinterpret_cast<V2*>(c.rptr[1]);
  }
  if (ran == 0) return;
  __shared__ double sred[kSeedBlock / 32];
  __shared__ double sums[kMaxSources];
  __shared__ double s_scale[kMaxSources], s_beta[kMaxSources];
  __shared__ double2 s_a[kMaxTotal], s_b[kMaxTotal];
  __shared__ int s_flag[kMaxTotal];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int NL = N * L;
  if (w == kSeedBlock / 32 - 1 && !c.split) {
    const int nblk = gridDim.x * gridDim.y;
    for (int qi = blockIdx.y * gridDim.x + blockIdx.x + lane * nblk; qi < NL; qi += 32 * nblk) {
      const int ls = qi / N;
      // all loads first (independent addresses), then the test
      const int lv = c.live[ls], ac = c.act[qi];
      const SeedState sd = c.seed[ls];
      const double alpha = c.alpha[ls];
      const double2 xc = c.xi_cur[qi], xp = c.xi_prev[qi], s = c.shift_s[qi];
      if (lv == 0 || !ac) continue;
      const double ap = sd.alpha_prev, bp = sd.beta_prev;
      const double inv_c = 1.0 / (xc.x * xc.x + xc.y * xc.y);  // independent of the chain below
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
      c.xi_next[qi] = xn;
      c.ratio[qi] = make_double2((xn.x * xc.x + xn.y * xc.y) * inv_c, (xn.y * xc.x - xn.x * xc.y) * inv_c);
    }
  }
  double acc0 = 0.0, acc1 = 0.0;
  if (live_l != 0) {
    const double alpha = alpha_l;
    const V2* rl = r_in + (long long)l * n;
    V2* ro = r_out + (long long)l * n;
    const V2* ql = q + (long long)l * n;
    // mixed precision: the FP64 seed solution x += alpha p / S (S: product of
    // the rescales of r and p so far), for the reliable updates
    double2* xl = c.x != nullptr ? c.x + (long long)l * n : nullptr;
    const V2* pl = p + (long long)l * n;
    const double ax = c.x != nullptr ? alpha / spad1_l : 0.0;
    using T = decltype(V2::x);
    const T af = (T)alpha;
    const T sc = (T)scale_l;  // rescale of r decided last iteration (exact power of two)
    const long long stride = (long long)gridDim.x * kSeedBlock;
    if constexpr (std::is_same<V2, float4>::value) {
      // float-float: r_out = s r_in - alpha q, ||r_out||^2 summed in float-float per thread
      const float2 naf = ff::split(-alpha);
      const float scf = (float)scale_l;
      float hs = 0.f, hl = 0.f;
      for (long long e = blockIdx.x * (long long)kSeedBlock + threadIdx.x; e < n; e += stride) {
        const float4 x1 = ff::caxpy(ff::cscale2(rl[e], scf), naf, ql[e]);
        ro[e] = x1;
        ff::norm2_acc(x1, hs, hl);
      }
      acc0 = (double)hs + (double)hl;
    } else {
      auto one = [&](long long e, double& acc) {
        V2 x0 = rl[e];
        const V2 y0 = ql[e];
        x0.x = fma(-af, y0.x, sc * x0.x);
        x0.y = fma(-af, y0.y, sc * x0.y);
        ro[e] = x0;
        const double xr = x0.x, xi = x0.y;
        acc = fma(xr, xr, fma(xi, xi, acc));
        if (xl != nullptr) {
          const V2 pv = pl[e];
          double2 xv = xl[e];
          xv.x = fma(ax, (double)pv.x, xv.x);
          xv.y = fma(ax, (double)pv.y, xv.y);
          xl[e] = xv;
        }
      };
      long long e = blockIdx.x * (long long)kSeedBlock + threadIdx.x;
      for (; e + stride < n; e += 2 * stride) {
        one(e, acc0);
        one(e + stride, acc1);
      }
      if (e < n) one(e, acc0);
    }
  }
  double acc = warp_sum(acc0 + acc1);
  if (lane == 0) sred[w] = acc;
  __syncthreads();
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
    const double t = ((sred[0] + sred[1]) + (sred[2] + sred[3])) + ((sred[4] + sred[5]) + (sred[6] + sred[7]));
    c.partial_rr[(size_t)l * nb + blockIdx.x] = t;
    pdl_trigger();
    __threadfence();
    const unsigned ticket = atomicAdd(&c.done[1], 1u);
    s_last = ticket == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  const int kb = c.tab != nullptr ? *c.seed_iters - 1 : 0;  // this iteration (Krylov-basis form)
  for (int ls = w; ls < L; ls += kSeedBlock / 32) {
    // the source's control words together with its partials
    const double pad0 = c.seed[ls].pad[0], vn2 = c.vnorm2[ls];  // pad[0] holds 1 / rr_k
    const int lv = c.live[ls];
    double a0 = 0.0, a1 = 0.0;
    int b = lane;
    for (; b + 32 < nb; b += 64) {
      a0 += __ldcg(c.partial_rr + (size_t)ls * nb + b);
      a1 += __ldcg(c.partial_rr + (size_t)ls * nb + b + 32);
    }
    if (b < nb) a0 += __ldcg(c.partial_rr + (size_t)ls * nb + b);
    const double a = warp_sum(a0 + a1);
    if (lane == 0) {
      sums[ls] = a;
      s_beta[ls] = a * pad0;
      s_scale[ls] = (lv != 0 && a < rescale_below * vn2 && a > 0.0) ? rescale_by : 1.0;
    }
  }
  if (c.tab != nullptr && threadIdx.x == 0) {  // slots of the next iteration
    const long long Ln = (long long)L * n;
    c.rptr[0] = reinterpret_cast<char*>(basis_slot<V2>(c, kb + 1, Ln));
    c.rptr[1] = reinterpret_cast<char*>(basis_slot<V2>(c, kb + 2, Ln));
  }
  __syncthreads();
  if (c.split) {
    // the seed state only; kernel S takes the shifts from this record
    for (int ls = threadIdx.x; ls < L; ls += blockDim.x) {
      const double sc = s_scale[ls];
      const SeedState sd = c.seed[ls];
      double* rec = c.srec + ((size_t)par * L + ls) * 4;
      rec[0] = sums[ls];
      rec[1] = s_beta[ls];
      rec[2] = sc;
      rec[3] = sd.pad[1];
      if (c.live[ls] != 0) {
        const double rr = sums[ls] * sc * sc;
        c.seed[ls] = SeedState{rr, c.alpha[ls], s_beta[ls], s_beta[ls], sc, {1.0 / rr, sd.pad[1] * sc, 0.0}};
      }
    }
    if (threadIdx.x == 0) {
      c.srec_k[par] = kb;
      c.done[1] = 0u;
      c.task_ctr[par] = 0u;
    }
    return;
  }
  // per shift: coefficients and the freeze test from xi_{k+1}
  for (int qi = threadIdx.x; qi < NL; qi += blockDim.x) {
    const int ls = qi / N;
    int flag = 0;
    // all loads first (independent addresses), then the test
    const int lv = c.live[ls], ac = c.act[qi];
    const double alpha = c.alpha[ls], vn2 = c.vnorm2[ls], spad1 = c.seed[ls].pad[1];
    const double2 xn = __ldcg(c.xi_next + qi), ratio = __ldcg(c.ratio + qi), xc = c.xi_cur[qi];
    if (lv != 0 && ac) {
      const double rr1 = sums[ls], beta = s_beta[ls];
      const double sc = s_scale[ls], inv_sc = sc == 1.0 ? 1.0 : 1.0 / rescale_by;
      s_a[qi] = make_double2(alpha * xn.x, alpha * xn.y);
      s_b[qi] = make_double2(sc * beta * ratio.x, sc * beta * ratio.y);
      if (c.tab != nullptr) {
        basis_coef(c, kb, NL, 0)[qi] = s_a[qi];
        basis_coef(c, kb, NL, 1)[qi] = s_b[qi];
      }
      const bool live = (xn.x * xn.x + xn.y * xn.y) * rr1 > tol2 * vn2;
      flag = live ? 2 : 1;
      c.xi_prev[qi] = make_double2(xc.x * inv_sc, xc.y * inv_sc);
      // a freezing shift leaves its unscaled xi (xi_{k+1} S, S = product of
      // the scales so far); a live one keeps it in the scale of r
      const double S = live ? inv_sc : spad1;
      c.xi_cur[qi] = make_double2(xn.x * S, xn.y * S);
      c.act[qi] = live ? 1 : 0;
      c.iters[qi] += 1;
    }
    s_flag[qi] = flag;
  }
  __syncthreads();
  // per source (one warp each): ordered list by ballots, live count, seed state
  for (int ls = w; ls < L; ls += kSeedBlock / 32) {
    int m = 0, live = 0;
    for (int j0 = 0; j0 < N; j0 += 32) {
      const int j = j0 + lane;
      const int f = j < N ? s_flag[ls * N + j] : 0;
      const unsigned upd = __ballot_sync(0xffffffffu, f != 0);
      const unsigned stay = __ballot_sync(0xffffffffu, f == 2);
      if (f) {
        const int pos = m + __popc(upd & ((1u << lane) - 1u));
        const int o = (par * L + ls) * N + pos;
        c.list_j[o] = j;
        c.list_a[o] = s_a[ls * N + j];
        c.list_b[o] = s_b[ls * N + j];
      }
      m += __popc(upd);
      live += __popc(stay);
    }
    if (lane == 0) {
      c.list_n[par * L + ls] = m;
      c.list_sc[par * L + ls] = s_scale[ls];
      if (c.tab != nullptr) basis_scale(c, kb, NL, L)[ls] = s_scale[ls];
      if (c.live[ls] != 0) {
        const double sc = s_scale[ls];
        const double rr = sums[ls] * sc * sc;
        c.seed[ls] = SeedState{rr, c.alpha[ls], s_beta[ls], s_beta[ls], sc, {1.0 / rr, c.seed[ls].pad[1] * sc, 0.0}};
      }
      c.live[ls] = live;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int ls = 0; ls < L; ++ls) tot += c.live[ls];
    *c.live_total = tot;
    c.done[1] = 0u;
    c.task_ctr[par] = 0u;
  }
}

// ---- P. seed direction p = s (r + beta p) ------------------------------------------------
// s: the power of two kernel B chose for this iteration (applied to the
// stored r by the next iteration's kernel B).  Runs on the main chain right
// after B, so the next stencil can start while kernel C still updates the
// shifts.
template <typename VR>
__global__ void __launch_bounds__(kUpdBlock)
cg_seed_p_kernel(Control c, const VR* __restrict__ r, VR* __restrict__ p, long long n) {
  pdl_wait();
  const int l = blockIdx.y;
  const int ran = *c.ran, live_l = c.live[l];
  const double scale_l = c.seed[l].scale, beta_l = c.seed[l].beta;
  if (c.tab != nullptr) r = reinterpret_cast<const VR*>(c.rptr[0]);  // r_{k+1}: kernel B advanced the slots
  if (ran == 0 || live_l == 0) return;
  const VR* rl = r + (long long)l * n;
  VR* pl = p + (long long)l * n;
  if constexpr (std::is_same<VR, float4>::value) {  // float-float
    const float scf = (float)scale_l;
    const float2 beta = ff::split(scale_l * beta_l);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
      pl[e] = ff::caxpy(ff::cscale2(rl[e], scf), beta, pl[e]);
  } else {
    using TR = decltype(VR::x);
    const TR sc = (TR)scale_l;
    const TR beta = (TR)(scale_l * beta_l);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
      const VR x = rl[e];
      VR pe = pl[e];
      pe.x = fma(beta, pe.x, sc * x.x);
      pe.y = fma(beta, pe.y, sc * x.y);
      pl[e] = pe;
    }
  }
  pdl_trigger();
}

// ---- S. shift scalars of the Krylov-basis loop (side stream) ---------------------------
// For every live shift of iteration k (record of parity par): xi_{k+1} from
// alpha_k and the older scalars, the coefficients a_j = alpha_k xi_{k+1} and
// b_j = s beta_k xi_{k+1} / xi_k into the coefficient records, the freeze
// test |xi_{k+1}|^2 rr_{k+1} <= tol^2 ||v||^2, and the live counts.  It runs
// beside P(k), A(k+1), B(k+1) of the main stream: they read the live counts
// only to skip finished work, and a count one iteration old only makes them
// do some of it once more (counts only fall).  A(k+2) waits for S(k), whose
// records (alpha_rec, srec of this parity) it and B(k+2) rewrite.  One block.
__global__ void __launch_bounds__(kSeedBlock)
cg_shift_kernel(Control c, int L, int N, int par, double tol2, double rescale_by) {
  if (c.rec_ran[par] == 0) return;
  __shared__ int s_live[kMaxSources];
  const int NL = N * L;
  const int kb = c.srec_k[par];
  for (int t = threadIdx.x; t < L; t += blockDim.x) s_live[t] = 0;
  __syncthreads();
  for (int qi = threadIdx.x; qi < NL; qi += blockDim.x) {
    const int ls = qi / N;
    const int lv = c.live[ls], ac = c.act[qi];
    const double* rec = c.srec + ((size_t)par * L + ls) * 4;
    const double rr1 = rec[0], beta = rec[1], sc = rec[2], spad1 = rec[3];
    const double alpha = c.alpha_rec[par * L + ls], ap = c.sprev[2 * ls], bp = c.sprev[2 * ls + 1];
    const double vn2 = c.vnorm2[ls];
    const double2 xc = c.xi_cur[qi], xp = c.xi_prev[qi], s = c.shift_s[qi];
    if (lv == 0 || !ac) continue;
    const double inv_c = 1.0 / (xc.x * xc.x + xc.y * xc.y);  // independent of the chain below
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
    const double2 ratio = make_double2((xn.x * xc.x + xn.y * xc.y) * inv_c, (xn.y * xc.x - xn.x * xc.y) * inv_c);
    const double inv_sc = sc == 1.0 ? 1.0 : 1.0 / rescale_by;
    basis_coef(c, kb, NL, 0)[qi] = make_double2(alpha * xn.x, alpha * xn.y);
    basis_coef(c, kb, NL, 1)[qi] = make_double2(sc * beta * ratio.x, sc * beta * ratio.y);
    const bool live = (xn.x * xn.x + xn.y * xn.y) * rr1 > tol2 * vn2;
    c.xi_prev[qi] = make_double2(xc.x * inv_sc, xc.y * inv_sc);
    // a freezing shift leaves its unscaled xi (xi_{k+1} S, S = product of
    // the scales so far); a live one keeps it in the scale of r
    const double S = live ? inv_sc : spad1;
    c.xi_cur[qi] = make_double2(xn.x * S, xn.y * S);
    c.act[qi] = live ? 1 : 0;
    c.iters[qi] += 1;
    if (live) atomicAdd(&s_live[ls], 1);
  }
  __syncthreads();
  for (int ls = threadIdx.x; ls < L; ls += blockDim.x) {
    const double* rec = c.srec + ((size_t)par * L + ls) * 4;
    basis_scale(c, kb, NL, L)[ls] = rec[2];
    if (c.live[ls] != 0) {
      c.sprev[2 * ls] = c.alpha_rec[par * L + ls];
      c.sprev[2 * ls + 1] = rec[1];
    }
    c.live[ls] = s_live[ls];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int ls = 0; ls < L; ++ls) tot += s_live[ls];
    *c.live_total = tot;
  }
}

// ---- C. fused multi-shift update -------------------------------------------------------
// Thread per EPT elements (stride blockDim) of one source; the block stages
// its source's list of shifts (the record of iteration parity par) in shared
// memory and every thread walks it, two shifts at a time, so each lane keeps
// 4 EPT loads in flight.  r (the buffer kernel B of the same iteration wrote)
// is only read, times the record's scale.  V2 = double2 (FP64 path: bound by
// the FP64 pipe) or float2 (bound by HBM).
template <typename T>
struct alignas(4 * sizeof(T)) Coef4 {
  T x, y, z, w;  // a.x, -a.y, b.x, -b.y (imaginary parts negated once per block)
};

template <typename VR, typename V2, int EPT>
__global__ void __launch_bounds__(kUpdBlock)
cg_update_kernel(Control c, int N, int par, const VR* __restrict__ r, V2* __restrict__ y, V2* __restrict__ ph,
                 long long n) {
  using T = decltype(V2::x);    // shift vectors (y, p-hat)
  using TR = decltype(VR::x);   // seed vectors (r)
  if (c.rec_ran[par] == 0) return;
  const int l = blockIdx.y, L = gridDim.y;
  const int m = c.list_n[par * L + l];
  if (m == 0) return;
  __shared__ int s_j[kMaxShifts];
  __shared__ Coef4<T> s_ab[kMaxShifts];
  __shared__ T s_ay[kMaxShifts], s_by[kMaxShifts];
  const int o = (par * L + l) * N;
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    const double2 a = c.list_a[o + t], b = c.list_b[o + t];
    s_j[t] = c.list_j[o + t];
    s_ab[t] = Coef4<T>{(T)a.x, (T)-a.y, (T)b.x, (T)-b.y};
    s_ay[t] = (T)a.y;
    s_by[t] = (T)b.y;
  }
  __syncthreads();
  const TR sc = (TR)c.list_sc[par * L + l];  // exact power of two, usually 1
  const VR* rl = r + (long long)l * n;
  V2* yl = y + (long long)l * N * n;
  V2* hl = ph + (long long)l * N * n;
  const long long chunk = (long long)kUpdBlock * EPT;
  for (long long base = blockIdx.x * chunk + threadIdx.x; base < n; base += (long long)gridDim.x * chunk) {
    V2 rv[EPT];   // s r in the shift precision
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const long long e = base + (long long)i * kUpdBlock;
      const VR x = e < n ? rl[e] : VR{0, 0};
      rv[i] = V2{(T)(sc * x.x), (T)(sc * x.y)};
    }
    int t = 0;
    for (; t + 2 <= m; t += 2) {
      const Coef4<T> c0 = s_ab[t], c1 = s_ab[t + 1];
      const T a0y = s_ay[t], b0y = s_by[t], a1y = s_ay[t + 1], b1y = s_by[t + 1];
      V2* y0 = yl + (long long)s_j[t] * n;
      V2* h0 = hl + (long long)s_j[t] * n;
      V2* y1 = yl + (long long)s_j[t + 1] * n;
      V2* h1 = hl + (long long)s_j[t + 1] * n;
      V2 yv0[EPT], hv0[EPT], yv1[EPT], hv1[EPT];
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        const long long e = base + (long long)i * kUpdBlock;
        if (e < n) {
          yv0[i] = y0[e];
          hv0[i] = h0[e];
          yv1[i] = y1[e];
          hv1[i] = h1[e];
        }
      }
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        const long long e = base + (long long)i * kUpdBlock;
        if (e < n) {
          V2 a, b;
          a.x = fma(c0.x, hv0[i].x, fma(c0.y, hv0[i].y, yv0[i].x));
          a.y = fma(c0.x, hv0[i].y, fma(a0y, hv0[i].x, yv0[i].y));
          b.x = fma(c0.z, hv0[i].x, fma(c0.w, hv0[i].y, rv[i].x));
          b.y = fma(c0.z, hv0[i].y, fma(b0y, hv0[i].x, rv[i].y));
          y0[e] = a;
          h0[e] = b;
          a.x = fma(c1.x, hv1[i].x, fma(c1.y, hv1[i].y, yv1[i].x));
          a.y = fma(c1.x, hv1[i].y, fma(a1y, hv1[i].x, yv1[i].y));
          b.x = fma(c1.z, hv1[i].x, fma(c1.w, hv1[i].y, rv[i].x));
          b.y = fma(c1.z, hv1[i].y, fma(b1y, hv1[i].x, rv[i].y));
          y1[e] = a;
          h1[e] = b;
        }
      }
    }
    if (t < m) {
      const Coef4<T> c0 = s_ab[t];
      const T a0y = s_ay[t], b0y = s_by[t];
      V2* y0 = yl + (long long)s_j[t] * n;
      V2* h0 = hl + (long long)s_j[t] * n;
#pragma unroll
      for (int i = 0; i < EPT; ++i) {
        const long long e = base + (long long)i * kUpdBlock;
        if (e < n) {
          const V2 yv = y0[e], hv = h0[e];
          V2 a, b;
          a.x = fma(c0.x, hv.x, fma(c0.y, hv.y, yv.x));
          a.y = fma(c0.x, hv.y, fma(a0y, hv.x, yv.y));
          b.x = fma(c0.z, hv.x, fma(c0.w, hv.y, rv[i].x));
          b.y = fma(c0.z, hv.y, fma(b0y, hv.x, rv[i].y));
          y0[e] = a;
          h0[e] = b;
        }
      }
    }
  }
}

// Software-pipelined form of kernel C for one element per thread: the loads
// of the next pair of shifts are issued before the current pair's FMAs, so
// each lane keeps eight 16-byte loads in flight across the pair boundary.
template <typename VR, typename V2>
__global__ void __launch_bounds__(kUpdBlock)
cg_update_pf_kernel(Control c, int N, int par, const VR* __restrict__ r, V2* __restrict__ y, V2* __restrict__ ph,
                    long long n) {
  using T = decltype(V2::x);
  if (c.rec_ran[par] == 0) return;
  const int l = blockIdx.y, L = gridDim.y;
  const int m = c.list_n[par * L + l];
  if (m == 0) return;
  __shared__ int s_j[kMaxShifts];
  __shared__ Coef4<T> s_ab[kMaxShifts];
  __shared__ T s_ay[kMaxShifts], s_by[kMaxShifts];
  const int o = (par * L + l) * N;
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    const double2 a = c.list_a[o + t], b = c.list_b[o + t];
    s_j[t] = c.list_j[o + t];
    s_ab[t] = Coef4<T>{(T)a.x, (T)-a.y, (T)b.x, (T)-b.y};
    s_ay[t] = (T)a.y;
    s_by[t] = (T)b.y;
  }
  __syncthreads();
  using TR = decltype(VR::x);
  const TR sc = (TR)c.list_sc[par * L + l];
  const VR* rl = r + (long long)l * n;
  V2* yl = y + (long long)l * N * n;
  V2* hl = ph + (long long)l * N * n;
  for (long long e = blockIdx.x * (long long)kUpdBlock + threadIdx.x; e < n; e += (long long)gridDim.x * kUpdBlock) {
    const VR x = rl[e];
    const V2 rv{(T)(sc * x.x), (T)(sc * x.y)};
    // current pair (t, t + 1) and the prefetched next pair
    V2 y0 = yl[(long long)s_j[0] * n + e], h0 = hl[(long long)s_j[0] * n + e];
    V2 y1{}, h1{};
    if (m > 1) {
      y1 = yl[(long long)s_j[1] * n + e];
      h1 = hl[(long long)s_j[1] * n + e];
    }
    for (int t = 0; t < m; t += 2) {
      V2 ny0{}, nh0{}, ny1{}, nh1{};
      if (t + 2 < m) {
        ny0 = yl[(long long)s_j[t + 2] * n + e];
        nh0 = hl[(long long)s_j[t + 2] * n + e];
      }
      if (t + 3 < m) {
        ny1 = yl[(long long)s_j[t + 3] * n + e];
        nh1 = hl[(long long)s_j[t + 3] * n + e];
      }
      {
        const Coef4<T> c0 = s_ab[t];
        const T a0y = s_ay[t], b0y = s_by[t];
        V2 a, b;
        a.x = fma(c0.x, h0.x, fma(c0.y, h0.y, y0.x));
        a.y = fma(c0.x, h0.y, fma(a0y, h0.x, y0.y));
        b.x = fma(c0.z, h0.x, fma(c0.w, h0.y, rv.x));
        b.y = fma(c0.z, h0.y, fma(b0y, h0.x, rv.y));
        yl[(long long)s_j[t] * n + e] = a;
        hl[(long long)s_j[t] * n + e] = b;
      }
      if (t + 1 < m) {
        const Coef4<T> c1 = s_ab[t + 1];
        const T a1y = s_ay[t + 1], b1y = s_by[t + 1];
        V2 a, b;
        a.x = fma(c1.x, h1.x, fma(c1.y, h1.y, y1.x));
        a.y = fma(c1.x, h1.y, fma(a1y, h1.x, y1.y));
        b.x = fma(c1.z, h1.x, fma(c1.w, h1.y, rv.x));
        b.y = fma(c1.z, h1.y, fma(b1y, h1.x, rv.y));
        yl[(long long)s_j[t + 1] * n + e] = a;
        hl[(long long)s_j[t + 1] * n + e] = b;
      }
      y0 = ny0;
      h0 = nh0;
      y1 = ny1;
      h1 = nh1;
    }
  }
}

// ---- fused update, float-float shift vectors ---------------------------------------------
// Kernel C of SSQCD_FP64_DFSHIFT: the seed vectors r, p stay FP64; y_j and
// p-hat_j are complex float-float (float4 {re.hi, im.hi, re.lo, im.lo}, 16
// bytes like an FP64 complex).  Work unit = (chunk of kUpdBlock * EPT
// elements, source, group of kDfGroup listed shifts): blockIdx = (chunk,
// source, group).  Blocks are short-lived and many (~5 waves at the 8^4
// size), so no wave runs nearly empty; r is re-read once per group (1/16 of
// the shift traffic at 8 shifts a group).
// The coefficients a_j, b_j (FP64, from kernel B) and r are split to
// float-float once per block / per element; each shift then costs two
// complex float-float multiply-adds on the FP32 pipes.
constexpr int kDfGroup = 8;

// s r as complex float-float: from FP64 (SSQCD_FP64_DFSHIFT) or float-float
// (SSQCD_DF) seed vectors
__device__ __forceinline__ float4 scaled_r(double2 x, double sc) {
  return ff::from_double2(make_double2(sc * x.x, sc * x.y));
}
__device__ __forceinline__ float4 scaled_r(float4 x, double sc) { return ff::cscale2(x, (float)sc); }

template <typename RT, int EPT>
__global__ void __launch_bounds__(kUpdBlock)
cg_update_df_kernel(Control c, int N, int par, const RT* __restrict__ r, float4* __restrict__ y,
                    float4* __restrict__ ph, long long n) {
  if (c.rec_ran[par] == 0) return;
  const int l = blockIdx.y, L = gridDim.y;
  const int m = c.list_n[par * L + l];
  const int t0 = blockIdx.z * kDfGroup, t1 = min(m, t0 + kDfGroup);
  if (t1 <= t0) return;
  __shared__ int s_j[kDfGroup];
  __shared__ float4 s_a[kDfGroup], s_b[kDfGroup];
  if (threadIdx.x < kDfGroup && t0 + (int)threadIdx.x < t1) {
    const int o = (par * L + l) * N + t0 + threadIdx.x;
    s_j[threadIdx.x] = c.list_j[o];
    s_a[threadIdx.x] = ff::from_double2(c.list_a[o]);
    s_b[threadIdx.x] = ff::from_double2(c.list_b[o]);
  }
  __syncthreads();
  const int mg = t1 - t0;
  const double sc = c.list_sc[par * L + l];  // exact power of two, usually 1
  const RT* rl = r + (long long)l * n;
  float4* yl = y + (long long)l * N * n;
  float4* hl = ph + (long long)l * N * n;
  const long long base = blockIdx.x * (long long)kUpdBlock * EPT + threadIdx.x;
  float4 rv[EPT];
#pragma unroll
  for (int i = 0; i < EPT; ++i) {
    const long long e = base + (long long)i * kUpdBlock;
    rv[i] = e < n ? scaled_r(rl[e], sc) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  int t = 0;
  for (; t + 2 <= mg; t += 2) {
    const float4 a0 = s_a[t], b0 = s_b[t], a1 = s_a[t + 1], b1 = s_b[t + 1];
    float4* y0 = yl + (long long)s_j[t] * n;
    float4* h0 = hl + (long long)s_j[t] * n;
    float4* y1 = yl + (long long)s_j[t + 1] * n;
    float4* h1 = hl + (long long)s_j[t + 1] * n;
    float4 yv0[EPT], hv0[EPT], yv1[EPT], hv1[EPT];
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const long long e = base + (long long)i * kUpdBlock;
      if (e < n) {
        yv0[i] = y0[e];
        hv0[i] = h0[e];
        yv1[i] = y1[e];
        hv1[i] = h1[e];
      }
    }
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const long long e = base + (long long)i * kUpdBlock;
      if (e < n) {
        y0[e] = ff::cfma(yv0[i], a0, hv0[i]);
        h0[e] = ff::cfma(rv[i], b0, hv0[i]);
        y1[e] = ff::cfma(yv1[i], a1, hv1[i]);
        h1[e] = ff::cfma(rv[i], b1, hv1[i]);
      }
    }
  }
  if (t < mg) {
    const float4 a0 = s_a[t], b0 = s_b[t];
    float4* y0 = yl + (long long)s_j[t] * n;
    float4* h0 = hl + (long long)s_j[t] * n;
#pragma unroll
    for (int i = 0; i < EPT; ++i) {
      const long long e = base + (long long)i * kUpdBlock;
      if (e < n) {
        const float4 yv = y0[e], hv = h0[e];
        y0[e] = ff::cfma(yv, a0, hv);
        h0[e] = ff::cfma(rv[i], b0, hv);
      }
    }
  }
}

// ---- fused update, float-float shift vectors, fed by bulk copies -----------------------
// Persistent form of the float-float kernel C: one CTA per SM with 8
// consumer warps and 1 producer warp and a ring of kTmaStages shared-memory
// stages.  A task is (source l, chunk of kTmaCh elements); the producer takes
// tasks from a per-parity counter, and for each listed shift of the task
// fills the next free stage with the y and p-hat segments of that shift
// (plus the r segment for the task's first shift) by bulk copies
// (cp.async.bulk, completion counted on the stage's mbarrier); consumer
// thread i updates elements i, i + 256, ... and writes y and p-hat back to
// global memory, then the warps release the stage.  A CTA this small leaves
// room on every SM for the blocks of the stencil and seed kernels that run
// beside it, while the stage ring keeps kTmaStages x 16 KB of loads in flight
// per SM.
// Every wait is bounded: after 1 s (device global timer; kSpinLimit polls as
// a backstop) the kernel sets c.err = 2, drains its outstanding copies
// (bounded again) and returns.  With
// producer_off set (a test of that path, SSQCD_TEST_UPDATE_STALL=1) the
// producer issues nothing, so the consumers' first wait runs out.
constexpr int kTmaConsumerWarps = 8;
constexpr int kTmaEpt = 2;  // elements per consumer thread and stage
constexpr int kTmaCh = kTmaConsumerWarps * 32 * kTmaEpt;
constexpr int kTmaStages = 4;
constexpr int kTmaThreads = (kTmaConsumerWarps + 1) * 32;
constexpr long long kSpinLimit = 1LL << 24;        // polls (backstop)
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s of device time

struct __align__(16) TmaStage {
  float4 y[kTmaCh];
  float4 h[kTmaCh];
  float4 r[kTmaCh];
};

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// true once the phase of the given parity has completed; false after
// kWaitLimitNs (or kSpinLimit polls)
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long i = 1; i < kSpinLimit; ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 255) == 0 && global_ns() - t0 > kWaitLimitNs) return false;
  }
  return false;
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

size_t tma_smem_bytes(int NL, int L) {
  return sizeof(TmaStage) * kTmaStages + 2 * kTmaStages * sizeof(unsigned long long) + kTmaStages * sizeof(int4) +
         (size_t)NL * (2 * sizeof(float4) + sizeof(int)) + (size_t)L * sizeof(int);
}

template <typename RT>
__global__ void __launch_bounds__(kTmaThreads, 1)
cg_update_tma_kernel(Control c, int N, int L, int par, const RT* __restrict__ r, float4* __restrict__ y,
                     float4* __restrict__ ph, long long n, int nchunks, int producer_off) {
  if (c.rec_ran[par] == 0) return;
  extern __shared__ __align__(128) unsigned char smem[];
  TmaStage* stage = reinterpret_cast<TmaStage*>(smem);
  unsigned long long* full = reinterpret_cast<unsigned long long*>(stage + kTmaStages);
  unsigned long long* empty = full + kTmaStages;
  int4* meta = reinterpret_cast<int4*>(empty + kTmaStages);
  const int NL = N * L;
  float4* la = reinterpret_cast<float4*>(meta + kTmaStages);
  float4* lb = la + NL;
  int* lj = reinterpret_cast<int*>(lb + NL);
  int* ln = lj + NL;
  // this iteration's record, coefficients split to float-float once
  for (int i = threadIdx.x; i < NL; i += blockDim.x) {
    const int l = i / N, t = i - l * N;
    if (t < c.list_n[par * L + l]) {
      const int o = par * NL + i;
      la[i] = ff::from_double2(c.list_a[o]);
      lb[i] = ff::from_double2(c.list_b[o]);
      lj[i] = c.list_j[o];
    }
  }
  for (int l = threadIdx.x; l < L; l += blockDim.x) ln[l] = c.list_n[par * L + l];
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTmaStages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, kTmaConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == kTmaConsumerWarps) {
    // ---- producer (one lane) ----
    if (lane != 0 || producer_off) return;
    const unsigned total = (unsigned)L * (unsigned)nchunks;
    long long s = 0;  // stages issued
    bool ok = true;
    for (;;) {
      const unsigned task = atomicAdd(c.task_ctr + par, 1u);
      if (task >= total) break;
      const int l = (int)(task / (unsigned)nchunks), ch = (int)(task % (unsigned)nchunks);
      const int m = ln[l];
      const long long e0 = (long long)ch * kTmaCh;
      const unsigned cnt = (unsigned)min((long long)kTmaCh, n - e0);
      for (int t = 0; t < m && ok; ++t, ++s) {
        const int slot = (int)(s % kTmaStages);
        if (s >= kTmaStages) ok = mbar_wait(empty + slot, (unsigned)((s / kTmaStages + 1) & 1));
        if (!ok) break;
        meta[slot] = make_int4(l, ch, t, (int)cnt);
        const long long off = ((long long)l * N + lj[l * N + t]) * n + e0;
        mbar_arrive_tx(full + slot, (t == 0 ? 3u : 2u) * cnt * 16u);
        bulk_load(stage[slot].y, y + off, cnt * 16u, full + slot);
        bulk_load(stage[slot].h, ph + off, cnt * 16u, full + slot);
        if (t == 0) bulk_load(stage[slot].r, r + (long long)l * n + e0, cnt * 16u, full + slot);
      }
      if (!ok) break;
    }
    if (ok) {  // end marker for the consumers
      const int slot = (int)(s % kTmaStages);
      if (s >= kTmaStages) ok = mbar_wait(empty + slot, (unsigned)((s / kTmaStages + 1) & 1));
      if (ok) {
        meta[slot] = make_int4(-1, 0, 0, 0);
        mbar_arrive(full + slot);
      }
    }
    if (!ok) {
      atomicExch(c.err, 2);
      // let the copies already issued land before the CTA can exit
      for (long long q = s - 1; q >= 0 && q >= s - kTmaStages; --q)
        (void)mbar_wait(full + (int)(q % kTmaStages), (unsigned)((q / kTmaStages) & 1));
    }
    return;
  }
  // ---- consumers: thread i <-> elements i + 256 e of the chunk ----
  constexpr int kConsumers = kTmaConsumerWarps * 32;
  const int i = threadIdx.x;
  float4 rv[kTmaEpt];
#pragma unroll
  for (int e = 0; e < kTmaEpt; ++e) rv[e] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long s = 0;; ++s) {
    const int slot = (int)(s % kTmaStages);
    if (!mbar_wait(full + slot, (unsigned)((s / kTmaStages) & 1))) {
      atomicExch(c.err, 2);
      return;
    }
    const int4 mt = meta[slot];
    if (mt.x < 0) return;
    const int l = mt.x, t = mt.z;
    const int q = l * N + t;
    const float4 a = la[q], b = lb[q];
    if (t == 0) {
      const double sc = c.list_sc[par * L + l];
#pragma unroll
      for (int e = 0; e < kTmaEpt; ++e)
        if (i + e * kConsumers < mt.w)
          rv[e] = scaled_r(reinterpret_cast<const RT*>(stage[slot].r)[i + e * kConsumers], sc);
    }
    const long long base = ((long long)l * N + lj[q]) * n + (long long)mt.y * kTmaCh + i;
    float4 yv[kTmaEpt], hv[kTmaEpt];
#pragma unroll
    for (int e = 0; e < kTmaEpt; ++e)
      if (i + e * kConsumers < mt.w) {
        yv[e] = stage[slot].y[i + e * kConsumers];
        hv[e] = stage[slot].h[i + e * kConsumers];
      }
#pragma unroll
    for (int e = 0; e < kTmaEpt; ++e)
      if (i + e * kConsumers < mt.w) {
        y[base + e * kConsumers] = ff::cfma(yv[e], a, hv[e]);
        ph[base + e * kConsumers] = ff::cfma(rv[e], b, hv[e]);
      }
    __syncwarp();
    if (lane == 0) mbar_arrive(empty + slot);
  }
}

// In-place conversion of float-float solutions to FP64 (same element size).
__global__ void df_to_f64_kernel(float4* __restrict__ y, long long count) {
  double2* out = reinterpret_cast<double2*>(y);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    out[e] = ff::to_double2(y[e]);
}

// ---- reliable update (mixed precision) -------------------------------------------------
// r = S (v - K x) from the FP64 seed solution x and kx = K x (FP64 stencil),
// replacing the FP32 recursive residual while ||r|| is above sqrt(floor2)
// ||v||.  Below that, the true residual of the FP64 operator is dominated by
// the difference between it and the reduced-precision operator the
// recursion uses (~3e-4 relative with FP16 links, ~1e-7 with FP32 links), and
// replacing r would break the Krylov recurrence the shifted systems are
// built on; the last block stores (r, r) and its reciprocal.  The stored r is
// divided by the scale chosen in the last iteration, which kernel B applies.
template <typename V2>
__global__ void __launch_bounds__(kSeedBlock)
cg_reliable_kernel(Control c, int L, const double2* __restrict__ v, const double2* __restrict__ kx,
                   V2* __restrict__ r, long long n, double floor2) {
  __shared__ double sred[kSeedBlock / 32];
  __shared__ bool s_last;
  const int l = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const SeedState sd = c.seed[l];
  const double S = sd.pad[1];
  const double inv_pending = 1.0 / sd.scale;  // kernel B applies sd.scale to the stored r
  const bool apply = c.live[l] != 0 && sd.rr > floor2 * S * S * c.vnorm2[l];
  double acc = 0.0;
  if (apply) {
    using T = decltype(V2::x);
    const double2* vl = v + (long long)l * n;
    const double2* kl = kx + (long long)l * n;
    V2* rl = r + (long long)l * n;
    for (long long e = blockIdx.x * (long long)kSeedBlock + threadIdx.x; e < n; e += (long long)gridDim.x * kSeedBlock) {
      const double2 a = vl[e], b = kl[e];
      const double tx = S * (a.x - b.x), ty = S * (a.y - b.y);
      rl[e] = V2{(T)(tx * inv_pending), (T)(ty * inv_pending)};
      acc = fma(tx, tx, fma(ty, ty, acc));
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) sred[w] = acc;
  __syncthreads();
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
    const double t = ((sred[0] + sred[1]) + (sred[2] + sred[3])) + ((sred[4] + sred[5]) + (sred[6] + sred[7]));
    c.partial_rr[(size_t)l * nb + blockIdx.x] = t;
    __threadfence();
    const unsigned ticket = atomicAdd(&c.done[1], 1u);
    s_last = ticket == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int ls = w; ls < L; ls += kSeedBlock / 32) {
    const SeedState sl = c.seed[ls];
    const bool ap = c.live[ls] != 0 && sl.rr > floor2 * sl.pad[1] * sl.pad[1] * c.vnorm2[ls];
    double a = 0.0;
    for (int b = lane; b < nb; b += 32) a += __ldcg(c.partial_rr + (size_t)ls * nb + b);
    a = warp_sum(a);
    if (lane == 0 && ap && a > 0.0) {
      SeedState sn = sl;
      sn.rr = a;
      sn.pad[0] = 1.0 / a;
      c.seed[ls] = sn;
      atomicAdd(c.seed_iters + 1, 1);  // reliable-update counter
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) c.done[1] = 0u;
}

// ---- Krylov-basis form: coefficients and the combination of stored residuals ----------
// g_j(s) scs(s) for every (source, shift) pair, one thread each: the backward
// recurrence g_j(s) = a_j(s) + b_j(s) g_j(s+1) from s = K_j = iters_j - 1
// (zero above); gam [L N][S].
__global__ void basis_gamma_kernel(Control c, int L, int N, int S, double2* __restrict__ gam) {
  const int qi = blockIdx.x * blockDim.x + threadIdx.x;
  const int NL = N * L;
  if (qi >= NL) return;
  const int l = qi / N;
  const int K = c.iters[qi] - 1;
  double2* gq = gam + (size_t)qi * S;
  for (int s = S - 1; s > K; --s) gq[s] = make_double2(0.0, 0.0);
  // the recurrence is a chain of dependent FMAs (64 cycles each); the loads
  // of the coefficients it needs are independent of it, so they are issued
  // kG steps ahead
  constexpr int kG = 8;
  double gx = 0.0, gy = 0.0;
  for (int s1 = K; s1 >= 0; s1 -= kG) {
    double2 a[kG], b[kG];
    double sc[kG];
#pragma unroll
    for (int i = 0; i < kG; ++i) {
      const int s = s1 - i;
      if (s >= 0) {
        a[i] = basis_coef(c, s, NL, 0)[qi];
        b[i] = basis_coef(c, s, NL, 1)[qi];
        sc[i] = s == 0 ? 1.0 : basis_scale(c, s - 1, NL, L)[l];
      }
    }
#pragma unroll
    for (int i = 0; i < kG; ++i) {
      const int s = s1 - i;
      if (s >= 0) {
        const double nx = fma(b[i].x, gx, fma(-b[i].y, gy, a[i].x));
        const double ny = fma(b[i].x, gy, fma(b[i].y, gx, a[i].y));
        gx = nx;
        gy = ny;
        gq[s] = make_double2(gx * sc[i], gy * sc[i]);
      }
    }
  }
}

// Coefficients of p-hat_j after k iterations for the shifts still live:
// p-hat_j(k) = sum_{s <= k} (prod_{m=s}^{k-1} b_j(m)) scs(s) r_s; zero for
// frozen shifts (their p-hat is never used again); P [L N][S].
__global__ void basis_phat_kernel(Control c, int L, int N, int k, int S, double2* __restrict__ P) {
  const int qi = blockIdx.x * blockDim.x + threadIdx.x;
  const int NL = N * L;
  if (qi >= NL) return;
  const int l = qi / N;
  const bool live = c.act[qi] != 0;
  double2* pq = P + (size_t)qi * S;
  double px = 1.0, py = 0.0;
  for (int s = S - 1; s >= 0; --s) {
    if (!live || s > k) {
      pq[s] = make_double2(0.0, 0.0);
      continue;
    }
    const double sc = s == 0 ? 1.0 : basis_scale(c, s - 1, NL, L)[l];
    pq[s] = make_double2(px * sc, py * sc);
    if (s > 0) {
      const double2 b = basis_coef(c, s - 1, NL, 1)[qi];
      const double nx = b.x * px - b.y * py, ny = b.x * py + b.y * px;
      px = nx;
      py = ny;
    }
  }
}

// Moment coefficients of one window: G[l][m][s] = sum_j W[j][m] gam[l][j][s]
// (j ascending: a fixed order).
__global__ void basis_window_kernel(const double2* __restrict__ gam, const double2* __restrict__ W, int N, int M,
                                    int L, int S, double2* __restrict__ G) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)L * M * S) return;
  const int s = (int)(t % S);
  const int m = (int)((t / S) % M);
  const int l = (int)(t / ((long long)S * M));
  double re = 0.0, im = 0.0;
  for (int j = 0; j < N; ++j) {
    const double2 w = W[j * M + m], g = gam[((size_t)l * N + j) * S + s];
    re = fma(w.x, g.x, fma(-w.y, g.y, re));
    im = fma(w.x, g.y, fma(w.y, g.x, im));
  }
  G[t] = make_double2(re, im);
}

__device__ __forceinline__ double2 to_d2(double2 x) { return x; }
__device__ __forceinline__ double2 to_d2(float4 x) { return ff::to_double2(x); }
__device__ __forceinline__ void put_out(double2& d, double2 x) { d = x; }
__device__ __forceinline__ void put_out(float4& d, double2 x) { d = ff::from_double2(x); }
__device__ __forceinline__ void put_out(float2& d, double2 x) {
  d = make_float2(__double2float_rn(x.x), __double2float_rn(x.y));
}

// out[l][o][e] = sum_{s < count[l]} C[l][o][s] r_s[l][e] for O outputs per
// source, kCombOut of them per block (grid.z): every thread keeps the
// accumulators of kCombOut outputs for one element and streams the stored
// residuals of its source once; the coefficients of kCombTile slots at a
// time sit in shared memory.  The complex products use three real
// multiplications (Gauss): with x = xr + i xi and w = wr + i wi,
//   Re(w x) = wr xr - wi xi,  Im(w x) = (wr + wi)(xr + xi) - wr xr - wi xi,
// accumulated as the three real sums A1 = sum wr xr, A2 = sum wi xi,
// A3 = sum (wr + wi)(xr + xi): 3 FMA per term instead of 4 (the kernel is
// bound by the FP64 pipe).  The imaginary part's rounding error is within a
// few units of 2^-53 (|A1| + |A2| + |A3|), the order of that of the direct
// product sum relative to sum |w| |x|.
constexpr int kCombOut = 8;
constexpr int kCombTile = 32;
// small blocks: the work per element is uniform, so the per-SM load is even
// only when blocks are small against it (8^4 x 4 sources: 3072 blocks of 64
// threads, ~20 an SM, against 768 of 256 filling 2.5 waves of 2 an SM)
constexpr int kCombThreads = 64;

// RC (real coefficients): only Re C is used, 2 FMA a term (Re and Im of the
// residual times the real coefficient).  The moments of a contour whose
// points and weights come in conjugate pairs (z, w), (conj z, conj w) have
// real coefficients: the seed's CG scalars are real (Hermitian A, real seed
// shift), so each shift's Krylov coefficients are rational functions of the
// shift with real coefficients, the pair's coefficients are conjugate, and
// the two terms of a pair sum to twice the real part.  Im C is then rounding
// noise of the sum over the points and is dropped.
template <typename VR, typename VO, int OUT, bool RC>
__global__ void __launch_bounds__(kCombThreads, 2)
basis_combine_kernel(char* const* __restrict__ tab, long long n, int L, const double2* __restrict__ C, int O, int S,
                     const int* __restrict__ count, VO* __restrict__ out, int l0) {
  __shared__ double s_w[RC ? 1 : 3][kCombTile][OUT];
  __shared__ const VR* s_p[kCombTile];
  const int l = blockIdx.y + l0, o0 = blockIdx.z * OUT;
  const int no = min(OUT, O - o0);
  const int Sl = count[l];
  const long long e = blockIdx.x * (long long)kCombThreads + threadIdx.x;
  const long long Ln = (long long)L * n;
  double a1[OUT], a2[OUT], a3[RC ? 1 : OUT];
#pragma unroll
  for (int o = 0; o < OUT; ++o) a1[o] = a2[o] = 0.0;
#pragma unroll
  for (int o = 0; o < (RC ? 1 : OUT); ++o) a3[o] = 0.0;
  for (int s0 = 0; s0 < Sl; s0 += kCombTile) {
    const int ns = min(kCombTile, Sl - s0);
    __syncthreads();
    for (int t = threadIdx.x; t < kCombTile * OUT; t += kCombThreads) {
      const int ss = t / OUT, oo = t % OUT;
      const double2 c = (ss < ns && oo < no) ? C[((size_t)l * O + o0 + oo) * S + s0 + ss] : make_double2(0.0, 0.0);
      s_w[0][ss][oo] = c.x;
      if (!RC) {
        s_w[RC ? 0 : 1][ss][oo] = c.y;
        s_w[RC ? 0 : 2][ss][oo] = c.x + c.y;
      }
    }
    if (threadIdx.x < kCombTile) {
      const int s = s0 + threadIdx.x;
      s_p[threadIdx.x] = threadIdx.x < ns ? reinterpret_cast<const VR*>(tab[s >> kBasisLog]) +
                                                (long long)(s & (kBasisBlock - 1)) * Ln + (long long)l * n
                                          : nullptr;
    }
    __syncthreads();
    if (e < n) {
#pragma unroll 4
      for (int ss = 0; ss < ns; ++ss) {
        const double2 x = to_d2(s_p[ss][e]);
        if (RC) {
#pragma unroll
          for (int o = 0; o < OUT; ++o) {
            a1[o] = fma(s_w[0][ss][o], x.x, a1[o]);
            a2[o] = fma(s_w[0][ss][o], x.y, a2[o]);
          }
        } else {
          const double xs = x.x + x.y;
#pragma unroll
          for (int o = 0; o < OUT; ++o) {
            a1[o] = fma(s_w[0][ss][o], x.x, a1[o]);
            a2[o] = fma(s_w[RC ? 0 : 1][ss][o], x.y, a2[o]);
            a3[RC ? 0 : o] = fma(s_w[RC ? 0 : 2][ss][o], xs, a3[RC ? 0 : o]);
          }
        }
      }
    }
  }
  if (e < n) {
#pragma unroll
    for (int o = 0; o < OUT; ++o)
      if (o < no)
        put_out(out[((size_t)l * O + o0 + o) * n + e],
                RC ? make_double2(a1[o], a2[o]) : make_double2(a1[o] - a2[o], (a3[RC ? 0 : o] - a1[o]) - a2[o]));
  }
}

// The same combination for float-float residuals (SSQCD_DF runs), on the
// FP32 pipes: within a tile of TILE slots each output accumulates c += w r
// in float-float, then the tile's sums enter FP64 accumulators, so at most
// TILE terms share a float-float sum (rounding ~TILE 2^-48 of their
// magnitudes, against the residuals' own 2^-48).  The FP64 pipe (1/64 of the
// FP32 rate) only sees the per-tile conversions, but every warp reaches them
// at once after the tile's barrier, so they are kept rare: real coefficients
// (RC, as in basis_combine_kernel) take tiles of 128 slots and come as
// float-float pairs from coef_real_to_ff_kernel (one FP64 split per
// coefficient and solve, not per block); complex ones tiles of kCombTile,
// split per tile.  The complex float-float multiply-adds run on register
// pairs (real and imaginary part in one paired instruction, floatfloat.cuh
// p_cfma), in the operation order of ff::cfma; RC: one float-float
// multiply-add a part, both parts in one paired instruction (ff::p_rfma).
constexpr int kCombTileRC = 128;

// cr[i] = (hi, lo) of Re c[i] as float-float
__global__ void coef_real_to_ff_kernel(const double2* __restrict__ c, long long count, float2* __restrict__ cr) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < count) cr[i] = ff::split(c[i].x);
}

template <int OUT, bool RC, int TILE>
__global__ void __launch_bounds__(kCombThreads, 2)
basis_combine_df_kernel(char* const* __restrict__ tab, long long n, int L, const double2* __restrict__ C,
                        const float2* __restrict__ Cr, int O, int S, const int* __restrict__ count,
                        double2* __restrict__ out, int l0) {
  // coefficients as the four register pairs of ff::p_cfma (real part in lane
  // 0, imaginary part in lane 1: one paired instruction for both); RC: the
  // pairs (hi, hi) and (lo, lo) of the real coefficient
  __shared__ ff::PCoef s_w[RC ? 1 : TILE][OUT];
  __shared__ f32x2_t s_rh[RC ? TILE : 1][OUT], s_rl[RC ? TILE : 1][OUT];
  __shared__ const float4* s_p[TILE];
  const int l = blockIdx.y + l0, o0 = blockIdx.z * OUT;
  const int no = min(OUT, O - o0);
  const int Sl = count[l];
  const long long e = blockIdx.x * (long long)kCombThreads + threadIdx.x;
  const long long Ln = (long long)L * n;
  double2 accd[OUT];
#pragma unroll
  for (int o = 0; o < OUT; ++o) accd[o] = make_double2(0.0, 0.0);
  for (int s0 = 0; s0 < Sl; s0 += TILE) {
    const int ns = min(TILE, Sl - s0);
    __syncthreads();
    for (int t = threadIdx.x; t < TILE * OUT; t += kCombThreads) {
      const int ss = t / OUT, oo = t % OUT;
      if (RC) {
        const float2 r = (ss < ns && oo < no) ? Cr[((size_t)l * O + o0 + oo) * S + s0 + ss] : make_float2(0.f, 0.f);
        s_rh[RC ? ss : 0][oo] = pk2(r.x, r.x);
        s_rl[RC ? ss : 0][oo] = pk2(r.y, r.y);
      } else {
        const double2 c = (ss < ns && oo < no) ? C[((size_t)l * O + o0 + oo) * S + s0 + ss] : make_double2(0.0, 0.0);
        s_w[RC ? 0 : ss][oo] = ff::p_coef(ff::from_double2(c));
      }
    }
    for (int t = threadIdx.x; t < TILE; t += kCombThreads) {
      const int s = s0 + t;
      s_p[t] = t < ns ? reinterpret_cast<const float4*>(tab[s >> kBasisLog]) + (long long)(s & (kBasisBlock - 1)) * Ln +
                            (long long)l * n
                      : nullptr;
    }
    __syncthreads();
    if (e < n) {
      f32x2_t ah[OUT], al[OUT];
#pragma unroll
      for (int o = 0; o < OUT; ++o) ah[o] = al[o] = 0ull;
#pragma unroll 2
      for (int ss = 0; ss < ns; ++ss) {
        const ff::PVal x = ff::p_val(s_p[ss][e]);
        if (RC) {
#pragma unroll
          for (int o = 0; o < OUT; ++o) ff::p_rfma(ah[o], al[o], s_rh[RC ? ss : 0][o], s_rl[RC ? ss : 0][o], x);
        } else {
#pragma unroll
          for (int o = 0; o < OUT; ++o) ff::p_cfma(ah[o], al[o], s_w[RC ? 0 : ss][o], x);
        }
      }
#pragma unroll
      for (int o = 0; o < OUT; ++o) {
        const double2 t = ff::to_double2(ff::make2(ah[o], al[o]));
        accd[o].x += t.x;
        accd[o].y += t.y;
      }
    }
  }
  if (e < n)
    for (int o = 0; o < no; ++o) out[((size_t)l * O + o0 + o) * n + e] = accd[o];
}

// sources [l0, l0 + nl) of L (all by default); rc: real coefficients
template <typename VR, typename VO>
int launch_combine(char* const* tab, long long n, int L, const double2* C, int O, int S, const int* count, VO* out,
                   cudaStream_t st, int l0 = 0, int nl = -1, bool rc = false) {
  if (nl < 0) nl = L - l0;
  // outputs a thread accumulates: 16 when there are at least 16 (a
  // 16-moment window reads the residuals once instead of twice, 48
  // accumulators a thread; headline workload: moments 6.17 against 6.26 s,
  // bit-identical sums), else 8; SSQCD_COMB_OUT=8 forces 8 for comparison
  static const int out_per_thread = [] {
    const char* e = std::getenv("SSQCD_COMB_OUT");
    return (e != nullptr && std::atoi(e) == 8) ? 8 : 16;
  }();
  const int per = (out_per_thread == 16 && O >= 16) ? 16 : kCombOut;
  const dim3 grid((unsigned)((n + kCombThreads - 1) / kCombThreads), nl, (O + per - 1) / per);
  if (per == 16 && rc)
    basis_combine_kernel<VR, VO, 16, true><<<grid, kCombThreads, 0, st>>>(tab, n, L, C, O, S, count, out, l0);
  else if (per == 16)
    basis_combine_kernel<VR, VO, 16, false><<<grid, kCombThreads, 0, st>>>(tab, n, L, C, O, S, count, out, l0);
  else if (rc)
    basis_combine_kernel<VR, VO, kCombOut, true><<<grid, kCombThreads, 0, st>>>(tab, n, L, C, O, S, count, out, l0);
  else
    basis_combine_kernel<VR, VO, kCombOut, false><<<grid, kCombThreads, 0, st>>>(tab, n, L, C, O, S, count, out, l0);
  SS_CHECK_LAUNCH();
  count_launches(1);
  return SSQCD_OK;
}

// Kernel launch with a scheduling priority (cudaLaunchAttributePriority; kept
// as a node attribute when captured into a graph).  The main chain A, B, P
// runs at the device's greatest priority so that its blocks are dispatched
// ahead of the remaining blocks of the concurrent shift update C.
// pdl: programmatic dependent launch on the previous kernel of the stream.
template <typename... KArgs, typename... Args>
void launch_prio_smem(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int prio,
                      bool pdl, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  attr[0].id = cudaLaunchAttributePriority;
  attr[0].val.priority = prio;
  attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 2 : 1;
  cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}
template <typename... KArgs, typename... Args>
void launch_prio(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, int prio, Args&&... args) {
  launch_prio_smem(kern, grid, block, 0, st, prio, false, std::forward<Args>(args)...);
}
template <typename... KArgs, typename... Args>
void launch_chain(void (*kern)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, int prio, bool pdl,
                  Args&&... args) {
  launch_prio_smem(kern, grid, block, 0, st, prio, pdl, std::forward<Args>(args)...);
}

// Programmatic dependent launch of the chain kernels in the Krylov-basis
// loop: off by default (measured 59.7 us per iteration without, 65.6 with,
// on the 8^4 x 4 workload); SSQCD_PDL=1 turns it on for comparison runs.
bool use_pdl() {
  static const bool v = [] {
    const char* e = std::getenv("SSQCD_PDL");
    return e && e[0] == '1';
  }();
  return v;
}

// Blocks per SM of the loop's stencil (register cap), SSQCD_STENCIL_MINB for
// comparison runs: 0 = the default of each form.
int stencil_minb() {
  static const int v = [] {
    const char* e = std::getenv("SSQCD_STENCIL_MINB");
    return e ? std::atoi(e) : 0;
  }();
  return v;
}

// The FP64 stencil of the solve loop: the balanced 16-site form (default) or
// the 32-site form (SSQCD_STENCIL_SITES=32, for comparison runs).
bool balanced_stencil() {
  static const bool v = [] {
    const char* e = std::getenv("SSQCD_STENCIL_SITES");
    return !(e && std::atoi(e) == 32);
  }();
  return v;
}

// Resident blocks an SM the seed direction kernel P aims at (256 threads,
// striding over its source): 2 for lattices whose vectors sit in L2 (8^4 x
// 4), 8 when the L vectors hold more than 2^21 elements and P streams from
// HBM (more loads in flight; 16^3 x 32 x 2 sources: 40 -> 32 us).
long long seed_blocks_per_sm(long long n, int L) { return n * L > (1LL << 21) ? 8 : 2; }

// Blocks per source of kernel P (it strides): seed_blocks_per_sm over all
// sources by default (8^4 x 4: 50.3 against 50.6 us an iteration with one
// element per thread and two blocks an SM); SSQCD_P_BLOCKS sets the cap for
// tuning runs.
unsigned p_blocks(long long n, int L) {
  static const long long env = [] {
    const char* e = std::getenv("SSQCD_P_BLOCKS");
    const long long v = e ? std::atoll(e) : 0;
    return v > 0 ? v : 0LL;
  }();
  const long long cap = env > 0 ? env : (152LL * seed_blocks_per_sm(n, L) + L - 1) / L;
  long long b = (n + kUpdBlock - 1) / kUpdBlock;
  if (b > cap) b = cap;
  return (unsigned)(b < 1 ? 1 : b);
}

int seed_blocks(long long n, int L) {
  static const int ept = [] {  // SSQCD_SEED_EPT: elements per thread (tuning runs)
    const char* e = std::getenv("SSQCD_SEED_EPT");
    const int v = e ? std::atoi(e) : 0;
    return (v >= 1 && v <= 64) ? v : 2;  // measured (8^4 x 4, stored-residual loop): 2 -> 51.9, 4 -> 53.3 us an iteration
  }();
  long long b = (n + (long long)ept * kSeedBlock - 1) / ((long long)ept * kSeedBlock);
  // B ends in a last-block reduction over its blocks' partials: two blocks
  // an SM at every size (16^3 x 32 x 2 sources: 62 us an iteration at two,
  // 67 at eight)
  const long long cap = (152LL * 2 + L - 1) / L;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// Elements per thread of the update kernel: 1 for FP64 shift vectors (the
// FP64 pipe, not memory, is the limit; measured 1 > 2 > 4), 2 for the
// memory-bound FP32 and float-float ones.  The environment variable
// SSQCD_UPDATE_EPT overrides it for tuning runs.
int update_epts(bool memory_bound) {
  static int v = [] {
    const char* e = std::getenv("SSQCD_UPDATE_EPT");
    const int x = e ? std::atoi(e) : 0;
    return (x == 1 || x == 2 || x == 4) ? x : 0;
  }();
  return v != 0 ? v : (memory_bound ? 2 : 1);
}

// One element per thread uses the software-pipelined kernel (3% faster on
// the FP64 path, whose pipe it keeps 94% busy); SSQCD_UPDATE_PREFETCH=0
// selects the plain loop for comparison runs.
bool use_prefetch_update() {
  static const bool v = [] {
    const char* e = std::getenv("SSQCD_UPDATE_PREFETCH");
    return !(e && e[0] == '0');
  }();
  return v;
}

template <typename VR, typename V2>
void launch_update(int ept, dim3 grid, cudaStream_t st, int prio, const Control& c, int N, int par, const VR* r,
                   V2* y, V2* ph, long long n) {
  if (ept == 1 && use_prefetch_update()) {
    launch_prio(cg_update_pf_kernel<VR, V2>, grid, kUpdBlock, st, prio, c, N, par, r, y, ph, n);
    return;
  }
  switch (ept) {
    case 1: launch_prio(cg_update_kernel<VR, V2, 1>, grid, kUpdBlock, st, prio, c, N, par, r, y, ph, n); break;
    case 2: launch_prio(cg_update_kernel<VR, V2, 2>, grid, kUpdBlock, st, prio, c, N, par, r, y, ph, n); break;
    default: launch_prio(cg_update_kernel<VR, V2, 4>, grid, kUpdBlock, st, prio, c, N, par, r, y, ph, n); break;
  }
}

template <typename RT>
void launch_update_df(int ept, int L, cudaStream_t st, int prio, const Control& c, int N, int par, const RT* r,
                      float4* y, float4* ph, long long n) {
  const long long chunks = (n + (long long)kUpdBlock * ept - 1) / ((long long)kUpdBlock * ept);
  const dim3 grid((unsigned)chunks, L, (N + kDfGroup - 1) / kDfGroup);
  switch (ept) {
    case 1: launch_prio(cg_update_df_kernel<RT, 1>, grid, kUpdBlock, st, prio, c, N, par, r, y, ph, n); break;
    case 2: launch_prio(cg_update_df_kernel<RT, 2>, grid, kUpdBlock, st, prio, c, N, par, r, y, ph, n); break;
    default: launch_prio(cg_update_df_kernel<RT, 4>, grid, kUpdBlock, st, prio, c, N, par, r, y, ph, n); break;
  }
}

// The TMA-fed float-float update (default; SSQCD_UPDATE_TMA=0 selects the
// grouped register kernel instead, for comparison runs).
bool use_tma_update() {
  static const bool v = [] {
    const char* e = std::getenv("SSQCD_UPDATE_TMA");
    return !(e && e[0] == '0');
  }();
  return v;
}

// Test of the bounded waits: SSQCD_TEST_UPDATE_STALL=1 keeps the producer of
// the TMA-fed update idle (the wait-limit error path, without a fault).
int update_stall_test() {
  static const int v = [] {
    const char* e = std::getenv("SSQCD_TEST_UPDATE_STALL");
    return (e && e[0] == '1') ? 1 : 0;
  }();
  return v;
}

// The shared-memory limit is an attribute of the kernel, shared by every run
// of the process: it is only ever raised, so that a run with fewer shifts
// does not lower it below what a concurrent run's launches need (the
// scheduler's requests run side by side).
template <typename RT>
int prepare_update_tma(int NL, int L) {
  static std::mutex mu;
  static size_t set = 0;
  const size_t smem = tma_smem_bytes(NL, L);
  std::lock_guard<std::mutex> lock(mu);
  if (smem <= set) return SSQCD_OK;
  SS_CUDA(cudaFuncSetAttribute(cg_update_tma_kernel<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  set = smem;
  return SSQCD_OK;
}

template <typename RT>
void launch_update_tma(int nblocks, int L, cudaStream_t st, int prio, const Control& c, int N, int par, const RT* r,
                       float4* y, float4* ph, long long n) {
  const int nchunks = (int)((n + kTmaCh - 1) / kTmaCh);
  launch_prio_smem(cg_update_tma_kernel<RT>, dim3(nblocks), dim3(kTmaThreads), tma_smem_bytes(N * L, L), st, prio,
                   false, c, N, L, par, r, y, ph, n, nchunks, update_stall_test());
}

int update_blocks(long long n, int L, int ept) {
  const long long chunks = (n + (long long)kUpdBlock * ept - 1) / ((long long)kUpdBlock * ept);
  const long long cap = (152LL * 8 + L - 1) / L;
  return (int)std::max(1LL, std::min(chunks, cap));
}

}  // namespace

namespace {

// The solve loop for one precision: VR is the type of the seed vectors (r, p,
// q and the stencil), V2 that of the shift vectors (y, p-hat): double2 /
// double2 (SSQCD_FP64), double2 / float2 (SSQCD_FP64_SHIFT32), double2 /
// float4 = complex float-float (SSQCD_FP64_DFSHIFT), float4 / float4
// (SSQCD_DF), float2 / float2 (the mixed precisions).  The final solutions
// are FP64.
//
// A run is resumable: init() allocates and initialises on the run's stream
// and captures the chunk graph; launch() enqueues one chunk of kChunk
// iterations followed by the read of the live-shift count and error flag
// into pinned memory (never blocks); poll() looks at the oldest launched
// chunk (waiting for it or not) and reports whether shifts are still live;
// finish() hands over the FP64 solutions and the counters.  ss_solve drives
// one run to the end; the request scheduler interleaves many.
template <typename VR, typename V2>
class CgRun final : public CgRunBase {
  static constexpr bool kFP32 = sizeof(VR) == sizeof(float2);       // seed vectors and stencil in FP32
  static constexpr bool kShift32 = sizeof(V2) == sizeof(float2);    // shift vectors in FP32
  static constexpr bool kShiftDF = std::is_same<V2, float4>::value;  // shift vectors in float-float
  static constexpr bool kSeedDF = std::is_same<VR, float4>::value;   // seed vectors and stencil in float-float
  static constexpr int kChunk = 16;  // even: every chunk starts at parity 0
  static constexpr int kSlots = 8;   // timing events per iteration: A, B, C, P start/stop
  static constexpr int kTimedEvery = 4;
  static constexpr int kInFlight = 2;  // chunks enqueued ahead of the poll

 public:
  ~CgRun() override {
    if (st_ != nullptr) cudaStreamSynchronize(st_);
    if (gexec_ != nullptr) cudaGraphExecDestroy(gexec_);
    if (gexec_t_ != nullptr) cudaGraphExecDestroy(gexec_t_);
    for (auto e : tev_) cudaEventDestroy(e);
    for (auto e : ev_) cudaEventDestroy(e);
    for (auto e : ev_poll_) cudaEventDestroy(e);
    if (e0_) cudaEventDestroy(e0_);
    if (e1_) cudaEventDestroy(e1_);
    if (side_) cudaStreamDestroy(side_);
    if (h_poll_) cudaFreeHost(h_poll_);
    if (h_iters_) cudaFreeHost(h_iters_);
    if (h_tab_) cudaFreeHost(h_tab_);
  }

  int init(ssqcd_lattice lat, int N, const double2* z_host, int L, const double2* v, double sigma, double tol,
           int max_iter, int reliable_every, double basis_cap, cudaStream_t st) {
    lat_ = lat;
    // the Krylov-basis form: 16-byte seed vectors (FP64 or float-float) and
    // shift vectors of the same type, no reliable updates
    basis_ = basis_cap > 0.0 && kBasisCapable && reliable_every <= 0;
    basis_cap_ = basis_cap;
    basis_state_ = basis_ ? 1 : 0;
    N_ = N;
    L_ = L;
    v_ = v;
    sigma_ = sigma;
    max_iter_ = max_iter;
    st_ = st;
    // lattice-owned data first, outside the run's stream-ordered allocations
    if constexpr (kSeedDF) SS_TRY(ensure_df_links(lat));
    AllocStream scope(st_);
    tma_ = kShiftDF && use_tma_update();
    {
      int dev = 0;
      SS_CUDA(cudaGetDevice(&dev));
      SS_CUDA(cudaDeviceGetAttribute(&n_sm_, cudaDevAttrMultiProcessorCount, dev));
    }
    tma_ctas_ = n_sm_;
    if (const char* e = std::getenv("SSQCD_UPDATE_CTAS")) {  // tuning runs: persistent CTAs of the update
      const int v = std::atoi(e);
      if (v >= 1 && v <= 4 * n_sm_) tma_ctas_ = v;
    }
    if constexpr (kShiftDF) {
      if (tma_) SS_TRY(prepare_update_tma<VR>(N * L, L));
    }
    const Geometry& g = lat->g;
    n_ = 12LL * g.V;
    const long long n = n_;
    const int NL = N * L;
    nbw_ = kFP32 ? (g.V + kSiteThreads - 1) / kSiteThreads
           : (kSeedDF || !balanced_stencil()) ? wilson_blocks(g)
                                              : (g.V + kSitesPerBlockH - 1) / kSitesPerBlockH;
    nbs_ = seed_blocks(n, L);
    ept_ = update_epts(kShift32 || kShiftDF);
    nbu_ = update_blocks(n, L, ept_);
    // r enters p-hat: with FP32 exponents (FP32 or float-float shift vectors)
    // ||r|| is kept within 2^-20 of ||v|| (its elements stay far above the
    // FP32 underflow); FP64 within 2^-200.
    rescale_below_ = (kShift32 || kShiftDF) ? 0x1p-40 : 0x1p-400;
    rescale_by_ = (kShift32 || kShiftDF) ? 0x1p+20 : 0x1p+200;
    tol2_ = tol * tol;

    SS_TRY(p_.alloc(sizeof(VR) * n * L));
    SS_TRY(q_.alloc(sizeof(VR) * n * L));
    if (basis_) {
      // block table (pinned host mirror, written once per entry) and the
      // first two blocks: slot 0 and the first chunk's residuals
      blk_vec_ = (sizeof(VR) * kBasisBlock * (size_t)L * n + 255) / 256 * 256;
      blk_bytes_ = basis_block_bytes(blk_vec_, NL, L);
      tab_cap_ = (max_iter + kChunk) / kBasisBlock + 2;
      SS_TRY(tab_.alloc(sizeof(char*) * tab_cap_));
      SS_CUDA(cudaMallocHost(&h_tab_, sizeof(char*) * (tab_cap_ + 2)));  // + the first two slot pointers
      SS_TRY(ensure_blocks(kChunk + 1));
      if (!basis_) return fail(SSQCD_ERR_OOM, "stored residuals: the memory cap is below two blocks");
    } else {
      SS_TRY(alloc_update_vectors());
    }
    if (kFP32 && reliable_every > 0) {
      SS_TRY(x_.alloc(sizeof(double2) * n * L));
      SS_TRY(kx_.alloc(sizeof(double2) * n * L));
      SS_CUDA(cudaMemsetAsync(x_.p, 0, sizeof(double2) * n * L, st_));
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
      const size_t o = off;
      off += (bytes + 255) / 256 * 256;
      return o;
    };
    const size_t o_seed = take(sizeof(SeedState) * L), o_alpha = take(sizeof(double) * L),
                 o_vn = take(sizeof(double) * L), o_live = take(sizeof(int) * L), o_tot = take(sizeof(int)),
                 o_ran = take(sizeof(int)), o_rran = take(sizeof(int) * 2), o_err = take(sizeof(int)),
                 o_si = take(sizeof(int) * 2), o_done = take(sizeof(unsigned) * 4),
                 o_s = take(sizeof(double2) * NL), o_xc = take(sizeof(double2) * NL),
                 o_xp = take(sizeof(double2) * NL), o_xn = take(sizeof(double2) * NL),
                 o_rt = take(sizeof(double2) * NL), o_act = take(sizeof(int) * NL), o_it = take(sizeof(int) * NL),
                 o_ln = take(sizeof(int) * 2 * L), o_lj = take(sizeof(int) * 2 * NL),
                 o_la = take(sizeof(double2) * 2 * NL), o_lb = take(sizeof(double2) * 2 * NL),
                 o_lsc = take(sizeof(double) * 2 * L), o_part = take(sizeof(double) * (size_t)nbw_ * L),
                 o_prr = take(sizeof(double) * (size_t)nbs_ * L), o_vp = take(sizeof(double) * (size_t)nbs_ * L),
                 o_vn2 = take(sizeof(double) * L), o_rptr = take(sizeof(char*) * 2),
                 o_arec = take(sizeof(double) * 2 * L), o_srec = take(sizeof(double) * 8 * L),
                 o_srk = take(sizeof(int) * 2), o_sprev = take(sizeof(double) * 2 * L);
    SS_TRY(ctl_.alloc(off));
    char* base = ctl_.as<char>();
    Control& c = c_;
    c.seed = reinterpret_cast<SeedState*>(base + o_seed);
    c.alpha = reinterpret_cast<double*>(base + o_alpha);
    c.vnorm2 = reinterpret_cast<double*>(base + o_vn);
    c.live = reinterpret_cast<int*>(base + o_live);
    c.live_total = reinterpret_cast<int*>(base + o_tot);
    c.ran = reinterpret_cast<int*>(base + o_ran);
    c.rec_ran = reinterpret_cast<int*>(base + o_rran);
    c.err = reinterpret_cast<int*>(base + o_err);
    c.seed_iters = reinterpret_cast<int*>(base + o_si);
    c.done = reinterpret_cast<unsigned*>(base + o_done);
    c.task_ctr = c.done + 2;
    c.shift_s = reinterpret_cast<double2*>(base + o_s);
    c.xi_cur = reinterpret_cast<double2*>(base + o_xc);
    c.xi_prev = reinterpret_cast<double2*>(base + o_xp);
    c.xi_next = reinterpret_cast<double2*>(base + o_xn);
    c.ratio = reinterpret_cast<double2*>(base + o_rt);
    c.act = reinterpret_cast<int*>(base + o_act);
    c.iters = reinterpret_cast<int*>(base + o_it);
    c.list_n = reinterpret_cast<int*>(base + o_ln);
    c.list_j = reinterpret_cast<int*>(base + o_lj);
    c.list_a = reinterpret_cast<double2*>(base + o_la);
    c.list_b = reinterpret_cast<double2*>(base + o_lb);
    c.list_sc = reinterpret_cast<double*>(base + o_lsc);
    c.partial = reinterpret_cast<double*>(base + o_part);
    c.partial_rr = reinterpret_cast<double*>(base + o_prr);
    c.x = x_.p != nullptr ? x_.as<double2>() : nullptr;
    c.tab = basis_ ? tab_.as<char*>() : nullptr;
    c.blk_vec = blk_vec_;
    c.rptr = reinterpret_cast<char**>(base + o_rptr);
    c.split = basis_ ? 1 : 0;
    c.alpha_rec = reinterpret_cast<double*>(base + o_arec);
    c.srec = reinterpret_cast<double*>(base + o_srec);
    c.srec_k = reinterpret_cast<int*>(base + o_srk);
    c.sprev = reinterpret_cast<double*>(base + o_sprev);
    if (basis_) {  // slots 0 and 1 for the first iteration
      h_tab_[tab_cap_] = h_tab_[0];
      h_tab_[tab_cap_ + 1] = h_tab_[0] + sizeof(VR) * (size_t)L * n;
      SS_CUDA(cudaMemcpyAsync(c.rptr, h_tab_ + tab_cap_, sizeof(char*) * 2, cudaMemcpyHostToDevice, st_));
    }
    double* vn_part = reinterpret_cast<double*>(base + o_vp);
    double* vn2 = reinterpret_cast<double*>(base + o_vn2);

    shift_host_.resize(NL);
    for (int l = 0; l < L; ++l)
      for (int j = 0; j < N; ++j) shift_host_[l * N + j] = make_double2(z_host[j].x - sigma, z_host[j].y);
    SS_CUDA(cudaMemcpyAsync(c.shift_s, shift_host_.data(), sizeof(double2) * NL, cudaMemcpyHostToDevice, st_));

    SS_TRY(norm2_partials(v, L, n, vn_part, nbs_, st_));
    SS_TRY(sum_partials(vn_part, L, nbs_, vn2, st_));
    if (basis_)  // r_0 = v into slot 0; no shift vectors
      init_vectors_kernel<<<dim3(nbu_, L), kUpdBlock, 0, st_>>>(v, blocks_[0]->as<VR>(), p_.as<VR>(), (V2*)nullptr,
                                                                (V2*)nullptr, 0, n);
    else
      init_vectors_kernel<<<dim3(nbu_, L), kUpdBlock, 0, st_>>>(v, r_.as<VR>(), p_.as<VR>(), yv_, ph_.as<V2>(), N, n);
    SS_CHECK_LAUNCH();
    init_control_kernel<<<1, 256, 0, st_>>>(c, vn2, L, N);
    SS_CHECK_LAUNCH();
    count_launches(2);

    SS_CUDA(cudaEventCreate(&e0_));
    SS_CUDA(cudaEventCreate(&e1_));
    SS_CUDA(cudaEventRecord(e0_, st_));
    SS_CUDA(cudaMallocHost(&h_poll_, sizeof(int) * 2 * kInFlight));
    ev_poll_.resize(kInFlight);
    for (auto& e : ev_poll_) SS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    timing_ = kernel_timing_enabled();
    ru_chunks_ = (kFP32 && reliable_every > 0) ? std::max(1, (reliable_every + kChunk / 2) / kChunk) : 0;
    // Two streams: the main chain A -> B -> P runs on the run's stream at
    // the greatest priority; C (the shift update of iteration k) runs on a
    // side stream beside A, B, P of iteration k + 1.  Dependencies: C(k)
    // after B(k) (coefficients, r_{k+1}) and after C(k-1) (stream order);
    // A(k) after C(k-2) (A and B of iteration k rewrite the parity-(k % 2)
    // record and r buffer that C(k-2) read).  Each chunk forks the side
    // stream from the main one and joins it back at the end.
    SS_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo_, &prio_hi_));
    // the stencil A one level below B and P: when the runs of two source
    // blocks share the GPU (opts.block_streams), the short seed kernels of one
    // run are dispatched ahead of the remaining stencil blocks of the other,
    // instead of queueing behind them (headline workload: CG loop 5.30 -> 4.99 s
    // FP64, 2.68 -> 2.27 s float-float); alone, A, B and P run in turn anyway
    prio_a_ = (prio_lo_ - prio_hi_ >= 2) ? prio_hi_ + 1 : prio_hi_;
    SS_CUDA(cudaStreamCreateWithPriority(&side_, cudaStreamNonBlocking, prio_lo_));
    ev_.resize(2 * kChunk + 1);
    for (auto& e : ev_) SS_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    if (timing_) {
      tev_.resize(kChunk * kSlots);
      for (auto& e : tev_) SS_CUDA(cudaEventCreate(&e));
      SS_CUDA(cudaMallocHost(&h_iters_, sizeof(int) * NL * kInFlight));
    }
    // A chunk of iterations is captured once as a CUDA graph and replayed
    // (the kernels read all per-iteration state from device memory, so every
    // replay is the same graph; node priorities are kept).  With kernel
    // timing on, a second graph also records an event around every kernel;
    // it replaces the plain one for one chunk in kTimedEvery (the event nodes
    // cost ~7% of the loop), and its events are read after that replay.  A
    // stream that cannot be captured (the legacy default stream) falls back
    // to direct launches.
    gexec_ = capture(false);
    gexec_t_ = (timing_ && gexec_ != nullptr) ? capture(true) : nullptr;
    return SSQCD_OK;
  }

  int launch() override {
    AllocStream scope(st_);
    const int chunk = std::min(kChunk, max_iter_ - k_);
    if (chunk <= 0) return SSQCD_OK;
    if (basis_) SS_TRY(ensure_blocks(k_ + chunk + 1));  // kernel B of the last iteration looks one slot ahead
    const int slot = (int)(launched_chunks_ % kInFlight);
    ChunkInfo info;
    info.k_start = k_;
    info.timed = timing_ && launched_chunks_ % kTimedEvery == 0 && (gexec_ == nullptr || gexec_t_ != nullptr);
    if (gexec_ != nullptr && chunk == kChunk) {
      cudaError_t ge = cudaGraphLaunch(info.timed ? gexec_t_ : gexec_, st_);
      if (ge != cudaSuccess) return cuda_fail(ge, "shifted CG graph launch", __FILE__, __LINE__);
    } else {
      mark_on_ = info.timed;
      run_chunk(chunk);
      mark_on_ = false;
      cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) return cuda_fail(le, "shifted CG launch", __FILE__, __LINE__);
    }
    count_launches(4LL * chunk);
    k_ += chunk;
    info.count = chunk;
    ++launched_chunks_;
    if (kFP32 && c_.x != nullptr && ru_chunks_ > 0 && launched_chunks_ % ru_chunks_ == 0) {
      // reliable update: r = S (v - K x) in FP64 with the FP64 links
      SS_TRY(wilson64(lat_->g, lat_->u64.as<double2>(), c_.x, kx_.as<double2>(), L_, sigma_, -1.0, nullptr, nullptr,
                      st_));
      const double floor2 = lat_->precision == SSQCD_MIXED ? 1e-4 : 1e-10;  // (1e-2 / 1e-5 of ||v||)^2
      // the next iteration (parity of the chunk length) reads this buffer
      VR* r_next = r_.as<VR>() + (size_t)(chunk & 1) * n_ * L_;
      cg_reliable_kernel<VR><<<dim3(nbs_, L_), kSeedBlock, 0, st_>>>(c_, L_, v_, kx_.as<double2>(), r_next, n_,
                                                                     floor2);
      SS_CHECK_LAUNCH();
      count_launches(1);
    }
    // live-shift count after the last iteration and the error flag
    SS_CUDA(cudaMemcpyAsync(h_poll_ + 2 * slot, c_.live_total, sizeof(int), cudaMemcpyDeviceToHost, st_));
    SS_CUDA(cudaMemcpyAsync(h_poll_ + 2 * slot + 1, c_.err, sizeof(int), cudaMemcpyDeviceToHost, st_));
    if (timing_)
      SS_CUDA(cudaMemcpyAsync(h_iters_ + (size_t)slot * N_ * L_, c_.iters, sizeof(int) * N_ * L_,
                              cudaMemcpyDeviceToHost, st_));
    SS_CUDA(cudaEventRecord(ev_poll_[slot], st_));
    pending_.push_back(info);
    return SSQCD_OK;
  }

  int in_flight() const override { return (int)pending_.size(); }

  int poll(bool wait, int* state) override {
    *state = kPollRunning;
    if (pending_.empty()) {
      if (k_ >= max_iter_) return fail(SSQCD_ERR_NOCONV, "shifted CG: max_iter reached");
      return SSQCD_OK;
    }
    const int slot = (int)(polled_chunks_ % kInFlight);
    if (wait) {
      SS_CUDA(cudaEventSynchronize(ev_poll_[slot]));
    } else {
      const cudaError_t q = cudaEventQuery(ev_poll_[slot]);
      if (q == cudaErrorNotReady) {
        *state = kPollBusy;
        return SSQCD_OK;
      }
      if (q != cudaSuccess) return cuda_fail(q, "shifted CG poll", __FILE__, __LINE__);
    }
    const ChunkInfo info = pending_.front();
    pending_.erase(pending_.begin());
    ++polled_chunks_;
    if (timing_) {
      // the counts after this chunk (each in-flight chunk has its own copy)
      long long units = 0;
      const int* hi = h_iters_ + (size_t)slot * N_ * L_;
      for (int qi = 0; qi < N_ * L_; ++qi) units += hi[qi];
      if (info.timed) {
        timed_units_ += units - units_prev_;
        for (int it = 0; it < info.count; ++it) {
          t_k_.push_back(info.k_start + it);
          for (int cls = 0; cls < 4; ++cls) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, tev_[it * kSlots + 2 * cls], tev_[it * kSlots + 2 * cls + 1]);
            t_iter_[cls].push_back(ms);
          }
        }
      }
      units_prev_ = units;
    }
    const int live = h_poll_[2 * slot], err = h_poll_[2 * slot + 1];
    if (err == 2) return fail(SSQCD_ERR_NOCONV, "shift update: a device-side wait hit its limit");
    // every shift frozen: done, even if an iteration that ran after the last
    // freeze (the Krylov-basis loop reads the live count one iteration late)
    // met a breakdown of the then useless seed recurrence
    if (live == 0) {
      *state = kPollDone;
      return SSQCD_OK;
    }
    if (err != 0) return fail(SSQCD_ERR_BREAKDOWN, "seed CG breakdown: |(p, K p)| < 1e-30 (r, r)");
    if (info.k_start + info.count >= max_iter_) {
      char buf[128];
      std::snprintf(buf, sizeof(buf), "shifted CG: %d shifts still above tol after %d iterations", live, max_iter_);
      return fail(SSQCD_ERR_NOCONV, buf);
    }
    return SSQCD_OK;
  }

  int finish(DevBuf& y_out, int* iters_host, double2* xi_host, ShiftedCGOut* out) override {
    AllocStream scope(st_);
    const long long n = n_;
    const int NL = N_ * L_;
    // chunks enqueued past convergence do no work; wait for them
    SS_CUDA(cudaStreamSynchronize(st_));
    pending_.clear();
    if (basis_) {
      SS_TRY(finish_basis());
    } else if (kShift32) {  // hand FP64 solutions to the FP64 moments and Rayleigh-Ritz
      SS_TRY(y_out_.alloc(sizeof(double2) * n * NL));
      SS_TRY(convert_f32_to_f64(reinterpret_cast<const float2*>(yv_), y_out_.as<double2>(), n * NL, st_));
    } else if (kShiftDF) {
      const long long cnt = n * NL;
      const int nb = (int)std::max(1LL, std::min((cnt + 255) / 256, 152LL * 16));
      df_to_f64_kernel<<<nb, 256, 0, st_>>>(reinterpret_cast<float4*>(yv_), cnt);
      SS_CHECK_LAUNCH();
      count_launches(1);
    }
    SS_CUDA(cudaEventRecord(e1_, st_));
    int counters[2] = {0, 0};
    std::vector<int> it_all(NL);
    SS_CUDA(cudaMemcpyAsync(counters, c_.seed_iters, sizeof(int) * 2, cudaMemcpyDeviceToHost, st_));
    SS_CUDA(cudaMemcpyAsync(it_all.data(), c_.iters, sizeof(int) * NL, cudaMemcpyDeviceToHost, st_));
    std::vector<int> act_all(xi_host ? NL : 0);
    std::vector<SeedState> seed_all(xi_host ? L_ : 0);
    if (xi_host) {
      SS_CUDA(cudaMemcpyAsync(xi_host, c_.xi_cur, sizeof(double2) * NL, cudaMemcpyDeviceToHost, st_));
      SS_CUDA(cudaMemcpyAsync(act_all.data(), c_.act, sizeof(int) * NL, cudaMemcpyDeviceToHost, st_));
      SS_CUDA(cudaMemcpyAsync(seed_all.data(), c_.seed, sizeof(SeedState) * L_, cudaMemcpyDeviceToHost, st_));
    }
    SS_CUDA(cudaStreamSynchronize(st_));
    if (xi_host)  // shifts still live at the end hold xi / S
      for (int qi = 0; qi < NL; ++qi)
        if (act_all[qi]) {
          const double S = seed_all[qi / N_].pad[1];
          xi_host[qi] = make_double2(xi_host[qi].x * S, xi_host[qi].y * S);
        }
    if (iters_host) std::copy(it_all.begin(), it_all.end(), iters_host);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0_, e1_);
    if (out) {
      // iterations that updated a shift: the stencil applications but for
      // at most one after the last freeze (Krylov-basis loop, see poll)
      out->seed_iters = it_all.empty() ? 0 : *std::max_element(it_all.begin(), it_all.end());
      out->reliable_updates = counters[1];
      out->ms = ms;
      out->shift_updates = 0;
      for (int v2 : it_all) out->shift_updates += v2;
      out->timed = timing_;
      out->timed_units = timed_units_;
      out->basis = basis_state_;
      out->basis_bytes = (double)basis_peak_;
      int n_timed = 0;
      for (int kk : t_k_) n_timed += kk < counters[0] ? 1 : 0;
      out->launches_update = n_timed;
      for (int cls = 0; cls < 4; ++cls) out->ms_k[cls] = 0.0;
      const int slot_of[4] = {0, 1, 3, 2};  // stencil, seed update + scalars, shift update, seed p
      for (int cls = 0; cls < 4; ++cls) {
        double acc = 0.0;
        // iterations after the last live one skip their work: not counted
        for (size_t i = 0; i < t_iter_[cls].size(); ++i)
          if (t_k_[i] < counters[0]) acc += t_iter_[cls][i];
        out->ms_k[slot_of[cls]] = acc;
      }
    }
    y_out.swap(y_out_);
    return SSQCD_OK;
  }

  bool take_basis(KrylovBasis* out) override {
    if (!basis_ || out == nullptr) return false;
    out->release();
    out->L = L_;
    out->N = N_;
    out->S = basis_S_;
    out->df = kSeedDF;
    out->n = n_;
    out->blocks.swap(blocks_);
    out->tab.swap(tab_);
    out->gam.swap(gam_);
    out->count.swap(count_);
    basis_ = false;
    return true;
  }

 private:
  static constexpr bool kBasisCapable = sizeof(VR) == 16 && std::is_same<VR, V2>::value;

  // y and p-hat of every shift (and r's parity buffers) for the update form
  int alloc_update_vectors() {
    const long long n = n_;
    const int NL = N_ * L_;
    SS_TRY(r_.alloc(2 * sizeof(VR) * n * L_));  // r_k and r_{k+1}: parity buffers
    SS_TRY(ph_.alloc(sizeof(V2) * n * NL));
    if (kShift32) {
      SS_TRY(y32_.alloc(sizeof(V2) * n * NL));
      yv_ = y32_.as<V2>();
    } else {  // FP64 solutions, or float-float ones converted in place at the end
      static_assert(kShift32 || sizeof(V2) == sizeof(double2), "in-place conversion needs equal element sizes");
      SS_TRY(y_out_.alloc(sizeof(double2) * n * NL));
      yv_ = reinterpret_cast<V2*>(y_out_.p);
    }
    return SSQCD_OK;
  }

  // Blocks for every slot up to kend (and the coefficient records of the
  // iterations before it); at the memory cap, switch to the update form.
  int ensure_blocks(int kend) {
    const size_t need = (size_t)(kend >> kBasisLog) + 1;
    while (blocks_.size() < need) {
      if (blocks_.size() >= tab_cap_) return fail(SSQCD_ERR_ARG, "stored residuals: block table full");
      if ((double)(basis_bytes_ + blk_bytes_) > basis_cap_ && blocks_.size() >= 2) return switch_to_updates();
      auto b = std::make_unique<DevBuf>();
      SS_TRY(b->alloc(blk_bytes_));
      const size_t i = blocks_.size();
      h_tab_[i] = b->as<char>();
      SS_CUDA(cudaMemcpyAsync(tab_.as<char*>() + i, h_tab_ + i, sizeof(char*), cudaMemcpyHostToDevice, st_));
      blocks_.push_back(std::move(b));
      basis_bytes_ += blk_bytes_;
      basis_peak_ = std::max(basis_peak_, basis_bytes_);
    }
    return SSQCD_OK;
  }

  // Slot counts from the per-shift iteration counts: S (the stride) and, per
  // source, the slots its solutions combine (k + 1 while a shift is live).
  int slot_counts(int k, bool with_live, std::vector<int>& it_all, std::vector<int>& act_all, int* S_out) {
    const int NL = N_ * L_;
    it_all.resize(NL);
    act_all.resize(NL);
    SS_CUDA(cudaMemcpyAsync(it_all.data(), c_.iters, sizeof(int) * NL, cudaMemcpyDeviceToHost, st_));
    SS_CUDA(cudaMemcpyAsync(act_all.data(), c_.act, sizeof(int) * NL, cudaMemcpyDeviceToHost, st_));
    SS_CUDA(cudaStreamSynchronize(st_));
    std::vector<int> cnt(L_, 0);
    for (int qi = 0; qi < NL; ++qi) {
      int c = it_all[qi];
      if (with_live && act_all[qi]) c = k + 1;
      cnt[qi / N_] = std::max(cnt[qi / N_], c);
    }
    int S = 1;
    for (int v : cnt) S = std::max(S, v);
    SS_TRY(count_.alloc(sizeof(int) * L_));
    SS_CUDA(cudaMemcpyAsync(count_.p, cnt.data(), sizeof(int) * L_, cudaMemcpyHostToDevice, st_));
    SS_CUDA(cudaStreamSynchronize(st_));  // cnt is a local array
    *S_out = S;
    return SSQCD_OK;
  }

  // End of a run in the Krylov-basis form: the coefficient of every slot in
  // every solution (the moments are formed from them later).
  int finish_basis() {
    int k = 0;
    SS_CUDA(cudaMemcpy(&k, c_.seed_iters, sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<int> it_all, act_all;
    SS_TRY(slot_counts(k, false, it_all, act_all, &basis_S_));
    const int NL = N_ * L_;
    SS_TRY(gam_.alloc(sizeof(double2) * (size_t)NL * basis_S_));
    basis_gamma_kernel<<<(NL + 127) / 128, 128, 0, st_>>>(c_, L_, N_, basis_S_, gam_.as<double2>());
    SS_CHECK_LAUNCH();
    count_launches(1);
    return SSQCD_OK;
  }

  // At the memory cap: form y_j and p-hat_j from the stored residuals, put
  // r_k into the parity buffer the next iteration reads, free the blocks and
  // continue with the per-iteration updates (new chunk graphs).
  int switch_to_updates() {
    SS_CUDA(cudaStreamSynchronize(st_));
    int k = 0;
    SS_CUDA(cudaMemcpy(&k, c_.seed_iters, sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<int> it_all, act_all;
    int S = 0;
    SS_TRY(slot_counts(k, true, it_all, act_all, &S));
    SS_TRY(alloc_update_vectors());
    const int NL = N_ * L_;
    DevBuf gy, gp;
    SS_TRY(gy.alloc(sizeof(double2) * (size_t)NL * S));
    SS_TRY(gp.alloc(sizeof(double2) * (size_t)NL * S));
    basis_gamma_kernel<<<(NL + 127) / 128, 128, 0, st_>>>(c_, L_, N_, S, gy.as<double2>());
    SS_CHECK_LAUNCH();
    basis_phat_kernel<<<(NL + 127) / 128, 128, 0, st_>>>(c_, L_, N_, k, S, gp.as<double2>());
    SS_CHECK_LAUNCH();
    count_launches(2);
    if constexpr (kBasisCapable) {
      SS_TRY((launch_combine<VR, V2>(tab_.as<char*>(), n_, L_, gy.as<double2>(), N_, S, count_.as<int>(), yv_, st_)));
      SS_TRY((launch_combine<VR, V2>(tab_.as<char*>(), n_, L_, gp.as<double2>(), N_, S, count_.as<int>(),
                                     ph_.as<V2>(), st_)));
    }
    const char* rk = h_tab_[k >> kBasisLog] + (size_t)(k & (kBasisBlock - 1)) * L_ * n_ * sizeof(VR);
    SS_CUDA(cudaMemcpyAsync(r_.p, rk, sizeof(VR) * L_ * n_, cudaMemcpyDeviceToDevice, st_));
    SS_CUDA(cudaStreamSynchronize(st_));
    gy.release();
    gp.release();
    blocks_.clear();
    basis_bytes_ = 0;
    basis_ = false;
    basis_state_ = 2;
    c_.tab = nullptr;
    c_.split = 0;  // kernel B takes the shift scalars again
    if (gexec_ != nullptr) cudaGraphExecDestroy(gexec_);
    if (gexec_t_ != nullptr) cudaGraphExecDestroy(gexec_t_);
    gexec_ = capture(false);
    gexec_t_ = (timing_ && gexec_ != nullptr) ? capture(true) : nullptr;
    return SSQCD_OK;
  }
  struct ChunkInfo {
    int k_start = 0, count = 0;
    bool timed = false;
  };

  void mark(int it, int slot, cudaStream_t s) {
    // during capture, only the External flag makes a real event-record node
    if (mark_on_) cudaEventRecordWithFlags(tev_[it * kSlots + slot], s, cudaEventRecordExternal);
  }

  void iteration(int it) {
    const Geometry& g = lat_->g;
    const long long n = n_;
    const int L = L_, N = N_;
    Control& c = c_;
    const dim3 grid_a(nbw_, L), grid_b(nbs_, L), grid_c(nbu_, L);
    const dim3 grid_p(p_blocks(n, L), L);
    VR* const r0 = r_.as<VR>();  // null in the Krylov-basis form (kernels B, P address the slots)
    const int par = it & 1;
    const VR* r_in = basis_ ? nullptr : r0 + (size_t)par * n * L;
    VR* r_out = basis_ ? nullptr : r0 + (size_t)(par ^ 1) * n * L;
    cudaStream_t st = st_;
    // A(k) after the side-stream kernel of k - 2 (C or S), which reads the
    // parity-(k % 2) records that A(k) and B(k) rewrite
    if (it >= 2) cudaStreamWaitEvent(st, ev_[kChunk + it - 2], 0);
    mark(it, 0, st);
    if constexpr (kFP32) {
      if (lat_->precision == SSQCD_MIXED)
        launch_chain(cg_stencil_kernel<Stencil32<LinksF16>, VR>, grid_a, kSiteThreads, st, prio_a_, basis_ && use_pdl(), c, L, par, g,
                    Stencil32<LinksF16>{LinksF16{lat_->u16.as<uint2>(), g.V}}, sigma_, p_.as<VR>(), q_.as<VR>());
      else
        launch_chain(cg_stencil_kernel<Stencil32<LinksF32>, VR>, grid_a, kSiteThreads, st, prio_a_, basis_ && use_pdl(), c, L, par, g,
                    Stencil32<LinksF32>{LinksF32{lat_->u32.as<float4>(), g.V}}, sigma_, p_.as<VR>(), q_.as<VR>());
    } else if constexpr (kSeedDF) {
      if (stencil_minb() == 3)
        launch_chain(cg_stencil_kernel<StencilDF<3>, VR>, grid_a, kStencilThreadsDF, st, prio_a_,
                     basis_ && use_pdl(), c, L, par, g, StencilDF<3>{lat_->udf.as<float4>()}, sigma_, p_.as<VR>(),
                     q_.as<VR>());
      else
        launch_chain(cg_stencil_kernel<StencilDF<4>, VR>, grid_a, kStencilThreadsDF, st, prio_a_,
                     basis_ && use_pdl(), c, L, par, g, StencilDF<4>{lat_->udf.as<float4>()}, sigma_, p_.as<VR>(),
                     q_.as<VR>());
    } else if (balanced_stencil()) {
      if (stencil_minb() == 8)
        launch_chain(cg_stencil_kernel<Stencil64h<8>, VR>, grid_a, kStencilThreads, st, prio_a_,
                     basis_ && use_pdl(), c, L, par, g, Stencil64h<8>{lat_->u64.as<double2>()}, sigma_,
                     p_.as<VR>(), q_.as<VR>());
      else
        launch_chain(cg_stencil_kernel<Stencil64h<7>, VR>, grid_a, kStencilThreads, st, prio_a_,
                     basis_ && use_pdl(), c, L, par, g, Stencil64h<7>{lat_->u64.as<double2>()}, sigma_,
                     p_.as<VR>(), q_.as<VR>());
    } else {
      launch_chain(cg_stencil_kernel<Stencil64, VR>, grid_a, kStencilThreads, st, prio_a_, basis_ && use_pdl(), c, L, par, g,
                  Stencil64{lat_->u64.as<double2>()}, sigma_, p_.as<VR>(), q_.as<VR>());
    }
    mark(it, 1, st);
    mark(it, 2, st);
    launch_chain(cg_seed_kernel<VR>, grid_b, kSeedBlock, st, prio_hi_, basis_ && use_pdl(), c, L, N, par, tol2_, r_in, r_out, q_.as<VR>(),
                p_.as<VR>(), n, rescale_below_, rescale_by_);
    mark(it, 3, st);
    cudaEventRecord(ev_[it], st);
    mark(it, 6, st);
    launch_chain(cg_seed_p_kernel<VR>, grid_p, kUpdBlock, st, prio_hi_, basis_ && use_pdl(), c, r_out, p_.as<VR>(), n);
    mark(it, 7, st);
    if (basis_) {  // no shift-vector update: the shift scalars on the side stream
      cudaStreamWaitEvent(side_, ev_[it], 0);
      mark(it, 4, side_);
      launch_prio(cg_shift_kernel, dim3(1), kSeedBlock, side_, prio_lo_, c, L, N, par, tol2_, rescale_by_);
      mark(it, 5, side_);
      cudaEventRecord(ev_[kChunk + it], side_);
      return;
    }
    cudaStreamWaitEvent(side_, ev_[it], 0);
    mark(it, 4, side_);
    if constexpr (kShiftDF) {
      if (tma_)
        launch_update_tma<VR>(tma_ctas_, L, side_, prio_lo_, c, N, par, r_out, yv_, ph_.as<float4>(), n);
      else
        launch_update_df<VR>(ept_, L, side_, prio_lo_, c, N, par, r_out, yv_, ph_.as<float4>(), n);
    } else {
      launch_update<VR, V2>(ept_, grid_c, side_, prio_lo_, c, N, par, r_out, yv_, ph_.as<V2>(), n);
    }
    mark(it, 5, side_);
    cudaEventRecord(ev_[kChunk + it], side_);
  }

  void run_chunk(int count) {
    cudaEvent_t ev_fork = ev_[2 * kChunk];
    cudaEventRecord(ev_fork, st_);
    cudaStreamWaitEvent(side_, ev_fork, 0);
    for (int it = 0; it < count; ++it) iteration(it);
    cudaStreamWaitEvent(st_, ev_[kChunk + count - 1], 0);
  }

  cudaGraphExec_t capture(bool with_events) {
    cudaGraphExec_t ge = nullptr;
    cudaGraph_t graph = nullptr;
    mark_on_ = with_events;
    if (cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      run_chunk(kChunk);
      if (cudaStreamEndCapture(st_, &graph) == cudaSuccess && graph != nullptr) {
        if (cudaGraphInstantiate(&ge, graph, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) ge = nullptr;
        cudaGraphDestroy(graph);
      }
    }
    (void)cudaGetLastError();  // a failed capture falls back to direct launches
    mark_on_ = false;
    return ge;
  }

  ssqcd_lattice lat_ = nullptr;
  int N_ = 0, L_ = 0, max_iter_ = 0;
  const double2* v_ = nullptr;
  double sigma_ = 0.0, tol2_ = 0.0, rescale_below_ = 0.0, rescale_by_ = 0.0;
  cudaStream_t st_ = nullptr, side_ = nullptr;
  long long n_ = 0;
  int nbw_ = 0, nbs_ = 0, nbu_ = 0, ept_ = 1, n_sm_ = 0, tma_ctas_ = 0, prio_lo_ = 0, prio_hi_ = 0, prio_a_ = 0, ru_chunks_ = 0;
  bool tma_ = false, timing_ = false, mark_on_ = false;
  // Krylov-basis form
  bool basis_ = false;
  int basis_state_ = 0, basis_S_ = 0;
  double basis_cap_ = 0.0;
  size_t blk_vec_ = 0, blk_bytes_ = 0, tab_cap_ = 0, basis_bytes_ = 0, basis_peak_ = 0;
  std::vector<std::unique_ptr<DevBuf>> blocks_;
  DevBuf tab_, gam_, count_;
  char** h_tab_ = nullptr;
  DevBuf r_, p_, q_, ph_, y32_, x_, kx_, y_out_, ctl_;
  V2* yv_ = nullptr;
  Control c_{};
  std::vector<double2> shift_host_;
  std::vector<cudaEvent_t> ev_, tev_, ev_poll_;
  cudaEvent_t e0_ = nullptr, e1_ = nullptr;
  cudaGraphExec_t gexec_ = nullptr, gexec_t_ = nullptr;
  int* h_poll_ = nullptr;
  int* h_iters_ = nullptr;
  int k_ = 0;
  long long launched_chunks_ = 0, polled_chunks_ = 0;
  std::vector<ChunkInfo> pending_;
  long long units_prev_ = 0, timed_units_ = 0;
  std::vector<int> t_k_;
  std::vector<double> t_iter_[4];
};

}  // namespace

int make_cg_run(ssqcd_lattice lat, int N, const double2* z_host, int L, const double2* v, double sigma, double tol,
                int max_iter, int precision, int reliable_every, double basis_cap, cudaStream_t st,
                std::unique_ptr<CgRunBase>* out) {
  if (!valid_precision(precision)) return fail(SSQCD_ERR_ARG, "unknown precision");
  if (is_mixed(precision) && precision != lat->precision)
    return fail(SSQCD_ERR_ARG, "a mixed-precision solve needs a lattice created with that precision");
  if (N < 1 || N > kMaxShifts) return fail(SSQCD_ERR_ARG, "N must be in [1, 512]");
  if (L < 1 || L > kMaxSources || N * L > kMaxTotal)
    return fail(SSQCD_ERR_ARG, "L must be in [1, 64] and N * L <= 1024");
  auto make = [&](auto* run) -> int {
    std::unique_ptr<CgRunBase> holder(run);
    if (!run) return fail(SSQCD_ERR_OOM, "host allocation failed");
    SS_TRY(run->init(lat, N, z_host, L, v, sigma, tol, max_iter, reliable_every, basis_cap, st));
    *out = std::move(holder);
    return SSQCD_OK;
  };
  if (precision == SSQCD_FP64) return make(new (std::nothrow) CgRun<double2, double2>());
  if (precision == SSQCD_DF) return make(new (std::nothrow) CgRun<float4, float4>());
  if (precision == SSQCD_FP64_DFSHIFT) return make(new (std::nothrow) CgRun<double2, float4>());
  if (precision == SSQCD_FP64_SHIFT32) return make(new (std::nothrow) CgRun<double2, float2>());
  return make(new (std::nothrow) CgRun<float2, float2>());
}

namespace {

// Drive a run to the end with two chunks in flight (the host polls one
// while the device works on the next; a chunk enqueued past convergence
// does no work).
int drive(CgRunBase* run) {
  int status = run->launch();
  if (status == SSQCD_OK) status = run->launch();
  while (status == SSQCD_OK) {
    int state = 0;
    if ((status = run->poll(true, &state)) != SSQCD_OK) break;
    if (state == CgRunBase::kPollDone) break;
    status = run->launch();
  }
  return status;
}

}  // namespace

int shifted_cg_device(ssqcd_lattice lat, int N, const double2* z_host, int L, const double2* v, double sigma,
                      double tol, int max_iter, int precision, int reliable_every, DevBuf& y, int* iters_host,
                      double2* xi_host, ShiftedCGOut* out) {
  std::unique_ptr<CgRunBase> run;
  SS_TRY(make_cg_run(lat, N, z_host, L, v, sigma, tol, max_iter, precision, reliable_every, 0.0, lat->stream,
                     &run));
  const int status = drive(run.get());
  if (status != SSQCD_OK && status != SSQCD_ERR_BREAKDOWN && status != SSQCD_ERR_NOCONV) return status;
  const int s2 = run->finish(y, iters_host, xi_host, out);
  return s2 != SSQCD_OK ? s2 : status;
}

int shifted_cg_solve(ssqcd_lattice lat, int N, const double2* z_host, int L, const double2* v, double sigma,
                     double tol, int max_iter, int precision, int reliable_every, double basis_cap, DevBuf& y,
                     KrylovBasis* basis, int* iters_host, ShiftedCGOut* out) {
  std::unique_ptr<CgRunBase> run;
  SS_TRY(make_cg_run(lat, N, z_host, L, v, sigma, tol, max_iter, precision, reliable_every, basis_cap, lat->stream,
                     &run));
  const int status = drive(run.get());
  if (status != SSQCD_OK && status != SSQCD_ERR_BREAKDOWN && status != SSQCD_ERR_NOCONV) return status;
  const int s2 = run->finish(y, iters_host, nullptr, out);
  if (s2 != SSQCD_OK) return s2;
  run->take_basis(basis);
  return status;
}

double basis_cap_for(int precision, int basis, double basis_max_bytes, long long n, int N, int L) {
  if (basis == 0 || !(precision == SSQCD_FP64 || precision == SSQCD_DF)) return 0.0;
  if (basis_max_bytes > 0.0) return basis_max_bytes;
  // sixteen times the memory of the shift vectors the update form would
  // hold (y and p-hat, 16 B a complex element: 32 N L n bytes), i.e. up to
  // 32 N iterations, and at least 4 GiB; a function of the problem only, so
  // that a solve makes the same choice (and the same arithmetic) wherever it
  // runs, unless the device has less than twice that free
  const double cap = std::max(16.0 * 32.0 * (double)n * N * L, 4.0 * (1ull << 30));
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0.0;
  return std::min(cap, 0.5 * (double)free_b);
}

void KrylovBasis::release() {
  blocks.clear();
  tab.release();
  gam.release();
  count.release();
  S = 0;
}

bool real_moments_enabled() {
  // SSQCD_REAL_MOMENTS=0 keeps the complex combination, for comparison
  static const bool on = [] {
    const char* e = std::getenv("SSQCD_REAL_MOMENTS");
    return !(e != nullptr && std::atoi(e) == 0);
  }();
  return on;
}

int basis_moments(const KrylovBasis& b, const double2* coef_host, int M, double2* s_hat, DevBuf& scratch,
                  cudaStream_t st, cudaStream_t side, const cudaEvent_t* src_ready, bool real_coef) {
  const int N = b.N, L = b.L, S = b.S;
  const size_t w_bytes = (sizeof(double2) * (size_t)N * M + 255) / 256 * 256;
  const long long cnt = (long long)L * M * S;
  const bool rc = real_coef && real_moments_enabled();
  // FP64 residuals with real coefficients: the tensor-core combination
  // (unless SSQCD_MOMENTS_TC=0), one source a launch, each with its work space
  const bool tc = !b.df && rc && combine_tc_enabled() && combine_tc_applicable(b.n, M, S);
  const size_t g_bytes = (sizeof(double2) * (size_t)cnt + (b.df ? sizeof(float2) * (size_t)cnt : 0) + 255) / 256 * 256;
  const size_t tc_src = tc ? (combine_tc_work_bytes(1, S) + 255) / 256 * 256 : 0;
  // W, G and (float-float residuals) Re G as float-float pairs
  SS_TRY(scratch.alloc(w_bytes + g_bytes + tc_src * (size_t)L));
  double2* W = scratch.as<double2>();
  double2* G = reinterpret_cast<double2*>(scratch.as<char>() + w_bytes);
  float2* Gr = reinterpret_cast<float2*>(G + cnt);
  char* tcw = scratch.as<char>() + w_bytes + g_bytes;
  SS_CUDA(cudaMemcpyAsync(W, coef_host, sizeof(double2) * (size_t)N * M, cudaMemcpyHostToDevice, st));
  basis_window_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(b.gam.as<double2>(), W, N, M, L, S, G);
  SS_CHECK_LAUNCH();
  count_launches(1);
  if (b.df && rc) {
    coef_real_to_ff_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(G, cnt, Gr);
    SS_CHECK_LAUNCH();
    count_launches(1);
  }
  auto one = [&](int l0, int nl, cudaStream_t s) -> int {
    if (b.df) {
      // outputs a thread accumulates: 8 (default) or 4 (SSQCD_COMB_DF_OUT=4:
      // fewer registers, more resident warps, the residuals read twice as often)
      static const int out_df = [] {
        const char* e = std::getenv("SSQCD_COMB_DF_OUT");
        return (e != nullptr && std::atoi(e) == 4) ? 4 : 8;
      }();
      const int per = out_df;
      const dim3 grid((unsigned)((b.n + kCombThreads - 1) / kCombThreads), nl, (M + per - 1) / per);
      char* const* tab = b.tab.as<char*>();
      const int* count = b.count.as<int>();
      // SSQCD_COMB_DF_TILE=32: real coefficients in tiles of 32 (comparison runs)
      static const bool tile32 = [] {
        const char* e = std::getenv("SSQCD_COMB_DF_TILE");
        return e != nullptr && std::atoi(e) == 32;
      }();
      if (per == 4 && rc)
        basis_combine_df_kernel<4, true, kCombTileRC>
            <<<grid, kCombThreads, 0, s>>>(tab, b.n, L, G, Gr, M, S, count, s_hat, l0);
      else if (per == 4)
        basis_combine_df_kernel<4, false, kCombTile>
            <<<grid, kCombThreads, 0, s>>>(tab, b.n, L, G, Gr, M, S, count, s_hat, l0);
      else if (rc && tile32)
        basis_combine_df_kernel<8, true, kCombTile>
            <<<grid, kCombThreads, 0, s>>>(tab, b.n, L, G, Gr, M, S, count, s_hat, l0);
      else if (rc)
        basis_combine_df_kernel<8, true, kCombTileRC>
            <<<grid, kCombThreads, 0, s>>>(tab, b.n, L, G, Gr, M, S, count, s_hat, l0);
      else
        basis_combine_df_kernel<8, false, kCombTile>
            <<<grid, kCombThreads, 0, s>>>(tab, b.n, L, G, Gr, M, S, count, s_hat, l0);
      SS_CHECK_LAUNCH();
      count_launches(1);
      return SSQCD_OK;
    }
    if (tc) {
      for (int l = l0; l < l0 + nl; ++l)
        SS_TRY(combine_tc(b.tab.as<char*>(), kBasisLog, b.n, L, G, M, S, b.count.as<int>(), s_hat, l, 1,
                          tcw + tc_src * (size_t)l, s));
      return SSQCD_OK;
    }
    return launch_combine<double2, double2>(b.tab.as<char*>(), b.n, L, G, M, S, b.count.as<int>(), s_hat, s, l0,
                                            nl, rc);
  };
  if (side == nullptr || src_ready == nullptr || L == 1) return one(0, L, st);
  // sources 0 .. L-2 in one launch on st (the orthogonalisation of their
  // moments follows in stream order), the last one on the side stream
  SS_TRY(one(0, L - 1, st));
  for (int l = 0; l < L - 1; ++l) SS_CUDA(cudaEventRecord(src_ready[l], st));
  SS_CUDA(cudaStreamWaitEvent(side, src_ready[0], 0));  // G and W are on st before
  SS_TRY(one(L - 1, 1, side));
  SS_CUDA(cudaEventRecord(src_ready[L - 1], side));
  return SSQCD_OK;
}

}  // namespace ssqcd
