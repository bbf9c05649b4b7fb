// Float-float versions of the Rayleigh-Ritz block operations (Section 2.1)
// for SSQCD_DF solves: CGS2 of the moment block, the Gram product T^H A T
// and the Ritz-vector combination, on the FP32 pipes.
//
// A complex float-float vector element is a float4 (re.hi, im.hi, re.lo,
// im.lo) (floatfloat.cuh); the arithmetic runs on register pairs with the
// real part in one lane and the imaginary part in the other (ff::p_cfma).
// Every sum keeps its float-float chains short -- a tile of elements or a
// tree of warp exchanges -- and adds the chains in FP64 (per block, or every
// few hundred elements), so the rounding stays within a few hundred units of
// 2^-48 of the terms; the FP64 pipe (1/64 of the FP32 rate on this GPU)
// only sees those per-chain conversions.  The reductions have a fixed order
// (block partials, then one pass over them in block order).
#include <algorithm>
#include <mutex>

#include "floatfloat.cuh"
#include "internal.h"

namespace ssqcd {
namespace {

using ff::cff;
constexpr int kRB = 256;     // threads a block
constexpr int kTPC = 4;      // columns a tile (CGS2)
constexpr int kEPT = 4;      // elements a thread (CGS2)
constexpr int kMaxCols = 128;

// A complex float-float value as its two register pairs (hi, lo).
struct C2 {
  f32x2_t h, l;
};
__device__ __forceinline__ C2 c2_of(cff z) { return C2{ff::hi2(z), ff::lo2(z)}; }
__device__ __forceinline__ cff cff_of(C2 a) { return ff::make2(a.h, a.l); }
__device__ __forceinline__ C2 c2_add(C2 a, C2 b) { return c2_of(ff::p_cadd(cff_of(a), cff_of(b))); }
__device__ __forceinline__ C2 c2_shfl_xor(C2 a, int o) {
  return C2{__shfl_xor_sync(0xffffffffu, a.h, o), __shfl_xor_sync(0xffffffffu, a.l, o)};
}
// p_cfma's coefficient pairs for conj(q)
__device__ __forceinline__ ff::PCoef coef_conj(cff q) {
  return ff::PCoef{pk2(q.x, q.x), pk2(q.z, q.z), pk2(q.y, -q.y), pk2(q.w, -q.w)};
}

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of 4 complex float-float values at once: two halving exchanges
// (at offset O a lane keeps one half of its values and adds the partner's
// copy of that half), then three over the low lane bits.  On return lane L
// holds the warp total of value (L >> 3) & 3.
template <int O, int HALF>
__device__ __forceinline__ void halve_c2(C2 (&v)[4], int lane) {
  const bool up = (lane & O) != 0;
#pragma unroll
  for (int i = 0; i < HALF; ++i) {
    const C2 send = up ? v[i] : v[i + HALF];
    const C2 keep = up ? v[i + HALF] : v[i];
    v[i] = c2_add(keep, c2_shfl_xor(send, O));
  }
}
__device__ __forceinline__ C2 warp_reduce_c2x4(C2 (&v)[4]) {
  const int lane = threadIdx.x & 31;
  halve_c2<16, 2>(v, lane);
  halve_c2<8, 1>(v, lane);
  C2 t = v[0];
  t = c2_add(t, c2_shfl_xor(t, 4));
  t = c2_add(t, c2_shfl_xor(t, 2));
  return c2_add(t, c2_shfl_xor(t, 1));
}
// FP64 warp sums of 8 values (lane L: value (L >> 2) & 7), for the last
// block's pass over the block partials
template <int O, int HALF>
__device__ __forceinline__ void halve8(double (&v)[8], int lane) {
  const bool up = (lane & O) != 0;
#pragma unroll
  for (int i = 0; i < HALF; ++i) {
    const double send = up ? v[i] : v[i + HALF];
    const double keep = up ? v[i + HALF] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
  }
}
__device__ __forceinline__ double warp_reduce8d(double (&v)[8]) {
  const int lane = threadIdx.x & 31;
  halve8<16, 4>(v, lane);
  halve8<8, 2>(v, lane);
  halve8<4, 1>(v, lane);
  const double t = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 2);
  return t + __shfl_xor_sync(0xffffffffu, t, 1);
}

// ---- CGS2 --------------------------------------------------------------------
// The same column-by-column CGS2 as the FP64 form (blas.cu): unnormalised
// columns v_a with nu_a^2 = ||v_a||^2, two launches a column, each launch's
// last block reducing the block partials in FP64 and forming the next
// subtraction coefficients; a column whose norm fell below 1e-15 of its
// original is dependent (zero).  Here the vectors and the projection
// arithmetic are float-float; the coefficients reach the next launch as
// float-float (negated, ready for p_cfma), the partial sums leave each block
// in FP64.
enum Mode : int { kStart = 0, kSubProj = 1, kSubNext = 2, kFinal = 3 };

struct CgsDf {
  double2* partial;   // [kMaxCols][nb]
  double* npart;      // [2][nb]
  float4* c;          // [kMaxCols] -c_a as complex float-float
  double* inv_nu2;    // [kMaxCols]
  double* inv_nu;     // [kMaxCols]
  double* orig2;      // [kMaxCols]
  unsigned* ticket;
};

__global__ void __launch_bounds__(kRB)
cgs2_df_step_kernel(CgsDf st, float4* __restrict__ Q, long long n, int m, int j, int mode,
                    double2* __restrict__ R) {
  __shared__ ff::PCoef s_c[kMaxCols];
  __shared__ C2 s_red[kRB / 32][kTPC];
  __shared__ double s_nred[2][kRB / 32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nb = gridDim.x;
  long long ei[kEPT];
  bool in[kEPT];
#pragma unroll
  for (int i = 0; i < kEPT; ++i) {
    ei[i] = blockIdx.x * (long long)(kRB * kEPT) + i * kRB + threadIdx.x;
    in[i] = ei[i] < n;
  }
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  if (mode == kFinal) {  // Q_a = v_a / nu_a for every column
    for (int a = 0; a < m; ++a) {
      const float2 s = ff::split(st.inv_nu[a]);
      const f32x2_t sh = pk2(s.x, s.x), sl = pk2(s.y, s.y);
#pragma unroll
      for (int i = 0; i < kEPT; ++i)
        if (in[i]) {
          C2 r{0ull, 0ull};
          ff::p_rfma(r.h, r.l, sh, sl, ff::p_val(Q[(long long)a * n + ei[i]]));
          Q[(long long)a * n + ei[i]] = cff_of(r);
        }
    }
    return;
  }
  // 1. the subtraction w -= sum_a v_a c_a on column j
  C2 x[kEPT];
#pragma unroll
  for (int i = 0; i < kEPT; ++i) x[i] = c2_of(in[i] ? Q[(long long)j * n + ei[i]] : zero4);
  if (mode == kSubProj || mode == kSubNext) {
    for (int a = threadIdx.x; a < j; a += kRB) s_c[a] = ff::p_coef(st.c[a]);
    __syncthreads();
    for (int a0 = 0; a0 < j; a0 += kTPC) {
      float4 q[kTPC][kEPT];
#pragma unroll
      for (int c = 0; c < kTPC; ++c)
#pragma unroll
        for (int i = 0; i < kEPT; ++i)
          q[c][i] = (a0 + c < j && in[i]) ? Q[(long long)(a0 + c) * n + ei[i]] : zero4;
#pragma unroll
      for (int c = 0; c < kTPC; ++c)
        if (a0 + c < j) {
          const ff::PCoef h = s_c[a0 + c];
#pragma unroll
          for (int i = 0; i < kEPT; ++i) ff::p_cfma(x[i].h, x[i].l, h, ff::p_val(q[c][i]));
        }
    }
#pragma unroll
    for (int i = 0; i < kEPT; ++i)
      if (in[i]) Q[(long long)j * n + ei[i]] = cff_of(x[i]);
  }
  // 2. partials of v_a^H y on the first np columns (FP64 per block)
  const int jp = mode == kSubNext ? j + 1 : j;
  const bool next = mode == kSubNext && jp < m;
  const int np = mode == kSubProj ? j : (next ? jp : 0);
  C2 y[kEPT];
#pragma unroll
  for (int i = 0; i < kEPT; ++i) y[i] = next ? c2_of(in[i] ? Q[(long long)jp * n + ei[i]] : zero4) : x[i];
  ff::PVal yv[kEPT];
#pragma unroll
  for (int i = 0; i < kEPT; ++i) yv[i] = ff::p_val(cff_of(y[i]));
  for (int a0 = 0; a0 < np; a0 += kTPC) {
    float4 q[kTPC][kEPT];
#pragma unroll
    for (int c = 0; c < kTPC; ++c) {
      const int a = a0 + c;
#pragma unroll
      for (int i = 0; i < kEPT; ++i)
        q[c][i] = (a < np && in[i]) ? ((next && a == j) ? cff_of(x[i]) : Q[(long long)a * n + ei[i]]) : zero4;
    }
    C2 acc[kTPC];
#pragma unroll
    for (int c = 0; c < kTPC; ++c) {
      acc[c] = C2{0ull, 0ull};
#pragma unroll
      for (int i = 0; i < kEPT; ++i) ff::p_cfma(acc[c].h, acc[c].l, coef_conj(q[c][i]), yv[i]);
    }
    const C2 t = warp_reduce_c2x4(acc);
    if ((lane & 7) == 0) s_red[w][lane >> 3] = t;
    __syncthreads();
    if (threadIdx.x < kTPC && a0 + (int)threadIdx.x < np) {
      C2 u = s_red[0][threadIdx.x];
      for (int ww = 1; ww < kRB / 32; ++ww) u = c2_add(u, s_red[ww][threadIdx.x]);
      st.partial[(long long)(a0 + threadIdx.x) * nb + blockIdx.x] = ff::to_double2(cff_of(u));
    }
    __syncthreads();
  }
  // norms (once a launch: float-float per thread, FP64 across the block)
  const bool norm_w = mode == kStart || mode == kSubNext;
  if (norm_w || next) {
    float s0 = 0.f, l0 = 0.f, s1 = 0.f, l1 = 0.f;
#pragma unroll
    for (int i = 0; i < kEPT; ++i) {
      ff::norm2_acc(cff_of(x[i]), s0, l0);
      if (next) ff::norm2_acc(cff_of(y[i]), s1, l1);
    }
    double v0 = wsum((double)s0 + (double)l0), v1 = wsum((double)s1 + (double)l1);
    if (lane == 0) {
      s_nred[0][w] = v0;
      s_nred[1][w] = v1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      double t = 0.0;
      for (int ww = 0; ww < kRB / 32; ++ww) t += s_nred[threadIdx.x][ww];
      st.npart[threadIdx.x * nb + blockIdx.x] = t;
    }
  }
  // 3. the last block reduces the partials in block order (FP64)
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(st.ticket, 1u) == (unsigned)nb - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (norm_w || next) {
    if (w < 2 && (w == 0 ? norm_w : next)) {
      double t = 0.0;
      for (int b = lane; b < nb; b += 32) t += __ldcg(st.npart + w * nb + b);
      t = wsum(t);
      if (lane == 0) {
        if (w == 0) {
          if (mode == kStart) st.orig2[j] = t;
          const bool dep = !(t > 1e-30 * (mode == kStart ? t : st.orig2[j]));
          st.inv_nu2[j] = dep ? 0.0 : 1.0 / t;
          st.inv_nu[j] = dep ? 0.0 : 1.0 / sqrt(t);
          R[(long long)j * m + j] = make_double2(dep ? 0.0 : sqrt(t), 0.0);
        } else {
          st.orig2[jp] = t;
        }
      }
    }
    __syncthreads();
  }
  for (int a0 = 4 * w; a0 < np; a0 += 4 * (kRB / 32)) {
    double acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = 0.0;
    for (int b = lane; b < nb; b += 32) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (a0 + c < np) {
          const double2 t = __ldcg(st.partial + (long long)(a0 + c) * nb + b);
          acc[2 * c] += t.x;
          acc[2 * c + 1] += t.y;
        }
    }
    const double t = warp_reduce8d(acc);
    const int a = a0 + (lane >> 3), comp = (lane >> 2) & 1;
    if ((lane & 3) == 0 && a < np) {
      const double i2 = __ldcg(st.inv_nu2 + a), i1 = __ldcg(st.inv_nu + a);
      // -c_a (float-float) for the subtraction of the next launch
      const double v = -t * i2;
      const float hv = __double2float_rn(v), lv = __double2float_rn(v - (double)hv);
      float* cf = reinterpret_cast<float*>(st.c + a);
      cf[comp] = hv;
      cf[2 + comp] = lv;
      reinterpret_cast<double*>(R)[2 * ((long long)a * m + jp) + comp] += t * i1;
    }
  }
  if (threadIdx.x == 0) *st.ticket = 0u;
}

// ---- Gram product G = X^H Y -------------------------------------------------
// 32 x 32 tiles of G per block (thread (ty, tx) of 16 x 16: entries ty + 16 i,
// tx + 16 j), the n elements split over blockIdx.z, staged through shared
// memory; float-float multiply-adds over kGEd elements at a time, whose sums
// enter FP64 accumulators every kFlushStages stages.
constexpr int kGTd = 32;
constexpr int kGEd = 32;
constexpr int kFlushStages = 8;

__global__ void __launch_bounds__(256)
gram_df_partial_kernel(const float4* __restrict__ X, int mx, const float4* __restrict__ Y, int my, long long n,
                       long long chunk, double2* __restrict__ partial, int herm) {
  __shared__ float4 sx[kGEd][kGTd + 1];
  __shared__ float4 sy[kGEd][kGTd + 1];
  if (herm && blockIdx.x > blockIdx.y) return;
  const int a0 = blockIdx.x * kGTd, b0 = blockIdx.y * kGTd;
  const int split = blockIdx.z;
  const long long e_begin = split * chunk;
  const long long e_end = min(n, e_begin + chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  double2 acc64[2][2];
  C2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      acc64[i][jj] = make_double2(0.0, 0.0);
      acc[i][jj] = C2{0ull, 0ull};
    }
  int stages = 0;
  for (long long e0 = e_begin; e0 < e_end; e0 += kGEd) {
    for (int t = threadIdx.x; t < kGTd * kGEd; t += 256) {
      const int col = t / kGEd, e = t % kGEd;
      const long long ee = e0 + e;
      const bool ine = ee < e_end;
      sx[e][col] = (a0 + col < mx && ine) ? X[(long long)(a0 + col) * n + ee] : zero4;
      sy[e][col] = (b0 + col < my && ine) ? Y[(long long)(b0 + col) * n + ee] : zero4;
    }
    __syncthreads();
#pragma unroll 2
    for (int e = 0; e < kGEd; ++e) {
      const ff::PCoef xa[2] = {coef_conj(sx[e][ty]), coef_conj(sx[e][ty + 16])};
      const ff::PVal yb[2] = {ff::p_val(sy[e][tx]), ff::p_val(sy[e][tx + 16])};
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) ff::p_cfma(acc[i][jj].h, acc[i][jj].l, xa[i], yb[jj]);
    }
    __syncthreads();
    if (++stages == kFlushStages || e0 + kGEd >= e_end) {
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int jj = 0; jj < 2; ++jj) {
          const double2 v = ff::to_double2(cff_of(acc[i][jj]));
          acc64[i][jj].x += v.x;
          acc64[i][jj].y += v.y;
          acc[i][jj] = C2{0ull, 0ull};
        }
      stages = 0;
    }
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * jj;
      if (a < mx && b < my) partial[((long long)split * mx + a) * my + b] = acc64[i][jj];
    }
}

__global__ void gram_df_reduce_kernel(const double2* __restrict__ partial, int nsplit, int count, int my, int herm,
                                      double2* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double2 acc = make_double2(0.0, 0.0);
  if (herm && (i / my) / kGTd > (i % my) / kGTd) {  // a tile below the diagonal: not formed
    G[i] = acc;
    return;
  }
  for (int sp = 0; sp < nsplit; ++sp) {
    const double2 v = partial[(long long)sp * count + i];
    acc.x += v.x;
    acc.y += v.y;
  }
  G[i] = acc;
}

// ---- combination X[c] = sum_a T[a] C[a][c] -----------------------------------
// C (FP64, ms x mc) as float-float coefficients in shared memory, kCCd
// outputs a thread, the output in FP64.
constexpr int kCCd = 8;

__global__ void __launch_bounds__(256)
combine_df_kernel(const float4* __restrict__ T, int ms, long long n, const double2* __restrict__ C, int mc,
                  double2* __restrict__ X) {
  extern __shared__ ff::PCoef scd[];
  const int c0 = blockIdx.y * kCCd;
  const int nc = min(kCCd, mc - c0);
  for (int t = threadIdx.x; t < ms * kCCd; t += blockDim.x) {
    const int a = t / kCCd, c = t % kCCd;
    scd[t] = ff::p_coef(ff::from_double2(c < nc ? C[(long long)a * mc + c0 + c] : make_double2(0.0, 0.0)));
  }
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    C2 acc[kCCd];
#pragma unroll
    for (int c = 0; c < kCCd; ++c) acc[c] = C2{0ull, 0ull};
    for (int a = 0; a < ms; ++a) {
      const ff::PVal v = ff::p_val(T[(long long)a * n + e]);
#pragma unroll
      for (int c = 0; c < kCCd; ++c) ff::p_cfma(acc[c].h, acc[c].l, scd[a * kCCd + c], v);
    }
#pragma unroll
    for (int c = 0; c < kCCd; ++c)
      if (c < nc) X[(long long)(c0 + c) * n + e] = ff::to_double2(cff_of(acc[c]));
  }
}

}  // namespace

int cgs2_df(const float4* S, int m, long long n, float4* Q, double2* R, DevBuf& scratch, cudaStream_t s) {
  if (m > kMaxCols) return fail(SSQCD_ERR_ARG, "CGS2 of more than 128 columns");
  if (m <= 0 || n <= 0) return SSQCD_OK;
  const long long nbl = (n + kRB * kEPT - 1) / (kRB * kEPT);
  if (nbl > (1LL << 30)) return fail(SSQCD_ERR_ARG, "CGS2 vectors too long");
  const int nb = (int)nbl;
  const size_t o_part = 0, o_np = o_part + sizeof(double2) * (size_t)kMaxCols * nb,
               o_c = (o_np + sizeof(double) * 2 * nb + 255) / 256 * 256, o_i2 = o_c + sizeof(float4) * kMaxCols,
               o_i1 = o_i2 + sizeof(double) * kMaxCols, o_or = o_i1 + sizeof(double) * kMaxCols,
               o_t = o_or + sizeof(double) * kMaxCols, total = o_t + 256;
  SS_TRY(scratch.alloc(total));
  char* base = scratch.as<char>();
  CgsDf st{reinterpret_cast<double2*>(base + o_part), reinterpret_cast<double*>(base + o_np),
           reinterpret_cast<float4*>(base + o_c), reinterpret_cast<double*>(base + o_i2),
           reinterpret_cast<double*>(base + o_i1), reinterpret_cast<double*>(base + o_or),
           reinterpret_cast<unsigned*>(base + o_t)};
  SS_CUDA(cudaMemsetAsync(st.ticket, 0, sizeof(unsigned), s));
  SS_CUDA(cudaMemsetAsync(R, 0, sizeof(double2) * m * m, s));
  SS_CUDA(cudaMemcpyAsync(Q, S, sizeof(float4) * n * m, cudaMemcpyDeviceToDevice, s));
  auto step = [&](int j, int mode) {
    cgs2_df_step_kernel<<<nb, kRB, 0, s>>>(st, Q, n, m, j, mode, R);
    count_launches(1);
  };
  step(0, kStart);
  if (m > 1) step(0, kSubNext);
  for (int j = 1; j < m; ++j) {
    step(j, kSubProj);
    step(j, kSubNext);
  }
  step(0, kFinal);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int gram_df(const float4* X, int mx, const float4* Y, int my, long long n, double2* G, DevBuf& scratch,
            cudaStream_t s, bool herm) {
  if (mx <= 0 || my <= 0) return SSQCD_OK;
  if (herm && mx != my) return fail(SSQCD_ERR_ARG, "gram_df: a Hermitian product needs mx == my");
  const int ta = (mx + kGTd - 1) / kGTd, tb = (my + kGTd - 1) / kGTd;
  const int tiles = herm ? ta * (ta + 1) / 2 : ta * tb;
  long long nsplit = (4LL * 152 + tiles - 1) / tiles;
  const long long min_chunk = 256;
  if (nsplit * min_chunk > n) nsplit = (n + min_chunk - 1) / min_chunk;
  if (nsplit < 1) nsplit = 1;
  long long chunk = (n + nsplit - 1) / nsplit;
  chunk = (chunk + kGEd - 1) / kGEd * kGEd;
  nsplit = (n + chunk - 1) / chunk;
  SS_TRY(scratch.alloc(sizeof(double2) * nsplit * mx * my));
  gram_df_partial_kernel<<<dim3(ta, tb, (unsigned)nsplit), 256, 0, s>>>(X, mx, Y, my, n, chunk,
                                                                         scratch.as<double2>(), herm ? 1 : 0);
  SS_CHECK_LAUNCH();
  const int count = mx * my;
  gram_df_reduce_kernel<<<grid_for(count, 256), 256, 0, s>>>(scratch.as<double2>(), (int)nsplit, count, my,
                                                              herm ? 1 : 0, G);
  count_launches(2);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int combine_df(const float4* T, int ms, long long n, const double2* C, int mc, double2* X, cudaStream_t s) {
  if (ms <= 0 || mc <= 0 || n <= 0) return SSQCD_OK;
  const int cy = (mc + kCCd - 1) / kCCd;
  long long bx = (n + 255) / 256;
  const long long cap = (4LL * 152 + cy - 1) / cy;
  if (bx > cap) bx = cap;
  const size_t shm = sizeof(ff::PCoef) * ms * kCCd;
  if (shm > 48 * 1024) {  // raised only: concurrent solves share the kernel's attribute
    static std::mutex mu;
    static size_t set = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (shm > set) {
      SS_CUDA(cudaFuncSetAttribute(combine_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      set = shm;
    }
  }
  combine_df_kernel<<<dim3((unsigned)bx, cy), 256, shm, s>>>(T, ms, n, C, mc, X);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

}  // namespace ssqcd
