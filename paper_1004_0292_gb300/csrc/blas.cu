// Layout conversions and the FP64 dense block operations of the post-solve
// steps: moment combination (Eq. 2), the Gram / projected matrices and the
// basis combinations of Rayleigh-Ritz (Section 2.1), residual norms.
//
// All reductions are two-stage with a fixed order (per-block partial sums,
// then one pass over the partials in block order), so results do not depend
// on scheduling.
#include <algorithm>
#include <mutex>

#include "internal.h"

namespace ssqcd {
namespace {

// user [nf][V][12] -> device [nf][12][V]
__global__ void pack_spinor_kernel(const double2* __restrict__ user, double2* __restrict__ dev, int nf,
                                   int V) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)nf * V) return;
  const long long f = i / V;
  const int s = (int)(i % V);
  const double2* src = user + (f * V + s) * 12;
  double2* dst = dev + f * 12 * (long long)V + s;
#pragma unroll
  for (int c = 0; c < 12; ++c) dst[(long long)c * V] = src[c];
}

__global__ void unpack_spinor_kernel(const double2* __restrict__ dev, double2* __restrict__ user, int nf,
                                     int V) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)nf * V) return;
  const long long f = i / V;
  const int s = (int)(i % V);
  const double2* src = dev + f * 12 * (long long)V + s;
  double2* dst = user + (f * V + s) * 12;
#pragma unroll
  for (int c = 0; c < 12; ++c) dst[c] = src[(long long)c * V];
}

// user [4][V][3][3] -> device [4][9][V]
__global__ void pack_gauge_kernel(const double2* __restrict__ user, double2* __restrict__ dev, int V) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= 4LL * V) return;
  const int mu = (int)(i / V), s = (int)(i % V);
  const double2* src = user + ((long long)mu * V + s) * 9;
#pragma unroll
  for (int e = 0; e < 9; ++e) dev[((long long)mu * 9 + e) * V + s] = src[e];
}

constexpr int kRedBlock = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_reduce(double v) {
  __shared__ double sh[kRedBlock / 32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < kRedBlock / 32; ++i) r += sh[i];
  return r;
}

// partial[v * nblocks + b] = sum over block b's stride of |x_v|^2
__global__ void norm2_partial_kernel(const double2* __restrict__ x, long long n, double* __restrict__ partial) {
  const int v = blockIdx.y;
  const double2* xv = x + (long long)v * n;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)kRedBlock + threadIdx.x; i < n; i += (long long)gridDim.x * kRedBlock) {
    const double2 z = xv[i];
    acc = fma(z.x, z.x, fma(z.y, z.y, acc));
  }
  const double r = block_reduce(acc);
  if (threadIdx.x == 0) partial[(long long)v * gridDim.x + blockIdx.x] = r;
}

// out[v] = sum_b partial[v * nblocks + b], one warp per v, fixed order
__global__ void sum_partials_kernel(const double* __restrict__ partial, int nvec, int nblocks,
                                    double* __restrict__ out) {
  const int v = blockIdx.x;
  if (v >= nvec) return;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 32) acc += partial[(long long)v * nblocks + b];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) out[v] = acc;
}

// Gram-type product G = X^H Y, X: [mx][n], Y: [my][n] (each vector
// contiguous).  Block (tile_a, tile_b, split) accumulates a 32 x 32 tile of
// G over its share of the n elements, staged through shared memory; thread
// (ty, tx) of the 16 x 16 block owns entries (ty + 16 i, tx + 16 j).
constexpr int kGT = 32;     // tile of G
constexpr int kGE = 32;     // elements per shared-memory stage

__global__ void __launch_bounds__(256)
gram_partial_kernel(const double2* __restrict__ X, int mx, const double2* __restrict__ Y, int my, long long n,
                    long long chunk, double2* __restrict__ partial, int herm) {
  __shared__ double2 sx[kGE][kGT + 1];
  __shared__ double2 sy[kGE][kGT + 1];
  // herm: G is Hermitian, only the tiles on and above the diagonal
  if (herm && blockIdx.x > blockIdx.y) return;
  const int a0 = blockIdx.x * kGT, b0 = blockIdx.y * kGT;
  const int split = blockIdx.z;
  const long long e_begin = split * chunk;
  const long long e_end = min(n, e_begin + chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
  for (long long e0 = e_begin; e0 < e_end; e0 += kGE) {
    // load kGT vectors x kGE elements of X and Y
    for (int t = threadIdx.x; t < kGT * kGE; t += 256) {
      const int col = t / kGE, e = t % kGE;
      const long long ee = e0 + e;
      const bool ine = ee < e_end;
      sx[e][col] = (a0 + col < mx && ine) ? X[(long long)(a0 + col) * n + ee] : make_double2(0.0, 0.0);
      sy[e][col] = (b0 + col < my && ine) ? Y[(long long)(b0 + col) * n + ee] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int e = 0; e < kGE; ++e) {
      double2 xa[2], yb[2];
      xa[0] = sx[e][ty];
      xa[1] = sx[e][ty + 16];
      yb[0] = sy[e][tx];
      yb[1] = sy[e][tx + 16];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          // conj(x) * y
          acc[i][j].x = fma(xa[i].x, yb[j].x, fma(xa[i].y, yb[j].y, acc[i][j].x));
          acc[i][j].y = fma(xa[i].x, yb[j].y, fma(-xa[i].y, yb[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
      if (a < mx && b < my) partial[((long long)split * mx + a) * my + b] = acc[i][j];
    }
}

__global__ void gram_reduce_kernel(const double2* __restrict__ partial, int nsplit, int count, int my, int herm,
                                   double2* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double2 acc = make_double2(0.0, 0.0);
  if (herm && (i / my) / kGT > (i % my) / kGT) {  // a tile below the diagonal: not computed
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

// Q[c][e] = sum_a S[a][e] C[a * mc + c] for c < mc; C (ms x mc, row-major) in
// shared memory; each thread owns one element and kCC output vectors.
constexpr int kCC = 8;

__global__ void __launch_bounds__(256)
combine_kernel(const double2* __restrict__ S, int ms, long long n, const double2* __restrict__ C, int mc,
               double2* __restrict__ Q) {
  extern __shared__ double2 sc[];
  const int c0 = blockIdx.y * kCC;
  const int nc = min(kCC, mc - c0);
  for (int t = threadIdx.x; t < ms * kCC; t += blockDim.x) {
    const int a = t / kCC, c = t % kCC;
    sc[t] = (c < nc) ? C[(long long)a * mc + c0 + c] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double2 acc[kCC];
#pragma unroll
    for (int c = 0; c < kCC; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int a = 0; a < ms; ++a) {
      const double2 s = S[(long long)a * n + e];
#pragma unroll
      for (int c = 0; c < kCC; ++c) {
        const double2 w = sc[a * kCC + c];
        acc[c].x = fma(s.x, w.x, fma(-s.y, w.y, acc[c].x));
        acc[c].y = fma(s.x, w.y, fma(s.y, w.x, acc[c].y));
      }
    }
#pragma unroll
    for (int c = 0; c < kCC; ++c)
      if (c < nc) Q[(long long)(c0 + c) * n + e] = acc[c];
  }
}

// partial[c * nb + b] = sum |AX_c - theta_c X_c|^2 and sum |X_c|^2
__global__ void resid_partial_kernel(const double2* __restrict__ AX, const double2* __restrict__ X,
                                     const double* __restrict__ theta, long long n, double* __restrict__ pr,
                                     double* __restrict__ px) {
  const int c = blockIdx.y;
  const double th = theta[c];
  const double2* ax = AX + (long long)c * n;
  const double2* x = X + (long long)c * n;
  double r = 0.0, xx = 0.0;
  for (long long i = blockIdx.x * (long long)kRedBlock + threadIdx.x; i < n; i += (long long)gridDim.x * kRedBlock) {
    const double2 a = ax[i], b = x[i];
    const double dx = fma(-th, b.x, a.x), dy = fma(-th, b.y, a.y);
    r = fma(dx, dx, fma(dy, dy, r));
    xx = fma(b.x, b.x, fma(b.y, b.y, xx));
  }
  const double rr = block_reduce(r);
  __syncthreads();
  const double rx = block_reduce(xx);
  if (threadIdx.x == 0) {
    pr[(long long)c * gridDim.x + blockIdx.x] = rr;
    px[(long long)c * gridDim.x + blockIdx.x] = rx;
  }
}

__global__ void resid_final_kernel(const double* __restrict__ pr, const double* __restrict__ px, int nb, int m,
                                   double* __restrict__ out) {
  const int c = blockIdx.x;
  if (c >= m) return;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += 32) {
    a += pr[(long long)c * nb + i];
    b += px[(long long)c * nb + i];
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if (threadIdx.x == 0) out[c] = sqrt(a) / sqrt(b);
}

__global__ void f64_to_f32_kernel(const double2* __restrict__ in, float2* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double2 z = in[i];
    out[i] = make_float2((float)z.x, (float)z.y);
  }
}

__global__ void f32_to_f64_kernel(const float2* __restrict__ in, double2* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float2 z = in[i];
    out[i] = make_double2((double)z.x, (double)z.y);
  }
}


// ---- classical Gram-Schmidt with one re-orthogonalisation pass (CGS2), two
// fused launches per column ------------------------------------------------------
// The columns are kept unnormalised (v_a, with nu_a^2 = ||v_a||^2 after both
// passes) until one final scaling launch; the projection on Q_a = v_a / nu_a
// is w -= v_a c_a with c_a = (v_a^H w) / nu_a^2 and R[a][j] += (v_a^H w) / nu_a.
// Column j (w = v_j) takes two launches, each over all elements, whose last
// block (ticket) reduces the block partials in block order:
//   kSubProj : w -= sum_a v_a c_a (pass 1)   then partials of v_a^H w (pass 2)
//   kSubNext : w -= sum_a v_a c'_a (pass 2)  then partials of ||w||^2, and for
//              column j + 1 (u): partials of v_a^H u (a <= j, v_j from
//              registers) and ||u||^2; the last block forms nu_j^2 first
// and kStart gives column 0's norm; a column whose norm fell below 1e-15 of
// its original is dependent: Q_j = 0, R[j][j] = 0 and c_j = 0 from then on.
// Per thread: kCE elements, kCE x kPT loads in flight (the grid covers n);
// the projections in tiles of kPT columns, each tile's 2 kPT sums over the
// thread's elements reduced by halving warp exchanges and one pass over the
// warps, so the reduction's FP64 additions are spread over kCE elements
// (one element a thread spent ~2 additions a column and element on them,
// against 8 FP64 operations of projection).
enum CgsMode : int { kStart = 0, kSubProj = 1, kSubNext = 2, kFinal = 3 };

// Warp sums of 8 values at once by halving exchanges: at the step with offset
// O a lane keeps one half of its values and adds the partner's copy of that
// half (4 + 2 + 1 additions), then two exchanges over the low lane bits.  On
// return lane L holds the warp total of value (L >> 2) & 7.
template <int O, int HALF>
__device__ __forceinline__ void halve_step8(double (&v)[8], int lane) {
  const bool up = (lane & O) != 0;
#pragma unroll
  for (int i = 0; i < HALF; ++i) {
    const double send = up ? v[i] : v[i + HALF];
    const double keep = up ? v[i + HALF] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
  }
}
__device__ __forceinline__ double warp_reduce8(double (&v)[8]) {
  const int lane = threadIdx.x & 31;
  halve_step8<16, 4>(v, lane);
  halve_step8<8, 2>(v, lane);
  halve_step8<4, 1>(v, lane);
  double t = v[0] + __shfl_xor_sync(0xffffffffu, v[0], 2);
  return t + __shfl_xor_sync(0xffffffffu, t, 1);
}
constexpr int kPT = 4;
constexpr int kCE = 4;
constexpr int kCgsMaxCols = 128;

struct CgsState {
  double2* partial;   // [kCgsMaxCols][nb]
  double* npart;      // [2][nb]: ||w||^2, ||u||^2
  double2* c;         // [kCgsMaxCols] subtraction coefficients of the next launch
  double* inv_nu2;    // [kCgsMaxCols] 1 / nu_a^2 (0: dependent)
  double* inv_nu;     // [kCgsMaxCols] 1 / nu_a   (0: dependent)
  double* orig2;      // [kCgsMaxCols] ||v_a||^2 before the projections
  unsigned* ticket;
};

__global__ void __launch_bounds__(kRedBlock)
cgs2_step_kernel(CgsState st, double2* __restrict__ Q, long long n, int m, int j, int mode,
                 double2* __restrict__ R) {
  __shared__ double2 s_c[kCgsMaxCols];
  __shared__ double s_red[kRedBlock / 32][2 * kPT];
  __shared__ double s_nred[2][kRedBlock / 32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nb = gridDim.x;
  long long ei[kCE];
  bool in[kCE];
#pragma unroll
  for (int i = 0; i < kCE; ++i) {
    ei[i] = blockIdx.x * (long long)(kRedBlock * kCE) + i * kRedBlock + threadIdx.x;
    in[i] = ei[i] < n;
  }
  if (mode == kFinal) {  // Q_a = v_a / nu_a for every column
    for (int a = 0; a < m; ++a) {
      const double s = st.inv_nu[a];
#pragma unroll
      for (int i = 0; i < kCE; ++i)
        if (in[i]) {
          double2 x = Q[(long long)a * n + ei[i]];
          Q[(long long)a * n + ei[i]] = make_double2(x.x * s, x.y * s);
        }
    }
    return;
  }
  // 1. the subtraction w -= sum_a v_a c_a on column j
  double2 x[kCE];
#pragma unroll
  for (int i = 0; i < kCE; ++i) x[i] = in[i] ? Q[(long long)j * n + ei[i]] : make_double2(0.0, 0.0);
  if (mode == kSubProj || mode == kSubNext) {
    for (int a = threadIdx.x; a < j; a += kRedBlock) s_c[a] = st.c[a];
    __syncthreads();
    for (int a0 = 0; a0 < j; a0 += kPT) {
      double2 q[kPT][kCE];
#pragma unroll
      for (int c = 0; c < kPT; ++c)
#pragma unroll
        for (int i = 0; i < kCE; ++i)
          q[c][i] = (a0 + c < j && in[i]) ? Q[(long long)(a0 + c) * n + ei[i]] : make_double2(0.0, 0.0);
#pragma unroll
      for (int c = 0; c < kPT; ++c) {
        if (a0 + c < j) {
          const double2 h = s_c[a0 + c];
#pragma unroll
          for (int i = 0; i < kCE; ++i) {
            x[i].x -= q[c][i].x * h.x - q[c][i].y * h.y;
            x[i].y -= q[c][i].x * h.y + q[c][i].y * h.x;
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kCE; ++i)
      if (in[i]) Q[(long long)j * n + ei[i]] = x[i];
  }
  // 2. partials: projections of column jp on its first np columns, norms
  const int jp = mode == kSubNext ? j + 1 : j;
  const bool next = mode == kSubNext && jp < m;
  const int np = mode == kSubProj ? j : (next ? jp : 0);
  double2 y[kCE];  // the vector being projected
#pragma unroll
  for (int i = 0; i < kCE; ++i) y[i] = next ? (in[i] ? Q[(long long)jp * n + ei[i]] : make_double2(0.0, 0.0)) : x[i];
  for (int a0 = 0; a0 < np; a0 += kPT) {
    double2 q[kPT][kCE];
#pragma unroll
    for (int c = 0; c < kPT; ++c) {
      const int a = a0 + c;
#pragma unroll
      for (int i = 0; i < kCE; ++i)
        q[c][i] = (a < np && in[i]) ? ((next && a == j) ? x[i] : Q[(long long)a * n + ei[i]]) : make_double2(0.0, 0.0);
    }
    double acc[2 * kPT];  // re, im of sum over the thread's elements of conj(v_a) y
#pragma unroll
    for (int c = 0; c < kPT; ++c) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int i = 0; i < kCE; ++i) {
        re = fma(q[c][i].x, y[i].x, fma(q[c][i].y, y[i].y, re));
        im = fma(q[c][i].x, y[i].y, fma(-q[c][i].y, y[i].x, im));
      }
      acc[2 * c] = re;
      acc[2 * c + 1] = im;
    }
    const double t = warp_reduce8(acc);
    if ((lane & 3) == 0) s_red[w][lane >> 2] = t;
    __syncthreads();
    if (threadIdx.x < 2 * kPT && a0 + (int)threadIdx.x / 2 < np) {
      double u = s_red[0][threadIdx.x];
      for (int ww = 1; ww < kRedBlock / 32; ++ww) u += s_red[ww][threadIdx.x];
      reinterpret_cast<double*>(st.partial)[2 * ((long long)(a0 + threadIdx.x / 2) * nb + blockIdx.x) +
                                            (threadIdx.x & 1)] = u;
    }
    __syncthreads();
  }
  // norms: kStart / kSubNext: ||w||^2 of column j; kSubNext with a next
  // column: also ||u||^2
  const bool norm_w = mode == kStart || mode == kSubNext;
  if (norm_w || next) {
    double v0 = 0.0, v1 = 0.0;
#pragma unroll
    for (int i = 0; i < kCE; ++i) {
      v0 = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, v0));
      if (next) v1 = fma(y[i].x, y[i].x, fma(y[i].y, y[i].y, v1));
    }
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    if (lane == 0) {
      s_nred[0][w] = v0;
      s_nred[1][w] = v1;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      double t = 0.0;
      for (int ww = 0; ww < kRedBlock / 32; ++ww) t += s_nred[threadIdx.x][ww];
      st.npart[threadIdx.x * nb + blockIdx.x] = t;
    }
  }
  // 3. the last block reduces the partials in block order
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(st.ticket, 1u) == (unsigned)nb - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (norm_w || next) {  // norms first: nu_j^2 enters the coefficients below
    if (w < 2 && (w == 0 ? norm_w : next)) {
      double t = 0.0;
      for (int b = lane; b < nb; b += 32) t += __ldcg(st.npart + w * nb + b);
      t = warp_sum(t);
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
  // warp w: columns [a0, a0 + kPT) for a0 = kPT w, kPT (w + 8), ...
  for (int a0 = kPT * w; a0 < np; a0 += kPT * (kRedBlock / 32)) {
    double acc[2 * kPT];
#pragma unroll
    for (int c = 0; c < 2 * kPT; ++c) acc[c] = 0.0;
    for (int b = lane; b < nb; b += 32) {
#pragma unroll
      for (int c = 0; c < kPT; ++c) {
        if (a0 + c < np) {
          const double2 t = __ldcg(st.partial + (long long)(a0 + c) * nb + b);
          acc[2 * c] += t.x;
          acc[2 * c + 1] += t.y;
        }
      }
    }
    const double t = warp_reduce8(acc);
    const int a = a0 + (lane >> 3), comp = (lane >> 2) & 1;
    if ((lane & 3) == 0 && a < np) {
      // v_a^H y: subtraction coefficient / nu_a^2, R entry / nu_a
      const double i2 = __ldcg(st.inv_nu2 + a), i1 = __ldcg(st.inv_nu + a);
      reinterpret_cast<double*>(st.c)[2 * a + comp] = t * i2;
      reinterpret_cast<double*>(R)[2 * ((long long)a * m + jp) + comp] += t * i1;
    }
  }
  if (threadIdx.x == 0) *st.ticket = 0u;
}

int reduce_blocks(long long n) {
  long long b = (n + kRedBlock - 1) / kRedBlock;
  if (b > 1216) b = 1216;  // 152 SMs x 8
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

int pack_spinors(const double2* user, double2* dev, int nfields, int V, cudaStream_t s) {
  const long long w = (long long)nfields * V;
  if (w == 0) return SSQCD_OK;
  pack_spinor_kernel<<<grid_for(w, 256), 256, 0, s>>>(user, dev, nfields, V);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int unpack_spinors(const double2* dev, double2* user, int nfields, int V, cudaStream_t s) {
  const long long w = (long long)nfields * V;
  if (w == 0) return SSQCD_OK;
  unpack_spinor_kernel<<<grid_for(w, 256), 256, 0, s>>>(dev, user, nfields, V);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int pack_gauge64(const double2* user, double2* dev, int V, cudaStream_t s) {
  pack_gauge_kernel<<<grid_for(4LL * V, 256), 256, 0, s>>>(user, dev, V);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int norm2_partials(const double2* x, int nvec, long long n, double* partial, int nblocks, cudaStream_t s) {
  norm2_partial_kernel<<<dim3(nblocks, nvec), kRedBlock, 0, s>>>(x, n, partial);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int sum_partials(const double* partial, int nvec, int nblocks, double* out, cudaStream_t s) {
  sum_partials_kernel<<<nvec, 32, 0, s>>>(partial, nvec, nblocks, out);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int gram(const double2* X, int mx, const double2* Y, int my, long long n, double2* G, DevBuf& scratch,
         cudaStream_t s, bool herm) {
  if (mx <= 0 || my <= 0) return SSQCD_OK;
  if (herm && mx != my) return fail(SSQCD_ERR_ARG, "gram: a Hermitian product needs mx == my");
  const int ta = (mx + kGT - 1) / kGT, tb = (my + kGT - 1) / kGT;
  const int tiles = herm ? ta * (ta + 1) / 2 : ta * tb;
  // enough splits to give every SM a few blocks
  long long nsplit = (4LL * 152 + tiles - 1) / tiles;
  const long long min_chunk = 256;
  if (nsplit * min_chunk > n) nsplit = (n + min_chunk - 1) / min_chunk;
  if (nsplit < 1) nsplit = 1;
  long long chunk = (n + nsplit - 1) / nsplit;
  chunk = (chunk + kGE - 1) / kGE * kGE;
  nsplit = (n + chunk - 1) / chunk;
  SS_TRY(scratch.alloc(sizeof(double2) * nsplit * mx * my));
  gram_partial_kernel<<<dim3(ta, tb, (unsigned)nsplit), 256, 0, s>>>(X, mx, Y, my, n, chunk,
                                                                      scratch.as<double2>(), herm ? 1 : 0);
  SS_CHECK_LAUNCH();
  const int count = mx * my;
  gram_reduce_kernel<<<grid_for(count, 256), 256, 0, s>>>(scratch.as<double2>(), (int)nsplit, count, my,
                                                           herm ? 1 : 0, G);
  count_launches(2);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}


int cgs2(const double2* S, int m, long long n, double2* Q, double2* R, DevBuf& scratch, cudaStream_t s,
         const cudaEvent_t* group_ready, int group) {
  if (m > kCgsMaxCols) return fail(SSQCD_ERR_ARG, "CGS2 of more than 128 columns");
  if (m <= 0 || n <= 0) return SSQCD_OK;
  const long long nbl = (n + kRedBlock * kCE - 1) / (kRedBlock * kCE);  // kCE elements a thread
  if (nbl > (1LL << 30)) return fail(SSQCD_ERR_ARG, "CGS2 vectors too long");
  const int nb = (int)nbl;
  const size_t o_part = 0, o_np = o_part + sizeof(double2) * (size_t)kCgsMaxCols * nb,
               o_c = (o_np + sizeof(double) * 2 * nb + 255) / 256 * 256, o_i2 = o_c + sizeof(double2) * kCgsMaxCols,
               o_i1 = o_i2 + sizeof(double) * kCgsMaxCols, o_or = o_i1 + sizeof(double) * kCgsMaxCols,
               o_t = o_or + sizeof(double) * kCgsMaxCols, total = o_t + 256;
  SS_TRY(scratch.alloc(total));
  char* base = scratch.as<char>();
  CgsState st{reinterpret_cast<double2*>(base + o_part), reinterpret_cast<double*>(base + o_np),
              reinterpret_cast<double2*>(base + o_c), reinterpret_cast<double*>(base + o_i2),
              reinterpret_cast<double*>(base + o_i1), reinterpret_cast<double*>(base + o_or),
              reinterpret_cast<unsigned*>(base + o_t)};
  SS_CUDA(cudaMemsetAsync(st.ticket, 0, sizeof(unsigned), s));
  SS_CUDA(cudaMemsetAsync(R, 0, sizeof(double2) * m * m, s));
  // the columns enter Q as they are first needed; with group_ready, group g
  // (columns [g group, (g + 1) group)) waits for its event first, so the
  // orthogonalisation can start while later columns are still being formed
  if (group_ready == nullptr || group <= 0) group = m;
  int copied = 0;  // columns [0, copied) are in Q
  auto need = [&](int j) -> int {
    while (copied <= j) {
      const int g = copied / group, c1 = std::min(m, copied + group);
      if (group_ready != nullptr && group_ready[g] != nullptr) SS_CUDA(cudaStreamWaitEvent(s, group_ready[g], 0));
      SS_CUDA(cudaMemcpyAsync(Q + (size_t)copied * n, S + (size_t)copied * n, sizeof(double2) * n * (c1 - copied),
                              cudaMemcpyDeviceToDevice, s));
      copied = c1;
    }
    return SSQCD_OK;
  };
  auto step = [&](int j, int mode) {
    cgs2_step_kernel<<<nb, kRedBlock, 0, s>>>(st, Q, n, m, j, mode, R);
    count_launches(1);
  };
  SS_TRY(need(0));
  step(0, kStart);    // nu_0 (column 0 has nothing to project on)
  if (m > 1) {
    // column 0's partials for column 1 (pass 1) come from a kSubNext on
    // column 0 with nothing to subtract
    SS_TRY(need(1));
    step(0, kSubNext);
  }
  for (int j = 1; j < m; ++j) {
    step(j, kSubProj);  // pass 1 subtraction, pass 2 partials
    if (j + 1 < m) SS_TRY(need(j + 1));
    step(j, kSubNext);  // pass 2 subtraction, nu_j, pass 1 partials of column j + 1
  }
  step(0, kFinal);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int combine(const double2* S, int ms, long long n, const double2* C, int mc, double2* Q, cudaStream_t s) {
  if (ms <= 0 || mc <= 0 || n <= 0) return SSQCD_OK;
  const int cy = (mc + kCC - 1) / kCC;
  long long bx = (n + 255) / 256;
  const long long cap = (4LL * 152 + cy - 1) / cy;
  if (bx > cap) bx = cap;
  const size_t shm = sizeof(double2) * ms * kCC;
  if (shm > 48 * 1024) {  // raised only: concurrent solves share the kernel's attribute
    static std::mutex mu;
    static size_t set = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (shm > set) {
      SS_CUDA(cudaFuncSetAttribute(combine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
      set = shm;
    }
  }
  combine_kernel<<<dim3((unsigned)bx, cy), 256, shm, s>>>(S, ms, n, C, mc, Q);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int col_residual_norms(const double2* AX, const double2* X, const double* theta, int m, long long n,
                       double* out, DevBuf& scratch, cudaStream_t s) {
  if (m <= 0) return SSQCD_OK;
  const int nb = reduce_blocks(n);
  SS_TRY(scratch.alloc(sizeof(double) * 2 * (size_t)nb * m));
  double* pr = scratch.as<double>();
  double* px = pr + (size_t)nb * m;
  resid_partial_kernel<<<dim3(nb, m), kRedBlock, 0, s>>>(AX, X, theta, n, pr, px);
  SS_CHECK_LAUNCH();
  resid_final_kernel<<<m, 32, 0, s>>>(pr, px, nb, m, out);
  count_launches(2);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int convert_f64_to_f32(const double2* in, float2* out, long long n, cudaStream_t s) {
  f64_to_f32_kernel<<<reduce_blocks(n), 256, 0, s>>>(in, out, n);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

int convert_f32_to_f64(const float2* in, double2* out, long long n, cudaStream_t s) {
  f32_to_f64_kernel<<<reduce_blocks(n), 256, 0, s>>>(in, out, n);
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}

}  // namespace ssqcd
