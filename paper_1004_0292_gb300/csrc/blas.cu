// Layout conversions and the FP64 dense block operations of the post-solve
// steps: moment combination (Eq. 2), the Gram / projected matrices and the
// basis combinations of Rayleigh-Ritz (Section 2.1), residual norms.
//
// All reductions are two-stage with a fixed order (per-block partial sums,
// then one pass over the partials in block order), so results do not depend
// on scheduling.
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
                    long long chunk, double2* __restrict__ partial) {
  __shared__ double2 sx[kGE][kGT + 1];
  __shared__ double2 sy[kGE][kGT + 1];
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

__global__ void gram_reduce_kernel(const double2* __restrict__ partial, int nsplit, int count,
                                   double2* __restrict__ G) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double2 acc = make_double2(0.0, 0.0);
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


// ---- classical Gram-Schmidt with one re-orthogonalisation pass (CGS2) ----
// Column j of the basis: h = Q[0:j]^H v; v -= Q[0:j] h (twice); R[0:j, j]
// accumulates both h; R[j, j] = ||v||; Q_j = v / ||v||.
constexpr int kPC = 8;  // basis vectors per thread in the projection kernel

// partial[(a) * nb + blk] = sum over block blk's elements of conj(Q_a) v
__global__ void __launch_bounds__(kRedBlock)
proj_partial_kernel(const double2* __restrict__ Q, int j, const double2* __restrict__ v, long long n,
                    double2* __restrict__ partial) {
  const int a0 = blockIdx.y * kPC;
  double2 acc[kPC];
#pragma unroll
  for (int c = 0; c < kPC; ++c) acc[c] = make_double2(0.0, 0.0);
  for (long long e = blockIdx.x * (long long)kRedBlock + threadIdx.x; e < n; e += (long long)gridDim.x * kRedBlock) {
    const double2 x = v[e];
#pragma unroll
    for (int c = 0; c < kPC; ++c) {
      if (a0 + c < j) {
        const double2 q = Q[(long long)(a0 + c) * n + e];
        acc[c].x = fma(q.x, x.x, fma(q.y, x.y, acc[c].x));
        acc[c].y = fma(q.x, x.y, fma(-q.y, x.x, acc[c].y));
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kPC; ++c) {
    const double rx = block_reduce(acc[c].x);
    __syncthreads();
    const double ry = block_reduce(acc[c].y);
    __syncthreads();
    if (threadIdx.x == 0 && a0 + c < j) partial[(long long)(a0 + c) * gridDim.x + blockIdx.x] = make_double2(rx, ry);
  }
}

// h[a] = sum_b partial[a * nb + b]; R[a * m + j] += h[a]; one warp per a
__global__ void proj_reduce_kernel(const double2* __restrict__ partial, int nb, int j, double2* __restrict__ h,
                                   double2* __restrict__ R, int m) {
  const int a = blockIdx.x;
  if (a >= j) return;
  double sx = 0.0, sy = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) {
    sx += partial[(long long)a * nb + b].x;
    sy += partial[(long long)a * nb + b].y;
  }
  sx = warp_sum(sx);
  sy = warp_sum(sy);
  if (threadIdx.x == 0) {
    h[a] = make_double2(sx, sy);
    R[(long long)a * m + j].x += sx;
    R[(long long)a * m + j].y += sy;
  }
}

// v -= Q[0:j] h
__global__ void __launch_bounds__(256)
proj_subtract_kernel(const double2* __restrict__ Q, int j, const double2* __restrict__ h, double2* __restrict__ v,
                     long long n) {
  extern __shared__ double2 sh_h[];
  for (int a = threadIdx.x; a < j; a += blockDim.x) sh_h[a] = h[a];
  __syncthreads();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double2 x = v[e];
    for (int a = 0; a < j; ++a) {
      const double2 q = Q[(long long)a * n + e];
      const double2 c = sh_h[a];
      x.x -= q.x * c.x - q.y * c.y;
      x.y -= q.x * c.y + q.y * c.x;
    }
    v[e] = x;
  }
}

// R[j, j] = ||v|| (from the summed square), Q_j = v / ||v||; a vector whose
// norm fell below 1e-15 of the original column's is numerically dependent
// and becomes zero (R[j, j] = 0).
__global__ void normalise_col_kernel(double2* __restrict__ v, long long n, const double* __restrict__ nrm2,
                                     const double* __restrict__ orig2, double2* __restrict__ R, int m, int j) {
  const double s2 = *nrm2;
  const bool dep = !(s2 > 1e-30 * (*orig2));
  const double inv = dep ? 0.0 : 1.0 / sqrt(s2);
  if (blockIdx.x == 0 && threadIdx.x == 0) R[(long long)j * m + j] = make_double2(dep ? 0.0 : sqrt(s2), 0.0);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double2 x = v[e];
    x.x *= inv;
    x.y *= inv;
    v[e] = x;
  }
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
         cudaStream_t s) {
  if (mx <= 0 || my <= 0) return SSQCD_OK;
  const int ta = (mx + kGT - 1) / kGT, tb = (my + kGT - 1) / kGT;
  // enough splits to give every SM a few blocks
  long long nsplit = (4LL * 152 + ta * tb - 1) / (ta * tb);
  const long long min_chunk = 256;
  if (nsplit * min_chunk > n) nsplit = (n + min_chunk - 1) / min_chunk;
  if (nsplit < 1) nsplit = 1;
  long long chunk = (n + nsplit - 1) / nsplit;
  chunk = (chunk + kGE - 1) / kGE * kGE;
  nsplit = (n + chunk - 1) / chunk;
  SS_TRY(scratch.alloc(sizeof(double2) * nsplit * mx * my));
  gram_partial_kernel<<<dim3(ta, tb, (unsigned)nsplit), 256, 0, s>>>(X, mx, Y, my, n, chunk,
                                                                      scratch.as<double2>());
  SS_CHECK_LAUNCH();
  const int count = mx * my;
  gram_reduce_kernel<<<grid_for(count, 256), 256, 0, s>>>(scratch.as<double2>(), (int)nsplit, count, G);
  count_launches(2);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}


int cgs2(const double2* S, int m, long long n, double2* Q, double2* R, DevBuf& scratch, cudaStream_t s) {
  const int nb = reduce_blocks(n);
  const size_t part_bytes = sizeof(double2) * (size_t)nb * m;
  SS_TRY(scratch.alloc(part_bytes + sizeof(double2) * m + sizeof(double) * (2 * (size_t)nb + 2)));
  double2* partial = scratch.as<double2>();
  double2* h = partial + (size_t)nb * m;
  double* npart = reinterpret_cast<double*>(h + m);
  double* nrm2 = npart + nb;
  double* orig2 = nrm2 + 1;
  SS_CUDA(cudaMemsetAsync(R, 0, sizeof(double2) * m * m, s));
  SS_CUDA(cudaMemcpyAsync(Q, S, sizeof(double2) * n * m, cudaMemcpyDeviceToDevice, s));
  if (m * sizeof(double2) > 48 * 1024)
    SS_CUDA(cudaFuncSetAttribute(proj_subtract_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(m * sizeof(double2))));
  for (int j = 0; j < m; ++j) {
    double2* v = Q + (long long)j * n;
    SS_TRY(norm2_partials(v, 1, n, npart, nb, s));
    SS_TRY(sum_partials(npart, 1, nb, orig2, s));
    for (int pass = 0; pass < 2 && j > 0; ++pass) {
      proj_partial_kernel<<<dim3(nb, (j + kPC - 1) / kPC), kRedBlock, 0, s>>>(Q, j, v, n, partial);
      proj_reduce_kernel<<<j, 32, 0, s>>>(partial, nb, j, h, R, m);
      proj_subtract_kernel<<<nb, 256, sizeof(double2) * j, s>>>(Q, j, h, v, n);
      count_launches(3);
      SS_CHECK_LAUNCH();
    }
    SS_TRY(norm2_partials(v, 1, n, npart, nb, s));
    SS_TRY(sum_partials(npart, 1, nb, nrm2, s));
    normalise_col_kernel<<<nb, 256, 0, s>>>(v, n, nrm2, orig2, R, m, j);
    count_launches(1);
    SS_CHECK_LAUNCH();
  }
  return SSQCD_OK;
}

int combine(const double2* S, int ms, long long n, const double2* C, int mc, double2* Q, cudaStream_t s) {
  if (ms <= 0 || mc <= 0 || n <= 0) return SSQCD_OK;
  const int cy = (mc + kCC - 1) / kCC;
  long long bx = (n + 255) / 256;
  const long long cap = (4LL * 152 + cy - 1) / cy;
  if (bx > cap) bx = cap;
  const size_t shm = sizeof(double2) * ms * kCC;
  if (shm > 48 * 1024) {
    SS_CUDA(cudaFuncSetAttribute(combine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
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
