// ssqcd_moments_noalloc: the moment combination s_hat[l][k] = sum_j c_jk y[l][j]
// with c_jk = w_j zeta_j^k, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// moments: programs that hand all device memory to their own pool or arena
// up front (a framework's caching allocator, an embedded solver inside a
// larger simulation), and allocation-free loops with fixed memory budgets.
// This entry point takes device pointers for the input and the output and
// keeps its only scratch -- the N x M coefficient table -- in a fixed
// file-scope device array, so a call allocates nothing.
//
// The weights and nodes reach the device by value, as kernel parameters (at
// most 256 of each: 8 KiB of parameters); a first kernel forms the table
// c_jk = w_j zeta_j^k in the device array, a second one forms the moments.
// No host buffer outlives the call and nothing is copied from host memory.
//
// The array holds at most kMaxCoef = 4096 complex coefficients (64 KiB), so
// N * M <= 4096 (and N <= 256); every GPU that loads this library holds it
// until the process exits.  All calls share the one array, which keeps the
// last call's table: each call overwrites the N * M entries it uses before
// its second kernel reads them, so nothing has to start at zero, but calls
// whose kernels overlap on the GPU (different streams, no ordering between
// them) race on the table.  Calls on one stream are ordered.
#include <mutex>
#include <vector>

#include "internal.h"

namespace ssqcd {
namespace {

constexpr int kMaxCoef = 4096;
constexpr int kMaxNoallocShifts = 256;
constexpr int kMaxDevices = 64;

// The scratch: one coefficient table per GPU (file scope, static storage).
static __device__ __align__(256) double2 g_moment_coef[kMaxCoef];

// In host code g_moment_coef is only a host-side stand-in, not a device
// address; the device address comes from cudaGetSymbolAddress, once per
// device and process, with that device current (the first call on a
// device).  The cached address belongs to that device's primary context: a
// process that destroys the context (cudaDeviceReset) must not call this
// entry point on that device again.
std::mutex g_setup_mutex;
double2* g_coef_ptr[kMaxDevices] = {nullptr};

int coef_table(int dev, double2** out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(SSQCD_ERR_ARG, "moments_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_coef_ptr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_moment_coef);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_moment_coef)", __FILE__, __LINE__);
    g_coef_ptr[dev] = static_cast<double2*>(p);
  }
  *out = g_coef_ptr[dev];
  return SSQCD_OK;
}

constexpr int kCols = 8;  // output vectors per thread

// Weights and nodes of one call, passed by value as a kernel parameter.
struct NodeSet {
  double2 w[kMaxNoallocShifts];
  double2 zeta[kMaxNoallocShifts];
};

// coef[j * M + k] = w_j zeta_j^k, one thread per node j (powers by repeated
// multiplication, k ascending).
__global__ void moment_coef_kernel(const NodeSet ns, int N, int M, double2* __restrict__ coef) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const double2 w = ns.w[j], a = ns.zeta[j];
  double zr = 1.0, zi = 0.0;
  for (int k = 0; k < M; ++k) {
    coef[j * M + k] = make_double2(w.x * zr - w.y * zi, w.x * zi + w.y * zr);
    const double nr = zr * a.x - zi * a.y, ni = zr * a.y + zi * a.x;
    zr = nr;
    zi = ni;
  }
}

// s_hat[l][c] (n complex) = sum_j y[l][j] coef[j * M + c]; blockIdx.z = l.
// The coefficient columns of this block are staged in shared memory.
__global__ void __launch_bounds__(256)
moments_noalloc_kernel(const double2* __restrict__ y, int N, int M, long long n, const double2* __restrict__ coef,
                       double2* __restrict__ s_hat) {
  extern __shared__ double2 sc[];
  const int l = blockIdx.z;
  const int c0 = blockIdx.y * kCols;
  const int nc = min(kCols, M - c0);
  for (int t = threadIdx.x; t < N * kCols; t += blockDim.x) {
    const int j = t / kCols, c = t % kCols;
    sc[t] = (c < nc) ? coef[j * M + c0 + c] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const double2* yl = y + (long long)l * N * n;
  double2* sl = s_hat + (long long)l * M * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double2 acc[kCols];
#pragma unroll
    for (int c = 0; c < kCols; ++c) acc[c] = make_double2(0.0, 0.0);
    for (int j = 0; j < N; ++j) {
      const double2 s = yl[(long long)j * n + e];
#pragma unroll
      for (int c = 0; c < kCols; ++c) {
        const double2 w = sc[j * kCols + c];
        acc[c].x = fma(s.x, w.x, fma(-s.y, w.y, acc[c].x));
        acc[c].y = fma(s.x, w.y, fma(s.y, w.x, acc[c].y));
      }
    }
#pragma unroll
    for (int c = 0; c < kCols; ++c)
      if (c < nc) sl[(long long)(c0 + c) * n + e] = acc[c];
  }
}

}  // namespace
}  // namespace ssqcd

extern "C" int ssqcd_moments_noalloc(int N, int M, int L, long long n, const double* w, const double* zeta,
                                     const double* y, double* s_hat, void* cuda_stream) {
  using namespace ssqcd;
  if (N < 1 || M < 1 || L < 1 || n < 1 || !w || !zeta || !y || !s_hat)
    return fail(SSQCD_ERR_ARG, "ssqcd_moments_noalloc: N, M, L, n must be >= 1 and pointers non-NULL");
  if (N > kMaxNoallocShifts || (long long)N * M > kMaxCoef)
    return fail(SSQCD_ERR_ARG, "ssqcd_moments_noalloc: N * M must be <= 4096 and N <= 256 (fixed scratch size)");
  int dev = 0;
  SS_CUDA(cudaGetDevice(&dev));
  double2* table = nullptr;
  SS_TRY(coef_table(dev, &table));
  // c_jk = w_j zeta_j^k, formed on the device from the nodes passed by value
  NodeSet ns;
  for (int j = 0; j < N; ++j) {
    ns.w[j] = make_double2(w[2 * j], w[2 * j + 1]);
    ns.zeta[j] = make_double2(zeta[2 * j], zeta[2 * j + 1]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  moment_coef_kernel<<<(N + 63) / 64, 64, 0, st>>>(ns, N, M, table);
  count_launches(1);
  SS_CHECK_LAUNCH();
  const int cy = (M + kCols - 1) / kCols;
  long long bx = (n + 255) / 256;
  const long long cap = (4LL * 152 + (long long)cy * L - 1) / ((long long)cy * L);
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  const size_t shm = sizeof(double2) * N * kCols;  // <= 32 KiB for N <= 256
  moments_noalloc_kernel<<<dim3((unsigned)bx, cy, L), 256, shm, st>>>(reinterpret_cast<const double2*>(y), N, M, n,
                                                                      table, reinterpret_cast<double2*>(s_hat));
  count_launches(1);
  SS_CHECK_LAUNCH();
  return SSQCD_OK;
}
