// Error reporting, device buffers and launch accounting shared by the library.
#include <atomic>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace ssqcd {

namespace {
thread_local std::string g_last_error;
std::atomic<long long> g_launches{0};
std::atomic<int> g_timing{0};
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

int fail(int code, const std::string& msg) {
  set_error(msg);
  return code;
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  set_error(buf);
  return e == cudaErrorMemoryAllocation ? SSQCD_ERR_OOM : SSQCD_ERR_CUDA;
}

void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

bool kernel_timing_enabled() { return g_timing.load() != 0; }

namespace {
thread_local cudaStream_t t_alloc_stream = nullptr;
thread_local bool t_alloc_on = false;
}  // namespace

AllocStream::AllocStream(cudaStream_t s, bool on) : prev_(t_alloc_stream), prev_on_(t_alloc_on) {
  t_alloc_stream = s;
  t_alloc_on = on;
}
AllocStream::~AllocStream() {
  t_alloc_stream = prev_;
  t_alloc_on = prev_on_;
}

namespace {
// The stream-ordered allocations come from the device's default memory pool.
// By default the pool hands its unused memory back to the driver at every
// synchronisation, so each solve would map its gigabytes of stored
// residuals afresh; keeping the freed memory in the pool (release threshold
// at the maximum, once per device) makes the next solve's allocations reuse
// it.  The setting lives in this process's context only.
void keep_pool_memory() {
  static std::atomic<unsigned long long> done_mask{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= 64) return;
  const unsigned long long bit = 1ull << dev;
  if (done_mask.fetch_or(bit) & bit) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    unsigned long long thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  (void)cudaGetLastError();
}
}  // namespace

int DevBuf::alloc(size_t nbytes) {
  if (p && bytes >= nbytes) return SSQCD_OK;
  release();
  if (nbytes == 0) return SSQCD_OK;
  async = t_alloc_on;
  stream = t_alloc_stream;
  if (async) keep_pool_memory();
  cudaError_t e = async ? cudaMallocAsync(&p, nbytes, stream) : cudaMalloc(&p, nbytes);
  if (e != cudaSuccess) {
    p = nullptr;
    bytes = 0;
    (void)cudaGetLastError();
    char buf[160];
    std::snprintf(buf, sizeof(buf), "device allocation of %zu bytes failed: %s", nbytes,
                  cudaGetErrorString(e));
    return fail(SSQCD_ERR_OOM, buf);
  }
  bytes = nbytes;
  return SSQCD_OK;
}

void DevBuf::release() {
  if (p) {
    if (async)
      cudaFreeAsync(p, stream);
    else
      cudaFree(p);
  }
  p = nullptr;
  bytes = 0;
  async = false;
  stream = nullptr;
}

int grid_for(long long work, int threads) {
  long long b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (1LL << 30)) b = 1LL << 30;
  return static_cast<int>(b);
}

}  // namespace ssqcd

extern "C" const char* ssqcd_last_error(void) { return ssqcd::g_last_error.c_str(); }

extern "C" long long ssqcd_kernel_launches(void) { return ssqcd::g_launches.load(); }

extern "C" int ssqcd_set_kernel_timing(int enable) {
  ssqcd::g_timing.store(enable ? 1 : 0);
  return SSQCD_OK;
}
