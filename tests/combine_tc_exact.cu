// Exactness check of the tensor-core moment combination (combine_tc.cu),
// built and run by tests/test_gpu_combine_tc.py: synthetic stored residuals
// in the basis layout (blocks of 16 slots, [slot][L][n] complex FP64) and
// random real coefficients; the device result must equal, bit for bit, a CPU
// copy of the same integer arithmetic (the 56-bit fixed-point digits, the
// exact slice-pair sums, the same final FP64 combination), and lie within a
// few units of 2^-52 of the long-double sum; a NaN in a residual must make
// the outputs of its source NaN.  Prints "checks: passed".
// With --time it times the combination on a half-size headline window.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../paper_1004_0292_gb300/csrc/combine_tc.cu"  // the kernels under test, same translation unit

namespace ssqcd {
void set_error(const std::string& m) { fprintf(stderr, "error: %s\n", m.c_str()); }
int fail(int code, const std::string& m) {
  fprintf(stderr, "fail %d: %s\n", code, m.c_str());
  return code;
}
int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  fprintf(stderr, "cuda %s at %s:%d: %s\n", cudaGetErrorString(e), file, line, what);
  return 5;
}
void count_launches(long long) {}
}  // namespace ssqcd

static unsigned long long rng_state = 12345;
static double urand() {
  rng_state = rng_state * 6364136223846793005ull + 1442695040888963407ull;
  return ((rng_state >> 11) & ((1ull << 53) - 1)) * (1.0 / 9007199254740992.0);
}

constexpr int kLog = 4, kBlk = 16;

struct Case {
  long long n;
  int L, S, O, cnt, l;
};

// exact CPU copy: returns out[o][2n]
static void cpu_tc(const std::vector<std::vector<double>>& R /*[s][2n]*/, const std::vector<double>& C /*[o][S]*/,
                   int O, int S, int cnt, long long n, std::vector<double>& out, std::vector<long double>& ref) {
  std::vector<int> e(cnt);
  for (int s = 0; s < cnt; ++s) {
    double m = 0;
    for (double v : R[s]) m = std::fmax(m, std::fabs(v));
    int E = 0;
    if (m > 0) std::frexp(m, &E);
    e[s] = E;
  }
  std::vector<double> sig(16, 1.0);
  std::vector<std::vector<long long>> Bd(16 * 7, std::vector<long long>(cnt, 0));
  for (int o = 0; o < O; ++o) {
    double m = 0;
    for (int s = 0; s < cnt; ++s) m = std::fmax(m, std::fabs(std::ldexp(C[(size_t)o * S + s], e[s])));
    int g = 0;
    if (m > 0) std::frexp(m, &g);
    sig[o] = std::ldexp(1.0, g);
    for (int s = 0; s < cnt; ++s) {
      const double b = std::ldexp(C[(size_t)o * S + s], e[s] - (g - 1) - 1);  // C 2^e / 2^g
      const long long X = std::llrint(std::ldexp(std::fabs(b), 56));
      const long long sg = b < 0 ? -1 : 1;
      for (int q = 0; q < 7; ++q) {
        const long long d = q == 0 ? (X >> 48) : ((X >> (48 - 8 * q)) & 255);
        Bd[q * 16 + o][s] = sg * d;
      }
    }
  }
  out.assign((size_t)O * 2 * n, 0.0);
  ref.assign((size_t)O * 2 * n, 0.0L);
  std::vector<long long> Ad(7 * cnt);
  for (long long r = 0; r < 2 * n; ++r) {
    for (int s = 0; s < cnt; ++s) {
      const double x = R[s][r];
      long long X = 0;
      if (x != 0.0) {
        int E = 0;
        const double f = std::frexp(std::fabs(x), &E);
        const long long m = (long long)std::ldexp(f, 53);
        int sh = E + 3 - e[s];
        if (sh > 4) sh = 4;
        if (sh >= 0)
          X = m << sh;
        else if (sh > -60)
          X = (m + (1ll << (-sh - 1))) >> (-sh);
      }
      const long long sg = x < 0 ? -1 : 1;
      for (int p = 0; p < 7; ++p) Ad[p * cnt + s] = sg * (p == 0 ? (X >> 48) : ((X >> (48 - 8 * p)) & 255));
    }
    for (int o = 0; o < O; ++o) {
      long long xh = 0, xl = 0;
      for (int p = 0; p < 7; ++p)
        for (int q = 0; p + q <= 6; ++q) {
          long long I = 0;
          for (int s = 0; s < cnt; ++s) I += Ad[p * cnt + s] * Bd[q * 16 + o][s];
          const int lv = p + q;
          if (lv <= 2)
            xh += I << (8 * (2 - lv));
          else
            xl += I << (8 * (6 - lv));
        }
      double v = std::fma((double)xl, 0x1p-48, (double)xh * 0x1p-16);
      v *= sig[o] * 0x1p-16;
      out[(size_t)o * 2 * n + r] = v;
      long double acc = 0;
      for (int s = 0; s < cnt; ++s) acc += (long double)C[(size_t)o * S + s] * (long double)R[s][r];
      ref[(size_t)o * 2 * n + r] = acc;
    }
  }
}

static int run_check(const Case& c) {
  const long long n = c.n;
  const int nblk = (c.S + kBlk - 1) / kBlk;
  // residuals: slot s of source l; magnitudes decay with s, spread over 4 decades within a slot
  std::vector<std::vector<double>> R(c.cnt, std::vector<double>(2 * n));
  for (int s = 0; s < c.cnt; ++s) {
    const double sc = std::pow(10.0, -8.0 * s / std::max(1, c.cnt - 1));
    for (long long r = 0; r < 2 * n; ++r) {
      const double u = urand();
      R[s][r] = (u < 0.02) ? 0.0 : sc * (urand() - 0.5) * std::pow(10.0, -4.0 * urand());
    }
  }
  std::vector<double> C((size_t)c.O * c.S, 0.0);
  for (int o = 0; o < c.O; ++o)
    for (int s = 0; s < c.cnt; ++s) C[(size_t)o * c.S + s] = (urand() - 0.5) * std::pow(10.0, 8.0 * s / c.cnt - 3.0 * urand());
  // device: blocks of [16][L][n] double2
  std::vector<char*> blocks(nblk);
  for (int b = 0; b < nblk; ++b) {
    if (cudaMalloc(&blocks[b], (size_t)kBlk * c.L * n * 16) != cudaSuccess) return 2;
    cudaMemset(blocks[b], 0xFF, (size_t)kBlk * c.L * n * 16);  // NaN fill: unused slots must not be read
  }
  for (int s = 0; s < c.cnt; ++s) {
    char* dst = blocks[s / kBlk] + ((size_t)(s % kBlk) * c.L + c.l) * n * 16;
    cudaMemcpy(dst, R[s].data(), (size_t)2 * n * 8, cudaMemcpyHostToDevice);
  }
  char** tab;
  cudaMalloc(&tab, sizeof(char*) * nblk);
  cudaMemcpy(tab, blocks.data(), sizeof(char*) * nblk, cudaMemcpyHostToDevice);
  // C[l][o][s] double2 for all L sources (only source l filled)
  std::vector<double2> Ch((size_t)c.L * c.O * c.S, make_double2(0, 0));
  for (int o = 0; o < c.O; ++o)
    for (int s = 0; s < c.S; ++s) Ch[((size_t)c.l * c.O + o) * c.S + s] = make_double2(C[(size_t)o * c.S + s], 0.0);
  double2 *Cd, *out;
  int* count;
  cudaMalloc(&Cd, sizeof(double2) * Ch.size());
  cudaMemcpy(Cd, Ch.data(), sizeof(double2) * Ch.size(), cudaMemcpyHostToDevice);
  std::vector<int> cnts(c.L, 0);
  cnts[c.l] = c.cnt;
  cudaMalloc(&count, sizeof(int) * c.L);
  cudaMemcpy(count, cnts.data(), sizeof(int) * c.L, cudaMemcpyHostToDevice);
  cudaMalloc(&out, sizeof(double2) * (size_t)c.L * c.O * n);
  cudaMemset(out, 0, sizeof(double2) * (size_t)c.L * c.O * n);
  void* work;
  cudaMalloc(&work, ssqcd::combine_tc_work_bytes(1, c.S));
  cudaStream_t st;
  cudaStreamCreate(&st);
  const int rc = ssqcd::combine_tc(tab, kLog, n, c.L, Cd, c.O, c.S, count, out, c.l, 1, work, st);
  cudaError_t ce = cudaDeviceSynchronize();
  printf("case n=%lld L=%d S=%d O=%d cnt=%d l=%d: status %d, cuda %s\n", n, c.L, c.S, c.O, c.cnt, c.l, rc,
         cudaGetErrorString(ce));
  if (rc != 0 || ce != cudaSuccess) return 1;
  std::vector<double> g((size_t)c.O * 2 * n);
  cudaMemcpy(g.data(), reinterpret_cast<double*>(out + (size_t)c.l * c.O * n), sizeof(double) * g.size(),
             cudaMemcpyDeviceToHost);
  std::vector<double> cpu;
  std::vector<long double> ref;
  cpu_tc(R, C, c.O, c.S, c.cnt, n, cpu, ref);
  long long nbad = 0;
  double worst = 0, worst_fp64 = 0;
  for (int o = 0; o < c.O; ++o) {
    long double num = 0, den = 0, num64 = 0;
    for (long long r = 0; r < 2 * n; ++r) {
      const size_t i = (size_t)o * 2 * n + r;
      if (g[i] != cpu[i] && !(std::isnan(g[i]) && std::isnan(cpu[i]))) {
        if (nbad < 5) printf("  mismatch o=%d r=%lld gpu %.17g cpu %.17g\n", o, r, g[i], cpu[i]);
        ++nbad;
      }
      num += (g[i] - ref[i]) * (g[i] - ref[i]);
      den += ref[i] * ref[i];
    }
    // plain FP64 sum for comparison
    for (long long r = 0; r < 2 * n; ++r) {
      double a = 0;
      for (int s = 0; s < c.cnt; ++s) a += C[(size_t)o * c.S + s] * R[s][r];
      const size_t i = (size_t)o * 2 * n + r;
      num64 += (a - ref[i]) * (a - ref[i]);
    }
    worst = std::fmax(worst, (double)std::sqrt(num / den));
    worst_fp64 = std::fmax(worst_fp64, (double)std::sqrt(num64 / den));
  }
  printf("  bitwise mismatches vs CPU copy: %lld of %lld; rel err vs long double: tc %.2e, fp64 sum %.2e\n", nbad,
         (long long)g.size(), worst, worst_fp64);
  for (auto b : blocks) cudaFree(b);
  cudaFree(tab);
  cudaFree(Cd);
  cudaFree(out);
  cudaFree(count);
  cudaFree(work);
  cudaStreamDestroy(st);
  return nbad == 0 && worst < 1e-13 ? 0 : 1;
}

// A NaN in one element of one slot: every output of that source is NaN
// (the tensor-core path marks the source through its scales; the FP64 sum
// would give NaN in the rows that element reaches).
static int run_nan_check() {
  const long long n = 64 * 4;
  const int S = 32, cnt = 20, O = 16;
  std::vector<double> h((size_t)2 * n * 16);
  for (auto& v : h) v = urand() - 0.5;
  std::vector<char*> blocks(2);
  for (int b = 0; b < 2; ++b) {
    if (cudaMalloc(&blocks[b], (size_t)16 * n * 16) != cudaSuccess) return 2;
    cudaMemcpy(blocks[b], h.data(), (size_t)16 * n * 16, cudaMemcpyHostToDevice);
  }
  const double nan = std::nan("");
  cudaMemcpy(reinterpret_cast<double*>(blocks[0] + (size_t)3 * n * 16) + 77, &nan, 8, cudaMemcpyHostToDevice);
  char** tab;
  cudaMalloc(&tab, sizeof(char*) * 2);
  cudaMemcpy(tab, blocks.data(), sizeof(char*) * 2, cudaMemcpyHostToDevice);
  std::vector<double2> Ch((size_t)O * S);
  for (auto& v : Ch) v = make_double2(urand() - 0.5, 0.0);
  double2 *Cd, *out;
  int* count;
  cudaMalloc(&Cd, sizeof(double2) * Ch.size());
  cudaMemcpy(Cd, Ch.data(), sizeof(double2) * Ch.size(), cudaMemcpyHostToDevice);
  cudaMalloc(&count, sizeof(int));
  cudaMemcpy(count, &cnt, sizeof(int), cudaMemcpyHostToDevice);
  cudaMalloc(&out, sizeof(double2) * O * n);
  void* work;
  cudaMalloc(&work, ssqcd::combine_tc_work_bytes(1, S));
  const int rc = ssqcd::combine_tc(tab, kLog, n, 1, Cd, O, S, count, out, 0, 1, work, 0);
  std::vector<double> g((size_t)O * 2 * n);
  cudaMemcpy(g.data(), out, sizeof(double) * g.size(), cudaMemcpyDeviceToHost);
  long long finite = 0;
  for (double v : g) finite += std::isnan(v) ? 0 : 1;
  printf("nan case: status %d, %lld of %lld outputs not NaN\n", rc, finite, (long long)g.size());
  for (auto b : blocks) cudaFree(b);
  cudaFree(tab);
  cudaFree(Cd);
  cudaFree(out);
  cudaFree(count);
  cudaFree(work);
  return rc == 0 && finite == 0 ? 0 : 1;
}

// --time: one window of the headline size (2502 slots of 786,432 complex
// elements, 31.5 GB, 16 moments), best of three after a warm-up
__global__ void fill_kernel(double* p, long long count, unsigned long long seed, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = (i + 1) * 0x9E3779B97F4A7C15ull ^ seed;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    p[i] = scale * ((double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5);
  }
}

static int run_timing(long long n, int S) {
  const int nblk = (S + kBlk - 1) / kBlk;
  std::vector<char*> blocks(nblk);
  for (int b = 0; b < nblk; ++b) {
    if (cudaMalloc(&blocks[b], (size_t)kBlk * n * 16) != cudaSuccess) {
      printf("timing: allocation failed\n");
      return 2;
    }
    fill_kernel<<<1024, 256>>>(reinterpret_cast<double*>(blocks[b]), (long long)kBlk * 2 * n, b, std::pow(10.0, -8.0 * b / nblk));
  }
  char** tab;
  cudaMalloc(&tab, sizeof(char*) * nblk);
  cudaMemcpy(tab, blocks.data(), sizeof(char*) * nblk, cudaMemcpyHostToDevice);
  std::vector<double2> Ch((size_t)16 * S);
  for (auto& v : Ch) v = make_double2(urand() - 0.5, 0.0);
  double2 *Cd, *out;
  int* count;
  cudaMalloc(&Cd, sizeof(double2) * Ch.size());
  cudaMemcpy(Cd, Ch.data(), sizeof(double2) * Ch.size(), cudaMemcpyHostToDevice);
  cudaMalloc(&count, sizeof(int));
  cudaMemcpy(count, &S, sizeof(int), cudaMemcpyHostToDevice);
  cudaMalloc(&out, sizeof(double2) * 16 * n);
  void* work;
  cudaMalloc(&work, ssqcd::combine_tc_work_bytes(1, S));
  cudaStream_t st;
  cudaStreamCreate(&st);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = ssqcd::combine_tc(tab, kLog, n, 1, Cd, 16, S, count, out, 0, 1, work, st);  // warm-up
  float best = 1e30f;
  for (int it = 0; it < 3 && rc == 0; ++it) {
    cudaEventRecord(e0, st);
    rc = ssqcd::combine_tc(tab, kLog, n, 1, Cd, 16, S, count, out, 0, 1, work, st);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    best = std::fmin(best, ms);
  }
  const double gb = (double)S * n * 16 / 1e9;
  printf("timing n=%lld S=%d (%.1f GB of residuals): status %d, %.2f ms (incl. scale pass and host sync), %.0f GB/s\n",
         n, S, gb, rc, best, gb / (best / 1e3));
  for (auto b : blocks) cudaFree(b);
  return rc;
}

int main(int argc, char** argv) {
  cudaFree(0);
  if (argc > 1 && std::strcmp(argv[1], "--time") == 0) return run_timing(786432, 2502);
  int bad = 0;
  bad |= run_check(Case{64 * 40, 1, 300, 16, 300, 0});
  bad |= run_check(Case{64 * 20, 3, 48, 5, 37, 1});
  bad |= run_check(Case{64 * 8, 1, 16, 16, 1, 0});
  bad |= run_nan_check();
  printf("checks: %s\n", bad ? "FAILED" : "passed");
  return bad ? 1 : 0;
}
