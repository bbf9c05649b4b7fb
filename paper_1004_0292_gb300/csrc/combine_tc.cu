// Moment combination on the tensor cores (tcgen05), FP64 stored residuals
// with real coefficients (the line-pair contours):
//
//   out[l][o][e] = sum_{s < count[l]} C[l][o][s] r_s[l][e]     (Eq. 2 through
//   the Krylov-basis identity: every shifted solution is a combination of
//   the seed residuals)
//
// GB300's tensor cores have no fast FP64 rate, so the FP64 products are
// split exactly into bf16 pieces (the error-free splitting of Ozaki et al.,
// "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications", 2012):
//
// * Each residual r_s (real and imaginary parts as separate rows) is scaled
//   by tau_s = 2^e_s >= max |r_s| and rounded to a 56-bit fixed-point
//   integer X = round(|r| 2^(56 - e_s)), whose seven base-256 digits
//   d_0 .. d_6 (d_0 <= 256) are the bf16 slices A_p = sign d_p (integers,
//   exact in bf16).
// * Each coefficient column o, B[s][o] = C[l][o][s] tau_s, is scaled by
//   sigma_o = 2^g_o >= max_s |B[s][o]| and split the same way into B_q.
// * A_p B_q sums 16-bit integer products; 256 of them stay below 2^24, so
//   the fp32 accumulator in tensor memory holds the sum of a chunk of 256
//   slots exactly.  The pairs with p + q <= 6 are kept: level l = p + q has
//   weight 2^(-8 (l + 2)), and the dropped levels lie below 2^-64 of the
//   scales.  The chunk sums of the levels I_l are added up exactly in two
//   64-bit integers per output, X_hi = I_0 2^16 +
//   I_1 2^8 + I_2 and X_lo = I_3 2^24 + I_4 2^16 + I_5 2^8 + I_6, and at the
//   end of a tile
//     out = sigma_o 2^-16 (2^-16 X_hi + 2^-48 X_lo)   in FP64.
// The result lies within about 2^-56 of the scales of the exact sum, the
// order of the FP64 sum's own rounding: a CPU emulation of this arithmetic
// on the 8^4 workload puts the moments within 2.3e-16 of the exact ones
// (the FP64 sum: 9.1e-16); on test data whose elements span 4 decades
// within a residual, the fixed-point grid leaves the small ones fewer bits
// (2.4e-15 against 6.5e-16).
//
// One persistent CTA per SM (18 warps):
// * warp 9, lane 0: bulk copies (cp.async.bulk) of a tile's 16 slots x 128
//   rows of FP64 into a ring of kF64Stages stages;
// * warps 10-17: cut the stage into the seven A slices (core-matrix layout,
//   K-major, no swizzle) and copy the K-step's B slices (prepared once per
//   launch in the same layout) into a ring of kSliceStages stages;
// * warp 8, lane 0: issues seven tcgen05.mma (M = 128, N = 16 (7 - p),
//   K = 16) a K-step into 448 tensor-memory columns, and commits the stage
//   and, every 256 slots, the accumulators;
// * warps 0-7: read the accumulators (tcgen05.ld; warp w: lanes 32 (w % 4),
//   outputs 8 (w / 4) ..), add them exactly into X_hi and X_lo, and at the
//   end of a tile form and store the outputs.
// Every wait is bounded (1 s of device time); past it the kernel sets *err,
// lets its issued copies and MMAs finish, frees its tensor memory and
// returns.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>

#include "internal.h"

namespace ssqcd {
namespace {

constexpr int kRows = 128;         // real rows (64 complex elements) per tile
constexpr int kKStep = 16;         // slots per MMA (K of kind::f16)
constexpr int kSlices = 7;         // base-256 digits of the 56-bit fixed point
constexpr int kOut = 16;           // outputs per launch
constexpr int kChunkSteps = 16;    // K-steps per accumulator flush (256 slots)
constexpr int kF64Stages = 4;
constexpr int kSliceStages = 4;
constexpr int kEpiWarps = 8;
constexpr int kMmaWarp = 8;
constexpr int kLoadWarp = 9;
constexpr int kSliceWarp0 = 10;
constexpr int kSliceWarps = 8;
constexpr int kTcThreads = (kSliceWarp0 + kSliceWarps) * 32;  // 576
constexpr int kTmemCols = 512;
constexpr int kABytes = kRows * kKStep * 2;       // one bf16 slice: 4096 B
constexpr int kBRows = kSlices * kOut;            // 112
constexpr int kBBytes = kBRows * kKStep * 2;      // 3584 B
constexpr int kMaxCount = 65535;                  // slots (grid.y of the scale kernel)
constexpr unsigned long long kTcWaitNs = 1000000000ull;
constexpr long long kTcSpin = 1LL << 26;

struct __align__(1024) SliceStage {
  unsigned char a[kSlices][kABytes];
  unsigned char b[kBBytes];
};
struct __align__(1024) F64Stage {
  double v[kKStep][kRows];
};
struct TcShared {
  F64Stage f64[kF64Stages];
  SliceStage sl[kSliceStages];
  unsigned long long full_f[kF64Stages], empty_f[kF64Stages];
  unsigned long long full_s[kSliceStages], empty_s[kSliceStages];
  unsigned long long tmem_full, tmem_empty, mma_done;
  unsigned tmem_base;
  int abort;
};

// column of tensor memory where the products of A slice p start (pairs
// (p, q), q = 0 .. 6 - p, 16 columns each)
__host__ __device__ constexpr int col_base(int p) { return 16 * (p * 7 - p * (p - 1) / 2); }

__device__ __forceinline__ unsigned su32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void bar_init(unsigned long long* b, unsigned c) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(c) : "memory");
}
__device__ __forceinline__ void bar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void bar_arrive_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool bar_test(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait for the phase of the given parity; false after kTcWaitNs or
// when another role has given up (abort)
__device__ __forceinline__ bool bar_wait(unsigned long long* b, unsigned parity, volatile int* abort) {
  if (bar_test(b, parity)) return true;
  const unsigned long long t0 = gtimer();
  for (long long i = 1; i < kTcSpin; ++i) {
    if (bar_test(b, parity)) return true;
    if ((i & 255) == 0) {
      if (*abort) return false;
      if (gtimer() - t0 > kTcWaitNs) return false;
    }
  }
  return false;
}
// the same for all 32 lanes of a warp together: every lane observes the
// phase (so every lane may read what it guards) and all leave together
__device__ __forceinline__ bool bar_wait_warp(unsigned long long* b, unsigned parity, volatile int* abort) {
  const unsigned long long t0 = gtimer();
  for (long long i = 0; i < kTcSpin; ++i) {
    if (__all_sync(0xffffffffu, bar_test(b, parity))) return true;
    if ((i & 255) == 255 && __any_sync(0xffffffffu, *abort != 0 || gtimer() - t0 > kTcWaitNs)) return false;
  }
  return false;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   su32(dst)),
               "l"(src), "r"(bytes), "r"(su32(bar))
               : "memory");
}

// ---- tcgen05 ---------------------------------------------------------------------------
// Shared-memory matrix descriptor, K-major without swizzle: core matrices of
// 8 rows x 16 bytes stored as 128 contiguous bytes; `lbo` = byte distance of
// the core matrices adjacent in K, `sbo` = of those adjacent in M (or N).
// Bits: start address >> 4 [0, 14), lbo >> 4 [16, 30), sbo >> 4 [32, 46),
// descriptor version 1 at [46, 48), base offset 0, swizzle mode 0 [61, 64).
__device__ __forceinline__ unsigned long long smem_desc(const void* p, unsigned lbo, unsigned sbo) {
  const unsigned long long a = (su32(p) & 0x3FFFFu) >> 4;
  return a | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) | ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) |
         (1ull << 46);
}
// Instruction descriptor of kind::f16: fp32 accumulator (bits [4, 6) = 1),
// A and B bf16 ([7, 10) = 1, [10, 13) = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at [17, 23), M >> 4 at [24, 29).
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(unsigned d_tmem, unsigned long long a, unsigned long long b, unsigned idesc,
                                       unsigned acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on the mbarrier once the MMAs issued so far by this thread are done
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// a[i] += 2^sh x (the 8 consecutive fp32 columns of this thread's lane),
// each column an integer of magnitude <= 2^24 (exact conversion); load,
// wait, conversion and addition in one statement
__device__ __forceinline__ void tc_ld8_add(unsigned taddr, unsigned sh, long long (&a)[8]) {
  asm volatile(
      "{\n .reg .f32 t<8>;\n .reg .s64 c<8>;\n"
      " tcgen05.ld.sync.aligned.32x32b.x8.b32 {t0, t1, t2, t3, t4, t5, t6, t7}, [%8];\n"
      " tcgen05.wait::ld.sync.aligned;\n"
      " cvt.rni.s64.f32 c0, t0;\n cvt.rni.s64.f32 c1, t1;\n cvt.rni.s64.f32 c2, t2;\n cvt.rni.s64.f32 c3, t3;\n"
      " cvt.rni.s64.f32 c4, t4;\n cvt.rni.s64.f32 c5, t5;\n cvt.rni.s64.f32 c6, t6;\n cvt.rni.s64.f32 c7, t7;\n"
      " shl.b64 c0, c0, %9;\n shl.b64 c1, c1, %9;\n shl.b64 c2, c2, %9;\n shl.b64 c3, c3, %9;\n"
      " shl.b64 c4, c4, %9;\n shl.b64 c5, c5, %9;\n shl.b64 c6, c6, %9;\n shl.b64 c7, c7, %9;\n"
      " add.s64 %0, %0, c0;\n add.s64 %1, %1, c1;\n add.s64 %2, %2, c2;\n add.s64 %3, %3, c3;\n"
      " add.s64 %4, %4, c4;\n add.s64 %5, %5, c5;\n add.s64 %6, %6, c6;\n add.s64 %7, %7, c7;\n}\n"
      : "+l"(a[0]), "+l"(a[1]), "+l"(a[2]), "+l"(a[3]), "+l"(a[4]), "+l"(a[5]), "+l"(a[6]), "+l"(a[7])
      : "r"(taddr), "r"(sh)
      : "memory");
}

// byte offset of element (row, k) of a K-major no-swizzle tile of 16 K:
// core matrix (row / 8, k / 8) at (row / 8) * 256 + (k / 8) * 128
__host__ __device__ constexpr int core_off(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}
constexpr unsigned kLbo = 128, kSbo = 256;

// bf16 bits of the signed integer digit d (0 <= d <= 256): d converted
// exactly to fp32 by the 2^23 offset, the sign set, the upper half kept
// (d has at most 9 significant bits and a power of two when it has 9)
__device__ __forceinline__ unsigned digit_f32(unsigned d, unsigned sgn) {
  const float f = __int_as_float(0x4B000000 | (int)d) - 8388608.0f;
  return (unsigned)__float_as_int(f) | sgn;
}
__device__ __forceinline__ unsigned pack_bf16(unsigned lo_f32, unsigned hi_f32) {
  return __byte_perm(lo_f32, hi_f32, 0x7632);
}
// 56-bit fixed point |x| 2^(56 - e), rounded to nearest (ties up); the sign
// bit in sgn (bit 31).  |x| <= 2^e is required (then X <= 2^56).  Without
// branches: the lanes of a warp hold elements of different exponents.
__device__ __forceinline__ unsigned long long fixed56(double x, int e, unsigned& sgn) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  sgn = (unsigned)(bits >> 32) & 0x80000000u;
  const int E = (int)((bits >> 52) & 0x7FF);
  const unsigned long long m = (bits & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const int sh = E - 1019 - e;                  // X = m 2^sh
  const int ls = min(max(sh, 0), 4), rs = min(max(-sh, 0), 62);
  const unsigned long long half = rs > 0 ? (1ull << (rs - 1)) : 0ull;
  const unsigned long long X = ((m << ls) + half) >> rs;
  // zero (and subnormals, far below any scale here) and shifts past the last digit
  return (E == 0 || sh <= -60) ? 0ull : X;
}

// ---- scales and coefficient slices --------------------------------------------------------
__device__ __forceinline__ const double* slot_ptr(char* const* tab, int basis_log, long long n, int L, int l, int s) {
  const int mask = (1 << basis_log) - 1;
  return reinterpret_cast<const double*>(tab[s >> basis_log]) + 2 * (((long long)(s & mask) * L + l) * n);
}

// mx[l'][s] = max |component| of r_s of source l0 + l' (as the bits of a
// non-negative double, so that integer atomicMax orders them); grid
// (x: element blocks, y: slot, z: source)
__global__ void tc_maxabs_kernel(char* const* __restrict__ tab, int basis_log, long long n, int L, int l0,
                                 const int* __restrict__ count, int S, unsigned long long* __restrict__ mx) {
  const int s = blockIdx.y, lz = blockIdx.z, l = l0 + lz;
  if (s >= count[l]) return;
  const double2* r = reinterpret_cast<const double2*>(slot_ptr(tab, basis_log, n, L, l, s));
  double m = 0.0;
  bool bad = false;  // a NaN or infinity (fmax would drop a NaN)
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const double2 v = r[e];
    bad |= !isfinite(v.x) || !isfinite(v.y);
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  bad = __any_sync(0xffffffffu, bad);
  __shared__ double wm[32];
  __shared__ int wb[32];
  if ((threadIdx.x & 31) == 0) {
    wm[threadIdx.x >> 5] = m;
    wb[threadIdx.x >> 5] = bad ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      m = fmax(m, wm[w]);
      bad |= wb[w] != 0;
    }
    // a non-finite element marks the slot with +infinity (above every finite bit pattern)
    atomicMax(mx + (size_t)lz * S + s, bad ? 0x7FF0000000000000ull : (unsigned long long)__double_as_longlong(m));
  }
}

// the exponent e with 2^(e - 1) <= x < 2^e (x > 0), 0 for x = 0
__device__ __forceinline__ int exp_above(double x) {
  int e = 0;
  if (x > 0.0) (void)frexp(x, &e);
  return e;
}

// e[l'][s] (slot scales) and sig[l'][o] = 2^g_o >= max_s |C[l][o][s] 2^e_s|;
// one block of 256 threads per (source, output).  A non-finite residual
// element or coefficient makes sig NaN, so that the outputs of that source
// come out NaN as the FP64 sum's would (the slices themselves stay finite).
__global__ void tc_scales_kernel(const unsigned long long* __restrict__ mx, const double2* __restrict__ C, int O,
                                 int S, int l0, const int* __restrict__ count, int* __restrict__ eslot,
                                 double* __restrict__ sig) {
  const int lz = blockIdx.x / kOut, o = blockIdx.x % kOut, l = l0 + lz;
  const int cnt = count[l];
  double m = 0.0;
  bool bad = false;
  for (int s = threadIdx.x; s < cnt; s += blockDim.x) {
    const double ms = __longlong_as_double((long long)mx[(size_t)lz * S + s]);
    const bool fin = isfinite(ms);
    const int e = fin ? exp_above(ms) : 0;
    bad |= !fin;
    if (o == 0) eslot[(size_t)lz * S + s] = e;
    if (o < O) {
      const double c = C[((size_t)l * O + o) * S + s].x;
      bad |= !isfinite(c);
      if (isfinite(c)) m = fmax(m, fabs(ldexp(c, e)));
    }
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, d));
  bad = __any_sync(0xffffffffu, bad);
  __shared__ double wm[32];
  __shared__ int wb[32];
  if ((threadIdx.x & 31) == 0) {
    wm[threadIdx.x >> 5] = m;
    wb[threadIdx.x >> 5] = bad ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
      m = fmax(m, wm[w]);
      bad |= wb[w] != 0;
    }
    // every output of the source: a bad slot of this source poisons them all
    sig[(size_t)lz * kOut + o] = (bad || !isfinite(m)) ? __longlong_as_double(0x7FF8000000000000ll)
                                                       : ldexp(1.0, exp_above(m));
  }
}

// B image of K-step kk for source l0 + l' (grid (kk, l'), 224 threads): row
// q * 16 + o of the N x 16 operand holds digit q of C[l][o][s] 2^(e_s - g_o)
// for the slots s = 16 kk + k; thread t writes the 8 slots k = 8 (t & 1) ..
// of row t / 2 (16 bytes of one core matrix).
__global__ void tc_bslices_kernel(const double2* __restrict__ C, int O, int S, int l0, const int* __restrict__ count,
                                  const int* __restrict__ eslot, const double* __restrict__ sig, int ksteps_cap,
                                  unsigned char* __restrict__ bimg) {
  const int kk = blockIdx.x, lz = blockIdx.y, l = l0 + lz;
  const int t = threadIdx.x, row = t >> 1, h = t & 1;
  const int q = row / kOut, o = row % kOut;
  const int cnt = count[l];
  unsigned w[4];
  unsigned f[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int s = kk * kKStep + 8 * h + i;
    unsigned d = 0, sgn = 0;
    if (o < O && s < cnt) {
      const int g = exp_above(sig[(size_t)lz * kOut + o]) - 1;  // sig = 2^g
      const double b = ldexp(C[((size_t)l * O + o) * S + s].x, eslot[(size_t)lz * S + s] - g);
      sgn = b < 0.0 ? 0x80000000u : 0u;
      const unsigned long long X = (unsigned long long)llrint(ldexp(fabs(b), 56));
      d = q == 0 ? (unsigned)(X >> 48) : (unsigned)((X >> (48 - 8 * q)) & 0xFFu);
    }
    f[i] = digit_f32(d, sgn);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = pack_bf16(f[2 * k], f[2 * k + 1]);
  unsigned char* dst = bimg + ((size_t)lz * ksteps_cap + kk) * kBBytes + core_off(row, 8 * h);
  *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// ---- the combination ------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1)
combine_tc_kernel(char* const* __restrict__ tab, int basis_log, long long n, int L, int l0, int nl,
                  const int* __restrict__ count, int S, const int* __restrict__ eslot,
                  const unsigned char* __restrict__ bimg, int ksteps_cap, const double* __restrict__ sig, int O,
                  double2* __restrict__ out, int* __restrict__ err) {
  extern __shared__ unsigned char tc_smem_raw[];
  TcShared* sh = reinterpret_cast<TcShared*>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long tiles_per_src = (2 * n) / kRows;
  const long long tiles = tiles_per_src * nl;
  volatile int* abort = &sh->abort;

  if (threadIdx.x == 0) {
    for (int i = 0; i < kF64Stages; ++i) {
      bar_init(sh->full_f + i, 1);
      bar_init(sh->empty_f + i, kSliceWarps);
    }
    for (int i = 0; i < kSliceStages; ++i) {
      bar_init(sh->full_s + i, kSliceWarps);
      bar_init(sh->empty_s + i, 1);
    }
    bar_init(&sh->tmem_full, 1);
    bar_init(&sh->tmem_empty, kEpiWarps);
    bar_init(&sh->mma_done, 1);
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&sh->tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = sh->tmem_base;

  auto give_up = [&]() {
    *abort = 1;
    atomicExch(err, 3);
  };

  if (warp == kLoadWarp) {
    // ---- bulk copies of the FP64 residual rows ----
    if (lane == 0) {
      long long fc = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int lz = (int)(t / tiles_per_src), l = l0 + lz;
        const long long row0 = (t % tiles_per_src) * kRows;
        const int cnt = count[l], ks = (cnt + kKStep - 1) / kKStep;
        for (int kk = 0; kk < ks; ++kk, ++fc) {
          const int st = (int)(fc % kF64Stages);
          if (fc >= kF64Stages && !bar_wait(sh->empty_f + st, (unsigned)((fc / kF64Stages - 1) & 1), abort)) {
            ok = false;
            break;
          }
          const int nv = min(kKStep, cnt - kk * kKStep);
          bar_arrive_tx(sh->full_f + st, (unsigned)nv * kRows * 8u);
          for (int j = 0; j < nv; ++j)
            bulk_copy(sh->f64[st].v[j], slot_ptr(tab, basis_log, n, L, l, kk * kKStep + j) + row0, kRows * 8u,
                      sh->full_f + st);
        }
      }
      if (!ok) {
        give_up();
        // the copies already issued land before the CTA can exit
        for (long long q = fc - 1; q >= 0 && q >= fc - kF64Stages; --q) {
          const int st = (int)(q % kF64Stages);
          const unsigned long long t0 = gtimer();
          while (!bar_test(sh->full_f + st, (unsigned)((q / kF64Stages) & 1)) && gtimer() - t0 < kTcWaitNs) {
          }
        }
      }
    }
  } else if (warp >= kSliceWarp0) {
    // ---- slices: thread u <-> row u % 128, slots 8 (u / 128) .. + 7 of a K-step ----
    const int u = threadIdx.x - kSliceWarp0 * 32;
    const int row = u & (kRows - 1), h = u >> 7;
    long long fc = 0, sc = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      const int lz = (int)(t / tiles_per_src), l = l0 + lz;
      const int cnt = count[l], ks = (cnt + kKStep - 1) / kKStep;
      for (int kk = 0; kk < ks; ++kk, ++fc, ++sc) {
        const int fs = (int)(fc % kF64Stages), ss = (int)(sc % kSliceStages);
        if (!bar_wait_warp(sh->full_f + fs, (unsigned)((fc / kF64Stages) & 1), abort)) {
          ok = false;
          break;
        }
        const int nv = min(kKStep, cnt - kk * kKStep);
        unsigned long long X[8];
        unsigned sg[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int j = 8 * h + i;
          X[i] = 0ull;
          sg[i] = 0u;
          if (j < nv) X[i] = fixed56(sh->f64[fs].v[j][row], __ldg(eslot + (size_t)lz * S + kk * kKStep + j), sg[i]);
        }
        __syncwarp();
        if (lane == 0) bar_arrive(sh->empty_f + fs);
        if (sc >= kSliceStages &&
            !bar_wait_warp(sh->empty_s + ss, (unsigned)((sc / kSliceStages - 1) & 1), abort)) {
          ok = false;
          break;
        }
#pragma unroll
        for (int p = 0; p < kSlices; ++p) {
          unsigned f[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const unsigned d = p == 0 ? (unsigned)(X[i] >> 48) : (unsigned)((X[i] >> (48 - 8 * p)) & 0xFFu);
            f[i] = digit_f32(d, sg[i]);
          }
          *reinterpret_cast<uint4*>(sh->sl[ss].a[p] + core_off(row, 8 * h)) =
              make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), pack_bf16(f[6], f[7]));
        }
        if (u < kBBytes / 16)
          reinterpret_cast<uint4*>(sh->sl[ss].b)[u] =
              __ldg(reinterpret_cast<const uint4*>(bimg + ((size_t)lz * ksteps_cap + kk) * kBBytes) + u);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) bar_arrive(sh->full_s + ss);
      }
    }
    if (!ok) give_up();
  } else if (warp == kMmaWarp) {
    // ---- MMA issue (one thread) ----
    if (lane == 0) {
      long long sc = 0, cc = 0;
      bool ok = true;
      for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int l = l0 + (int)(t / tiles_per_src);
        const int cnt = count[l], ks = (cnt + kKStep - 1) / kKStep;
        for (int kk = 0; kk < ks; ++kk, ++sc) {
          const int ss = (int)(sc % kSliceStages);
          if (kk % kChunkSteps == 0) {
            if (cc >= 1 && !bar_wait(&sh->tmem_empty, (unsigned)((cc - 1) & 1), abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
          }
          if (!bar_wait(sh->full_s + ss, (unsigned)((sc / kSliceStages) & 1), abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const unsigned acc = (kk % kChunkSteps) != 0 ? 1u : 0u;
          const unsigned long long bd = smem_desc(sh->sl[ss].b, kLbo, kSbo);
#pragma unroll
          for (int p = 0; p < kSlices; ++p)
            tc_mma(tmem + (unsigned)col_base(p), smem_desc(sh->sl[ss].a[p], kLbo, kSbo), bd,
                   idesc_bf16(kRows, kOut * (kSlices - p)), acc);
          tc_commit(sh->empty_s + ss);
          if (kk % kChunkSteps == kChunkSteps - 1 || kk == ks - 1) {
            tc_commit(&sh->tmem_full);
            ++cc;
          }
        }
      }
      if (!ok) give_up();
      // every MMA issued has completed before the tensor memory is freed
      tc_commit(&sh->mma_done);
      const unsigned long long t0 = gtimer();
      while (!bar_test(&sh->mma_done, 0u) && gtimer() - t0 < kTcWaitNs) {
      }
    }
  } else {
    // ---- epilogue: warp w reads lanes 32 (w % 4) .., outputs 8 (w / 4) .. ----
    const int quarter = warp & 3, half = warp >> 2;
    const unsigned lane_addr = tmem + ((unsigned)(32 * quarter) << 16);
    long long cc = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      const int lz = (int)(t / tiles_per_src), l = l0 + lz;
      const long long row0 = (t % tiles_per_src) * kRows;
      const int cnt = count[l], ks = (cnt + kKStep - 1) / kKStep;
      const int nch = (ks + kChunkSteps - 1) / kChunkSteps;
      // level sums combined exactly as they arrive: xh = I_0 2^16 + I_1 2^8 +
      // I_2 (< 2^48), xl = I_3 2^24 + I_4 2^16 + I_5 2^8 + I_6 (< 2^56)
      long long xh[8], xl[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) xh[i] = xl[i] = 0;
      for (int c = 0; c < nch; ++c, ++cc) {
        if (!bar_wait_warp(&sh->tmem_full, (unsigned)(cc & 1), abort)) {
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int p = 0; p < kSlices; ++p)
#pragma unroll
          for (int q = 0; q < kSlices - p; ++q) {
            const unsigned ta = lane_addr + (unsigned)(col_base(p) + kOut * q + 8 * half);
            if (p + q <= 2)
              tc_ld8_add(ta, 8u * (2 - p - q), xh);
            else
              tc_ld8_add(ta, 8u * (6 - p - q), xl);
          }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) bar_arrive(&sh->tmem_empty);
      }
      if (!ok) break;
      // the output addresses are formed here, not kept live across the chunks
      long long r = row0 + 32 * quarter + lane;  // real row: element r / 2, part r % 2
      int lo = l, lzo = lz;
      asm volatile("" : "+l"(r), "+r"(lo), "+r"(lzo));
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int o = 8 * half + i;
        if (o < O) {
          // sum_l I_l 2^(-8 l) = 2^-16 xh + 2^-48 xl
          double v = fma((double)xl[i], 0x1p-48, (double)xh[i] * 0x1p-16);
          v *= sig[(size_t)lzo * kOut + o] * 0x1p-16;
          reinterpret_cast<double*>(out + ((size_t)lo * O + o) * n)[r] = v;
        }
      }
    }
    if (!ok) give_up();
  }
  __syncthreads();
  if (warp == kMmaWarp) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

struct TcWork {
  unsigned long long* mx;
  int* eslot;
  double* sig;
  unsigned char* bimg;
  int* err;
};
size_t align256(size_t b) { return (b + 255) / 256 * 256; }
TcWork carve(void* w, int nl, int S, int ksteps_cap) {
  char* p = static_cast<char*>(w);
  TcWork t;
  t.mx = reinterpret_cast<unsigned long long*>(p);
  p += align256(sizeof(unsigned long long) * (size_t)nl * S);
  t.eslot = reinterpret_cast<int*>(p);
  p += align256(sizeof(int) * (size_t)nl * S);
  t.sig = reinterpret_cast<double*>(p);
  p += align256(sizeof(double) * (size_t)nl * kOut);
  t.err = reinterpret_cast<int*>(p);
  p += 256;
  t.bimg = reinterpret_cast<unsigned char*>(p);
  return t;
}

}  // namespace

bool combine_tc_enabled() {
  // SSQCD_MOMENTS_TC=0: the FP64-pipe combination instead (comparison runs)
  static const bool on = [] {
    const char* e = std::getenv("SSQCD_MOMENTS_TC");
    return !(e != nullptr && std::atoi(e) == 0);
  }();
  return on;
}

bool combine_tc_applicable(long long n, int O, int S) {
  return O >= 1 && O <= kOut && n > 0 && (2 * n) % kRows == 0 && S >= 1 && S <= kMaxCount;
}

size_t combine_tc_work_bytes(int nl, int S) {
  const int ks = (S + kKStep - 1) / kKStep;
  return align256(sizeof(unsigned long long) * (size_t)nl * S) + align256(sizeof(int) * (size_t)nl * S) +
         align256(sizeof(double) * (size_t)nl * kOut) + 256 + (size_t)nl * ks * kBBytes;
}

int combine_tc(char* const* tab, int basis_log, long long n, int L, const double2* C, int O, int S,
               const int* count, double2* out, int l0, int nl, void* work, cudaStream_t st) {
  if (!combine_tc_applicable(n, O, S)) return fail(SSQCD_ERR_ARG, "combine_tc: shape not supported");
  const int ks = (S + kKStep - 1) / kKStep;
  TcWork w = carve(work, nl, S, ks);
  SS_CUDA(cudaMemsetAsync(w.mx, 0, sizeof(unsigned long long) * (size_t)nl * S, st));
  SS_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
  tc_maxabs_kernel<<<dim3(64, S, nl), 256, 0, st>>>(tab, basis_log, n, L, l0, count, S, w.mx);
  SS_CHECK_LAUNCH();
  tc_scales_kernel<<<nl * kOut, 256, 0, st>>>(w.mx, C, O, S, l0, count, w.eslot, w.sig);
  SS_CHECK_LAUNCH();
  tc_bslices_kernel<<<dim3(ks, nl), 2 * kBRows, 0, st>>>(C, O, S, l0, count, w.eslot, w.sig, ks, w.bimg);
  SS_CHECK_LAUNCH();
  static const size_t smem = sizeof(TcShared) + 1024;
  static const cudaError_t attr =
      cudaFuncSetAttribute(combine_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  SS_CUDA(attr);
  int dev = 0, sms = 0;
  SS_CUDA(cudaGetDevice(&dev));
  SS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const long long tiles = (2 * n / kRows) * nl;
  const int grid = (int)(tiles < sms ? tiles : sms);
  combine_tc_kernel<<<grid, kTcThreads, smem, st>>>(tab, basis_log, n, L, l0, nl, count, S, w.eslot, w.bimg, ks,
                                                  w.sig, O, out, w.err);
  SS_CHECK_LAUNCH();
  count_launches(4);
  int h_err = 0;
  SS_CUDA(cudaMemcpyAsync(&h_err, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  SS_CUDA(cudaStreamSynchronize(st));
  if (h_err != 0) return fail(SSQCD_ERR_NOCONV, "moment combination (tensor cores): a device-side wait hit its limit");
  return SSQCD_OK;
}

}  // namespace ssqcd
