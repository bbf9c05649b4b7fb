// Internal declarations of the ssqcd library (not part of the C ABI).
//
// Device layout ("component-major, site-fastest"):
//   spinor field    : [12][V] complex, component c = 3*spin + colour;
//   block of L      : [L][12][V];
//   FP64 gauge      : [4][9][V] double2, element (a,b) of U_mu(s) at
//                     (mu*9 + 3a + b)*V + s;
//   FP16 gauge      : [4][3][V] uint2 (rows 0 and 1 as six half2);
//   FP32 gauge      : [4][3][V] float4 (rows 0 and 1 as six float2).
// A warp of consecutive sites then reads 32 consecutive complex numbers for
// every component, for the site itself and for each of its 8 neighbours
// (neighbours of consecutive sites are consecutive except at wraps).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cstddef>
#include <cstdint>
#include <memory>
#include <utility>
#include <string>
#include <vector>

#include "../../include/ssqcd.h"

namespace ssqcd {

// ---- error handling --------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define SS_CUDA(call)                                                          \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) return ::ssqcd::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define SS_CHECK_LAUNCH()                                                      \
  do {                                                                         \
    cudaError_t e_ = cudaGetLastError();                                       \
    if (e_ != cudaSuccess) return ::ssqcd::cuda_fail(e_, "kernel launch", __FILE__, __LINE__); \
  } while (0)

#define SS_TRY(expr)                                                           \
  do {                                                                         \
    int s_ = (expr);                                                           \
    if (s_ != SSQCD_OK) return s_;                                             \
  } while (0)

void count_launches(long long k);

// ---- device buffers --------------------------------------------------------
// Allocation is stream-ordered (cudaMallocAsync / cudaFreeAsync) on the
// stream of the innermost AllocStream scope of the calling thread, else
// plain cudaMalloc / cudaFree (which synchronise the device on free).  A
// buffer remembers the stream it was allocated on and frees on it; the code
// that uses a buffer on other streams joins them into that stream first.
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  bool async = false;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  int alloc(size_t nbytes);          // no-op when already that large
  void release();
  void swap(DevBuf& o) {
    std::swap(p, o.p);
    std::swap(bytes, o.bytes);
    std::swap(stream, o.stream);
    std::swap(async, o.async);
  }
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

// RAII: DevBuf allocations of this thread use stream-ordered allocation on s
// (on = false: plain allocation inside an enclosing scope).
struct AllocStream {
  explicit AllocStream(cudaStream_t s, bool on = true);
  ~AllocStream();
  AllocStream(const AllocStream&) = delete;
  AllocStream& operator=(const AllocStream&) = delete;

 private:
  cudaStream_t prev_;
  bool prev_on_;
};

// ---- lattice -------------------------------------------------------------------
struct Geometry {
  int X, Y, Z, T;
  int V;
  double kappa;
  double bc_t;
};

}  // namespace ssqcd

struct ssqcd_lattice_s {
  ssqcd::Geometry g;
  int precision;
  cudaStream_t stream;
  bool has_gauge = false;
  ssqcd::DevBuf u64;     // FP64 links [4][9][V] double2
  ssqcd::DevBuf u16;     // FP16 12-parameter links, SSQCD_MIXED only
  ssqcd::DevBuf u32;     // FP32 12-parameter links, SSQCD_MIXED_F32LINKS only
  ssqcd::DevBuf udf;     // float-float links [4][9][V] float4, built on first SSQCD_DF use
  int gauge_version = 0; // bumped by every upload
  int udf_version = -1;  // gauge_version udf was built from
  ssqcd::DevBuf stage;   // staging for host <-> device copies
};

namespace ssqcd {

// ---- kernels and their host launchers (each .cu file documents its own) ----
constexpr int kThreads = 256;

int grid_for(long long work, int threads);

// layout conversions (blas.cu)
int pack_spinors(const double2* user, double2* dev, int nfields, int V, cudaStream_t s);
int unpack_spinors(const double2* dev, double2* user, int nfields, int V, cudaStream_t s);
int pack_gauge64(const double2* user, double2* dev, int V, cudaStream_t s);

// stencil (wilson.cu): out = c0 * in + c1 * A in, for nrhs fields of layout
// [nrhs][12][V]; if dot_partial != nullptr, also per-block partial sums of
// Re <in, out> into dot_partial[rhs * nblocks + block] (nblocks returned by
// wilson_blocks).
int wilson_blocks(const Geometry& g);
int wilson64(const Geometry& g, const double2* u, const double2* in, double2* out, int nrhs,
             double c0, double c1, double* dot_partial, const int* skip_if_zero, cudaStream_t s);
// link_bits 16: FP16 12-parameter links [4][3][V] uint2; 32: FP32 [4][3][V] float4
int wilson32(const Geometry& g, const void* links, int link_bits, const float2* in, float2* out, int nrhs,
             float c0, float c1, float* dot_partial, const int* skip_if_zero, cudaStream_t s);
int pack_gauge16(const double2* u64dev, void* u16, int V, cudaStream_t s);
// FP32 stencil variants (wilson.cu): -1 tuned per (V, nrhs, link bits), 0..3 forced
int set_fp32_stencil_variant(int v);
int fp32_stencil_tuning(int V, int nrhs, int link_bits, int* variant, float* us);  // us[8]
int wilson32_kernel_only(const Geometry& g, const void* links, int link_bits, const float2* in, float2* out, int nrhs,
                         float c0, float c1, cudaStream_t s);
int wilson_df(const Geometry& g, const float4* u, const float4* in, float4* out, int nrhs, double c0, double c1,
              cudaStream_t s);
int convert_f64_to_df(const double2* a, float4* b, long long n, cudaStream_t s);
int convert_df_to_f64(const float4* a, double2* b, long long n, cudaStream_t s);
int pack_gauge_df(const double2* u64dev, float4* udf, int V, cudaStream_t s);
// float-float links of the current gauge field (built or rebuilt on demand)
int ensure_df_links(ssqcd_lattice lat);
int pack_gauge32(const double2* u64dev, void* u32, int V, cudaStream_t s);

// reductions / dense block ops in FP64 (blas.cu)
int norm2_partials(const double2* x, int nvec, long long n, double* partial, int nblocks, cudaStream_t s);
int sum_partials(const double* partial, int nvec, int nblocks, double* out, cudaStream_t s);
// G = X^H Y (mx x my row-major, device).  herm: X^H Y is Hermitian (mx ==
// my, e.g. Q^H A Q): only the 32 x 32 tiles on and above the diagonal are
// formed, the others are left zero (the upper triangle is always complete)
int gram(const double2* X, int mx, const double2* Y, int my, long long n, double2* G, DevBuf& scratch,
         cudaStream_t s, bool herm = false);
// Q[c] = sum_a S[a] C[a][c] (C ms x mc row-major, device)
int combine(const double2* S, int ms, long long n, const double2* C, int mc, double2* Q, cudaStream_t s);
// CGS2 QR of the m vectors S (device): Q [m][n] with orthonormal (or zero)
// vectors and R (m x m row-major, device, upper triangular), S = Q R.
// group_ready (optional): events after which column groups of `group`
// columns of S are complete (the orthogonalisation waits per group)
int cgs2(const double2* S, int m, long long n, double2* Q, double2* R, DevBuf& scratch, cudaStream_t s,
         const cudaEvent_t* group_ready = nullptr, int group = 0);
// Float-float forms of cgs2, gram and combine (blas_df.cu) for SSQCD_DF
// solves: S, Q, X (gram), T: complex float-float vectors [m][n] (float4);
// R, G: FP64 (m x m row-major, device); combine_df writes X in FP64.
int cgs2_df(const float4* S, int m, long long n, float4* Q, double2* R, DevBuf& scratch, cudaStream_t s);
int gram_df(const float4* X, int mx, const float4* Y, int my, long long n, double2* G, DevBuf& scratch,
            cudaStream_t s, bool herm = false);
int combine_df(const float4* T, int ms, long long n, const double2* C, int mc, double2* X, cudaStream_t s);
int col_residual_norms(const double2* AX, const double2* X, const double* theta, int m, long long n,
                       double* out, DevBuf& scratch, cudaStream_t s);
int convert_f64_to_f32(const double2* in, float2* out, long long n, cudaStream_t s);
int convert_f32_to_f64(const float2* in, double2* out, long long n, cudaStream_t s);

// contour (contour.cu, host)
int contour_nodes(int path, double gamma, double rho, double beta, int N,
                  std::vector<double2>& z, std::vector<double2>& w);

// small Hermitian eigenproblem (eigh.cu, host)
int small_eigh(int m, const double2* a, double* evals, double2* evecs);
int small_svd_min_right(int rows, int cols, const double2* a, double* smin, double2* v);
// left singular vectors of a small complex matrix (m x m row-major, host):
// sigma[m] descending, U[m][m] row-major with singular vector k in column k
int small_svd_left(int m, const double2* a, double* sigma, double2* U);

// shifted CG (mshift.cu)
struct ShiftedCGOut {
  int seed_iters = 0;
  int reliable_updates = 0;
  float ms = 0.f;
  long long shift_updates = 0;
  bool timed = false;
  int launches_update = 0;        // timed iterations (with work)
  long long timed_units = 0;      // (source, shift) updates in the timed iterations
  double ms_k[4] = {0, 0, 0, 0};  // stencil, seed update, seed direction, shift update (timed iterations)
  int basis = 0;                  // 1 Krylov-basis form, 2 switched to updates at the cap, 0 updates
  double basis_bytes = 0.0;       // peak bytes of the stored residuals
};
bool kernel_timing_enabled();
inline bool is_mixed(int precision) { return precision == SSQCD_MIXED || precision == SSQCD_MIXED_F32LINKS; }
inline bool valid_precision(int precision) {
  return precision == SSQCD_FP64 || precision == SSQCD_FP64_SHIFT32 || precision == SSQCD_FP64_DFSHIFT ||
         precision == SSQCD_DF || is_mixed(precision);
}
// The stored seed residuals of a shifted-CG run in the Krylov-basis form
// (mshift.cu): slot s holds r_s (slot 0: the source), kBasisBlock slots and
// as many iterations' shift coefficients per device block; gam[l][j][s] is
// the coefficient of slot s in the solution y_j of source l, so
//   y_j = sum_s gam[l][j][s] r_s   and   s_hat_m = sum_j w_j zeta_j^m y_j
//       = sum_s (sum_j w_j zeta_j^m gam[l][j][s]) r_s.
struct KrylovBasis {
  int L = 0, N = 0, S = 0;     // sources, shifts, slot stride of gam
  bool df = false;             // float-float residuals (else FP64)
  long long n = 0;
  std::vector<std::unique_ptr<DevBuf>> blocks;  // the stored residuals and coefficient records
  DevBuf tab;                  // device table of the block pointers
  DevBuf gam;                  // [L][N][S] complex FP64
  DevBuf count;                // [L] int: slots of source l that enter (the rest are unused)
  void release();
};
// s_hat [L][M][n] = sum_s (sum_j coef[j][m] gam[l][j][s]) r_s; coef_host [N][M]
// With side and src_ready (L events): sources 0 .. L-2 on st, the last one on
// the side stream, each source followed by its event, so that the
// orthogonalisation of the first sources' moments overlaps the combination
// of the last (scratch must then stay allocated until st has waited for
// every event).  real_coef: the coefficients' points and weights come in
// conjugate pairs, so the combined coefficients are real and only their
// real parts are applied (half the FP64 work of complex coefficients).
int basis_moments(const KrylovBasis& b, const double2* coef_host, int M, double2* s_hat, DevBuf& scratch,
                  cudaStream_t st, cudaStream_t side = nullptr, const cudaEvent_t* src_ready = nullptr,
                  bool real_coef = false);
// false when the environment sets SSQCD_REAL_MOMENTS=0 (complex coefficients
// throughout, for comparison)
bool real_moments_enabled();

// The moment combination on the tensor cores (combine_tc.cu): FP64 residuals
// (tab: the basis block table, 2^basis_log slots a block, [slot][L][n]),
// real coefficients C[l][o][s] (.x), O <= 16 outputs, out[l][o][n] for the
// sources l0 .. l0 + nl - 1; work: combine_tc_work_bytes(nl, S) bytes.
// Synchronises st (reads the kernel's error word).
bool combine_tc_enabled();
bool combine_tc_applicable(long long n, int O, int S);
size_t combine_tc_work_bytes(int nl, int S);
int combine_tc(char* const* tab, int basis_log, long long n, int L, const double2* C, int O, int S,
               const int* count, double2* out, int l0, int nl, void* work, cudaStream_t st);

// Solves for L sources already packed on device (v: [L][12][V]); y out
// [L][N][12][V] (device, FP64).  iters/xi: host arrays [L*N] (may be null).
// A resumable shifted-CG run (mshift.cu): see CgRun there.
class CgRunBase {
 public:
  enum { kPollRunning = 0, kPollDone = 1, kPollBusy = 2 };
  virtual ~CgRunBase() = default;
  virtual int launch() = 0;                          // enqueue one chunk and its poll read
  virtual int poll(bool wait, int* state) = 0;       // the oldest enqueued chunk's outcome
  virtual int in_flight() const = 0;                 // chunks enqueued, not yet polled
  // y: FP64 solutions, or left empty when the run ended in the Krylov-basis
  // form (then take_basis hands over the stored residuals)
  virtual int finish(DevBuf& y, int* iters_host, double2* xi_host, ShiftedCGOut* out) = 0;
  virtual bool take_basis(KrylovBasis* out) = 0;
};
// basis_cap: bytes the stored residuals may take (Krylov-basis form, FP64 and
// DF precisions); 0 selects the per-iteration shift-vector updates
int make_cg_run(ssqcd_lattice lat, int N, const double2* z_host, int L, const double2* v, double sigma, double tol,
                int max_iter, int precision, int reliable_every, double basis_cap, cudaStream_t st,
                std::unique_ptr<CgRunBase>* out);
// the basis_cap of a solve from its options and size (n, N points, L
// sources): 0 when the form does not apply
double basis_cap_for(int precision, int basis, double basis_max_bytes, long long n, int N, int L);
int shifted_cg_device(ssqcd_lattice lat, int N, const double2* z_host, int L, const double2* v,
                      double sigma, double tol, int max_iter, int precision, int reliable_every,
                      DevBuf& y, int* iters, double2* xi, ShiftedCGOut* out);
// The same driven to the end with basis_cap (see make_cg_run): y, or y left
// empty and *basis filled
int shifted_cg_solve(ssqcd_lattice lat, int N, const double2* z_host, int L, const double2* v, double sigma,
                     double tol, int max_iter, int precision, int reliable_every, double basis_cap, DevBuf& y,
                     KrylovBasis* basis, int* iters, ShiftedCGOut* out);

// moments (moments.cu): s_hat [L][M][12][V] from y [L][N][12][V]
int moments_device(const double2* y, int N, int M, int L, long long n, const double2* coef_host,
                   double2* s_hat, DevBuf& scratch, cudaStream_t s);

}  // namespace ssqcd
