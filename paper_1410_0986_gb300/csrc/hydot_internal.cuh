// Internal declarations shared by the translation units of libhydot.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "hydot.h"

namespace hydot {

// ----------------------------------------------------------------------------- scalars
// Minimal complex type for the frequency-domain (complex-symmetric) solves. All products
// used by COCG are bilinear (no conjugation); |z| is used only for norms.
template <typename R>
struct cpx {
  R re, im;
};
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <typename R>
__host__ __device__ __forceinline__ cpx<R> operator/(cpx<R> a, cpx<R> b) {
  R den = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}

template <typename T> struct Traits;
template <> struct Traits<float> {
  using R = float;
  static constexpr bool cplx = false;
  __host__ __device__ static float zero() { return 0.f; }
  __host__ __device__ static float make(float re, float) { return re; }
  __host__ __device__ static float from(double re, double) { return (float)re; }
  __host__ __device__ static double re(float v) { return v; }
  __host__ __device__ static double im(float) { return 0.0; }
  __host__ __device__ static float abs2(float v) { return v * v; }
  __host__ __device__ static float rre(float v) { return v; }
  __host__ __device__ static float rim(float) { return 0.f; }
};
template <> struct Traits<double> {
  using R = double;
  static constexpr bool cplx = false;
  __host__ __device__ static double zero() { return 0.0; }
  __host__ __device__ static double make(double re, double) { return re; }
  __host__ __device__ static double from(double re, double) { return re; }
  __host__ __device__ static double re(double v) { return v; }
  __host__ __device__ static double im(double) { return 0.0; }
  __host__ __device__ static double abs2(double v) { return v * v; }
  __host__ __device__ static double rre(double v) { return v; }
  __host__ __device__ static double rim(double) { return 0.0; }
};
template <> struct Traits<cpx<float>> {
  using R = float;
  static constexpr bool cplx = true;
  __host__ __device__ static cpx<float> zero() { return {0.f, 0.f}; }
  __host__ __device__ static cpx<float> make(float re, float im) { return {re, im}; }
  __host__ __device__ static cpx<float> from(double re, double im) { return {(float)re, (float)im}; }
  __host__ __device__ static double re(cpx<float> v) { return v.re; }
  __host__ __device__ static double im(cpx<float> v) { return v.im; }
  __host__ __device__ static float abs2(cpx<float> v) { return v.re * v.re + v.im * v.im; }
  __host__ __device__ static float rre(cpx<float> v) { return v.re; }
  __host__ __device__ static float rim(cpx<float> v) { return v.im; }
};
template <> struct Traits<cpx<double>> {
  using R = double;
  static constexpr bool cplx = true;
  __host__ __device__ static cpx<double> zero() { return {0.0, 0.0}; }
  __host__ __device__ static cpx<double> make(double re, double im) { return {re, im}; }
  __host__ __device__ static cpx<double> from(double re, double im) { return {re, im}; }
  __host__ __device__ static double re(cpx<double> v) { return v.re; }
  __host__ __device__ static double im(cpx<double> v) { return v.im; }
  __host__ __device__ static double abs2(cpx<double> v) { return v.re * v.re + v.im * v.im; }
  __host__ __device__ static double rre(cpx<double> v) { return v.re; }
  __host__ __device__ static double rim(cpx<double> v) { return v.im; }
};

// ----------------------------------------------------------------------------- double-float
// An unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2: about 48 significant
// bits in the exponent range of FP32. GB300 runs FP32 at ~64x its FP64 rate, so the refinement
// iterate of the mixed real path is held in this form and updated with error-free transformations
// (Knuth's TwoSum, Dekker's FastTwoSum, the FMA-based exact product). The rounded-to-nearest
// intrinsics keep the compiler from fusing the operations these rely on.
struct __align__(8) df32 {
  float hi, lo;
};

// A complex number with double-float parts: the refinement iterate of the mixed complex path.
struct __align__(16) cdf32 {
  df32 re, im;
};

__host__ __device__ inline df32 df_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

#ifdef __CUDACC__
// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ df32 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
// p + e = a * b exactly
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
}
// a + b, accurate also under cancellation (both pairs of parts added with TwoSum)
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  df32 r = fast_two_sum(s, __fadd_rn(e, t));
  r = fast_two_sum(r.hi, __fadd_rn(r.lo, f));
  return r;
}
// the biased FP64 exponent of |v.hi| (0 for zero and FP32 subnormals): integer operations only
__device__ __forceinline__ int bexp(df32 v) {
  const int e = (__float_as_int(v.hi) >> 23) & 0xff;
  return e ? e + (1023 - 127) : 0;
}
__device__ __forceinline__ int bexp_f(float v) {
  const int e = (__float_as_int(v) >> 23) & 0xff;
  return e ? e + (1023 - 127) : 0;
}
#endif

// ----------------------------------------------------------------------------- coefficients
// Per-wavelength coefficients of the scaled operator  Ahat = A / (D h):
//   off-diagonal -1 to each existing neighbour,
//   diagonal 6 + sigma + sum over boundary faces of the cell of (bhat_f - 1),
//   sigma = mu_a h^2 / D (+ i omega h^2 / (c D)),  bhat_f = 2 h / (h + 4 A_f D).
// The field of a unit source is phi = x / (D h) where Ahat x = e_cell.
struct LamCoef {
  double sigma_re, sigma_im;
  double bhat[6];
  double inv_Dh;
  double mua, D;
};

// The same coefficients in FP32 for the inner kernels (no FP64 conversion on the device).
struct LamCoefF {
  float dint;   // 6 + sigma_re: diagonal of an interior cell
  float dim;    // sigma_im
  float idint;  // 1 / dint
  float fa[6];  // bhat_f - 1
  float dint_lo;   // 6 + sigma_re - dint: with dint, the diagonal as a double-float
  float fa_lo[6];  // bhat_f - 1 - fa[f]
  float dim_lo;    // sigma_im - dim
};

// Solver state of one simultaneous field (right-hand side) of a batch.
enum RhsStatus : int { RHS_INNER = 0, RHS_FINISHED = 1, RHS_DONE = 2 };

struct Tiling {
  int tx, ty, tz;     // tile extent in cells (tx = 32, ty = 8 threads; tz planes per thread)
  int ntx, nty, ntz;  // tiles per axis
  int ntiles;         // tiles per field
};

// Event-based per-kernel timing (instrumentation, off by default).
struct KernelTimer {
  struct Pend {
    cudaEvent_t a, b;
    int kind;
  };
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<Pend> pending;
  double ms[HYDOT_KERNEL_COUNT] = {0};
  long long n[HYDOT_KERNEL_COUNT] = {0};
  double bytes[HYDOT_KERNEL_COUNT] = {0};
};

}  // namespace hydot

// ----------------------------------------------------------------------------- context
struct hydot_ctx {
  int device = 0;  // CUDA device current at hydot_setup (all of the context's memory lives there)
  // problem
  int nx, ny, nz;
  long long N;
  double h;
  double robin_A[6];
  int n_lambda, n_chrom, n_src, n_det;
  std::vector<double> eps;        // [n_lambda][n_chrom]
  std::vector<double> c_bg;       // [n_chrom]
  std::vector<double> mus_prime;  // [n_lambda]
  double omega, c_medium;
  std::vector<int> optode_voxel;  // [n_src + n_det] sources then detectors
  int precision;
  double tol, tol_cw, inner_tol, cw_floor;
  int max_iter;
  int deflation_k;
  int max_fields;                 // simultaneous fields the workspace holds
  bool cplx;

  cudaStream_t stream = nullptr;
  std::string err;

  // per-wavelength tables
  std::vector<hydot::LamCoef> coef;  // host copy
  hydot::LamCoef* d_coef = nullptr;
  hydot::LamCoefF* d_coef_f = nullptr;
  double* d_eps = nullptr;           // [n_lambda][n_chrom]
  int* d_optode = nullptr;           // [n_src + n_det]

  // solver workspace (sized for max_fields simultaneous fields)
  hydot::Tiling tiling{};
  void* d_x64 = nullptr;   // [max_fields][N] double (or cpx<double>)
  void* d_e = nullptr;     // [max_fields][N] inner scalar
  void* d_r = nullptr;     // [max_fields][N]
  void* d_p[2] = {nullptr, nullptr};
  double* d_part = nullptr;  // reduction partials, see solver.cu
  size_t part_stride = 0;    // doubles per (field) in d_part
  int* d_status = nullptr;   // [max_fields]
  int* d_iters = nullptr;    // [max_fields] Krylov iterations, all cycles
  int* d_cycles = nullptr;   // [max_fields]
  double* d_scale = nullptr; // [max_fields] 1 / (scale of the FP32 residual) of the current cycle
  double* d_next = nullptr;  // [max_fields] ||r64|| of the latest residual (next cycle's scale)
  double* d_rr0 = nullptr;   // [max_fields] ||r32||^2 at the start of the inner solve
  double* d_theta = nullptr; // [max_fields] floor of the componentwise test
  double* d_final = nullptr; // [max_fields][2] final residual norm, componentwise error
  int* d_counter = nullptr;  // [counter_len] active-field counters (one per inner iteration)
  int counter_len = 0;
  int* h_pinned = nullptr;   // pinned host words for polling
  int* d_err = nullptr;      // set by a kernel whose bounded wait gave up
  bool use_tma = false;      // FP32 real inner kernels with TMA tile loads (nx % 4 == 0)
  // 4-D maps {nx, ny, nz, max_fields} per slab depth 2, 4, 8: d_r, d_p[0], d_p[1] in slabs with the
  // x-y halo (40 x 10 x depth), d_e and d_r in slabs of the tile alone (32 x 8 x depth)
  CUtensorMap tm_rh[3]{}, tm_ph[3][2]{}, tm_e[3]{}, tm_rv[3]{};
  CUtensorMap tm_rh2[3]{}, tm_ph2[3][2]{};  // pass 1 on 32 x 16 tiles: r and p_old in 40 x 18 boxes
  CUtensorMap tm_rx[2][3]{}, tm_px[2][3][2]{};  // pass 1 on x-pairs: 72 x 10 and 72 x 18 boxes
  // single-sweep inner iteration (FP32 real fields on the TMA path): a second residual buffer,
  // per-field scalars {gamma, alpha} per parity [2][max_fields][2], and maps per slab depth 3, 4:
  // r (both buffers) and p (both) in boxes of the tile plus a two-cell ring (40 x 12 x depth), e in
  // boxes of the tile
  bool sweep_ok = false;   // single-sweep resources allocated (real FP32 fields on the TMA path)
  bool use_sweep = false;  // launched iterations use the single-sweep form (else the two passes)
  // persistent form of a cycle's inner solve: mode -1 while the tuner compares it with launched
  // iterations (ms per active cell-iteration, per mode), then 0 (launched) or 1 (persistent)
  struct {
    int mode = -1;
    int samples[2] = {0, 0};
    double ms[2] = {0.0, 0.0};
    double cells[2] = {0.0, 0.0};
  } persist;
  unsigned* d_gsync = nullptr;  // grid barrier words {count, generation}
  // adjoint solves: detector slot of every cell (-1 elsewhere), normalised weights [max_fields][n_det]
  // and their norms [max_fields] (allocated at the first adjoint solve)
  int* d_rhs_slot = nullptr;
  double* d_rhs_w = nullptr;
  double* d_rhs_scale = nullptr;
  int persist_blocks = 0;       // co-resident blocks of the persistent kernel (whole GPU)
  void* d_r2 = nullptr;
  double* d_cgsc = nullptr;
  CUtensorMap tm_r2[2][2]{}, tm_p2[2][2]{}, tm_e2[2]{};
  CUtensorMap tm_r4[2][2]{}, tm_p4[2][2]{}, tm_e4[2]{};  // the same for 32 x 16 tiles (40 x 20 boxes)
  // autotuner of the rolling inner passes: variant -1 while groups of iterations are being timed
  struct {
    int variant = -1;
    int samples[HYDOT_ROLL_VARIANTS] = {};
    double ms[HYDOT_ROLL_VARIANTS] = {};
    double cells[HYDOT_ROLL_VARIANTS] = {};
  } tune;
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  int* d_it = nullptr;               // device-resident base of the inner iteration index
  // absorption perturbation dc [n_chrom][N] (mM, FP64) and the per-slice diagonal increments
  double* d_dc = nullptr;
  double* d_dsig_d = nullptr;        // [max_lambda_per_call][N]
  float* d_dsig_f = nullptr;
  bool use_graphs = true;            // replay groups of inner iterations from a CUDA graph
  void* inner_exec = nullptr;        // cudaGraphExec_t of one group
  cudaStream_t cap_stream = nullptr;  // private non-blocking stream the group is captured on
  std::vector<unsigned char> inner_key;  // what the graph was captured for
  int dir_seg = 0;           // z-planes per block of the rolling pass-1 kernel (multiple of the tile depth)
  // deflation (recycled subspace): W [k][N] FP64 and the k x k Gram blocks
  double* d_W = nullptr;
  std::vector<double> gram_L, gram_I, gram_B;  // W^T Lg W, W^T W, W^T B_f W (6 blocks)
  double* d_Ginv = nullptr;                    // [n_lambda][k][k] inverse of W^T Ahat_j W
  double* d_defl_coef = nullptr;               // [max_fields][k] G_j^-1 W^T b per field
  std::vector<double> deflation_ritz;          // Ritz values of the base operator (ascending)

  // shift-invariant initial guesses: per optode field an FP32 orthonormal basis of the Krylov space
  // of the mean-shift operator started at the optode cell, with its Lanczos coefficients and the
  // boundary blocks V^T B_f V
  int sg_m = 0;                // basis size (0: off)
  float* d_sgV = nullptr;      // [n_src + n_det][sg_m][N]
  double* d_sgA = nullptr;     // [n_src + n_det][64] Lanczos diagonal
  double* d_sgB = nullptr;     // [n_src + n_det][64] Lanczos off-diagonal
  double* d_sgP = nullptr;     // [n_src + n_det][6][sg_m][sg_m]
  int* d_sgMeff = nullptr;     // [n_src + n_det] basis size (smaller after a breakdown)
  float* d_sgY = nullptr;      // [max_fields][sg_m] Galerkin coefficients of a batch
  double sg_base[7] = {0, 0, 0, 0, 0, 0, 0};  // mean sigma, mean bhat_f of the base operator

  long long launches = 0;  // kernels enqueued by this context
  hydot::KernelTimer timer;

  // sketch operand workspace (BF16 B operands)
  void* d_sketch_ws = nullptr;
  size_t sketch_ws_bytes = 0;

  // Born apply workspace
  void* d_apply_ws = nullptr;
  size_t apply_ws_bytes = 0;
};

namespace hydot {

#define HYDOT_CUDA_TRY(ctx, call)                                                     \
  do {                                                                               \
    cudaError_t e__ = (call);                                                        \
    if (e__ != cudaSuccess) {                                                        \
      (ctx)->err = std::string(#call) + ": " + cudaGetErrorString(e__);              \
      return e__ == cudaErrorMemoryAllocation ? HYDOT_ERR_OOM : HYDOT_ERR_CUDA;       \
    }                                                                                \
  } while (0)

inline int fail(hydot_ctx* ctx, int code, const std::string& msg) {
  ctx->err = msg;
  return code;
}

// Raises a kernel's dynamic shared-memory limit on the current device to at least `bytes`, never
// lowering it. Contexts solving concurrently from several host threads can need different sizes
// of one kernel; a lower limit set between another thread's raise and its launch would fail that
// launch, so the limit only grows (under a lock). The limit bounds what a launch may ask for and
// does not change what a smaller launch gets.
cudaError_t raise_smem_limit_raw(const void* func, size_t bytes);
template <typename F>
cudaError_t raise_smem_limit(F* func, size_t bytes) {
  return raise_smem_limit_raw(reinterpret_cast<const void*>(func), bytes);
}

// solver.cu
int solve_fields_impl(hydot_ctx* ctx, int lam0, int nlam, void* phi_src, void* phi_det, hydot_stats* st);
int solve_adjoint_impl(hydot_ctx* ctx, int lam0, int nlam, const void* y, void* psi, hydot_stats* st);
int born_apply_T_adjoint_impl(hydot_ctx* ctx, const void* phi_src, const void* psi, int lam0, int nlam, void* g);
int get_tuning_impl(const hydot_ctx* ctx, int* variant, int* planes, int* buffers, double* ns_per_cell);
int wait_selftest_impl(hydot_ctx* ctx, int polls);
int get_launch_mode_impl(const hydot_ctx* ctx, int* mode, double* ns_launched, double* ns_persistent);
int set_absorption_impl(hydot_ctx* ctx, const double* dc);
int solver_alloc(hydot_ctx* ctx);
void solver_free(hydot_ctx* ctx);

// sketch.cu
int sketch_range_impl(hydot_ctx* ctx, const float* ps, const float* pd, int lam0, int nlam, int src0, int nsr,
                      const void* omega_t, int ncols, float* Y, long long ldY);
int sketch_project_impl(hydot_ctx* ctx, const float* ps, const float* pd, int lam0, int nlam, int src0, int nsr,
                        const float* Q, int ncols, long long ldQ, float* Bt, long long ldB);
int sketch_orthonormalize_impl(hydot_ctx* ctx, float* Y, long long rows, int ncols, long long ldY, int* rank_out,
                               double* smax_out);
int sketch_rank_impl(hydot_ctx* ctx, const float* Q, long long ldQ, long long rows, int nq, const float* Y2,
                     long long ldY2, int k, double s1, double tol, int* rank, double* estimate);
int source_tree_impl(const double* xy, int n, double x_lo, double y_lo, double x_hi, double y_hi, int leaf_max,
                     int* order, int* nodes, int* n_nodes, int* root);
int sketch_merge_impl(hydot_ctx* ctx, const float* U1, long long ldU1, long long m1, const double* S1, const float* V1,
                      long long ldV1, int r1, const float* U2, long long ldU2, long long m2, const double* S2,
                      const float* V2, long long ldV2, int r2, long long n, double tol, int max_rank, float* U,
                      long long ldU, double* S, float* V, long long ldV, int* rank_out);
int sketch_factor_impl(hydot_ctx* ctx, const float* Q, long long rows, long long ldQ, const float* Bt, long long nb,
                       long long ldB, int ncols, int rank, float* U, long long ldU, double* S, float* V, long long ldV);

int tall_cross(hydot_ctx* ctx, const float* X, long long ldx, int nx, const float* Y, long long ldy, int ny,
               long long rows, std::vector<double>& C);

// deflation.cu
int build_deflation(hydot_ctx* ctx);
// x64: double [nrhs][N], or df32 (double-float) when df
int deflate_initial_guess(hydot_ctx* ctx, int lam0, int f_begin, int nf, int nrhs, void* x64, bool df);

// recon.cu
int pals_reconstruct_impl(hydot_ctx* ctx, const float* U, long long ldU, long long rows, const double* S,
                          const float* V, long long ldV, int rank, const float* y, int n_basis, double* p, double* c,
                          const hydot_pals_options* opt, hydot_pals_result* res);
int pals_shape_impl(hydot_ctx* ctx, int n_basis, const double* p, double tau, double eps, double nu, float* mu);
int pals_project_impl(hydot_ctx* ctx, const float* V, long long ldV, int rank, int n_basis, const double* p, double tau,
                      double eps, double nu, double* A);
int shape_compare_impl(hydot_ctx* ctx, const float* mu, const float* mu_hat, double level, double* rel_l2,
                       double* dice);

// shiftguess.cu
int set_shift_guess_impl(hydot_ctx* ctx, int m);
int shift_initial_guess(hydot_ctx* ctx, int lam0, int f_begin, int nf, int nrhs, void* x64, bool df);
int shift_guess_fields_impl(hydot_ctx* ctx, int lam0, int nlam, void* phi_src, void* phi_det);
void shift_guess_free(hydot_ctx* ctx);

// api.cu
void set_context_free_error(const std::string& msg);

// Runs the body of a C-ABI entry point so that no C++ exception crosses the ABI: a failed host
// allocation (std::bad_alloc, e.g. from a std::vector or std::string) becomes HYDOT_ERR_OOM and any
// other exception HYDOT_ERR_HOST, with the message kept in the context (or, for calls without
// one, in the calling thread's context-free message).
template <typename F>
int abi_guard(const hydot_ctx* ctx, F&& body) noexcept {
  auto note = [ctx](const char* what) noexcept {
    try {
      if (ctx) const_cast<hydot_ctx*>(ctx)->err = what;
      else set_context_free_error(what);
    } catch (...) {  // no memory even for the message: the status alone reports it
    }
  };
  try {
    return body();
  } catch (const std::bad_alloc&) {
    note("host memory allocation failed");
    return HYDOT_ERR_OOM;
  } catch (const std::exception& e) {
    note(e.what());
    return HYDOT_ERR_HOST;
  } catch (...) {
    note("unknown host-side exception");
    return HYDOT_ERR_HOST;
  }
}

// Instrumentation helpers (api.cu): a timed launch is bracketed by timer_begin/timer_end;
// timer_flush reads the completed events (call after the stream was synchronised).
cudaEvent_t timer_begin(hydot_ctx* ctx);
void timer_end(hydot_ctx* ctx, cudaEvent_t a, int kind, double bytes, int count = 1);
void timer_flush(hydot_ctx* ctx);

// born.cu
int born_assemble_impl(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam,
                       long long row0, long long nrows, void* J, long long ldJ);
int born_apply_impl(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam,
                    const void* x, void* y);
int born_apply_T_impl(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam,
                      const void* y, void* g);

}  // namespace hydot
