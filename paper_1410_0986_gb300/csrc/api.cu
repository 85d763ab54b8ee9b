// C ABI of libhydot: validation, per-wavelength coefficients, context lifetime, dispatch.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "hydot_internal.cuh"

using hydot::fail;

namespace {

thread_local std::string g_setup_error;  // this thread's last failure with no context to hold it

// Per-wavelength coefficients of the scaled operator (Section 2.1-2.2):
//   mu_a = sum_c eps_c(lambda) c_bg,c            (eqn:perturbation for the background)
//   D    = 1 / (3 (mu_a + mu_s'))
//   sigma = mu_a h^2 / D (+ i omega h^2 / (c_m D)),  bhat_f = 2 h / (h + 4 A_f D),  1/(D h).
void compute_coefficients(hydot_ctx* c) {
  c->coef.resize(c->n_lambda);
  for (int j = 0; j < c->n_lambda; ++j) {
    double mua = 0.0;
    for (int l = 0; l < c->n_chrom; ++l) mua += c->eps[(size_t)j * c->n_chrom + l] * c->c_bg[l];
    const double D = 1.0 / (3.0 * (mua + c->mus_prime[j]));
    hydot::LamCoef& k = c->coef[j];
    k.mua = mua;
    k.D = D;
    k.sigma_re = mua * c->h * c->h / D;
    k.sigma_im = (c->omega != 0.0) ? c->omega * c->h * c->h / (c->c_medium * D) : 0.0;
    for (int f = 0; f < 6; ++f) k.bhat[f] = 2.0 * c->h / (c->h + 4.0 * c->robin_A[f] * D);
    k.inv_Dh = 1.0 / (D * c->h);
  }
}

int validate(const hydot_problem* p, std::string& msg) {
  auto bad = [&](const std::string& m) { msg = m; return HYDOT_ERR_ARG; };
  if (!p) return bad("problem is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return bad("grid extents must be >= 1");
  if (!(p->h_mm > 0.0) || !std::isfinite(p->h_mm)) return bad("h_mm must be finite and > 0");
  for (int f = 0; f < 6; ++f)
    if (!(p->robin_A[f] >= 0.0) || !std::isfinite(p->robin_A[f])) return bad("robin_A must be finite and >= 0");
  if (p->n_lambda < 1) return bad("n_lambda must be >= 1");
  if (p->n_chrom < 1 || p->n_chrom > 16) return bad("n_chrom must be in 1..16");
  if (!p->eps || !p->c_bg || !p->mus_prime) return bad("eps, c_bg and mus_prime must be given");
  for (long long q = 0; q < (long long)p->n_lambda * p->n_chrom; ++q)
    if (!std::isfinite(p->eps[q]) || p->eps[q] < 0.0) return bad("eps must be finite and >= 0");
  for (int l = 0; l < p->n_chrom; ++l)
    if (!std::isfinite(p->c_bg[l]) || p->c_bg[l] < 0.0) return bad("c_bg must be finite and >= 0");
  for (int j = 0; j < p->n_lambda; ++j)
    if (!(p->mus_prime[j] > 0.0) || !std::isfinite(p->mus_prime[j])) return bad("mus_prime must be finite and > 0");
  if (!std::isfinite(p->omega)) return bad("omega must be finite");
  if (p->omega != 0.0 && !(p->c_medium > 0.0)) return bad("c_medium must be > 0 when omega != 0");
  if (p->n_src < 0 || p->n_det < 0 || p->n_src + p->n_det < 1) return bad("need at least one source or detector");
  if ((p->n_src && !p->src_ijk) || (p->n_det && !p->det_ijk)) return bad("optode arrays must be given");
  std::set<long long> cells;
  for (int q = 0; q < p->n_src + p->n_det; ++q) {
    const int* ijk = q < p->n_src ? p->src_ijk + 3 * q : p->det_ijk + 3 * (q - p->n_src);
    if (ijk[0] < 0 || ijk[0] >= p->nx || ijk[1] < 0 || ijk[1] >= p->ny || ijk[2] < 0 || ijk[2] >= p->nz)
      return bad("optode outside the grid");
    long long v = ((long long)ijk[2] * p->ny + ijk[1]) * p->nx + ijk[0];
    if (!cells.insert(v).second) return bad("two optodes share a cell");
  }
  if (p->precision != HYDOT_FP64 && p->precision != HYDOT_MIXED) return bad("unknown precision");
  if (!(p->tol > 0.0) || !(p->tol < 1.0)) return bad("tol must be in (0, 1)");
  if (!(p->tol_cw >= 0.0) || !(p->tol_cw < 1.0)) return bad("tol_cw must be in [0, 1)");
  if (!(p->inner_tol >= 0.0) || !(p->inner_tol < 1.0)) return bad("inner_tol must be in [0, 1)");
  if (p->max_iter < 0) return bad("max_iter must be >= 0");
  if (p->deflation_k < 0 || p->deflation_k > 32) return bad("deflation_k must be in 0..32");
  if (p->max_lambda_per_call < 0 || p->max_lambda_per_call > p->n_lambda)
    return bad("max_lambda_per_call must be in 0..n_lambda");
  if (!(p->cw_floor >= 0.0) || !std::isfinite(p->cw_floor)) return bad("cw_floor must be finite and >= 0");
  return HYDOT_OK;
}

void free_all(hydot_ctx* c) {
  cudaStreamSynchronize(c->stream);
  for (cudaEvent_t e : c->timer.pool) cudaEventDestroy(e);
  c->timer.pool.clear();
  hydot::solver_free(c);
  cudaFree(c->d_coef);
  cudaFree(c->d_coef_f);
  cudaFree(c->d_eps);
  cudaFree(c->d_optode);
  cudaFree(c->d_W);
  cudaFree(c->d_Ginv);
  cudaFree(c->d_defl_coef);
  hydot::shift_guess_free(c);
  cudaFree(c->d_apply_ws);
  cudaFree(c->d_sketch_ws);
}

}  // namespace

namespace hydot {
// Message of a failed call that has no context (reported by hydot_last_error(NULL)).
void set_context_free_error(const std::string& msg) { g_setup_error = msg; }

cudaError_t raise_smem_limit_raw(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> limit;  // (kernel, device) -> bytes set
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& cur = limit[{func, dev}];
  if (bytes <= cur) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

cudaEvent_t timer_begin(hydot_ctx* ctx) {
  KernelTimer& t = ctx->timer;
  if (!t.on) return nullptr;
  if (t.used + 2 > t.pool.size()) {
    for (int q = 0; q < 64; ++q) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      t.pool.push_back(e);
    }
  }
  cudaEvent_t a = t.pool[t.used++];
  cudaEventRecord(a, ctx->stream);
  return a;
}

void timer_end(hydot_ctx* ctx, cudaEvent_t a, int kind, double bytes, int count) {
  KernelTimer& t = ctx->timer;
  if (!t.on || !a) return;
  cudaEvent_t b = t.pool[t.used++];
  cudaEventRecord(b, ctx->stream);
  t.pending.push_back({a, b, kind});
  t.n[kind] += count;
  t.bytes[kind] += bytes;
}

void timer_flush(hydot_ctx* ctx) {
  KernelTimer& t = ctx->timer;
  for (const auto& p : t.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess)
      t.ms[p.kind] += ms;
  }
  t.pending.clear();
  t.used = 0;
}
}  // namespace hydot

extern "C" {

int hydot_version(void) { return 10000; }

int hydot_setup(const hydot_problem* p, void* stream, hydot_ctx** out) {
  return hydot::abi_guard(nullptr, [&]() -> int {
    if (!out) {
      g_setup_error = "out is NULL";
      return HYDOT_ERR_ARG;
    }
    *out = nullptr;
    std::string msg;
    int rc = validate(p, msg);
    if (rc) {
      g_setup_error = msg;
      return rc;
    }
    hydot_ctx* c = new (std::nothrow) hydot_ctx();
    if (!c) {
      g_setup_error = "host allocation failed";
      return HYDOT_ERR_OOM;
    }
    c->nx = p->nx;
    c->ny = p->ny;
    c->nz = p->nz;
    c->N = (long long)p->nx * p->ny * p->nz;
    c->h = p->h_mm;
    std::memcpy(c->robin_A, p->robin_A, sizeof(c->robin_A));
    c->n_lambda = p->n_lambda;
    c->n_chrom = p->n_chrom;
    c->n_src = p->n_src;
    c->n_det = p->n_det;
    c->eps.assign(p->eps, p->eps + (size_t)p->n_lambda * p->n_chrom);
    c->c_bg.assign(p->c_bg, p->c_bg + p->n_chrom);
    c->mus_prime.assign(p->mus_prime, p->mus_prime + p->n_lambda);
    c->omega = p->omega;
    c->c_medium = p->c_medium;
    c->cplx = p->omega != 0.0;
    for (int q = 0; q < p->n_src + p->n_det; ++q) {
      const int* ijk = q < p->n_src ? p->src_ijk + 3 * q : p->det_ijk + 3 * (q - p->n_src);
      c->optode_voxel.push_back((int)(((long long)ijk[2] * p->ny + ijk[1]) * p->nx + ijk[0]));
    }
    c->precision = p->precision;
    c->tol = p->tol;
    c->tol_cw = p->tol_cw;
    c->inner_tol = p->inner_tol;
    c->max_iter = p->max_iter > 0 ? p->max_iter : 20000;
    c->deflation_k = p->deflation_k;
    c->cw_floor = p->cw_floor;
    if (p->deflation_k > 0 && p->omega != 0.0) {
      g_setup_error = "deflation is available for continuous-wave (real) fields only";
      delete c;
      return HYDOT_ERR_ARG;
    }
    c->max_fields = (p->max_lambda_per_call > 0 ? p->max_lambda_per_call : p->n_lambda) * (p->n_src + p->n_det);
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    compute_coefficients(c);

    auto bail = [&](int code) {
      g_setup_error = c->err;
      free_all(c);
      delete c;
      return code;
    };
  #define SETUP_TRY(call)                                                                  \
    do {                                                                                   \
      cudaError_t e__ = (call);                                                            \
      if (e__ != cudaSuccess) {                                                            \
        c->err = std::string(#call) + ": " + cudaGetErrorString(e__);                      \
        return bail(e__ == cudaErrorMemoryAllocation ? HYDOT_ERR_OOM : HYDOT_ERR_CUDA);     \
      }                                                                                    \
    } while (0)
    SETUP_TRY(cudaMalloc(&c->d_coef, sizeof(hydot::LamCoef) * c->n_lambda));
    SETUP_TRY(cudaMemcpy(c->d_coef, c->coef.data(), sizeof(hydot::LamCoef) * c->n_lambda, cudaMemcpyHostToDevice));
    {
      std::vector<hydot::LamCoefF> cf(c->n_lambda);
      for (int j = 0; j < c->n_lambda; ++j) {
        const double d = 6.0 + c->coef[j].sigma_re;
        cf[j].dint = (float)d;
        cf[j].dint_lo = (float)(d - (double)cf[j].dint);
        cf[j].dim = (float)c->coef[j].sigma_im;
        cf[j].dim_lo = (float)(c->coef[j].sigma_im - (double)cf[j].dim);
        cf[j].idint = (float)(1.0 / d);
        for (int f = 0; f < 6; ++f) {
          const double a = c->coef[j].bhat[f] - 1.0;
          cf[j].fa[f] = (float)a;
          cf[j].fa_lo[f] = (float)(a - (double)cf[j].fa[f]);
        }
      }
      SETUP_TRY(cudaMalloc(&c->d_coef_f, sizeof(hydot::LamCoefF) * c->n_lambda));
      SETUP_TRY(cudaMemcpy(c->d_coef_f, cf.data(), sizeof(hydot::LamCoefF) * c->n_lambda, cudaMemcpyHostToDevice));
    }
    SETUP_TRY(cudaMalloc(&c->d_eps, sizeof(double) * c->eps.size()));
    SETUP_TRY(cudaMemcpy(c->d_eps, c->eps.data(), sizeof(double) * c->eps.size(), cudaMemcpyHostToDevice));
    SETUP_TRY(cudaMalloc(&c->d_optode, sizeof(int) * c->optode_voxel.size()));
    SETUP_TRY(cudaMemcpy(c->d_optode, c->optode_voxel.data(), sizeof(int) * c->optode_voxel.size(),
                         cudaMemcpyHostToDevice));
  #undef SETUP_TRY
    rc = hydot::solver_alloc(c);
    if (rc) return bail(rc);
    rc = hydot::build_deflation(c);
    if (rc) return bail(rc);
    *out = c;
    return HYDOT_OK;
  });
}

int hydot_set_stream(hydot_ctx* ctx, void* stream) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return HYDOT_OK;
  });
}

int hydot_solve_fields(hydot_ctx* ctx, int lam0, int nlam, void* phi_src, void* phi_det, hydot_stats* st) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    if (lam0 < 0 || nlam < 1 || lam0 + nlam > ctx->n_lambda) return fail(ctx, HYDOT_ERR_ARG, "wavelength slice out of range");
    if (!phi_src && !phi_det) return fail(ctx, HYDOT_ERR_ARG, "phi_src and phi_det are both NULL");
    if ((phi_src && ctx->n_src == 0) || (phi_det && ctx->n_det == 0))
      return fail(ctx, HYDOT_ERR_ARG, "output given for an empty optode set");
    const int nf = (phi_src ? ctx->n_src : 0) + (phi_det ? ctx->n_det : 0);
    if ((long long)nf * nlam > ctx->max_fields)
      return fail(ctx, HYDOT_ERR_ARG, "nlam exceeds max_lambda_per_call given to hydot_setup");
    return hydot::solve_fields_impl(ctx, lam0, nlam, phi_src, phi_det, st);
  });
}

int hydot_solve_batch(hydot_ctx* const* ctxs, int n, const int* lam0, const int* nlam, void* const* phi_src,
                      void* const* phi_det, hydot_stats* st, int* status) {
  return hydot::abi_guard(nullptr, [&]() -> int {
    g_setup_error.clear();  // set again below only when the lists themselves are rejected
    auto bad = [&](const char* m) {  // the lists themselves are wrong: no context ran
      g_setup_error = m;
      if (status && n > 0)
        for (int i = 0; i < n; ++i) status[i] = HYDOT_ERR_ARG;
      return (int)HYDOT_ERR_ARG;
    };
    if (n < 0) return bad("batch size is negative");
    if (n > 0 && (!ctxs || !lam0 || !nlam || !phi_src || !phi_det)) return bad("a batch list is NULL");
    std::set<const hydot_ctx*> seen;
    for (int i = 0; i < n; ++i) {
      if (!ctxs[i]) return bad("a batch context is NULL");
      if (!seen.insert(ctxs[i]).second) return bad("a context appears twice in the batch");
    }
    if (n == 0) return HYDOT_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
      g_setup_error = "cudaGetDevice failed";
      if (status)
        for (int i = 0; i < n; ++i) status[i] = HYDOT_ERR_CUDA;
      return HYDOT_ERR_CUDA;
    }
    for (int i = 0; i < n; ++i)
      if (ctxs[i]->device != dev) {
        if (status)
          for (int q = 0; q < n; ++q) status[q] = HYDOT_ERR_ARG;
        g_setup_error = "context " + std::to_string(i) + " is not on the caller's current device";
        return fail(ctxs[i], HYDOT_ERR_ARG, g_setup_error);
      }
    std::vector<int> rc(n, HYDOT_OK);
    auto one = [&](int i) {
      // a new host thread starts on device 0: adopt the caller's device before any CUDA call
      if (cudaSetDevice(dev) != cudaSuccess) {
        rc[i] = fail(ctxs[i], HYDOT_ERR_CUDA, "cudaSetDevice failed in a batch worker");
        return;
      }
      rc[i] = hydot_solve_fields(ctxs[i], lam0[i], nlam[i], phi_src[i], phi_det[i], st ? st + i : nullptr);
    };
    std::vector<std::thread> workers;
    workers.reserve(n > 0 ? n - 1 : 0);
    try {
      for (int i = 1; i < n; ++i) workers.emplace_back(one, i);
    } catch (...) {  // no thread could be started: run the rest here, in order
      for (int i = 1 + (int)workers.size(); i < n; ++i) one(i);
    }
    if (n > 0) one(0);
    for (auto& w : workers) w.join();
    int out = HYDOT_OK;
    for (int i = 0; i < n; ++i) {
      if (status) status[i] = rc[i];
      if (rc[i] == HYDOT_ERR_NOT_CONVERGED) {
        if (out == HYDOT_OK) out = HYDOT_ERR_NOT_CONVERGED;
      } else if (rc[i] != HYDOT_OK && (out == HYDOT_OK || out == HYDOT_ERR_NOT_CONVERGED)) {
        out = rc[i];
      }
    }
    return out;
  });
}

int hydot_solve_adjoint(hydot_ctx* ctx, int lam0, int nlam, const void* y, void* psi, hydot_stats* st) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::solve_adjoint_impl(ctx, lam0, nlam, y, psi, st);
  });
}

int hydot_born_apply_T_adjoint(hydot_ctx* ctx, const void* phi_src, const void* psi, int lam0, int nlam, void* g) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::born_apply_T_adjoint_impl(ctx, phi_src, psi, lam0, nlam, g);
  });
}

int hydot_born_assemble(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam, long long row0,
                        long long nrows, void* J, long long ldJ) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::born_assemble_impl(ctx, phi_src, phi_det, lam0, nlam, row0, nrows, J, ldJ);
  });
}

int hydot_born_apply(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam, const void* x,
                     void* y) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::born_apply_impl(ctx, phi_src, phi_det, lam0, nlam, x, y);
  });
}

int hydot_born_apply_T(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam, const void* y,
                       void* g) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::born_apply_T_impl(ctx, phi_src, phi_det, lam0, nlam, y, g);
  });
}

static int sketch_finish(hydot_ctx* ctx, int rc) {
  if (rc) return rc;
  int timed_out = 0;
  HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(&timed_out, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (timed_out) return fail(ctx, HYDOT_ERR_TIMEOUT, "a bounded wait in the sketch kernel gave up; output is not valid");
  return HYDOT_OK;
}

int hydot_sketch_range(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam, int src0,
                       int nsrc, const void* omega_t, int ncols, float* Y, long long ldY) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return sketch_finish(ctx, hydot::sketch_range_impl(ctx, (const float*)phi_src, (const float*)phi_det, lam0, nlam,
                                                       src0, nsrc, omega_t, ncols, Y, ldY));
  });
}

int hydot_sketch_project(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam, int src0,
                         int nsrc, const float* Q, int ncols, long long ldQ, float* Bt, long long ldB) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return sketch_finish(ctx, hydot::sketch_project_impl(ctx, (const float*)phi_src, (const float*)phi_det, lam0, nlam,
                                                         src0, nsrc, Q, ncols, ldQ, Bt, ldB));
  });
}

int hydot_sketch_orthonormalize(hydot_ctx* ctx, float* Y, long long rows, int ncols, long long ldY, int* rank_out,
                                double* smax_out) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::sketch_orthonormalize_impl(ctx, Y, rows, ncols, ldY, rank_out, smax_out);
  });
}

int hydot_sketch_rank(hydot_ctx* ctx, const float* Q, long long ldQ, long long rows, int nq, const float* Y2,
                      long long ldY2, int k, double s1, double tol, int* rank, double* estimate) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::sketch_rank_impl(ctx, Q, ldQ, rows, nq, Y2, ldY2, k, s1, tol, rank, estimate);
  });
}

int hydot_source_tree(const double* xy, int n, double x_lo, double y_lo, double x_hi, double y_hi, int leaf_max,
                      int* order, int* nodes, int* n_nodes, int* root) {
  return hydot::abi_guard(nullptr, [&]() -> int {
    return hydot::source_tree_impl(xy, n, x_lo, y_lo, x_hi, y_hi, leaf_max, order, nodes, n_nodes, root);
  });
}

int hydot_sketch_merge(hydot_ctx* ctx, const float* U1, long long ldU1, long long m1, const double* S1, const float* V1,
                       long long ldV1, int r1, const float* U2, long long ldU2, long long m2, const double* S2,
                       const float* V2, long long ldV2, int r2, long long n, double tol, int max_rank, float* U,
                       long long ldU, double* S, float* V, long long ldV, int* rank_out) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::sketch_merge_impl(ctx, U1, ldU1, m1, S1, V1, ldV1, r1, U2, ldU2, m2, S2, V2, ldV2, r2, n, tol,
                                    max_rank, U, ldU, S, V, ldV, rank_out);
  });
}

int hydot_sketch_factor(hydot_ctx* ctx, const float* Q, long long rows, long long ldQ, const float* Bt, long long nb,
                        long long ldB, int ncols, int rank, float* U, long long ldU, double* S, float* V,
                        long long ldV) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::sketch_factor_impl(ctx, Q, rows, ldQ, Bt, nb, ldB, ncols, rank, U, ldU, S, V, ldV);
  });
}

long long hydot_kernel_launches(const hydot_ctx* ctx) { return ctx ? ctx->launches : 0; }

int hydot_set_absorption(hydot_ctx* ctx, const double* dc) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::set_absorption_impl(ctx, dc);
  });
}

int hydot_pals_reconstruct(hydot_ctx* ctx, const float* U, long long ldU, long long rows, const double* S,
                           const float* V, long long ldV, int rank, const float* y, int n_basis, double* p,
                           double* c, const hydot_pals_options* opt, hydot_pals_result* res) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::pals_reconstruct_impl(ctx, U, ldU, rows, S, V, ldV, rank, y, n_basis, p, c, opt, res);
  });
}

int hydot_pals_shape(hydot_ctx* ctx, int n_basis, const double* p, double tau, double eps, double nu, float* mu) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::pals_shape_impl(ctx, n_basis, p, tau, eps, nu, mu);
  });
}

int hydot_pals_project(hydot_ctx* ctx, const float* V, long long ldV, int rank, int n_basis, const double* p,
                       double tau, double eps, double nu, double* A) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::pals_project_impl(ctx, V, ldV, rank, n_basis, p, tau, eps, nu, A);
  });
}

int hydot_shape_compare(hydot_ctx* ctx, const float* mu, const float* mu_hat, double level, double* rel_l2,
                        double* dice) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::shape_compare_impl(ctx, mu, mu_hat, level, rel_l2, dice);
  });
}

int hydot_set_shift_guess(hydot_ctx* ctx, int m) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::set_shift_guess_impl(ctx, m);
  });
}

int hydot_shift_guess_fields(hydot_ctx* ctx, int lam0, int nlam, void* phi_src, void* phi_det) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::shift_guess_fields_impl(ctx, lam0, nlam, phi_src, phi_det);
  });
}

int hydot_wait_selftest(hydot_ctx* ctx, int polls) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::wait_selftest_impl(ctx, polls);
  });
}

int hydot_get_tuning(const hydot_ctx* ctx, int* variant, int* planes, int* buffers, double* ns_per_cell) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::get_tuning_impl(ctx, variant, planes, buffers, ns_per_cell);
  });
}

int hydot_set_kernel_timing(hydot_ctx* ctx, int on) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    cudaStreamSynchronize(ctx->stream);
    hydot::timer_flush(ctx);
    hydot::KernelTimer& t = ctx->timer;
    t.on = on != 0;
    for (int k = 0; k < HYDOT_KERNEL_COUNT; ++k) {
      t.ms[k] = 0.0;
      t.n[k] = 0;
      t.bytes[k] = 0.0;
    }
    return HYDOT_OK;
  });
}

int hydot_get_launch_mode(const hydot_ctx* ctx, int* mode, double* ns_launched, double* ns_persistent) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    return hydot::get_launch_mode_impl(ctx, mode, ns_launched, ns_persistent);
  });
}

int hydot_set_graphs(hydot_ctx* ctx, int on) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    ctx->use_graphs = on != 0;
    return HYDOT_OK;
  });
}

int hydot_kernel_stats(hydot_ctx* ctx, int kernel, double* ms, long long* launches, double* bytes) {
  return hydot::abi_guard(ctx, [&]() -> int {
    if (!ctx) return HYDOT_ERR_ARG;
    if (kernel < 0 || kernel >= HYDOT_KERNEL_COUNT) return fail(ctx, HYDOT_ERR_ARG, "unknown kernel id");
    HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    hydot::timer_flush(ctx);
    const hydot::KernelTimer& t = ctx->timer;
    if (ms) *ms = t.ms[kernel];
    if (launches) *launches = t.n[kernel];
    if (bytes) *bytes = t.bytes[kernel];
    return HYDOT_OK;
  });
}

const char* hydot_last_error(const hydot_ctx* ctx) { return ctx ? ctx->err.c_str() : g_setup_error.c_str(); }

void hydot_destroy(hydot_ctx* ctx) {
  if (!ctx) return;
  try {
    free_all(ctx);
  } catch (...) {  // freeing must not throw across the ABI; the device memory is released above
  }
  delete ctx;
}

}  // extern "C"
