// Shape reconstruction with parametric level sets (Section 5: eqn:pals, eqn:minimization,
// Algorithm alg:opt) on the compressed Born operator J ~ U diag(S) V^T.
//
// Shape: mu(r) = H_eps(phi(r) - tau), phi(r) = sum_k alpha_k psi(beta_k |r - chi_k|_nu), |v|_nu =
// sqrt(|v|^2 + nu^2), with Wendland's compactly supported psi(t) = (1 - t)_+^4 (4t + 1) and the
// arctan-smoothed Heaviside H_eps(t) = 1/2 + arctan(pi t / eps) / pi; p = [alpha, beta, chi_x,
// chi_y, chi_z] (N_p = 5 n_p), positions in mm at voxel centres.
// With U orthonormal, |y - D(p) c|^2 = (|y|^2 - |U^T y|^2) + |U^T y - S M c|^2 where M[:, c] =
// V_c^T mu (V_c: the rows of V of chromophore c), and the residual's Jacobian is
// -S sum_c c_c V_c^T dmu/dp. So one evaluation is: a kernel writes F = [mu, dmu/dp] per voxel
// (FP32), and tall-skinny products give A_c = V_c^T F (FP32 products, FP64 sums); the rest works
// on r x (1 + N_p) matrices on the host: the linear least-squares step for c and the
// Levenberg-Marquardt steps (J^T J + nu I) dp = -J^T eps of alg:opt, stopped by the discrepancy
// principle |eps| <= gamma |eta| (the loop conditions printed in the algorithm have the inequality
// reversed; the text's rule is followed).
#include <algorithm>
#include <cmath>
#include <vector>

#include "dense.h"
#include "hydot_internal.cuh"

namespace hydot {

namespace {

constexpr int PALS_MAXB = 8;  // basis functions

struct PalsGeo {
  int nx, ny, nz, nb;
  float h, tau, eps, nu;
};

// F[x][0] = mu(x) and, with grad, F[x][1 + q] = dmu/dp_q(x)
__global__ void __launch_bounds__(256) k_pals_features(PalsGeo g, const float* __restrict__ pdev, float* __restrict__ F,
                                                       int ldf, int grad) {
  __shared__ float sp[5 * PALS_MAXB];
  for (int q = threadIdx.x; q < 5 * g.nb; q += blockDim.x) sp[q] = pdev[q];
  __syncthreads();
  const int nb = g.nb;
  const float* al = sp;
  const float* be = sp + nb;
  const float* cx = sp + 2 * nb;
  const float* cy = sp + 3 * nb;
  const float* cz = sp + 4 * nb;
  const long long N = (long long)g.nx * g.ny * g.nz;
  const float kpi = 3.14159265358979f / g.eps;
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(x % g.nx), j = (int)((x / g.nx) % g.ny), k = (int)(x / ((long long)g.nx * g.ny));
    const float px = (i + 0.5f) * g.h, py = (j + 0.5f) * g.h, pz = (k + 0.5f) * g.h;
    float psi[PALS_MAXB], dpsi[PALS_MAXB], rn[PALS_MAXB], dx[PALS_MAXB], dy[PALS_MAXB], dz[PALS_MAXB];
    float phi = 0.f;
#pragma unroll
    for (int b = 0; b < PALS_MAXB; ++b) {
      if (b < nb) {
        dx[b] = px - cx[b];
        dy[b] = py - cy[b];
        dz[b] = pz - cz[b];
        rn[b] = sqrtf(dx[b] * dx[b] + dy[b] * dy[b] + dz[b] * dz[b] + g.nu * g.nu);
        const float t = be[b] * rn[b];
        const float u = 1.f - t;
        psi[b] = t < 1.f ? u * u * u * u * (4.f * t + 1.f) : 0.f;
        dpsi[b] = t < 1.f ? -20.f * t * u * u * u : 0.f;
        phi = fmaf(al[b], psi[b], phi);
      }
    }
    const float s = phi - g.tau;
    float* f = F + x * ldf;
    f[0] = 0.5f + atanf(kpi * s) / 3.14159265358979f;
    if (grad) {
      const float de = (1.f / g.eps) / (1.f + (kpi * s) * (kpi * s));
#pragma unroll
      for (int b = 0; b < PALS_MAXB; ++b) {
        if (b < nb) {
          f[1 + b] = de * psi[b];
          f[1 + nb + b] = de * al[b] * dpsi[b] * rn[b];
          const float gg = de * al[b] * dpsi[b] * be[b] / rn[b];
          f[1 + 2 * nb + b] = -gg * dx[b];
          f[1 + 3 * nb + b] = -gg * dy[b];
          f[1 + 4 * nb + b] = -gg * dz[b];
        }
      }
    }
  }
}

// per-block partials [blk][5]: sum (a - b)^2, sum a^2, |a > level|, |b > level|, |both|
__global__ void __launch_bounds__(256) k_shape_compare(const float* __restrict__ a, const float* __restrict__ b,
                                                       long long N, float level, double* __restrict__ part) {
  __shared__ double sm[5][8];
  double v[5] = {0, 0, 0, 0, 0};
  for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
    const float av = a[x], bv = b[x];
    const double d = (double)av - (double)bv;
    v[0] += d * d;
    v[1] += (double)av * av;
    const bool ia = av > level, ib = bv > level;
    v[2] += ia;
    v[3] += ib;
    v[4] += ia && ib;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 5; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if (lane == 0) sm[q][w] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < 5) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += sm[threadIdx.x][q];
    part[(size_t)blockIdx.x * 5 + threadIdx.x] = s;
  }
}

// x = G^-1 b for symmetric positive definite G (n x n, row-major); false if the factorisation fails
bool spd_solve(const std::vector<double>& G, int n, const std::vector<double>& b, std::vector<double>& x) {
  std::vector<double> R;
  if (!cholesky_upper(G, n, R)) return false;  // G = R^T R
  std::vector<double> z(n);
  for (int i = 0; i < n; ++i) {  // R^T z = b
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= R[(size_t)k * n + i] * z[k];
    z[i] = s / R[(size_t)i * n + i];
  }
  x.assign(n, 0.0);
  for (int i = n - 1; i >= 0; --i) {  // R x = z
    double s = z[i];
    for (int k = i + 1; k < n; ++k) s -= R[(size_t)i * n + k] * x[k];
    x[i] = s / R[(size_t)i * n + i];
  }
  return true;
}

struct PalsWork {
  hydot_ctx* ctx;
  PalsGeo g;
  const float* V;
  long long ldV;
  int r, nc, Q;
  float* F = nullptr;   // [N][Q]
  float* pd = nullptr;  // [5 nb]
  ~PalsWork() {
    cudaFree(F);
    cudaFree(pd);
  }
  int alloc() {
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&F, sizeof(float) * (size_t)ctx->N * Q));
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&pd, sizeof(float) * 5 * PALS_MAXB));
    return HYDOT_OK;
  }
  // A [nc][r][Q] = V_c^T [mu, dmu/dp] at p
  int project(const std::vector<double>& p, std::vector<double>& A) {
    float pf[5 * PALS_MAXB];
    for (int q = 0; q < 5 * g.nb; ++q) pf[q] = (float)p[q];
    HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(pd, pf, sizeof(float) * 5 * g.nb, cudaMemcpyHostToDevice, ctx->stream));
    const unsigned blocks = (unsigned)std::min<long long>((ctx->N + 255) / 256, 152 * 16);
    k_pals_features<<<blocks, 256, 0, ctx->stream>>>(g, pd, F, Q, 1);
    ++ctx->launches;
    HYDOT_CUDA_TRY(ctx, cudaGetLastError());
    A.assign((size_t)nc * r * Q, 0.0);
    std::vector<double> Ac;
    for (int c = 0; c < nc; ++c) {
      int rc = tall_cross(ctx, V + (size_t)c * ctx->N * ldV, ldV, r, F, Q, Q, ctx->N, Ac);
      if (rc) return rc;
      std::copy(Ac.begin(), Ac.end(), A.begin() + (size_t)c * r * Q);
    }
    return HYDOT_OK;
  }
};

PalsGeo make_pals_geo(const hydot_ctx* ctx, int nb, double tau, double eps, double nu) {
  PalsGeo g;
  g.nx = ctx->nx;
  g.ny = ctx->ny;
  g.nz = ctx->nz;
  g.nb = nb;
  g.h = (float)ctx->h;
  g.tau = (float)tau;
  g.eps = (float)eps;
  g.nu = (float)nu;
  return g;
}

}  // namespace

int pals_shape_impl(hydot_ctx* ctx, int n_basis, const double* p, double tau, double eps, double nu, float* mu) {
  if (n_basis < 1 || n_basis > PALS_MAXB) return fail(ctx, HYDOT_ERR_ARG, "n_basis must be in 1..8");
  if (!p || !mu) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  if (!(eps > 0.0) || !(nu >= 0.0)) return fail(ctx, HYDOT_ERR_ARG, "eps must be > 0 and nu >= 0");
  float pf[5 * PALS_MAXB];
  for (int q = 0; q < 5 * n_basis; ++q) pf[q] = (float)p[q];
  float* pd = nullptr;
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&pd, sizeof(pf)));
  cudaError_t e = cudaMemcpyAsync(pd, pf, sizeof(float) * 5 * n_basis, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) {
    const unsigned blocks = (unsigned)std::min<long long>((ctx->N + 255) / 256, 152 * 16);
    k_pals_features<<<blocks, 256, 0, ctx->stream>>>(make_pals_geo(ctx, n_basis, tau, eps, nu), pd, mu, 1, 0);
    ++ctx->launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // pf and pd go out of scope
  cudaFree(pd);
  if (e != cudaSuccess) return fail(ctx, HYDOT_ERR_CUDA, std::string("pals shape: ") + cudaGetErrorString(e));
  return HYDOT_OK;
}

int pals_project_impl(hydot_ctx* ctx, const float* V, long long ldV, int rank, int n_basis, const double* p, double tau,
                      double eps, double nu, double* A) {
  if (n_basis < 1 || n_basis > PALS_MAXB) return fail(ctx, HYDOT_ERR_ARG, "n_basis must be in 1..8");
  if (!V || !p || !A || rank < 1 || ldV < rank) return fail(ctx, HYDOT_ERR_ARG, "bad V, rank or pointer");
  if (!(eps > 0.0) || !(nu >= 0.0)) return fail(ctx, HYDOT_ERR_ARG, "eps must be > 0 and nu >= 0");
  PalsWork w{ctx, make_pals_geo(ctx, n_basis, tau, eps, nu), V, ldV, rank, ctx->n_chrom, 1 + 5 * n_basis};
  int rc = w.alloc();
  if (rc) return rc;
  std::vector<double> pv(p, p + 5 * n_basis), Av;
  rc = w.project(pv, Av);
  if (rc) return rc;
  std::copy(Av.begin(), Av.end(), A);
  return HYDOT_OK;
}

int shape_compare_impl(hydot_ctx* ctx, const float* mu, const float* mu_hat, double level, double* rel_l2,
                       double* dice) {
  if (!mu || !mu_hat) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  const long long N = ctx->N;
  const unsigned blocks = (unsigned)std::min<long long>((N + 255) / 256, 152 * 4);
  double* part = nullptr;
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&part, sizeof(double) * 5 * blocks));
  k_shape_compare<<<blocks, 256, 0, ctx->stream>>>(mu, mu_hat, N, (float)level, part);
  ++ctx->launches;
  std::vector<double> h((size_t)5 * blocks);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(part);
  if (e != cudaSuccess) return fail(ctx, HYDOT_ERR_CUDA, std::string("shape compare: ") + cudaGetErrorString(e));
  double s[5] = {0, 0, 0, 0, 0};
  for (unsigned b = 0; b < blocks; ++b)
    for (int q = 0; q < 5; ++q) s[q] += h[(size_t)b * 5 + q];
  if (rel_l2) *rel_l2 = s[1] > 0 ? std::sqrt(s[0] / s[1]) : 0.0;
  if (dice) *dice = (s[2] + s[3]) > 0 ? 2.0 * s[4] / (s[2] + s[3]) : 1.0;
  return HYDOT_OK;
}

// Algorithm alg:opt. U [rows][rank] (ldU), V [n_chrom * N][rank] (ldV), y [rows]: device FP32;
// S [rank], p [5 n_basis], c [n_chrom]: host FP64 (p, c in and out).
int pals_reconstruct_impl(hydot_ctx* ctx, const float* U, long long ldU, long long rows, const double* S,
                          const float* V, long long ldV, int rank, const float* y, int n_basis, double* p, double* c,
                          const hydot_pals_options* opt, hydot_pals_result* res) {
  if (n_basis < 1 || n_basis > PALS_MAXB) return fail(ctx, HYDOT_ERR_ARG, "n_basis must be in 1..8");
  if (!U || !S || !V || !y || !p || !c || !opt) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  if (rank < 1 || ldU < rank || ldV < rank || rows < 1) return fail(ctx, HYDOT_ERR_ARG, "bad rank or leading dimension");
  if (!(opt->eps > 0.0) || !(opt->nu >= 0.0)) return fail(ctx, HYDOT_ERR_ARG, "eps must be > 0 and nu >= 0");
  const int nc = ctx->n_chrom, r = rank, np = 5 * n_basis;
  PalsWork w{ctx, make_pals_geo(ctx, n_basis, opt->tau, opt->eps, opt->nu), V, ldV, r, nc, 1 + np};
  int rc = w.alloc();
  if (rc) return rc;
  const int Q = w.Q;
  // yh = U^T y and |y|^2: the part of y outside range(U) is a constant of the problem
  std::vector<double> yh, y2;
  if ((rc = tall_cross(ctx, U, ldU, r, y, 1, 1, rows, yh))) return rc;
  if ((rc = tall_cross(ctx, y, 1, 1, y, 1, 1, rows, y2))) return rc;
  double yh2 = 0.0;
  for (int k = 0; k < r; ++k) yh2 += yh[k] * yh[k];
  const double out2 = std::max(y2[0] - yh2, 0.0);
  std::vector<double> P(p, p + np), C(c, c + nc);
  int evals = 0, accepted = 0;
  std::vector<double> A, e(r), Jp((size_t)r * np);
  double resid = 0.0;
  // residual eps_h = yh - S M c and Jacobian -S sum_c c_c V_c^T dmu/dp from A
  auto terms = [&](const std::vector<double>& Am, const std::vector<double>& Cv, std::vector<double>& ev,
                   std::vector<double>& Jv) {
    double ee = 0.0;
    for (int k = 0; k < r; ++k) {
      double m = 0.0;
      for (int cc = 0; cc < nc; ++cc) m += Am[((size_t)cc * r + k) * Q] * Cv[cc];
      ev[k] = yh[k] - S[k] * m;
      ee += ev[k] * ev[k];
      for (int q = 0; q < np; ++q) {
        double j = 0.0;
        for (int cc = 0; cc < nc; ++cc) j += Cv[cc] * Am[((size_t)cc * r + k) * Q + 1 + q];
        Jv[(size_t)k * np + q] = -S[k] * j;
      }
    }
    return std::sqrt(out2 + ee);
  };
  auto evaluate = [&](const std::vector<double>& Pv, const std::vector<double>& Cv, std::vector<double>& Am,
                      std::vector<double>& ev, std::vector<double>& Jv, double& rs) -> int {
    ++evals;
    int rr = w.project(Pv, Am);
    if (rr) return rr;
    rs = terms(Am, Cv, ev, Jv);
    return (int)HYDOT_OK;
  };
  if ((rc = evaluate(P, C, A, e, Jp, resid))) return rc;
  const double resid0 = resid;
  const double target = opt->gamma * opt->noise_norm;
  std::vector<double> A2, e2(r), Jp2((size_t)r * np), G((size_t)np * np), g(np), dp;
  for (int outer = 0; outer < opt->max_outer; ++outer) {
    if (resid <= target) break;
    const double outer_start = resid;
    if (!opt->fix_c) {
      // the linear least-squares step: min |yh - D c|, D = S M, by the normal equations
      std::vector<double> DD((size_t)nc * nc, 0.0), Db(nc, 0.0), cn;
      for (int k = 0; k < r; ++k)
        for (int a = 0; a < nc; ++a) {
          const double da = S[k] * A[((size_t)a * r + k) * Q];
          Db[a] += da * yh[k];
          for (int b2 = 0; b2 < nc; ++b2) DD[(size_t)a * nc + b2] += da * S[k] * A[((size_t)b2 * r + k) * Q];
        }
      if (spd_solve(DD, nc, Db, cn)) {
        C = cn;
        resid = terms(A, C, e, Jp);
      }
    }
    double jmax = 0.0;
    for (int q = 0; q < np; ++q) {
      double d = 0.0;
      for (int k = 0; k < r; ++k) d += Jp[(size_t)k * np + q] * Jp[(size_t)k * np + q];
      jmax = std::max(jmax, d);
    }
    double nu = opt->lm_nu0 * jmax;
    for (int inner = 0; inner < opt->max_inner; ++inner) {
      if (resid <= target) break;
      // (J^T J + nu I) dp = -J^T eps
      for (int a = 0; a < np; ++a) {
        double gs = 0.0;
        for (int k = 0; k < r; ++k) gs += Jp[(size_t)k * np + a] * e[k];
        g[a] = -gs;
        for (int b2 = 0; b2 < np; ++b2) {
          double s2 = 0.0;
          for (int k = 0; k < r; ++k) s2 += Jp[(size_t)k * np + a] * Jp[(size_t)k * np + b2];
          G[(size_t)a * np + b2] = s2 + (a == b2 ? nu : 0.0);
        }
      }
      if (!spd_solve(G, np, g, dp)) {
        nu *= 4.0;
        continue;
      }
      std::vector<double> P2(np);
      double dn = 0.0, pn = 0.0;
      for (int q = 0; q < np; ++q) {
        P2[q] = P[q] + dp[q];
        dn += dp[q] * dp[q];
        pn += P2[q] * P2[q];
      }
      double resid2 = 0.0;
      if ((rc = evaluate(P2, C, A2, e2, Jp2, resid2))) return rc;
      if (resid2 < resid) {
        P.swap(P2);
        A.swap(A2);
        e.swap(e2);
        Jp.swap(Jp2);
        resid = resid2;
        ++accepted;
        nu /= 3.0;
        if (std::sqrt(dn) <= 1e-10 * (1.0 + std::sqrt(pn))) break;
      } else {
        nu *= 4.0;
      }
    }
    if (resid >= outer_start * (1.0 - 1e-6)) break;
  }
  std::copy(P.begin(), P.end(), p);
  std::copy(C.begin(), C.end(), c);
  if (res) {
    res->evaluations = evals;
    res->accepted = accepted;
    res->residual0 = resid0;
    res->residual = resid;
  }
  return HYDOT_OK;
}

}  // namespace hydot
