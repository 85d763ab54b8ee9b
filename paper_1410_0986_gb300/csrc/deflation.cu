// Recycled deflation subspace shared by all wavelengths (Section 3).
//
// The paper builds one approximately invariant subspace from a Krylov space of the
// shift-independent part of the operator and reuses it for every wavelength, updating only small
// k x k quantities per shift (Section 3.2: the Gram matrix of the updated basis from precomputed
// k x k blocks, then a Cholesky factorisation, O(k^3) per wavelength). For the symmetric CG setting
// here that becomes:
//   1. m Lanczos steps (FP64, full reorthogonalisation) on the base operator
//      Ahat_0 = Lg + mean(sigma) I + sum_f mean(bhat_f) B_f, i.e. with the mean shift and the mean
//      boundary term folded in (the mean-shift transformation of Section 6.1);
//   2. W = the Ritz vectors of the k smallest Ritz values, orthonormalised by CholeskyQR2;
//   3. shift-independent blocks W^T Lg W and W^T B_f W (Lg: graph Laplacian of the grid, B_f: the
//      indicator of the cells on face f), so that for every wavelength
//        G_j = W^T Ahat_j W = W^T Lg W + sigma_j I + sum_f bhat_{f,j} W^T B_f W,
//      and its inverse via Cholesky (k x k, host, FP64);
//   4. each field starts from the Galerkin projection x0 = W G_j^-1 W^T b (b = e_cell, so
//      W^T b is the optode cell's row of W).
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "dense.h"
#include "hydot_internal.cuh"

namespace hydot {

namespace {

constexpr int DT = 256;  // threads per block of the setup kernels

// y = (Lg + s I + sum_f bf[f] B_f) v for one FP64 vector (setup only).
__global__ void k_op64(int nx, int ny, int nz, double s, double b0, double b1, double b2, double b3, double b4,
                       double b5, const double* __restrict__ v, double* __restrict__ y) {
  const long long N = (long long)nx * ny * nz;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % nx);
    const int j = (int)((id / nx) % ny);
    const int k = (int)(id / ((long long)nx * ny));
    double d = s, acc = 0.0;
    if (i > 0) { d += 1.0; acc += v[id - 1]; } else d += b0;
    if (i < nx - 1) { d += 1.0; acc += v[id + 1]; } else d += b1;
    if (j > 0) { d += 1.0; acc += v[id - nx]; } else d += b2;
    if (j < ny - 1) { d += 1.0; acc += v[id + nx]; } else d += b3;
    if (k > 0) { d += 1.0; acc += v[id - (long long)nx * ny]; } else d += b4;
    if (k < nz - 1) { d += 1.0; acc += v[id + (long long)nx * ny]; } else d += b5;
    y[id] = d * v[id] - acc;
  }
}

// Partial dot products of vectors A[a] (stride lda) with B[b] for all pairs: grid (blocks, na*nb).
__global__ void k_dots(const double* __restrict__ A, long long lda, int na, const double* __restrict__ B, long long ldb,
                       long long N, double* __restrict__ part) {
  __shared__ double sm[DT / 32];
  const int pair = blockIdx.y;
  const int a = pair % na, b = pair / na;
  const double* x = A + (size_t)a * lda;
  const double* y = B + (size_t)b * ldb;
  double acc = 0.0;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x)
    acc += x[id] * y[id];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < DT / 32; ++w) s += sm[w];
    part[(size_t)pair * gridDim.x + blockIdx.x] = s;
  }
}

// out[p] = sum over blocks of part[p][*], in a fixed order.
__global__ void k_sum_parts(const double* __restrict__ part, int nblk, int npairs, double* __restrict__ out) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  double s = 0.0;
  for (int q = 0; q < nblk; ++q) s += part[(size_t)p * nblk + q];
  out[p] = s;
}

// w -= sum_j h[j] V[j]  (V: nv vectors of length N, contiguous)
__global__ void k_sub_comb(double* __restrict__ w, const double* __restrict__ V, const double* __restrict__ h, int nv,
                           long long N) {
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s += h[j] * V[(size_t)j * N + id];
    w[id] -= s;
  }
}

__global__ void k_scale_copy(const double* __restrict__ w, double a, double* __restrict__ v, long long N) {
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x)
    v[id] = a * w[id];
}

// Wt[i][cell] = sum_j V[j][cell] * Y[j][i]  (Ritz vectors), or in place W <- W Rinv (triangular)
__global__ void k_combine(const double* __restrict__ V, int m, const double* __restrict__ Y, int k, long long N,
                          double* __restrict__ Wt) {
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x) {
    double acc[32];
    for (int i = 0; i < k; ++i) acc[i] = 0.0;
    for (int j = 0; j < m; ++j) {
      const double v = V[(size_t)j * N + id];
      for (int i = 0; i < k; ++i) acc[i] += v * Y[j * k + i];
    }
    for (int i = 0; i < k; ++i) Wt[(size_t)i * N + id] = acc[i];
  }
}

// Wt[i] <- sum_j Wt[j] Rinv[j][i] (upper-triangular Rinv), in place per cell
__global__ void k_right_tri(double* __restrict__ Wt, const double* __restrict__ Rinv, int k, long long N) {
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x) {
    double w[32], o[32];
    for (int j = 0; j < k; ++j) w[j] = Wt[(size_t)j * N + id];
    for (int i = 0; i < k; ++i) {
      double s = 0.0;
      for (int j = 0; j <= i; ++j) s += w[j] * Rinv[j * k + i];
      o[i] = s;
    }
    for (int i = 0; i < k; ++i) Wt[(size_t)i * N + id] = o[i];
  }
}

// Y[i] = B_f W[i]: W restricted to the cells of face f
__global__ void k_face_mask(const double* __restrict__ Wt, int k, int nx, int ny, int nz, int f, double* __restrict__ Y) {
  const long long N = (long long)nx * ny * nz;
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(id % nx), j = (int)((id / nx) % ny), kk = (int)(id / ((long long)nx * ny));
    const bool on = (f == 0 && i == 0) || (f == 1 && i == nx - 1) || (f == 2 && j == 0) || (f == 3 && j == ny - 1) ||
                    (f == 4 && kk == 0) || (f == 5 && kk == nz - 1);
    for (int q = 0; q < k; ++q) Y[(size_t)q * N + id] = on ? Wt[(size_t)q * N + id] : 0.0;
  }
}

struct Dev {
  hydot_ctx* ctx;
  double* part = nullptr;
  double* res = nullptr;
  int nblk = 152 * 2;
  ~Dev() {
    cudaFree(part);
    cudaFree(res);
  }
};

// all pairwise dots of na vectors of A with nb vectors of B -> host out[b*na + a]
int dots(Dev& d, const double* A, int na, const double* B, int nb, long long N, std::vector<double>& out) {
  hydot_ctx* ctx = d.ctx;
  const int np = na * nb;
  dim3 grid(d.nblk, np);
  k_dots<<<grid, DT, 0, ctx->stream>>>(A, N, na, B, N, N, d.part);
  k_sum_parts<<<(np + 255) / 256, 256, 0, ctx->stream>>>(d.part, d.nblk, np, d.res);
  ctx->launches += 2;
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  out.resize(np);
  HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(out.data(), d.res, sizeof(double) * np, cudaMemcpyDeviceToHost, ctx->stream));
  HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return HYDOT_OK;
}

}  // namespace

int build_deflation(hydot_ctx* ctx) {
  const int k = ctx->deflation_k;
  if (k == 0) return HYDOT_OK;
  if (ctx->cplx) return fail(ctx, HYDOT_ERR_ARG, "deflation is available for continuous-wave (real) fields only");
  const long long N = ctx->N;
  if (N < 4LL * k) return fail(ctx, HYDOT_ERR_ARG, "grid too small for the requested deflation_k");
  const int m = (int)std::min<long long>(std::max(4 * k, 48), std::min<long long>(N, 128));
  cudaStream_t s = ctx->stream;
  const int nx = ctx->nx, ny = ctx->ny, nz = ctx->nz;
  // base operator: mean shift and mean boundary terms over the wavelengths
  double sbar = 0.0, bbar[6] = {0, 0, 0, 0, 0, 0};
  for (int j = 0; j < ctx->n_lambda; ++j) {
    sbar += ctx->coef[j].sigma_re / ctx->n_lambda;
    for (int f = 0; f < 6; ++f) bbar[f] += ctx->coef[j].bhat[f] / ctx->n_lambda;
  }
  Dev d{ctx};
  double *V = nullptr, *w = nullptr, *Wt = nullptr, *Y = nullptr, *h = nullptr;
  bool keep_w = false;
  auto cleanup = [&]() {
    cudaFree(V);
    cudaFree(w);
    cudaFree(Y);
    cudaFree(h);
    if (!keep_w) cudaFree(Wt);
  };
#define DTRY(call)                                                                   \
  do {                                                                              \
    cudaError_t e__ = (call);                                                       \
    if (e__ != cudaSuccess) {                                                       \
      cleanup();                                                                    \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e__);               \
      return e__ == cudaErrorMemoryAllocation ? HYDOT_ERR_OOM : HYDOT_ERR_CUDA;      \
    }                                                                               \
  } while (0)
  DTRY(cudaMalloc(&d.part, sizeof(double) * (size_t)d.nblk * std::max(m, k * k)));
  DTRY(cudaMalloc(&d.res, sizeof(double) * std::max(m, k * k)));
  DTRY(cudaMalloc(&V, sizeof(double) * (size_t)(m + 1) * N));
  DTRY(cudaMalloc(&w, sizeof(double) * N));
  DTRY(cudaMalloc(&Wt, sizeof(double) * (size_t)k * N));
  DTRY(cudaMalloc(&Y, sizeof(double) * (size_t)k * N));
  DTRY(cudaMalloc(&h, sizeof(double) * (m + 1)));
  const unsigned g1 = (unsigned)std::min<long long>((N + DT - 1) / DT, 4096);
  // start vector: all ones (smooth, overlaps the lowest modes), normalised
  {
    std::vector<double> ones(N, 1.0 / std::sqrt((double)N));
    DTRY(cudaMemcpy(V, ones.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
  }
  std::vector<double> alpha, beta;
  std::vector<double> hv;
  int steps = 0;
  for (int j = 0; j < m; ++j) {
    double* vj = V + (size_t)j * N;
    k_op64<<<g1, DT, 0, s>>>(nx, ny, nz, sbar, bbar[0], bbar[1], bbar[2], bbar[3], bbar[4], bbar[5], vj, w);
    ++ctx->launches;
    // full reorthogonalisation (twice): h = V^T w; w -= V h
    for (int pass = 0; pass < 2; ++pass) {
      int rc = dots(d, V, j + 1, w, 1, N, hv);
      if (rc) { cleanup(); return rc; }
      if (pass == 0) alpha.push_back(hv[j]);
      DTRY(cudaMemcpyAsync(h, hv.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, s));
      k_sub_comb<<<g1, DT, 0, s>>>(w, V, h, j + 1, N);
      ++ctx->launches;
    }
    std::vector<double> nn;
    int rc = dots(d, w, 1, w, 1, N, nn);
    if (rc) { cleanup(); return rc; }
    const double b = std::sqrt(std::max(nn[0], 0.0));
    steps = j + 1;
    if (j + 1 < m) {
      if (!(b > 1e-12 * std::fabs(alpha[j]))) break;  // invariant subspace found
      beta.push_back(b);
      k_scale_copy<<<g1, DT, 0, s>>>(w, 1.0 / b, V + (size_t)(j + 1) * N, N);
      ++ctx->launches;
    }
  }
  const int mm = steps;
  if (mm < k) { cleanup(); return fail(ctx, HYDOT_ERR_STATE, "Lanczos found fewer vectors than deflation_k"); }
  // Ritz pairs of the tridiagonal T_mm; keep the k smallest
  std::vector<double> T((size_t)mm * mm, 0.0), lam, Z;
  for (int i = 0; i < mm; ++i) {
    T[(size_t)i * mm + i] = alpha[i];
    if (i + 1 < mm) T[(size_t)i * mm + i + 1] = T[(size_t)(i + 1) * mm + i] = beta[i];
  }
  if (!sym_eig(T, mm, lam, Z)) {
    cleanup();
    return fail(ctx, HYDOT_ERR_NOT_CONVERGED, "host eigensolver did not converge on the Lanczos tridiagonal");
  }
  std::vector<int> order(mm);
  for (int i = 0; i < mm; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return lam[a] < lam[b]; });
  std::vector<double> Yk((size_t)mm * k);
  for (int j = 0; j < mm; ++j)
    for (int i = 0; i < k; ++i) Yk[(size_t)j * k + i] = Z[(size_t)j * mm + order[i]];
  double* dY = nullptr;
  DTRY(cudaMalloc(&dY, sizeof(double) * (size_t)mm * k));
  DTRY(cudaMemcpy(dY, Yk.data(), sizeof(double) * (size_t)mm * k, cudaMemcpyHostToDevice));
  k_combine<<<g1, DT, 0, s>>>(V, mm, dY, k, N, Wt);
  ++ctx->launches;
  DTRY(cudaStreamSynchronize(s));
  cudaFree(dY);
  // CholeskyQR2: W <- W R^-1, twice
  double* dRi = nullptr;
  DTRY(cudaMalloc(&dRi, sizeof(double) * k * k));
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<double> G, R;
    int rc = dots(d, Wt, k, Wt, k, N, G);
    if (rc) { cudaFree(dRi); cleanup(); return rc; }
    if (!cholesky_upper(G, k, R)) { cudaFree(dRi); cleanup(); return fail(ctx, HYDOT_ERR_STATE, "CholeskyQR2 of the deflation basis failed"); }
    std::vector<double> Ri = tri_inv_upper(R, k);
    DTRY(cudaMemcpy(dRi, Ri.data(), sizeof(double) * k * k, cudaMemcpyHostToDevice));
    k_right_tri<<<g1, DT, 0, s>>>(Wt, dRi, k, N);
    ++ctx->launches;
  }
  cudaFree(dRi);
  // shift-independent k x k blocks: W^T Lg W and W^T B_f W
  std::vector<double> GL, GI;
  for (int q = 0; q < k; ++q) {
    k_op64<<<g1, DT, 0, s>>>(nx, ny, nz, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, Wt + (size_t)q * N, Y + (size_t)q * N);
    ++ctx->launches;
  }
  int rc = dots(d, Wt, k, Y, k, N, GL);
  if (!rc) rc = dots(d, Wt, k, Wt, k, N, GI);
  if (rc) { cleanup(); return rc; }
  std::vector<std::vector<double>> GB(6);
  for (int f = 0; f < 6; ++f) {
    k_face_mask<<<g1, DT, 0, s>>>(Wt, k, nx, ny, nz, f, Y);
    ++ctx->launches;
    rc = dots(d, Wt, k, Y, k, N, GB[f]);
    if (rc) { cleanup(); return rc; }
  }
  ctx->gram_L = GL;
  ctx->gram_I = GI;
  ctx->gram_B.clear();
  for (int f = 0; f < 6; ++f) ctx->gram_B.insert(ctx->gram_B.end(), GB[f].begin(), GB[f].end());
  // per wavelength: G_j = W^T Lg W + sigma_j W^T W + sum_f bhat_{f,j} W^T B_f W; store G_j^-1
  std::vector<double> Ginv((size_t)ctx->n_lambda * k * k);
  for (int j = 0; j < ctx->n_lambda; ++j) {
    std::vector<double> G((size_t)k * k), R;
    for (int q = 0; q < k * k; ++q) {
      double v = GL[q] + ctx->coef[j].sigma_re * GI[q];
      for (int f = 0; f < 6; ++f) v += ctx->coef[j].bhat[f] * GB[f][q];
      G[q] = v;
    }
    for (int a = 0; a < k; ++a)  // symmetrise (the blocks are symmetric up to rounding)
      for (int b = a + 1; b < k; ++b) G[(size_t)a * k + b] = G[(size_t)b * k + a] = 0.5 * (G[(size_t)a * k + b] + G[(size_t)b * k + a]);
    if (!cholesky_upper(G, k, R)) { cleanup(); return fail(ctx, HYDOT_ERR_STATE, "Galerkin matrix of the deflation basis is not positive definite"); }
    std::vector<double> Ri = tri_inv_upper(R, k);  // G^-1 = Ri Ri^T
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        double v = 0.0;
        for (int p = std::max(a, b); p < k; ++p) v += Ri[(size_t)a * k + p] * Ri[(size_t)b * k + p];
        Ginv[((size_t)j * k + a) * k + b] = v;
      }
  }
  DTRY(cudaMalloc(&ctx->d_Ginv, sizeof(double) * Ginv.size()));
  DTRY(cudaMemcpy(ctx->d_Ginv, Ginv.data(), sizeof(double) * Ginv.size(), cudaMemcpyHostToDevice));
  DTRY(cudaMalloc(&ctx->d_defl_coef, sizeof(double) * (size_t)ctx->max_fields * k));
  ctx->d_W = Wt;  // [k][N], owned by the context from here on
  keep_w = true;
  ctx->deflation_ritz.assign(lam.begin(), lam.end());
  std::sort(ctx->deflation_ritz.begin(), ctx->deflation_ritz.end());
  cleanup();
#undef DTRY
  return HYDOT_OK;
}

// x0 = W G_j^-1 W^T e_src for every field of the batch (the Galerkin initial guess).
__global__ void k_deflate_coef(const double* __restrict__ Wt, const double* __restrict__ Ginv, int k, long long N,
                               const int* __restrict__ optode, int lam0, int f_begin, int nf, int nrhs,
                               double* __restrict__ C) {
  int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= nrhs) return;
  const int lam = lam0 + rhs / nf;
  const long long src = optode[f_begin + rhs % nf];
  const double* G = Ginv + (size_t)lam * k * k;
  for (int a = 0; a < k; ++a) {
    double s = 0.0;
    for (int b = 0; b < k; ++b) s += G[a * k + b] * Wt[(size_t)b * N + src];
    C[(size_t)rhs * k + a] = s;
  }
}

template <typename X>
__global__ void k_deflate_x0(const double* __restrict__ Wt, const double* __restrict__ C, int k, long long N, int nrhs,
                             X* __restrict__ x64) {
  for (long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x; id < N; id += (long long)gridDim.x * blockDim.x) {
    double wrow[32];
    for (int a = 0; a < k; ++a) wrow[a] = Wt[(size_t)a * N + id];
    for (int rhs = blockIdx.y; rhs < nrhs; rhs += gridDim.y) {
      double s = 0.0;
      for (int a = 0; a < k; ++a) s += wrow[a] * C[(size_t)rhs * k + a];
      if constexpr (std::is_same<X, df32>::value) x64[(size_t)rhs * N + id] = df_from(s);
      else x64[(size_t)rhs * N + id] = s;
    }
  }
}

int deflate_initial_guess(hydot_ctx* ctx, int lam0, int f_begin, int nf, int nrhs, void* x64, bool df) {
  const int k = ctx->deflation_k;
  double* C = ctx->d_defl_coef;
  k_deflate_coef<<<(nrhs + 127) / 128, 128, 0, ctx->stream>>>(ctx->d_W, ctx->d_Ginv, k, ctx->N, ctx->d_optode, lam0,
                                                               f_begin, nf, nrhs, C);
  dim3 grid((unsigned)std::min<long long>((ctx->N + 255) / 256, 1024), (unsigned)std::min(nrhs, 64));
  if (df) k_deflate_x0<df32><<<grid, 256, 0, ctx->stream>>>(ctx->d_W, C, k, ctx->N, nrhs, (df32*)x64);
  else k_deflate_x0<double><<<grid, 256, 0, ctx->stream>>>(ctx->d_W, C, k, ctx->N, nrhs, (double*)x64);
  ctx->launches += 2;
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  return HYDOT_OK;
}

}  // namespace hydot
