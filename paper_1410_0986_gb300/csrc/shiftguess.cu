// Shift-invariant initial guesses (Section 3, 3.2; the base operator at the mean shift, Section 6.1).
//
// Every field of every wavelength solves Ahat_j x = e_c, where the scaled operators of the
// wavelengths differ only by the shift sigma_j and the boundary terms bhat_{f,j}:
//   Ahat_j = Lg + sigma_j I + sum_f bhat_{f,j} B_f.
// One Krylov space per optode cell c, built once on the base operator
//   Ahat_0 = Lg + mean(sigma) I + sum_f mean(bhat_f) B_f,
// serves all wavelengths: with V an orthonormal basis of K_m(Ahat_0, e_c),
//   V^T Ahat_j V = T + (sigma_j - mean sigma) I + sum_f (bhat_{f,j} - mean bhat_f) V^T B_f V,
// where T = V^T Ahat_0 V is the Lanczos tridiagonal and V^T B_f V involves only the cells of face f;
// the guess x_j = V (V^T Ahat_j V)^-1 V^T e_c then needs no product with Ahat_j (Section 3.2: the
// projected matrices are updated per shift from quantities computed once).
//
// Build (hydot_set_shift_guess), batched over all n_src + n_det fields, vectors in FP32:
//   Lanczos with two passes of full reorthogonalisation per step; dot products as FP32 partial sums
//   over runs of cells, added in FP64 in a fixed order; alpha, beta kept in FP64 on the device.
//   Then V^T B_f V for the six faces.
// Per solve (shift_initial_guess): one block per (wavelength, field) forms V^T Ahat_j V, factors
// it (Cholesky, FP64) and solves for the coefficients; one pass over the bases forms x_j in FP32
// and stores it as the FP64 iterate the refinement starts from. The bases only have to span the
// space: their FP32 rounding changes the guess by ~1e-7 relative, which the refinement removes.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "hydot_internal.cuh"

namespace hydot {

namespace {

constexpr int SG_T = 256;      // threads per block
constexpr int SG_MAXM = 64;    // largest basis
constexpr int SG_CELLS = 4096; // cells per block of the dot-product kernel

// y[f] = Ahat_0 v[f] for F vectors (stride ldv between fields), FP32
__global__ void k_sg_op(int nx, int ny, int nz, float s, const float* __restrict__ bb, const float* __restrict__ v,
                        long long ldv, int F, float* __restrict__ y) {
  const long long N = (long long)nx * ny * nz;
  const long long tot = N * F;
  const float b0 = bb[0], b1 = bb[1], b2 = bb[2], b3 = bb[3], b4 = bb[4], b5 = bb[5];
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / N);
    const long long id = q - (long long)f * N;
    const float* vf = v + (size_t)f * ldv;
    const int i = (int)(id % nx);
    const int j = (int)((id / nx) % ny);
    const int k = (int)(id / ((long long)nx * ny));
    float d = s, acc = 0.f;
    if (i > 0) { d += 1.f; acc += vf[id - 1]; } else d += b0;
    if (i < nx - 1) { d += 1.f; acc += vf[id + 1]; } else d += b1;
    if (j > 0) { d += 1.f; acc += vf[id - nx]; } else d += b2;
    if (j < ny - 1) { d += 1.f; acc += vf[id + nx]; } else d += b3;
    if (k > 0) { d += 1.f; acc += vf[id - (long long)nx * ny]; } else d += b4;
    if (k < nz - 1) { d += 1.f; acc += vf[id + (long long)nx * ny]; } else d += b5;
    y[(size_t)f * N + id] = d * vf[id] - acc;
  }
}

// part[f][blk][i] = sum over the block's cells of V[f][i][x] * w[f][x], i < nv. Grid (nblk, F).
// A thread sums its cells in FP32; warps and blocks add in FP64.
__global__ void __launch_bounds__(SG_T) k_sg_dots(const float* __restrict__ V, long long ldf, int nv,
                                                  const float* __restrict__ w, long long N, double* __restrict__ part,
                                                  int mstride) {
  __shared__ double red[SG_MAXM][SG_T / 32];
  const int f = blockIdx.y;
  const long long c0 = (long long)blockIdx.x * SG_CELLS;
  const long long c1 = c0 + SG_CELLS < N ? c0 + SG_CELLS : N;
  const float* wf = w + (size_t)f * N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < nv; ++i) {
    const float* vi = V + (size_t)f * ldf + (size_t)i * N;
    float acc = 0.f;
    for (long long x = c0 + threadIdx.x; x < c1; x += SG_T) acc = fmaf(vi[x], wf[x], acc);
    double a = acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) red[i][warp] = a;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nv; i += SG_T) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < SG_T / 32; ++q) s += red[i][q];
    part[((size_t)f * gridDim.x + blockIdx.x) * mstride + i] = s;
  }
}

// c[f][i] = sum over blocks of part[f][*][i] (fixed order), also as FP32; for i == j (the first
// pass of step j) alpha[f][j] = c[f][j].
__global__ void k_sg_sum(const double* __restrict__ part, int nblk, int nv, int F, int mstride, double* __restrict__ c,
                         float* __restrict__ cf, double* __restrict__ alpha, int j) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= F * nv) return;
  const int f = q / nv, i = q % nv;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[((size_t)f * nblk + b) * mstride + i];
  c[(size_t)f * SG_MAXM + i] = s;
  cf[(size_t)f * SG_MAXM + i] = (float)s;
  if (alpha && i == j) alpha[(size_t)f * SG_MAXM + j] = s;
}

// w[f] -= sum_{i < nv} c[f][i] V[f][i]
__global__ void k_sg_sub(const float* __restrict__ V, long long ldf, int nv, const float* __restrict__ cf, long long N,
                         int F, float* __restrict__ w) {
  const long long tot = N * F;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / N);
    const long long x = q - (long long)f * N;
    const float* vf = V + (size_t)f * ldf + x;
    const float* cc = cf + (size_t)f * SG_MAXM;
    float s = 0.f;
    for (int i = 0; i < nv; ++i) s = fmaf(cc[i], vf[(size_t)i * N], s);
    w[q] -= s;
  }
}

// beta[f][j] = ||w[f]||; V[f][j+1] = w[f] / beta (zeros, and the basis size fixed at j + 1, when
// the recurrence has broken down: the Krylov space is invariant)
__global__ void k_sg_beta(const double* __restrict__ nrm2, int F, int j, const double* __restrict__ alpha,
                          double* __restrict__ beta, int* __restrict__ meff, float* __restrict__ scale) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const double b = sqrt(fmax(nrm2[(size_t)f * SG_MAXM], 0.0));
  const double ref = fabs(alpha[(size_t)f * SG_MAXM + j]) + (j > 0 ? beta[(size_t)f * SG_MAXM + j - 1] : 0.0);
  beta[(size_t)f * SG_MAXM + j] = b;
  const bool broken = meff[f] <= j || !(b > 1e-4 * ref);
  if (broken && meff[f] > j + 1) meff[f] = j + 1;
  scale[f] = broken ? 0.f : (float)(1.0 / b);
}

__global__ void k_sg_next(const float* __restrict__ w, const float* __restrict__ scale, long long N, int F,
                          float* __restrict__ V, long long ldf, int j1) {
  const long long tot = N * F;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(q / N);
    const long long x = q - (long long)f * N;
    V[(size_t)f * ldf + (size_t)j1 * N + x] = w[q] * scale[f];
  }
}

__global__ void k_sg_start(const int* __restrict__ optode, int F, long long N, float* __restrict__ V, long long ldf) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < F) V[(size_t)f * ldf + optode[f]] = 1.f;
}

// P[f][face][a][b] = sum over the cells of `face` of V[f][a][x] V[f][b][x] (a, b < m); grid (F, 6).
// Runs of 32 face cells are staged in shared memory; FP32 sums per run, FP64 across runs.
__global__ void __launch_bounds__(SG_T) k_sg_face(const float* __restrict__ V, long long ldf, int m, int nx, int ny,
                                                  int nz, double* __restrict__ P) {
  __shared__ float S[SG_MAXM][33];
  const int f = blockIdx.x, face = blockIdx.y;
  const long long N = (long long)nx * ny * nz;
  const int ua = face < 2 ? ny : nx;                      // fastest index along the face
  const long long ncell = face < 2 ? (long long)ny * nz : face < 4 ? (long long)nx * nz : (long long)nx * ny;
  const float* vf = V + (size_t)f * ldf;
  constexpr int QMAX = SG_MAXM * SG_MAXM / SG_T;
  double acc[QMAX];
#pragma unroll
  for (int q = 0; q < QMAX; ++q) acc[q] = 0.0;
  for (long long c0 = 0; c0 < ncell; c0 += 32) {
    for (int e = threadIdx.x; e < m * 32; e += SG_T) {
      const int a = e / 32, cc = e % 32;
      const long long c = c0 + cc;
      float v = 0.f;
      if (c < ncell) {
        const int u = (int)(c % ua), w = (int)(c / ua);
        long long x;
        if (face < 2) x = ((long long)w * ny + u) * nx + (face == 0 ? 0 : nx - 1);
        else if (face < 4) x = ((long long)w * ny + (face == 2 ? 0 : ny - 1)) * nx + u;
        else x = ((long long)(face == 4 ? 0 : nz - 1) * ny + w) * nx + u;
        v = vf[(size_t)a * N + x];
      }
      S[a][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int e = threadIdx.x + q * SG_T;
      if (e < m * m) {
        const int a = e / m, b = e % m;
        float sum = 0.f;
#pragma unroll 8
        for (int cc = 0; cc < 32; ++cc) sum = fmaf(S[a][cc], S[b][cc], sum);
        acc[q] += sum;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < QMAX; ++q) {
    const int e = threadIdx.x + q * SG_T;
    if (e < m * m) P[((size_t)f * 6 + face) * m * m + e] = acc[q];
  }
}

struct SgBase {
  double sbar;
  double bbar[6];
};

// Coefficients Y[rhs][a] of the guess of field f = f_begin + rhs % nf at wavelength lam0 + rhs / nf:
// G = T + (sigma_j - mean sigma) I + sum_face (bhat_{face,j} - mean bhat_face) P[f][face], G y = V^T e_c.
// One block per rhs; Cholesky in shared memory (FP64). A field whose G is not positive definite
// gets y = 0 (it starts from zero).
__global__ void __launch_bounds__(SG_MAXM) k_sg_solve(const double* __restrict__ alpha, const double* __restrict__ beta,
                                                       const double* __restrict__ P, const int* __restrict__ meff,
                                                       const float* __restrict__ V, long long ldf, long long N,
                                                       const int* __restrict__ optode, const LamCoef* __restrict__ coef,
                                                       SgBase base, int lam0, int f_begin, int nf, int m,
                                                       float* __restrict__ Y) {
  __shared__ double G[SG_MAXM][SG_MAXM + 1];
  __shared__ double r[SG_MAXM];
  __shared__ int bad;
  const int rhs = blockIdx.x, t = threadIdx.x;
  const int f = f_begin + rhs % nf, lam = lam0 + rhs / nf;
  const int me = meff[f];
  const LamCoef cj = coef[lam];
  const double ds = cj.sigma_re - base.sbar;
  double db[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) db[q] = cj.bhat[q] - base.bbar[q];
  const double* A = alpha + (size_t)f * SG_MAXM;
  const double* B = beta + (size_t)f * SG_MAXM;
  for (int e = t; e < me * me; e += blockDim.x) {
    const int a = e / me, b = e % me;
    double g = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) g += db[q] * P[((size_t)f * 6 + q) * m * m + (size_t)a * m + b];
    if (a == b) g += A[a] + ds;
    if (b == a + 1) g += B[a];
    if (a == b + 1) g += B[b];
    G[a][b] = g;
  }
  for (int a = t; a < me; a += blockDim.x) r[a] = V[(size_t)f * ldf + (size_t)a * N + optode[f]];
  if (t == 0) bad = 0;
  __syncthreads();
  for (int k = 0; k < me; ++k) {
    if (t == 0) {
      const double d = G[k][k];
      if (!(d > 0.0)) bad = 1;
      G[k][k] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    for (int i = k + 1 + t; i < me; i += blockDim.x) G[i][k] /= G[k][k];
    __syncthreads();
    const int w = me - k - 1;
    for (int e = t; e < w * w; e += blockDim.x) {
      const int i = k + 1 + e / w, jj = k + 1 + e % w;
      if (jj <= i) G[i][jj] -= G[i][k] * G[jj][k];
    }
    __syncthreads();
  }
  if (t == 0) {
    for (int i = 0; i < me; ++i) {  // L z = r
      double s = r[i];
      for (int q = 0; q < i; ++q) s -= G[i][q] * r[q];
      r[i] = s / G[i][i];
    }
    for (int i = me - 1; i >= 0; --i) {  // L^T y = z
      double s = r[i];
      for (int q = i + 1; q < me; ++q) s -= G[q][i] * r[q];
      r[i] = s / G[i][i];
    }
  }
  __syncthreads();
  for (int a = t; a < m; a += blockDim.x) Y[(size_t)rhs * m + a] = (a < me && !bad) ? (float)r[a] : 0.f;
}

// x64[(l * nf + fl)][x] = sum_a V[f_begin + fl][a][x] Y[(l * nf + fl)][a] for wavelengths l of
// [l0, l0 + nl), nl <= SG_LB; grid (cell blocks, nf)
constexpr int SG_LB = 16;
template <typename X>
__global__ void __launch_bounds__(SG_T) k_sg_x0(const float* __restrict__ V, long long ldf, long long N,
                                                const float* __restrict__ Y, int nf, int f_begin, int l0, int nl, int m,
                                                const int* __restrict__ meff, X* __restrict__ x64) {
  // coefficients as ys[a][l] (zero for l >= nl): the 16 of one basis vector are four 16-byte loads
  __shared__ __align__(16) float ys[SG_MAXM][SG_LB];
  const int fl = blockIdx.y, f = f_begin + fl;
  for (int e = threadIdx.x; e < SG_LB * m; e += SG_T) {
    const int l = e / m, a = e % m;
    ys[a][l] = l < nl ? Y[((size_t)(l0 + l) * nf + fl) * m + a] : 0.f;
  }
  __syncthreads();
  const int me = meff[f];
  const float* vf = V + (size_t)f * ldf;
  for (long long x = (long long)blockIdx.x * SG_T + threadIdx.x; x < N; x += (long long)gridDim.x * SG_T) {
    float acc[SG_LB];
#pragma unroll
    for (int l = 0; l < SG_LB; ++l) acc[l] = 0.f;
    for (int a = 0; a < me; ++a) {
      const float v = vf[(size_t)a * N + x];
      const float4* y4 = reinterpret_cast<const float4*>(ys[a]);
#pragma unroll
      for (int q = 0; q < SG_LB / 4; ++q) {
        const float4 c = y4[q];
        acc[4 * q] = fmaf(v, c.x, acc[4 * q]);
        acc[4 * q + 1] = fmaf(v, c.y, acc[4 * q + 1]);
        acc[4 * q + 2] = fmaf(v, c.z, acc[4 * q + 2]);
        acc[4 * q + 3] = fmaf(v, c.w, acc[4 * q + 3]);
      }
    }
#pragma unroll
    for (int l = 0; l < SG_LB; ++l) {
      if (l < nl) {
        if constexpr (std::is_same<X, df32>::value) x64[((size_t)(l0 + l) * nf + fl) * N + x] = df32{acc[l], 0.f};
        else x64[((size_t)(l0 + l) * nf + fl) * N + x] = (X)acc[l];
      }
    }
  }
}

// phi[l][f][x] = x64[(l * nf + fl)][x] / (D h) of the wavelength, for the fields of a batch
template <typename O>
__global__ void k_sg_out(const double* __restrict__ x64, const LamCoef* __restrict__ coef, int lam0, int nlam, int nf,
                         int f_begin, int n_src, long long N, O* __restrict__ phi_src, O* __restrict__ phi_det) {
  const long long tot = (long long)nlam * nf * N;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < tot; q += (long long)gridDim.x * blockDim.x) {
    const long long rhs = q / N;
    const long long x = q - rhs * N;
    const int l = (int)(rhs / nf), f = f_begin + (int)(rhs % nf);
    const double v = x64[q] * coef[lam0 + l].inv_Dh;
    if (f < n_src) phi_src[((size_t)l * n_src + f) * N + x] = (O)v;
    else phi_det[((size_t)l * (nf - n_src) + (f - n_src)) * N + x] = (O)v;
  }
}

}  // namespace

void shift_guess_free(hydot_ctx* ctx) {
  cudaFree(ctx->d_sgV);
  cudaFree(ctx->d_sgA);
  cudaFree(ctx->d_sgB);
  cudaFree(ctx->d_sgP);
  cudaFree(ctx->d_sgMeff);
  cudaFree(ctx->d_sgY);
  ctx->d_sgV = nullptr;
  ctx->d_sgA = ctx->d_sgB = ctx->d_sgP = nullptr;
  ctx->d_sgMeff = nullptr;
  ctx->d_sgY = nullptr;
  ctx->sg_m = 0;
}

int set_shift_guess_impl(hydot_ctx* ctx, int m) {
  if (m < 0 || m > SG_MAXM) return fail(ctx, HYDOT_ERR_ARG, "basis size m must be in 0..64");
  HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));  // the old bases may still be in use
  shift_guess_free(ctx);
  if (m == 0) return HYDOT_OK;
  if (ctx->cplx) return fail(ctx, HYDOT_ERR_STATE, "shift-invariant guesses are built for continuous-wave fields only");
  if (ctx->deflation_k > 0)
    return fail(ctx, HYDOT_ERR_STATE, "shift-invariant guesses and the recycled deflation basis are exclusive");
  const long long N = ctx->N;
  m = (int)std::min<long long>(m, N);
  const int F = ctx->n_src + ctx->n_det;
  const int nx = ctx->nx, ny = ctx->ny, nz = ctx->nz;
  cudaStream_t s = ctx->stream;
  // base operator: the mean shift and the mean boundary terms over the wavelengths
  SgBase base{};
  for (int j = 0; j < ctx->n_lambda; ++j) {
    base.sbar += ctx->coef[j].sigma_re / ctx->n_lambda;
    for (int f = 0; f < 6; ++f) base.bbar[f] += ctx->coef[j].bhat[f] / ctx->n_lambda;
  }
  const long long ldf = (long long)m * N;
  const int nblk = (int)((N + SG_CELLS - 1) / SG_CELLS);
  float *w = nullptr, *cf = nullptr, *scale = nullptr, *bb = nullptr;
  double *part = nullptr, *c = nullptr;
  auto cleanup = [&]() {
    cudaFree(w);
    cudaFree(cf);
    cudaFree(scale);
    cudaFree(bb);
    cudaFree(part);
    cudaFree(c);
  };
#define STRY(call)                                                                   \
  do {                                                                              \
    cudaError_t e__ = (call);                                                       \
    if (e__ != cudaSuccess) {                                                       \
      cleanup();                                                                    \
      shift_guess_free(ctx);                                                        \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e__);               \
      return e__ == cudaErrorMemoryAllocation ? HYDOT_ERR_OOM : HYDOT_ERR_CUDA;      \
    }                                                                               \
  } while (0)
  STRY(cudaMalloc(&ctx->d_sgV, sizeof(float) * (size_t)F * ldf));
  STRY(cudaMalloc(&ctx->d_sgA, sizeof(double) * (size_t)F * SG_MAXM));
  STRY(cudaMalloc(&ctx->d_sgB, sizeof(double) * (size_t)F * SG_MAXM));
  STRY(cudaMalloc(&ctx->d_sgP, sizeof(double) * (size_t)F * 6 * m * m));
  STRY(cudaMalloc(&ctx->d_sgMeff, sizeof(int) * F));
  STRY(cudaMalloc(&ctx->d_sgY, sizeof(float) * (size_t)ctx->max_fields * m));
  STRY(cudaMalloc(&w, sizeof(float) * (size_t)F * N));
  STRY(cudaMalloc(&cf, sizeof(float) * (size_t)F * SG_MAXM));
  STRY(cudaMalloc(&scale, sizeof(float) * F));
  STRY(cudaMalloc(&bb, sizeof(float) * 6));
  STRY(cudaMalloc(&part, sizeof(double) * (size_t)F * nblk * SG_MAXM));
  STRY(cudaMalloc(&c, sizeof(double) * (size_t)F * SG_MAXM));
  {
    float bbf[6];
    for (int f = 0; f < 6; ++f) bbf[f] = (float)base.bbar[f];
    STRY(cudaMemcpyAsync(bb, bbf, sizeof(bbf), cudaMemcpyHostToDevice, s));
    std::vector<int> me(F, m);
    STRY(cudaMemcpyAsync(ctx->d_sgMeff, me.data(), sizeof(int) * F, cudaMemcpyHostToDevice, s));
    STRY(cudaStreamSynchronize(s));  // the host staging arrays go out of scope
  }
  STRY(cudaMemsetAsync(ctx->d_sgV, 0, sizeof(float) * (size_t)F * ldf, s));
  STRY(cudaMemsetAsync(ctx->d_sgA, 0, sizeof(double) * (size_t)F * SG_MAXM, s));
  STRY(cudaMemsetAsync(ctx->d_sgB, 0, sizeof(double) * (size_t)F * SG_MAXM, s));
  k_sg_start<<<(F + 127) / 128, 128, 0, s>>>(ctx->d_optode, F, N, ctx->d_sgV, ldf);
  ++ctx->launches;
  const unsigned gv = (unsigned)std::min<long long>((N * F + SG_T - 1) / SG_T, 152 * 16);
  const dim3 gd(nblk, F);
  for (int j = 0; j < m; ++j) {
    k_sg_op<<<gv, SG_T, 0, s>>>(nx, ny, nz, (float)base.sbar, bb, ctx->d_sgV + (size_t)j * N, ldf, F, w);
    ++ctx->launches;
    for (int pass = 0; pass < 2; ++pass) {  // full reorthogonalisation, twice
      k_sg_dots<<<gd, SG_T, 0, s>>>(ctx->d_sgV, ldf, j + 1, w, N, part, SG_MAXM);
      k_sg_sum<<<(F * (j + 1) + 127) / 128, 128, 0, s>>>(part, nblk, j + 1, F, SG_MAXM, c, cf,
                                                          pass == 0 ? ctx->d_sgA : nullptr, j);
      k_sg_sub<<<gv, SG_T, 0, s>>>(ctx->d_sgV, ldf, j + 1, cf, N, F, w);
      ctx->launches += 3;
    }
    if (j + 1 < m) {
      k_sg_dots<<<gd, SG_T, 0, s>>>(w, N, 1, w, N, part, SG_MAXM);
      k_sg_sum<<<(F + 127) / 128, 128, 0, s>>>(part, nblk, 1, F, SG_MAXM, c, cf, nullptr, 0);
      k_sg_beta<<<(F + 127) / 128, 128, 0, s>>>(c, F, j, ctx->d_sgA, ctx->d_sgB, ctx->d_sgMeff, scale);
      k_sg_next<<<gv, SG_T, 0, s>>>(w, scale, N, F, ctx->d_sgV, ldf, j + 1);
      ctx->launches += 4;
    }
    STRY(cudaGetLastError());
  }
  k_sg_face<<<dim3(F, 6), SG_T, 0, s>>>(ctx->d_sgV, ldf, m, nx, ny, nz, ctx->d_sgP);
  ++ctx->launches;
  STRY(cudaGetLastError());
  STRY(cudaStreamSynchronize(s));
  cleanup();
#undef STRY
  ctx->sg_m = m;
  ctx->sg_base[0] = base.sbar;
  for (int f = 0; f < 6; ++f) ctx->sg_base[1 + f] = base.bbar[f];
  return HYDOT_OK;
}

// x64 of a batch (nrhs = nlam * nf fields, rhs = l * nf + fl) = the Galerkin guesses
int shift_initial_guess(hydot_ctx* ctx, int lam0, int f_begin, int nf, int nrhs, void* x64, bool df) {
  const int m = ctx->sg_m;
  const long long N = ctx->N, ldf = (long long)m * N;
  const int nlam = nrhs / nf;
  SgBase base{};
  base.sbar = ctx->sg_base[0];
  for (int f = 0; f < 6; ++f) base.bbar[f] = ctx->sg_base[1 + f];
  cudaStream_t s = ctx->stream;
  k_sg_solve<<<nrhs, SG_MAXM, 0, s>>>(ctx->d_sgA, ctx->d_sgB, ctx->d_sgP, ctx->d_sgMeff, ctx->d_sgV, ldf, N,
                                      ctx->d_optode, ctx->d_coef, base, lam0, f_begin, nf, m, ctx->d_sgY);
  ++ctx->launches;
  const unsigned gx = (unsigned)std::min<long long>((N + SG_T - 1) / SG_T, std::max<long long>(1, 152 * 8 / nf));
  for (int l0 = 0; l0 < nlam; l0 += SG_LB) {
    if (df)
      k_sg_x0<df32><<<dim3(gx, nf), SG_T, 0, s>>>(ctx->d_sgV, ldf, N, ctx->d_sgY, nf, f_begin, l0,
                                                  std::min(SG_LB, nlam - l0), m, ctx->d_sgMeff, (df32*)x64);
    else
      k_sg_x0<double><<<dim3(gx, nf), SG_T, 0, s>>>(ctx->d_sgV, ldf, N, ctx->d_sgY, nf, f_begin, l0,
                                                    std::min(SG_LB, nlam - l0), m, ctx->d_sgMeff, (double*)x64);
    ++ctx->launches;
  }
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  return HYDOT_OK;
}

int shift_guess_fields_impl(hydot_ctx* ctx, int lam0, int nlam, void* phi_src, void* phi_det) {
  if (ctx->sg_m == 0) return fail(ctx, HYDOT_ERR_STATE, "no shift-invariant bases: call hydot_set_shift_guess first");
  if (lam0 < 0 || nlam < 1 || lam0 + nlam > ctx->n_lambda) return fail(ctx, HYDOT_ERR_ARG, "wavelength slice out of range");
  if (!phi_src || !phi_det) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  const int nf = ctx->n_src + ctx->n_det;
  if ((long long)nlam * nf > ctx->max_fields) return fail(ctx, HYDOT_ERR_ARG, "nlam exceeds max_lambda_per_call");
  double* x64 = (double*)ctx->d_x64;
  int rc = shift_initial_guess(ctx, lam0, 0, nf, nlam * nf, x64, false);
  if (rc) return rc;
  const long long tot = (long long)nlam * nf * ctx->N;
  const unsigned g = (unsigned)std::min<long long>((tot + 255) / 256, 152 * 32);
  if (ctx->precision == HYDOT_MIXED)
    k_sg_out<float><<<g, 256, 0, ctx->stream>>>(x64, ctx->d_coef, lam0, nlam, nf, 0, ctx->n_src, ctx->N,
                                                (float*)phi_src, (float*)phi_det);
  else
    k_sg_out<double><<<g, 256, 0, ctx->stream>>>(x64, ctx->d_coef, lam0, nlam, nf, 0, ctx->n_src, ctx->N,
                                                 (double*)phi_src, (double*)phi_det);
  ++ctx->launches;
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  return HYDOT_OK;
}

}  // namespace hydot
