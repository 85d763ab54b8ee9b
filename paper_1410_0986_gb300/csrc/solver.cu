// Batched field solves: matrix-free FV diffusion operator, Jacobi-preconditioned CG (COCG for
// the complex-symmetric frequency-domain operator) with iterative refinement: on the mixed paths FP32
// inner solves and a double-float iterate and residual, on the FP64 paths FP64 throughout.
//
// Each simultaneous field ("rhs") solves  Ahat x = e_cell  with Ahat = A_j / (D_j h) (the
// operator of eqn:discincident restated as finite volumes, see hydot.h); the field is
// phi = x / (D_j h). One refinement cycle:
//   K_theta  floor of the componentwise test from the partner optode cells (optional)
//   K_res    r64 = b - Ahat x64 to well beyond FP32 accuracy, ||r64||_2, the componentwise backward
//            error max_i |r64_i| / (|Ahat||x64| + |b| + theta)_i, and the inner right-hand side
//            r = r64 / scale in the inner precision with rho_0 = r^T D^-1 r  [per-tile partials]
//            (FP64 iterate and arithmetic for the FP64 paths; for the mixed paths, real and
//            complex, the iterate x64 is double-float and the residual uses FP32 error-free
//            transformations, as FP64 runs at ~1/64 of the FP32 rate on this GPU)
//   K_decide stop, or start a cycle                                        [one thread per rhs]
//   K_A/K_B  inner PCG/COCG on Ahat e = r (two kernels per iteration, see below)
//   K_fold   x64 += scale * e
// The inner iteration is split in two passes over memory because alpha needs the global
// p^T Ahat p before x and r can move:
//   K_A  p_new = D^-1 r + beta p_old (formed on the fly, also at the stencil neighbours),
//        gamma = p_new^T Ahat p_new;  writes p_new          (reads r, p_old; writes p_new)
//   K_B  alpha = rho / gamma; e += alpha p; r -= alpha Ahat p (Ahat p recomputed from p);
//        rho' = r^T D^-1 r, ||r||^2                         (reads e, r, p; writes e, r)
// Scalars are never stored: every block of a field sums the per-tile partials of the previous
// pass in the same fixed order, so all blocks agree bit for bit and the result is reproducible.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <cudaTypedefs.h>

#include "hydot_internal.cuh"
#include "tma.cuh"

namespace hydot {

namespace {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NTHREADS = TX * TY;
constexpr int NWARPS = NTHREADS / 32;
constexpr int MAX_INNER_PER_CYCLE = 4096;
constexpr int MAX_CYCLES = 64;
constexpr int POLL_GROUP = 8;

struct Geo {
  int nx, ny, nz;
  long long N;
  int ntx, nty, ntz, tz, ntiles;
};

// Per-field partial layout (doubles), with T = ntiles:
//   [0, 4T)   rho[parity][tile][re,im]
//   [4T, 6T)  rr[parity][tile]
//   [6T, 8T)  gamma[tile][re,im]
//   [8T, 10T) res[tile][rr64, omega]
__host__ __device__ inline size_t part_stride(int T) { return (size_t)10 * T; }

struct Batch {
  const LamCoef* coef;
  const int* optode;  // voxel of optode f (sources then detectors)
  int lam0, f_begin, nf, nrhs;
  int* status;
  int* iters;
  int* cycles;
  double* scale;
  double* next;
  double* rr0;
  double* theta;
  double* fin;
  double* part;
  int* counter;
  int* err;
  double tol_in2;
  int max_inner, max_iter;
  double tol, tol_cw, cw_floor;
  // inner solves may also stop once their residual, scaled back, is half the outer tolerance (an
  // FP64 inner recurrence tracks the true residual; with no componentwise target the outer test
  // then passes): a good initial guess then saves iterations instead of only shrinking the target
  int abs_inner;
  int n_src, n_det;
  // per-voxel increment of the scaled diagonal, h^2 dmu_a(x; lambda) / D(lambda), for the
  // wavelengths of the slice ([nlam][N]); null without an absorption perturbation
  const float* dsig_f;
  const double* dsig_d;
  // general sparse right-hand side (adjoint solves, Section 5's gradient by one extra solve per
  // source): b_rhs = sum_k w[rhs][k] e_(cell k) with the weights of each field normalised to unit
  // 2-norm (rhs_scale holds the norms, applied to the output); rhs_slot[x] is k for the cells of
  // the right-hand side, -1 elsewhere. Null for the one-hot optode right-hand sides.
  const int* rhs_slot;
  const double* rhs_w;
  const double* rhs_scale;
  int n_rhs_cells;
};

// Increment of the diagonal of field rhs at voxel id in precision T (real part only).
template <typename T>
__device__ __forceinline__ T dsig_at(const Batch& b, int rhs, long long id, long long N) {
  if constexpr (sizeof(typename Traits<T>::R) == 8) {
    return Traits<T>::make(b.dsig_d[(size_t)(rhs / b.nf) * N + id], 0.0);
  } else {
    return Traits<T>::make(b.dsig_f[(size_t)(rhs / b.nf) * N + id], 0.0);
  }
}

__device__ __forceinline__ int rhs_lambda(const Batch& b, int rhs) { return b.lam0 + rhs / b.nf; }

// Entry `id` of field rhs's right-hand side: 1 at the optode cell `src`, or the field's weight at
// the cells of a general right-hand side.
__device__ __forceinline__ double rhs_value(const Batch& b, int rhs, long long id, long long src) {
  if (b.rhs_slot) {
    const int k = b.rhs_slot[id];
    return k >= 0 ? b.rhs_w[(size_t)rhs * b.n_rhs_cells + k] : 0.0;
  }
  return id == src ? 1.0 : 0.0;
}
__device__ __forceinline__ long long rhs_source(const Batch& b, int rhs) {
  return (long long)b.optode[b.f_begin + rhs % b.nf];
}

// Diagonal of Ahat in precision R: 6 + sigma on interior cells; a cell on boundary face f adds
// bhat_f - 1 (one neighbour fewer, one boundary term more). The face set of a cell is a 6-bit
// mask, so interior cells (mask 0) do no arithmetic for it -- in the FP64 kernels that keeps
// the slow FP64 pipe for the residual itself.
template <typename R>
struct DiagT {
  R dre, dim;  // 6 + sigma
  R fa[6];     // bhat_f - 1
  __device__ void load(const LamCoef& c) {
    dre = (R)(6.0 + c.sigma_re);
    dim = (R)c.sigma_im;
#pragma unroll
    for (int f = 0; f < 6; ++f) fa[f] = (R)(c.bhat[f] - 1.0);
  }
  __device__ __forceinline__ R add(int m) const {
    R a = 0;
#pragma unroll
    for (int f = 0; f < 6; ++f)
      if (m & (1 << f)) a += fa[f];
    return a;
  }
};

__device__ __forceinline__ int face_mask(const Geo& g, int i, int j, int k) {
  return (i == 0) | ((i == g.nx - 1) << 1) | ((j == 0) << 2) | ((j == g.ny - 1) << 3) | ((k == 0) << 4) |
         ((k == g.nz - 1) << 5);
}

template <typename T, typename R>
__device__ __forceinline__ T diag_at(const DiagT<R>& d, int m) {
  return Traits<T>::make(m ? d.dre + d.add(m) : d.dre, d.dim);
}

// Biased binary exponent of |v| (0 for zero and subnormals), read from the bits: integer ops only.
__device__ __forceinline__ int bexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }
__device__ __forceinline__ int bexp(cpx<double> v) { return max(bexp(v.re), bexp(v.im)); }

template <typename T>
__device__ __forceinline__ T inv(T v) {
  if constexpr (Traits<T>::cplx) {
    using R = typename Traits<T>::R;
    R den = v.re * v.re + v.im * v.im;
    return T{v.re / den, -v.im / den};
  } else {
    return (T)1 / v;
  }
}
template <typename T>
__device__ __forceinline__ T scal(typename Traits<T>::R s, T v) {
  if constexpr (Traits<T>::cplx) return s * v; else return s * v;
}

// ---------------------------------------------------------------- block reductions
template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum NV per-thread values over the block (deterministic); result valid in thread 0.
template <int NV, typename R>
__device__ void block_sum(R (&v)[NV], double (&out)[NV], double* sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    R s = warp_sum(v[q]);
    if (lane == 0) sm[q * NWARPS + warp] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = 0.0;
      for (int w = 0; w < NWARPS; ++w) s += sm[q * NWARPS + w];
      out[q] = s;
    }
  }
  __syncthreads();
}

// Sum NV strided partial arrays over the tiles of one field; every thread gets the result.
// p points at the first value; element (q, t) is p[q*qstride + t*tstride]. One warp does the
// FP64 work (fixed lane assignment and shuffle tree: every block of a field gets the same bits).
template <int NV>
__device__ void tile_sum(const double* p, int qstride, int tstride, int ntiles, double (&out)[NV], double* sm) {
  if (threadIdx.x < 32) {
    double v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = 0.0;
    for (int t = threadIdx.x; t < ntiles; t += 32) {
#pragma unroll
      for (int q = 0; q < NV; ++q) v[q] += p[q * qstride + (size_t)t * tstride];
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double s = warp_sum(v[q]);
      if (threadIdx.x == 0) sm[64 + q] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) out[q] = sm[64 + q];
  __syncthreads();
}

struct TileCoord {
  int rhs, tile, i, j, k0, k1;
  bool in;
};
__device__ __forceinline__ TileCoord tile_coord(const Geo& g) {
  TileCoord c;
  c.rhs = blockIdx.x / g.ntiles;
  c.tile = blockIdx.x % g.ntiles;
  int tx = c.tile % g.ntx;
  int rem = c.tile / g.ntx;
  int ty = rem % g.nty;
  int tzi = rem / g.nty;
  c.i = tx * TX + (threadIdx.x % TX);
  c.j = ty * TY + (threadIdx.x / TX);
  c.k0 = tzi * g.tz;
  c.k1 = min(c.k0 + g.tz, g.nz);
  c.in = (c.i < g.nx) && (c.j < g.ny);
  return c;
}

__device__ __forceinline__ long long vidx(const Geo& g, int i, int j, int k) {
  return ((long long)k * g.ny + j) * g.nx + i;
}

// ---------------------------------------------------------------- FP64 residual
// One pass per refinement cycle over the fields that finished an inner solve:
//   r64 = b - Ahat x64 in FP64 (six adds and one fused multiply-add per cell on the FP64 pipe),
//   ||r64||^2, and a bound on the componentwise backward error
//     omega = max_i |r64_i| / (|Ahat||x|_i + |b_i| + theta)
//   from binary exponents in the integer pipes: |r_i| < 2^(e_r - 1022) and the denominator is
//   >= 2^(max(e_xc + 2, e_nbr, e_b, e_theta) - 1023) (|diagonal| >= 4), so 2^(e_r + 1 - max)
//   >= omega_i; the bound exceeds the true value by at most a factor ~30 (conservative).
// It also writes the next inner solve's right-hand side r = r64 / s in the inner precision,
// with s = ||r64|| of the previous cycle (known before this pass; the inner solve's tolerance is
// relative to its own start, so r need not have unit norm), and the partials of
// rho_0 = r^T D^-1 r and ||r||^2 that the first inner iteration needs.
template <typename T, typename X>
__global__ void __launch_bounds__(NTHREADS) k_residual(Geo g, Batch b, const X* __restrict__ x64, T* __restrict__ R) {
  __shared__ double sm[96];
  __shared__ int smi[NWARPS];
  TileCoord c = tile_coord(g);
  if (b.status[c.rhs] != RHS_FINISHED) return;
  using Rt = typename Traits<T>::R;
  const LamCoef& lc = b.coef[rhs_lambda(b, c.rhs)];
  DiagT<double> dg;
  dg.load(lc);
  DiagT<Rt> dgi;
  dgi.load(lc);
  const T idint = inv(diag_at<T>(dgi, 0));
  const long long src = rhs_source(b, c.rhs);
  const double pre = 1.0 / b.next[c.rhs];
  const int etheta = bexp(b.theta[c.rhs]);
  const X* x = x64 + (size_t)c.rhs * g.N;
  T* r = R + (size_t)c.rhs * g.N;
  double rr = 0.0;
  Rt acc[3] = {0, 0, 0};  // rho_0 re, im, ||r||^2
  int om_e = -4096;
  constexpr int cplx_extra = Traits<X>::cplx ? 1 : 0;
  if (c.in) {
    auto ld = [&](int k) { return x[vidx(g, c.i, c.j, k)]; };
    X zero = Traits<X>::zero();
    X xm = c.k0 > 0 ? ld(c.k0 - 1) : zero;
    X xc = ld(c.k0);
    for (int k = c.k0; k < c.k1; ++k) {
      X xp = (k + 1 < g.nz) ? ld(k + 1) : zero;
      X sn = xm + xp;
      int ed = max(max(bexp(xm), bexp(xp)), etheta);
      if (c.i > 0) { X v = x[vidx(g, c.i - 1, c.j, k)]; sn = sn + v; ed = max(ed, bexp(v)); }
      if (c.i < g.nx - 1) { X v = x[vidx(g, c.i + 1, c.j, k)]; sn = sn + v; ed = max(ed, bexp(v)); }
      if (c.j > 0) { X v = x[vidx(g, c.i, c.j - 1, k)]; sn = sn + v; ed = max(ed, bexp(v)); }
      if (c.j < g.ny - 1) { X v = x[vidx(g, c.i, c.j + 1, k)]; sn = sn + v; ed = max(ed, bexp(v)); }
      const int m = face_mask(g, c.i, c.j, k);
      long long id = vidx(g, c.i, c.j, k);
      X d = diag_at<X>(dg, m);
      if (b.dsig_d) d = d + dsig_at<X>(b, c.rhs, id, g.N);
      X ax = d * xc - sn;
      const double bv = rhs_value(b, c.rhs, id, src);
      X r64 = Traits<X>::make(bv, 0.0) - ax;
      rr += Traits<X>::abs2(r64);
      int ec = bexp(xc);
      ed = max(ed, ec ? ec + 2 : 0);
      if (bv != 0.0) ed = max(ed, bexp(bv));
      int er = bexp(r64);
      if (er) om_e = max(om_e, ed ? er + 1 + cplx_extra - ed : 4096);
      T rv = Traits<T>::from(Traits<X>::re(r64) * pre, Traits<X>::im(r64) * pre);
      r[id] = rv;
      T rz = rv * (rv * ((m || b.dsig_f) ? inv(diag_at<T>(dgi, m) + (b.dsig_f ? dsig_at<T>(b, c.rhs, id, g.N) : Traits<T>::zero()))
                                           : idint));
      acc[0] += Traits<T>::rre(rz);
      acc[1] += Traits<T>::rim(rz);
      acc[2] += Traits<T>::abs2(rv);
      xm = xc;
      xc = xp;
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s1 = warp_sum(rr);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) om_e = max(om_e, __shfl_down_sync(0xffffffffu, om_e, o));
  if (lane == 0) { sm[32 + warp] = s1; smi[warp] = om_e; }
  double out[3];
  block_sum<3, Rt>(acc, out, sm);  // (its barriers also publish sm[32..] and smi)
  if (threadIdx.x == 0) {
    double sr = 0.0;
    int mx = -4096;
    for (int w = 0; w < NWARPS; ++w) { sr += sm[32 + w]; mx = max(mx, smi[w]); }
    const int T_ = g.ntiles;
    double* pb = b.part + (size_t)c.rhs * part_stride(T_);
    pb[8 * T_ + 2 * c.tile] = sr;
    pb[8 * T_ + 2 * c.tile + 1] = (mx <= -4096) ? 0.0 : (mx >= 4096 ? INFINITY : ldexp(1.0, mx));
    pb[2 * c.tile] = out[0];          // rho parity 0
    pb[2 * c.tile + 1] = out[1];
    pb[4 * T_ + c.tile] = out[2];     // ||r||^2 parity 0
  }
}

// Stages a tile of the iterate with its one-cell halo, [nzl][TY + 2][TX + 2] elements of X, zeros
// outside the grid, into xs: thread t takes plane positions t and t + NTHREADS of every staged
// plane, and every load of the block is issued before any cell is summed.
template <typename X>
__device__ __forceinline__ void stage_halo_tile(const Geo& g, const TileCoord& c, const X* __restrict__ x, X* xs) {
  constexpr int SX = TX + 2, SY = TY + 2;
  const int i0 = c.i - (int)(threadIdx.x % TX), j0 = c.j - (int)(threadIdx.x / TX);
  const int nzl = c.k1 - c.k0 + 2;
  const long long plane = (long long)g.nx * g.ny;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int q = threadIdx.x + u * NTHREADS;
    if (q < SX * SY) {
      const int ii = i0 - 1 + q % SX, jj = j0 - 1 + q / SX;
      const bool inxy = ii >= 0 && ii < g.nx && jj >= 0 && jj < g.ny;
      const X* src_p = x + ((long long)(c.k0 - 1) * g.ny + jj) * g.nx + ii;
      for (int kk = 0; kk < nzl; ++kk) {
        const int kz = c.k0 - 1 + kk;
        xs[kk * SX * SY + q] = (inxy && kz >= 0 && kz < g.nz) ? src_p[kk * plane] : X{};
      }
    }
  }
}

// Block sums of the residual pass in FP32 (each partial needs only ~1e-7 relative accuracy; the
// FP64 pipe is slow on this GPU), one conversion per partial, written to the tile's slots:
// v = {||r64||^2, rho re, rho im, ||r||^2}; the per-field sums over tiles stay FP64.
__device__ __forceinline__ void residual_partials(const Geo& g, const Batch& b, const TileCoord& c, float (&v)[4],
                                                  int om_e, double* sm, int* smi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) om_e = max(om_e, __shfl_down_sync(0xffffffffu, om_e, o));
  float* smf = reinterpret_cast<float*>(sm);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) smf[q * NWARPS + warp] = v[q];
    smi[warp] = om_e;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float t4[4] = {0.f, 0.f, 0.f, 0.f};
    int mx = -4096;
    for (int w = 0; w < NWARPS; ++w) {
#pragma unroll
      for (int q = 0; q < 4; ++q) t4[q] += smf[q * NWARPS + w];
      mx = max(mx, smi[w]);
    }
    const int T_ = g.ntiles;
    double* pb = b.part + (size_t)c.rhs * part_stride(T_);
    pb[8 * T_ + 2 * c.tile] = (double)t4[0];
    pb[8 * T_ + 2 * c.tile + 1] = (mx <= -4096) ? 0.0 : (mx >= 4096 ? INFINITY : ldexp(1.0, mx));
    pb[2 * c.tile] = (double)t4[1];  // rho parity 0
    pb[2 * c.tile + 1] = (double)t4[2];
    pb[4 * T_ + c.tile] = (double)t4[3];  // ||r||^2 parity 0
  }
}

// The same pass for the mixed real path, whose iterate is double-float (df32). Per cell the
// residual r = b - (d x_c - sum of the six neighbours) is a short signed sum; it is accumulated as
// s + c: the high parts enter through TwoSum (exact), the low parts and the TwoSum errors through
// the FP32 compensation c (the compensated summation of Ogita, Rump & Oishi), and the diagonal
// product d x_c through the exact FMA product. The error of r is then ~n^2 2^-48 (|Ahat||x|)_i
// (n <= 9 terms), far below the componentwise target, with FP32 operations only. r is rounded to
// FP32 for the norm, the exponent bound and the inner right-hand side, which need no more.
// What does not change down a column is set up once per thread: the diagonal of its x and y faces
// (a double-float sum for the residual; in FP32, in the face order of diag_at, for the Jacobi
// weight of rho_0, with its reciprocal). The per-cell body is compiled once per kind of plane
// (interior, k = 0, k = nz - 1, both): the z faces belong to whole planes, the same plane for
// every thread of a block, so interior planes carry no face terms at all. GEN selects the body
// with a per-cell absorption shift or a general right-hand side; the common case (a unit point
// source, no shift) is compiled without either.
template <int ZF>
struct ZFace {
  static constexpr bool lo = (ZF & 1) != 0, hi = (ZF & 2) != 0;
};

template <bool GEN>
__global__ void __launch_bounds__(NTHREADS) k_residual_df(Geo g, Batch b, const LamCoefF* __restrict__ coef_f,
                                                          const df32* __restrict__ x64, float* __restrict__ R) {
  extern __shared__ __align__(16) unsigned char rsm_raw[];
  __shared__ double sm[96];
  __shared__ int smi[NWARPS];
  TileCoord c = tile_coord(g);
  if (b.status[c.rhs] != RHS_FINISHED) return;
  // coefficients from the FP32 table (no FP64 arithmetic in this kernel)
  const LamCoefF cf = coef_f[rhs_lambda(b, c.rhs)];
  const long long src = rhs_source(b, c.rhs);
  const float pre = 1.f / (float)b.next[c.rhs];
  const int etheta = bexp(b.theta[c.rhs]);
  const df32* x = x64 + (size_t)c.rhs * g.N;
  float* r = R + (size_t)c.rhs * g.N;
  // the tile with a one-cell halo, [tz + 2][TY + 2][TX + 2], zeros outside the grid
  df32* xs = reinterpret_cast<df32*>(rsm_raw);
  constexpr int SX = TX + 2, SY = TY + 2;
  stage_halo_tile(g, c, x, xs);
  __syncthreads();
  float rr = 0.f;
  float acc[3] = {0.f, 0.f, 0.f};  // rho_0, (unused), ||r||^2
  int om_e = -4096;
  // s + c += coefficient * v, the product exact up to the coefficient's and v's low parts
  auto add_prod = [](float& s, float& cc, df32 k, df32 v) {
    float p, e, t;
    two_prod(k.hi, v.hi, p, e);
    e = fmaf(k.hi, v.lo, fmaf(k.lo, v.hi, e));
    two_sum(s, p, s, t);
    cc += t + e;
  };
  if (c.in) {
    const int li = (int)(threadIdx.x % TX) + 1, lj = (int)(threadIdx.x / TX) + 1;
    const int mxy = face_mask(g, c.i, c.j, 0) & 15;  // the x and y faces of the column
    df32 dcol{cf.dint, cf.dint_lo};
    float axy = 0.f;
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (mxy & (1 << f)) {
        dcol = df_add(dcol, df32{cf.fa[f], cf.fa_lo[f]});
        axy += cf.fa[f];
      }
    const float wcol = mxy ? 1.f / (cf.dint + axy) : cf.idint;
    const long long plane = (long long)g.nx * g.ny;
    long long id = vidx(g, c.i, c.j, c.k0);
    const df32* xq = xs + (SY + lj) * SX + li;
    auto cell = [&](auto zf) {
      constexpr bool zlo = decltype(zf)::lo, zhi = decltype(zf)::hi;
      const df32 xc = xq[0];
      // A x = d x_c - sum of the neighbours, as s + cc (neighbours outside the grid are zero)
      float s, cc;
      two_prod(dcol.hi, xc.hi, s, cc);
      cc = fmaf(dcol.hi, xc.lo, fmaf(dcol.lo, xc.hi, cc));
      if constexpr (zlo) add_prod(s, cc, df32{cf.fa[4], cf.fa_lo[4]}, xc);
      if constexpr (zhi) add_prod(s, cc, df32{cf.fa[5], cf.fa_lo[5]}, xc);
      if constexpr (GEN)
        if (b.dsig_d) add_prod(s, cc, df_from(dsig_at<double>(b, c.rhs, id, g.N)), xc);
      // the denominator's exponent comes once from the largest of |d x_c| >= 4 |x_c| and the
      // neighbours' moduli
      float amax = 4.f * fabsf(xc.hi);
      auto sub_nb = [&](df32 v) {
        float t;
        two_sum(s, -v.hi, s, t);
        cc += t - v.lo;
        amax = fmaxf(amax, fabsf(v.hi));
      };
      sub_nb(xq[-SX * SY]);
      sub_nb(xq[SX * SY]);
      sub_nb(xq[-1]);
      sub_nb(xq[1]);
      sub_nb(xq[-SX]);
      sub_nb(xq[SX]);
      // r = b - A x
      float rh = -s, rl = -cc;
      int eb = 0;  // binary exponent of |b| at this cell (0: b is zero here)
      if (GEN && b.rhs_slot) {
        const double bv = rhs_value(b, c.rhs, id, src);
        if (bv != 0.0) {
          const df32 bd = df_from(bv);
          float t;
          two_sum(bd.hi, rh, rh, t);
          rl += t + bd.lo;
          eb = bexp(bv);
        }
      } else if (id == src) {
        float t;
        two_sum(1.f, rh, rh, t);
        rl += t;
        eb = 1023;
      }
      const float rf = rh + rl;
      rr = fmaf(rf, rf, rr);
      const int ed = max(max(etheta, bexp_f(amax)), eb);
      const int er = bexp_f(rf);
      if (er) om_e = max(om_e, ed ? er + 1 - ed : 4096);
      const float rv = rf * pre;
      r[id] = rv;
      // the Jacobi weight 1 / d_i: the column's, except on z-face planes and with a per-cell shift
      float dinv = wcol;
      if constexpr (zlo || zhi || GEN) {
        float a = axy;
        if constexpr (zlo) a += cf.fa[4];
        if constexpr (zhi) a += cf.fa[5];
        const int m = mxy | (zlo << 4) | (zhi << 5);
        const bool sh = GEN && b.dsig_f;
        if (m || sh) dinv = 1.f / ((m ? cf.dint + a : cf.dint) + (sh ? dsig_at<float>(b, c.rhs, id, g.N) : 0.f));
        else dinv = cf.idint;
      }
      acc[0] = fmaf(rv * dinv, rv, acc[0]);
      acc[2] = fmaf(rv, rv, acc[2]);
    };
    for (int k = c.k0; k < c.k1; ++k, id += plane, xq += SX * SY) {
      const int zf = (k == 0) | ((k == g.nz - 1) << 1);  // the same for the whole block
      if (zf == 0) cell(ZFace<0>{});
      else if (zf == 1) cell(ZFace<1>{});
      else if (zf == 2) cell(ZFace<2>{});
      else cell(ZFace<3>{});
    }
  }
  float v4[4] = {rr, acc[0], 0.f, acc[2]};
  residual_partials(g, b, c, v4, om_e, sm, smi);
}

// The same pass for complex fields with a double-float iterate (re and im each a df32). The
// operator is the real stencil plus one imaginary shift on the diagonal, so
//   Re(A x) = d x_re - sigma_im x_im - (neighbours of x_re),
//   Im(A x) = d x_im + sigma_im x_re - (neighbours of x_im),
// each accumulated as s + cc exactly as in k_residual_df (TwoSum for the high parts, FP32
// compensation for the rest, exact FMA products for the diagonal terms). The exponent bound of
// the componentwise backward error takes the larger part of each complex number and one more
// bit for |z| <= sqrt(2) max(|re|, |im|), as the FP64 kernel does.
// The diagonal and D^-1 of a column are set up once, and the per-cell body is compiled per kind
// of plane and with or without a per-cell shift (GEN), as in k_residual_df.
template <bool GEN>
__global__ void __launch_bounds__(NTHREADS) k_residual_cdf(Geo g, Batch b, const LamCoefF* __restrict__ coef_f,
                                                           const cdf32* __restrict__ x64, float2* __restrict__ R) {
  extern __shared__ __align__(16) unsigned char rsm_raw[];
  __shared__ double sm[96];
  __shared__ int smi[NWARPS];
  TileCoord c = tile_coord(g);
  if (b.status[c.rhs] != RHS_FINISHED) return;
  const LamCoefF cf = coef_f[rhs_lambda(b, c.rhs)];
  const df32 d0{cf.dint, cf.dint_lo};
  const df32 dsi{cf.dim, cf.dim_lo}, ndsi{-cf.dim, -cf.dim_lo};
  df32 dfa[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) dfa[f] = df32{cf.fa[f], cf.fa_lo[f]};
  const long long src = rhs_source(b, c.rhs);
  const float pre = 1.f / (float)b.next[c.rhs];
  const int etheta = bexp(b.theta[c.rhs]);
  const cdf32* x = x64 + (size_t)c.rhs * g.N;
  float2* r = R + (size_t)c.rhs * g.N;
  cdf32* xs = reinterpret_cast<cdf32*>(rsm_raw);
  constexpr int SX = TX + 2, SY = TY + 2;
  stage_halo_tile(g, c, x, xs);
  __syncthreads();
  float rr = 0.f;
  float acc[3] = {0.f, 0.f, 0.f};  // rho_0 re, im, ||r||^2
  int om_e = -4096;
  auto add_prod = [](float& s, float& cc, df32 k, df32 v) {
    float p, e, t;
    two_prod(k.hi, v.hi, p, e);
    e = fmaf(k.hi, v.lo, fmaf(k.lo, v.hi, e));
    two_sum(s, p, s, t);
    cc += t + e;
  };
  if (c.in) {
    const int li = (int)(threadIdx.x % TX) + 1, lj = (int)(threadIdx.x / TX) + 1;
    const int mxy = face_mask(g, c.i, c.j, 0) & 15;
    df32 dcol = d0;
    float dre_col = cf.dint;  // the real diagonal in FP32, faces added in order
#pragma unroll
    for (int f = 0; f < 4; ++f)
      if (mxy & (1 << f)) {
        dcol = df_add(dcol, dfa[f]);
        dre_col += cf.fa[f];
      }
    const float den_col = fmaf(dre_col, dre_col, cf.dim * cf.dim);
    const float2 dinv_col = make_float2(dre_col / den_col, -cf.dim / den_col);
    const long long plane = (long long)g.nx * g.ny;
    const long long col = vidx(g, c.i, c.j, 0);
    long long id = col + (long long)c.k0 * plane;
    const cdf32* xq = xs + (SY + lj) * SX + li;
    auto cell = [&](auto zf) {
      constexpr bool zlo = decltype(zf)::lo, zhi = decltype(zf)::hi;
      const cdf32 xc = xq[0];
      float sr, cr, si, ci;
      two_prod(dcol.hi, xc.re.hi, sr, cr);
      cr = fmaf(dcol.hi, xc.re.lo, fmaf(dcol.lo, xc.re.hi, cr));
      two_prod(dcol.hi, xc.im.hi, si, ci);
      ci = fmaf(dcol.hi, xc.im.lo, fmaf(dcol.lo, xc.im.hi, ci));
      if constexpr (zlo) {
        add_prod(sr, cr, dfa[4], xc.re);
        add_prod(si, ci, dfa[4], xc.im);
      }
      if constexpr (zhi) {
        add_prod(sr, cr, dfa[5], xc.re);
        add_prod(si, ci, dfa[5], xc.im);
      }
      if constexpr (GEN)
        if (b.dsig_d) {
          const df32 ds = df_from(dsig_at<double>(b, c.rhs, id, g.N));
          add_prod(sr, cr, ds, xc.re);
          add_prod(si, ci, ds, xc.im);
        }
      add_prod(sr, cr, ndsi, xc.im);
      add_prod(si, ci, dsi, xc.re);
      // |d x_c| >= 4 max(|re|, |im|) enters the denominator's exponent with the neighbours
      float amax = 4.f * fmaxf(fabsf(xc.re.hi), fabsf(xc.im.hi));
      auto sub_nb = [&](const cdf32& v) {
        float t;
        two_sum(sr, -v.re.hi, sr, t);
        cr += t - v.re.lo;
        two_sum(si, -v.im.hi, si, t);
        ci += t - v.im.lo;
        amax = fmaxf(amax, fmaxf(fabsf(v.re.hi), fabsf(v.im.hi)));
      };
      sub_nb(xq[-SX * SY]);
      sub_nb(xq[SX * SY]);
      sub_nb(xq[-1]);
      sub_nb(xq[1]);
      sub_nb(xq[-SX]);
      sub_nb(xq[SX]);
      float rh = -sr, rl = -cr;
      int ed = max(etheta, bexp_f(amax));
      if (id == src) {
        float t;
        two_sum(1.f, rh, rh, t);
        rl += t;
        ed = max(ed, 1023);
      }
      const float fr = rh + rl, fi = -si + -ci;
      rr = fmaf(fr, fr, fmaf(fi, fi, rr));
      const int er = max(bexp_f(fr), bexp_f(fi));
      if (er) om_e = max(om_e, ed ? er + 2 - ed : 4096);
      const float2 rv = make_float2(fr * pre, fi * pre);
      r[id] = rv;
      // D^-1 of the cell: the real diagonal (faces, absorption perturbation) plus i sigma_im
      float2 dinv = dinv_col;
      if constexpr (zlo || zhi || GEN) {
        float dre = dre_col;
        if constexpr (zlo) dre += cf.fa[4];
        if constexpr (zhi) dre += cf.fa[5];
        if (GEN && b.dsig_f) dre += dsig_at<float>(b, c.rhs, id, g.N);
        if (zlo || zhi || (GEN && b.dsig_f)) {
          const float den = fmaf(dre, dre, cf.dim * cf.dim);
          dinv = make_float2(dre / den, -cf.dim / den);
        }
      }
      // rho_0 = r^T D^-1 r (bilinear), ||r||^2
      const float2 zr = make_float2(fmaf(rv.x, dinv.x, -rv.y * dinv.y), fmaf(rv.x, dinv.y, rv.y * dinv.x));
      acc[0] = fmaf(rv.x, zr.x, fmaf(-rv.y, zr.y, acc[0]));
      acc[1] = fmaf(rv.x, zr.y, fmaf(rv.y, zr.x, acc[1]));
      acc[2] = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, acc[2]));
    };
    for (int k = c.k0; k < c.k1; ++k, id += plane, xq += SX * SY) {
      const int zf = (k == 0) | ((k == g.nz - 1) << 1);  // the same for the whole block
      if (zf == 0) cell(ZFace<0>{});
      else if (zf == 1) cell(ZFace<1>{});
      else if (zf == 2) cell(ZFace<2>{});
      else cell(ZFace<3>{});
    }
  }
  float v4[4] = {rr, acc[0], acc[1], acc[2]};
  residual_partials(g, b, c, v4, om_e, sm, smi);
}

// Floor of the componentwise test: theta = cw_floor * sigma * min |x| over the field's partner
// optode cells (detectors for a source field, sources for a detector field); sigma is the real
// shift and |x| the modulus for complex fields.
template <typename X>
__global__ void k_theta(Geo g, Batch b, const X* __restrict__ x64, const int* __restrict__ optode) {
  int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= b.nrhs) return;
  if (b.status[rhs] != RHS_FINISHED) return;
  const int f = b.f_begin + rhs % b.nf;
  const bool is_src = f < b.n_src;
  // a general right-hand side (adjoint field of source f) is weighed against its own source's field
  const int p0 = b.rhs_slot ? f : (is_src ? b.n_src : 0);
  const int np = b.rhs_slot ? 1 : (is_src ? b.n_det : b.n_src);
  double th = 0.0;
  if (b.cw_floor > 0.0 && np > 0) {
    const X* x = x64 + (size_t)rhs * g.N;
    double mn = INFINITY;
    for (int q = 0; q < np; ++q) {
      if constexpr (std::is_same<X, df32>::value) {
        mn = fmin(mn, fabs((double)x[optode[p0 + q]].hi));
      } else if constexpr (std::is_same<X, cdf32>::value) {
        const cdf32 v = x[optode[p0 + q]];
        mn = fmin(mn, hypot((double)v.re.hi, (double)v.im.hi));
      } else {
        mn = fmin(mn, sqrt(Traits<X>::abs2(x[optode[p0 + q]])));
      }
    }
    th = b.cw_floor * b.coef[rhs_lambda(b, rhs)].sigma_re * mn;
  }
  b.theta[rhs] = th;
}

__global__ void k_decide(Geo g, Batch b) {
  int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= b.nrhs) return;
  if (b.status[rhs] != RHS_FINISHED) return;
  const int T_ = g.ntiles;
  const double* pb = b.part + (size_t)rhs * part_stride(T_);
  double rr = 0.0, om = 0.0, rr0 = 0.0;
  for (int t = 0; t < T_; ++t) {
    rr += pb[8 * T_ + 2 * t];
    om = fmax(om, pb[8 * T_ + 2 * t + 1]);
    rr0 += pb[4 * T_ + t];
  }
  double res = sqrt(rr);  // ||b|| = 1 for a unit point source
  b.fin[2 * rhs] = res;
  b.fin[2 * rhs + 1] = om;
  bool conv = (res <= b.tol) && (b.tol_cw <= 0.0 || om <= b.tol_cw);
  if (conv || b.iters[rhs] >= b.max_iter || b.cycles[rhs] >= MAX_CYCLES || rr == 0.0) {
    b.status[rhs] = RHS_DONE;
  } else {
    b.status[rhs] = RHS_INNER;
    const double sc = b.next[rhs];
    b.scale[rhs] = sc;  // the inner right-hand side is r64 / scale: x += scale * e
    b.next[rhs] = res;
    // stop the inner solve at ||r||^2 <= tol_in2 * rr0, or (abs_inner) at scale * ||r|| <= tol / 2
    b.rr0[rhs] = b.abs_inner ? fmax(rr0, 0.25 * b.tol * b.tol / (sc * sc * b.tol_in2)) : rr0;
    b.cycles[rhs] += 1;
    atomicAdd(&b.counter[0], 1);
  }
}

// ---------------------------------------------------------------- inner K_A
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_dir(Geo g, Batch b, int it, const T* __restrict__ R,
                                                  const T* __restrict__ Pold, T* __restrict__ Pnew) {
  __shared__ double sm[96];
  __shared__ int s_status;
  TileCoord c = tile_coord(g);
  // the tile-0 block of this field may flip its status during this launch: read it once
  if (threadIdx.x == 0) s_status = b.status[c.rhs];
  __syncthreads();
  if (s_status != RHS_INNER) return;
  using Rt = typename Traits<T>::R;
  const int T_ = g.ntiles;
  double* pb = b.part + (size_t)c.rhs * part_stride(T_);
  const int par = it & 1;
  double cur[3];
  {
    double t2[2];
    tile_sum<2>(pb + 2 * T_ * par, 1, 2, T_, t2, sm);  // rho (re, im) of the current residual
    cur[0] = t2[0];
    cur[1] = t2[1];
    double t1[1];
    tile_sum<1>(pb + 4 * T_ + T_ * par, 0, 1, T_, t1, sm);
    cur[2] = t1[0];
  }
  // convergence of the inner solve (residual norm relative to the normalised start)
  if (cur[2] <= b.tol_in2 * b.rr0[c.rhs] || it >= b.max_inner || b.iters[c.rhs] >= b.max_iter || cur[2] == 0.0) {
    if (c.tile == 0 && threadIdx.x == 0) b.status[c.rhs] = RHS_FINISHED;
    return;
  }
  if (c.tile == 0 && threadIdx.x == 0) atomicAdd(&b.counter[1 + it], 1);
  T beta = Traits<T>::zero();
  if (it > 0) {
    double prev[2];
    tile_sum<2>(pb + 2 * T_ * (par ^ 1), 1, 2, T_, prev, sm);
    // beta = rho_cur / rho_prev (complex division in double, once per block)
    double den = prev[0] * prev[0] + prev[1] * prev[1];
    double br = (cur[0] * prev[0] + cur[1] * prev[1]) / den;
    double bi = (cur[1] * prev[0] - cur[0] * prev[1]) / den;
    beta = Traits<T>::from(br, bi);
  }
  const LamCoef& lc = b.coef[rhs_lambda(b, c.rhs)];
  DiagT<Rt> dg;
  dg.load(lc);
  const T* r = R + (size_t)c.rhs * g.N;
  const T* po = Pold + (size_t)c.rhs * g.N;
  T* pn = Pnew + (size_t)c.rhs * g.N;
  const T dint = diag_at<T>(dg, 0);
  const T idint = inv(dint);
  const bool first = (it == 0);
  Rt acc[2] = {0, 0};
  const bool het = b.dsig_f != nullptr;  // per-voxel absorption perturbation on the diagonal
  if (c.in) {
    auto P = [&](int ii, int jj, int kk) -> T {
      long long id = vidx(g, ii, jj, kk);
      const int m = face_mask(g, ii, jj, kk);
      T z = het ? r[id] * inv((m ? diag_at<T>(dg, m) : dint) + dsig_at<T>(b, c.rhs, id, g.N))
                : r[id] * (m ? inv(diag_at<T>(dg, m)) : idint);
      return first ? z : z + beta * po[id];
    };
    T zero = Traits<T>::zero();
    T pm = c.k0 > 0 ? P(c.i, c.j, c.k0 - 1) : zero;
    T pc = P(c.i, c.j, c.k0);
    for (int k = c.k0; k < c.k1; ++k) {
      T pp = (k + 1 < g.nz) ? P(c.i, c.j, k + 1) : zero;
      T s = pm + pp;
      if (c.i > 0) s = s + P(c.i - 1, c.j, k);
      if (c.i < g.nx - 1) s = s + P(c.i + 1, c.j, k);
      if (c.j > 0) s = s + P(c.i, c.j - 1, k);
      if (c.j < g.ny - 1) s = s + P(c.i, c.j + 1, k);
      const int m = face_mask(g, c.i, c.j, k);
      T dk = m ? diag_at<T>(dg, m) : dint;
      if (het) dk = dk + dsig_at<T>(b, c.rhs, vidx(g, c.i, c.j, k), g.N);
      T q = dk * pc - s;
      T pq = pc * q;
      acc[0] += Traits<T>::rre(pq);
      acc[1] += Traits<T>::rim(pq);
      pn[vidx(g, c.i, c.j, k)] = pc;
      pm = pc;
      pc = pp;
    }
  }
  double out[2];
  block_sum<2, Rt>(acc, out, sm);
  if (threadIdx.x == 0) {
    pb[6 * T_ + 2 * c.tile] = out[0];
    pb[6 * T_ + 2 * c.tile + 1] = out[1];
  }
}

// ---------------------------------------------------------------- inner K_B
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_update(Geo g, Batch b, int it, T* __restrict__ E, T* __restrict__ R,
                                                     const T* __restrict__ Pn) {
  __shared__ double sm[96];
  TileCoord c = tile_coord(g);
  if (b.status[c.rhs] != RHS_INNER) return;
  using Rt = typename Traits<T>::R;
  const int T_ = g.ntiles;
  double* pb = b.part + (size_t)c.rhs * part_stride(T_);
  const int par = it & 1;
  double rho[2], gam[2];
  tile_sum<2>(pb + 2 * T_ * par, 1, 2, T_, rho, sm);
  tile_sum<2>(pb + 6 * T_, 1, 2, T_, gam, sm);
  double den = gam[0] * gam[0] + gam[1] * gam[1];
  double ar = (rho[0] * gam[0] + rho[1] * gam[1]) / den;
  double ai = (rho[1] * gam[0] - rho[0] * gam[1]) / den;
  const T alpha = Traits<T>::from(ar, ai);
  const LamCoef& lc = b.coef[rhs_lambda(b, c.rhs)];
  DiagT<Rt> dg;
  dg.load(lc);
  T* e = E + (size_t)c.rhs * g.N;
  T* r = R + (size_t)c.rhs * g.N;
  const T* p = Pn + (size_t)c.rhs * g.N;
  const T dint = diag_at<T>(dg, 0);
  const T idint = inv(dint);
  const bool first = (it == 0);
  Rt acc[3] = {0, 0, 0};
  if (c.in) {
    auto ld = [&](int k) { return p[vidx(g, c.i, c.j, k)]; };
    T zero = Traits<T>::zero();
    T pm = c.k0 > 0 ? ld(c.k0 - 1) : zero;
    T pc = ld(c.k0);
    for (int k = c.k0; k < c.k1; ++k) {
      T pp = (k + 1 < g.nz) ? ld(k + 1) : zero;
      T s = pm + pp;
      if (c.i > 0) s = s + p[vidx(g, c.i - 1, c.j, k)];
      if (c.i < g.nx - 1) s = s + p[vidx(g, c.i + 1, c.j, k)];
      if (c.j > 0) s = s + p[vidx(g, c.i, c.j - 1, k)];
      if (c.j < g.ny - 1) s = s + p[vidx(g, c.i, c.j + 1, k)];
      const int m = face_mask(g, c.i, c.j, k);
      long long id = vidx(g, c.i, c.j, k);
      T d = m ? diag_at<T>(dg, m) : dint;
      const bool het = b.dsig_f != nullptr;
      if (het) d = d + dsig_at<T>(b, c.rhs, id, g.N);
      T q = d * pc - s;
      T ev = first ? alpha * pc : e[id] + alpha * pc;
      T rv = r[id] - alpha * q;
      e[id] = ev;
      r[id] = rv;
      T z = rv * ((m || het) ? inv(d) : idint);
      T rz = rv * z;
      acc[0] += Traits<T>::rre(rz);
      acc[1] += Traits<T>::rim(rz);
      acc[2] += Traits<T>::abs2(rv);
      pm = pc;
      pc = pp;
    }
  }
  double out[3];
  block_sum<3, Rt>(acc, out, sm);
  if (threadIdx.x == 0) {
    pb[2 * T_ * (par ^ 1) + 2 * c.tile] = out[0];
    pb[2 * T_ * (par ^ 1) + 2 * c.tile + 1] = out[1];
    pb[4 * T_ + T_ * (par ^ 1) + c.tile] = out[2];
    if (c.tile == 0) b.iters[c.rhs] += 1;
  }
}

// ---------------------------------------------------------------- inner passes with TMA slabs
// FP32 real fields whose row pitch is a multiple of 16 bytes (nx % 4 == 0), and complex64 fields
// (8-byte elements: nx even). Tiles are 32 x 8 cells in x-y; TMA copies bring planes of a tile plus
// its one-cell x-y halo (x rounded out to x0 - 4 so the x coordinate stays 16-byte aligned for
// either element size); cells outside the grid arrive as zeros, so the stencil
// adds its six neighbours without branches (the Robin/Dirichlet faces live in the diagonal).
// Every wait on an mbarrier is bounded: on timeout the block flags b.err, waits (bounded) for the
// copies it issued and returns. The partial sums of a block go to the slot of its first 8-plane
// tile and zeros to the others (the per-tile layout of the partials is shared with the generic
// kernels). Per-field scalars (convergence, alpha, beta) are formed once per block by one lane.
constexpr int TZT = 8;               // planes per partial-sum tile on this path
constexpr int BXT = 40, BYT = 10;    // x-y extent of a halo box

// The dynamic shared-memory block rounded up to 128 bytes. The rounding is added to the __shared__
// pointer itself (not done on an integer), so the compiler keeps the shared address space and the
// slab accesses stay 32-bit shared-memory operations.
template <typename E>
__device__ __forceinline__ E* align128(unsigned char* p) {
  return reinterpret_cast<E*>(p + ((128u - (smem_addr(p) & 127u)) & 127u));
}

__device__ __forceinline__ float diag_f(const LamCoefF& cf, int m) {
  float a = cf.dint;
#pragma unroll
  for (int f = 0; f < 6; ++f)
    if (m & (1 << f)) a += cf.fa[f];
  return a;
}

// Element arithmetic of the rolling passes: float for real fields, float2 (re, im) for complex64
// fields, whose COCG uses the unconjugated bilinear form (x^T y, not x^H y), so a "product" is
// the plain complex product and the only conjugate-free norm is |r|^2 for the stopping test.
__device__ __forceinline__ float e_add(float a, float b) { return a + b; }
__device__ __forceinline__ float2 e_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float e_sub(float a, float b) { return a - b; }
__device__ __forceinline__ float2 e_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float e_mul(float a, float b) { return a * b; }
__device__ __forceinline__ float2 e_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a b rounded on its own: never merged into a multiply-add (complex: the product as e_mul forms it)
__device__ __forceinline__ float e_mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float2 e_mul_rn(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float e_fma(float a, float b, float c) { return fmaf(a, b, c); }  // a b + c
__device__ __forceinline__ float2 e_fma(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, fmaf(-a.y, b.y, c.x)), fmaf(a.x, b.y, fmaf(a.y, b.x, c.y)));
}
__device__ __forceinline__ float e_neg(float a) { return -a; }
__device__ __forceinline__ float2 e_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float e_abs2_fma(float v, float acc) { return fmaf(v, v, acc); }  // |v|^2 + acc
__device__ __forceinline__ float e_abs2_fma(float2 v, float acc) { return fmaf(v.x, v.x, fmaf(v.y, v.y, acc)); }
__device__ __forceinline__ float e_re(float a) { return a; }
__device__ __forceinline__ float e_re(float2 a) { return a.x; }
__device__ __forceinline__ float e_im(float) { return 0.f; }
__device__ __forceinline__ float e_im(float2 a) { return a.y; }

// Quotient (a_re + i a_im) / (b_re + i b_im) of per-field FP64 sums, rounded to the element type.
template <typename E>
__device__ __forceinline__ E e_quot(double ar, double ai, double br, double bi) {
  if constexpr (std::is_same<E, float>::value) {
    return (float)(ar / br);
  } else {
    const double den = br * br + bi * bi;
    return make_float2((float)((ar * br + ai * bi) / den), (float)((ai * br - ar * bi) / den));
  }
}

// Pass 1 with a rolling window of planes. A block owns a (field, x-tile, y-tile, z-segment)
// column; r and p_old arrive by TMA in slabs of RP planes (box 40 x 10 x RP: the tile plus its
// one-cell x-y halo, x rounded out to x0-4 for the 16-byte rule; no z-halo), RS slab buffers.
// Per slab: (B) p_new = D^-1 r + beta p_old is formed once per cell of the tile and its x-y
// halo, in place over r; a barrier; (D) the stencil runs on the planes whose upper neighbour is
// now formed (the slab's planes shifted down by one, the first of them in the previous slab's
// buffer). The z-neighbours of a cell are the same thread's values of the adjacent planes, kept
// in registers. A slab buffer is refilled at the barrier after its last read, so RS - 2 slabs
// are in flight while a slab is processed. The diagonal and its inverse depend on the cell only
// through its face mask: each thread precomputes them for its column and its halo cell (four z
// cases: interior, bottom, top, both).
// E is float (real fields) or float2 (complex64 fields: the same passes in complex arithmetic,
// 8-byte elements in the slabs). RP (planes per slab) and RS (slab buffers) are template
// parameters; the variants compute the same values in the same order (bitwise identical results)
// and differ only in how much data is in flight per block and how many blocks fit on an SM,
// which the autotuner times.
constexpr int PLN = BXT * BYT;  // elements in one box plane (32 x 8 tiles)
template <typename E, int RP, int RS, int CY = 1>
constexpr size_t roll_smem() { return (size_t)RS * 2 * RP * (BXT * (TY * CY + 2)) * sizeof(E) + 128; }

__device__ __forceinline__ void col_diag(const LamCoefF& cf, int mxy, float (&d)[4], float (&di)[4]) {
#pragma unroll
  for (int zb = 0; zb < 4; ++zb) {
    const int m = mxy | ((zb & 1) << 4) | ((zb >> 1) << 5);
    d[zb] = m ? diag_f(cf, m) : cf.dint;
    di[zb] = m ? 1.f / d[zb] : cf.idint;
  }
}
// complex diagonal (6 + sigma + face terms) + i sigma_im and its inverse
__device__ __forceinline__ void col_diag(const LamCoefF& cf, int mxy, float2 (&d)[4], float2 (&di)[4]) {
#pragma unroll
  for (int zb = 0; zb < 4; ++zb) {
    const int m = mxy | ((zb & 1) << 4) | ((zb >> 1) << 5);
    const float re = m ? diag_f(cf, m) : cf.dint;
    d[zb] = make_float2(re, cf.dim);
    const float den = fmaf(re, re, cf.dim * cf.dim);
    di[zb] = make_float2(re / den, -cf.dim / den);
  }
}
// v[zb] with selects (a dynamic index would put the array in local memory)
template <typename E>
__device__ __forceinline__ E pick4(const E (&v)[4], int zb) {
  return zb == 0 ? v[0] : (zb == 1 ? v[1] : (zb == 2 ? v[2] : v[3]));
}

// Pass-1 prologue, run by one warp: the stopping test on ||r||^2 and beta = rho / rho_prev, from
// the per-tile partials in FP64 in a fixed order (every block of a field decides alike). Sets
// *s_go (1: iterate) and *s_beta in thread 0; the field's lead block marks a finished field.
template <typename E>
__device__ __forceinline__ void dir_scalars(const Batch& b, const double* pb, int T_, int it, int rhs, bool lead,
                                            int* s_go, E* s_beta) {
  constexpr bool CPLX = !std::is_same<E, float>::value;
  const int par = it & 1;
  const bool first = (it == 0);
  // rho of the current residual (re, im), ||r||^2, and rho of the previous one (re, im)
  double v0 = 0.0, v0i = 0.0, v1 = 0.0, v2 = 0.0, v2i = 0.0;
  for (int t = threadIdx.x; t < T_; t += 32) {
    v0 += pb[2 * T_ * par + 2 * t];
    v1 += pb[4 * T_ + T_ * par + t];
    if (!first) v2 += pb[2 * T_ * (par ^ 1) + 2 * t];
    if constexpr (CPLX) {
      v0i += pb[2 * T_ * par + 2 * t + 1];
      if (!first) v2i += pb[2 * T_ * (par ^ 1) + 2 * t + 1];
    }
  }
  v0 = warp_sum(v0);
  v1 = warp_sum(v1);
  v2 = warp_sum(v2);
  if constexpr (CPLX) {
    v0i = warp_sum(v0i);
    v2i = warp_sum(v2i);
  }
  if (threadIdx.x == 0) {
    int go = 0;
    E beta{};
    const bool done = v1 <= b.tol_in2 * b.rr0[rhs] || it >= b.max_inner || b.iters[rhs] >= b.max_iter || v1 == 0.0;
    if (done) {
      if (lead) b.status[rhs] = RHS_FINISHED;
    } else {
      go = 1;
      if (!first) beta = e_quot<E>(v0, v0i, v2, v2i);
      if (lead) atomicAdd(&b.counter[1 + it], 1);
    }
    *s_go = go;
    *s_beta = beta;
  }
}

template <typename E, int RP, int RS, int CY, int MINB>
__global__ void __launch_bounds__(NTHREADS, MINB) k_dir_roll(Geo g, Batch b, const int* __restrict__ it_dev, int k,
                                                             int seg,
                                                          const LamCoefF* __restrict__ coef_f,
                                                          const __grid_constant__ CUtensorMap mapR,
                                                          const __grid_constant__ CUtensorMap mapPold,
                                                          E* __restrict__ Pnew) {
  static_assert(RS >= 3, "a slab buffer is refilled two slabs after its own");
  constexpr bool CPLX = !std::is_same<E, float>::value;
  static_assert(CY == 1 || !CPLX, "complex fields use 32 x 8 tiles");
  constexpr int TYB = TY * CY;          // tile rows
  constexpr int PLB = BXT * (TYB + 2);  // elements in one box plane (tile plus a one-cell x-y ring)
  extern __shared__ unsigned char dsm[];
  E* slab = align128<E>(dsm);  // [RS][r -> p_new, p_old][RP planes]
  __shared__ uint64_t mbar[RS];
  __shared__ double sm[96];
  __shared__ E s_beta;
  __shared__ int s_go, s_st;
  constexpr uint32_t SLAB_BYTES = RP * PLB * sizeof(E);
  const int it = *it_dev + k;  // iteration index: group base on the device + offset in the group
  const int nty2 = (g.nty + CY - 1) / CY;
  const int ncol = g.ntx * nty2;
  const int nseg = (g.nz + seg - 1) / seg;
  const int rhs = blockIdx.x / (ncol * nseg);
  const int rem = blockIdx.x - rhs * ncol * nseg;
  const int zs = rem / ncol, col = rem - zs * ncol;
  const int cx = col % g.ntx, cy2 = col / g.ntx;
  const int x0 = cx * TX, y0 = cy2 * TYB;
  const int z0 = zs * seg, z1 = min(z0 + seg, g.nz);
  const bool lead = (col == 0 && zs == 0);
  const int T_ = g.ntiles;
  double* pb = b.part + (size_t)rhs * part_stride(T_);
  const bool first = (it == 0);
  const int np = z1 - z0 + 2;  // planes z0-1 .. z1 (t = plane - (z0 - 1))
  const int nslab = (np + RP - 1) / RP;
  const int nfirst = min(RS, nslab);
  const uint32_t tx_bytes = (first ? 1u : 2u) * SLAB_BYTES;
  auto issue = [&](int q) {
    E* dst = slab + (q % RS) * 2 * RP * PLB;
    mbar_expect_tx(&mbar[q % RS], tx_bytes);
    tma_load_4d(dst, &mapR, &mbar[q % RS], x0 - 4, y0 - 1, z0 - 1 + q * RP, rhs);
    if (!first) tma_load_4d(dst + RP * PLB, &mapPold, &mbar[q % RS], x0 - 4, y0 - 1, z0 - 1 + q * RP, rhs);
  };
  // A field still iterating gets its first slabs requested at once; the convergence test and
  // beta (FP64 sums of the per-tile partials) are formed while they are in flight. A field that
  // stops here still waits (bounded) for those copies before the block exits.
  if (threadIdx.x == 0) {
    const int st = b.status[rhs];
    s_st = st;
    if (st == RHS_INNER) {
      for (int q = 0; q < RS; ++q) mbar_init(&mbar[q], 1);
      mbar_fence_init();
      for (int q = 0; q < nfirst; ++q) issue(q);
    }
  }
  __syncthreads();
  if (s_st != RHS_INNER) return;
  if (threadIdx.x < 32) dir_scalars<E>(b, pb, T_, it, rhs, lead, &s_go, &s_beta);
  const LamCoefF cf = coef_f[rhs_lambda(b, rhs)];
  __syncthreads();
  if (!s_go) {
    if (threadIdx.x == 0)
      for (int q = 0; q < nfirst; ++q) mbar_wait_bounded(&mbar[q % RS], 0u);
    return;
  }
  const E beta = s_beta;

  // own cells (tx, ty + 8 c) and the halo cell of this thread
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int i = x0 + tx;
  bool in[CY];
  int ob[CY];
  E dd[CY][4], di[CY][4];
#pragma unroll
  for (int c = 0; c < CY; ++c) {
    const int j = y0 + ty + TY * c;
    in[c] = (i < g.nx) && (j < g.ny);
    ob[c] = (ty + TY * c + 1) * BXT + tx + 4;
    col_diag(cf, (i == 0) | ((i == g.nx - 1) << 1) | ((j == 0) << 2) | ((j == g.ny - 1) << 3), dd[c], di[c]);
  }
  // halo: the first 64 threads take the rows y0-1 and y0+TYB, the next 2 TYB the columns x0-1 and x0+32
  const int h = threadIdx.x;
  const bool has_halo = h < 2 * TX + 2 * TYB;
  int hb = 0;
  E hdi[4] = {};
  if (has_halo) {
    int hx, hy;
    if (h < 2 * TX) {
      hx = h % TX;
      hy = (h < TX) ? -1 : TYB;
    } else {
      hx = (h - 2 * TX < TYB) ? -1 : TX;
      hy = (h - 2 * TX) % TYB;
    }
    hb = (hy + 1) * BXT + hx + 4;
    const int gi = x0 + hx, gj = y0 + hy;
    E hd[4];
    col_diag(cf, (gi == 0) | ((gi == g.nx - 1) << 1) | ((gj == 0) << 2) | ((gj == g.ny - 1) << 3), hd, hdi);
  }
  const int plane_n = g.nx * g.ny;
  E* out = Pnew + (size_t)rhs * g.N + (size_t)(y0 + ty) * g.nx + i;
  const int row8 = TY * g.nx;  // offset of the cell eight rows further
  // own p_new of the previous slab's last two planes; gamma per 32 x 8 column (each column's sum
  // in the same order whatever CY is)
  E acc[CY], pm2[CY], pm1[CY];
#pragma unroll
  for (int c = 0; c < CY; ++c) acc[c] = pm2[c] = pm1[c] = E{};
  const E* prev = slab;  // previous slab's p_new planes
  for (int q = 0; q < nslab; ++q) {
    E* cur = slab + (q % RS) * 2 * RP * PLB;
    const bool ok = mbar_wait_bounded(&mbar[q % RS], (uint32_t)((q / RS) & 1));
    const int t0 = q * RP;
    const int a0 = z0 - 1 + t0;  // first plane formed from this slab
    E pv[CY][RP];
    // (B) p_new in place; slabs without a grid z-face take the interior diagonal. The product
    // D^-1 r is rounded on its own (never merged into a multiply-add), so that every variant rounds
    // alike.
    auto form = [&](auto edge) {
#pragma unroll
      for (int u = 0; u < RP; ++u) {
        int zb = 0;
        if constexpr (decltype(edge)::value) zb = (a0 + u == 0) | ((a0 + u == g.nz - 1) << 1);
        E* pl = cur + u * PLB;
#pragma unroll
        for (int c = 0; c < CY; ++c) {
          E v = e_mul_rn(pl[ob[c]], decltype(edge)::value ? pick4(di[c], zb) : di[c][0]);
          if (!first) v = e_fma(beta, pl[RP * PLB + ob[c]], v);
          pl[ob[c]] = v;
          pv[c][u] = v;
        }
        if (has_halo) {
          E hv = e_mul_rn(pl[hb], decltype(edge)::value ? pick4(hdi, zb) : hdi[0]);
          if (!first) hv = e_fma(beta, pl[RP * PLB + hb], hv);
          pl[hb] = hv;
        }
      }
    };
    if (a0 <= 0 || a0 + RP - 1 >= g.nz - 1) form(std::true_type{});
    else form(std::false_type{});
    // the in-place writes are ordered before the copy that later refills this buffer
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(ok)) {
      // a slab never arrived: flag it, wait (bounded) for the copies issued so far, return
      if (threadIdx.x == 0) {
        atomicExch(b.err, 1);
        const int last = min(max(RS - 1, q + RS - 3), nslab - 1);
        for (int u = q; u <= last; ++u) mbar_wait_bounded(&mbar[u % RS], (uint32_t)((u / RS) & 1));
      }
      return;
    }
    // every thread is past the stencils that read slab q - 2: refill its buffer
    if (threadIdx.x == 0 && q >= 2 && q - 2 + RS < nslab) issue(q - 2 + RS);
    // (D) stencils of the planes t0 - 1 .. t0 + RP - 2 (plane t0 - 1 lies in the previous slab)
    auto stencil = [&](auto edge) {
#pragma unroll
      for (int u = 0; u < RP; ++u) {
        const int zc = a0 - 1 + u;
        int zb = 0;
        if constexpr (decltype(edge)::value) {
          if (zc < z0 || zc >= z1) continue;
          zb = (zc == 0) | ((zc == g.nz - 1) << 1);
        }
        const E* pl = (u == 0) ? prev + (RP - 1) * PLB : cur + (u - 1) * PLB;
#pragma unroll
        for (int c = 0; c < CY; ++c) {
          if (!in[c]) continue;
          const int o = ob[c];
          const E d = decltype(edge)::value ? pick4(dd[c], zb) : dd[c][0];
          const E below = (u == 0) ? pm2[c] : (u == 1 ? pm1[c] : pv[c][u - 2]);
          const E centre = (u == 0) ? pm1[c] : pv[c][u - 1];
          const E sn = e_add(e_add(e_add(pl[o - 1], pl[o + 1]), e_add(pl[o - BXT], pl[o + BXT])),
                             e_add(below, pv[c][u]));
          if constexpr (CPLX) acc[c] = e_fma(centre, e_sub(e_mul(d, centre), sn), acc[c]);
          else acc[c] = e_fma(centre, e_fma(d, centre, e_neg(sn)), acc[c]);  // s = d p - sum: one rounding
          out[(ptrdiff_t)zc * plane_n + c * row8] = centre;
        }
      }
    };
    if (a0 - 1 < max(z0, 1) || a0 + RP - 2 > min(z1 - 1, g.nz - 2)) stencil(std::true_type{});
    else stencil(std::false_type{});
#pragma unroll
    for (int c = 0; c < CY; ++c) {
      pm2[c] = pv[c][RP - 2];
      pm1[c] = pv[c][RP - 1];
    }
    prev = cur;
  }
  float a2[2 * CY];
#pragma unroll
  for (int c = 0; c < CY; ++c) {
    a2[2 * c] = e_re(acc[c]);
    a2[2 * c + 1] = e_im(acc[c]);
  }
  double o2[2 * CY];
  if constexpr (CPLX) {
    block_sum<2 * CY, float>(a2, o2, sm);
  } else {
    float a1[CY];
#pragma unroll
    for (int c = 0; c < CY; ++c) a1[c] = a2[2 * c];
    double o1[CY];
    block_sum<CY, float>(a1, o1, sm);
#pragma unroll
    for (int c = 0; c < CY; ++c) {
      o2[2 * c] = o1[c];
      o2[2 * c + 1] = 0.0;
    }
  }
  // each 32 x 8 column's gamma goes to its partial slot of the segment's first 8-plane tile, zeros
  // to the segment's later tiles
  const int nsl = (z1 - z0 + g.tz - 1) / g.tz;
  const int ncols = min(CY, g.nty - cy2 * CY);
  const int ncol8 = g.ntx * g.nty;
  if (threadIdx.x < nsl * ncols) {
    const int ct = threadIdx.x / nsl, zt = threadIdx.x - ct * nsl;
    if (zt > 0) {
      const int slot = (cy2 * CY + ct) * g.ntx + cx + (z0 / g.tz + zt) * ncol8;
      pb[6 * T_ + 2 * slot] = 0.0;
      pb[6 * T_ + 2 * slot + 1] = 0.0;
    }
  }
  if (threadIdx.x == 0) {  // the sums (valid in thread 0) for the first tile of each column
#pragma unroll
    for (int c = 0; c < CY; ++c) {
      if (c >= ncols) break;
      const int slot = (cy2 * CY + c) * g.ntx + cx + (z0 / g.tz) * ncol8;
      pb[6 * T_ + 2 * slot] = o2[2 * c];
      pb[6 * T_ + 2 * slot + 1] = o2[2 * c + 1];
    }
  }
}

// Pass 1 on 64 x 8 CY tiles with two x-adjacent cells per thread (real fields). The same rolling
// slabs as k_dir_roll, with boxes 72 wide (x0 - 4 .. x0 + 67) and 8 CY + 2 rows, but a thread owns
// the cells (x0 + 2m, y) and (x0 + 2m + 1, y) for y = y0 + ty + 8 c: it forms both with one 8-byte
// shared load of r and of p_old and one 8-byte store, and in the stencil each cell of the pair is
// the other's x-neighbour (a register), so a pair takes two 4-byte loads (x - 1, x + 2) and two
// 8-byte loads (the rows above and below) where two single cells take eight 4-byte loads. The
// arithmetic per cell and the order of every sum are those of k_dir_roll: gamma per 32 x 8
// column is formed as its warp reduction forms it (the even and the odd cells of a row as two
// shuffle trees over 16 lanes, then their sum; the rows in order in FP64), so both kernels give
// the same bits. The diagonal of a cell on a grid z-face is formed when that plane comes up (it
// is rare); the cell's interior-z diagonal and its inverse stay in registers. Needs nx % 4 == 0
// (the TMA row pitch), so the pairs never straddle the grid's x-extent and 8-byte global stores
// are aligned.
constexpr int TXP = 64;  // tile width of the paired-cell pass 1
constexpr int BXP = 72;  // its box width: x0 - 4 .. x0 + 67
template <typename E, int RP, int RS, int CY>
constexpr size_t xp_smem() { return (size_t)RS * 2 * RP * (BXP * (TY * CY + 2)) * sizeof(E) + 128; }

// Diagonal of the cell with face mask m (bits: x low, x high, y low, y high, z low, z high) and its
// inverse, as col_diag forms them (real, and complex: the face terms on the real part, sigma_im on
// the imaginary part).
__device__ __forceinline__ void cell_diag(const LamCoefF& cf, int m, float& d, float& di) {
  d = m ? diag_f(cf, m) : cf.dint;
  di = m ? 1.f / d : cf.idint;
}
__device__ __forceinline__ void cell_diag(const LamCoefF& cf, int m, float2& d, float2& di) {
  const float re = m ? diag_f(cf, m) : cf.dint;
  d = make_float2(re, cf.dim);
  const float den = fmaf(re, re, cf.dim * cf.dim);
  di = make_float2(re / den, -cf.dim / den);
}
__device__ __forceinline__ int zmask(int zb) { return ((zb & 1) << 4) | ((zb >> 1) << 5); }

// Two x-adjacent cells of element type E, moved as one 8-byte (real) or 16-byte (complex) word.
template <typename E>
struct CellPair;
template <>
struct CellPair<float> {
  using T = float2;
  static __device__ __forceinline__ float a(float2 p) { return p.x; }
  static __device__ __forceinline__ float b(float2 p) { return p.y; }
  static __device__ __forceinline__ float2 make(float u, float v) { return make_float2(u, v); }
};
template <>
struct CellPair<float2> {
  using T = float4;
  static __device__ __forceinline__ float2 a(float4 p) { return make_float2(p.x, p.y); }
  static __device__ __forceinline__ float2 b(float4 p) { return make_float2(p.z, p.w); }
  static __device__ __forceinline__ float4 make(float2 u, float2 v) { return make_float4(u.x, u.y, v.x, v.y); }
};

template <typename E, int RP, int RS, int CY, int MINB>
__global__ void __launch_bounds__(NTHREADS, MINB) k_dir_xp(Geo g, Batch b, const int* __restrict__ it_dev, int k,
                                                           int seg, const LamCoefF* __restrict__ coef_f,
                                                           const __grid_constant__ CUtensorMap mapR,
                                                           const __grid_constant__ CUtensorMap mapPold,
                                                           E* __restrict__ Pnew) {
  static_assert(RS >= 3, "a slab buffer is refilled two slabs after its own");
  constexpr bool CPLX = !std::is_same<E, float>::value;
  constexpr int NV = CPLX ? 2 : 1;      // real and imaginary parts of gamma
  using CP = CellPair<E>;
  using PT = typename CP::T;
  constexpr int TYB = TY * CY;          // tile rows
  constexpr int PLB = BXP * (TYB + 2);  // elements in one box plane
  extern __shared__ unsigned char dsm[];
  E* slab = align128<E>(dsm);  // [RS][r -> p_new, p_old][RP planes]
  __shared__ uint64_t mbar[RS];
  __shared__ double sm[NV * 2 * CY * NWARPS];  // row sums per (part, 8-row group, 32-column half, row)
  __shared__ LamCoefF s_cf;
  __shared__ E s_beta;
  __shared__ int s_go, s_st;
  constexpr uint32_t SLAB_BYTES = RP * PLB * sizeof(E);
  const int it = *it_dev + k;
  const int ntxp = (g.nx + TXP - 1) / TXP;
  const int nty2 = (g.nty + CY - 1) / CY;
  const int ncol = ntxp * nty2;
  const int nseg = (g.nz + seg - 1) / seg;
  const int rhs = blockIdx.x / (ncol * nseg);
  const int rem = blockIdx.x - rhs * ncol * nseg;
  const int zs = rem / ncol, col = rem - zs * ncol;
  const int cx = col % ntxp, cy2 = col / ntxp;
  const int x0 = cx * TXP, y0 = cy2 * TYB;
  const int z0 = zs * seg, z1 = min(z0 + seg, g.nz);
  const bool lead = (col == 0 && zs == 0);
  const int T_ = g.ntiles;
  double* pb = b.part + (size_t)rhs * part_stride(T_);
  const bool first = (it == 0);
  const int np = z1 - z0 + 2;  // planes z0-1 .. z1
  const int nslab = (np + RP - 1) / RP;
  const int nfirst = min(RS, nslab);
  const uint32_t tx_bytes = (first ? 1u : 2u) * SLAB_BYTES;
  auto issue = [&](int q) {
    E* dst = slab + (q % RS) * 2 * RP * PLB;
    mbar_expect_tx(&mbar[q % RS], tx_bytes);
    tma_load_4d(dst, &mapR, &mbar[q % RS], x0 - 4, y0 - 1, z0 - 1 + q * RP, rhs);
    if (!first) tma_load_4d(dst + RP * PLB, &mapPold, &mbar[q % RS], x0 - 4, y0 - 1, z0 - 1 + q * RP, rhs);
  };
  if (threadIdx.x == 0) {
    const int st = b.status[rhs];
    s_st = st;
    if (st == RHS_INNER) {
      for (int q = 0; q < RS; ++q) mbar_init(&mbar[q], 1);
      mbar_fence_init();
      for (int q = 0; q < nfirst; ++q) issue(q);
    }
  }
  __syncthreads();
  if (s_st != RHS_INNER) return;
  if (threadIdx.x < 32) dir_scalars<E>(b, pb, T_, it, rhs, lead, &s_go, &s_beta);
  if (threadIdx.x == 32) s_cf = coef_f[rhs_lambda(b, rhs)];
  __syncthreads();
  if (!s_go) {
    if (threadIdx.x == 0)
      for (int q = 0; q < nfirst; ++q) mbar_wait_bounded(&mbar[q % RS], 0u);
    return;
  }
  const E beta = s_beta;
  const LamCoefF& cf = s_cf;

  // own pairs (x0 + 2m + {0, 1}, y0 + ty + 8 c): face masks, interior-z diagonals and inverses
  const int m = threadIdx.x % 32, ty = threadIdx.x / 32;
  const int i = x0 + 2 * m;  // even; i < nx implies i + 1 < nx (nx even on this path)
  bool in[CY];
  int ob[CY], msk[CY][2];
  E d0[CY][2], i0[CY][2];
#pragma unroll
  for (int c = 0; c < CY; ++c) {
    const int j = y0 + ty + TY * c;
    in[c] = (i < g.nx) && (j < g.ny);
    ob[c] = (ty + TY * c + 1) * BXP + 4 + 2 * m;
    const int my = ((j == 0) << 2) | ((j == g.ny - 1) << 3);
    msk[c][0] = (i == 0) | my;
    msk[c][1] = ((i + 1 == g.nx - 1) << 1) | my;
    cell_diag(cf, msk[c][0], d0[c][0], i0[c][0]);
    cell_diag(cf, msk[c][1], d0[c][1], i0[c][1]);
  }
  // halo: threads 0..63 form the pairs of the rows y0 - 1 and y0 + TYB, threads 64 .. 64 + 2 TYB - 1
  // the cells of the columns x0 - 1 and x0 + 64
  const int h = threadIdx.x;
  const bool hpair = h < 2 * 32;
  const bool hcol = !hpair && h < 2 * 32 + 2 * TYB;
  int hb = 0, hm0 = 0, hm1 = 0;
  E hi0{}, hi1{};
  if (hpair) {
    const int hx = 2 * (h % 32), hy = h < 32 ? -1 : TYB;
    hb = (hy + 1) * BXP + 4 + hx;
    const int gi = x0 + hx, gj = y0 + hy;
    const int my = ((gj == 0) << 2) | ((gj == g.ny - 1) << 3);
    hm0 = (gi == 0) | my;
    hm1 = ((gi + 1 == g.nx - 1) << 1) | my;
  } else if (hcol) {
    const int q = h - 2 * 32;
    const int hx = q < TYB ? -1 : TXP, hy = q % TYB;
    hb = (hy + 1) * BXP + 4 + hx;
    const int gi = x0 + hx, gj = y0 + hy;
    hm0 = (gi == 0) | ((gi == g.nx - 1) << 1) | ((gj == 0) << 2) | ((gj == g.ny - 1) << 3);
  }
  {
    E dd;
    cell_diag(cf, hm0, dd, hi0);
    cell_diag(cf, hm1, dd, hi1);
  }
  const int plane_n = g.nx * g.ny;
  E* out = Pnew + (size_t)rhs * g.N + (size_t)(y0 + ty) * g.nx + i;
  const int row8 = TY * g.nx;  // offset of the cell eight rows further
  E acc[CY][2];
  PT pm2[CY], pm1[CY];  // own p_new of the previous slab's last two planes
#pragma unroll
  for (int c = 0; c < CY; ++c) {
    acc[c][0] = acc[c][1] = E{};
    pm2[c] = pm1[c] = PT{};
  }
  const E* prev = slab;
  for (int q = 0; q < nslab; ++q) {
    E* cur = slab + (q % RS) * 2 * RP * PLB;
    const bool ok = mbar_wait_bounded(&mbar[q % RS], (uint32_t)((q / RS) & 1));
    const int a0 = z0 - 1 + q * RP;  // first plane formed from this slab
    PT pv[CY][RP];
    // (B) p_new = D^-1 r + beta p_old in place (the product rounded on its own, as k_dir_roll)
    auto form = [&](auto edge) {
#pragma unroll
      for (int u = 0; u < RP; ++u) {
        int zm = 0;
        if constexpr (decltype(edge)::value) zm = zmask((a0 + u == 0) | ((a0 + u == g.nz - 1) << 1));
        E* pl = cur + u * PLB;
#pragma unroll
        for (int c = 0; c < CY; ++c) {
          E ia = i0[c][0], ib = i0[c][1];
          if constexpr (decltype(edge)::value) {
            if (zm) {
              E dd;
              cell_diag(cf, msk[c][0] | zm, dd, ia);
              cell_diag(cf, msk[c][1] | zm, dd, ib);
            }
          }
          const PT rv = *reinterpret_cast<const PT*>(pl + ob[c]);
          E va = e_mul_rn(CP::a(rv), ia), vb = e_mul_rn(CP::b(rv), ib);
          if (!first) {
            const PT po = *reinterpret_cast<const PT*>(pl + RP * PLB + ob[c]);
            va = e_fma(beta, CP::a(po), va);
            vb = e_fma(beta, CP::b(po), vb);
          }
          const PT v = CP::make(va, vb);
          *reinterpret_cast<PT*>(pl + ob[c]) = v;
          pv[c][u] = v;
        }
        if (hpair || hcol) {
          E ia = hi0, ib = hi1;
          if constexpr (decltype(edge)::value) {
            if (zm) {
              E dd;
              cell_diag(cf, hm0 | zm, dd, ia);
              cell_diag(cf, hm1 | zm, dd, ib);
            }
          }
          if (hpair) {
            const PT rv = *reinterpret_cast<const PT*>(pl + hb);
            E va = e_mul_rn(CP::a(rv), ia), vb = e_mul_rn(CP::b(rv), ib);
            if (!first) {
              const PT po = *reinterpret_cast<const PT*>(pl + RP * PLB + hb);
              va = e_fma(beta, CP::a(po), va);
              vb = e_fma(beta, CP::b(po), vb);
            }
            *reinterpret_cast<PT*>(pl + hb) = CP::make(va, vb);
          } else {
            E v = e_mul_rn(pl[hb], ia);
            if (!first) v = e_fma(beta, pl[RP * PLB + hb], v);
            pl[hb] = v;
          }
        }
      }
    };
    if (a0 <= 0 || a0 + RP - 1 >= g.nz - 1) form(std::true_type{});
    else form(std::false_type{});
    // the in-place writes are ordered before the copy that later refills this buffer
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) {
        atomicExch(b.err, 1);
        const int last = min(max(RS - 1, q + RS - 3), nslab - 1);
        for (int u = q; u <= last; ++u) mbar_wait_bounded(&mbar[u % RS], (uint32_t)((u / RS) & 1));
      }
      return;
    }
    if (threadIdx.x == 0 && q >= 2 && q - 2 + RS < nslab) issue(q - 2 + RS);
    // (D) stencils of the planes a0 - 1 .. a0 + RP - 2 (the first lies in the previous slab)
    auto stencil = [&](auto edge) {
#pragma unroll
      for (int u = 0; u < RP; ++u) {
        const int zc = a0 - 1 + u;
        int zm = 0;
        if constexpr (decltype(edge)::value) {
          if (zc < z0 || zc >= z1) continue;
          zm = zmask((zc == 0) | ((zc == g.nz - 1) << 1));
        }
        const E* pl = (u == 0) ? prev + (RP - 1) * PLB : cur + (u - 1) * PLB;
#pragma unroll
        for (int c = 0; c < CY; ++c) {
          if (!in[c]) continue;
          const int o = ob[c];
          E da = d0[c][0], db = d0[c][1];
          if constexpr (decltype(edge)::value) {
            if (zm) {
              E dummy;
              cell_diag(cf, msk[c][0] | zm, da, dummy);
              cell_diag(cf, msk[c][1] | zm, db, dummy);
            }
          }
          const PT below = (u == 0) ? pm2[c] : (u == 1 ? pm1[c] : pv[c][u - 2]);
          const PT centre = (u == 0) ? pm1[c] : pv[c][u - 1];
          const PT above = pv[c][u];
          const PT ylo = *reinterpret_cast<const PT*>(pl + o - BXP);
          const PT yhi = *reinterpret_cast<const PT*>(pl + o + BXP);
          const E ca = CP::a(centre), cb = CP::b(centre);
          const E sa = e_add(e_add(e_add(pl[o - 1], cb), e_add(CP::a(ylo), CP::a(yhi))),
                             e_add(CP::a(below), CP::a(above)));
          const E sb = e_add(e_add(e_add(ca, pl[o + 2]), e_add(CP::b(ylo), CP::b(yhi))),
                             e_add(CP::b(below), CP::b(above)));
          if constexpr (CPLX) {
            acc[c][0] = e_fma(ca, e_sub(e_mul(da, ca), sa), acc[c][0]);
            acc[c][1] = e_fma(cb, e_sub(e_mul(db, cb), sb), acc[c][1]);
          } else {
            acc[c][0] = e_fma(ca, e_fma(da, ca, e_neg(sa)), acc[c][0]);
            acc[c][1] = e_fma(cb, e_fma(db, cb, e_neg(sb)), acc[c][1]);
          }
          *reinterpret_cast<PT*>(out + (ptrdiff_t)zc * plane_n + c * row8) = centre;
        }
      }
    };
    if (a0 - 1 < max(z0, 1) || a0 + RP - 2 > min(z1 - 1, g.nz - 2)) stencil(std::true_type{});
    else stencil(std::false_type{});
#pragma unroll
    for (int c = 0; c < CY; ++c) {
      pm2[c] = pv[c][RP - 2];
      pm1[c] = pv[c][RP - 1];
    }
    prev = cur;
  }
  // gamma per 32 x 8 column (each part): each row's even and odd cells as shuffle trees over the
  // half-warp (the first four steps of k_dir_roll's lane tree), then even + odd (its last step); the
  // rows are summed in order in FP64 as block_sum does
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < CY; ++c)
#pragma unroll
    for (int pv2 = 0; pv2 < NV; ++pv2) {
      float ea = pv2 ? e_im(acc[c][0]) : e_re(acc[c][0]), oa = pv2 ? e_im(acc[c][1]) : e_re(acc[c][1]);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        ea += __shfl_down_sync(0xffffffffu, ea, o, 16);
        oa += __shfl_down_sync(0xffffffffu, oa, o, 16);
      }
      if ((lane & 15) == 0) sm[((pv2 * CY + c) * 2 + (lane >> 4)) * NWARPS + warp] = (double)(ea + oa);
    }
  __syncthreads();
  const int nsl = (z1 - z0 + g.tz - 1) / g.tz;
  const int nyc = min(CY, g.nty - cy2 * CY), nxc = min(2, g.ntx - 2 * cx);
  const int ncol8 = g.ntx * g.nty;
  // each 32 x 8 column's gamma goes to its partial slot of the segment's first 8-plane tile, zeros
  // to the segment's later tiles
  for (int idx = threadIdx.x; idx < nsl * 2 * CY; idx += NTHREADS) {
    const int qc = idx / nsl, zt = idx - qc * nsl;
    const int c = qc >> 1, hf = qc & 1;
    if (c < nyc && hf < nxc) {
      const int slot = (cy2 * CY + c) * g.ntx + 2 * cx + hf + (z0 / g.tz + zt) * ncol8;
      double vr = 0.0, vi = 0.0;
      if (zt == 0) {
        for (int w = 0; w < NWARPS; ++w) vr += sm[qc * NWARPS + w];
        if constexpr (CPLX)
          for (int w = 0; w < NWARPS; ++w) vi += sm[(CY * 2 + qc) * NWARPS + w];
      }
      pb[6 * T_ + 2 * slot] = vr;
      pb[6 * T_ + 2 * slot + 1] = vi;
    }
  }
}

// Pass 2 with the same rolling window: a slab holds RP planes of p (tile + x-y halo) and of e
// and r (tile only), all by TMA; the stencil of plane k runs once plane k+1 of p is resident.
// Threads write nothing to shared memory, so one barrier per slab only guards the refill.
template <typename E, int RP>
__host__ __device__ constexpr uint32_t upd_slab() {  // p | e | r
  return (uint32_t)((RP * PLN + 2 * RP * TX * TY) * sizeof(E));
}
template <typename E, int RP, int RS>
constexpr size_t upd_smem() { return (size_t)RS * upd_slab<E, RP>() + 128; }

template <typename E, int RP, int RS, int MINB>
__global__ void __launch_bounds__(NTHREADS, MINB) k_update_roll(Geo g, Batch b, const int* __restrict__ it_dev,
                                                                int k, int seg,
                                                             const LamCoefF* __restrict__ coef_f,
                                                             E* __restrict__ Eo, E* __restrict__ R,
                                                             const __grid_constant__ CUtensorMap mapP,
                                                             const __grid_constant__ CUtensorMap mapE,
                                                             const __grid_constant__ CUtensorMap mapR) {
  static_assert(RS >= 3, "a slab buffer is refilled two slabs after its own");
  constexpr bool CPLX = !std::is_same<E, float>::value;
  extern __shared__ unsigned char dsm[];
  unsigned char* slab = reinterpret_cast<unsigned char*>(align128<E>(dsm));  // [RS][p | e | r]
  __shared__ uint64_t mbar[RS];
  __shared__ double sm[96];
  __shared__ E s_alpha;
  __shared__ int s_st;
  constexpr uint32_t UP_P = RP * PLN * sizeof(E);      // p planes of a slab (bytes)
  constexpr uint32_t UP_V = RP * TX * TY * sizeof(E);  // e or r planes of a slab (bytes)
  constexpr uint32_t UP_SLAB = upd_slab<E, RP>();
  const int it = *it_dev + k;  // iteration index: group base on the device + offset in the group
  const int ncol = g.ntx * g.nty;
  const int nseg = (g.nz + seg - 1) / seg;
  const int rhs = blockIdx.x / (ncol * nseg);
  const int rem = blockIdx.x - rhs * ncol * nseg;
  const int zs = rem / ncol, col = rem - zs * ncol;
  const int x0 = (col % g.ntx) * TX, y0 = (col / g.ntx) * TY;
  const int z0 = zs * seg, z1 = min(z0 + seg, g.nz);
  const bool lead = (col == 0 && zs == 0);
  const int T_ = g.ntiles;
  double* pb = b.part + (size_t)rhs * part_stride(T_);
  const int par = it & 1;
  const bool first = (it == 0);
  const int np = z1 - z0 + 2;
  const int nslab = (np + RP - 1) / RP;
  const uint32_t tx_bytes = UP_P + (first ? 1u : 2u) * UP_V;
  auto issue = [&](int q) {
    unsigned char* dst = slab + (size_t)(q % RS) * UP_SLAB;
    const int zq = z0 - 1 + q * RP;
    mbar_expect_tx(&mbar[q % RS], tx_bytes);
    tma_load_4d(dst, &mapP, &mbar[q % RS], x0 - 4, y0 - 1, zq, rhs);
    if (!first) tma_load_4d(dst + UP_P, &mapE, &mbar[q % RS], x0, y0, zq, rhs);
    tma_load_4d(dst + UP_P + UP_V, &mapR, &mbar[q % RS], x0, y0, zq, rhs);
  };
  // a field still iterating (pass 1 ran for it) gets its first slabs requested at once; alpha is
  // formed from the partials while they are in flight
  if (threadIdx.x == 0) {
    const int st = b.status[rhs];
    s_st = st;
    if (st == RHS_INNER) {
      for (int q = 0; q < RS; ++q) mbar_init(&mbar[q], 1);
      mbar_fence_init();
      for (int q = 0; q < min(RS, nslab); ++q) issue(q);
    }
  }
  __syncthreads();
  if (s_st != RHS_INNER) return;
  if (threadIdx.x < 32) {
    // alpha = rho / gamma (complex for complex fields)
    double v0 = 0.0, v0i = 0.0, v1 = 0.0, v1i = 0.0;
    for (int t = threadIdx.x; t < T_; t += 32) {
      v0 += pb[2 * T_ * par + 2 * t];
      v1 += pb[6 * T_ + 2 * t];
      if constexpr (CPLX) {
        v0i += pb[2 * T_ * par + 2 * t + 1];
        v1i += pb[6 * T_ + 2 * t + 1];
      }
    }
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    if constexpr (CPLX) {
      v0i = warp_sum(v0i);
      v1i = warp_sum(v1i);
    }
    if (threadIdx.x == 0) s_alpha = e_quot<E>(v0, v0i, v1, v1i);
  }
  const LamCoefF cf = coef_f[rhs_lambda(b, rhs)];
  __syncthreads();
  const E alpha = s_alpha;
  const E nalpha = e_neg(alpha);

  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int i = x0 + tx, j = y0 + ty;
  const bool in = (i < g.nx) && (j < g.ny);
  const int ob = (ty + 1) * BXT + tx + 4;
  const int ov = threadIdx.x;  // (ty, tx) in an e / r plane
  E dd[4], di[4];
  col_diag(cf, (i == 0) | ((i == g.nx - 1) << 1) | ((j == 0) << 2) | ((j == g.ny - 1) << 3), dd, di);
  const int plane_n = g.nx * g.ny;
  const size_t base = (size_t)rhs * g.N + (size_t)j * g.nx + i;
  E acc0{}, pm2{}, pm1{};
  float acc1 = 0.f;
  const unsigned char* prev = slab;
  for (int q = 0; q < nslab; ++q) {
    const unsigned char* cur = slab + (size_t)(q % RS) * UP_SLAB;
    const bool ok = mbar_wait_bounded(&mbar[q % RS], (uint32_t)((q / RS) & 1));
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) {
        atomicExch(b.err, 1);
        const int last = min(max(RS - 1, q + RS - 3), nslab - 1);
        for (int u = q; u <= last; ++u) mbar_wait_bounded(&mbar[u % RS], (uint32_t)((u / RS) & 1));
      }
      return;
    }
    // every thread is past the stencils that read slab q - 2: refill its buffer
    if (threadIdx.x == 0 && q >= 2 && q - 2 + RS < nslab) issue(q - 2 + RS);
    const int a0 = z0 - 1 + q * RP;
    const E* cp = reinterpret_cast<const E*>(cur);
    E pv[RP];
#pragma unroll
    for (int u = 0; u < RP; ++u) pv[u] = cp[u * PLN + ob];
    auto stencil = [&](auto edge) {
      const size_t o0 = base + (ptrdiff_t)(a0 - 1) * plane_n;
#pragma unroll
      for (int u = 0; u < RP; ++u) {
        const int c = a0 - 1 + u;
        E d = dd[0], dinv = di[0];
        if constexpr (decltype(edge)::value) {
          if (c < z0 || c >= z1) continue;
          const int zc = (c == 0) | ((c == g.nz - 1) << 1);
          d = pick4(dd, zc);
          dinv = pick4(di, zc);
        }
        const unsigned char* sl = (u == 0) ? prev : cur;
        const int pu = (u == 0) ? RP - 1 : u - 1;
        const E* pl = reinterpret_cast<const E*>(sl) + pu * PLN;
        const E* ev = reinterpret_cast<const E*>(sl + UP_P) + pu * TX * TY;
        const E* rv = reinterpret_cast<const E*>(sl + UP_P + UP_V) + pu * TX * TY;
        const E below = (u == 0) ? pm2 : (u == 1 ? pm1 : pv[u - 2]);
        const E centre = (u == 0) ? pm1 : pv[u - 1];
        const E sn = e_add(e_add(e_add(pl[ob - 1], pl[ob + 1]), e_add(pl[ob - BXT], pl[ob + BXT])),
                           e_add(below, pv[u]));
        const E qv = e_sub(e_mul(d, centre), sn);
        const E en = first ? e_mul(alpha, centre) : e_fma(alpha, centre, ev[ov]);
        const E rn = e_fma(nalpha, qv, rv[ov]);
        const size_t id = o0 + (size_t)u * plane_n;
        Eo[id] = en;
        R[id] = rn;
        acc0 = e_fma(rn, e_mul(rn, dinv), acc0);
        acc1 = e_abs2_fma(rn, acc1);
      }
    };
    if (in) {
      if (a0 - 1 < max(z0, 1) || a0 + RP - 2 > min(z1 - 1, g.nz - 2)) stencil(std::true_type{});
      else stencil(std::false_type{});
    }
    pm2 = pv[RP - 2];
    pm1 = pv[RP - 1];
    prev = cur;
  }
  double outs[3] = {0.0, 0.0, 0.0};
  if constexpr (CPLX) {
    float accs[3] = {e_re(acc0), acc1, e_im(acc0)};
    block_sum<3, float>(accs, outs, sm);
  } else {
    float accs[2] = {e_re(acc0), acc1};
    double o2[2];
    block_sum<2, float>(accs, o2, sm);
    outs[0] = o2[0];
    outs[1] = o2[1];
  }
  const int nsl = (z1 - z0 + g.tz - 1) / g.tz;
  if (threadIdx.x < nsl) {
    const int slot = col + (z0 / g.tz + threadIdx.x) * ncol;
    const bool z = threadIdx.x == 0;
    pb[2 * T_ * (par ^ 1) + 2 * slot] = z ? outs[0] : 0.0;
    pb[2 * T_ * (par ^ 1) + 2 * slot + 1] = z ? outs[2] : 0.0;
    pb[4 * T_ + T_ * (par ^ 1) + slot] = z ? outs[1] : 0.0;
    if (z && lead) b.iters[rhs] += 1;
  }
}

// ---------------------------------------------------------------- single-sweep inner iteration
// One pass over memory per inner iteration: Jacobi-preconditioned CG in the form of Chronopoulos
// & Gear (1989), whose two inner products of an iteration, gamma = r^T u and delta = (Ahat u)^T u
// with u = D^-1 r, come from the same sweep, so that alpha and beta of the next iteration are
// known before it starts:
//   beta_k = gamma_k / gamma_(k-1),  alpha_k = gamma_k / (delta_k - beta_k gamma_k / alpha_(k-1))
//   (alpha_0 = gamma_0 / delta_0, beta_0 = 0), and then, in one sweep,
//   p_k = u_k + beta_k p_(k-1),  s_k = Ahat p_k,  e_(k+1) = e_k + alpha_k p_k,
//   r_(k+1) = r_k - alpha_k s_k,  u_(k+1) = D^-1 r_(k+1),  w_(k+1) = Ahat u_(k+1),
//   gamma_(k+1) = r_(k+1)^T u_(k+1),  delta_(k+1) = w_(k+1)^T u_(k+1),  ||r_(k+1)||^2.
// s_k is recomputed from p_k instead of carried by a recurrence, so the sweep reads r, p and e once
// and writes them once (6 words per cell: the least a CG iteration moves). Recomputing s on the
// tile and its one-cell ring and w on the tile needs p on a two-cell ring: a block's slabs are
// boxes of 40 x 12 cells (the 32 x 8 tile, two cells around it, x rounded out to x0 - 4 for the
// 16-byte rule) of r and p_(k-1), plus the tile's e, arriving by TMA. Per slab of RP planes:
//   (A) p_k on the tile and both rings, in place over p_(k-1);            barrier
//   (B) s, r_(k+1), u_(k+1) on the tile and the inner ring one plane behind (u in place over r);
//       e, p and r of the tile cells to global memory;                      barrier
//   (C) w = Ahat u and the inner products on the tile two planes behind.
// r is double-buffered (neighbouring blocks read r_k on their ring while this block writes
// r_(k+1)); p already is. A block of the first sweep of a cycle reads neither p nor e (both zero).
// The priming launch of a cycle (PRIME) computes only gamma_0, delta_0 and ||r_0||^2 from r_0.
// Per-field scalars: every block of a field forms the same gamma_k, delta_k from the per-tile
// partials in the same order; gamma_k and alpha_k of iteration k are kept per field (one block
// writes them) for iteration k + 1. Threads 0..91 form p on the outer ring, threads 172..255 run
// (A) and (B) on the inner ring as well; the z-neighbours of every column are registers.
constexpr int BX2 = 40;  // x extent of a box: x0 - 4 .. x0 + 35 (the 16-byte rule rounds x0 - 2 down)

// Tile shape of the single sweep: 32 x (8 CY) cells, one thread per column of 8-row groups (a thread
// owns the CY cells (tx, ty + 8 c)); boxes of the tile plus a two-cell ring, 40 x (8 CY + 4) cells.
template <int CY>
struct SweepShape {
  static constexpr int TYB = TY * CY;               // tile rows
  static constexpr int BYB = TYB + 4;               // box rows
  static constexpr int PLANE = BX2 * BYB;           // cells of one box plane
  static constexpr int TILE_PLANE = TX * TYB;       // cells of one tile plane
  static constexpr int RING2 = 2 * (TX + 4) + 2 * (TYB + 2);  // outer-ring cells (p only)
  static constexpr int RING1 = 2 * (TX + 2) + 2 * TYB;        // inner-ring cells (p, s, r, u)
  static_assert(RING2 <= NTHREADS - RING1, "the two rings go to disjoint threads");
};
template <int RP, int CY>
__host__ __device__ constexpr uint32_t sw_slab_bytes() {  // r | p | e
  return (uint32_t)((2 * RP * SweepShape<CY>::PLANE + RP * SweepShape<CY>::TILE_PLANE) * sizeof(float));
}
template <int RP, int RS, int CY>
constexpr size_t sw_smem() { return (size_t)RS * sw_slab_bytes<RP, CY>() + 128; }

// (hx, hy) of ring cell q, relative to the tile origin, for a tile of TX x tyb cells: ring 1 (one cell
// out) or ring 2 (two)
__device__ __forceinline__ void ring_cell(int ring, int q, int tyb, int& hx, int& hy) {
  const int w = TX + 2 * ring, h = tyb + 2 * ring;  // extent of the ring's outline
  if (q < 2 * w) {
    hx = q % w - ring;
    hy = (q < w) ? -ring : tyb - 1 + ring;
  } else {
    q -= 2 * w;
    const int hh = h - 2;
    hx = (q < hh) ? -ring : TX - 1 + ring;
    hy = q % hh - ring + 1;
  }
}

// Per-field scalars of the single-sweep iteration: [parity][field] {gamma, alpha}.
struct SweepScalars {
  double* s;  // [2][nrhs_max][2]
  int stride; // fields per parity
};

// Shared scalars and barriers of one block of the single-sweep iteration.
template <int RS>
struct SweepShared {
  uint64_t mbar[RS];
  double sm[96];
  float beta, alpha;
  int go, st;
};

// One work item of the single-sweep iteration: the (field, x-y column, z-segment) `item` at inner
// iteration `it` (or the cycle's priming pass). Run by all threads of a block; slab is the block's
// dynamic shared memory rounded to 128 bytes. Returns false when a TMA slab never arrived (the
// device error flag is then set and the copies issued so far have been waited for).
template <int RP, int RS, int CY, bool PRIME>
__device__ __forceinline__ bool sweep_item(const Geo& g, const Batch& b, const int it, const int item, const int seg,
                                           const LamCoefF* __restrict__ coef_f, const SweepScalars& sc,
                                           const CUtensorMap* mapR0, const CUtensorMap* mapR1,
                                           const CUtensorMap* mapP0, const CUtensorMap* mapP1,
                                           const CUtensorMap* mapE, float* __restrict__ R0, float* __restrict__ R1,
                                           float* __restrict__ P0, float* __restrict__ P1, float* __restrict__ Eo,
                                           float* slab, SweepShared<RS>& sh) {
  static_assert(RP >= 3 && RS >= 3, "stage C reads u one slab back; a buffer is refilled two slabs after its own");
  // Products that later sums take in are rounded on their own (__fmul_rn is never merged into a
  // multiply-add), so every slab shape, tile shape and launch form rounds alike: the same bits.
  using Sh = SweepShape<CY>;
  constexpr int PLB = Sh::PLANE, TPB = Sh::TILE_PLANE;
  constexpr int SLAB = 2 * RP * PLB + RP * TPB;  // floats per slab buffer
  uint64_t* mbar = sh.mbar;
  double* sm = sh.sm;
  const int nty2 = (g.nty + CY - 1) / CY;  // tile rows of this shape
  const int ncol = g.ntx * nty2;
  const int nseg = (g.nz + seg - 1) / seg;
  const int rhs = item / (ncol * nseg);
  const int rem = item - rhs * ncol * nseg;
  const int zs = rem / ncol, col = rem - zs * ncol;
  const int cx = col % g.ntx, cy2 = col / g.ntx;
  const int x0 = cx * TX, y0 = cy2 * Sh::TYB;
  const int z0 = zs * seg, z1 = min(z0 + seg, g.nz);
  const bool lead = (col == 0 && zs == 0);
  const int T_ = g.ntiles;
  double* pb = b.part + (size_t)rhs * part_stride(T_);
  const int par = it & 1;
  const bool first = PRIME || it == 0;
  const int np = z1 - z0 + 4;  // planes z0-2 .. z1+1 (t = plane - (z0 - 2))
  const int nslab = (np + RP - 1) / RP;
  const int nfirst = min(RS, nslab);
  const CUtensorMap* mr = par ? mapR1 : mapR0;
  const CUtensorMap* mp = par ? mapP0 : mapP1;  // p_(k-1) was written by iteration k-1 into P[k & 1 ^ 1]
  const uint32_t tx_bytes = first ? RP * PLB * 4u : (2u * RP * PLB + RP * TPB) * 4u;
  auto issue = [&](int q) {
    float* dst = slab + (q % RS) * SLAB;
    const int zq = z0 - 2 + q * RP;
    mbar_expect_tx(&mbar[q % RS], tx_bytes);
    tma_load_4d(dst, mr, &mbar[q % RS], x0 - 4, y0 - 2, zq, rhs);
    if (!first) {
      tma_load_4d(dst + RP * PLB, mp, &mbar[q % RS], x0 - 4, y0 - 2, zq, rhs);
      tma_load_4d(dst + 2 * RP * PLB, mapE, &mbar[q % RS], x0, y0, zq, rhs);
    }
  };
  __syncthreads();  // the previous item's threads are done with the barriers re-initialised below
  if (threadIdx.x == 0) {
    const int st = b.status[rhs];
    sh.st = st;
    if (st == RHS_INNER) {
      for (int q = 0; q < RS; ++q) mbar_init(&mbar[q], 1);
      mbar_fence_init();
      for (int q = 0; q < nfirst; ++q) issue(q);
    }
  }
  __syncthreads();
  if (sh.st != RHS_INNER) return true;
  if (!PRIME) {
    if (threadIdx.x < 32) {
      double vg = 0.0, vd = 0.0, vr = 0.0;
      for (int t = threadIdx.x; t < T_; t += 32) {
        vg += pb[T_ * par + t];
        vd += pb[2 * T_ + T_ * par + t];
        vr += pb[4 * T_ + T_ * par + t];
      }
      vg = warp_sum(vg);
      vd = warp_sum(vd);
      vr = warp_sum(vr);
      if (threadIdx.x == 0) {
        bool done = vr <= b.tol_in2 * b.rr0[rhs] || it >= b.max_inner || b.iters[rhs] >= b.max_iter || vr == 0.0;
        double alpha = 0.0, beta = 0.0;
        if (!done) {
          if (it == 0) {
            alpha = vg / vd;
          } else {
            const double* prev = sc.s + ((size_t)(par ^ 1) * sc.stride + rhs) * 2;
            beta = vg / prev[0];
            const double den = vd - beta * vg / prev[1];
            alpha = vg / den;
            done = !(den > 0.0);  // breakdown (p^T Ahat p not positive in rounding): end this inner solve
          }
          done = done || !(vd > 0.0) || !isfinite(alpha);
        }
        if (done) {
          if (lead) b.status[rhs] = RHS_FINISHED;
        } else if (lead) {
          double* cur = sc.s + ((size_t)par * sc.stride + rhs) * 2;
          cur[0] = vg;
          cur[1] = alpha;
          atomicAdd(&b.counter[1 + it], 1);
        }
        sh.go = done ? 0 : 1;
        sh.alpha = (float)alpha;
        sh.beta = (float)beta;
      }
    }
  } else if (threadIdx.x == 0) {
    sh.go = 1;
    sh.alpha = 0.f;
    sh.beta = 0.f;
  }
  const LamCoefF cf = coef_f[rhs_lambda(b, rhs)];
  __syncthreads();
  if (!sh.go) {
    if (threadIdx.x == 0)
      for (int q = 0; q < nfirst; ++q) mbar_wait_bounded(&mbar[q % RS], 0u);
    return true;
  }
  const float alpha = sh.alpha, beta = sh.beta;

  // own cells: column (tx, ty + 8 c) of the tile for c < CY
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int i = x0 + tx;
  bool in[CY];
  int ob[CY];
  float dd[CY][4], di[CY][4];
#pragma unroll
  for (int c = 0; c < CY; ++c) {
    const int j = y0 + ty + TY * c;
    in[c] = (i < g.nx) && (j < g.ny);
    ob[c] = (ty + TY * c + 2) * BX2 + tx + 4;
    col_diag(cf, (i == 0) | ((i == g.nx - 1) << 1) | ((j == 0) << 2) | ((j == g.ny - 1) << 3), dd[c], di[c]);
  }
  // ring cells: outer ring (p only) for the first threads, inner ring (p, s, r, u) for the last
  const bool has2 = threadIdx.x < Sh::RING2;
  const bool has1 = threadIdx.x >= NTHREADS - Sh::RING1;
  int h2b = 0, h1b = 0;
  bool h1in = false;
  float h2di[4] = {}, h1d[4] = {}, h1di[4] = {};
  if (has2) {
    int hx, hy;
    ring_cell(2, threadIdx.x, Sh::TYB, hx, hy);
    h2b = (hy + 2) * BX2 + hx + 4;
    const int gi = x0 + hx, gj = y0 + hy;
    float d4[4];
    col_diag(cf, (gi == 0) | ((gi == g.nx - 1) << 1) | ((gj == 0) << 2) | ((gj == g.ny - 1) << 3), d4, h2di);
  }
  if (has1) {
    int hx, hy;
    ring_cell(1, threadIdx.x - (NTHREADS - Sh::RING1), Sh::TYB, hx, hy);
    h1b = (hy + 2) * BX2 + hx + 4;
    const int gi = x0 + hx, gj = y0 + hy;
    h1in = gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny;
    col_diag(cf, (gi == 0) | ((gi == g.nx - 1) << 1) | ((gj == 0) << 2) | ((gj == g.ny - 1) << 3), h1d, h1di);
  }
  const int plane_n = g.nx * g.ny;
  // the column's cells in this field's part of e, r_(k+1) and p_k (offsets within a field fit 32 bits)
  const size_t fbase = (size_t)rhs * g.N + (size_t)(y0 + ty) * g.nx + i;
  float* const eo = Eo + fbase;
  float* const rn_out = (par ? R0 : R1) + fbase;  // r_(k+1)
  float* const pn_out = (par ? P1 : P0) + fbase;  // p_k (read back as p_(k-1) from the other buffer)
  const int row8 = TY * g.nx;                     // offset of the cell eight rows further
  // z-queues: p of the own cells and inner-ring cell (two planes back), u and r_(k+1) of the own cells
  float pq2[CY], pq1[CY], uq2[CY], uq1[CY], rq1[CY];
#pragma unroll
  for (int c = 0; c < CY; ++c) pq2[c] = pq1[c] = uq2[c] = uq1[c] = rq1[c] = 0.f;
  float hq2 = 0.f, hq1 = 0.f;
  // inner products per 32 x 8 column (each column's sums in the same order whatever CY is)
  float ag[CY], ad[CY], ar[CY];
#pragma unroll
  for (int c = 0; c < CY; ++c) ag[c] = ad[c] = ar[c] = 0.f;
  const float* prev = slab;
  // One slab: (A), barrier, (B), barrier, (C). EDGE: a slab whose planes touch a grid z-face or
  // lie outside the block's segment (per-plane checks, z-face diagonals); otherwise every plane of
  // (A), (B) and (C) is an interior plane of the segment and the diagonals are the column's
  // interior ones. Returns false when a TMA slab never arrived.
  auto run_slab = [&](int q, auto edge_t) -> bool {
    constexpr bool EDGE = decltype(edge_t)::value;
    float* cur = slab + (q % RS) * SLAB;
    // one lane per warp polls the slab's barrier; the warp's other lanes are ordered after it by
    // __syncwarp (the copy's writes are visible to every thread that synchronises with the observer)
    bool ok = true;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait_bounded(&mbar[q % RS], (uint32_t)((q / RS) & 1));
    ok = __shfl_sync(0xffffffffu, (int)ok, 0) != 0;
    __syncwarp();
    const int zA = z0 - 2 + q * RP;  // plane of (A)'s first slab plane
    auto zcase = [&](int zt) { return EDGE ? ((zt == 0) | ((zt == g.nz - 1) << 1)) : 0; };
    auto dsel = [&](const float (&v)[4], int zb) { return EDGE ? pick4(v, zb) : v[0]; };
    float pA[CY][RP], hA[RP];
#pragma unroll
    for (int u = 0; u < RP; ++u) {
      hA[u] = 0.f;
#pragma unroll
      for (int c = 0; c < CY; ++c) pA[c][u] = 0.f;
    }
    // (A) p_k = D^-1 r_k + beta p_(k-1) on the tile and both rings (zero outside the grid: r and
    // p arrive as zeros there)
    if (!PRIME) {
#pragma unroll
      for (int u = 0; u < RP; ++u) {
        const int zb = zcase(zA + u);
        float* rp = cur + u * PLB;
        float* pp = cur + RP * PLB + u * PLB;
#pragma unroll
        for (int c = 0; c < CY; ++c) {
          float v = __fmul_rn(rp[ob[c]], dsel(di[c], zb));
          if (!first) v = fmaf(beta, pp[ob[c]], v);
          pp[ob[c]] = v;
          pA[c][u] = v;
        }
        if (has2) {
          float hv = __fmul_rn(rp[h2b], dsel(h2di, zb));
          if (!first) hv = fmaf(beta, pp[h2b], hv);
          pp[h2b] = hv;
        }
        if (has1) {
          float hv = __fmul_rn(rp[h1b], dsel(h1di, zb));
          if (!first) hv = fmaf(beta, pp[h1b], hv);
          pp[h1b] = hv;
          hA[u] = hv;
        }
      }
    }
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) {
        atomicExch(b.err, 1);
        const int last = min(max(RS - 1, q + RS - 3), nslab - 1);
        for (int u = q; u <= last; ++u) mbar_wait_bounded(&mbar[u % RS], (uint32_t)((u / RS) & 1));
      }
      return false;
    }
    // every thread is past (C) of slab q - 1, the last reader of slab q - 2: refill its buffer
    if (threadIdx.x == 0 && q >= 2 && q - 2 + RS < nslab) issue(q - 2 + RS);
    // (B) planes zA - 1 .. zA + RP - 2 (the first in the previous slab's buffer)
    float uB[CY][RP], rB[CY][RP];
#pragma unroll
    for (int u = 0; u < RP; ++u) {
      const int zt = zA - 1 + u;
#pragma unroll
      for (int c = 0; c < CY; ++c) uB[c][u] = rB[c][u] = 0.f;
      if (EDGE && (zt < z0 - 1 || zt > z1)) continue;  // not needed by (C)
      const bool zin = !EDGE || (zt >= 0 && zt < g.nz);
      const int zb = zcase(zt);
      float* rpl = (u == 0) ? const_cast<float*>(prev) + (RP - 1) * PLB : cur + (u - 1) * PLB;
      const float* ppl = rpl + RP * PLB;
      if (PRIME) {
#pragma unroll
        for (int c = 0; c < CY; ++c) {
          const float rv = rpl[ob[c]];
          const float uv = (in[c] && zin) ? __fmul_rn(rv, dsel(di[c], zb)) : 0.f;
          rpl[ob[c]] = uv;
          uB[c][u] = uv;
          rB[c][u] = rv;
        }
        if (has1) rpl[h1b] = (h1in && zin) ? __fmul_rn(rpl[h1b], dsel(h1di, zb)) : 0.f;
        continue;
      }
      const bool wr = !EDGE || (zt >= z0 && zt < z1);
      const int off = zt * plane_n;
#pragma unroll
      for (int c = 0; c < CY; ++c) {
        const int o = ob[c];
        const float below = (u == 0) ? pq2[c] : (u == 1 ? pq1[c] : pA[c][u - 2]);
        const float centre = (u == 0) ? pq1[c] : pA[c][u - 1];
        const float sn = (ppl[o - 1] + ppl[o + 1]) + (ppl[o - BX2] + ppl[o + BX2]) + (below + pA[c][u]);
        const float s = fmaf(dsel(dd[c], zb), centre, -sn);
        const float rn = fmaf(-alpha, s, rpl[o]);
        const float uv = (in[c] && zin) ? __fmul_rn(rn, dsel(di[c], zb)) : 0.f;
        rpl[o] = uv;
        uB[c][u] = uv;
        rB[c][u] = rn;
        if (in[c] && wr) {
          const float* epl = (u == 0) ? prev + 2 * RP * PLB + (RP - 1) * TPB : cur + 2 * RP * PLB + (u - 1) * TPB;
          const int oc = off + c * row8;
          eo[oc] = first ? __fmul_rn(alpha, centre) : fmaf(alpha, centre, epl[threadIdx.x + c * NTHREADS]);
          pn_out[oc] = centre;
          rn_out[oc] = rn;
        }
      }
      if (has1) {
        const float below = (u == 0) ? hq2 : (u == 1 ? hq1 : hA[u - 2]);
        const float centre = (u == 0) ? hq1 : hA[u - 1];
        const float sn = (ppl[h1b - 1] + ppl[h1b + 1]) + (ppl[h1b - BX2] + ppl[h1b + BX2]) + (below + hA[u]);
        const float s = fmaf(dsel(h1d, zb), centre, -sn);
        const float rn = fmaf(-alpha, s, rpl[h1b]);
        rpl[h1b] = (h1in && zin) ? __fmul_rn(rn, dsel(h1di, zb)) : 0.f;
      }
    }
    // the in-place writes are ordered before the copies that later refill these buffers
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    // (C) planes zA - 2 .. zA + RP - 3: w = Ahat u and the inner products
#pragma unroll
    for (int u = 0; u < RP; ++u) {
      const int zt = zA - 2 + u;
      if (EDGE && (zt < z0 || zt >= z1)) continue;
      const int zb = zcase(zt);
      const float* upl = (u <= 1) ? prev + (RP - 2 + u) * PLB : cur + (u - 2) * PLB;
#pragma unroll
      for (int c = 0; c < CY; ++c) {
        if (!in[c]) continue;
        const int o = ob[c];
        const float below = (u == 0) ? uq2[c] : (u == 1 ? uq1[c] : uB[c][u - 2]);
        const float centre = (u == 0) ? uq1[c] : uB[c][u - 1];
        const float rn = (u == 0) ? rq1[c] : rB[c][u - 1];
        const float sn = (upl[o - 1] + upl[o + 1]) + (upl[o - BX2] + upl[o + BX2]) + (below + uB[c][u]);
        const float w = fmaf(dsel(dd[c], zb), centre, -sn);
        ag[c] = fmaf(rn, centre, ag[c]);
        ad[c] = fmaf(w, centre, ad[c]);
        ar[c] = fmaf(rn, rn, ar[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < CY; ++c) {
      pq2[c] = pA[c][RP - 2];
      pq1[c] = pA[c][RP - 1];
      uq2[c] = uB[c][RP - 2];
      uq1[c] = uB[c][RP - 1];
      rq1[c] = rB[c][RP - 1];
    }
    hq2 = hA[RP - 2];
    hq1 = hA[RP - 1];
    prev = cur;
    return true;
  };
  for (int q = 0; q < nslab; ++q) {
    const int zA = z0 - 2 + q * RP;
    // interior: (A)'s planes zA .. zA+RP-1, (B)'s zA-1 .. zA+RP-2 and (C)'s zA-2 .. zA+RP-3 all
    // inside the segment and away from the grid's z-faces
    const bool interior = zA - 2 >= max(z0, 1) && zA + RP - 1 <= min(z1 - 1, g.nz - 2);
    const bool ok = interior ? run_slab(q, std::false_type{}) : run_slab(q, std::true_type{});
    if (!ok) return false;
  }
  float a3[3 * CY];
#pragma unroll
  for (int c = 0; c < CY; ++c) {
    a3[3 * c] = ag[c];
    a3[3 * c + 1] = ad[c];
    a3[3 * c + 2] = ar[c];
  }
  double o3[3 * CY];
  block_sum<3 * CY, float>(a3, o3, sm);
  // each 32 x 8 column's sums go to its partial slot of the segment's first 8-plane tile, zeros to
  // the segment's later tiles (the per-tile layout the per-field sums read)
  const int npar = PRIME ? 0 : (par ^ 1);
  const int nsl = (z1 - z0 + g.tz - 1) / g.tz;
  const int ncols = min(CY, g.nty - cy2 * CY);
  const int ncol8 = g.ntx * g.nty;
  if (threadIdx.x < nsl * ncols) {  // zeros for the later tiles of each column
    const int ct = threadIdx.x / nsl, zt = threadIdx.x - ct * nsl;
    if (zt > 0) {
      const int slot = (cy2 * CY + ct) * g.ntx + cx + (z0 / g.tz + zt) * ncol8;
      pb[T_ * npar + slot] = 0.0;
      pb[2 * T_ + T_ * npar + slot] = 0.0;
      pb[4 * T_ + T_ * npar + slot] = 0.0;
    }
  }
  if (threadIdx.x == 0) {  // the sums (valid in thread 0) for the first tile of each column
#pragma unroll
    for (int c = 0; c < CY; ++c) {
      if (c >= ncols) break;
      const int slot = (cy2 * CY + c) * g.ntx + cx + (z0 / g.tz) * ncol8;
      pb[T_ * npar + slot] = o3[3 * c];
      pb[2 * T_ + T_ * npar + slot] = o3[3 * c + 1];
      pb[4 * T_ + T_ * npar + slot] = o3[3 * c + 2];
    }
    if (!PRIME && lead) b.iters[rhs] += 1;
  }
  return true;

}


template <int RP, int RS, int CY, int MINB, bool PRIME>
__global__ void __launch_bounds__(NTHREADS, MINB) k_cg_sweep(Geo g, Batch b, const int* __restrict__ it_dev, int k,
                                                             int seg, const LamCoefF* __restrict__ coef_f,
                                                             SweepScalars sc,
                                                             const __grid_constant__ CUtensorMap mapR0,
                                                             const __grid_constant__ CUtensorMap mapR1,
                                                             const __grid_constant__ CUtensorMap mapP0,
                                                             const __grid_constant__ CUtensorMap mapP1,
                                                             const __grid_constant__ CUtensorMap mapE,
                                                             float* __restrict__ R0, float* __restrict__ R1,
                                                             float* __restrict__ P0, float* __restrict__ P1,
                                                             float* __restrict__ Eo) {
  extern __shared__ unsigned char dsm[];
  __shared__ SweepShared<RS> sh;
  const int it = PRIME ? 0 : *it_dev + k;
  sweep_item<RP, RS, CY, PRIME>(g, b, it, blockIdx.x, seg, coef_f, sc, &mapR0, &mapR1, &mapP0, &mapP1, &mapE, R0,
                                R1, P0, P1, Eo, align128<float>(dsm), sh);
}

// Grid-wide barrier of the persistent iteration (its blocks are co-resident: cooperative launch).
// Arrivals count up; the last arrival resets the count and advances the generation the others
// poll. Every wait is bounded: a block that gives up raises the device error flag and returns false
// (the kernel then ends; blocks still waiting for it give up in turn), so no launch can hang.
struct GridSync {
  unsigned* count;
  unsigned* gen;
  uint32_t polls;  // bound on the polls of one wait (64 ns pauses between polls)
};

__device__ __forceinline__ bool grid_sync(const GridSync& gs, int* err) {
  __shared__ int s_ok;
  // this block's global writes (fields, partials, per-field scalars) are ordered before the
  // arrival, also for the TMA (async-proxy) reads of the next iteration
  asm volatile("fence.proxy.async;" ::: "memory");
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned g0 = *(volatile unsigned*)gs.gen;
    bool ok = true;
    if (atomicAdd(gs.count, 1u) == gridDim.x - 1) {
      *(volatile unsigned*)gs.count = 0u;
      __threadfence();
      atomicAdd(gs.gen, 1u);
    } else {
      uint32_t n = 0;
      while (*(volatile unsigned*)gs.gen == g0) {
        if (++n > gs.polls) {
          ok = false;
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    asm volatile("fence.proxy.async;" ::: "memory");
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Persistent form of one refinement cycle's inner solve (small batches, where per-iteration launch
// and polling latency matter): one cooperative launch of co-resident blocks runs the priming pass
// and then the single-sweep iterations, each block taking work items (field, column, segment)
// in turn, with a grid barrier after every pass. The iteration stops on the device once an
// iteration finds no field still iterating (per-field convergence as in the launched form) or at
// the per-cycle cap. Block 0 writes the number of iterations run to *it_out. A wait that gives up
// ends the launch with the device error flag set.
template <int RP, int RS, int MINB>
__global__ void __launch_bounds__(NTHREADS, MINB) k_cg_persist(Geo g, Batch b, int seg,
                                                               const LamCoefF* __restrict__ coef_f, SweepScalars sc,
                                                               const __grid_constant__ CUtensorMap mapR0,
                                                               const __grid_constant__ CUtensorMap mapR1,
                                                               const __grid_constant__ CUtensorMap mapP0,
                                                               const __grid_constant__ CUtensorMap mapP1,
                                                               const __grid_constant__ CUtensorMap mapE,
                                                               float* __restrict__ R0, float* __restrict__ R1,
                                                               float* __restrict__ P0, float* __restrict__ P1,
                                                               float* __restrict__ Eo, GridSync gs, int nitems,
                                                               int* __restrict__ it_out) {
  extern __shared__ unsigned char dsm[];
  __shared__ SweepShared<RS> sh;
  float* slab = align128<float>(dsm);
  for (int w = blockIdx.x; w < nitems; w += gridDim.x)
    if (!sweep_item<RP, RS, 1, true>(g, b, 0, w, seg, coef_f, sc, &mapR0, &mapR1, &mapP0, &mapP1, &mapE, R0, R1,
                                     P0, P1, Eo, slab, sh))
      return;
  if (!grid_sync(gs, b.err)) return;
  int it = 0;
  for (; it < b.max_inner; ++it) {
    for (int w = blockIdx.x; w < nitems; w += gridDim.x)
      if (!sweep_item<RP, RS, 1, false>(g, b, it, w, seg, coef_f, sc, &mapR0, &mapR1, &mapP0, &mapP1, &mapE, R0,
                                        R1, P0, P1, Eo, slab, sh))
        return;
    if (!grid_sync(gs, b.err)) return;
    if (*(volatile int*)&b.counter[1 + it] == 0) break;  // no field iterated: every one has finished
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *it_out = min(it + 1, b.max_inner);
}

// ---------------------------------------------------------------- fold, output
template <typename T, typename X>
__global__ void k_fold(Geo g, Batch b, X* __restrict__ x64, const T* __restrict__ E) {
  for (int rhs = blockIdx.y; rhs < b.nrhs; rhs += gridDim.y) {
    if (b.status[rhs] != RHS_FINISHED) continue;
    const double s = b.scale[rhs];
    X* x = x64 + (size_t)rhs * g.N;
    const T* e = E + (size_t)rhs * g.N;
    if constexpr (std::is_same<X, cdf32>::value) {
      // complex: both parts as in the real double-float update below
      const df32 sd = df_from(s);
      const cpx<float>* ec = reinterpret_cast<const cpx<float>*>(e);
      for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < g.N;
           v += (long long)gridDim.x * blockDim.x) {
        const cpx<float> ev = ec[v];
        cdf32 xv = x[v];
        float p, q;
        two_prod(sd.hi, ev.re, p, q);
        q = fmaf(sd.lo, ev.re, q);
        xv.re = df_add(xv.re, fast_two_sum(p, q));
        two_prod(sd.hi, ev.im, p, q);
        q = fmaf(sd.lo, ev.im, q);
        xv.im = df_add(xv.im, fast_two_sum(p, q));
        x[v] = xv;
      }
    } else if constexpr (std::is_same<X, df32>::value) {
      // x += s e with the product exact up to s's low part and the sum accurate (double-float);
      // four independent cells per thread and pass keep the dependent TwoSum chains overlapped
      const df32 sd = df_from(s);
      const long long step = (long long)gridDim.x * blockDim.x;
      auto upd = [&](long long v) {
        float p, q;
        two_prod(sd.hi, e[v], p, q);
        q = fmaf(sd.lo, e[v], q);
        x[v] = df_add(x[v], fast_two_sum(p, q));
      };
      long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
      for (; v + 3 * step < g.N; v += 4 * step) {
        float p[4], q[4];
        df32 xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float ev = e[v + u * step];
          xv[u] = x[v + u * step];
          two_prod(sd.hi, ev, p[u], q[u]);
          q[u] = fmaf(sd.lo, ev, q[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) x[v + u * step] = df_add(xv[u], fast_two_sum(p[u], q[u]));
      }
      for (; v < g.N; v += step) upd(v);
    } else {
      for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (long long)gridDim.x * blockDim.x) {
        T ev = e[v];
        x[v] = x[v] + Traits<X>::from(s * Traits<T>::re(ev), s * Traits<T>::im(ev));
      }
    }
  }
}

template <typename X, typename O>
__global__ void k_output(Geo g, Batch b, const X* __restrict__ x64, O* __restrict__ phi_src,
                         O* __restrict__ phi_det, int n_src, int n_det) {
  for (int rhs = blockIdx.y; rhs < b.nrhs; rhs += gridDim.y) {
    int a = rhs / b.nf;
    int f = b.f_begin + rhs % b.nf;
    const double sc = b.coef[b.lam0 + a].inv_Dh * (b.rhs_scale ? b.rhs_scale[rhs] : 1.0);
    O* out = (f < n_src) ? phi_src + ((size_t)a * n_src + f) * g.N : phi_det + ((size_t)a * n_det + (f - n_src)) * g.N;
    const X* x = x64 + (size_t)rhs * g.N;
    if constexpr (std::is_same<X, cdf32>::value) {
      const float scf = (float)sc;
      for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (long long)gridDim.x * blockDim.x) {
        const cdf32 xv = x[v];
        out[v] = O{(xv.re.hi + xv.re.lo) * scf, (xv.im.hi + xv.im.lo) * scf};
      }
    } else if constexpr (std::is_same<X, df32>::value) {
      const float scf = (float)sc;
      for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (long long)gridDim.x * blockDim.x) {
        const df32 xv = x[v];
        out[v] = (O)((xv.hi + xv.lo) * scf);
      }
    } else {
      for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (long long)gridDim.x * blockDim.x) {
        X xv = x[v];
        out[v] = Traits<O>::from(sc * Traits<X>::re(xv), sc * Traits<X>::im(xv));
      }
    }
  }
}

__global__ void k_reset(Batch b) {
  int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= b.nrhs) return;
  b.status[rhs] = RHS_FINISHED;
  b.iters[rhs] = 0;
  b.cycles[rhs] = 0;
  b.scale[rhs] = 1.0;
  b.next[rhs] = 1.0;
  b.theta[rhs] = 0.0;
}

Geo make_geo(const hydot_ctx* ctx) {
  Geo g;
  g.nx = ctx->nx;
  g.ny = ctx->ny;
  g.nz = ctx->nz;
  g.N = ctx->N;
  g.ntx = ctx->tiling.ntx;
  g.nty = ctx->tiling.nty;
  g.ntz = ctx->tiling.ntz;
  g.tz = ctx->tiling.tz;
  g.ntiles = ctx->tiling.ntiles;
  return g;
}

// ---------------------------------------------------------------- absorption perturbation
// dsig[l][x] = h^2 sum_c eps_c(lambda_(lam0+l)) dc_c(x) / D(lambda): the perturbation
// h^3 dmu_a(x) of the absorption term (the diffusion coefficient stays the background's, as in
// the Born model of eqn:lippschwin) in the scaled operator A / (D h).
__global__ void k_dsig(const double* __restrict__ dc, const double* __restrict__ eps, const LamCoef* __restrict__ coef,
                       int lam0, int nlam, int nc, long long N, double h2, double* __restrict__ out_d,
                       float* __restrict__ out_f) {
  const long long total = (long long)nlam * N;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const int l = (int)(q / N);
    const long long x = q - (long long)l * N;
    double dm = 0.0;
    for (int c = 0; c < nc; ++c) dm += eps[(size_t)(lam0 + l) * nc + c] * dc[(size_t)c * N + x];
    const double v = h2 * dm / coef[lam0 + l].D;
    out_d[q] = v;
    out_f[q] = (float)v;
  }
}

// ---------------------------------------------------------------- rolling-pass variants
// {planes per slab, slab buffers}; the autotuner picks one per context (they give identical bits).
// Complex64 slabs take twice the shared memory per plane, hence their own, shallower set; complex
// variants 0 and 3 share the 2 x 4 slabs and differ in pass 1's register budget (three or four
// blocks per SM), and variant 2 runs pass 1 on 64 x 8 tiles of paired cells (16-byte pairs).
struct RollVariant {
  int rp, rs;
  int cy = 1;       // cells per thread in y (tiles of 32 x 8 cy, or 64 x 8 cy with xp)
  bool xp = false;  // pass 1 on paired x-adjacent cells (k_dir_xp)
};
// Real fields, pass 1 on: 32 x 8 tiles (variant 0); 64 x 8 tiles, x-pairs (1); 32 x 16 tiles, two
// cells per thread (2); 64 x 16 tiles, two x-pairs per thread (3). Pass 2 runs on 32 x 8 tiles.
constexpr RollVariant ROLL_VARIANTS[HYDOT_ROLL_VARIANTS] = {{4, 4, 1}, {2, 6, 1, true}, {2, 6, 2}, {2, 4, 2, true}};
constexpr RollVariant ROLL_VARIANTS_C[HYDOT_ROLL_VARIANTS] = {{2, 4}, {2, 6}, {2, 3, 1, true}, {2, 4}};

__host__ __device__ constexpr int rp_index(int rp) { return rp == 2 ? 0 : (rp == 4 ? 1 : 2); }

// Single-sweep variants {planes per slab, slab buffers, cells per thread in y} (real FP32 fields);
// bitwise identical results (each 32 x 8 column's inner products are summed in the same order). The
// blocks-per-SM bounds are what their shared memory allows: 32 x 8 tiles {4,3} and {3,4} 58 KB (three
// blocks per SM); 32 x 16 tiles {3,3} 76 KB and {4,3} 101 KB (two).
constexpr RollVariant SWEEP_VARIANTS[HYDOT_ROLL_VARIANTS] = {{4, 3, 1}, {3, 4, 1}, {3, 3, 2}, {4, 3, 2}};
__host__ __device__ constexpr int sw_index(int rp) { return rp == 3 ? 0 : 1; }

template <int RP, int RS, int CY, int MB>
int sweep_attrs(hydot_ctx* ctx) {
  HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_cg_sweep<RP, RS, CY, MB, false>, sw_smem<RP, RS, CY>()));
  HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_cg_sweep<RP, RS, CY, MB, true>, sw_smem<RP, RS, CY>()));
  return HYDOT_OK;
}

// Work items of the single sweep: (field, 32 x 8CY column, z-segment).
unsigned sweep_items(const hydot_ctx* ctx, const Geo& g, const Batch& b, int cy) {
  return (unsigned)((long long)b.nrhs * g.ntx * ((g.nty + cy - 1) / cy) * ((g.nz + ctx->dir_seg - 1) / ctx->dir_seg));
}

// One single-sweep iteration (k_off: offset of the iteration in its group; the group's base index
// is on the device) or, with PRIME, the cycle's priming pass.
template <int RP, int RS, int CY, int MB, bool PRIME>
void sweep_launch(hydot_ctx* ctx, const Geo& g, const Batch& b, int k_off) {
  const int d = sw_index(RP);
  const SweepScalars sc{ctx->d_cgsc, ctx->max_fields};
  const CUtensorMap* mr = CY == 1 ? ctx->tm_r2[d] : ctx->tm_r4[d];
  const CUtensorMap* mp = CY == 1 ? ctx->tm_p2[d] : ctx->tm_p4[d];
  const CUtensorMap& me = CY == 1 ? ctx->tm_e2[d] : ctx->tm_e4[d];
  cudaEvent_t t0 = timer_begin(ctx);
  k_cg_sweep<RP, RS, CY, MB, PRIME><<<sweep_items(ctx, g, b, CY), NTHREADS, sw_smem<RP, RS, CY>(), ctx->stream>>>(
      g, b, ctx->d_it, k_off, ctx->dir_seg, ctx->d_coef_f, sc, mr[0], mr[1], mp[0], mp[1], me, (float*)ctx->d_r,
      (float*)ctx->d_r2, (float*)ctx->d_p[0], (float*)ctx->d_p[1], (float*)ctx->d_e);
  ++ctx->launches;
  timer_end(ctx, t0, PRIME ? HYDOT_KERNEL_PRIME : HYDOT_KERNEL_SWEEP, 0.0);
}

// The persistent kernel runs the {3 planes, 4 buffers} slabs (58 KB: three blocks per SM).
constexpr int PERSIST_RP = 3, PERSIST_RS = 4, PERSIST_MB = 3;
constexpr uint32_t GRID_WAIT_POLLS = 1u << 24;  // about a second of 64 ns pauses per grid barrier

int persist_setup(hydot_ctx* ctx) {
  auto kern = k_cg_persist<PERSIST_RP, PERSIST_RS, PERSIST_MB>;
  const size_t smem = sw_smem<PERSIST_RP, PERSIST_RS, 1>();
  HYDOT_CUDA_TRY(ctx, raise_smem_limit(kern, smem));
  int per_sm = 0, sms = 0, coop = 0;
  HYDOT_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NTHREADS, smem));
  HYDOT_CUDA_TRY(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  HYDOT_CUDA_TRY(ctx, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
  ctx->persist_blocks = coop ? per_sm * sms : 0;
  if (ctx->persist_blocks <= 0) ctx->persist.mode = 0;  // no co-resident launch possible: launched only
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_gsync, 2 * sizeof(unsigned)));
  HYDOT_CUDA_TRY(ctx, cudaMemset(ctx->d_gsync, 0, 2 * sizeof(unsigned)));
  return HYDOT_OK;
}

// One cooperative launch for the whole inner solve of a cycle; returns the iterations it ran in *iters.
int persist_launch(hydot_ctx* ctx, const Geo& g, const Batch& b, unsigned nitems, int* iters) {
  const int d = sw_index(PERSIST_RP);
  SweepScalars sc{ctx->d_cgsc, ctx->max_fields};
  GridSync gs{ctx->d_gsync, ctx->d_gsync + 1, GRID_WAIT_POLLS};
  int seg = ctx->dir_seg;
  int ni = (int)nitems;
  int* it_out = ctx->d_it;
  float* r0 = (float*)ctx->d_r;
  float* r1 = (float*)ctx->d_r2;
  float* p0 = (float*)ctx->d_p[0];
  float* p1 = (float*)ctx->d_p[1];
  float* e = (float*)ctx->d_e;
  Geo gg = g;
  Batch bb = b;
  const LamCoefF* cf = ctx->d_coef_f;
  void* args[] = {&gg, &bb, &seg, &cf, &sc, &ctx->tm_r2[d][0], &ctx->tm_r2[d][1], &ctx->tm_p2[d][0],
                  &ctx->tm_p2[d][1], &ctx->tm_e2[d], &r0, &r1, &p0, &p1, &e, &gs, &ni, &it_out};
  const unsigned grid = std::min<unsigned>(nitems, (unsigned)ctx->persist_blocks);
  HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_gsync, 0, 2 * sizeof(unsigned), ctx->stream));
  HYDOT_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((const void*)k_cg_persist<PERSIST_RP, PERSIST_RS, PERSIST_MB>,
                                                  dim3(grid), dim3(NTHREADS), args,
                                                  sw_smem<PERSIST_RP, PERSIST_RS, 1>(), ctx->stream));
  ++ctx->launches;
  HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(iters, ctx->d_it, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return HYDOT_OK;
}

// Mode of the next cycle's inner solve: the chosen one, else (tuning) the mode with fewer samples.
int persist_pick(const hydot_ctx* ctx) {
  if (ctx->persist.mode >= 0) return ctx->persist.mode;
  return ctx->persist.samples[1] < ctx->persist.samples[0] ? 1 : 0;
}
void persist_record(hydot_ctx* ctx, int mode, double ms, double cell_iters) {
  if (ctx->persist.mode >= 0 || cell_iters <= 0.0) return;
  ctx->persist.ms[mode] += ms;
  ctx->persist.cells[mode] += cell_iters;
  ctx->persist.samples[mode] += 1;
  if (ctx->persist.samples[0] >= 2 && ctx->persist.samples[1] >= 2)
    ctx->persist.mode = (ctx->persist.ms[1] / ctx->persist.cells[1] < ctx->persist.ms[0] / ctx->persist.cells[0]) ? 1 : 0;
}

template <bool PRIME>
void sweep_dispatch(hydot_ctx* ctx, int v, const Geo& g, const Batch& b, int k_off) {
  switch (v) {
    case 1: sweep_launch<3, 4, 1, 3, PRIME>(ctx, g, b, k_off); break;
    case 2: sweep_launch<3, 3, 2, 2, PRIME>(ctx, g, b, k_off); break;
    case 3: sweep_launch<4, 3, 2, 2, PRIME>(ctx, g, b, k_off); break;
    default: sweep_launch<4, 3, 1, 3, PRIME>(ctx, g, b, k_off); break;
  }
}

template <typename E, int RP, int RS, int CY, int MB1, int MB2, bool XP = false, int RS2 = RS>
int roll_attrs(hydot_ctx* ctx) {
  if constexpr (XP) {
    HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_dir_xp<E, RP, RS, CY, MB1>, xp_smem<E, RP, RS, CY>()));
  } else {
    HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_dir_roll<E, RP, RS, CY, MB1>, roll_smem<E, RP, RS, CY>()));
  }
  HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_update_roll<E, RP, RS2, MB2>, upd_smem<E, RP, RS2>()));
  return HYDOT_OK;
}

// One inner iteration (pass 1, pass 2) with variant <RP, RS, CY, XP>: pass 1 on tiles of 32 x 8 CY, or
// with XP 64 x 8 CY (its blocks cover the tile rows and columns of that size), pass 2 on 32 x 8
// tiles (nrb blocks) with RS2 slab buffers.
template <typename E, int RP, int RS, int CY, int MB1, int MB2, bool XP = false, int RS2 = RS>
void roll_iteration(hydot_ctx* ctx, const Geo& g, const Batch& b, int it, unsigned nrb, E* Ev, E* R, E* const* P) {
  const int k = rp_index(RP);
  const int seg = ctx->dir_seg;
  cudaStream_t s = ctx->stream;
  cudaEvent_t t0 = timer_begin(ctx);
  const int o = it % POLL_GROUP;  // groups start at multiples of POLL_GROUP (even): parity of it = parity of o
  if constexpr (XP) {
    const unsigned nrb1 = (unsigned)((long long)b.nrhs * ((g.nx + TXP - 1) / TXP) * ((g.nty + CY - 1) / CY) *
                                     ((g.nz + seg - 1) / seg));
    const int c = CY - 1;
    k_dir_xp<E, RP, RS, CY, MB1><<<nrb1, NTHREADS, xp_smem<E, RP, RS, CY>(), s>>>(
        g, b, ctx->d_it, o, seg, ctx->d_coef_f, ctx->tm_rx[c][k], ctx->tm_px[c][k][it & 1], P[(it + 1) & 1]);
  } else {
    const unsigned nrb1 = CY == 1 ? nrb : sweep_items(ctx, g, b, CY);
    const CUtensorMap& mr = CY == 1 ? ctx->tm_rh[k] : ctx->tm_rh2[k];
    const CUtensorMap& mp = CY == 1 ? ctx->tm_ph[k][it & 1] : ctx->tm_ph2[k][it & 1];
    k_dir_roll<E, RP, RS, CY, MB1><<<nrb1, NTHREADS, roll_smem<E, RP, RS, CY>(), s>>>(
        g, b, ctx->d_it, o, seg, ctx->d_coef_f, mr, mp, P[(it + 1) & 1]);
  }
  ++ctx->launches;
  timer_end(ctx, t0, HYDOT_KERNEL_DIR, 0.0);
  t0 = timer_begin(ctx);
  k_update_roll<E, RP, RS2, MB2><<<nrb, NTHREADS, upd_smem<E, RP, RS2>(), s>>>(
      g, b, ctx->d_it, o, seg, ctx->d_coef_f, Ev, R, ctx->tm_ph[k][(it + 1) & 1], ctx->tm_e[k], ctx->tm_rv[k]);
  ++ctx->launches;
  timer_end(ctx, t0, HYDOT_KERNEL_UPDATE, 0.0);
}

// The variants' template arguments follow ROLL_VARIANTS / ROLL_VARIANTS_C; the blocks-per-SM
// bounds are what their shared memory allows (228 KB per SM).
void roll_dispatch(hydot_ctx* ctx, int v, const Geo& g, const Batch& b, int it, unsigned nrb, void* Ev, void* R,
                   void* const* P) {
  if (ctx->use_sweep) {
    sweep_dispatch<false>(ctx, v, g, b, it % POLL_GROUP);
    return;
  }
  if (ctx->cplx) {
    float2* e = (float2*)Ev;
    float2* r = (float2*)R;
    float2* p[2] = {(float2*)P[0], (float2*)P[1]};
    switch (v) {
      case 1: roll_iteration<float2, 2, 6, 1, 2, 2>(ctx, g, b, it, nrb, e, r, p); break;
      case 2: roll_iteration<float2, 2, 3, 1, 3, 3, true, 4>(ctx, g, b, it, nrb, e, r, p); break;
      case 3: roll_iteration<float2, 2, 4, 1, 4, 3>(ctx, g, b, it, nrb, e, r, p); break;
      default: roll_iteration<float2, 2, 4, 1, 3, 3>(ctx, g, b, it, nrb, e, r, p); break;
    }
    return;
  }
  float* e = (float*)Ev;
  float* r = (float*)R;
  float* p[2] = {(float*)P[0], (float*)P[1]};
  switch (v) {
    case 1: roll_iteration<float, 2, 6, 1, 3, 4, true>(ctx, g, b, it, nrb, e, r, p); break;
    case 2: roll_iteration<float, 2, 6, 2, 3, 4>(ctx, g, b, it, nrb, e, r, p); break;
    case 3: roll_iteration<float, 2, 4, 2, 2, 4, true, 6>(ctx, g, b, it, nrb, e, r, p); break;
    default: roll_iteration<float, 4, 4, 1, 4, 3>(ctx, g, b, it, nrb, e, r, p); break;
  }
}

int roll_setup(hydot_ctx* ctx) {
  if (ctx->use_sweep) {
    int rc = sweep_attrs<4, 3, 1, 3>(ctx);
    if (!rc) rc = sweep_attrs<3, 4, 1, 3>(ctx);
    if (!rc) rc = sweep_attrs<3, 3, 2, 2>(ctx);
    if (!rc) rc = sweep_attrs<4, 3, 2, 2>(ctx);
    return rc;
  }
  if (ctx->cplx) {
    int rc = roll_attrs<float2, 2, 4, 1, 3, 3>(ctx);
    if (!rc) rc = roll_attrs<float2, 2, 6, 1, 2, 2>(ctx);
    if (!rc) rc = roll_attrs<float2, 2, 3, 1, 3, 3, true, 4>(ctx);
    if (!rc) rc = roll_attrs<float2, 2, 4, 1, 4, 3>(ctx);
    return rc;
  }
  int rc = roll_attrs<float, 4, 4, 1, 4, 3>(ctx);
  if (!rc) rc = roll_attrs<float, 2, 6, 1, 3, 4, true>(ctx);
  if (!rc) rc = roll_attrs<float, 2, 6, 2, 3, 4>(ctx);
  if (!rc) rc = roll_attrs<float, 2, 4, 2, 2, 4, true, 6>(ctx);
  return rc;
}

// Variant for the next group of inner iterations: the chosen one, else (tuning) the variant with
// the fewest timed groups so far.
int roll_pick(hydot_ctx* ctx) {
  if (ctx->tune.variant >= 0) return ctx->tune.variant;
  int best = 0;
  for (int v = 1; v < HYDOT_ROLL_VARIANTS; ++v)
    if (ctx->tune.samples[v] < ctx->tune.samples[best]) best = v;
  return best;
}

// Record a timed group; once every variant has TUNE_SAMPLES groups, keep the fastest per cell-iteration.
constexpr int TUNE_SAMPLES = 2;
void roll_record(hydot_ctx* ctx, int v, double ms, double cell_iters) {
  if (ctx->tune.variant >= 0 || cell_iters <= 0.0) return;
  ctx->tune.ms[v] += ms;
  ctx->tune.cells[v] += cell_iters;
  ctx->tune.samples[v] += 1;
  for (int q = 0; q < HYDOT_ROLL_VARIANTS; ++q)
    if (ctx->tune.samples[q] < TUNE_SAMPLES) return;
  int best = 0;
  for (int q = 1; q < HYDOT_ROLL_VARIANTS; ++q)
    if (ctx->tune.ms[q] / ctx->tune.cells[q] < ctx->tune.ms[best] / ctx->tune.cells[best]) best = q;
  ctx->tune.variant = best;
}

// Advances the device-resident iteration base by one group (the last node of a group).
__global__ void k_bump(int* v, int d) { *v += d; }

// One group of POLL_GROUP inner iterations of the rolling passes plus the base advance, captured
// once into a CUDA graph and replayed while the batch, the variant and the grid stay the same
// (the iteration index comes from the device, so every group of a cycle replays the same graph).
struct GraphKey {
  Batch b;
  Geo g;
  int variant, seg;
  unsigned nrb;
  const void *E, *R, *P0, *P1;
};

int inner_graph_launch(hydot_ctx* ctx, const Geo& g, const Batch& b, int variant, unsigned nrb, void* E, void* R,
                       void* const* P) {
  GraphKey key;
  std::memset(&key, 0, sizeof(key));
  key.b = b;
  key.g = g;
  key.variant = variant;
  key.seg = ctx->dir_seg;
  key.nrb = nrb;
  key.E = E;
  key.R = R;
  key.P0 = P[0];
  key.P1 = P[1];
  cudaStream_t s = ctx->stream;
  const bool same = ctx->inner_exec && ctx->inner_key.size() == sizeof(key) &&
                    std::memcmp(ctx->inner_key.data(), &key, sizeof(key)) == 0;
  if (!same) {
    // captured on the context's private stream (the caller's may be the legacy default stream,
    // which cannot be captured); the graph is then launched on the caller's stream
    const long long launches = ctx->launches;
    cudaGraph_t graph = nullptr;
    cudaStream_t cs = ctx->cap_stream;
    HYDOT_CUDA_TRY(ctx, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    ctx->stream = cs;
    const bool timing = ctx->timer.on;  // no per-pass events inside the graph: it is timed whole
    ctx->timer.on = false;
    for (int o = 0; o < POLL_GROUP; ++o) roll_dispatch(ctx, variant, g, b, o, nrb, E, R, P);
    k_bump<<<1, 1, 0, cs>>>(ctx->d_it, POLL_GROUP);
    ctx->timer.on = timing;
    ctx->stream = s;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    ctx->launches = launches;
    if (e != cudaSuccess) return fail(ctx, HYDOT_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    cudaGraphExec_t exec = (cudaGraphExec_t)ctx->inner_exec;
    bool updated = false;
    if (exec) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(exec, graph, &info) == cudaSuccess;
      if (!updated) {
        (void)cudaGetLastError();
        cudaGraphExecDestroy(exec);
        ctx->inner_exec = nullptr;
      }
    }
    if (!updated) {
      e = cudaGraphInstantiate(&exec, graph, 0);
      if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(ctx, HYDOT_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
      }
      ctx->inner_exec = exec;
    }
    cudaGraphDestroy(graph);
    ctx->inner_key.assign(reinterpret_cast<const unsigned char*>(&key),
                          reinterpret_cast<const unsigned char*>(&key) + sizeof(key));
  }
  HYDOT_CUDA_TRY(ctx, cudaGraphLaunch((cudaGraphExec_t)ctx->inner_exec, s));
  ctx->launches += 2 * POLL_GROUP + 1;
  return HYDOT_OK;
}

// A general right-hand side for run_solve (adjoint solves): see Batch.
struct GeneralRhs {
  const int* slot;
  const double* w;
  const double* scale;
  int n_cells;
};

template <typename T, typename X, typename O>
int run_solve(hydot_ctx* ctx, int lam0, int nlam, O* phi_src, O* phi_det, hydot_stats* st,
              const GeneralRhs* gr = nullptr) {
  Geo g = make_geo(ctx);
  Batch b{};
  if (gr) {
    b.rhs_slot = gr->slot;
    b.rhs_w = gr->w;
    b.rhs_scale = gr->scale;
    b.n_rhs_cells = gr->n_cells;
  }
  b.coef = ctx->d_coef;
  b.optode = ctx->d_optode;
  b.lam0 = lam0;
  if (phi_src && phi_det) { b.f_begin = 0; b.nf = ctx->n_src + ctx->n_det; }
  else if (phi_src) { b.f_begin = 0; b.nf = ctx->n_src; }
  else { b.f_begin = ctx->n_src; b.nf = ctx->n_det; }
  b.nrhs = b.nf * nlam;
  b.status = ctx->d_status;
  b.iters = ctx->d_iters;
  b.cycles = ctx->d_cycles;
  b.scale = ctx->d_scale;
  b.next = ctx->d_next;
  b.rr0 = ctx->d_rr0;
  b.theta = ctx->d_theta;
  b.cw_floor = ctx->cw_floor;
  b.n_src = ctx->n_src;
  b.n_det = ctx->n_det;
  b.fin = ctx->d_final;
  b.part = ctx->d_part;
  b.counter = ctx->d_counter;
  b.err = ctx->d_err;
  b.dsig_d = nullptr;
  b.dsig_f = nullptr;
  if (ctx->d_dc) {
    const long long tot = (long long)nlam * ctx->N;
    k_dsig<<<(unsigned)std::min<long long>((tot + 255) / 256, 152 * 64), 256, 0, ctx->stream>>>(
        ctx->d_dc, ctx->d_eps, ctx->d_coef, lam0, nlam, ctx->n_chrom, ctx->N, ctx->h * ctx->h, ctx->d_dsig_d,
        ctx->d_dsig_f);
    ++ctx->launches;
    HYDOT_CUDA_TRY(ctx, cudaGetLastError());
    b.dsig_d = ctx->d_dsig_d;
    b.dsig_f = ctx->d_dsig_f;
  }
  const bool mixed = ctx->precision == HYDOT_MIXED;
  const double tin = mixed ? (ctx->inner_tol > 0 ? ctx->inner_tol : 1e-5) : ctx->tol;
  b.tol_in2 = tin * tin;
  b.max_inner = MAX_INNER_PER_CYCLE;
  b.max_iter = ctx->max_iter;
  b.tol = ctx->tol;
  b.tol_cw = ctx->tol_cw;
  b.abs_inner = (!mixed && ctx->tol_cw <= 0.0) ? 1 : 0;
  cudaStream_t s = ctx->stream;

  X* x64 = (X*)ctx->d_x64;
  T* E = (T*)ctx->d_e;
  T* R = (T*)ctx->d_r;
  T* P[2] = {(T*)ctx->d_p[0], (T*)ctx->d_p[1]};
  const unsigned nblk = (unsigned)((long long)b.nrhs * g.ntiles);
  const dim3 blk(NTHREADS);

  if constexpr (std::is_same<X, double>::value || std::is_same<X, df32>::value) {
    constexpr bool df = std::is_same<X, df32>::value;
    if (gr) {
      // the starting subspaces are built for the one-hot optode right-hand sides: start from zero
      HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(x64, 0, sizeof(X) * (size_t)b.nrhs * g.N, s));
    } else if (ctx->deflation_k > 0) {
      // Galerkin initial guess from the recycled subspace (shared by all wavelengths)
      int rc = deflate_initial_guess(ctx, lam0, b.f_begin, b.nf, b.nrhs, x64, df);
      if (rc) return rc;
    } else if (ctx->sg_m > 0) {
      // Galerkin initial guess from each optode's Krylov space of the mean-shift operator
      int rc = shift_initial_guess(ctx, lam0, b.f_begin, b.nf, b.nrhs, x64, df);
      if (rc) return rc;
    } else {
      HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(x64, 0, sizeof(X) * (size_t)b.nrhs * g.N, s));
    }
  } else {
    HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(x64, 0, sizeof(X) * (size_t)b.nrhs * g.N, s));
  }
  HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(b.err, 0, sizeof(int), s));
  if constexpr (std::is_same<X, df32>::value) {  // the residual's halo tile: up to 18 x 10 x 34 double-floats
    HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_residual_df<false>, sizeof(df32) * (g.tz + 2) * (TY + 2) * (TX + 2)));
    HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_residual_df<true>, sizeof(df32) * (g.tz + 2) * (TY + 2) * (TX + 2)));
  }
  if constexpr (std::is_same<X, cdf32>::value) {
    HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_residual_cdf<false>, sizeof(cdf32) * (g.tz + 2) * (TY + 2) * (TX + 2)));
    HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_residual_cdf<true>, sizeof(cdf32) * (g.tz + 2) * (TY + 2) * (TX + 2)));
  }
  k_reset<<<(b.nrhs + 255) / 256, 256, 0, s>>>(b);
  ++ctx->launches;
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());

  volatile int* hp = ctx->h_pinned;
  int prev_active = b.nrhs;
  for (int cycle = 0; cycle <= MAX_CYCLES; ++cycle) {
    if (b.cw_floor > 0.0) {
      k_theta<X><<<(b.nrhs + 255) / 256, 256, 0, s>>>(g, b, x64, ctx->d_optode);
      ++ctx->launches;
    }
    cudaEvent_t t_res = timer_begin(ctx);
    if constexpr (std::is_same<X, df32>::value) {
      // the general body only where a field has a per-cell shift or a general right-hand side
      const size_t sm_df = sizeof(df32) * (g.tz + 2) * (TY + 2) * (TX + 2);
      if (b.dsig_d || b.dsig_f || b.rhs_slot)
        k_residual_df<true><<<nblk, blk, sm_df, s>>>(g, b, ctx->d_coef_f, x64, R);
      else
        k_residual_df<false><<<nblk, blk, sm_df, s>>>(g, b, ctx->d_coef_f, x64, R);
    } else if constexpr (std::is_same<X, cdf32>::value) {
      const size_t sm_c = sizeof(cdf32) * (g.tz + 2) * (TY + 2) * (TX + 2);
      if (b.dsig_d || b.dsig_f)
        k_residual_cdf<true><<<nblk, blk, sm_c, s>>>(g, b, ctx->d_coef_f, x64, (float2*)R);
      else
        k_residual_cdf<false><<<nblk, blk, sm_c, s>>>(g, b, ctx->d_coef_f, x64, (float2*)R);
    } else {
      k_residual<T, X><<<nblk, blk, 0, s>>>(g, b, x64, R);
    }
    ++ctx->launches;
    timer_end(ctx, t_res, HYDOT_KERNEL_RESIDUAL,
              (double)(cycle == 0 ? b.nrhs : prev_active) * (double)g.N * (double)(sizeof(X) + sizeof(T)));
    HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(b.counter, 0, sizeof(int) * (size_t)ctx->counter_len, s));
    k_decide<<<(b.nrhs + 255) / 256, 256, 0, s>>>(g, b);
    ++ctx->launches;
    HYDOT_CUDA_TRY(ctx, cudaGetLastError());
    HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync((void*)&hp[0], b.counter, sizeof(int), cudaMemcpyDeviceToHost, s));
    HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (hp[0] == 0) break;
    prev_active = hp[0];
    // inner iterations in groups; the group after the one being polled is already queued
    int it = 0;
    int pending = -1;  // index of the iteration whose counter is in flight
    cudaEvent_t ev[2];
    HYDOT_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
    HYDOT_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
    int slot = 0;
    bool stop = false;
    // rolling passes (FP32 real or complex64 fields, TMA): the iteration index lives on the device
    const bool roll = (std::is_same<T, float>::value || std::is_same<T, cpx<float>>::value) && ctx->use_tma &&
                      !ctx->d_dc;
    void* const Pv[2] = {P[0], P[1]};
    const unsigned nrb =
        roll ? (unsigned)((long long)b.nrhs * g.ntx * g.nty * ((g.nz + ctx->dir_seg - 1) / ctx->dir_seg)) : 0u;
    if (roll) HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_it, 0, sizeof(int), s));
    // persistent form: only once the slab variant of the launched form is settled, so that the
    // two forms are compared at their best
    const int mode = (roll && ctx->sweep_ok && ctx->tune.variant >= 0) ? persist_pick(ctx) : 0;
    const bool persistent = mode == 1;
    const bool tuning_mode = roll && ctx->sweep_ok && ctx->tune.variant >= 0 && ctx->persist.mode < 0;
    if (tuning_mode) HYDOT_CUDA_TRY(ctx, cudaEventRecord(ctx->tune_ev[0], s));
    if (persistent) {
      cudaEvent_t t_grp = timer_begin(ctx);
      int ran = 0;
      int rc = persist_launch(ctx, g, b, nrb, &ran);
      if (rc) return rc;
      timer_end(ctx, t_grp, HYDOT_KERNEL_ITER, 0.0, ran);
      it = ran;
      stop = true;
    }
    if (roll && ctx->use_sweep && !persistent) {
      // the cycle's first inner products (gamma_0, delta_0, ||r_0||^2) from r_0
      sweep_dispatch<true>(ctx, roll_pick(ctx), g, b, 0);
      if (ctx->timer.on) ctx->timer.bytes[HYDOT_KERNEL_PRIME] += (double)prev_active * (double)g.N * sizeof(T);
      HYDOT_CUDA_TRY(ctx, cudaGetLastError());
    }
    std::vector<unsigned char> replayed;  // per group: 1 if it ran as a graph replay (no per-pass events)
    if (persistent) replayed.assign((it + POLL_GROUP - 1) / POLL_GROUP, 1);
    while (!stop && it < MAX_INNER_PER_CYCLE) {
      int g_end = std::min(it + POLL_GROUP, MAX_INNER_PER_CYCLE);
      // autotuning: a group that does not start the cycle runs one candidate variant and is timed
      const int variant = roll ? roll_pick(ctx) : 0;
      const bool tuning = roll && ctx->tune.variant < 0 && it > 0;
      const int g_begin = it;
      if (tuning) HYDOT_CUDA_TRY(ctx, cudaEventRecord(ctx->tune_ev[0], s));
      cudaEvent_t t_grp = timer_begin(ctx);  // the whole group: every pass of its iterations
      if (roll) {
        if (ctx->use_graphs && !tuning && ctx->tune.variant >= 0) {
          int rc = inner_graph_launch(ctx, g, b, variant, nrb, E, R, Pv);
          if (rc) return rc;
          it = g_end;
          replayed.push_back(1);
        } else {
          replayed.push_back(0);
          for (; it < g_end; ++it) roll_dispatch(ctx, variant, g, b, it, nrb, E, R, Pv);
          k_bump<<<1, 1, 0, s>>>(ctx->d_it, POLL_GROUP);
          ++ctx->launches;
        }
      }
      for (; it < g_end; ++it) {
        cudaEvent_t t0 = timer_begin(ctx);
        k_dir<T><<<nblk, blk, 0, s>>>(g, b, it, R, P[it & 1], P[(it + 1) & 1]);
        ++ctx->launches;
        timer_end(ctx, t0, HYDOT_KERNEL_DIR, 0.0);
        t0 = timer_begin(ctx);
        k_update<T><<<nblk, blk, 0, s>>>(g, b, it, E, R, P[(it + 1) & 1]);
        ++ctx->launches;
        timer_end(ctx, t0, HYDOT_KERNEL_UPDATE, 0.0);
      }
      timer_end(ctx, t_grp, HYDOT_KERNEL_ITER, 0.0, g_end - g_begin);
      HYDOT_CUDA_TRY(ctx, cudaGetLastError());
      if (tuning) {
        // time of the group per active cell-iteration (fields that ran x cells)
        HYDOT_CUDA_TRY(ctx, cudaEventRecord(ctx->tune_ev[1], s));
        int cnt[POLL_GROUP];
        HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(cnt, b.counter + 1 + g_begin, sizeof(int) * (it - g_begin),
                                            cudaMemcpyDeviceToHost, s));
        HYDOT_CUDA_TRY(ctx, cudaEventSynchronize(ctx->tune_ev[1]));
        float ms = 0.f;
        HYDOT_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->tune_ev[0], ctx->tune_ev[1]));
        double work = 0.0;
        for (int q = 0; q < it - g_begin; ++q) work += (double)cnt[q] * (double)g.N;
        // a group in which fields converged mixes full and empty launches: only whole groups count
        if (cnt[0] == cnt[it - g_begin - 1]) roll_record(ctx, variant, ms, work);
      }
      HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync((void*)&hp[1 + slot], b.counter + 1 + (it - 1), sizeof(int),
                                          cudaMemcpyDeviceToHost, s));
      HYDOT_CUDA_TRY(ctx, cudaEventRecord(ev[slot], s));
      if (pending >= 0) {
        int ps = slot ^ 1;
        HYDOT_CUDA_TRY(ctx, cudaEventSynchronize(ev[ps]));
        if (hp[1 + ps] == 0) stop = true;
      }
      pending = it - 1;
      slot ^= 1;
    }
    HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (tuning_mode && it > 0) {
      // the cycle's inner solve per active cell-iteration, in the mode it ran
      HYDOT_CUDA_TRY(ctx, cudaEventRecord(ctx->tune_ev[1], s));
      std::vector<int> cnt(it);
      HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(cnt.data(), b.counter + 1, sizeof(int) * it, cudaMemcpyDeviceToHost, s));
      HYDOT_CUDA_TRY(ctx, cudaEventSynchronize(ctx->tune_ev[1]));
      float ms = 0.f;
      HYDOT_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, ctx->tune_ev[0], ctx->tune_ev[1]));
      double work = 0.0;
      for (int q = 0; q < it; ++q) work += (double)cnt[q] * (double)g.N;
      if (it >= POLL_GROUP) persist_record(ctx, mode, ms, work);
    }
    if (ctx->timer.on) {
      // algorithmic bytes of the inner passes: fields active at each iteration (the counters
      // k_dir increments) x 12 B (pass 1) or 20 B (pass 2) per cell in the inner precision
      std::vector<int> cnt(it);
      if (it > 0) {  // on the context's stream: a legacy-stream copy would serialise concurrent contexts
        HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(cnt.data(), b.counter + 1, sizeof(int) * it, cudaMemcpyDeviceToHost, s));
        HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(s));
      }
      // (per-pass kinds only for the groups whose passes were launched, and timed, directly)
      double active = 0.0, direct = 0.0;
      for (int q = 0; q < it; ++q) {
        active += cnt[q];
        const size_t grp = (size_t)(q / POLL_GROUP);
        if (grp >= replayed.size() || !replayed[grp]) direct += cnt[q];
      }
      if (roll && (ctx->use_sweep || persistent)) {
        ctx->timer.bytes[HYDOT_KERNEL_SWEEP] += direct * 6.0 * (double)g.N * sizeof(T);
      } else {
        ctx->timer.bytes[HYDOT_KERNEL_DIR] += direct * 3.0 * (double)g.N * sizeof(T);
        ctx->timer.bytes[HYDOT_KERNEL_UPDATE] += direct * 5.0 * (double)g.N * sizeof(T);
      }
      ctx->timer.bytes[HYDOT_KERNEL_ITER] += active * 6.0 * (double)g.N * sizeof(T);
      timer_flush(ctx);
    }
    // any field still marked INNER hit the per-cycle cap: finish it
    {
      dim3 fg((unsigned)std::min<long long>((g.N + 2047) / 2048, 1024), (unsigned)std::min(b.nrhs, 65535));  // 8 cells per thread
      // fields that were still iterating when the cap hit are FINISHED by a k_dir at the cap; a
      // launched loop that stopped on a zero count of iterating fields left none (the persistent
      // form may stop at the cap itself)
      if (!stop || persistent) {
        k_dir<T><<<nblk, blk, 0, s>>>(g, b, MAX_INNER_PER_CYCLE, R, P[0], P[1]);
        ++ctx->launches;
      }
      k_fold<T, X><<<fg, 256, 0, s>>>(g, b, x64, E);
      ++ctx->launches;
      HYDOT_CUDA_TRY(ctx, cudaGetLastError());
    }
  }
  {
    dim3 fg((unsigned)std::min<long long>((g.N + 2047) / 2048, 1024), (unsigned)std::min(b.nrhs, 65535));  // 8 cells per thread
    k_output<X, O><<<fg, 256, 0, s>>>(g, b, x64, phi_src, phi_det, ctx->n_src, ctx->n_det);
    ++ctx->launches;
    HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  }
  // statistics
  std::vector<int> iters(b.nrhs), cycles(b.nrhs);
  std::vector<double> fin(2 * (size_t)b.nrhs);
  HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(iters.data(), b.iters, sizeof(int) * b.nrhs, cudaMemcpyDeviceToHost, s));
  HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(cycles.data(), b.cycles, sizeof(int) * b.nrhs, cudaMemcpyDeviceToHost, s));
  HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(fin.data(), b.fin, sizeof(double) * 2 * b.nrhs, cudaMemcpyDeviceToHost, s));
  int timed_out = 0;
  HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(&timed_out, b.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (timed_out) return fail(ctx, HYDOT_ERR_TIMEOUT, "a bounded wait for a TMA tile gave up; fields are not valid");
  int nnc = 0, imax = 0, cmax = 0;
  double isum = 0, rmax = 0, omax = 0;
  for (int i = 0; i < b.nrhs; ++i) {
    bool conv = fin[2 * i] <= ctx->tol && (ctx->tol_cw <= 0 || fin[2 * i + 1] <= ctx->tol_cw);
    nnc += conv ? 0 : 1;
    imax = std::max(imax, iters[i]);
    cmax = std::max(cmax, cycles[i]);
    isum += iters[i];
    rmax = std::max(rmax, fin[2 * i]);
    omax = std::max(omax, fin[2 * i + 1]);
  }
  if (st) {
    st->n_fields = b.nrhs;
    st->n_not_converged = nnc;
    st->iters_max = imax;
    st->iters_mean = b.nrhs ? isum / b.nrhs : 0.0;
    st->cycles_max = cmax;
    st->resid_max = rmax;
    st->cw_max = omax;
  }
  if (nnc) {
    ctx->err = std::to_string(nnc) + " of " + std::to_string(b.nrhs) + " fields missed the tolerance";
    return HYDOT_ERR_NOT_CONVERGED;
  }
  return HYDOT_OK;
}

}  // namespace

namespace {

bool getenv_flag(const char* name) {
  const char* v = std::getenv(name);
  return v && *v && std::strcmp(v, "0") != 0;
}

// 4-D tensor map {nx, ny, nz, max_fields} of an FP32 (real) or complex64 (8-byte elements, copied
// as opaque 64-bit words) field buffer with a bx x by x bz box.
int encode_field_map(hydot_ctx* ctx, void* base, CUtensorMap* map, int bx, int by, int bz) {
  // looked up once (a function-local static is initialised once even when batch workers race here)
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    return (e == cudaSuccess && q == cudaDriverEntryPointSuccess) ? reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn)
                                                                   : nullptr;
  }();
  if (!encode) return fail(ctx, HYDOT_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t nx = ctx->nx, ny = ctx->ny, nz = ctx->nz, F = ctx->max_fields;
  cuuint64_t dims[4] = {nx, ny, nz, F};
  const cuuint64_t w = ctx->cplx ? 8 : 4;
  cuuint64_t strides[3] = {nx * w, nx * ny * w, nx * ny * nz * w};
  cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, 1};
  cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt = ctx->cplx ? CU_TENSOR_MAP_DATA_TYPE_UINT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUresult r = encode(map, dt, 4, base, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, HYDOT_ERR_CUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
  return HYDOT_OK;
}

}  // namespace

int solver_alloc(hydot_ctx* ctx) {
  Tiling& t = ctx->tiling;
  t.tx = TX;
  t.ty = TY;
  // FP32 real / complex64 fields with a 16-byte row pitch take the TMA inner kernels (8-plane tiles)
  ctx->use_tma = ctx->precision == HYDOT_MIXED && (ctx->nx % (ctx->cplx ? 2 : 4) == 0) && !getenv_flag("HYDOT_NO_TMA");
  t.tz = ctx->use_tma ? std::min(ctx->nz, TZT) : std::min(ctx->nz, 16);
  t.ntx = (ctx->nx + TX - 1) / TX;
  t.nty = (ctx->ny + TY - 1) / TY;
  t.ntz = (ctx->nz + t.tz - 1) / t.tz;
  t.ntiles = t.ntx * t.nty * t.ntz;
  const size_t F = (size_t)ctx->max_fields, N = (size_t)ctx->N;
  const bool mixed = ctx->precision == HYDOT_MIXED;
  const size_t xw = ctx->cplx ? 16 : 8;
  const size_t iw = (mixed ? 4 : 8) * (ctx->cplx ? 2 : 1);
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_x64, xw * F * N));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_e, iw * F * N));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_r, iw * F * N));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_p[0], iw * F * N));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_p[1], iw * F * N));
  ctx->part_stride = part_stride(t.ntiles);
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_part, sizeof(double) * ctx->part_stride * F));
  HYDOT_CUDA_TRY(ctx, cudaMemset(ctx->d_part, 0, sizeof(double) * ctx->part_stride * F));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_status, sizeof(int) * F));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_iters, sizeof(int) * F));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_cycles, sizeof(int) * F));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_scale, sizeof(double) * F));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_next, sizeof(double) * F));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_rr0, sizeof(double) * F));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_theta, sizeof(double) * F));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_final, sizeof(double) * 2 * F));
  ctx->counter_len = MAX_INNER_PER_CYCLE + 8;
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_counter, sizeof(int) * ctx->counter_len));
  HYDOT_CUDA_TRY(ctx, cudaMallocHost(&ctx->h_pinned, sizeof(int) * 8));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_err, sizeof(int)));
  HYDOT_CUDA_TRY(ctx, cudaMemset(ctx->d_err, 0, sizeof(int)));
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_it, sizeof(int)));
  HYDOT_CUDA_TRY(ctx, cudaMemset(ctx->d_it, 0, sizeof(int)));
  ctx->use_graphs = !getenv_flag("HYDOT_NO_GRAPHS");
  HYDOT_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  // Real FP32 fields on the TMA path iterate in two passes (measured faster on every workload
  // here), or in single sweeps with HYDOT_SINGLE_SWEEP=1. Only with single sweeps is the persistent
  // form tuned against launched iterations: the two do the same arithmetic, so the tuner never
  // changes a result's bits (HYDOT_PERSISTENT=0 or 1 fixes the launch form; 1 implies sweeps).
  ctx->sweep_ok = ctx->use_tma && !ctx->cplx;
  if (ctx->sweep_ok) {
    ctx->use_sweep = getenv_flag("HYDOT_SINGLE_SWEEP");
    ctx->persist.mode = ctx->use_sweep ? -1 : 0;
  }
  if (ctx->sweep_ok) {
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_r2, iw * F * N));
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_cgsc, sizeof(double) * 4 * F));
    HYDOT_CUDA_TRY(ctx, cudaMemset(ctx->d_cgsc, 0, sizeof(double) * 4 * F));
    if (const char* v = std::getenv("HYDOT_PERSISTENT")) ctx->persist.mode = (std::atoi(v) != 0) ? 1 : 0;
    if (ctx->persist.mode == 1 && !ctx->use_sweep) ctx->use_sweep = true;  // the persistent form iterates in sweeps
  }
  if (ctx->use_tma) {
    int rc = roll_setup(ctx);
    if (!rc && ctx->sweep_ok && !ctx->use_sweep) {  // the sweep kernels also serve the priming pass
      rc = sweep_attrs<4, 3, 1, 3>(ctx);
      if (!rc) rc = sweep_attrs<3, 4, 1, 3>(ctx);
      if (!rc) rc = sweep_attrs<3, 3, 2, 2>(ctx);
      if (!rc) rc = sweep_attrs<4, 3, 2, 2>(ctx);
    }
    if (!rc && ctx->sweep_ok) rc = persist_setup(ctx);
    for (int d = 0; d < 2 && !rc && ctx->sweep_ok; ++d) {
      const int bz = 3 + d;
      constexpr int B1 = SweepShape<1>::BYB, B2 = SweepShape<2>::BYB;
      rc = encode_field_map(ctx, ctx->d_r, &ctx->tm_r2[d][0], BX2, B1, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_r2, &ctx->tm_r2[d][1], BX2, B1, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_p[0], &ctx->tm_p2[d][0], BX2, B1, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_p[1], &ctx->tm_p2[d][1], BX2, B1, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_e, &ctx->tm_e2[d], TX, TY, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_r, &ctx->tm_r4[d][0], BX2, B2, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_r2, &ctx->tm_r4[d][1], BX2, B2, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_p[0], &ctx->tm_p4[d][0], BX2, B2, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_p[1], &ctx->tm_p4[d][1], BX2, B2, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_e, &ctx->tm_e4[d], TX, 2 * TY, bz);
    }
    // per slab depth (2, 4, 8 planes): halo slabs of r and p (pass 1 reads r and p_old, pass 2 reads
    // p_new), plain slabs of e and r
    for (int k = 0; k < 3 && !rc; ++k) {
      const int bz = 2 << k;
      rc = encode_field_map(ctx, ctx->d_r, &ctx->tm_rh[k], BXT, BYT, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_p[0], &ctx->tm_ph[k][0], BXT, BYT, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_p[1], &ctx->tm_ph[k][1], BXT, BYT, bz);
      if (!rc && !ctx->cplx) {  // pass 1 on 32 x 16 tiles (real fields)
        rc = encode_field_map(ctx, ctx->d_r, &ctx->tm_rh2[k], BXT, 2 * TY + 2, bz);
        if (!rc) rc = encode_field_map(ctx, ctx->d_p[0], &ctx->tm_ph2[k][0], BXT, 2 * TY + 2, bz);
        if (!rc) rc = encode_field_map(ctx, ctx->d_p[1], &ctx->tm_ph2[k][1], BXT, 2 * TY + 2, bz);
      }
      if (!rc) {  // pass 1 on paired cells: 64 x 8 and 64 x 16 tiles
        for (int c = 0; c < 2 && !rc; ++c) {
          rc = encode_field_map(ctx, ctx->d_r, &ctx->tm_rx[c][k], BXP, (c + 1) * TY + 2, bz);
          if (!rc) rc = encode_field_map(ctx, ctx->d_p[0], &ctx->tm_px[c][k][0], BXP, (c + 1) * TY + 2, bz);
          if (!rc) rc = encode_field_map(ctx, ctx->d_p[1], &ctx->tm_px[c][k][1], BXP, (c + 1) * TY + 2, bz);
        }
      }
      if (!rc) rc = encode_field_map(ctx, ctx->d_e, &ctx->tm_e[k], TX, TY, bz);
      if (!rc) rc = encode_field_map(ctx, ctx->d_r, &ctx->tm_rv[k], TX, TY, bz);
    }
    if (rc) return rc;
    HYDOT_CUDA_TRY(ctx, cudaEventCreate(&ctx->tune_ev[0]));
    HYDOT_CUDA_TRY(ctx, cudaEventCreate(&ctx->tune_ev[1]));
    if (const char* v = std::getenv("HYDOT_ROLL_VARIANT")) {
      const int want = std::atoi(v);
      if (want >= 0 && want < HYDOT_ROLL_VARIANTS) ctx->tune.variant = want;
    }
    // whole columns unless the blocks of one wavelength's fields would leave most SMs idle
    ctx->dir_seg = t.ntz * t.tz;
    if (const char* v = std::getenv("HYDOT_DIR_SEG")) {
      const int want = std::atoi(v);
      if (want > 0) ctx->dir_seg = std::max(t.tz, (want + t.tz - 1) / t.tz * t.tz);
    }
  }
  return HYDOT_OK;
}

void solver_free(hydot_ctx* ctx) {
  cudaFree(ctx->d_x64);
  cudaFree(ctx->d_r2);
  cudaFree(ctx->d_cgsc);
  cudaFree(ctx->d_gsync);
  cudaFree(ctx->d_rhs_slot);
  cudaFree(ctx->d_rhs_w);
  cudaFree(ctx->d_rhs_scale);
  cudaFree(ctx->d_e);
  cudaFree(ctx->d_r);
  cudaFree(ctx->d_p[0]);
  cudaFree(ctx->d_p[1]);
  cudaFree(ctx->d_part);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_iters);
  cudaFree(ctx->d_cycles);
  cudaFree(ctx->d_scale);
  cudaFree(ctx->d_next);
  cudaFree(ctx->d_rr0);
  cudaFree(ctx->d_theta);
  cudaFree(ctx->d_final);
  cudaFree(ctx->d_counter);
  cudaFree(ctx->d_err);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  cudaFree(ctx->d_it);
  cudaFree(ctx->d_dc);
  cudaFree(ctx->d_dsig_d);
  cudaFree(ctx->d_dsig_f);
  if (ctx->inner_exec) cudaGraphExecDestroy((cudaGraphExec_t)ctx->inner_exec);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->tune_ev[0]) cudaEventDestroy(ctx->tune_ev[0]);
  if (ctx->tune_ev[1]) cudaEventDestroy(ctx->tune_ev[1]);
}

namespace {
// One thread waits on a shared-memory mbarrier that nothing arrives at, through the same bounded
// poll loop as the pipelined kernels, then raises the error flag and returns.
__global__ void k_wait_selftest(int* err, uint32_t polls) {
  __shared__ uint64_t m;
  if (threadIdx.x == 0) {
    mbar_init(&m, 1);
    mbar_fence_init();
    if (!mbar_wait_polls(&m, 0u, polls)) atomicExch(err, 1);
  }
}
}  // namespace

// Two co-resident blocks; only block 0 arrives at the grid barrier, so its bounded wait runs out.
__global__ void k_grid_wait_selftest(GridSync gs, int* err) {
  if (blockIdx.x == 0) grid_sync(gs, err);
}

int wait_selftest_impl(hydot_ctx* ctx, int polls) {
  if (polls < 1 || (uint32_t)polls > WAIT_POLLS) return fail(ctx, HYDOT_ERR_ARG, "polls must be in 1..2^22");
  int flag[2] = {0, 0};
  // (1) an mbarrier that nothing arrives at, polled as the pipelined kernels poll their slabs
  HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  k_wait_selftest<<<1, 32, 0, ctx->stream>>>(ctx->d_err, (uint32_t)polls);
  ++ctx->launches;
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(&flag[0], ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  // (2) the persistent kernel's grid barrier with one of two blocks never arriving
  HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  unsigned* words = ctx->d_gsync;
  bool own = false;
  if (!words) {
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&words, 2 * sizeof(unsigned)));
    own = true;
  }
  HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(words, 0, 2 * sizeof(unsigned), ctx->stream));
  GridSync gs{words, words + 1, (uint32_t)polls};
  int* err = ctx->d_err;
  void* args[] = {&gs, &err};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_grid_wait_selftest, dim3(2), dim3(32), args, 0,
                                              ctx->stream);
  ++ctx->launches;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&flag[1], ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (own) cudaFree(words);
  if (e != cudaSuccess) return fail(ctx, HYDOT_ERR_CUDA, std::string("grid-barrier self-test: ") + cudaGetErrorString(e));
  HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (flag[0] && flag[1]) return fail(ctx, HYDOT_ERR_TIMEOUT, "bounded waits gave up (self-test: mbarrier and grid barrier)");
  return fail(ctx, HYDOT_ERR_STATE, std::string("self-test: a bounded wait did not give up (mbarrier ") +
                                        (flag[0] ? "yes" : "no") + ", grid barrier " + (flag[1] ? "yes" : "no") + ")");
}

int get_launch_mode_impl(const hydot_ctx* ctx, int* mode, double* ns_launched, double* ns_persistent) {
  const auto& p = ctx->persist;
  if (mode) *mode = ctx->sweep_ok ? p.mode : 0;
  if (ns_launched) *ns_launched = p.cells[0] > 0.0 ? 1e6 * p.ms[0] / p.cells[0] : 0.0;
  if (ns_persistent) *ns_persistent = p.cells[1] > 0.0 ? 1e6 * p.ms[1] / p.cells[1] : 0.0;
  return HYDOT_OK;
}

int set_absorption_impl(hydot_ctx* ctx, const double* dc) {
  if (!dc) {
    cudaFree(ctx->d_dc);
    cudaFree(ctx->d_dsig_d);
    cudaFree(ctx->d_dsig_f);
    ctx->d_dc = nullptr;
    ctx->d_dsig_d = nullptr;
    ctx->d_dsig_f = nullptr;
    return HYDOT_OK;
  }
  const size_t n = (size_t)ctx->n_chrom * ctx->N;
  // one increment per wavelength of the largest slice (max_fields / (n_src + n_det) wavelengths)
  const size_t m = (size_t)std::max(1, ctx->max_fields / std::max(1, ctx->n_src + ctx->n_det)) * ctx->N;
  if (!ctx->d_dc) {
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_dc, sizeof(double) * n));
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_dsig_d, sizeof(double) * m));
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_dsig_f, sizeof(float) * m));
  }
  HYDOT_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->d_dc, dc, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
  HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return HYDOT_OK;
}

int get_tuning_impl(const hydot_ctx* ctx, int* variant, int* planes, int* buffers, double* ns_per_cell) {
  if (variant) *variant = ctx->use_tma ? ctx->tune.variant : -1;
  for (int v = 0; v < HYDOT_ROLL_VARIANTS; ++v) {
    const RollVariant& rv = ctx->use_sweep ? SWEEP_VARIANTS[v] : (ctx->cplx ? ROLL_VARIANTS_C[v] : ROLL_VARIANTS[v]);
    if (planes) planes[v] = rv.rp;
    if (buffers) buffers[v] = rv.rs;
    if (ns_per_cell)
      ns_per_cell[v] = ctx->tune.cells[v] > 0.0 ? 1e6 * ctx->tune.ms[v] / ctx->tune.cells[v] : 0.0;
  }
  return HYDOT_OK;
}

namespace {
// w[rhs][d] = y[(s*nd + d)*nlam + a] / |w[rhs]|_2 and scale[rhs] = |w[rhs]|_2 for rhs = a*ns + s: the
// adjoint right-hand side sum_d y[s,d,lambda] e_d of source s at wavelength a of the slice.
template <typename Y>
__global__ void k_adjoint_weights(const Y* __restrict__ y, int nlam, int ns, int nd, double* __restrict__ w,
                                  double* __restrict__ scale) {
  const int rhs = blockIdx.x * blockDim.x + threadIdx.x;
  if (rhs >= nlam * ns) return;
  const int a = rhs / ns, s = rhs - a * ns;
  double n2 = 0.0;
  for (int d = 0; d < nd; ++d) {
    const double v = (double)y[((size_t)s * nd + d) * nlam + a];
    n2 += v * v;
  }
  const double n = sqrt(n2);
  const double inv = n > 0.0 ? 1.0 / n : 0.0;
  for (int d = 0; d < nd; ++d) w[(size_t)rhs * nd + d] = (double)y[((size_t)s * nd + d) * nlam + a] * inv;
  scale[rhs] = n;
}

// slot[x] = d at the cell of detector d, -1 elsewhere
__global__ void k_detector_slots(const int* __restrict__ optode, int ns, int nd, int* __restrict__ slot) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d < nd) slot[optode[ns + d]] = d;
}
}  // namespace

int solve_adjoint_impl(hydot_ctx* ctx, int lam0, int nlam, const void* y, void* psi, hydot_stats* st) {
  if (ctx->cplx) return fail(ctx, HYDOT_ERR_STATE, "adjoint solves are available for continuous-wave (real) fields only");
  if (ctx->n_src < 1 || ctx->n_det < 1) return fail(ctx, HYDOT_ERR_STATE, "adjoint solves need sources and detectors");
  if (!y || !psi) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  if (lam0 < 0 || nlam < 1 || lam0 + nlam > ctx->n_lambda) return fail(ctx, HYDOT_ERR_ARG, "wavelength slice out of range");
  if ((long long)nlam * ctx->n_src > ctx->max_fields)
    return fail(ctx, HYDOT_ERR_ARG, "nlam * n_src exceeds the fields the workspace holds");
  cudaStream_t s = ctx->stream;
  if (!ctx->d_rhs_slot) {
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_rhs_slot, sizeof(int) * (size_t)ctx->N));
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_rhs_w, sizeof(double) * (size_t)ctx->max_fields * ctx->n_det));
    HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_rhs_scale, sizeof(double) * (size_t)ctx->max_fields));
    HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_rhs_slot, 0xff, sizeof(int) * (size_t)ctx->N, s));
    k_detector_slots<<<(ctx->n_det + 127) / 128, 128, 0, s>>>(ctx->d_optode, ctx->n_src, ctx->n_det, ctx->d_rhs_slot);
    ++ctx->launches;
    HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  }
  const int nrhs = nlam * ctx->n_src;
  const bool mixed = ctx->precision == HYDOT_MIXED;
  if (mixed)
    k_adjoint_weights<float><<<(nrhs + 127) / 128, 128, 0, s>>>((const float*)y, nlam, ctx->n_src, ctx->n_det,
                                                                ctx->d_rhs_w, ctx->d_rhs_scale);
  else
    k_adjoint_weights<double><<<(nrhs + 127) / 128, 128, 0, s>>>((const double*)y, nlam, ctx->n_src, ctx->n_det,
                                                                 ctx->d_rhs_w, ctx->d_rhs_scale);
  ++ctx->launches;
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  const GeneralRhs gr{ctx->d_rhs_slot, ctx->d_rhs_w, ctx->d_rhs_scale, ctx->n_det};
  if (mixed) return run_solve<float, df32, float>(ctx, lam0, nlam, (float*)psi, (float*)nullptr, st, &gr);
  return run_solve<double, double, double>(ctx, lam0, nlam, (double*)psi, (double*)nullptr, st, &gr);
}

int solve_fields_impl(hydot_ctx* ctx, int lam0, int nlam, void* phi_src, void* phi_det, hydot_stats* st) {
  const bool mixed = ctx->precision == HYDOT_MIXED;
  if (!ctx->cplx) {
    if (mixed) return run_solve<float, df32, float>(ctx, lam0, nlam, (float*)phi_src, (float*)phi_det, st);
    return run_solve<double, double, double>(ctx, lam0, nlam, (double*)phi_src, (double*)phi_det, st);
  }
  using cf = cpx<float>;
  using cd = cpx<double>;
  if (mixed) return run_solve<cf, cdf32, cf>(ctx, lam0, nlam, (cf*)phi_src, (cf*)phi_det, st);
  return run_solve<cd, cd, cd>(ctx, lam0, nlam, (cd*)phi_src, (cd*)phi_det, st);
}


}  // namespace hydot
