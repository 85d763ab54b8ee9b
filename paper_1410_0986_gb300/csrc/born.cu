// Born rows and implicit Born products (eqn:lippschwin, eqn:perturbation, eqn:measurement).
//
//   J[(s,d,a),(c,x)] = -h^3 eps_c(lambda_a) phi_s[a][s][x] phi_d[a][d][x]
//   y[(s,d,a)]       = -h^3 sum_x phi_s[a][s][x] phi_d[a][d][x] mu_a[x],  mu_a[x] = sum_c eps_c(lambda_a) x[c*N+x]
//   g[c*N+x]        += -h^3 sum_a eps_c(lambda_a) sum_s phi_s[a][s][x] sum_d Y_a[s][d] phi_d[a][d][x]
// with slice rows r = (s*n_det + d)*nlam + a.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>

#include "hydot_internal.cuh"

namespace hydot {

namespace {

constexpr int MAXC = 16;

// ---------------------------------------------------------------- assembly (write streaming)
// Blocks walk the slice's rows wavelength-major (all (s,d) of one wavelength, then the next),
// so the n_src+n_det fields of a wavelength stay in L2 while their rows are written; every
// element of J is written once with an evict-first store.
template <typename E, int VEC>
struct Vec;
template <> struct Vec<float, 4> { using V = float4; };
template <> struct Vec<double, 2> { using V = double2; };

template <typename E, int VEC>
__global__ void __launch_bounds__(256) k_born_rows(const E* __restrict__ ps, const E* __restrict__ pd,
                                                   const double* __restrict__ eps, int lam0, int nlam, int ns,
                                                   int nd, int nc, long long N, double h3, long long row0,
                                                   long long nrows, int sd_lo, int n_sd, E* __restrict__ J,
                                                   long long ldJ) {
  using V = typename Vec<E, VEC>::V;
  const long long nvec = N / VEC;
  const long long total_rows = (long long)nlam * n_sd;
  for (long long yy = blockIdx.y; yy < total_rows; yy += gridDim.y) {
    const int a = (int)(yy / n_sd);
    const int sd = sd_lo + (int)(yy % n_sd);
    const long long r = (long long)sd * nlam + a;
    if (r < row0 || r >= row0 + nrows) continue;
    const int s = sd / nd, d = sd % nd;
    const E* fs = ps + ((size_t)a * ns + s) * N;
    const E* fd = pd + ((size_t)a * nd + d) * N;
    E* row = J + (size_t)(r - row0) * ldJ;
    E w[MAXC];
    for (int c = 0; c < nc; ++c) w[c] = (E)(-h3 * eps[(size_t)(lam0 + a) * nc + c]);
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nvec; v += (long long)gridDim.x * blockDim.x) {
      V a4 = reinterpret_cast<const V*>(fs)[v];
      V b4 = reinterpret_cast<const V*>(fd)[v];
      V hv;
      if constexpr (VEC == 4) {
        hv = make_float4(a4.x * b4.x, a4.y * b4.y, a4.z * b4.z, a4.w * b4.w);
      } else {
        hv = make_double2(a4.x * b4.x, a4.y * b4.y);
      }
      for (int c = 0; c < nc; ++c) {
        V o;
        if constexpr (VEC == 4) {
          o = make_float4(w[c] * hv.x, w[c] * hv.y, w[c] * hv.z, w[c] * hv.w);
        } else {
          o = make_double2(w[c] * hv.x, w[c] * hv.y);
        }
        __stcs(reinterpret_cast<V*>(row + (size_t)c * N) + v, o);
      }
    }
    // tail (N not a multiple of VEC) -- also the whole row on the unaligned path
    for (long long x = nvec * VEC + (long long)blockIdx.x * blockDim.x + threadIdx.x; x < N;
         x += (long long)gridDim.x * blockDim.x) {
      E hv = fs[x] * fd[x];
      for (int c = 0; c < nc; ++c) row[(size_t)c * N + x] = w[c] * hv;
    }
  }
}

template <typename E>
__global__ void __launch_bounds__(256) k_born_rows_scalar(const E* __restrict__ ps, const E* __restrict__ pd,
                                                          const double* __restrict__ eps, int lam0, int nlam, int ns,
                                                          int nd, int nc, long long N, double h3, long long row0,
                                                          long long nrows, int sd_lo, int n_sd, E* __restrict__ J,
                                                          long long ldJ) {
  const long long total_rows = (long long)nlam * n_sd;
  for (long long yy = blockIdx.y; yy < total_rows; yy += gridDim.y) {
    const int a = (int)(yy / n_sd);
    const int sd = sd_lo + (int)(yy % n_sd);
    const long long r = (long long)sd * nlam + a;
    if (r < row0 || r >= row0 + nrows) continue;
    const int s = sd / nd, d = sd % nd;
    const E* fs = ps + ((size_t)a * ns + s) * N;
    const E* fd = pd + ((size_t)a * nd + d) * N;
    E* row = J + (size_t)(r - row0) * ldJ;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
      E hv = fs[x] * fd[x];
      for (int c = 0; c < nc; ++c) row[(size_t)c * N + x] = (E)(-h3 * eps[(size_t)(lam0 + a) * nc + c]) * hv;
    }
  }
}

// ---------------------------------------------------------------- J x
// Block = (wavelength a, chunk of spb x AP_XC voxels, TILE x TILE tile of (s, d), TILE = 4U
// with U in {8, 6, 4, 2} chosen per problem so that the tiles pad n_src and n_det little). Each stage of
// AP_XC voxels (phi_s and phi_d rows of the tile, and the chromophore maps x_c) is copied into
// shared memory with cp.async two stages ahead of the one being contracted (three buffers). 256 threads =
// 16 voxel groups x 16 (s, d) sub-tiles; a thread accumulates s-rows si0 + 4u and d-rows
// di0 + 4v (u, v < U), which with a row stride of AP_XC + 16 bytes keeps the tile reads of a warp
// on distinct banks. mu_a(x) = sum_c eps_c(lambda_a) x_c is formed by each thread for its voxels.
// Block partials go to a workspace and a second kernel sums them in a fixed order.
constexpr int AP_XC = 128;   // voxels per stage
constexpr int AP_STAGES = 8; // stages per block of the allocation-free entry point (the library picks
                              // 4 .. 64 per problem, see apply_spb)
constexpr int AP_NBUF = 3;    // stage buffers: two stages in flight while one is contracted

template <typename E>
__host__ __device__ constexpr int ap_ld() { return AP_XC + 16 / (int)sizeof(E); }  // padded row stride (elements)
// elements of one stage buffer: S [TILE][LD], D [TILE][LD], X [nc][AP_XC]
template <typename E, int U>
__host__ __device__ constexpr size_t apply_buf_elems(int nc) {
  return (size_t)8 * U * ap_ld<E>() + (size_t)nc * AP_XC;
}
// Narrow tiles (U <= 6, FP32) need fewer registers: three blocks per SM with a two-stage ring
// (three stages would not fit three blocks' shared memory); U = 8 keeps two blocks and three stages.
template <typename E, int U>
__host__ __device__ constexpr int apply_nbuf() { return (U <= 6 && sizeof(E) == 4) ? 2 : AP_NBUF; }
template <typename E, int U>
__host__ __device__ constexpr int apply_min_blocks() { return sizeof(E) == 4 ? (U <= 6 ? 3 : 2) : 1; }
template <typename E, int U>
size_t apply_smem_bytes(int nc) {
  return std::max(sizeof(E) * apply_nbuf<E, U>() * apply_buf_elems<E, U>(nc), sizeof(E) * 8 * 1024);  // the reduction reuses it
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
template <int B>
__device__ __forceinline__ void cp_async_small(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "n"(B), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N_>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N_) : "memory"); }

template <typename E, int U>
__global__ void __launch_bounds__(256, apply_min_blocks<E, U>()) k_apply_partial(const E* __restrict__ ps, const E* __restrict__ pd,
                                                       const E* __restrict__ xin, const double* __restrict__ eps,
                                                       int lam0, int ns, int nd, int nc, long long N, int nxb, int spb,
                                                       int vec, E* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int LD = ap_ld<E>();
  constexpr int VE = 16 / (int)sizeof(E);  // elements per 16-byte copy
  constexpr int TILE = 4 * U;
  E* buf0 = reinterpret_cast<E*>(smraw);   // per buffer: S [TILE][LD], D [TILE][LD], X [nc][AP_XC]
  E* red = buf0;                           // [8][1024], reused after the voxel loop
  const int xb = blockIdx.x;
  const int a = blockIdx.y;
  const int tsd = blockIdx.z;  // (s-tile, d-tile)
  const int nts = (ns + TILE - 1) / TILE;
  const int s0 = (tsd % nts) * TILE, d0 = (tsd / nts) * TILE;
  const int t = threadIdx.x;
  const int grp = t / 16, sub = t % 16;
  const int si0 = sub / 4, di0 = sub % 4;
  __shared__ E w[MAXC];  // eps_c(lambda_a)
  __shared__ __align__(16) E mu[AP_XC];  // mu_a of the stage's voxels
  if (t < nc) w[t] = (E)eps[(size_t)(lam0 + a) * nc + t];
  const E* srow = ps + ((size_t)a * ns + s0) * N;
  const E* drow = pd + ((size_t)a * nd + d0) * N;
  auto load = [&](int st, E* b) {
    const long long xbase = ((long long)xb * spb + st) * AP_XC;
    E* S = b;
    E* D = b + TILE * LD;
    E* X = b + 2 * TILE * LD;
    if (vec) {
      // thread t copies 16-byte chunk t % CH of rows t / CH + RPI * i of S, D and X
      constexpr int CH = AP_XC / VE;  // 16-byte chunks per row
      constexpr int RPI = 256 / CH;   // rows per pass of the block
      const int r0 = t / CH, col = (t % CH) * VE;
      const long long x = xbase + col;
      const bool xok = x < N;  // N is a multiple of VE here: a chunk is inside or outside as a whole
      const E* sp = srow + (size_t)r0 * N + x;
      const E* dp = drow + (size_t)r0 * N + x;
#pragma unroll
      for (int i = 0; i < TILE / RPI; ++i) {
        const bool ok = xok && s0 + r0 + RPI * i < ns;
        cp_async16(S + (r0 + RPI * i) * LD + col, ok ? (const void*)(sp + (size_t)RPI * i * N) : (const void*)xin,
                   ok ? 16u : 0u);
      }
#pragma unroll
      for (int i = 0; i < TILE / RPI; ++i) {
        const bool ok = xok && d0 + r0 + RPI * i < nd;
        cp_async16(D + (r0 + RPI * i) * LD + col, ok ? (const void*)(dp + (size_t)RPI * i * N) : (const void*)xin,
                   ok ? 16u : 0u);
      }
      for (int r = r0; r < nc; r += RPI)
        cp_async16(X + r * AP_XC + col, xok ? (const void*)(xin + (size_t)r * N + x) : (const void*)xin, xok ? 16u : 0u);
    } else {
      for (int q = t; q < (2 * TILE + nc) * AP_XC; q += 256) {
        const int row = q / AP_XC, col = q % AP_XC;
        const long long x = xbase + col;
        const E* src;
        E* dst;
        bool ok;
        if (row < TILE) {
          ok = s0 + row < ns;
          src = srow + (size_t)row * N + x;
          dst = S + row * LD + col;
        } else if (row < 2 * TILE) {
          ok = d0 + row - TILE < nd;
          src = drow + (size_t)(row - TILE) * N + x;
          dst = D + (row - TILE) * LD + col;
        } else {
          ok = true;
          src = xin + (size_t)(row - 2 * TILE) * N + x;
          dst = X + (row - 2 * TILE) * AP_XC + col;
        }
        ok = ok && x < N;
        cp_async_small<(int)sizeof(E)>(dst, ok ? src : xin, ok ? (uint32_t)sizeof(E) : 0u);
      }
    }
    cp_async_commit();
  };
  E acc[U][U];
#pragma unroll
  for (int u = 0; u < U; ++u)
#pragma unroll
    for (int v = 0; v < U; ++v) acc[u][v] = 0;
  const long long nstage = min((long long)spb, (N - (long long)xb * spb * AP_XC + AP_XC - 1) / AP_XC);
  const size_t be = apply_buf_elems<E, U>(nc);  // elements per stage buffer
  constexpr int NB = apply_nbuf<E, U>();
  static_assert(NB == 2 || NB == 3, "two or three stage buffers");
  load(0, buf0);
  if (NB == 3 && nstage > 1) load(1, buf0 + be);
  for (int st = 0; st < nstage; ++st) {
    E* b = buf0 + (st % NB) * be;
    // stage st has landed (the copies still pending are stage st's and, with three buffers, the
    // next one's); after the barrier every thread is done with stage st - 1, whose buffer the copy
    // issued next refills, so one barrier per stage orders both
    if (NB == 3 && st + 1 < nstage) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
    if (st + NB - 1 < nstage) load(st + NB - 1, buf0 + ((st + NB - 1) % NB) * be);
    const E* S = b;
    const E* D = b + TILE * LD;
    const E* X = b + 2 * TILE * LD;
    if constexpr (sizeof(E) == 4) {
      // scale the source rows by mu once, then contract 4-voxel quads with 16-byte reads:
      // per quad 8 + 8 vector reads feed 256 FMAs. Thread t scales voxel quad t % 32 of rows
      // t / 32 + 8i and forms mu for those 4 voxels itself.
      {
        const int cq = 4 * (t & 31), r0 = t >> 5;
        float4 m4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = 0; c < nc; ++c) {
          const float4 x4 = *reinterpret_cast<const float4*>(X + c * AP_XC + cq);
          m4.x = fmaf(w[c], x4.x, m4.x); m4.y = fmaf(w[c], x4.y, m4.y);
          m4.z = fmaf(w[c], x4.z, m4.z); m4.w = fmaf(w[c], x4.w, m4.w);
        }
#pragma unroll
        for (int i = 0; i < TILE / 8; ++i) {
          float4* sp = reinterpret_cast<float4*>(const_cast<E*>(S) + (r0 + 8 * i) * LD + cq);
          float4 v4 = *sp;
          v4.x *= m4.x; v4.y *= m4.y; v4.z *= m4.z; v4.w *= m4.w;
          *sp = v4;
        }
      }
      __syncthreads();
      // quads of warp w = grp / 2: (w / 2) * 8 + (w % 2) * 2 + {0, 1, 4, 5}, the odd group 4 quads
      // (16 banks) after the even one; with the 4-bank row skew the 8 distinct 16-byte words a
      // warp reads cover the 32 banks once
      const int qbase = (grp >> 2) * 8 + ((grp >> 1) & 1) * 2 + (grp & 1) * 4;
#pragma unroll 1
      for (int qd = 0; qd < 2; ++qd) {
        const int x0 = (qbase + qd) * 4;
        float4 dv[U];
#pragma unroll
        for (int v = 0; v < U; ++v) dv[v] = *reinterpret_cast<const float4*>(D + (di0 + 4 * v) * LD + x0);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const float4 sv = *reinterpret_cast<const float4*>(S + (si0 + 4 * u) * LD + x0);
#pragma unroll
          for (int v = 0; v < U; ++v) {
            acc[u][v] = fmaf(sv.x, dv[v].x, acc[u][v]);
            acc[u][v] = fmaf(sv.y, dv[v].y, acc[u][v]);
            acc[u][v] = fmaf(sv.z, dv[v].z, acc[u][v]);
            acc[u][v] = fmaf(sv.w, dv[v].w, acc[u][v]);
          }
        }
      }
    } else {
      if (t < AP_XC) {
        E m = 0;
        for (int c = 0; c < nc; ++c) m += w[c] * X[c * AP_XC + t];
        mu[t] = m;
      }
      __syncthreads();
      for (int q = grp; q < AP_XC; q += 16) {
        const E m = mu[q];
        E sv[U], dv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) sv[u] = S[(si0 + 4 * u) * LD + q] * m;
#pragma unroll
        for (int v = 0; v < U; ++v) dv[v] = D[(di0 + 4 * v) * LD + q];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int v = 0; v < U; ++v) acc[u][v] += sv[u] * dv[v];
      }
    }
  }
  // tree reduction over the 16 voxel groups (fixed order -> deterministic)
  for (int half = 8; half >= 1; half >>= 1) {
    __syncthreads();
    // element (u, v) of sub-tile `sub` at (u*U + v)*16 + sub: the 16 sub-tiles of a voxel group
    // hit 16 consecutive words
    if (grp >= half && grp < 2 * half) {
      E* dst = red + (size_t)(grp - half) * 1024 + sub;
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) dst[(u * U + v) * 16] = acc[u][v];
    }
    __syncthreads();
    if (grp < half) {
      const E* src = red + (size_t)grp * 1024 + sub;
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int v = 0; v < U; ++v) acc[u][v] += src[(u * U + v) * 16];
    }
  }
  if (grp == 0) {
    E* out = part + (((size_t)a * gridDim.z + tsd) * nxb + xb) * 1024;
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int v = 0; v < U; ++v) out[(si0 + 4 * u) * 32 + (di0 + 4 * v)] = acc[u][v];
  }
}

// 16-byte copies need 16-byte aligned rows: N * element size a multiple of 16 and aligned bases.
inline int apply_vec_ok(const void* a, const void* b, const void* c, long long N, size_t es) {
  const auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  return ((N * (long long)es) % 16 == 0 && al(a) && al(b) && al(c)) ? 1 : 0;
}

// Block = one source row (32 slots) of one (wavelength, optode tile) partial block; its 8 warps
// take every 8th voxel block (reads of 128 contiguous bytes per warp) and the 8 FP64 sums are added
// in warp order, so the result does not depend on scheduling. A partial block holds the tile's
// entry (s, d) at slot s * 32 + d; slots with d >= tile are never written, and their sums are dropped.
template <typename E>
__global__ void __launch_bounds__(256) k_apply_reduce(const E* __restrict__ part, int nlam, int ns, int nd, int nts,
                                                      int ntd, int tile_w, int nxb, double h3, E* __restrict__ y) {
  __shared__ double red[8][32];
  const int ntile = nts * ntd;
  const int sl = (int)(blockIdx.x % tile_w);
  const long long at = blockIdx.x / tile_w;  // a * ntile + tile
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const E* p = part + (size_t)at * nxb * 1024 + sl * 32 + lane;
  double sum = 0.0;
#pragma unroll 4
  for (int xb = w; xb < nxb; xb += 8) sum += (double)p[(size_t)xb * 1024];
  red[w][lane] = sum;
  __syncthreads();
  if (w == 0) {
    double tot = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) tot += red[i][lane];
    const int a = (int)(at / ntile), tile = (int)(at % ntile);
    const int s = (tile % nts) * tile_w + sl, d = (tile / nts) * tile_w + lane;
    if (lane < tile_w && s < ns && d < nd) y[((size_t)s * nd + d) * nlam + a] = (E)(-h3 * tot);
  }
}

template <typename E>
cudaError_t launch_apply_reduce(const E* part, int nlam, int ns, int nd, int nts, int ntd, int tile_w, int nxb,
                                double h3, E* y, cudaStream_t st) {
  const unsigned blocks = (unsigned)((size_t)nlam * nts * ntd * tile_w);
  k_apply_reduce<E><<<blocks, 256, 0, st>>>(part, nlam, ns, nd, nts, ntd, tile_w, nxb, h3, y);
  return cudaGetLastError();
}

// J x tile width 4U: per voxel quad a tile costs 4 U^2 FMAs, 2U shared reads and about 8 issue
// slots of staging, so pick the U with the fewest tiles x (4 U^2 + 2U + 8)
int apply_u(int ns, int nd) {
  int best = 8;
  long long cost = -1;
  for (int u : {8, 6, 4, 2}) {
    const long long c = (long long)((ns + 4 * u - 1) / (4 * u)) * ((nd + 4 * u - 1) / (4 * u)) * (4 * u * u + 2 * u + 8);
    if (cost < 0 || c < cost) best = u, cost = c;
  }
  return best;
}

template <typename E, int U>
cudaError_t launch_apply_partial(dim3 grid, cudaStream_t st, const E* ps, const E* pd, const E* x, const double* eps,
                                 int lam0, int ns, int nd, int nc, long long N, int nxb, int spb, int vec, E* part) {
  const size_t smem = apply_smem_bytes<E, U>(nc);
  cudaError_t e = raise_smem_limit(k_apply_partial<E, U>, smem);
  if (e != cudaSuccess) return e;
  k_apply_partial<E, U><<<grid, 256, smem, st>>>(ps, pd, x, eps, lam0, ns, nd, nc, N, nxb, spb, vec, part);
  return cudaGetLastError();
}

template <typename E>
cudaError_t launch_apply_partial_u(int u, dim3 grid, cudaStream_t st, const E* ps, const E* pd, const E* x,
                                   const double* eps, int lam0, int ns, int nd, int nc, long long N, int nxb, int spb,
                                   int vec, E* part) {
  switch (u) {
    case 6: return launch_apply_partial<E, 6>(grid, st, ps, pd, x, eps, lam0, ns, nd, nc, N, nxb, spb, vec, part);
    case 4: return launch_apply_partial<E, 4>(grid, st, ps, pd, x, eps, lam0, ns, nd, nc, N, nxb, spb, vec, part);
    case 2: return launch_apply_partial<E, 2>(grid, st, ps, pd, x, eps, lam0, ns, nd, nc, N, nxb, spb, vec, part);
    default: return launch_apply_partial<E, 8>(grid, st, ps, pd, x, eps, lam0, ns, nd, nc, N, nxb, spb, vec, part);
  }
}

// Stages (of AP_XC voxels) per block of the J x kernel. Its blocks are bound by instruction issue
// on their SM, so a partial last wave of blocks takes as long as a full one: the count chosen is
// the one with the fewest whole waves x (stages per block + about two stages of per-block cost: the
// pipeline fill, the block reduction and its partial write). 1,536 blocks of 16 stages on 304
// resident slots (5.05 waves) take as long as six full waves; 608 blocks of 41 stages fill two.
int apply_spb(long long N, int nlam, int ntiles, int resident) {
  const long long nst = (N + AP_XC - 1) / AP_XC;
  int best = 4;
  double best_t = 0.0;
  for (int spb = 4; spb <= 64; ++spb) {
    const long long nxb = (nst + spb - 1) / spb;
    const long long waves = (nxb * nlam * ntiles + resident - 1) / resident;
    const double t = (double)waves * (spb + 2.0);
    if (spb == 4 || t < best_t) best = spb, best_t = t;
  }
  return best;
}

// SMs of the current GPU
int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0)
    sms = 152;
  return sms;
}

// resident blocks of the J x kernel on this GPU for tile parameter u (the launch bounds fix the
// blocks per SM: two at u = 8 and three below in FP32, one in FP64)
template <typename E>
int apply_resident(int u) {
  return device_sms() * (u == 8 ? apply_min_blocks<E, 8>() : apply_min_blocks<E, 6>());
}

// ---------------------------------------------------------------- J^T y
// Thread per voxel; loops over the wavelengths of its group. Per wavelength and block of (up to)
// 32 detectors x 32 sources, the thread first loads the 64 field values of its voxel (independent
// coalesced loads, all in flight together), then t_a += sum_s phi_s (sum_d Y_a[s][d] phi_d) with
// Y_a in shared memory (rows padded to a multiple of 4, read as 16-byte broadcasts), and
// acc_c += eps_c(lambda_a) t_a.
constexpr int AT_B = 32;

template <typename E>
__host__ __device__ constexpr int at_ld(int nd) { return (nd + 3) / 4 * 4; }  // padded row of Y

// FULL: n_src and n_det are multiples of 32 (no guards inside the blocks)
template <typename E, bool FULL>
__global__ void __launch_bounds__(256, 2) k_apply_T_partial(const E* __restrict__ ps, const E* __restrict__ pd,
                                                         const E* __restrict__ y, const double* __restrict__ eps,
                                                         int lam0, int nlam, int ns, int nd, int nc, long long N,
                                                         int lam_per_group, E* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int LDY = at_ld<E>(nd);
  E* Y = reinterpret_cast<E*>(smraw);          // [ns][LDY] of one wavelength, zero-padded
  E* Tl = Y + (size_t)ns * LDY;                // [wavelengths of the group][256]: t_a per voxel
  const int grp = blockIdx.y;
  const int a0 = grp * lam_per_group, a1 = min(nlam, a0 + lam_per_group);
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = x < N;
  for (int a = a0; a < a1; ++a) {
    __syncthreads();
    for (int q = threadIdx.x; q < ns * LDY; q += blockDim.x) {
      const int s = q / LDY, d = q % LDY;
      Y[q] = d < nd ? y[((size_t)s * nd + d) * nlam + a] : (E)0;
    }
    __syncthreads();
    E ta = 0;
    if (in) {
      for (int d0 = 0; d0 < nd; d0 += AT_B) {
        const int dn = FULL ? AT_B : min(AT_B, nd - d0);
        E fd[AT_B];
#pragma unroll
        for (int q = 0; q < AT_B; ++q) fd[q] = (q < dn) ? pd[((size_t)a * nd + d0 + q) * N + x] : (E)0;
        const int dq = FULL ? AT_B / 4 : (dn + 3) / 4;  // 4-wide groups of Y within this detector block
        for (int s0 = 0; s0 < ns; s0 += AT_B) {
          const int sn = FULL ? AT_B : min(AT_B, ns - s0);
          E fs[AT_B];
#pragma unroll
          for (int q = 0; q < AT_B; ++q) fs[q] = (q < sn) ? ps[((size_t)a * ns + s0 + q) * N + x] : (E)0;
#pragma unroll
          for (int s = 0; s < AT_B; ++s) {
            if (s >= sn) break;
            const E* Ys = Y + (size_t)(s0 + s) * LDY + d0;
            E z = 0;
            if constexpr (sizeof(E) == 4) {
              // four independent partial sums (no serial chain of 32 dependent FMAs)
              float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
              for (int g = 0; g < AT_B / 4; ++g) {
                if (g < dq) {
                  const float4 yv = *reinterpret_cast<const float4*>(Ys + 4 * g);
                  z0 = fmaf(yv.x, fd[4 * g], z0);
                  z1 = fmaf(yv.y, fd[4 * g + 1], z1);
                  z2 = fmaf(yv.z, fd[4 * g + 2], z2);
                  z3 = fmaf(yv.w, fd[4 * g + 3], z3);
                }
              }
              z = (z0 + z1) + (z2 + z3);
            } else {
#pragma unroll
              for (int q = 0; q < AT_B; ++q)
                if (q < dn) z += Ys[q] * fd[q];
            }
            ta += fs[s] * z;
          }
        }
      }
    }
    Tl[(a - a0) * 256 + threadIdx.x] = ta;
  }
  // acc_c = sum_a eps_c(lambda_a) t_a (the t_a wait in shared memory, not in registers)
  if (in)
    for (int c = 0; c < nc; ++c) {
      E acc = 0;
      for (int a = a0; a < a1; ++a) acc += (E)eps[(size_t)(lam0 + a) * nc + c] * Tl[(a - a0) * 256 + threadIdx.x];
      part[((size_t)grp * nc + c) * N + x] = acc;
    }
}

// Register-tiled variant (FP32, up to 4 chromophores, N a multiple of 4). Block = 256-voxel chunk x
// group of wavelengths; 256 threads = 64 voxel quads x 4 source groups (thread t: quad t / 4, group
// t % 4). The sources are taken in tiles of 4 * SPT; a thread owns SPT sources of the tile and the
// 4 voxels of its quad and accumulates W[s][x] = sum_d Y_a[s][d] phi_d(x) over detector chunks of
// TT_DC, staged (phi_d rows of the chunk and Y_a of the tile) in shared memory by cp.async, two
// stages in flight. Per detector a warp reads one 16-byte word of phi_d per quad (8 quads: 128
// contiguous bytes) and two of Y (4 groups: distinct banks) for 4 * SPT FMAs. After the last chunk
// of a tile t_a(x) += sum_s phi_s(x) W[s][x] with phi_s read from global memory straight into
// registers (issued before the detector loop), and after the last tile of a wavelength
// acc_c(x) += eps_c(lambda_a) t_a(x). The 4 groups' partial sums are added by shuffles at the end.
constexpr int TT_XC = 256;  // voxels per block
constexpr int TT_DC = 32;   // detectors per stage
constexpr int TT_NC = 4;    // chromophores held in registers
constexpr size_t TT_STAGE_FLOATS = (size_t)TT_DC * TT_XC + (size_t)TT_DC * 32;  // phi_d chunk + Y tile
constexpr int TT_NBUF = 2;  // stage buffers: one stage in flight while one is contracted
constexpr size_t TT_SMEM = TT_NBUF * TT_STAGE_FLOATS * sizeof(float);

template <int SPT>
__global__ void __launch_bounds__(256, 2) k_apply_T_tile(const float* __restrict__ ps, const float* __restrict__ pd,
                                                      const float* __restrict__ yT, const double* __restrict__ eps,
                                                      int lam0, int nlam, int ns, int nd, int nc, long long N,
                                                      int lam_per_group, float* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float* buf0 = reinterpret_cast<float*>(smraw);
  float* epsf = buf0 + TT_NBUF * TT_STAGE_FLOATS;  // [lam_per_group][TT_NC] eps_c(lambda) of the group, FP32
  const int t = threadIdx.x;
  const int q = t >> 2, g = t & 3;
  const int grp = blockIdx.y;
  const int a0 = grp * lam_per_group, a1 = min(nlam, a0 + lam_per_group);
  const long long xb = (long long)blockIdx.x * TT_XC;
  const long long x0 = xb + 4 * q;
  const bool in = x0 < N;  // N % 4 == 0: a quad is inside or outside as a whole
  constexpr int ST = 4 * SPT;  // sources per tile
  const int nst = (ns + ST - 1) / ST, ndc = (nd + TT_DC - 1) / TT_DC;
  const int nstage = (a1 - a0) * nst * ndc;
  for (int e = t; e < (a1 - a0) * TT_NC; e += 256) {
    const int c = e % TT_NC;
    epsf[e] = c < nc ? (float)eps[(size_t)(lam0 + a0 + e / TT_NC) * nc + c] : 0.f;
  }
  // staging roles, fixed for the whole block: detector rows (t >> 6) + 4i at voxel column 4 (t & 63)
  // (i < 8); Y entries of detectors (t >> 5) + 8i (i < 4), source slot j = t & 7 of group (t & 31) >> 3
  const int dr = t >> 6, dcol = (t & 63) * 4;
  const bool dok = xb + dcol < N;
  const int yr = t >> 5, yg = (t & 31) >> 3, yj = t & 7;
  const size_t N4 = (size_t)4 * N;
  // stage k = ((a - a0) * nst + st) * ndc + dc, kept as counters rather than divisions
  int la = a0, lst = 0, ldc = 0;  // stage to load next
  auto load = [&](float* b) {
    const int d0 = ldc * TT_DC, dn = min(TT_DC, nd - d0);
    float* Dt = b + dr * TT_XC + dcol;
    const float* src = pd + ((size_t)la * nd + d0 + dr) * N + xb + dcol;
#pragma unroll
    for (int i = 0; i < TT_DC / 4; ++i) {
      if (dr + 4 * i < dn)
        cp_async16(Dt + i * 4 * TT_XC, dok ? (const void*)(src + i * N4) : (const void*)pd, dok ? 16u : 0u);
    }
    const int s = lst * ST + yg * SPT + yj;
    const bool sok = yj < SPT && s < ns;
    float* Yt = b + (size_t)TT_DC * TT_XC + yr * 32 + yg * 8 + yj;  // Y_a[s][d0 + d] at d*32 + group*8 + j
    // yT [nlam][nd][ns]: the sources of one detector are contiguous, a warp reads one 128-byte row
    const float* ysrc = yT + ((size_t)la * nd + d0 + yr) * ns + (sok ? s : 0);
#pragma unroll
    for (int i = 0; i < TT_DC / 8; ++i) {
      const bool ok = sok && yr + 8 * i < dn;
      cp_async_small<4>(Yt + i * 8 * 32, ok ? (const void*)(ysrc + (size_t)i * 8 * ns) : (const void*)yT,
                        ok ? 4u : 0u);
    }
    cp_async_commit();
    if (++ldc == ndc) {
      ldc = 0;
      if (++lst == nst) lst = 0, ++la;
    }
  };
  float acc[TT_NC][4], tacc[4], W[SPT][4];
  float4 fs[SPT];
#pragma unroll
  for (int c = 0; c < TT_NC; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[c][i] = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) tacc[i] = 0.f;
#pragma unroll
  for (int j = 0; j < SPT; ++j) {
    fs[j] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int i = 0; i < 4; ++i) W[j][i] = 0.f;
  }
  static_assert(TT_NBUF == 2 || TT_NBUF == 3, "two or three stage buffers");
  if (nstage > 0) load(buf0);
  if (TT_NBUF == 3 && nstage > 1) load(buf0 + TT_STAGE_FLOATS);
  int a = a0, st = 0, dc = 0;  // stage being contracted
  for (int k = 0; k < nstage; ++k) {
    if (dc == 0 && in) {  // phi_s of this tile: consumed after the tile's last detector chunk
      const int sb = st * ST + g * SPT;
      const float* sp = ps + ((size_t)a * ns + sb) * N + x0;
#pragma unroll
      for (int j = 0; j < SPT; ++j)
        fs[j] = sb + j < ns ? *reinterpret_cast<const float4*>(sp + (size_t)j * N) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float* b = buf0 + (k % TT_NBUF) * TT_STAGE_FLOATS;
    // stage k has landed; after the barrier every thread is done with stage k - 1, whose buffer
    // the copy issued next refills (one barrier per stage)
    if (TT_NBUF == 3 && k + 1 < nstage) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
    if (k + TT_NBUF - 1 < nstage) load(buf0 + ((k + TT_NBUF - 1) % TT_NBUF) * TT_STAGE_FLOATS);
    const float* Dt = b + 4 * q;
    const float* Yt = b + (size_t)TT_DC * TT_XC + g * 8;
    const int dn = min(TT_DC, nd - dc * TT_DC);
#pragma unroll 4
    for (int d = 0; d < dn; ++d) {
      const float4 f = *reinterpret_cast<const float4*>(Dt + d * TT_XC);
      const float4 ya = *reinterpret_cast<const float4*>(Yt + d * 32);
      float yv[8] = {ya.x, ya.y, ya.z, ya.w, 0.f, 0.f, 0.f, 0.f};
      if constexpr (SPT > 4) {
        const float4 yb = *reinterpret_cast<const float4*>(Yt + d * 32 + 4);
        yv[4] = yb.x; yv[5] = yb.y; yv[6] = yb.z; yv[7] = yb.w;
      }
#pragma unroll
      for (int j = 0; j < SPT; ++j) {
        W[j][0] = fmaf(yv[j], f.x, W[j][0]);
        W[j][1] = fmaf(yv[j], f.y, W[j][1]);
        W[j][2] = fmaf(yv[j], f.z, W[j][2]);
        W[j][3] = fmaf(yv[j], f.w, W[j][3]);
      }
    }
    if (dc == ndc - 1) {
#pragma unroll
      for (int j = 0; j < SPT; ++j) {
        tacc[0] = fmaf(fs[j].x, W[j][0], tacc[0]);
        tacc[1] = fmaf(fs[j].y, W[j][1], tacc[1]);
        tacc[2] = fmaf(fs[j].z, W[j][2], tacc[2]);
        tacc[3] = fmaf(fs[j].w, W[j][3], tacc[3]);
#pragma unroll
        for (int i = 0; i < 4; ++i) W[j][i] = 0.f;
      }
      if (st == nst - 1) {
        const float4 e4 = *reinterpret_cast<const float4*>(epsf + (a - a0) * TT_NC);
        const float ev[TT_NC] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
        for (int c = 0; c < TT_NC; ++c)
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[c][i] = fmaf(ev[c], tacc[i], acc[c][i]);
#pragma unroll
        for (int i = 0; i < 4; ++i) tacc[i] = 0.f;
      }
    }
    if (++dc == ndc) {
      dc = 0;
      if (++st == nst) st = 0, ++a;
    }
  }
  // sum the 4 source groups of a quad (lanes 4q' .. 4q' + 3 of a warp), fixed order
#pragma unroll
  for (int c = 0; c < TT_NC; ++c)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      acc[c][i] += __shfl_xor_sync(0xffffffffu, acc[c][i], 1);
      acc[c][i] += __shfl_xor_sync(0xffffffffu, acc[c][i], 2);
    }
  if (in && g < nc) {
    float4 o;
    // lane g writes chromophore g (g < nc <= 4)
    o.x = g == 0 ? acc[0][0] : g == 1 ? acc[1][0] : g == 2 ? acc[2][0] : acc[3][0];
    o.y = g == 0 ? acc[0][1] : g == 1 ? acc[1][1] : g == 2 ? acc[2][1] : acc[3][1];
    o.z = g == 0 ? acc[0][2] : g == 1 ? acc[1][2] : g == 2 ? acc[2][2] : acc[3][2];
    o.w = g == 0 ? acc[0][3] : g == 1 ? acc[1][3] : g == 2 ? acc[2][3] : acc[3][3];
    *reinterpret_cast<float4*>(part + ((size_t)grp * nc + g) * N + x0) = o;
  }
}


template <typename E>
__global__ void k_apply_T_reduce(const E* __restrict__ part, int ngrp, int nc, long long N, double h3,
                                 E* __restrict__ g) {
  long long total = (long long)nc * N;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    E sum = 0;
    for (int gg = 0; gg < ngrp; ++gg) sum += part[(size_t)gg * total + q];
    g[q] += (E)(-h3) * sum;
  }
}

int check_slice(hydot_ctx* ctx, int lam0, int nlam) {
  if (ctx->cplx) return fail(ctx, HYDOT_ERR_STATE, "Born products are defined for continuous-wave (real) fields only");
  if (lam0 < 0 || nlam < 1 || lam0 + nlam > ctx->n_lambda) return fail(ctx, HYDOT_ERR_ARG, "wavelength slice out of range");
  if (ctx->n_chrom > MAXC) return fail(ctx, HYDOT_ERR_ARG, "too many chromophores");
  return HYDOT_OK;
}

template <typename E>
int assemble_t(hydot_ctx* ctx, const E* ps, const E* pd, int lam0, int nlam, long long row0, long long nrows, E* J,
               long long ldJ) {
  const long long N = ctx->N;
  const int ns = ctx->n_src, nd = ctx->n_det, nc = ctx->n_chrom;
  const double h3 = ctx->h * ctx->h * ctx->h;
  const int sd_lo = (int)(row0 / nlam);
  const int sd_hi = (int)((row0 + nrows - 1) / nlam);
  const int n_sd = sd_hi - sd_lo + 1;
  const long long total_rows = (long long)nlam * n_sd;
  constexpr int VEC = sizeof(E) == 4 ? 4 : 2;
  const bool aligned = (N % VEC == 0) && ((uintptr_t)J % 16 == 0) && ((ldJ * (long long)sizeof(E)) % 16 == 0) &&
                       ((uintptr_t)ps % 16 == 0) && ((uintptr_t)pd % 16 == 0);
  const long long per_row = aligned ? N / VEC : N;
  unsigned gx = (unsigned)std::max<long long>(1, std::min<long long>((per_row + 1023) / 1024, 1024));
  unsigned gy = (unsigned)std::min<long long>(total_rows, 65535);
  dim3 grid(gx, gy);
  cudaEvent_t t0 = timer_begin(ctx);
  if (aligned)
    k_born_rows<E, VEC><<<grid, 256, 0, ctx->stream>>>(ps, pd, ctx->d_eps, lam0, nlam, ns, nd, nc, N, h3, row0, nrows,
                                                       sd_lo, n_sd, J, ldJ);
  else
    k_born_rows_scalar<E><<<grid, 256, 0, ctx->stream>>>(ps, pd, ctx->d_eps, lam0, nlam, ns, nd, nc, N, h3, row0,
                                                         nrows, sd_lo, n_sd, J, ldJ);
  ++ctx->launches;
  timer_end(ctx, t0, HYDOT_KERNEL_BORN_ROWS, (double)nrows * nc * (double)N * sizeof(E));
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  return HYDOT_OK;
}

int ensure_ws(hydot_ctx* ctx, size_t bytes) {
  if (ctx->apply_ws_bytes >= bytes) return HYDOT_OK;
  if (ctx->d_apply_ws) {
    // the previous workspace may still be used by queued work on this stream
    HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->d_apply_ws);
    ctx->d_apply_ws = nullptr;
    ctx->apply_ws_bytes = 0;
  }
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_apply_ws, bytes));
  ctx->apply_ws_bytes = bytes;
  return HYDOT_OK;
}

template <typename E>
int apply_t(hydot_ctx* ctx, const E* ps, const E* pd, int lam0, int nlam, const E* x, E* y) {
  const long long N = ctx->N;
  const int ns = ctx->n_src, nd = ctx->n_det, nc = ctx->n_chrom;
  const int u = apply_u(ns, nd), tw = 4 * u;
  const int nts = (ns + tw - 1) / tw, ntd = (nd + tw - 1) / tw;
  const int spb = apply_spb(N, nlam, nts * ntd, apply_resident<E>(u));
  const long long per_blk = (long long)AP_XC * spb;
  const int nxb = (int)((N + per_blk - 1) / per_blk);
  size_t bytes = sizeof(E) * (size_t)nlam * nts * ntd * nxb * 1024;
  int rc = ensure_ws(ctx, bytes);
  if (rc) return rc;
  E* part = (E*)ctx->d_apply_ws;
  dim3 grid(nxb, nlam, nts * ntd);
  const int vec = apply_vec_ok(ps, pd, x, N, sizeof(E));
  cudaEvent_t t0 = timer_begin(ctx);
  HYDOT_CUDA_TRY(ctx, launch_apply_partial_u<E>(u, grid, ctx->stream, ps, pd, x, ctx->d_eps, lam0, ns, nd, nc, N,
                                                nxb, spb, vec, part));
  ++ctx->launches;
  HYDOT_CUDA_TRY(ctx, launch_apply_reduce<E>(part, nlam, ns, nd, nts, ntd, tw, nxb, ctx->h * ctx->h * ctx->h, y,
                                              ctx->stream));
  ++ctx->launches;
  timer_end(ctx, t0, HYDOT_KERNEL_APPLY, ((double)nlam * (ns + nd) + nc) * (double)N * sizeof(E));
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  return HYDOT_OK;
}

// yT[(a * nd + d) * ns + s] = y[(s * nd + d) * nlam + a]: the slice's residual with the sources of
// each (wavelength, detector) contiguous, for the register-tiled J^T y kernel's staging
__global__ void k_transpose_y(const float* __restrict__ y, int nlam, int ns, int nd, float* __restrict__ yT) {
  const long long M = (long long)nlam * ns * nd;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < M; r += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(r % ns);
    const long long ad = r / ns;
    const int d = (int)(ad % nd), a = (int)(ad / nd);
    yT[r] = y[((size_t)s * nd + d) * nlam + a];
  }
}

// sources per thread of the register-tiled J^T y kernel: per detector a source tile costs 4 * SPT
// FMAs plus about 6 issue slots of loads and addressing, so pick the SPT with the fewest
// tiles x (4 * SPT + 6)
int tile_spt(int ns) {
  int best = 8, cost = 1 << 30;
  for (int spt : {8, 6, 4, 2}) {
    const int c = (ns + 4 * spt - 1) / (4 * spt) * (4 * spt + 6);
    if (c < cost) best = spt, cost = c;
  }
  return best;
}

int apply_T_tile(hydot_ctx* ctx, const float* ps, const float* pd, int lam0, int nlam, const float* y, float* g) {
  const long long N = ctx->N;
  const int ns = ctx->n_src, nd = ctx->n_det, nc = ctx->n_chrom;
  const long long xblocks = (N + TT_XC - 1) / TT_XC;
  // wavelength groups (each writes its own partial sums). Among the counts that give at least four
  // waves of two blocks per SM (fewer leave HBM idle in the last wave: one group of 768 blocks on
  // 304 slots, 2.53 waves, ran 5 % slower than two), the one with the fewest whole waves x
  // (wavelengths per block + about one of per-block cost); with none, the most waves
  const long long resident = 2LL * device_sms();
  int lpg = nlam;
  double best = -1.0;
  long long most = -1;
  int lpg_most = 1;
  for (int ng = 1; ng <= nlam; ++ng) {
    const int l = (nlam + ng - 1) / ng, ngr = (nlam + l - 1) / l;
    const long long blocks = xblocks * ngr;
    if (blocks > most) most = blocks, lpg_most = l;
    if (blocks < 4 * resident) continue;
    const double t = (double)((blocks + resident - 1) / resident) * (l + 1.0);
    if (best < 0.0 || t < best) best = t, lpg = l;
  }
  if (best < 0.0) lpg = lpg_most;
  const int ngrp = (nlam + lpg - 1) / lpg;
  const size_t part_elems = (size_t)ngrp * nc * N;
  const long long M = (long long)nlam * ns * nd;
  int rc = ensure_ws(ctx, sizeof(float) * (part_elems + (size_t)M));
  if (rc) return rc;
  float* part = (float*)ctx->d_apply_ws;
  float* yT = part + part_elems;
  const int spt = tile_spt(ns);
  auto kern = spt == 8 ? k_apply_T_tile<8> : spt == 6 ? k_apply_T_tile<6> : spt == 4 ? k_apply_T_tile<4>
                                                                                      : k_apply_T_tile<2>;
  const size_t smem = TT_SMEM + sizeof(float) * (size_t)lpg * TT_NC;
  if (smem > 200 * 1024) return fail(ctx, HYDOT_ERR_ARG, "too many wavelengths per J^T y call");
  HYDOT_CUDA_TRY(ctx, raise_smem_limit(kern, smem));
  dim3 grid((unsigned)xblocks, ngrp);
  cudaEvent_t t0 = timer_begin(ctx);
  k_transpose_y<<<(unsigned)std::min<long long>((M + 255) / 256, 4096), 256, 0, ctx->stream>>>(y, nlam, ns, nd, yT);
  ++ctx->launches;
  kern<<<grid, 256, smem, ctx->stream>>>(ps, pd, yT, ctx->d_eps, lam0, nlam, ns, nd, nc, N, lpg, part);
  ++ctx->launches;
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  long long tot = (long long)nc * N;
  k_apply_T_reduce<float><<<(unsigned)std::min<long long>((tot + 255) / 256, 8192), 256, 0, ctx->stream>>>(
      part, ngrp, nc, N, ctx->h * ctx->h * ctx->h, g);
  ++ctx->launches;
  timer_end(ctx, t0, HYDOT_KERNEL_APPLY_T, ((double)nlam * (ns + nd) + 2.0 * nc) * (double)N * sizeof(float));
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  return HYDOT_OK;
}

template <typename E>
int apply_T_t(hydot_ctx* ctx, const E* ps, const E* pd, int lam0, int nlam, const E* y, E* g) {
  const long long N = ctx->N;
  const int ns = ctx->n_src, nd = ctx->n_det, nc = ctx->n_chrom;
  if constexpr (sizeof(E) == 4) {
    if (nc <= TT_NC && N % 4 == 0 && (uintptr_t)ps % 16 == 0 && (uintptr_t)pd % 16 == 0 && !getenv("HYDOT_NO_TILE_T"))
      return apply_T_tile(ctx, ps, pd, lam0, nlam, y, g);
  }
  // enough blocks to fill the GPU: split the wavelengths into groups with their own partials
  const long long xblocks = (N + 255) / 256;
  int ngrp = (int)std::max<long long>(1, std::min<long long>(nlam, (4 * 152 * 8 + xblocks - 1) / xblocks));
  const int lpg = (nlam + ngrp - 1) / ngrp;
  ngrp = (nlam + lpg - 1) / lpg;
  size_t bytes = sizeof(E) * (size_t)ngrp * nc * N;
  int rc = ensure_ws(ctx, bytes);
  if (rc) return rc;
  E* part = (E*)ctx->d_apply_ws;
  dim3 grid((unsigned)xblocks, ngrp);
  // one wavelength's Y block and the per-wavelength t_a of the block's voxels
  const size_t smem = sizeof(E) * ((size_t)ns * at_ld<E>(nd) + (size_t)lpg * 256);
  if (smem > 200 * 1024) return fail(ctx, HYDOT_ERR_ARG, "n_src x n_det too large for the J^T y kernel");
  const bool full = ns % AT_B == 0 && nd % AT_B == 0;
  auto kern = full ? k_apply_T_partial<E, true> : k_apply_T_partial<E, false>;
  if (smem > 48 * 1024) {
    HYDOT_CUDA_TRY(ctx, raise_smem_limit(kern, smem));
  }
  cudaEvent_t t0 = timer_begin(ctx);
  kern<<<grid, 256, smem, ctx->stream>>>(ps, pd, y, ctx->d_eps, lam0, nlam, ns, nd, nc, N, lpg, part);
  ++ctx->launches;
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  long long tot = (long long)nc * N;
  k_apply_T_reduce<E><<<(unsigned)std::min<long long>((tot + 255) / 256, 8192), 256, 0, ctx->stream>>>(
      part, ngrp, nc, N, ctx->h * ctx->h * ctx->h, g);
  ++ctx->launches;
  timer_end(ctx, t0, HYDOT_KERNEL_APPLY_T, ((double)nlam * (ns + nd) + 2.0 * nc) * (double)N * sizeof(E));
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  return HYDOT_OK;
}

}  // namespace

int born_assemble_impl(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam, long long row0,
                       long long nrows, void* J, long long ldJ) {
  int rc = check_slice(ctx, lam0, nlam);
  if (rc) return rc;
  const long long M = (long long)ctx->n_src * ctx->n_det * nlam;
  if (!phi_src || !phi_det || !J) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  if (row0 < 0 || nrows < 0 || row0 + nrows > M) return fail(ctx, HYDOT_ERR_ARG, "row range outside the slice");
  if (ldJ < (long long)ctx->n_chrom * ctx->N) return fail(ctx, HYDOT_ERR_ARG, "ldJ < n_chrom*N");
  if (nrows == 0) return HYDOT_OK;
  if (ctx->precision == HYDOT_MIXED)
    return assemble_t<float>(ctx, (const float*)phi_src, (const float*)phi_det, lam0, nlam, row0, nrows, (float*)J, ldJ);
  return assemble_t<double>(ctx, (const double*)phi_src, (const double*)phi_det, lam0, nlam, row0, nrows, (double*)J,
                            ldJ);
}

int born_apply_impl(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam, const void* x,
                    void* y) {
  int rc = check_slice(ctx, lam0, nlam);
  if (rc) return rc;
  if (!phi_src || !phi_det || !x || !y) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  if (ctx->precision == HYDOT_MIXED)
    return apply_t<float>(ctx, (const float*)phi_src, (const float*)phi_det, lam0, nlam, (const float*)x, (float*)y);
  return apply_t<double>(ctx, (const double*)phi_src, (const double*)phi_det, lam0, nlam, (const double*)x, (double*)y);
}

// J^T y from the adjoint fields (Section 5, the gradient by one extra solve per source):
//   g[c*N + x] += -h^3 sum_a eps_c(lambda_a) sum_s phi_s[a][s][x] psi[a][s][x]
// with psi[a][s] = A^-1 (sum_d y[s,d,a] e_d) from hydot_solve_adjoint. One thread per voxel, the
// wavelengths and sources of the slice in a fixed order (the same bits on every run); reads each
// field value once, coalesced along x.
template <typename E>
__global__ void __launch_bounds__(256) k_apply_T_adjoint(const E* __restrict__ ps, const E* __restrict__ psi,
                                                        const double* __restrict__ eps, int lam0, int nlam, int ns,
                                                        int nc, long long N, E scale, E* __restrict__ g) {
  __shared__ E w[64 * MAXC];  // eps of up to 64 wavelengths of the slice at a time
  for (long long x0 = (long long)blockIdx.x * blockDim.x; x0 < N; x0 += (long long)gridDim.x * blockDim.x) {
    const long long x = x0 + threadIdx.x;
    E acc[MAXC];
#pragma unroll
    for (int c = 0; c < MAXC; ++c) acc[c] = E(0);
    for (int a0 = 0; a0 < nlam; a0 += 64) {
      const int na = min(64, nlam - a0);
      __syncthreads();
      for (int q = threadIdx.x; q < na * nc; q += blockDim.x) w[q] = (E)eps[(size_t)(lam0 + a0) * nc + q];
      __syncthreads();
      if (x < N) {
        for (int a = 0; a < na; ++a) {
          const size_t f0 = (size_t)(a0 + a) * ns;
          E t = E(0);
          for (int s = 0; s < ns; ++s) t = fma(ps[(f0 + s) * N + x], psi[(f0 + s) * N + x], t);
#pragma unroll
          for (int c = 0; c < MAXC; ++c)
            if (c < nc) acc[c] = fma(w[a * nc + c], t, acc[c]);
        }
      }
    }
    if (x < N) {
#pragma unroll
      for (int c = 0; c < MAXC; ++c)
        if (c < nc) g[(size_t)c * N + x] += scale * acc[c];
    }
  }
}

int born_apply_T_adjoint_impl(hydot_ctx* ctx, const void* phi_src, const void* psi, int lam0, int nlam, void* g) {
  int rc = check_slice(ctx, lam0, nlam);
  if (rc) return rc;
  if (!phi_src || !psi || !g) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  if (ctx->n_src < 1) return fail(ctx, HYDOT_ERR_STATE, "no sources");
  const double h3 = ctx->h * ctx->h * ctx->h;
  const unsigned blocks = (unsigned)std::min<long long>((ctx->N + 255) / 256, 152LL * 16);
  cudaEvent_t t0 = timer_begin(ctx);
  if (ctx->precision == HYDOT_MIXED)
    k_apply_T_adjoint<float><<<blocks, 256, 0, ctx->stream>>>((const float*)phi_src, (const float*)psi, ctx->d_eps, lam0,
                                                              nlam, ctx->n_src, ctx->n_chrom, ctx->N, (float)(-h3),
                                                              (float*)g);
  else
    k_apply_T_adjoint<double><<<blocks, 256, 0, ctx->stream>>>((const double*)phi_src, (const double*)psi, ctx->d_eps,
                                                               lam0, nlam, ctx->n_src, ctx->n_chrom, ctx->N, -h3,
                                                               (double*)g);
  ++ctx->launches;
  timer_end(ctx, t0, HYDOT_KERNEL_APPLY_T,
            2.0 * nlam * ctx->n_src * (double)ctx->N * (ctx->precision == HYDOT_MIXED ? 4.0 : 8.0));
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  return HYDOT_OK;
}

int born_apply_T_impl(hydot_ctx* ctx, const void* phi_src, const void* phi_det, int lam0, int nlam, const void* y,
                      void* g) {
  int rc = check_slice(ctx, lam0, nlam);
  if (rc) return rc;
  if (!phi_src || !phi_det || !y || !g) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  if (ctx->precision == HYDOT_MIXED)
    return apply_T_t<float>(ctx, (const float*)phi_src, (const float*)phi_det, lam0, nlam, (const float*)y, (float*)g);
  return apply_T_t<double>(ctx, (const double*)phi_src, (const double*)phi_det, lam0, nlam, (const double*)y,
                           (double*)g);
}

}  // namespace hydot

// ---------------------------------------------------------------- J x without device allocation
// For callers that cannot allocate device memory themselves (code running where cudaMalloc is
// not allowed, or under an allocator owned by someone else):
// the per-block partial sums of J x live in a fixed file-scope device array instead of a
// library workspace, and the wavelength slice's extinction coefficients are staged there too.
// Every GPU that loads the library holds this array until the process exits.
namespace {

constexpr size_t NOALLOC_EPS_BYTES = 64 * 1024;                 // eps slice: up to 8,192 doubles
constexpr size_t NOALLOC_PART_BYTES = 16u * 1024u * 1024u;      // J x partial sums: 16 MiB
constexpr size_t NOALLOC_BYTES = NOALLOC_EPS_BYTES + NOALLOC_PART_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
// device address of the array, per device; host threads may make their first call on a device at
// the same time, so each slot is atomic (both then look up the same address)
std::atomic<void*> g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

}  // namespace

extern "C" int hydot_born_apply_noalloc(long long N, int n_src, int n_det, int n_chrom, int nlam, double h_mm,
                                        const double* eps, const float* phi_src, const float* phi_det,
                                        const float* x, float* y, void* stream) {
  using namespace hydot;
  return abi_guard(nullptr, [&]() -> int {
    auto bad = [](const std::string& m) {
      set_context_free_error(m);
      return (int)HYDOT_ERR_ARG;
    };
    if (N < 1 || n_src < 1 || n_det < 1 || nlam < 1 || n_chrom < 1) return bad("sizes must be >= 1");
    if (n_chrom > MAXC) return bad("n_chrom must be <= 16");
    if (!(h_mm > 0.0)) return bad("h_mm must be > 0");
    if (!eps || !phi_src || !phi_det || !x || !y) return bad("null pointer");
    const size_t eps_bytes = sizeof(double) * (size_t)nlam * n_chrom;
    if (eps_bytes > NOALLOC_EPS_BYTES) return bad("nlam * n_chrom exceeds the static limit of 8192");
    const int nts = (n_src + 31) / 32, ntd = (n_det + 31) / 32;
    const long long per_blk = (long long)AP_XC * AP_STAGES;
    const long long nxb = (N + per_blk - 1) / per_blk;
    const double part_bytes = 4.0 * (double)nlam * nts * ntd * (double)nxb * 1024.0;
    if (part_bytes > (double)NOALLOC_PART_BYTES)
      return bad("nlam * ceil(n_src/32) * ceil(n_det/32) * ceil(N/1024) * 4 KiB exceeds the 16 MiB static scratch");
    if (nlam > 65535 || nts * ntd > 65535) return bad("too many wavelengths or optode tiles for one launch");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
      set_context_free_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
      return HYDOT_ERR_CUDA;
    }
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
      set_context_free_error("device index " + std::to_string(dev) + " exceeds the 64 devices this call supports");
      return HYDOT_ERR_CUDA;
    }
    // once per device, with that device current: the array's device address (the host-side name
    // of a __device__ array is only a stand-in and must not be passed to a kernel)
    void* addr = g_noalloc_ptr[dev].load(std::memory_order_acquire);
    if (!addr) {
      e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess || !addr) {
        set_context_free_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        return HYDOT_ERR_CUDA;
      }
      g_noalloc_ptr[dev].store(addr, std::memory_order_release);
    }
    unsigned char* base = static_cast<unsigned char*>(addr);
    double* d_eps = reinterpret_cast<double*>(base);
    float* part = reinterpret_cast<float*>(base + NOALLOC_EPS_BYTES);
    cudaStream_t s = (cudaStream_t)stream;
    e = cudaMemcpyAsync(d_eps, eps, eps_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      set_context_free_error(std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
      return HYDOT_ERR_CUDA;
    }
    {
      dim3 grid((unsigned)nxb, nlam, nts * ntd);
      // 32-wide optode tiles; every partial slot that is summed is written first, so nothing in the
      // array needs clearing
      e = launch_apply_partial<float, 8>(grid, s, phi_src, phi_det, x, d_eps, 0, n_src, n_det, n_chrom, N, (int)nxb,
                                         AP_STAGES, apply_vec_ok(phi_src, phi_det, x, N, 4), part);
      if (e == cudaSuccess)
        e = launch_apply_reduce<float>(part, nlam, n_src, n_det, nts, ntd, 32, (int)nxb, h_mm * h_mm * h_mm, y, s);
    }
    if (e != cudaSuccess) {
      set_context_free_error(std::string("launch: ") + cudaGetErrorString(e));
      return HYDOT_ERR_CUDA;
    }
    return HYDOT_OK;
  });
}
