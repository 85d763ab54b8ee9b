// Randomised low-rank sketch of the Born matrix on the tcgen05 tensor cores (Appendix A.1,
// alg:randsvd, at a fixed rank; Section 4.2 agglomeration as a sum over row blocks).
//
//   pass 1 (range):       Y = J Omega,  Y[(s,d,l), k] = -h^3 sum_x phi_s(x) phi_d(x) M_l[x, k],
//                         M_l = sum_c eps_c(lambda_l) Omega_c                 (rows of one slice)
//   pass 2 (projection):  B^T[(c,x), k] += -h^3 sum_(s,d,l) eps_c(lambda_l) phi_s(x) phi_d(x) Q[(s,d,l), k]
//                         (summing over wavelength slices merges the row blocks)
//
// Both passes are BF16 x BF16 -> FP32 tcgen05 GEMMs with two 128 x 224 accumulators in tensor
// memory: the A tiles (Hadamard products of source and detector fields) are formed by the CTA's
// threads straight into shared memory in the 128-byte swizzled K-major layout, the B tiles (M_l or
// eps-scaled Q, prepared once per call in BF16) arrive by TMA with the same swizzle, and one
// thread issues the MMAs. Multi-stage mbarrier pipelines (the range pass: three operand stages and
// two A stages; the projection: four B stages, two A stages, two field buffers); every wait is
// bounded. The general-shape projection kernel below is a simpler two-stage form.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cudaTypedefs.h>
#include <array>
#include <vector>

#include <cuda_bf16.h>

#include "dense.h"
#include "hydot_internal.cuh"
#include "tcgen05.cuh"

namespace hydot {

namespace {

constexpr int SK_M = 128;                      // accumulator rows (TMEM lanes)
constexpr int SK_N = 224;                      // sketch columns (rank + oversampling, padded to 16)
constexpr int SK_K = 64;                       // K per stage: one 128-byte swizzle row of BF16
constexpr int SK_A_BYTES = SK_M * SK_K * 2;    // 16 KiB
constexpr int SK_B_BYTES = SK_N * SK_K * 2;    // 28 KiB
constexpr int SK_STAGE = SK_A_BYTES + SK_B_BYTES;
constexpr int SK_STAGES = 2;
constexpr size_t SK_SMEM = (size_t)SK_STAGES * SK_STAGE + 1024;
constexpr uint32_t SK_TMEM_COLS = 256;

struct SketchArgs {
  const float* ps;   // [nlam][nsf][N]
  const float* pd;   // [nlam][nd][N]
  int ns, nd, nlam;  // ns: sources of the range src0 .. src0 + ns - 1
  int nsf, src0;     // sources in the field array; first source of the range
  long long N;
  long long P;       // pairs of the slice: nlam * ns * nd (internal order (l, s, d), d fastest)
  int chrom;         // chromophore of this launch
  float scale;       // -h^3
  float* out;
  long long ldo;
  int* err;
};

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~uintptr_t(1023));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&h);
}

// 16-byte store to a shared-memory address
__device__ __forceinline__ void sts_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
               : "memory");
}

// Bounded wait by one thread; on timeout the error flag is raised and the wait is retried once
// (bounded) so that no copy or MMA is left writing into shared memory that is about to be reused.
__device__ __forceinline__ void wait_or_flag(uint64_t* m, uint32_t parity, int* err) {
  if (!mbar_wait_bounded(m, parity)) {
    atomicExch(err, 1);
    mbar_wait_bounded(m, parity);
  }
}

// Projection pass for general optode counts (rows = voxels, K = pairs of the slice), one
// chromophore per launch; the A tile is formed from global loads.
__global__ void __launch_bounds__(128) k_project_generic(SketchArgs a, const __grid_constant__ CUtensorMap mapB) {
  extern __shared__ uint8_t sk_dsm[];
  uint8_t* base = align1024(sk_dsm);
  __shared__ uint64_t full[SK_STAGES], empty[SK_STAGES], done;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5;
  const long long x0 = (long long)blockIdx.x * SK_M;
  const long long K = a.P;
  const int nk = (int)((K + SK_K - 1) / SK_K);
  if (warp == 0) tmem_alloc(&s_tmem, SK_TMEM_COLS);
  if (tid == 0) {
    for (int q = 0; q < SK_STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 1);
    }
    mbar_init(&done, 1);
    mbar_fence_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  constexpr uint32_t IDESC = idesc_bf16_f32(SK_M, SK_N);

  for (int t = 0; t < nk; ++t) {
    const int st = t & 1;
    uint8_t* As = base + st * SK_STAGE;
    uint8_t* Bs = As + SK_A_BYTES;
    if (t >= SK_STAGES) {
      if (tid == 0) wait_or_flag(&empty[st], (uint32_t)(((t - SK_STAGES) >> 1) & 1), a.err);
      __syncthreads();
    }
    if (tid == 0) {
      mbar_expect_tx(&full[st], SK_B_BYTES);
      tma_load_3d(Bs, &mapB, &full[st], t * SK_K, 0, a.chrom);
    }
    // ---- A tile: 128 rows x 64 K of Hadamard products, BF16, swizzled K-major
    {
      const long long x = x0 + tid;
      const long long p0 = (long long)t * SK_K;
      // decode p0 once, then step (l, s, d) with d fastest
      int d = (int)(p0 % a.nd);
      const long long ls0 = p0 / a.nd;
      int s = (int)(ls0 % a.ns), l = (int)(ls0 / a.ns);
      const bool xin = x < a.N;
      float fsv = (xin && p0 < a.P) ? __ldg(a.ps + ((size_t)l * a.nsf + a.src0 + s) * a.N + x) : 0.f;
      for (int ch = 0; ch < 8; ++ch) {
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const long long p = p0 + ch * 8 + i;
          v[i] = (xin && p < a.P) ? fsv * __ldg(a.pd + ((size_t)l * a.nd + d) * a.N + x) : 0.f;
          if (++d == a.nd) {
            d = 0;
            if (++s == a.ns) {
              s = 0;
              ++l;
            }
            if (xin && p + 1 < a.P) fsv = __ldg(a.ps + ((size_t)l * a.nsf + a.src0 + s) * a.N + x);
          }
        }
        uint4 pk;
        pk.x = pack_bf16x2(v[0], v[1]);
        pk.y = pack_bf16x2(v[2], v[3]);
        pk.z = pack_bf16x2(v[4], v[5]);
        pk.w = pack_bf16x2(v[6], v[7]);
        *reinterpret_cast<uint4*>(As + sw128_offset(tid, ch * 8)) = pk;
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      wait_or_flag(&full[st], (uint32_t)((t >> 1) & 1), a.err);
      tc_fence_after();
      const uint32_t a_addr = smem_addr(As), b_addr = smem_addr(Bs);
#pragma unroll
      for (int kk = 0; kk < SK_K / 16; ++kk) {
        tc_mma_bf16(tmem, smem_desc_sw128(a_addr + kk * 32), smem_desc_sw128(b_addr + kk * 32), IDESC,
                    (t > 0 || kk > 0) ? 1u : 0u);
      }
      tc_commit(&empty[st]);
    }
  }
  if (tid == 0) {
    tc_commit(&done);
    wait_or_flag(&done, 0, a.err);
  }
  __syncthreads();
  tc_fence_after();
  // ---- epilogue: warp w owns TMEM lanes 32w..32w+31, i.e. accumulator rows 32w + lane
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const int row = tid;
  const long long x = x0 + row;
  const bool ok = x < a.N;
  float* dst = a.out + ((long long)a.chrom * a.N + (ok ? x : 0)) * a.ldo;
  for (int c0 = 0; c0 < SK_N; c0 += 16) {
    float v[16];
    tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
    if (ok) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        dst[c0 + q] += a.scale * v[q];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, SK_TMEM_COLS);
}

// ---------------------------------------------------------------- warp-specialised range pass
// Y = J Omega for a (wavelength, source block, detector block) item and a range of K-steps:
//   warp 0        TMA producer: per K-step the B tile (M_l, 224 x 64 BF16, 128-byte swizzle) and
//                 the FP32 field slabs of the item's sources (2 S_a rows) and detectors (D_t rows);
//   warp 1        one thread issues the MMAs: two 128 x 224 accumulators in tensor memory (the
//                 item's first and second S_a sources x D_t detectors) share each B tile;
//   warps 2..9    form the A tiles (Hadamard products, BF16, swizzled K-major) from the field
//                 slabs in shared memory, then read the accumulators back (epilogue).
// RG_STAGES operand stages and 2 A stages; the K range of an item is split over CTAs (partials
// summed by a second kernel in a fixed order) so that the grid covers the SMs.
constexpr int RG_THREADS = 320;
constexpr int RG_STAGES = 3;
constexpr int RG_FROWS = 72;                                   // field rows per stage (2 S_a + D_t <= 72)
constexpr int RG_ND = 4, RG_NS = 2;                            // detectors and sources of a former's work unit
constexpr uint32_t RG_B_BYTES = SK_N * SK_K * 2;               // 28,672
constexpr uint32_t RG_F_BYTES = RG_FROWS * SK_K * 4;           // 18,432
constexpr uint32_t RG_STAGE = RG_B_BYTES + RG_F_BYTES;         // 47,104 = 46 x 1024
constexpr uint32_t RG_A_STAGE = 2 * SK_A_BYTES;                // two 128 x 64 A tiles
constexpr size_t RG_SMEM = (size_t)RG_STAGES * RG_STAGE + 2 * RG_A_STAGE + 1024;
constexpr uint32_t RG_TMEM_COLS = 512;                         // accumulators at columns 0 and 256

struct RangeArgs {
  int ns, nd, nlam;          // ns: sources of the range src0 .. src0 + ns - 1
  int src0;
  long long N;
  int S_a, D_t, nsb, ndb;    // sources per accumulator, detectors per block, source / detector blocks
  int nk, k_per_split, nsplit;
  long long P;               // rows of Y in the slice
  float* out;                // Y (nsplit == 1, scaled) or partials [nsplit][P][SK_N]
  long long ldo;
  float scale;
  int* err;
};

__global__ void __launch_bounds__(RG_THREADS, 1)
    k_range_ws(RangeArgs a, const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapPs,
               const __grid_constant__ CUtensorMap mapPd) {
  extern __shared__ uint8_t sk_dsm[];
  uint8_t* base = align1024(sk_dsm);
  uint8_t* abuf = base + (size_t)RG_STAGES * RG_STAGE;
  __shared__ uint64_t full[RG_STAGES], empty[RG_STAGES], afull[2], aempty[2], accf;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int item = blockIdx.x / a.nsplit, ks = blockIdx.x - item * a.nsplit;
  const int l = item / (a.nsb * a.ndb);
  const int rem = item - l * a.nsb * a.ndb;
  const int sb = rem / a.ndb, db = rem - sb * a.ndb;
  const int s0 = a.src0 + sb * 2 * a.S_a, d0 = db * a.D_t;
  const int kt0 = ks * a.k_per_split, kt1 = min(a.nk, kt0 + a.k_per_split);
  const int nku = max(kt1 - kt0, 0);
  if (tid == 0) {
    for (int q = 0; q < RG_STAGES; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&empty[q], 9);  // 8 former warps + the MMA commit
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&afull[q], 8);
      mbar_init(&aempty[q], 1);
    }
    mbar_init(&accf, 1);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(&s_tmem, RG_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  const uint32_t fbytes = (uint32_t)(2 * a.S_a + a.D_t) * SK_K * 4;

  if (warp == 0) {
    if (lane == 0) {
      for (int u = 0; u < nku; ++u) {
        const int st = u % RG_STAGES;
        if (u >= RG_STAGES) wait_or_flag(&empty[st], (uint32_t)((u / RG_STAGES - 1) & 1), a.err);
        uint8_t* sb_ = base + (size_t)st * RG_STAGE;
        const int x = (kt0 + u) * SK_K;
        mbar_expect_tx(&full[st], RG_B_BYTES + fbytes);
        tma_load_3d(sb_, &mapB, &full[st], x, 0, l);
        tma_load_3d(sb_ + RG_B_BYTES, &mapPs, &full[st], x, s0, l);
        tma_load_3d(sb_ + RG_B_BYTES + 2 * a.S_a * SK_K * 4, &mapPd, &full[st], x, d0, l);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t IDESC = idesc_bf16_f32(SK_M, SK_N);
      for (int u = 0; u < nku; ++u) {
        const int st = u % RG_STAGES, as = u & 1;
        wait_or_flag(&full[st], (uint32_t)((u / RG_STAGES) & 1), a.err);
        wait_or_flag(&afull[as], (uint32_t)((u >> 1) & 1), a.err);
        tc_fence_after();
        const uint32_t b_addr = smem_addr(base + (size_t)st * RG_STAGE);
        const uint32_t a_addr = smem_addr(abuf + (size_t)as * RG_A_STAGE);
#pragma unroll
        for (int acc = 0; acc < 2; ++acc)
#pragma unroll
          for (int kk = 0; kk < SK_K / 16; ++kk)
            tc_mma_bf16(tmem + (uint32_t)(acc * 256), smem_desc_sw128(a_addr + acc * SK_A_BYTES + kk * 32),
                        smem_desc_sw128(b_addr + kk * 32), IDESC, (u > 0 || kk > 0) ? 1u : 0u);
        tc_commit(&empty[st]);
        tc_commit(&aempty[as]);
      }
      tc_commit(&accf);
    }
  } else {
    // ---- A formers. Work unit (chunk ch of 8 voxels, a group of RG_ND detectors, a group of RG_NS
    // sources): the unit's RG_ND detector and RG_NS source chunks are read into registers once and
    // give RG_NS x RG_ND chunk products, so a K-step reads each detector chunk 2 S_a / RG_NS times and
    // each source chunk D_t / RG_ND times from shared memory, whose bandwidth the TMA copies and the
    // MMAs share with these loads (one product per detector and source chunk read 8 times over).
    // The eight lanes of a 16-byte load phase read chunks ch = 0..7 of one row: lanes with ch >= 4
    // read their chunk's second half first, so that the phase's eight 16-byte words fall on distinct
    // bank groups (ch * 32 + 16 * (ch >> 2) mod 128 is a permutation of 16 * 0..7); [0] is the half
    // read first, and the products are stored in that order.
    const int f = tid - 64;
    const int rows = a.S_a * a.D_t;
    const int nsrc = 2 * a.S_a;
    const int ndg = (a.D_t + RG_ND - 1) / RG_ND, nsg = (nsrc + RG_NS - 1) / RG_NS;
    const int nunit = 8 * ndg * nsg;  // at most 400 (D_t = 5): two rounds of 256 formers
    // this thread's work units w = f and f + 256 (chunk, detector group, source group), fixed over K
    const int nrounds = f < nunit ? (f + 256 < nunit ? 2 : 1) : 0;
    int uch[2], udg[2], usg[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int w = f + r * 256;
      uch[r] = w & 7;
      udg[r] = (w >> 3) % ndg;
      usg[r] = (w >> 3) / ndg;
    }
    // rows that no pair maps to stay zero: write them once in both A stages
    for (int e = f; e < 2 * 2 * (SK_M - rows) * 8; e += 256) {
      const int ch = e & 7, rr = rows + ((e >> 3) % (SK_M - rows)), sa = (e >> 3) / (SK_M - rows);
      *reinterpret_cast<uint4*>(abuf + (size_t)(sa >> 1) * RG_A_STAGE + (sa & 1) * SK_A_BYTES +
                                sw128_offset(rr, ch * 8)) = make_uint4(0u, 0u, 0u, 0u);
    }
    for (int u = 0; u < nku; ++u) {
      const int st = u % RG_STAGES, as = u & 1;
      if (!mbar_wait_bounded(&full[st], (uint32_t)((u / RG_STAGES) & 1))) atomicExch(a.err, 1);
      if (u >= 2 && !mbar_wait_bounded(&aempty[as], (uint32_t)((u / 2 - 1) & 1))) atomicExch(a.err, 1);
      const float* fps = reinterpret_cast<const float*>(base + (size_t)st * RG_STAGE + RG_B_BYTES);
      const float* fpd = fps + 2 * a.S_a * SK_K;
      const uint32_t At = smem_addr(abuf + (size_t)as * RG_A_STAGE);
      for (int r = 0; r < 2; ++r) {
        if (r >= nrounds) break;
        const int ch = uch[r], dg = udg[r], sg = usg[r];
        const int h0 = (ch >> 2) * 4, h1 = 4 - h0;
        float4 dv[RG_ND][2], sv[RG_NS][2];
#pragma unroll
        for (int j = 0; j < RG_ND; ++j) {
          const int d = min(dg * RG_ND + j, a.D_t - 1);
          dv[j][0] = *reinterpret_cast<const float4*>(fpd + d * SK_K + ch * 8 + h0);
          dv[j][1] = *reinterpret_cast<const float4*>(fpd + d * SK_K + ch * 8 + h1);
        }
#pragma unroll
        for (int i = 0; i < RG_NS; ++i) {
          const int sl = min(sg * RG_NS + i, nsrc - 1);
          sv[i][0] = *reinterpret_cast<const float4*>(fps + sl * SK_K + ch * 8 + h0);
          sv[i][1] = *reinterpret_cast<const float4*>(fps + sl * SK_K + ch * 8 + h1);
        }
#pragma unroll
        for (int i = 0; i < RG_NS; ++i) {
          const int sl = sg * RG_NS + i;
          const int acc = sl >= a.S_a ? 1 : 0;
#pragma unroll
          for (int j = 0; j < RG_ND; ++j) {
            const int dl = dg * RG_ND + j;
            if (sl >= nsrc || dl >= a.D_t) continue;
            const int rr = (sl - acc * a.S_a) * a.D_t + dl;
            const uint32_t p0 = pack_bf16x2(sv[i][0].x * dv[j][0].x, sv[i][0].y * dv[j][0].y);
            const uint32_t p1 = pack_bf16x2(sv[i][0].z * dv[j][0].z, sv[i][0].w * dv[j][0].w);
            const uint32_t p2 = pack_bf16x2(sv[i][1].x * dv[j][1].x, sv[i][1].y * dv[j][1].y);
            const uint32_t p3 = pack_bf16x2(sv[i][1].z * dv[j][1].z, sv[i][1].w * dv[j][1].w);
            // chunks ch >= 4 keep the order they were read in (second half first): M_l's K order
            // within those chunks is the same (k_form_mt)
            sts_v4(At + acc * SK_A_BYTES + sw128_offset(rr, ch * 8), make_uint4(p0, p1, p2, p3));
          }
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&afull[as]);
        mbar_arrive(&empty[st]);
      }
    }
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of accumulator (w - 2) / 4
    if (!mbar_wait_bounded(&accf, 0u)) atomicExch(a.err, 1);
    tc_fence_after();
    const int q4 = warp & 3, acc = (warp - 2) >> 2;
    const int rr = q4 * 32 + lane;
    bool ok = nku > 0 && rr < rows;
    long long r_out = 0;
    if (ok) {
      const int s = s0 + acc * a.S_a + rr / a.D_t, d = d0 + rr % a.D_t;
      ok = s < a.src0 + a.ns && d < a.nd;
      r_out = ((long long)(s - a.src0) * a.nd + d) * a.nlam + l;
    }
    float* dst = nullptr;
    float sc = 1.f;
    if (a.nsplit == 1) {
      dst = a.out + r_out * a.ldo;
      sc = a.scale;
    } else {
      dst = a.out + ((long long)ks * a.P + r_out) * SK_N;
    }
    const uint32_t tbase = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(acc * 256);
    for (int c0 = 0; c0 < SK_N; c0 += 16) {
      float v[16];
      tmem_ld16(tbase + (uint32_t)c0, v);
      if (ok) {
#pragma unroll
        for (int q = 0; q < 16; q += 4)
          *reinterpret_cast<float4*>(dst + c0 + q) = make_float4(sc * v[q], sc * v[q + 1], sc * v[q + 2], sc * v[q + 3]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, RG_TMEM_COLS);
}

// Y[r][k] = scale * sum_s part[s][r][k] (fixed order over the K splits)
__global__ void k_range_reduce(const float* __restrict__ part, int nsplit, long long P, float scale,
                               float* __restrict__ Y, long long ldY) {
  const long long total = P * (SK_N / 4);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const long long r = q / (SK_N / 4);
    const int k4 = (int)(q - r * (SK_N / 4)) * 4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int sp = 0; sp < nsplit; ++sp) {
      const float4 v = *reinterpret_cast<const float4*>(part + ((long long)sp * P + r) * SK_N + k4);
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
    *reinterpret_cast<float4*>(Y + r * ldY + k4) = make_float4(scale * acc.x, scale * acc.y, scale * acc.z, scale * acc.w);
  }
}

// ---------------------------------------------------------------- warp-specialised projection pass
// B^T[(c,x), k] += -h^3 sum_(l,s,d) eps_c(l) phi_s(x) phi_d(x) Q[(s,d,l), k] for a tile of 128 voxels
// and two chromophores (two 128 x 224 accumulators sharing each A tile). K runs over the pairs of
// each wavelength (padded to a multiple of 64 per wavelength). The tile's fields of the current
// wavelength (n_src + n_det rows of 128 voxels, FP32) stay in shared memory while its K-steps run;
// with n_src + n_det <= 64 the field buffer holds two wavelengths, so the next one arrives while
// the current one is formed.
//   warp 0        TMA: the B tiles (eps_c-scaled Q, 224 x 64 BF16), one stage per (K-step,
//                 chromophore): four stages of one tile each, so that loads run 1.5 K-steps ahead;
//   warp 1        one thread issues the MMAs;
//   warp 2        TMA: the field block of each wavelength, once its buffer is consumed;
//   warps 3..10   form the A tiles and read the accumulators back.
constexpr int PJ_THREADS = 352;
constexpr int PJ_M = 128;                                     // voxels per tile
constexpr uint32_t PJ_B_TILE = SK_N * SK_K * 2;               // one B tile: 28,672 B
constexpr int PJ_B_STAGES = 4;
constexpr int PJ_BT0_COLS = 116;                              // epilogue boxes: columns 0..115, 116..223
constexpr uint32_t PJ_STG_BYTES = 32 * PJ_BT0_COLS * 4;       // one warp's staged rows: 14,848 B (116 x 128)
constexpr uint32_t PJ_F_BYTES = 128 * PJ_M * 4;               // n_src + n_det <= 128 rows: 65,536 B
constexpr size_t PJ_SMEM = PJ_B_STAGES * (size_t)PJ_B_TILE + 2 * (size_t)SK_A_BYTES + PJ_F_BYTES + 1024;

struct ProjArgs {
  int ns, nd, nlam, nc, Kl;  // ns: sources of the range src0 .. src0 + ns - 1; Kl: K-steps per wavelength
  int src0;
  long long N;
  float* Bt;
  long long ldB;
  float scale;
  int* err;
};

__global__ void __launch_bounds__(PJ_THREADS, 1)
    k_project_ws(ProjArgs a, const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapPs,
                 const __grid_constant__ CUtensorMap mapPd, const __grid_constant__ CUtensorMap mapBt0,
                 const __grid_constant__ CUtensorMap mapBt1) {
  extern __shared__ uint8_t sk_dsm[];
  uint8_t* base = align1024(sk_dsm);
  uint8_t* abuf = base + PJ_B_STAGES * (size_t)PJ_B_TILE;
  float* fld = reinterpret_cast<float*>(abuf + 2 * (size_t)SK_A_BYTES);  // [nfb][ns + nd][128]
  __shared__ uint64_t bfull[PJ_B_STAGES], bempty[PJ_B_STAGES], afull[2], aempty[2], ffull[2], fempty[2], accf;
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tile = blockIdx.x / ((a.nc + 1) / 2), cp = blockIdx.x - tile * ((a.nc + 1) / 2);
  const long long x0 = (long long)tile * PJ_M;
  const int c0 = 2 * cp;
  const int nku = a.nlam * a.Kl;
  const int frow = (a.ns + a.nd) * PJ_M;                        // floats of one wavelength's field block
  const int nfb = 2 * frow * 4 <= (int)PJ_F_BYTES ? 2 : 1;      // field buffers
  if (tid == 0) {
    for (int q = 0; q < PJ_B_STAGES; ++q) {
      mbar_init(&bfull[q], 1);
      mbar_init(&bempty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&afull[q], 8);
      mbar_init(&aempty[q], 1);
      mbar_init(&ffull[q], 1);
      mbar_init(&fempty[q], 8);
    }
    mbar_init(&accf, 1);
    mbar_fence_init();
  }
  if (warp == 1) tmem_alloc(&s_tmem, RG_TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    if (lane == 0) {
      // stage use q = 2 u + h: K-step u, chromophore c0 + h
      for (int q = 0; q < 2 * nku; ++q) {
        const int bs = q % PJ_B_STAGES;
        if (q >= PJ_B_STAGES) wait_or_flag(&bempty[bs], (uint32_t)((q / PJ_B_STAGES - 1) & 1), a.err);
        mbar_expect_tx(&bfull[bs], PJ_B_TILE);
        tma_load_3d(base + (size_t)bs * PJ_B_TILE, &mapB, &bfull[bs], (q >> 1) * SK_K, 0, c0 + (q & 1));
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t IDESC = idesc_bf16_f32(SK_M, SK_N);
      for (int u = 0; u < nku; ++u) {
        const int as = u & 1;
        wait_or_flag(&afull[as], (uint32_t)((u >> 1) & 1), a.err);
        const uint32_t a_addr = smem_addr(abuf + (size_t)as * SK_A_BYTES);
#pragma unroll
        for (int acc = 0; acc < 2; ++acc) {
          const int q = 2 * u + acc, bs = q % PJ_B_STAGES;
          wait_or_flag(&bfull[bs], (uint32_t)((q / PJ_B_STAGES) & 1), a.err);
          tc_fence_after();
          const uint32_t b_addr = smem_addr(base + (size_t)bs * PJ_B_TILE);
#pragma unroll
          for (int kk = 0; kk < SK_K / 16; ++kk)
            tc_mma_bf16(tmem + (uint32_t)(acc * 256), smem_desc_sw128(a_addr + kk * 32),
                        smem_desc_sw128(b_addr + kk * 32), IDESC, (u > 0 || kk > 0) ? 1u : 0u);
          tc_commit(&bempty[bs]);
        }
        tc_commit(&aempty[as]);
      }
      tc_commit(&accf);
    }
  } else if (warp == 2) {
    if (lane == 0) {
      const uint32_t fb = (uint32_t)frow * 4;
      for (int l = 0; l < a.nlam; ++l) {
        const int b = l % nfb;
        float* dst = fld + (size_t)b * frow;
        if (l >= nfb) wait_or_flag(&fempty[b], (uint32_t)((l / nfb - 1) & 1), a.err);
        mbar_expect_tx(&ffull[b], fb);
        tma_load_3d(dst, &mapPs, &ffull[b], (int)x0, a.src0, l);
        tma_load_3d(dst + a.ns * PJ_M, &mapPd, &ffull[b], (int)x0, 0, l);
      }
    }
  } else {
    // ---- A formers: thread f takes voxel row (id & 127) and pair chunk (id >> 7) for id = j*256 + f.
    // With n_det % 8 == 0 the chunk's eight pairs share their source and take detectors d .. d + 7;
    // the thread keeps those eight detector values of its row in registers while d stays the same
    // (for every K-step of a wavelength when n_det divides 64 or 64 divides it), so a K-step mostly
    // reads one source value per chunk from shared memory.
    const int f = tid - 96;
    const int npairs = a.ns * a.nd;
    const bool nd8 = (a.nd & 7) == 0;
    float dreg[4][8];
    int dkey[4];       // detector offset d of the values in dreg[j] (-1: none)
    int sj[4], dj[4];  // source and detector of the first pair of item j's chunk at this K-step
    int l = 0, kq = 0, fbi = 0;  // wavelength, K-step in it, field buffer (no divisions in the loop)
    for (int u = 0; u < nku; ++u) {
      const int as = u & 1;
      const float* psm = fld + (size_t)fbi * frow;
      const float* pdm = psm + a.ns * PJ_M;
      if (kq == 0) {
        const uint32_t fpar = (uint32_t)((nfb == 2 ? (l >> 1) : l) & 1);
        if (!mbar_wait_bounded(&ffull[fbi], fpar)) atomicExch(a.err, 1);
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // a new wavelength's fields
          const int q0 = ((j * 256 + f) >> 7) * 8;
          sj[j] = q0 / a.nd;
          dj[j] = q0 - sj[j] * a.nd;
          dkey[j] = -1;
        }
      }
      if (u >= 2 && !mbar_wait_bounded(&aempty[as], (uint32_t)(((u >> 1) - 1) & 1))) atomicExch(a.err, 1);
      const uint32_t At = smem_addr(abuf + (size_t)as * SK_A_BYTES);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int id = j * 256 + f;
        const int row = id & (PJ_M - 1), ch = id >> 7;
        const int q0 = kq * SK_K + ch * 8;
        int s = sj[j], d = dj[j];
        // the next K-step's first pair of this chunk is 64 pairs on
        dj[j] += SK_K;
        while (dj[j] >= a.nd) {
          dj[j] -= a.nd;
          ++sj[j];
        }
        float v[8];
        if (nd8 && q0 + 8 <= npairs) {
          if (d != dkey[j]) {
            const float* pr = pdm + d * PJ_M + row;
#pragma unroll
            for (int i = 0; i < 8; ++i) dreg[j][i] = pr[i * PJ_M];
            dkey[j] = d;
          }
          const float sv = psm[s * PJ_M + row];
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = sv * dreg[j][i];
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            // clamped indices keep every read inside the field block; the padding pairs give 0
            const float pv = psm[min(s, a.ns - 1) * PJ_M + row] * pdm[d * PJ_M + row];
            v[i] = (q0 + i < npairs) ? pv : 0.f;
            if (++d == a.nd) {
              d = 0;
              ++s;
            }
          }
        }
        uint4 pk;
        pk.x = pack_bf16x2(v[0], v[1]);
        pk.y = pack_bf16x2(v[2], v[3]);
        pk.z = pack_bf16x2(v[4], v[5]);
        pk.w = pack_bf16x2(v[6], v[7]);
        sts_v4(At + sw128_offset(row, ch * 8), pk);
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&afull[as]);
        if (kq == a.Kl - 1) mbar_arrive(&fempty[fbi]);
      }
      if (++kq == a.Kl) {
        kq = 0;
        ++l;
        fbi = nfb == 2 ? fbi ^ 1 : 0;
      }
    }
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of accumulator (w - 3) / 4, i.e. the
    // scaled rows of 32 voxels, stages them in the (now idle) B / A stage buffers and adds them to
    // B^T with TMA reductions, columns 0..115 and then 116..223 (row pitches of 29 and 27 16-byte
    // units: the lanes' 16-byte stores fall on distinct bank groups). B^T is never read by the SM.
    if (!mbar_wait_bounded(&accf, 0u)) atomicExch(a.err, 1);
    tc_fence_after();
    const int q4 = warp & 3, acc = (warp - 3) >> 2;
    const int c = c0 + acc;
    const long long xr = x0 + q4 * 32;  // first voxel of the warp's rows
    const bool ok = nku > 0 && xr < a.N && c < a.nc;
    float* stg = reinterpret_cast<float*>(base + (size_t)(warp - 3) * PJ_STG_BYTES);
    const uint32_t tbase = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(acc * 256);
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
      const int g0 = h ? PJ_BT0_COLS / 4 : 0, g1 = h ? SK_N / 4 : PJ_BT0_COLS / 4;  // 4-column groups
      const int pitch = h ? SK_N - PJ_BT0_COLS : PJ_BT0_COLS;                          // floats per staged row
      for (int k0 = (g0 * 4) & ~15; k0 < g1 * 4; k0 += 16) {
        float v[16];
        tmem_ld16(tbase + (uint32_t)k0, v);
#pragma unroll
        for (int q = 0; q < 16; q += 4) {
          const int g = (k0 + q) >> 2;
          if (g < g0 || g >= g1) continue;
          *reinterpret_cast<float4*>(stg + lane * pitch + (g - g0) * 4) =
              make_float4(a.scale * v[q], a.scale * v[q + 1], a.scale * v[q + 2], a.scale * v[q + 3]);
        }
      }
      fence_async_smem();
      __syncwarp();
      if (lane == 0 && ok) {
        tma_reduce_add_3d(h ? &mapBt1 : &mapBt0, stg, g0 * 4, (int)xr, c);
        bulk_commit_group();
        bulk_wait_read_all();  // the staging rows are reused by the second half
      }
      __syncwarp();
    }
    if (lane == 0 && ok) bulk_wait_all();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, RG_TMEM_COLS);
}

// Qc[c][k][l * Pl + q] = eps_c(lambda_l) * Q[row][k] for the pairs q = s * nd + d < ns * nd of
// wavelength l (row = (s*nd + d)*nlam + l), zero on the padding q >= ns * nd and for k >= ncols.
__global__ void k_form_qc_padded(const float* __restrict__ Q, long long ldq, const double* __restrict__ eps, int lam0,
                                 int nlam, int ns, int nd, int nc, int ncols, long long Pl,
                                 __nv_bfloat16* __restrict__ Qc) {
  const long long Pt = (long long)nlam * Pl;
  const long long total = (long long)nc * SK_N * Pt;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long pp = i % Pt;
    const int k = (int)((i / Pt) % SK_N);
    const int c = (int)(i / (Pt * SK_N));
    const int l = (int)(pp / Pl);
    const long long q = pp - (long long)l * Pl;
    float v = 0.f;
    if (q < (long long)ns * nd && k < ncols) {
      const long long r = q * nlam + l;
      v = (float)eps[(size_t)(lam0 + l) * nc + c] * Q[r * ldq + k];
    }
    Qc[i] = __float2bfloat16_rn(v);
  }
}

// Mt[l][k][x] = sum_c eps_c(lambda_(lam0+l)) * Omega_t[c][k][x] in BF16 (k >= ncols: 0); 8 voxels per thread.
// Within each 64-voxel K-step, 8-voxel chunks 4..7 are stored with their halves swapped (voxels 4..7,
// then 0..3): the range pass's A formers read those chunks' halves in that order (a bank-conflict
// rule) and store their products as read; the K order of A and B is permuted alike, so the product
// A B^T is unchanged.
__global__ void k_form_mt(const __nv_bfloat16* __restrict__ om, const double* __restrict__ eps, int lam0, int nlam,
                          int nc, int ncols, long long N, __nv_bfloat16* __restrict__ Mt) {
  const long long nv = N / 8;
  const long long total = (long long)nlam * SK_N * nv;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const long long xv = q % nv;
    const int k = (int)((q / nv) % SK_N);
    const int l = (int)(q / (nv * SK_N));
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (k < ncols) {
      for (int c = 0; c < nc; ++c) {
        const float e = (float)eps[(size_t)(lam0 + l) * nc + c];
        const uint4 raw = *reinterpret_cast<const uint4*>(om + ((size_t)c * ncols + k) * N + xv * 8);
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 f = __bfloat1622float2(h[i]);
          acc[2 * i] = fmaf(e, f.x, acc[2 * i]);
          acc[2 * i + 1] = fmaf(e, f.y, acc[2 * i + 1]);
        }
      }
    }
    uint4 out;
    out.x = pack_bf16x2(acc[0], acc[1]);
    out.y = pack_bf16x2(acc[2], acc[3]);
    out.z = pack_bf16x2(acc[4], acc[5]);
    out.w = pack_bf16x2(acc[6], acc[7]);
    if ((xv & 7) >= 4) out = make_uint4(out.z, out.w, out.x, out.y);
    *reinterpret_cast<uint4*>(Mt + ((size_t)l * SK_N + k) * N + xv * 8) = out;
  }
}

// Qc[c][k][p] = eps_c(lambda of pair p) * Q[row(p)][k] in BF16, pairs p = (l, s, d) of the slice
// (d fastest), row(p) = (s*nd + d)*nlam + l; p >= P or k >= ncols: 0.
__global__ void k_form_qc(const float* __restrict__ Q, long long ldq, const double* __restrict__ eps, int lam0,
                          int nlam, int ns, int nd, int nc, int ncols, long long P, long long Pp,
                          __nv_bfloat16* __restrict__ Qc) {
  const long long total = (long long)nc * SK_N * Pp;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const long long p = q % Pp;
    const int k = (int)((q / Pp) % SK_N);
    const int c = (int)(q / (Pp * SK_N));
    float v = 0.f;
    if (p < P && k < ncols) {
      const int d = (int)(p % nd);
      const long long ls = p / nd;
      const int s = (int)(ls % ns), l = (int)(ls / ns);
      const long long r = ((long long)s * nd + d) * nlam + l;
      v = (float)eps[(size_t)(lam0 + l) * nc + c] * Q[r * ldq + k];
    }
    Qc[q] = __float2bfloat16_rn(v);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder(hydot_ctx* ctx) {
  static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    return (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
               ? reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p)
               : nullptr;
  }();
  if (!fn) fail(ctx, HYDOT_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  return fn;
}

// 3-D BF16 map {inner, 224, outer} with a {64, 224, 1} box in the 128-byte swizzle.
int encode_b_map(hydot_ctx* ctx, void* base, long long inner, long long outer, CUtensorMap* map) {
  auto enc = tensor_map_encoder(ctx);
  if (!enc) return HYDOT_ERR_CUDA;
  cuuint64_t dims[3] = {(cuuint64_t)inner, (cuuint64_t)SK_N, (cuuint64_t)outer};
  cuuint64_t strides[2] = {(cuuint64_t)inner * 2, (cuuint64_t)inner * 2 * SK_N};
  cuuint32_t box[3] = {(cuuint32_t)SK_K, (cuuint32_t)SK_N, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, HYDOT_ERR_CUDA, "cuTensorMapEncodeTiled failed for a sketch operand");
  return HYDOT_OK;
}

// 3-D FP32 map {d0, d1, d2} (d0 innermost, contiguous) with a {b0, b1, 1} box, no swizzle.
int encode_f32_map(hydot_ctx* ctx, const void* base, long long d0, long long d1, long long d2, int b0, int b1,
                   CUtensorMap* map) {
  auto enc = tensor_map_encoder(ctx);
  if (!enc) return HYDOT_ERR_CUDA;
  cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
  cuuint64_t strides[2] = {(cuuint64_t)d0 * 4, (cuuint64_t)d0 * 4 * d1};
  cuuint32_t box[3] = {(cuuint32_t)b0, (cuuint32_t)b1, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, HYDOT_ERR_CUDA, "cuTensorMapEncodeTiled failed for a field slab map");
  return HYDOT_OK;
}

// 3-D FP32 map over B^T [(c, x)][ldB] as {224 columns, N voxels, nc chromophores} with a {b0, 32, 1}
// box, for the projection epilogue's TMA reductions (voxels past N are outside the map, so a partial
// voxel tile never reaches the next chromophore's rows).
int encode_bt_map(hydot_ctx* ctx, float* Bt, long long N, int nc, long long ldB, int b0, CUtensorMap* map) {
  auto enc = tensor_map_encoder(ctx);
  if (!enc) return HYDOT_ERR_CUDA;
  cuuint64_t dims[3] = {(cuuint64_t)SK_N, (cuuint64_t)N, (cuuint64_t)nc};
  cuuint64_t strides[2] = {(cuuint64_t)ldB * 4, (cuuint64_t)ldB * 4 * N};
  cuuint32_t box[3] = {(cuuint32_t)b0, 32, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, Bt, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, HYDOT_ERR_CUDA, "cuTensorMapEncodeTiled failed for the B^T map");
  return HYDOT_OK;
}

int sketch_ws(hydot_ctx* ctx, size_t bytes) {
  if (ctx->sketch_ws_bytes >= bytes) return HYDOT_OK;
  if (ctx->d_sketch_ws) {
    HYDOT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->d_sketch_ws);
    ctx->d_sketch_ws = nullptr;
    ctx->sketch_ws_bytes = 0;
  }
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&ctx->d_sketch_ws, bytes));
  ctx->sketch_ws_bytes = bytes;
  return HYDOT_OK;
}

int sketch_check(hydot_ctx* ctx, int lam0, int nlam, int ncols) {
  if (ctx->cplx) return fail(ctx, HYDOT_ERR_STATE, "the sketch is defined for continuous-wave (real) fields only");
  if (ctx->precision != HYDOT_MIXED) return fail(ctx, HYDOT_ERR_STATE, "the sketch takes FP32 fields (HYDOT_MIXED)");
  if (lam0 < 0 || nlam < 1 || lam0 + nlam > ctx->n_lambda) return fail(ctx, HYDOT_ERR_ARG, "wavelength slice out of range");
  if (ncols < 1 || ncols > SK_N) return fail(ctx, HYDOT_ERR_ARG, "ncols must be in 1..224");
  if (ctx->N % 8 != 0) return fail(ctx, HYDOT_ERR_ARG, "the sketch needs N divisible by 8");
  return HYDOT_OK;
}

int set_sketch_smem(hydot_ctx* ctx) {
  HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_project_generic, SK_SMEM));
  HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_range_ws, RG_SMEM));
  HYDOT_CUDA_TRY(ctx, raise_smem_limit(k_project_ws, PJ_SMEM));
  return HYDOT_OK;
}

}  // namespace

int sketch_range_impl(hydot_ctx* ctx, const float* ps, const float* pd, int lam0, int nlam, int src0, int nsr,
                      const void* omega_t, int ncols, float* Y, long long ldY) {
  int rc = sketch_check(ctx, lam0, nlam, ncols);
  if (rc) return rc;
  if (src0 < 0 || nsr < 1 || src0 + nsr > ctx->n_src) return fail(ctx, HYDOT_ERR_ARG, "source range out of range");
  if (!ps || !pd || !omega_t || !Y) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  if (ldY < SK_N || ldY % 4 != 0 || (reinterpret_cast<uintptr_t>(Y) & 15) != 0)
    return fail(ctx, HYDOT_ERR_ARG, "Y must be 16-byte aligned with ldY >= 224 and ldY % 4 == 0");
  const long long N = ctx->N;
  const int ns = nsr, nd = ctx->n_det;
  const long long P = (long long)nlam * ns * nd;
  // items: (wavelength, block of 2 S_a sources, block of D_t detectors); each accumulator holds
  // S_a x D_t pairs (<= 128 rows)
  const int D_t = std::min(nd, 64);
  const int S_a = std::min(32, SK_M / D_t);
  const int nsb = (ns + 2 * S_a - 1) / (2 * S_a), ndb = (nd + D_t - 1) / D_t;
  const long long items = (long long)nlam * nsb * ndb;
  const int nk = (int)((N + SK_K - 1) / SK_K);
  // split K so that the grid fills about eight waves of one CTA per SM, each split >= 32 K-steps
  int nsplit = (int)std::max<long long>(1, std::min<long long>((8 * 152 + items - 1) / items, std::max(1, nk / 32)));
  const int kps = (nk + nsplit - 1) / nsplit;
  nsplit = (nk + kps - 1) / kps;
  const size_t mt_bytes = ((size_t)nlam * SK_N * N * 2 + 255) / 256 * 256;
  const size_t part_bytes = nsplit > 1 ? (size_t)nsplit * P * SK_N * 4 : 0;
  if ((rc = sketch_ws(ctx, mt_bytes + part_bytes))) return rc;
  if ((rc = set_sketch_smem(ctx))) return rc;
  __nv_bfloat16* Mt = (__nv_bfloat16*)ctx->d_sketch_ws;
  float* part = (float*)((uint8_t*)ctx->d_sketch_ws + mt_bytes);
  const long long tot = (long long)nlam * SK_N * (N / 8);
  k_form_mt<<<(unsigned)std::min<long long>((tot + 255) / 256, 152 * 32), 256, 0, ctx->stream>>>(
      (const __nv_bfloat16*)omega_t, ctx->d_eps, lam0, nlam, ctx->n_chrom, ncols, N, Mt);
  ++ctx->launches;
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  CUtensorMap mapB, mapPs, mapPd;
  if ((rc = encode_b_map(ctx, Mt, N, nlam, &mapB))) return rc;
  if ((rc = encode_f32_map(ctx, ps, N, ctx->n_src, nlam, SK_K, 2 * S_a, &mapPs))) return rc;
  if ((rc = encode_f32_map(ctx, pd, N, nd, nlam, SK_K, D_t, &mapPd))) return rc;
  RangeArgs a{};
  a.ns = ns;
  a.src0 = src0;
  a.nd = nd;
  a.nlam = nlam;
  a.N = N;
  a.S_a = S_a;
  a.D_t = D_t;
  a.nsb = nsb;
  a.ndb = ndb;
  a.nk = nk;
  a.k_per_split = kps;
  a.nsplit = nsplit;
  a.P = P;
  a.out = nsplit > 1 ? part : Y;
  a.ldo = ldY;
  a.scale = (float)(-ctx->h * ctx->h * ctx->h);
  a.err = ctx->d_err;
  HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  if (nd * ns * nlam == 0) return HYDOT_OK;
  cudaEvent_t t0 = timer_begin(ctx);
  k_range_ws<<<(unsigned)(items * nsplit), RG_THREADS, RG_SMEM, ctx->stream>>>(a, mapB, mapPs, mapPd);
  ++ctx->launches;
  if (nsplit > 1) {
    const long long tq = P * (SK_N / 4);
    k_range_reduce<<<(unsigned)std::min<long long>((tq + 255) / 256, 152 * 16), 256, 0, ctx->stream>>>(
        part, nsplit, P, a.scale, Y, ldY);
    ++ctx->launches;
  }
  timer_end(ctx, t0, HYDOT_KERNEL_SKETCH_RANGE, 2.0 * (double)P * (double)N * ncols);
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  return HYDOT_OK;
}

int sketch_project_impl(hydot_ctx* ctx, const float* ps, const float* pd, int lam0, int nlam, int src0, int nsr,
                        const float* Q, int ncols, long long ldQ, float* Bt, long long ldB) {
  int rc = sketch_check(ctx, lam0, nlam, ncols);
  if (rc) return rc;
  if (src0 < 0 || nsr < 1 || src0 + nsr > ctx->n_src) return fail(ctx, HYDOT_ERR_ARG, "source range out of range");
  if (!ps || !pd || !Q || !Bt) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  if (ldB < SK_N || ldQ < ncols) return fail(ctx, HYDOT_ERR_ARG, "ldB must be >= 224 and ldQ >= ncols");
  const long long N = ctx->N;
  const int nc = ctx->n_chrom, ns = nsr, nd = ctx->n_det;
  const long long P = (long long)nlam * ns * nd;
  if ((rc = set_sketch_smem(ctx))) return rc;
  HYDOT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  if (P == 0) return HYDOT_OK;
  const float scale = (float)(-ctx->h * ctx->h * ctx->h);
  if (ns + nd <= 128 && ldB % 4 == 0 && (reinterpret_cast<uintptr_t>(Bt) & 15) == 0) {
    // warp-specialised kernel: per-wavelength pair blocks padded to whole K-steps
    const int Kl = (int)(((long long)ns * nd + SK_K - 1) / SK_K);
    const long long Pl = (long long)Kl * SK_K;
    if ((rc = sketch_ws(ctx, (size_t)nc * SK_N * nlam * Pl * 2))) return rc;
    __nv_bfloat16* Qc = (__nv_bfloat16*)ctx->d_sketch_ws;
    const long long tot = (long long)nc * SK_N * nlam * Pl;
    k_form_qc_padded<<<(unsigned)std::min<long long>((tot + 255) / 256, 152 * 32), 256, 0, ctx->stream>>>(
        Q, ldQ, ctx->d_eps, lam0, nlam, ns, nd, nc, ncols, Pl, Qc);
    ++ctx->launches;
    HYDOT_CUDA_TRY(ctx, cudaGetLastError());
    CUtensorMap mapB, mapPs, mapPd;
    if ((rc = encode_b_map(ctx, Qc, nlam * Pl, nc, &mapB))) return rc;
    if ((rc = encode_f32_map(ctx, ps, N, ctx->n_src, nlam, PJ_M, ns, &mapPs))) return rc;
    if ((rc = encode_f32_map(ctx, pd, N, nd, nlam, PJ_M, nd, &mapPd))) return rc;
    CUtensorMap mapBt0, mapBt1;
    if ((rc = encode_bt_map(ctx, Bt, N, nc, ldB, PJ_BT0_COLS, &mapBt0))) return rc;
    if ((rc = encode_bt_map(ctx, Bt, N, nc, ldB, SK_N - PJ_BT0_COLS, &mapBt1))) return rc;
    ProjArgs a{};
    a.ns = ns;
    a.src0 = src0;
    a.nd = nd;
    a.nlam = nlam;
    a.nc = nc;
    a.Kl = Kl;
    a.N = N;
    a.Bt = Bt;
    a.ldB = ldB;
    a.scale = scale;
    a.err = ctx->d_err;
    const long long grid = ((N + PJ_M - 1) / PJ_M) * ((nc + 1) / 2);
    cudaEvent_t t0 = timer_begin(ctx);
    k_project_ws<<<(unsigned)grid, PJ_THREADS, PJ_SMEM, ctx->stream>>>(a, mapB, mapPs, mapPd, mapBt0, mapBt1);
    ++ctx->launches;
    timer_end(ctx, t0, HYDOT_KERNEL_SKETCH_PROJECT, 2.0 * (double)nc * (double)N * (double)P * ncols);
    HYDOT_CUDA_TRY(ctx, cudaGetLastError());
    return HYDOT_OK;
  }
  // general shapes: one launch per chromophore, A tiles formed from global loads
  const long long Pp = (P + 7) / 8 * 8;
  if ((rc = sketch_ws(ctx, (size_t)nc * SK_N * Pp * 2))) return rc;
  __nv_bfloat16* Qc = (__nv_bfloat16*)ctx->d_sketch_ws;
  const long long tot = (long long)nc * SK_N * Pp;
  k_form_qc<<<(unsigned)std::min<long long>((tot + 255) / 256, 152 * 32), 256, 0, ctx->stream>>>(
      Q, ldQ, ctx->d_eps, lam0, nlam, ns, nd, nc, ncols, P, Pp, Qc);
  ++ctx->launches;
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  CUtensorMap map;
  if ((rc = encode_b_map(ctx, Qc, Pp, nc, &map))) return rc;
  SketchArgs a{};
  a.ps = ps;
  a.pd = pd;
  a.ns = ns;
  a.nsf = ctx->n_src;
  a.src0 = src0;
  a.nd = nd;
  a.nlam = nlam;
  a.N = N;
  a.P = P;
  a.scale = scale;
  a.out = Bt;
  a.ldo = ldB;
  a.err = ctx->d_err;
  const unsigned grid = (unsigned)((N + SK_M - 1) / SK_M);
  cudaEvent_t t0 = timer_begin(ctx);
  for (int c = 0; c < nc; ++c) {
    a.chrom = c;
    k_project_generic<<<grid, 128, SK_SMEM, ctx->stream>>>(a, map);
    ++ctx->launches;
  }
  timer_end(ctx, t0, HYDOT_KERNEL_SKETCH_PROJECT, 2.0 * (double)nc * (double)N * (double)P * ncols);
  HYDOT_CUDA_TRY(ctx, cudaGetLastError());
  return HYDOT_OK;
}

}  // namespace hydot

// ---------------------------------------------------------------- tall-skinny helpers
// Orthonormalisation of the range sketch, the final factors and the merges use the n x n (n <= 224)
// Gram matrices and cross products of tall-skinny operands: FP32 products summed in FP32 within
// 64-row blocks and in FP64 across blocks (the Gram squares the condition number; the second round
// of the orthonormalisation restores what the block sums lose), and products with small n x m
// matrices.
namespace hydot {
namespace {

constexpr int GT = 32;  // Gram tile (columns)

// partial[chunk][pair][GT][GT] = X[rows of chunk][tile i]^T X[rows of chunk][tile j], pair = (i <= j)
__global__ void __launch_bounds__(256) k_gram64(const float* __restrict__ X, long long rows, long long ldx, int n,
                                                int ntile, long long rows_per_chunk, double* __restrict__ part) {
  __shared__ float Xi[64][GT + 1], Xj[64][GT + 1];
  const int chunk = blockIdx.x, pair = blockIdx.y;
  int ti = 0, rem = pair;
  while (rem >= ntile - ti) {
    rem -= ntile - ti;
    ++ti;
  }
  const int tj = ti + rem;
  const int t = threadIdx.x;
  const int ii = t >> 3, jj = (t & 7) * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long r0 = (long long)chunk * rows_per_chunk;
  const long long r1 = min(rows, r0 + rows_per_chunk);
  for (long long rb = r0; rb < r1; rb += 64) {
    for (int q = t; q < 64 * GT; q += 256) {
      const int rr = q / GT, cc = q % GT;
      const long long r = rb + rr;
      const int ci = ti * GT + cc, cj = tj * GT + cc;
      Xi[rr][cc] = (r < r1 && ci < n) ? X[r * ldx + ci] : 0.f;
      Xj[rr][cc] = (r < r1 && cj < n) ? X[r * ldx + cj] : 0.f;
    }
    __syncthreads();
    // FP32 products and sums within the 64-row block, FP64 across blocks (GB300's FP64 rate is
    // ~1/64 of FP32; the block sums carry ~1e-6 relative error)
    float blk[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int rr = 0; rr < 64; ++rr) {
      const float a = Xi[rr][ii];
#pragma unroll
      for (int q = 0; q < 4; ++q) blk[q] = fmaf(a, Xj[rr][jj + q], blk[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += (double)blk[q];
    __syncthreads();
  }
  double* out = part + (((size_t)chunk * gridDim.y + pair) * GT + ii) * GT + jj;
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = acc[q];
}

__global__ void k_gram_reduce(const double* __restrict__ part, int nchunk, int npair, int ntile, int n,
                              double* __restrict__ G) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npair * GT * GT) return;
  const int pair = idx / (GT * GT), ij = idx % (GT * GT), ii = ij / GT, jj = ij % GT;
  int ti = 0, rem = pair;
  while (rem >= ntile - ti) {
    rem -= ntile - ti;
    ++ti;
  }
  const int tj = ti + rem;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[((size_t)c * npair + pair) * GT * GT + ij];
  const int a = ti * GT + ii, b = tj * GT + jj;
  if (a < n && b < n) {
    G[(size_t)a * n + b] = s;
    G[(size_t)b * n + a] = s;
  }
}

// partial[chunk][ti][tj][GT][GT] = X[rows of chunk][tile ti]^T Y[rows of chunk][tile tj] (FP64 across blocks)
__global__ void __launch_bounds__(256) k_cross64(const float* __restrict__ X, long long ldx, int nx,
                                                 const float* __restrict__ Y, long long ldy, int ny, long long rows,
                                                 long long rows_per_chunk, double* __restrict__ part) {
  __shared__ float Xi[64][GT + 1], Yj[64][GT + 1];
  const int chunk = blockIdx.x, ti = blockIdx.y, tj = blockIdx.z;
  const int t = threadIdx.x;
  const int ii = t >> 3, jj = (t & 7) * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long r0 = (long long)chunk * rows_per_chunk;
  const long long r1 = min(rows, r0 + rows_per_chunk);
  for (long long rb = r0; rb < r1; rb += 64) {
    for (int q = t; q < 64 * GT; q += 256) {
      const int rr = q / GT, cc = q % GT;
      const long long r = rb + rr;
      const int ci = ti * GT + cc, cj = tj * GT + cc;
      Xi[rr][cc] = (r < r1 && ci < nx) ? X[r * ldx + ci] : 0.f;
      Yj[rr][cc] = (r < r1 && cj < ny) ? Y[r * ldy + cj] : 0.f;
    }
    __syncthreads();
    float blk[4] = {0.f, 0.f, 0.f, 0.f};  // FP32 within the block, FP64 across blocks
#pragma unroll 4
    for (int rr = 0; rr < 64; ++rr) {
      const float a = Xi[rr][ii];
#pragma unroll
      for (int q = 0; q < 4; ++q) blk[q] = fmaf(a, Yj[rr][jj + q], blk[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += (double)blk[q];
    __syncthreads();
  }
  double* out = part + ((((size_t)chunk * gridDim.y + ti) * gridDim.z + tj) * GT + ii) * GT + jj;
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = acc[q];
}

__global__ void k_cross_reduce(const double* __restrict__ part, int nchunk, int ntx, int nty, int nx, int ny,
                               double* __restrict__ G) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ntx * nty * GT * GT) return;
  const int tile = idx / (GT * GT), ij = idx % (GT * GT), ii = ij / GT, jj = ij % GT;
  const int ti = tile / nty, tj = tile % nty;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[((size_t)c * ntx * nty + tile) * GT * GT + ij];
  const int a = ti * GT + ii, b = tj * GT + jj;
  if (a < nx && b < ny) G[(size_t)a * ny + b] = s;
}

// Z[r][j] (+)= sum_k X[r][k] W[k][j] for j < m (Z columns m..ldz-1 untouched), FP32.
__global__ void __launch_bounds__(256) k_right_mul(const float* __restrict__ X, long long rows, long long ldx, int n,
                                                   const float* __restrict__ W, int m, float* __restrict__ Z,
                                                   long long ldz, int accumulate) {
  __shared__ float Xs[64][33];
  __shared__ float Ws[32][64];
  const int t = threadIdx.x, tr = t >> 4, tc = t & 15;
  const long long r0 = (long long)blockIdx.x * 64;
  const int c0 = blockIdx.y * 64;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int q = t; q < 64 * 32; q += 256) {
      const int rr = q / 32, kk = q % 32;
      const long long r = r0 + rr;
      Xs[rr][kk] = (r < rows && k0 + kk < n) ? X[r * ldx + k0 + kk] : 0.f;
    }
    for (int q = t; q < 32 * 64; q += 256) {
      const int kk = q / 64, cc = q % 64;
      Ws[kk][cc] = (k0 + kk < n && c0 + cc < m) ? W[(size_t)(k0 + kk) * m + c0 + cc] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      float a[4], w[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) a[u] = Xs[tr * 4 + u][kk];
#pragma unroll
      for (int v = 0; v < 4; ++v) w[v] = Ws[kk][tc * 4 + v];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], w[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const long long r = r0 + tr * 4 + u;
    if (r >= rows) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int c = c0 + tc * 4 + v;
      if (c < m) Z[r * ldz + c] = accumulate ? Z[r * ldz + c] + acc[u][v] : acc[u][v];
    }
  }
}

// G = X[:, :n]^T X[:, :n] (n x n, FP64) to the host.
int gram(hydot_ctx* ctx, const float* X, long long rows, long long ldx, int n, std::vector<double>& G) {
  const int ntile = (n + GT - 1) / GT;
  const int npair = ntile * (ntile + 1) / 2;
  const long long want = std::max<long long>(1, 4 * 152 / npair);
  const long long nchunk = std::max<long long>(1, std::min<long long>(want, (rows + 63) / 64));
  const long long rpc = ((rows + nchunk - 1) / nchunk + 63) / 64 * 64;
  const long long nch = (rows + rpc - 1) / rpc;
  double *part = nullptr, *dG = nullptr;
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&part, sizeof(double) * (size_t)nch * npair * GT * GT));
  cudaError_t e = cudaMalloc(&dG, sizeof(double) * (size_t)n * n);
  if (e != cudaSuccess) {
    cudaFree(part);
    return fail(ctx, HYDOT_ERR_OOM, "cudaMalloc of the Gram matrix failed");
  }
  k_gram64<<<dim3((unsigned)nch, npair), 256, 0, ctx->stream>>>(X, rows, ldx, n, ntile, rpc, part);
  k_gram_reduce<<<(npair * GT * GT + 255) / 256, 256, 0, ctx->stream>>>(part, (int)nch, npair, ntile, n, dG);
  ctx->launches += 2;
  G.assign((size_t)n * n, 0.0);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(G.data(), dG, sizeof(double) * n * n, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(part);
  cudaFree(dG);
  if (e != cudaSuccess) return fail(ctx, HYDOT_ERR_CUDA, std::string("Gram: ") + cudaGetErrorString(e));
  return HYDOT_OK;
}

// C = X[:, :nx]^T Y[:, :ny] (nx x ny, FP64, row-major) to the host.
int cross(hydot_ctx* ctx, const float* X, long long ldx, int nx, const float* Y, long long ldy, int ny, long long rows,
          std::vector<double>& Cm) {
  const int ntx = (nx + GT - 1) / GT, nty = (ny + GT - 1) / GT;
  const long long want = std::max<long long>(1, 4 * 152 / (ntx * nty));
  const long long nchunk = std::max<long long>(1, std::min<long long>(want, (rows + 63) / 64));
  const long long rpc = ((rows + nchunk - 1) / nchunk + 63) / 64 * 64;
  const long long nch = (rows + rpc - 1) / rpc;
  double *part = nullptr, *dC = nullptr;
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&part, sizeof(double) * (size_t)nch * ntx * nty * GT * GT));
  cudaError_t e = cudaMalloc(&dC, sizeof(double) * (size_t)nx * ny);
  if (e != cudaSuccess) {
    cudaFree(part);
    return fail(ctx, HYDOT_ERR_OOM, "cudaMalloc of a cross product failed");
  }
  k_cross64<<<dim3((unsigned)nch, ntx, nty), 256, 0, ctx->stream>>>(X, ldx, nx, Y, ldy, ny, rows, rpc, part);
  k_cross_reduce<<<(ntx * nty * GT * GT + 255) / 256, 256, 0, ctx->stream>>>(part, (int)nch, ntx, nty, nx, ny, dC);
  ctx->launches += 2;
  Cm.assign((size_t)nx * ny, 0.0);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(Cm.data(), dC, sizeof(double) * nx * ny, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(part);
  cudaFree(dC);
  if (e != cudaSuccess) return fail(ctx, HYDOT_ERR_CUDA, std::string("cross: ") + cudaGetErrorString(e));
  return HYDOT_OK;
}

// Z = X W (or Z += X W) with W (n x m) given on the host.
int right_mul(hydot_ctx* ctx, const float* X, long long rows, long long ldx, int n, const std::vector<float>& W, int m,
              float* Z, long long ldz, bool accumulate = false) {
  float* dW = nullptr;
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&dW, sizeof(float) * (size_t)n * m));
  cudaError_t e = cudaMemcpyAsync(dW, W.data(), sizeof(float) * (size_t)n * m, cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) {
    k_right_mul<<<dim3((unsigned)((rows + 63) / 64), (m + 63) / 64), 256, 0, ctx->stream>>>(X, rows, ldx, n, dW, m, Z, ldz,
                                                                                          accumulate ? 1 : 0);
    ++ctx->launches;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(dW);
  if (e != cudaSuccess) return fail(ctx, HYDOT_ERR_CUDA, std::string("right_mul: ") + cudaGetErrorString(e));
  return HYDOT_OK;
}

// eigen-pairs of a symmetric n x n matrix, descending
// (false when the host eigensolver did not converge)
bool eig_desc(const std::vector<double>& G, int n, std::vector<double>& lam, std::vector<double>& V) {
  std::vector<double> l, Z;
  if (!sym_eig(G, n, l, Z)) return false;
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return l[a] > l[b]; });
  lam.resize(n);
  V.assign((size_t)n * n, 0.0);
  for (int j = 0; j < n; ++j) {
    lam[j] = l[ord[j]];
    for (int i = 0; i < n; ++i) V[(size_t)i * n + j] = Z[(size_t)i * n + ord[j]];
  }
  return true;
}

}  // namespace

// Orthonormal basis of range(Y) in place: two rounds of Y <- Y V_k diag(lambda_k^-1/2) from the FP64
// Gram Y^T Y = V diag(lambda) V^T, keeping the directions whose singular value exceeds 1e-6 of the
// largest (the rest are set to zero columns). *rank_out receives the number kept.
int sketch_orthonormalize_impl(hydot_ctx* ctx, float* Y, long long rows, int ncols, long long ldY, int* rank_out,
                               double* smax_out) {
  if (!Y || rows < 1 || ncols < 1 || ncols > SK_N || ldY < ncols) return fail(ctx, HYDOT_ERR_ARG, "bad Y shape");
  float* Z = nullptr;
  HYDOT_CUDA_TRY(ctx, cudaMalloc(&Z, sizeof(float) * (size_t)rows * ncols));
  int kept = ncols;
  for (int round = 0; round < 2; ++round) {
    std::vector<double> G, lam, V;
    int rc = gram(ctx, Y, rows, ldY, ncols, G);
    if (rc) { cudaFree(Z); return rc; }
    if (!eig_desc(G, ncols, lam, V)) {
      cudaFree(Z);
      return fail(ctx, HYDOT_ERR_NOT_CONVERGED, "host eigensolver did not converge on the Gram of Y");
    }
    const double smax = std::sqrt(std::max(lam[0], 0.0));
    if (round == 0 && smax_out) *smax_out = smax;
    kept = 0;
    std::vector<float> W((size_t)ncols * ncols, 0.f);
    for (int j = 0; j < ncols; ++j) {
      const double sj = std::sqrt(std::max(lam[j], 0.0));
      if (!(sj > 1e-6 * smax) || smax == 0.0) break;
      ++kept;
      for (int i = 0; i < ncols; ++i) W[(size_t)i * ncols + j] = (float)(V[(size_t)i * ncols + j] / sj);
    }
    rc = right_mul(ctx, Y, rows, ldY, ncols, W, ncols, Z, ncols);
    if (!rc) {
      cudaError_t e = cudaMemcpy2DAsync(Y, sizeof(float) * ldY, Z, sizeof(float) * ncols, sizeof(float) * ncols, rows,
                                        cudaMemcpyDeviceToDevice, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) rc = fail(ctx, HYDOT_ERR_CUDA, std::string("copy: ") + cudaGetErrorString(e));
    }
    if (rc) { cudaFree(Z); return rc; }
  }
  cudaFree(Z);
  if (rank_out) *rank_out = kept;
  return HYDOT_OK;
}

// Rank-r factors from the projected sketch: with B = Q^T J (given as Bt = B^T, nb x ncols) the Gram
// B B^T = U_B diag(S^2) U_B^T gives S, V = B^T U_B diag(1/S) and U = Q U_B, so J ~ U diag(S) V^T
// (the final recompression of Section 4.4, truncated to `rank`).
int sketch_factor_impl(hydot_ctx* ctx, const float* Q, long long rows, long long ldQ, const float* Bt, long long nb,
                       long long ldB, int ncols, int rank, float* U, long long ldU, double* S, float* V, long long ldV) {
  if (!Q || !Bt || !U || !S || !V) return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  if (ncols < 1 || ncols > SK_N || rank < 1 || rank > ncols || ldQ < ncols || ldB < ncols || ldU < rank || ldV < rank)
    return fail(ctx, HYDOT_ERR_ARG, "bad sketch factor shapes");
  std::vector<double> G, lam, UB;
  int rc = gram(ctx, Bt, nb, ldB, ncols, G);
  if (rc) return rc;
  if (!eig_desc(G, ncols, lam, UB))
    return fail(ctx, HYDOT_ERR_NOT_CONVERGED, "host eigensolver did not converge on the Gram of B");
  std::vector<float> WV((size_t)ncols * rank, 0.f), WU((size_t)ncols * rank, 0.f);
  for (int j = 0; j < rank; ++j) {
    const double sj = std::sqrt(std::max(lam[j], 0.0));
    S[j] = sj;
    for (int i = 0; i < ncols; ++i) {
      WU[(size_t)i * rank + j] = (float)UB[(size_t)i * ncols + j];
      WV[(size_t)i * rank + j] = sj > 0.0 ? (float)(UB[(size_t)i * ncols + j] / sj) : 0.f;
    }
  }
  rc = right_mul(ctx, Bt, nb, ldB, ncols, WV, rank, V, ldV);
  if (!rc) rc = right_mul(ctx, Q, rows, ldQ, ncols, WU, rank, U, ldU);
  return rc;
}

// Adaptive rank (Appendix A.1, alg:randsvd error estimator): with Q the orthonormal basis of range(A
// Omega_1) (columns in descending singular-value order) and Y2 = A Omega_2 for k further Gaussian
// columns, the smallest r with e_r = || Y2 - Q_r Q_r^T Y2 ||_2 <= tol * s1. Because Q is orthonormal,
// (Y2 - Q_r Q_r^T Y2)^T (Y2 - Q_r Q_r^T Y2) = Y2^T Y2 - sum_(i<r) c_i c_i^T with c_i = Q[:, i]^T Y2, so all
// e_r follow from the k x k Gram of Y2 and the nq x k product Q^T Y2 (both FP64).
int sketch_rank_impl(hydot_ctx* ctx, const float* Q, long long ldQ, long long rows, int nq, const float* Y2,
                     long long ldY2, int k, double s1, double tol, int* rank, double* estimate) {
  if (!Q || !Y2 || !rank || rows < 1 || nq < 1 || nq > SK_N || k < 1 || k > 32 || ldQ < nq || ldY2 < k)
    return fail(ctx, HYDOT_ERR_ARG, "bad arguments to the rank estimator");
  std::vector<double> C, G2;
  int rc = cross(ctx, Q, ldQ, nq, Y2, ldY2, k, rows, C);
  if (!rc) rc = cross(ctx, Y2, ldY2, k, Y2, ldY2, k, rows, G2);
  if (rc) return rc;
  std::vector<double> R = G2, lam, V;
  int r = 0;
  double e = 0.0;
  for (;; ++r) {
    if (!sym_eig(R, k, lam, V))
      return fail(ctx, HYDOT_ERR_NOT_CONVERGED, "host eigensolver did not converge in the rank estimator");
    double lmax = 0.0;
    for (double v : lam) lmax = std::max(lmax, v);
    e = std::sqrt(std::max(lmax, 0.0));
    if (e <= tol * s1 || r == nq) break;
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) R[(size_t)a * k + b] -= C[(size_t)r * k + a] * C[(size_t)r * k + b];
  }
  *rank = std::max(r, 1);
  if (estimate) *estimate = s1 > 0.0 ? e / s1 : 0.0;
  return HYDOT_OK;
}

// Agglomeration of two low-rank factorisations of stacked row blocks (Section 4.3):
//   [H1; H2] ~ [U1 S1 V1^T; U2 S2 V2^T] = blockdiag(U1, U2) W,  W = [S1 V1^T; S2 V2^T].
// W W^T = [[S1 V1^T V1 S1, S1 V1^T V2 S2], [S2 V2^T V1 S1, S2 V2^T V2 S2]] ((r1+r2)^2, FP64 from the
// tall-skinny products) = E diag(lambda) E^T; keeping the r directions with sqrt(lambda_i) >
// tol * sqrt(lambda_1) (at most max_rank) gives W ~ E_r diag(S) V^T with S = sqrt(lambda_r) and
// V = W^T E_r diag(1/S), hence U = blockdiag(U1, U2) E_r: the merged factors are again a truncated SVD.
int sketch_merge_impl(hydot_ctx* ctx, const float* U1, long long ldU1, long long m1, const double* S1, const float* V1,
                      long long ldV1, int r1, const float* U2, long long ldU2, long long m2, const double* S2,
                      const float* V2, long long ldV2, int r2, long long n, double tol, int max_rank, float* U,
                      long long ldU, double* S, float* V, long long ldV, int* rank_out) {
  if (!U1 || !S1 || !V1 || !U2 || !S2 || !V2 || !U || !S || !V || !rank_out)
    return fail(ctx, HYDOT_ERR_ARG, "null pointer");
  const int rt = r1 + r2;
  if (r1 < 1 || r2 < 1 || rt > 2 * SK_N || max_rank < 1 || m1 < 1 || m2 < 1 || n < 1 || ldU1 < r1 || ldU2 < r2 ||
      ldV1 < r1 || ldV2 < r2)
    return fail(ctx, HYDOT_ERR_ARG, "bad factor shapes for the merge");
  std::vector<double> C12, G11, G22;
  int rc = cross(ctx, V1, ldV1, r1, V2, ldV2, r2, n, C12);
  if (!rc) rc = cross(ctx, V1, ldV1, r1, V1, ldV1, r1, n, G11);
  if (!rc) rc = cross(ctx, V2, ldV2, r2, V2, ldV2, r2, n, G22);
  if (rc) return rc;
  std::vector<double> G((size_t)rt * rt, 0.0);
  for (int i = 0; i < r1; ++i)
    for (int j = 0; j < r1; ++j) G[(size_t)i * rt + j] = S1[i] * G11[(size_t)i * r1 + j] * S1[j];
  for (int i = 0; i < r2; ++i)
    for (int j = 0; j < r2; ++j) G[(size_t)(r1 + i) * rt + r1 + j] = S2[i] * G22[(size_t)i * r2 + j] * S2[j];
  for (int i = 0; i < r1; ++i)
    for (int j = 0; j < r2; ++j) {
      const double v = S1[i] * C12[(size_t)i * r2 + j] * S2[j];
      G[(size_t)i * rt + r1 + j] = v;
      G[(size_t)(r1 + j) * rt + i] = v;
    }
  std::vector<double> lam, E;
  if (!eig_desc(G, rt, lam, E))
    return fail(ctx, HYDOT_ERR_NOT_CONVERGED, "host eigensolver did not converge on the merge Gram");
  const double s_1 = std::sqrt(std::max(lam[0], 0.0));
  int r = 0;
  while (r < rt && r < max_rank && std::sqrt(std::max(lam[r], 0.0)) > tol * s_1 && lam[r] > 0.0) ++r;
  r = std::max(r, 1);
  if (ldU < r || ldV < r) return fail(ctx, HYDOT_ERR_ARG, "ldU / ldV smaller than the merged rank");
  std::vector<float> E1((size_t)r1 * r), E2((size_t)r2 * r), W1((size_t)r1 * r), W2((size_t)r2 * r);
  for (int j = 0; j < r; ++j) {
    const double sj = std::sqrt(std::max(lam[j], 0.0));
    S[j] = sj;
    for (int i = 0; i < r1; ++i) {
      E1[(size_t)i * r + j] = (float)E[(size_t)i * rt + j];
      W1[(size_t)i * r + j] = sj > 0.0 ? (float)(S1[i] * E[(size_t)i * rt + j] / sj) : 0.f;
    }
    for (int i = 0; i < r2; ++i) {
      E2[(size_t)i * r + j] = (float)E[(size_t)(r1 + i) * rt + j];
      W2[(size_t)i * r + j] = sj > 0.0 ? (float)(S2[i] * E[(size_t)(r1 + i) * rt + j] / sj) : 0.f;
    }
  }
  rc = right_mul(ctx, U1, m1, ldU1, r1, E1, r, U, ldU);
  if (!rc) rc = right_mul(ctx, U2, m2, ldU2, r2, E2, r, U + m1 * ldU, ldU);
  if (!rc) rc = right_mul(ctx, V1, n, ldV1, r1, W1, r, V, ldV);
  if (!rc) rc = right_mul(ctx, V2, n, ldV2, r2, W2, r, V, ldV, true);
  if (rc) return rc;
  *rank_out = r;
  return HYDOT_OK;
}

// C = X^T Y for tall-skinny FP32 X [rows][nx] and Y [rows][ny] (row strides ldx, ldy): FP32
// products summed in FP64 across 64-row blocks and chunks, in a fixed order; C on the host [nx][ny].
int tall_cross(hydot_ctx* ctx, const float* X, long long ldx, int nx, const float* Y, long long ldy, int ny,
               long long rows, std::vector<double>& C) {
  return cross(ctx, X, ldx, nx, Y, ldy, ny, rows, C);
}


// ---------------------------------------------------------------- source tree (alg:geom)
namespace {
struct TreeBuild {
  const double* xy;
  int leaf_max;
  int* order;
  int* nodes;
  int pos = 0, cnt = 0;
};

// Node of the positions idx inside the box [lo, hi]; returns its index (a split with one empty side
// returns the other side's node).
int tree_split(TreeBuild& t, const std::vector<int>& idx, std::array<double, 2> lo, std::array<double, 2> hi,
               int depth) {
  const int start = t.pos;
  if ((int)idx.size() <= t.leaf_max || depth > 64) {
    for (int i : idx) t.order[t.pos++] = i;
    const int id = t.cnt++;
    t.nodes[4 * id] = start;
    t.nodes[4 * id + 1] = t.pos;
    t.nodes[4 * id + 2] = t.nodes[4 * id + 3] = -1;
    return id;
  }
  const int j = (hi[0] - lo[0] >= hi[1] - lo[1]) ? 0 : 1;  // direction of the larger extent
  const double gamma = 0.5 * (lo[j] + hi[j]);                 // midpoint split
  std::vector<int> t1, t2;
  for (int i : idx) (t.xy[2 * i + j] <= gamma ? t1 : t2).push_back(i);
  std::array<double, 2> hi1 = hi, lo2 = lo;
  hi1[j] = gamma;
  lo2[j] = gamma;
  int kids[2], nk = 0;
  if (!t1.empty()) kids[nk++] = tree_split(t, t1, lo, hi1, depth + 1);
  if (!t2.empty()) kids[nk++] = tree_split(t, t2, lo2, hi, depth + 1);
  if (nk == 1) return kids[0];
  const int id = t.cnt++;
  t.nodes[4 * id] = start;
  t.nodes[4 * id + 1] = t.pos;
  t.nodes[4 * id + 2] = kids[0];
  t.nodes[4 * id + 3] = kids[1];
  return id;
}
}  // namespace

int source_tree_impl(const double* xy, int n, double x_lo, double y_lo, double x_hi, double y_hi, int leaf_max,
                     int* order, int* nodes, int* n_nodes, int* root) {
  if (!xy || !order || !nodes || !n_nodes || !root || n < 1 || leaf_max < 1) {
    set_context_free_error("hydot_source_tree: null pointer, n < 1 or leaf_max < 1");
    return HYDOT_ERR_ARG;
  }
  TreeBuild t{xy, leaf_max, order, nodes};
  std::vector<int> all((size_t)n);
  for (int i = 0; i < n; ++i) all[(size_t)i] = i;
  *root = tree_split(t, all, {x_lo, y_lo}, {x_hi, y_hi}, 0);
  *n_nodes = t.cnt;
  return HYDOT_OK;
}

}  // namespace hydot
