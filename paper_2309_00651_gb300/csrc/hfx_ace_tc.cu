// The two grid-sized contractions of the ACE operator (Sec. 2.1, Eq. vx_ace: M = <psi|W>, the
// screen's |psi_i||psi_j| sums, P = W L^-T and V_x^ACE psi = -P <P|psi>) on the fifth-generation
// tensor cores, for FP32 contexts: TF32 x 3 split products with FP32 accumulation in TMEM.
//
// Every FP64 operand value is rounded once to FP32 and split into two TF32 values, hi + lo
// (tc::split_tf32); a product is formed as hi.hi + hi.lo + lo.hi, which reproduces the FP32
// product to about 2^-21 relative.  The tensor core rounds each addition into its FP32
// accumulator toward zero, so a long accumulation drifts: about half a unit of the running sum
// per MMA, always in the same direction (measured: 6e-6 on the 373248-point Gram of 128 water
// orbitals when one accumulator took a whole run).  Hence the hi.hi products and the two
// correction products (2^-10 smaller) go to separate accumulators, and the Gram form restarts
// its accumulators every k-block of 32 points and adds them to round-to-nearest FP32 sums in
// registers (4 MMAs per accumulator and k-block: about 1e-7 of drift).  The left multiply
// contracts over the orbitals only (K <= a few hundred) and keeps its accumulators for the job.
//
// Block: 256 threads (8 warps), one per SM (two pipeline stages of shared memory).  Per k-block
// of 32 contraction steps the threads load the FP64 operands of the next k-block into registers
// while the tensor core works on the current one, then round, split and store them into the
// stage's SWIZZLE_128B K-major tiles; thread 0 issues the MMAs and commits them to the stage's
// mbarrier, which the threads wait on before they overwrite that stage two k-blocks later.  Every
// wait has an iteration limit: a wait that runs out sets the timeout bit of the error word, the
// block drains its MMAs (again with a limit), frees its TMEM and returns.
//
//   Gram form (k_gram_tc): one job = output tile (a, b) of 128 x 128 over one run of grid points;
//     A = X rows, B = Y rows (both K-major as stored); the FP32 accumulator of the job is
//     widened exactly and written as the job's FP64 partial (summed in a fixed order later).
//   Left multiply (k_lmul_tc): one job = 128 grid points p (the MMA's M) x all m (its N, <= 256);
//     A[p][k] = Y[k][p] (transposed while it is stored), B[m][k] = T[m][k] from the transposed
//     FP32 copy tt[k][m]; D[p][m] is written to C[m][p] with lanes on consecutive p (coalesced).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fp_convert.cuh"
#include "hfx_ace_internal.h"
#include "hfx_kernels.cuh"
#include "tc_sm100.cuh"

namespace hfx {
namespace ace {

namespace {

constexpr int kTcThreads = 256;
constexpr int kTcBK = 32;                   // contraction steps per k-block (128 bytes of TF32)
constexpr int kTcTile = 128;                // the MMA's M, and N of the Gram form
constexpr long long kWaitLimit = 1LL << 26; // polls of one mbarrier wait before giving up
constexpr uint32_t kTileBytes = 16384;      // one 128-row operand tile

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return (unsigned char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

template <bool ABS>
__device__ __forceinline__ float to_f32(double v) {
  return f64_to_f32_rn(ABS ? fabs(v) : v);
}

}  // namespace

// ------------------------------------------------------------------------------------
// Gram form: partial C[a][b] = sum_{p in run} X[a][p] Y[b][p]
// ------------------------------------------------------------------------------------
template <bool ABS>
__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(const MmArgs a, int* err) {
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* base = align1024(smem_dyn);  // stage st: [A hi | A lo | B hi | B lo] at st * 64 KiB
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init_fence();
    s_abort = 0;
  }
  // TMEM: k-block buffer b in {0, 1}: hi.hi accumulator at column 256 b, corrections at 256 b + 128
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = tc::idesc_tf32(kTcTile, kTcTile);
  const double* X = reinterpret_cast<const double*>(a.x);
  const int cp = tid & 15, r0 = tid >> 4;  // loads: column pair cp, rows r0 + 16 i
  const int q = warp & 3, h = warp >> 2;   // drains: TMEM lanes 32q.. (rows a), columns 64h.. (b)
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  const int tiles = a.tiles_x * a.tiles_y;

  long long g = 0;  // k-blocks this block has issued: stage and TMEM buffer g & 1, use g >> 1
  bool aborted = false;
  double2 xr[8], yr[8];
  float acc[64];
  // k-block g - 1's products (its commit) into the round-to-nearest sums
  auto drain = [&](long long gd) -> bool {
    if (!tc::mbar_wait(&mbar[gd & 1], (uint32_t)((gd >> 1) & 1), kWaitLimit)) return false;
    tc::fence_after_sync();
    const uint32_t tb0 = tmem + lane_off + 256u * (uint32_t)(gd & 1) + 64u * h;
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      float vm[32], vc[32];
      tc::tmem_ld32(tb0 + 32u * cc, vm);
      tc::tmem_ld32(tb0 + 128u + 32u * cc, vc);
#pragma unroll
      for (int j = 0; j < 32; ++j) acc[32 * cc + j] += vm[j] + vc[j];
    }
    tc::fence_before_sync();
    return true;
  };
  for (int job = blockIdx.x; job < a.njobs && !aborted; job += gridDim.x) {
    const int s = job / tiles, t = job - s * tiles;
    const int ta = t % a.tiles_x, tb = t / a.tiles_x;
    const long long p0 = (long long)s * a.chunk, p1 = min(a.K, p0 + a.chunk);
    const int nkb = (int)((p1 - p0 + kTcBK - 1) / kTcBK);
#pragma unroll
    for (int j = 0; j < 64; ++j) acc[j] = 0.f;
    auto load = [&](int kb) {
      const long long p = p0 + (long long)kb * kTcBK + 2 * cp;
      const bool pin = p < p1;  // runs start and end on even points, so p + 1 < p1 as well
      const double2 zero = make_double2(0.0, 0.0);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = r0 + 16 * i;
        const int ga = ta * kTcTile + r, gb = tb * kTcTile + r;
        xr[i] = (pin && ga < a.nx) ? __ldcs(reinterpret_cast<const double2*>(X + (long long)ga * a.ldx + p)) : zero;
        yr[i] = (pin && gb < a.ny) ? __ldcs(reinterpret_cast<const double2*>(a.y + (long long)gb * a.ldy + p)) : zero;
      }
    };
    load(0);
    for (int kb = 0; kb < nkb; ++kb, ++g) {
      const int st = (int)(g & 1);
      unsigned char* sah = base + st * 4 * kTileBytes;
      unsigned char* sal = sah + kTileBytes;
      unsigned char* sbh = sah + 2 * kTileBytes;
      unsigned char* sbl = sah + 3 * kTileBytes;
      // stage st and TMEM buffer st were last used by k-block g - 2, drained in the previous
      // iteration (or at the end of the previous job)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = r0 + 16 * i;
        const uint32_t o = tc::swz128(r, 2 * cp);
        float h0, l0, h1, l1;
        tc::split_tf32(to_f32<ABS>(xr[i].x), h0, l0);
        tc::split_tf32(to_f32<ABS>(xr[i].y), h1, l1);
        *reinterpret_cast<float2*>(sah + o) = make_float2(h0, h1);
        *reinterpret_cast<float2*>(sal + o) = make_float2(l0, l1);
        tc::split_tf32(to_f32<ABS>(yr[i].x), h0, l0);
        tc::split_tf32(to_f32<ABS>(yr[i].y), h1, l1);
        *reinterpret_cast<float2*>(sbh + o) = make_float2(h0, h1);
        *reinterpret_cast<float2*>(sbl + o) = make_float2(l0, l1);
      }
      tc::fence_proxy_async();
      __syncthreads();
      if (s_abort) { aborted = true; break; }
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t ah = tc::smem_u32(sah), al = tc::smem_u32(sal), bh = tc::smem_u32(sbh), bl = tc::smem_u32(sbl);
        const uint32_t dm = tmem + 256u * (uint32_t)st, dc = dm + 128u;
#pragma unroll
        for (int ks = 0; ks < kTcBK / 8; ++ks) {
          const uint32_t off = 32u * ks;
          tc::mma_tf32(dm, tc::desc_sw128(ah + off), tc::desc_sw128(bh + off), idesc, ks > 0 ? 1u : 0u);
          tc::mma_tf32(dc, tc::desc_sw128(ah + off), tc::desc_sw128(bl + off), idesc, ks > 0 ? 1u : 0u);
          tc::mma_tf32(dc, tc::desc_sw128(al + off), tc::desc_sw128(bh + off), idesc, 1u);
        }
        tc::mma_commit(&mbar[st]);
      }
      if (kb + 1 < nkb) load(kb + 1);
      if (kb > 0 && !drain(g - 1)) s_abort = 1;
    }
    if (aborted) break;
    // the job's last k-block
    if (!drain(g - 1)) s_abort = 1;
    __syncthreads();
    if (s_abort) { aborted = true; break; }
    const int ga = ta * kTcTile + 32 * q + (tid & 31);
    if (ga < a.nx) {
      double* out = a.out + (size_t)s * a.nx * a.ny + (size_t)ga * a.ny;
#pragma unroll
      for (int j = 0; j < 64; ++j) {
        const int gb = tb * kTcTile + 64 * h + j;
        if (gb < a.ny) out[gb] = f32_to_f64_exact(acc[j]);
      }
    }
  }
  if (aborted) {
    if (tid == 0) atomicOr(err, kErrTimeout);
    if (tid == 0 && g > 0) tc::mbar_wait(&mbar[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1), kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------------------------------
// left multiply: C[m][p] (+)= sum_k T[m][k] Y[k][p], T given as tt[k][m] (FP32)
// ------------------------------------------------------------------------------------
template <int NCOL>
__global__ void __launch_bounds__(kTcThreads, 1) k_lmul_tc(const MmArgs a, int* err) {
  constexpr uint32_t kBBytes = (uint32_t)NCOL * 128;     // one B tile (NCOL rows)
  constexpr uint32_t kStage = 2 * kTileBytes + 2 * kBBytes;
  constexpr int kBTasks = NCOL * 8 / kTcThreads;         // (m, k-quad) tasks of B per thread
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* base = align1024(smem_dyn);  // stage st: [A hi | A lo | B hi | B lo]
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
    tc::mbar_init_fence();
    s_abort = 0;
  }
  // TMEM: hi.hi accumulator at column 0, corrections at column NCOL
  if (warp == 0) tc::tmem_alloc(&tmem_base, 2 * NCOL);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = tc::idesc_tf32(kTcTile, NCOL);
  const float* TT = reinterpret_cast<const float*>(a.x);
  const int nkb = (int)((a.K + kTcBK - 1) / kTcBK);
  const int pa = tid & 127, qa = tid >> 7;  // A tasks: point pa, k-quads qa + 2 j (j < 4)

  long long g = 0;
  bool aborted = false;
  double ya[4][4];
  float tb[kBTasks][4];
  for (int job = blockIdx.x; job < a.njobs && !aborted; job += gridDim.x) {
    const long long p0 = (long long)job * kTcTile;
    auto load = [&](int kb) {
      const long long k0 = (long long)kb * kTcBK;
      const long long gp = p0 + pa;
#pragma unroll
      for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const long long k = k0 + 4 * (qa + 2 * j) + e;
          ya[j][e] = (k < a.K && gp < a.N) ? __ldcs(a.y + k * a.ldy + gp) : 0.0;
        }
#pragma unroll
      for (int j = 0; j < kBTasks; ++j) {
        const int idx = tid + kTcThreads * j;
        const int m = idx % NCOL, kq = idx / NCOL;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const long long k = k0 + 4 * kq + e;
          tb[j][e] = (k < a.K && m < a.nx) ? __ldg(TT + k * a.ldx + m) : 0.f;
        }
      }
    };
    load(0);
    for (int kb = 0; kb < nkb; ++kb, ++g) {
      const int st = (int)(g & 1);
      unsigned char* sah = base + st * kStage;
      unsigned char* sal = sah + kTileBytes;
      unsigned char* sbh = sah + 2 * kTileBytes;
      unsigned char* sbl = sbh + kBBytes;
      if (g >= 2 && !tc::mbar_wait(&mbar[st], (uint32_t)(((g >> 1) - 1) & 1), kWaitLimit)) s_abort = 1;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int kq = qa + 2 * j;
        float4 hv, lv;
        tc::split_tf32(f64_to_f32_rn(ya[j][0]), hv.x, lv.x);
        tc::split_tf32(f64_to_f32_rn(ya[j][1]), hv.y, lv.y);
        tc::split_tf32(f64_to_f32_rn(ya[j][2]), hv.z, lv.z);
        tc::split_tf32(f64_to_f32_rn(ya[j][3]), hv.w, lv.w);
        const uint32_t o = tc::swz128(pa, 4 * kq);
        *reinterpret_cast<float4*>(sah + o) = hv;
        *reinterpret_cast<float4*>(sal + o) = lv;
      }
#pragma unroll
      for (int j = 0; j < kBTasks; ++j) {
        const int idx = tid + kTcThreads * j;
        const int m = idx % NCOL, kq = idx / NCOL;
        float4 hv, lv;
        tc::split_tf32(tb[j][0], hv.x, lv.x);
        tc::split_tf32(tb[j][1], hv.y, lv.y);
        tc::split_tf32(tb[j][2], hv.z, lv.z);
        tc::split_tf32(tb[j][3], hv.w, lv.w);
        const uint32_t o = tc::swz128(m, 4 * kq);
        *reinterpret_cast<float4*>(sbh + o) = hv;
        *reinterpret_cast<float4*>(sbl + o) = lv;
      }
      tc::fence_proxy_async();
      __syncthreads();
      if (s_abort) { aborted = true; break; }
      if (tid == 0) {
        tc::fence_after_sync();
        const uint32_t ah = tc::smem_u32(sah), al = tc::smem_u32(sal), bh = tc::smem_u32(sbh), bl = tc::smem_u32(sbl);
#pragma unroll
        for (int ks = 0; ks < kTcBK / 8; ++ks) {
          const uint32_t off = 32u * ks;
          const uint32_t first = (kb > 0 || ks > 0) ? 1u : 0u;
          tc::mma_tf32(tmem, tc::desc_sw128(ah + off), tc::desc_sw128(bh + off), idesc, first);
          tc::mma_tf32(tmem + NCOL, tc::desc_sw128(ah + off), tc::desc_sw128(bl + off), idesc, first);
          tc::mma_tf32(tmem + NCOL, tc::desc_sw128(al + off), tc::desc_sw128(bh + off), idesc, 1u);
        }
        tc::mma_commit(&mbar[st]);
      }
      if (kb + 1 < nkb) load(kb + 1);
    }
    if (aborted) break;
    const long long gl = g - 1;
    if (!tc::mbar_wait(&mbar[gl & 1], (uint32_t)((gl >> 1) & 1), kWaitLimit)) s_abort = 1;
    __syncthreads();
    if (s_abort) { aborted = true; break; }
    tc::fence_after_sync();
    const int q = warp & 3, h = warp >> 2;  // TMEM lanes 32q.. (points p), columns (NCOL/2) h.. (m)
    const long long gp = p0 + 32 * q + (tid & 31);
#pragma unroll 1
    for (int cc = 0; cc < NCOL / 64; ++cc) {
      float v[32], vc[32];
      const int m0 = (NCOL / 2) * h + 32 * cc;
      tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)m0, v);
      tc::tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(NCOL + m0), vc);
      if (gp < a.N) {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int m = m0 + j;
          if (m < a.nx) {
            double* o = a.out + (long long)m * a.ldo + gp;
            const double w = f32_to_f64_exact(v[j] + vc[j]);
            *o = a.accumulate ? *o + w : w;
          }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
  }
  if (aborted) {
    if (tid == 0) atomicOr(err, kErrTimeout);
    if (tid == 0 && g > 0) tc::mbar_wait(&mbar[(g - 1) & 1], (uint32_t)(((g - 1) >> 1) & 1), kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, 2 * NCOL);
  }
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

bool gram_tc_ok(const double* x, long long ldx, const double* y, long long ldy, long long K, const GramPlan& plan) {
  return aligned16(x) && aligned16(y) && ldx % 2 == 0 && ldy % 2 == 0 && K % 2 == 0 && plan.chunk % 2 == 0;
}

cudaError_t gram_tc(bool absval, const double* x, long long ldx, int nx, const double* y, long long ldy, int ny,
                    long long K, const GramPlan& plan, double* partials, int* err, int sm_count, cudaStream_t st) {
  MmArgs a{};
  a.x = x; a.y = y; a.out = partials;
  a.K = K; a.ldx = ldx; a.ldy = ldy; a.ldo = 0;
  a.nx = nx; a.ny = ny; a.N = 0;
  a.chunk = plan.chunk;
  a.tiles_x = plan.tiles_x; a.tiles_y = plan.tiles_y; a.njobs = plan.njobs;
  const size_t smem = 2 * 4 * (size_t)kTileBytes + 1024;
  const int grid = std::min(a.njobs, sm_count);
  if (absval) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_tc<true><<<grid, kTcThreads, smem, st>>>(a, err);
  } else {
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_gram_tc<false><<<grid, kTcThreads, smem, st>>>(a, err);
  }
  return cudaGetLastError();
}

bool lmul_tc_ok(const void* tt, int m, const double* y, double* out) {
  return m >= 1 && m <= 256 && aligned16(tt) && aligned16(y) && aligned16(out);
}

template <int NCOL>
static cudaError_t launch_lmul_tc(const MmArgs& a, int* err, int sm_count, cudaStream_t st) {
  const size_t smem = 2 * (2 * (size_t)kTileBytes + 2 * (size_t)NCOL * 128) + 1024;
  cudaError_t e = cudaFuncSetAttribute(k_lmul_tc<NCOL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_lmul_tc<NCOL><<<std::min(a.njobs, sm_count), kTcThreads, smem, st>>>(a, err);
  return cudaGetLastError();
}

cudaError_t lmul_tc(const float* tt, long long ldt, int m, int k, const double* y, long long ldy, long long n,
                    bool accumulate, double* out, long long ldo, int* err, int sm_count, cudaStream_t st) {
  MmArgs a{};
  a.x = tt; a.y = y; a.out = out;
  a.K = k; a.ldx = ldt; a.ldy = ldy; a.ldo = ldo;
  a.nx = m; a.ny = 0; a.N = n;
  a.tiles_x = 1;
  a.tiles_y = (int)((n + kTcTile - 1) / kTcTile);
  a.njobs = a.tiles_y;
  a.accumulate = accumulate ? 1 : 0;
  if (m <= 128) return launch_lmul_tc<128>(a, err, sm_count, st);
  return launch_lmul_tc<256>(a, err, sm_count, st);
}

}  // namespace ace
}  // namespace hfx
