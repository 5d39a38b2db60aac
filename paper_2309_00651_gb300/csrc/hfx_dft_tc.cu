// The forward plane pass (pair product, forward DFT along z and y of one x-plane) with its DFT
// stages on the fifth-generation tensor cores: the HFX_PREC_MIXED_TC precision of the exchange
// path (Sec. 2.1, Eqs. vij and HFX; the per-pair forward transform of the Poisson solve).
//
// Each axis is one complex DFT of length N, written as one real GEMM with split TF32 operands:
//   [X_re | X_im](row) = [Z_re | Z_im](row) . B,  B = [[C, -S], [S, C]] over (input, output),
// C = cos(2 pi t f / N), S = sin(2 pi t f / N) for input index t and output frequency f, with
// the output columns in the digit-reversed position order of the stage plan of N, so the result
// lands where the x/Coulomb and inverse-y passes (hfx_ct.cuh) expect it.  The data is the A
// operand (M = 128 rows: the plane's N lines, the rest zero), the DFT matrix B (N_mma = 2N
// columns, K = 2N) comes pre-split (hi + lo TF32) and pre-swizzled from a table, one k-block of
// 32 inputs at a time.  Every data value is rounded to FP32 and split hi + lo; products are
// hi.hi + hi.lo + lo.hi, the hi.hi products and the two corrections in separate TMEM
// accumulators that restart every k-block and are added, with round-to-nearest, to FP32 sums
// (the tensor core's own accumulation rounds toward zero).
//   z: rows y, inputs z -> P[y][f] (shared memory, FP32);
//   y: rows f (from P, transposed as it is stored), inputs y -> registers -> W[cl][x][fy][fz].
// Block: 256 threads; thread 0 issues the MMAs; every mbarrier wait has an iteration limit after
// which the block records the timeout bit in the error word, frees its TMEM and returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "hfx_internal.h"
#include "hfx_kernels.cuh"
#include "tc_sm100.cuh"

namespace hfx {
namespace dft {

namespace {

constexpr int kThreads = 256;
constexpr long long kWaitLimit = 1LL << 26;

template <int N>
struct TcGeo {
  static constexpr int NB = 2 * N;       // MMA N: (re, im) of the N outputs
  static constexpr int KB = 2 * N / 32;  // k-blocks of one axis (K = 2N)
  static constexpr uint32_t kA = 16384;  // one 128-row A tile
  static constexpr uint32_t kB = NB * 128;
  static constexpr int PS = NB + 1;      // row stride (floats) of P: odd, so columns are conflict-free
  static constexpr uint32_t kTmem = 2 * NB <= 128 ? 128 : (2 * NB <= 256 ? 256 : 512);
  static constexpr size_t kSmem = 1024 + 2 * (size_t)kA + 2 * (size_t)kB + (size_t)N * PS * sizeof(float);
  static_assert(N % 16 == 0 && NB <= 256, "edge must be a multiple of 16 and at most 128");
};

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return (unsigned char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

__device__ __forceinline__ void split4(float4 v, float4& h, float4& l) {
  tc::split_tf32(v.x, h.x, l.x);
  tc::split_tf32(v.y, h.y, l.y);
  tc::split_tf32(v.z, h.z, l.z);
  tc::split_tf32(v.w, h.w, l.w);
}

}  // namespace

template <int N>
__global__ void __launch_bounds__(kThreads, 1)
k_fwd_yz_tc(const float* __restrict__ orb, long long Ntot, const int4* __restrict__ couples, int c0, int c1,
            float2* __restrict__ W, const unsigned char* __restrict__ dftb, int* err) {
  using G = TcGeo<N>;
  constexpr int NB = G::NB, KB = G::KB, PS = G::PS, PLANE = N * N;
  constexpr uint32_t kA = G::kA, kB = G::kB;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char* base = align1024(smem_dyn);
  unsigned char* sah = base;
  unsigned char* sal = base + kA;
  unsigned char* sbh = base + 2 * kA;
  unsigned char* sbl = sbh + kB;
  float* P = reinterpret_cast<float*>(sbl + kB);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_abort;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    tc::mbar_init(&mbar, 1);
    tc::mbar_init_fence();
    s_abort = 0;
  }
  if (warp == 0) tc::tmem_alloc(&tmem_base, G::kTmem);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tmem_base;
  constexpr uint32_t idesc = tc::idesc_tf32(128, NB);
  const int q = warp & 3, h = warp >> 2;   // drains: TMEM lanes 32q.., columns h NB/2 ..
  const uint32_t lane_off = (uint32_t)(32 * q) << 16;
  const int rr = tid >> 1, hf = tid & 1;   // A tiles: row rr, inputs 16 hf .. 16 hf + 15 of the k-block
  uint32_t phase = 0;
  bool aborted = false;
  float acc[NB / 2];

  // the k-block's B tiles (hi, lo), contiguous in the table and in shared memory
  auto copy_b = [&](int kb) {
    const uint4* src = reinterpret_cast<const uint4*>(dftb + (size_t)kb * 2 * kB);
    uint4* dst = reinterpret_cast<uint4*>(sbh);
    for (int i = tid; i < (int)(2 * kB / 16); i += kThreads) dst[i] = __ldg(src + i);
  };
  // the k-block's MMAs (hi.hi into column 0, the corrections into column NB), then wait for them
  auto mma_wait = [&]() -> bool {
    tc::fence_proxy_async();
    __syncthreads();
    if (s_abort) return false;
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t ah = tc::smem_u32(sah), al = tc::smem_u32(sal), bh = tc::smem_u32(sbh), bl = tc::smem_u32(sbl);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t off = 32u * ks;
        tc::mma_tf32(tmem, tc::desc_sw128(ah + off), tc::desc_sw128(bh + off), idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32(tmem + NB, tc::desc_sw128(ah + off), tc::desc_sw128(bl + off), idesc, ks > 0 ? 1u : 0u);
        tc::mma_tf32(tmem + NB, tc::desc_sw128(al + off), tc::desc_sw128(bh + off), idesc, 1u);
      }
      tc::mma_commit(&mbar);
    }
    const bool ok = tc::mbar_wait(&mbar, phase, kWaitLimit);
    phase ^= 1u;
    if (!ok) s_abort = 1;
    tc::fence_after_sync();
    return ok;
  };

  const int items = (c1 - c0) * N;
  for (int it = blockIdx.x; it < items && !aborted; it += gridDim.x) {
    const int cl = it / N;
    const int x = it - cl * N;
    const int4 cp = couples[c0 + cl];
    if (couple_empty(cp)) continue;
    const long long off = (long long)x * PLANE;
    const bool hasa = cp.x >= 0, hasb = cp.z >= 0;
    const float* pa1 = orb + (long long)(hasa ? cp.x : 0) * Ntot + off;
    const float* pa2 = orb + (long long)(hasa ? cp.y : 0) * Ntot + off;
    const float* pb1 = orb + (long long)(hasb ? cp.z : 0) * Ntot + off;
    const float* pb2 = orb + (long long)(hasb ? cp.w : 0) * Ntot + off;

    // ---- z: rows y, inputs [Re z | Im z] -> P[y][column]
    for (int kb = 0; kb < KB && !aborted; ++kb) {
      // this thread's 16 inputs 32 kb + 16 hf ..: all real or all imaginary parts (N is a
      // multiple of 16), of points z0 .. z0 + 15
      const int k0 = 32 * kb + 16 * hf;
      const bool re = k0 < N;
      const int z0 = re ? k0 : k0 - N;
      const bool live = rr < N && (re ? hasa : hasb);
      const float* p1 = (re ? pa1 : pb1) + rr * N + z0;
      const float* p2 = (re ? pa2 : pb2) + rr * N + z0;
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        float4 hv = make_float4(0.f, 0.f, 0.f, 0.f), lv = hv;
        if (live) {
          const float4 u = __ldg(reinterpret_cast<const float4*>(p1 + 4 * q4));
          const float4 v = __ldg(reinterpret_cast<const float4*>(p2 + 4 * q4));
          split4(make_float4(u.x * v.x, u.y * v.y, u.z * v.z, u.w * v.w), hv, lv);
        }
        const uint32_t o = tc::swz128(rr, 16 * hf + 4 * q4);
        *reinterpret_cast<float4*>(sah + o) = hv;
        *reinterpret_cast<float4*>(sal + o) = lv;
      }
      copy_b(kb);
      if (!mma_wait()) { aborted = true; break; }
#pragma unroll
      for (int c16 = 0; c16 < NB / 32; ++c16) {
        const int j0 = h * (NB / 2) + 16 * c16;
        float vm[16], vc[16];
        tc::tmem_ld16(tmem + lane_off + (uint32_t)j0, vm);
        tc::tmem_ld16(tmem + lane_off + (uint32_t)(NB + j0), vc);
        const int y = 32 * q + lane;
        if (y < N) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float* pp = P + y * PS + j0 + j;
            *pp = (kb > 0 ? *pp : 0.f) + (vm[j] + vc[j]);
          }
        }
      }
      tc::fence_before_sync();
      __syncthreads();  // P updated; TMEM and the operand tiles free for the next k-block
    }
    if (aborted) break;

    // ---- y: rows = z position f (P's column), inputs [Re y | Im y] -> acc (this thread: lane f,
    // columns h NB/2 ..)
#pragma unroll
    for (int j = 0; j < NB / 2; ++j) acc[j] = 0.f;
    for (int kb = 0; kb < KB && !aborted; ++kb) {
      const int k0 = 32 * kb + 16 * hf;
      const bool re = k0 < N;
      const int y0 = re ? k0 : k0 - N;
      const int col = rr + (re ? 0 : N);
#pragma unroll
      for (int q4 = 0; q4 < 4; ++q4) {
        float4 hv = make_float4(0.f, 0.f, 0.f, 0.f), lv = hv;
        if (rr < N) {
          const int y = y0 + 4 * q4;
          split4(make_float4(P[(y + 0) * PS + col], P[(y + 1) * PS + col], P[(y + 2) * PS + col],
                             P[(y + 3) * PS + col]), hv, lv);
        }
        const uint32_t o = tc::swz128(rr, 16 * hf + 4 * q4);
        *reinterpret_cast<float4*>(sah + o) = hv;
        *reinterpret_cast<float4*>(sal + o) = lv;
      }
      copy_b(kb);
      if (!mma_wait()) { aborted = true; break; }
#pragma unroll
      for (int c16 = 0; c16 < NB / 32; ++c16) {
        const int j0 = h * (NB / 2) + 16 * c16;
        float vm[16], vc[16];
        tc::tmem_ld16(tmem + lane_off + (uint32_t)j0, vm);
        tc::tmem_ld16(tmem + lane_off + (uint32_t)(NB + j0), vc);
#pragma unroll
        for (int j = 0; j < 16; ++j) acc[16 * c16 + j] += vm[j] + vc[j];
      }
      tc::fence_before_sync();
      __syncthreads();
    }
    if (aborted) break;
    // ---- W[cl][x][fy][fz]: this thread holds fz = lane row, columns jj: Re (jj < N) or Im of fy
    const int fz = 32 * q + lane;
    if (fz < N) {
      float* wb = reinterpret_cast<float*>(W + ((long long)cl * N + x) * PLANE);
#pragma unroll
      for (int j = 0; j < NB / 2; ++j) {
        const int jj = h * (NB / 2) + j;
        const int fy = jj < N ? jj : jj - N;
        wb[2 * ((long long)fy * N + fz) + (jj < N ? 0 : 1)] = acc[j];
      }
    }
  }
  if (aborted && tid == 0) {
    atomicOr(err, kErrTimeout);
    tc::mbar_wait(&mbar, phase ^ 1u, kWaitLimit);  // the last commit, if it is still in flight
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, G::kTmem);
  }
}

// ------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------
bool tc_edge(int n) { return n == 32 || n == 48 || n == 64 || n == 96; }

size_t tc_table_bytes(int n) { return (size_t)(2 * n / 32) * 2 * (size_t)(2 * n) * 128; }

template <int N>
static cudaError_t prep(int* blocks) {
  using G = TcGeo<N>;
  cudaError_t e = cudaFuncSetAttribute(k_fwd_yz_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::kSmem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, k_fwd_yz_tc<N>, kThreads, G::kSmem);
}

cudaError_t tc_prepare(int n, int* blocks) {
  switch (n) {
    case 32: return prep<32>(blocks);
    case 48: return prep<48>(blocks);
    case 64: return prep<64>(blocks);
    case 96: return prep<96>(blocks);
    default: return cudaErrorInvalidValue;
  }
}

template <int N>
static void launch(int grid, cudaStream_t st, const float* orb, long long Ntot, const int4* couples, int c0, int c1,
                   float2* W, const unsigned char* dftb, int* err) {
  k_fwd_yz_tc<N><<<grid, kThreads, TcGeo<N>::kSmem, st>>>(orb, Ntot, couples, c0, c1, W, dftb, err);
}

void fwd_yz_tc(int n, int grid, cudaStream_t st, const float* orb, long long Ntot, const int4* couples, int c0,
               int c1, float2* W, const unsigned char* dftb, int* err) {
  switch (n) {
    case 32: launch<32>(grid, st, orb, Ntot, couples, c0, c1, W, dftb, err); break;
    case 48: launch<48>(grid, st, orb, Ntot, couples, c0, c1, W, dftb, err); break;
    case 64: launch<64>(grid, st, orb, Ntot, couples, c0, c1, W, dftb, err); break;
    case 96: launch<96>(grid, st, orb, Ntot, couples, c0, c1, W, dftb, err); break;
    default: break;
  }
}

}  // namespace dft
}  // namespace hfx
