// Compile-time-geometry versions of the exchange passes for cubic grids of edge N.
//
// Same algorithm and the same in-place DIF/DIT stage order as the runtime kernels in
// hfx_kernels.cuh (so the digit-reversed storage order, and therefore the Coulomb table, are
// identical), but every length, stride, radix and loop trip count is a constant: butterfly
// element offsets become immediate offsets, divisions by constants become multiply-shifts, and
// each stage reads its twiddles from its own [m][r] table (w_L^{j1 k}), one row per butterfly.
#pragma once
#include "hfx_kernels.cuh"
#include "tma_sm100.cuh"

namespace hfx {
namespace ct {

template <int N> struct Plan { static constexpr StagePlan p = stage_plan(N); };

// one in-place stage over LINES lines (element e of line l at buf[l*LS + e*ES])
template <int R, int M, bool INV, int LINES, int LS, int ES, int N, int NT, typename C>
__device__ __forceinline__ void stage(C* __restrict__ buf, const C* __restrict__ twt) {
  constexpr int NQ = N / R;
  constexpr int TOTAL = LINES * NQ;
  constexpr int STEP = M * ES;
  constexpr int ITERS = (TOTAL + NT - 1) / NT;
#pragma unroll 1
  for (int it = 0; it < ITERS; ++it) {
    const int id = threadIdx.x + it * NT;
    if ((TOTAL % NT) != 0 && id >= TOTAL) break;
    const int q = id / LINES;
    const int line = id - q * LINES;
    const int j1 = q % M;
    C* p = buf + line * LS + ((q - j1) * R + j1) * ES;
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = p[k * STEP];
    if constexpr (!INV) {
      Dft<R, -1, C>::run(v);
      if constexpr (M > 1) {
        const C* t = twt + j1 * R;
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = cmul(v[k], t[k]);
      }
    } else {
      if constexpr (M > 1) {
        const C* t = twt + j1 * R;
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], t[k]);
      }
      Dft<R, 1, C>::run(v);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) p[k * STEP] = v[k];
  }
}

// forward stages S0 .. S1-1, or inverse stages S1-1 .. S0; a barrier after each
template <int N, bool INV, int S0, int S1, int LINES, int LS, int ES, int NT, typename C>
__device__ __forceinline__ void stages(C* buf, const C* tw) {
  constexpr StagePlan P = Plan<N>::p;
  if constexpr (S0 < S1) {
    if constexpr (!INV) {
      stage<P.r[S0], P.m[S0], false, LINES, LS, ES, N, NT>(buf, tw + P.twoff[S0]);
      __syncthreads();
      stages<N, false, S0 + 1, S1, LINES, LS, ES, NT>(buf, tw);
    } else {
      stage<P.r[S1 - 1], P.m[S1 - 1], true, LINES, LS, ES, N, NT>(buf, tw + P.twoff[S1 - 1]);
      __syncthreads();
      stages<N, true, S0, S1 - 1, LINES, LS, ES, NT>(buf, tw);
    }
  }
}

// forward stage 0 of column lines reading its input from global memory: line l's element e at
// src[l + e*GES]; results go to buf[l*SLS + e*SES].  A barrier follows.  The loads go through L2
// only (read once; in a persistent launch another block of the same launch may have written them).
template <int R, int M, int LINES, int GES, int SLS, int SES, int N, int NT, typename C>
__device__ __forceinline__ void stage_fwd_g2s(const C* __restrict__ src, C* __restrict__ buf,
                                              const C* __restrict__ twt) {
  constexpr int TOTAL = LINES * (N / R);
  constexpr int ITERS = (TOTAL + NT - 1) / NT;
#pragma unroll 1
  for (int it = 0; it < ITERS; ++it) {
    const int id = threadIdx.x + it * NT;
    if ((TOTAL % NT) != 0 && id >= TOTAL) break;
    const int q = id / LINES;
    const int line = id - q * LINES;
    const int j1 = q % M;
    const int e0 = (q - j1) * R + j1;
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = __ldcg(src + line + (e0 + k * M) * GES);
    Dft<R, -1, C>::run(v);
    if constexpr (M > 1) {
      const C* t = twt + j1 * R;
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmul(v[k], t[k]);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) buf[line * SLS + (e0 + k * M) * SES] = v[k];
  }
  __syncthreads();
}

// last forward stage (m = 1, no twiddles) of column lines writing its output to global memory
template <int R, int LINES, int SLS, int SES, int GES, int N, int NT, typename C>
__device__ __forceinline__ void stage_fwd_last_s2g(const C* __restrict__ buf, C* __restrict__ dst) {
  constexpr int TOTAL = LINES * (N / R);
  constexpr int ITERS = (TOTAL + NT - 1) / NT;
#pragma unroll 1
  for (int it = 0; it < ITERS; ++it) {
    const int id = threadIdx.x + it * NT;
    if ((TOTAL % NT) != 0 && id >= TOTAL) break;
    const int q = id / LINES;
    const int line = id - q * LINES;
    const int e0 = q * R;
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[line * SLS + (e0 + k) * SES];
    Dft<R, -1, C>::run(v);
#pragma unroll
    for (int k = 0; k < R; ++k) dst[line + (e0 + k) * GES] = v[k];
  }
}

// inverse stage 0 (the last one applied) of column lines writing its output to global memory
template <int R, int M, int LINES, int SLS, int SES, int GES, int N, int NT, typename C>
__device__ __forceinline__ void stage_inv_s2g(const C* __restrict__ buf, C* __restrict__ dst,
                                              const C* __restrict__ twt) {
  constexpr int TOTAL = LINES * (N / R);
  constexpr int ITERS = (TOTAL + NT - 1) / NT;
#pragma unroll 1
  for (int it = 0; it < ITERS; ++it) {
    const int id = threadIdx.x + it * NT;
    if ((TOTAL % NT) != 0 && id >= TOTAL) break;
    const int q = id / LINES;
    const int line = id - q * LINES;
    const int j1 = q % M;
    const int e0 = (q - j1) * R + j1;
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[line * SLS + (e0 + k * M) * SES];
    if constexpr (M > 1) {
      const C* t = twt + j1 * R;
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], t[k]);
    }
    Dft<R, 1, C>::run(v);
#pragma unroll
    for (int k = 0; k < R; ++k) dst[line + (e0 + k * M) * GES] = v[k];
  }
}

template <typename T> struct Two;  // two consecutive reals
template <> struct Two<float> { using type = float2; };
template <> struct Two<double> { using type = double2; };

// store two consecutive complex values (16 or 32 bytes) to global memory
__device__ __forceinline__ void st2(float2* dst, float2 a, float2 b) {
  *reinterpret_cast<float4*>(dst) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st2(double2* dst, double2 a, double2 b) { dst[0] = a; dst[1] = b; }
__device__ __forceinline__ void ld2(const float2* src, float2& a, float2& b) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(src));
  a = make_float2(v.x, v.y);
  b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void ld2(const double2* src, double2& a, double2& b) {
  a = __ldg(src);
  b = __ldg(src + 1);
}

// FP32 -> FP64, exact for normal numbers and +-0, with integer operations only (sign, exponent
// rebias 127 -> 1023, fraction widened); FP32 subnormals flush to zero.  The flushes below use it
// so that their only FP64 instruction is the final add (the FP64 pipe of this part is narrow).
__device__ __forceinline__ double widen_exact(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned mag = u & 0x7fffffffu, sign = u & 0x80000000u;
  const bool tiny = mag < 0x00800000u;
  const unsigned hi = tiny ? sign : (((mag >> 3) + 0x38000000u) | sign);
  const unsigned lo = tiny ? 0u : (mag << 29);
  return __hiloint2double((int)hi, (int)lo);
}

constexpr int kUnroll = 4;

// threads per block of the compile-time plane kernels: 256, but 512 where the padded plane is so
// large that one block fills an SM's shared memory (N = 128), so that 16 warps rather than 8 hide
// the latency of each SM's single plane
template <int N> struct PlaneThreads {
  static constexpr int value = N * (N + 1) * 8 > 114 * 1024 ? 2 * kThreadsPlane : kThreadsPlane;
};

// resident blocks per SM the plane kernels of edge N are built for: at most `cap`, and no more than
// the padded plane (N (N+1) complex FP32 plus the twiddles, ~1 KB) lets fit in an SM's 228 KB of
// shared memory (asking for more would only cap the registers a thread may use)
template <int N, int cap> struct PlaneBlocks {
  static constexpr int bytes = N * (N + 1) * 8 + 1024 + 1024;
  static constexpr int fit = (228 * 1024) / bytes;
  static constexpr int value = fit < 1 ? 1 : (fit < cap ? fit : cap);
};

// an asynchronous prefetch of `bytes` (a multiple of 16) at the 16-byte-aligned global address p
// into L2; nothing is returned to the issuing thread
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ----------------------------------------------------------------------------------
// pass 1: pair product + forward FFT along z and y of one x-plane
// ----------------------------------------------------------------------------------
// one item (couple cl = it / N, x-plane x = it mod N); buf holds the padded plane, tw the per-stage
// twiddles in shared memory (loaded before the caller's first barrier)
template <typename T, int N>
__device__ __forceinline__ void fwd_yz_ct_item(const T* __restrict__ orb, long long Ntot,
                                               const int4* __restrict__ couples, int c0, cx<T>* __restrict__ W,
                                               cx<T>* buf, const cx<T>* tw, int it) {
  using C = cx<T>;
  using T2 = typename Two<T>::type;
  constexpr int S = N + 1, PLANE = N * N, NT = PlaneThreads<N>::value, NV = PLANE / 2;
  constexpr StagePlan P = Plan<N>::p;
  const int cl = it / N;
  const int x = it - cl * N;
  const int4 cp = couples[c0 + cl];
  if (couple_empty(cp)) return;
  const long long off = (long long)x * PLANE;
  const bool hasa = cp.x >= 0, hasb = cp.z >= 0;
  const T2* pa1 = reinterpret_cast<const T2*>(orb + (long long)(hasa ? cp.x : 0) * Ntot + off);
  const T2* pa2 = reinterpret_cast<const T2*>(orb + (long long)(hasa ? cp.y : 0) * Ntot + off);
  const T2* pb1 = reinterpret_cast<const T2*>(orb + (long long)(hasb ? cp.z : 0) * Ntot + off);
  const T2* pb2 = reinterpret_cast<const T2*>(orb + (long long)(hasb ? cp.w : 0) * Ntot + off);
  __syncthreads();  // the previous item's store is done with buf (and the table is loaded)
  for (int i0 = threadIdx.x; i0 < NV; i0 += kUnroll * NT) {
    T2 a1[kUnroll], a2[kUnroll], b1[kUnroll], b2[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * NT;
      const bool in = (NV % (kUnroll * NT) == 0) || i < NV;
      const T2 zero = {};
      a1[u] = (in && hasa) ? __ldg(pa1 + i) : zero;
      a2[u] = (in && hasa) ? __ldg(pa2 + i) : zero;
      b1[u] = (in && hasb) ? __ldg(pb1 + i) : zero;
      b2[u] = (in && hasb) ? __ldg(pb2 + i) : zero;
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int i = i0 + u * NT;
      if ((NV % (kUnroll * NT) == 0) || i < NV) {
        const int p = 2 * i;
        const int y = p / N, z = p - y * N;  // N even: both points in row y
        const C c0 = mk<C>(a1[u].x * a2[u].x, b1[u].x * b2[u].x);
        const C c1 = mk<C>(a1[u].y * a2[u].y, b1[u].y * b2[u].y);
        // which of its two points a thread stores first: with ((i / 8) ^ y) odd the second, so that
        // each store instruction of a warp covers every shared-memory bank twice (consecutive
        // threads' points are 16 bytes apart; in one order they would use half of the banks)
        const int sw = ((i >> 3) ^ y) & 1;
        buf[y * S + z + sw] = sw ? c1 : c0;
        buf[y * S + z + 1 - sw] = sw ? c0 : c1;
      }
    }
  }
  __syncthreads();
  stages<N, false, 0, P.ns, N, S, 1, NT>(buf, tw);      // z: N rows
  stages<N, false, 0, P.ns - 1, N, 1, S, NT>(buf, tw);  // y: N columns, all but the last stage
  // last y stage straight to W[cl][x][y][z] (consecutive threads on consecutive z)
  stage_fwd_last_s2g<P.r[P.ns - 1], N, 1, S, N, N, NT>(buf, W + ((long long)cl * N + x) * PLANE);
}

template <typename T, int N>
__global__ void __launch_bounds__(PlaneThreads<N>::value, (PlaneBlocks<N, 3>::value))
k_fwd_yz_ct(const T* __restrict__ orb, long long Ntot, const int4* __restrict__ couples, int c0, int c1,
            cx<T>* __restrict__ W, const cx<T>* __restrict__ twg, int prefetch) {
  using C = cx<T>;
  constexpr int S = N + 1;
  constexpr StagePlan P = Plan<N>::p;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw = buf + N * S;
  for (int i = threadIdx.x; i < P.twtotal; i += PlaneThreads<N>::value) tw[i] = twg[i];
  const int ncl = c1 - c0, items = ncl * N;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    // x-major order: the blocks in flight work on the same x-plane of many couples, whose orbital
    // planes (the batch's orbitals at that x) are then read from DRAM once and from L2 after
    const int x = it / ncl, cl = it - x * ncl;
    // the four orbital planes of this block's next item head for L2 while this one runs
    const int nx = it + gridDim.x;
    if (prefetch && nx < items && threadIdx.x < 4) {
      const int x2 = nx / ncl;
      const int4 cp = couples[c0 + nx - x2 * ncl];
      const int o = threadIdx.x == 0 ? cp.x : threadIdx.x == 1 ? cp.y : threadIdx.x == 2 ? cp.z : cp.w;
      if (o >= 0) prefetch_l2(orb + (long long)o * Ntot + (long long)x2 * N * N, N * N * sizeof(T));
    }
    fwd_yz_ct_item<T, N>(orb, Ntot, couples, c0, W, buf, tw, cl * N + x);
  }
}

// ----------------------------------------------------------------------------------
// pass 2: forward FFT along x, Coulomb multiply + energy, inverse along x and z
// ----------------------------------------------------------------------------------
// one item (couple cl = it / N, y-plane y = it mod N); red: [2][32] floats of shared memory used
// alternately (par) by consecutive items of a block
template <typename T, int N>
__device__ __forceinline__ void x_coulomb_ct_item(const int4* __restrict__ couples, int c0, cx<T>* __restrict__ W,
                                                  const T* __restrict__ vtab, double* __restrict__ epart,
                                                  int energy_only, cx<T>* buf, const cx<T>* tw, float (*red)[32],
                                                  int par, int it) {
  using C = cx<T>;
  constexpr int S = N + 1, PLANE = N * N, NT = PlaneThreads<N>::value;
  constexpr StagePlan P = Plan<N>::p;
  constexpr int RL = P.r[P.ns - 1];  // last forward stage (m = 1)
  static_assert(P.ns >= 2, "compile-time x pass needs at least two stages");
  const int cl = it / N;
  const int y = it - cl * N;
  if (couple_empty(couples[c0 + cl])) return;
  C* wc = W + (long long)cl * N * PLANE + (long long)y * N;
  __syncthreads();
  // x stage 0 straight from W[cl][x][y][z] (line z, element x at stride PLANE)
  stage_fwd_g2s<P.r[0], P.m[0], N, PLANE, 1, S, N, NT>(wc, buf, tw + P.twoff[0]);
  stages<N, false, 1, P.ns - 1, N, 1, S, NT>(buf, tw);  // remaining x stages but the last
  // last forward x stage (no twiddles) + Coulomb + energy + first inverse x stage
  // the plane's energy partial in FP32 (a few terms per thread, then a tree over the block),
  // widened once; the partials of all planes and couples are summed in FP64
  T e_acc = T(0);
  {
    constexpr int TOTAL = N * (N / RL);
    const T* vy = vtab + (long long)y * N;
#pragma unroll 1
    for (int id = threadIdx.x; id < TOTAL; id += NT) {
      const int q = id / N, z = id - q * N;
      C* p = buf + q * RL * S + z;
      T vg[RL];
#pragma unroll
      for (int k = 0; k < RL; ++k) vg[k] = __ldg(vy + (long long)(q * RL + k) * PLANE + z);
      C v[RL];
#pragma unroll
      for (int k = 0; k < RL; ++k) v[k] = p[k * S];
      Dft<RL, -1, C>::run(v);
      T e = T(0);
#pragma unroll
      for (int k = 0; k < RL; ++k) {
        e += vg[k] * (v[k].x * v[k].x + v[k].y * v[k].y);
        v[k].x *= vg[k];
        v[k].y *= vg[k];
      }
      e_acc += e;
      if (!energy_only) {
        Dft<RL, 1, C>::run(v);
#pragma unroll
        for (int k = 0; k < RL; ++k) p[k * S] = v[k];
      }
    }
  }
  static_assert(sizeof(T) == 4, "compile-time passes are FP32");
  // block sum without barriers of its own: a shuffle tree per warp, the warp partials to
  // red[par] now, and warp 0 adds them (a second tree) after the barrier that the inverse
  // stages need anyway
  {
    float v = e_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[par][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    constexpr int NW = (NT + 31) / 32;
    float r = threadIdx.x < NW ? red[par][threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    if (threadIdx.x == 0) epart[(long long)(c0 + cl) * N + y] = widen_exact(r);
  }
  if (energy_only) return;
  // inverse transforms along different axes commute: z first (rows), then the remaining x
  // stages, the last of which writes W directly
  stages<N, true, 0, P.ns, N, S, 1, NT>(buf, tw);      // z inverse: N rows
  stages<N, true, 1, P.ns - 1, N, 1, S, NT>(buf, tw);  // x inverse stages ns-2 .. 1
  stage_inv_s2g<P.r[0], P.m[0], N, 1, S, PLANE, N, NT>(buf, wc, tw + P.twoff[0]);
}

template <typename T, int N>
__global__ void __launch_bounds__(PlaneThreads<N>::value, (PlaneBlocks<N, 4>::value))
k_x_coulomb_ct(const int4* __restrict__ couples, int c0, int c1, cx<T>* __restrict__ W, const T* __restrict__ vtab,
               const cx<T>* __restrict__ twg, double* __restrict__ epart, int energy_only, int prefetch) {
  using C = cx<T>;
  constexpr int S = N + 1;
  constexpr StagePlan P = Plan<N>::p;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw = buf + N * S;
  __shared__ float red[2][32];  // warp partials of the plane energy, double-buffered by item parity
  for (int i = threadIdx.x; i < P.twtotal; i += PlaneThreads<N>::value) tw[i] = twg[i];
  int par = 0;
  const int items = (c1 - c0) * N;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    // the N rows (576 bytes at N = 72) of this block's next y-plane head for L2 while this one runs
    const int nx = it + gridDim.x;
    if (prefetch && nx < items && threadIdx.x < N)
      prefetch_l2(W + ((long long)nx / N * N + threadIdx.x) * N * N + (long long)(nx % N) * N, N * sizeof(C));
    if (couple_empty(couples[c0 + it / N])) continue;
    x_coulomb_ct_item<T, N>(couples, c0, W, vtab, epart, energy_only, buf, tw, red, par, it);
    par ^= 1;
  }
}

// ----------------------------------------------------------------------------------
// pass 3a with compile-time geometry: see k_y_acc_dense
// ----------------------------------------------------------------------------------
template <typename T, int N> struct DenseGeo {
  static constexpr int ZC = ZChunk<T>::value;
  static constexpr int PTS = N * ZC;
  // points per thread: one up to 640 points (more warps hide the pass's load latency), else as
  // few as keep the block within 512 threads
  static constexpr int NP = PTS <= 640 ? 1 : (PTS + 511) / 512;
  static constexpr int NT = ((PTS + NP - 1) / NP + 31) / 32 * 32;   // threads
  // orbital rows per iteration of the off-diagonal pass: two up to N = 72; one beyond, which
  // halves the ring of couple tiles so that two blocks fit an SM at N = 96
  static constexpr int RPI = dense_rows_ct(N);
  static constexpr int MINB = N <= 96 ? 2 : 1;  // resident blocks per SM the passes are built for
};

template <typename T, int N, int B>
__global__ void __launch_bounds__(DenseGeo<T, N>::NT, DenseGeo<T, N>::MINB)
k_y_acc_dense_ct(const T* __restrict__ orb, long long Ntot, const int4* __restrict__ couples,
                 const int* __restrict__ slot_list, const int* __restrict__ slot_couple_base,
                 const int2* __restrict__ slot_blocks, int c0, const cx<T>* __restrict__ W,
                 const cx<T>* __restrict__ twg, T* __restrict__ V, double vscale) {
  using C = cx<T>;
  using G = DenseGeo<T, N>;
  constexpr int ZC = G::ZC, PTS = G::PTS, NP = G::NP, NT = G::NT;
  constexpr int HB = B / 2;
  constexpr int RPI = G::RPI;  // orbital rows per iteration
  constexpr int RING = kDenseRingCt;
  constexpr int LN = RPI * HB * ZC;  // lines of the interleaved tile [y][u][t][zz]
  constexpr int ITERS = B / RPI;
  static_assert(B % RPI == 0, "rows per iteration must divide the block");
  constexpr int PER = 16 / int(sizeof(C));
  constexpr int PLANE = N * N;
  constexpr StagePlan P = Plan<N>::p;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int z0 = blockIdx.x * ZC;
  const int zcn = min(ZC, N - z0);
  const int x = blockIdx.y;
  const int slot = slot_list[blockIdx.z];
  C* tiles = reinterpret_cast<C*>(smem_raw);  // RING x [N][LN]
  C* tw = tiles + RING * N * LN;
  T* phiI = reinterpret_cast<T*>(tw + P.twtotal);  // [B][PTS]
  T* accI = phiI + B * PTS;                         // [B][PTS]

  const int2 blk = slot_blocks[slot];
  const int I0 = blk.x * B, J0 = blk.y * B;
  const int cs = slot_couple_base[slot];
  const long long rowoff = (long long)x * PLANE + z0;

  // which couples of the block pair hold pairs (bit t of the mask: couple cs + t)
  static_assert(B * HB <= 32, "one mask word per block pair");
  __shared__ unsigned live_mask;
  if (threadIdx.x < 32) {
    const unsigned m = __ballot_sync(0xffffffffu, threadIdx.x < B * HB && !couple_empty(couples[cs + threadIdx.x]));
    if (threadIdx.x == 0) live_mask = m;
  }
  __syncthreads();
  const unsigned live = live_mask;

  // phi_I (kept) and phi_J (staged in the accI area until it moves to registers) tiles, rows of
  // ZC reals; they join the first copy group
  {
    // reals per copy: 16 bytes where every orbital row starts on a 16-byte boundary (N a multiple
    // of 16 / sizeof(T)), else 8 bytes
    constexpr int CPB = (N * int(sizeof(T))) % 16 == 0 ? 16 : 8;
    constexpr int RPER = CPB / int(sizeof(T));
    constexpr int VPR = ZC / RPER;
    for (int i = threadIdx.x; i < 2 * B * N * VPR; i += NT) {
      const int v = i % VPR;
      const int rest = i / VPR;
      const int y = rest % N;
      const int oo = rest / N;  // 0..2B-1: I block then J block
      const int o = oo < B ? I0 + oo : J0 + (oo - B);
      T* dst = (oo < B ? phiI + oo * PTS : accI + (oo - B) * PTS) + y * ZC + v * RPER;
      const int valid = zcn - v * RPER;
      const int bytes = valid >= RPER ? CPB : (valid > 0 ? valid * int(sizeof(T)) : 0);
      const T* src = orb + (long long)o * Ntot + rowoff + (long long)y * N + v * RPER;
      if constexpr (CPB == 16) cp_async16(dst, bytes ? (const void*)src : (const void*)orb, bytes);
      else cp_async8(dst, bytes ? (const void*)src : (const void*)orb, bytes);
    }
  }

  // the couple tiles of orbital rows k*RPI .. k*RPI+RPI-1 -> ring buffer k % RING (empty couples and
  // columns past N read as zero); an iteration past the block commits an empty group
  auto issue_it = [&](int k) {
    if (k >= ITERS) { cp_async_commit(); return; }
    C* dstb = tiles + (k % RING) * N * LN;
    constexpr int VPR = ZC / PER;
    for (int i = threadIdx.x; i < RPI * HB * N * VPR; i += NT) {
      const int v = i % VPR;
      const int rest = i / VPR;
      const int ut = rest % (RPI * HB), y = rest / (RPI * HB);  // ut = u * HB + t
      const int cr = k * RPI * HB + ut;                          // couple within the block pair
      const bool ok_c = ((live >> cr) & 1u) && v * PER < zcn;
      const C* src = W + ((long long)(cs + cr - c0) * N + x) * PLANE + (long long)y * N + z0 + v * PER;
      cp_async16(dstb + y * LN + ut * ZC + v * PER, ok_c ? (const void*)src : (const void*)W, ok_c ? 16 : 0);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < RING - 1; ++k) issue_it(k);

  for (int i = threadIdx.x; i < P.twtotal; i += NT) tw[i] = twg[i];

  long long goff[NP];
  bool ok[NP];
  T phiJ[NP][B], accJ[NP][B];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int p = threadIdx.x + k * NT;
    const int y = p / ZC, zz = p - y * ZC;
    ok[k] = p < PTS && zz < zcn;
    goff[k] = rowoff + (long long)y * N + zz;
#pragma unroll
    for (int j = 0; j < B; ++j) accJ[k][j] = T(0);
  }

  for (int kk = 0; kk < ITERS; ++kk) {
    issue_it(kk + RING - 1);
    cp_async_wait<RING - 1>();
    __syncthreads();
    if (kk == 0) {
      // phi_J to registers (the staging area becomes accI after the barriers of the first row)
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int p = threadIdx.x + k * NT;
#pragma unroll
        for (int j = 0; j < B; ++j) phiJ[k][j] = ok[k] ? accI[j * PTS + p] : T(0);
      }
    }
    C* buf = tiles + (kk % RING) * N * LN;
    stages<N, true, 0, P.ns, LN, 1, LN, NT>(buf, tw);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = threadIdx.x + k * NT;
      if (!ok[k]) continue;
      const int y = p / ZC, zz = p - y * ZC;
#pragma unroll
      for (int u = 0; u < RPI; ++u) {
        const int r = kk * RPI + u;
        const C* vp = buf + y * LN + u * HB * ZC + zz;
        const T phii = phiI[r * PTS + p];
        T acci = T(0);
#pragma unroll
        for (int t = 0; t < HB; ++t) {
          const C v = vp[t * ZC];
          acci += v.x * phiJ[k][2 * t] + v.y * phiJ[k][2 * t + 1];
          accJ[k][2 * t] += v.x * phii;
          accJ[k][2 * t + 1] += v.y * phii;
        }
        accI[r * PTS + p] = acci;
      }
    }
    __syncthreads();
  }
  // flush into the call's FP32 accumulator of V_x phi (widened to FP64 once at the end of the
  // call): read-modify-write of V_J (registers) and V_I (shared memory), every load issued before
  // any store (a store could alias a later load, which would serialise the round trips)
  const T vs = (T)vscale;
  T old[NP][B];
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int j = 0; j < B; ++j) old[k][j] = ok[k] ? __ldcg(V + (long long)(J0 + j) * Ntot + goff[k]) : T(0);
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    if (!ok[k]) continue;
#pragma unroll
    for (int j = 0; j < B; ++j) V[(long long)(J0 + j) * Ntot + goff[k]] = old[k][j] + vs * accJ[k][j];
  }
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int j = 0; j < B; ++j) old[k][j] = ok[k] ? __ldcg(V + (long long)(I0 + j) * Ntot + goff[k]) : T(0);
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    if (!ok[k]) continue;
    const int p = threadIdx.x + k * NT;
#pragma unroll
    for (int j = 0; j < B; ++j) V[(long long)(I0 + j) * Ntot + goff[k]] = old[k][j] + vs * accI[j * PTS + p];
  }
}

// pass 3a with compile-time geometry, tiles moved by TMA: the work of k_y_acc_dense_ct, but one
// thread issues each iteration's couple tile as one tensor copy (the 4-D box of 2 ZC reals x
// RPI * HB couples x N rows of y at plane x, landing as [y][couple][zz]) and the two blocks'
// orbital tiles as two more (box ZC x N x B, landing as [orbital][y][zz]); the copies complete on
// mbarriers that every thread waits on with a time limit.  The same boxes of the FP32 V_x phi
// accumulator (tmV, laid out like the orbitals) are prefetched into L2 at the start, and the
// block's scaled sums are added into them at the end by two tensor reduce-adds.  Couples without
// pairs are read like the others (their slots of W hold stale values) and cleared in shared
// memory before the transform.
constexpr long long kTmaWaitCycles = 1LL << 30;  // about half a second

template <typename T, int N, int B>
__global__ void __launch_bounds__(DenseGeo<T, N>::NT, DenseGeo<T, N>::MINB)
k_y_acc_dense_tma(const __grid_constant__ CUtensorMap tmW, const __grid_constant__ CUtensorMap tmOrb,
                  const __grid_constant__ CUtensorMap tmV, const int4* __restrict__ couples,
                  const int* __restrict__ slot_list, const int* __restrict__ slot_couple_base, const int2* __restrict__ slot_blocks, int c0,
                  const cx<T>* __restrict__ twg, double vscale, int* __restrict__ err, int stall) {
  using C = cx<T>;
  using G = DenseGeo<T, N>;
  constexpr int ZC = G::ZC, PTS = G::PTS, NP = G::NP, NT = G::NT;
  constexpr int HB = B / 2;
  constexpr int RPI = G::RPI;        // orbital rows per iteration
  constexpr int CPI = RPI * HB;      // couples per iteration
  constexpr int LN = CPI * ZC;       // lines of the tile [y][couple][zz]
  constexpr int RING = kDenseRingCt;
  constexpr int ITERS = B / RPI;
  constexpr uint32_t kTileBytes = N * LN * sizeof(C);
  constexpr uint32_t kOrbTileBytes = B * PTS * sizeof(T);
  constexpr StagePlan P = Plan<N>::p;
  static_assert(B % RPI == 0, "rows per iteration must divide the block");
  static_assert(B * HB <= 32, "one mask word per block pair");
  static_assert(kTileBytes % 128 == 0 && kOrbTileBytes % 128 == 0, "tensor-copy destinations stay 128-byte aligned");
  // the host encodes boxes of 16 x couples x N (transforms) and 8 x N x 8 (orbitals): the byte
  // counts the mbarriers expect are those boxes only when ZC = 8 and B = 8
  static_assert(ZC == 8 && B == 8, "box sizes of the host's tensor maps");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[RING + 1];  // the ring's slots, then the orbital tiles
  __shared__ unsigned live_mask;
  unsigned char* base = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
  C* tiles = reinterpret_cast<C*>(base);                   // RING x [N][LN]
  T* phiI = reinterpret_cast<T*>(tiles + RING * N * LN);   // [B][PTS]
  T* accI = phiI + B * PTS;                                // [B][PTS]: phi_J on arrival, then the V_I sums
  C* tw = reinterpret_cast<C*>(accI + B * PTS);
  const CUtensorMap* mapW = &tmW;
  const CUtensorMap* mapOrb = &tmOrb;

  const int z0 = blockIdx.x * ZC;
  const int zcn = min(ZC, N - z0);
  const int x = blockIdx.y;
  const int slot = slot_list[blockIdx.z];
  const int2 blk = slot_blocks[slot];
  const int I0 = blk.x * B, J0 = blk.y * B;
  const int cs = slot_couple_base[slot];
  // thread 0's account of its copies: couple tiles issued, tiles it has seen land (in order), and
  // whether the orbital tiles have landed; what it has not seen land is waited for before exit
  int issued = 0, landed = 0;
  bool orb_landed = false;
  // iteration k's couple tile -> ring slot k % RING (thread 0 only).  stall (a failure-detection
  // test): the first tile's mbarrier expects 16 bytes more than the copy brings, so its wait can
  // only end by running out
  auto issue = [&](int k) {
    if (k >= ITERS) return;
    uint64_t* bar = &bars[k % RING];
    tma::expect_tx(bar, kTileBytes + (stall && k == 0 ? 16u : 0u));
    tma::load4d(tiles + (k % RING) * N * LN, mapW, 2 * z0, cs - c0 + k * CPI, 0, x, bar);
    issued = k + 1;
  };
  // thread 0 starts the copies at once: they do not depend on which couples hold pairs
  __shared__ int skip;
  __shared__ int failed;  // set by any thread whose wait ran out; read after the next barrier
  if (threadIdx.x == 0) {
    failed = 0;
    for (int i = 0; i <= RING; ++i) tc::mbar_init(&bars[i], 1);
    tc::mbar_init_fence();
    // a block of this launch whose copies never arrived: the result is void, start no more copies
    skip = *(volatile const int*)err & kErrTimeout;
    if (!skip) {
      tma::expect_tx(&bars[RING], 2 * kOrbTileBytes);
      tma::load4d(phiI, mapOrb, z0, 0, I0, x, &bars[RING]);
      tma::load4d(accI, mapOrb, z0, 0, J0, x, &bars[RING]);
#pragma unroll
      for (int k = 0; k < RING - 1; ++k) issue(k);
      // the V_x phi tiles that the flush reads and rewrites at the end head for L2 now
      tma::prefetch4d(&tmV, z0, 0, I0, x);
      tma::prefetch4d(&tmV, z0, 0, J0, x);
    }
  }
  // which couples of the block pair hold pairs (bit t of the mask: couple cs + t)
  if (threadIdx.x < 32) {
    const unsigned m = __ballot_sync(0xffffffffu, threadIdx.x < B * HB && !couple_empty(couples[cs + threadIdx.x]));
    if (threadIdx.x == 0) live_mask = m;
  }
  for (int i = threadIdx.x; i < P.twtotal; i += NT) tw[i] = twg[i];
  __syncthreads();
  if (skip) return;  // the same for every thread of the block
  const unsigned live = live_mask;

  // a wait that runs out is retried once (the copy may still land); after that this thread waits
  // no more, and the block stops at its next vote
  bool waits_ok = true;
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (!waits_ok) return false;
    if (tc::mbar_wait_cycles(bar, parity, kTmaWaitCycles) || tc::mbar_wait_cycles(bar, parity, kTmaWaitCycles))
      return true;
    waits_ok = false;
    failed = 1;
    return false;
  };
  orb_landed = wait(&bars[RING], 0);

  bool ok[NP];
  T phiJ[NP][B], accJ[NP][B];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int p = threadIdx.x + k * NT;
    const int y = p / ZC, zz = p - y * ZC;
    ok[k] = p < PTS && zz < zcn;  // (points past z = N lie outside tmV: the flush skips them)
#pragma unroll
    for (int j = 0; j < B; ++j) {
      phiJ[k][j] = ok[k] ? accI[j * PTS + p] : T(0);
      accJ[k][j] = T(0);
    }
  }
  // (a thread rewrites accI only at its own points, after it has read phi_J there)

  const T vs = (T)vscale;
  // every thread's waits so far have ended with their copies landed: the same verdict for the block
  __syncthreads();
  bool block_ok = *(volatile int*)&failed == 0;
  // (a constant trip count, so the loop unrolls; after a failed vote the iterations do nothing)
#pragma unroll
  for (int kk = 0; kk < ITERS; ++kk) {
    if (!block_ok) continue;
    if (threadIdx.x == 0) issue(kk + RING - 1);
    C* buf = tiles + (kk % RING) * N * LN;
    if (wait(&bars[kk % RING], (uint32_t)((kk / RING) & 1))) landed = kk + 1;
    const unsigned dead = (~live >> (kk * CPI)) & ((1u << CPI) - 1u);
    if (dead) {  // the same for every thread of the block
      for (int i = threadIdx.x; i < N * LN; i += NT)
        if ((dead >> ((i / ZC) % CPI)) & 1u) buf[i] = C{};
      __syncthreads();
    }
    stages<N, true, 0, P.ns, LN, 1, LN, NT>(buf, tw);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = threadIdx.x + k * NT;
      if (!ok[k]) continue;
      const int y = p / ZC, zz = p - y * ZC;
#pragma unroll
      for (int u = 0; u < RPI; ++u) {
        const int r = kk * RPI + u;
        const C* vp = buf + y * LN + u * HB * ZC + zz;
        const T phii = phiI[r * PTS + p];
        T acci = T(0);
#pragma unroll
        for (int t = 0; t < HB; ++t) {
          const C v = vp[t * ZC];
          acci += v.x * phiJ[k][2 * t] + v.y * phiJ[k][2 * t + 1];
          accJ[k][2 * t] += v.x * phii;
          accJ[k][2 * t + 1] += v.y * phii;
        }
        accI[r * PTS + p] = vs * acci;
      }
    }
    // this thread's writes of the slot are ordered before the tensor copy that refills it; the
    // barrier also takes the block's vote on its waits (a copy that never landed stops the block
    // before it starts another)
    tc::fence_proxy_async();
    __syncthreads();
    block_ok = *(volatile int*)&failed == 0;
  }
  if (!block_ok) {
    if (threadIdx.x == 0) {
      atomicOr(err, kErrTimeout);
      // the copies this block started and has not seen land: waited for, again with a limit, so
      // that none is still writing into this block's shared memory when it exits
      if (!orb_landed) tc::mbar_wait_cycles(&bars[RING], 0, kTmaWaitCycles);
      for (int k = landed; k < issued; ++k)
        tc::mbar_wait_cycles(&bars[k % RING], (uint32_t)((k / RING) & 1), kTmaWaitCycles);
    }
    return;  // the call's result is void; hfx_sync_status reports HFX_ERR_TIMEOUT
  }
  // flush: V_J (registers, scaled) goes where phi_I was, V_I (scaled as stored) is in accI; both
  // are added into the call's FP32 accumulator of V_x phi by two tensor reduce-adds, which run at
  // L2 (no block of this launch touches the same elements: its block pairs are disjoint)
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int p = threadIdx.x + k * NT;
    if (p >= PTS) continue;
#pragma unroll
    for (int j = 0; j < B; ++j) phiI[j * PTS + p] = vs * accJ[k][j];
  }
  tc::fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    tma::reduce_add4d(&tmV, z0, 0, J0, x, phiI);
    tma::reduce_add4d(&tmV, z0, 0, I0, x, accI);
    tma::bulk_commit();
    tma::bulk_wait_read_all();  // the sources stay in place until the tensor unit has read them
  }
}

}  // namespace ct
}  // namespace hfx
