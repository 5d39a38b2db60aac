// Register-resident forms of the forward plane pass and the x/Coulomb pass for FP32 cubic grids
// with edges up to 72 (compile-time edge N).
//
// One thread holds one whole grid line (N complex values) in registers and transforms it there:
// the N-point DFT is split N = P x Q, P-point DFTs, the twiddles w_N^(j1 k2) and Q-point DFTs, all
// with compile-time indices, so the twiddles are immediate constants and no stage goes through
// shared memory.  Shared memory is used only to turn a plane from rows into columns (one write and
// one read per point) -- two such exchanges per pass, against four write/read rounds of the
// stage-by-stage form in hfx_ct.cuh.  Orders: z and x stay natural; the forward pass stores y in
// the digit-reversed position order of the stage plan of edge N, which is the order the inverse-y
// accumulate passes (hfx_ct.cuh, hfx_ct_diag.cuh) read, so those passes are shared unchanged.
#pragma once
#include "hfx_ct.cuh"

namespace hfx {
namespace line {

template <int N> struct Split;
template <> struct Split<32> { static constexpr int P = 4, Q = 8; };
template <> struct Split<48> { static constexpr int P = 6, Q = 8; };
template <> struct Split<64> { static constexpr int P = 8, Q = 8; };
template <> struct Split<72> { static constexpr int P = 8, Q = 9; };

template <int N> struct Has { static constexpr bool value = N == 32 || N == 48 || N == 64 || N == 72; };

// DFT of N values in registers, natural order in and out: X[k] = sum_j x[j] exp(DIR 2 pi i jk/N)
template <int N, int DIR, typename C>
__device__ __forceinline__ void dft_line(C (&x)[N]) {
  dft_composite<Split<N>::P, Split<N>::Q, DIR>(x);
}

// position, in the stage plan's digit-reversed storage order, of frequency k
__host__ __device__ constexpr int pos_of_freq(const StagePlan& p, int k) {
  int pos = 0;
  for (int s = 0; s < p.ns; ++s) {
    const int d = k % p.r[s];
    k /= p.r[s];
    pos += d * p.m[s];
  }
  return pos;
}

template <int N> struct YPos {
  int v[N];
  constexpr YPos() : v() {
    constexpr StagePlan p = stage_plan(N);
    for (int k = 0; k < N; ++k) v[k] = pos_of_freq(p, k);
  }
};

template <int N> struct Geo {
  static constexpr int S = N + 1;                 // padded row stride (odd: conflict-free columns)
  static constexpr int NT = (N + 31) / 32 * 32;   // threads per block: one per line, whole warps
};

// ----------------------------------------------------------------------------------
// pass 1: pair product, forward z (rows) and y (columns) of one x-plane
// ----------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Geo<N>::NT)
k_fwd_line(const float* __restrict__ orb, long long Ntot, const int4* __restrict__ couples, int c0, int c1,
           float2* __restrict__ W) {
  constexpr int S = Geo<N>::S, NT = Geo<N>::NT, PLANE = N * N, NV = PLANE / 2;
  constexpr int U = ct::kUnroll;
  constexpr YPos<N> ypos{};
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  const int t = threadIdx.x;

  const int items = (c1 - c0) * N;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int cl = it / N;
    const int x = it - cl * N;
    const int4 cp = couples[c0 + cl];
    if (couple_empty(cp)) continue;
    const long long off = (long long)x * PLANE;
    const bool hasa = cp.x >= 0, hasb = cp.z >= 0;
    const float2* pa1 = reinterpret_cast<const float2*>(orb + (long long)(hasa ? cp.x : 0) * Ntot + off);
    const float2* pa2 = reinterpret_cast<const float2*>(orb + (long long)(hasa ? cp.y : 0) * Ntot + off);
    const float2* pb1 = reinterpret_cast<const float2*>(orb + (long long)(hasb ? cp.z : 0) * Ntot + off);
    const float2* pb2 = reinterpret_cast<const float2*>(orb + (long long)(hasb ? cp.w : 0) * Ntot + off);
    __syncthreads();  // the previous item's column reads are done with buf
    // Z = phi_a1 phi_a2 + i phi_b1 phi_b2 on the plane, two points per thread and load
    for (int i0 = t; i0 < NV; i0 += U * NT) {
      float2 a1[U], a2[U], b1[U], b2[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * NT;
        const bool in = (NV % (U * NT) == 0) || i < NV;
        const float2 zero = {0.f, 0.f};
        a1[u] = (in && hasa) ? __ldg(pa1 + i) : zero;
        a2[u] = (in && hasa) ? __ldg(pa2 + i) : zero;
        b1[u] = (in && hasb) ? __ldg(pb1 + i) : zero;
        b2[u] = (in && hasb) ? __ldg(pb2 + i) : zero;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u * NT;
        if ((NV % (U * NT) == 0) || i < NV) {
          const int p = 2 * i;
          const int y = p / N, z = p - y * N;  // N even: both points in row y
          buf[y * S + z] = make_float2(a1[u].x * a2[u].x, b1[u].x * b2[u].x);
          buf[y * S + z + 1] = make_float2(a1[u].y * a2[u].y, b1[u].y * b2[u].y);
        }
      }
    }
    __syncthreads();
    if (t < N) {  // row y = t: forward z, in place (the row stays with this thread)
      float2 v[N];
      float2* row = buf + t * S;
#pragma unroll
      for (int k = 0; k < N; ++k) v[k] = row[k];
      dft_line<N, -1>(v);
#pragma unroll
      for (int k = 0; k < N; ++k) row[k] = v[k];
    }
    __syncthreads();
    if (t < N) {  // column z = t: forward y, stored at the digit-reversed y positions
      float2 v[N];
#pragma unroll
      for (int y = 0; y < N; ++y) v[y] = buf[y * S + t];
      dft_line<N, -1>(v);
      float2* dst = W + ((long long)cl * N + x) * PLANE + t;
#pragma unroll
      for (int k = 0; k < N; ++k) dst[ypos.v[k] * N] = v[k];
    }
  }
}

// ----------------------------------------------------------------------------------
// pass 2: forward x, Coulomb multiply + energy, inverse x (columns, registers), inverse z (rows)
// ----------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(Geo<N>::NT)
k_x_line(const int4* __restrict__ couples, int c0, int c1, float2* __restrict__ W, const float* __restrict__ vline,
         double* __restrict__ epart, int energy_only) {
  constexpr int S = Geo<N>::S, NT = Geo<N>::NT, NW = NT / 32, PLANE = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  __shared__ double red[2][NW];
  const int t = threadIdx.x;
  int par = 0;

  const int items = (c1 - c0) * N;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int cl = it / N;
    const int y = it - cl * N;
    if (couple_empty(couples[c0 + cl])) continue;
    float2* wc = W + (long long)cl * N * PLANE + (long long)y * N;  // (x, z) at wc[x * PLANE + z]
    __syncthreads();  // the previous item's column reads are done with buf
    float e = 0.f;    // this thread's N terms in FP32; FP64 from the warp sums on
    if (t < N) {      // column z = t of the (x, z) plane
      float2 v[N];
#pragma unroll
      for (int k = 0; k < N; ++k) v[k] = __ldcg(wc + (long long)k * PLANE + t);
      dft_line<N, -1>(v);
      const float* vg = vline + (long long)y * N + t;  // v(G) at [kx][y position][kz]
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float g = __ldg(vg + (long long)k * PLANE);
        e += g * (v[k].x * v[k].x + v[k].y * v[k].y);
        v[k].x *= g;
        v[k].y *= g;
      }
      if (!energy_only) {
        dft_line<N, 1>(v);
#pragma unroll
        for (int k = 0; k < N; ++k) buf[k * S + t] = v[k];
      }
    }
    {
      double d = (double)e;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
      if ((t & 31) == 0) red[par][t >> 5] = d;
    }
    __syncthreads();
    if (t < 32) {
      double r = t < NW ? red[par][t] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
      if (t == 0) epart[(long long)(c0 + cl) * N + y] = r;
    }
    par ^= 1;
    if (energy_only) continue;
    if (t < N) {  // row x = t: inverse z, in place
      float2 v[N];
      float2* row = buf + t * S;
#pragma unroll
      for (int k = 0; k < N; ++k) v[k] = row[k];
      dft_line<N, 1>(v);
#pragma unroll
      for (int k = 0; k < N; ++k) row[k] = v[k];
    }
    __syncthreads();
    if (t < N) {
#pragma unroll
      for (int k = 0; k < N; ++k) wc[(long long)k * PLANE + t] = buf[k * S + t];
    }
  }
}

}  // namespace line
}  // namespace hfx
