// Kernels of the exchange path.  One call runs, per batch of packed pair couples (two real pair
// densities per complex transform, Z = rho_a + i rho_b):
//
//   k_fwd_yz    (couple, x-plane)   Z = phi_a1 phi_a2 + i phi_b1 phi_b2; forward FFT along z
//                                    and y in shared memory -> W
//   k_x_coulomb (couple, y-plane)   forward FFT along x; v(G) multiply and the energy sum
//                                    sum_G v |Z|^2 (FP64); inverse FFT along x and z -> W
//   k_y_acc_dense (off-diagonal block pair of full blocks, x-plane, z-chunk)
//                                    inverse FFT along y of the block pair's couples one orbital
//                                    row at a time; V_i and V_J accumulated in registers
//   k_y_acc_generic (any other block pair, x-plane, z-chunk)
//                                    the same with the accumulators in shared memory
//
// Transforms are in place: forward stages are decimation in frequency (natural order in,
// digit-reversed out), inverse stages decimation in time (digit-reversed in, natural out), so no
// reordering pass exists; v(G) is tabulated in the digit-reversed storage order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_codelets.cuh"
#include "fft_plan.h"

namespace hfx {

// Division by a fixed divisor d < 2^16 for dividends x < 2^16: q = floor(x * ceil(2^32/d) / 2^32).
// The product's error is below x / 2^32 < 2^-16 < 1/d, so the floor is exact.
struct FastDiv {
  uint32_t d, M;
  static FastDiv make(uint32_t d_) {
    FastDiv f;
    f.d = d_;
    f.M = d_ > 1 ? 0xFFFFFFFFu / d_ + 1u : 0u;
    return f;
  }
  __device__ __forceinline__ int div(int x) const { return d == 1 ? x : (int)__umulhi((uint32_t)x, M); }
};

__device__ __forceinline__ FastDiv fastdiv_dev(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.M = d > 1 ? 0xFFFFFFFFu / d + 1u : 0u;
  return f;
}

struct DimPlan {
  int n;                    // length
  int ns;                   // number of stages
  int r[kMaxStages];        // radix of stage s (stage 0 first in the forward transform)
  int m[kMaxStages];        // sub-length after stage s: m[s] = n / (r[0] ... r[s]); m[ns-1] = 1
  FastDiv mdiv[kMaxStages];
  FastDiv ndiv;             // division by n (lines of this length in a plane)
};

struct Geo {
  int n1, n2, n3;
  long long N;              // n1 n2 n3
  int S;                    // padded shared-memory row stride of the planes: n3 + 1 (odd)
  DimPlan d[3];
};

// Error bits of the device error word.
constexpr int kErrBadPair = 1;
constexpr int kErrTimeout = 2;
// HFX_DEBUG builds: a workspace guard band lost its pattern; a placed couple is off its canonical place
constexpr int kErrGuard = 16;
constexpr int kErrLayout = 32;

constexpr int kThreadsPlane = 256;  // k_fwd_yz / k_x_coulomb

template <typename T> struct ZChunk;
template <> struct ZChunk<float> { static constexpr int value = 8; };   // 64-byte rows
template <> struct ZChunk<double> { static constexpr int value = 4; };  // 64-byte rows

__device__ __forceinline__ bool couple_empty(int4 cp) { return cp.x < 0 && cp.z < 0; }

// ----------------------------------------------------------------------------------
// one in-place radix-R stage over `lines` lines of length n held in shared memory.
// Element e of line l lives at buf[l*ls + e*es].  Butterfly q in [0, n/R): j1 = q mod m,
// elements (q - j1) R + j1 + k m, k < R.  Forward (DIF): DFT then twiddle w_L^{j1 k};
// inverse (DIT): conj twiddle then inverse DFT (L = R m).  Consecutive threads take the same
// butterfly of consecutive lines, so twiddle reads are broadcasts and, with an odd or unit
// line stride, the data accesses hit distinct banks.
// ----------------------------------------------------------------------------------
template <int R, bool INV, typename C>
__device__ __forceinline__ void fft_stage(C* __restrict__ buf, const C* __restrict__ tw, int lines,
                                          FastDiv ldiv, int n, int m, FastDiv mdiv, int ls, int es) {
  const int nq = n / R;
  const int total = lines * nq;
  const int tstride = n / (R * m);
  const int step = m * es;
  for (int id = threadIdx.x; id < total; id += blockDim.x) {
    const int q = ldiv.div(id);
    const int line = id - q * lines;
    const int blk = mdiv.div(q);
    const int j1 = q - blk * m;
    const int base = line * ls + (blk * R * m + j1) * es;
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[base + k * step];
    if (!INV) {
      Dft<R, -1, C>::run(v);
      if (m > 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = cmul(v[k], tw[j1 * k * tstride]);
      }
    } else {
      if (m > 1) {
#pragma unroll
        for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], tw[j1 * k * tstride]);
      }
      Dft<R, 1, C>::run(v);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) buf[base + k * step] = v[k];
  }
}

template <bool INV, typename C>
__device__ __forceinline__ void fft_stage_rt(int R, C* buf, const C* tw, int lines, FastDiv ldiv, int n, int m,
                                             FastDiv mdiv, int ls, int es) {
  switch (R) {
    case 2: fft_stage<2, INV>(buf, tw, lines, ldiv, n, m, mdiv, ls, es); break;
    case 3: fft_stage<3, INV>(buf, tw, lines, ldiv, n, m, mdiv, ls, es); break;
    case 4: fft_stage<4, INV>(buf, tw, lines, ldiv, n, m, mdiv, ls, es); break;
    case 5: fft_stage<5, INV>(buf, tw, lines, ldiv, n, m, mdiv, ls, es); break;
    case 6: fft_stage<6, INV>(buf, tw, lines, ldiv, n, m, mdiv, ls, es); break;
    case 8: fft_stage<8, INV>(buf, tw, lines, ldiv, n, m, mdiv, ls, es); break;
    case 9: fft_stage<9, INV>(buf, tw, lines, ldiv, n, m, mdiv, ls, es); break;
    case 10: fft_stage<10, INV>(buf, tw, lines, ldiv, n, m, mdiv, ls, es); break;
    case 12: fft_stage<12, INV>(buf, tw, lines, ldiv, n, m, mdiv, ls, es); break;
    case 16: fft_stage<16, INV>(buf, tw, lines, ldiv, n, m, mdiv, ls, es); break;
    default: break;
  }
}

// forward stages [s_begin, s_end) of one dimension, a barrier after each
template <typename C>
__device__ __forceinline__ void fft_forward(const DimPlan& d, int s_begin, int s_end, C* buf, const C* tw, int lines,
                                            FastDiv ldiv, int ls, int es) {
  for (int s = s_begin; s < s_end; ++s) {
    fft_stage_rt<false>(d.r[s], buf, tw, lines, ldiv, d.n, d.m[s], d.mdiv[s], ls, es);
    __syncthreads();
  }
}
// inverse stages s = s_hi-1 down to s_lo, a barrier after each
template <typename C>
__device__ __forceinline__ void fft_inverse(const DimPlan& d, int s_lo, int s_hi, C* buf, const C* tw, int lines,
                                            FastDiv ldiv, int ls, int es) {
  for (int s = s_hi - 1; s >= s_lo; --s) {
    fft_stage_rt<true>(d.r[s], buf, tw, lines, ldiv, d.n, d.m[s], d.mdiv[s], ls, es);
    __syncthreads();
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  // deterministic tree: warp shuffles, then warp 0 over the warp partials
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    r = (l < nw) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

// plane copies, one complex value per thread step (consecutive threads on consecutive z: 8- or
// 16-byte coalesced global accesses and conflict-free shared accesses into the padded rows); the
// loads go through L2 only (the plane is read once, and in a persistent launch another block of
// the same launch may have written it)
constexpr int kLoadUnroll = 4;  // loads each thread keeps in flight per copy step

template <typename C>
__device__ __forceinline__ void plane_g2s(C* __restrict__ buf, int S, const C* __restrict__ src, long long gstride,
                                          int rows, int n3, FastDiv n3div) {
  const int total = rows * n3;
  for (int p0 = threadIdx.x; p0 < total; p0 += kLoadUnroll * blockDim.x) {
    C v[kLoadUnroll];
#pragma unroll
    for (int u = 0; u < kLoadUnroll; ++u) {
      const int p = p0 + u * blockDim.x;
      if (p < total) {
        const int r = n3div.div(p), z = p - r * n3;
        v[u] = __ldcg(src + r * gstride + z);
      }
    }
#pragma unroll
    for (int u = 0; u < kLoadUnroll; ++u) {
      const int p = p0 + u * blockDim.x;
      if (p < total) {
        const int r = n3div.div(p), z = p - r * n3;
        buf[r * S + z] = v[u];
      }
    }
  }
}
template <typename C>
__device__ __forceinline__ void plane_s2g(C* __restrict__ dst, long long gstride, const C* __restrict__ buf, int S,
                                          int rows, int n3, FastDiv n3div) {
  const int total = rows * n3;
  for (int p = threadIdx.x; p < total; p += blockDim.x) {
    const int r = n3div.div(p), z = p - r * n3;
    dst[r * gstride + z] = buf[r * S + z];
  }
}

// ----------------------------------------------------------------------------------
// pass 1: pair product + forward FFT along z and y of one x-plane
// ----------------------------------------------------------------------------------
// one item (couple cl = it / n1, x-plane x = it mod n1); buf holds the padded plane, tw2/tw3 the
// twiddles in shared memory (loaded by the caller before its first barrier)
template <typename T>
__device__ __forceinline__ void fwd_yz_item(const Geo& g, const T* __restrict__ orb, const int4* __restrict__ couples,
                                            int c0, cx<T>* __restrict__ W, const cx<T>* tw2, const cx<T>* tw3,
                                            cx<T>* buf, long long it) {
  using C = cx<T>;
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3, S = g.S;
  const int plane = n2 * n3;
  const int cl = int(it / n1);
  const int x = int(it - (long long)cl * n1);
  const int4 cp = couples[c0 + cl];
  if (couple_empty(cp)) return;
  const long long off = (long long)x * plane;
  const bool hasa = cp.x >= 0, hasb = cp.z >= 0;
  const T* pa1 = orb + (long long)(hasa ? cp.x : 0) * g.N + off;
  const T* pa2 = orb + (long long)(hasa ? cp.y : 0) * g.N + off;
  const T* pb1 = orb + (long long)(hasb ? cp.z : 0) * g.N + off;
  const T* pb2 = orb + (long long)(hasb ? cp.w : 0) * g.N + off;
  __syncthreads();  // previous item's store has finished reading buf (and tables are loaded)
  const FastDiv n3div = g.d[2].ndiv;
  for (int p0 = threadIdx.x; p0 < plane; p0 += kLoadUnroll * blockDim.x) {
    T a1[kLoadUnroll], a2[kLoadUnroll], b1[kLoadUnroll], b2[kLoadUnroll];
#pragma unroll
    for (int u = 0; u < kLoadUnroll; ++u) {
      const int p = p0 + u * blockDim.x;
      const bool in = p < plane;
      a1[u] = (in && hasa) ? __ldg(pa1 + p) : T(0);
      a2[u] = (in && hasa) ? __ldg(pa2 + p) : T(0);
      b1[u] = (in && hasb) ? __ldg(pb1 + p) : T(0);
      b2[u] = (in && hasb) ? __ldg(pb2 + p) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kLoadUnroll; ++u) {
      const int p = p0 + u * blockDim.x;
      if (p < plane) {
        const int y = n3div.div(p), z = p - y * n3;
        buf[y * S + z] = mk<C>(a1[u] * a2[u], b1[u] * b2[u]);
      }
    }
  }
  __syncthreads();
  // z: n2 rows (stride S) of length n3; y: n3 columns (stride 1) of length n2 (element stride S)
  fft_forward(g.d[2], 0, g.d[2].ns, buf, tw3, n2, g.d[1].ndiv, S, 1);
  fft_forward(g.d[1], 0, g.d[1].ns, buf, tw2, n3, g.d[2].ndiv, 1, S);
  plane_s2g(W + ((long long)cl * n1 + x) * plane, n3, buf, S, n2, n3, g.d[2].ndiv);
}

template <typename T>
__global__ void __launch_bounds__(kThreadsPlane, 3)
k_fwd_yz(const __grid_constant__ Geo g, const T* __restrict__ orb, const int4* __restrict__ couples, int c0, int c1, cx<T>* __restrict__ W,
         const cx<T>* __restrict__ tw2g, const cx<T>* __restrict__ tw3g) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3, S = g.S;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw2 = buf + n2 * S;
  C* tw3 = tw2 + n2;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = tw2g[i];
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw3[i] = tw3g[i];
  const long long items = (long long)(c1 - c0) * n1;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) fwd_yz_item(g, orb, couples, c0, W, tw2, tw3, buf, it);
}

// ----------------------------------------------------------------------------------
// pass 2: forward FFT along x, Coulomb multiply + energy, inverse along x and z
// ----------------------------------------------------------------------------------
template <int R, typename C, typename T>
__device__ __forceinline__ double x_last_coulomb(C* __restrict__ buf, int S, int n1, int n3, FastDiv zdiv,
                                                 const T* __restrict__ vy, long long vstride_x, bool energy_only) {
  double e_acc = 0.0;
  // last forward stage of x (m = 1: no twiddles) fused with the first inverse stage (also m = 1)
  const int total = n3 * (n1 / R);
  for (int id = threadIdx.x; id < total; id += blockDim.x) {
    const int q = zdiv.div(id);
    const int z = id - q * n3;
    const int base = q * R * S + z;
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[base + k * S];
    Dft<R, -1, C>::run(v);
    T e = T(0);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const T vg = __ldg(vy + (q * R + k) * vstride_x + z);
      e += vg * (v[k].x * v[k].x + v[k].y * v[k].y);
      v[k].x *= vg;
      v[k].y *= vg;
    }
    e_acc += double(e);
    if (!energy_only) {
      Dft<R, 1, C>::run(v);
#pragma unroll
      for (int k = 0; k < R; ++k) buf[base + k * S] = v[k];
    }
  }
  return e_acc;
}

template <typename C, typename T>
__device__ __forceinline__ double x_last_coulomb_rt(int R, C* buf, int S, int n1, int n3, FastDiv zdiv, const T* vy,
                                                    long long vsx, bool eo) {
  switch (R) {
    case 2: return x_last_coulomb<2>(buf, S, n1, n3, zdiv, vy, vsx, eo);
    case 3: return x_last_coulomb<3>(buf, S, n1, n3, zdiv, vy, vsx, eo);
    case 4: return x_last_coulomb<4>(buf, S, n1, n3, zdiv, vy, vsx, eo);
    case 5: return x_last_coulomb<5>(buf, S, n1, n3, zdiv, vy, vsx, eo);
    case 6: return x_last_coulomb<6>(buf, S, n1, n3, zdiv, vy, vsx, eo);
    case 8: return x_last_coulomb<8>(buf, S, n1, n3, zdiv, vy, vsx, eo);
    case 9: return x_last_coulomb<9>(buf, S, n1, n3, zdiv, vy, vsx, eo);
    case 10: return x_last_coulomb<10>(buf, S, n1, n3, zdiv, vy, vsx, eo);
    case 12: return x_last_coulomb<12>(buf, S, n1, n3, zdiv, vy, vsx, eo);
    case 16: return x_last_coulomb<16>(buf, S, n1, n3, zdiv, vy, vsx, eo);
    default: return 0.0;
  }
}

// one item (couple cl = it / n2, y-plane y = it mod n2); red: 32 doubles of shared memory
template <typename T>
__device__ __forceinline__ void x_coulomb_item(const Geo& g, const int4* __restrict__ couples, int c0,
                                               cx<T>* __restrict__ W, const T* __restrict__ vtab, const cx<T>* tw1,
                                               const cx<T>* tw3, double* __restrict__ epart, bool energy_only,
                                               cx<T>* buf, double* red, long long it) {
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3, S = g.S;
  const long long plane = (long long)n2 * n3;
  const int cl = int(it / n2);
  const int y = int(it - (long long)cl * n2);
  if (couple_empty(couples[c0 + cl])) return;
  cx<T>* wc = W + (long long)cl * n1 * plane + (long long)y * n3;
  __syncthreads();
  plane_g2s(buf, S, wc, plane, n1, n3, g.d[2].ndiv);  // rows x: W[cl][x][y][:]
  __syncthreads();
  const DimPlan& dx = g.d[0];
  // x: n3 columns of length n1 (element stride S)
  fft_forward(dx, 0, dx.ns - 1, buf, tw1, n3, g.d[2].ndiv, 1, S);
  const double e = x_last_coulomb_rt(dx.r[dx.ns - 1], buf, S, n1, n3, g.d[2].ndiv, vtab + (long long)y * n3, plane,
                                     energy_only);
  const double es = block_sum(e, red);
  if (threadIdx.x == 0) epart[(long long)(c0 + cl) * n2 + y] = es;
  if (energy_only) return;
  __syncthreads();
  fft_inverse(dx, 0, dx.ns - 1, buf, tw1, n3, g.d[2].ndiv, 1, S);
  fft_inverse(g.d[2], 0, g.d[2].ns, buf, tw3, n1, g.d[0].ndiv, S, 1);  // z: n1 rows
  plane_s2g(wc, plane, buf, S, n1, n3, g.d[2].ndiv);
}

template <typename T>
__global__ void __launch_bounds__(kThreadsPlane, 3)
k_x_coulomb(const __grid_constant__ Geo g, const int4* __restrict__ couples, int c0, int c1, cx<T>* __restrict__ W, const T* __restrict__ vtab,
            const cx<T>* __restrict__ tw1g, const cx<T>* __restrict__ tw3g, double* __restrict__ epart,
            int energy_only) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = g.n1, n3 = g.n3, S = g.S;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw1 = buf + n1 * S;
  C* tw3 = tw1 + n1;
  __shared__ double red[32];
  for (int i = threadIdx.x; i < n1; i += blockDim.x) tw1[i] = tw1g[i];
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw3[i] = tw3g[i];
  const long long items = (long long)(c1 - c0) * g.n2;
  for (long long it = blockIdx.x; it < items; it += gridDim.x)
    x_coulomb_item(g, couples, c0, W, vtab, tw1, tw3, epart, energy_only != 0, buf, red, it);
}

// ----------------------------------------------------------------------------------
// Pencil form of passes 1 and 2, for grids whose planes do not fit in one SM's shared memory
// (FP64 on 128^3): the same transforms one or two axes at a time.
//   k_fwd_z_rows   (couple, x, row block)   pair product + forward FFT along z of rows -> W
//   k_fwd_y_cols   (couple, x, z-chunk)     forward FFT along y -> W
//   k_x_cols       (couple, y, z-chunk)     forward FFT along x, Coulomb + energy, inverse FFT
//                                           along x -> W
//   k_inv_z_rows   (couple, x, row block)   inverse FFT along z -> W
// The energy partials are per (couple, y, z-chunk).  Requires n3 % ZChunk == 0.
// ----------------------------------------------------------------------------------
constexpr int kThreadsPencil = 128;

template <typename T>
__global__ void __launch_bounds__(kThreadsPencil)
k_fwd_z_rows(const __grid_constant__ Geo g, const T* __restrict__ orb, const int4* __restrict__ couples, int c0, int c1,
             int rb, cx<T>* __restrict__ W, const cx<T>* __restrict__ tw3g) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3, S = g.S;
  C* buf = reinterpret_cast<C*>(smem_raw);  // [rb][S]
  C* tw3 = buf + rb * S;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw3[i] = tw3g[i];
  const int nrb = (n2 + rb - 1) / rb;
  const long long items = (long long)(c1 - c0) * n1 * nrb;
  const long long plane = (long long)n2 * n3;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int cl = int(it / ((long long)n1 * nrb));
    const int rem = int(it - (long long)cl * n1 * nrb);
    const int x = rem / nrb, y0 = (rem - x * nrb) * rb;
    const int rows = min(rb, n2 - y0);
    const int4 cp = couples[c0 + cl];
    if (couple_empty(cp)) continue;
    const bool hasa = cp.x >= 0, hasb = cp.z >= 0;
    const long long off = (long long)x * plane + (long long)y0 * n3;
    const T* pa1 = orb + (long long)(hasa ? cp.x : 0) * g.N + off;
    const T* pa2 = orb + (long long)(hasa ? cp.y : 0) * g.N + off;
    const T* pb1 = orb + (long long)(hasb ? cp.z : 0) * g.N + off;
    const T* pb2 = orb + (long long)(hasb ? cp.w : 0) * g.N + off;
    __syncthreads();
    for (int p = threadIdx.x; p < rows * n3; p += blockDim.x) {
      const int r = g.d[2].ndiv.div(p), z = p - r * n3;
      const T a = hasa ? __ldg(pa1 + p) * __ldg(pa2 + p) : T(0);
      const T b = hasb ? __ldg(pb1 + p) * __ldg(pb2 + p) : T(0);
      buf[r * S + z] = mk<C>(a, b);
    }
    __syncthreads();
    fft_forward(g.d[2], 0, g.d[2].ns, buf, tw3, rows, fastdiv_dev(rows), S, 1);
    plane_s2g(W + ((long long)cl * n1 + x) * plane + (long long)y0 * n3, n3, buf, S, rows, n3, g.d[2].ndiv);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreadsPencil)
k_inv_z_rows(const __grid_constant__ Geo g, const int4* __restrict__ couples, int c0, int c1, int rb,
             cx<T>* __restrict__ W, const cx<T>* __restrict__ tw3g) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3, S = g.S;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw3 = buf + rb * S;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw3[i] = tw3g[i];
  const int nrb = (n2 + rb - 1) / rb;
  const long long items = (long long)(c1 - c0) * n1 * nrb;
  const long long plane = (long long)n2 * n3;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int cl = int(it / ((long long)n1 * nrb));
    const int rem = int(it - (long long)cl * n1 * nrb);
    const int x = rem / nrb, y0 = (rem - x * nrb) * rb;
    const int rows = min(rb, n2 - y0);
    if (couple_empty(couples[c0 + cl])) continue;
    C* base = W + ((long long)cl * n1 + x) * plane + (long long)y0 * n3;
    __syncthreads();
    plane_g2s(buf, S, base, n3, rows, n3, g.d[2].ndiv);
    __syncthreads();
    fft_inverse(g.d[2], 0, g.d[2].ns, buf, tw3, rows, fastdiv_dev(rows), S, 1);
    plane_s2g(base, n3, buf, S, rows, n3, g.d[2].ndiv);
  }
}

// tile [n][ZC] of one z-chunk: load / store rows of ZC complex values (stride gstride apart)
template <typename C, int ZC>
__device__ __forceinline__ void chunk_g2s(C* __restrict__ buf, const C* __restrict__ src, long long gstride, int n) {
  for (int i = threadIdx.x; i < n * ZC; i += blockDim.x) {
    const int r = i / ZC, zz = i - r * ZC;
    buf[i] = __ldg(src + r * gstride + zz);
  }
}
template <typename C, int ZC>
__device__ __forceinline__ void chunk_s2g(C* __restrict__ dst, long long gstride, const C* __restrict__ buf, int n) {
  for (int i = threadIdx.x; i < n * ZC; i += blockDim.x) {
    const int r = i / ZC, zz = i - r * ZC;
    dst[r * gstride + zz] = buf[i];
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreadsPencil)
k_fwd_y_cols(const __grid_constant__ Geo g, const int4* __restrict__ couples, int c0, int c1, cx<T>* __restrict__ W,
             const cx<T>* __restrict__ tw2g) {
  using C = cx<T>;
  constexpr int ZC = ZChunk<T>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  C* buf = reinterpret_cast<C*>(smem_raw);  // [n2][ZC]
  C* tw2 = buf + n2 * ZC;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = tw2g[i];
  const int nzc = n3 / ZC;
  const long long items = (long long)(c1 - c0) * n1 * nzc;
  const long long plane = (long long)n2 * n3;
  const FastDiv zcdiv = fastdiv_dev(ZC);
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int cl = int(it / ((long long)n1 * nzc));
    const int rem = int(it - (long long)cl * n1 * nzc);
    const int x = rem / nzc, z0 = (rem - x * nzc) * ZC;
    if (couple_empty(couples[c0 + cl])) continue;
    C* base = W + ((long long)cl * n1 + x) * plane + z0;
    __syncthreads();
    chunk_g2s<C, ZC>(buf, base, n3, n2);
    __syncthreads();
    fft_forward(g.d[1], 0, g.d[1].ns, buf, tw2, ZC, zcdiv, 1, ZC);
    chunk_s2g<C, ZC>(base, n3, buf, n2);
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreadsPencil)
k_x_cols(const __grid_constant__ Geo g, const int4* __restrict__ couples, int c0, int c1, cx<T>* __restrict__ W,
         const T* __restrict__ vtab, const cx<T>* __restrict__ tw1g, double* __restrict__ epart, int energy_only) {
  using C = cx<T>;
  constexpr int ZC = ZChunk<T>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[32];
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  C* buf = reinterpret_cast<C*>(smem_raw);  // [n1][ZC]
  C* tw1 = buf + n1 * ZC;
  for (int i = threadIdx.x; i < n1; i += blockDim.x) tw1[i] = tw1g[i];
  const int nzc = n3 / ZC;
  const long long items = (long long)(c1 - c0) * n2 * nzc;
  const long long plane = (long long)n2 * n3;
  const FastDiv zcdiv = fastdiv_dev(ZC);
  const DimPlan& dx = g.d[0];
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int cl = int(it / ((long long)n2 * nzc));
    const int rem = int(it - (long long)cl * n2 * nzc);
    const int y = rem / nzc, zc = rem - y * nzc, z0 = zc * ZC;
    if (couple_empty(couples[c0 + cl])) continue;
    C* base = W + (long long)cl * n1 * plane + (long long)y * n3 + z0;
    __syncthreads();
    chunk_g2s<C, ZC>(buf, base, plane, n1);
    __syncthreads();
    fft_forward(dx, 0, dx.ns - 1, buf, tw1, ZC, zcdiv, 1, ZC);
    const double e = x_last_coulomb_rt(dx.r[dx.ns - 1], buf, ZC, n1, ZC, zcdiv, vtab + (long long)y * n3 + z0,
                                       plane, energy_only != 0);
    const double es = block_sum(e, red);
    if (threadIdx.x == 0) epart[((long long)(c0 + cl) * n2 + y) * nzc + zc] = es;
    if (energy_only) continue;
    __syncthreads();
    fft_inverse(dx, 0, dx.ns - 1, buf, tw1, ZC, zcdiv, 1, ZC);
    chunk_s2g<C, ZC>(base, plane, buf, n1);
  }
}

// ----------------------------------------------------------------------------------
// asynchronous 16-byte global -> shared copies (zero-filled when src_bytes == 0)
// ----------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
// 8-byte variant, for rows that start on 8-byte boundaries only
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ----------------------------------------------------------------------------------
// pass 3a: off-diagonal block pair (I, J) of two full blocks of B orbitals.  Couples sit in
// canonical order: couple c holds pairs (I0 + c / (B/2), J0 + 2 (c mod B/2)) and (.., +1).
// For each orbital row i the B/2 couples of the row are inverse-transformed along y together
// (the next row's tiles stream in meanwhile); then every thread, for its own points, forms
// V_i = sum_j v_ij phi_j (kept on chip) and V_j += v_ij phi_i (registers).  V_x phi is read and
// written once per block pair and point, in FP64.
// ----------------------------------------------------------------------------------
constexpr int kDenseMaxThreads = 512;
constexpr int kDenseRing = 3;  // orbital rows of couple tiles in flight
// compile-time dense pass: ring depth (its orbital rows per iteration are DenseGeo::RPI)
constexpr int kDenseRingCt = 2;
__host__ __device__ constexpr int dense_rows_ct(int n) { return n <= 72 ? 2 : 1; }
template <int NP> struct DenseBounds;
template <> struct DenseBounds<2> { static constexpr int threads = 320, blocks = 2; };
template <> struct DenseBounds<4> { static constexpr int threads = 512, blocks = 1; };

template <typename T, int B, int NP>
__global__ void __launch_bounds__(DenseBounds<NP>::threads, DenseBounds<NP>::blocks)
k_y_acc_dense(const __grid_constant__ Geo g, const T* __restrict__ orb, const int4* __restrict__ couples,
              const int* __restrict__ slot_list, const int* __restrict__ slot_couple_base,
              const int2* __restrict__ slot_blocks, int c0, const cx<T>* __restrict__ W,
              const cx<T>* __restrict__ tw2g, T* __restrict__ V, double vscale) {
  using C = cx<T>;
  constexpr int ZC = ZChunk<T>::value;
  constexpr int HB = B / 2;
  constexpr int LN = HB * ZC;                  // lines of the interleaved tile [y][t][zz]
  constexpr int PER = 16 / int(sizeof(C));     // complex values per 16-byte copy
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const int z0 = blockIdx.x * ZC;
  const int zcn = min(ZC, n3 - z0);
  const int x = blockIdx.y;
  const int slot = slot_list[blockIdx.z];
  const int pts = n2 * ZC;
  C* tiles = reinterpret_cast<C*>(smem_raw);   // kDenseRing x [n2][LN]
  C* tw2 = tiles + kDenseRing * n2 * LN;
  T* phiI = reinterpret_cast<T*>(tw2 + n2);    // [B][pts]
  T* accI = phiI + B * pts;                    // [B][pts]

  const int2 blk = slot_blocks[slot];
  const int I0 = blk.x * B, J0 = blk.y * B;
  const int cs = slot_couple_base[slot];
  const long long plane = (long long)n2 * n3;
  const long long rowoff = (long long)x * plane + z0;

  // tiles of orbital row r -> ring buffer r % kDenseRing (empty couples and columns past n3 read as
  // zero); a row past the block commits an empty group so the group count stays uniform
  auto issue_row = [&](int r) {
    if (r >= B) { cp_async_commit(); return; }
    C* dstb = tiles + (r % kDenseRing) * n2 * LN;
    for (int i = threadIdx.x; i < HB * n2 * (ZC / PER); i += blockDim.x) {
      const int v = i % (ZC / PER);
      const int rest = i / (ZC / PER);
      const int t = rest % HB, y = rest / HB;
      const int c = cs + r * HB + t;
      const bool live = !couple_empty(couples[c]) && v * PER < zcn;
      const C* src = W + ((long long)(c - c0) * n1 + x) * plane + (long long)y * n3 + z0 + v * PER;
      cp_async16(dstb + y * LN + t * ZC + v * PER, live ? (const void*)src : (const void*)W, live ? 16 : 0);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int r = 0; r < kDenseRing - 1; ++r) issue_row(r);

  for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = tw2g[i];
  for (int i = threadIdx.x; i < B * pts; i += blockDim.x) {
    const int o = i / pts, p = i - o * pts;
    const int y = p / ZC, zz = p - y * ZC;
    phiI[i] = zz < zcn ? __ldg(orb + (long long)(I0 + o) * g.N + rowoff + (long long)y * n3 + zz) : T(0);
  }

  // this thread's points
  long long goff[NP];
  bool ok[NP];
  int pp[NP];
  T phiJ[NP][B], accJ[NP][B];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int p = threadIdx.x + k * blockDim.x;
    const int y = p / ZC, zz = p - (p / ZC) * ZC;
    ok[k] = p < pts && zz < zcn;
    pp[k] = p;
    goff[k] = rowoff + (long long)y * n3 + zz;
#pragma unroll
    for (int j = 0; j < B; ++j) {
      phiJ[k][j] = ok[k] ? __ldg(orb + (long long)(J0 + j) * g.N + goff[k]) : T(0);
      accJ[k][j] = T(0);
    }
  }

  const FastDiv ldiv = fastdiv_dev(LN);
  for (int r = 0; r < B; ++r) {
    issue_row(r + kDenseRing - 1);  // its buffer was last read in row r - 1 (barrier passed)
    cp_async_wait<kDenseRing - 1>();
    __syncthreads();  // row r's tiles (and the tables) visible to all threads
    C* buf = tiles + (r % kDenseRing) * n2 * LN;
    fft_inverse(g.d[1], 0, g.d[1].ns, buf, tw2, LN, ldiv, 1, LN);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      if (!ok[k]) continue;
      const int p = pp[k];
      const int y = p / ZC, zz = p - y * ZC;
      const C* vp = buf + y * LN + zz;
      const T phii = phiI[r * pts + p];
      T acci = T(0);
#pragma unroll
      for (int t = 0; t < HB; ++t) {
        const C v = vp[t * ZC];
        acci += v.x * phiJ[k][2 * t] + v.y * phiJ[k][2 * t + 1];
        accJ[k][2 * t] += v.x * phii;
        accJ[k][2 * t + 1] += v.y * phii;
      }
      accI[r * pts + p] = acci;
    }
    __syncthreads();  // buffer r % kDenseRing is refilled by the copies issued in the next iteration
  }
  // flush, read-modify-write of V (FP64 on the FP64 path, the call's FP32 accumulator on the FP32
  // path): V_J from registers, V_I from shared memory; all loads first (a store could alias a later
  // load, which would serialise the round trips)
  const T vs = (T)vscale;
  T old[NP][B];
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int j = 0; j < B; ++j) old[k][j] = ok[k] ? __ldcg(V + (long long)(J0 + j) * g.N + goff[k]) : T(0);
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    if (!ok[k]) continue;
#pragma unroll
    for (int j = 0; j < B; ++j) V[(long long)(J0 + j) * g.N + goff[k]] = old[k][j] + vs * accJ[k][j];
  }
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int j = 0; j < B; ++j) old[k][j] = ok[k] ? __ldcg(V + (long long)(I0 + j) * g.N + goff[k]) : T(0);
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    if (!ok[k]) continue;
    const int p = pp[k];
#pragma unroll
    for (int j = 0; j < B; ++j) V[(long long)(I0 + j) * g.N + goff[k]] = old[k][j] + vs * accI[j * pts + p];
  }
}

// ----------------------------------------------------------------------------------
// pass 3b: any block pair (diagonal, ragged, sparse, or a block size without a dense kernel).
// The block pair's couples are taken `grp` at a time (the next group streams in while the current
// one is transformed): inverse FFT along y of the group's tiles on one (x, z-chunk), then each
// thread adds, for its own points, v_a phi_a2 to the accumulator of a1 (and v_a phi_a1 to a2's
// when a1 != a2), likewise for the b half.  Accumulators (FP32 or FP64 as the path) and, when
// they fit, the orbital tiles live in shared memory; V_x phi is read and written once per block
// pair and point, in FP64.
// ----------------------------------------------------------------------------------
constexpr int kThreadsGen = 256;
constexpr int kGenRing = 2;

// one tile of the generic accumulate pass: z-chunk zi, x-plane x, block pair `slot`; the dynamic
// shared memory `smem_raw` holds the tiles, twiddles, accumulators, orbital tiles and couple table
template <typename T>
__device__ __forceinline__ void acc_generic_item(const Geo& g, const T* __restrict__ orb,
                                                 const int4* __restrict__ couples, int slot,
                                                 const int* __restrict__ slot_couple_base,
                                                 const int2* __restrict__ slot_blocks, int bsize, int n_orb, int c0,
                                                 const cx<T>* __restrict__ W, const cx<T>* __restrict__ tw2g,
                                                 T* __restrict__ V, double vscale, int grp, int phi_smem,
                                                 int cap_max, unsigned char* smem_raw, int zi, int x) {
  using C = cx<T>;
  constexpr int ZC = ZChunk<T>::value;
  constexpr int PER = 16 / int(sizeof(C));
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const int z0 = zi * ZC;
  const int zcn = min(ZC, n3 - z0);
  const int pts = n2 * ZC;
  const int LN = grp * ZC;
  const int nloc_max = 2 * bsize;
  C* tiles = reinterpret_cast<C*>(smem_raw);          // kGenRing x [n2][LN]
  C* tw2 = tiles + kGenRing * n2 * LN;
  T* acc = reinterpret_cast<T*>(tw2 + n2);             // [nloc][pts]
  T* phi = acc + nloc_max * pts;                       // [nloc][pts] when phi_smem
  int4* cloc = reinterpret_cast<int4*>(phi + (phi_smem ? nloc_max * pts : 0));  // [cap] local indices

  const int2 blk = slot_blocks[slot];
  const int i0 = blk.x * bsize, ni = min(bsize, n_orb - i0);
  const int j0 = blk.y * bsize, nj = min(bsize, n_orb - j0);
  const bool same = blk.x == blk.y;
  const int nloc = same ? ni : ni + nj;
  auto local = [&](int o) { return (o >= i0 && o - i0 < ni) ? o - i0 : ni + (o - j0); };
  auto orbital = [&](int lo) { return lo < ni ? i0 + lo : j0 + (lo - ni); };
  const int cs = slot_couple_base[slot], nc = min(slot_couple_base[slot + 1] - cs, cap_max);
  const int ngroups = (nc + grp - 1) / grp;
  const long long plane = (long long)n2 * n3;
  const long long rowoff = (long long)x * plane + z0;

  // couple table with local orbital indices (-1: absent half)
  for (int c = threadIdx.x; c < nc; c += blockDim.x) {
    const int4 cp = couples[cs + c];
    int4 l;
    l.x = cp.x >= 0 ? local(cp.x) : -1;
    l.y = cp.x >= 0 ? local(cp.y) : -1;
    l.z = cp.z >= 0 ? local(cp.z) : -1;
    l.w = cp.z >= 0 ? local(cp.w) : -1;
    cloc[c] = l;
  }
  // orbital tiles (first copy group), in 8-byte pieces: with n3 even every row of reals starts on
  // an 8-byte boundary, but on a 16-byte one only when n3 is a multiple of 16 / sizeof(T)
  if (phi_smem) {
    constexpr int EPER = 8 / int(sizeof(T));  // reals per 8-byte copy
    constexpr int VPR = ZC / EPER;
    for (int i = threadIdx.x; i < nloc * n2 * VPR; i += blockDim.x) {
      const int v = i % VPR;
      const int rest = i / VPR;
      const int y = rest % n2, lo = rest / n2;
      const int valid = zcn - v * EPER;
      const int bytes = valid >= EPER ? 8 : (valid > 0 ? valid * int(sizeof(T)) : 0);
      const T* src = orb + (long long)orbital(lo) * g.N + rowoff + (long long)y * n3 + v * EPER;
      cp_async8(phi + lo * pts + y * ZC + v * EPER, bytes ? (const void*)src : (const void*)orb, bytes);
    }
  }
  __syncthreads();  // cloc ready for the copy issue below
  auto issue_group = [&](int q) {
    if (q < ngroups) {
      C* dstb = tiles + (q % kGenRing) * n2 * LN;
      const int VPR = ZC / PER;
      for (int i = threadIdx.x; i < grp * n2 * VPR; i += blockDim.x) {
        const int v = i % VPR;
        const int rest = i / VPR;
        const int t = rest % grp, y = rest / grp;
        const int c = q * grp + t;
        const bool live = c < nc && (cloc[c].x >= 0 || cloc[c].z >= 0) && v * PER < zcn;
        const C* src = W + ((long long)(cs + c - c0) * n1 + x) * plane + (long long)y * n3 + z0 + v * PER;
        cp_async16(dstb + y * LN + t * ZC + v * PER, live ? (const void*)src : (const void*)W, live ? 16 : 0);
      }
    }
    cp_async_commit();
  };
  for (int q = 0; q < kGenRing - 1; ++q) issue_group(q);
  for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = tw2g[i];
  for (int i = threadIdx.x; i < nloc * pts; i += blockDim.x) acc[i] = T(0);

  const FastDiv ldiv = fastdiv_dev(LN);
  for (int q = 0; q < ngroups; ++q) {
    issue_group(q + kGenRing - 1);
    cp_async_wait<kGenRing - 1>();
    __syncthreads();
    C* buf = tiles + (q % kGenRing) * n2 * LN;
    fft_inverse(g.d[1], 0, g.d[1].ns, buf, tw2, LN, ldiv, 1, LN);
    for (int p = threadIdx.x; p < pts; p += blockDim.x) {
      const int y = p / ZC, zz = p - y * ZC;
      if (zz >= zcn) continue;
      const long long go = rowoff + (long long)y * n3 + zz;
      for (int t = 0; t < grp; ++t) {
        const int c = q * grp + t;
        if (c >= nc) break;
        const int4 l = cloc[c];
        const C v = buf[y * LN + t * ZC + zz];
        if (l.x >= 0) {
          const T f1 = phi_smem ? phi[l.x * pts + p] : __ldg(orb + (long long)orbital(l.x) * g.N + go);
          const T f2 = phi_smem ? phi[l.y * pts + p] : __ldg(orb + (long long)orbital(l.y) * g.N + go);
          acc[l.x * pts + p] += v.x * f2;
          if (l.x != l.y) acc[l.y * pts + p] += v.x * f1;
        }
        if (l.z >= 0) {
          const T f1 = phi_smem ? phi[l.z * pts + p] : __ldg(orb + (long long)orbital(l.z) * g.N + go);
          const T f2 = phi_smem ? phi[l.w * pts + p] : __ldg(orb + (long long)orbital(l.w) * g.N + go);
          acc[l.z * pts + p] += v.y * f2;
          if (l.z != l.w) acc[l.w * pts + p] += v.y * f1;
        }
      }
    }
    __syncthreads();  // buffer q % kGenRing is refilled by the copies issued next
  }
  cp_async_wait<0>();
  __syncthreads();
  // flush: V[o][x][y][z0 + zz] += vscale * acc, in groups whose loads all precede their stores
  constexpr int GF = 8;
  const int total = nloc * pts;
  const T vs = (T)vscale;
  for (int i0f = threadIdx.x; i0f < total; i0f += GF * blockDim.x) {
    T old[GF];
    long long off[GF];
    bool on[GF];
#pragma unroll
    for (int u = 0; u < GF; ++u) {
      const int i = i0f + u * blockDim.x;
      const int lo = i / pts;
      const int p = i - lo * pts;
      const int yy = p / ZC, zz = p - yy * ZC;
      on[u] = i < total && zz < zcn;
      off[u] = (long long)orbital(lo) * g.N + rowoff + (long long)yy * n3 + zz;
      old[u] = on[u] ? __ldcg(V + off[u]) : T(0);
    }
#pragma unroll
    for (int u = 0; u < GF; ++u)
      if (on[u]) V[off[u]] = old[u] + vs * acc[i0f + u * blockDim.x];
  }
}


template <typename T>
__global__ void __launch_bounds__(kThreadsGen)
k_y_acc_generic(const __grid_constant__ Geo g, const T* __restrict__ orb, const int4* __restrict__ couples,
                const int* __restrict__ slot_list, const int* __restrict__ slot_couple_base,
                const int2* __restrict__ slot_blocks, int bsize, int n_orb, int c0, const cx<T>* __restrict__ W,
                const cx<T>* __restrict__ tw2g, T* __restrict__ V, double vscale, int grp, int phi_smem,
                int cap_max) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  acc_generic_item(g, orb, couples, slot_list[blockIdx.z], slot_couple_base, slot_blocks, bsize, n_orb, c0, W, tw2g, V,
                   vscale, grp, phi_smem, cap_max, smem_raw, (int)blockIdx.x, (int)blockIdx.y);
}

}  // namespace hfx
