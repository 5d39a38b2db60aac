// Kernels of the exchange path.  One call runs, per batch of packed pair couples:
//
//   k_fwd_yz   (per couple, per x-plane)   Z = phi_a1 phi_a2 + i phi_b1 phi_b2, forward FFT
//                                           along z then y in shared memory -> W
//   k_x_coulomb(per couple, per y-plane)   forward FFT along x; v(G) multiply and the energy
//                                           sum sum_G v |Z|^2 (FP64); inverse FFT along x,
//                                           inverse FFT along z -> W
//   k_y_inv_acc(per block pair, per x-plane, per z-chunk)
//                                           inverse FFT along y of every couple of the block
//                                           pair, V_a1 += v_a phi_a2, V_a2 += v_a phi_a1,
//                                           ... accumulated on chip, then added to V_x phi (FP64)
//
// Transforms are in place: forward stages are decimation in frequency (natural order in,
// digit-reversed out), inverse stages are decimation in time (digit-reversed in, natural out),
// so no reordering pass exists; v(G) is tabulated in the digit-reversed storage order.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fft_codelets.cuh"

namespace hfx {

constexpr int kMaxStages = 8;

struct DimPlan {
  int n;                 // length
  int ns;                // number of stages
  int r[kMaxStages];     // radix of stage s (stage 0 first in the forward transform)
  int m[kMaxStages];     // sub-length after stage s: m[s] = n / (r[0] ... r[s]); m[ns-1] = 1
};

struct Geo {
  int n1, n2, n3;
  long long N;           // n1 n2 n3
  DimPlan d[3];
};

// Error bits of the device error word.
constexpr int kErrBadPair = 1;
constexpr int kErrTimeout = 2;

constexpr int kThreadsPlane = 256;  // k_fwd_yz / k_x_coulomb
constexpr int kThreadsAcc = 128;    // k_y_inv_acc

template <typename T> struct ZChunk;
template <> struct ZChunk<float> { static constexpr int value = 8; };   // 64-byte rows
template <> struct ZChunk<double> { static constexpr int value = 4; };  // 64-byte rows

// ----------------------------------------------------------------------------------
// one in-place radix-R stage over `lines` lines of length n held in shared memory.
// Element e of line l lives at buf[l*ls + e*es].  Butterfly q in [0, n/R): j1 = q mod m,
// elements (q - j1) R + j1 + k m, k < R.  Forward (DIF): DFT then twiddle w_L^{j1 k};
// inverse (DIT): conj twiddle then inverse DFT.  L = R m.  LINE_FAST maps consecutive
// threads to consecutive lines (column lines), else to consecutive butterflies of a line.
// ----------------------------------------------------------------------------------
template <int R, bool INV, bool LINE_FAST, typename C>
__device__ __forceinline__ void fft_stage(C* __restrict__ buf, const C* __restrict__ tw, int lines,
                                          int n, int m, int ls, int es) {
  const int nq = n / R;
  const int total = lines * nq;
  const int tstride = n / (R * m);
  for (int id = threadIdx.x; id < total; id += blockDim.x) {
    int line, q;
    if (LINE_FAST) { line = id % lines; q = id / lines; }
    else { q = id % nq; line = id / nq; }
    const int j1 = q % m;
    const int base = line * ls + ((q - j1) * R + j1) * es;
    const int step = m * es;
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

template <bool INV, bool LINE_FAST, typename C>
__device__ __forceinline__ void fft_stage_rt(int R, C* buf, const C* tw, int lines, int n, int m,
                                             int ls, int es) {
  switch (R) {
    case 2: fft_stage<2, INV, LINE_FAST>(buf, tw, lines, n, m, ls, es); break;
    case 3: fft_stage<3, INV, LINE_FAST>(buf, tw, lines, n, m, ls, es); break;
    case 4: fft_stage<4, INV, LINE_FAST>(buf, tw, lines, n, m, ls, es); break;
    case 5: fft_stage<5, INV, LINE_FAST>(buf, tw, lines, n, m, ls, es); break;
    case 6: fft_stage<6, INV, LINE_FAST>(buf, tw, lines, n, m, ls, es); break;
    case 8: fft_stage<8, INV, LINE_FAST>(buf, tw, lines, n, m, ls, es); break;
    case 9: fft_stage<9, INV, LINE_FAST>(buf, tw, lines, n, m, ls, es); break;
    case 10: fft_stage<10, INV, LINE_FAST>(buf, tw, lines, n, m, ls, es); break;
    case 12: fft_stage<12, INV, LINE_FAST>(buf, tw, lines, n, m, ls, es); break;
    case 16: fft_stage<16, INV, LINE_FAST>(buf, tw, lines, n, m, ls, es); break;
    default: break;
  }
}

// all forward stages [s_begin, s_end) of one dimension; a barrier after each
template <bool LINE_FAST, typename C>
__device__ __forceinline__ void fft_forward(const DimPlan& d, int s_begin, int s_end, C* buf, const C* tw,
                                            int lines, int ls, int es) {
  for (int s = s_begin; s < s_end; ++s) {
    fft_stage_rt<false, LINE_FAST>(d.r[s], buf, tw, lines, d.n, d.m[s], ls, es);
    __syncthreads();
  }
}
// inverse stages s = s_hi-1 down to s_lo; a barrier after each
template <bool LINE_FAST, typename C>
__device__ __forceinline__ void fft_inverse(const DimPlan& d, int s_lo, int s_hi, C* buf, const C* tw,
                                            int lines, int ls, int es) {
  for (int s = s_hi - 1; s >= s_lo; --s) {
    fft_stage_rt<true, LINE_FAST>(d.r[s], buf, tw, lines, d.n, d.m[s], ls, es);
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------------
// vectorised copies between global and shared memory (16-byte units)
// ----------------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ void copy_g2s(C* __restrict__ dst, const C* __restrict__ src, int count) {
  // count complex values, both 16-byte aligned, count * sizeof(C) multiple of 16
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  const int nv = count * int(sizeof(C)) / 16;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) d[i] = __ldg(s + i);
}
template <typename C>
__device__ __forceinline__ void copy_s2g(C* __restrict__ dst, const C* __restrict__ src, int count) {
  const int4* s = reinterpret_cast<const int4*>(src);
  int4* d = reinterpret_cast<int4*>(dst);
  const int nv = count * int(sizeof(C)) / 16;
  for (int i = threadIdx.x; i < nv; i += blockDim.x) d[i] = s[i];
}

template <typename T>
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

// ----------------------------------------------------------------------------------
// pass 1: pair product + forward FFT along z and y of one x-plane
// ----------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreadsPlane)
k_fwd_yz(Geo g, const T* __restrict__ orb, const int4* __restrict__ couples,
         const int* __restrict__ batch_begin, int batch, cx<T>* __restrict__ W,
         const cx<T>* __restrict__ tw2g, const cx<T>* __restrict__ tw3g) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const int plane = n2 * n3;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw2 = buf + plane;
  C* tw3 = tw2 + n2;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = tw2g[i];
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw3[i] = tw3g[i];

  const int c0 = batch_begin[batch], c1 = batch_begin[batch + 1];
  const long long items = (long long)(c1 - c0) * n1;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int cl = int(it / n1);
    const int x = int(it - (long long)cl * n1);
    const int4 cp = couples[c0 + cl];
    const long long off = (long long)x * plane;
    const T* pa1 = orb + (long long)cp.x * g.N + off;
    const T* pa2 = orb + (long long)cp.y * g.N + off;
    const bool hasb = cp.z >= 0;
    const T* pb1 = orb + (long long)(hasb ? cp.z : 0) * g.N + off;
    const T* pb2 = orb + (long long)(hasb ? cp.w : 0) * g.N + off;
    __syncthreads();  // previous item's store has finished reading buf
    if constexpr (sizeof(T) == 4) {
      const int nv = plane / 4;
      for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        float4 a1 = __ldg(reinterpret_cast<const float4*>(pa1) + i);
        float4 a2 = __ldg(reinterpret_cast<const float4*>(pa2) + i);
        float4 b1 = make_float4(0.f, 0.f, 0.f, 0.f), b2 = b1;
        if (hasb) {
          b1 = __ldg(reinterpret_cast<const float4*>(pb1) + i);
          b2 = __ldg(reinterpret_cast<const float4*>(pb2) + i);
        }
        float4* d = reinterpret_cast<float4*>(buf + 4 * i);
        d[0] = make_float4(a1.x * a2.x, b1.x * b2.x, a1.y * a2.y, b1.y * b2.y);
        d[1] = make_float4(a1.z * a2.z, b1.z * b2.z, a1.w * a2.w, b1.w * b2.w);
      }
    } else {
      const int nv = plane / 2;
      for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        double2 a1 = __ldg(reinterpret_cast<const double2*>(pa1) + i);
        double2 a2 = __ldg(reinterpret_cast<const double2*>(pa2) + i);
        double2 b1 = make_double2(0.0, 0.0), b2 = b1;
        if (hasb) {
          b1 = __ldg(reinterpret_cast<const double2*>(pb1) + i);
          b2 = __ldg(reinterpret_cast<const double2*>(pb2) + i);
        }
        buf[2 * i] = make_double2(a1.x * a2.x, b1.x * b2.x);
        buf[2 * i + 1] = make_double2(a1.y * a2.y, b1.y * b2.y);
      }
    }
    __syncthreads();
    // z: n2 rows of length n3 (contiguous), butterflies of a row on consecutive threads
    fft_forward<false>(g.d[2], 0, g.d[2].ns, buf, tw3, n2, n3, 1);
    // y: n3 columns of length n2 (stride n3), consecutive threads on consecutive columns
    fft_forward<true>(g.d[1], 0, g.d[1].ns, buf, tw2, n3, 1, n3);
    copy_s2g(W + ((long long)cl * n1 + x) * plane, buf, plane);
  }
}

// ----------------------------------------------------------------------------------
// pass 2: forward FFT along x, Coulomb multiply + energy, inverse along x and z
// ----------------------------------------------------------------------------------
template <int R, typename C, typename T>
__device__ __forceinline__ void x_last_coulomb(C* __restrict__ buf, int n1, int n3, const T* __restrict__ vy,
                                               long long vstride_x, bool energy_only, double& e_acc) {
  // last forward stage of x (m = 1: no twiddles) fused with the first inverse stage (also m = 1)
  const int nq = n1 / R;
  const int total = n3 * nq;
  for (int id = threadIdx.x; id < total; id += blockDim.x) {
    const int z = id % n3, q = id / n3;
    const int base = q * R * n3 + z;
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[base + k * n3];
    Dft<R, -1, C>::run(v);
    T e = T(0);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const T vg = vy[(long long)(q * R + k) * vstride_x + z];
      e += vg * (v[k].x * v[k].x + v[k].y * v[k].y);
      v[k].x *= vg;
      v[k].y *= vg;
    }
    e_acc += double(e);
    if (!energy_only) {
      Dft<R, 1, C>::run(v);
#pragma unroll
      for (int k = 0; k < R; ++k) buf[base + k * n3] = v[k];
    }
  }
}

template <typename C, typename T>
__device__ __forceinline__ void x_last_coulomb_rt(int R, C* buf, int n1, int n3, const T* vy, long long vsx,
                                                  bool eo, double& e) {
  switch (R) {
    case 2: x_last_coulomb<2>(buf, n1, n3, vy, vsx, eo, e); break;
    case 3: x_last_coulomb<3>(buf, n1, n3, vy, vsx, eo, e); break;
    case 4: x_last_coulomb<4>(buf, n1, n3, vy, vsx, eo, e); break;
    case 5: x_last_coulomb<5>(buf, n1, n3, vy, vsx, eo, e); break;
    case 6: x_last_coulomb<6>(buf, n1, n3, vy, vsx, eo, e); break;
    case 8: x_last_coulomb<8>(buf, n1, n3, vy, vsx, eo, e); break;
    case 9: x_last_coulomb<9>(buf, n1, n3, vy, vsx, eo, e); break;
    case 10: x_last_coulomb<10>(buf, n1, n3, vy, vsx, eo, e); break;
    case 12: x_last_coulomb<12>(buf, n1, n3, vy, vsx, eo, e); break;
    case 16: x_last_coulomb<16>(buf, n1, n3, vy, vsx, eo, e); break;
    default: break;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreadsPlane)
k_x_coulomb(Geo g, const int* __restrict__ batch_begin, int batch, cx<T>* __restrict__ W,
            const T* __restrict__ vtab, const cx<T>* __restrict__ tw1g, const cx<T>* __restrict__ tw3g,
            double* __restrict__ epart, int energy_only) {
  using C = cx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const int tile = n1 * n3;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw1 = buf + tile;
  C* tw3 = tw1 + n1;
  __shared__ double red[32];
  for (int i = threadIdx.x; i < n1; i += blockDim.x) tw1[i] = tw1g[i];
  for (int i = threadIdx.x; i < n3; i += blockDim.x) tw3[i] = tw3g[i];

  const int c0 = batch_begin[batch], c1 = batch_begin[batch + 1];
  const long long items = (long long)(c1 - c0) * n2;
  const long long plane = (long long)n2 * n3;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const int cl = int(it / n2);
    const int y = int(it - (long long)cl * n2);
    C* wc = W + (long long)cl * n1 * plane + (long long)y * n3;
    __syncthreads();
    // rows x of the tile: W[cl][x][y][:], n3 contiguous complex values each
    const int vpr = n3 * int(sizeof(C)) / 16;
    for (int i = threadIdx.x; i < n1 * vpr; i += blockDim.x) {
      const int xx = i / vpr, vv = i - xx * vpr;
      reinterpret_cast<int4*>(buf + xx * n3)[vv] = reinterpret_cast<const int4*>(wc + xx * plane)[vv];
    }
    __syncthreads();
    const DimPlan& dx = g.d[0];
    fft_forward<true>(dx, 0, dx.ns - 1, buf, tw1, n3, 1, n3);
    double e = 0.0;
    x_last_coulomb_rt(dx.r[dx.ns - 1], buf, n1, n3, vtab + (long long)y * n3, plane, energy_only != 0, e);
    const double es = block_sum<T>(e, red);
    if (threadIdx.x == 0) epart[(long long)(c0 + cl) * n2 + y] = es;
    if (energy_only) continue;
    __syncthreads();
    fft_inverse<true>(dx, 0, dx.ns - 1, buf, tw1, n3, 1, n3);
    fft_inverse<false>(g.d[2], 0, g.d[2].ns, buf, tw3, n1, n3, 1);
    for (int i = threadIdx.x; i < n1 * vpr; i += blockDim.x) {
      const int xx = i / vpr, vv = i - xx * vpr;
      reinterpret_cast<int4*>(wc + xx * plane)[vv] = reinterpret_cast<const int4*>(buf + xx * n3)[vv];
    }
  }
}

// ----------------------------------------------------------------------------------
// pass 3: inverse FFT along y for every couple of one block pair on one (x, z-chunk) tile,
// V_x phi accumulation on chip, one FP64 read-modify-write of V per block pair
// ----------------------------------------------------------------------------------
struct AccCtx {
  int i0, ni;   // block I: orbitals [i0, i0 + ni)
  int j0, nj;   // block J (same as I for a diagonal block pair)
  bool same;
  __device__ __forceinline__ int local(int o) const { return (o - i0 < ni && o >= i0) ? o - i0 : ni + (o - j0); }
};

template <int R, typename C, typename T>
__device__ __forceinline__ void y_last_acc(C* __restrict__ buf, const C* __restrict__ tw, int n2, int m, int zc,
                                           int zcn, T* __restrict__ acc, int tile_pts, const T* __restrict__ orb,
                                           long long N, long long rowoff, int n3, int4 cp, const AccCtx& ac) {
  // final inverse stage (stage 0: L = n2, one block, m = n2 / R), natural-order outputs
  const int total = zcn * m;
  const int la1 = ac.local(cp.x), la2 = ac.local(cp.y);
  const bool hasb = cp.z >= 0;
  const int lb1 = hasb ? ac.local(cp.z) : 0, lb2 = hasb ? ac.local(cp.w) : 0;
  const T* pa1 = orb + (long long)cp.x * N + rowoff;
  const T* pa2 = orb + (long long)cp.y * N + rowoff;
  const T* pb1 = orb + (long long)(hasb ? cp.z : 0) * N + rowoff;
  const T* pb2 = orb + (long long)(hasb ? cp.w : 0) * N + rowoff;
  const bool adiag = cp.x == cp.y, bdiag = cp.z == cp.w;
  for (int id = threadIdx.x; id < total; id += blockDim.x) {
    const int zz = id % zcn, j1 = id / zcn;
    C v[R];
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = buf[(j1 + k * m) * zc + zz];
    if (m > 1) {
#pragma unroll
      for (int k = 1; k < R; ++k) v[k] = cmulc(v[k], tw[j1 * k]);
    }
    Dft<R, 1, C>::run(v);
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const int y = j1 + k * m;
      const int p = y * zc + zz;
      const long long go = (long long)y * n3 + zz;
      const T va = v[k].x, vb = v[k].y;
      const T fa1 = __ldg(pa1 + go), fa2 = __ldg(pa2 + go);
      acc[la1 * tile_pts + p] += va * fa2;
      if (!adiag) acc[la2 * tile_pts + p] += va * fa1;
      if (hasb) {
        const T fb1 = __ldg(pb1 + go), fb2 = __ldg(pb2 + go);
        acc[lb1 * tile_pts + p] += vb * fb2;
        if (!bdiag) acc[lb2 * tile_pts + p] += vb * fb1;
      }
    }
  }
}

template <typename C, typename T>
__device__ __forceinline__ void y_last_acc_rt(int R, C* buf, const C* tw, int n2, int m, int zc, int zcn, T* acc,
                                              int tp, const T* orb, long long N, long long ro, int n3, int4 cp,
                                              const AccCtx& ac) {
  switch (R) {
    case 2: y_last_acc<2>(buf, tw, n2, m, zc, zcn, acc, tp, orb, N, ro, n3, cp, ac); break;
    case 3: y_last_acc<3>(buf, tw, n2, m, zc, zcn, acc, tp, orb, N, ro, n3, cp, ac); break;
    case 4: y_last_acc<4>(buf, tw, n2, m, zc, zcn, acc, tp, orb, N, ro, n3, cp, ac); break;
    case 5: y_last_acc<5>(buf, tw, n2, m, zc, zcn, acc, tp, orb, N, ro, n3, cp, ac); break;
    case 6: y_last_acc<6>(buf, tw, n2, m, zc, zcn, acc, tp, orb, N, ro, n3, cp, ac); break;
    case 8: y_last_acc<8>(buf, tw, n2, m, zc, zcn, acc, tp, orb, N, ro, n3, cp, ac); break;
    case 9: y_last_acc<9>(buf, tw, n2, m, zc, zcn, acc, tp, orb, N, ro, n3, cp, ac); break;
    case 10: y_last_acc<10>(buf, tw, n2, m, zc, zcn, acc, tp, orb, N, ro, n3, cp, ac); break;
    case 12: y_last_acc<12>(buf, tw, n2, m, zc, zcn, acc, tp, orb, N, ro, n3, cp, ac); break;
    case 16: y_last_acc<16>(buf, tw, n2, m, zc, zcn, acc, tp, orb, N, ro, n3, cp, ac); break;
    default: break;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreadsAcc)
k_y_inv_acc(Geo g, const T* __restrict__ orb, const int4* __restrict__ couples,
            const int* __restrict__ batch_begin, int batch, const int* __restrict__ slot_begin,
            const int2* __restrict__ slot_blocks, int slot0, int bsize, int n_orb,
            const cx<T>* __restrict__ W, const cx<T>* __restrict__ tw2g, double* __restrict__ V,
            double vscale) {
  using C = cx<T>;
  constexpr int ZC = ZChunk<T>::value;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = g.n1, n2 = g.n2, n3 = g.n3;
  const int z0 = blockIdx.x * ZC;
  const int zcn = min(ZC, n3 - z0);
  const int x = blockIdx.y;
  const int slot = slot0 + blockIdx.z;
  const int tile_pts = n2 * ZC;
  C* buf = reinterpret_cast<C*>(smem_raw);
  C* tw2 = buf + tile_pts;
  T* acc = reinterpret_cast<T*>(tw2 + n2);

  const int2 blk = slot_blocks[slot];
  AccCtx ac;
  ac.i0 = blk.x * bsize; ac.ni = min(bsize, n_orb - ac.i0);
  ac.j0 = blk.y * bsize; ac.nj = min(bsize, n_orb - ac.j0);
  ac.same = blk.x == blk.y;
  const int nloc = ac.same ? ac.ni : ac.ni + ac.nj;

  for (int i = threadIdx.x; i < n2; i += blockDim.x) tw2[i] = tw2g[i];
  for (int i = threadIdx.x; i < nloc * tile_pts; i += blockDim.x) acc[i] = T(0);

  const int cb0 = batch_begin[batch];
  const int cs = slot_begin[slot], ce = slot_begin[slot + 1];
  const long long plane = (long long)n2 * n3;
  const long long rowoff = (long long)x * plane + z0;
  const DimPlan& dy = g.d[1];
  for (int c = cs; c < ce; ++c) {
    const int4 cp = couples[c];
    const C* src = W + ((long long)(c - cb0) * n1 + x) * plane + z0;
    __syncthreads();  // previous couple done with buf (and acc/tw init complete)
    // tile [n2][ZC]: rows of zcn complex (zcn even, 16-byte multiples)
    const int vpr = zcn * int(sizeof(C)) / 16;
    for (int i = threadIdx.x; i < n2 * vpr; i += blockDim.x) {
      const int yy = i / vpr, vv = i - yy * vpr;
      reinterpret_cast<int4*>(buf + yy * ZC)[vv] = __ldg(reinterpret_cast<const int4*>(src + (long long)yy * n3) + vv);
    }
    __syncthreads();
    fft_inverse<true>(dy, 1, dy.ns, buf, tw2, zcn, 1, ZC);
    y_last_acc_rt(dy.r[0], buf, tw2, n2, dy.m[0], ZC, zcn, acc, tile_pts, orb, g.N, rowoff, n3, cp, ac);
  }
  __syncthreads();
  // flush: V[o][x][y][z0 + zz] += vscale * acc
  for (int i = threadIdx.x; i < nloc * n2 * zcn; i += blockDim.x) {
    const int lo = i / (n2 * zcn);
    const int rem = i - lo * (n2 * zcn);
    const int yy = rem / zcn, zz = rem - yy * zcn;
    const int o = (lo < ac.ni) ? ac.i0 + lo : ac.j0 + (lo - ac.ni);
    double* dst = V + (long long)o * g.N + rowoff + (long long)yy * n3 + zz;
    *dst += vscale * double(acc[lo * tile_pts + yy * ZC + zz]);
  }
}

}  // namespace hfx
