// Kernels of the ACE operator and of the pair-list overlap screen (Sec. 2.1, Eq. vx_ace and
// the definitions of P, W, L and M after it; the overlap cut of the localised-orbital variant).
//
// Two contraction shapes carry all the grid-sized work:
//   * split contraction over the grid ("Gram"): C[a][b] = sum_p f(X[a][p]) f(Y[b][p]) with a, b
//     over orbitals (<= a few hundred) and p over N grid points; each job takes one 128 x 128
//     output tile and one run of grid points and writes an FP64 partial, and a second kernel
//     sums the partials in a fixed order (deterministic, no atomics);
//   * left multiply by a small matrix ("lmul"): C[m][p] = T[m][k] Y[k][p] (+ C), k over
//     orbitals, p over the grid, one 128 x 128 output tile per job.
// Both read FP64 operands through a three-deep cp.async ring of raw staging buffers, round
// them once to the compute type in a double-buffered shared tile, and run an 8 x 8 register
// tile per thread (256 threads, 128 x 128 per block); blocks are persistent and walk their jobs
// with the ring running across job boundaries.
//
// The Cholesky factorisation of -(M + M^T)/2 and the triangular inverse are small FP64
// kernels; the screen's pair compaction is a count / scan / write sequence over rows.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "fp_convert.cuh"
#include "hfx_ace_internal.h"

namespace hfx {
namespace ace {

namespace {

constexpr int kT = 128;                // output tile edge
constexpr int kBK = 16;                // contraction depth per stage
constexpr int kStages = 3;             // cp.async ring depth
constexpr int kThreads = 256;
constexpr int kRawStride = kBK + 2;    // doubles per staged row: 144 B, 16-byte aligned, conflict-free reads
constexpr int kSubStages = 256 / kBK;  // FP32: stages per inner partial sum (runs of 256 terms)

constexpr size_t kRawRowsBytes = size_t(kT) * kRawStride * sizeof(double);  // a [128][18] staging tile
constexpr size_t kRawColsBytes = size_t(kBK) * kT * sizeof(double);         // a [16][128] staging tile

__device__ __forceinline__ void cp_async_zfill16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_zfill8(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <typename T>
__device__ __forceinline__ double to_double(T v);
template <>
__device__ __forceinline__ double to_double<float>(float v) { return f32_to_f64_exact(v); }
template <>
__device__ __forceinline__ double to_double<double>(double v) { return v; }

template <typename T>
__device__ __forceinline__ T to_compute(double v);
template <>
__device__ __forceinline__ float to_compute<float>(double v) { return f64_to_f32_rn(v); }
template <>
__device__ __forceinline__ double to_compute<double>(double v) { return v; }

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ __forceinline__ void load(const float* p, float* r) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  }
};
template <>
struct Vec4<double> {
  static __device__ __forceinline__ void load(const double* p, double* r) {
    const double2 a = *reinterpret_cast<const double2*>(p);
    const double2 b = *reinterpret_cast<const double2*>(p + 2);
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
  }
};

// A job is one output tile and its run of stages.  Gram jobs: tile (ta, tb) of split s,
// job = s * tiles + tb * tiles_x + ta (the tiles of one split are neighbours, so they run
// together and share the split's operand rows in L2).  lmul jobs: tile (tm, tp),
// job = tp * tiles_x + tm.
struct Cursor {
  int job, ks, nst;
  int t0, t1;        // Gram: (ta, tb); lmul: (tm, tp)
  long long p0, p1;  // Gram: the split's grid points [p0, p1)
};

}  // namespace

// ------------------------------------------------------------------------------------
// the contraction kernel (both shapes)
// ------------------------------------------------------------------------------------
template <typename T, int FORM, bool VEC16, bool ABS>
__global__ void __launch_bounds__(kThreads, 1) k_ace_mm(const MmArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* rawx = reinterpret_cast<double*>(smem_raw);  // Gram: [kStages][128][kRawStride]; lmul: [kStages][16][128] T
  double* rawy = reinterpret_cast<double*>(smem_raw + kStages * kRawRowsBytes);
  // Gram: y staged like x ([128][kRawStride]); lmul: y staged as [16][128]
  constexpr size_t ybytes = FORM == kFormGram ? kRawRowsBytes : kRawColsBytes;
  T* cx = reinterpret_cast<T*>(smem_raw + kStages * (kRawRowsBytes + ybytes));  // [2][16][128]
  T* cy = cx + 2 * kBK * kT;                                                     // [2][16][128]

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;

  auto decode = [&](Cursor& c) {
    c.ks = 0;
    c.nst = 0;
    if (c.job >= a.njobs) return;
    if (FORM == kFormGram) {
      const int tiles = a.tiles_x * a.tiles_y;
      const int s = c.job / tiles, t = c.job - s * tiles;
      c.t0 = t % a.tiles_x;
      c.t1 = t / a.tiles_x;
      c.p0 = (long long)s * a.chunk;
      c.p1 = min(a.K, c.p0 + a.chunk);
      c.nst = (int)((c.p1 - c.p0 + kBK - 1) / kBK);
    } else {
      c.t0 = c.job % a.tiles_x;
      c.t1 = c.job / a.tiles_x;
      const long long k1 = a.lower ? min(a.K, (long long)(c.t0 + 1) * kT) : a.K;
      c.nst = (int)((k1 + kBK - 1) / kBK);
    }
  };
  auto next = [&](Cursor& c) {
    if (++c.ks >= c.nst) {
      c.job += gridDim.x;
      decode(c);
    }
  };

  // issue the cp.async copies of stage (job, ks) into ring slot `slot`
  auto issue = [&](const Cursor& c, int slot) {
    if (c.job >= a.njobs) return;
    if (FORM == kFormGram) {
      double* rx = rawx + (size_t)slot * kT * kRawStride;
      double* ry = rawy + (size_t)slot * kT * kRawStride;
      const long long p = c.p0 + (long long)c.ks * kBK;
      const long long valid = c.p1 - p;  // >= 1
      const double* X = reinterpret_cast<const double*>(a.x);
      if (VEC16) {
        // 128 rows x 8 pieces of 16 B per operand; this thread: rows r0 + 32 q, piece pc
        const int r0 = tid >> 3, pc = tid & 7;
        const long long left = valid - 2 * pc;
        const int bytes_in = left >= 2 ? 16 : (left == 1 ? 8 : 0);
        const int gx = c.t0 * kT + r0, gy = c.t1 * kT + r0;
        const double* sx = X + (long long)gx * a.ldx + p + 2 * pc;
        const double* sy = a.y + (long long)gy * a.ldy + p + 2 * pc;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const bool vx = gx + 32 * q < a.nx, vy = gy + 32 * q < a.ny;
          cp_async_zfill16(rx + (r0 + 32 * q) * kRawStride + 2 * pc, vx ? sx + q * 32 * a.ldx : X, vx ? bytes_in : 0);
          cp_async_zfill16(ry + (r0 + 32 * q) * kRawStride + 2 * pc, vy ? sy + q * 32 * a.ldy : a.y, vy ? bytes_in : 0);
        }
      } else {
        // 128 rows x 16 pieces of 8 B per operand; this thread: rows r0 + 16 q, piece pc
        const int r0 = tid >> 4, pc = tid & 15;
        const int bytes_in = pc < valid ? 8 : 0;
        const int gx = c.t0 * kT + r0, gy = c.t1 * kT + r0;
        const double* sx = X + (long long)gx * a.ldx + p + pc;
        const double* sy = a.y + (long long)gy * a.ldy + p + pc;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const bool vx = gx + 16 * q < a.nx, vy = gy + 16 * q < a.ny;
          cp_async_zfill8(rx + (r0 + 16 * q) * kRawStride + pc, vx ? sx + q * 16 * a.ldx : X, vx ? bytes_in : 0);
          cp_async_zfill8(ry + (r0 + 16 * q) * kRawStride + pc, vy ? sy + q * 16 * a.ldy : a.y, vy ? bytes_in : 0);
        }
      }
    } else {
      // x: rows k0..k0+15 of the transposed, pre-rounded T, 128 entries each (16-byte pieces)
      T* rx = reinterpret_cast<T*>(rawx + (size_t)slot * kT * kRawStride);
      const T* Xt = reinterpret_cast<const T*>(a.x);
      const long long k0 = (long long)c.ks * kBK;
      constexpr int EPP = 16 / sizeof(T);     // entries per piece
      constexpr int PPR = kT / EPP;           // pieces per row
      constexpr int PPT = kBK * PPR / kThreads;
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int e = tid + q * kThreads;
        const int kk = e / PPR, pc = e % PPR;
        const int m = c.t0 * kT + pc * EPP;
        const int left = a.nx - m;
        const int bytes_in = (k0 + kk < a.K && left > 0) ? min(left, EPP) * (int)sizeof(T) : 0;
        const T* src = bytes_in ? Xt + (k0 + kk) * a.ldx + m : Xt;
        cp_async_zfill16(rx + kk * kT + pc * EPP, src, bytes_in);
      }
      // y: grid rows [16][128]
      double* ry = rawy + (size_t)slot * kBK * kT;
      const long long p0 = (long long)c.t1 * kT;
      if (VEC16) {
#pragma unroll
        for (int q = 0; q < (kBK * 64) / kThreads; ++q) {
          const int e = tid + q * kThreads;
          const int kk = e >> 6, pc = e & 63;
          const long long gk = k0 + kk;
          const long long left = a.N - (p0 + 2 * pc);
          const int bytes_in = gk < a.K ? (left >= 2 ? 16 : (left == 1 ? 8 : 0)) : 0;
          const double* src = a.y + (bytes_in ? gk * a.ldy + p0 + 2 * pc : 0);
          cp_async_zfill16(ry + kk * kT + 2 * pc, src, bytes_in);
        }
      } else {
#pragma unroll 4
        for (int q = 0; q < (kBK * kT) / kThreads; ++q) {
          const int e = tid + q * kThreads;
          const int kk = e >> 7, pc = e & 127;
          const long long gk = k0 + kk;
          const int bytes_in = (gk < a.K && p0 + pc < a.N) ? 8 : 0;
          const double* src = a.y + (bytes_in ? gk * a.ldy + p0 + pc : 0);
          cp_async_zfill8(ry + kk * kT + pc, src, bytes_in);
        }
      }
    }
  };

  // ring slot `slot` -> compute buffer `buf` (rounded to T)
  auto convert = [&](int slot, int buf) {
    T* ox = cx + buf * kBK * kT;
    T* oy = cy + buf * kBK * kT;
    if (FORM == kFormGram) {
      // transpose [128][16] -> [16][128]: thread (row, half) reads 8 consecutive doubles
      const int row = tid & (kT - 1), half = tid >> 7;
      const double* srcx = rawx + (size_t)slot * kT * kRawStride + row * kRawStride + half * 8;
      const double* srcy = rawy + (size_t)slot * kT * kRawStride + row * kRawStride + half * 8;
#pragma unroll
      for (int j = 0; j < 8; j += 2) {
        const double2 u = *reinterpret_cast<const double2*>(srcx + j);
        const double2 v = *reinterpret_cast<const double2*>(srcy + j);
        ox[(half * 8 + j) * kT + row] = to_compute<T>(ABS ? fabs(u.x) : u.x);
        ox[(half * 8 + j + 1) * kT + row] = to_compute<T>(ABS ? fabs(u.y) : u.y);
        oy[(half * 8 + j) * kT + row] = to_compute<T>(ABS ? fabs(v.x) : v.x);
        oy[(half * 8 + j + 1) * kT + row] = to_compute<T>(ABS ? fabs(v.y) : v.y);
      }
    } else {
      // x is already in compute layout: a 16-byte copy
      const uint4* srcx = reinterpret_cast<const uint4*>(rawx + (size_t)slot * kT * kRawStride);
      uint4* dstx = reinterpret_cast<uint4*>(ox);
      constexpr int NV = kBK * kT * (int)sizeof(T) / 16;
#pragma unroll
      for (int q = 0; q < NV / kThreads; ++q) dstx[tid + q * kThreads] = srcx[tid + q * kThreads];
      // y: [16][128] doubles -> T, thread (p, half) converts 8 rows of one column
      const double* ry = rawy + (size_t)slot * kBK * kT;
      const int p = tid & (kT - 1), half = tid >> 7;
#pragma unroll
      for (int j = 0; j < 8; ++j) oy[(half * 8 + j) * kT + p] = to_compute<T>(ry[(half * 8 + j) * kT + p]);
    }
  };

  T acc[8][8];
  T acc2[8][8];  // FP32: sum of the inner partial sums
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) { acc[i][j] = T(0); acc2[i][j] = T(0); }

  auto fold = [&]() {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) { acc2[i][j] += acc[i][j]; acc[i][j] = T(0); }
  };

  auto store = [&](const Cursor& c) {
    if (FORM == kFormGram) {
      const int s = (int)(c.p0 / a.chunk);
      double* out = a.out + (size_t)s * a.nx * a.ny;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int ga = c.t0 * kT + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (ga >= a.nx) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int gb = c.t1 * kT + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
          if (gb < a.ny) out[(size_t)ga * a.ny + gb] = to_double<T>(acc2[i][j] + acc[i][j]);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int gm = c.t0 * kT + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
        if (gm >= a.nx) continue;
        double* orow = a.out + (size_t)gm * a.ldo;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const long long p = (long long)c.t1 * kT + h * 64 + tx * 4;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (p + j >= a.N) break;
            double v = to_double<T>(acc2[i][h * 4 + j] + acc[i][h * 4 + j]);
            if (a.accumulate) v += orow[p + j];
            orow[p + j] = v;
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) { acc[i][j] = T(0); acc2[i][j] = T(0); }
  };

  Cursor cmp;
  cmp.job = (int)blockIdx.x;
  decode(cmp);
  if (cmp.job >= a.njobs) return;
  // stages of this block over all its jobs
  int total = 0;
  {
    Cursor t;
    t.job = cmp.job;
    decode(t);
    while (t.job < a.njobs) {
      total += t.nst;
      t.job += gridDim.x;
      decode(t);
    }
  }
  Cursor ld = cmp;

  // prologue: stages 0 .. kStages-2 in flight, stage 0 converted, stage kStages-1 in flight
#pragma unroll
  for (int s = 0; s < kStages - 1; ++s) {
    issue(ld, s);
    cp_async_commit();
    next(ld);
  }
  cp_async_wait<kStages - 2>();
  __syncthreads();
  convert(0, 0);
  issue(ld, kStages - 1);
  cp_async_commit();
  next(ld);

  for (int it = 0; it < total; ++it) {
    cp_async_wait<kStages - 2>();  // stage it+1 landed (this thread's copies)
    __syncthreads();               // ... everyone's; buffer (it+1)&1 and slot it%kStages free
    if (it + 1 < total) convert((it + 1) % kStages, (it + 1) & 1);
    issue(ld, it % kStages);
    cp_async_commit();
    next(ld);

    const T* bx = cx + (it & 1) * kBK * kT;
    const T* by = cy + (it & 1) * kBK * kT;
#pragma unroll
    for (int k = 0; k < kBK; ++k) {
      T xa[8], yb[8];
      Vec4<T>::load(bx + k * kT + ty * 4, xa);
      Vec4<T>::load(bx + k * kT + 64 + ty * 4, xa + 4);
      Vec4<T>::load(by + k * kT + tx * 4, yb);
      Vec4<T>::load(by + k * kT + 64 + tx * 4, yb + 4);
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fma(xa[i], yb[j], acc[i][j]);
    }
    const bool last = cmp.ks + 1 >= cmp.nst;
    if (sizeof(T) == 4 && ((cmp.ks + 1) % kSubStages == 0) && !last) fold();
    if (last) store(cmp);
    next(cmp);
  }
  cp_async_wait<0>();
}

}  // namespace ace
}  // namespace hfx

namespace hfx {
namespace ace {

// ------------------------------------------------------------------------------------
// fixed-order sum of the split partials: lane -> output element, warp w -> splits w, w+8, ...
// Writes scale * sum to out[a][b] (FP64, row stride ldo) and/or to the transposed, rounded
// copy outt[b][a] (compute type, row stride ldt) that the left multiply reads.
// ------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_gram_reduce(const double* __restrict__ part, int splits, int nx, int ny,
                                                     double scale, double* __restrict__ out, long long ldo,
                                                     T* __restrict__ outt, long long ldt) {
  __shared__ double red[8][33];
  const long long total = (long long)nx * ny;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long idx = (long long)blockIdx.x * 32 + lane;
  double s0 = 0.0, s1 = 0.0;
  if (idx < total) {
    int s = w;
    for (; s + 8 < splits; s += 16) {
      s0 += part[(long long)s * total + idx];
      s1 += part[(long long)(s + 8) * total + idx];
    }
    if (s < splits) s0 += part[(long long)s * total + idx];
  }
  red[w][lane] = s0 + s1;
  __syncthreads();
  if (w == 0 && idx < total) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) t += red[q][lane];
    t *= scale;
    const long long a = idx / ny, b = idx % ny;
    if (out) out[a * ldo + b] = t;
    if (outt) outt[b * ldt + a] = to_compute<T>(t);
  }
}

// ------------------------------------------------------------------------------------
// Cholesky factor of A = -(M + M^T)/2, right-looking, one block; A in shared memory when it
// fits, else in `gwork`.  Step k: one thread takes the pivot's square root and reciprocals,
// then column k of L and the rank-one update of the trailing lower triangle (which never
// writes column k).
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_cholesky(const double* __restrict__ m, long long ldm, int n,
                                                   double* __restrict__ l, double* gwork, int use_smem, int* err) {
  extern __shared__ __align__(16) double sw[];  // [n][n] lower triangle of A (when it fits), then col[n]
  __shared__ double piv[2];
  __shared__ int bad;
  double* A = use_smem ? sw : gwork;
  double* col = use_smem ? sw + (size_t)n * n : gwork + (size_t)n * n;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const int nthr = blockDim.x * blockDim.y;
  if (tid == 0) bad = 0;
  for (long long idx = tid; idx < (long long)n * n; idx += nthr) {
    const int i = (int)(idx / n), j = (int)(idx % n);
    if (j <= i) A[idx] = -0.5 * (m[(long long)i * ldm + j] + m[(long long)j * ldm + i]);
    else l[idx] = 0.0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    // column k of the updated A into a vector (read along rows of A: one pass per step)
    for (int i = k + tid; i < n; i += nthr) col[i] = A[(long long)i * n + k];
    if (tid == 0) {
      const double d = A[(long long)k * n + k];
      if (!(d > 0.0)) bad = 1;
      const double r = rsqrt(d);
      piv[0] = r;      // column scale 1/sqrt(d)
      piv[1] = r * r;  // update scale 1/d
    }
    __syncthreads();
    const double inv_sd = piv[0], inv_d = piv[1];
    for (int i = k + tid; i < n; i += nthr) l[(long long)i * n + k] = col[i] * inv_sd;
    for (int i = k + 1 + threadIdx.y; i < n; i += blockDim.y) {
      const double aik = col[i] * inv_d;
      for (int j = k + 1 + threadIdx.x; j <= i; j += 32) A[(long long)i * n + j] -= aik * col[j];
    }
    __syncthreads();
  }
  if (tid == 0 && bad) atomicOr(err, kErrNotPosDef);
}

// The same factorisation spread over a cluster of kCholCluster CTAs, one per SM, so that the
// trailing updates use the FP64 pipes of eight SMs.  CTA r keeps rows i = r + kCholCluster q of
// the lower triangle in shared memory.  Step k reads column k of the updated A and the pivot's
// reciprocal square root from a double-buffered column buffer that every CTA holds; whoever
// updates A[i][k+1] during step k writes it straight into every CTA's next buffer (distributed
// shared memory), the thread that updates the diagonal element A[k+1][k+1] adds 1/sqrt(d) and
// 1/d, and one cluster barrier per step orders those writes before their use.
constexpr int kCholCluster = 8;
constexpr int kCholThreads = 512;
constexpr int kCholMaxN = 256;
constexpr size_t kCholSmemOneCta = 120 * 1024;  // more than half an SM: one CTA of the cluster per SM

__global__ void __cluster_dims__(kCholCluster, 1, 1) __launch_bounds__(kCholThreads, 1)
    k_cholesky_cluster(const double* __restrict__ m, long long ldm, int n, double* __restrict__ l, int* err) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  constexpr int C = kCholCluster;
  const int rank = (int)cluster.block_rank();
  const int rows_max = (n + C - 1) / C;
  const int rows = (n - rank + C - 1) / C;  // local rows q: global row i = rank + C q
  extern __shared__ __align__(16) double sc[];
  double* A = sc;                                    // [rows_max][n], row q holds columns 0..i
  double* colbuf = sc + (size_t)rows_max * n;        // [2][n + 2]: column entries, 1/sqrt(d), 1/d
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int NW = kCholThreads / 32;

  // write value v as entry e of column buffer b in every CTA of the cluster
  auto bcast = [&](int b, int e, double v) {
#pragma unroll
    for (int r = 0; r < C; ++r) cluster.map_shared_rank(colbuf, r)[(size_t)b * (n + 2) + e] = v;
  };
  auto pivot = [&](int b, double d) {
    if (!(d > 0.0)) atomicOr(err, kErrNotPosDef);
    const double r = rsqrt(d);
    bcast(b, n, r);
    bcast(b, n + 1, r * r);
  };

  for (int idx = threadIdx.x; idx < rows * n; idx += kCholThreads) {
    const int q = idx / n, j = idx % n, i = rank + C * q;
    if (j <= i) A[(size_t)q * n + j] = -0.5 * (m[(long long)i * ldm + j] + m[(long long)j * ldm + i]);
    else l[(long long)i * n + j] = 0.0;
  }
  __syncthreads();
  // column 0 and the first pivot
  for (int q = w; q < rows; q += NW) {
    if (lane != 0) continue;
    const int i = rank + C * q;
    const double v = A[(size_t)q * n];
    bcast(0, i, v);
    if (i == 0) pivot(0, v);
  }
  cluster.sync();

  for (int k = 0; k < n; ++k) {
    const double* cb = colbuf + (size_t)(k & 1) * (n + 2);
    const int nb = (k + 1) & 1;
    const double inv_sd = cb[n], inv_d = cb[n + 1];
    for (int q = w; q < rows; q += NW) {
      const int i = rank + C * q;
      if (i < k) continue;
      double* row = A + (size_t)q * n;
      const double aik = row[k];
      if (lane == 0) l[(long long)i * n + k] = aik * inv_sd;
      if (i == k) continue;
      const double s = aik * inv_d;
      for (int j = k + 1 + lane; j <= i; j += 32) {
        const double v = row[j] - s * cb[j];
        row[j] = v;
        if (j == k + 1) {  // column k+1 of the updated A, and the next pivot
          bcast(nb, i, v);
          if (i == k + 1) pivot(nb, v);
        }
      }
    }
    cluster.sync();
  }
}

// ------------------------------------------------------------------------------------
// L^-1 by forward substitution, one block per column j; L's rows j..n-1 are staged in shared
// memory when they fit.  Column j of L^-1 is row j of the transposed output linvt (compute
// type, row stride ldt), which the left multiply reads as its small operand.
// ------------------------------------------------------------------------------------
template <bool SMEM_L, typename T>
__global__ void __launch_bounds__(128) k_tri_inverse(const double* __restrict__ l, int n, T* __restrict__ linvt,
                                                     long long ldt) {
  extern __shared__ __align__(16) double sm[];
  double* x = sm;            // [n]
  double* dinv = sm + n;     // [n] reciprocal diagonal
  double* Ls = sm + 2 * n;   // [n][n] when staged
  const int j = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    x[i] = (i == j) ? 1.0 : 0.0;
    if (i >= j) dinv[i] = 1.0 / l[(long long)i * n + i];
  }
  if (SMEM_L)
    for (long long idx = (long long)j * n + threadIdx.x; idx < (long long)n * n; idx += blockDim.x) Ls[idx] = l[idx];
  const double* L = SMEM_L ? Ls : l;
  __syncthreads();
  T* row = linvt + (long long)j * ldt;
  for (int k = j; k < n; ++k) {
    const double xk = x[k] * dinv[k];
    if (threadIdx.x == 0) row[k] = to_compute<T>(xk);
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) x[i] -= L[(long long)i * n + k] * xk;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < j; i += blockDim.x) row[i] = T(0);
}

// ------------------------------------------------------------------------------------
// screen compaction
// ------------------------------------------------------------------------------------
__device__ __forceinline__ bool keep_pair(const double* s, int n, int i, int j, double cut) {
  return j == i || s[(long long)i * n + j] > cut;
}

__global__ void __launch_bounds__(256) k_screen_count(const double* __restrict__ s, int n, double cut, int* rowbuf) {
  __shared__ int part[8];
  const int i = blockIdx.x;
  int c = 0;
  for (int j = i + threadIdx.x; j < n; j += blockDim.x) c += keep_pair(s, n, i, j, cut) ? 1 : 0;
#pragma unroll
  for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int q = 0; q < 8; ++q) t += part[q];
    rowbuf[i] = t;
  }
}

// exclusive scan of the n row counts in place (rowbuf[n] = total), one block of 1024
__global__ void __launch_bounds__(1024) k_screen_scan(int* rowbuf, int n, int64_t* n_pairs) {
  __shared__ long long sums[1024];
  const int per = (n + 1023) / 1024;
  const int b = threadIdx.x * per, e = min(n, b + per);
  long long loc = 0;
  for (int i = b; i < e; ++i) loc += rowbuf[i];
  sums[threadIdx.x] = loc;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const long long v = threadIdx.x >= o ? sums[threadIdx.x - o] : 0;
    __syncthreads();
    sums[threadIdx.x] += v;
    __syncthreads();
  }
  long long run = sums[threadIdx.x] - loc;
  for (int i = b; i < e; ++i) {
    const int c = rowbuf[i];
    rowbuf[i] = (int)run;
    run += c;
  }
  if (threadIdx.x == 1023) {
    rowbuf[n] = (int)sums[1023];
    *n_pairs = sums[1023];
  }
}

__global__ void __launch_bounds__(256) k_screen_write(const double* __restrict__ s, int n, double cut,
                                                      const int* __restrict__ rowbuf, int32_t* pairs) {
  __shared__ int wsum[8];
  const int i = blockIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int base = rowbuf[i];
  for (int j0 = i; j0 < n; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    const bool k = j < n && keep_pair(s, n, i, j, cut);
    const unsigned bal = __ballot_sync(0xffffffffu, k);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      off += q < w ? wsum[q] : 0;
      tot += wsum[q];
    }
    if (k) {
      const int pos = base + off + __popc(bal & ((1u << lane) - 1u));
      pairs[2 * (long long)pos] = i;
      pairs[2 * (long long)pos + 1] = j;
    }
    base += tot;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
GramPlan gram_plan(int nx, int ny, long long K, int sm_count) {
  GramPlan p;
  p.tiles_x = (nx + kT - 1) / kT;
  p.tiles_y = (ny + kT - 1) / kT;
  const int tiles = p.tiles_x * p.tiles_y;
  const long long want = std::max(1LL, (2LL * sm_count + tiles - 1) / tiles);
  long long chunk = (K + want - 1) / want;
  chunk = std::max<long long>(kBK, (chunk + kBK - 1) / kBK * kBK);
  p.chunk = chunk;
  p.splits = (int)((K + chunk - 1) / chunk);
  p.njobs = p.splits * tiles;
  return p;
}

size_t gram_partial_bytes(const GramPlan& p, int nx, int ny) { return (size_t)p.splits * nx * ny * sizeof(double); }

template <typename T, int FORM, bool VEC16, bool ABS>
static cudaError_t launch_mm(const MmArgs& a, int sm_count, cudaStream_t st) {
  const size_t ybytes = FORM == kFormGram ? kRawRowsBytes : kRawColsBytes;
  const size_t smem = kStages * (kRawRowsBytes + ybytes) + 4 * size_t(kBK) * kT * sizeof(T);
  const cudaError_t e =
      cudaFuncSetAttribute(k_ace_mm<T, FORM, VEC16, ABS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = std::min(a.njobs, sm_count);
  k_ace_mm<T, FORM, VEC16, ABS><<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

cudaError_t gram(bool fp32, bool absval, const double* x, long long ldx, int nx, const double* y, long long ldy,
                 int ny, long long K, const GramPlan& plan, double* partials, int sm_count, cudaStream_t st) {
  MmArgs a{};
  a.x = x; a.y = y; a.out = partials;
  a.K = K; a.ldx = ldx; a.ldy = ldy; a.ldo = 0;
  a.nx = nx; a.ny = ny; a.N = 0;
  a.chunk = plan.chunk;
  a.tiles_x = plan.tiles_x; a.tiles_y = plan.tiles_y; a.njobs = plan.njobs;
  a.lower = 0; a.accumulate = 0;
  const bool v16 = (ldx % 2 == 0) && (ldy % 2 == 0) && aligned16(x) && aligned16(y);
#define HFX_ACE_GRAM(TT, V, AB) return launch_mm<TT, kFormGram, V, AB>(a, sm_count, st)
  if (fp32) {
    if (v16) { if (absval) HFX_ACE_GRAM(float, true, true); else HFX_ACE_GRAM(float, true, false); }
    else { if (absval) HFX_ACE_GRAM(float, false, true); else HFX_ACE_GRAM(float, false, false); }
  } else {
    if (v16) { if (absval) HFX_ACE_GRAM(double, true, true); else HFX_ACE_GRAM(double, true, false); }
    else { if (absval) HFX_ACE_GRAM(double, false, true); else HFX_ACE_GRAM(double, false, false); }
  }
#undef HFX_ACE_GRAM
}

// m <- (m + m^T) / 2 in place (exact when m is already symmetric): a symmetric quantity whose two
// halves were summed in different orders (split tensor-core products) becomes exactly symmetric
__global__ void k_symmetrise(double* __restrict__ m, int n, long long ld) {
  const long long total = (long long)n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(i / n), b = (int)(i % n);
    if (a >= b) continue;
    const double v = 0.5 * (m[(long long)a * ld + b] + m[(long long)b * ld + a]);
    m[(long long)a * ld + b] = v;
    m[(long long)b * ld + a] = v;
  }
}

cudaError_t symmetrise(double* m, int n, long long ld, cudaStream_t st) {
  const long long total = (long long)n * n;
  const int grid = (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 1024));
  k_symmetrise<<<grid, 256, 0, st>>>(m, n, ld);
  return cudaGetLastError();
}

cudaError_t gram_reduce(bool fp32, const double* partials, int splits, int nx, int ny, double scale, double* out,
                        long long ldo, void* outt, long long ldt, cudaStream_t st) {
  const long long total = (long long)nx * ny;
  const int grid = (int)((total + 31) / 32);
  if (fp32)
    k_gram_reduce<float><<<grid, 256, 0, st>>>(partials, splits, nx, ny, scale, out, ldo, (float*)outt, ldt);
  else
    k_gram_reduce<double><<<grid, 256, 0, st>>>(partials, splits, nx, ny, scale, out, ldo, (double*)outt, ldt);
  return cudaGetLastError();
}

long long lmul_ldt(bool fp32, int m) { return fp32 ? (m + 3) / 4 * 4 : (m + 1) / 2 * 2; }

cudaError_t lmul(bool fp32, const void* tt, long long ldt, int m, int k, bool lower, const double* y, long long ldy,
                 long long n, bool accumulate, double* out, long long ldo, int sm_count, cudaStream_t st) {
  MmArgs a{};
  a.x = tt; a.y = y; a.out = out;
  a.K = k; a.ldx = ldt; a.ldy = ldy; a.ldo = ldo;
  a.nx = m; a.ny = 0; a.N = n;
  a.chunk = 0;
  a.tiles_x = (m + kT - 1) / kT;
  a.tiles_y = (int)((n + kT - 1) / kT);
  a.njobs = a.tiles_x * a.tiles_y;
  a.lower = lower ? 1 : 0; a.accumulate = accumulate ? 1 : 0;
  const bool v16 = (ldy % 2 == 0) && aligned16(y);
  if (fp32) {
    if (v16) return launch_mm<float, kFormLmul, true, false>(a, sm_count, st);
    return launch_mm<float, kFormLmul, false, false>(a, sm_count, st);
  }
  if (v16) return launch_mm<double, kFormLmul, true, false>(a, sm_count, st);
  return launch_mm<double, kFormLmul, false, false>(a, sm_count, st);
}

cudaError_t cholesky_neg_sym(const double* m, long long ldm, int n, double* l, double* work, int* err, int max_smem,
                             cudaStream_t st) {
  if (n <= kCholMaxN) {
    const size_t need = ((size_t)((n + kCholCluster - 1) / kCholCluster) * n + 2 * (n + 2)) * sizeof(double);
    const size_t smem = std::max(need, kCholSmemOneCta);
    if (smem + 1024 <= (size_t)max_smem) {
      const cudaError_t e =
          cudaFuncSetAttribute(k_cholesky_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_cholesky_cluster<<<kCholCluster, kCholThreads, smem, st>>>(m, ldm, n, l, err);
      return cudaGetLastError();
    }
  }
  const size_t need = ((size_t)n * n + n) * sizeof(double);
  const bool use_smem = need + 64 <= (size_t)max_smem;
  if (use_smem) {
    const cudaError_t e = cudaFuncSetAttribute(k_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    if (e != cudaSuccess) return e;
  }
  k_cholesky<<<1, dim3(32, 32), use_smem ? need : 0, st>>>(m, ldm, n, l, work, use_smem ? 1 : 0, err);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t tri_inverse_t(const double* l, int n, T* linvt, long long ldt, int max_smem, cudaStream_t st) {
  const size_t full = ((size_t)n * n + 2 * n) * sizeof(double);
  if (full <= (size_t)max_smem) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_tri_inverse<true, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)full);
    if (e != cudaSuccess) return e;
    k_tri_inverse<true, T><<<n, 128, full, st>>>(l, n, linvt, ldt);
  } else {
    k_tri_inverse<false, T><<<n, 128, 2 * n * sizeof(double), st>>>(l, n, linvt, ldt);
  }
  return cudaGetLastError();
}

cudaError_t tri_inverse(bool fp32, const double* l, int n, void* linvt, long long ldt, int max_smem, cudaStream_t st) {
  return fp32 ? tri_inverse_t(l, n, (float*)linvt, ldt, max_smem, st)
              : tri_inverse_t(l, n, (double*)linvt, ldt, max_smem, st);
}

cudaError_t screen_compact(const double* s, int n, double cut, int32_t* pairs, int64_t* n_pairs, int* rowbuf,
                           cudaStream_t st) {
  k_screen_count<<<n, 256, 0, st>>>(s, n, cut, rowbuf);
  k_screen_scan<<<1, 1024, 0, st>>>(rowbuf, n, n_pairs);
  k_screen_write<<<n, 256, 0, st>>>(s, n, cut, rowbuf, pairs);
  return cudaGetLastError();
}

}  // namespace ace
}  // namespace hfx
