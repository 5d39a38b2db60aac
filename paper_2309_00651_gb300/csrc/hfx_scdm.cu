// SCDM localisation on the GPU (the selected-columns-of-the-density-matrix method that the
// paper's localised-orbital variant uses, Sec. 2.1; the algorithm follows the published method):
// a column-pivoted QR factorisation of Psi^T by greedy residual-norm pivoting picks n grid points,
// and the localised orthonormal orbitals are Phi = Psi Q with q_j the Gram-Schmidt vectors of the
// picked columns.
//
// Per step j (two launches, stream ordered):
//   k_scdm_pick   (one block)  the grid point p_j of largest residual norm (from the per-block
//                              maxima of the previous launch, lowest index on a tie); its column
//                              a = Psi^T[:, p_j] orthogonalised twice against q_0..q_{j-1}
//                              (classical Gram-Schmidt with one re-orthogonalisation), q_j = r/|r|.
//   k_scdm_update (grid)       c_p = q_j . Psi^T[:, p] for every grid point, nu_p -= c_p^2, and the
//                              per-block maxima of nu for the next pick.
// Both run in the context's precision (FP32: the orbitals rounded once to an FP32 copy in the
// workspace, FP32 dot products, FP64 residual norms; FP64: FP64 throughout).  The last step is
// followed by the left multiply Phi = Q^T Psi of hfx_ace.cu.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "hfx_ace_internal.h"

namespace hfx {
namespace ace {

namespace {

constexpr int kUpdThreads = 256;
constexpr int kUpdPoints = 4;  // grid points per thread per sweep (independent dot products)
constexpr int kUpdBlocksPerSm = 3;  // resident update blocks per SM at its launch bounds

template <typename T>
__device__ __forceinline__ T round_to(double v);
template <>
__device__ __forceinline__ float round_to<float>(double v) { return __double2float_rn(v); }
template <>
__device__ __forceinline__ double round_to<double>(double v) { return v; }

// (value, index) maximum with the lowest index on a tie
__device__ __forceinline__ void take_max(double& v, long long& i, double v2, long long i2) {
  if (v2 > v || (v2 == v && i2 < i)) { v = v2; i = i2; }
}

__device__ __forceinline__ void block_argmax(double& v, long long& i, double* sv, long long* si) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
    take_max(v, i, v2, i2);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) { sv[w] = v; si[w] = i; }
  __syncthreads();
  if (w == 0) {
    v = lane < nw ? sv[lane] : -2.0;
    i = lane < nw ? si[lane] : (long long)1 << 62;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
      const long long i2 = __shfl_xor_sync(0xffffffffu, i, o);
      take_max(v, i, v2, i2);
    }
  }
}

// sum of v over threads 0..n-1 (one element each, n <= blockDim.x), returned to every thread;
// the FP64 adds run in the warps that hold data and in one thread, not in the whole block (the
// FP64 pipe of this part is narrow)
__device__ __forceinline__ double sum_first_n(double v, int n, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = (n + 31) >> 5;
  __syncthreads();  // red may still be read from an earlier call
  if (w < nw) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[w] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += red[q];
    red[32] = t;
  }
  __syncthreads();
  return red[32];
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

}  // namespace

// residual norms nu_p = |Psi^T[:, p]|^2 (in the compute type, widened), the FP32 copy of the
// orbitals when T = float, and the per-block maxima
template <typename T>
__global__ void __launch_bounds__(kUpdThreads) k_scdm_init(const double* __restrict__ psi, long long N, int n,
                                                           T* __restrict__ a32, double* __restrict__ nu,
                                                           double* __restrict__ bmax, long long* __restrict__ bidx) {
  __shared__ double sv[32];
  __shared__ long long si[32];
  double best = -2.0;
  long long bi = (long long)1 << 62;
  for (long long p = (long long)blockIdx.x * kUpdThreads + threadIdx.x; p < N; p += (long long)gridDim.x * kUpdThreads) {
    T acc = T(0);
    for (int i = 0; i < n; ++i) {
      const T v = round_to<T>(psi[(long long)i * N + p]);
      if (a32) a32[(long long)i * N + p] = v;
      acc = fma(v, v, acc);
    }
    const double x = (double)acc;
    nu[p] = x;
    take_max(best, bi, x, p);
  }
  block_argmax(best, bi, sv, si);
  if (threadIdx.x == 0) { bmax[blockIdx.x] = best; bidx[blockIdx.x] = bi; }
}

// step j: pick p_j and form q_j (one block of kPickThreads threads; dynamic shared memory holds
// a[n], h[n] and the per-warp partial sums hp[32][n], all in T, and with QS a copy of
// q_0..q_{j-1} at the row stride of qt).  The kernel is a chain of short phases, so each phase
// issues all of its global loads before it uses any of them: the argmax reads at most two
// per-block maxima per thread, and the Gram-Schmidt products read up to kPickChunks x kPickRows
// entries of Q per lane at once -- from shared memory when QS, where the copy of Q is started
// before the argmax (Q does not depend on the pick) and lands while the argmax and the column
// load wait on memory.
constexpr int kPickThreads = 1024;
constexpr int kPickChunks = 4;  // 32-column chunks of Q a lane holds in flight (128 columns)
constexpr int kPickRows = 4;    // rows of Q a warp takes at once in a -= Q h
constexpr size_t kPickSmemBudget = 200 * 1024;  // shared memory for the QS variant
template <typename T, bool QS>
__global__ void __launch_bounds__(kPickThreads, 1) k_scdm_pick(const double* __restrict__ psi, long long N, int n, int j,
                                                            const double* __restrict__ bmax,
                                                            const long long* __restrict__ bidx, int nb,
                                                            long long* __restrict__ piv, T* __restrict__ qt,
                                                            double* __restrict__ q64, long long ldt,
                                                            double* __restrict__ rdiag, int* err) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* a = reinterpret_cast<T*>(smem);  // [n]
  T* h = a + n;                       // [n]
  T* hp = h + n;                      // [32][n]
  __shared__ double red[33];
  __shared__ double scal[2];
  __shared__ double sv[32];
  __shared__ long long si[32];
  __shared__ long long pick;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int nw = kPickThreads / 32;
  // Q's rows (16-byte aligned: ldt is a multiple of 16 bytes), columns 0 .. j-1 rounded up to
  // whole 16-byte pieces, which stay inside the row
  T* qs = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(hp + 32 * n) + 15) & ~uintptr_t(15));
  const T* Q = QS ? qs : qt;
  if (QS && j > 0) {
    constexpr int EPC = 16 / (int)sizeof(T);
    const int cpr = (j + EPC - 1) / EPC;
    for (int c = threadIdx.x; c < n * cpr; c += kPickThreads) {
      const int i = c / cpr, kc = c - i * cpr;
      cp_async16(qs + (long long)i * ldt + kc * EPC, qt + (long long)i * ldt + kc * EPC);
    }
  }
  {  // argmax over the per-block maxima (lowest index on a tie), the whole block
    double best = -2.0;
    long long bi = (long long)1 << 62;
    for (int b = threadIdx.x; b < nb; b += kPickThreads) take_max(best, bi, bmax[b], bidx[b]);
    block_argmax(best, bi, sv, si);
    if (threadIdx.x == 0) {
      const bool ok = best > 0.0 && bi < N;
      if (!ok) atomicOr(err, kErrRankDeficient);
      pick = ok ? bi : 0;
      piv[j] = pick;
    }
  }
  __syncthreads();
  const long long p = pick;
  double sa = 0.0;
  if (threadIdx.x < n) {
    a[threadIdx.x] = round_to<T>(psi[(long long)threadIdx.x * N + p]);
    sa = (double)a[threadIdx.x] * (double)a[threadIdx.x];
  }
  if (QS) cp_async_wait_all();  // this thread's pieces of Q; the barriers below publish them
  const double an2 = sum_first_n(sa, n, red);
  // two passes of classical Gram-Schmidt against q_0..q_{j-1} (Q[i][k] = q_k[i])
  for (int pass = 0; pass < 2; ++pass) {
    // h = Q^T a: warp w takes rows i = w, w + 32, ...; lane takes columns k = K0 + lane + 32 c
    for (int K0 = 0; K0 < j; K0 += 32 * kPickChunks) {
      T s[kPickChunks];
#pragma unroll
      for (int c = 0; c < kPickChunks; ++c) s[c] = T(0);
#pragma unroll 4
      for (int i = w; i < n; i += nw) {
        const T ai = a[i];
        const T* row = Q + (long long)i * ldt;
#pragma unroll
        for (int c = 0; c < kPickChunks; ++c) {
          const int k = K0 + lane + 32 * c;
          if (k < j) s[c] = fma(row[k], ai, s[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < kPickChunks; ++c) {
        const int k = K0 + lane + 32 * c;
        if (k < j) hp[w * n + k] = s[c];
      }
    }
    __syncthreads();
    // h[k] = sum over the 32 warp partials, eight threads per column
    for (int base = 0; base < j; base += kPickThreads / 8) {
      const int k = base + (threadIdx.x >> 3), part = threadIdx.x & 7;
      T s = T(0);
      if (k < j)
        for (int q = part; q < nw; q += 8) s += hp[q * n + k];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      s += __shfl_xor_sync(0xffffffffu, s, 4);
      if (k < j && part == 0) h[k] = s;
    }
    __syncthreads();
    // a -= Q h: warp w takes kPickRows rows at once (i = i0 + r * 32); lanes take columns
    for (int i0 = w; i0 < n; i0 += kPickRows * nw) {
      T s[kPickRows];
#pragma unroll
      for (int r = 0; r < kPickRows; ++r) s[r] = T(0);
      for (int K0 = 0; K0 < j; K0 += 32 * kPickChunks) {
#pragma unroll
        for (int c = 0; c < kPickChunks; ++c) {
          const int k = K0 + lane + 32 * c;
          if (k < j) {
            const T hk = h[k];
#pragma unroll
            for (int r = 0; r < kPickRows; ++r) {
              const int i = i0 + r * nw;
              if (i < n) s[r] = fma(Q[(long long)i * ldt + k], hk, s[r]);
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < kPickRows; ++r) {
        T t = s[r];
#pragma unroll
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        const int i = i0 + r * nw;
        if (lane == 0 && i < n) a[i] -= t;
      }
    }
    __syncthreads();
  }
  const double ss = threadIdx.x < n ? (double)a[threadIdx.x] * (double)a[threadIdx.x] : 0.0;
  const double rn2 = sum_first_n(ss, n, red);
  if (threadIdx.x == 0) {
    const double rn = sqrt(rn2);
    // the picked column lies in the span of q_0..q_{j-1} to working precision: no new direction
    const double floor_rel = 1e3 * (sizeof(T) == 4 ? 5.96e-8 : 1.11e-16);
    if (!(rn > floor_rel * sqrt(an2))) atomicOr(err, kErrRankDeficient);
    scal[0] = rn > 0.0 ? 1.0 / rn : 0.0;
    rdiag[j] = rn;
  }
  __syncthreads();
  const double inv = scal[0];
  if (threadIdx.x < n) {
    const double q = (double)a[threadIdx.x] * inv;
    qt[(long long)threadIdx.x * ldt + j] = round_to<T>(q);
    if (q64) q64[(long long)threadIdx.x * n + j] = q;
  }
}

// step j: c_p = q_j . Psi^T[:, p], nu_p -= c_p^2 (picked points stay at -1), per-block maxima;
// each thread takes kUpdPoints grid points, rows unrolled for loads in flight
template <typename T>
__global__ void __launch_bounds__(kUpdThreads, kUpdBlocksPerSm) k_scdm_update(const T* __restrict__ A, long long N, int n,
                                                             const T* __restrict__ qt, long long ldt, int j,
                                                             const long long* __restrict__ piv,
                                                             double* __restrict__ nu, double* __restrict__ bmax,
                                                             long long* __restrict__ bidx) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* q = reinterpret_cast<T*>(smem);  // [n]
  __shared__ double sv[32];
  __shared__ long long si[32];
  for (int i = threadIdx.x; i < n; i += blockDim.x) q[i] = qt[(long long)i * ldt + j];
  __syncthreads();
  const long long picked = piv[j];
  double best = -2.0;
  long long bi = (long long)1 << 62;
  // block b takes the contiguous run [b chunk, (b+1) chunk) of grid points (chunk a multiple of
  // 32), in sweeps of kUpdThreads x kUpdPoints points: every block gets the same share
  const long long chunk = ((N + gridDim.x - 1) / gridDim.x + 31) / 32 * 32;
  const long long b0 = (long long)blockIdx.x * chunk;
  const long long b1 = min(N, b0 + chunk);
  for (long long p0 = b0 + threadIdx.x; p0 < b1; p0 += (long long)kUpdThreads * kUpdPoints) {
    T c[kUpdPoints];
    bool in[kUpdPoints];
#pragma unroll
    for (int u = 0; u < kUpdPoints; ++u) {
      c[u] = T(0);
      in[u] = p0 + u * kUpdThreads < b1;
    }
#pragma unroll 8
    for (int i = 0; i < n; ++i) {
      const T qi = q[i];
      const T* row = A + (long long)i * N + p0;
#pragma unroll
      for (int u = 0; u < kUpdPoints; ++u)
        if (in[u]) c[u] = fma(qi, row[u * kUpdThreads], c[u]);
    }
#pragma unroll
    for (int u = 0; u < kUpdPoints; ++u) {
      const long long p = p0 + u * kUpdThreads;
      if (!in[u]) continue;
      const double old = nu[p];
      const double cc = (double)c[u];
      const double v = (old < 0.0 || p == picked) ? -1.0 : old - cc * cc;
      nu[p] = v;
      take_max(best, bi, v, p);
    }
  }
  block_argmax(best, bi, sv, si);
  if (threadIdx.x == 0) { bmax[blockIdx.x] = best; bidx[blockIdx.x] = bi; }
}

// blocks of the init / update launches: one wave of kUpdBlocksPerSm blocks on every SM (equal
// shares of the grid, so no SM runs a block more than the others), fewer for small grids (at
// least kUpdThreads points per block)
static int scdm_blocks(long long N, int sm_count) {
  const long long cover = (N + kUpdThreads - 1) / kUpdThreads;
  return (int)std::max(1LL, std::min<long long>(cover, (long long)sm_count * kUpdBlocksPerSm));
}

template <typename T>
static cudaError_t scdm_run(const double* psi, long long N, int n, T* a32, double* nu, double* bmax, long long* bidx,
                            long long* piv, T* qt, long long ldt, double* q64, double* rdiag, int* err, int sm_count,
                            cudaStream_t st) {
  const int nb = scdm_blocks(N, sm_count);
  const T* A = a32 ? a32 : reinterpret_cast<const T*>(psi);
  k_scdm_init<T><<<nb, kUpdThreads, 0, st>>>(psi, N, n, a32, nu, bmax, bidx);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t base_smem = 34 * (size_t)n * sizeof(T);
  const size_t qs_smem = base_smem + 16 + (size_t)n * ldt * sizeof(T);
  const bool qs = qs_smem <= kPickSmemBudget;
  const size_t pick_smem = qs ? qs_smem : base_smem;
  if (pick_smem > 48 * 1024) {
    e = qs ? cudaFuncSetAttribute(k_scdm_pick<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pick_smem)
           : cudaFuncSetAttribute(k_scdm_pick<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pick_smem);
    if (e != cudaSuccess) return e;
  }
  const size_t upd_smem = (size_t)n * sizeof(T);
  for (int j = 0; j < n; ++j) {
    if (qs)
      k_scdm_pick<T, true><<<1, kPickThreads, pick_smem, st>>>(psi, N, n, j, bmax, bidx, nb, piv, qt, q64, ldt, rdiag, err);
    else
      k_scdm_pick<T, false><<<1, kPickThreads, pick_smem, st>>>(psi, N, n, j, bmax, bidx, nb, piv, qt, q64, ldt, rdiag, err);
    if (j + 1 < n) k_scdm_update<T><<<nb, kUpdThreads, upd_smem, st>>>(A, N, n, qt, ldt, j, piv, nu, bmax, bidx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

size_t scdm_scratch_bytes(bool fp32, int n, long long N, int sm_count) {
  const int nb = scdm_blocks(N, sm_count);
  auto r = [](size_t b) { return (b + 255) / 256 * 256; };
  return r((size_t)N * sizeof(double)) + r(nb * sizeof(double)) + r(nb * sizeof(long long)) +
         r((size_t)n * sizeof(double)) + (fp32 ? r((size_t)n * N * sizeof(float)) : 0);
}

cudaError_t scdm_pivots_q(bool fp32, const double* psi, long long N, int n, void* scratch, long long* piv, void* qt,
                          long long ldt, double* q64, int* err, int sm_count, cudaStream_t st) {
  const int nb = scdm_blocks(N, sm_count);
  auto r = [](size_t b) { return (b + 255) / 256 * 256; };
  char* s = (char*)scratch;
  double* nu = (double*)s;
  s += r((size_t)N * sizeof(double));
  double* bmax = (double*)s;
  s += r(nb * sizeof(double));
  long long* bidx = (long long*)s;
  s += r(nb * sizeof(long long));
  double* rdiag = (double*)s;
  s += r((size_t)n * sizeof(double));
  if (fp32)
    return scdm_run<float>(psi, N, n, (float*)s, nu, bmax, bidx, piv, (float*)qt, ldt, q64, rdiag, err, sm_count, st);
  return scdm_run<double>(psi, N, n, nullptr, nu, bmax, bidx, piv, (double*)qt, ldt, q64, rdiag, err, sm_count, st);
}

}  // namespace ace
}  // namespace hfx
