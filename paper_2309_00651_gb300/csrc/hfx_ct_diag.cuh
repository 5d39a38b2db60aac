// Inverse-y / accumulate pass for full diagonal orbital-block pairs, compile-time geometry (FP32).
//
// A diagonal block pair (I == J, B orbitals) holds the B(B-1)/2 pairs a < b and the B pairs
// (a, a) of the block.  Its couples sit in the canonical layout of the pair staging: the
// off-diagonal pairs in the order t = a B - a(a+1)/2 + (b - a - 1), couple t/2, half t&1 (real part
// for even t), then the diagonal pairs, couple B(B-1)/4 + a/2, half a&1.  That layout is fixed,
// so the pair behind every half of every couple is known at compile time, and the whole block
// pair accumulates into B register accumulators per grid point:
//   v from the couple's half for pair (a, b):  V_a += v phi_b,  V_b += v phi_a   (a < b)
//                                              V_a += v phi_a                    (a == b)
// (Eq. vx with the pair potential v_ab of Eq. vij), with the V rows read and rewritten once per
// block pair in FP64.  The couple tiles stream through a cp.async ring and get their y-inverse
// stages in shared memory, as in the off-diagonal dense pass.
#pragma once
#include "hfx_ct.cuh"
#include "tma_sm100.cuh"
#include "hfx_internal.h"

namespace hfx {
namespace ct {

template <int B> struct DiagLayout {
  static constexpr int NOFF = B * (B - 1) / 2;
  static constexpr int NCPL = NOFF / 2 + B / 2;  // couples of the block pair
  static_assert(B % 2 == 0 && NOFF % 2 == 0, "full couples only (B a multiple of 4)");
  // orbitals (a, b), a <= b, local to the block, behind half h of couple c
  __host__ __device__ static constexpr int first(int c, int h) {
    if (c >= NOFF / 2) return 2 * (c - NOFF / 2) + h;
    int t = 2 * c + h, a = 0;
    while (t >= B - 1 - a) { t -= B - 1 - a; ++a; }
    return a;
  }
  __host__ __device__ static constexpr int second(int c, int h) {
    if (c >= NOFF / 2) return 2 * (c - NOFF / 2) + h;
    int t = 2 * c + h, a = 0;
    while (t >= B - 1 - a) { t -= B - 1 - a; ++a; }
    return a + 1 + t;
  }
};

template <typename T, int N, int B>
__global__ void __launch_bounds__(DenseGeo<T, N>::NT, DenseGeo<T, N>::MINB)
k_y_acc_diag_ct(const T* __restrict__ orb, long long Ntot, const int4* __restrict__ couples,
                const int* __restrict__ slot_list, const int* __restrict__ slot_couple_base,
                const int2* __restrict__ slot_blocks, int c0, const cx<T>* __restrict__ W,
                const cx<T>* __restrict__ twg, T* __restrict__ V, double vscale,
                const __grid_constant__ CUtensorMap tmV, int tma_flush) {
  using C = cx<T>;
  using G = DenseGeo<T, N>;
  using D = DiagLayout<B>;
  constexpr int ZC = G::ZC, PTS = G::PTS, NP = G::NP, NT = G::NT;
  constexpr int CPI = kDiagCouplesPerItCt;
  constexpr int ITERS = D::NCPL / CPI;
  static_assert(D::NCPL % CPI == 0, "couples per iteration must divide the block pair's couples");
  static_assert(D::NCPL <= 32, "one mask word per block pair");
  constexpr int RING = kDenseRingCt;
  constexpr int LN = CPI * ZC;  // lines of the interleaved tile [y][u][zz]
  constexpr int PER = 16 / int(sizeof(C));
  constexpr int PLANE = N * N;
  constexpr StagePlan P = Plan<N>::p;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int z0 = blockIdx.x * ZC;
  const int zcn = min(ZC, N - z0);
  const int x = blockIdx.y;
  const int slot = slot_list[blockIdx.z];
  static_assert((RING * N * LN * sizeof(C)) % 128 == 0, "the staging tile starts on a 128-byte boundary");
  unsigned char* base = smem_raw + ((128u - (tc::smem_u32(smem_raw) & 127u)) & 127u);
  C* tiles = reinterpret_cast<C*>(base);  // RING x [N][LN]
  // [B][PTS] staging of the block's orbitals; at the end, of the scaled V_x phi sums
  T* phis = reinterpret_cast<T*>(tiles + RING * N * LN);
  C* tw = reinterpret_cast<C*>(phis + B * PTS);

  const int I0 = slot_blocks[slot].x * B;
  const int cs = slot_couple_base[slot];
  const long long rowoff = (long long)x * PLANE + z0;

  __shared__ unsigned live_mask;
  if (threadIdx.x < 32) {
    const unsigned m = __ballot_sync(0xffffffffu, threadIdx.x < D::NCPL && !couple_empty(couples[cs + threadIdx.x]));
    if (threadIdx.x == 0) live_mask = m;
  }
  __syncthreads();
  const unsigned live = live_mask;

  // the block's orbital tiles (rows of ZC reals) join the first copy group
  {
    // reals per copy: 16 bytes where every orbital row starts on a 16-byte boundary (N a multiple
    // of 16 / sizeof(T)), else 8 bytes
    constexpr int CPB = (N * int(sizeof(T))) % 16 == 0 ? 16 : 8;
    constexpr int RPER = CPB / int(sizeof(T));
    constexpr int VPR = ZC / RPER;
    for (int i = threadIdx.x; i < B * N * VPR; i += NT) {
      const int v = i % VPR;
      const int rest = i / VPR;
      const int y = rest % N;
      const int o = rest / N;
      T* dst = phis + o * PTS + y * ZC + v * RPER;
      const int valid = zcn - v * RPER;
      const int bytes = valid >= RPER ? CPB : (valid > 0 ? valid * int(sizeof(T)) : 0);
      const T* src = orb + (long long)(I0 + o) * Ntot + rowoff + (long long)y * N + v * RPER;
      if constexpr (CPB == 16) cp_async16(dst, bytes ? (const void*)src : (const void*)orb, bytes);
      else cp_async8(dst, bytes ? (const void*)src : (const void*)orb, bytes);
    }
  }

  // couples k*CPI .. k*CPI+CPI-1 -> ring slot k % RING (empty couples and columns past N read as
  // zero); an iteration past the block pair commits an empty group
  auto issue_it = [&](int k) {
    if (k >= ITERS) { cp_async_commit(); return; }
    C* dstb = tiles + (k % RING) * N * LN;
    constexpr int VPR = ZC / PER;
    for (int i = threadIdx.x; i < CPI * N * VPR; i += NT) {
      const int v = i % VPR;
      const int rest = i / VPR;
      const int u = rest % CPI, y = rest / CPI;
      const int cr = k * CPI + u;
      const bool ok_c = ((live >> cr) & 1u) && v * PER < zcn;
      const C* src = W + ((long long)(cs + cr - c0) * N + x) * PLANE + (long long)y * N + z0 + v * PER;
      cp_async16(dstb + y * LN + u * ZC + v * PER, ok_c ? (const void*)src : (const void*)W, ok_c ? 16 : 0);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int k = 0; k < RING - 1; ++k) issue_it(k);

  for (int i = threadIdx.x; i < P.twtotal; i += NT) tw[i] = twg[i];

  long long goff[NP];
  bool ok[NP];
  T phi[NP][B], acc[NP][B];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const int p = threadIdx.x + k * NT;
    const int y = p / ZC, zz = p - y * ZC;
    ok[k] = p < PTS && zz < zcn;
    goff[k] = rowoff + (long long)y * N + zz;
#pragma unroll
    for (int j = 0; j < B; ++j) acc[k][j] = T(0);
  }

  static_for<0, ITERS>([&](auto KK) {
    constexpr int kk = decltype(KK)::value;
    issue_it(kk + RING - 1);
    cp_async_wait<RING - 1>();
    __syncthreads();
    if (kk == 0) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const int p = threadIdx.x + k * NT;
#pragma unroll
        for (int j = 0; j < B; ++j) phi[k][j] = ok[k] ? phis[j * PTS + p] : T(0);
      }
    }
    C* buf = tiles + (kk % RING) * N * LN;
    stages<N, true, 0, P.ns, LN, 1, LN, NT>(buf, tw);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = threadIdx.x + k * NT;
      const int y = p / ZC, zz = p - y * ZC;
      const C* vp = buf + y * LN + zz;
      static_for<0, CPI>([&](auto U) {
        constexpr int u = decltype(U)::value;
        constexpr int c = kk * CPI + u;
        constexpr int a0 = D::first(c, 0), b0 = D::second(c, 0);
        constexpr int a1 = D::first(c, 1), b1 = D::second(c, 1);
        const C v = ok[k] ? vp[u * ZC] : C{T(0), T(0)};
        if constexpr (a0 == b0) {
          acc[k][a0] += v.x * phi[k][a0];
        } else {
          acc[k][a0] += v.x * phi[k][b0];
          acc[k][b0] += v.x * phi[k][a0];
        }
        if constexpr (a1 == b1) {
          acc[k][a1] += v.y * phi[k][a1];
        } else {
          acc[k][a1] += v.y * phi[k][b1];
          acc[k][b1] += v.y * phi[k][a1];
        }
      });
    }
    __syncthreads();
  });

  const T vs = (T)vscale;
  if (tma_flush) {
    // the scaled sums go where the orbital tiles were (read into registers in the first
    // iteration) and are added into the call's FP32 accumulator of V_x phi at L2 by one tensor
    // reduce-add (tmV: the accumulator as (z, y, orbital, x), box 8 x N x 8)
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const int p = threadIdx.x + k * NT;
      if (p >= PTS) continue;
#pragma unroll
      for (int j = 0; j < B; ++j) phis[j * PTS + p] = vs * acc[k][j];
    }
    tc::fence_proxy_async();
    __syncthreads();
    if (threadIdx.x == 0) {
      tma::reduce_add4d(&tmV, z0, 0, I0, x, phis);
      tma::bulk_commit();
      tma::bulk_wait_read_all();
    }
    return;
  }
  // read-modify-write of the block's rows of the call's FP32 accumulator of V_x phi: every load
  // before any store
  T old[NP][B];
#pragma unroll
  for (int k = 0; k < NP; ++k)
#pragma unroll
    for (int j = 0; j < B; ++j) old[k][j] = ok[k] ? __ldcg(V + (long long)(I0 + j) * Ntot + goff[k]) : T(0);
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    if (!ok[k]) continue;
#pragma unroll
    for (int j = 0; j < B; ++j) V[(long long)(I0 + j) * Ntot + goff[k]] = old[k][j] + vs * acc[k][j];
  }
}

}  // namespace ct
}  // namespace hfx
