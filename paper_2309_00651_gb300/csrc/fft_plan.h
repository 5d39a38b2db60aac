// Split of an FFT length into in-register radices, shared by the host tables and the
// compile-time kernels (both must agree: the Coulomb table is stored in the digit-reversed
// order that this split produces).
//
// Radices {16,12,10,9,8,6,5,4,3,2}; fewest stages first (each stage is one shared-memory round
// trip), then the lowest estimated flop count per point.
#pragma once

namespace hfx {

constexpr int kMaxStages = 8;

struct Factors {
  int ns;                 // number of stages (-1: no split exists)
  int r[kMaxStages];      // radix of stage s, stage 0 first in the forward transform
  double cost;
};

__host__ __device__ constexpr double radix_cost(int r) {
  return r == 2 ? 2.0 : r == 3 ? 4.0 : r == 4 ? 4.0 : r == 5 ? 6.8 : r == 6 ? 5.3 : r == 8 ? 5.5
       : r == 9 ? 7.6 : r == 10 ? 7.2 : r == 12 ? 7.3 : r == 16 ? 7.5 : 99.0;
}

__host__ __device__ constexpr Factors best_factors(int n) {
  Factors best{0, {0, 0, 0, 0, 0, 0, 0, 0}, 0.0};
  if (n == 1) return best;
  const int radices[10] = {16, 12, 10, 9, 8, 6, 5, 4, 3, 2};
  bool found = false;
  for (int i = 0; i < 10; ++i) {
    const int r = radices[i];
    if (n % r) continue;
    const Factors rest = best_factors(n / r);
    if (rest.ns < 0 || rest.ns + 1 > kMaxStages) continue;
    Factors f{rest.ns + 1, {0, 0, 0, 0, 0, 0, 0, 0}, 0.0};
    f.r[0] = r;
    for (int k = 0; k < rest.ns; ++k) f.r[k + 1] = rest.r[k];
    f.cost = rest.cost + radix_cost(r) + 6.0 * (r - 1) / r + 1000.0;
    if (!found || f.cost < best.cost) { best = f; found = true; }
  }
  if (!found) best.ns = -1;
  return best;
}

// Per-stage data of one length: radices, sub-lengths m[s] = n / (r[0] ... r[s]) and the offset of
// stage s's twiddle table [m][r] (w_L^{j1 k}, L = r m; stages with m = 1 have none).
struct StagePlan {
  int n, ns;
  int r[kMaxStages];
  int m[kMaxStages];
  int twoff[kMaxStages];
  int twtotal;
};

__host__ __device__ constexpr StagePlan stage_plan(int n) {
  StagePlan p{n, 0, {0}, {0}, {0}, 0};
  const Factors f = best_factors(n);
  p.ns = f.ns;
  int m = n, off = 0;
  for (int s = 0; s < (f.ns > 0 ? f.ns : 0); ++s) {
    p.r[s] = f.r[s];
    m /= f.r[s];
    p.m[s] = m;
    p.twoff[s] = off;
    off += m > 1 ? m * f.r[s] : 0;
  }
  p.twtotal = off;
  return p;
}

}  // namespace hfx
