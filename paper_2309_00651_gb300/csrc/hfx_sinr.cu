// SIN(R) isokinetic-thermostat updates of the multiple-time-step integrator (the paper's
// appendix, updates A, B and C, applied in its XI-RESPA factorisation; equations of motion
// eq. eom, constraint eq. kecons).  One thread per physical degree of freedom I, its L thermostat
// velocities v1_{I,j}, v2_{I,j} in registers; FP64 throughout.  The FP64 pipe of this part is
// narrow, so the quotients that do not depend on the degree of freedom are taken once on the host
// (Delta/(4 Q2), -Delta/2, sqrt(Lambda), L Q1/(L+1)) and H comes from one reciprocal square root.
//
//   A  exp(iL_N Delta/2), n_res x n_sy factors with Delta = w_k dt / n_res:
//        v2 += (Delta/4) (Q1 v1^2 - kT)/Q2
//        H   = sqrt(Lambda / (M V^2 + L/(L+1) sum_j Q1 v1_j^2 exp(-v2_j Delta)))
//        V  *= H,  v1_j *= H exp(-v2_j Delta/2)
//        v2 += (Delta/4) (Q1 v1^2 - kT)/Q2
//   B  exp(iL_V dt/2), force F constant:  a = F V/Lambda, b = F^2/(M Lambda), x = sqrt(b) dt/2,
//        s = sinh(x)/sqrt(b) + (a/b)(cosh x - 1),  sdot = cosh x + (a/sqrt(b)) sinh x,
//        V = (V + s F/M)/sdot,  v1_j /= sdot
//      with cosh x - 1 taken as 2 sinh(x/2)^2 and, for x < 1e-4, the series of s and sdot in x.
//   C  X += V dt;  v2 = v2 e^{-gamma dt} + sigma R sqrt((1 - e^{-2 gamma dt})/(2 gamma)),
//        sigma = sqrt(2 kT gamma / Q2), R a standard normal draw supplied by the caller.
// Lambda is the constraint value L kT.
#include <cuda_runtime.h>
#include <stdint.h>

#include "hfx_ace_internal.h"

namespace hfx {
namespace sinr {

namespace {

constexpr int kThreads = 256;

// per Suzuki-Yoshida factor k: c = Delta_k / (4 Q2) and hd = -Delta_k / 2
struct SubSteps {
  double c[5], hd[5];
};

__global__ void __launch_bounds__(kThreads) k_update_n(SinrArgs a, long long n_dof, int n_res, int n_sy, SubSteps ss,
                                                       double sqrt_lam, double cq, const double* __restrict__ mass,
                                                       double* __restrict__ V, double* __restrict__ v1,
                                                       double* __restrict__ v2) {
  const long long I = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (I >= n_dof) return;
  const int L = a.L;
  double x1[kMaxChain], x2[kMaxChain];
  for (int j = 0; j < L; ++j) {
    x1[j] = v1[I * L + j];
    x2[j] = v2[I * L + j];
  }
  const double M = mass[I];
  double vel = V[I];
  for (int r = 0; r < n_res; ++r) {
    for (int k = 0; k < n_sy; ++k) {
      const double c = ss.c[k], hd = ss.hd[k];
      // e_j = exp(-v2_j Delta/2) serves both the rescaling of v1 and, squared, the denominator of H
      double e[kMaxChain];
      double den = M * vel * vel;
      for (int j = 0; j < L; ++j) {
        x2[j] += c * fma(a.Q1 * x1[j], x1[j], -a.kT);
        e[j] = exp(hd * x2[j]);
        den += cq * (x1[j] * x1[j]) * (e[j] * e[j]);
      }
      const double H = sqrt_lam * rsqrt(den);
      vel *= H;
      for (int j = 0; j < L; ++j) {
        x1[j] *= H * e[j];
        x2[j] += c * fma(a.Q1 * x1[j], x1[j], -a.kT);
      }
    }
  }
  V[I] = vel;
  for (int j = 0; j < L; ++j) {
    v1[I * L + j] = x1[j];
    v2[I * L + j] = x2[j];
  }
}

__global__ void __launch_bounds__(kThreads) k_update_v(SinrArgs a, long long n_dof, double dt, double inv_lam,
                                                       const double* __restrict__ mass, const double* __restrict__ force,
                                                       const double* __restrict__ force_extra, double* __restrict__ V,
                                                       double* __restrict__ v1) {
  const long long I = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (I >= n_dof) return;
  const int L = a.L;
  const double M = mass[I], inv_m = 1.0 / M;
  const double F = force[I] + (force_extra ? force_extra[I] : 0.0);
  const double vel = V[I];
  const double ca = F * vel * inv_lam, cb = F * F * inv_m * inv_lam;
  const double rb = sqrt(cb), h = 0.5 * dt, x = rb * h;
  double s, sd;
  if (x < 1e-4) {
    s = h * (1.0 + cb * h * h / 6.0 + cb * cb * h * h * h * h / 120.0) + ca * h * h * (0.5 + cb * h * h / 24.0);
    sd = 1.0 + cb * h * h / 2.0 + cb * cb * h * h * h * h / 24.0 + ca * h * (1.0 + cb * h * h / 6.0);
  } else {
    // one hyperbolic function: sinh x = 2 sinh(x/2) cosh(x/2), cosh x - 1 = 2 sinh(x/2)^2,
    // cosh(x/2) = sqrt(1 + sinh(x/2)^2); a/b = V M / F (F != 0 on this branch)
    const double shh = sinh(0.5 * x);
    const double chh = sqrt(fma(shh, shh, 1.0));
    const double sh = 2.0 * shh * chh, chm1 = 2.0 * shh * shh;
    const double inv_rb = 1.0 / rb;
    s = sh * inv_rb + (vel * M / F) * chm1;
    sd = 1.0 + chm1 + ca * inv_rb * sh;
  }
  const double inv = 1.0 / sd;
  V[I] = (vel + s * F * inv_m) * inv;
  for (int j = 0; j < L; ++j) v1[I * L + j] *= inv;
}

__global__ void __launch_bounds__(kThreads) k_update_x(SinrArgs a, long long n_dof, double dt, double decay,
                                                       double noise, const double* __restrict__ V,
                                                       double* __restrict__ X, double* __restrict__ v2,
                                                       const double* __restrict__ R) {
  const long long I = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (I >= n_dof) return;
  X[I] += V[I] * dt;
  const int L = a.L;
  for (int j = 0; j < L; ++j) v2[I * L + j] = v2[I * L + j] * decay + noise * R[I * L + j];
}

int blocks(long long n) { return (int)((n + kThreads - 1) / kThreads); }

}  // namespace

cudaError_t update_n(const SinrArgs& a, long long n_dof, double dt, int n_res, const SyWeights& w, int n_sy,
                     const double* mass, double* V, double* v1, double* v2, cudaStream_t st) {
  if (n_dof == 0) return cudaSuccess;
  SubSteps ss{};
  for (int k = 0; k < n_sy; ++k) {
    const double delta = w.w[k] * dt / n_res;
    ss.c[k] = 0.25 * delta / a.Q2;
    ss.hd[k] = -0.5 * delta;
  }
  const double sqrt_lam = sqrt(a.L * a.kT), cq = (double)a.L / (a.L + 1.0) * a.Q1;
  k_update_n<<<blocks(n_dof), kThreads, 0, st>>>(a, n_dof, n_res, n_sy, ss, sqrt_lam, cq, mass, V, v1, v2);
  return cudaGetLastError();
}

cudaError_t update_v(const SinrArgs& a, long long n_dof, double dt, const double* mass, const double* force,
                     const double* force_extra, double* V, double* v1, cudaStream_t st) {
  if (n_dof == 0) return cudaSuccess;
  k_update_v<<<blocks(n_dof), kThreads, 0, st>>>(a, n_dof, dt, 1.0 / (a.L * a.kT), mass, force, force_extra, V, v1);
  return cudaGetLastError();
}

cudaError_t update_x(const SinrArgs& a, long long n_dof, double dt, const double* V, double* X, double* v2,
                     const double* R, cudaStream_t st) {
  if (n_dof == 0) return cudaSuccess;
  // the Ornstein-Uhlenbeck coefficients are the same for every degree of freedom
  const double decay = exp(-a.gamma * dt);
  const double sigma = sqrt(2.0 * a.kT * a.gamma / a.Q2);
  const double noise = sigma * sqrt((1.0 - exp(-2.0 * a.gamma * dt)) / (2.0 * a.gamma));
  k_update_x<<<blocks(n_dof), kThreads, 0, st>>>(a, n_dof, dt, decay, noise, V, X, v2, R);
  return cudaGetLastError();
}

}  // namespace sinr
}  // namespace hfx
