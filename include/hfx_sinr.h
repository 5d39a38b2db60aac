/* hfx_sinr.h -- C ABI of the SIN(R) isokinetic-thermostat updates of the multiple-time-step
 * integrator (the paper's appendix, updates A, B and C; they are applied in its XI-RESPA
 * factorisation, Sec. 2.3 eq. trotter-sinr; equations of motion eq. eom; constraint eq. kecons).
 * The paper has no code for them; each entry applies one operator to every degree of freedom.
 *
 * State per physical degree of freedom I = 0..n_dof-1 (Cartesian components of all atoms), all
 * device FP64 arrays owned by the caller:
 *   X[I], V[I], mass[I], force[I];  thermostat velocities v1[I][j], v2[I][j], j < L (row per I).
 * Constraint: Lambda_I = mass V^2 + L/(L+1) sum_j Q1 v1_j^2 = L kT, kept exactly (up to rounding)
 * by A and B; C leaves V and v1 alone.  Lambda in A and B is the constraint value L kT.
 *
 * Errors: HFX_ERR_INVALID_ARG on the host for NULL arrays (when n_dof > 0), n_dof < 0, L outside
 * 1..16, kT, Q1, Q2 <= 0 (gamma <= 0 for C), n_res < 1, n_sy not 1, 3 or 5, pointers that are
 * not 8-byte aligned.  Calls are asynchronous on `cuda_stream`.
 */
#ifndef HFX_SINR_H
#define HFX_SINR_H

#include "hfx.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  double kT;     /* k_B T (Hartree)                                  */
  double Q1;     /* thermostat mass of v1 (Q = k_B T tau^2)          */
  double Q2;     /* thermostat mass of v2                            */
  double gamma;  /* Ornstein-Uhlenbeck friction of v2 (1/time)       */
  int32_t L;     /* thermostat chain length, 1..16                   */
} hfx_sinr_params;

/* Update A (the paper's appendix, update A; eq. eom): exp(iL_N dt/2) as n_res x n_sy factors
 * (Suzuki-Yoshida order n_sy = 1, 3 or 5, the standard weights w_k), each with
 * Delta = w_k dt / n_res:
 *   v2 += (Delta/4) G(v1)/Q2, G(v1) = Q1 v1^2 - kT;  V *= H;  v1 *= H exp(-v2 Delta/2);
 *   v2 += (Delta/4) G(v1)/Q2;  H = sqrt(Lambda/(M V^2 + L/(L+1) sum_j Q1 v1_j^2 exp(-v2_j Delta))). */
hfx_status hfx_sinr_update_n(const hfx_sinr_params* p, int64_t n_dof, double dt, int32_t n_res, int32_t n_sy,
                             const double* mass, double* V, double* v1, double* v2, void* cuda_stream);

/* Update B (the paper's appendix, update B): exp(iL_V dt/2) with the force F = force +
 * force_extra held constant (force_extra may be NULL; the XI-RESPA steps pass n_MTS F_slow there
 * at the ends of an outer step):
 *   V = (V + s F/M)/sdot, v1 /= sdot, with s, sdot of a = F V/Lambda, b = F^2/(M Lambda). */
hfx_status hfx_sinr_update_v(const hfx_sinr_params* p, int64_t n_dof, double dt, const double* mass,
                             const double* force, const double* force_extra, double* V, double* v1,
                             void* cuda_stream);

/* Update C (the paper's appendix, update C): X += V dt and the exact Ornstein-Uhlenbeck step of
 * v2 over dt,
 *   v2 = v2 e^{-gamma dt} + sigma R sqrt((1 - e^{-2 gamma dt})/(2 gamma)), sigma = sqrt(2 kT gamma/Q2),
 * with R[I][j] standard normal draws supplied by the caller (read only). */
hfx_status hfx_sinr_update_x(const hfx_sinr_params* p, int64_t n_dof, double dt, const double* V, double* X,
                             double* v2, const double* R, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* HFX_SINR_H */
