"""FP64 CPU oracle for the SIN(R) isokinetic-thermostat updates of the multiple-time-step integrator.

TEST INFRASTRUCTURE ONLY.  Plain numpy statements of the operator updates the paper lists in its
appendix (updates A, B and C, applied in the XI-RESPA factorisation, Sec. 2.3 eq. "trotter-sinr";
equations of motion eq. "eom", constraint eq. "kecons").  Only the test suite, the smoke check and
the CPU-baseline leg of the benchmark may import it; the library never does, and it shares no code
with the CUDA kernels.

State per physical degree of freedom I (arrays over I; thermostat arrays [n_dof, L]):
  X_I, V_I, mass M_I, force F_I; thermostat velocities v1_{I,j}, v2_{I,j}, j = 1..L.
Parameters: kT, Q1, Q2 (thermostat masses), gamma (friction), L (chain length).
Constraint (eq. kecons): Lambda_I = M_I V_I^2 + L/(L+1) sum_j Q1 v1_{I,j}^2 = L kT.

* update_n (A): one factor exp(iL_N Delta/2): quarter kick of v2 by G(v1)/Q2, the isokinetic
  rescaling of V and v1 (factor H_I, with v1 also damped by exp(-v2 Delta/2)), quarter kick again.
* update_v (B): exp(iL_V dt/2) with a force held constant: V = (V + s F/M)/sdot, v1 = v1/sdot.
* update_x (C): X += V dt and the exact Ornstein-Uhlenbeck step of v2 over dt with a given
  standard normal draw R_{I,j}.

Readings where the paper is silent: Lambda_I in updates A and B is the constraint value L kT; the
Suzuki-Yoshida weights are the standard third- and fifth-order ones (Yoshida 1990); in B,
cosh(x) - 1 is evaluated as 2 sinh(x/2)^2 (the same quantity without cancellation), and where
x = sqrt(b) dt/2 < 1e-4 the printed expressions (which divide by b) are replaced by their series
in x through x^4.
"""
from __future__ import annotations

import math
import numpy as np


def suzuki_yoshida_weights(n_sy: int) -> np.ndarray:
    if n_sy == 1:
        return np.array([1.0])
    if n_sy == 3:
        w = 1.0 / (2.0 - 2.0 ** (1.0 / 3.0))
        return np.array([w, 1.0 - 2.0 * w, w])
    if n_sy == 5:
        w = 1.0 / (4.0 - 4.0 ** (1.0 / 3.0))
        return np.array([w, w, 1.0 - 4.0 * w, w, w])
    raise ValueError("n_sy must be 1, 3 or 5")


def constraint(M, V, v1, Q1, L):
    """Lambda_I = M V^2 + L/(L+1) sum_j Q1 v1_j^2 (eq. kecons)."""
    return M * V * V + (L / (L + 1.0)) * Q1 * np.sum(v1 * v1, axis=-1)


def update_n(V, v1, v2, M, kT, Q1, Q2, L, delta):
    """Update A for one sub-step length Delta (one factor exp(iL_N Delta/2)); returns new arrays."""
    lam = L * kT
    v2 = v2 + 0.25 * delta * (Q1 * v1 * v1 - kT) / Q2
    H = np.sqrt(lam / (M * V * V + (L / (L + 1.0)) * Q1 * np.sum(v1 * v1 * np.exp(-v2 * delta), axis=-1)))
    V = V * H
    v1 = v1 * H[:, None] * np.exp(-0.5 * v2 * delta)
    v2 = v2 + 0.25 * delta * (Q1 * v1 * v1 - kT) / Q2
    return V, v1, v2


def update_n_half_step(V, v1, v2, M, kT, Q1, Q2, L, dt, n_res=1, n_sy=1):
    """exp(iL_N dt/2) as the product of n_res x n_sy factors with Delta = w_k dt / n_res."""
    for _ in range(n_res):
        for w in suzuki_yoshida_weights(n_sy):
            V, v1, v2 = update_n(V, v1, v2, M, kT, Q1, Q2, L, w * dt / n_res)
    return V, v1, v2


def update_v(V, v1, F, M, kT, L, dt):
    """Update B (exp(iL_V dt/2) with F constant): a = F V / Lambda, b = F^2 / (M Lambda)."""
    lam = L * kT
    a = F * V / lam
    b = F * F / (M * lam)
    rb = np.sqrt(b)
    x = rb * 0.5 * dt
    small = x < 1e-4
    with np.errstate(divide="ignore", invalid="ignore"):
        s_big = np.sinh(x) / rb + (a / b) * (2.0 * np.sinh(0.5 * x) ** 2)
        sd_big = np.cosh(x) + (a / rb) * np.sinh(x)
    h = 0.5 * dt
    # series of the same expressions in x = sqrt(b) dt/2 (terms through x^4)
    s_small = h * (1.0 + b * h * h / 6.0 + b * b * h ** 4 / 120.0) + a * h * h * (0.5 + b * h * h / 24.0)
    sd_small = 1.0 + b * h * h / 2.0 + b * b * h ** 4 / 24.0 + a * h * (1.0 + b * h * h / 6.0)
    s = np.where(small, s_small, s_big)
    sd = np.where(small, sd_small, sd_big)
    V = (V + s * F / M) / sd
    v1 = v1 / sd[:, None]
    return V, v1


def update_x(X, V, v2, R, kT, Q2, gamma, dt):
    """Update C: X += V dt; v2 = v2 e^{-gamma dt} + sigma R sqrt((1 - e^{-2 gamma dt}) / (2 gamma)),
    sigma = sqrt(2 kT gamma / Q2)."""
    sigma = math.sqrt(2.0 * kT * gamma / Q2)
    X = X + V * dt
    v2 = v2 * math.exp(-gamma * dt) + sigma * R * math.sqrt((1.0 - math.exp(-2.0 * gamma * dt)) / (2.0 * gamma))
    return X, v2


def xi_respa_inner(X, V, v1, v2, M, F_fast, kT, Q1, Q2, L, gamma, dt, R, n_res=1, n_sy=1, F_first=None,
                   F_last=None):
    """One inner factor of eq. trotter-sinr, updates applied in the order
    N(dt/2) V(dt/2) [X(dt/2) OU(dt) X(dt/2) = C] V(dt/2) N(dt/2).  F_fast is a callable of X; the
    slow kick n_MTS F_slow enters the first velocity update of the outer step's first inner step
    (F_first, an array) and the second velocity update of its last one (F_last, a callable of the
    position after C)."""
    V, v1, v2 = update_n_half_step(V, v1, v2, M, kT, Q1, Q2, L, dt, n_res, n_sy)
    F = F_fast(X) if F_first is None else F_fast(X) + F_first
    V, v1 = update_v(V, v1, F, M, kT, L, dt)
    X, v2 = update_x(X, V, v2, R, kT, Q2, gamma, dt)
    F = F_fast(X) if F_last is None else F_fast(X) + F_last(X)
    V, v1 = update_v(V, v1, F, M, kT, L, dt)
    V, v1, v2 = update_n_half_step(V, v1, v2, M, kT, Q1, Q2, L, dt, n_res, n_sy)
    return X, V, v1, v2
