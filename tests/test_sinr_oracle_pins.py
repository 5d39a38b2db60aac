"""Pins of the SIN(R) update oracle (appendix updates A, B, C; eqs. eom, kecons, trotter-sinr)
against the mathematics:

* the isokinetic constraint Lambda_I = L kT is kept exactly by updates A and B, and untouched by C;
* B is the exact flow of dV = (F/M - lambda V) dt, dv1 = -lambda v1 dt with lambda = F V / Lambda
  for a constant force (compared with a fine Runge-Kutta integration), in both of its branches;
* A is a second-order splitting of the N flow of eq. eom (error ratio 8 when the step halves), with
  the thermostat equilibrium Q1 v1^2 = kT, v2 = 0 as a fixed point;
* C moves X by V dt exactly and its Ornstein-Uhlenbeck step has the stationary law N(0, kT/Q2);
* the Suzuki-Yoshida weights satisfy the third-order conditions;
* a long XI-RESPA run with harmonic fast and slow forces keeps every Lambda_I at L kT.
"""
import math

import numpy as np
import pytest

from oracle import sinr_oracle as S

KT, Q1, Q2, L, GAMMA = 0.0019, 0.0019 * 40.0 ** 2, 0.0019 * 40.0 ** 2, 4, 0.01


def random_state(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.uniform(1000.0, 30000.0, n)
    V = rng.standard_normal(n) * 1e-3
    v1 = rng.standard_normal((n, L)) * math.sqrt(KT / Q1)
    v2 = rng.standard_normal((n, L)) * math.sqrt(KT / Q2)
    lam = S.constraint(M, V, v1, Q1, L)
    f = np.sqrt(L * KT / lam)  # place every degree of freedom on the constraint surface
    return M, V * f, v1 * f[:, None], v2


def rk4(f, y, t, steps):
    h = t / steps
    for _ in range(steps):
        k1 = f(y)
        k2 = f(y + 0.5 * h * k1)
        k3 = f(y + 0.5 * h * k2)
        k4 = f(y + h * k3)
        y = y + (h / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


def test_constraint_kept_by_a_and_b():
    M, V, v1, v2 = random_state(50, 1)
    F = np.random.default_rng(2).standard_normal(50) * 0.05
    for delta in (0.5, 5.0, 40.0):
        V2, v12, v22 = S.update_n(V, v1, v2, M, KT, Q1, Q2, L, delta)
        assert np.allclose(S.constraint(M, V2, v12, Q1, L), L * KT, rtol=1e-13, atol=0)
    for dt in (1.0, 20.0, 200.0):
        V2, v12 = S.update_v(V, v1, F, M, KT, L, dt)
        assert np.allclose(S.constraint(M, V2, v12, Q1, L), L * KT, rtol=1e-13, atol=0)


@pytest.mark.parametrize("fscale", [1e-9, 0.05])
def test_update_b_is_the_exact_constant_force_flow(fscale):
    n = 6
    M, V, v1, v2 = random_state(n, 3)
    F = np.random.default_rng(4).standard_normal(n) * fscale
    dt = 40.0
    lam = L * KT

    def rhs(y):
        Vy, v1y = y[:n], y[n:].reshape(n, L)
        lmb = F * Vy / lam
        return np.concatenate([F / M - lmb * Vy, (-lmb[:, None] * v1y).ravel()])

    y = rk4(rhs, np.concatenate([V, v1.ravel()]), 0.5 * dt, 4000)
    V2, v12 = S.update_v(V, v1, F, M, KT, L, dt)
    assert np.allclose(V2, y[:n], rtol=1e-10, atol=1e-16)
    assert np.allclose(v12, y[n:].reshape(n, L), rtol=1e-10, atol=1e-16)


def test_update_a_second_order_splitting_of_the_n_flow():
    n = 5
    M, V, v1, v2 = random_state(n, 5)
    lam = L * KT

    def rhs(y):
        Vy, v1y, v2y = y[:n], y[n:n + n * L].reshape(n, L), y[n + n * L:].reshape(n, L)
        lmb = -(1.0 / lam) * (L / (L + 1.0)) * Q1 * np.sum(v1y * v1y * v2y, axis=1)
        dV = -lmb * Vy
        dv1 = -lmb[:, None] * v1y - v2y * v1y
        dv2 = (Q1 * v1y * v1y - KT) / Q2
        return np.concatenate([dV, dv1.ravel(), dv2.ravel()])

    errs = []
    for delta in (40.0, 20.0, 10.0):
        exact = rk4(rhs, np.concatenate([V, v1.ravel(), v2.ravel()]), 0.5 * delta, 2000)
        got = np.concatenate([a.ravel() for a in S.update_n(V, v1, v2, M, KT, Q1, Q2, L, delta)])
        errs.append(np.linalg.norm(got - exact) / np.linalg.norm(exact))
    assert errs[0] / errs[1] == pytest.approx(8.0, rel=0.15)
    assert errs[1] / errs[2] == pytest.approx(8.0, rel=0.15)


def test_update_a_thermostat_equilibrium_is_fixed():
    n = 4
    M = np.full(n, 1837.0)
    v1 = np.full((n, L), math.sqrt(KT / Q1)) * np.array([1, -1, 1, -1])
    v2 = np.zeros((n, L))
    V = np.sqrt((L * KT - (L / (L + 1.0)) * L * KT) / M)
    V2, v12, v22 = S.update_n(V, v1, v2, M, KT, Q1, Q2, L, 10.0)
    assert np.allclose(V2, V, rtol=1e-15) and np.allclose(v12, v1, rtol=1e-15)
    assert np.max(np.abs(v22)) < 1e-12 * math.sqrt(KT / Q2)  # G(v1) = 0 up to the rounding of v1


def test_update_c_and_ou_stationary_law():
    rng = np.random.default_rng(6)
    n = 200000
    X = rng.standard_normal(n)
    V = rng.standard_normal(n)
    X2, _ = S.update_x(X, V, np.zeros(n), np.zeros(n), KT, Q2, GAMMA, 3.0)
    assert np.array_equal(X2, X + V * 3.0)
    v2 = np.zeros(n)
    for _ in range(60):  # 60 steps of gamma dt = 0.5: the initial condition is forgotten
        _, v2 = S.update_x(X, V, v2, rng.standard_normal(n), KT, Q2, GAMMA, 50.0)
    var = KT / Q2
    assert abs(np.mean(v2)) < 5 * math.sqrt(var / n)
    assert np.var(v2) == pytest.approx(var, rel=5 * math.sqrt(2.0 / n))


def test_suzuki_yoshida_weights():
    for n_sy in (1, 3, 5):
        w = S.suzuki_yoshida_weights(n_sy)
        assert sum(w) == pytest.approx(1.0, abs=1e-15)
        if n_sy > 1:
            assert sum(w ** 3) == pytest.approx(0.0, abs=1e-14)


def test_xi_respa_keeps_the_constraint():
    n = 30
    M, V, v1, v2 = random_state(n, 7)
    X = np.random.default_rng(8).standard_normal(n) * 0.1
    kf, ks = 0.3, 0.02
    rng = np.random.default_rng(9)
    n_mts, dt = 4, 20.0
    for outer in range(5):
        F_slow = -ks * X
        for k in range(n_mts):
            X, V, v1, v2 = S.xi_respa_inner(X, V, v1, v2, M, lambda x: -kf * x, KT, Q1, Q2, L, GAMMA, dt,
                                            rng.standard_normal((n, L)), n_res=2, n_sy=3,
                                            F_first=n_mts * F_slow if k == 0 else None,
                                            F_last=(lambda x: n_mts * (-ks * x)) if k == n_mts - 1 else None)
            assert np.allclose(S.constraint(M, V, v1, Q1, L), L * KT, rtol=1e-12, atol=0)
