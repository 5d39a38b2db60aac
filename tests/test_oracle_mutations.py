"""The oracle pins catch plausible mistakes: each test plants one mistake in the oracle (on the
CPU, through monkeypatch) and checks that a pin which the correct oracle passes now fails.

Exchange (Eqs. vx, vij, HFX): Coulomb kernel with the wrong power of |G|, a dropped 1/N in the
pair potential, a dropped 1/2 in the energy scale, off-diagonal pairs counted once, the pair
density taken from the wrong orbitals.  ACE (Eq. vx_ace): the grid inner product without Omega/N,
a flipped sign of the compressed operator, L^-1 applied where L^-T belongs.  SIN(R): update B
without the isokinetic division by sdot.
"""
import math

import numpy as np

from oracle import ace_oracle as A
from oracle import hfx_oracle as O
from oracle import sinr_oracle as S
from paper_2309_00651_gb300 import inputs as I

KSET = np.array([[1, 0, 0], [0, 2, -1], [1, 1, 1]])
L_BOX, N_GRID = 7.0, 8


def real_closed_form_holds(rtol=1e-10):
    """E_x and V_x phi of cos/sin plane waves against the closed form (the pin of Eqs. vx/HFX)."""
    lat = np.diag([L_BOX] * 3)
    phi = I.real_plane_wave_orbitals(KSET, L_BOX, N_GRID)
    E0, eps = O.closed_form_real(KSET, lat)
    E, V = O.exchange(phi, I.all_pairs(len(phi)), lat)
    eps_o = np.repeat(eps, 2)
    okE = abs(E - E0) <= rtol * abs(E0)
    okV = np.allclose(V, eps_o[:, None, None, None] * phi, rtol=rtol, atol=rtol * np.max(np.abs(V)))
    return okE and okV


def homogeneity_holds(rtol=1e-12):
    """E_x = 1/2 (Omega/N) sum_i <phi_i, V_i> on random orbitals (degree-4 homogeneity)."""
    L = 6.5
    lat = np.diag([L] * 3)
    raw = I.random_pw_orbitals(4, L, 8, ecut=0.5 * (2 * math.pi * 2.5 / L) ** 2, seed=3)
    phi, _ = I.loewdin(raw, L ** 3)
    E, V = O.exchange(phi, I.all_pairs(4), lat)
    return abs(0.5 * (L ** 3 / 8 ** 3) * np.sum(phi * V) - E) <= rtol * abs(E)


def test_correct_oracle_passes_the_pins():
    assert real_closed_form_holds()
    assert homogeneity_holds()


def test_wrong_power_of_G(monkeypatch):
    good = O.coulomb_kernel

    def bad(lattice, grid, sphere_ecut=None):
        v = good(lattice, grid, sphere_ecut)
        g2 = O.g_squared(lattice, grid)
        return np.where(g2 > 0, v * np.sqrt(g2), 0.0)  # 4 pi / |G|

    monkeypatch.setattr(O, "coulomb_kernel", bad)
    assert not real_closed_form_holds()


def test_dropped_inverse_normalisation(monkeypatch):
    good = O.pair_potential
    monkeypatch.setattr(O, "pair_potential", lambda F, v, direct=None: F.size * good(F, v, direct))
    assert not real_closed_form_holds()
    assert not homogeneity_holds()


def test_dropped_half_in_energy(monkeypatch):
    good = O.energy_scale
    monkeypatch.setattr(O, "energy_scale", lambda lattice, grid, alpha: 2.0 * good(lattice, grid, alpha))
    assert not real_closed_form_holds()
    assert not homogeneity_holds()


def test_off_diagonal_weight_one(monkeypatch):
    # count every i != j pair once: its energy term halves when its transform is scaled by 1/sqrt 2
    # (its potential is scaled too, a second symptom of the same mistake)
    good_t = O.pair_transform

    def bad_t(phi_i, phi_j, direct=None):
        F = good_t(phi_i, phi_j, direct)
        same = phi_i.__array_interface__["data"][0] == phi_j.__array_interface__["data"][0]
        return F if same else F / math.sqrt(2.0)

    monkeypatch.setattr(O, "pair_transform", bad_t)
    assert not real_closed_form_holds()


def test_wrong_pair_density(monkeypatch):
    good = O.pair_transform
    monkeypatch.setattr(O, "pair_transform", lambda phi_i, phi_j, direct=None: good(phi_i, phi_i, direct))
    assert not real_closed_form_holds()


# ----------------------------------------------------------------------------- ACE

def ace_span_identity_holds(rtol=1e-10):
    L, n = 6.5, 8
    lat = np.diag([L] * 3)
    raw = I.random_pw_orbitals(5, L, n, ecut=0.5 * (2 * math.pi * 2.5 / L) ** 2, seed=5)
    phi, _ = I.loewdin(raw, L ** 3)
    _, W = O.exchange(phi, I.all_pairs(5), lat)
    try:
        _, _, P = A.ace_build(phi, W, lat)
    except np.linalg.LinAlgError:
        return False
    Y = A.ace_apply(P, phi, lat)
    return np.linalg.norm(Y - W) <= rtol * np.linalg.norm(W)


def ace_closed_form_holds(rtol=1e-10):
    lat = np.diag([L_BOX] * 3)
    phi = I.real_plane_wave_orbitals(KSET, L_BOX, N_GRID)
    _, eps_k = O.closed_form_real(KSET, lat)
    eps = np.repeat(eps_k, 2)
    W = eps[:, None, None, None] * phi
    try:
        M, _, P = A.ace_build(phi, W, lat)
    except np.linalg.LinAlgError:
        return False
    Y = A.ace_apply(P, phi, lat)
    okM = np.allclose(M, np.diag(eps), rtol=rtol, atol=rtol * np.max(np.abs(eps)))
    okP = np.allclose(P, -np.sqrt(-eps)[:, None, None, None] * phi, rtol=rtol, atol=rtol * np.max(np.abs(P)))
    return okM and okP and np.allclose(Y, W, rtol=rtol, atol=rtol * np.max(np.abs(W)))


def test_correct_ace_oracle_passes():
    assert ace_span_identity_holds() and ace_closed_form_holds()


def test_ace_missing_volume_weight(monkeypatch):
    good = A.grid_inner

    def bad(f, g, lattice):
        F = np.asarray(f).reshape(np.shape(f)[0], -1)
        return good(f, g, lattice) * F.shape[1] / O.cell_volume(lattice)

    monkeypatch.setattr(A, "grid_inner", bad)
    # (V_ACE psi itself is unchanged by a consistent rescaling of the inner product; M and P are not)
    assert not ace_closed_form_holds()


def test_ace_flipped_sign(monkeypatch):
    good = A.ace_apply
    monkeypatch.setattr(A, "ace_apply", lambda P, psi, lattice: -good(P, psi, lattice))
    assert not ace_closed_form_holds()
    assert not ace_span_identity_holds()


def test_ace_wrong_triangular_side(monkeypatch):
    import scipy.linalg

    def bad_build(phi, w, lattice):
        M = A.grid_inner(phi, w, lattice)
        Lf = np.linalg.cholesky(-0.5 * (M + M.T))
        Wr = np.asarray(w).reshape(np.shape(w)[0], -1)
        P = scipy.linalg.solve_triangular(Lf.T, Wr, lower=False)  # L^-T W_rows instead of L^-1 W_rows
        return M, Lf, P.reshape(np.shape(w))

    monkeypatch.setattr(A, "ace_build", bad_build)
    assert not ace_span_identity_holds()


# ----------------------------------------------------------------------------- SIN(R)

def test_sinr_update_b_without_sdot_breaks_the_constraint(monkeypatch):
    kT, Q1, L = 0.0019, 0.0019 * 1600.0, 4
    rng = np.random.default_rng(1)
    M = rng.uniform(1000.0, 30000.0, 20)
    V = rng.standard_normal(20) * 1e-3
    v1 = rng.standard_normal((20, L)) * math.sqrt(kT / Q1)
    f = np.sqrt(L * kT / S.constraint(M, V, v1, Q1, L))
    V, v1 = V * f, v1 * f[:, None]
    F = rng.standard_normal(20) * 0.05
    V2, v12 = S.update_v(V, v1, F, M, kT, L, 40.0)
    assert np.allclose(S.constraint(M, V2, v12, Q1, L), L * kT, rtol=1e-13)
    good = S.update_v

    def bad(V, v1, F, M, kT, L, dt):
        Vn, _ = good(V, v1, F, M, kT, L, dt)
        return Vn, v1  # thermostat velocities not rescaled
    monkeypatch.setattr(S, "update_v", bad)
    V3, v13 = S.update_v(V, v1, F, M, kT, L, 40.0)
    assert not np.allclose(S.constraint(M, V3, v13, Q1, L), L * kT, rtol=1e-10)
