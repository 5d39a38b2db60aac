"""Pins of the ACE and screening oracle against facts fixed by the mathematics.

* closed form: real plane-wave orbitals are eigenfunctions of V_x (V_x phi = eps phi, itself
  pinned by the exchange closed form), so M = diag(eps), L = diag(sqrt(-eps)),
  P_k = -sqrt(-eps_k) phi_k, and the ACE operator annihilates plane waves outside the span;
* the defining property of the compression (Sec. 2.1, Eq. vx_ace): V_x^ACE psi_i = V_x psi_i on
  every occupied orbital, with W from the exchange oracle;
* the energy from the compressed operator, 1/2 tr M, equals E_x (Euler homogeneity);
* the operator depends only on the occupied span (orthogonal rotation of the occupied set);
* the symmetric-part reading for a screened pair list: L L^T = -(M + M^T)/2;
* the screen quantity: closed values for indicator functions of boxes, s_ii = 1 for orthonormal
  orbitals, the Cauchy-Schwarz bounds, and the row-major kept-pair order.
"""
import math

import numpy as np
import pytest

from oracle import ace_oracle as A
from oracle import hfx_oracle as O
from paper_2309_00651_gb300 import inputs as I


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def small_orbitals(n_orb, n, L, seed):
    ecut = 0.5 * (2 * math.pi * (n / 4 + 0.5) / L) ** 2
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=ecut, seed=seed)
    phi, _ = I.loewdin(raw, L ** 3)
    return phi


KSET = np.array([[1, 0, 0], [0, 2, -1], [1, 1, 1]])


def plane_wave_case(L=7.0, n=8):
    lat = np.diag([L, L, L])
    phi = I.real_plane_wave_orbitals(KSET, L, n)
    _, eps_k = O.closed_form_real(KSET, lat)
    eps = np.repeat(eps_k, 2)  # cos and sin of the same k share eps
    W = eps[:, None, None, None] * phi
    return lat, phi, W, eps


def test_closed_form_plane_waves():
    lat, phi, W, eps = plane_wave_case()
    M, L, P = A.ace_build(phi, W, lat)
    assert np.max(np.abs(M - np.diag(eps))) < 1e-13 * np.max(np.abs(eps))
    assert np.max(np.abs(L - np.diag(np.sqrt(-eps)))) < 1e-12
    expect_P = -np.sqrt(-eps)[:, None, None, None] * phi
    assert rel(P, expect_P) < 1e-12
    # a plane wave outside the occupied span is annihilated; the span is scaled by eps
    q = np.array([[2, -1, 0]])
    chi = I.real_plane_wave_orbitals(q, 7.0, 8)
    assert np.max(np.abs(A.ace_apply(P, chi, lat))) < 1e-12
    mix = phi[2] + 0.5 * chi[0]
    assert rel(A.ace_apply(P, mix[None], lat)[0], eps[2] * phi[2]) < 1e-12


def test_exact_on_occupied_span():
    L, n = 6.5, 10
    lat = np.diag([L, L, L])
    phi = small_orbitals(6, n, L, seed=3)
    E, W = O.exchange(phi, I.all_pairs(6), lat)
    M, Lf, P = A.ace_build(phi, W, lat)
    assert rel(A.ace_apply(P, phi, lat), W) < 1e-12
    # M is symmetric for the full pair list, and 1/2 tr M is the exchange energy
    assert np.max(np.abs(M - M.T)) < 1e-13 * np.max(np.abs(M))
    assert 0.5 * np.trace(M) == pytest.approx(E, rel=1e-12)
    # the Cholesky factor: lower triangular, positive diagonal, reproduces -M
    assert np.all(np.triu(Lf, 1) == 0) and np.all(np.diag(Lf) > 0)
    assert rel(Lf @ Lf.T, -0.5 * (M + M.T)) < 1e-14
    # the compressed energy -1/2 sum_i |P^T psi_i|^2 agrees too
    X = A.grid_inner(phi, P, lat)
    assert -0.5 * np.sum(X ** 2) == pytest.approx(E, rel=1e-12)


def test_operator_depends_only_on_span():
    L, n = 6.0, 8
    lat = np.diag([L, L, L])
    phi = small_orbitals(5, n, L, seed=11)
    pairs = I.all_pairs(5)
    _, W = O.exchange(phi, pairs, lat)
    U, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((5, 5)))
    phiU = np.einsum("ia,i...->a...", U, phi)
    _, WU = O.exchange(phiU, pairs, lat)
    _, _, P = A.ace_build(phi, W, lat)
    _, _, PU = A.ace_build(phiU, WU, lat)
    chi = np.random.default_rng(4).standard_normal((3, n, n, n))
    assert rel(A.ace_apply(PU, chi, lat), A.ace_apply(P, chi, lat)) < 1e-11


def test_screened_list_uses_symmetric_part():
    L, n = 6.0, 8
    lat = np.diag([L, L, L])
    phi = small_orbitals(6, n, L, seed=5)
    pairs = I.all_pairs(6)
    keep = np.array([(i == j) or ((i + j) % 3 != 1) for i, j in pairs])
    _, W = O.exchange(phi, pairs[keep], lat)
    M, Lf, P = A.ace_build(phi, W, lat)
    assert np.max(np.abs(M - M.T)) > 1e-6 * np.max(np.abs(M))  # really not symmetric
    assert rel(Lf @ Lf.T, -0.5 * (M + M.T)) < 1e-14
    # <psi_i|V_ACE|psi_j> = -(X X^T)_ij with X = M L^-T, i.e. M Msym^-1 M^T
    X = A.grid_inner(phi, P, lat)
    Msym = 0.5 * (M + M.T)
    assert rel(-(X @ X.T), M @ np.linalg.solve(Msym, M.T)) < 1e-12


def test_screen_indicator_boxes():
    # phi_a = c_a 1[box_a]: s_ab = c_a c_b (Omega/N) |box_a & box_b|
    n, L = 8, 5.0
    lat = np.diag([L, L, L])
    boxes = [(slice(0, 4), slice(0, 4), slice(0, 8)), (slice(2, 6), slice(0, 8), slice(4, 8)),
             (slice(6, 8), slice(6, 8), slice(0, 2))]
    c = [0.7, -1.3, 2.0]
    phi = np.zeros((3, n, n, n))
    masks = []
    for a, (b, ca) in enumerate(zip(boxes, c)):
        phi[a][b] = ca
        m = np.zeros((n, n, n), bool)
        m[b] = True
        masks.append(m)
    s = A.overlap_screen(phi, lat)
    for a in range(3):
        for b in range(3):
            expect = abs(c[a] * c[b]) * (L ** 3 / n ** 3) * np.count_nonzero(masks[a] & masks[b])
            assert s[a, b] == pytest.approx(expect, rel=1e-14, abs=1e-300)
    pairs, _ = A.screen_pairs(phi, lat, 1e-9)
    # box 2 overlaps neither of the others
    assert pairs.tolist() == [[0, 0], [0, 1], [1, 1], [2, 2]]


def test_screen_bounds_and_order():
    L, n = 6.0, 8
    lat = np.diag([L, L, L])
    phi = small_orbitals(7, n, L, seed=8)
    s = A.overlap_screen(phi, lat)
    S = A.grid_inner(phi, phi, lat)
    assert np.allclose(np.diag(s), 1.0, atol=1e-13)
    assert np.all(s <= np.sqrt(np.outer(np.diag(s), np.diag(s))) * (1 + 1e-13))
    assert np.all(s >= np.abs(S) - 1e-13)
    cut = float(np.median(s[np.triu_indices(7, 1)]))
    pairs, _ = A.screen_pairs(phi, lat, cut)
    assert np.array_equal(pairs, I.screened_pairs(phi, L ** 3, cut))
    key = pairs[:, 0] * 7 + pairs[:, 1]
    assert np.all(np.diff(key) > 0)


# ----------------------------------------------------------------------------- SCDM localisation

def test_scdm_pivots_match_library_qrcp():
    import scipy.linalg
    L, n = 6.0, 8
    phi = small_orbitals(7, n, L, seed=21)
    piv, Q, rdiag = A.scdm_pivots(phi)
    At = phi.reshape(7, -1)
    Ql, Rl, Pl = scipy.linalg.qr(At, pivoting=True, mode="economic")
    assert np.array_equal(piv, Pl[:7])
    assert np.allclose(rdiag, np.abs(np.diag(Rl)), rtol=1e-12, atol=0)
    sgn = np.sign(np.diag(Rl))
    assert np.allclose(Q, Ql * sgn[None, :], atol=1e-12)
    # the greedy factor is the QR factor of the selected columns
    assert np.allclose(A.scdm_q_from_pivots(phi, piv), Q, atol=1e-12)
    assert np.all(A.scdm_pivot_slack(phi, piv) == 1.0)


def test_scdm_recovers_disjoint_localised_orbitals():
    # orthonormal indicator functions of disjoint boxes, mixed by an orthogonal rotation: SCDM
    # returns the boxes again (up to sign and order)
    n, L = 8, 6.0
    w = L ** 3 / n ** 3
    boxes = [(slice(0, 2), slice(0, 3), slice(0, 4)), (slice(3, 6), slice(0, 2), slice(0, 8)),
             (slice(6, 8), slice(4, 8), slice(2, 5)), (slice(0, 4), slice(5, 8), slice(6, 8))]
    loc = np.zeros((4, n, n, n))
    for k, b in enumerate(boxes):
        loc[k][b] = 1.0
        loc[k] /= np.sqrt(w * np.sum(loc[k] ** 2))
    U, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((4, 4)))
    psi = np.einsum("ki,k...->i...", U, loc)
    piv, Q, Phi = A.scdm_localise(psi)
    O = w * Phi.reshape(4, -1) @ loc.reshape(4, -1).T   # overlaps with the boxes
    assert np.allclose(np.sort(np.abs(O), axis=1)[:, -1], 1.0, atol=1e-12)
    assert np.allclose(np.sort(np.abs(O), axis=1)[:, :-1], 0.0, atol=1e-12)


def test_scdm_orthonormal_same_span():
    L, n = 6.5, 8
    lat = np.diag([L, L, L])
    phi = small_orbitals(6, n, L, seed=22)
    piv, Q, Phi = A.scdm_localise(phi)
    assert np.allclose(Q.T @ Q, np.eye(6), atol=1e-13)
    S = A.grid_inner(Phi, Phi, lat)
    assert np.allclose(S, np.eye(6), atol=1e-12)
    # same occupied projector: sum_i |phi_i><phi_i| = sum_j |Phi_j><Phi_j|
    f, F = phi.reshape(6, -1), Phi.reshape(6, -1)
    assert np.allclose(f.T @ f, F.T @ F, atol=1e-12)
