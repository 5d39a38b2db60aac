"""Pins of the FP64 oracle against facts fixed by the mathematics, not by the oracle itself.

* transforms: brute-force DFT vs an independent library FFT, and the plane-wave delta;
* Coulomb kernel: 4 pi / |G|^2 at hand-chosen G, G = 0 rule, sphere cut;
* closed forms for plane-wave orbitals (complex form of the exchange energy, and the real
  cos/sin form derived from the same definition, with V_x phi = eps phi);
* invariants: orthogonal rotation of the occupied set, v_ij = v_ji, Parseval (real-space
  energy), Euler homogeneity E = 1/2 sum_i <phi_i, V_x phi_i>, the gradient identity
  dE/dphi = 2 (Omega/N) V_x phi by a 5-point stencil (exact for a quartic), linearity in
  the pair list, the two-pairs-per-complex-transform packing identity, independence of the basis
  a cell is written in (a skewed basis of the same cubic cell);
* an independent pure-Python brute force of Eqs. vx/vij/HFX on a 4^3 grid.
"""
import math

import numpy as np
import pytest

from oracle import hfx_oracle as O
from paper_2309_00651_gb300 import inputs as I


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def small_orbitals(n_orb, n, L, seed):
    # cutoff sphere reaching about a quarter of the grid: pair products stay resolved
    ecut = 0.5 * (2 * math.pi * (n / 4 + 0.5) / L) ** 2
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=ecut, seed=seed)
    phi, _ = I.loewdin(raw, L ** 3)
    return phi


# ----------------------------------------------------------------------------- transforms

@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 6, 6), (8, 8, 8), (12, 12, 12), (4, 6, 10)])
def test_direct_dft_matches_library_fft(shape):
    rng = np.random.default_rng(1)
    f = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    assert rel(O.dft3_direct(f), np.fft.fftn(f)) < 1e-13
    assert rel(O.dft3_direct(f, inverse=True) / f.size, np.fft.ifftn(f)) < 1e-13


def test_direct_dft_plane_wave_is_delta():
    n = 6
    p = np.arange(n) / n
    m = (1, -2, 3)
    f = np.exp(2j * np.pi * (m[0] * p[:, None, None] + m[1] * p[None, :, None] + m[2] * p[None, None, :]))
    F = O.dft3_direct(f)
    expect = np.zeros((n, n, n), complex)
    expect[m[0] % n, m[1] % n, m[2] % n] = n ** 3
    assert np.max(np.abs(F - expect)) < 1e-10


# ----------------------------------------------------------------------------- kernel

def test_coulomb_kernel_closed_values():
    L, n = 7.0, 8
    v = O.coulomb_kernel(np.diag([L, L, L]), (n, n, n))
    assert v[0, 0, 0] == 0.0
    g = 2 * math.pi / L
    for (a, b, c) in [(1, 0, 0), (1, 2, 3), (4, 4, 4), (7, 1, 5)]:  # index 7 -> m = -1, index 4 -> m = 4 (Nyquist)
        m = [x if x <= n // 2 else x - n for x in (a, b, c)]
        assert v[a, b, c] == pytest.approx(4 * math.pi / (g * g * sum(x * x for x in m)), rel=1e-14)
    # orthorhombic box: G = 2 pi (m1/L1, m2/L2, m3/L3)
    Ls = (5.0, 6.0, 9.0)
    v2 = O.coulomb_kernel(np.diag(Ls), (6, 8, 10))
    m = (1, -3, 2)
    G2 = sum((2 * math.pi * mi / Li) ** 2 for mi, Li in zip(m, Ls))
    assert v2[1, 8 - 3, 2] == pytest.approx(4 * math.pi / G2, rel=1e-14)
    # even in G
    neg = (-np.arange(8)) % 8
    assert np.array_equal(v, v[neg][:, neg][:, :, neg])


def test_coulomb_sphere_cut():
    L, n, ecut = 10.0, 16, 2.0
    v = O.coulomb_kernel(np.diag([L] * 3), (n,) * 3, sphere_ecut=ecut)
    g2 = O.g_squared(np.diag([L] * 3), (n,) * 3)
    assert np.all(v[0.5 * g2 >= 4 * ecut] == 0.0)
    inside = (0.5 * g2 < 4 * ecut) & (g2 > 0)
    assert np.allclose(v[inside], 4 * math.pi / g2[inside], rtol=1e-15)


def test_skewed_basis_of_the_same_cell():
    """E_x and V_x phi of a cell do not depend on the basis it is written in (pins the general-
    lattice reciprocal vectors: a transposed or non-inverted lattice matrix fails)."""
    phi, phi_s, lat, lat_s, src = I.skewed_basis_case()
    n = phi.shape[1]
    pairs = I.all_pairs(phi.shape[0])
    E, V = O.exchange(phi, pairs, lat)
    E_s, V_s = O.exchange(phi_s, pairs, lat_s)
    assert abs(E_s - E) <= 1e-12 * abs(E)
    assert rel(V_s, V[:, src, np.arange(n)[None, :], :]) <= 1e-12
    # the skewed cell really is skewed: its reciprocal rows are not orthogonal
    B = O.reciprocal_vectors(lat_s)
    assert abs(B[0] @ B[1]) > 1e-3


def test_symmetric_part_of_the_kernel_on_a_triclinic_cell(monkeypatch):
    """On a non-orthogonal cell with even edges the kernel on the grid is not inversion-symmetric
    (a Nyquist point and its mirror have different |G|), yet for real orbitals E_x = sum v |F|^2 and
    V_x phi = Re ifft(v F) are the same with v replaced by its symmetric part (v(k) + v(-k))/2:
    |F(k)| = |F(-k)| for real pair densities, and the real part keeps only the symmetric part."""
    lat = np.array([[9.0, 0.0, 0.0], [2.5, 8.0, 0.0], [1.0, -1.5, 10.0]])
    grid = (10, 8, 12)
    v = O.coulomb_kernel(lat, grid)
    mirror = tuple((-np.arange(n)) % n for n in grid)
    v_m = v[mirror[0]][:, mirror[1]][:, :, mirror[2]]
    assert np.max(np.abs(v - v_m)) > 1e-3 * np.max(v)  # the raw kernel is not symmetric here
    rng = np.random.default_rng(12)
    phi, _ = I.loewdin(rng.standard_normal((4,) + grid), abs(float(np.linalg.det(lat))))
    pairs = I.all_pairs(4)
    E, V = O.exchange(phi, pairs, lat)
    kernel = O.coulomb_kernel

    def symmetric(lattice, g, sphere_ecut=None):
        w = kernel(lattice, g, sphere_ecut)
        m = tuple((-np.arange(n)) % n for n in g)
        return 0.5 * (w + w[m[0]][:, m[1]][:, :, m[2]])

    monkeypatch.setattr(O, "coulomb_kernel", symmetric)
    E_s, V_s = O.exchange(phi, pairs, lat)
    assert abs(E_s - E) <= 1e-13 * abs(E)
    assert rel(V_s, V) <= 1e-13


def test_result_does_not_depend_on_the_nyquist_tie_break(monkeypatch):
    """Folding the Nyquist index to -n/2 instead of +n/2 swaps v between a Nyquist point and its
    mirror on a triclinic cell; for real orbitals E_x and V_x phi stay the same."""
    lat = np.array([[9.0, 0.0, 0.0], [2.5, 8.0, 0.0], [1.0, -1.5, 10.0]])
    grid = (10, 8, 12)
    rng = np.random.default_rng(13)
    phi, _ = I.loewdin(rng.standard_normal((3,) + grid), abs(float(np.linalg.det(lat))))
    pairs = I.all_pairs(3)
    E, V = O.exchange(phi, pairs, lat)
    v_plus = O.coulomb_kernel(lat, grid)
    monkeypatch.setattr(O, "frequencies", lambda n: np.where(np.arange(n) < n // 2, np.arange(n),
                                                             np.arange(n) - n))
    assert not np.allclose(O.coulomb_kernel(lat, grid), v_plus)  # the tie-break matters to v
    E_m, V_m = O.exchange(phi, pairs, lat)
    assert abs(E_m - E) <= 1e-13 * abs(E)
    assert rel(V_m, V) <= 1e-13


def test_skewed_basis_catches_a_transposed_reciprocal_matrix(monkeypatch):
    phi, phi_s, lat, lat_s, _ = I.skewed_basis_case()
    pairs = I.all_pairs(phi.shape[0])
    E, _ = O.exchange(phi, pairs, lat, want_v=False)
    monkeypatch.setattr(O, "reciprocal_vectors",
                        lambda A: 2.0 * np.pi * np.linalg.inv(np.asarray(A, dtype=np.float64)))
    E_bad, _ = O.exchange(phi_s, pairs, lat_s, want_v=False)
    assert abs(E_bad - E) > 1e-6 * abs(E)


# ----------------------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n,direct", [(8, True), (16, False)])
def test_closed_form_complex_plane_waves(n, direct):
    L = 9.0
    lat = np.diag([L] * 3)
    kset = np.array([[0, 0, 0], [1, 0, 0], [0, 1, -1], [1, 1, 1], [-1, 2, 0]])
    phi = I.complex_plane_wave_orbitals(kset, L, n)
    E, V = O.exchange_complex(phi, lat, alpha=0.25, direct=direct)
    E_ref, eps = O.closed_form_complex(kset, lat, alpha=0.25)
    assert E == pytest.approx(E_ref, rel=1e-12)
    for i in range(len(kset)):
        assert rel(V[i], eps[i] * phi[i]) < 1e-11


@pytest.mark.parametrize("n,direct", [(12, True), (16, False)])
def test_closed_form_real_plane_waves(n, direct):
    L = 8.5
    lat = np.diag([L] * 3)
    # no two equal or opposite; all k +- q inside (-n/2, n/2)
    kset = np.array([[1, 0, 0], [0, 2, 1], [1, -1, 2], [2, 1, -1]])
    phi = I.real_plane_wave_orbitals(kset, L, n)
    # exact orthonormality on the grid
    S = (L ** 3 / n ** 3) * phi.reshape(len(phi), -1) @ phi.reshape(len(phi), -1).T
    assert np.allclose(S, np.eye(len(phi)), atol=1e-13)
    pairs = I.all_pairs(len(phi))
    E, V = O.exchange(phi, pairs, lat, alpha=0.25, direct=direct)
    E_ref, eps = O.closed_form_real(kset, lat, alpha=0.25)
    assert E == pytest.approx(E_ref, rel=1e-12)
    for a in range(len(kset)):
        for b in (2 * a, 2 * a + 1):
            assert rel(V[b], eps[a] * phi[b]) < 1e-11


def test_closed_form_real_per_pair_terms():
    L, n = 8.0, 12
    lat = np.diag([L] * 3)
    kset = np.array([[1, 0, 0], [0, 2, 1], [1, -1, 2]])
    phi = I.real_plane_wave_orbitals(kset, L, n)
    pairs = I.all_pairs(len(phi))
    e = O.pair_energy_terms(phi, pairs, lat)
    N, omega = n ** 3, L ** 3
    for (i, j), eij in zip(pairs, e):
        k, q = kset[i // 2], kset[j // 2]
        expect = (2 * math.pi / omega) * (O._inv_sq(k - q, lat) + O._inv_sq(k + q, lat))
        # Omega * sum_G v |F/N|^2
        assert omega * eij / N ** 2 == pytest.approx(expect, rel=1e-12, abs=1e-15)


# ----------------------------------------------------------------------------- invariants

def test_rotation_invariance():
    L, n = 6.0, 10
    lat = np.diag([L] * 3)
    phi = small_orbitals(5, n, L, seed=3)
    pairs = I.all_pairs(5)
    E, V = O.exchange(phi, pairs, lat)
    rng = np.random.default_rng(4)
    U, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    phiU = np.einsum("ji,jxyz->ixyz", U, phi)  # phi'_i = sum_j phi_j U_ji
    E2, V2 = O.exchange(phiU, pairs, lat)
    assert E2 == pytest.approx(E, rel=1e-12)
    assert rel(V2, np.einsum("ji,jxyz->ixyz", U, V)) < 1e-11


def test_pair_potential_symmetric():
    L, n = 6.0, 10
    lat = np.diag([L] * 3)
    phi = small_orbitals(3, n, L, seed=5)
    v = O.coulomb_kernel(lat, (n,) * 3)
    a = O.pair_potential(O.pair_transform(phi[0], phi[2]), v)
    b = O.pair_potential(O.pair_transform(phi[2], phi[0]), v)
    assert rel(a, b) < 1e-15


def test_parseval_real_space_energy():
    L, n = 6.0, 12
    lat = np.diag([L] * 3)
    phi = small_orbitals(4, n, L, seed=6)
    pairs = I.all_pairs(4)
    E, _ = O.exchange(phi, pairs, lat)
    v = O.coulomb_kernel(lat, (n,) * 3)
    N, omega = n ** 3, L ** 3
    acc = 0.0
    for i, j in pairs:
        rho = phi[i] * phi[j]
        vij = O.pair_potential(O.pair_transform(phi[i], phi[j]), v)
        acc += (1.0 if i == j else 2.0) * float(np.sum(rho * vij))
    assert -0.5 * 0.25 * (omega / N) * acc == pytest.approx(E, rel=1e-12)


def test_homogeneity_identity():
    L, n = 7.0, 12
    lat = np.diag([L] * 3)
    phi = small_orbitals(5, n, L, seed=7)
    pairs = I.all_pairs(5)
    E, V = O.exchange(phi, pairs, lat)
    N, omega = n ** 3, L ** 3
    assert 0.5 * (omega / N) * float(np.sum(phi * V)) == pytest.approx(E, rel=1e-12)
    # also for a partial list
    sub = pairs[::3]
    E2, V2 = O.exchange(phi, sub, lat)
    assert 0.5 * (omega / N) * float(np.sum(phi * V2)) == pytest.approx(E2, rel=1e-12)


def test_gradient_identity_five_point():
    L, n = 6.0, 8
    lat = np.diag([L] * 3)
    phi = small_orbitals(4, n, L, seed=8)
    pairs = I.all_pairs(4)
    _, V = O.exchange(phi, pairs, lat)
    N, omega = n ** 3, L ** 3
    for s in (1, 2):
        d = np.random.default_rng(s).standard_normal(phi.shape)
        h = 1e-3 * np.linalg.norm(phi) / np.linalg.norm(d)
        Ef = [O.exchange(phi + c * h * d, pairs, lat, want_v=False)[0] for c in (-2, -1, 1, 2)]
        fd = (Ef[0] - 8 * Ef[1] + 8 * Ef[2] - Ef[3]) / (12 * h)
        an = 2.0 * (omega / N) * float(np.sum(V * d))
        assert fd == pytest.approx(an, rel=1e-9)


def test_pair_list_linearity():
    L, n = 6.0, 10
    lat = np.diag([L] * 3)
    phi = small_orbitals(5, n, L, seed=9)
    pairs = I.all_pairs(5)
    E, V = O.exchange(phi, pairs, lat)
    E1, V1 = O.exchange(phi, pairs[::2], lat)
    E2, V2 = O.exchange(phi, pairs[1::2], lat)
    assert E1 + E2 == pytest.approx(E, rel=1e-13)
    assert rel(V1 + V2, V) < 1e-13


def test_packing_identity():
    """Two real pair densities in one complex transform: sum_G v |F_a + i F_b|^2 = e_a + e_b,
    and sum_G v Re(Z(G) Z(-G)) = e_a - e_b (what a packed kernel relies on)."""
    L, n = 6.0, 10
    lat = np.diag([L] * 3)
    phi = small_orbitals(4, n, L, seed=10)
    v = O.coulomb_kernel(lat, (n,) * 3)
    Fa = O.pair_transform(phi[0], phi[1])
    Fb = O.pair_transform(phi[2], phi[2])
    Z = O.fft3(phi[0] * phi[1] + 1j * phi[2] * phi[2])
    ea, eb = O.pair_energy_sum(Fa, v), O.pair_energy_sum(Fb, v)
    assert float(np.sum(v * np.abs(Z) ** 2)) == pytest.approx(ea + eb, rel=1e-13)
    neg = (-np.arange(n)) % n
    Zm = Z[neg][:, neg][:, :, neg]
    assert float(np.sum(v * np.real(Z * Zm))) == pytest.approx(ea - eb, rel=1e-12)
    # and the inverse transform of v Z is v_a + i v_b
    w = O.ifft3(v * Z)
    assert rel(w.real, O.pair_potential(Fa, v)) < 1e-13
    assert rel(w.imag, O.pair_potential(Fb, v)) < 1e-13


# ----------------------------------------------------------------------------- brute force

def _brute_force_exchange(phi, L, alpha):
    """Eqs. vx, vij, HFX by explicit loops over grid points and wavevectors (no FFT, no numpy
    vector maths), over all ordered pairs of real orbitals."""
    n_orb, n = len(phi), len(phi[0])
    N, omega = n ** 3, L ** 3
    pts = [(a, b, c) for a in range(n) for b in range(n) for c in range(n)]
    freqs = [k if k <= n // 2 else k - n for k in range(n)]
    Gs = [(freqs[a], freqs[b], freqs[c]) for (a, b, c) in pts]
    E = 0.0
    V = [[0.0] * N for _ in range(n_orb)]
    for i in range(n_orb):
        for j in range(n_orb):
            rho = [phi[i][a][b][c] * phi[j][a][b][c] for (a, b, c) in pts]
            pot = [0.0] * N
            for (m1, m2, m3) in Gs:
                g2 = (2 * math.pi / L) ** 2 * (m1 * m1 + m2 * m2 + m3 * m3)
                if g2 == 0.0:
                    continue
                vg = 4 * math.pi / g2
                re = im = 0.0
                for (a, b, c), r in zip(pts, rho):
                    ang = -2 * math.pi * (m1 * a + m2 * b + m3 * c) / n
                    re += r * math.cos(ang)
                    im += r * math.sin(ang)
                E += vg * (re * re + im * im)
                for t, (a, b, c) in enumerate(pts):
                    ang = 2 * math.pi * (m1 * a + m2 * b + m3 * c) / n
                    pot[t] += vg * (re * math.cos(ang) - im * math.sin(ang)) / N
            for t, (a, b, c) in enumerate(pts):
                V[i][t] -= alpha * pot[t] * phi[j][a][b][c]
    return -0.5 * alpha * omega / N ** 2 * E, V


def test_bruteforce_pure_python():
    L, n = 5.0, 4
    # unrestricted random real orbitals: the definition holds for any grid function
    raw = np.random.default_rng(11).standard_normal((3, n, n, n))
    phi, _ = I.loewdin(raw, L ** 3)
    E_bf, V_bf = _brute_force_exchange(phi.tolist(), L, 0.25)
    E, V = O.exchange(phi, I.all_pairs(3), np.diag([L] * 3), alpha=0.25)
    assert E == pytest.approx(E_bf, rel=1e-12)
    assert rel(V.reshape(3, -1), np.array(V_bf)) < 1e-12


# ----------------------------------------------------------------------------- planted mistakes

def test_planted_mistakes_are_caught(monkeypatch):
    """Each plausible slip in the oracle breaks at least one of the pins above."""
    L, n = 8.5, 12
    lat = np.diag([L] * 3)
    kset = np.array([[1, 0, 0], [0, 2, 1], [1, -1, 2]])
    phi = I.real_plane_wave_orbitals(kset, L, n)
    pairs = I.all_pairs(len(phi))
    E_ref, eps = O.closed_form_real(kset, lat)

    def pin_holds():
        E, V = O.exchange(phi, pairs, lat)
        ok_e = abs(E - E_ref) <= 1e-10 * abs(E_ref)
        ok_v = all(rel(V[b], eps[b // 2] * phi[b]) < 1e-9 for b in range(len(phi)))
        return ok_e and ok_v

    assert pin_holds()
    orig_energy_scale = O.energy_scale
    mutants = {
        # dropped 1/2 of the ordered double sum
        "scale": lambda m: m.setattr(O, "energy_scale", lambda lat_, g, a: 2 * orig_energy_scale(lat_, g, a)),
        # reciprocal vectors without the 2 pi
        "kernel": lambda m: m.setattr(O, "reciprocal_vectors", lambda A: np.linalg.inv(np.asarray(A)).T),
        # inverse transform taken with the forward sign
        "sign": lambda m: m.setattr(O, "pair_potential", lambda F, v, d=None: np.real(O.fft3(v * F)) / F.size),
        # wrong operand in the pair product: phi_i * phi_i
        "operand": lambda m: m.setattr(O, "pair_transform", lambda a, b, d=None: O.fft3(a * a, d)),
    }
    for name, plant in mutants.items():
        with monkeypatch.context() as m:
            plant(m)
            assert not pin_holds(), f"mutant {name!r} not caught"


# ----------------------------------------------------------------------------- sampled rows

def _rows_case():
    """7 orbitals on a 10^3 grid with a partial pair list: orbital 6 appears in no pair, rows 1
    and 4 appear as the first and as the second member of off-diagonal pairs and with their own
    diagonal pair."""
    L, n = 7.0, 10
    lat = np.diag([L] * 3)
    phi = small_orbitals(7, n, L, seed=21)
    allp = I.all_pairs(7)
    keep = np.random.default_rng(22).random(len(allp)) < 0.6
    sub = allp[keep & (allp[:, 0] != 6) & (allp[:, 1] != 6)]
    for must in ([1, 1], [4, 4], [0, 1], [1, 5], [2, 4], [4, 5]):
        if not any((sub[:, 0] == must[0]) & (sub[:, 1] == must[1])):
            sub = np.concatenate([sub, np.array([must], dtype=np.int32)])
    return phi, sub, lat


def test_exchange_rows_matches_full_exchange():
    """exchange_rows (the checker of every full-size parity row) equals the rows of the full
    V_x phi over the same partial list, including diagonal pairs, both pair positions and a row
    that no pair contains (exactly zero)."""
    phi, sub, lat = _rows_case()
    _, V = O.exchange(phi, sub, lat)
    rows = [1, 4, 6, 0, 5]
    R = O.exchange_rows(phi, sub, rows, lat)
    for r, k in enumerate(rows):
        if k == 6:
            assert np.all(R[r] == 0.0)
        else:
            assert rel(R[r], V[k]) < 1e-13
    # reversing the pair list (order inside the sums only) changes nothing beyond rounding
    R2 = O.exchange_rows(phi, sub[::-1].copy(), rows, lat)
    assert rel(R2, R) < 1e-13


def test_exchange_rows_closed_form_real():
    """Rows of the real plane-wave closed form: every orbital of the k pair gets eps_k phi."""
    L, n = 8.5, 12
    lat = np.diag([L] * 3)
    kset = np.array([[1, 0, 0], [0, 2, 1], [1, -1, 2]])
    phi = I.real_plane_wave_orbitals(kset, L, n)
    _, eps = O.closed_form_real(kset, lat)
    rows = [0, 3, 5]
    R = O.exchange_rows(phi, I.all_pairs(len(phi)), rows, lat)
    for r, b in enumerate(rows):
        assert rel(R[r], eps[b // 2] * phi[b]) < 1e-12


def test_exchange_rows_planted_slips_are_caught():
    """Plausible slips in a rows checker (the partner index taken as the row itself, diagonal
    pairs skipped, off-diagonal pairs counted only where the row is the first member) written
    out here as variants: each one disagrees with the full exchange that the real one matches."""
    phi, sub, lat = _rows_case()
    _, V = O.exchange(phi, sub, lat)
    v = O.coulomb_kernel(lat, phi.shape[1:])

    def variant(k, slip):
        out = np.zeros(phi.shape[1:])
        for i, j in sub:
            if i != k and j != k:
                continue
            if slip == "first_only" and i != k:
                continue
            if slip == "no_diag" and i == j:
                continue
            other = k if slip == "self" else (j if i == k else i)
            out -= 0.25 * O.pair_potential(O.pair_transform(phi[i], phi[j]), v) * phi[other]
        return out

    for k in (1, 4):
        assert rel(variant(k, "none"), V[k]) < 1e-13
        for slip in ("self", "no_diag", "first_only"):
            assert rel(variant(k, slip), V[k]) > 1e-3, (k, slip)
    assert rel(O.exchange_rows(phi, sub, [4], lat)[0], V[4]) < 1e-13
