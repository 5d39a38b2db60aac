"""FP64 CPU oracle for the Gamma-point Hartree-Fock exact-exchange evaluation.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct
statement of what the exchange path computes.  Only the test suite, the smoke
check and the CPU-baseline leg of the benchmark may import it; the library never
does, and it shares no code, table or helper with the CUDA kernels.

What it computes (paper Sec. 2.1, Eqs. "vx", "vij", "HFX"):

* occupied real orbitals phi_i(r_p) on the grid r_p = A^T (p / n), p in {0..n-1}^3;
* pair density           rho_ij(r) = phi_i(r) phi_j(r);
* its transform          F_ij(G)   = sum_p rho_ij(r_p) exp(-i G.r_p)   (numpy.fft.fftn);
* Coulomb kernel         v(G) = 4 pi / |G|^2, v(0) = 0 (optionally also 0 outside
                          the pair-density sphere |G|^2/2 >= 4 ecut);
* pair potential (Eq. vij, solved on the grid by FFT)
                          v_ij(r_p) = (1/N) sum_G v(G) F_ij(G) exp(i G.r_p);
* exchange energy (Eq. HFX, with the hybrid fraction alpha and the 1/2 of an ordered
  double sum)             E_x = -(alpha/2) (Omega/N^2) sum_{i,j ordered} sum_G v(G) |F_ij(G)|^2;
* exchange action (Eq. vx, scaled by alpha)
                          (V_x phi)_i(r) = -alpha sum_j v_ij(r) phi_j(r).

A pair list holds unordered pairs i <= j; an off-diagonal pair stands for (i,j) and
(j,i) (weight 2, and it feeds both V_i and V_j since v_ij = v_ji), a diagonal pair for
itself (weight 1).

Transforms: a brute-force O(N^2) direct DFT (``dft3_direct``) on grids whose edges are
all <= 12, ``numpy.fft`` beyond.  Everything is float64 / complex128.
"""
from __future__ import annotations

import math
from typing import Iterable, Optional, Sequence, Tuple

import numpy as np

DIRECT_DFT_MAX_EDGE = 12


# ------------------------------------------------------------------------------------
# geometry and Coulomb kernel
# ------------------------------------------------------------------------------------

def reciprocal_vectors(lattice: np.ndarray) -> np.ndarray:
    """Rows b_k with a_i . b_k = 2 pi delta_ik, for lattice rows a_i (bohr)."""
    A = np.asarray(lattice, dtype=np.float64)
    return 2.0 * np.pi * np.linalg.inv(A).T


def cell_volume(lattice: np.ndarray) -> float:
    return float(abs(np.linalg.det(np.asarray(lattice, dtype=np.float64))))


def frequencies(n: int) -> np.ndarray:
    """Integer frequency m of FFT output index k: m = k for k <= n/2, k - n above."""
    k = np.arange(n)
    return np.where(k <= n // 2, k, k - n)


def g_squared(lattice: np.ndarray, grid: Sequence[int]) -> np.ndarray:
    """|G|^2 for G = m1 b1 + m2 b2 + m3 b3 on the full grid (FFT output order)."""
    B = reciprocal_vectors(lattice)
    m1, m2, m3 = (frequencies(n).astype(np.float64) for n in grid)
    G = (m1[:, None, None, None] * B[0] + m2[None, :, None, None] * B[1]
         + m3[None, None, :, None] * B[2])
    return np.sum(G * G, axis=-1)


def coulomb_kernel(lattice: np.ndarray, grid: Sequence[int], sphere_ecut: Optional[float] = None) -> np.ndarray:
    """v(G) = 4 pi / |G|^2 with v(0) = 0; with ``sphere_ecut`` also v = 0 where |G|^2/2 >= 4 ecut."""
    g2 = g_squared(lattice, grid)
    v = np.zeros_like(g2)
    nz = g2 > 0.0
    v[nz] = 4.0 * np.pi / g2[nz]
    if sphere_ecut is not None:
        v[0.5 * g2 >= 4.0 * sphere_ecut] = 0.0
    return v


# ------------------------------------------------------------------------------------
# transforms
# ------------------------------------------------------------------------------------

def dft3_direct(f: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Brute-force 3D DFT: F(k) = sum_p f(p) exp(-+ 2 pi i sum_d k_d p_d / n_d) (no 1/N).

    Builds the full N x N phase matrix, so it is only meant for tiny grids.
    """
    f = np.asarray(f, dtype=np.complex128)
    n1, n2, n3 = f.shape
    idx = np.indices((n1, n2, n3)).reshape(3, -1).T.astype(np.float64)  # [N, 3] integer points
    frac = idx / np.array([n1, n2, n3], dtype=np.float64)
    sign = 1.0 if inverse else -1.0
    phase = np.exp(sign * 2j * np.pi * (idx @ frac.T))  # [k, p]
    return (phase @ f.reshape(-1)).reshape(n1, n2, n3)


def _tiny(shape: Sequence[int]) -> bool:
    return max(shape) <= DIRECT_DFT_MAX_EDGE


def fft3(f: np.ndarray, direct: Optional[bool] = None) -> np.ndarray:
    """Unnormalised forward transform (the convention of numpy.fft.fftn)."""
    if direct is None:
        direct = _tiny(f.shape)
    return dft3_direct(f) if direct else np.fft.fftn(f)


def ifft3(F: np.ndarray, direct: Optional[bool] = None) -> np.ndarray:
    """Normalised inverse transform (1/N included, the convention of numpy.fft.ifftn)."""
    if direct is None:
        direct = _tiny(F.shape)
    if direct:
        return dft3_direct(F, inverse=True) / F.size
    return np.fft.ifftn(F)


# ------------------------------------------------------------------------------------
# the exchange evaluation
# ------------------------------------------------------------------------------------

def pair_transform(phi_i: np.ndarray, phi_j: np.ndarray, direct: Optional[bool] = None) -> np.ndarray:
    """F_ij = F[rho_ij] with rho_ij = phi_i phi_j (Eq. vij: the density whose potential is taken)."""
    return fft3(phi_i * phi_j, direct)


def pair_potential(F: np.ndarray, v: np.ndarray, direct: Optional[bool] = None) -> np.ndarray:
    """v_ij(r_p) = (1/N) sum_G v(G) F_ij(G) exp(i G.r_p): the Poisson solution of Eq. vij (real for real phi)."""
    return np.real(ifft3(v * F, direct))


def pair_energy_sum(F: np.ndarray, v: np.ndarray) -> float:
    """e_ij = sum_G v(G) |F_ij(G)|^2 (the unscaled per-pair term of Eq. HFX)."""
    return float(np.sum(v * (F.real * F.real + F.imag * F.imag)))


def energy_scale(lattice: np.ndarray, grid: Sequence[int], alpha: float) -> float:
    """E_x = scale * sum_ordered e_ij with scale = -(alpha/2) Omega / N^2."""
    N = int(np.prod(grid))
    return -0.5 * alpha * cell_volume(lattice) / float(N) ** 2


def _check_pairs(pairs: np.ndarray, n_orb: int) -> np.ndarray:
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    if pairs.size and (pairs.min() < 0 or pairs.max() >= n_orb or np.any(pairs[:, 0] > pairs[:, 1])):
        raise ValueError("pair list entries must satisfy 0 <= i <= j < n_orb")
    return pairs


def exchange(phi: np.ndarray, pairs: np.ndarray, lattice: np.ndarray, alpha: float = 0.25,
             sphere_ecut: Optional[float] = None, want_v: bool = True,
             direct: Optional[bool] = None) -> Tuple[float, Optional[np.ndarray]]:
    """E_x and V_x phi for real orbitals phi [n_orb, n1, n2, n3] over an unordered pair list.

    For each listed pair (i, j): rho_ij -> F_ij -> e_ij and v_ij; E gets weight 2 (i != j)
    or 1 (i == j); V_i -= alpha v_ij phi_j and, for i != j, V_j -= alpha v_ij phi_i.
    """
    phi = np.asarray(phi, dtype=np.float64)
    n_orb = phi.shape[0]
    grid = phi.shape[1:]
    pairs = _check_pairs(pairs, n_orb)
    v = coulomb_kernel(lattice, grid, sphere_ecut)
    total = 0.0
    V = np.zeros_like(phi) if want_v else None
    for i, j in pairs:
        F = pair_transform(phi[i], phi[j], direct)
        weight = 1.0 if i == j else 2.0
        total += weight * pair_energy_sum(F, v)
        if want_v:
            vij = pair_potential(F, v, direct)
            V[i] -= alpha * vij * phi[j]
            if i != j:
                V[j] -= alpha * vij * phi[i]
    return energy_scale(lattice, grid, alpha) * total, V


def pair_energy_terms(phi: np.ndarray, pairs: np.ndarray, lattice: np.ndarray,
                      sphere_ecut: Optional[float] = None) -> np.ndarray:
    """Unscaled, unweighted e_ij = sum_G v |F_ij|^2 for each listed pair."""
    phi = np.asarray(phi, dtype=np.float64)
    pairs = _check_pairs(pairs, phi.shape[0])
    v = coulomb_kernel(lattice, phi.shape[1:], sphere_ecut)
    return np.array([pair_energy_sum(pair_transform(phi[i], phi[j]), v) for i, j in pairs])


def exchange_rows(phi: np.ndarray, pairs: np.ndarray, rows: Iterable[int], lattice: np.ndarray,
                  alpha: float = 0.25, sphere_ecut: Optional[float] = None) -> np.ndarray:
    """(V_x phi)_k for the orbitals k in ``rows`` only, from the listed pairs that contain k."""
    phi = np.asarray(phi, dtype=np.float64)
    pairs = _check_pairs(pairs, phi.shape[0])
    v = coulomb_kernel(lattice, phi.shape[1:], sphere_ecut)
    rows = list(rows)
    out = np.zeros((len(rows),) + phi.shape[1:])
    for r, k in enumerate(rows):
        for i, j in pairs:
            if i != k and j != k:
                continue
            other = j if i == k else i
            vij = pair_potential(pair_transform(phi[i], phi[j]), v)
            out[r] -= alpha * vij * phi[other]
    return out


def exchange_complex(phi: np.ndarray, lattice: np.ndarray, alpha: float = 0.25,
                     direct: Optional[bool] = None) -> Tuple[float, np.ndarray]:
    """Complex-orbital form over all ordered pairs: rho_ij = conj(phi_i) phi_j,
    E_x = -(alpha/2)(Omega/N^2) sum_ij sum_G v |F_ij|^2, (V_x phi)_i = -alpha sum_j v[conj(phi_j) phi_i] phi_j.

    Used for the plane-wave closed form; the GPU path is real-only.
    """
    phi = np.asarray(phi, dtype=np.complex128)
    n_orb = phi.shape[0]
    grid = phi.shape[1:]
    v = coulomb_kernel(lattice, grid)
    total = 0.0
    V = np.zeros_like(phi)
    for i in range(n_orb):
        for j in range(n_orb):
            F = fft3(np.conj(phi[i]) * phi[j], direct)
            total += pair_energy_sum(F, v)
            # potential of conj(phi_j) phi_i acting on phi_j, accumulated into V_i
            Fji = fft3(np.conj(phi[j]) * phi[i], direct)
            V[i] -= alpha * ifft3(v * Fji, direct) * phi[j]
    return energy_scale(lattice, grid, alpha) * total, V


# ------------------------------------------------------------------------------------
# closed forms (plane-wave orbitals), stated from the definition above
# ------------------------------------------------------------------------------------

def _inv_sq(m: np.ndarray, lattice: np.ndarray) -> float:
    """S(m) = 1/|G(m)|^2 with S(0) = 0 for an integer wavevector m."""
    if not np.any(m):
        return 0.0
    G = np.asarray(m, dtype=np.float64) @ reciprocal_vectors(lattice)
    return 1.0 / float(G @ G)


def closed_form_complex(kset: np.ndarray, lattice: np.ndarray, alpha: float = 0.25):
    """phi_i = exp(i k_i.r)/sqrt(Omega): E_x = -(alpha/2)(4 pi/Omega) sum_{i != j} 1/|k_i - k_j|^2,
    V_x phi_i = eps_i phi_i with eps_i = -alpha (4 pi / Omega) sum_{j != i} 1/|k_i - k_j|^2."""
    omega = cell_volume(lattice)
    K = np.asarray(kset)
    eps = np.array([-alpha * 4.0 * math.pi / omega * sum(_inv_sq(K[i] - K[j], lattice)
                    for j in range(len(K)) if j != i) for i in range(len(K))])
    return 0.5 * float(np.sum(eps)), eps


def closed_form_real(kset: np.ndarray, lattice: np.ndarray, alpha: float = 0.25):
    """Orbitals sqrt(2/Omega) cos(k.r), sqrt(2/Omega) sin(k.r), k in K (none equal or opposite):
    E_x = -alpha (4 pi/Omega) sum_{k,q in K} [S(k-q) + S(k+q)], and both members of the k pair
    get V_x phi = eps_k phi with eps_k = -alpha (4 pi/Omega) sum_{q in K} [S(k-q) + S(k+q)]."""
    omega = cell_volume(lattice)
    K = np.asarray(kset)
    eps = np.array([-alpha * 4.0 * math.pi / omega * sum(_inv_sq(K[a] - K[b], lattice) + _inv_sq(K[a] + K[b], lattice)
                    for b in range(len(K))) for a in range(len(K))])
    return float(np.sum(eps)), eps
