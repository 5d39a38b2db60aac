"""FP64 CPU oracle for the adaptively compressed exchange (ACE) operator and the pair screen.

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously correct statements of what the ACE and
screening entry points compute.  Only the test suite, the smoke check and the CPU-baseline
leg of the benchmark may import it; the library never does, and it shares no code, table or
helper with the CUDA kernels.

ACE (paper Sec. 2.1, Eq. "vx_ace" and the definitions of P, W, L and M that follow it), for
real orbitals on the grid with the grid inner product <f|g> = (Omega/N) sum_p f(r_p) g(r_p):

* W_l = V_x psi_l                      (the exchange action of the occupied set);
* M_kl = <psi_k | V_x psi_l> = <psi_k | W_l>;
* L = Cholesky factor of -M            (lower triangular, positive diagonal);
* P = W L^{-T}                         (columns P_k; stored here as rows, P_rows = L^{-1} W_rows);
* V_x^ACE = - sum_k |P_k><P_k|,  so V_x^ACE chi = - sum_k P_k <P_k | chi>.

Readings where the paper is silent:

* M is symmetric in exact arithmetic for the full pair list (V_x is Hermitian); the Cholesky
  factorisation takes its symmetric part (M + M^T)/2, which also defines the operator for a
  screened pair list, where M itself is not symmetric.
* W is whatever exchange action the caller passes (here: the hybrid-scaled action of the
  exchange entry point, alpha included), so V_x^ACE reproduces alpha V_x on the occupied span.

Screening (Sec. 2.1, the s-MTACE overlap cut): s_ij = (Omega/N) sum_p |phi_i(r_p)| |phi_j(r_p)|,
a pair i <= j is kept when s_ij > cut; diagonal pairs are always kept.  Pairs come out in
row-major (i, then j) order.

SCDM localisation (the method the paper cites for its localised orbitals, Sec. 2.1; the paper
prints no algorithm, so this follows the published method): column-pivoted QR of Psi^T by greedy
residual-norm pivoting picks n grid points; Phi = Psi Q with Q from Psi(C, :)^T = Q R.

Linear algebra steps use numpy/scipy library routines (a matrix product, a Cholesky
factorisation, a triangular solve); nothing is blocked, fused or reordered.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np
import scipy.linalg

from .hfx_oracle import cell_volume


def _rows(f: np.ndarray) -> np.ndarray:
    """[n, n1, n2, n3] -> [n, N] view (grid point index fastest along z)."""
    f = np.asarray(f, dtype=np.float64)
    return f.reshape(f.shape[0], -1)


def grid_inner(f: np.ndarray, g: np.ndarray, lattice: np.ndarray) -> np.ndarray:
    """Matrix of grid inner products <f_a | g_b> = (Omega/N) sum_p f_a(r_p) g_b(r_p), [n_f, n_g]."""
    F, G = _rows(f), _rows(g)
    return (cell_volume(lattice) / F.shape[1]) * (F @ G.T)


def ace_build(phi: np.ndarray, w: np.ndarray, lattice: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """ACE construction (Sec. 2.1, Eq. vx_ace; P = W L^-T; L L^T = -M; M_kl = <psi_k|V_x psi_l>).

    phi, w: [n_orb, n1, n2, n3] occupied orbitals and their exchange action W_l = V_x psi_l.
    Returns (M [n_orb, n_orb] as defined, unsymmetrised; L lower triangular; P [n_orb, n1, n2, n3]).
    Raises numpy.linalg.LinAlgError when -(M + M^T)/2 is not positive definite.
    """
    M = grid_inner(phi, w, lattice)
    Msym = 0.5 * (M + M.T)
    L = np.linalg.cholesky(-Msym)
    P = scipy.linalg.solve_triangular(L, _rows(w), lower=True)  # L^-1 W_rows = (W L^-T)^T
    return M, L, P.reshape(np.shape(w))


def ace_apply(P: np.ndarray, psi: np.ndarray, lattice: np.ndarray) -> np.ndarray:
    """V_x^ACE psi_i = - sum_k P_k <P_k | psi_i> (Sec. 2.1, Eq. vx_ace), for every row psi_i."""
    X = grid_inner(psi, P, lattice)  # X[i, k] = <psi_i | P_k>
    return (-(X @ _rows(P))).reshape(np.shape(psi))


def overlap_screen(phi: np.ndarray, lattice: np.ndarray) -> np.ndarray:
    """s_ij = (Omega/N) sum_p |phi_i(r_p)| |phi_j(r_p)| (the s-MTACE cut quantity, Sec. 2.1)."""
    a = np.abs(_rows(phi))
    return grid_inner(a, a, lattice)


def screen_pairs(phi: np.ndarray, lattice: np.ndarray, cut: float) -> Tuple[np.ndarray, np.ndarray]:
    """Pairs i <= j with s_ij > cut, diagonal always kept, row-major order; returns (pairs int32 [P, 2], s)."""
    s = overlap_screen(phi, lattice)
    n = s.shape[0]
    out = [(i, j) for i in range(n) for j in range(i, n) if i == j or s[i, j] > cut]
    return np.array(out, dtype=np.int32).reshape(-1, 2), s


# ---------------------------------------------------------------------------------------------
# SCDM localisation (the selected-columns-of-the-density-matrix method the paper cites for its
# localised orbitals, Sec. 2.1): a column-pivoted QR factorisation of Psi^T picks n grid points
# C; the localised orthonormal orbitals are Phi = Psi Q with Q from the QR factorisation of the
# selected columns, Psi(C, :)^T = Q R (Q orthogonal, R upper triangular with positive diagonal).
# ---------------------------------------------------------------------------------------------

def scdm_pivots(phi: np.ndarray) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Column-pivoted QR of A = Psi^T ([n][N], column p = the n orbital values at grid point p) by
    greedy pivoting on residual column norms (Businger-Golub): at step j take the column of largest
    residual norm (lowest index on a tie), orthogonalise it against q_0..q_{j-1}, normalise to q_j,
    and remove its q_j component from every column.

    Returns (pivots [n] int64, Q [n][n] with columns q_j, diag(R) [n] = residual norms at the picks).
    """
    A = _rows(phi).copy()          # [n][N]; A[:, p] is column p
    n = A.shape[0]
    nu = np.sum(A * A, axis=0)     # squared residual column norms
    Q = np.zeros((n, n))
    piv = np.zeros(n, dtype=np.int64)
    rdiag = np.zeros(n)
    for j in range(n):
        p = int(np.argmax(nu))     # first maximum
        r = A[:, p].copy()
        rn = float(np.linalg.norm(r))
        q = r / rn
        Q[:, j] = q
        piv[j] = p
        rdiag[j] = rn
        A -= np.outer(q, q @ A)    # residual of every column
        nu = np.sum(A * A, axis=0)
        nu[piv[: j + 1]] = -1.0    # picked columns are exhausted
    return piv, Q, rdiag


def scdm_q_from_pivots(phi: np.ndarray, piv: np.ndarray) -> np.ndarray:
    """Q of the QR factorisation Psi(C, :)^T = Q R with diag(R) > 0, for given pivots C."""
    B = _rows(phi)[:, np.asarray(piv)]   # [n][n]: column j = orbital values at pivot j
    Q, R = np.linalg.qr(B)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s[None, :]


def scdm_localise(phi: np.ndarray, piv: np.ndarray = None) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """SCDM-localised orthonormal orbitals Phi = Psi Q (rows: Phi_j = sum_i Q[i][j] psi_i).

    Returns (pivots, Q, Phi [n, n1, n2, n3]); with `piv` given, Q is formed from those pivots."""
    if piv is None:
        piv, _, _ = scdm_pivots(phi)
    Q = scdm_q_from_pivots(phi, piv)
    Phi = (Q.T @ _rows(phi)).reshape(np.shape(phi))
    return np.asarray(piv), Q, Phi


def scdm_pivot_slack(phi: np.ndarray, piv: np.ndarray) -> np.ndarray:
    """For a proposed pivot sequence, the FP64 squared residual norm of each pick relative to the
    largest one available at that step (1 = a greedy choice; below 1 = how far from it)."""
    A = _rows(phi).copy()
    out = np.zeros(len(piv))
    taken = []
    for j, p in enumerate(piv):
        nu = np.sum(A * A, axis=0)
        nu[taken] = -1.0
        out[j] = nu[p] / nu.max()
        q = A[:, p] / np.linalg.norm(A[:, p])
        A -= np.outer(q, q @ A)
        taken.append(int(p))
    return out
