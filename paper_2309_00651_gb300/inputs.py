"""Seeded synthetic inputs for the Gamma-point exact-exchange path.

This module builds the occupied orbitals, the box and the orbital-pair lists that
both the CUDA path and the FP64 oracle consume.  It holds none of the exchange
arithmetic itself (no Coulomb kernel, no pair densities, no energies): only the
construction of real orbitals on the FFT grid, their Loewdin orthonormalisation
and the pair lists.

Workload shapes follow the paper's systems (Sec. "Computational Details" and the
system table): 4 doubly occupied orbitals per H2O, liquid-water density (32 H2O in
a 9.85 A box, 128 H2O in a 15.64 A box), an 80 Ry (= 40 Ha) wavefunction cutoff.

Orbital recipes
---------------
* ``pw``: plane-wave coefficients c(G) drawn N(0,1) (real and imaginary parts) on
  the cutoff sphere |G|^2/2 < ecut, damped by exp(-|G|^2/8), made Hermitian
  (c(-G) = conj c(G)) so that phi(r) is real.
* ``gauss``: the analytic periodic Fourier transform of a normalised Gaussian of
  width sigma centred at c, c(G) ~ exp(-sigma^2 |G|^2 / 2) exp(-i G.c), on the same
  cutoff sphere.  Centres: 4 per molecule, 0.7 bohr from the molecule site along
  the even-parity tetrahedron (+-1,+-1,+-1)/sqrt(3); molecule sites are the first
  N_mol points of a seeded permutation of a ceil(N_mol^(1/3))^3 simple cubic
  lattice, jittered uniformly by +-0.25 lattice spacings.
* Both are Loewdin-orthonormalised on the grid: S_ij = (Omega/N) sum_r phi_i phi_j,
  phi <- S^(-1/2) phi.

Grid convention: phi has shape [n_orb, n1, n2, n3], point r_p = L p / n, the last
axis (z) contiguous.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.529177210903
# Volume per H2O at 1 g/cm^3: 30 A^3 (the paper's 9.85 A / 32 H2O and 15.64 A / 128 H2O boxes).
WATER_VOLUME_BOHR3 = 30.0 * BOHR_PER_ANGSTROM ** 3  # ~202.4 bohr^3


@dataclasses.dataclass(frozen=True)
class Workload:
    """One exchange workload: box, grid, orbital recipe and pair-list rule."""

    name: str
    n_orb: int
    L: float                      # cubic box edge, bohr
    n: int                        # grid points per edge (n1 = n2 = n3)
    ecut: float                   # Ha, PW cutoff used to build the orbitals
    kind: str                     # "pw" or "gauss"
    seed: int = 0
    sigma: float = 1.2            # Gaussian width (bohr) for kind == "gauss"
    screen: Optional[float] = None  # keep pairs with s_ij > screen (None: all pairs)

    @property
    def grid(self) -> Tuple[int, int, int]:
        return (self.n, self.n, self.n)

    @property
    def lattice(self) -> np.ndarray:
        return np.diag([self.L, self.L, self.L]).astype(np.float64)

    @property
    def volume(self) -> float:
        return float(self.L ** 3)


# The five workloads the exchange path is measured and checked on.
WORKLOADS = {
    # 16 random-PW orbitals, L = 10 bohr, 32^3, Ecut = 20 Ha, all 136 pairs.
    "pw16_n32": Workload("pw16_n32", 16, 10.0, 32, 20.0, "pw", seed=0),
    # 32 H2O water box (paper's 9.85 A cell = 18.6 bohr), 128 orbitals, 72^3, 40 Ha, 8256 pairs.
    "water32_n72": Workload("water32_n72", 128, 18.6, 72, 40.0, "gauss", seed=0, sigma=1.2),
    # 64 H2O box (paper's Fe3+/64-water cell size), 256 random-PW orbitals, 96^3, 20 Ha.
    "water64_n96": Workload("water64_n96", 256, 23.5, 96, 20.0, "pw", seed=0),
    # the 96^3 box with 64 random-PW orbitals (16 H2O worth): a profiling case of the 96^3 kernels
    # whose transforms and orbital copies still exceed L2 (2080 pairs, about 2 GB on the device)
    "water16_n96": Workload("water16_n96", 64, 23.5, 96, 20.0, "pw", seed=0),
    # small case of the water-box workload for profiling captures: 32 orbitals in the same
    # 18.6 bohr cell and 72^3 grid (528 pairs; one batch of transforms still exceeds L2).
    "water8_n72": Workload("water8_n72", 32, 18.6, 72, 40.0, "gauss", seed=0, sigma=1.2),
    # 128 H2O box (paper's 15.64 A cell = 29.6 bohr), 512 Gaussian orbitals, 128^3, 40 Ha,
    # overlap-screened pair list s_ij > 1e-6.
    "water128_n128": Workload("water128_n128", 512, 29.6, 128, 40.0, "gauss", seed=0,
                              sigma=1.5, screen=1e-6),
}


def smooth_even_at_least(x: float) -> int:
    """Smallest even integer >= x whose prime factors are all in {2, 3, 5}."""
    n = max(2, int(math.ceil(x - 1e-12)))
    while True:
        if n % 2 == 0:
            m = n
            for p in (2, 3, 5):
                while m % p == 0:
                    m //= p
            if m == 1:
                return n
        n += 1


def batched_workloads(count: int = 24, seed: int = 0, lo: int = 32, hi: int = 256) -> List[Workload]:
    """The uneven batch: `count` independent water-density boxes.

    N_orb ~ U{lo..hi}; L = (30 A^3 * N_orb / 4)^(1/3); grid = smallest even
    {2,3,5}-smooth n >= 4.03 L (no aliasing of pair products at Ecut = 20 Ha);
    random-PW orbitals with sub-seeds spawned from SeedSequence(seed).
    """
    ss = np.random.SeedSequence(seed)
    rng = np.random.default_rng(ss)
    n_orbs = rng.integers(lo, hi + 1, size=count)
    children = ss.spawn(count)
    out = []
    for k, (no, child) in enumerate(zip(n_orbs, children)):
        no = int(no)
        L = (WATER_VOLUME_BOHR3 * no / 4.0) ** (1.0 / 3.0)
        n = smooth_even_at_least(4.03 * L)
        sub_seed = int(child.generate_state(1)[0])
        out.append(Workload(f"batch{k:02d}_o{no}_n{n}", no, float(L), n, 20.0, "pw", seed=sub_seed))
    return out


# ----------------------------------------------------------------------------------------
# reciprocal-space helpers (input construction only)
# ----------------------------------------------------------------------------------------

def _gvec_sq(L: float, n: int) -> np.ndarray:
    """|G|^2 on the full FFT grid (fftfreq order), cubic box."""
    m = np.fft.fftfreq(n, d=1.0 / n)
    g = 2.0 * np.pi * m / L
    return g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2


def _gvec(L: float, n: int):
    m = np.fft.fftfreq(n, d=1.0 / n)
    g = 2.0 * np.pi * m / L
    return g


def _neg_index(n: int) -> np.ndarray:
    return (-np.arange(n)) % n


def _hermitise(c: np.ndarray) -> np.ndarray:
    """Return (c + conj(c(-G)))/2 so that the inverse transform is real."""
    n1, n2, n3 = c.shape[-3:]
    cm = c[..., _neg_index(n1), :, :][..., :, _neg_index(n2), :][..., :, :, _neg_index(n3)]
    return 0.5 * (c + np.conj(cm))


def _coeffs_to_real(c: np.ndarray) -> np.ndarray:
    """phi(r_p) = sum_G c(G) exp(i G.r_p) for Hermitian c (numpy inverse FFT times N)."""
    n = c.shape[-1] * c.shape[-2] * c.shape[-3]
    return np.real(np.fft.ifftn(c, axes=(-3, -2, -1))) * n


def random_pw_orbitals(n_orb: int, L: float, n: int, ecut: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    g2 = _gvec_sq(L, n)
    sphere = 0.5 * g2 < ecut
    amp = np.exp(-g2 / 8.0) * sphere
    phi = np.empty((n_orb, n, n, n), dtype=np.float64)
    for i in range(n_orb):
        c = (rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))) * amp
        phi[i] = _coeffs_to_real(_hermitise(c))
    return phi


def water_sites(n_mol: int, L: float, rng: np.random.Generator) -> np.ndarray:
    m = int(math.ceil(n_mol ** (1.0 / 3.0) - 1e-12))
    a = L / m
    idx = np.array([(i, j, k) for i in range(m) for j in range(m) for k in range(m)], dtype=np.float64)
    perm = rng.permutation(len(idx))[:n_mol]
    sites = (idx[perm] + 0.5) * a
    sites += rng.uniform(-0.25 * a, 0.25 * a, size=sites.shape)
    return np.mod(sites, L)


TETRAHEDRON = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) / math.sqrt(3.0)


def gaussian_orbitals(n_orb: int, L: float, n: int, ecut: float, sigma: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    n_mol = (n_orb + 3) // 4
    sites = water_sites(n_mol, L, rng)
    centres = (sites[:, None, :] + 0.7 * TETRAHEDRON[None, :, :]).reshape(-1, 3)[:n_orb]
    g = _gvec(L, n)
    g2 = g[:, None, None] ** 2 + g[None, :, None] ** 2 + g[None, None, :] ** 2
    amp = np.exp(-0.5 * sigma * sigma * g2) * (0.5 * g2 < ecut)
    phi = np.empty((n_orb, n, n, n), dtype=np.float64)
    for i, c in enumerate(centres):
        phase = np.exp(-1j * (g[:, None, None] * c[0] + g[None, :, None] * c[1] + g[None, None, :] * c[2]))
        phi[i] = _coeffs_to_real(amp * phase)
    return phi


def loewdin(phi: np.ndarray, volume: float) -> Tuple[np.ndarray, float]:
    """Symmetric orthonormalisation on the grid; returns (phi S^-1/2, cond(S))."""
    n_orb = phi.shape[0]
    npts = phi[0].size
    flat = phi.reshape(n_orb, npts)
    S = (volume / npts) * (flat @ flat.T)
    w, U = np.linalg.eigh(S)
    cond = float(w.max() / w.min())
    S_mhalf = (U * (1.0 / np.sqrt(w))) @ U.T
    out = (S_mhalf @ flat).reshape(phi.shape)
    return out, cond


def all_pairs(n_orb: int) -> np.ndarray:
    """Unordered pairs (i, j), i <= j, row-major: n_orb (n_orb + 1) / 2 entries, int32 [P, 2]."""
    i, j = np.triu_indices(n_orb)
    return np.stack([i, j], axis=1).astype(np.int32)


def screened_pairs(phi: np.ndarray, volume: float, threshold: float) -> np.ndarray:
    """Pairs i <= j with s_ij = (Omega/N) sum_r |phi_i||phi_j| > threshold (diagonal always kept).

    The overlap-screening rule of s-MTACE (Sec. 2.1) with the grid sum in place of the integral.
    """
    n_orb = phi.shape[0]
    a = np.abs(phi.reshape(n_orb, -1))
    s = (volume / a.shape[1]) * (a @ a.T)
    i, j = np.triu_indices(n_orb)
    keep = (s[i, j] > threshold) | (i == j)
    return np.stack([i[keep], j[keep]], axis=1).astype(np.int32)


def make_orbitals(w: Workload) -> Tuple[np.ndarray, float]:
    if w.kind == "pw":
        raw = random_pw_orbitals(w.n_orb, w.L, w.n, w.ecut, w.seed)
    elif w.kind == "gauss":
        raw = gaussian_orbitals(w.n_orb, w.L, w.n, w.ecut, w.sigma, w.seed)
    else:
        raise ValueError(f"unknown orbital kind {w.kind!r}")
    return loewdin(raw, w.volume)


def make_workload(w: Workload):
    """Return (phi [n_orb,n,n,n] float64, pairs int32 [P,2], info dict)."""
    phi, cond = make_orbitals(w)
    if w.screen is None:
        pairs = all_pairs(w.n_orb)
    else:
        pairs = screened_pairs(phi, w.volume, w.screen)
    info = {"name": w.name, "n_orb": w.n_orb, "L": w.L, "n": w.n, "ecut": w.ecut,
            "kind": w.kind, "seed": w.seed, "cond_S": cond, "n_pairs": int(len(pairs))}
    return phi, pairs, info


def save_workload(path: str, w: Workload, phi: np.ndarray, pairs: np.ndarray, info: Optional[dict] = None) -> None:
    """Write a generated workload to one .npz file: the orbitals, the pair list and, as JSON, the
    workload record (seed included) plus make_workload's info (cond(S), pair count).  A run can then
    restart from exactly these inputs, or rebuild them from the record (make_workload(w) reproduces
    the arrays bit for bit)."""
    import json
    meta = {"format": 1, "workload": dataclasses.asdict(w), "info": info or {}}
    np.savez(path, phi=np.ascontiguousarray(phi, dtype=np.float64), pairs=np.ascontiguousarray(pairs, dtype=np.int32),
             meta=np.array(json.dumps(meta)))


def load_workload(path: str) -> Tuple[Workload, np.ndarray, np.ndarray, dict]:
    """Read a file written by save_workload: (workload record, phi, pairs, info)."""
    import json
    with np.load(path, allow_pickle=False) as f:
        meta = json.loads(str(f["meta"]))
        if meta.get("format") != 1:
            raise ValueError(f"{path}: unknown workload file format {meta.get('format')!r}")
        return Workload(**meta["workload"]), f["phi"].copy(), f["pairs"].copy(), meta["info"]


def random_pairs_subset(pairs: np.ndarray, k: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(pairs), size=min(k, len(pairs)), replace=False))
    return pairs[idx]


# ----------------------------------------------------------------------------------------
# closed-form test orbitals (plane waves), used by both the oracle pins and GPU parity
# ----------------------------------------------------------------------------------------

def real_plane_wave_orbitals(kset: np.ndarray, L: float, n: int) -> np.ndarray:
    """sqrt(2/Omega) cos(k.r) and sqrt(2/Omega) sin(k.r) for each integer k in kset (k = 2 pi m / L)."""
    p = np.arange(n) / n  # fractional coordinate
    out = []
    for m in kset:
        arg = 2.0 * np.pi * (m[0] * p[:, None, None] + m[1] * p[None, :, None] + m[2] * p[None, None, :])
        out.append(np.sqrt(2.0 / L ** 3) * np.cos(arg))
        out.append(np.sqrt(2.0 / L ** 3) * np.sin(arg))
    return np.array(out)


def complex_plane_wave_orbitals(kset: np.ndarray, L: float, n: int) -> np.ndarray:
    """exp(i k.r)/sqrt(Omega) for each integer k in kset."""
    p = np.arange(n) / n
    out = []
    for m in kset:
        arg = 2.0 * np.pi * (m[0] * p[:, None, None] + m[1] * p[None, :, None] + m[2] * p[None, None, :])
        out.append(np.exp(1j * arg) / np.sqrt(L ** 3))
    return np.array(out)


def skewed_basis_case(n: int = 24, L: float = 8.0, n_orb: int = 4, seed: int = 7):
    """One cubic cell written in two bases: rows a1, a2, a3 and the skewed rows a1, a1 + a2, a3.

    Grid point p of the skewed basis is r = ((p1 + p2)/n) a1 + (p2/n) a2 + (p3/n) a3, i.e. point
    ((p1 + p2) mod n, p2, p3) of the cubic one, so phi_s[p1, p2] = phi[(p1 + p2) mod n, p2] is the
    same periodic function.  The orbitals carry |m| <= 2 per axis, their pair densities |m| <= 4,
    which in skewed indices is (m1, m1 + m2) with |m1 + m2| <= 8 < n/2: no Fourier coefficient of
    a pair density lies where the two bases fold frequencies differently, so the discrete exchange
    is the same in both.  Returns (phi, phi_s, lattice, skewed lattice, src) with
    src[p1, p2] = (p1 + p2) mod n."""
    ecut = 0.5 * (2 * math.pi * 2.5 / L) ** 2  # |m|^2 < 6.25
    raw = random_pw_orbitals(n_orb, L, n, ecut=ecut, seed=seed)
    phi, _ = loewdin(raw, L ** 3)
    lat = np.diag([L, L, L])
    lat_s = np.array([[L, 0.0, 0.0], [L, L, 0.0], [0.0, 0.0, L]])
    p = np.arange(n)
    src = (p[:, None] + p[None, :]) % n
    phi_s = np.ascontiguousarray(phi[:, src, p[None, :], :])
    return phi, phi_s, lat, lat_s, src


def _make_workload_task(w: Workload):
    return make_workload(w)


def make_workloads_parallel(ws: List[Workload], procs: Optional[int] = None):
    """make_workload for several workloads at once, one spawned process per host core (spawn, so
    it is safe in a process that has initialised CUDA).  Every workload is built from its own
    seed, so the arrays equal those of make_workload called one by one; returned in order."""
    import multiprocessing as mp
    import os
    procs = procs or max(1, min(len(ws), len(os.sched_getaffinity(0))))
    if procs == 1 or len(ws) == 1:
        return [make_workload(w) for w in ws]
    # largest first, so the longest jobs do not start last
    order = sorted(range(len(ws)), key=lambda k: -ws[k].n_orb * ws[k].n ** 3)
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_make_workload_task, [ws[k] for k in order], chunksize=1)
    out = [None] * len(ws)
    for k, r in zip(order, res):
        out[k] = r
    return out
