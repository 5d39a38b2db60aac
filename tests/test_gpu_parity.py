"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: the FP64 path must match to 1e-8 relative and the FP32 path to 1e-6 relative in
E_x and in ||V_x phi||_F (the stated accuracy targets of the two paths).  Integer work (pair
staging) is checked exactly through its effect: every listed pair is counted once.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hfx_oracle as O  # noqa: E402
from paper_2309_00651_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-8, "fp32": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_00651_gb300 import build
    build.build()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def maxrel(a, b):
    """max |a - b| / max |b|: a localised error (one plane, one ragged chunk) is not diluted by the
    grid size the way it is in a Frobenius norm."""
    return float(np.max(np.abs(np.ravel(a - b))) / max(np.max(np.abs(np.ravel(b))), 1e-300))


def assert_v_close(V, V_ref, tol):
    assert rel(V, V_ref) <= tol
    assert maxrel(V, V_ref) <= tol


def run_gpu(phi, pairs, lattice, prec, **kw):
    from paper_2309_00651_gb300 import hfx
    ex = hfx.Exchange(lattice, phi.shape[1:], alpha=kw.pop("alpha", 0.25), precision=prec,
                      kernel=kw.pop("kernel", "coulomb"), ecut=kw.pop("ecut", 0.0))
    phi_d = torch.from_numpy(np.ascontiguousarray(phi)).cuda()
    pairs_d = torch.from_numpy(np.ascontiguousarray(pairs, dtype=np.int32)).cuda()
    E, V = ex.apply(phi_d, pairs_d, **kw)
    ex.sync_status()
    out = (E.item(), None if V is None else V.cpu().numpy())
    ex.close()
    return out


def band_limited(n_orb, n, L, seed, frac=0.25):
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=0.5 * (2 * math.pi * (frac * n + 0.5) / L) ** 2, seed=seed)
    phi, _ = I.loewdin(raw, L ** 3)
    return phi


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_real_plane_wave_closed_form(prec):
    L, n = 8.5, 16
    lat = np.diag([L] * 3)
    kset = np.array([[1, 0, 0], [0, 2, 1], [1, -1, 2], [2, 1, -1]])
    phi = I.real_plane_wave_orbitals(kset, L, n)
    E, V = run_gpu(phi, I.all_pairs(len(phi)), lat, prec)
    E_ref, eps = O.closed_form_real(kset, lat)
    assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
    for b in range(len(phi)):
        assert rel(V[b], eps[b // 2] * phi[b]) <= 10 * TOL[prec]
        assert maxrel(V[b], eps[b // 2] * phi[b]) <= 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,n_orb", [(8, 5), (18, 13), (30, 9), (24, 17)])
def test_small_grids_all_pairs(prec, n, n_orb):
    """Several tiles, ragged blocks (n_orb not a multiple of the block), ragged z-chunks."""
    L = 0.6 * n
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=n + n_orb)
    pairs = I.all_pairs(n_orb)
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    E, V = run_gpu(phi, pairs, lat, prec)
    assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
    assert_v_close(V, V_ref, TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_orthorhombic_non_cubic_grid(prec):
    Ls = (9.0, 7.5, 11.0)
    grid = (20, 16, 24)
    lat = np.diag(Ls)
    rng = np.random.default_rng(3)
    raw = rng.standard_normal((7,) + grid)
    phi, _ = I.loewdin(raw, float(np.prod(Ls)))
    pairs = I.all_pairs(7)
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    E, V = run_gpu(phi, pairs, lat, prec)
    assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
    assert_v_close(V, V_ref, TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_triclinic_cell(prec):
    """A general (non-orthogonal) cell: the reciprocal vectors and |G| of the Coulomb table come
    from the full lattice matrix on both sides."""
    lat = np.array([[9.0, 0.0, 0.0], [2.5, 8.0, 0.0], [1.0, -1.5, 10.0]])
    grid = (20, 18, 24)
    rng = np.random.default_rng(11)
    raw = rng.standard_normal((6,) + grid)
    phi, _ = I.loewdin(raw, abs(float(np.linalg.det(lat))))
    pairs = I.all_pairs(6)
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    E, V = run_gpu(phi, pairs, lat, prec)
    assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
    assert_v_close(V, V_ref, TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_skewed_basis_of_the_same_cell(prec):
    """The cubic cell written in the skewed basis a1, a1 + a2, a3 with the grid data index-mapped
    accordingly (band-limited orbitals, so no pair density reaches where the two bases fold
    frequencies differently): against the oracle in the skewed basis, and against the GPU's own
    result in the cubic basis mapped to the skewed grid."""
    phi, phi_s, lat, lat_s, src = I.skewed_basis_case()
    n = phi.shape[1]
    pairs = I.all_pairs(phi.shape[0])
    E_ref, V_ref = O.exchange(phi_s, pairs, lat_s)
    E_s, V_s = run_gpu(phi_s, pairs, lat_s, prec)
    assert abs(E_s - E_ref) <= TOL[prec] * abs(E_ref)
    assert_v_close(V_s, V_ref, TOL[prec])
    E, V = run_gpu(phi, pairs, lat, prec)
    assert abs(E_s - E) <= TOL[prec] * abs(E)
    assert_v_close(V_s, V[:, src, np.arange(n)[None, :], :], TOL[prec])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("grid,n_orb", [((4, 4, 4), 3), ((2, 4, 6), 2), ((6, 2, 4), 5), ((8, 8, 8), 1)])
def test_degenerate_sizes(prec, grid, n_orb):
    """The smallest grids (one radix per axis, an edge of 2, z rows shorter than a z-chunk) and a
    single orbital (one diagonal pair), against the oracle's brute-force DFT."""
    Ls = (5.0, 6.0, 7.0)
    lat = np.diag(Ls)
    rng = np.random.default_rng(sum(grid) + n_orb)
    phi, _ = I.loewdin(rng.standard_normal((n_orb,) + grid), float(np.prod(Ls)))
    pairs = I.all_pairs(n_orb)
    E_ref, V_ref = O.exchange(phi, pairs, lat, direct=True)
    E, V = run_gpu(phi, pairs, lat, prec)
    assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
    assert_v_close(V, V_ref, TOL[prec])


@pytest.mark.parametrize("n,n_orb", [(32, 16), (24, 11)])
def test_fp32_orbitals_flag(n, n_orb):
    """HFX_ORBITALS_F32: FP32 orbitals taken straight from the caller give bit for bit what the FP64
    orbitals give after the library's own round-to-nearest FP32 copy (a compile-time grid with the
    TMA dense pass, and a runtime-geometry grid), in one call and in a batched call."""
    from paper_2309_00651_gb300 import hfx
    L = 0.6 * n
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=21 + n)
    pairs = I.all_pairs(n_orb)
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    ex = hfx.Exchange(lat, (n, n, n), alpha=0.25, precision="fp32")
    phi64 = torch.from_numpy(phi).cuda()
    phi32 = phi64.float().contiguous()
    pairs_d = torch.from_numpy(pairs).cuda()
    E1, V1 = ex.apply(phi64, pairs_d)
    E2, V2 = ex.apply(phi32, pairs_d)
    ex.sync_status()
    assert E2.item() == E1.item() and torch.equal(V2, V1)
    assert abs(E2.item() - E_ref) <= TOL["fp32"] * abs(E_ref)
    assert_v_close(V2.cpu().numpy(), V_ref, TOL["fp32"])
    E3 = torch.zeros(1, dtype=torch.float64, device="cuda")
    V3 = torch.empty_like(phi64)
    hfx.hfx_apply_batched([ex.ctx], [(phi32, pairs_d, E3, V3, hfx.HFX_ORBITALS_F32)])
    ex.sync_status()
    assert abs(E3.item() - E_ref) <= TOL["fp32"] * abs(E_ref)
    assert_v_close(V3.cpu().numpy(), V_ref, TOL["fp32"])
    ex.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pw16_n32_full(prec):
    """The 16-orbital random-PW workload: L = 10 bohr, 32^3, Ecut = 20 Ha, all 136 pairs."""
    w = I.WORKLOADS["pw16_n32"]
    phi, pairs, _ = I.make_workload(w)
    E_ref, V_ref = O.exchange(phi, pairs, w.lattice)
    E, V = run_gpu(phi, pairs, w.lattice, prec)
    assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
    assert_v_close(V, V_ref, TOL[prec])
    # per-orbital norm-wise error as well
    worst = max(rel(V[i], V_ref[i]) for i in range(len(V)))
    assert worst <= 10 * TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_shuffled_subset_with_diagonals_and_accumulate(prec):
    n, L, n_orb = 24, 12.0, 20
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=5)
    allp = I.all_pairs(n_orb)
    rng = np.random.default_rng(6)
    sub = allp[rng.permutation(len(allp))[: len(allp) // 3]]
    E_ref, V_ref = O.exchange(phi, sub, lat)
    E, V = run_gpu(phi, sub, lat, prec)
    assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
    assert_v_close(V, V_ref, TOL[prec])
    # linearity: two halves with HFX_ACCUMULATE equal the whole list
    from paper_2309_00651_gb300 import hfx
    ex = hfx.Exchange(lat, (n, n, n), precision=prec)
    phi_d = torch.from_numpy(phi).cuda()
    h1 = torch.from_numpy(sub[::2].copy()).cuda()
    h2 = torch.from_numpy(sub[1::2].copy()).cuda()
    E1, V1 = ex.apply(phi_d, h1)
    E2, V2 = ex.apply(phi_d, h2, accumulate=True, ex=E1, vxphi=V1)
    assert abs(E2.item() - E_ref) <= TOL[prec] * abs(E_ref)
    assert_v_close(V2.cpu().numpy(), V_ref, TOL[prec])
    # energy only
    Ee, Ve = ex.apply(phi_d, torch.from_numpy(sub).cuda(), energy_only=True)
    assert Ve is None and abs(Ee.item() - E_ref) <= TOL[prec] * abs(E_ref)
    ex.close()


def test_empty_list_and_determinism():
    from paper_2309_00651_gb300 import hfx
    n, L, n_orb = 16, 8.0, 6
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=9)
    ex = hfx.Exchange(lat, (n, n, n), precision="fp32")
    phi_d = torch.from_numpy(phi).cuda()
    empty = torch.zeros((0, 2), dtype=torch.int32, device="cuda")
    E, V = ex.apply(phi_d, empty)
    assert E.item() == 0.0 and float(V.abs().max()) == 0.0
    pairs = torch.from_numpy(I.all_pairs(n_orb)).cuda()
    Ea, Va = ex.apply(phi_d, pairs)
    Eb, Vb = ex.apply(phi_d, pairs)
    assert Ea.item() == Eb.item() and torch.equal(Va, Vb)
    ex.close()


def test_result_independent_of_pair_order():
    """Pairs are placed canonically per block pair, so any ordering gives bit-identical results."""
    from paper_2309_00651_gb300 import hfx
    n, L, n_orb = 18, 9.0, 21
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=12)
    pairs = I.all_pairs(n_orb)
    ex = hfx.Exchange(lat, (n, n, n), precision="fp32")
    phi_d = torch.from_numpy(phi).cuda()
    Ea, Va = ex.apply(phi_d, torch.from_numpy(pairs).cuda())
    perm = np.random.default_rng(13).permutation(len(pairs))
    Eb, Vb = ex.apply(phi_d, torch.from_numpy(pairs[perm].copy()).cuda())
    assert Ea.item() == Eb.item() and torch.equal(Va, Vb)
    ex.close()


def test_duplicate_pairs_are_reported_and_counted_once():
    from paper_2309_00651_gb300 import hfx
    n, L, n_orb = 16, 8.0, 10
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=14)
    good = I.all_pairs(n_orb)
    dup = np.concatenate([good, good[[3, 17, 40]]])
    E_ref, V_ref = O.exchange(phi, good, lat)
    ex = hfx.Exchange(lat, (n, n, n), precision="fp64")
    E, V = ex.apply(torch.from_numpy(phi).cuda(), torch.from_numpy(dup).cuda())
    with pytest.raises(hfx.HFXError) as ei:
        ex.sync_status()
    assert ei.value.status == -5
    assert abs(E.item() - E_ref) <= 1e-8 * abs(E_ref)
    assert_v_close(V.cpu().numpy(), V_ref, 1e-8)
    ex.close()


@pytest.mark.parametrize("block", ["4", "8", "5"])
def test_orbital_block_sizes(block, monkeypatch):
    """Block sizes with a register-accumulating kernel (4, 8) and without one (5: generic path)."""
    monkeypatch.setenv("HFX_BLOCK", block)
    n, L, n_orb = 16, 8.0, 19
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=15)
    pairs = I.all_pairs(n_orb)
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    for prec in ("fp64", "fp32"):
        E, V = run_gpu(phi, pairs, lat, prec)
        assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
        assert_v_close(V, V_ref, TOL[prec])


def test_large_tile_sparse_block_pair():
    """A 90^3 grid (more tile points than one thread block holds two to a thread) and a block pair
    with missing pairs."""
    n, L, n_orb = 90, 22.0, 16
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=16, frac=0.15)
    blk = np.array([[i, j] for i in range(8) for j in range(8, 16) if (i + j) % 5 != 0], dtype=np.int32)
    extra = np.array([[0, 0], [3, 5], [9, 12], [15, 15]], dtype=np.int32)
    pairs = np.concatenate([blk, extra])
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    for prec in ("fp64", "fp32"):
        E, V = run_gpu(phi, pairs, lat, prec)
        assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
        assert_v_close(V, V_ref, TOL[prec])


@pytest.mark.parametrize("n", [48, 64, 80, 90, 96])
@pytest.mark.parametrize("no_ct", ["0", "1"])
def test_compile_time_and_runtime_kernels(n, no_ct, monkeypatch):
    """FP32 cubic grids with an instantiated edge use compile-time-geometry kernels; HFX_NO_CT=1
    forces the runtime kernels. Both must match the oracle."""
    monkeypatch.setenv("HFX_NO_CT", no_ct)
    L, n_orb = 0.4 * n, 18
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=n + 1, frac=0.2)
    pairs = I.all_pairs(n_orb)
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    E, V = run_gpu(phi, pairs, lat, "fp32")
    assert abs(E - E_ref) <= 1e-6 * abs(E_ref)
    assert_v_close(V, V_ref, 1e-6)


def test_cuda_graph_capture_and_replay():
    """After one ordinary call (which uploads the schedule), a call can be captured in a CUDA graph
    (the two internal streams join inside the capture) and replayed with identical results."""
    from paper_2309_00651_gb300 import hfx
    n, L, n_orb = 32, 10.0, 20
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=17)
    pairs = torch.from_numpy(I.all_pairs(n_orb)).cuda()
    phi_d = torch.from_numpy(phi).cuda()
    ex = hfx.Exchange(lat, (n, n, n), precision="fp32")
    E_ref, V_ref = ex.apply(phi_d, pairs)
    E_ref, V_ref = E_ref.clone(), V_ref.clone()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    V = torch.empty_like(phi_d)
    ex.apply(phi_d, pairs, ex=E, vxphi=V)  # warm-up on the side stream used for capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ex.apply(phi_d, pairs, ex=E, vxphi=V)
    E.zero_()
    V.zero_()
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert E.item() == E_ref.item() and torch.equal(V, V_ref)
    ex.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_pencil_form(prec, monkeypatch):
    """The row-block / z-chunk pencil form of the forward and x passes (used when a grid plane does
    not fit in shared memory, e.g. FP64 on 128^3), forced here on small grids."""
    monkeypatch.setenv("HFX_PENCIL", "1")
    for grid, Ls, n_orb in [((24, 16, 32), (9.0, 7.5, 11.0), 11), ((40, 40, 40), (12.0, 12.0, 12.0), 17)]:
        lat = np.diag(Ls)
        raw = I.random_pw_orbitals(n_orb, Ls[0], grid[0], ecut=1.0, seed=18) if grid[0] == grid[2] else None
        if raw is None or raw.shape[1:] != grid:
            raw = np.random.default_rng(19).standard_normal((n_orb,) + grid)
        phi, _ = I.loewdin(raw, float(np.prod(Ls)))
        pairs = I.all_pairs(n_orb)
        E_ref, V_ref = O.exchange(phi, pairs, lat)
        E, V = run_gpu(phi, pairs, lat, prec)
        assert abs(E - E_ref) <= TOL[prec] * abs(E_ref)
        assert_v_close(V, V_ref, TOL[prec])
        Ee, _ = run_gpu(phi, pairs, lat, prec, energy_only=True)
        assert abs(Ee - E_ref) <= TOL[prec] * abs(E_ref)


def test_fp64_on_128_grid_uses_pencils_and_matches_oracle():
    """FP64 on a 128^3 grid (planes larger than shared memory), checked on a few pairs."""
    n, L, n_orb = 128, 29.6, 6
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=20, frac=0.1)
    pairs = I.all_pairs(n_orb)[::2]
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    E, V = run_gpu(phi, pairs, lat, "fp64")
    assert abs(E - E_ref) <= 1e-8 * abs(E_ref)
    assert_v_close(V, V_ref, 1e-8)


def test_bad_pairs_are_reported_and_skipped():
    from paper_2309_00651_gb300 import hfx
    n, L, n_orb = 16, 8.0, 6
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=10)
    good = I.all_pairs(n_orb)
    bad = np.concatenate([good, np.array([[3, 1], [0, 6], [-1, 2]], dtype=np.int32)])
    E_ref, V_ref = O.exchange(phi, good, lat)
    ex = hfx.Exchange(lat, (n, n, n), precision="fp64")
    E, V = ex.apply(torch.from_numpy(phi).cuda(), torch.from_numpy(bad).cuda())
    with pytest.raises(hfx.HFXError) as ei:
        ex.sync_status()
    assert ei.value.status == -5
    assert abs(E.item() - E_ref) <= 1e-8 * abs(E_ref)
    assert_v_close(V.cpu().numpy(), V_ref, 1e-8)
    ex.sync_status()  # cleared
    ex.close()


def test_sphere_kernel_matches_oracle():
    n, L, n_orb, ecut = 24, 10.0, 7, 3.0
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=11)
    pairs = I.all_pairs(n_orb)
    E_ref, V_ref = O.exchange(phi, pairs, lat, sphere_ecut=ecut)
    E, V = run_gpu(phi, pairs, lat, "fp64", kernel="coulomb_sphere", ecut=ecut)
    assert abs(E - E_ref) <= 1e-8 * abs(E_ref)
    assert_v_close(V, V_ref, 1e-8)


def test_compile_time_passes_with_sparse_pair_list():
    """FP32 on a compile-time grid (32^3) with a random third of the pairs: the dense and the
    diagonal-block accumulate passes see couples with one or both halves missing."""
    w = I.WORKLOADS["pw16_n32"]
    phi, allp, _ = I.make_workload(w)
    rng = np.random.default_rng(17)
    sub = allp[np.sort(rng.permutation(len(allp))[: len(allp) // 3])]
    assert any(i == j for i, j in sub) and any(i != j for i, j in sub)
    E_ref, V_ref = O.exchange(phi, sub, w.lattice)
    E, V = run_gpu(phi, sub, w.lattice, "fp32")
    assert abs(E - E_ref) <= TOL["fp32"] * abs(E_ref)
    assert_v_close(V, V_ref, TOL["fp32"])


@pytest.mark.parametrize("dense_tma", ["1", "0"])
@pytest.mark.parametrize("n,n_orb", [(32, 16), (48, 24), (80, 16), (90, 16)])
def test_dense_pass_ignores_stale_transforms_of_empty_couples(dense_tma, n, n_orb, monkeypatch):
    """The compile-time dense accumulate pass reads whole couple tiles of the transform buffer (by
    TMA, or with HFX_DENSE_TMA=0 by per-thread copies).  Couples whose two pairs are both missing
    are never transformed, so their slots hold whatever was there before; they must contribute
    nothing.  The workspace is filled with NaN bytes first and a sparse pair list leaves such
    couples in the full off-diagonal block pairs."""
    monkeypatch.setenv("HFX_DENSE_TMA", dense_tma)
    from paper_2309_00651_gb300 import hfx
    L = 0.4 * n
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=n + 5, frac=0.2)
    allp = I.all_pairs(n_orb)
    rng = np.random.default_rng(n)
    sub = allp[np.sort(rng.permutation(len(allp))[: len(allp) // 4])]
    E_ref, V_ref = O.exchange(phi, sub, lat)
    ex = hfx.Exchange(lat, (n, n, n), precision="fp32")
    st = hfx.hfx_plan_stats(ex.ctx, n_orb, len(sub))
    ex.ensure_workspace(n_orb, len(sub))
    ex._ws.fill_(0xFF)  # every FP32 word of the workspace is a NaN
    phi_d = torch.from_numpy(phi).cuda()
    E, V = ex.apply(phi_d, torch.from_numpy(sub.astype(np.int32)).cuda())
    ex.sync_status()
    V = V.cpu().numpy()
    ex.close()
    assert st["dense_couples"] > 0
    assert np.isfinite(V).all()
    assert abs(E.item() - E_ref) <= TOL["fp32"] * abs(E_ref)
    assert_v_close(V, V_ref, TOL["fp32"])


@pytest.mark.parametrize("prefetch,waves", [("0", "1"), ("1", "1"), ("0", "64")])
def test_compile_time_passes_launch_shapes(prefetch, waves, monkeypatch):
    """The compile-time forward and x passes loop over work items with a grid of HFX_GRID_WAVES
    blocks per resident slot and send the next item's data to L2 ahead (HFX_PREFETCH); neither
    setting may change the result."""
    monkeypatch.setenv("HFX_PREFETCH", prefetch)
    monkeypatch.setenv("HFX_GRID_WAVES", waves)
    n, n_orb = 48, 20
    L = 0.4 * n
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=n + 9, frac=0.2)
    pairs = I.all_pairs(n_orb)
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    E, V = run_gpu(phi, pairs, lat, "fp32")
    assert abs(E - E_ref) <= TOL["fp32"] * abs(E_ref)
    assert_v_close(V, V_ref, TOL["fp32"])


def test_compile_time_passes_128():
    """128^3: the compile-time plane kernels run 512 threads per block (one block fills an SM's
    shared memory), the dense accumulate pass one block of 512 per SM."""
    n, n_orb = 128, 10
    L = 0.4 * n
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=n + 3, frac=0.2)
    pairs = I.all_pairs(n_orb)
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    E, V = run_gpu(phi, pairs, lat, "fp32")
    assert abs(E - E_ref) <= TOL["fp32"] * abs(E_ref)
    assert_v_close(V, V_ref, TOL["fp32"])
