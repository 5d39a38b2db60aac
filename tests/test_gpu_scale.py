"""Differentiation at scale: the 128-H2O box (512 Gaussian orbitals, sigma = 1.5 bohr, 29.6 bohr,
128^3 grid, overlap-screened pair list s_ij > 1e-6).

* The FP32 path over the whole screened list: the homogeneity identity on the full result.
  E_x of a seeded sample of the screened pairs, run as the GPU's own pair list, against the oracle.
* The FP32 compile-time 128^3 passes against the oracle: the screened pairs among the first 24
  orbitals (three full orbital blocks: diagonal and off-diagonal block pairs), sampled rows of
  V_x phi from the oracle's per-row evaluation and E_x of a seeded pair sample.
* The FP64 path (pencil form on this grid) over the screened pairs among the first 48 orbitals:
  E_x through the autograd wrapper, its backward pass checked against 5-point finite
  differences along 8 random perturbations (E is a quartic in the step, so the stencil is exact
  up to rounding) and, on a sampled orbital row, against the oracle gradient 2 (Omega/N) V_x phi;
  the FP32 path agreeing with it on the same list.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hfx_oracle as O  # noqa: E402
from paper_2309_00651_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_00651_gb300 import build
    build.build()
    w = I.WORKLOADS["water128_n128"]
    phi, pairs, info = I.make_workload(w)
    return w, phi, pairs, info


def test_full_screened_list_fp32(workload):
    from paper_2309_00651_gb300 import hfx
    w, phi, pairs, info = workload
    assert 512 <= len(pairs) <= 512 * 513 // 2 and np.all(pairs[:, 0] <= pairs[:, 1])
    phi_d = torch.from_numpy(phi).cuda()
    ex = hfx.Exchange(w.lattice, w.grid, precision="fp32")
    E, V = ex.apply(phi_d, torch.from_numpy(pairs).cuda())
    ex.sync_status()
    N = w.n ** 3
    hom = 0.5 * (w.volume / N) * float(torch.sum(phi_d * V).item())
    assert E.item() < 0 and abs(hom - E.item()) <= 1e-5 * abs(E.item())
    del V
    # a seeded sample of the screened list as the GPU's own pair list, against the oracle
    sample = I.random_pairs_subset(pairs, 16, seed=23)
    Es, _ = ex.apply(phi_d, torch.from_numpy(sample).cuda(), energy_only=True)
    E_ref, _ = O.exchange(phi, sample, w.lattice, want_v=False)
    assert abs(Es.item() - E_ref) <= 1e-6 * abs(E_ref)
    ex.close()
    del phi_d
    torch.cuda.empty_cache()


def test_fp32_compile_time_128_against_oracle(workload):
    """The FP32 compile-time 128^3 kernels (forward, x/Coulomb, dense and diagonal-block
    accumulate) on the screened pairs among the first 24 orbitals, checked against the oracle."""
    from paper_2309_00651_gb300 import hfx
    w, phi, pairs, _ = workload
    k = 24
    sub = pairs[pairs[:, 1] < k]
    phi_k = np.ascontiguousarray(phi[:k])
    ex = hfx.Exchange(w.lattice, w.grid, precision="fp32")
    phi_d = torch.from_numpy(phi_k).cuda()
    E, V = ex.apply(phi_d, torch.from_numpy(sub).cuda())
    ex.sync_status()
    rows = [3, 13]
    V_rows = O.exchange_rows(phi_k, sub, rows, w.lattice)
    for r, kk in enumerate(rows):
        Vk = V[kk].cpu().numpy()
        assert np.linalg.norm(Vk - V_rows[r]) <= 1e-6 * np.linalg.norm(V_rows[r])
        assert np.max(np.abs(Vk - V_rows[r])) <= 1e-6 * np.max(np.abs(V_rows[r]))
    sample = I.random_pairs_subset(sub, 16, seed=29)
    Es, _ = ex.apply(phi_d, torch.from_numpy(sample).cuda(), energy_only=True)
    E_ref, _ = O.exchange(phi_k, sample, w.lattice, want_v=False)
    assert abs(Es.item() - E_ref) <= 1e-6 * abs(E_ref)
    N = w.n ** 3
    hom = 0.5 * (w.volume / N) * float(torch.sum(phi_d * V).item())
    assert abs(hom - E.item()) <= 1e-5 * abs(E.item())
    ex.close()


def test_fd_gradient_fp64_sublist(workload):
    from paper_2309_00651_gb300 import hfx
    from paper_2309_00651_gb300.autograd import exchange_energy
    w, phi, pairs, _ = workload
    k = 48
    sub = pairs[(pairs[:, 1] < k)]
    phi_k = np.ascontiguousarray(phi[:k])
    ex = hfx.Exchange(w.lattice, w.grid, precision="fp64")
    phi_d = torch.from_numpy(phi_k).cuda().requires_grad_(True)
    pairs_d = torch.from_numpy(sub).cuda()
    E = exchange_energy(ex, phi_d, pairs_d)
    (g,) = torch.autograd.grad(E, phi_d)
    for s in range(1, 9):
        d = torch.from_numpy(np.random.default_rng(s).standard_normal(phi_k.shape)).cuda()
        h = 1e-3 * float(torch.linalg.norm(phi_d.detach())) / float(torch.linalg.norm(d))
        with torch.no_grad():
            Es = [exchange_energy(ex, phi_d.detach() + c * h * d, pairs_d).item() for c in (-2, -1, 1, 2)]
        fd = (Es[0] - 8 * Es[1] + 8 * Es[2] - Es[3]) / (12 * h)
        an = float(torch.sum(g * d))
        assert fd == pytest.approx(an, rel=1e-8)
    # the gradient's sampled row against the oracle gradient 2 (Omega/N) (V_x phi)_row
    row = 29
    N = w.n ** 3
    g_ref = 2.0 * (w.volume / N) * O.exchange_rows(phi_k, sub, [row], w.lattice)[0]
    g_row = g[row].cpu().numpy()
    assert np.linalg.norm(g_row - g_ref) <= 1e-8 * np.linalg.norm(g_ref)
    assert np.max(np.abs(g_row - g_ref)) <= 1e-8 * np.max(np.abs(g_ref))
    # the FP32 path on the same list
    ex32 = hfx.Exchange(w.lattice, w.grid, precision="fp32")
    E32, V32 = ex32.apply(phi_d.detach(), pairs_d)
    E64, V64 = ex.apply(phi_d.detach(), pairs_d)
    assert abs(E32.item() - E64.item()) <= 1e-6 * abs(E64.item())
    assert float(torch.linalg.norm(V32 - V64) / torch.linalg.norm(V64)) <= 1e-6
    ex.close()
    ex32.close()
