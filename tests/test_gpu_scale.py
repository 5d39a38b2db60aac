"""Differentiation at scale: the 128-H2O box (512 Gaussian orbitals, sigma = 1.5 bohr, 29.6 bohr,
128^3 grid, overlap-screened pair list s_ij > 1e-6).

* The FP32 path over the whole screened list: the homogeneity identity on the full result.
* The FP64 path (pencil form on this grid) over the screened pairs among the first 48 orbitals:
  E_x through the autograd wrapper, its backward pass checked against 5-point finite
  differences along 8 random perturbations (E is a quartic in the step, so the stencil is exact
  up to rounding), and the FP32 path agreeing with it on the same list.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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
    ex.close()
    del phi_d, V
    torch.cuda.empty_cache()


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
    # the FP32 path on the same list
    ex32 = hfx.Exchange(w.lattice, w.grid, precision="fp32")
    E32, V32 = ex32.apply(phi_d.detach(), pairs_d)
    E64, V64 = ex.apply(phi_d.detach(), pairs_d)
    assert abs(E32.item() - E64.item()) <= 1e-6 * abs(E64.item())
    assert float(torch.linalg.norm(V32 - V64) / torch.linalg.norm(V64)) <= 1e-6
    ex.close()
    ex32.close()
