"""HFX_PREC_MIXED_TC: the forward DFTs of the plane pass (along z and y) on the tensor cores,
each axis one complex DFT as a dense GEMM with split TF32 operands and FP32 accumulation, the
other stages as on the FP32 path.  Against the FP64 oracle at the mixed path's stated accuracy
(1e-6 relative in E_x and V_x phi, Frobenius and max-abs), on every supported edge, with a
ragged orbital block and a partial pair list, energy only; then the 256-orbital 96^3 workload
(all 32896 pairs) on sampled rows of V_x phi and on E_x of a seeded pair sample."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hfx_oracle as O  # noqa: E402
from paper_2309_00651_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_00651_gb300 import build
    build.build()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def maxrel(a, b):
    return float(np.max(np.abs(np.ravel(a - b))) / np.max(np.abs(np.ravel(b))))


def band_limited(n_orb, n, L, seed, frac=0.2):
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=0.5 * (2 * math.pi * (frac * n + 0.5) / L) ** 2, seed=seed)
    phi, _ = I.loewdin(raw, L ** 3)
    return phi


@pytest.mark.parametrize("n", [32, 48, 64, 96])
def test_mixed_tc_against_oracle(n):
    from paper_2309_00651_gb300 import hfx
    L, n_orb = 0.28 * n, 11
    lat = np.diag([L] * 3)
    phi = band_limited(n_orb, n, L, seed=7 * n)
    allp = I.all_pairs(n_orb)
    pairs = allp[np.random.default_rng(n).permutation(len(allp))[: 2 * len(allp) // 3]]
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    ex = hfx.Exchange(lat, (n, n, n), precision="mixed_tc")
    phi_d = torch.from_numpy(phi).cuda()
    pairs_d = torch.from_numpy(np.ascontiguousarray(pairs)).cuda()
    E, V = ex.apply(phi_d, pairs_d)
    Ee, _ = ex.apply(phi_d, pairs_d, energy_only=True)
    ex.sync_status()
    V = V.cpu().numpy()
    assert abs(E.item() - E_ref) <= 1e-6 * abs(E_ref)
    assert abs(Ee.item() - E_ref) <= 1e-6 * abs(E_ref)
    assert rel(V, V_ref) <= 1e-6
    assert maxrel(V, V_ref) <= 1e-6
    ex.close()


def test_mixed_tc_unsupported_edge_is_refused():
    from paper_2309_00651_gb300 import hfx
    with pytest.raises(hfx.HFXError) as ei:
        hfx.Exchange(np.diag([10.0] * 3), (72, 72, 72), precision="mixed_tc")
    assert ei.value.status == -2


def test_mixed_tc_water64_n96():
    """The 256-orbital 96^3 workload, all 32896 pairs: sampled rows of V_x phi (the oracle from
    every listed pair containing the row) and E_x of a seeded pair sample run as the GPU's own
    list, within 1e-6; the whole result against the FP32 path and on the homogeneity identity."""
    from paper_2309_00651_gb300 import hfx
    w = I.WORKLOADS["water64_n96"]
    phi, pairs, _ = I.make_workload(w)
    rows = (77,)
    V_rows = O.exchange_rows(phi, pairs, rows, w.lattice)
    sub = I.random_pairs_subset(pairs, 16, seed=13)
    E_sub, _ = O.exchange(phi, sub, w.lattice, want_v=False)
    phi_d = torch.from_numpy(phi).cuda()
    pairs_d = torch.from_numpy(pairs).cuda()
    ex = hfx.Exchange(w.lattice, w.grid, precision="mixed_tc")
    E, V = ex.apply(phi_d, pairs_d)
    Es, _ = ex.apply(phi_d, torch.from_numpy(sub).cuda(), energy_only=True)
    ex.sync_status()
    for r, k in enumerate(rows):
        Vk = V[k].cpu().numpy()
        assert rel(Vk, V_rows[r]) <= 1e-6
        assert maxrel(Vk, V_rows[r]) <= 1e-6
    assert abs(Es.item() - E_sub) <= 1e-6 * abs(E_sub)
    N = w.n ** 3
    hom = 0.5 * (w.volume / N) * float(torch.sum(phi_d * V).item())
    assert abs(hom - E.item()) <= 1e-5 * abs(E.item())
    ex32 = hfx.Exchange(w.lattice, w.grid, precision="fp32")
    E32, V32 = ex32.apply(phi_d, pairs_d)
    assert abs(E.item() - E32.item()) <= 1e-6 * abs(E32.item())
    assert float(torch.linalg.norm(V - V32) / torch.linalg.norm(V32)) <= 1e-6
    ex.close()
    ex32.close()
