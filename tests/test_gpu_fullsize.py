"""Full-size workloads, in the launch configuration bench.py times, checked on sampled outputs.

* water32_n72 (128 orbitals, 72^3, all 8256 pairs) and water64_n96 (256 orbitals, 96^3, all
  32896 pairs): the full call on both precision paths; the oracle recomputes, one by one,
  (V_x phi)_k for sampled orbitals k (from every listed pair that contains k) and E_x over a
  seeded sample of pairs, which the GPU evaluates as its own pair list.  Properties that hold at
  any size are checked on the full result: the homogeneity identity E_x = 1/2 (Omega/N) sum
  <phi_i, (V_x phi)_i>, and agreement between the FP32 and FP64 paths.
"""
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
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("name,rows,n_sample", [("water32_n72", (5, 77), 48), ("water64_n96", (130,), 24)])
def test_full_workload_sampled(name, rows, n_sample):
    from paper_2309_00651_gb300 import hfx
    w = I.WORKLOADS[name]
    phi, pairs, _ = I.make_workload(w)
    phi_d = torch.from_numpy(phi).cuda()
    pairs_d = torch.from_numpy(pairs).cuda()
    N = w.n ** 3
    # oracle references, once: sampled rows of V_x phi and E_x over a seeded sample of pairs
    V_rows = O.exchange_rows(phi, pairs, rows, w.lattice)
    sub = I.random_pairs_subset(pairs, n_sample, seed=11)
    E_ref, _ = O.exchange(phi, sub, w.lattice, want_v=False)
    results = {}
    for prec in ("fp32", "fp64"):
        ex = hfx.Exchange(w.lattice, w.grid, precision=prec)
        E, V = ex.apply(phi_d, pairs_d)
        ex.sync_status()
        Ef = E.item()
        # homogeneity identity on the full result
        hom = 0.5 * (w.volume / N) * float(torch.sum(phi_d * V).item())
        assert abs(hom - Ef) <= 10 * TOL[prec] * abs(Ef)
        for r, k in enumerate(rows):
            assert rel(V[k].cpu().numpy(), V_rows[r]) <= TOL[prec]
        # the sampled pairs as the GPU's own pair list
        Es, _ = ex.apply(phi_d, torch.from_numpy(sub).cuda(), energy_only=True)
        assert abs(Es.item() - E_ref) <= TOL[prec] * abs(E_ref)
        results[prec] = (Ef, V.cpu().numpy())
        ex.close()
    # the two precision paths agree to the FP32 tolerance
    assert abs(results["fp32"][0] - results["fp64"][0]) <= 1e-6 * abs(results["fp64"][0])
    assert rel(results["fp32"][1], results["fp64"][1]) <= 1e-6


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_ace_full_workload(precision):
    """ACE at full size (water32_n72, W from the exchange call itself): M against the oracle's
    full grid contraction, L against its Cholesky factor, the first rows of P against forward
    substitution, the occupied-span identity and 1/2 tr M = E_x on the whole result."""
    import scipy.linalg
    from oracle import ace_oracle as A
    from paper_2309_00651_gb300 import hfx
    w = I.WORKLOADS["water32_n72"]
    phi, pairs, _ = I.make_workload(w)
    phi_d = torch.from_numpy(phi).cuda()
    ex = hfx.Exchange(w.lattice, w.grid, precision=precision)
    E, V = ex.apply(phi_d, torch.from_numpy(pairs).cuda())
    M, Lf, P = ex.ace_build(phi_d, V)
    Y = ex.ace_apply(P, phi_d)
    ex.sync_status()
    tol = TOL[precision]
    Vh = V.cpu().numpy()
    M0 = A.grid_inner(phi, Vh, w.lattice)
    L0 = np.linalg.cholesky(-0.5 * (M0 + M0.T))
    assert rel(M.cpu().numpy(), M0) <= tol
    assert rel(Lf.cpu().numpy(), L0) <= 10 * tol
    k = 4
    P0 = scipy.linalg.solve_triangular(L0[:k, :k], Vh[:k].reshape(k, -1), lower=True)
    assert rel(P[:k].cpu().numpy().reshape(k, -1), P0) <= 10 * tol
    assert float(torch.linalg.norm(Y - V) / torch.linalg.norm(V)) <= 10 * tol
    assert 0.5 * float(torch.trace(M)) == pytest.approx(E.item(), rel=10 * tol)
    ex.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_scdm_full_workload(precision):
    """SCDM at full size (water32_n72, 128 orbitals on 72^3): every pick is a greedy choice within
    the stated slack of the FP64 residual norms, Q matches the oracle's QR of the picked columns,
    sampled rows of Phi match, Phi is orthonormal."""
    from oracle import ace_oracle as A
    from paper_2309_00651_gb300 import hfx
    w = I.WORKLOADS["water32_n72"]
    phi, _, _ = I.make_workload(w)
    ex = hfx.Exchange(w.lattice, w.grid, precision=precision)
    piv, Q, Phi = ex.scdm_localise(torch.from_numpy(phi).cuda())
    ex.sync_status()
    piv = piv.cpu().numpy()
    slack = A.scdm_pivot_slack(phi, piv)
    assert slack.min() >= (1 - 1e-9 if precision == "fp64" else 1 - 1e-4)
    Q0 = A.scdm_q_from_pivots(phi, piv)
    tol = TOL[precision]
    assert rel(Q.cpu().numpy(), Q0) <= 10 * tol
    rows = [0, 63, 127]
    Phi0 = Q0[:, rows].T @ phi.reshape(128, -1)
    assert rel(Phi[rows].cpu().numpy().reshape(3, -1), Phi0) <= 10 * tol
    G = (w.volume / w.n ** 3) * (Phi.reshape(128, -1) @ Phi.reshape(128, -1).T)
    assert float(torch.max(torch.abs(G - torch.eye(128, dtype=G.dtype, device=G.device)))) <= 10 * tol
    ex.close()
