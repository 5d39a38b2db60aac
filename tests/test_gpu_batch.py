"""The uneven batch (24 independent water-density boxes, 32..256 orbitals on 48^3..96^3 grids)
through hfx_apply_batched: all passes of all problems in one persistent launch with a device work
queue and bounded waits.

* All 24 problems at full size: every problem against the oracle on a sampled orbital row of
  V_x phi and on E_x of a seeded pair sample (the sample run as a second batch), against
  hfx_apply_sequential (one hfx_apply per problem, the separately oracle-checked path) on the
  whole result, and on the homogeneity identity.  The oracle work runs in spawned processes, one
  per host core, each rebuilding its problem's orbitals from the problem's seed.
* Flags in a batch (energy only, accumulate, an empty pair list) against hfx_apply_sequential.
* Capture of one batched call in a CUDA graph, replayed with bit-identical results.
* Failure detection without a GPU fault: HFX_TEST_STALL makes one wait expect an item that never
  comes; with a small wait budget the call ends, HFX_ERR_TIMEOUT is reported for that problem,
  and the next call on the same contexts is correct.
"""
import math
import multiprocessing as mp

import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def _oracle_checks(task):
    """Oracle values of one batch problem, rebuilt from its seed: (V_x phi)_row from every listed
    pair containing the row, and E_x of a seeded pair sample."""
    from oracle import hfx_oracle as O
    w, row, sample = task
    phi, pairs, _ = I.make_workload(w)
    V_row = O.exchange_rows(phi, pairs, [row], w.lattice)[0]
    E_s, _ = O.exchange(phi, sample, w.lattice, want_v=False)
    return V_row, E_s


def _setup(ws, data, precision="fp32"):
    from paper_2309_00651_gb300 import hfx
    exs, phis, pairss = [], [], []
    for w, (phi, pairs, _) in zip(ws, data):
        ex = hfx.Exchange(w.lattice, w.grid, precision=precision)
        ex.ensure_workspace(w.n_orb, len(pairs))
        exs.append(ex)
        phis.append(torch.from_numpy(phi).cuda())
        pairss.append(torch.from_numpy(pairs).cuda())
    return exs, phis, pairss


def test_all_24_problems_one_launch():
    from paper_2309_00651_gb300 import hfx
    ws = I.batched_workloads()
    assert len(ws) == 24
    rows = [w.n_orb // 3 for w in ws]
    samples = [I.random_pairs_subset(I.all_pairs(w.n_orb), 6, seed=100 + k) for k, w in enumerate(ws)]
    # the oracle work starts first (spawned processes), the GPU work runs meanwhile
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(min(len(ws), max(1, len(__import__("os").sched_getaffinity(0)))))
    order = sorted(range(len(ws)), key=lambda k: -ws[k].n_orb * ws[k].n ** 3)
    pending = {k: pool.apply_async(_oracle_checks, ((ws[k], rows[k], samples[k]),)) for k in order}
    try:
        data = I.make_workloads_parallel(ws)
        exs, phis, pairss = _setup(ws, data)
        Es = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in ws]
        Vs = [torch.empty_like(p) for p in phis]
        hfx.hfx_apply_batched([e.ctx for e in exs], [(p, q, E, V, 0) for p, q, E, V in zip(phis, pairss, Es, Vs)])
        torch.cuda.synchronize()
        for e in exs:
            e.sync_status()
        # the same problems one by one
        Es2 = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in ws]
        Vs2 = [torch.empty_like(p) for p in phis]
        hfx.hfx_apply_sequential([e.ctx for e in exs], [(p, q, E, V, 0) for p, q, E, V in zip(phis, pairss, Es2, Vs2)])
        # the seeded pair samples as a second batch, energy only
        Ess = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in ws]
        smp = [torch.from_numpy(s).cuda() for s in samples]
        hfx.hfx_apply_batched([e.ctx for e in exs],
                              [(p, s, E, None, hfx.HFX_ENERGY_ONLY) for p, s, E in zip(phis, smp, Ess)])
        torch.cuda.synchronize()
        for k, w in enumerate(ws):
            N = w.n ** 3
            E, E2 = Es[k].item(), Es2[k].item()
            hom = 0.5 * (w.volume / N) * float(torch.sum(phis[k] * Vs[k]).item())
            assert abs(hom - E) <= 1e-5 * abs(E), w.name
            assert abs(E - E2) <= 1e-6 * abs(E2), w.name
            assert float(torch.linalg.norm(Vs[k] - Vs2[k]) / torch.linalg.norm(Vs2[k])) <= 1e-6, w.name
        for k, w in enumerate(ws):
            V_row, E_s = pending[k].get(timeout=1800)
            Vk = Vs[k][rows[k]].cpu().numpy()
            assert rel(Vk, V_row) <= 1e-6, w.name
            assert np.max(np.abs(Vk - V_row)) <= 1e-6 * np.max(np.abs(V_row)), w.name
            assert abs(Ess[k].item() - E_s) <= 1e-6 * abs(E_s), w.name
        for e in exs:
            e.close()
    finally:
        pool.terminate()
        pool.join()
    torch.cuda.empty_cache()


def _small_batch(precision):
    specs = [(9, 24, 9.0), (13, 30, 10.0), (5, 18, 7.0), (17, 32, 11.0)]
    ws, data = [], []
    for k, (n_orb, n, L) in enumerate(specs):
        w = I.Workload(f"small{k}", n_orb, L, n, 0.5 * (2 * math.pi * (0.2 * n + 0.5) / L) ** 2, "pw", seed=50 + k)
        ws.append(w)
        data.append(I.make_workload(w))
    return ws, data


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_flags_in_a_batch(precision):
    """Energy only, accumulate and an empty pair list mixed in one batch, against one-by-one calls."""
    from paper_2309_00651_gb300 import hfx
    ws, data = _small_batch(precision)
    exs, phis, pairss = _setup(ws, data, precision)
    tol = 1e-6 if precision == "fp32" else 1e-8
    flags = [0, hfx.HFX_ENERGY_ONLY, hfx.HFX_ACCUMULATE, 0]
    lists = [pairss[0], pairss[1], pairss[2], pairss[3][:0]]
    outs = []
    for runner in (hfx.hfx_apply_batched, hfx.hfx_apply_sequential):
        Es = [torch.full((1,), 0.5, dtype=torch.float64, device="cuda") for _ in ws]
        Vs = [torch.full_like(p, 0.25) for p in phis]
        runner([e.ctx for e in exs],
               [(p, q, E, None if f & hfx.HFX_ENERGY_ONLY else V, f)
                for p, q, E, V, f in zip(phis, lists, Es, Vs, flags)])
        torch.cuda.synchronize()
        for e in exs:
            e.sync_status()
        outs.append((Es, Vs))
    (Eb, Vb), (Es_, Vs_) = outs
    for k in range(len(ws)):
        assert abs(Eb[k].item() - Es_[k].item()) <= tol * max(abs(Es_[k].item()), 1e-300), k
        if k in (0, 2):  # 1: energy only, 3: empty list (both checked exactly below)
            assert float(torch.linalg.norm(Vb[k] - Vs_[k]) / torch.linalg.norm(Vs_[k])) <= tol, k
    assert Eb[3].item() == 0.0 and float(Vb[3].abs().max()) == 0.0
    assert bool(torch.all(Vb[1] == 0.25))  # energy only leaves V alone
    for e in exs:
        e.close()


def test_graph_capture_and_replay():
    from paper_2309_00651_gb300 import hfx
    ws, data = _small_batch("fp32")
    exs, phis, pairss = _setup(ws, data)
    Es = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in ws]
    Vs = [torch.empty_like(p) for p in phis]
    args = [(p, q, E, V, 0) for p, q, E, V in zip(phis, pairss, Es, Vs)]
    ctxs = [e.ctx for e in exs]
    hfx.hfx_apply_batched(ctxs, args)  # sizes the queue tables and uploads the schedules
    torch.cuda.synchronize()
    ref = [(E.clone(), V.clone()) for E, V in zip(Es, Vs)]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        hfx.hfx_apply_batched(ctxs, args)
    for E, V in zip(Es, Vs):
        E.zero_()
        V.zero_()
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for (E, V), (Er, Vr) in zip(zip(Es, Vs), ref):
            assert E.item() == Er.item() and torch.equal(V, Vr)
    for e in exs:
        e.close()


def test_wait_budget_runs_out_and_is_reported():
    """No GPU fault: a wait that nothing completes gives up after its budget, the call ends,
    HFX_ERR_TIMEOUT is reported, and the next calls on the same contexts are correct.  The
    stalled problem runs alone, so its never-completed wait is the only wait of the launch."""
    from paper_2309_00651_gb300 import hfx
    ws, data = _small_batch("fp32")
    exs, phis, pairss = _setup(ws, data)
    ctxs = [e.ctx for e in exs]
    Es = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in ws]
    Vs = [torch.empty_like(p) for p in phis]
    hfx.hfx_apply_sequential(ctxs, [(p, q, E, V, 0) for p, q, E, V in zip(phis, pairss, Es, Vs)])
    torch.cuda.synchronize()
    ref = [(E.item(), V.clone()) for E, V in zip(Es, Vs)]
    hfx.hfx_set_wait_budget(ctxs[1], 200000)  # about 0.1 ms
    hfx.hfx_apply_batched([ctxs[1]], [(phis[1], pairss[1], Es[1], Vs[1], hfx.HFX_TEST_STALL)])
    torch.cuda.synchronize()
    with pytest.raises(hfx.HFXError) as ei:
        exs[1].sync_status()
    assert ei.value.status == -6
    exs[1].sync_status()  # cleared
    # the contexts stay usable: the stalled problem alone, then all four in one batched call
    hfx.hfx_set_wait_budget(ctxs[1], 0)
    hfx.hfx_apply_batched([ctxs[1]], [(phis[1], pairss[1], Es[1], Vs[1], 0)])
    hfx.hfx_apply_batched(ctxs, [(p, q, E, V, 0) for p, q, E, V in zip(phis, pairss, Es, Vs)])
    torch.cuda.synchronize()
    for e in exs:
        e.sync_status()
    for (E, V), (Er, Vr) in zip(zip(Es, Vs), ref):
        assert abs(E.item() - Er) <= 1e-6 * abs(Er)
        assert float(torch.linalg.norm(V - Vr) / torch.linalg.norm(Vr)) <= 1e-6
    for e in exs:
        e.close()
