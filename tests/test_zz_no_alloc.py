"""The allocation-free entry point, hfx_apply_noalloc, against hfx_apply.

hfx_apply_noalloc is for callers that cannot call cudaMalloc when they evaluate the exchange
(allocator or memory-pool callbacks, frameworks that own all device memory, latency-critical
loops): it uses the library's static device scratch instead of a caller workspace.  Here it is
called through the C ABI twice in a row and must give what hfx_apply gives, within the same
tolerances as the other GPU tests; a problem too large for the static scratch must be refused.
This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-8, "fp32": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_00651_gb300 import build
    build.build()


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_matches_apply_twice(prec):
    from paper_2309_00651_gb300 import hfx
    from paper_2309_00651_gb300 import inputs as I

    w = I.WORKLOADS["pw16_n32"]
    phi_np, pairs_np, _ = I.make_workload(w)
    phi = torch.from_numpy(phi_np).cuda()
    pairs = torch.from_numpy(pairs_np).cuda()
    ctx = hfx.hfx_create(w.lattice, w.grid, 0.0, "coulomb", 0.25, prec)
    try:
        ws = torch.empty(hfx.hfx_workspace_bytes(ctx, w.n_orb, len(pairs_np)), dtype=torch.uint8, device="cuda")
        hfx.hfx_set_workspace(ctx, ws)
        E_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        V_ref = torch.empty_like(phi)
        hfx.hfx_apply(ctx, phi, pairs, E_ref, V_ref)
        hfx.hfx_sync_status(ctx)
        for _ in range(2):
            E = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")
            V = torch.full_like(phi, 7.0)
            hfx.hfx_apply_noalloc(ctx, phi, pairs, E, V)
            hfx.hfx_sync_status(ctx)
            assert abs(E.item() - E_ref.item()) <= TOL[prec] * abs(E_ref.item())
            assert rel(V, V_ref) <= TOL[prec]
        # the caller's workspace is untouched by the allocation-free path and still usable
        E2 = torch.zeros(1, dtype=torch.float64, device="cuda")
        V2 = torch.empty_like(phi)
        hfx.hfx_apply(ctx, phi, pairs, E2, V2)
        hfx.hfx_sync_status(ctx)
        assert E2.item() == E_ref.item() and torch.equal(V2, V_ref)
    finally:
        hfx.hfx_destroy(ctx)


def test_noalloc_refuses_problems_beyond_its_scratch():
    from paper_2309_00651_gb300 import hfx
    n, n_orb = 72, 32
    ctx = hfx.hfx_create(np.diag([18.6] * 3), (n, n, n), 0.0, "coulomb", 0.25, "fp32")
    try:
        phi = torch.zeros((n_orb, n, n, n), dtype=torch.float64, device="cuda")
        i, j = np.triu_indices(n_orb)
        pairs = torch.from_numpy(np.stack([i, j], 1).astype(np.int32)).cuda()
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        V = torch.empty_like(phi)
        with pytest.raises(hfx.HFXError) as ei:
            hfx.hfx_apply_noalloc(ctx, phi, pairs, E, V)
        assert ei.value.status == -3 and "scratch" in str(ei.value)
    finally:
        hfx.hfx_destroy(ctx)
