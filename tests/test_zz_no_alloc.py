"""The allocation-free entry point, hfx_apply_noalloc, against hfx_apply.

hfx_apply_noalloc is for callers that cannot call cudaMalloc when they evaluate the exchange
(allocator or memory-pool callbacks, frameworks that own all device memory, latency-critical
loops): it uses the library's static device scratch instead of a caller workspace.  Here it is
called through the C ABI twice in a row and must give what hfx_apply gives, within the same
tolerances as the other GPU tests, with the caller's workspace left exactly as it was; the
accumulate and energy-only flags go through it too; a problem whose default batches exceed the
static scratch runs in smaller batches; a problem whose single block pair does not fit is refused.
This file is named so that pytest collects it last.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-8, "fp32": 1e-6}
SCRATCH = 32 << 20  # HFX_NOALLOC_SCRATCH_BYTES


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_00651_gb300 import build
    build.build()


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _reference(hfx, ctx, phi, pairs, flags=0, E0=None, V0=None):
    E = torch.zeros(1, dtype=torch.float64, device="cuda") if E0 is None else E0.clone()
    V = torch.empty_like(phi) if V0 is None else V0.clone()
    hfx.hfx_apply(ctx, phi, pairs, E, None if flags & hfx.HFX_ENERGY_ONLY else V, flags=flags)
    hfx.hfx_sync_status(ctx)
    return E, V


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
        E_ref, V_ref = _reference(hfx, ctx, phi, pairs)
        # a sentinel in the caller's workspace: the allocation-free path must not touch it
        ws.fill_(0xA5)
        for _ in range(2):
            E = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")
            V = torch.full_like(phi, 7.0)
            hfx.hfx_apply_noalloc(ctx, phi, pairs, E, V)
            hfx.hfx_sync_status(ctx)
            assert abs(E.item() - E_ref.item()) <= TOL[prec] * abs(E_ref.item())
            assert rel(V, V_ref) <= TOL[prec]
            assert float(torch.max(torch.abs(V - V_ref))) <= TOL[prec] * float(torch.max(torch.abs(V_ref)))
        assert bool(torch.all(ws == 0xA5))
        # accumulate: half the list by hfx_apply, the other half added by the allocation-free path
        h1, h2 = pairs[0::2].contiguous(), pairs[1::2].contiguous()
        E_a, V_a = _reference(hfx, ctx, phi, h1)
        ws.fill_(0xA5)
        hfx.hfx_apply_noalloc(ctx, phi, h2, E_a, V_a, flags=hfx.HFX_ACCUMULATE)
        hfx.hfx_sync_status(ctx)
        assert bool(torch.all(ws == 0xA5))
        assert abs(E_a.item() - E_ref.item()) <= TOL[prec] * abs(E_ref.item())
        assert rel(V_a, V_ref) <= TOL[prec]
        # energy only: vxphi may be NULL
        E_e = torch.full((1,), -5.0, dtype=torch.float64, device="cuda")
        hfx.hfx_apply_noalloc(ctx, phi, pairs, E_e, None, flags=hfx.HFX_ENERGY_ONLY)
        hfx.hfx_sync_status(ctx)
        assert abs(E_e.item() - E_ref.item()) <= TOL[prec] * abs(E_ref.item())
    finally:
        hfx.hfx_destroy(ctx)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_noalloc_splits_batches_to_fit(prec):
    """32 orbitals on 32^3: the default batches need more than the static scratch, so the
    allocation-free path runs the block pairs in smaller batches; results match hfx_apply."""
    from paper_2309_00651_gb300 import hfx
    from paper_2309_00651_gb300 import inputs as I

    n, L, n_orb = 32, 10.0, 32
    lat = np.diag([L] * 3)
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=0.5 * (2 * math.pi * 6.5 / L) ** 2, seed=41)
    phi_np, _ = I.loewdin(raw, L ** 3)
    pairs_np = I.all_pairs(n_orb)
    phi = torch.from_numpy(phi_np).cuda()
    pairs = torch.from_numpy(pairs_np).cuda()
    ctx = hfx.hfx_create(lat, (n, n, n), 0.0, "coulomb", 0.25, prec)
    try:
        need = hfx.hfx_workspace_bytes(ctx, n_orb, len(pairs_np))
        assert need > SCRATCH
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        hfx.hfx_set_workspace(ctx, ws)
        E_ref, V_ref = _reference(hfx, ctx, phi, pairs)
        for _ in range(2):
            E = torch.zeros(1, dtype=torch.float64, device="cuda")
            V = torch.full_like(phi, 3.0)
            hfx.hfx_apply_noalloc(ctx, phi, pairs, E, V)
            hfx.hfx_sync_status(ctx)
            assert abs(E.item() - E_ref.item()) <= TOL[prec] * abs(E_ref.item())
            assert rel(V, V_ref) <= TOL[prec]
    finally:
        hfx.hfx_destroy(ctx)


def test_noalloc_refuses_problems_beyond_its_scratch():
    """72^3 in FP32: one block pair's 32 transforms alone (95 MB) exceed the static scratch."""
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
