"""Failure injection on the host: a device allocation that fails.

Every device allocation libhfx makes for itself goes through one allocator, which the test entry
point hfx_test_fail_allocation(k) makes fail on the (k+1)-th call from now, as cudaMalloc does on a
full device.  For each allocation of hfx_create, of the first hfx_apply of an orbital count (its
schedule tables) and of the first hfx_apply_batched (its queue tables), the call must return
HFX_ERR_OOM, hold no device allocation it did not hold before (hfx_test_live_allocations), and the
next call without a failure must give the same result as a context that never saw one.  Nothing
here faults or exhausts the GPU: the failing allocation never reaches cudaMalloc.
"""
import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

OOM = -3  # HFX_ERR_OOM


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_00651_gb300 import build
    build.build()
    yield
    from paper_2309_00651_gb300 import hfx
    hfx.hfx_test_fail_allocation(-1)


@pytest.fixture(autouse=True)
def _no_collection_during_counts():
    """Contexts that earlier tests left in reference cycles are freed now, and the cyclic collector
    is held off while a test compares allocation counts (a context it freed mid-test would lower
    the count by its tables)."""
    gc.collect()
    gc.disable()
    yield
    gc.enable()


def _workload(n_orb, seed):
    from paper_2309_00651_gb300 import inputs as I
    L, n = 10.0, 32
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=20.0, seed=seed)
    phi, _ = I.loewdin(raw, L ** 3)
    return np.diag([L] * 3), (n, n, n), torch.from_numpy(phi).cuda(), torch.from_numpy(I.all_pairs(n_orb)).cuda()


def _expect_oom(fn):
    from paper_2309_00651_gb300 import hfx
    with pytest.raises(hfx.HFXError) as ei:
        fn()
    assert ei.value.status == OOM, str(ei.value)


@pytest.mark.parametrize("prec", ["fp32", "fp64", "mixed_tc"])
def test_create_fails_cleanly_at_every_allocation(prec):
    from paper_2309_00651_gb300 import hfx
    lat, grid, _, _ = _workload(4, 0)
    live0 = hfx.hfx_test_live_allocations()
    ctx = hfx.hfx_create(lat, grid, 0.0, "coulomb", 0.25, prec)
    n_create = hfx.hfx_test_live_allocations() - live0
    hfx.hfx_destroy(ctx)
    assert hfx.hfx_test_live_allocations() == live0
    assert n_create >= 5  # three twiddle tables, the Coulomb table, the error word (and more)
    for k in range(n_create):
        hfx.hfx_test_fail_allocation(k)
        _expect_oom(lambda: hfx.hfx_create(lat, grid, 0.0, "coulomb", 0.25, prec))
        assert hfx.hfx_test_live_allocations() == live0, f"allocation {k} of hfx_create: tables leaked"
    # the failure was used up: the next create succeeds and holds what the first one held
    ctx = hfx.hfx_create(lat, grid, 0.0, "coulomb", 0.25, prec)
    assert hfx.hfx_test_live_allocations() == live0 + n_create
    hfx.hfx_destroy(ctx)
    assert hfx.hfx_test_live_allocations() == live0


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_first_apply_fails_cleanly_at_every_schedule_allocation(prec):
    from paper_2309_00651_gb300 import hfx
    lat, grid, phi, pairs = _workload(16, 1)
    ref = hfx.Exchange(lat, grid, alpha=0.25, precision=prec)
    live0 = hfx.hfx_test_live_allocations()
    E_ref, V_ref = ref.apply(phi, pairs)
    ref.sync_status()
    n_sched = hfx.hfx_test_live_allocations() - live0  # the schedule tables of 16 orbitals
    assert n_sched >= 1
    ex = hfx.Exchange(lat, grid, alpha=0.25, precision=prec)
    ex.ensure_workspace(16, len(pairs))
    live1 = hfx.hfx_test_live_allocations()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    V = torch.empty_like(phi)
    for k in range(n_sched):
        hfx.hfx_test_fail_allocation(k)
        _expect_oom(lambda: hfx.hfx_apply(ex.ctx, phi, pairs, E, V))
        assert hfx.hfx_test_live_allocations() == live1, f"schedule allocation {k}: tables leaked"
    hfx.hfx_apply(ex.ctx, phi, pairs, E, V)
    hfx.hfx_sync_status(ex.ctx)
    assert hfx.hfx_test_live_allocations() == live1 + n_sched
    assert E.item() == E_ref.item()
    assert torch.equal(V, V_ref)
    ex.close()
    ref.close()


def test_batched_call_fails_cleanly_when_its_tables_cannot_be_allocated():
    from paper_2309_00651_gb300 import hfx
    probs = [_workload(16, 2), _workload(12, 3)]
    exs = []
    for lat, grid, phi, pairs in probs:
        ex = hfx.Exchange(lat, grid, alpha=0.25, precision="fp32")
        ex.ensure_workspace(phi.shape[0], len(pairs))
        ex.apply(phi, pairs)  # the schedules exist: the batch tables are the call's only allocation
        ex.sync_status()
        exs.append(ex)
    ctxs = [e.ctx for e in exs]
    Es = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in probs]
    Vs = [torch.empty_like(p[2]) for p in probs]
    args = [(p[2], p[3], E, V, 0) for p, E, V in zip(probs, Es, Vs)]
    live1 = hfx.hfx_test_live_allocations()
    hfx.hfx_test_fail_allocation(0)
    _expect_oom(lambda: hfx.hfx_apply_batched(ctxs, args))
    assert hfx.hfx_test_live_allocations() == live1
    hfx.hfx_apply_batched(ctxs, args)
    for e in exs:
        e.sync_status()
    assert hfx.hfx_test_live_allocations() == live1 + 1
    # the same batch on contexts that never saw a failure
    fresh = [hfx.Exchange(p[0], p[1], alpha=0.25, precision="fp32") for p in probs]
    for f, p in zip(fresh, probs):
        f.ensure_workspace(p[2].shape[0], len(p[3]))
    Es2 = [torch.zeros(1, dtype=torch.float64, device="cuda") for _ in probs]
    Vs2 = [torch.empty_like(p[2]) for p in probs]
    hfx.hfx_apply_batched([f.ctx for f in fresh], [(p[2], p[3], E, V, 0) for p, E, V in zip(probs, Es2, Vs2)])
    for f in fresh:
        f.sync_status()
    for E, V, E2, V2 in zip(Es, Vs, Es2, Vs2):
        assert abs(E.item() - E2.item()) <= 1e-6 * abs(E2.item())
        assert float(torch.linalg.norm(V - V2) / torch.linalg.norm(V2)) <= 1e-6
    for e in exs + fresh:
        e.close()
