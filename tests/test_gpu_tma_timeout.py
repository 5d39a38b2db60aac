"""Failure detection of the TMA dense accumulate pass without a GPU fault.

With HFX_TEST_STALL, the first tile barrier of every dense block expects 16 bytes more than its
tensor copy brings, so each block's wait can only end by running out of its time limit.  The
block then waits, again with a limit, for the copies it started, skips its flush and returns;
blocks that start later skip their work.  hfx_sync_status reports HFX_ERR_TIMEOUT, and the next
call on the same context gives the result of an ordinary call.
"""
import time

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


def test_dense_tma_wait_runs_out_and_is_reported(monkeypatch):
    from paper_2309_00651_gb300 import hfx
    monkeypatch.setenv("HFX_DENSE_TMA", "1")
    w = I.WORKLOADS["pw16_n32"]  # 16 orbitals on 32^3: one full off-diagonal block pair
    phi, pairs, _ = I.make_workload(w)
    ex = hfx.Exchange(w.lattice, phi.shape[1:], precision="fp32")
    phi_d = torch.from_numpy(phi).cuda()
    pairs_d = torch.from_numpy(pairs.astype(np.int32)).cuda()
    assert hfx.hfx_plan_stats(ex.ctx, phi.shape[0], len(pairs))["dense_couples"] > 0
    E_ref, V_ref = ex.apply(phi_d, pairs_d)
    E_ref, V_ref = E_ref.item(), V_ref.clone()
    ex.sync_status()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    V = torch.empty_like(phi_d)
    ex.ensure_workspace(phi.shape[0], len(pairs))
    t0 = time.time()
    hfx.hfx_apply(ex.ctx, phi_d, pairs_d, E, V, flags=hfx.HFX_TEST_STALL)
    torch.cuda.synchronize()
    assert time.time() - t0 < 60.0  # each resident block gives up after about a second
    with pytest.raises(hfx.HFXError) as ei:
        ex.sync_status()
    assert ei.value.status == -6  # HFX_ERR_TIMEOUT
    ex.sync_status()  # cleared
    E2, V2 = ex.apply(phi_d, pairs_d)
    ex.sync_status()
    assert E2.item() == E_ref
    assert torch.equal(V2, V_ref)
    ex.close()
