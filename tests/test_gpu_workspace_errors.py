"""A caller workspace that is missing or short: hfx_apply returns HFX_ERR_OOM before it enqueues any
work, and the same context computes the right result once the caller hands it enough memory."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hfx_oracle as O  # noqa: E402
from paper_2309_00651_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

OOM = -3  # HFX_ERR_OOM


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_00651_gb300 import build
    build.build()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_missing_or_short_workspace_is_refused_then_recovered(prec):
    from paper_2309_00651_gb300 import hfx
    L, n, n_orb = 8.0, 16, 6
    lat = np.diag([L] * 3)
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=0.5 * (2 * np.pi * 4.5 / L) ** 2, seed=8)
    phi_np, _ = I.loewdin(raw, L ** 3)
    pairs_np = I.all_pairs(n_orb)
    phi = torch.from_numpy(phi_np).cuda()
    pairs = torch.from_numpy(pairs_np).cuda()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    V = torch.zeros_like(phi)
    ctx = hfx.hfx_create(lat, (n, n, n), 0.0, "coulomb", 0.25, prec)
    try:
        # no workspace at all
        with pytest.raises(hfx.HFXError) as ei:
            hfx.hfx_apply(ctx, phi, pairs, E, V)
        assert ei.value.status == OOM
        # 256 bytes short of what hfx_workspace_bytes asks for
        need = hfx.hfx_workspace_bytes(ctx, n_orb, len(pairs_np))
        assert need > 256
        short = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
        hfx.hfx_set_workspace(ctx, short)
        with pytest.raises(hfx.HFXError) as ei:
            hfx.hfx_apply(ctx, phi, pairs, E, V)
        assert ei.value.status == OOM
        torch.cuda.synchronize()
        assert E.item() == 0.0 and float(V.abs().max()) == 0.0  # nothing ran
        # enough memory: the same context gives the oracle's result
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
        hfx.hfx_set_workspace(ctx, ws)
        hfx.hfx_apply(ctx, phi, pairs, E, V)
        hfx.hfx_sync_status(ctx)
        E_ref, V_ref = O.exchange(phi_np, pairs_np, lat)
        tol = 1e-6 if prec == "fp32" else 1e-8
        assert abs(E.item() - E_ref) <= tol * abs(E_ref)
        V_np = V.cpu().numpy()
        assert np.linalg.norm(V_np - V_ref) <= tol * np.linalg.norm(V_ref)
    finally:
        hfx.hfx_destroy(ctx)
