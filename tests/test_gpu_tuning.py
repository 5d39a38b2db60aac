"""Schedule settings (block size, batch budget, pipelining) change speed, not results; the
autotuner picks one of them and remembers it."""
import json

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


def _problem():
    n, L, n_orb = 32, 10.0, 24
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=0.5 * (2 * np.pi * 8.5 / L) ** 2, seed=41)
    phi, _ = I.loewdin(raw, L ** 3)
    return phi, I.all_pairs(n_orb), np.diag([L] * 3)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("fp64", 1e-8)])
def test_settings_agree_with_oracle(prec, tol):
    from paper_2309_00651_gb300 import hfx
    phi, pairs, lat = _problem()
    E_ref, V_ref = O.exchange(phi, pairs, lat)
    ex = hfx.Exchange(lat, phi.shape[1:], precision=prec)
    phi_d = torch.from_numpy(phi).cuda()
    pairs_d = torch.from_numpy(pairs).cuda()
    for block, mb, pipe in [(8, 1024, True), (8, 4, True), (4, 8, False), (5, 16, True), (16, 64, False)]:
        ex.set_tuning(block, mb << 20, pipe)
        E, V = ex.apply(phi_d, pairs_d)
        ex.sync_status()
        assert abs(E.item() - E_ref) <= tol * abs(E_ref), (block, mb, pipe)
        assert float(np.linalg.norm(V.cpu().numpy() - V_ref)) <= tol * float(np.linalg.norm(V_ref)), (block, mb, pipe)
    ex.close()


def test_bad_tuning_is_rejected():
    from paper_2309_00651_gb300 import hfx
    ex = hfx.Exchange(np.diag([10.0] * 3), (32, 32, 32), precision="fp32")
    with pytest.raises(hfx.HFXError):
        ex.set_tuning(0, 1 << 30, True)
    with pytest.raises(hfx.HFXError):
        ex.set_tuning(8, 0, True)
    ex.close()


def test_autotuner_picks_and_caches(tmp_path):
    from paper_2309_00651_gb300 import autotune, hfx
    phi, pairs, lat = _problem()
    ex = hfx.Exchange(lat, phi.shape[1:], precision="fp32")
    phi_d = torch.from_numpy(phi).cuda()
    pairs_d = torch.from_numpy(pairs).cuda()
    path = str(tmp_path / "tune.json")
    cands = [{"block": 8, "batch_bytes": 1 << 30, "pipeline": True}, {"block": 4, "batch_bytes": 8 << 20, "pipeline": False}]
    r1 = autotune.tune(ex, phi_d, pairs_d, candidates=cands, steps=2, path=path)
    assert not r1["cached"] and r1["setting"] in cands and len(r1["trials"]) == 2
    with open(path) as f:
        table = json.load(f)
    assert autotune.shape_key(ex, phi.shape[0]) in table
    r2 = autotune.tune(ex, phi_d, pairs_d, candidates=cands, steps=2, path=path)
    assert r2["cached"] and r2["setting"] == r1["setting"]
    ex.close()
