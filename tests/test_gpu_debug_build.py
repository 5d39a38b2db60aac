"""The HFX_DEBUG build (libhfx_debug.so, the stand-in for compute-sanitizer, which is closed on
this pool): guard bands between the workspace slices, filled before and checked after every call,
and a device-side check that every placed pair couple sits at its canonical place in its block
pair, both writing into the context's error word (no trap).

In a child process that loads the debug library: a small exchange on both precisions matches the
oracle and the release library bit for bit, the checks stay silent on a correct call, and a
workspace overwritten after the call (guard bands included) is reported as HFX_ERR_CORRUPTION.
The release library refuses the guard check with HFX_ERR_INVALID_ARG."""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2309_00651_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N, L, N_ORB = 24, 9.0, 13


def _inputs():
    raw = I.random_pw_orbitals(N_ORB, L, N, ecut=0.5 * (2 * math.pi * 5.5 / L) ** 2, seed=61)
    phi, _ = I.loewdin(raw, L ** 3)
    return phi, I.all_pairs(N_ORB)


CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
from oracle import hfx_oracle as O
from paper_2309_00651_gb300 import hfx, inputs as I
import math
raw = I.random_pw_orbitals({n_orb}, {L}, {n}, ecut=0.5 * (2 * math.pi * 5.5 / {L}) ** 2, seed=61)
phi, _ = I.loewdin(raw, {L} ** 3)
pairs = I.all_pairs({n_orb})
lat = np.diag([{L}] * 3)
E_ref, V_ref = O.exchange(phi, pairs, lat)
assert hfx.load_library()._name.endswith("libhfx_debug.so")
out = {{}}
for prec in ("fp64", "fp32"):
    ex = hfx.Exchange(lat, ({n}, {n}, {n}), precision=prec)
    E, V = ex.apply(torch.from_numpy(phi).cuda(), torch.from_numpy(pairs).cuda())
    ex.sync_status()
    hfx.hfx_debug_check_guards(ex.ctx)
    ex.sync_status()
    V = V.cpu().numpy()
    ex._ws.fill_(0)
    hfx.hfx_debug_check_guards(ex.ctx)
    try:
        ex.sync_status()
        status = 0
    except hfx.HFXError as e:
        status = e.status
    out[prec] = {{"E": repr(E.item()), "E_err": abs(E.item() - E_ref) / abs(E_ref),
                 "V_err": float(np.linalg.norm(V - V_ref) / np.linalg.norm(V_ref)), "after_overwrite": status}}
    ex.close()
print(json.dumps(out))
"""


@pytest.fixture(scope="module", autouse=True)
def _libs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_00651_gb300 import build
    build.build()
    build.build(debug=True)


def test_debug_build_checks_and_matches_release():
    from paper_2309_00651_gb300 import hfx
    phi, pairs = _inputs()
    lat = np.diag([L] * 3)
    release = {}
    for prec in ("fp64", "fp32"):
        ex = hfx.Exchange(lat, (N, N, N), precision=prec)
        E, _ = ex.apply(torch.from_numpy(phi).cuda(), torch.from_numpy(pairs).cuda())
        ex.sync_status()
        release[prec] = E.item()
        with pytest.raises(hfx.HFXError) as ei:  # the release library has no guard bands
            hfx.hfx_debug_check_guards(ex.ctx)
        assert ei.value.status == -1
        ex.close()
    env = dict(os.environ, HFX_DEBUG_LIB="1")
    code = CHILD.format(root=ROOT, n_orb=N_ORB, L=L, n=N)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for prec, tol in (("fp64", 1e-8), ("fp32", 1e-6)):
        assert res[prec]["E_err"] <= tol and res[prec]["V_err"] <= tol, res[prec]
        assert float(res[prec]["E"]) == release[prec]
        assert res[prec]["after_overwrite"] == -9
