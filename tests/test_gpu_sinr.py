"""GPU parity of the SIN(R) updates (appendix A, B, C) and of an XI-RESPA run against the FP64
oracle: ragged n_dof (not a multiple of the 256-thread block), chain lengths 1, 4 and 16,
Suzuki-Yoshida orders 1, 3, 5 with n_res = 2, both branches of update B (tiny and large forces),
the constraint Lambda_I = L kT after every update.  Tolerance 1e-12 relative (FP64; the device
exp/sinh/cosh/sqrt differ from the host's by an ulp or so)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sinr_oracle as S  # noqa: E402

pytestmark = pytest.mark.gpu

KT = 0.0019


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_00651_gb300 import build
    build.build()


def params(L, gamma=0.01):
    return {"kT": KT, "Q1": KT * 40.0 ** 2, "Q2": KT * 45.0 ** 2, "gamma": gamma, "L": L}


def state(n, L, seed):
    rng = np.random.default_rng(seed)
    p = params(L)
    M = rng.uniform(1000.0, 30000.0, n)
    V = rng.standard_normal(n) * 1e-3
    v1 = rng.standard_normal((n, L)) * math.sqrt(KT / p["Q1"])
    v2 = rng.standard_normal((n, L)) * math.sqrt(KT / p["Q2"])
    lam = S.constraint(M, V, v1, p["Q1"], L)
    f = np.sqrt(L * KT / lam)
    return M, V * f, v1 * f[:, None], v2


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.mark.parametrize("L", [1, 4, 16])
@pytest.mark.parametrize("n_sy", [1, 3, 5])
def test_update_a(L, n_sy):
    from paper_2309_00651_gb300 import hfx
    n = 1000
    M, V, v1, v2 = state(n, L, 10 + L + n_sy)
    p = params(L)
    Md, Vd, v1d, v2d = dev(M), dev(V), dev(v1), dev(v2)
    hfx.hfx_sinr_update_n(p, 30.0, Md, Vd, v1d, v2d, n_res=2, n_sy=n_sy)
    V0, v10, v20 = S.update_n_half_step(V, v1, v2, M, KT, p["Q1"], p["Q2"], L, 30.0, n_res=2, n_sy=n_sy)
    assert rel(Vd.cpu().numpy(), V0) < 1e-12
    assert rel(v1d.cpu().numpy(), v10) < 1e-12
    assert rel(v2d.cpu().numpy(), v20) < 1e-12
    lam = S.constraint(M, Vd.cpu().numpy(), v1d.cpu().numpy(), p["Q1"], L)
    assert np.allclose(lam, L * KT, rtol=1e-13, atol=0)


@pytest.mark.parametrize("fscale", [1e-12, 0.05])
@pytest.mark.parametrize("with_extra", [False, True])
def test_update_b(fscale, with_extra):
    from paper_2309_00651_gb300 import hfx
    n, L = 777, 4
    M, V, v1, _ = state(n, L, 3)
    p = params(L)
    rng = np.random.default_rng(4)
    F = rng.standard_normal(n) * fscale
    Fx = rng.standard_normal(n) * fscale if with_extra else None
    Vd, v1d = dev(V), dev(v1)
    hfx.hfx_sinr_update_v(p, 40.0, dev(M), dev(F), Vd, v1d, None if Fx is None else dev(Fx))
    V0, v10 = S.update_v(V, v1, F if Fx is None else F + Fx, M, KT, L, 40.0)
    assert rel(Vd.cpu().numpy(), V0) < 1e-12
    assert rel(v1d.cpu().numpy(), v10) < 1e-12
    lam = S.constraint(M, Vd.cpu().numpy(), v1d.cpu().numpy(), p["Q1"], L)
    assert np.allclose(lam, L * KT, rtol=1e-13, atol=0)


def test_update_c():
    from paper_2309_00651_gb300 import hfx
    n, L = 1025, 4
    rng = np.random.default_rng(5)
    X, V = rng.standard_normal(n), rng.standard_normal(n) * 1e-3
    v2, R = rng.standard_normal((n, L)) * 0.01, rng.standard_normal((n, L))
    p = params(L)
    Xd, v2d = dev(X), dev(v2)
    hfx.hfx_sinr_update_x(p, 20.0, dev(V), Xd, v2d, dev(R))
    X0, v20 = S.update_x(X, V, v2, R, KT, p["Q2"], p["gamma"], 20.0)
    assert rel(Xd.cpu().numpy(), X0) < 1e-15  # the device may fuse X + V dt into one rounding
    assert rel(v2d.cpu().numpy(), v20) < 1e-14


def test_xi_respa_run_matches_oracle():
    """Three outer steps (n_MTS = 4) with harmonic fast and slow forces, n_res = 2, n_sy = 3."""
    from paper_2309_00651_gb300.sinr import SinR
    n, L = 300, 4
    M, V, v1, v2 = state(n, L, 6)
    X = np.random.default_rng(7).standard_normal(n) * 0.1
    p = params(L)
    kf, ks, dt, n_mts = 0.3, 0.02, 20.0, 4
    draws = [np.random.default_rng(100 + k).standard_normal((n, L)) for k in range(3 * n_mts)]
    # oracle
    Xo, Vo, v1o, v2o = X.copy(), V.copy(), v1.copy(), v2.copy()
    c = 0
    for outer in range(3):
        for k in range(n_mts):
            Xo, Vo, v1o, v2o = S.xi_respa_inner(
                Xo, Vo, v1o, v2o, M, lambda x: -kf * x, KT, p["Q1"], p["Q2"], L, p["gamma"], dt, draws[c],
                n_res=2, n_sy=3, F_first=n_mts * (-ks * Xo) if k == 0 else None,
                F_last=(lambda x: n_mts * (-ks * x)) if k == n_mts - 1 else None)
            c += 1
    # GPU
    integ = SinR(p["kT"], p["Q1"], p["Q2"], p["gamma"], L, n_res=2, n_sy=3)
    Xd, Vd, v1d, v2d, Md = dev(X), dev(V), dev(v1), dev(v2), dev(M)
    it = iter(draws)
    for outer in range(3):
        integ.outer(Xd, Vd, v1d, v2d, Md, lambda x: -kf * x, lambda x: -ks * x, dt, n_mts, lambda: dev(next(it)))
        lam = integ.constraint(Md, Vd, v1d)
        assert float(torch.max(torch.abs(lam / (L * KT) - 1.0))) < 1e-12
    assert rel(Xd.cpu().numpy(), Xo) < 1e-11
    assert rel(Vd.cpu().numpy(), Vo) < 1e-11
    assert rel(v1d.cpu().numpy(), v1o) < 1e-11
    assert rel(v2d.cpu().numpy(), v2o) < 1e-11
