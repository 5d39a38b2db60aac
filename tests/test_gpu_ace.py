"""GPU parity of the ACE operator and the overlap screen against the FP64 oracle.

* construction (M, L, P) and application, FP64 and FP32 contexts, on grids that span several
  split runs with a ragged tail (10^3 and 18^3 points: 62.5 and 364.5 stages of 16), orbital
  counts below,
  at and above one 128-row tile, and operands whose 8-byte offset forces the 8-byte copy path;
* the defining property on the occupied span (V_x^ACE psi_i = W_i) with W from the exchange
  entry point itself;
* accumulate, a non-positive-definite -M reported through the device error word, a short
  workspace rejected on the host;
* the Cholesky factorisation on both sides of the cluster kernel's size limit (200, 256, 257);
* the screen: s against the oracle, the kept-pair list identical (FP64) or identical away from
  the cut (FP32).

Tolerances: FP64 1e-10 relative (sums reassociated over the split runs), FP32 1e-6 relative
(operands rounded once to FP32, sums of at most 256 terms in FP32, FP64 beyond).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ace_oracle as A  # noqa: E402
from oracle import hfx_oracle as O  # noqa: E402
from paper_2309_00651_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_00651_gb300 import build
    build.build()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def small_orbitals(n_orb, n, L, seed):
    ecut = 0.5 * (2 * math.pi * (n / 4 + 0.5) / L) ** 2
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=ecut, seed=seed)
    phi, _ = I.loewdin(raw, L ** 3)
    return phi


def synthetic_action(phi, seed):
    """W = A phi with A symmetric negative definite: a valid exchange-like action, M = A."""
    n = phi.shape[0]
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    Aneg = -(B @ B.T / n + 0.5 * np.eye(n))
    return np.einsum("kl,l...->k...", Aneg, phi)


def localised(n_orb, n, L, seed, sigma=0.9):
    """Periodic Gaussians exp(-d^2 / 2 sigma^2) at random centres (minimum image): overlaps that
    spread from ~1 down to far below any cut."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0, L, size=(n_orb, 3))
    x = np.arange(n) * (L / n)
    out = np.empty((n_orb, n, n, n))
    for i in range(n_orb):
        d = [(x - c[i, a] + L / 2) % L - L / 2 for a in range(3)]
        r2 = d[0][:, None, None] ** 2 + d[1][None, :, None] ** 2 + d[2][None, None, :] ** 2
        out[i] = np.exp(-r2 / (2 * sigma * sigma)) * (1 if i % 2 else -1)
    return out


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def make_exchange(L, n, precision):
    from paper_2309_00651_gb300 import hfx
    return hfx.Exchange(np.diag([L, L, L]), (n, n, n), precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n_orb,n,seed", [(6, 10, 1), (128, 16, 2), (130, 18, 3)])
def test_build_and_apply_parity(precision, n_orb, n, seed):
    L = 7.0 + 0.1 * seed
    lat = np.diag([L, L, L])
    phi = small_orbitals(n_orb, n, L, seed)
    if n_orb <= 8:
        _, W = O.exchange(phi, I.all_pairs(n_orb), lat)
    else:
        W = synthetic_action(phi, seed)
    M0, L0, P0 = A.ace_build(phi, W, lat)
    ex = make_exchange(L, n, precision)
    M, Lf, P = ex.ace_build(dev(phi), dev(W))
    ex.sync_status()
    tol = TOL[precision]
    assert rel(M.cpu().numpy(), M0) < tol
    assert rel(Lf.cpu().numpy(), L0) < 10 * tol
    assert np.all(np.triu(Lf.cpu().numpy(), 1) == 0)
    assert rel(P.cpu().numpy(), P0) < 10 * tol
    psi = np.random.default_rng(seed + 10).standard_normal((n_orb + 3, n, n, n))
    Y = ex.ace_apply(P, dev(psi))
    assert rel(Y.cpu().numpy(), A.ace_apply(P0, psi, lat)) < 10 * tol
    # accumulate: out += V_ACE psi
    base = np.random.default_rng(seed + 20).standard_normal(psi.shape)
    out = dev(base)
    ex.ace_apply(P, dev(psi), out=out, accumulate=True)
    assert rel(out.cpu().numpy(), base + A.ace_apply(P0, psi, lat)) < 10 * tol
    ex.sync_status()
    ex.close()


@pytest.mark.parametrize("no_tc", ["0", "1"])
@pytest.mark.parametrize("n_orb,n_psi,n,seed", [(40, 40, 18, 4), (120, 270, 16, 5), (200, 64, 18, 6)])
def test_tensor_core_and_simt_contractions(no_tc, n_orb, n_psi, n, seed, monkeypatch):
    """FP32 contexts run the grid contractions on the tensor cores (tcgen05, TF32 x 3 split
    products, FP32 accumulation in TMEM); HFX_NO_TC=1 keeps them on the FP32 SIMT kernels.  Both
    against the oracle: M (Gram form, several output tiles when n_orb > 128), P and V_x^ACE psi
    (left multiply with up to 128 or 256 columns; 270 functions exceed that and take the SIMT
    kernel), and the screen (absolute values)."""
    monkeypatch.setenv("HFX_NO_TC", no_tc)
    L = 7.5
    lat = np.diag([L, L, L])
    phi = small_orbitals(n_orb, n, L, seed)
    W = synthetic_action(phi, seed)
    M0, L0, P0 = A.ace_build(phi, W, lat)
    ex = make_exchange(L, n, "fp32")
    M, Lf, P = ex.ace_build(dev(phi), dev(W))
    psi = np.random.default_rng(seed + 10).standard_normal((n_psi, n, n, n))
    Y = ex.ace_apply(P, dev(psi))
    ex.sync_status()
    assert rel(M.cpu().numpy(), M0) < TOL["fp32"]
    assert rel(P.cpu().numpy(), P0) < 10 * TOL["fp32"]
    Y0 = A.ace_apply(P0, psi, lat)
    assert rel(Y.cpu().numpy(), Y0) < 10 * TOL["fp32"]
    assert np.max(np.abs(Y.cpu().numpy() - Y0)) < 10 * TOL["fp32"] * np.max(np.abs(Y0))
    ex.close()


@pytest.mark.parametrize("n_orb", [200, 256, 257])
def test_cholesky_paths(n_orb):
    # 200 and 256 orbitals: the cluster factorisation with one and two local rows per warp (256 is
    # its largest size); 257: the single-block factorisation with A in global scratch
    n, L = 12, 6.0
    lat = np.diag([L, L, L])
    N = n ** 3
    q, _ = np.linalg.qr(np.random.default_rng(n_orb).standard_normal((N, n_orb)))
    phi = (q.T * math.sqrt(N / L ** 3)).reshape(n_orb, n, n, n)
    W = synthetic_action(phi, n_orb + 1)
    M0, L0, P0 = A.ace_build(phi, W, lat)
    ex = make_exchange(L, n, "fp64")
    M, Lf, P = ex.ace_build(dev(phi), dev(W))
    ex.sync_status()
    assert rel(M.cpu().numpy(), M0) < TOL["fp64"]
    assert rel(Lf.cpu().numpy(), L0) < 10 * TOL["fp64"]
    assert np.all(np.triu(Lf.cpu().numpy(), 1) == 0)
    assert rel(P.cpu().numpy(), P0) < 10 * TOL["fp64"]
    ex.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_eight_byte_aligned_operands(precision):
    # operands at an 8-byte (not 16-byte) offset take the 8-byte copy path
    n_orb, n, L = 20, 12, 6.5
    lat = np.diag([L, L, L])
    phi = small_orbitals(n_orb, n, L, 5)
    W = synthetic_action(phi, 5)
    M0, L0, P0 = A.ace_build(phi, W, lat)
    ex = make_exchange(L, n, precision)
    N = n ** 3

    def offset_copy(x):
        buf = torch.empty(x.size + 1, dtype=torch.float64, device="cuda")
        v = buf[1:].view(x.shape)
        v.copy_(dev(x))
        assert v.data_ptr() % 16 == 8
        return v

    phid, Wd = offset_copy(phi), offset_copy(W)
    M, Lf, P = ex.ace_build(phid, Wd)
    tol = TOL[precision]
    assert rel(M.cpu().numpy(), M0) < tol
    assert rel(P.cpu().numpy(), P0) < 10 * tol
    Y = ex.ace_apply(P, phid)
    assert rel(Y.cpu().numpy(), A.ace_apply(P0, phi, lat)) < 10 * tol
    ex.sync_status()
    ex.close()
    assert N == phid[0].numel()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_exact_on_occupied_span_with_gpu_exchange(precision):
    n_orb, n, L = 24, 16, 8.0
    phi = small_orbitals(n_orb, n, L, 7)
    ex = make_exchange(L, n, precision)
    phid = dev(phi)
    E, W = ex.apply(phid, dev(I.all_pairs(n_orb)))
    M, Lf, P = ex.ace_build(phid, W)
    Y = ex.ace_apply(P, phid)
    ex.sync_status()
    tol = TOL[precision]
    assert float(torch.linalg.norm(Y - W) / torch.linalg.norm(W)) < 10 * tol
    # 1/2 tr M is the exchange energy (homogeneity)
    assert 0.5 * float(torch.trace(M)) == pytest.approx(E.item(), rel=10 * tol)
    ex.close()


def test_not_positive_definite_is_reported():
    from paper_2309_00651_gb300 import hfx
    n_orb, n, L = 8, 8, 6.0
    phi = small_orbitals(n_orb, n, L, 9)
    ex = make_exchange(L, n, "fp64")
    phid = dev(phi)
    ex.ace_build(phid, phid)  # W = +phi: M = +I, so -M is negative definite
    with pytest.raises(hfx.HFXError) as e:
        ex.sync_status()
    assert e.value.status == -7
    ex.sync_status()  # the error word was cleared
    ex.close()


def test_short_workspace_rejected_on_host():
    from paper_2309_00651_gb300 import hfx
    ex = make_exchange(6.0, 8, "fp32")
    phi = dev(small_orbitals(4, 8, 6.0, 1))
    need = hfx.hfx_ace_workspace_bytes(ex.ctx, 4, 0)
    ws = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    p = torch.empty_like(phi)
    with pytest.raises(hfx.HFXError) as e:
        hfx.hfx_ace_build(ex.ctx, phi, phi, None, None, p, ws)
    assert e.value.status == -3
    ex.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n_orb,n", [(9, 10), (140, 12)])
def test_screen_parity(precision, n_orb, n):
    L = 9.0
    lat = np.diag([L, L, L])
    phi = localised(n_orb, n, L, seed=4)
    s0 = A.overlap_screen(phi, lat)
    # a cut halfway between two neighbouring values, so that both sides decide every pair alike
    v = np.sort(s0[np.triu_indices(n_orb, 1)])
    k = int(0.4 * len(v))
    cut = float(0.5 * (v[k] + v[k + 1]))
    pairs0, _ = A.screen_pairs(phi, lat, cut)
    ex = make_exchange(L, n, precision)
    pairs, s = ex.screen_pairs(dev(phi), cut)
    ex.sync_status()
    s = s.cpu().numpy()
    assert rel(s, s0) < TOL[precision]
    assert np.array_equal(s, s.T)
    got = pairs.cpu().numpy()
    if precision == "fp64":
        assert np.array_equal(got, pairs0)
    else:
        # identical away from the cut; near it each side decides in its own precision
        near = np.abs(s0 - cut) <= 1e-5 * cut
        key = lambda P: {(int(i), int(j)) for i, j in P if not near[i, j]}
        assert key(got) == key(pairs0)
        k = got[:, 0].astype(np.int64) * n_orb + got[:, 1]
        assert np.all(np.diff(k) > 0) and np.all(got[:, 0] <= got[:, 1])
        assert all((i, i) in {(int(a), int(b)) for a, b in got} for i in range(n_orb))
    ex.close()


# ----------------------------------------------------------------------------- SCDM localisation
# Pivots: FP64 picks equal the oracle's greedy picks; FP32 picks are checked for validity (each is
# within a relative 1e-4 of the largest FP64 residual norm available at its step, given the
# earlier picks).  Q and Phi are compared with the oracle's, formed from the GPU's own pivots.

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n_orb,n,seed", [(6, 10, 31), (40, 12, 32), (130, 18, 33)])
def test_scdm_parity(precision, n_orb, n, seed):
    L = 8.0
    lat = np.diag([L, L, L])
    phi = small_orbitals(n_orb, n, L, seed)
    ex = make_exchange(L, n, precision)
    piv, Q, Phi = ex.scdm_localise(dev(phi))
    ex.sync_status()
    piv = piv.cpu().numpy()
    assert len(set(piv.tolist())) == n_orb and piv.min() >= 0 and piv.max() < n ** 3
    slack = A.scdm_pivot_slack(phi, piv)
    if precision == "fp64":
        ref_piv, _, _ = A.scdm_pivots(phi)
        assert np.array_equal(piv, ref_piv)
    else:
        assert slack.min() >= 1 - 1e-4
    _, Q0, Phi0 = A.scdm_localise(phi, piv)
    tol = TOL[precision]
    assert rel(Q.cpu().numpy(), Q0) < 10 * tol
    assert rel(Phi.cpu().numpy(), Phi0) < 10 * tol
    S = A.grid_inner(Phi.cpu().numpy(), Phi.cpu().numpy(), lat)
    assert np.max(np.abs(S - np.eye(n_orb))) < 10 * tol
    ex.close()


def test_scdm_recovers_disjoint_boxes():
    n, L = 8, 6.0
    w = L ** 3 / n ** 3
    boxes = [(slice(0, 2), slice(0, 3), slice(0, 4)), (slice(3, 6), slice(0, 2), slice(0, 8)),
             (slice(6, 8), slice(4, 8), slice(2, 5)), (slice(0, 4), slice(5, 8), slice(6, 8))]
    loc = np.zeros((4, n, n, n))
    for k, b in enumerate(boxes):
        loc[k][b] = 1.0
        loc[k] /= np.sqrt(w * np.sum(loc[k] ** 2))
    U, _ = np.linalg.qr(np.random.default_rng(3).standard_normal((4, 4)))
    psi = np.einsum("ki,k...->i...", U, loc)
    for precision in ("fp64", "fp32"):
        ex = make_exchange(L, n, precision)
        _, _, Phi = ex.scdm_localise(dev(psi))
        ex.sync_status()
        O = w * Phi.cpu().numpy().reshape(4, -1) @ loc.reshape(4, -1).T
        assert np.allclose(np.sort(np.abs(O), axis=1)[:, -1], 1.0, atol=1e-6)
        assert np.allclose(np.sort(np.abs(O), axis=1)[:, :-1], 0.0, atol=1e-6)
        ex.close()


def test_scdm_rank_deficient_is_reported():
    from paper_2309_00651_gb300 import hfx
    n, L = 8, 6.0
    phi = small_orbitals(5, n, L, 34)
    phi = np.concatenate([phi, phi[:1]])  # a repeated orbital: rank 5 of 6
    ex = make_exchange(L, n, "fp64")
    ex.scdm_localise(dev(phi))
    with pytest.raises(hfx.HFXError) as e:
        ex.sync_status()
    assert e.value.status == -8
    ex.close()
