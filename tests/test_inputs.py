"""The synthetic input generator: orthonormality, pair-list shapes and the workload rules."""
import numpy as np

from paper_2309_00651_gb300 import inputs as I


def test_smooth_even():
    assert I.smooth_even_at_least(47.3) == 48
    assert I.smooth_even_at_least(94.7) == 96
    assert I.smooth_even_at_least(49.0) == 50
    assert I.smooth_even_at_least(55.0) == 60
    for x in range(3, 200):
        n = I.smooth_even_at_least(x)
        assert n >= x and n % 2 == 0


def test_pw16_n32_workload():
    w = I.WORKLOADS["pw16_n32"]
    phi, pairs, info = I.make_workload(w)
    assert phi.shape == (16, 32, 32, 32) and phi.dtype == np.float64
    assert len(pairs) == 136 and info["n_pairs"] == 136
    S = (w.volume / 32 ** 3) * phi.reshape(16, -1) @ phi.reshape(16, -1).T
    assert np.allclose(S, np.eye(16), atol=1e-12)
    assert np.all(pairs[:, 0] <= pairs[:, 1])


def test_gaussian_orbitals_small():
    phi = I.gaussian_orbitals(8, 10.0, 24, 20.0, 1.2, seed=0)
    assert np.isfinite(phi).all()
    lo, cond = I.loewdin(phi, 1000.0)
    S = (1000.0 / 24 ** 3) * lo.reshape(8, -1) @ lo.reshape(8, -1).T
    assert np.allclose(S, np.eye(8), atol=1e-11)
    assert cond > 1.0


def test_batched_rules():
    ws = I.batched_workloads()
    assert len(ws) == 24
    for w in ws:
        assert 32 <= w.n_orb <= 256
        assert w.n >= 4.03 * w.L and w.n % 2 == 0
        assert abs(w.L ** 3 - I.WATER_VOLUME_BOHR3 * w.n_orb / 4) < 1e-6 * w.L ** 3
    grids = {w.n for w in ws}
    assert min(grids) >= 48 and max(grids) <= 96


def test_screened_pairs_keep_diagonal():
    phi = I.gaussian_orbitals(12, 12.0, 24, 20.0, 1.0, seed=1)
    phi, _ = I.loewdin(phi, 12.0 ** 3)
    p = I.screened_pairs(phi, 12.0 ** 3, 1e30)
    assert np.array_equal(p[:, 0], p[:, 1]) and len(p) == 12
    q = I.screened_pairs(phi, 12.0 ** 3, 0.0)
    assert len(q) == 12 * 13 // 2


def test_save_and_load_workload_round_trip(tmp_path):
    """Inputs saved with their record come back bit for bit, and the record alone rebuilds them."""
    w = I.Workload("small_gauss", 10, 11.0, 20, 20.0, "gauss", seed=5, sigma=1.1, screen=1e-6)
    phi, pairs, info = I.make_workload(w)
    path = str(tmp_path / "small_gauss.npz")
    I.save_workload(path, w, phi, pairs, info)
    w2, phi2, pairs2, info2 = I.load_workload(path)
    assert w2 == w
    assert phi2.dtype == np.float64 and np.array_equal(phi2, phi)
    assert pairs2.dtype == np.int32 and np.array_equal(pairs2, pairs)
    assert info2 == info
    phi3, pairs3, _ = I.make_workload(w2)
    assert np.array_equal(phi3, phi) and np.array_equal(pairs3, pairs)


def test_load_workload_rejects_unknown_format(tmp_path):
    import json
    path = str(tmp_path / "bad.npz")
    np.savez(path, phi=np.zeros((1, 2, 2, 2)), pairs=np.zeros((1, 2), np.int32),
             meta=np.array(json.dumps({"format": 99, "workload": {}, "info": {}})))
    import pytest
    with pytest.raises(ValueError, match="format"):
        I.load_workload(path)
