"""The autograd wrapper: backward = 2 (Omega/N) V_x phi, checked by 5-point finite differences
(exact for the quartic E(phi + eps d) up to rounding) and against the oracle's gradient."""
import math

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


def _setup(n_orb=12, n=24, L=11.0, seed=31, screen=False):
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=0.5 * (2 * math.pi * (n / 4 + 0.5) / L) ** 2, seed=seed)
    phi, _ = I.loewdin(raw, L ** 3)
    pairs = I.all_pairs(n_orb)
    if screen:
        pairs = pairs[::2]
    return phi, pairs, np.diag([L] * 3)


@pytest.mark.parametrize("recompute", [False, True])
@pytest.mark.parametrize("screen", [False, True])
def test_fd_directional_derivatives_fp64(recompute, screen):
    from paper_2309_00651_gb300 import hfx
    from paper_2309_00651_gb300.autograd import exchange_energy
    phi, pairs, lat = _setup(screen=screen)
    ex = hfx.Exchange(lat, phi.shape[1:], precision="fp64")
    phi_d = torch.from_numpy(phi).cuda().requires_grad_(True)
    pairs_d = torch.from_numpy(pairs).cuda()
    E = exchange_energy(ex, phi_d, pairs_d, recompute=recompute)
    (g,) = torch.autograd.grad(E, phi_d)
    # oracle gradient 2 (Omega/N) V_x phi
    _, V_ref = O.exchange(phi, pairs, lat)
    scale = 2 * lat[0, 0] ** 3 / phi[0].size
    assert float(torch.linalg.norm(g.cpu() - torch.from_numpy(scale * V_ref))) <= 1e-8 * float(
        np.linalg.norm(scale * V_ref))
    for s in range(1, 9):
        d = torch.from_numpy(np.random.default_rng(s).standard_normal(phi.shape)).cuda()
        h = 1e-3 * float(torch.linalg.norm(phi_d.detach())) / float(torch.linalg.norm(d))
        with torch.no_grad():
            Es = [exchange_energy(ex, phi_d.detach() + c * h * d, pairs_d).item() for c in (-2, -1, 1, 2)]
        fd = (Es[0] - 8 * Es[1] + 8 * Es[2] - Es[3]) / (12 * h)
        an = float(torch.sum(g * d))
        assert fd == pytest.approx(an, rel=1e-9)
    ex.close()


def test_fd_fp32_path_loose():
    """The FP32 path's gradient agrees with its own finite differences to the FP32 noise level."""
    from paper_2309_00651_gb300 import hfx
    from paper_2309_00651_gb300.autograd import exchange_energy
    phi, pairs, lat = _setup(seed=33)
    ex = hfx.Exchange(lat, phi.shape[1:], precision="fp32")
    phi_d = torch.from_numpy(phi).cuda().requires_grad_(True)
    pairs_d = torch.from_numpy(pairs).cuda()
    E = exchange_energy(ex, phi_d, pairs_d)
    (g,) = torch.autograd.grad(E, phi_d)
    d = torch.from_numpy(np.random.default_rng(3).standard_normal(phi.shape)).cuda()
    h = 1e-2 * float(torch.linalg.norm(phi_d.detach())) / float(torch.linalg.norm(d))
    with torch.no_grad():
        Es = [exchange_energy(ex, phi_d.detach() + c * h * d, pairs_d).item() for c in (-2, -1, 1, 2)]
    fd = (Es[0] - 8 * Es[1] + 8 * Es[2] - Es[3]) / (12 * h)
    assert fd == pytest.approx(float(torch.sum(g * d)), rel=1e-4)
    ex.close()
