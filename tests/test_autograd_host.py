"""The autograd wrapper's own logic on the CPU (paper_2309_00651_gb300/autograd.py): the backward
pass is grad_E * 2 (Omega/N) V_x phi, with V_x phi kept from the forward call or, with
recompute=True, from a second full call made only in the backward pass.  The library call is
replaced here by a stand-in that evaluates the FP64 oracle on CPU tensors, so the test checks the
wrapper (scale, chain rule, what is saved, when the second call happens), not the CUDA path
(tests/test_gpu_autograd.py does that)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hfx_oracle as O  # noqa: E402
from paper_2309_00651_gb300 import autograd as A  # noqa: E402
from paper_2309_00651_gb300 import inputs as I  # noqa: E402


class OracleExchange:
    """Stand-in for hfx.Exchange with the same apply() contract, evaluated by the oracle."""

    def __init__(self, L, n):
        self.lattice = np.diag([L] * 3)
        self.volume = L ** 3
        self.npoints = n ** 3
        self.calls = []

    def apply(self, phi, pairs, energy_only=False):
        self.calls.append("energy" if energy_only else "full")
        E, V = O.exchange(phi.numpy(), pairs.numpy(), self.lattice, want_v=not energy_only)
        E_t = torch.tensor([E], dtype=torch.float64)
        return E_t, (None if energy_only else torch.from_numpy(V))


def _case():
    L, n, n_orb = 6.0, 8, 4
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=0.5 * (2 * np.pi * 2.5 / L) ** 2, seed=3)
    phi, _ = I.loewdin(raw, L ** 3)
    pairs = I.random_pairs_subset(I.all_pairs(n_orb), 7, seed=4)
    return L, n, torch.from_numpy(phi), torch.from_numpy(pairs)


@pytest.mark.parametrize("recompute", [False, True])
def test_backward_is_the_scaled_adjoint(recompute):
    L, n, phi, pairs = _case()
    ex = OracleExchange(L, n)
    x = phi.clone().requires_grad_(True)
    E = A.exchange_energy(ex, x, pairs, recompute=recompute)
    assert E.dim() == 0
    (3.0 * E).backward()  # the chain rule through an outer factor
    _, V = O.exchange(phi.numpy(), pairs.numpy(), ex.lattice)
    expect = 3.0 * 2.0 * (L ** 3 / n ** 3) * V
    assert np.allclose(x.grad.numpy(), expect, rtol=1e-12, atol=1e-15)
    # what ran: one full call, or an energy-only forward and a full call in the backward pass
    assert ex.calls == (["energy", "full"] if recompute else ["full"])


@pytest.mark.parametrize("recompute", [False, True])
def test_what_the_forward_pass_keeps(recompute):
    """Without recompute the forward pass keeps V_x phi for the backward pass; with it, only the
    orbitals (and no V_x phi has been computed yet)."""
    L, n, phi, pairs = _case()
    ex = OracleExchange(L, n)
    x = phi.clone().requires_grad_(True)
    E = A.exchange_energy(ex, x, pairs, recompute=recompute)
    grids = [t for t in E.grad_fn.saved_tensors if t.dim() == 4]
    assert len(grids) == 1
    _, V = O.exchange(phi.numpy(), pairs.numpy(), ex.lattice)
    if recompute:
        assert torch.equal(grids[0], phi) and ex.calls == ["energy"]
    else:
        assert np.array_equal(grids[0].numpy(), V) and ex.calls == ["full"]


def test_gradient_matches_finite_differences_of_the_wrapped_energy():
    """A directional derivative of the wrapped E_x by a 5-point stencil (E is a quartic along any
    direction, so the stencil is exact up to rounding) against <grad, d>."""
    L, n, phi, pairs = _case()
    ex = OracleExchange(L, n)
    x = phi.clone().requires_grad_(True)
    A.exchange_energy(ex, x, pairs).backward()
    d = torch.from_numpy(np.random.default_rng(5).standard_normal(phi.shape))
    h = 1e-3

    def e(t):
        return A.exchange_energy(ex, phi + t * d, pairs).item()
    fd = (-e(2 * h) + 8 * e(h) - 8 * e(-h) + e(-2 * h)) / (12 * h)
    assert abs(fd - float((x.grad * d).sum())) <= 1e-9 * abs(fd)
