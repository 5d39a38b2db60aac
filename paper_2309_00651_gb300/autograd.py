"""E_x as a differentiable function of the orbitals.

`exchange_energy(exch, phi, pairs)` returns E_x (Eq. HFX) as a 0-dim float64 tensor whose
backward pass is the hand-written adjoint: dE_x/dphi_i(r) = 2 (Omega/N) (V_x phi)_i(r), with
V_x phi from Eq. vx computed by the same CUDA library call.  With `recompute=True` the forward
pass evaluates the energy only (no V_x phi kept in memory) and the backward pass runs the full
call again, trading a second evaluation for the memory of one orbital-sized FP64 array.
"""
from __future__ import annotations

import torch

from .hfx import Exchange


class HFXEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi: torch.Tensor, pairs: torch.Tensor, exch: Exchange, recompute: bool) -> torch.Tensor:
        phi_c = phi.detach().contiguous()
        E, V = exch.apply(phi_c, pairs, energy_only=recompute)
        ctx.exch = exch
        ctx.recompute = recompute
        ctx.scale = 2.0 * exch.volume / exch.npoints
        if recompute:
            ctx.save_for_backward(phi_c, pairs)
        else:
            ctx.save_for_backward(V, pairs)
        return E.reshape(())

    @staticmethod
    def backward(ctx, grad_E: torch.Tensor):
        saved, pairs = ctx.saved_tensors
        if ctx.recompute:
            _, V = ctx.exch.apply(saved, pairs)
        else:
            V = saved
        grad = (grad_E.to(torch.float64) * ctx.scale) * V
        return grad, None, None, None


def exchange_energy(exch: Exchange, phi: torch.Tensor, pairs: torch.Tensor, recompute: bool = False) -> torch.Tensor:
    """E_x for orbitals `phi` [n_orb, n1, n2, n3] (float64, CUDA) over `pairs` (int32 [P, 2], CUDA)."""
    return HFXEnergy.apply(phi, pairs, exch, recompute)
