"""XI-RESPA outer step of the SIN(R) integrator (Sec. 2.3, eq. trotter-sinr) over the library's
update entry points (include/hfx_sinr.h); forces come from caller-supplied callables.

One outer step of length n_MTS dt applies n_MTS inner factors, each
    A(dt/2)  B(dt/2; F_fast)  C(dt)  B(dt/2; F_fast at the new X)  A(dt/2),
with the slow kick n_MTS F_slow added to the first B of the first inner factor and to the last B
of the last one.  The updates A, B and C run in the CUDA library; this module orders the calls.
Two things here are plain torch work on the caller's tensors rather than library kernels: the
slow kick's scaling n_MTS F_slow (one multiply per element, passed to update B as its extra
force) and constraint(), the diagnostic sum M V^2 + L/(L+1) Q1 sum v1^2 of eq. kecons.
"""
from __future__ import annotations

from typing import Callable, Optional

import torch

from . import hfx


class SinR:
    def __init__(self, kT: float, Q1: float, Q2: float, gamma: float, L: int, n_res: int = 1, n_sy: int = 1):
        self.params = hfx.HfxSinrParams(kT, Q1, Q2, gamma, L)
        self.n_res, self.n_sy = int(n_res), int(n_sy)

    def constraint(self, mass: torch.Tensor, V: torch.Tensor, v1: torch.Tensor) -> torch.Tensor:
        """Isokinetic constraint value per degree of freedom (eq. kecons), a diagnostic in torch."""
        L = self.params.L
        return mass * V * V + (L / (L + 1.0)) * self.params.Q1 * torch.sum(v1 * v1, dim=-1)

    def inner(self, X, V, v1, v2, mass, fast_force: Callable[[torch.Tensor], torch.Tensor], dt: float,
              R: torch.Tensor, slow_first: Optional[torch.Tensor] = None,
              slow_last: Optional[torch.Tensor] = None) -> None:
        p = self.params
        hfx.hfx_sinr_update_n(p, dt, mass, V, v1, v2, self.n_res, self.n_sy)
        hfx.hfx_sinr_update_v(p, dt, mass, fast_force(X), V, v1, slow_first)
        hfx.hfx_sinr_update_x(p, dt, V, X, v2, R)
        hfx.hfx_sinr_update_v(p, dt, mass, fast_force(X), V, v1, slow_last)
        hfx.hfx_sinr_update_n(p, dt, mass, V, v1, v2, self.n_res, self.n_sy)

    def outer(self, X, V, v1, v2, mass, fast_force, slow_force: Callable[[torch.Tensor], torch.Tensor], dt: float,
              n_mts: int, draw: Callable[[], torch.Tensor]) -> None:
        """One outer step (n_mts >= 1 inner factors); `draw()` returns standard normal [n_dof, L]."""
        for k in range(n_mts):
            first = n_mts * slow_force(X) if k == 0 else None
            if k == n_mts - 1:
                # the slow force of the last kick is taken at the position after this factor's C
                p = self.params
                hfx.hfx_sinr_update_n(p, dt, mass, V, v1, v2, self.n_res, self.n_sy)
                hfx.hfx_sinr_update_v(p, dt, mass, fast_force(X), V, v1, first)
                hfx.hfx_sinr_update_x(p, dt, V, X, v2, draw())
                hfx.hfx_sinr_update_v(p, dt, mass, fast_force(X), V, v1, n_mts * slow_force(X))
                hfx.hfx_sinr_update_n(p, dt, mass, V, v1, v2, self.n_res, self.n_sy)
            else:
                self.inner(X, V, v1, v2, mass, fast_force, dt, draw(), first, None)
