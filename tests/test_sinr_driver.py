"""Host logic of the XI-RESPA outer step (paper_2309_00651_gb300/sinr.py) on the CPU: the order of
the update calls within one outer step (appendix updates A, B, C in the factorisation of eq.
trotter-sinr), where the slow kick n_MTS F_slow enters, and the position at which the last slow
force is evaluated.  The library's update entry points are replaced by recorders, so nothing runs
on a GPU; the arithmetic of the updates is covered against the oracle in test_gpu_sinr.py."""
import types

import pytest

torch = pytest.importorskip("torch")

from paper_2309_00651_gb300 import sinr as S  # noqa: E402


class Recorder:
    """Stands in for the binding: logs each call; update C moves X by V dt so that forces taken
    after it see the new position."""

    def __init__(self):
        self.calls = []

    def module(self):
        rec = self

        def update_n(p, dt, mass, V, v1, v2, n_res, n_sy):
            rec.calls.append(("A", dt, n_res, n_sy))

        def update_v(p, dt, mass, force, V, v1, extra=None):
            rec.calls.append(("B", dt, float(force[0]), None if extra is None else float(extra[0])))

        def update_x(p, dt, V, X, v2, R):
            X += V * dt
            rec.calls.append(("C", dt, float(R[0, 0])))

        return types.SimpleNamespace(HfxSinrParams=lambda *a: a, hfx_sinr_update_n=update_n,
                                     hfx_sinr_update_v=update_v, hfx_sinr_update_x=update_x)


@pytest.mark.parametrize("n_mts", [1, 3])
def test_outer_step_call_order_and_slow_kicks(monkeypatch, n_mts):
    rec = Recorder()
    monkeypatch.setattr(S, "hfx", rec.module())
    integ = S.SinR(kT=0.0019, Q1=3.0, Q2=4.0, gamma=0.01, L=4, n_res=2, n_sy=3)
    n = 5
    X = torch.zeros(n, dtype=torch.float64)
    V = torch.ones(n, dtype=torch.float64)
    v1 = torch.zeros(n, 4, dtype=torch.float64)
    v2 = torch.zeros(n, 4, dtype=torch.float64)
    mass = torch.ones(n, dtype=torch.float64)
    dt = 0.5
    draws = iter(range(100))
    fast = lambda x: 10.0 + x          # noqa: E731  (fast force at position x)
    slow = lambda x: 100.0 + x         # noqa: E731  (slow force at position x)
    integ.outer(X, V, v1, v2, mass, fast, slow, dt, n_mts,
                lambda: torch.full((n, 4), float(next(draws)), dtype=torch.float64))
    kinds = "".join(c[0] for c in rec.calls)
    assert kinds == "ABCBA" * n_mts
    # every update gets the inner step and A its n_res x n_sy factorisation
    assert all(c[1] == dt for c in rec.calls)
    assert all(c[2:] == (2, 3) for c in rec.calls if c[0] == "A")
    # one draw per inner factor, in order
    assert [c[2] for c in rec.calls if c[0] == "C"] == [float(k) for k in range(n_mts)]
    b = [c for c in rec.calls if c[0] == "B"]
    # X advances by V dt = 0.5 at each C: the k-th factor's B kicks see X = k/2 and (k+1)/2
    for k in range(n_mts):
        assert b[2 * k][2] == 10.0 + 0.5 * k
        assert b[2 * k + 1][2] == 10.0 + 0.5 * (k + 1)
    # slow kick n_MTS F_slow: on the first B (at the start position) and the last B (at the
    # position after the last C); no other kick carries it
    assert b[0][3] == n_mts * (100.0 + 0.0)
    assert b[-1][3] == n_mts * (100.0 + 0.5 * n_mts)
    assert all(c[3] is None for c in b[1:-1])
    if n_mts == 1:
        assert len(b) == 2
