"""ctypes binding of libhfx (include/hfx.h, include/hfx_ace.h): same entry points, torch tensors in, no compute here.

Every step of the exchange path runs in the CUDA library; this module only marshals device
pointers, sizes and the current CUDA stream.  If libhfx.so is missing it raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhfx.so")
LIB_DEBUG_PATH = os.path.join(_PKG, "libhfx_debug.so")

HFX_OK = 0
STATUS_NAMES = {0: "HFX_OK", -1: "HFX_ERR_INVALID_ARG", -2: "HFX_ERR_UNSUPPORTED_GRID", -3: "HFX_ERR_OOM",
                -4: "HFX_ERR_CUDA", -5: "HFX_ERR_BAD_PAIR_LIST", -6: "HFX_ERR_TIMEOUT",
                -7: "HFX_ERR_NOT_POSITIVE_DEFINITE", -8: "HFX_ERR_RANK_DEFICIENT",
                -9: "HFX_ERR_CORRUPTION"}
PRECISION = {"fp64": 0, "fp32": 1, "mixed_tc": 2}
KERNEL = {"coulomb": 0, "coulomb_sphere": 1}
HFX_ENERGY_ONLY = 0x1
HFX_ACCUMULATE = 0x2
HFX_ORBITALS_F32 = 0x4
HFX_TEST_STALL = 0x100

# every symbol include/hfx.h and include/hfx_ace.h declare
EXPORTED = ("hfx_create", "hfx_workspace_bytes", "hfx_set_workspace", "hfx_apply", "hfx_apply_batched",
            "hfx_apply_sequential", "hfx_set_wait_budget", "hfx_apply_noalloc", "hfx_sync_status", "hfx_set_tuning", "hfx_plan_stats", "hfx_profile_enable",
            "hfx_profile_read",
            "hfx_last_error", "hfx_destroy",
            "hfx_ace_workspace_bytes", "hfx_ace_build", "hfx_ace_apply", "hfx_screen_pairs", "hfx_ace_profile_read",
            "hfx_scdm_workspace_bytes", "hfx_scdm_localise",
            "hfx_sinr_update_n", "hfx_sinr_update_v", "hfx_sinr_update_x", "hfx_fma_peak",
            "hfx_debug_check_guards", "hfx_test_fail_allocation", "hfx_test_live_allocations")
HFX_NOALLOC_SCRATCH_BYTES = 32 << 20
PASS_NAMES = ("stage", "fwd_yz", "x_coulomb", "y_acc_dense", "energy", "y_acc_generic")
ACE_KERNEL_NAMES = ("ace_gram", "ace_lmul", "ace_small")


class HfxBox(ctypes.Structure):
    _fields_ = [("lattice", (ctypes.c_double * 3) * 3)]


class HfxApplyArgs(ctypes.Structure):
    _fields_ = [("orbitals", ctypes.c_void_p), ("n_orb", ctypes.c_int32), ("pairs", ctypes.c_void_p),
                ("n_pairs", ctypes.c_int64), ("flags", ctypes.c_uint32), ("ex_dev", ctypes.c_void_p),
                ("vxphi", ctypes.c_void_p)]


class HfxSinrParams(ctypes.Structure):
    _fields_ = [("kT", ctypes.c_double), ("Q1", ctypes.c_double), ("Q2", ctypes.c_double),
                ("gamma", ctypes.c_double), ("L", ctypes.c_int32)]


class HFXError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libhfx.so (built by paper_2309_00651_gb300.build.build()), or libhfx_debug.so when the
    environment sets HFX_DEBUG_LIB=1 (build(debug=True)); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = LIB_DEBUG_PATH if os.environ.get("HFX_DEBUG_LIB") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libhfx.so not found at {path}: build it with paper_2309_00651_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, u32, dbl, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                   ctypes.c_double, ctypes.c_size_t)
    L.hfx_create.argtypes = [ctypes.POINTER(HfxBox), ctypes.POINTER(i32), dbl, ctypes.c_int, dbl, ctypes.c_int,
                             ctypes.POINTER(vp)]
    L.hfx_create.restype = ctypes.c_int
    L.hfx_workspace_bytes.argtypes = [vp, i32, i64]
    L.hfx_workspace_bytes.restype = sz
    L.hfx_set_workspace.argtypes = [vp, vp, sz]
    L.hfx_set_workspace.restype = ctypes.c_int
    L.hfx_apply.argtypes = [vp, vp, i32, vp, i64, u32, vp, vp, vp]
    L.hfx_apply.restype = ctypes.c_int
    L.hfx_apply_noalloc.argtypes = [vp, vp, i32, vp, i64, u32, vp, vp, vp]
    L.hfx_apply_noalloc.restype = ctypes.c_int
    L.hfx_apply_batched.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(HfxApplyArgs), i32, vp]
    L.hfx_apply_batched.restype = ctypes.c_int
    L.hfx_apply_sequential.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(HfxApplyArgs), i32, vp]
    L.hfx_apply_sequential.restype = ctypes.c_int
    L.hfx_set_wait_budget.argtypes = [vp, i64]
    L.hfx_set_wait_budget.restype = ctypes.c_int
    L.hfx_sync_status.argtypes = [vp, vp]
    L.hfx_sync_status.restype = ctypes.c_int
    L.hfx_set_tuning.argtypes = [vp, i32, sz, i32]
    L.hfx_set_tuning.restype = ctypes.c_int
    L.hfx_plan_stats.argtypes = [vp, i32, i64, u32, ctypes.POINTER(i64)]
    L.hfx_plan_stats.restype = ctypes.c_int
    L.hfx_profile_enable.argtypes = [vp, ctypes.c_int]
    L.hfx_profile_enable.restype = ctypes.c_int
    L.hfx_profile_read.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64)]
    L.hfx_profile_read.restype = ctypes.c_int
    L.hfx_last_error.argtypes = []
    L.hfx_last_error.restype = ctypes.c_char_p
    L.hfx_destroy.argtypes = [vp]
    L.hfx_destroy.restype = None
    L.hfx_ace_workspace_bytes.argtypes = [vp, i32, i32]
    L.hfx_ace_workspace_bytes.restype = sz
    L.hfx_ace_build.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, sz, vp]
    L.hfx_ace_build.restype = ctypes.c_int
    L.hfx_ace_apply.argtypes = [vp, vp, i32, vp, i32, u32, vp, vp, sz, vp]
    L.hfx_ace_apply.restype = ctypes.c_int
    L.hfx_screen_pairs.argtypes = [vp, vp, i32, dbl, vp, vp, vp, vp, sz, vp]
    L.hfx_screen_pairs.restype = ctypes.c_int
    L.hfx_ace_profile_read.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(i64)]
    L.hfx_ace_profile_read.restype = ctypes.c_int
    L.hfx_scdm_workspace_bytes.argtypes = [vp, i32]
    L.hfx_scdm_workspace_bytes.restype = sz
    L.hfx_scdm_localise.argtypes = [vp, vp, i32, vp, vp, vp, vp, sz, vp]
    L.hfx_scdm_localise.restype = ctypes.c_int
    sp = ctypes.POINTER(HfxSinrParams)
    L.hfx_sinr_update_n.argtypes = [sp, i64, dbl, i32, i32, vp, vp, vp, vp, vp]
    L.hfx_sinr_update_n.restype = ctypes.c_int
    L.hfx_sinr_update_v.argtypes = [sp, i64, dbl, vp, vp, vp, vp, vp, vp]
    L.hfx_sinr_update_v.restype = ctypes.c_int
    L.hfx_sinr_update_x.argtypes = [sp, i64, dbl, vp, vp, vp, vp, vp]
    L.hfx_sinr_update_x.restype = ctypes.c_int
    L.hfx_fma_peak.argtypes = [i32, i32, ctypes.POINTER(dbl), vp]
    L.hfx_fma_peak.restype = ctypes.c_int
    L.hfx_debug_check_guards.argtypes = [vp, vp]
    L.hfx_debug_check_guards.restype = ctypes.c_int
    L.hfx_test_fail_allocation.argtypes = [i64]
    L.hfx_test_fail_allocation.restype = None
    L.hfx_test_live_allocations.argtypes = []
    L.hfx_test_live_allocations.restype = i64
    _lib = L
    return L


def _check(status: int) -> None:
    if status != HFX_OK:
        msg = load_library().hfx_last_error()
        raise HFXError(status, msg.decode() if msg else "")


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


# ---------------------------------------------------------------------------------------
# entry points, same names as the C ABI
# ---------------------------------------------------------------------------------------

def hfx_create(lattice, grid: Sequence[int], ecut: float = 0.0, kernel: str = "coulomb", alpha: float = 0.25,
               precision: str = "fp32") -> ctypes.c_void_p:
    L = load_library()
    box = HfxBox()
    for a in range(3):
        for b in range(3):
            box.lattice[a][b] = float(lattice[a][b])
    g = (ctypes.c_int32 * 3)(*[int(x) for x in grid])
    out = ctypes.c_void_p()
    _check(L.hfx_create(ctypes.byref(box), g, float(ecut), KERNEL[kernel], float(alpha), PRECISION[precision],
                        ctypes.byref(out)))
    return out


def hfx_workspace_bytes(ctx, n_orb: int, n_pairs: int) -> int:
    return int(load_library().hfx_workspace_bytes(ctx, int(n_orb), int(n_pairs)))


def hfx_set_workspace(ctx, buf: torch.Tensor) -> None:
    _check(load_library().hfx_set_workspace(ctx, _ptr(buf), buf.numel() * buf.element_size()))


def hfx_apply(ctx, orbitals: torch.Tensor, pairs: torch.Tensor, ex: torch.Tensor, vxphi: Optional[torch.Tensor],
              flags: int = 0, stream: Optional[torch.cuda.Stream] = None) -> None:
    n_orb = orbitals.shape[0]
    _check(load_library().hfx_apply(ctx, _ptr(orbitals), int(n_orb), _ptr(pairs), int(pairs.shape[0]), int(flags),
                                    _ptr(ex), _ptr(vxphi), _stream_handle(stream)))


def hfx_apply_noalloc(ctx, orbitals: torch.Tensor, pairs: torch.Tensor, ex: torch.Tensor,
                      vxphi: Optional[torch.Tensor], flags: int = 0, stream: Optional[torch.cuda.Stream] = None) -> None:
    """hfx_apply without a workspace, for callers that cannot allocate device memory at call time:
    the library's own static device scratch (HFX_NOALLOC_SCRATCH_BYTES) is used instead."""
    n_orb = orbitals.shape[0]
    _check(load_library().hfx_apply_noalloc(ctx, _ptr(orbitals), int(n_orb), _ptr(pairs), int(pairs.shape[0]),
                                            int(flags), _ptr(ex), _ptr(vxphi), _stream_handle(stream)))


def _batch_args(ctxs, args):
    n = len(ctxs)
    carr = (ctypes.c_void_p * n)(*[c.value for c in ctxs])
    aarr = (HfxApplyArgs * n)()
    for k, (orb, pairs, ex, v, flags) in enumerate(args):
        aarr[k] = HfxApplyArgs(_ptr(orb), int(orb.shape[0]), _ptr(pairs), int(pairs.shape[0]), int(flags), _ptr(ex),
                               _ptr(v))
    return n, carr, aarr


def hfx_apply_batched(ctxs, args, stream: Optional[torch.cuda.Stream] = None) -> None:
    """All problems in one persistent launch.  ctxs: list of contexts; args: list of
    (orbitals, pairs, ex, vxphi, flags)."""
    n, carr, aarr = _batch_args(ctxs, args)
    _check(load_library().hfx_apply_batched(carr, aarr, n, _stream_handle(stream)))


def hfx_apply_sequential(ctxs, args, stream: Optional[torch.cuda.Stream] = None) -> None:
    """The same problems as one hfx_apply each, back to back on the stream."""
    n, carr, aarr = _batch_args(ctxs, args)
    _check(load_library().hfx_apply_sequential(carr, aarr, n, _stream_handle(stream)))


def hfx_set_wait_budget(ctx, cycles: int) -> None:
    _check(load_library().hfx_set_wait_budget(ctx, int(cycles)))


def hfx_sync_status(ctx, stream: Optional[torch.cuda.Stream] = None) -> None:
    _check(load_library().hfx_sync_status(ctx, _stream_handle(stream)))


def hfx_set_tuning(ctx, block: int = 8, batch_bytes: int = 1 << 30, pipeline: bool = True) -> None:
    _check(load_library().hfx_set_tuning(ctx, int(block), int(batch_bytes), 1 if pipeline else 0))


def hfx_plan_stats(ctx, n_orb: int, n_pairs: int, flags: int = 0) -> dict:
    out = (ctypes.c_int64 * 6)()
    _check(load_library().hfx_plan_stats(ctx, int(n_orb), int(n_pairs), int(flags), out))
    return {"launches": int(out[0]), "batches": int(out[1]), "block": int(out[2]), "max_batch_couples": int(out[3]),
            "couples": int(out[4]), "dense_couples": int(out[5])}


def hfx_profile_enable(ctx, on: bool) -> None:
    _check(load_library().hfx_profile_enable(ctx, 1 if on else 0))


def hfx_profile_read(ctx) -> dict:
    ms = (ctypes.c_double * 6)()
    n = (ctypes.c_int64 * 6)()
    _check(load_library().hfx_profile_read(ctx, ms, n))
    return {name: {"ms": float(ms[k]), "launches": int(n[k])} for k, name in enumerate(PASS_NAMES)}


def hfx_scdm_workspace_bytes(ctx, n_orb: int) -> int:
    return int(load_library().hfx_scdm_workspace_bytes(ctx, int(n_orb)))


def hfx_scdm_localise(ctx, orbitals: torch.Tensor, pivots: torch.Tensor, q: Optional[torch.Tensor],
                      phi_loc: torch.Tensor, workspace: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> None:
    _check(load_library().hfx_scdm_localise(ctx, _ptr(orbitals), int(orbitals.shape[0]), _ptr(pivots), _ptr(q),
                                            _ptr(phi_loc), _ptr(workspace), _nbytes(workspace), _stream_handle(stream)))


def _sinr_params(p) -> HfxSinrParams:
    return p if isinstance(p, HfxSinrParams) else HfxSinrParams(float(p["kT"]), float(p["Q1"]), float(p["Q2"]),
                                                                float(p.get("gamma", 0.0)), int(p["L"]))


def hfx_sinr_update_n(params, dt: float, mass: torch.Tensor, V: torch.Tensor, v1: torch.Tensor, v2: torch.Tensor,
                      n_res: int = 1, n_sy: int = 1, stream: Optional[torch.cuda.Stream] = None) -> None:
    _check(load_library().hfx_sinr_update_n(ctypes.byref(_sinr_params(params)), int(V.numel()), float(dt), int(n_res),
                                            int(n_sy), _ptr(mass), _ptr(V), _ptr(v1), _ptr(v2), _stream_handle(stream)))


def hfx_sinr_update_v(params, dt: float, mass: torch.Tensor, force: torch.Tensor, V: torch.Tensor,
                      v1: torch.Tensor, force_extra: Optional[torch.Tensor] = None,
                      stream: Optional[torch.cuda.Stream] = None) -> None:
    _check(load_library().hfx_sinr_update_v(ctypes.byref(_sinr_params(params)), int(V.numel()), float(dt), _ptr(mass),
                                            _ptr(force), _ptr(force_extra), _ptr(V), _ptr(v1),
                                            _stream_handle(stream)))


def hfx_sinr_update_x(params, dt: float, V: torch.Tensor, X: torch.Tensor, v2: torch.Tensor, R: torch.Tensor,
                      stream: Optional[torch.cuda.Stream] = None) -> None:
    _check(load_library().hfx_sinr_update_x(ctypes.byref(_sinr_params(params)), int(V.numel()), float(dt), _ptr(V),
                                            _ptr(X), _ptr(v2), _ptr(R), _stream_handle(stream)))


def hfx_ace_profile_read(ctx) -> dict:
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_int64 * 3)()
    _check(load_library().hfx_ace_profile_read(ctx, ms, n))
    return {name: {"ms": float(ms[k]), "launches": int(n[k])} for k, name in enumerate(ACE_KERNEL_NAMES)}


def hfx_last_error() -> str:
    m = load_library().hfx_last_error()
    return m.decode() if m else ""


def hfx_destroy(ctx) -> None:
    load_library().hfx_destroy(ctx)


def hfx_ace_workspace_bytes(ctx, n_orb: int, n_psi: int = 0) -> int:
    return int(load_library().hfx_ace_workspace_bytes(ctx, int(n_orb), int(n_psi)))


def _nbytes(t: torch.Tensor) -> int:
    return t.numel() * t.element_size()


def hfx_ace_build(ctx, orbitals: torch.Tensor, w: torch.Tensor, m: Optional[torch.Tensor], l: Optional[torch.Tensor],
                  p: torch.Tensor, workspace: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> None:
    _check(load_library().hfx_ace_build(ctx, _ptr(orbitals), _ptr(w), int(orbitals.shape[0]), _ptr(m), _ptr(l), _ptr(p),
                                        _ptr(workspace), _nbytes(workspace), _stream_handle(stream)))


def hfx_ace_apply(ctx, p: torch.Tensor, psi: torch.Tensor, out: torch.Tensor, workspace: torch.Tensor,
                  flags: int = 0, stream: Optional[torch.cuda.Stream] = None) -> None:
    _check(load_library().hfx_ace_apply(ctx, _ptr(p), int(p.shape[0]), _ptr(psi), int(psi.shape[0]), int(flags),
                                        _ptr(out), _ptr(workspace), _nbytes(workspace), _stream_handle(stream)))


def hfx_screen_pairs(ctx, orbitals: torch.Tensor, cut: float, s: Optional[torch.Tensor], pairs: torch.Tensor,
                     n_pairs: torch.Tensor, workspace: torch.Tensor, stream: Optional[torch.cuda.Stream] = None) -> None:
    _check(load_library().hfx_screen_pairs(ctx, _ptr(orbitals), int(orbitals.shape[0]), float(cut), _ptr(s),
                                           _ptr(pairs), _ptr(n_pairs), _ptr(workspace), _nbytes(workspace),
                                           _stream_handle(stream)))


# ---------------------------------------------------------------------------------------
# convenience wrapper: one context + a torch-owned workspace
# ---------------------------------------------------------------------------------------

class Exchange:
    """Exact exchange for one cell and grid on the current CUDA device.

    ``apply(phi, pairs)`` returns (E_x as a 1-element float64 device tensor, V_x phi float64
    [n_orb, n1, n2, n3] or None with energy_only).
    """

    def __init__(self, lattice, grid: Sequence[int], ecut: float = 0.0, alpha: float = 0.25,
                 precision: str = "fp32", kernel: str = "coulomb"):
        self.lattice = [[float(x) for x in row] for row in lattice]
        self.grid = tuple(int(x) for x in grid)
        self.alpha = float(alpha)
        self.precision = precision
        self.ctx = hfx_create(self.lattice, self.grid, ecut, kernel, alpha, precision)
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._ws: Optional[torch.Tensor] = None

    @property
    def volume(self) -> float:
        import numpy as np
        return float(abs(np.linalg.det(np.array(self.lattice))))

    @property
    def npoints(self) -> int:
        return self.grid[0] * self.grid[1] * self.grid[2]

    def ensure_workspace(self, n_orb: int, n_pairs: int) -> None:
        need = hfx_workspace_bytes(self.ctx, n_orb, n_pairs)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
            hfx_set_workspace(self.ctx, self._ws)

    def apply(self, phi: torch.Tensor, pairs: torch.Tensor, energy_only: bool = False, accumulate: bool = False,
              ex: Optional[torch.Tensor] = None, vxphi: Optional[torch.Tensor] = None,
              stream: Optional[torch.cuda.Stream] = None) -> Tuple[torch.Tensor, Optional[torch.Tensor]]:
        if not phi.is_cuda or not pairs.is_cuda:
            raise ValueError("phi and pairs must be CUDA tensors")
        if phi.dtype not in (torch.float64, torch.float32) or not phi.is_contiguous():
            raise ValueError("phi must be a contiguous float64 (or float32) tensor [n_orb, n1, n2, n3]")
        if tuple(phi.shape[1:]) != self.grid:
            raise ValueError(f"phi grid {tuple(phi.shape[1:])} != context grid {self.grid}")
        if pairs.dtype != torch.int32 or pairs.dim() != 2 or pairs.shape[1] != 2 or not pairs.is_contiguous():
            raise ValueError("pairs must be a contiguous int32 tensor [n_pairs, 2]")
        flags = 0
        if energy_only:
            flags |= HFX_ENERGY_ONLY
        if accumulate:
            flags |= HFX_ACCUMULATE
        if phi.dtype == torch.float32:
            flags |= HFX_ORBITALS_F32
        n_orb = phi.shape[0]
        self.ensure_workspace(n_orb, pairs.shape[0])
        if ex is None:
            ex = torch.zeros(1, dtype=torch.float64, device=phi.device)
        if vxphi is None and not energy_only:
            vxphi = torch.empty(phi.shape, dtype=torch.float64, device=phi.device)
        hfx_apply(self.ctx, phi, pairs, ex, None if energy_only else vxphi, flags, stream)
        return ex, (None if energy_only else vxphi)

    def sync_status(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        hfx_sync_status(self.ctx, stream)

    # ---- ACE operator and overlap screen (include/hfx_ace.h)

    def _grid_rows(self, name: str, t: torch.Tensor) -> None:
        if not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous() or tuple(t.shape[1:]) != self.grid:
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor [n, {self.grid[0]}, {self.grid[1]}, "
                             f"{self.grid[2]}]")

    def _ace_workspace(self, n_orb: int, n_psi: int) -> torch.Tensor:
        need = hfx_ace_workspace_bytes(self.ctx, n_orb, n_psi)
        ws = getattr(self, "_ace_ws", None)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device=self.device)
            self._ace_ws = ws
        return ws

    def ace_build(self, phi: torch.Tensor, w: torch.Tensor, stream: Optional[torch.cuda.Stream] = None):
        """(M, L, P) of the ACE operator built from orbitals phi and W = V_x phi (both FP64)."""
        self._grid_rows("phi", phi)
        self._grid_rows("w", w)
        if w.shape != phi.shape:
            raise ValueError("w must have the shape of phi")
        n = phi.shape[0]
        m = torch.empty((n, n), dtype=torch.float64, device=phi.device)
        l = torch.empty((n, n), dtype=torch.float64, device=phi.device)
        p = torch.empty_like(phi)
        hfx_ace_build(self.ctx, phi, w, m, l, p, self._ace_workspace(n, 0), stream)
        return m, l, p

    def ace_apply(self, p: torch.Tensor, psi: torch.Tensor, out: Optional[torch.Tensor] = None,
                  accumulate: bool = False, stream: Optional[torch.cuda.Stream] = None) -> torch.Tensor:
        """V_x^ACE psi for every row of psi (FP64)."""
        self._grid_rows("p", p)
        self._grid_rows("psi", psi)
        if out is None:
            out = torch.zeros_like(psi) if accumulate else torch.empty_like(psi)
        hfx_ace_apply(self.ctx, p, psi, out, self._ace_workspace(p.shape[0], psi.shape[0]),
                      HFX_ACCUMULATE if accumulate else 0, stream)
        return out

    def scdm_localise(self, phi: torch.Tensor, stream: Optional[torch.cuda.Stream] = None):
        """(pivots int64 [n], Q [n, n], Phi = Psi Q [n, n1, n2, n3]) of the SCDM localisation."""
        self._grid_rows("phi", phi)
        n = phi.shape[0]
        need = hfx_scdm_workspace_bytes(self.ctx, n)
        if need == 0:
            raise ValueError(f"SCDM needs 1 <= n_orb <= min(N, 768); got {n}")
        ws = getattr(self, "_scdm_ws", None)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=self.device)
            self._scdm_ws = ws
        piv = torch.empty(n, dtype=torch.int64, device=phi.device)
        q = torch.empty((n, n), dtype=torch.float64, device=phi.device)
        out = torch.empty_like(phi)
        hfx_scdm_localise(self.ctx, phi, piv, q, out, ws, stream)
        return piv, q, out

    def screen_pairs(self, phi: torch.Tensor, cut: float, stream: Optional[torch.cuda.Stream] = None):
        """(pairs int32 [P, 2] device tensor, s [n, n]) of the overlap screen s_ij > cut (diagonal kept).

        Reads the pair count back to size the result, so it synchronises with `stream`."""
        self._grid_rows("phi", phi)
        n = phi.shape[0]
        s = torch.empty((n, n), dtype=torch.float64, device=phi.device)
        pairs = torch.empty((n * (n + 1) // 2, 2), dtype=torch.int32, device=phi.device)
        count = torch.zeros(1, dtype=torch.int64, device=phi.device)
        hfx_screen_pairs(self.ctx, phi, cut, s, pairs, count, self._ace_workspace(n, 0), stream)
        return pairs[: int(count.item())], s

    def set_tuning(self, block: int = 8, batch_bytes: int = 1 << 30, pipeline: bool = True) -> None:
        hfx_set_tuning(self.ctx, block, batch_bytes, pipeline)
        self.tuning = {"block": int(block), "batch_bytes": int(batch_bytes), "pipeline": bool(pipeline)}

    def close(self) -> None:
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            hfx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hfx_fma_peak(fp64: bool, iters: int = 20000, stream: Optional[torch.cuda.Stream] = None) -> float:
    """Measured FMA throughput of the current device in TFLOP/s (FP64 or FP32)."""
    out = ctypes.c_double(0.0)
    _check(load_library().hfx_fma_peak(1 if fp64 else 0, int(iters), ctypes.byref(out), _stream_handle(stream)))
    return float(out.value)


def hfx_debug_check_guards(ctx, stream: Optional[torch.cuda.Stream] = None) -> None:
    """HFX_DEBUG builds: enqueue the check of the workspace guard bands (see hfx_sync_status)."""
    _check(load_library().hfx_debug_check_guards(ctx, _stream_handle(stream)))


def hfx_test_fail_allocation(k: int) -> None:
    """Failure injection (tests): the library's device allocation after the next k fails as out of
    memory; k < 0 cancels."""
    load_library().hfx_test_fail_allocation(int(k))


def hfx_test_live_allocations() -> int:
    """Device allocations the library holds, all contexts."""
    return int(load_library().hfx_test_live_allocations())
