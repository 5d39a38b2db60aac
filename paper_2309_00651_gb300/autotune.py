"""Schedule autotuner for the exchange call.

For one (GPU, grid, orbital-count bucket, precision) it times a few settings of the orbital block
size, the per-batch transform budget and the two-stream batch pipelining (`hfx_set_tuning`) on
the caller's actual inputs, keeps the fastest, and remembers it in a JSON cache so later
contexts of the same shape start tuned.  Results never depend on the setting beyond rounding
order.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, Optional

import torch

from .hfx import Exchange

DEFAULT_CANDIDATES = tuple(
    {"block": b, "batch_bytes": mb << 20, "pipeline": p}
    for b in (8, 4) for mb in (1024, 2048, 512, 256) for p in (True, False))


def cache_path() -> str:
    return os.environ.get("HFX_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "hfx_gb300_tuning.json"))


def shape_key(exch: Exchange, n_orb: int) -> str:
    bucket = 1
    while bucket * 2 <= n_orb:
        bucket *= 2
    gpu = torch.cuda.get_device_name(exch.device)
    return f"{gpu}|{'x'.join(map(str, exch.grid))}|norb{bucket}|{exch.precision}"


def _load(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, table: Dict[str, dict]) -> None:
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only loses the memory of the result


def time_call(exch: Exchange, phi: torch.Tensor, pairs: torch.Tensor, steps: int) -> float:
    """Median-free mean milliseconds of `steps` calls after one warm-up call."""
    exch.ensure_workspace(phi.shape[0], pairs.shape[0])
    E = torch.zeros(1, dtype=torch.float64, device=phi.device)
    V = torch.empty(phi.shape, dtype=torch.float64, device=phi.device)
    exch.apply(phi, pairs, ex=E, vxphi=V)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        exch.apply(phi, pairs, ex=E, vxphi=V)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def tune(exch: Exchange, phi: torch.Tensor, pairs: torch.Tensor,
         candidates: Iterable[dict] = DEFAULT_CANDIDATES, steps: int = 3,
         use_cache: bool = True, path: Optional[str] = None) -> dict:
    """Pick and apply the fastest setting; returns {"setting": ..., "ms": ..., "trials": [...]}."""
    path = path or cache_path()
    key = shape_key(exch, phi.shape[0])
    table = _load(path) if use_cache else {}
    if use_cache and key in table:
        best = table[key]
        exch.set_tuning(**best["setting"])
        return dict(best, cached=True)
    trials = []
    for cand in candidates:
        try:
            exch.set_tuning(**cand)
            ms = time_call(exch, phi, pairs, steps)
        except Exception as err:  # a setting that does not fit this grid is skipped
            trials.append({"setting": cand, "error": str(err)})
            continue
        trials.append({"setting": cand, "ms": ms})
    ok = [t for t in trials if "ms" in t]
    if not ok:
        raise RuntimeError(f"no tuning candidate ran: {trials}")
    best = min(ok, key=lambda t: t["ms"])
    exch.set_tuning(**best["setting"])
    result = {"setting": best["setting"], "ms": best["ms"], "trials": trials}
    if use_cache:
        table[key] = {"setting": best["setting"], "ms": best["ms"]}
        _store(path, table)
    return dict(result, cached=False)
