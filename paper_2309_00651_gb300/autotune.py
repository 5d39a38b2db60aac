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
        tmp = f"{path}.{os.getpid()}.tmp"  # per process: concurrent writers never share it
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


BATCH_BUDGETS = (1 << 30, 512 << 20, 256 << 20, 2 << 30)


def tune_batch(exchanges, run_persistent, run_sequential, n_orbs, n_pairs,
               budgets: Iterable[int] = BATCH_BUDGETS, steps: int = 2, timer=None) -> dict:
    """Pick the pair-batch size (per-context transform budget) of the uneven batch's persistent
    launch, then keep the persistent form or the one-call-per-problem form, whichever is faster.

    exchanges: the Exchange of every problem; run_persistent / run_sequential: callables that
    run the whole batch once in that form; n_orbs, n_pairs: per problem (for the workspaces).
    Returns {"setting": {"batch_bytes", "mode"}, "ms": ..., "trials": [...]} with the setting
    applied to every context."""
    timer = timer or _time_batch

    def apply(budget):
        for ex, no, npair in zip(exchanges, n_orbs, n_pairs):
            ex.set_tuning(8, budget, True)
            ex.ensure_workspace(no, npair)

    trials = []
    for b in budgets:
        try:
            apply(b)
            ms = timer(run_persistent, steps)
        except Exception as err:  # a budget whose workspaces do not fit is skipped
            trials.append({"setting": {"batch_bytes": b, "mode": "persistent"}, "error": str(err)})
            continue
        trials.append({"setting": {"batch_bytes": b, "mode": "persistent"}, "ms": ms})
    ok = [t for t in trials if "ms" in t]
    if not ok:
        raise RuntimeError(f"no batch setting ran: {trials}")
    best = min(ok, key=lambda t: t["ms"])
    apply(best["setting"]["batch_bytes"])
    try:
        ms_seq = timer(run_sequential, steps)
        trials.append({"setting": {"batch_bytes": best["setting"]["batch_bytes"], "mode": "sequential"}, "ms": ms_seq})
        if ms_seq < best["ms"]:
            best = trials[-1]
    except Exception as err:
        trials.append({"setting": {"mode": "sequential"}, "error": str(err)})
    return {"setting": best["setting"], "ms": best["ms"], "trials": trials}


def _time_batch(run, steps: int) -> float:
    run()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        run()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps
