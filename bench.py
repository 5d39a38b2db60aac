"""Benchmark of the Gamma-point exact-exchange path (E_x + V_x phi) on GB300.

One step = one full hfx_apply over the whole pair list of the workload (pair-list staging,
pair products, forward 3D FFTs, Coulomb multiply + energy, inverse 3D FFTs, V_x phi
accumulation, energy reduction).  Metric: orbital pairs per second.

Default workload: the 32-H2O water box: 128 Gaussian-type orbitals (sigma = 1.2 bohr, four
per jittered lattice site), L = 18.6 bohr, 72^3 grid, Ecut = 40 Ha, all 8256 pairs, seeded
synthetic data standing in for the paper's 32-water system.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp32|fp64]
                       [--impl reference] [--no-fp64-compare] [--no-cpu-baseline]
Under torchrun each rank runs an independent replica of the workload on its own GPU (pairs of
independent problems need no exchange); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HF-exchange orbital pairs/s (E_x+V_xφ), mixed vs FP64 GPU path at stated error"
UNIT = "pairs/s"
L2_BYTES = 129 * 1024 * 1024


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="libhfx", choices=["libhfx", "reference"])
    ap.add_argument("--workload", default="water32_n72")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "mixed_tc"])
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-ace", action="store_true", help="skip the ACE / screen rows")
    ap.add_argument("--no-extra", action="store_true", help="skip the 96^3 (256-orbital) sub-measurement")
    ap.add_argument("--with-128", action="store_true",
                    help="also measure the 512-orbital 128^3 screened workload (minutes of input generation)")
    ap.add_argument("--rows-only", action="store_true",
                    help="one exchange call, then the ACE / screen / SCDM / SIN(R) rows with 2 repetitions each; "
                         "prints their JSON (a short run to profile those kernels)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_desc(w, n_pairs):
    return {
        "workload": f"{w.name}: {w.n_orb} orbitals, cubic L={w.L} bohr, {w.n}^3 grid, Ecut={w.ecut} Ha, "
                    f"{'Gaussian sigma=' + str(w.sigma) if w.kind == 'gauss' else 'random PW'} orbitals, "
                    f"Loewdin, {n_pairs} pairs, seed {w.seed}",
        "n_orb": w.n_orb, "grid": [w.n, w.n, w.n], "L_bohr": w.L, "n_pairs": int(n_pairs), "alpha": 0.25,
    }


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peak_tf32():
    """Dense TF32 tensor rate: the measured BF16 burst rate x the nominal TF32/BF16 ratio (1.1/2.25)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 burst x nominal tf32/bf16 ratio"
    except Exception:
        return 1900.0 * 1.1 / 2.25, "fallback bf16 x nominal tf32/bf16 ratio"


def measured_peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------------------------------------
# reference arm and CPU baseline: the FP64 oracle on a bounded sample of the same workload
# ------------------------------------------------------------------------------------------------

def oracle_rate(phi, pairs, lattice, n_sample, seed=0):
    """Time the oracle (as it stands) on a seeded sample of pairs; returns (pairs/s, seconds, E, V)."""
    from oracle import hfx_oracle as O
    from paper_2309_00651_gb300 import inputs as I
    sub = I.random_pairs_subset(pairs, n_sample, seed)
    t0 = time.perf_counter()
    E, V = O.exchange(phi, sub, lattice, alpha=0.25)
    dt = time.perf_counter() - t0
    return len(sub) / dt, dt, sub, E, V


def _oracle_chunk(task):
    """Worker of the all-cores oracle leg: the oracle, as it stands, over one chunk of the pair
    sample, on orbitals shared through a named shared-memory block."""
    from multiprocessing import shared_memory

    import numpy as np
    from oracle import hfx_oracle as O
    name, shape, lattice, chunk = task
    shm = shared_memory.SharedMemory(name=name)
    try:
        phi = np.ndarray(shape, dtype=np.float64, buffer=shm.buf)
        t0 = time.perf_counter()
        E, V = O.exchange(phi, chunk, lattice, alpha=0.25)
        dt = time.perf_counter() - t0
        return E, dt
    finally:
        shm.close()


class OraclePool:
    """The oracle on every host core: one spawned process per core (started with spawn, so it is
    safe after CUDA initialisation), the orbitals shared read-only through shared memory, each
    process evaluating its own slice of a pair sample."""

    def __init__(self, phi, lattice, procs=None):
        import multiprocessing as mp
        from multiprocessing import shared_memory

        import numpy as np
        self.procs = procs or len(os.sched_getaffinity(0))
        self.shm = shared_memory.SharedMemory(create=True, size=phi.nbytes)
        buf = np.ndarray(phi.shape, dtype=np.float64, buffer=self.shm.buf)
        buf[...] = phi
        self.shape = phi.shape
        self.lattice = np.asarray(lattice, dtype=np.float64)
        self.pool = mp.get_context("spawn").Pool(self.procs)
        # first use in every process (imports, FFT plans) outside any timed region
        self.pool.map(_oracle_chunk, [(self.shm.name, self.shape, self.lattice, np.zeros((1, 2), np.int32))] * self.procs)

    def rate(self, pairs, n_sample, seed):
        """pairs/s of the whole pool over a seeded sample (wall clock), and its E_x."""
        import numpy as np
        from paper_2309_00651_gb300 import inputs as I
        sub = I.random_pairs_subset(pairs, n_sample, seed)
        chunks = [c for c in np.array_split(sub, self.procs) if len(c)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_chunk, [(self.shm.name, self.shape, self.lattice, c) for c in chunks], chunksize=1)
        dt = time.perf_counter() - t0
        return len(sub) / dt, dt, sum(r[0] for r in res)

    def close(self):
        self.pool.close()
        self.pool.join()
        self.shm.close()
        self.shm.unlink()


FP32_FFMA_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12  # SMs x FP32 lanes x 2 flop x max SM clock
FP64_PEAK_TFLOPS = 1.25                                  # nominal FP64 rate of this part
# FMA throughput measured on this device by hfx_fma_peak (filled in before the measurements; the
# figures above are the fallbacks)
MEASURED_ALU = {}


def alu_peak(fp64: bool):
    key = "fp64_tflops" if fp64 else "fp32_tflops"
    if key in MEASURED_ALU:
        return MEASURED_ALU[key], "measured (hfx_fma_peak)"
    return (FP64_PEAK_TFLOPS, "nominal FP64 rate") if fp64 else (FP32_FFMA_PEAK_TFLOPS, "derived FP32 rate")


def ace_rows(ex, phi, V, E, w, precision, hfx, reps=10):
    """ACE construction / application (Sec. 2.1, Eq. vx_ace) and the overlap screen on this
    workload, W = V_x phi from the exchange call: call times, per-kernel roofline of the split
    grid contraction and of the left multiply, identities that hold at any size.  Returns the
    row and (M, P) for the oracle comparison of the CPU-baseline leg."""
    import torch
    n_orb, N = phi.shape[0], phi[0].numel()
    M, Lf, Pm = ex.ace_build(phi, V)
    Y = ex.ace_apply(Pm, phi)
    ex.sync_status()
    out = torch.empty_like(phi)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    t_build = timed(lambda: ex.ace_build(phi, V))
    t_apply = timed(lambda: ex.ace_apply(Pm, phi, out=out))
    t_screen = timed(lambda: ex.screen_pairs(phi, 1e-6))
    t_scdm = timed(lambda: ex.scdm_localise(phi))
    # per-kernel device time over `reps` applications (CUDA events around each launch)
    hfx.hfx_profile_enable(ex.ctx, True)
    hfx.hfx_ace_profile_read(ex.ctx)
    for _ in range(reps):
        ex.ace_apply(Pm, phi, out=out)
    torch.cuda.synchronize()
    hfx.hfx_profile_enable(ex.ctx, False)
    kp = hfx.hfx_ace_profile_read(ex.ctx)
    g_ms = kp["ace_gram"]["ms"] / max(1, kp["ace_gram"]["launches"])
    l_ms = kp["ace_lmul"]["ms"] / max(1, kp["ace_lmul"]["launches"])
    flops = 2.0 * n_orb * n_orb * N            # one contraction over the grid, n_psi = n_orb
    gram_bytes = 2.0 * n_orb * N * 8           # both FP64 operands read once
    lmul_bytes = 2.0 * n_orb * N * 8           # Y read once, C written once
    peak_tf, peak_tf_kind = alu_peak(precision == "fp64")
    hbm = measured_peak_hbm()[0]

    tf32_peak, tf32_kind = measured_peak_tf32()

    def roof(ms, nbytes, kernel):
        tf = flops / (ms / 1e3) / 1e12
        gbs = nbytes / (ms / 1e3) / 1e9
        if precision != "fp64":
            # tcgen05 TF32 x 3: three tensor-core products per FP32 product; the FP64 operands
            # stream from HBM once, which is the bound
            return {"bound": "hbm", "kernel": kernel, "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
                    "avg_launch_ms": ms, "alg_bytes_per_launch": nbytes, "alg_flops_per_launch": flops,
                    "tensor_tflops": 3 * tf, "tensor_peak_tflops": tf32_peak, "tensor_frac": 3 * tf / tf32_peak,
                    "tensor_peak_kind": tf32_kind, "peak_kind": "measured"}
        return {"bound": "alu", "kernel": kernel, "achieved": tf, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": tf / peak_tf, "avg_launch_ms": ms, "alg_flops_per_launch": flops,
                "alg_bytes_per_launch": nbytes, "hbm_frac": gbs / hbm, "peak_kind": peak_tf_kind}

    # SCDM: n - 1 residual updates, each a pass over the orbital copy in the compute type plus the
    # FP64 residual norms (read + write); the picks between them are latency-bound single blocks
    esize = 4 if precision != "fp64" else 8
    scdm_bytes = (n_orb - 1) * (n_orb * N * esize + 16 * N)
    scdm_gbs = scdm_bytes / (t_scdm / 1e3) / 1e9
    row = {
        "ms": {"build": t_build, "apply": t_apply, "screen": t_screen, "scdm": t_scdm},
        "scdm_roofline": {"bound": "hbm", "achieved": scdm_gbs, "peak": hbm, "unit": "GB/s", "frac": scdm_gbs / hbm,
                          "alg_bytes_per_call": scdm_bytes,
                          "measured": "whole call (picks included) with CUDA events"},
        "apply_vs_exchange_call": None,
        "roofline": roof(g_ms, gram_bytes, ("k_gram_tc (tcgen05 TF32x3" if precision != "fp64" else "k_ace_mm (FP64") +
                         ", split grid contraction <psi|P>)"),
        "roofline_lmul": roof(l_ms, lmul_bytes, ("k_lmul_tc (tcgen05 TF32x3" if precision != "fp64" else "k_ace_mm (FP64") +
                              ", left multiply -X P)"),
        "kernel_ms_per_apply": {k: v["ms"] / reps for k, v in kp.items()},
        "checks": {"span_rel_err": float(torch.linalg.norm(Y - V) / torch.linalg.norm(V)),
                   "half_trace_M_vs_E_rel": abs(0.5 * float(torch.trace(M)) - E) / abs(E)},
        "n_orb": n_orb, "n_psi": n_orb, "precision": precision,
    }
    return row, (M, Pm)


def sinr_rows(hfx, n_dof=3 * 1048576, L=4, reps=20):
    """SIN(R) integrator updates (appendix A, B, C) on a synthetic 1M-atom state: time per update
    and the bytes each moves per degree of freedom against measured HBM (A and B carry a few dozen
    FP64 transcendental operations per degree of freedom, which the narrow FP64 pipe of this part
    bounds)."""
    import torch
    g = torch.Generator(device="cuda").manual_seed(0)
    kT = 0.0019
    p = {"kT": kT, "Q1": kT * 1600.0, "Q2": kT * 1600.0, "gamma": 0.01, "L": L}
    M = torch.rand(n_dof, device="cuda", dtype=torch.float64, generator=g) * 29000.0 + 1000.0
    V = torch.randn(n_dof, device="cuda", dtype=torch.float64, generator=g) * 1e-3
    v1 = torch.randn(n_dof, L, device="cuda", dtype=torch.float64, generator=g) * (kT / p["Q1"]) ** 0.5
    lam = M * V * V + (L / (L + 1.0)) * p["Q1"] * torch.sum(v1 * v1, dim=1)
    f = torch.sqrt(L * kT / lam)
    V *= f
    v1 *= f[:, None]
    v2 = torch.randn(n_dof, L, device="cuda", dtype=torch.float64, generator=g) * (kT / p["Q2"]) ** 0.5
    X = torch.randn(n_dof, device="cuda", dtype=torch.float64, generator=g)
    F = torch.randn(n_dof, device="cuda", dtype=torch.float64, generator=g) * 0.01
    R = torch.randn(n_dof, L, device="cuda", dtype=torch.float64, generator=g)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    t_a = timed(lambda: hfx.hfx_sinr_update_n(p, 20.0, M, V, v1, v2, 1, 3))
    t_b = timed(lambda: hfx.hfx_sinr_update_v(p, 20.0, M, F, V, v1))
    t_c = timed(lambda: hfx.hfx_sinr_update_x(p, 20.0, V, X, v2, R))
    hbm = measured_peak_hbm()[0]
    per_dof = {"A": 8 * (2 + 2 * L) + 8 * (1 + 2 * L), "B": 8 * (3 + L) + 8 * (1 + L),
               "C": 8 * (2 + 2 * L) + 8 * (1 + L)}
    ms = {"A": t_a, "B": t_b, "C": t_c}
    lam2 = M * V * V + (L / (L + 1.0)) * p["Q1"] * torch.sum(v1 * v1, dim=1)
    return {"n_dof": n_dof, "L": L, "n_sy": 3, "ms": ms,
            "hbm_frac": {k: per_dof[k] * n_dof / (ms[k] / 1e3) / 1e9 / hbm for k in ms},
            "bytes_per_dof": per_dof,
            "constraint_max_rel_dev": float(torch.max(torch.abs(lam2 / (L * kT) - 1.0)))}


def run_reference(args):
    """The oracle as it stands on every host core (one process per core), on bounded samples of
    the same workload; the GPU path's metric, unit and config."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2309_00651_gb300 import inputs as I
    w = I.WORKLOADS[args.workload]
    phi, pairs, info = I.make_workload(w)
    pool = OraclePool(phi, w.lattice)
    try:
        # calibrate the per-pair cost, then size each step so the whole run stays within ~3 minutes
        rate, _, _ = pool.rate(pairs, 2 * pool.procs, seed=123)
        per_step = max(pool.procs, int(150.0 / max(1, args.steps + args.warmup) * rate))
        per_step = min(per_step, len(pairs))
        for k in range(args.warmup):
            pool.rate(pairs, per_step, seed=1000 + k)
        total_pairs, total_t = 0, 0.0
        for k in range(args.steps):
            r, dt, _ = pool.rate(pairs, per_step, seed=k)
            total_pairs += per_step
            total_t += dt
    finally:
        pool.close()
    value = total_pairs / total_t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_desc(w, len(pairs)),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                         "sample": f"{per_step} seeded random pairs of the {len(pairs)}-pair list per step, split "
                                   f"over {pool.procs} processes (numpy FP64, one per host core)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


PASS_KEYS = ("fwd_yz", "x_coulomb", "y_acc_dense", "y_acc_generic")


def measured_traffic(n, precision):
    """DRAM bytes per couple of each pass from profiles/traffic.json (ncu counters of the bench
    workload's own launches), for the grid edge and precision they were taken on and only while the
    kernel sources are the ones they were taken on; {} otherwise."""
    from paper_2309_00651_gb300 import build as B
    prof_file = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(prof_file) as f:
            tj = json.load(f)
    except (OSError, ValueError):
        return {}
    if tj.get("kernel_hash") != B.kernel_hash():
        return {}
    return {k: e["dram_bytes_per_couple"] for k, e in tj.get("kernels", {}).items()
            if e.get("grid") == n and e.get("precision") == precision}


def pass_rooflines(prof, steps, stats, N, csize, P, ms_step, peak, traffic=None):
    """Per pass: algorithmic bytes per step (per couple: forward pass writes the packed transform,
    8 N B in FP32; the x pass reads and writes it; the accumulate passes read it), device time per
    step from the library's per-launch CUDA events, and the fraction of the measured HBM peak;
    plus the whole call at 16 N B per pair (FP32; 32 N B in FP64).  Where `traffic` holds a pass's
    measured DRAM bytes per couple, the pass also gets the DRAM bytes it moves per step and the
    fraction of the HBM peak those bytes run at (`dram_frac`): how close the pass is to the DRAM
    roofline in the bytes it really moves, compulsory re-reads included."""
    per_couple = {"fwd_yz": csize * N, "x_coulomb": 2 * csize * N, "y_acc_dense": csize * N,
                  "y_acc_generic": csize * N}
    couples_of = {"fwd_yz": stats["couples"], "x_coulomb": stats["couples"],
                  "y_acc_dense": stats["dense_couples"], "y_acc_generic": stats["couples"] - stats["dense_couples"]}
    out = {}
    for k in PASS_KEYS:
        ms = prof[k]["ms"] / steps
        if ms <= 0:
            continue
        b = per_couple[k] * couples_of[k]
        out[k] = {"ms_per_step": ms, "alg_bytes_per_step": b, "achieved_gbs": b / (ms / 1e3) / 1e9,
                  "frac": b / (ms / 1e3) / 1e9 / peak}
        if traffic and k in traffic:
            d = traffic[k] * couples_of[k]
            out[k]["dram_bytes_per_step"] = d
            out[k]["dram_frac"] = d / (ms / 1e3) / 1e9 / peak
    whole = 2 * csize * N * P
    out["whole_call"] = {"ms_per_step": ms_step, "alg_bytes_per_step": whole,
                         "achieved_gbs": whole / (ms_step / 1e3) / 1e9, "frac": whole / (ms_step / 1e3) / 1e9 / peak}
    return out


def graph_steps(step, stream, steps, barrier):
    """Capture one step in a CUDA graph and time `steps` replays: CUDA events around the whole
    region (the contract's timing) and around each replay (for the median)."""
    import torch
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):  # captured on torch's own side stream, replayed on `stream`
        step()
    g.replay()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    barrier()
    evs[0].record(stream)
    for k in range(steps):
        g.replay()
        evs[k + 1].record(stream)
    barrier()
    per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
    return evs[0].elapsed_time(evs[-1]), per, g


def measure_workload(name, precision, hfx, I, O, dev, reps=3, n_check=12):
    """A further workload of the scope table at full size: ms per call (median of `reps` replays
    of a captured call), pairs/s, per-pass rooflines, and E_x over a seeded pair sample against
    the oracle (the sample run as the GPU's own pair list)."""
    import numpy as np
    import torch
    w = I.WORKLOADS[name]
    t0 = time.time()
    phi_np, pairs_np, info = I.make_workload(w)
    gen_s = time.time() - t0
    P, N = len(pairs_np), w.n ** 3
    phi = torch.from_numpy(phi_np).to(dev)
    pairs = torch.from_numpy(pairs_np).to(dev)
    ex = hfx.Exchange(w.lattice, w.grid, alpha=0.25, precision=precision)
    ex.ensure_workspace(w.n_orb, P)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    V = torch.empty_like(phi)
    stream = torch.cuda.current_stream()

    def step():
        ex.apply(phi, pairs, ex=E, vxphi=V)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    ex.sync_status()
    total, per, g = graph_steps(step, stream, reps, torch.cuda.synchronize)
    del g
    med = statistics.median(per)
    stats = hfx.hfx_plan_stats(ex.ctx, w.n_orb, P, 0)
    ex.set_tuning(8, 1 << 30, False)
    ex.ensure_workspace(w.n_orb, P)
    step()
    hfx.hfx_profile_enable(ex.ctx, True)
    hfx.hfx_profile_read(ex.ctx)
    step()
    torch.cuda.synchronize()
    hfx.hfx_profile_enable(ex.ctx, False)
    prof = hfx.hfx_profile_read(ex.ctx)
    csize = 16 if precision == "fp64" else 8
    peak = measured_peak_hbm()[0]
    E_val = float(E.item())
    hom = 0.5 * (w.volume / N) * float(torch.sum(phi * V).item())
    sub = I.random_pairs_subset(pairs_np, n_check, seed=5)
    Es, _ = ex.apply(phi, torch.from_numpy(sub).to(dev), energy_only=True)
    E_ref, _ = O.exchange(phi_np, sub, w.lattice, want_v=False)
    ex.close()
    del phi, V, pairs
    torch.cuda.empty_cache()
    return {"config": workload_desc(w, P), "precision": precision, "value": P / (med / 1e3), "unit": UNIT,
            "ms_per_call_median": med, "ms_per_call_mean": total / reps, "replays": reps,
            "roofline_passes": pass_rooflines(prof, 1, stats, N, csize, P, med, peak),
            "checks": {"E_x": E_val, "homogeneity_rel_err": abs(hom - E_val) / abs(E_val),
                       "E_rel_err_vs_oracle_on_sample": abs(Es.item() - E_ref) / abs(E_ref),
                       "sample": f"{len(sub)} seeded pairs as the GPU's own list"},
            "input_generation_s": gen_s}


def measure_batch(hfx, I, dev, precision, reps=3):
    """The uneven batch (24 independent water-density boxes, 32..256 orbitals, 48^3..96^3 grids,
    all pairs of every box): one hfx_apply_batched call (staging per problem, then every pass of
    every problem in one persistent launch), captured in a CUDA graph and replayed, against the
    same problems as back-to-back hfx_apply calls (hfx_apply_sequential), also replayed."""
    import torch
    ws = I.batched_workloads()
    t0 = time.time()
    data = I.make_workloads_parallel(ws)
    gen_s = time.time() - t0
    exs, phis, pairss, Es, Vs = [], [], [], [], []
    for w, (phi_np, pairs_np, _) in zip(ws, data):
        ex = hfx.Exchange(w.lattice, w.grid, alpha=0.25, precision=precision)
        ex.ensure_workspace(w.n_orb, len(pairs_np))
        exs.append(ex)
        phis.append(torch.from_numpy(phi_np).to(dev))
        pairss.append(torch.from_numpy(pairs_np).to(dev))
        Es.append(torch.zeros(1, dtype=torch.float64, device=dev))
        Vs.append(torch.empty(phi_np.shape, dtype=torch.float64, device=dev))
    del data
    P = sum(int(p.shape[0]) for p in pairss)
    ctxs = [e.ctx for e in exs]
    args = [(p, q, E, V, 0) for p, q, E, V in zip(phis, pairss, Es, Vs)]
    stream = torch.cuda.current_stream()
    out = {"config": {"workload": f"uneven batch: {len(ws)} independent water-density boxes (30 A^3 per H2O), "
                                  f"{min(w.n_orb for w in ws)}..{max(w.n_orb for w in ws)} random-PW orbitals, "
                                  f"{min(w.n for w in ws)}^3..{max(w.n for w in ws)}^3 grids, Ecut=20 Ha, all pairs, "
                                  f"sub-seeds of SeedSequence(0)", "problems": len(ws), "n_pairs": P},
           "input_generation_s": gen_s}
    # the autotuner picks the pair-batch size of the persistent launch and the faster form
    from paper_2309_00651_gb300 import autotune
    tuned = autotune.tune_batch(exs, lambda: hfx.hfx_apply_batched(ctxs, args),
                                lambda: hfx.hfx_apply_sequential(ctxs, args),
                                [w.n_orb for w in ws], [int(q.shape[0]) for q in pairss])
    out["tuning"] = {"setting": tuned["setting"],
                     "trials": [{**t["setting"], "ms": round(t.get("ms", -1), 2)} for t in tuned["trials"]]}
    res = {}
    for name, fn in (("persistent", hfx.hfx_apply_batched), ("sequential", hfx.hfx_apply_sequential)):
        fn(ctxs, args)
        fn(ctxs, args)
        torch.cuda.synchronize()
        total, per, g = graph_steps(lambda: fn(ctxs, args), stream, reps, torch.cuda.synchronize)
        del g
        med = statistics.median(per)
        res[name] = {"ms_per_call_median": med, "value": P / (med / 1e3), "unit": UNIT,
                     "E": [float(E.item()) for E in Es], "V_norm": [float(torch.linalg.norm(V)) for V in Vs]}
        for e in exs:
            e.sync_status()
    hom = []
    for w, phi, V, E in zip(ws, phis, Vs, Es):
        N = w.n ** 3
        hom.append(abs(0.5 * (w.volume / N) * float(torch.sum(phi * V).item()) - E.item()) / abs(E.item()))
    pe, se = res["persistent"]["E"], res["sequential"]["E"]
    out["persistent"] = {k: v for k, v in res["persistent"].items() if k not in ("E", "V_norm")}
    out["sequential"] = {k: v for k, v in res["sequential"].items() if k not in ("E", "V_norm")}
    out["persistent"]["launches"] = "per problem: V clear, couple reset, pair placement, FP32 copy; then one persistent launch"
    out["persistent_over_sequential"] = out["persistent"]["value"] / out["sequential"]["value"]
    out["value"] = out[tuned["setting"]["mode"]]["value"]
    out["unit"] = UNIT
    out["checks"] = {"max_E_rel_diff_persistent_vs_sequential": max(abs(a - b) / abs(b) for a, b in zip(pe, se)),
                     "max_homogeneity_rel_err": max(hom)}
    for e in exs:
        e.close()
    del phis, Vs, pairss
    torch.cuda.empty_cache()
    return out


# ------------------------------------------------------------------------------------------------
# the CUDA arm
# ------------------------------------------------------------------------------------------------

def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    rank, world, local = dist_env()
    import numpy as np
    import torch

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2309_00651_gb300 import build as B
    B.build()
    from paper_2309_00651_gb300 import hfx
    from paper_2309_00651_gb300 import inputs as I

    try:
        MEASURED_ALU["fp64_tflops"] = hfx.hfx_fma_peak(True)
        MEASURED_ALU["fp32_tflops"] = hfx.hfx_fma_peak(False)
    except Exception:
        MEASURED_ALU.clear()
    w = I.WORKLOADS[args.workload]
    phi_np, pairs_np, info = I.make_workload(w)
    n_orb, N = w.n_orb, w.n ** 3
    P = len(pairs_np)
    phi = torch.from_numpy(phi_np).to(dev)
    pairs = torch.from_numpy(pairs_np).to(dev)
    if args.rows_only:
        ex = hfx.Exchange(w.lattice, w.grid, alpha=0.25, precision=args.precision)
        E, V = ex.apply(phi, pairs)
        ex.sync_status()
        rows, _ = ace_rows(ex, phi, V, float(E.item()), w, args.precision, hfx, reps=2)
        if rank == 0:
            print(json.dumps({"workload": args.workload, "ace": rows, "sinr": sinr_rows(hfx, reps=2)}), flush=True)
        ex.close()
        return

    ex = hfx.Exchange(w.lattice, w.grid, alpha=0.25, precision=args.precision)
    # schedule autotuner (block size, transform batch, two-stream pipelining), on these inputs
    from paper_2309_00651_gb300 import autotune
    tuned = autotune.tune(ex, phi, pairs, use_cache=False) if not args.no_autotune else {
        "setting": {"block": 8, "batch_bytes": 1 << 30, "pipeline": True}}
    setting = tuned["setting"]
    ex.set_tuning(**setting)
    ex.ensure_workspace(n_orb, P)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    V = torch.empty(phi.shape, dtype=torch.float64, device=dev)
    stats = hfx.hfx_plan_stats(ex.ctx, n_orb, P, 0)
    stream = torch.cuda.current_stream()

    def step():
        ex.apply(phi, pairs, ex=E, vxphi=V)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ex.sync_status()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    # timed region: K full steps, each one replay of a captured call (the schedule and tables
    # were uploaded by the warm-up calls); CUDA events around the region and around each replay
    with ClockSampler(dev.index) as clk:
        ms_total, per_step_ms, graph = graph_steps(step, stream, args.steps, barrier)
    del graph
    median_ms = statistics.median(per_step_ms)

    # per-kernel durations for the roofline: a second timed region of K steps with the batches on
    # one stream (pipelined batches share the GPU, which would stretch every kernel's duration);
    # the library records CUDA events around each pass on the stream it launches it on
    ex.set_tuning(setting["block"], setting["batch_bytes"], False)
    ex.ensure_workspace(n_orb, P)
    step()
    hfx.hfx_profile_enable(ex.ctx, True)
    hfx.hfx_profile_read(ex.ctx)
    barrier()
    for _ in range(args.steps):
        step()
    barrier()
    hfx.hfx_profile_enable(ex.ctx, False)
    prof = hfx.hfx_profile_read(ex.ctx)
    ex.set_tuning(**setting)
    ex.ensure_workspace(n_orb, P)
    if world > 1:
        t = torch.tensor([ms_total], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms_total = float(t.item())
    ms_step = ms_total / args.steps
    value = world * P * args.steps / (ms_total / 1000.0)

    # roofline of the dominant kernel (largest device time), algorithmic bytes per couple:
    #   fwd_yz writes the packed transform (8 N B per couple, FP32 complex);
    #   x_coulomb reads and writes it (16 N B); the accumulate passes read it (8 N B).
    csize = 16 if args.precision == "fp64" else 8
    per_couple = {"fwd_yz": csize * N, "x_coulomb": 2 * csize * N, "y_acc_dense": csize * N,
                  "y_acc_generic": csize * N}
    # couples handled by each kernel per call (full pair list: every block pair full)
    couples_of = {"fwd_yz": stats["couples"], "x_coulomb": stats["couples"],
                  "y_acc_dense": stats["dense_couples"], "y_acc_generic": stats["couples"] - stats["dense_couples"]}
    dom = max(per_couple, key=lambda k: prof[k]["ms"])
    launches = max(1, prof[dom]["launches"])
    avg_ms = prof[dom]["ms"] / launches
    couples_per_launch = couples_of[dom] * args.steps / launches
    alg_bytes = per_couple[dom] * couples_per_launch
    achieved = alg_bytes / (avg_ms / 1000.0) / 1e9
    peak, peak_kind = measured_peak_hbm()
    # measured DRAM bytes per couple of this kernel (ncu, small case of the same grid; the traffic
    # grows in proportion to the couples of a launch), valid only for the sources it was taken on
    traffic = None
    prof_file = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof_file):
        try:
            with open(prof_file) as f:
                tj = json.load(f)
            ent = tj.get("kernels", {}).get(dom, {})
            if tj.get("kernel_hash") == B.kernel_hash() and ent.get("grid") == w.n and \
                    ent.get("precision") == args.precision:
                traffic = ent["dram_bytes_per_couple"] * couples_per_launch
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom, "peak_kind": peak_kind,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_ms,
                "measured": "CUDA events around each launch, batches on one stream, K steps",
                "pass_ms_per_step": {k: prof[k]["ms"] / args.steps for k in prof},
                "passes": pass_rooflines(prof, args.steps, stats, N, csize, P, ms_step, peak,
                                         measured_traffic(w.n, args.precision))}

    # end to end through the public API with host buffers: every step copies its orbitals and pair
    # list in from pinned host memory and its E_x and V_x phi back out.  Steps are pipelined the way
    # a caller feeding successive MD configurations would run them: step k+1's inputs travel in on
    # one copy stream and step k-1's result travels out on another while step k computes (two
    # device buffer sets; events order every reuse).
    phi_h = torch.from_numpy(phi_np).pin_memory()
    pairs_h = torch.from_numpy(pairs_np).pin_memory()
    V_h = [torch.empty(phi.shape, dtype=torch.float64).pin_memory() for _ in range(2)]
    E_h = [torch.empty(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    phi_dev = [torch.empty_like(phi) for _ in range(2)]
    pairs_dev = [torch.empty_like(pairs) for _ in range(2)]
    V_dev = [V, torch.empty_like(V)]
    E_dev = [E, torch.zeros_like(E)]
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def e2e_run(K, serial):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        s_in.wait_event(t0)
        for k in range(K):
            b = 0 if serial else (k & 1)
            with torch.cuda.stream(s_in):
                if serial or k >= 2:
                    s_in.wait_event(ev_out[b] if serial else ev_done[b])
                phi_dev[b].copy_(phi_h, non_blocking=True)
                pairs_dev[b].copy_(pairs_h, non_blocking=True)
                ev_in[b].record(s_in)
            stream.wait_event(ev_in[b])
            if k >= 2 or (serial and k >= 1):
                stream.wait_event(ev_out[b])
            ex.apply(phi_dev[b], pairs_dev[b], ex=E_dev[b], vxphi=V_dev[b], stream=stream)
            ev_done[b].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[b])
                V_h[b].copy_(V_dev[b], non_blocking=True)
                E_h[b].copy_(E_dev[b], non_blocking=True)
                ev_out[b].record(s_out)
        t1.record(s_out)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / K

    e2e_run(2, False)
    barrier()
    e2e_ms = e2e_run(args.e2e_steps, False)
    e2e_serial_ms = e2e_run(args.e2e_steps, True)
    barrier()
    e2e = {"value": world * P / (e2e_ms / 1000.0), "unit": UNIT,
           "h2d_bytes_per_step": phi_h.numel() * 8 + pairs_h.numel() * 4,
           "d2h_bytes_per_step": V_h[0].numel() * 8 + 8, "ms_per_step": e2e_ms,
           "pipelined": "inputs of step k+1 in and result of step k-1 out while step k computes",
           "serial_ms_per_step": e2e_serial_ms}
    if world > 1:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e["value"] = world * P / (float(t.item()) / 1000.0)

    # homogeneity check of this result: E_x = 1/2 (Omega/N) sum_i <phi_i, V_i>
    E_val = float(E.item())
    hom = 0.5 * (w.volume / N) * float(torch.sum(phi * V).item())
    checks = {"E_x": E_val, "homogeneity_rel_err": abs(hom - E_val) / abs(E_val)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "median_ms_per_step": median_ms,
        "value_at_median": world * P / (median_ms / 1000.0),
        "timing": "each step is one replay of a CUDA graph of the full call; value = K steps / CUDA-event time "
                  "of the K-step region (max over ranks); median over the K per-replay event times beside it",
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
        "data": "synthetic (seeded water-box-shaped orbitals; no dataset)",
        "config": dict(workload_desc(w, P), precision=args.precision,
                       l2="inputs larger than L2 (FP64 orbitals %.0f MB + transform batches %.0f MB per step)" % (
                           phi_np.nbytes / 1e6, stats["max_batch_couples"] * N * csize / 1e6),
                       parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                       block=stats["block"], batches=stats["batches"],
                       tuning=dict(setting, autotuned=not args.no_autotune,
                                   trials=[{**t["setting"], "ms": round(t.get("ms", -1), 3)}
                                           for t in tuned.get("trials", [])])),
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": stats["launches"] * args.steps,
        "clocks": clk.summary(),
        "checks": checks,
        "measured_alu_peaks": dict(MEASURED_ALU, how="hfx_fma_peak: 8 independent FMA chains per thread, every SM full, "
                                                      "CUDA events"),
    }

    ace_out = None
    if rank == 0 and not args.no_ace:
        line["ace"], ace_out = ace_rows(ex, phi, V, E_val, w, args.precision, hfx)
        line["ace"]["apply_vs_exchange_call"] = ms_step / line["ace"]["ms"]["apply"]
        line["sinr"] = sinr_rows(hfx)

    if rank == 0 and args.precision == "fp32" and not args.no_fp64_compare:
        ex64 = hfx.Exchange(w.lattice, w.grid, alpha=0.25, precision="fp64")
        ex64.ensure_workspace(n_orb, P)
        E64 = torch.zeros(1, dtype=torch.float64, device=dev)
        V64 = torch.empty_like(V)
        ex64.apply(phi, pairs, ex=E64, vxphi=V64)
        torch.cuda.synchronize()
        k64 = 10
        s3, t3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s3.record(stream)
        for _ in range(k64):
            ex64.apply(phi, pairs, ex=E64, vxphi=V64)
        t3.record(stream)
        torch.cuda.synchronize()
        ms64 = s3.elapsed_time(t3) / k64
        flops_pair = 5.0 * N * math.log2(N) + 20.0 * N  # one packed transform pair per 2 pairs, pointwise work
        pk64, pk64_kind = alu_peak(True)
        line["fp64_gpu_path"] = {
            "value": P / (ms64 / 1000.0), "unit": UNIT, "ms_per_step": ms64, "steps": k64,
            "roofline": {"bound": "alu", "achieved": flops_pair * P / (ms64 / 1e3) / 1e12, "peak": pk64,
                         "unit": "TFLOP/s", "frac": flops_pair * P / (ms64 / 1e3) / 1e12 / pk64, "peak_kind": pk64_kind,
                         "alg_flops_per_call": flops_pair * P},
            "mixed_speedup": (P / (ms_step / 1000.0)) / (P / (ms64 / 1000.0)),
            "E_rel_diff_fp32_vs_fp64": abs(E_val - E64.item()) / abs(E64.item()),
            "V_rel_diff_fp32_vs_fp64": float(torch.linalg.norm(V - V64) / torch.linalg.norm(V64)),
        }
        ex64.close()

    if rank == 0 and not args.no_cpu_baseline:
        # the oracle as it stands on the host cores, on a bounded sample of the same workload;
        # the GPU path runs the same sample list for the stated error
        ncpu = len(os.sched_getaffinity(0))
        rate, dt, _, _, _ = oracle_rate(phi_np, pairs_np, w.lattice, 4, seed=321)
        n_sample = int(max(8, min(P, 20.0 * rate)))
        rate, dt, sub, E_o, V_o = oracle_rate(phi_np, pairs_np, w.lattice, n_sample, seed=7)
        sub_d = torch.from_numpy(sub).to(dev)
        Es, Vs = ex.apply(phi, sub_d)
        torch.cuda.synchronize()
        Vs_np = Vs.cpu().numpy()
        # the same oracle on every host core (one process per core) over a larger sample
        pool = OraclePool(phi_np, w.lattice)
        try:
            n_all = int(max(pool.procs, min(P, 15.0 * rate * pool.procs)))
            rate_all, dt_all, _ = pool.rate(pairs_np, n_all, seed=8)
        finally:
            pool.close()
        line["cpu_baseline_all_cores"] = {
            "value": rate_all, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
            "sample": f"{n_all} seeded random pairs of the {P}-pair list split over {pool.procs} processes "
                      f"({dt_all:.1f} s wall, numpy FP64, one process per host core)"}
        line["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(sub)} seeded random pairs of the {P}-pair list ({dt:.1f} s, numpy FP64, "
                      f"1 thread of {ncpu} host cores)",
            "gpu_error_on_sample": {"precision": args.precision,
                                    "E_rel": abs(Es.item() - E_o) / abs(E_o),
                                    "V_rel": float(np.linalg.norm(Vs_np - V_o) / np.linalg.norm(V_o))},
        }
        if ace_out is not None:
            # the ACE oracle at full size on the same phi and W (numpy FP64, default BLAS threads)
            from oracle import ace_oracle as AO
            M_g, P_g = ace_out
            t0 = time.time()
            M0, _, P0 = AO.ace_build(phi_np, V.cpu().numpy(), np.asarray(w.lattice))
            dt_ace = time.time() - t0

            def rel(a, b):
                return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))

            line["cpu_baseline"]["ace_build"] = {
                "seconds": dt_ace, "gpu_ms": line["ace"]["ms"]["build"],
                "sample": f"full ACE construction, {n_orb} orbitals on {N} points",
                "M_rel_gpu_vs_oracle": rel(M_g.cpu().numpy(), M0), "P_rel_gpu_vs_oracle": rel(P_g.cpu().numpy(), P0)}

    if rank == 0 and not args.no_extra:
        from oracle import hfx_oracle as O
        ex.close()
        del V, phi
        torch.cuda.empty_cache()
        extra = {"water64_n96": measure_workload("water64_n96", args.precision, hfx, I, O, dev),

                 "uneven_batch": measure_batch(hfx, I, dev, args.precision)}
        # the 96^3 workload with the forward DFTs on the tensor cores (HFX_PREC_MIXED_TC: each
        # axis one dense split-TF32 GEMM), beside the FP32 SIMT stages on the same inputs
        mt = measure_workload("water64_n96", "mixed_tc", hfx, I, O, dev)
        f32 = extra["water64_n96"]
        line["mixed_tc"] = {
            "config": mt["config"], "value": mt["value"], "unit": UNIT, "ms_per_call": mt["ms_per_call_median"],
            "fwd_pass_ms": mt["roofline_passes"]["fwd_yz"]["ms_per_step"],
            "errors": {"E_rel_err_vs_oracle_on_sample": mt["checks"]["E_rel_err_vs_oracle_on_sample"],
                       "homogeneity_rel_err": mt["checks"]["homogeneity_rel_err"],
                       "sample": mt["checks"]["sample"]},
            "fp32_simt_same_inputs": {"value": f32["value"], "ms_per_call": f32["ms_per_call_median"],
                                      "fwd_pass_ms": f32["roofline_passes"]["fwd_yz"]["ms_per_step"],
                                      "E_rel_err_vs_oracle_on_sample": f32["checks"]["E_rel_err_vs_oracle_on_sample"]},
            "tc_over_simt": mt["value"] / f32["value"],
            "roofline_passes": mt["roofline_passes"]}
        if args.with_128:
            extra["water128_n128"] = measure_workload("water128_n128", args.precision, hfx, I, O, dev, reps=2, n_check=8)
        line["other_workloads"] = extra
    else:
        ex.close()

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
