"""Host logic of the schedule autotuner (paper_2309_00651_gb300/autotune.py) on the CPU: the
fastest candidate is applied and cached under its shape key, a candidate that raises is skipped
and reported, a cached entry is applied without timing, and a run where nothing works raises.
The exchange context and the timing are fakes; tests/test_gpu_tuning.py times real calls."""
import pytest

torch = pytest.importorskip("torch")

from paper_2309_00651_gb300 import autotune as T  # noqa: E402


class FakeExchange:
    def __init__(self):
        self.applied = []

    def set_tuning(self, block, batch_bytes, pipeline):
        self.applied.append((block, batch_bytes, pipeline))


CANDS = (
    {"block": 8, "batch_bytes": 1 << 30, "pipeline": True},
    {"block": 8, "batch_bytes": 1 << 29, "pipeline": True},
    {"block": 4, "batch_bytes": 1 << 30, "pipeline": False},
)


def fake_timer(table):
    def time_call(exch, phi, pairs, steps):
        setting = exch.applied[-1]
        ms = table[setting]
        if ms is None:
            raise RuntimeError("does not fit")
        return ms
    return time_call


def run(monkeypatch, tmp_path, times, use_cache=True):
    monkeypatch.setattr(T, "shape_key", lambda exch, n_orb: f"fake|72x72x72|norb{n_orb}|fp32")
    monkeypatch.setattr(T, "time_call", fake_timer(times))
    ex = FakeExchange()
    phi = torch.zeros(128, 1)
    pairs = torch.zeros(8256, 2, dtype=torch.int32)
    res = T.tune(ex, phi, pairs, candidates=CANDS, use_cache=use_cache, path=str(tmp_path / "tune.json"))
    return ex, res


def test_fastest_applied_failures_skipped_and_cached(monkeypatch, tmp_path):
    times = {(8, 1 << 30, True): 19.1, (8, 1 << 29, True): 18.9, (4, 1 << 30, False): None}
    ex, res = run(monkeypatch, tmp_path, times)
    assert res["cached"] is False
    assert res["setting"] == CANDS[1] and res["ms"] == 18.9
    assert ex.applied[-1] == (8, 1 << 29, True)          # the winner is left applied
    assert sum("error" in t for t in res["trials"]) == 1  # the raising candidate is reported
    # a second context of the same shape starts from the cache, without timing anything
    ex2, res2 = run(monkeypatch, tmp_path, {})
    assert res2["cached"] is True and res2["setting"] == CANDS[1]
    assert ex2.applied == [(8, 1 << 29, True)]


def test_no_cache_times_again(monkeypatch, tmp_path):
    times = {(8, 1 << 30, True): 5.0, (8, 1 << 29, True): 6.0, (4, 1 << 30, False): 7.0}
    run(monkeypatch, tmp_path, times)
    times2 = {(8, 1 << 30, True): 9.0, (8, 1 << 29, True): 6.0, (4, 1 << 30, False): 7.0}
    _, res = run(monkeypatch, tmp_path, times2, use_cache=False)
    assert res["cached"] is False and res["setting"] == CANDS[1]


def test_nothing_runs_raises(monkeypatch, tmp_path):
    times = {(8, 1 << 30, True): None, (8, 1 << 29, True): None, (4, 1 << 30, False): None}
    with pytest.raises(RuntimeError):
        run(monkeypatch, tmp_path, times)


class FakeBatchExchange:
    def __init__(self, log):
        self.log = log

    def set_tuning(self, block, batch_bytes, pipeline):
        self.log.append(("tune", batch_bytes))

    def ensure_workspace(self, n_orb, n_pairs):
        self.log.append(("ws", n_orb, n_pairs))


def test_batch_tuner_picks_budget_then_form():
    """The batch tuner times the persistent launch per transform budget (a budget that raises is
    skipped), applies the fastest to every context with its workspace, then keeps the
    one-call-per-problem form only if that is faster."""
    log = []
    exs = [FakeBatchExchange(log), FakeBatchExchange(log)]
    current = {"b": None}
    orig = exs[0].set_tuning

    def set_tuning(block, batch_bytes, pipeline):
        current["b"] = batch_bytes
        orig(block, batch_bytes, pipeline)
    exs[0].set_tuning = set_tuning
    ms_of = {1 << 30: 9.0, 512 << 20: 7.0, 256 << 20: None, 2 << 30: 8.0}

    def timer(run, steps):
        return run()

    def persistent():
        ms = ms_of[current["b"]]
        if ms is None:
            raise RuntimeError("does not fit")
        return ms

    res = T.tune_batch(exs, persistent, lambda: 7.5, [10, 20], [55, 210], timer=timer)
    assert res["setting"] == {"batch_bytes": 512 << 20, "mode": "persistent"} and res["ms"] == 7.0
    assert any("error" in t for t in res["trials"])
    assert log[-4:] == [("tune", 512 << 20), ("ws", 10, 55), ("tune", 512 << 20), ("ws", 20, 210)]
    res2 = T.tune_batch(exs, persistent, lambda: 6.0, [10, 20], [55, 210], timer=timer)
    assert res2["setting"]["mode"] == "sequential" and res2["ms"] == 6.0
