"""Multi-rank pair sharding on CPU with the gloo backend (world size 2).

Each rank evaluates its share of the pair list with the FP64 oracle, the shares are summed with
one all-reduce (the CP-group global sum of Sec. 2.2), and the sum must equal the single-process
result.  A rank that dies before the collective must make the survivor's collective fail within
its timeout (failure detection on the host, no GPU involved).
"""
import datetime
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    from paper_2309_00651_gb300 import inputs as I
    L, n, n_orb = 7.0, 10, 6
    raw = I.random_pw_orbitals(n_orb, L, n, ecut=0.5 * (2 * np.pi * 3.0 / L) ** 2, seed=21)
    phi, _ = I.loewdin(raw, L ** 3)
    return phi, I.all_pairs(n_orb), np.diag([L] * 3)


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    from oracle import hfx_oracle as O
    from paper_2309_00651_gb300 import shard
    phi, pairs, lat = _problem()
    mine = shard.partition_pairs(pairs, world, rank)
    E, V = O.exchange(phi, mine, lat)
    Et = torch.tensor([E], dtype=torch.float64)
    Vt = torch.from_numpy(V)
    shard.reduce_exchange(Et, Vt)
    if rank == 0:
        np.savez(out_path, E=Et.numpy(), V=Vt.numpy(), n=len(mine))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_covers_every_pair_once():
    from paper_2309_00651_gb300 import inputs as I
    from paper_2309_00651_gb300 import shard
    pairs = I.all_pairs(13)
    rng = np.random.default_rng(0)
    shuffled = pairs[rng.permutation(len(pairs))]
    for world in (1, 2, 3, 8):
        parts = [shard.partition_pairs(shuffled, world, r) for r in range(world)]
        cat = np.concatenate(parts)
        assert len(cat) == len(pairs)
        assert {tuple(p) for p in cat} == {tuple(p) for p in pairs}
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_sum_to_the_full_result(tmp_path):
    from oracle import hfx_oracle as O
    out = str(tmp_path / "r0.npz")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    phi, pairs, lat = _problem()
    E, V = O.exchange(phi, pairs, lat)
    got = np.load(out)
    assert got["E"][0] == pytest.approx(E, rel=1e-13)
    assert np.linalg.norm(got["V"] - V) <= 1e-13 * np.linalg.norm(V)
    assert int(got["n"]) == len(pairs) // 2 + len(pairs) % 2


def _dying_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        os._exit(0)  # leaves between steps, before the collective, with nothing in flight
    t = torch.ones(4, dtype=torch.float64)
    failed = False
    try:
        dist.all_reduce(t)
    except Exception:
        failed = True
    with open(out_path, "w") as f:
        f.write("failed" if failed else "completed")
    os._exit(0)


def test_lost_rank_is_detected_by_the_survivor(tmp_path):
    out = str(tmp_path / "status.txt")
    ctx = mp.start_processes(_dying_worker, args=(2, _free_port(), out), nprocs=2, join=False, start_method="spawn")
    for p in ctx.processes:
        p.join(timeout=120)
    with open(out) as f:
        assert f.read() == "failed"
