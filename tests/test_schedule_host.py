"""The library's pair-block schedule (host code, csrc/hfx_schedule.h), built on the CPU through a
small probe program and checked against what the accumulate passes rely on:

* every orbital-block pair I <= J is scheduled exactly once, and slot_of_bp finds it;
* no two block pairs of one batch share a block (each V_x phi tile has one writer per launch,
  which is what makes the accumulation race-free and deterministic without atomics);
* a block pair's couple capacity holds its pairs two per couple, off-diagonal pairs with
  off-diagonal ones and diagonal pairs with diagonal ones (equal-weight couples), with no spare
  couple beyond the one an odd count needs;
* batches cover the slots in order and keep within the transform budget (a single block pair
  larger than the budget gets a batch of its own);
* the dense, diagonal-block and generic accumulation lists partition every batch's slots by the
  rule the kernels assume (full off-diagonal pairs, full diagonal pairs, the rest).
"""
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROBE = os.path.join(ROOT, "tests", "schedule_probe.cpp")
CUDA_INCLUDE = "/usr/local/cuda/include"


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INCLUDE):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path_factory.mktemp("schedule") / "probe")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CUDA_INCLUDE, PROBE, "-o", exe], check=True)

    def run(n_orb, b, budget_couples, dense=True, diag=True, bytes_per_couple=1000):
        out = subprocess.run([exe, str(n_orb), str(b), str(budget_couples * bytes_per_couple), str(bytes_per_couple),
                              str(int(dense)), str(int(diag))], check=True, capture_output=True, text=True).stdout
        return json.loads(out)
    return run


def block_size(bi, b, n_orb):
    return min(b, n_orb - bi * b)


CASES = [  # n_orb, block, budget (couples), dense, diag
    (128, 8, 1 << 30, True, True),     # the 72^3 water box with an unlimited budget
    (128, 8, 300, True, True),         # one round split over batches
    (128, 8, 40, True, True),          # budget below one block pair: one slot per batch
    (100, 8, 500, True, True),         # ragged last block
    (255, 8, 1000, True, False),       # odd block count (a dummy partner per round)
    (13, 4, 9, False, False),          # small blocks, no specialised passes
    (7, 8, 100, True, True),           # a single ragged block
    (1, 8, 100, True, True),           # a single orbital
    (512, 8, 2000, True, True),        # the 512-orbital workload's block count
    (40, 5, 30, True, True),           # block size 5
]


@pytest.mark.parametrize("n_orb,b,budget,dense,diag", CASES)
def test_schedule_invariants(probe, n_orb, b, budget, dense, diag):
    S = probe(n_orb, b, budget, dense, diag)
    nb = (n_orb + b - 1) // b
    assert S["nb"] == nb and S["nslots"] == len(S["slot_blocks"]) == nb * (nb + 1) // 2
    # every block pair exactly once, found through slot_of_bp
    seen = [tuple(bp) for bp in S["slot_blocks"]]
    assert sorted(seen) == sorted((i, j) for i in range(nb) for j in range(i, nb))
    for I in range(nb):
        for J in range(nb):
            k = S["slot_of_bp"][I * nb + J]
            if I <= J:
                assert tuple(S["slot_blocks"][k]) == (I, J)
            else:
                assert k == -1
    # capacities: two pairs per couple, equal-weight couples
    for k, (I, J) in enumerate(seen):
        si, sj = block_size(I, b, n_orb), block_size(J, b, n_orb)
        if I != J:
            need = (si * sj + 1) // 2
        else:
            need = (si * (si - 1) // 2 + 1) // 2 + (si + 1) // 2
        assert S["slot_cap"][k] == need
        assert S["slot_couple_base"][k + 1] - S["slot_couple_base"][k] == need
    assert S["slot_couple_base"][0] == 0 and S["slot_couple_base"][-1] == S["max_total_couples"]
    # batches: in order, within the budget, blocks disjoint inside a batch
    begin = S["batch_slot_begin"]
    assert begin[0] == 0 and begin[-1] == S["nslots"] and len(begin) == S["nbatches"] + 1
    assert all(a < c for a, c in zip(begin, begin[1:]))
    assert S["nbatches"] >= (nb if nb > 1 else 1)  # at least one batch per round
    biggest = 0
    for bt in range(S["nbatches"]):
        slots = range(begin[bt], begin[bt + 1])
        couples = sum(S["slot_cap"][k] for k in slots)
        biggest = max(biggest, couples)
        assert couples <= budget or len(slots) == 1
        blocks = []
        for k in slots:
            I, J = S["slot_blocks"][k]
            blocks += [I] if I == J else [I, J]
        assert len(blocks) == len(set(blocks)), f"batch {bt} has two block pairs sharing a block"
    assert S["max_batch_couples"] == biggest
    # accumulation lists: a partition of each batch by the kernels' rule
    for bt in range(S["nbatches"]):
        slots = set(range(begin[bt], begin[bt + 1]))
        lists = {name: S[f"{name}_slots"][S[f"{name}_begin"][bt]:S[f"{name}_begin"][bt + 1]]
                 for name in ("dense", "diag", "generic")}
        got = [k for v in lists.values() for k in v]
        assert sorted(got) == sorted(slots)
        for k in slots:
            I, J = S["slot_blocks"][k]
            full = block_size(I, b, n_orb) == b and block_size(J, b, n_orb) == b
            want = "dense" if (dense and I != J and full) else "diag" if (diag and I == J and full) else "generic"
            assert k in lists[want]


def test_rounds_pair_every_block_once(probe):
    """With an unlimited budget a batch is a whole round: for an even block count every round of
    the circle method but the last pairs all blocks off-diagonally, and the last holds the diagonal
    pairs; for an odd count each round leaves one block to its diagonal pair."""
    for n_orb, nb in ((128, 16), (120, 15)):
        S = probe(n_orb, 8, 1 << 30)
        begin = S["batch_slot_begin"]
        assert S["nbatches"] == nb  # nb - 1 rounds and the diagonal one, or nb rounds with a dummy
        for bt in range(S["nbatches"]):
            pairs = [tuple(S["slot_blocks"][k]) for k in range(begin[bt], begin[bt + 1])]
            covered = sorted(x for I, J in pairs for x in ({I, J}))
            assert covered == list(range(nb))
