"""Host logic of the multi-GPU replica mode, run as two ``gloo`` ranks on CPU.

Each rank owns whole problems (round-robin), the timed duration of the job is
the maximum over ranks and the throughput counts the units of every rank.  A
rank that leaves before the timing reduction makes the other rank's
collective end with an error after a short process-group timeout.
"""
import datetime
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir, scenario):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2103_00081_gb300 import replicas as R

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world, timeout=datetime.timedelta(seconds=5))
    res = {"rank": rank}
    try:
        if scenario == "timing":
            n = 11
            mine = R.shard(n, rank, world)
            res["mine"] = mine
            # rank r "took" (r + 1) s of wall time and processed len(mine) problems
            (t_max,) = R.max_over_ranks([rank + 1.0], dist)
            (units,) = R.sum_over_ranks([len(mine)], dist)
            res["t_max"] = t_max
            res["units"] = units
            res["rate"] = R.job_rate(units, t_max)
            res["mixed"] = R.max_over_ranks([float(rank), -float(rank), 3.0], dist)
        elif scenario == "rank_leaves":
            if rank == 1:
                res["left"] = True  # leaves between steps, before the reduction
            else:
                try:
                    R.max_over_ranks([1.0], dist)
                    res["error"] = None
                except Exception as exc:  # the process-group timeout surfaces here
                    res["error"] = type(exc).__name__
    finally:
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(res, f)
        if scenario != "rank_leaves":
            dist.destroy_process_group()


def _run(scenario, tmp_path, world=2):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path), scenario), nprocs=world,
                       join=True, start_method="spawn")
    out = []
    for r in range(world):
        with open(tmp_path / f"rank{r}.json") as f:
            out.append(json.load(f))
    return out


def test_shard_covers_every_problem_once():
    from paper_2103_00081_gb300 import replicas as R
    for n in (0, 1, 7, 64):
        for world in (1, 2, 3, 8):
            parts = [R.shard(n, r, world) for r in range(world)]
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        R.shard(4, 2, 2)
    with pytest.raises(ValueError):
        R.job_rate(1.0, 0.0)


def test_single_process_reductions_are_identity():
    from paper_2103_00081_gb300 import replicas as R
    assert R.max_over_ranks([1.5, 2]) == [1.5, 2.0]
    assert R.sum_over_ranks([3]) == [3.0]


def test_two_gloo_ranks_max_time_and_summed_units(tmp_path):
    r0, r1 = _run("timing", tmp_path)
    assert sorted(r0["mine"] + r1["mine"]) == list(range(11))
    assert not set(r0["mine"]) & set(r1["mine"])
    for r in (r0, r1):
        assert r["t_max"] == 2.0          # the slowest rank's duration
        assert r["units"] == 11.0         # every rank's problems
        assert r["rate"] == pytest.approx(5.5)
        assert r["mixed"] == [1.0, 0.0, 3.0]


def test_rank_that_leaves_ends_the_others_collective_with_an_error(tmp_path):
    r0, r1 = _run("rank_leaves", tmp_path)
    assert r1["left"]
    assert r0["error"] is not None
