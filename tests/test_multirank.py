"""The multi-rank host logic on CPU: two gloo ranks (no GPU)."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_2312_05890_gb300 import multirank
    w, r, lr = multirank.rank_env()
    dist = multirank.init(w)
    multirank.barrier(dist)
    # rank r: (10 (r + 1)) ms for 100 (r + 1) units
    res = multirank.job_rate(10.0 * (r + 1), 100 * (r + 1), dist)
    seed = multirank.weak_seed(7, r)
    # shard brackets beyond 2^32: the sums stay exact
    counts = multirank.sum_counts((1 << 40) + r, (1 << 41) + 3 * r, dist)
    multirank.finish(dist)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"env": [w, r, lr], "rate": res, "seed": seed, "counts": counts}, f)


@pytest.mark.timeout(120)
def test_two_gloo_ranks_reduce_time_and_units(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, g in enumerate(got):
        assert g["env"] == [world, r, r]
        max_ms, total, rate = g["rate"]
        # the job took as long as its slowest rank and did every rank's units
        assert max_ms == 20.0 and total == 300.0
        assert rate == pytest.approx(300.0 / 0.020)
        assert g["seed"] == 7 + r
        assert g["counts"] == [(1 << 41) + 1, (1 << 42) + 3]
    assert got[0]["seed"] != got[1]["seed"]


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2312_05890_gb300 import multirank
    w, r, lr = multirank.rank_env()
    assert (w, r, lr) == (1, 0, 0)
    dist = multirank.init(w)
    assert dist is None
    assert multirank.job_rate(40.0, 8, dist) == (40.0, 8.0, 200.0)
