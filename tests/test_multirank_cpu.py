"""The N>1 path of bench.py on the CPU: two gloo ranks run the same rank
plumbing the GPU bench uses under torchrun (environment, per-rank shards of
boxes, slowest-rank timing, whole-job rate) and the reference arm's rule that
only rank 0 works.  The path has no data exchange, so nothing else crosses
ranks."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, lr = bench.rank_env()
    Q = 300
    boxes = bench.rank_boxes(2, Q, r)
    again = bench.rank_boxes(2, Q, r)
    shards = [None] * w
    dist.all_gather_object(shards, boxes.tolist())
    # each rank's own step time; the job is timed by the slowest
    t = bench.max_over_ranks(10.0 + 5.0 * r, w, "cpu")
    rate = bench.whole_job_rate(w, Q, t / 4)
    ref = bench.run_reference(bench.parse(["--impl", "reference"])) if r != 0 else "skipped"
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % r), "w") as f:
        json.dump(dict(env=[w, r, lr], deterministic=bool(np.array_equal(boxes, again)), shards=shards,
                       t=t, rate=rate, ref=ref), f)


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    dims = np.array((512, 512, 384))
    for r, x in enumerate(res):
        assert x["env"] == [world, r, r]
        assert x["deterministic"]
        # slowest rank (15 ms) times the job; rate counts the units of both ranks
        assert x["t"] == 15.0
        assert x["rate"] == pytest.approx(world * 300 / (15.0 / 4 / 1e3))
    # both ranks saw the same shards, and the shards are different, valid batches
    assert res[0]["shards"] == res[1]["shards"]
    a, b = (np.array(s) for s in res[0]["shards"])
    assert not np.array_equal(a, b)
    for s in (a, b):
        assert s.shape == (300, 6)
        assert (s[:, :3] >= 0).all() and (s[:, 3:] >= 1).all() and (s[:, :3] + s[:, 3:] <= dims).all()
    # the reference arm: ranks other than 0 exit without work
    assert res[1]["ref"] is None
