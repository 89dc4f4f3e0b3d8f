"""Host logic of multi-rank runs on CPU (gloo, world size 2): every rank runs its own share of
an ensemble (no data-path collective) and the whole-job figures are the slowest rank's time
and the summed work.  No GPU is used."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = bench.shard(bench.ensemble_specs(64), ws, rank)
        # per-rank figures that differ: time, work and simulated time
        ms, n_rhs, sim = 10.0 + 5.0 * rank, 100 + rank, 0.5 * (rank + 1)
        agg = bench.aggregate(dist, ws, ms, n_rhs, sim, "cpu")
        q.put((rank, [s[3] for s in mine], agg))
    finally:
        dist.destroy_process_group()


def test_ensemble_sharding_and_whole_job_figures_two_ranks():
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = dict((r, (ids, agg)) for r, ids, agg in (q.get(timeout=120) for _ in range(ws)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every instance runs on exactly one rank
    ids = sorted(out[0][0] + out[1][0])
    assert ids == list(range(64)) and not set(out[0][0]) & set(out[1][0])
    # both ranks see the same whole-job figures: max time, summed work
    for r in range(ws):
        assert out[r][1] == (15.0, 201.0, 1.5)


def test_single_rank_is_the_identity():
    import bench
    assert bench.aggregate(None, 1, 3.0, 7, 0.25, "cpu") == (3.0, 7.0, 0.25)
    assert bench.shard(range(5), 1, 0) == [0, 1, 2, 3, 4]
    assert bench.shard(range(5), 2, 1) == [1, 3]
