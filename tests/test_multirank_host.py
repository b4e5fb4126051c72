"""The multi-GPU path on CPU: two gloo ranks each serve their round-robin
share of a render stream (fake backend) and merge their latency records; the
shares cover every render exactly once and the merged summary equals the
single-process one. Also the max-over-ranks time reduction bench.py uses."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2202_00086_gb300 import serve, workloads


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from test_serve_host import FakeBackend
    stream = [(0.0, rd) for rd in workloads.uneven_batch(n=24, seed=4, sides=(16, 32, 64))]
    mine = serve.shard(stream, rank, world)
    ref = [None]
    srv = serve.RenderServer(backend=FakeBackend(ref), keep_outputs=True, round_rays=5000,
                             min_chunk=500)
    ref[0] = srv
    srv.run(mine, realtime=False, poll_s=0)
    rec = serve.local_record(srv.done)
    recs = [None] * world
    dist.all_gather_object(recs, rec)
    ids = [[(rd["nx"], rd["a"]) for _, rd in mine]]
    all_ids = [None] * world
    dist.all_gather_object(all_ids, ids[0])
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        results["merged"] = serve.merge_records(recs)
        results["ids"] = all_ids
        results["tmax"] = float(t.item())
        results["n_stream"] = len(stream)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_shards_and_merge():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        results = m.dict()
        mp.spawn(_worker, args=(world, port, results), nprocs=world, join=True)
        merged = dict(results["merged"])
        ids = list(results["ids"])
        assert results["tmax"] == 2.0
        n = results["n_stream"]
    flat = [x for part in ids for x in part]
    assert len(flat) == n and len(set(flat)) == n  # every render once
    assert merged["renders"] == n
    assert merged["p99_latency_s"] >= merged["p50_latency_s"] >= 0.0
