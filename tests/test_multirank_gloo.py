"""The multi-process (N > 1) path on CPU ranks with the gloo backend: the
bench's max-over-ranks timing and the replicas-only served stream (each rank
serves its shard with its own server; rank 0 gathers every result)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2302_08843_gb300 import binding
    from paper_2302_08843_gb300.serving import Server, latency_summary
    from test_serving_host import FakeBatch, _requests
    binding.Batch = FakeBatch
    # max over ranks: every rank sees the largest value
    m = bench.max_over_ranks(torch, dist, 1.5 + rank, "cpu")
    reqs = _requests(7, 23, [(8, 8, 1), (16, 4, 2)])
    srv = Server(hbm_cap=1e12, capacity=4)
    res, elapsed = bench.serve_replicas(torch, dist, rank, world, reqs, srv)
    srv.close()
    if rank == 0:
        steps = [r["steps"] for r in res]
        expect = [int(w.Ms // 1e5) for (_, w) in reqs]
        summ = latency_summary(res, elapsed)
        np.save(os.path.join(outdir, "out.npy"), np.array([m, elapsed, summ["converged"]] + steps + expect))
    else:
        np.save(os.path.join(outdir, "out%d.npy" % rank), np.array([m]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    tmp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    out = np.load(tmp_path / "out.npy")
    m, elapsed, converged = out[0], out[1], int(out[2])
    rest = out[3:]
    steps, expect = rest[:23], rest[23:]
    assert m == 2.5 and np.load(tmp_path / "out1.npy")[0] == 2.5
    assert elapsed >= 0 and converged == 23
    # every request served exactly once, its result independent of the shard it landed in
    assert np.array_equal(steps, expect)
