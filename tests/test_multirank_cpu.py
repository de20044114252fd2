"""Multi-rank logic on CPU (gloo, world size 2).

- The benchmark's whole-job aggregation: max time over ranks, summed work.
- The space-charge exchange of a pack-sharded run: each rank deposits its
  own packs, one all-reduce (sum) of the int64 charge grid gives exactly the
  single-rank deposit (integer addition is exact and order-independent).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _init(rank, ws, port):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)


def _agg_worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    _init(rank, ws, port)
    import bench
    t, p = bench.aggregate(10.0 + 5 * rank, 1000 * (rank + 1), torch.device("cpu"), ws)
    q.put((rank, t, p))
    dist.destroy_process_group()


def _deposit_worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    _init(rank, ws, port)
    import oracle
    from paper_2609_31258_b300 import workloads as W
    w = W.cylinder_space_charge(n_packs=6001, n_steps=0, pic_nr=33, pic_nz=129)
    s = oracle.Sim(w)
    s.inject()
    xq, yq, zq = s.quantized()
    lo, hi = rank * s.n // ws, (rank + 1) * s.n // ws
    Q = oracle.deposit_fixed(w.fields.pic, xq[lo:hi], yq[lo:hi], zq[lo:hi], s.status[lo:hi],
                             w.ion.charge * w.source.weight)
    t = torch.from_numpy(Q.copy())
    dist.all_reduce(t)
    full = oracle.deposit_fixed(w.fields.pic, xq, yq, zq, s.status[:s.n], w.ion.charge * w.source.weight)
    q.put((rank, bool((t.numpy() == full).all()), int(full.sum())))
    dist.destroy_process_group()


def _run(worker, ws=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_bench_aggregation_two_ranks():
    out = _run(_agg_worker)
    for rank, t, p in out:
        assert t == 15.0 and p == 3000.0


def test_sharded_deposit_allreduce_is_exact():
    out = _run(_deposit_worker)
    assert all(ok for _, ok, _ in out)
    assert out[0][2] == 6001 * 1000 * 2 ** 30
