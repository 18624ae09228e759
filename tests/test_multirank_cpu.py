"""The multi-process side of the benchmark and the sharding of events over ranks,
as world_size-2 gloo process groups on the CPU (rendezvous on 127.0.0.1):
the timing reduction takes the max over ranks, and filling each rank's
share of the events and summing the histograms over ranks gives the
histogram of all events (bins and counts exact, as the merge a multi-GPU
fill would do)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        m = bench.max_over_ranks(1.5 + rank, world)
        import oracle
        from paper_2401_13310_gb300 import workloads as W
        wl = W.cfg2a(n=20_000)
        lo, hi = rank * 10_000, (rank + 1) * 10_000
        r = oracle.fill(wl.axes, np.ascontiguousarray(wl.values[:, lo:hi]), np.ascontiguousarray(wl.weights[lo:hi]))
        counts = torch.from_numpy(r.counts.astype(np.int64))
        bins = torch.from_numpy(r.bins_acc.copy())
        dist.all_reduce(counts, op=dist.ReduceOp.SUM)
        dist.all_reduce(bins, op=dist.ReduceOp.SUM)
        out[rank] = (m, counts.numpy().tolist(), bins.numpy().tolist())
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_merged_histogram():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=180)
            assert p.exitcode == 0
        res = dict(out)
    import oracle
    from paper_2401_13310_gb300 import workloads as W
    wl = W.cfg2a(n=20_000)
    full = oracle.fill(wl.axes, wl.values, wl.weights)
    for rank in range(2):
        m, counts, bins = res[rank]
        assert m == 2.5
        assert np.array_equal(np.asarray(counts), full.counts.astype(np.int64))
        assert np.all(np.abs(np.asarray(bins) - full.bins_acc) <= 1e-12 * full.bins_abs + 1e-300)
