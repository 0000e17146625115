"""World-size-2 gloo tests of the multi-process host logic (no GPU): timing
reduction as bench.py uses it, and target sharding whose union equals a
single-process network inference (CPU oracle as the per-rank engine)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1902_06828_gb300.shard import shard_targets


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from oracle import network as onet
    from paper_1902_06828_gb300.shard import combine_timing, gather_results
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        times, counts = combine_timing(dist, [100.0 + rank, 5.0 * (rank + 1)], [10 * (rank + 1)])
        x, _, _ = synth.var_er(n=4, p=0.4, T=250, seed=2, lo=0.4, hi=0.7, max_lag=2)
        s = synth.standardise_jitter(x, 2)
        p = onet.Params(n_surr=20, alpha_max=0.1, alpha_min=0.1, alpha_omnibus=0.1,
                        max_lag_target=2, max_lag_sources=2, seed=4, n_threads=1)
        mine = shard_targets(4, rank, world)
        res = [(r.target, r.sel_sources, r.omnibus_p)
               for r in (onet.infer_target(s, t, p) for t in mine)]
        allres = gather_results(dist, res)
        q.put((rank, times, counts, allres))
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_target_shards():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    outs = [q.get(timeout=240) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, times, counts, allres in outs:
        assert times == [101.0, 10.0]          # max over ranks
        assert counts == [30.0]                # sum over ranks
    # the union of the shards equals one process running every target
    from oracle import network as onet
    import synth
    x, _, _ = synth.var_er(n=4, p=0.4, T=250, seed=2, lo=0.4, hi=0.7, max_lag=2)
    s = synth.standardise_jitter(x, 2)
    p = onet.Params(n_surr=20, alpha_max=0.1, alpha_min=0.1, alpha_omnibus=0.1,
                    max_lag_target=2, max_lag_sources=2, seed=4, n_threads=1)
    single = {t: (r.sel_sources, r.omnibus_p) for t, r in
              ((t, onet.infer_target(s, t, p)) for t in range(4))}
    union = {}
    for shard in outs[0][3]:
        for t, sel, pv in shard:
            union[t] = (sel, pv)
    assert union == single


def test_shard_targets_partition():
    for n, w in ((10, 1), (10, 3), (100, 8), (3, 4)):
        parts = [shard_targets(n, r, w) for r in range(w)]
        flat = sorted(t for part in parts for t in part)
        assert flat == list(range(n))
    with pytest.raises(ValueError):
        shard_targets(5, 2, 2)
