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


def _fdr_worker(rank, world, port, q):
    import torch.distributed as dist

    from oracle import network as onet
    from paper_1902_06828_gb300.shard import gather_results, merge_network_shards
    import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, _, _ = synth.var_er(n=5, p=0.35, T=260, seed=9, lo=0.3, hi=0.6, max_lag=2)
        s = synth.standardise_jitter(x, 9)
        p = onet.Params(n_surr=20, alpha_max=0.1, alpha_min=0.1, alpha_omnibus=0.1,
                        max_lag_target=2, max_lag_sources=2, seed=6, n_threads=1)
        targets = []
        n_est = 0
        for t in shard_targets(5, rank, world):      # each rank: its targets, no FDR
            r = onet.infer_target(s, t, p)
            n_est += r.n_estimates
            targets.append(dict(target=t, sel_target=r.sel_target, sel_sources=r.sel_sources,
                                omnibus_p=r.omnibus_p, omnibus_tested=r.omnibus_tested,
                                significant=r.significant))
        shards = gather_results(dist, dict(targets=targets, n_estimates=n_est))
        q.put((rank, merge_network_shards(shards, 5, fdr=True, alpha_fdr=0.06)))
    finally:
        dist.destroy_process_group()


def test_sharded_network_with_fdr_equals_one_process():
    """FDR across targets needs every omnibus p-value: the shards are merged
    after the gather, and the result equals one process inferring every
    target with FDR (CPU oracle as the per-rank engine)."""
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_fdr_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    outs = [q.get(timeout=240) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    from oracle import network as onet
    import synth
    x, _, _ = synth.var_er(n=5, p=0.35, T=260, seed=9, lo=0.3, hi=0.6, max_lag=2)
    s = synth.standardise_jitter(x, 9)
    p = onet.Params(n_surr=20, alpha_max=0.1, alpha_min=0.1, alpha_omnibus=0.1,
                    max_lag_target=2, max_lag_sources=2, seed=6, n_threads=1, fdr=True,
                    alpha_fdr=0.06)
    adj, res = onet.infer_network(s, p)
    for _rank, merged in outs:
        np.testing.assert_array_equal(merged["adjacency"], adj)
        assert [t["target"] for t in merged["targets"]] == list(range(5))
        for t, r in zip(merged["targets"], res):
            assert list(t["sel_sources"]) == list(r.sel_sources)
            assert t["significant"] == r.significant
        assert merged["n_estimates"] == sum(r.n_estimates for r in res)


def test_merge_applies_fdr_across_shards_by_hand():
    # four tested targets over two shards, p = 0.01, 0.04, 0.03, 0.20; with
    # alpha = 0.05 and m = 4 the BH thresholds are 0.0125, 0.025, 0.0375, 0.05:
    # only rank 1 (p = 0.01) passes, so targets 1, 2 and 3 lose their sources;
    # target 4 had no omnibus test and is not counted in m
    from paper_1902_06828_gb300.shard import merge_network_shards

    def t(target, p, tested=True, src=((0, 1),)):
        return dict(target=target, sel_target=[(target, 1)], sel_sources=list(src) if tested else [],
                    omnibus_p=p, omnibus_tested=tested, significant=tested)
    shards = [dict(targets=[t(2, 0.04), t(0, 0.01, src=((3, 2),))], n_estimates=10),
              dict(targets=[t(1, 0.03, src=((2, 1),)), t(3, 0.20), t(4, 1.0, tested=False)],
                   n_estimates=7)]
    m = merge_network_shards(shards, 5, fdr=True, alpha_fdr=0.05)
    assert [x["target"] for x in m["targets"]] == [0, 1, 2, 3, 4]
    assert [bool(x["sel_sources"]) for x in m["targets"]] == [True, False, False, False, False]
    assert m["adjacency"].sum() == 1 and m["adjacency"][3, 0] == 1 and m["min_lag"][3, 0] == 2
    assert m["n_estimates"] == 17
    # without FDR every tested target keeps its sources
    m = merge_network_shards(shards, 5, fdr=False)
    assert int(m["adjacency"].sum()) == 4
    # equal p-values pass or fail together: m = 2, thresholds alpha / 2 and
    # alpha, so p = 0.02 passes at alpha = 0.02 (rank 2) and fails below it
    tie = [dict(targets=[t(0, 0.02), t(1, 0.02, src=((2, 1),))], n_estimates=0)]
    assert int(merge_network_shards(tie, 3, fdr=True, alpha_fdr=0.02)["adjacency"].sum()) == 2
    assert int(merge_network_shards(tie, 3, fdr=True, alpha_fdr=0.015)["adjacency"].sum()) == 0
    with pytest.raises(ValueError):
        merge_network_shards([dict(targets=[t(0, 0.1)], n_estimates=0)] * 2, 3)
