"""Host-side multi-process helpers.

Targets of a network are independent (Supporting Information, Run-time on CPU
and GPU: one computing node per target), so several processes, one per GPU,
split them without exchanging any data on the compute path; only the final
per-target results and timing are gathered on the host.
"""
from __future__ import annotations


def shard_targets(n_proc: int, rank: int, world: int) -> list:
    """Round-robin split of targets 0..n_proc-1 over `world` ranks."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return list(range(rank, n_proc, world))


def combine_timing(dist, times_ms, counts, device="cpu"):
    """Max over ranks of each time and sum over ranks of each count (every
    rank gets the result).  `dist` is torch.distributed or None (one rank)."""
    import torch
    t = torch.tensor([float(v) for v in times_ms], dtype=torch.float64, device=device)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


def gather_results(dist, obj):
    """All ranks' Python objects, in rank order (one rank: [obj])."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


def merge_network_shards(shards, n_proc: int, fdr: bool = False, alpha_fdr: float = 0.05) -> dict:
    """One network from te_network_infer results of disjoint target shards,
    each run with fdr=False (Statistical tests, Combining across multiple
    targets: the FDR step needs every target's omnibus p-value, so it runs
    here, after the gather).  Targets come out in ascending order; with fdr,
    Benjamini-Hochberg over the targets whose omnibus test ran (p-values in
    ascending order, ties in target order; the largest rank r with
    p_(r) <= alpha_fdr r / m and every smaller one rejected), and a target not
    rejected loses its sources.  Then the adjacency [src, tgt] and the
    smallest selected lag per link; seconds is the slowest shard's time."""
    import numpy as np
    targets = sorted((dict(t) for sh in shards for t in sh["targets"]), key=lambda t: t["target"])
    seen = [t["target"] for t in targets]
    if len(set(seen)) != len(seen):
        raise ValueError("a target appears in more than one shard")
    if fdr:
        tested = [t for t in targets if t["omnibus_tested"]]
        order = sorted(range(len(tested)), key=lambda i: tested[i]["omnibus_p"])   # stable
        m = len(tested)
        last = 0
        for r, i in enumerate(order, start=1):
            if tested[i]["omnibus_p"] <= alpha_fdr * r / m:
                last = r
        for r, i in enumerate(order, start=1):
            if r > last:
                tested[i]["sel_sources"] = []
                tested[i]["significant"] = False
    adj = np.zeros((n_proc, n_proc), np.uint8)
    lag = np.zeros((n_proc, n_proc), np.int32)
    for t in targets:
        t["significant"] = bool(t["significant"]) and bool(t["sel_sources"])
        for src, l in t["sel_sources"]:
            adj[src, t["target"]] = 1
            if lag[src, t["target"]] == 0 or l < lag[src, t["target"]]:
                lag[src, t["target"]] = l
    return dict(adjacency=adj, min_lag=lag, targets=targets,
                n_estimates=sum(int(sh["n_estimates"]) for sh in shards),
                seconds=max([float(sh.get("seconds", 0.0)) for sh in shards] or [0.0]),
                theiler=next((sh["theiler"] for sh in shards if "theiler" in sh), None))


def infer_network_sharded(ctx, data, n_proc: int, dist=None, fdr: bool = False,
                          alpha_fdr: float = 0.05, **params) -> dict:
    """te_network_infer with the targets split round-robin over the ranks of
    `dist` (torch.distributed, or None for one process): each rank infers its
    own targets on its own GPU, the per-target results are gathered on the
    host and merged (FDR across all targets included).  Every rank gets the
    whole network."""
    import paper_1902_06828_gb300 as te
    rank = dist.get_rank() if dist is not None and dist.is_initialized() else 0
    world = dist.get_world_size() if dist is not None and dist.is_initialized() else 1
    mine = shard_targets(n_proc, rank, world)
    res = te.te_network_infer(ctx, data, targets=mine, fdr=False, **params) if mine else \
        dict(targets=[], n_estimates=0)
    shard = {k: res[k] for k in ("targets", "n_estimates", "seconds", "theiler") if k in res}
    return merge_network_shards(gather_results(dist, shard), n_proc, fdr, alpha_fdr)
