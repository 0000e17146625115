"""Autotuner of the member-lane KSG kernel's launch shape.

Times every launch shape (points per staged tile 64 / 128 / 256, one or two
members per lane) on batches shaped like the greedy loop's source steps: the
source candidates of target 0 of a seeded 10-node VAR at T = 1000, 3000 and
10000 points, each with its 200 surrogates, conditioned on 0, 1, 2, 4 or 8
variables.  For each bucket (points, conditioning dimensions, and whether
every group has the 64 members that two members per lane need) it keeps the
fastest shape and writes csrc/ksg_tune_table.h, which the library compiles in.
Timing is the KSG kernels' own device time (CUDA events around the launch,
from the context's counters), best of three.

    python -m paper_1902_06828_gb300.tune_ksg --header csrc/ksg_tune_table.h \
        --json timings.json           # tune (needs a GPU)
    python -m paper_1902_06828_gb300.tune_ksg --verify --json verify.json
                                      # the compiled table against every shape

It also times, on the same batches, the persistent-grid and graph-captured
forms (te_ctx_set_option) against the default, for the record.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

TS = (1000, 3000, 10000)
DZS = (0, 1, 2, 4, 8)
N_BUCKETS = (1500, 4500, 1 << 30)        # n_max of the table rows, by T above
DZ_BUCKETS = (0, 1, 3, 7, 1 << 30)        # dz_max of the rows, by DZS above
SHAPES = [(jt, ms) for ms in (2, 1) for jt in (256, 128, 64)]
S = 200


def _z(dz):
    """dz conditioning variables: the target's own lags first, then lag 1 of
    other processes (as the greedy loop accumulates them)."""
    own = [(0, l) for l in range(1, 6)]
    other = [(q, 1) for q in range(1, 10)]
    return (own + other)[:dz]


def _jobs(te, data, dz, wide):
    z = _z(dz)
    used = set(z)
    cands = [(q, l) for q in range(1, 10) for l in range(1, 6) if (q, l) not in used]
    if not wide:                      # one candidate, 20 surrogates: 21 members
        return [te.Job(data, [cands[0]], [(0, 0)], z, k=4, max_lag=5, n_surr=20, seed=3,
                       stream_tag=1)]
    return [te.Job(data, [c], [(0, 0)], z, k=4, max_lag=5, n_surr=S, seed=3, stream_tag=1)
            for c in cands]


def _time(te, ctx, jobs, reps=3):
    best = None
    keys0 = None
    for _ in range(reps):
        s0 = ctx.stats()
        _, keys = te.cmi_ksg_batch(ctx, jobs, return_keys=True)
        s1 = ctx.stats()
        ms = s1["kernel_ms"] - s0["kernel_ms"]
        best = ms if best is None else min(best, ms)
        keys0 = keys0 or keys
        assert keys == keys0
    return best, keys0


def tune(args):
    import paper_1902_06828_gb300 as te
    import synth
    ctx = te.Context(0)
    rows, record = [], []
    for T, nb in zip(TS, N_BUCKETS):
        data = te.te_data_create(ctx, synth.workload_var10(T=T, seed=1)["series"])
        for dz, zb in zip(DZS, DZ_BUCKETS):
            for wide in (True, False):
                jobs = _jobs(te, data, dz, wide)
                _time(te, ctx, jobs, reps=1)              # warm-up
                times, ref = {}, None
                for jt, ms in SHAPES:
                    if ms == 2 and not wide:
                        continue
                    ctx.set_option("ksg_tile", jt)
                    ctx.set_option("ksg_members_per_lane", ms)
                    t, keys = _time(te, ctx, jobs)
                    ref = ref or keys
                    assert keys == ref, "a launch shape changed a key"
                    times[(jt, ms)] = t
                ctx.set_option("ksg_tile", 0)
                ctx.set_option("ksg_members_per_lane", 0)
                best = min(times, key=times.get)
                rows.append((nb, zb, 64 if wide else 0, best[0], best[1]))
                members = sum(j.n_surr + 1 for j in jobs)
                record.append(dict(T=T, dz=dz, members=members,
                                   times_ms={f"jt{jt}_ms{ms}": round(v, 3)
                                             for (jt, ms), v in times.items()},
                                   best=f"jt{best[0]}_ms{best[1]}"))
                print(json.dumps(record[-1]), flush=True)
        data.close()
    # rows: per (n bucket, dz bucket) the >= 64-member row first, then the small one
    lines = ["    {%d, %d, %d, %d, %d}," % r for r in rows]
    hdr = open(os.path.join(HERE, "csrc", "ksg_tune_table.h")).read()
    head = hdr[:hdr.index("static const KsgTuneEntry kKsgTune[] = {")]
    head = head.replace("// default before tuning: 256-point tiles, two members per lane when every\n"
                        "// group has 64 members\n", "")
    body = ("// tuned: T = 1000 / 3000 / 10000 points, conditioning dims 0 / 1 / 2 / 4 / 8,\n"
            "// 45 candidates x 201 members (rows with min_members 64) or 21 members\n"
            "static const KsgTuneEntry kKsgTune[] = {\n" + "\n".join(lines) +
            "\n    {1 << 30, 1 << 30, 0, 256, 1},\n};\n\n}  // namespace teksg\n")
    with open(args.header, "w") as f:
        f.write(head + body)
    if args.json:
        with open(args.json, "w") as f:
            json.dump(record, f, indent=1)


def verify(args):
    """The compiled table's choice against every forced shape, and the
    persistent and graph-captured forms against the default."""
    import paper_1902_06828_gb300 as te
    import synth
    ctx = te.Context(0)
    out = []
    for T in TS:
        data = te.te_data_create(ctx, synth.workload_var10(T=T, seed=1)["series"])
        for dz in DZS:
            for wide in (True, False):
                jobs = _jobs(te, data, dz, wide)
                _time(te, ctx, jobs, reps=1)
                auto, ref = _time(te, ctx, jobs)
                forced = {}
                for jt, ms in SHAPES:
                    if ms == 2 and not wide:
                        continue
                    ctx.set_option("ksg_tile", jt)
                    ctx.set_option("ksg_members_per_lane", ms)
                    forced[f"jt{jt}_ms{ms}"], keys = _time(te, ctx, jobs)
                    assert keys == ref
                ctx.set_option("ksg_tile", 0)
                ctx.set_option("ksg_members_per_lane", 0)
                ctx.set_option("persistent", 1)
                pers, keys = _time(te, ctx, jobs)
                assert keys == ref
                ctx.set_option("persistent", 0)
                best = min(forced.values())
                out.append(dict(T=T, dz=dz, members=sum(j.n_surr + 1 for j in jobs),
                                auto_ms=round(auto, 3), best_forced_ms=round(best, 3),
                                auto_over_best=round(auto / best, 4),
                                persistent_ms=round(pers, 3), forced_ms={
                                    k: round(v, 3) for k, v in forced.items()}))
                print(json.dumps(out[-1]), flush=True)
        data.close()
    # graph capture of whole network inference rounds, wall time per network
    net = []
    for T in (1000, 10000):
        data = te.te_data_create(ctx, synth.workload_var10(T=T, seed=1)["series"])
        kw = dict(k=4, max_lag_target=5, max_lag_sources=5, n_surr=200, seed=1)
        res = {}
        for g in (0, 1):
            ctx.set_option("graph", g)
            r0 = te.te_network_infer(ctx, data, **kw)
            walls = []
            for _ in range(3):
                t = time.perf_counter()
                r = te.te_network_infer(ctx, data, **kw)
                walls.append(time.perf_counter() - t)
                assert np.array_equal(r["adjacency"], r0["adjacency"])
            res[f"graph{g}_s"] = round(min(walls), 4)
        ctx.set_option("graph", 0)
        net.append(dict(T=T, workload="var10 network, all targets", **res,
                        estimates=r0["n_estimates"]))
        print(json.dumps(net[-1]), flush=True)
        data.close()
    if args.json:
        with open(args.json, "w") as f:
            json.dump(dict(shapes=out, graph=net), f, indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--header", default=os.path.join(HERE, "csrc", "ksg_tune_table.h"))
    ap.add_argument("--json", default=None)
    ap.add_argument("--verify", action="store_true")
    args = ap.parse_args()
    (verify if args.verify else tune)(args)


if __name__ == "__main__":
    main()
