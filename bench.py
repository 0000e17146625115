"""Benchmark: KSG CMI estimates per second (surrogates included) at T = 10000.

Workload (default "clm100"): 100-node coupled logistic maps (directed ER
graph, expected in-degree 3, lags 1-5, x_i(t) = f(0.5 x_i(t-1) + 0.5 mean_j
x_j(t - d_ji)) + N(0, 0.1^2) mod 1, f(x) = 4x(1-x)), T = 10000 float32
samples, max lag 5, KSG k = 4, 200 surrogates per test, alpha = 0.05.  One
step = the complete greedy inference of one target (te_network_infer with
that target: embeddings, permutations, fused kNN + counts + digamma keys,
test statistics, greedy control), the steps cycling through the targets
(warm-up steps take targets 0 .. W-1, timed steps the next K).  "var10"
instead infers the whole 10-node VAR network per step.

value : estimates / s with the series already resident on the device.
e2e   : the same through the C ABI from a host buffer: each step uploads the
        series (te_data_create from pinned host memory) and reads results back.
Under torchrun each rank infers its own replica data set (seed + rank), no
collective on the data path ("scaling": "weak").

--impl reference times the CPU oracle (brute-force C, all host cores) on a
bounded sample of the same workload: the members of step-2 groups.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "KSG CMI estimates/s incl. surrogates at T=10000"
UNIT = "estimates/s"
TRAFFIC_PER_MEMBER_POINT = (146883584.0 + 4136448.0) / (9045 * 3995)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _workload(name, T, seed):
    import synth
    if name == "var10":
        w = synth.workload_var10(T=T, seed=seed)
        params = dict(k=4, max_lag_target=5, max_lag_sources=5, n_surr=200, alpha_max=0.05,
                      alpha_min=0.05, alpha_omnibus=0.05, seed=seed)
        desc = (f"var10: 10-node VAR, ER p=0.3, T={T}, max lag 5, k=4, S=200, alpha=0.05, "
                "full greedy inference over all targets")
    elif name == "clm100":
        w = synth.workload_clm100(T=T, seed=seed)
        params = dict(k=4, max_lag_target=5, max_lag_sources=5, n_surr=200, alpha_max=0.05,
                      alpha_min=0.05, alpha_omnibus=0.05, seed=seed)
        desc = f"clm100: 100-node coupled logistic maps, T={T}, max lag 5, k=4, S=200"
    else:
        raise SystemExit(f"unknown workload {name}")
    return w["series"], params, desc


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.device)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_sample(series, params, budget_s=20.0, members=None, threads=None):
    """Time the oracle on members of the first step-2 group of target 0
    (Y = target present, Z = its lag-1 past, X = each source candidate,
    identity plus surrogates), all host cores (or `threads` of them)."""
    from oracle import ksg as oksg
    n_proc, T = series.shape
    t0 = max(params["max_lag_target"], params["max_lag_sources"])
    N = T - t0
    cands = [(q, l) for q in range(1, n_proc) for l in range(1, params["max_lag_sources"] + 1)]
    S = 7
    perms = np.stack([oksg.permutation(params["seed"], 0, 2, 0, s, N) for s in range(1, S + 1)])
    threads = threads or oksg.max_threads()
    # calibrate with one member per thread, then size the sample to the budget
    def run(nm):
        xs, pidx = [], []
        for a in range(nm):
            xs.append([cands[a % len(cands)]])
            pidx.append((a % (S + 1)) - 1)
        t = time.perf_counter()
        oksg.cmi_ksg_batch(series, xs, [(0, 0)], [(0, 1)], perms=perms, perm_idx=pidx,
                           k=params["k"], max_lag=t0, n_threads=threads)
        return time.perf_counter() - t
    if members is None:
        dt = run(threads)
        per = dt / threads
        members = max(threads, int(budget_s / max(per, 1e-6)) // threads * threads)
        members = min(members, 40 * threads)
    dt = run(members)
    return {"value": members / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"{members} members (step-2 group of target 0: source candidates x "
                       f"identity/7 surrogates, Z = target lag 1) at N={N}, brute-force C "
                       f"oracle, {threads} OpenMP thread{'s' if threads > 1 else ''}, "
                       f"{dt:.1f} s")}


def plain_path(te, ctx, data, params, calls, stream):
    """The plain path: one cmi_ksg call per estimate (no surrogates batched),
    on a step-2-shaped estimate of target 0 (X = a source candidate, Y = the
    target present, Z = its lag-1 past), timed call by call (host wall clock
    around each blocking call), plus the latency of one request of the
    batched form (the same estimate with its 200 surrogates in one call)."""
    import torch
    n_proc = data.n_proc
    ml = max(params["max_lag_target"], params["max_lag_sources"])
    cands = [(q, l) for q in range(1, n_proc) for l in range(1, params["max_lag_sources"] + 1)]

    def one(c, S):
        t = time.perf_counter()
        te.cmi_ksg(ctx, data, [c], [(0, 0)], [(0, 1)], k=params["k"], max_lag=ml, n_surr=S,
                   seed=params["seed"], stream_tag=7)
        return time.perf_counter() - t

    one(cands[0], 0)
    one(cands[0], 200)
    lat = [one(cands[a % len(cands)], 0) for a in range(calls)]
    req = [one(cands[a % len(cands)], 200) for a in range(max(3, calls // 3))]
    lat_ms = np.array(lat) * 1e3
    req_ms = np.array(req) * 1e3
    return {"value": calls / float(np.sum(lat)), "unit": UNIT, "calls": calls,
            "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
            "request_201_p50_ms": float(np.percentile(req_ms, 50)),
            "request_201_p99_ms": float(np.percentile(req_ms, 99)),
            "request_201_estimates_per_s": 201 * len(req) / float(np.sum(req)),
            "shape": "X=(q,l) candidate, Y=(0,0), Z=(0,1), N=%d, k=%d" % (data.T - ml, params["k"])}


def run_serve(args):
    """Serving workload: requests from independent target loops over mixed
    coupled-logistic-map and VAR data (T in {1000, 3000, 10000}), each a KSG
    CMI job with joint dims 2-30 and 100-1000 surrogates, Poisson arrivals at
    several rates.  Reports per rate p50/p99 latency (submit to completion) and
    estimates/s, and the plain one-call-per-estimate rate on the same mix."""
    import threading

    import torch
    import paper_1902_06828_gb300 as te
    import synth

    torch.cuda.set_device(0)
    rng = np.random.default_rng(7)
    ctx = te.Context(0)
    sets = []
    for kind, T, seed in (("clm", 1000, 1), ("clm", 3000, 2), ("clm", 10000, 3),
                          ("var", 1000, 4), ("var", 3000, 5), ("var", 10000, 6)):
        n = 17
        if kind == "clm":
            x, _, _ = synth.clm_er(n=n, T=T, seed=seed)
        else:
            x, _, _ = synth.var_er(n=n, p=3.0 / 16, T=T, seed=seed)
        sets.append((te.te_data_create(ctx, synth.standardise_jitter(x, seed)), n))

    def request(i):
        d, n = sets[int(rng.integers(len(sets)))]
        tgt = int(rng.integers(n))
        pool = [(tgt, l) for l in range(1, 6)] + [(q, l) for q in range(n) if q != tgt
                                                  for l in range(1, 6)]
        dz = int(rng.integers(0, 29))                 # joint dims 2 .. 30
        idx = rng.permutation(len(pool))
        z = [pool[a] for a in idx[:dz]]
        x = next(pool[a] for a in idx[dz:] if pool[a][0] != tgt)
        return te.Job(d, [x], [(tgt, 0)], z, k=4, max_lag=5,
                      n_surr=int(rng.integers(100, 1001)), seed=7, stream_tag=i)

    te.te_serve_start(ctx, hbm_budget_bytes=16 << 30, max_inflight=2, max_batch_jobs=256)
    # warm-up
    for j in [request(i) for i in range(6)]:
        te.te_serve_poll(ctx, te.te_serve_submit(ctx, j), j.n_surr)
    rates = []
    nreq = args.serve_requests
    for lam in (10.0, 30.0, 100.0, 1000.0, 10000.0):
        reqs = [request(1000 + i) for i in range(nreq)]
        t_sub = [0.0] * nreq
        t_done = [0.0] * nreq
        tickets = [None] * nreq
        ready = threading.Semaphore(0)

        def poller():
            for a in range(nreq):
                ready.acquire()
                te.te_serve_poll(ctx, tickets[a], reqs[a].n_surr)
                t_done[a] = time.perf_counter()

        th = threading.Thread(target=poller)
        th.start()
        t0 = time.perf_counter()
        gaps = rng.exponential(1.0 / lam, nreq)
        due = t0
        for a in range(nreq):
            due += gaps[a]
            while time.perf_counter() < due:
                pass
            t_sub[a] = time.perf_counter()
            tickets[a] = te.te_serve_submit(ctx, reqs[a])
            ready.release()
        th.join()
        lat = (np.array(t_done) - np.array(t_sub)) * 1e3
        est = sum(1 + r.n_surr for r in reqs)
        span = max(t_done) - t0
        rates.append({"rate_per_s": lam, "requests": nreq, "p50_ms": float(np.percentile(lat, 50)),
                      "p99_ms": float(np.percentile(lat, 99)),
                      "estimates_per_s": est / span, "requests_per_s": nreq / span})
    st = te.te_serve_get_stats(ctx)
    te.te_serve_stop(ctx)
    greedy = serve_greedy(te, seconds=args.serve_seconds)
    # plain path on the same mix: one call per estimate, no surrogates batched
    plain = [request(5000 + i) for i in range(max(20, nreq // 4))]
    te.cmi_ksg(ctx, plain[0].data, plain[0].x, plain[0].y, plain[0].z, k=4, max_lag=5)
    t0 = time.perf_counter()
    for j in plain:
        te.cmi_ksg(ctx, j.data, j.x, j.y, j.z, k=4, max_lag=5)
    plain_rate = len(plain) / (time.perf_counter() - t0)
    best = max(r["estimates_per_s"] for r in rates)
    line = {"metric": "serving: KSG CMI estimates/s and p50/p99 request latency under Poisson "
                      "arrivals", "value": best, "unit": UNIT, "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "6 data sets (CLM and VAR, 17 nodes, T in {1000,3000,10000}); "
                                   "requests: joint dims 2-30, S ~ U{100..1000}, k=4",
                       "max_inflight": 2, "max_batch_jobs": 256, "budget_GiB": 16},
            "rates": rates, "plain_path_estimates_per_s": plain_rate,
            "served_over_plain": best / plain_rate, "batches": st["batches"],
            "peak_admitted_bytes": st["peak_bytes"], "greedy_loops": greedy}
    print(json.dumps(line), flush=True)


def serve_greedy(te, seconds=15.0, n_loops=100, plain_calls=40):
    """Serving fed by greedy loops: n_loops concurrent target loops (each one
    target's greedy inference, every test one request of one job per
    candidate with the loop's S surrogates) over 6 data sets of 10 processes
    (coupled logistic maps and VAR, T = 1000, 3000, 10000), S ~ U{100..1000}
    per loop, joint dims growing with the selections, one server.  The loops
    run for `seconds` after a warm-up; the line reports request latency
    (submit of a test's jobs to its last result) and estimates/s over the
    completed requests, and the plain path (one cmi_ksg call per estimate, no
    surrogates) on a sample of the served jobs."""
    import synth
    from paper_1902_06828_gb300.serve_loops import TargetLoop, run_served
    rng = np.random.default_rng(7)
    ctx = te.Context(0)
    sets = []
    for kind, T, seed in (("clm", 1000, 11), ("var", 1000, 12), ("clm", 3000, 13),
                          ("var", 3000, 14), ("clm", 10000, 15), ("var", 10000, 16)):
        x = (synth.clm_er(n=10, T=T, seed=seed)[0] if kind == "clm"
             else synth.var_er(n=10, p=0.3, T=T, seed=seed)[0])
        sets.append((te.te_data_create(ctx, synth.standardise_jitter(x, seed)), kind, T))

    def make(i, tag0):
        d, kind, T = sets[i % len(sets)]
        return TargetLoop(te, d, 10, (i // len(sets)) % 10, n_surr=int(rng.integers(100, 1001)),
                          seed=7, tag_base=tag0 + (i << 20), loop_id=i)

    te.te_serve_start(ctx, hbm_budget_bytes=16 << 30, max_inflight=2, max_batch_jobs=512)
    warm = [make(i, 1 << 41) for i in range(len(sets))]
    for lp in warm:   # one request of every data set
        req = lp.next_request()
        tk = [te.te_serve_submit(ctx, j) for j in req.jobs]
        for t, j in zip(tk, req.jobs):
            te.te_serve_poll(ctx, t, j.n_surr)
    loops = [make(i, 1 << 42) for i in range(n_loops)]
    t0 = time.perf_counter()
    reqs = run_served(te, ctx, loops, deadline_s=seconds)
    span = max(r.t_done for r in reqs) - t0
    st = te.te_serve_get_stats(ctx)
    te.te_serve_stop(ctx)
    lat = np.array([(r.t_done - r.t_submit) * 1e3 for r in reqs])
    est = sum(r.estimates for r in reqs)
    jobs = [j for r in reqs for j in r.jobs]
    pick = [jobs[int(a)] for a in rng.integers(0, len(jobs), plain_calls)]
    te.cmi_ksg(ctx, pick[0].data, pick[0].x, pick[0].y, pick[0].z, k=4, max_lag=5)
    t1 = time.perf_counter()
    for j in pick:
        te.cmi_ksg(ctx, j.data, j.x, j.y, j.z, k=4, max_lag=5)
    plain = plain_calls / (time.perf_counter() - t1)
    served = est / span
    by_stage = {}
    for r in reqs:
        by_stage[r.stage] = by_stage.get(r.stage, 0) + 1
    ctx.close()
    return {"value": served, "unit": UNIT, "loops": n_loops, "seconds": round(span, 2),
            "requests": len(reqs), "requests_by_stage": by_stage, "estimates": est,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "plain_estimates_per_s": plain, "served_over_plain": served / plain,
            "loops_finished": sum(1 for lp in loops if lp.done), "batches": st["batches"],
            "peak_admitted_bytes": st["peak_bytes"],
            "workload": "100 greedy target loops (steps 1-4 of one target each) over 6 data "
                        "sets of 10 processes: CLM and VAR at T = 1000, 3000, 10000; "
                        "S ~ U{100..1000} per loop; every test one request of one job per "
                        "candidate; max_inflight 2, 16 GiB admission budget"}


def run_gauss(args):
    """Linear-Gaussian estimator path on the 100-node VAR shape (ER p = 0.03,
    T = 10^4): cmi_gauss calls of one source candidate against the target
    present given 1..29 conditioning dims, 1000 surrogates each; error of
    sampled results against the FP64 oracle beside the returned bounds."""
    import torch
    import paper_1902_06828_gb300 as te
    import synth
    from oracle import gauss as ogauss
    from oracle import ksg as oksg
    x, _, _ = synth.var_er(n=100, p=0.03, T=args.T, seed=1)
    series = synth.standardise_jitter(x, 1)
    ctx = te.Context(0)
    data = te.te_data_create(ctx, series)
    S, L = 1000, 5
    calls = []
    # joint dims 3, 5, .., 39 and 40 (the Gaussian limit; above 33 the W block
    # takes two 32-column tensor-core passes)
    for a, dz in enumerate(list(range(1, 39, 2)) + [38]):
        z = [(0, l) for l in range(1, 6)][:dz] + [(1 + q, 1 + (q % 5)) for q in range(max(0, dz - 5))]
        calls.append(dict(x=[(60 + a, 1 + a % 5)], y=[(0, 0)], z=z[:dz], tag=a))
    for c in calls[:2]:
        te.cmi_gauss(ctx, data, c["x"], c["y"], c["z"], max_lag=L, n_surr=S, seed=2,
                     stream_tag=c["tag"])
    torch.cuda.synchronize()
    lat = []
    res = []
    t0 = time.perf_counter()
    for c in calls:
        t1 = time.perf_counter()
        res.append(te.cmi_gauss(ctx, data, c["x"], c["y"], c["z"], max_lag=L, n_surr=S, seed=2,
                                stream_tag=c["tag"]))
        lat.append((time.perf_counter() - t1) * 1e3)
    span = time.perf_counter() - t0
    est = len(calls) * (S + 1)
    # FP64 oracle on sampled surrogates of the first and last call
    N = series.shape[1] - L
    errs, bounds = [], []
    for ci in (0, len(calls) - 1):
        c = calls[ci]
        idx = [0, 1, 500, 1000]
        perms = np.stack([oksg.permutation(2, c["tag"], 0, 0, s, N) for s in idx[1:]])
        want = ogauss.cmi_gauss(series, c["x"], c["y"], c["z"], max_lag=L, perms=perms)
        got = res[ci][0][idx]
        errs += list(np.abs(got - want))
        bounds += list(res[ci][1][idx])
    line = {"metric": "linear-Gaussian CMI estimates/s incl. surrogates at T=%d" % args.T,
            "value": est / span, "unit": UNIT, "n_gpus": 1, "higher_is_better": True,
            "dtype": "f64 (tf32-split contraction)", "data": "synthetic",
            "config": {"workload": "100-node VAR (ER p=0.03, T=%d), x = 1 source lag, y = target "
                                   "present, z = 1..38 dims (joint 3..40), 1000 surrogates per "
                                   "call" % args.T,
                       "calls": len(calls)},
            "p50_ms_per_call": float(np.percentile(lat, 50)),
            "p99_ms_per_call": float(np.percentile(lat, 99)),
            "max_abs_err_vs_fp64_oracle": float(max(errs)),
            "max_err_bound_returned": float(max(bounds)),
            "errors_within_bounds": bool(all(e <= b for e, b in zip(errs, bounds)))}
    print(json.dumps(line), flush=True)


def run_gauss_network(args):
    """The workload's full greedy network inference with the linear-Gaussian
    estimator (te_network_infer, estimator "gauss": FP64 contraction, every
    round's estimates in one batched launch per kernel).  Each step is one
    blocking network inference; the rate is estimates per wall second."""
    import torch
    import paper_1902_06828_gb300 as te
    series, params, desc = _workload(args.workload, args.T, 1)
    params = {k: v for k, v in params.items() if k != "k"}
    ctx = te.Context(0)
    data = te.te_data_create(ctx, series)
    for _ in range(args.warmup):
        te.te_network_infer(ctx, data, estimator="gauss", **params)
    torch.cuda.synchronize()
    st0 = ctx.stats()
    n_est, secs = 0, []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        g = te.te_network_infer(ctx, data, estimator="gauss", **params)
        secs.append(time.perf_counter() - t1)
        n_est += g["n_estimates"]
    st1 = ctx.stats()
    line = {"metric": "linear-Gaussian CMI estimates/s incl. surrogates, network inference at "
                      "T=%d" % args.T,
            "value": n_est / sum(secs), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / args.steps,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc.replace("k=4, ", "") + ", Gaussian estimator",
                       "estimates_per_step": n_est / args.steps},
            "gpu_launches_per_step": (st1["launches"] - st0["launches"]) / args.steps,
            "edges": int(g["adjacency"].sum())}
    print(json.dumps(line), flush=True)


def var10_network(te, ctx, stream, T):
    """The whole 10-node VAR network (all targets) once, as an extra figure
    beside the per-target headline: estimates per second of device time."""
    import torch
    series, params, desc = _workload("var10", T, 1)
    data = te.te_data_create(ctx, series)
    te.te_network_infer(ctx, data, **params)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    r = te.te_network_infer(ctx, data, **params)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    data.close()
    return {"value": r["n_estimates"] / (ms / 1e3), "unit": UNIT, "ms": ms,
            "estimates": r["n_estimates"], "workload": desc, "edges": int(r["adjacency"].sum())}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    series, params, desc = _workload(args.workload, args.T, 1)
    from oracle import ksg as oksg
    threads = oksg.max_threads()
    # size one step so that all steps take about two minutes of CPU work (at
    # most 20 s each)
    calib = cpu_oracle_sample(series, params, members=threads)
    per_member = 1.0 / calib["value"]          # seconds per member with all threads busy
    budget = min(20.0, 120.0 / max(args.steps, 1))
    members = max(threads, int(budget / per_member) // threads * threads)
    for _ in range(args.warmup):
        cpu_oracle_sample(series, params, members=threads)
    vals = []
    t_all = 0.0
    n_all = 0
    for _ in range(args.steps):
        r = cpu_oracle_sample(series, params, members=members)
        vals.append(r)
        t_all += members / r["value"]
        n_all += members
    value = n_all / t_all
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": desc, "sample": vals[-1]["sample"]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clm100")
    ap.add_argument("--T", type=int, default=10000)
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--no-extra", dest="extra", action="store_false",
                    help="skip the extra var10 whole-network figure")
    ap.add_argument("--targets", default="all", help="comma list of targets, or 'all'")
    ap.add_argument("--serve", action="store_true",
                    help="run the serving workload instead of the network benchmark")
    ap.add_argument("--serve-requests", type=int, default=80)
    ap.add_argument("--serve-seconds", type=float, default=15.0,
                    help="length of the greedy-loop serving phase (extra key 'serving')")
    ap.add_argument("--gauss", action="store_true",
                    help="linear-Gaussian estimator path (cmi_gauss) instead of the KSG network")
    ap.add_argument("--gauss-network", action="store_true",
                    help="the workload's network inference with the linear-Gaussian estimator")
    ap.add_argument("--plain-calls", type=int, default=30,
                    help="one-call-per-estimate calls timed for the plain-path comparison")
    args = ap.parse_args()

    if args.impl == "reference":
        run_reference(args)
        return
    if args.gauss:
        return run_gauss(args)
    if args.gauss_network:
        return run_gauss_network(args)
    if args.serve:
        run_serve(args)
        return

    import torch
    import paper_1902_06828_gb300 as te

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    series, params, desc = _workload(args.workload, args.T, 1 + rank)
    n_proc = series.shape[0]
    # clm100 (the default): one target per step, cycling through the targets;
    # var10: the whole network per step; --targets: that list every step
    per_target = args.targets == "all" and args.workload == "clm100"
    if args.targets != "all":
        params["targets"] = [int(v) for v in args.targets.split(",")]
        desc += f", targets {args.targets}"

    ctx = te.Context(local)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream)
    data = te.te_data_create(ctx, series)
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    counter = [0]

    def step(d):
        if per_target:
            t = counter[0] % n_proc
            counter[0] += 1
            return te.te_network_infer(ctx, d, targets=[t], **params)
        return te.te_network_infer(ctx, d, **params)

    for _ in range(args.warmup):
        step(data)
    torch.cuda.synchronize()
    first_timed = counter[0]

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    s0 = ctx.stats()
    n_est = 0
    barrier()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    step_est = []
    ev0.record(stream)
    step_ev[0].record(stream)
    for a in range(args.steps):
        if flush is not None:
            flush.fill_(1)
        r = step(data)
        n_est += r["n_estimates"]
        step_est.append(r["n_estimates"])
        step_ev[a + 1].record(stream)
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    s1 = ctx.stats()
    ms = ev0.elapsed_time(ev1)
    if per_target:
        last = counter[0] - 1
        desc += (f"; one step = the complete greedy inference of one target; warm-up targets "
                 f"0-{first_timed - 1}, timed targets {first_timed}-{last} (mod {n_proc})")

    # end to end through the C ABI with host buffers, over the same work as
    # the first e2e_steps timed steps (per target: the same targets again)
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else min(args.steps, 5)
    e2e_steps = min(e2e_steps, args.steps)
    counter[0] = first_timed
    same_ms = sum(step_ev[a].elapsed_time(step_ev[a + 1]) for a in range(e2e_steps))
    same_est = sum(step_est[:e2e_steps])
    host = torch.from_numpy(series).pin_memory()
    e_est = 0
    sb = ctx.stats()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        if flush is not None:
            flush.fill_(1)
        d = te.te_data_create(ctx, host)
        r = step(d)
        e_est += r["n_estimates"]
        d.close()
    e1.record(stream)
    barrier()
    se = ctx.stats()
    e_ms = e0.elapsed_time(e1)

    from paper_1902_06828_gb300.shard import combine_timing
    (ms, e_ms), (n_est, e_est) = combine_timing(dist, [ms, e_ms], [n_est, e_est], device="cuda")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peaks = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    kernel_ms = s1["kernel_ms"] - s0["kernel_ms"]
    pair_evals = s1["pair_evals"] - s0["pair_evals"]
    pair_evals_bf = s1["pair_evals_bruteforce"] - s0["pair_evals_bruteforce"]
    ksg_launches = s1["ksg_launches"] - s0["ksg_launches"]
    ops = s1["ksg_ops"] - s0["ksg_ops"]
    achieved = ops / (kernel_ms / 1e3) / 1e12 if kernel_ms > 0 else None
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    peak = sm_count * 128 * sm_max * 1e6 / 1e12
    # DRAM traffic of the KSG kernel per launch: the ncu capture of the same
    # kernel (var10 at T = 4000, step-2 launch of target 0, 9045 members x 3995
    # points) read 147.02 MB and wrote 4.22 MB, i.e. 4.19 bytes per
    # member-point (each member's X row read once); scaled here by the
    # member-points one launch processes.  Algorithmic bytes: 4 N per member
    # (its X row) + 16 (key).
    n_pts = args.T - 5
    mp_per_launch = (n_est / world) * n_pts / max(ksg_launches, 1)   # this rank's launches
    traffic = TRAFFIC_PER_MEMBER_POINT * mp_per_launch if ksg_launches else None
    alg_bytes = (4.0 * n_pts + 16.0) * (n_est / world) / max(ksg_launches, 1)
    value = n_est / (ms / 1e3)
    # measured ceiling of the counted instruction mix (te_alu_peak, after the
    # timed region): the kNN-pass and count-pass patterns run from registers,
    # weighted by this run's counted ops (pair_evals = e1 + e2 and
    # ksg_ops = 3 e1 + 7 e2 give the two passes' shares)
    p_knn = te.te_alu_peak(ctx, "knn") / 1e12
    p_cnt = te.te_alu_peak(ctx, "count") / 1e12
    p_add = te.te_alu_peak(ctx, "fadd") / 1e12
    e2 = (ops - 3.0 * pair_evals) / 4.0
    ops1, ops2 = 3.0 * (pair_evals - e2), 7.0 * e2
    peak_mix = (ops1 + ops2) / (ops1 / p_knn + ops2 / p_cnt) if ops > 0 else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "estimates_per_step": n_est / args.steps / world,
                   "l2": "flushed before every step (256 MB write)" if flush is not None
                   else "not flushed", "parallelism": f"replicas{world}"},
        "e2e": {"value": e_est / (e_ms / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": (se["h2d_bytes"] - sb["h2d_bytes"]) / max(e2e_steps, 1),
                "d2h_bytes_per_step": (se["d2h_bytes"] - sb["d2h_bytes"]) / max(e2e_steps, 1),
                "steps": e2e_steps,
                "device_resident_same_steps": (same_est / (same_ms / 1e3)) if same_ms > 0
                else None,
                "note": "the work of the first timed steps again (same targets), each step "
                        "uploading the series from pinned host memory"},
        "gpu_launches": s1["launches"] - s0["launches"],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_note": "dram read+write bytes per launch, scaled from the ncu "
                                     "capture of this kernel at T=4000 by member-points",
                     "algorithmic_bytes_per_launch": alg_bytes,
                     "kernel": "ksg_lane_kernel", "kernel_ms_per_launch":
                     kernel_ms / max(ksg_launches, 1), "launches": ksg_launches,
                     "peak_note": f"{sm_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz "
                                  "(derived; SM count read from the device)",
                     "peak_measured_mix": peak_mix,
                     "frac_of_measured_mix": (achieved / peak_mix) if achieved and peak_mix
                     else None,
                     "peak_measured": {"knn_pass_pattern": p_knn, "count_pass_pattern": p_cnt,
                                       "fp32_add_issue": p_add,
                                       "count_pass_share_of_ops": (ops2 / ops) if ops else None,
                                       "note": "te_alu_peak: each pass's counted instruction "
                                               "pattern from registers at full occupancy, this "
                                               "run; the mix weights them by this run's ops"},
                     "work": "3 ops per executed kNN-pass member-pair, 7 per count-pass one",
                     "pair_evals_executed": pair_evals, "pair_evals_bruteforce": pair_evals_bf,
                     "pruned_fraction": (1.0 - pair_evals / pair_evals_bf) if pair_evals_bf
                     else None},
        "clocks": clk,
    }
    if args.plain_calls > 0:
        line["plain_path"] = plain_path(te, ctx, data, params, args.plain_calls, stream)
        line["plain_path"]["batched_over_plain"] = value / line["plain_path"]["value"]
    if args.extra and args.workload != "var10" and world == 1:
        line["var10_network"] = var10_network(te, ctx, stream, args.T)
    if args.extra and world == 1:
        line["serving"] = serve_greedy(te, seconds=args.serve_seconds)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_oracle_sample(series, params)
        one = cpu_oracle_sample(series, params, members=3, threads=1)
        line["cpu_baseline"]["one_core"] = {"value": one["value"], "sample": one["sample"]}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
