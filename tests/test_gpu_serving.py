"""Serving (continuous batching): results in the mix equal results alone.

Jobs of uneven shape (three data sets of different T, joint dims 2-8,
different surrogate counts and k) are submitted from several host threads
while batches run; each job's keys must equal the same job run alone through
cmi_ksg, bit for bit, and its values within the parity tolerance."""
import threading

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
REL, ABS = 1e-9, 1e-12


@pytest.fixture(scope="module")
def env():
    import paper_1902_06828_gb300 as te
    ctx = te.Context(0)
    yield te, ctx
    ctx.close()


def _jobs(te, ctx, rng):
    sets = []
    for T, seed in ((600, 1), (1100, 2), (1700, 3)):
        x, _, _ = synth.var_er(n=6, p=0.4, T=T, seed=seed, max_lag=3)
        sets.append(te.te_data_create(ctx, synth.standardise_jitter(x, seed)))
    jobs = []
    for a in range(36):
        d = sets[a % 3]
        tgt = int(rng.integers(0, 6))
        src = [(int(q), int(l)) for q, l in zip(rng.integers(0, 6, 2), rng.integers(1, 4, 2))]
        x = src[:1] if a % 5 else src
        z = [(tgt, l) for l in range(1, int(rng.integers(1, 4)) + 1)]
        if a % 7 == 0:
            z = []
        jobs.append(te.Job(d, x, [(tgt, 0)], z, k=4 if a % 4 else 3, max_lag=3,
                           n_surr=int(rng.choice([0, 9, 40, 120])), seed=5, stream_tag=a))
    return jobs


def test_mixed_jobs_equal_alone(env):
    te, ctx = env
    rng = np.random.default_rng(0)
    jobs = _jobs(te, ctx, rng)
    alone = [te.cmi_ksg(ctx, j.data, j.x, j.y, j.z, k=j.k, max_lag=j.max_lag, n_surr=j.n_surr,
                        seed=j.seed, stream_tag=j.stream_tag, return_keys=True) for j in jobs]
    te.te_serve_start(ctx, max_inflight=2, max_batch_jobs=5)
    results = [None] * len(jobs)

    def worker(idx):
        for a in idx:
            t = te.te_serve_submit(ctx, jobs[a])
            results[a] = te.te_serve_poll(ctx, t, jobs[a].n_surr, return_keys=True)

    threads = [threading.Thread(target=worker, args=(list(range(w, len(jobs), 4)),))
               for w in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    st = te.te_serve_get_stats(ctx)
    assert st["completed"] == len(jobs) and st["batches"] >= 2
    for (ref, rkeys), (got, gkeys) in zip(alone, results):
        assert gkeys == rkeys
        assert np.all(np.abs(got - ref) <= REL * np.abs(ref) + ABS)
    # submit everything at once, then poll in reverse order
    tickets = [te.te_serve_submit(ctx, j) for j in jobs]
    for a in reversed(range(len(jobs))):
        got, gkeys = te.te_serve_poll(ctx, tickets[a], jobs[a].n_surr, return_keys=True)
        assert gkeys == alone[a][1]
    te.te_serve_stop(ctx)


def test_cancel_budget_and_timeout(env):
    te, ctx = env
    w = synth.workload_var10(T=10000, seed=3)
    d = te.te_data_create(ctx, w["series"])
    te.te_serve_start(ctx, hbm_budget_bytes=256 << 20, max_inflight=1, max_batch_jobs=1)
    big = te.Job(d, [(1, 1)], [(0, 0)], [(0, 1)], k=4, max_lag=5, n_surr=400, seed=1)
    huge = te.Job(d, [(1, 1)], [(0, 0)], [(0, 1)], k=4, max_lag=5, n_surr=4000, seed=1)
    with pytest.raises(te.TEError, match="TE_EBUSY"):
        te.te_serve_submit(ctx, huge)          # about 12 S N bytes > 256 MiB
    t1 = te.te_serve_submit(ctx, big)
    t2 = te.te_serve_submit(ctx, big)          # waits behind t1 (one job per batch)
    te.te_serve_cancel(ctx, t2)
    with pytest.raises(te.TEError, match="TE_ECANCELLED"):
        te.te_serve_poll(ctx, t2, 400)
    with pytest.raises(te.TEError, match="TE_ETIMEOUT"):
        te.te_serve_poll(ctx, t1, 400, timeout_ms=0)
    got = te.te_serve_poll(ctx, t1, 400)
    ref = te.cmi_ksg(ctx, d, [(1, 1)], [(0, 0)], [(0, 1)], k=4, max_lag=5, n_surr=400, seed=1)
    assert np.array_equal(got, ref)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_serve_poll(ctx, t1, 400)         # released
    te.te_serve_stop(ctx)


def test_greedy_loops_served_equal_direct_and_oracle():
    """Six greedy target loops (steps 1-4 of one target each, every test one
    request of one job per candidate) run concurrently against one server;
    each loop takes exactly the requests and decisions of the same loop whose
    tests run directly through cmi_ksg_batch, every key equal, and sampled
    served jobs equal the CPU oracle's keys (permutations drawn from the
    jobs' seed and stream tag)."""
    import paper_1902_06828_gb300 as te
    from oracle import ksg as oksg
    from paper_1902_06828_gb300.serve_loops import TargetLoop, run_served
    ctx = te.Context(0)
    sets = []
    for kind, T, seed in (("clm", 500, 3), ("var", 700, 4)):
        x = (synth.clm_er(n=4, T=T, seed=seed, max_lag=3)[0] if kind == "clm"
             else synth.var_er(n=4, p=0.5, T=T, seed=seed, lo=0.4, hi=0.7, max_lag=3)[0])
        s = synth.standardise_jitter(x, seed)
        sets.append((te.te_data_create(ctx, s), s))

    def loops():
        return [TargetLoop(te, sets[i % 2][0], 4, i // 2, n_surr=30 + 10 * i, alpha=0.1,
                           max_lag=3, seed=5, tag_base=1000 * (i + 1), loop_id=i)
                for i in range(6)]

    lk = threading.Lock()   # a context serves one thread at a time

    def direct_eval(r):
        with lk:
            return te.cmi_ksg_batch(ctx, r.jobs, return_keys=True)[1]

    direct_loops = loops()
    direct = run_served(te, ctx, direct_loops, evaluate=direct_eval)
    te.te_serve_start(ctx, hbm_budget_bytes=1 << 30, max_inflight=2, max_batch_jobs=64)
    try:
        served_loops = loops()
        served = run_served(te, ctx, served_loops)
    finally:
        te.te_serve_stop(ctx)
    assert all(lp.done for lp in served_loops)
    key = lambda r: (r.loop, r.stage, r.it)
    d_by = {key(r): r for r in direct}
    assert sorted(d_by) == sorted(key(r) for r in served)
    for r in served:
        assert r.keys == d_by[key(r)].keys, key(r)
    for a, b in zip(served_loops, direct_loops):
        assert a.result() == b.result()
    assert any(r.stage == 2 for r in served) and any(lp.sel_x for lp in served_loops)
    # the oracle on a sample of served jobs
    rng = np.random.default_rng(2)
    jobs = [(j, r.keys[a]) for r in served for a, j in enumerate(r.jobs)]
    for i in rng.choice(len(jobs), 8, replace=False):
        j, got = jobs[int(i)]
        s = sets[0][1] if j.data is sets[0][0] else sets[1][1]
        N = s.shape[1] - j.max_lag
        perms = np.stack([oksg.permutation(j.seed, j.stream_tag, 0, 0, q, N)
                          for q in range(1, j.n_surr + 1)])
        want, _, _ = oksg.cmi_ksg_batch(s, [j.x] * (j.n_surr + 1), j.y, j.z, perms=perms,
                                        perm_idx=[-1] + list(range(j.n_surr)), k=j.k,
                                        max_lag=j.max_lag)
        assert got == want
    ctx.close()
