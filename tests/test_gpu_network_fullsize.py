"""te_network_infer at the benchmark's full size (T = 10^4, N = 9995, max lag
5, k = 4) against the CPU oracle's greedy loop for one target of each
benchmark workload: the same requests in the same order (stage, iteration,
candidates), every key of every candidate and surrogate of every request,
the selected pasts, the omnibus estimate and p-value, and the estimate count
(Methods, Inference algorithm steps 1-4; Statistical tests, maximum /
minimum statistic and omnibus tests).

The oracle's brute-force run of such a target takes hours, so its trace is
stored by tests/golden/make_network_fullsize.py (which calls only the
oracle): per request the SHA-256 of all keys and the first keys in clear.
The surrogate count is reduced to S = 20 (alpha = 0.1, so S * alpha > 1);
every other size is the benchmark's.  The input series is regenerated from
its seed and checked against the stored hash before anything else.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
CASES = [("var10", 0), ("clm100", 5)]


def _keys_sha(keys):
    flat = ",".join(str(int(k)) for row in keys for k in row)
    return hashlib.sha256(flat.encode()).hexdigest()


@pytest.fixture(scope="module")
def env():
    import paper_1902_06828_gb300 as te
    ctx = te.Context(0)
    yield te, ctx
    ctx.set_trace(None)
    ctx.close()


@pytest.mark.parametrize("workload,target", CASES)
def test_network_target_matches_oracle_trace_at_full_size(env, workload, target):
    te, ctx = env
    path = os.path.join(GOLDEN, f"network_{workload}_T10000_target{target}_S20.json")
    with open(path) as f:
        g = json.load(f)
    gen = {"var10": synth.workload_var10, "clm100": synth.workload_clm100}[workload]
    s = np.ascontiguousarray(gen(T=g["T"], seed=g["seed"])["series"], dtype=np.float32)
    sha = hashlib.sha256(s.tobytes()).hexdigest()
    assert sha == g["series_sha256"], "the input generator gives a different series here"

    trace = []
    ctx.set_trace(lambda *a: trace.append(a))
    data = te.te_data_create(ctx, s)
    try:
        res = te.te_network_infer(ctx, data, targets=[target], **g["params"])
    finally:
        ctx.set_trace(None)
    assert len(trace) == len(g["trace"]), (len(trace), len(g["trace"]))
    for i, ((tg, stage, it, vs, n_cand, n_surr, keys), want) in enumerate(zip(trace, g["trace"])):
        assert tg == target
        assert (stage, it) == (want["stage"], want["iter"]), i
        assert [list(v) for v in vs] == want["cands"], i
        assert n_cand == want["n_cand"] and n_surr == g["params"]["n_surr"], i
        assert [str(k) for k in keys[0][:len(want["keys_head"])]] == want["keys_head"], i
        assert _keys_sha(keys) == want["keys_sha256"], f"request {i}: some key differs"

    r = res["targets"][0]
    w = g["result"]
    assert r["target"] == target
    assert [list(v) for v in r["sel_target"]] == w["sel_target"]
    assert [list(v) for v in r["sel_sources"]] == w["sel_sources"]
    assert r["omnibus_tested"] == w["omnibus_tested"]
    assert r["omnibus_p"] == w["omnibus_p"]
    assert r["omnibus_cmi"] == float.fromhex(w["omnibus_cmi"])
    assert r["significant"] == w["significant"]
    assert r["n_estimates"] == w["n_estimates"] == res["n_estimates"]
