"""GPU at the full sizes of the benchmark workloads: step-2-shaped batches at
T = 10^4 (the launch shape the benchmark times: every source candidate of
target 0 x 201 members sharing one conditioning set) checked on sampled
members the oracle computes one by one, every per-point eps and count of one
surrogate, and the greedy chain recovery at T = 10^4."""
import numpy as np
import pytest

import synth
from oracle import ksg as oksg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def te():
    import paper_1902_06828_gb300 as te
    return te


@pytest.fixture(scope="module")
def ctx(te):
    c = te.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("name", ["var10", "clm100"])
def test_fullsize_step2_batch_sampled_members(te, ctx, name):
    w = (synth.workload_var10 if name == "var10" else synth.workload_clm100)(T=10000, seed=1)
    s = w["series"]
    n_proc = s.shape[0]
    data = te.te_data_create(ctx, s)
    z = [(0, 1), (0, 2)]
    cands = [(p, l) for p in range(1, n_proc) for l in range(1, 6)]
    S, tag = 200, 77
    jobs = [te.Job(data, [c], [(0, 0)], z, k=4, max_lag=5, n_surr=S, seed=1, stream_tag=tag)
            for c in cands]
    cmi, keys = te.cmi_ksg_batch(ctx, jobs, return_keys=True)
    assert len(keys) == len(cands) and all(len(k) == S + 1 for k in keys)
    N = s.shape[1] - 5
    rng = np.random.default_rng(len(cands))
    picks = [(0, 0), (len(cands) - 1, S)] + [(int(rng.integers(len(cands))),
                                               int(rng.integers(1, S + 1))) for _ in range(2)]
    for ci, m in picks:
        perm = None if m == 0 else oksg.permutation(1, tag, 0, 0, m, N)
        o = oksg.cmi_ksg(s, [cands[ci]], [(0, 0)], z, k=4, max_lag=5, perm=perm)
        assert keys[ci][m] == o["key"], (name, ci, m)
        assert cmi[ci][m] == o["i_key"]
    ci, m = picks[-1]
    g = te.cmi_ksg_debug(ctx, data, [cands[ci]], [(0, 0)], z, member=m, k=4, max_lag=5,
                         n_surr=S, seed=1, stream_tag=tag)
    o = oksg.cmi_ksg(s, [cands[ci]], [(0, 0)], z, k=4, max_lag=5,
                     perm=oksg.permutation(1, tag, 0, 0, m, N), per_point=True)
    np.testing.assert_array_equal(g["eps"], o["eps"])
    for c in ("n_xz", "n_yz", "n_z"):
        np.testing.assert_array_equal(g[c], o[c])


def test_greedy_recovers_chain_at_full_length(te, ctx):
    # the 3-node chain of the single-estimate workload at T = 10^4: exactly
    # the links 0 -> 1 and 1 -> 2, each at lag 1
    w = synth.workload_chain3(T=10000, seed=1)
    data = te.te_data_create(ctx, w["series"])
    g = te.te_network_infer(ctx, data, k=4, max_lag_target=2, max_lag_sources=2, n_surr=200,
                            alpha_max=0.05, alpha_min=0.05, alpha_omnibus=0.05, seed=3)
    np.testing.assert_array_equal(g["adjacency"], w["adj"])
    lags = {(src, t["target"]): lag for t in g["targets"] for src, lag in t["sel_sources"]}
    assert lags == {(0, 1): 1, (1, 2): 1}
