"""Execution options (te_ctx_set_option) change how the work is launched,
never a result: forced tile lengths and members per lane, persistent grids,
batches captured as CUDA graphs and either spatial order of the points give
the same keys and the same network as the default (the tuning table)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import paper_1902_06828_gb300 as te
    ctx = te.Context(0)
    yield te, ctx
    ctx.close()


def _reset(ctx):
    for name in ("ksg_tile", "ksg_members_per_lane", "persistent", "graph", "ksg_order"):
        ctx.set_option(name, 0)


def test_launch_shapes_and_forms_give_identical_keys(env):
    te, ctx = env
    s = synth.workload_var10(T=1500, seed=2)["series"]
    data = te.te_data_create(ctx, s)
    z = [(0, 1), (0, 2)]
    jobs = [te.Job(data, [(q, l)], [(0, 0)], z, k=4, max_lag=5, n_surr=70, seed=9,
                   stream_tag=4) for q in range(1, 4) for l in (1, 3)]
    _reset(ctx)
    _, ref = te.cmi_ksg_batch(ctx, jobs, return_keys=True)
    try:
        for opts in ({"ksg_tile": 64}, {"ksg_tile": 128, "ksg_members_per_lane": 1},
                     {"ksg_tile": 256, "ksg_members_per_lane": 2}, {"persistent": 1},
                     {"graph": 1}, {"persistent": 1, "graph": 1, "ksg_tile": 128}):
            _reset(ctx)
            for name, v in opts.items():
                ctx.set_option(name, v)
            _, keys = te.cmi_ksg_batch(ctx, jobs, return_keys=True)
            assert keys == ref, opts
    finally:
        _reset(ctx)


@pytest.mark.parametrize("z", [[(0, 1)], [(0, 1), (4, 2), (7, 1)],
                               [(0, 1), (0, 2), (1, 3), (2, 1), (5, 4), (8, 2), (9, 1)]])
def test_morton_and_kd_orders_give_identical_keys(env, z):
    """The Morton curve and the k-d tree order prune differently; every key of
    every member agrees between them, and the unpermuted estimates agree with
    the oracle (KSG estimator, Methods; conditioning sets of 1, 3 and 7
    variables)."""
    from oracle import ksg as oksg
    te, ctx = env
    s = np.asarray(synth.workload_var10(T=2000, seed=4)["series"], dtype=np.float32)
    data = te.te_data_create(ctx, s)
    cands = [(q, l) for q in (1, 3, 6) for l in (1, 2, 4) if (q, l) not in z][:7]
    jobs = [te.Job(data, [c], [(0, 0)], z, k=4, max_lag=5, n_surr=40, seed=12,
                   stream_tag=6) for c in cands]
    got = {}
    try:
        for order in (1, 2):
            _reset(ctx)
            ctx.set_option("ksg_order", order)
            _, got[order] = te.cmi_ksg_batch(ctx, jobs, return_keys=True)
    finally:
        _reset(ctx)
    assert got[1] == got[2]
    for c, keys in zip(cands, got[2]):
        o = oksg.cmi_ksg(s, [c], [(0, 0)], z, k=4, max_lag=5)
        assert keys[0] == o["key"], c
    data.close()


@pytest.mark.parametrize("T", [25, 16389])
def test_orders_at_the_sorted_path_limits(env, T):
    """The spatial orders at the smallest and largest group the sorted path
    takes (N = 20 and N = 16384 points, where the k-d tree build fills its
    shared-memory node list): identical keys, originals equal to the oracle."""
    from oracle import ksg as oksg
    te, ctx = env
    s = np.asarray(synth.workload_var10(T=T, seed=6)["series"], dtype=np.float32)
    data = te.te_data_create(ctx, s)
    z = [(0, 1), (2, 1)]
    cands = [(1, 1), (4, 2)]
    jobs = [te.Job(data, [c], [(0, 0)], z, k=4, max_lag=5, n_surr=8, seed=3,
                   stream_tag=2) for c in cands]
    got = {}
    try:
        for order in (1, 2):
            _reset(ctx)
            ctx.set_option("ksg_order", order)
            _, got[order] = te.cmi_ksg_batch(ctx, jobs, return_keys=True)
    finally:
        _reset(ctx)
    assert got[1] == got[2]
    for c, keys in zip(cands, got[2]):
        assert keys[0] == oksg.cmi_ksg(s, [c], [(0, 0)], z, k=4, max_lag=5)["key"], c
    data.close()


def test_network_with_graph_capture_and_persistent_grid(env):
    te, ctx = env
    w = synth.workload_chain3(T=800, seed=3)
    data = te.te_data_create(ctx, w["series"])
    kw = dict(k=4, max_lag_target=2, max_lag_sources=2, n_surr=30, alpha_max=0.1,
              alpha_min=0.1, alpha_omnibus=0.1, seed=5)
    _reset(ctx)
    ref = te.te_network_infer(ctx, data, **kw)
    try:
        ctx.set_option("graph", 1)
        ctx.set_option("persistent", 1)
        got = te.te_network_infer(ctx, data, **kw)
    finally:
        _reset(ctx)
    np.testing.assert_array_equal(got["adjacency"], ref["adjacency"])
    for a, b in zip(got["targets"], ref["targets"]):
        assert a["omnibus_cmi"] == b["omnibus_cmi"] and a["omnibus_p"] == b["omnibus_p"]


def test_bad_options_rejected(env):
    te, ctx = env
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        ctx.set_option("ksg_tile", 96)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        ctx.set_option("graph", 2)
    with pytest.raises(ValueError):
        ctx.set_option("no_such_option", 1)
