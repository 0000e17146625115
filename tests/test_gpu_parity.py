"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Bar: per-point eps bit-exact, counts exact, 128-bit keys exact, CMI values
identical (both sides evaluate I = Q[k] 2^-52 + K / (2^52 N) from the same
exact key in the same FP64 operation order; the test still states the
1e-9 relative / 1e-12 absolute tolerance the estimate is held to), surrogate
orderings and inferred networks identical.
"""
import os

import numpy as np
import pytest

import synth
from oracle import ksg as oksg
from oracle import network as onet

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
REL, ABS = 1e-9, 1e-12


@pytest.fixture(scope="module")
def te():
    import paper_1902_06828_gb300 as te
    return te


@pytest.fixture(scope="module")
def ctx(te):
    c = te.Context(0)
    yield c
    c.close()


def _close(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= REL * np.abs(b) + ABS)


def _oracle_members(series, x, y, z, k, theiler, max_lag, S, seed, tag):
    T = series.shape[1]
    N = T - max_lag
    perms = (np.stack([oksg.permutation(seed, tag, 0, 0, s, N) for s in range(1, S + 1)])
             if S else None)
    keys, ik, ip = oksg.cmi_ksg_batch(series, [x] * (S + 1), y, z, perms=perms,
                                      perm_idx=[-1] + list(range(S)), k=k, theiler=theiler,
                                      max_lag=max_lag)
    return keys, ik, ip, perms


def test_hand_enumerated_8_points(te, ctx):
    from tests.test_oracle_pins import CASES, PTS
    s = np.ascontiguousarray(PTS.T.astype(np.float32))
    data = te.te_data_create(ctx, s)
    for k, w, eps, nxz, nyz, nz in CASES:
        r = te.cmi_ksg_debug(ctx, data, [(0, 0)], [(1, 0)], [(2, 0)], k=k, theiler=w, max_lag=0)
        np.testing.assert_array_equal(r["eps"], eps.astype(np.float32))
        np.testing.assert_array_equal(r["n_xz"], nxz)
        np.testing.assert_array_equal(r["n_yz"], nyz)
        np.testing.assert_array_equal(r["n_z"], nz)


def test_chain3_config_all_surrogates_bit_exact(te, ctx):
    """3-node VAR(1) chain, T = 1000, target 2, source (1,1), Z = target lags
    1-2, k = 4, 200 surrogates: every key and value equal to the oracle's."""
    w = synth.workload_chain3(T=1000, seed=1)
    data = te.te_data_create(ctx, w["series"])
    S = 200
    cmi, keys = te.cmi_ksg(ctx, data, w["x"], w["y"], w["z"], k=4, max_lag=2, n_surr=S, seed=11,
                           stream_tag=5, return_keys=True)
    ok, ik, ip, perms = _oracle_members(w["series"], w["x"], w["y"], w["z"], 4, 0, 2, S, 11, 5)
    assert keys == ok
    assert np.array_equal(cmi, ik)
    assert _close(cmi, ip)                      # against the plain FP64 sum
    assert np.argsort(keys, kind="stable").tolist() == np.argsort(ok, kind="stable").tolist()
    # per-point eps and counts for the original and two surrogates
    for member in (0, 1, 137):
        g = te.cmi_ksg_debug(ctx, data, w["x"], w["y"], w["z"], member=member, k=4, max_lag=2,
                             n_surr=S, seed=11, stream_tag=5)
        o = oksg.cmi_ksg(w["series"], w["x"], w["y"], w["z"], k=4, max_lag=2,
                         perm=None if member == 0 else perms[member - 1], per_point=True)
        np.testing.assert_array_equal(g["eps"], o["eps"])
        for c in ("n_xz", "n_yz", "n_z"):
            np.testing.assert_array_equal(g[c], o[c])


CASES_SHAPES = [
    # (T, n_proc, x, y, z, k, theiler)   ragged N, every kernel variant
    (257, 4, [(0, 1)], [(1, 0)], [], 4, 0),                                 # empty Z
    (300, 4, [(0, 1)], [(1, 0)], [(1, 1)], 4, 0),
    (513, 5, [(0, 2)], [(1, 0)], [(1, 1), (2, 3), (3, 1), (4, 2)], 4, 3),   # Theiler window
    (400, 4, [(0, 1)], [(1, 0)], [(1, 1), (2, 2)], 1, 0),                   # k = 1 (runtime k)
    (389, 4, [(0, 1)], [(1, 0)], [(1, 2)], 7, 2),                           # k = 7
    (333, 5, [(0, 1), (2, 1), (3, 2)], [(1, 0)], [(1, 1)], 4, 0),           # dx = 3
    (301, 5, [(0, 1), (2, 2)], [(1, 0), (4, 0)], [(1, 1)], 3, 1),           # dx = 2, dy = 2
    (150, 6, [(0, 1)], [(1, 0)], [(p, l) for p in range(1, 6) for l in (1, 2)], 4, 0),  # dz = 10
    # the limits: 32 joint dimensions with the largest k, and k = 16 alone
    (211, 9, [(0, 1)], [(1, 0)], [(p, l) for p in range(1, 9) for l in range(1, 5)][:30], 16, 0),
    (260, 4, [(0, 1)], [(1, 0)], [(1, 1)], 16, 1),
]


@pytest.mark.parametrize("T,n_proc,x,y,z,k,w", CASES_SHAPES)
def test_shapes_and_variants(te, ctx, T, n_proc, x, y, z, k, w):
    rng = np.random.default_rng(T * 7 + n_proc)
    s = rng.normal(size=(n_proc, T))
    s[1, 1:] += 0.6 * s[0, :-1]
    s = synth.standardise_jitter(s, T)
    data = te.te_data_create(ctx, s)
    ml = max(l for _, l in x + y + z)
    S = 9
    cmi, keys = te.cmi_ksg(ctx, data, x, y, z, k=k, theiler=w, max_lag=ml, n_surr=S, seed=3,
                           stream_tag=T, return_keys=True)
    ok, ik, ip, perms = _oracle_members(s, x, y, z, k, w, ml, S, 3, T)
    assert keys == ok
    assert np.array_equal(cmi, ik) and _close(cmi, ip)
    g = te.cmi_ksg_debug(ctx, data, x, y, z, member=4, k=k, theiler=w, max_lag=ml, n_surr=S,
                         seed=3, stream_tag=T)
    o = oksg.cmi_ksg(s, x, y, z, k=k, theiler=w, max_lag=ml, perm=perms[3], per_point=True)
    np.testing.assert_array_equal(g["eps"], o["eps"])
    for c in ("n_xz", "n_yz", "n_z"):
        np.testing.assert_array_equal(g[c], o[c])


CASES_WIDE = [
    # (T, z, theiler)  71 members: two members per lane, second member block ragged
    (301, [], 0),                                   # empty Z (sorted-column counts)
    (389, [(1, 1), (2, 2)], 0),
    (257, [(1, 1)], 3),
]


@pytest.mark.parametrize("T,z,w", CASES_WIDE)
def test_two_members_per_lane(te, ctx, T, z, w):
    """Groups of at least 64 members run two members per lane; keys stay
    bit-exact, including the ragged last member block."""
    rng = np.random.default_rng(T + 17)
    s = rng.normal(size=(3, T))
    s[1, 1:] += 0.5 * s[0, :-1]
    s = synth.standardise_jitter(s, T)
    data = te.te_data_create(ctx, s)
    x, y, S = [(0, 1)], [(1, 0)], 70
    ml = max(l for _, l in x + y + z)
    cmi, keys = te.cmi_ksg(ctx, data, x, y, z, k=4, theiler=w, max_lag=ml, n_surr=S, seed=8,
                           stream_tag=T, return_keys=True)
    ok, ik, ip, perms = _oracle_members(s, x, y, z, 4, w, ml, S, 8, T)
    assert keys == ok
    assert np.array_equal(cmi, ik) and _close(cmi, ip)
    for member in (33, 70):      # second slot of a lane; last (ragged) block
        g = te.cmi_ksg_debug(ctx, data, x, y, z, member=member, k=4, theiler=w, max_lag=ml,
                             n_surr=S, seed=8, stream_tag=T)
        o = oksg.cmi_ksg(s, x, y, z, k=4, theiler=w, max_lag=ml, perm=perms[member - 1],
                         per_point=True)
        for c in ("eps", "n_xz", "n_yz", "n_z"):
            np.testing.assert_array_equal(g[c], o[c])


def test_batch_beyond_grid_limits(te, ctx):
    """330 jobs x 200 surrogates: more composed permutations (66,000) than one
    launch's grid y extent; sampled jobs equal their single calls and the
    oracle."""
    T, S = 120, 200
    rng = np.random.default_rng(5)
    s = synth.standardise_jitter(rng.normal(size=(6, T)), 5)
    data = te.te_data_create(ctx, s)
    y, z = [(0, 0)], [(0, 1), (1, 2)]
    cands = [(p, l) for p in range(1, 6) for l in range(1, 6) if (p, l) != (1, 2)]
    jobs = [te.Job(data, [cands[a % len(cands)]], y, z, k=4, max_lag=5, n_surr=S, seed=4,
                   stream_tag=a) for a in range(330)]
    cmi, keys = te.cmi_ksg_batch(ctx, jobs, return_keys=True)
    for a in (0, 167, 329):
        j = jobs[a]
        one, okeys = te.cmi_ksg(ctx, data, j.x, y, z, k=4, max_lag=5, n_surr=S, seed=4,
                                stream_tag=a, return_keys=True)
        assert keys[a] == okeys
        assert np.array_equal(cmi[a], one)
    ok, _, _, _ = _oracle_members(s, jobs[329].x, y, z, 4, 0, 5, S, 4, 329)
    assert keys[329] == ok


@pytest.mark.parametrize("z", [[], [(2, 1), (2, 3)]])
def test_beyond_the_ordering_limit(te, ctx, z):
    """N = 19997 points (above the 16384 that one ordering CTA sorts): groups
    stay in time order; keys and per-point counts equal the oracle's."""
    rng = np.random.default_rng(19)
    T = 20000
    s = rng.normal(size=(3, T))
    s[2, 1:] += 0.5 * s[1, :-1]
    s = synth.standardise_jitter(s, 19)
    data = te.te_data_create(ctx, s)
    x, y = [(1, 1)], [(2, 0)]
    cmi, keys = te.cmi_ksg(ctx, data, x, y, z, k=4, max_lag=3, n_surr=2, seed=5, stream_tag=1,
                           return_keys=True)
    ok, ik, ip, perms = _oracle_members(s, x, y, z, 4, 0, 3, 2, 5, 1)
    assert keys == ok
    assert np.array_equal(cmi, ik) and _close(cmi, ip)
    g = te.cmi_ksg_debug(ctx, data, x, y, z, member=2, k=4, max_lag=3, n_surr=2, seed=5,
                         stream_tag=1)
    o = oksg.cmi_ksg(s, x, y, z, k=4, max_lag=3, perm=perms[1], per_point=True)
    for c in ("eps", "n_xz", "n_yz", "n_z"):
        np.testing.assert_array_equal(g[c], o[c])


def test_duplicates_and_minimum_size(te, ctx):
    s = np.array([[0, 0, 0, 5, 1, 1], [0, 0, 0, 5, 2, 2]], np.float32)
    data = te.te_data_create(ctx, s)
    g = te.cmi_ksg_debug(ctx, data, [(0, 0)], [(1, 0)], [], k=1, max_lag=0)
    o = oksg.cmi_ksg(s, [(0, 0)], [(1, 0)], [], k=1, max_lag=0, per_point=True)
    for c in ("eps", "n_xz", "n_yz", "n_z"):
        np.testing.assert_array_equal(g[c], o[c])
    # k = N - 1: every other point is a neighbour
    cmi = te.cmi_ksg(ctx, data, [(0, 0)], [(1, 0)], [], k=5, max_lag=0)
    assert cmi[0] == oksg.cmi_ksg(s, [(0, 0)], [(1, 0)], [], k=5, max_lag=0)["i_key"]


def test_batch_equals_single_calls(te, ctx):
    w = synth.workload_var10(T=700, seed=2)
    s = w["series"]
    data = te.te_data_create(ctx, s)
    jobs, singles = [], []
    for a, (x, z) in enumerate([([(0, 1)], [(3, 1)]), ([(2, 3)], [(3, 1)]), ([(4, 2)], []),
                                ([(5, 1), (6, 2)], [(3, 1), (3, 2)]), ([(7, 5)], [(3, 1)])]):
        jobs.append(te.Job(data, x, [(3, 0)], z, k=4, max_lag=5, n_surr=6, seed=9, stream_tag=a))
        singles.append(te.cmi_ksg(ctx, data, x, [(3, 0)], z, k=4, max_lag=5, n_surr=6, seed=9,
                                  stream_tag=a))
    outs = te.cmi_ksg_batch(ctx, jobs)
    for a in range(len(jobs)):
        assert np.array_equal(outs[a], singles[a])
    # and against the oracle for one job with a multi-dim X
    ok, ik, _, _ = _oracle_members(s, [(5, 1), (6, 2)], [(3, 0)], [(3, 1), (3, 2)], 4, 0, 5, 6, 9, 3)
    assert np.array_equal(outs[3], ik)


def test_full_size_sampled_members(te, ctx):
    """T = 10000 (N = 9995) 10-node VAR data, a step-2-shaped group launched
    like the benchmark (45 candidates x 11 members, M = 16 kernel): sampled
    members against the oracle one by one."""
    w = synth.workload_var10(T=10000, seed=1)
    s = w["series"]
    data = te.te_data_create(ctx, s)
    cands = [(q, l) for q in range(10) if q != 0 for l in range(1, 6)]
    S = 10
    jobs = [te.Job(data, [c], [(0, 0)], [(0, 1)], k=4, max_lag=5, n_surr=S, seed=1,
                   stream_tag=0) for c in cands]
    outs, keys = te.cmi_ksg_batch(ctx, jobs, return_keys=True)
    N = 10000 - 5
    perms = np.stack([oksg.permutation(1, 0, 0, 0, s_, N) for s_ in range(1, S + 1)])
    rng = np.random.default_rng(0)
    picks = [(int(c), int(m)) for c, m in zip(rng.integers(0, len(cands), 4),
                                              rng.integers(0, S + 1, 4))] + [(0, 0)]
    for c, m in picks:
        o = oksg.cmi_ksg(s, [cands[c]], [(0, 0)], [(0, 1)], k=4, max_lag=5,
                         perm=None if m == 0 else perms[m - 1])
        assert keys[c][m] == o["key"]
        assert outs[c][m] == o["i_key"]


def test_validation_errors(te, ctx):
    s = np.zeros((2, 10), np.float32)
    data = te.te_data_create(ctx, s)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.cmi_ksg(ctx, data, [(0, 1)], [(1, 0)], [], k=20, max_lag=1)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.cmi_ksg(ctx, data, [(5, 1)], [(1, 0)], [], k=2, max_lag=1)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.cmi_ksg(ctx, data, [(0, 3)], [(1, 0)], [], k=2, max_lag=1)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.cmi_ksg(ctx, data, [(0, 1)], [(1, 0)], [], k=2, max_lag=1, n_surr=-1)
    bad = np.ones((2, 10), np.float32)
    bad[1, 3] = np.nan
    with pytest.raises(te.TEError, match="non-finite"):
        te.te_data_create(ctx, bad)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_network_infer(ctx, data, n_surr=10, alpha_max=0.05)   # S * alpha <= 1
    # 33 joint dimensions, one more than the limit
    wide = te.te_data_create(ctx, np.random.default_rng(1).normal(size=(9, 60)).astype(np.float32))
    z31 = [(p, l) for p in range(1, 9) for l in range(1, 5)][:31]
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.cmi_ksg(ctx, wide, [(0, 1)], [(1, 0)], z31, k=4, max_lag=4)


def test_torch_device_tensor_input(te, ctx):
    torch = pytest.importorskip("torch")
    w = synth.workload_chain3(T=400, seed=4)
    t = torch.from_numpy(w["series"]).cuda()
    d1 = te.te_data_create(ctx, t)
    d2 = te.te_data_create(ctx, w["series"])
    ctx.set_stream(torch.cuda.current_stream())
    a = te.cmi_ksg(ctx, d1, w["x"], w["y"], w["z"], k=4, max_lag=2, n_surr=5)
    ctx.set_stream(None)
    b = te.cmi_ksg(ctx, d2, w["x"], w["y"], w["z"], k=4, max_lag=2, n_surr=5)
    assert np.array_equal(a, b)


def _compare_networks(gpu, adj_o, res_o):
    np.testing.assert_array_equal(gpu["adjacency"], adj_o)
    for g, o in zip(gpu["targets"], res_o):
        assert g["target"] == o.target
        assert g["sel_target"] == [tuple(v) for v in o.sel_target]
        assert g["sel_sources"] == [tuple(v) for v in o.sel_sources]
        assert g["omnibus_tested"] == o.omnibus_tested
        assert g["omnibus_p"] == o.omnibus_p
        assert g["omnibus_cmi"] == o.omnibus_cmi
        assert g["significant"] == o.significant
        assert g["n_estimates"] == o.n_estimates


@pytest.mark.parametrize("seq,fdr", [(False, False), (True, True)])
def test_network_inference_matches_oracle(te, ctx, seq, fdr):
    x, adj, lags = synth.var_er(n=5, p=0.35, T=400, seed=4, lo=0.4, hi=0.7, max_lag=3)
    s = synth.standardise_jitter(x, 4)
    data = te.te_data_create(ctx, s)
    kw = dict(k=4, max_lag_target=3, max_lag_sources=3, n_surr=30, alpha_max=0.1,
              alpha_min=0.1, alpha_omnibus=0.1, alpha_seq=0.1, seq_test=seq, fdr=fdr,
              alpha_fdr=0.1, seed=21)
    g = te.te_network_infer(ctx, data, **kw)
    p = onet.Params(**kw)
    adj_o, res_o = onet.infer_network(s, p)
    _compare_networks(g, adj_o, res_o)
    assert g["n_estimates"] == sum(r.n_estimates for r in res_o)


def test_network_independent_surrogates_match_oracle(te, ctx):
    """Every test draws one permutation set per candidate (counter
    s + c * 2^32); networks, p-values and keys equal the oracle's."""
    x, adj, lags = synth.var_er(n=4, p=0.4, T=350, seed=6, lo=0.4, hi=0.7, max_lag=2)
    s = synth.standardise_jitter(x, 6)
    data = te.te_data_create(ctx, s)
    kw = dict(k=4, max_lag_target=2, max_lag_sources=2, n_surr=30, alpha_max=0.1,
              alpha_min=0.1, alpha_omnibus=0.1, alpha_seq=0.1, seq_test=True, seed=13,
              indep_surr=True)
    g = te.te_network_infer(ctx, data, **kw)
    adj_o, res_o = onet.infer_network(s, onet.Params(**kw))
    _compare_networks(g, adj_o, res_o)
    assert g["n_estimates"] == sum(r.n_estimates for r in res_o)


def test_network_targets_subset(te, ctx):
    w = synth.workload_chain3(T=600, seed=2, coupling=0.7)
    data = te.te_data_create(ctx, w["series"])
    kw = dict(k=4, max_lag_target=2, max_lag_sources=2, n_surr=25, alpha_max=0.08,
              alpha_min=0.08, alpha_omnibus=0.08, seed=5)
    g = te.te_network_infer(ctx, data, targets=[2, 1], **kw)
    res_o = [onet.infer_target(w["series"], t, onet.Params(**kw)) for t in (2, 1)]
    assert [t["target"] for t in g["targets"]] == [2, 1]
    for gt, o in zip(g["targets"], res_o):
        assert gt["sel_sources"] == [tuple(v) for v in o.sel_sources]
        assert gt["omnibus_p"] == o.omnibus_p
