"""GPU: te_network_infer with the linear-Gaussian estimator against the
oracle's network inference with the same estimator.

Test decisions compare estimates, so the network path sums its
cross-covariances in FP64 (differences from the FP64 oracle are rounding
noise, far below 1e-10), and a decision can only differ where the oracle's
own decision is closer than that to a tie.  Each case first checks on the
oracle's trace that every deciding comparison (best against runner-up,
observed against each surrogate statistic) is separated by more than 1e-9;
exact ties (a surrogate whose permutation reproduces the original data) are
equal on both sides.  Then edges, selections, p-values and counts must be
identical and the omnibus estimates equal within 1e-10."""
import numpy as np
import pytest

import synth
from oracle import network as onet

pytestmark = pytest.mark.gpu

MARGIN = 1e-9      # smallest deciding gap the cases must have
TOL = 1e-10        # omnibus estimates, GPU against oracle


@pytest.fixture(scope="module")
def te():
    import paper_1902_06828_gb300 as te
    return te


@pytest.fixture(scope="module")
def ctx(te):
    c = te.Context(0)
    yield c
    c.close()


_margin = onet.decision_margin


def _compare(g, adj_o, res_o):
    np.testing.assert_array_equal(g["adjacency"], adj_o)
    for gt, o in zip(g["targets"], res_o):
        assert gt["target"] == o.target
        assert gt["sel_target"] == [tuple(v) for v in o.sel_target]
        assert gt["sel_sources"] == [tuple(v) for v in o.sel_sources]
        assert gt["omnibus_tested"] == o.omnibus_tested
        assert gt["omnibus_p"] == o.omnibus_p
        assert abs(gt["omnibus_cmi"] - o.omnibus_cmi) <= TOL
        assert gt["significant"] == o.significant
        assert gt["n_estimates"] == o.n_estimates
    assert g["theiler"] == 0


@pytest.mark.parametrize("seed,seq,fdr", [(5, False, False), (7, True, True)])
def test_gauss_network_matches_oracle(te, ctx, seed, seq, fdr):
    x, _adj, _lags = synth.var_er(n=5, p=0.35, T=1500, seed=seed, lo=0.3, hi=0.6, max_lag=3)
    s = synth.standardise_jitter(x, seed)
    kw = dict(max_lag_target=3, max_lag_sources=3, n_surr=50, alpha_max=0.1, alpha_min=0.1,
              alpha_omnibus=0.1, alpha_seq=0.1, seq_test=seq, fdr=fdr, alpha_fdr=0.1, seed=21,
              estimator="gauss")
    adj_o, res_o = onet.infer_network(s, onet.Params(**kw))
    assert _margin(res_o) > MARGIN
    g = te.te_network_infer(ctx, te.te_data_create(ctx, s), **kw)
    _compare(g, adj_o, res_o)
    assert g["n_estimates"] == sum(r.n_estimates for r in res_o)


def test_gauss_network_independent_surrogates_match_oracle(te, ctx):
    x, _adj, _lags = synth.var_er(n=4, p=0.4, T=1200, seed=6, lo=0.3, hi=0.6, max_lag=2)
    s = synth.standardise_jitter(x, 6)
    kw = dict(max_lag_target=2, max_lag_sources=2, n_surr=40, alpha_max=0.1, alpha_min=0.1,
              alpha_omnibus=0.1, alpha_seq=0.1, seq_test=True, seed=13, indep_surr=True,
              estimator="gauss")
    adj_o, res_o = onet.infer_network(s, onet.Params(**kw))
    assert _margin(res_o) > MARGIN
    g = te.te_network_infer(ctx, te.te_data_create(ctx, s), **kw)
    _compare(g, adj_o, res_o)


def _trials(R, T, seed):
    rows = []
    for r in range(R):
        x, _ = synth.var_chain3(T, seed + r, coupling=0.6)
        rows.append(synth.standardise_jitter(x, seed + r))
    return np.ascontiguousarray(np.stack(rows, axis=1).astype(np.float32))   # [3][R][T]


@pytest.mark.parametrize("seed,mode", [(1, "trials"), (2, "within")])
def test_gauss_network_trial_surrogates_match_oracle(te, ctx, seed, mode):
    s3 = _trials(5, 300, seed)
    kw = dict(max_lag_target=2, max_lag_sources=2, n_surr=40, alpha_max=0.1, alpha_min=0.1,
              alpha_omnibus=0.1, seed=seed, estimator="gauss")
    adj_o, res_o = onet.infer_network(s3, onet.Params(**kw), trials=mode)
    assert _margin(res_o) > MARGIN
    data = te.te_data_create_trials(ctx, s3, 2)
    g = te.te_network_infer(ctx, data, surr_mode=mode, **kw)
    _compare(g, adj_o, res_o)


def test_gauss_network_rejects_theiler_window(te, ctx):
    s = synth.workload_chain3(T=300, seed=1)["series"]
    data = te.te_data_create(ctx, s)
    for w in (1, -1):
        with pytest.raises(te.TEError, match="TE_EINVAL"):
            te.te_network_infer(ctx, data, theiler=w, n_surr=40, estimator="gauss")
    # k is not used by the Gaussian estimator
    g = te.te_network_infer(ctx, data, k=0, max_lag_target=2, max_lag_sources=2, n_surr=40,
                            estimator="gauss")
    assert g["adjacency"][1, 2] == 1


def test_gauss_network_full_length_target(te, ctx):
    """var10 at T = 10^4 (N = 9995), all lags up to 5, S = 100: target 3,
    whose closest deciding gap in the oracle is about 3e-8 (a split-TF32
    contraction, ~1e-7, could flip it)."""
    s = synth.workload_var10(T=10000, seed=1)["series"]
    kw = dict(max_lag_target=5, max_lag_sources=5, n_surr=100, alpha_max=0.05,
              alpha_min=0.05, alpha_omnibus=0.05, seed=3, estimator="gauss")
    r = onet.infer_target(s, 3, onet.Params(**kw))
    assert MARGIN < _margin([r]) < 1e-7
    g = te.te_network_infer(ctx, te.te_data_create(ctx, s), targets=[3], **kw)
    gt = g["targets"][0]
    assert gt["sel_target"] == [tuple(v) for v in r.sel_target]
    assert gt["sel_sources"] == [tuple(v) for v in r.sel_sources]
    assert gt["omnibus_p"] == r.omnibus_p
    assert abs(gt["omnibus_cmi"] - r.omnibus_cmi) <= TOL
    assert gt["n_estimates"] == r.n_estimates
