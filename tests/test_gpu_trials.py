"""GPU: replications (trials) pooled by te_data_create_trials and network
inference with trial surrogates, against the oracle's pooling and network."""
import numpy as np
import pytest

import synth
from oracle import ksg as oksg
from oracle import network as onet

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


def _trials(R, T, seed):
    rows = []
    for r in range(R):
        x, _ = synth.var_chain3(T, seed + r, coupling=0.6)
        rows.append(synth.standardise_jitter(x, seed + r))
    return np.ascontiguousarray(np.stack(rows, axis=1).astype(np.float32))   # [3][R][T]


def test_pooled_estimates_match_oracle(te, ctx):
    s3 = _trials(4, 90, 3)
    L = 2
    data = te.te_data_create_trials(ctx, s3, L)
    pooled = oksg.pool_trials(s3, L)
    assert (data.n_proc, data.T) == pooled.shape
    m = lambda v: [te.trial_var(p, l, L) for p, l in v]
    x, y, z = [(1, 1)], [(2, 0)], [(2, 1), (2, 2)]
    cmi, keys = te.cmi_ksg(ctx, data, m(x), m(y), m(z), k=4, max_lag=0, n_surr=5, seed=2,
                           stream_tag=7, return_keys=True)
    N = pooled.shape[1]
    perms = np.stack([oksg.permutation(2, 7, 0, 0, s, N) for s in range(1, 6)])
    ok, _, _ = oksg.cmi_ksg_batch(pooled, [m(x)] * 6, m(y), m(z), perms=perms,
                                  perm_idx=[-1] + list(range(5)), k=4, max_lag=0)
    assert keys == ok


@pytest.mark.parametrize("mode,R", [("trials", 6), ("within", 4), ("auto", 3), ("auto", 5)])
def test_network_with_trial_surrogates_matches_oracle(te, ctx, mode, R):
    from tests.test_gpu_parity import _compare_networks
    s3 = _trials(R, 110, 10 + R)
    kw = dict(k=4, max_lag_target=2, max_lag_sources=2, n_surr=30, alpha_max=0.1,
              alpha_min=0.1, alpha_omnibus=0.1, seed=6)
    data = te.te_data_create_trials(ctx, s3, 2)
    g = te.te_network_infer(ctx, data, surr_mode=mode, **kw)
    adj_o, res_o = onet.infer_network(s3, onet.Params(**kw), trials=mode)
    _compare_networks(g, adj_o, res_o)


def test_trial_data_rejects_window_and_lag_mismatch(te, ctx):
    data = te.te_data_create_trials(ctx, _trials(3, 60, 1), 2)
    kw = dict(k=4, max_lag_target=2, max_lag_sources=2, n_surr=30, alpha_max=0.1,
              alpha_min=0.1, alpha_omnibus=0.1)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_network_infer(ctx, data, theiler=1, **kw)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_network_infer(ctx, data, **dict(kw, max_lag_sources=3))
