"""GPU: the Theiler-window heuristic (autocorrelation decay time) through the
C ABI against the FP64 oracle, and network inference with the automatic
window against the network oracle."""
import numpy as np
import pytest
from scipy.signal import lfilter

import synth
from oracle import network as onet
from oracle import theiler as oth

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


def _series():
    rng = np.random.default_rng(21)
    rows = [lfilter([1.0], [1.0, -phi], rng.normal(size=5000)) for phi in (0.3, 0.6, 0.85, 0.95)]
    t = np.arange(5000)
    rows.append(np.sin(2 * np.pi * t / 50) + 0.05 * rng.normal(size=5000))
    rows.append(np.arange(5000) % 97)            # sawtooth: slow decay
    rows.append(np.full(5000, 1.5))              # constant
    rows.append(rng.normal(size=5000))           # white noise
    return np.ascontiguousarray(np.stack(rows).astype(np.float32))


def _margin_ok(x, tau):
    # the oracle's decision at tau - 1 and tau is far from the threshold, so a
    # different FP64 summation order cannot flip it
    ok = True
    for t in (tau - 1, tau):
        if 1 <= t < len(x):
            ok &= abs(oth.acf(x, t) - oth.INV_E) > 1e-9
    return ok


def test_decay_time_per_process_matches_oracle(te, ctx):
    s = _series()
    data = te.te_data_create(ctx, s)
    for p in range(s.shape[0]):
        want = oth.autocorr_decay_time(s[p])
        assert _margin_ok(s[p], want)
        assert te.te_autocorr_decay(ctx, data, p) == want, p
    assert te.te_autocorr_decay(ctx, data, -1) == oth.theiler_window(s)


def test_decay_time_edge_cases(te, ctx):
    ramp = np.arange(1, 9, dtype=np.float32)[None, :]
    assert te.te_autocorr_decay(ctx, te.te_data_create(ctx, ramp), 0) == 2
    two = np.array([[1.0, 2.0]], np.float32)                  # T = 2: r(1) = -0.5
    assert te.te_autocorr_decay(ctx, te.te_data_create(ctx, two), 0) == 1
    data = te.te_data_create(ctx, _series())
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_autocorr_decay(ctx, data, 8)
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.te_autocorr_decay(ctx, data, -2)


def test_network_with_automatic_window_matches_oracle(te, ctx):
    rng = np.random.default_rng(12)
    s = np.stack([lfilter([1.0], [1.0, -0.7], rng.normal(size=220)) for _ in range(3)])
    s[1, 1:] += 0.8 * s[0, :-1]
    s[2, 1:] += 0.8 * s[1, :-1]
    s = synth.standardise_jitter(s, 12).astype(np.float32)
    kw = dict(k=4, max_lag_target=2, max_lag_sources=2, n_surr=25, alpha_max=0.08,
              alpha_min=0.08, alpha_omnibus=0.08, seed=5)
    data = te.te_data_create(ctx, s)
    g = te.te_network_infer(ctx, data, theiler=-1, **kw)
    adj_o, res_o = onet.infer_network(s, onet.Params(theiler=-1, **kw))
    from tests.test_gpu_parity import _compare_networks
    assert g["theiler"] == oth.theiler_window(s) >= 2
    _compare_networks(g, adj_o, res_o)
