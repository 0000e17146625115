"""Host logic of the validation harness: confusion counts, the per-target
false positive rate and its expected range under the complete null, and the
structure of the paper's validation processes."""
import math

import numpy as np

from paper_1902_06828_gb300 import validation as val


def test_scores_hand_example():
    t = np.zeros((3, 3), np.uint8)
    t[0, 1] = t[1, 2] = 1
    f = np.zeros((3, 3), np.uint8)
    f[0, 1] = f[2, 0] = 1
    f[1, 1] = 1                       # diagonal entries are not links
    s = val.scores(t, f)
    assert (s["tp"], s["fp"], s["fn"], s["tn"]) == (1, 1, 1, 3)
    assert s["precision"] == 0.5 and s["recall"] == 0.5 and s["specificity"] == 0.75


def test_scores_empty_denominators():
    z = np.zeros((4, 4), np.uint8)
    s = val.scores(z, z)
    assert s["precision"] is None and s["recall"] is None and s["specificity"] == 1.0


def test_fpr_target_counts_targets_with_any_source():
    a = np.zeros((4, 4), np.uint8)
    a[0, 1] = a[2, 1] = a[3, 2] = 1
    a[3, 3] = 1                       # self entry ignored
    assert val.fpr_target(a) == 0.5   # targets 1 and 2 of 4


def _binom_ppf_by_hand(q, m, p):
    c = 0.0
    for k in range(m + 1):
        c += math.comb(m, k) * p ** k * (1 - p) ** (m - k)
        if c >= q - 1e-12:
            return k
    return m


def test_fpr_expected_range_is_binomial_mean_percentiles():
    for n, alpha, sims in [(4, 0.3, 1), (2, 0.1, 3), (10, 0.05, 5)]:
        m = n * sims
        lo, hi = val.fpr_expected_range(n, alpha, sims)
        assert lo == _binom_ppf_by_hand(0.05, m, alpha) / m
        assert hi == _binom_ppf_by_hand(0.95, m, alpha) / m


def test_paper_couplings_structure():
    import synth
    from synth.generators import _paper_couplings
    rng = np.random.default_rng(4)
    adj, lags, w = _paper_couplings(30, 0.1, rng)
    for t in range(30):
        srcs = np.nonzero(adj[:, t])[0]
        assert adj[t, t] == 0
        if len(srcs):
            assert np.allclose(w[srcs, t], 0.4 / len(srcs))
            assert np.all((lags[srcs, t] >= 1) & (lags[srcs, t] <= 5))
        assert np.all(w[adj[:, t] == 0, t] == 0)
    x, _, _ = synth.var_paper(8, 3000, 2)
    assert np.all(np.isfinite(x)) and np.abs(x).max() < 5       # stable (row sums 0.9)
    x, _, _ = synth.clm_paper(5, 500, 2)
    assert x.min() >= 0.0 and x.max() < 1.0
