"""Pins of the oracle's network inference with the linear-Gaussian estimator
(Methods, Vector autoregressive process: the paper's estimator for its VAR
networks): on the 3-node VAR(1) chain the true links are recovered, and the
omnibus transfer entropy of each target agrees with the closed form computed
from the process's true stationary covariance."""
import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import network as onet

# x(t) = A x(t - 1) + e(t), e ~ N(0, I): edges 0 -> 1 and 1 -> 2 at lag 1
A_CHAIN = np.array([[0.4, 0.0, 0.0], [0.3, 0.4, 0.0], [0.0, 0.3, 0.4]])


def _true_cov(A):
    """cov(x_p(t - a), x_q(t - b)) of the stationary VAR(1) process, from
    Gamma_0 = A Gamma_0 A^T + I and Gamma_h = cov(x(t), x(t - h)) = A^h Gamma_0."""
    g0 = scipy.linalg.solve_discrete_lyapunov(A, np.eye(A.shape[0]))

    def cov(u, v):
        (p, a), (q, b) = u, v
        if a <= b:
            return (np.linalg.matrix_power(A, b - a) @ g0)[p, q]
        return (np.linalg.matrix_power(A, a - b) @ g0)[q, p]
    return cov


def _true_cmi(cov, x, y, z):
    """1/2 [ln|S_XZ| + ln|S_YZ| - ln|S_Z| - ln|S_XYZ|] on the true covariance."""
    def ld(vs):
        if not vs:
            return 0.0
        return np.linalg.slogdet(np.array([[cov(u, v) for v in vs] for u in vs]))[1]
    return 0.5 * (ld(x + z) + ld(y + z) - ld(z) - ld(x + y + z))


def test_gauss_network_recovers_chain():
    for seed in (1, 2, 3):
        s = synth.workload_chain3(T=2000, seed=seed)["series"]
        p = onet.Params(max_lag_target=2, max_lag_sources=2, n_surr=100, seed=seed,
                        estimator="gauss")
        adj, res = onet.infer_network(s, p)
        want = np.zeros((3, 3), np.uint8)
        want[0, 1] = want[1, 2] = 1
        np.testing.assert_array_equal(adj, want)
        for r in res:
            assert r.sel_target and r.sel_target[0] == (r.target, 1)
            if r.target > 0:
                assert r.sel_sources == [(r.target - 1, 1)]
                assert r.omnibus_p == 0.0


def test_gauss_omnibus_matches_closed_form():
    # z = (estimate - truth) / sd with the large-sample sd of the plug-in
    # estimate of one partial correlation, sqrt((1 - exp(-2 I)) / N)
    cov = _true_cov(A_CHAIN)
    zs = []
    for seed in range(1, 7):
        s = synth.workload_chain3(T=5000, seed=seed)["series"]
        p = onet.Params(max_lag_target=2, max_lag_sources=2, n_surr=50, seed=seed,
                        estimator="gauss")
        _, res = onet.infer_network(s, p, targets=[1, 2])
        for r in res:
            if len(r.sel_sources) != 1:
                continue
            truth = _true_cmi(cov, r.sel_sources, [(r.target, 0)], r.sel_target)
            assert truth > 0.04
            N = 5000 - 2
            zs.append((r.omnibus_cmi - truth) / np.sqrt((1 - np.exp(-2 * truth)) / N))
    assert len(zs) >= 8
    assert np.max(np.abs(zs)) < 4.0, zs
    assert abs(np.mean(zs)) < 3.0 / np.sqrt(len(zs)), zs


def test_gauss_closed_form_helper_reduces_to_noise_ratio():
    # target 1 given its own past and x_0(t - 1): the residual is the unit
    # noise, so I = 1/2 ln var(x_1(t) | x_1(t - 1))
    cov = _true_cov(A_CHAIN)
    v = cov((1, 0), (1, 0)) - cov((1, 0), (1, 1)) ** 2 / cov((1, 1), (1, 1))
    assert _true_cmi(cov, [(0, 1)], [(1, 0)], [(1, 1)]) == pytest.approx(0.5 * np.log(v),
                                                                           rel=1e-12)


def test_gauss_network_has_no_theiler_window():
    s = synth.workload_chain3(T=300, seed=1)["series"]
    with pytest.raises(ValueError, match="Theiler"):
        onet.infer_network(s, onet.Params(theiler=2, estimator="gauss"))
