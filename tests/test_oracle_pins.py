"""Pins for the CPU oracle, each against something other than the oracle itself:
hand-worked examples, closed forms, invariants, special cases that reduce to a
textbook routine, published generator outputs and exact rational arithmetic."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy.special import digamma

from oracle import ksg
from oracle import network as onet
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _hand8():
    cases = []
    pts = None
    with open(os.path.join(GOLDEN, "hand8.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("points"):
                pts = np.array([[float(v) for v in p.split(",")] for p in line.split()[1:]])
            elif line.startswith("case"):
                head, *parts = line.split("|")
                _, k, w = head.split()
                arr = [np.array([float(v) for v in p.split()]) for p in parts]
                cases.append((int(k), int(w), arr[0], *(a.astype(int) for a in arr[1:])))
    return pts, cases


def _lag0_series(cols):
    """Each coordinate its own process at lag 0, so point i is time i."""
    return np.ascontiguousarray(np.stack(cols).astype(np.float32))


PTS, CASES = _hand8()


@pytest.mark.parametrize("k,w,eps,nxz,nyz,nz", CASES)
def test_hand_enumerated_8_points(k, w, eps, nxz, nyz, nz):
    s = _lag0_series([PTS[:, 0], PTS[:, 1], PTS[:, 2]])
    r = ksg.cmi_ksg(s, [(0, 0)], [(1, 0)], [(2, 0)], k=k, theiler=w, max_lag=0, per_point=True)
    np.testing.assert_array_equal(r["eps"], eps.astype(np.float32))
    np.testing.assert_array_equal(r["n_xz"], nxz)
    np.testing.assert_array_equal(r["n_yz"], nyz)
    np.testing.assert_array_equal(r["n_z"], nz)
    # the estimate from the hand counts with scipy's digamma
    want = digamma(k) + np.mean(digamma(nz + 1) - digamma(nxz + 1) - digamma(nyz + 1))
    assert abs(r["i_plain"] - want) < 1e-12
    assert abs(r["i_key"] - want) < 1e-12


def test_duplicates_give_zero_eps_and_empty_z_counts_all():
    # x = y = [0, 0, 0, 5], empty Z, k = 1: eps = 0 for the three duplicates
    s = _lag0_series([[0, 0, 0, 5], [0, 0, 0, 5]])
    r = ksg.cmi_ksg(s, [(0, 0)], [(1, 0)], [], k=1, max_lag=0, per_point=True)
    np.testing.assert_array_equal(r["eps"], np.array([0, 0, 0, 5], np.float32))
    np.testing.assert_array_equal(r["n_xz"], [0, 0, 0, 0])
    np.testing.assert_array_equal(r["n_yz"], [0, 0, 0, 0])
    np.testing.assert_array_equal(r["n_z"], [3, 3, 3, 3])


def test_digamma_table_exact_rational():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    n_max = 70000
    q, margin = ksg.digamma_q(n_max)
    # the fixed-point sum carries < n_max units of 2^-100 error, so every entry
    # must sit further than that from a rounding tie
    assert margin > 4 * n_max
    gamma = mpmath.euler
    for n in [1, 2, 3, 4, 5, 7, 10, 100, 999, 1000, 9996, 65537, n_max]:
        h = Fraction(0)
        if n <= 1000:
            for m in range(1, n):
                h += Fraction(1, m)
            psi = mpmath.mpf(h.numerator) / h.denominator - gamma
        else:
            psi = mpmath.digamma(n)
        want = int(mpmath.nint(psi * mpmath.mpf(2) ** 52))
        assert int(q[n]) == want, n
    # plain long-double digamma agrees with scipy to FP64 accuracy
    for n in [1, 2, 5, 17, 1000, 65537]:
        assert abs(ksg.digamma_plain(n) - digamma(n)) < 4e-16 * max(1.0, abs(digamma(n)))


def test_splitmix64_published_outputs():
    # SplitMix64 from state 0 (Steele, Lea & Flood 2014): the widely published
    # first outputs of the reference generator.
    assert ksg.splitmix64_stream(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                           0x06C45D188009454F]
    # the key chain is four generator steps, each from state (previous ^ field)
    G = 0x9E3779B97F4A7C15
    first = ksg.splitmix64_stream(0, 1)[0]
    assert ksg.perm_key(0, 0, 0, 0, 0) == _step(_step(_step(first)))
    assert ksg.perm_key(5, 1, 2, 3, 4) == _step(_step(_step(_step(5 ^ 1) ^ 2) ^ 3) ^ 4)
    assert _step(0) == first and _step(G) == 0x6E789E6AA1B965F4


def _step(x):
    """one output of a generator whose state is x (state advanced once)"""
    return ksg.splitmix64_stream(x, 1)[0]


def test_fisher_yates_uniform_on_four_items():
    from itertools import permutations
    counts = {p: 0 for p in permutations(range(4))}
    n = 24000
    for s in range(n):
        p = tuple(ksg.permutation(7, 3, 2, 1, s, 4))
        counts[p] += 1
    obs = np.array(list(counts.values()))
    chi2 = ((obs - n / 24) ** 2 / (n / 24)).sum()
    assert chi2 < 50.0  # chi^2 with 23 dof: 99.99th percentile ~ 54
    p = ksg.permutation(1, 2, 3, 4, 5, 1000)
    assert sorted(p) == list(range(1000))


def test_empty_z_reduces_to_kraskov_mi():
    """dz = 0: I = psi(k) + psi(N) - <psi(n_x + 1) + psi(n_y + 1)> (Kraskov's I^(1))
    computed here from a numpy distance matrix."""
    x, _ = synth.gaussian_cmi_data(300, 4)
    s = x.astype(np.float32)
    r = ksg.cmi_ksg(s, [(0, 0)], [(1, 0)], [], k=4, max_lag=0, per_point=True)
    a, b = s[0], s[1]
    dxm = np.abs(a[:, None] - a[None, :])
    dym = np.abs(b[:, None] - b[None, :])
    d = np.maximum(dxm, dym)
    N = len(a)
    np.fill_diagonal(d, np.inf)
    eps = np.sort(d, axis=1)[:, 3]
    np.fill_diagonal(dxm, np.inf)
    np.fill_diagonal(dym, np.inf)
    nx = (dxm < eps[:, None]).sum(1)
    ny = (dym < eps[:, None]).sum(1)
    want = digamma(4) + digamma(N) - np.mean(digamma(nx + 1) + digamma(ny + 1))
    np.testing.assert_array_equal(r["n_z"], np.full(N, N - 1))
    assert abs(r["i_plain"] - want) < 1e-12


def _cmi_key(s, x, y, z, **kw):
    return ksg.cmi_ksg(s, x, y, z, **kw)["key"]


def test_symmetry_x_y():
    w = synth.workload_chain3(T=400, seed=3)
    s = w["series"]
    a = _cmi_key(s, w["x"], w["y"], w["z"], k=4, max_lag=2)
    b = _cmi_key(s, w["y"], w["x"], w["z"], k=4, max_lag=2)
    assert a == b


def test_joint_time_permutation_invariance():
    rng = np.random.default_rng(5)
    s = rng.normal(size=(4, 300)).astype(np.float32)
    s[1] += 0.5 * s[0]
    a = _cmi_key(s, [(0, 0)], [(1, 0)], [(2, 0), (3, 0)], k=4, max_lag=0)
    pi = rng.permutation(300)
    b = _cmi_key(np.ascontiguousarray(s[:, pi]), [(0, 0)], [(1, 0)], [(2, 0), (3, 0)], k=4, max_lag=0)
    assert a == b


def test_column_order_and_power_of_two_scale():
    w = synth.workload_chain3(T=400, seed=2)
    s = w["series"]
    a = _cmi_key(s, w["x"], w["y"], w["z"], k=4, max_lag=2)
    b = _cmi_key(s, w["x"], w["y"], w["z"][::-1], k=4, max_lag=2)
    c = _cmi_key(np.ascontiguousarray(s * np.float32(8.0)), w["x"], w["y"], w["z"], k=4, max_lag=2)
    d = _cmi_key(np.ascontiguousarray(s * np.float32(0.25)), w["x"], w["y"], w["z"], k=4, max_lag=2)
    assert a == b == c == d


def test_permutation_pointer_equals_permuted_data():
    """X read through pi (x at point i = x[pi(i)]) equals physically permuting
    the X column; pins the direction of the index."""
    rng = np.random.default_rng(9)
    s = rng.normal(size=(3, 200)).astype(np.float32)
    s[1] += s[0]
    pi = rng.permutation(200).astype(np.int32)
    a = ksg.cmi_ksg(s, [(0, 0)], [(1, 0)], [(2, 0)], k=3, max_lag=0, perm=pi)["key"]
    s2 = s.copy()
    s2[0] = s[0][pi]
    b = ksg.cmi_ksg(s2, [(0, 0)], [(1, 0)], [(2, 0)], k=3, max_lag=0)["key"]
    assert a == b


def test_key_vs_plain_fp64():
    w = synth.workload_chain3(T=600, seed=1)
    for z in (w["z"], [], [(2, 1)]):
        r = ksg.cmi_ksg(w["series"], w["x"], w["y"], z, k=4, max_lag=2)
        assert abs(r["i_key"] - r["i_plain"]) <= 1e-12


def _gauss_cmi_closed(cov):
    def ld(idx):
        return np.linalg.slogdet(cov[np.ix_(idx, idx)])[1]
    return 0.5 * (ld([0, 2]) + ld([1, 2]) - ld([2]) - ld([0, 1, 2]))


def test_gaussian_closed_form():
    vals = []
    cov = None
    for seed in range(12):
        x, cov = synth.gaussian_cmi_data(2000, seed)
        s = x.astype(np.float32)
        vals.append(ksg.cmi_ksg(s, [(0, 0)], [(1, 0)], [(2, 0)], k=4, max_lag=0)["i_key"])
    want = _gauss_cmi_closed(cov)
    m, se = np.mean(vals), np.std(vals, ddof=1) / math.sqrt(len(vals))
    assert abs(m - want) < max(0.02, 3 * se), (m, want, se)


def test_independent_series_near_zero():
    vals = []
    for seed in range(12):
        s = synth.independent(3, 1500, seed).astype(np.float32)
        vals.append(ksg.cmi_ksg(s, [(0, 0)], [(1, 0)], [(2, 0)], k=4, max_lag=0)["i_key"])
    m, se = np.mean(vals), np.std(vals, ddof=1) / math.sqrt(len(vals))
    assert abs(m) < max(3 * se, 0.01), (m, se)


def test_validation_rejects_bad_arguments():
    s = np.zeros((2, 10), np.float32)
    with pytest.raises(ValueError):
        ksg.cmi_ksg(s, [(0, 1)], [(1, 0)], [], k=20, max_lag=1)     # too few neighbours
    with pytest.raises(ValueError):
        ksg.cmi_ksg(s, [(5, 1)], [(1, 0)], [], k=2, max_lag=1)      # bad process
    with pytest.raises(ValueError):
        ksg.cmi_ksg(s, [(0, 3)], [(1, 0)], [], k=2, max_lag=1)      # lag > max lag


# ---- statistical tests ------------------------------------------------------

def test_max_statistic_hand_counted():
    # 3 candidates x (1 + 5 surrogates); null maxima per surrogate:
    # s1: max(1,2,0)=2, s2: max(7,1,1)=7, s3: max(0,0,3)=3, s4: max(2,9,1)=9, s5: max(1,1,1)=1
    keys = [[5, 1, 7, 0, 2, 1], [6, 2, 1, 0, 9, 1], [4, 0, 1, 3, 1, 1]]
    b, p, sig, null = onet.max_statistic_test(keys, alpha=0.5)
    assert b == 1 and null == [2, 7, 3, 9, 1]
    assert p == 2 / 5 and sig          # 7 and 9 exceed 6
    b, p, sig, _ = onet.max_statistic_test(keys, alpha=0.4)
    assert not sig                     # p < alpha is strict


def test_max_statistic_tie_goes_to_first_candidate():
    keys = [[3, 0, 0], [5, 0, 0], [5, 0, 0]]
    b, p, sig, _ = onet.max_statistic_test(keys, alpha=0.6)
    assert b == 1 and p == 0.0


def test_min_statistic_hand_counted():
    # minima per surrogate: s1 min(4,3)=3, s2 min(1,8)=1, s3 min(6,5)=5
    keys = [[2, 4, 1, 6], [7, 3, 8, 5]]
    w, p, sig, null = onet.min_statistic_test(keys, alpha=0.5)
    assert w == 0 and null == [3, 1, 5] and p == 2 / 3 and not sig


def test_max_statistic_fwer_matches_sidak_form():
    """Monte Carlo over i.i.d. continuous nulls: the rate at which one fixed
    null variable beats the empirical (1 - alpha) threshold of the maximum over
    n variables is v_FPR = 1 - (1 - alpha)^(1/n) (Statistical tests, FWER)."""
    rng = np.random.default_rng(11)
    n, S, alpha, trials = 10, 1000, 0.05, 4000
    hits = 0
    for _ in range(trials):
        sur = rng.integers(0, 1 << 40, size=(n, S))
        obs = int(rng.integers(0, 1 << 40))
        keys = [[obs] + [int(v) for v in sur[0]]] + [[-1] + [int(v) for v in sur[c]] for c in range(1, n)]
        _, p, sig, _ = onet.max_statistic_test(keys, alpha)
        hits += sig
    v = 1 - (1 - alpha) ** (1 / n)
    se = math.sqrt(v * (1 - v) / trials)
    assert abs(hits / trials - v) < 4 * se + 1e-3, (hits / trials, v)


def test_fdr_bh_hand():
    # sorted p: 0.001 (r1, thr .0125), 0.01 (r2, .025), 0.03 (r3, .0375), 0.2 (r4, .05)
    assert onet.fdr_bh([0.03, 0.2, 0.001, 0.01], 0.05) == [True, False, True, True]
    assert onet.fdr_bh([0.04, 0.2], 0.05) == [False, False]


def test_greedy_selects_a_planted_lagged_copy():
    rng = np.random.default_rng(3)
    T = 400
    src = rng.normal(size=T)
    tgt = np.zeros(T)
    tgt[2:] = src[:-2]
    tgt += 1e-3 * rng.normal(size=T)
    s = np.stack([tgt, src, rng.normal(size=T)]).astype(np.float32)
    p = onet.Params(n_surr=20, alpha_max=0.1, alpha_min=0.1, alpha_omnibus=0.1,
                    max_lag_target=2, max_lag_sources=3, seed=1)
    r = onet.infer_target(s, 0, p)
    assert (1, 2) in r.sel_sources
    assert all(src_ != 2 for src_, _ in r.sel_sources)
    assert r.omnibus_p == 0.0 and r.significant


@pytest.mark.slow
def test_greedy_recovers_chain():
    # coupling 0.7 so that T = 1000 suffices (the paper needs T ~ 10^4 for
    # the weak couplings of its validation networks)
    w = synth.workload_chain3(T=1000, seed=1, coupling=0.7)
    p = onet.Params(n_surr=40, alpha_max=0.05, alpha_min=0.05, alpha_omnibus=0.05,
                    max_lag_target=2, max_lag_sources=2, seed=3)
    adj, res = onet.infer_network(w["series"], p)
    np.testing.assert_array_equal(adj, w["adj"])
    lags = {(src, r.target): lag for r in res for src, lag in r.sel_sources}
    assert lags == {(0, 1): 1, (1, 2): 1}


# ---- linear-Gaussian estimator ------------------------------------------------

def _resid_var(target, regressors):
    """Residual variance of least squares with an intercept (numpy lstsq)."""
    A = np.column_stack([np.ones(len(target))] + list(regressors))
    coef, *_ = np.linalg.lstsq(A, target, rcond=None)
    r = target - A @ coef
    return float(r @ r)


def test_gauss_equals_regression_residual_identity():
    """For 1-D X and Y: I(X;Y|Z) = 1/2 ln(var(Y | Z) / var(Y | X, Z)), the
    Granger form, computed here by least squares instead of determinants."""
    from oracle import gauss
    w = synth.workload_chain3(T=800, seed=5)
    s = w["series"].astype(np.float64)
    N = s.shape[1] - 2
    Y = s[2, 2:]
    X = s[1, 1:-1]
    Z = [s[2, 1:-1], s[2, 0:-2]]
    want = 0.5 * np.log(_resid_var(Y, Z) / _resid_var(Y, [X] + Z))
    got = gauss.cmi_gauss(w["series"], w["x"], w["y"], w["z"], max_lag=2)[0]
    assert abs(got - want) < 1e-12
    # empty Z: mutual information 1/2 ln(var(Y) / var(Y | X)) = -1/2 ln(1 - r^2)
    r = np.corrcoef(X, Y)[0, 1]
    got0 = gauss.cmi_gauss(w["series"], w["x"], w["y"], [], max_lag=2)[0]
    assert abs(got0 + 0.5 * np.log(1 - r * r)) < 1e-12


def test_gauss_symmetry_affine_and_identity_permutation():
    from oracle import gauss
    w = synth.workload_chain3(T=500, seed=6)
    s = w["series"]
    a = gauss.cmi_gauss(s, w["x"], w["y"], w["z"], max_lag=2)[0]
    b = gauss.cmi_gauss(s, w["y"], w["x"], w["z"], max_lag=2)[0]
    s2 = s.copy()
    s2[1] = s[1] * np.float32(4.0)           # exact in float32
    c = gauss.cmi_gauss(s2, w["x"], w["y"], w["z"], max_lag=2)[0]
    s3 = s.copy()
    s3[1] = s[1] + np.float32(3.0)           # rounds the data at float32 ulp
    e = gauss.cmi_gauss(s3, w["x"], w["y"], w["z"], max_lag=2)[0]
    assert abs(a - e) < 1e-7
    N = s.shape[1] - 2
    d = gauss.cmi_gauss(s, w["x"], w["y"], w["z"], max_lag=2,
                        perms=np.arange(N)[None, :])
    assert abs(a - b) < 1e-12 and abs(a - c) < 1e-12 and abs(d[1] - a) < 1e-15


def test_gauss_population_closed_form():
    from oracle import gauss
    vals = []
    cov = None
    for seed in range(8):
        x, cov = synth.gaussian_cmi_data(20000, seed)
        vals.append(gauss.cmi_gauss(x.astype(np.float32), [(0, 0)], [(1, 0)], [(2, 0)],
                                    max_lag=0)[0])
    want = _gauss_cmi_closed(cov)
    assert abs(np.mean(vals) - want) < 3 * np.std(vals, ddof=1) / math.sqrt(len(vals)) + 2e-4


# ---- Theiler-window heuristic: autocorrelation decay time ---------------------
# (Supporting Information, dynamic correlation exclusion: shortest shift at
# which the autocorrelation drops by 1/e)

from oracle import theiler as oth


def test_inv_e_constant_is_nearest_double():
    import sympy
    exact = sympy.exp(-1).evalf(50)
    assert abs(sympy.Float(oth.INV_E, 50) - exact) <= sympy.Float(2.0 ** -55, 50)


def test_decay_time_linear_ramp_by_hand():
    # x = 1..8: deviations -3.5..3.5, sum of squares 42; lag-1 products sum to
    # 26.25 (r = 0.625 > 1/e), lag-2 products to 11.5 (r = 0.274 <= 1/e)
    x = np.arange(1, 9, dtype=np.float32)
    assert oth.acf(x, 1) == 26.25 / 42
    assert oth.acf(x, 2) == 11.5 / 42
    assert oth.autocorr_decay_time(x) == 2


@pytest.mark.parametrize("phi,tau", [(0.5, 2), (0.8, 5), (0.9, 10)])
def test_decay_time_ar1_closed_form(phi, tau):
    # AR(1) has r(t) = phi^t, so the decay time is the first t with phi^t <= 1/e
    # (every case keeps phi^t at least 0.019 away from 1/e, over 6 standard
    # errors of the sample autocorrelation at T = 10^6)
    from scipy.signal import lfilter
    assert phi ** (tau - 1) > math.exp(-1) + 0.019 and phi ** tau < math.exp(-1) - 0.019
    rng = np.random.default_rng(int(phi * 100))
    x = lfilter([1.0], [1.0, -phi], rng.normal(size=1_000_000))
    assert oth.autocorr_decay_time(x.astype(np.float32)) == tau


def test_decay_time_sine_closed_form():
    # r(t) -> cos(2 pi t / P) for a long sine: first t with cos <= 1/e at P = 50
    # is 10 (cos = 0.309; t = 9 gives 0.426)
    t = np.arange(100_000)
    x = np.sin(2 * np.pi * t / 50).astype(np.float32)
    assert oth.autocorr_decay_time(x) == 10


def test_decay_time_white_noise_and_constant():
    rng = np.random.default_rng(3)
    assert oth.autocorr_decay_time(rng.normal(size=5000).astype(np.float32)) == 1
    assert oth.autocorr_decay_time(np.full(100, 2.5, np.float32)) == 1


def test_theiler_window_is_max_over_processes():
    x = np.stack([np.arange(1, 9), np.arange(8, 0, -1), [1, -1] * 4]).astype(np.float32)
    assert [oth.autocorr_decay_time(r) for r in x] == [2, 2, 1]
    assert oth.theiler_window(x) == 2


def test_network_automatic_theiler_equals_explicit_window():
    # an automatic window is the same run as the explicit largest decay time
    rng = np.random.default_rng(12)
    from scipy.signal import lfilter
    s = np.stack([lfilter([1.0], [1.0, -0.7], rng.normal(size=160)) for _ in range(3)])
    s[1, 1:] += 0.8 * s[0, :-1]
    s = synth.standardise_jitter(s, 12).astype(np.float32)
    w = oth.theiler_window(s)
    assert w >= 2
    kw = dict(k=4, max_lag_target=1, max_lag_sources=1, n_surr=20, alpha_max=0.1,
              alpha_min=0.1, alpha_omnibus=0.1, seed=3)
    auto = onet.infer_network(s, onet.Params(theiler=-1, **kw))
    expl = onet.infer_network(s, onet.Params(theiler=w, **kw))
    assert np.array_equal(auto[0], expl[0])
    assert [r.sel_sources for r in auto[1]] == [r.sel_sources for r in expl[1]]


def test_independent_surrogates_follow_their_definition():
    # with indep_surr, every candidate's surrogate keys are the estimates with
    # the permutation of counter s + c * 2^32, recomputed here one by one
    w = synth.workload_chain3(T=300, seed=4, coupling=0.7)
    s = w["series"]
    kw = dict(k=4, max_lag_target=2, max_lag_sources=1, n_surr=12, alpha_max=0.1,
              alpha_min=0.1, alpha_omnibus=0.1, seed=9)
    r = onet.infer_target(s, 2, onet.Params(indep_surr=True, **kw))
    stage, it, cands, keys, null, pval, sig = r.trace[0]
    assert stage == onet.STAGE_TARGET and len(cands) == 2
    N = s.shape[1] - 2
    for ci, c in enumerate(cands):
        for sidx in (1, 7, 12):
            perm = ksg.permutation(9, 2, onet.STAGE_TARGET, it, sidx + (ci << 32), N)
            o = ksg.cmi_ksg(s, [c], [(2, 0)], [], k=4, max_lag=2, perm=perm)
            assert keys[ci][sidx] == o["key"]
    # candidate 0 keeps the shared permutations; candidate 1 does not
    shared = onet.infer_target(s, 2, onet.Params(**kw)).trace[0][3]
    assert shared[0] == keys[0] and shared[1][0] == keys[1][0] and shared[1] != keys[1]


# ---- replications (trials): pooled embedding and trial surrogates ------------

_M64 = (1 << 64) - 1


def _sm64_py(state):
    """SplitMix64 written out in Python: (new state, output)."""
    state = (state + 0x9E3779B97F4A7C15) & _M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return state, z ^ (z >> 31)


def _fy_py(items, state):
    """Fisher-Yates from the last position down, j = floor(r (i + 1) / 2^64)."""
    a = list(items)
    for i in range(len(a) - 1, 0, -1):
        state, r = _sm64_py(state)
        j = (r * (i + 1)) >> 64
        a[i], a[j] = a[j], a[i]
    return a, state


def test_trial_permutations_follow_their_definition():
    key = ksg.perm_key(11, 2, 1, 0, 5)
    R, n = 6, 9
    # mode 0: the trial order is a Fisher-Yates shuffle of the R trials
    sigma, _ = _fy_py(range(R), key)
    want = [sigma[r] * n + t for r in range(R) for t in range(n)]
    assert ksg.permutation_trials(11, 2, 1, 0, 5, R, n, 0).tolist() == want
    # mode 1: one shuffle per trial, trial 0 first, one continuing generator
    state, want = key, []
    for r in range(R):
        blk, state = _fy_py(range(r * n, (r + 1) * n), state)
        want += blk
    assert ksg.permutation_trials(11, 2, 1, 0, 5, R, n, 1).tolist() == want
    # one trial shuffled inside is the ordinary permutation
    assert np.array_equal(ksg.permutation_trials(11, 2, 1, 0, 5, 1, 40, 1),
                          ksg.permutation(11, 2, 1, 0, 5, 40))


def test_pool_trials_layout_and_single_trial_estimate():
    rng = np.random.default_rng(8)
    s3 = rng.normal(size=(2, 3, 7)).astype(np.float32)
    pooled = ksg.pool_trials(s3, 2)
    assert pooled.shape == (6, 15)
    # row p * 3 + l, point r * 5 + t holds process p of trial r at time 2 + t - l
    for p in range(2):
        for l in range(3):
            for r in range(3):
                for t in range(5):
                    assert pooled[p * 3 + l, r * 5 + t] == s3[p, r, 2 + t - l]
    # one trial: estimates on the pooled view equal the ordinary ones
    w = synth.workload_chain3(T=300, seed=2, coupling=0.7)
    one = w["series"][:, None, :]
    pv = ksg.pool_trials(one, 2)
    m = lambda v: [(p * 3 + l, 0) for p, l in v]
    a = ksg.cmi_ksg(pv, m(w["x"]), m(w["y"]), m(w["z"]), k=4, max_lag=0)
    b = ksg.cmi_ksg(w["series"], w["x"], w["y"], w["z"], k=4, max_lag=2)
    assert a["key"] == b["key"]


def test_network_with_one_trial_equals_ordinary_network():
    w = synth.workload_chain3(T=260, seed=5, coupling=0.7)
    kw = dict(k=4, max_lag_target=2, max_lag_sources=2, n_surr=20, alpha_max=0.1,
              alpha_min=0.1, alpha_omnibus=0.1, seed=4)
    adj1, r1 = onet.infer_network(w["series"], onet.Params(**kw))
    adj2, r2 = onet.infer_network(w["series"][:, None, :], onet.Params(**kw), trials="within")
    assert np.array_equal(adj1, adj2)
    assert [t.trace for t in r1] == [t.trace for t in r2]


def test_surrogate_rank_uniform_under_independence():
    # With X independent of Y and Z, the original and its S surrogates are
    # exchangeable, so cnt = #{surrogate > original} is uniform on 0..S; over
    # 200 seeds a chi-square test (19 dof, 99.99th percentile 52.6) holds.
    S = 19
    counts = np.zeros(S + 1, int)
    for seed in range(200):
        s = synth.independent(3, 260, seed).astype(np.float32)
        N = 259
        perms = np.stack([ksg.permutation(seed, 0, 0, 0, q, N) for q in range(1, S + 1)])
        keys, _, _ = ksg.cmi_ksg_batch(s, [[(0, 1)]] * (S + 1), [(1, 0)], [(2, 1)], perms=perms,
                                       perm_idx=[-1] + list(range(S)), k=4, max_lag=1)
        counts[sum(1 for v in keys[1:] if v > keys[0])] += 1
    exp = 200 / (S + 1)
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 52.6, (chi2, counts.tolist())
