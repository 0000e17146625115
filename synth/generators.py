"""Seeded synthetic workloads shaped like the paper's validation data.

* Vector autoregressive process (Methods, Validation tasks, "Vector
  autoregressive process"): Y_t = beta Y_{t-1} + sum_X alpha_X X_{t-l_X} + eta_t.
* Coupled logistic maps (Methods, Validation tasks, "Coupled logistic maps
  process"): a_t = beta Y_{t-1} + sum_X alpha_X X_{t-l_X},
  Y_t = (4 a_t (1 - a_t) + eta_t) mod 1.
* Directed Erdos-Renyi graphs (Methods, Validation tasks: link probability
  chosen for an expected in-degree).

All generators use numpy's PCG64 through default_rng(seed), so a seed gives the
same float32 array on x86_64 and aarch64.  `standardise_jitter` is the fixture
preprocessing (per-process z-score in float64 with ddof=0, plus N(0, 1e-8)
jitter, cast to float32); it happens before either the oracle or the CUDA
library sees the data.
"""
from __future__ import annotations

import numpy as np

__all__ = ["er_graph", "var_chain3", "var_er", "clm_er", "standardise_jitter", "independent",
           "gaussian_cmi_data", "workload_chain3", "workload_var10", "workload_clm100",
           "var_paper", "clm_paper"]


def er_graph(n: int, p: float, rng) -> np.ndarray:
    """adj[src, tgt] = 1 with probability p, no self loops."""
    a = (rng.random((n, n)) < p).astype(np.uint8)
    np.fill_diagonal(a, 0)
    return a


def standardise_jitter(x: np.ndarray, seed: int, sigma: float = 1e-8) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    mu = x.mean(axis=1, keepdims=True)
    sd = x.std(axis=1, keepdims=True)
    sd[sd == 0] = 1.0
    z = (x - mu) / sd
    rng = np.random.default_rng(seed + 0x5EED)
    z = z + rng.normal(0.0, sigma, size=z.shape)
    return np.ascontiguousarray(z.astype(np.float32))


def _simulate_var(coef: np.ndarray, T: int, noise_sd: float, rng, burn: int = 1000) -> np.ndarray:
    """coef[l-1, i, j] = weight of x_j(t - l) in x_i(t)."""
    L, n, _ = coef.shape
    total = T + burn
    x = np.zeros((total, n))
    eta = rng.normal(0.0, noise_sd, size=(total, n))
    for t in range(total):
        acc = eta[t].copy()
        for l in range(1, L + 1):
            if t - l >= 0:
                acc += coef[l - 1] @ x[t - l]
        x[t] = acc
    return x[burn:].T.copy()


def spectral_radius(coef: np.ndarray) -> float:
    L, n, _ = coef.shape
    comp = np.zeros((L * n, L * n))
    for l in range(L):
        comp[:n, l * n:(l + 1) * n] = coef[l]
    if L > 1:
        comp[n:, :-n] = np.eye((L - 1) * n)
    return float(np.max(np.abs(np.linalg.eigvals(comp))))


def var_chain3(T: int = 1000, seed: int = 1, coupling: float = 0.3):
    """3-node VAR(1): x_i(t) = 0.4 x_i(t-1) + sum_{j->i} c x_j(t-1) + N(0,1),
    c = 0.3 by default, edges 0->1 and 1->2.  Returns (float64 [3][T], adjacency)."""
    rng = np.random.default_rng(seed)
    c = coupling
    A = np.array([[0.4, 0.0, 0.0], [c, 0.4, 0.0], [0.0, c, 0.4]])
    x = _simulate_var(A[None], T, 1.0, rng)
    adj = np.zeros((3, 3), np.uint8)
    adj[0, 1] = adj[1, 2] = 1
    return x, adj


def var_er(n: int = 10, p: float = 0.3, T: int = 10000, seed: int = 1, self_coupling: float = 0.5,
           lo: float = 0.1, hi: float = 0.5, max_lag: int = 5, radius: float = 0.9,
           noise_sd: float = 1.0):
    """VAR with a directed ER graph: self coupling at lag 1, each edge a
    U(lo, hi) weight at a random lag in 1..max_lag; the lag-l coefficients are
    scaled by c^l so that the companion matrix has the requested spectral
    radius.  Returns (float64 [n][T], adjacency, lags[src, tgt] (0 = none))."""
    rng = np.random.default_rng(seed)
    adj = er_graph(n, p, rng)
    coef = np.zeros((max_lag, n, n))
    lags = np.zeros((n, n), np.int32)
    for i in range(n):
        coef[0, i, i] = self_coupling
    for s in range(n):
        for t in range(n):
            if adj[s, t]:
                l = int(rng.integers(1, max_lag + 1))
                lags[s, t] = l
                coef[l - 1, t, s] = rng.uniform(lo, hi)
    rho = spectral_radius(coef)
    if rho > 0:
        c = radius / rho
        for l in range(max_lag):
            coef[l] *= c ** (l + 1)
    x = _simulate_var(coef, T, noise_sd, rng)
    return x, adj, lags


def clm_er(n: int = 100, T: int = 10000, seed: int = 1, p: float | None = None, max_lag: int = 5,
           self_w: float = 0.5, noise_sd: float = 0.1, burn: int = 1000):
    """Coupled logistic maps: x_i(t) = f(0.5 x_i(t-1) + 0.5 mean_j x_j(t - d_ji))
    + N(0, noise_sd^2), mod 1, with f(x) = 4x(1-x).  A node without in-links
    gets an empty mean = 0.  Returns (float64 [n][T], adjacency, lags)."""
    rng = np.random.default_rng(seed)
    if p is None:
        p = 3.0 / (n - 1)
    adj = er_graph(n, p, rng)
    lags = np.zeros((n, n), np.int32)
    for s in range(n):
        for t in range(n):
            if adj[s, t]:
                lags[s, t] = int(rng.integers(1, max_lag + 1))
    total = T + burn
    x = np.zeros((total, n))
    x[:max_lag] = rng.random((max_lag, n))
    eta = rng.normal(0.0, noise_sd, size=(total, n))
    srcs = [np.nonzero(adj[:, t])[0] for t in range(n)]
    for t in range(max_lag, total):
        for i in range(n):
            a = self_w * x[t - 1, i]
            if len(srcs[i]):
                m = np.mean([x[t - lags[s, i], s] for s in srcs[i]])
                a += (1.0 - self_w) * m
            v = 4.0 * a * (1.0 - a) + eta[t, i]
            x[t, i] = v - np.floor(v)
    return x[burn:].T.copy(), adj, lags


def _paper_couplings(n: int, p: float, rng, max_lag: int = 5, total: float = 0.4):
    """ER topology with link probability p; every source of a target gets one
    random lag in 1..max_lag and the same weight, the weights of a target
    summing to `total`.  Returns (adjacency, lags, weights[src, tgt])."""
    adj = er_graph(n, p, rng)
    lags = np.zeros((n, n), np.int32)
    wts = np.zeros((n, n))
    for t in range(n):
        srcs = np.nonzero(adj[:, t])[0]
        for s_ in srcs:
            lags[s_, t] = int(rng.integers(1, max_lag + 1))
            wts[s_, t] = total / len(srcs)
    return adj, lags, wts


def var_paper(n: int, T: int, seed: int, p: float | None = None, beta: float = 0.5,
              noise_sd: float = 0.1, burn: int = 1000, max_lag: int = 5):
    """The validation VAR of the paper (Methods, "Vector autoregressive
    process"): Y_t = beta Y_{t-1} + sum_X alpha_X X_{t - l_X} + eta_t with
    beta = 0.5, one random lag l_X in 1..5 per source, equal cross-couplings
    summing to 0.4 per target, eta ~ N(0, 0.1^2); ER topology with p = 3 / N.
    Returns (float64 [n][T], adjacency, lags)."""
    rng = np.random.default_rng(seed)
    adj, lags, wts = _paper_couplings(n, 3.0 / n if p is None else p, rng, max_lag)
    coef = np.zeros((max_lag, n, n))
    for i in range(n):
        coef[0, i, i] = beta
    for s_ in range(n):
        for t in range(n):
            if adj[s_, t]:
                coef[lags[s_, t] - 1, t, s_] += wts[s_, t]
    return _simulate_var(coef, T, noise_sd, rng, burn), adj, lags


def clm_paper(n: int, T: int, seed: int, p: float | None = None, beta: float = 0.5,
              noise_sd: float = 0.1, burn: int = 1000, max_lag: int = 5):
    """The validation coupled logistic maps of the paper (Methods, "Coupled
    logistic maps process"): a_t = beta Y_{t-1} + sum_X alpha_X X_{t - l_X}
    with the lags and couplings of var_paper, Y_t = (4 a_t (1 - a_t) + eta_t)
    mod 1.  Returns (float64 [n][T], adjacency, lags)."""
    rng = np.random.default_rng(seed)
    adj, lags, wts = _paper_couplings(n, 3.0 / n if p is None else p, rng, max_lag)
    total = T + burn
    x = np.zeros((total, n))
    x[:max_lag] = rng.random((max_lag, n))
    eta = rng.normal(0.0, noise_sd, size=(total, n))
    srcs = [np.nonzero(adj[:, t])[0] for t in range(n)]
    for t in range(max_lag, total):
        a = beta * x[t - 1]
        for i in range(n):
            for s_ in srcs[i]:
                a[i] += wts[s_, i] * x[t - lags[s_, i], s_]
        v = 4.0 * a * (1.0 - a) + eta[t]
        x[t] = v - np.floor(v)
    return x[burn:].T.copy(), adj, lags


def independent(n: int, T: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, T))


def gaussian_cmi_data(T: int, seed: int, rho_xy: float = 0.6, rho_xz: float = 0.5,
                      rho_yz: float = 0.4):
    """Three jointly Gaussian unit-variance series (i.i.d. over time) with the
    given correlations; returns (float64 [3][T], covariance)."""
    cov = np.array([[1.0, rho_xy, rho_xz], [rho_xy, 1.0, rho_yz], [rho_xz, rho_yz, 1.0]])
    rng = np.random.default_rng(seed)
    L = np.linalg.cholesky(cov)
    x = (L @ rng.normal(size=(3, T)))
    return x, cov


# --- named workloads ---------------------------------------------------------

def workload_chain3(T: int = 1000, seed: int = 1, coupling: float = 0.3):
    """Single estimate workload: 3-node VAR(1) chain, target 2, source (1, lag 1),
    conditioning on the target's lags 1 and 2, k = 4, max lag 2."""
    x, adj = var_chain3(T, seed, coupling)
    s = standardise_jitter(x, seed)
    return dict(series=s, adj=adj, x=[(1, 1)], y=[(2, 0)], z=[(2, 1), (2, 2)], k=4, max_lag=2)


def workload_var10(T: int = 10000, seed: int = 1):
    x, adj, lags = var_er(10, 0.3, T, seed)
    return dict(series=standardise_jitter(x, seed), adj=adj, lags=lags)


def workload_clm100(T: int = 10000, seed: int = 1, n: int = 100):
    x, adj, lags = clm_er(n, T, seed)
    return dict(series=standardise_jitter(x, seed), adj=adj, lags=lags)
