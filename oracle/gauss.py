"""Linear-Gaussian CMI oracle (test infrastructure only; see oracle/__init__).

The paper uses a Gaussian estimator for the VAR runs and notes that transfer
entropy equals Granger causality for Gaussian variables (Methods, Vector
autoregressive process); it prints no formula.  Reading used here: the
plug-in estimate from the sample covariance (ddof = 1) of the embedded
variables,

    I(X; Y | Z) = 1/2 [ln|S_XZ| + ln|S_YZ| - ln|S_Z| - ln|S_XYZ|]

(|S_Z| = 1 for an empty Z), in float64 with numpy's slogdet.  Surrogate s
reads the rows of the whole X block through permutation s (X at point i is
X at point pi_s(i)); Y and Z are never permuted.  Points are as for the KSG
oracle: point i at time t0 + i, variable (p, lag) = series[p][t0 + i - lag].
"""
from __future__ import annotations

import numpy as np


def _cols(series, vars_, t0, N, perm=None):
    s = np.asarray(series, dtype=np.float32).astype(np.float64)
    idx = np.arange(N) if perm is None else np.asarray(perm)
    return np.stack([s[p, t0 - lag + idx] for p, lag in vars_], axis=1) if len(vars_) else \
        np.zeros((N, 0))


def _logdet(c):
    if c.shape[0] == 0:
        return 0.0
    sign, ld = np.linalg.slogdet(c)
    if sign <= 0:
        raise ValueError("covariance is not positive definite")
    return float(ld)


def cmi_gauss(series, x, y, z, *, max_lag, perms=None):
    """Original estimate and one per row of `perms` (int [S][N]) -> float64 [1 + S]."""
    s = np.asarray(series)
    T = s.shape[1]
    t0 = int(max_lag)
    N = T - t0
    Y = _cols(s, y, t0, N)
    Z = _cols(s, z, t0, N)
    dx, dy, dz = len(x), len(y), len(z)
    out = []
    plist = [None] + ([] if perms is None else list(perms))
    for p in plist:
        X = _cols(s, x, t0, N, p)
        A = np.concatenate([X, Y, Z], axis=1)
        C = np.cov(A, rowvar=False, ddof=1).reshape(A.shape[1], A.shape[1])
        ix = list(range(dx))
        iy = list(range(dx, dx + dy))
        iz = list(range(dx + dy, dx + dy + dz))
        sub = lambda ii: C[np.ix_(ii, ii)]
        out.append(0.5 * (_logdet(sub(ix + iz)) + _logdet(sub(iy + iz)) - _logdet(sub(iz))
                          - _logdet(sub(ix + iy + iz))))
    return np.array(out)
