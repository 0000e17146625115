"""Theiler-window heuristic -- plain numpy FP64 (test infrastructure only;
only tests/, the smoke check and the benchmark's CPU leg use it).

Dynamic correlation exclusion (Supporting Information, "Validation of false
positive rate on real fMRI data"): the window size is the autocorrelation
decay time of the data, the shortest time shift at which the autocorrelation
function has dropped by a factor 1/e from its zero-shift value.

Readings (also in the design notes):
  * the autocorrelation is the biased sample estimator with the mean of the
    whole series, r(tau) = sum_{t < T - tau} (x_t - m)(x_{t+tau} - m) /
    sum_t (x_t - m)^2;
  * the decay time is the smallest tau >= 1 with r(tau) <= 1/e, the constant
    1/e taken as the FP64 number nearest to e^-1 (0x3FD78B56362CEF38); a
    series that never drops that far within T - 1 shifts gets T - 1, and a
    constant series gets 1;
  * a network run with an automatic window uses the largest decay time over
    all processes for every estimate.
"""
from __future__ import annotations

import struct

import numpy as np

INV_E = struct.unpack("<d", bytes.fromhex("38ef2c36568bd73f"))[0]   # nearest FP64 to e^-1


def acf(x, tau: int) -> float:
    """Biased sample autocorrelation of x at shift tau (FP64)."""
    x = np.asarray(x, dtype=np.float64)
    d = x - x.mean()
    den = float(np.dot(d, d))
    if den == 0.0:
        return 0.0
    return float(np.dot(d[: len(d) - tau], d[tau:])) / den


def autocorr_decay_time(x) -> int:
    """Smallest tau >= 1 with r(tau) <= 1/e (T - 1 if none, 1 if constant)."""
    x = np.asarray(x, dtype=np.float64)
    T = len(x)
    d = x - x.mean()
    den = float(np.dot(d, d))
    if den == 0.0:
        return 1
    for tau in range(1, T):
        if float(np.dot(d[: T - tau], d[tau:])) / den <= INV_E:
            return tau
    return T - 1


def theiler_window(series) -> int:
    """Largest decay time over the processes (rows) of the series."""
    series = np.asarray(series, dtype=np.float64)
    return max(autocorr_decay_time(row) for row in series)
