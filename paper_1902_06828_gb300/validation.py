"""Validation harness: network inference against known ground truth.

* precision = TP / (TP + FP), recall = TP / (TP + FN), specificity =
  TN / (TN + FP) of the inferred network against the generating one, over the
  off-diagonal links (Results, "Influence of network size and length of the
  time series");
* the false positive rate per target on empty networks (every inferred link
  is false): the fraction of targets with at least one inferred source,
  averaged over simulations, with the 5th / 95th percentiles of its expected
  value under the complete null, the mean of n_sims i.i.d. Binomial(N,
  alpha_max) / N (Results, "Validation of false positive rate").

Networks come from the seeded generators in synth (random Erdos-Renyi
topology with link probability p = 3 / N; the paper's VAR or coupled logistic
map dynamics); the estimates are te_network_infer's KSG estimator, or with
--estimator gauss its linear-Gaussian one (the paper's choice for the VAR
runs).

    python -m paper_1902_06828_gb300.validation --e1 --dynamics var \\
        --sizes 10 40 --lengths 1000 10000 --sims 2 --surr 200 --alpha 0.05 \\
        --estimator gauss
    python -m paper_1902_06828_gb300.validation --e2 --sizes 10 --alphas 0.05 0.01 \\
        --sims 20 --lengths 10000 --surr 200

Each run prints one JSON line per (size, length, simulation) and a summary line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def scores(adj_true, adj_inf) -> dict:
    """Confusion counts and precision / recall / specificity over the
    off-diagonal entries (adj[src, tgt]).  A ratio with an empty denominator
    is reported as None."""
    t = np.asarray(adj_true, dtype=bool)
    f = np.asarray(adj_inf, dtype=bool)
    off = ~np.eye(t.shape[0], dtype=bool)
    tp = int(np.sum(t & f & off))
    fp = int(np.sum(~t & f & off))
    tn = int(np.sum(~t & ~f & off))
    fn = int(np.sum(t & ~f & off))

    def ratio(a, b):
        return a / (a + b) if a + b else None

    return dict(tp=tp, fp=fp, tn=tn, fn=fn, precision=ratio(tp, fp), recall=ratio(tp, fn),
                specificity=ratio(tn, fp))


def fpr_target(adj_inf) -> float:
    """Fraction of targets (columns) with at least one inferred source."""
    a = np.asarray(adj_inf, dtype=bool) & ~np.eye(np.asarray(adj_inf).shape[0], dtype=bool)
    return float(np.mean(a.any(axis=0)))


def fpr_expected_range(n: int, alpha: float, n_sims: int, q=(0.05, 0.95)):
    """Percentiles of the mean over n_sims i.i.d. Binomial(n, alpha) / n, i.e.
    of Binomial(n * n_sims, alpha) / (n * n_sims)."""
    from scipy.stats import binom
    m = n * n_sims
    return tuple(float(binom.ppf(p, m, alpha)) / m for p in q)


def _network(dynamics: str, n: int, T: int, seed: int, empty: bool = False):
    """The paper's validation processes (Methods, "Vector autoregressive
    process" and "Coupled logistic maps process") on an ER network with
    p = 3 / N, or with no links at all."""
    import synth
    if dynamics == "var":
        x, adj, _ = synth.var_paper(n, T, seed, p=0.0 if empty else None)
    elif dynamics == "clm":
        x, adj, _ = synth.clm_paper(n, T, seed, p=0.0 if empty else None)
    else:
        raise ValueError(f"unknown dynamics {dynamics!r}")
    return synth.standardise_jitter(x, seed), adj


def _infer(te, ctx, series, alpha, n_surr, seed, theiler=0, estimator="ksg"):
    data = te.te_data_create(ctx, series)
    return te.te_network_infer(ctx, data, k=4, theiler=theiler, max_lag_target=5,
                               max_lag_sources=5, n_surr=n_surr, alpha_max=alpha,
                               alpha_min=alpha, alpha_omnibus=alpha, seed=seed,
                               estimator=estimator)


def run_e1(ctx, dynamics="var", sizes=(10,), lengths=(1000,), n_sims=1, alpha=0.05,
           n_surr=200, seed=0, out=print, estimator="ksg"):
    """Precision / recall / specificity over (size, length, simulation)."""
    import paper_1902_06828_gb300 as te
    rows = []
    for n in sizes:
        for T in lengths:
            for s in range(n_sims):
                series, adj = _network(dynamics, n, T, seed + 1000 * s + n)
                t0 = time.time()
                g = _infer(te, ctx, series, alpha, n_surr, seed + s, estimator=estimator)
                row = dict(test="e1", dynamics=dynamics, estimator=estimator, n=n, T=T, sim=s,
                           alpha=alpha, n_surr=n_surr, links=int(adj.sum()),
                           seconds=time.time() - t0,
                           n_estimates=g["n_estimates"], **scores(adj, g["adjacency"]))
                rows.append(row)
                out(json.dumps(row))
    return rows


def run_e2(ctx, dynamics="var", sizes=(10,), alphas=(0.05,), n_sims=10, T=10000, n_surr=200,
           seed=0, out=print, estimator="ksg"):
    """False positive rate per target on empty networks, with its expected range."""
    import paper_1902_06828_gb300 as te
    rows = []
    for n in sizes:
        for alpha in alphas:
            rates = []
            for s in range(n_sims):
                series, _ = _network(dynamics, n, T, seed + 1000 * s + n, empty=True)
                g = _infer(te, ctx, series, alpha, n_surr, seed + s, estimator=estimator)
                rates.append(fpr_target(g["adjacency"]))
            lo, hi = fpr_expected_range(n, alpha, n_sims)
            row = dict(test="e2", dynamics=dynamics, estimator=estimator, n=n, T=T, alpha=alpha,
                       n_surr=n_surr,
                       sims=n_sims, fpr_target=float(np.mean(rates)), expected_p05=lo,
                       expected_p95=hi, within=bool(lo <= np.mean(rates) <= hi))
            rows.append(row)
            out(json.dumps(row))
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--e1", action="store_true")
    ap.add_argument("--e2", action="store_true")
    ap.add_argument("--dynamics", default="var", choices=("var", "clm"))
    ap.add_argument("--sizes", type=int, nargs="+", default=[10])
    ap.add_argument("--lengths", type=int, nargs="+", default=[1000])
    ap.add_argument("--alphas", type=float, nargs="+", default=[0.05])
    ap.add_argument("--alpha", type=float, default=0.05)
    ap.add_argument("--sims", type=int, default=1)
    ap.add_argument("--surr", type=int, default=200)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--estimator", default="ksg", choices=("ksg", "gauss"))
    a = ap.parse_args(argv)
    import paper_1902_06828_gb300 as te
    ctx = te.Context(0)
    if a.e1:
        rows = run_e1(ctx, a.dynamics, a.sizes, a.lengths, a.sims, a.alpha, a.surr, a.seed,
                      estimator=a.estimator)
        for n in a.sizes:
            for T in a.lengths:
                rs = [r for r in rows if r["n"] == n and r["T"] == T]
                mean = {k: float(np.mean([r[k] for r in rs if r[k] is not None] or [np.nan]))
                        for k in ("precision", "recall", "specificity")}
                print(json.dumps(dict(test="e1_summary", dynamics=a.dynamics,
                                      estimator=a.estimator, n=n, T=T, sims=len(rs), **mean)))
    if a.e2:
        run_e2(ctx, a.dynamics, a.sizes, a.alphas, a.sims, a.lengths[0], a.surr, a.seed,
               estimator=a.estimator)
    ctx.close()


if __name__ == "__main__":
    main()
