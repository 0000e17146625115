"""Greedy multivariate transfer-entropy network inference with hierarchical
statistical tests -- plain Python over the C estimator (test infrastructure
only; only tests/, the smoke check and the benchmark's CPU leg use it).

Follows the paper's Methods section step by step:
  Step 1  select the target past         (Inference algorithm, Step 1 a-c)
  Step 2  select the sources past        (Inference algorithm, Step 2 a-c)
  Step 3  prune the selected sources     (Inference algorithm, Step 3 a-c)
  Step 4  omnibus test                   (Inference algorithm, Step 4;
                                          Statistical tests, Omnibus test)
  maximum / minimum statistic tests      (Statistical tests, Maximum statistic
                                          test a-d and Table 1; Minimum
                                          statistic test)
  link rule                              (Results, Influence of network size:
                                          a link X->Y whenever X has a variable
                                          in the selected sources past)
  optional FDR over omnibus p-values     (Statistical tests, Combining across
                                          multiple targets)

Readings where the paper is silent or garbled (each also listed in the design
notes):
  * decisions compare exact integer keys; CMI values are I_key;
  * p = #{surrogate statistic strictly greater than the observed} / S and a
    test is significant iff p < alpha;
  * ties in argmax / argmin go to the first candidate in canonical order
    (target lags ascending in step 1; process then lag ascending in step 2;
    (process, lag) ascending in steps 3 and the sequential test);
  * one permutation per (stage, iteration, surrogate) is shared by every
    candidate of that test (the classic maximum-statistic permutation test);
    with indep_surr each candidate draws its own (counter s + c * 2^32 for
    candidate c of the test in canonical order);
  * pruning repeats until the minimum contribution IS significant or the set
    is empty (the paper's "until ... not significant" contradicts step b);
  * the minimum-statistic p-value uses the same direction as the maximum test;
  * the omnibus surrogate permutes the rows of the whole selected-sources block
    jointly; a failed omnibus test empties the selected sources;
  * the optional step-down ("sequential") stage follows the footnote on
    step-down tests: candidates ordered by their contribution, largest first,
    tested against the null of the maximum over candidates; at the first
    non-significant one it and all smaller ones are removed;
  * a negative Theiler window selects the automatic one: the largest
    autocorrelation decay time over the processes (oracle/theiler.py);
  * replications (trials) are embedded trial by trial and pooled point by
    point (t = L .. T - 1 of trial 0, then of trial 1, ...); their
    surrogates shuffle the candidate's trial order when the R! orders cover
    the S surrogates, else its samples inside each trial (Statistical tests,
    surrogate paragraph); no Theiler window is defined across trials;
  * estimator "gauss" runs the same four steps with the linear-Gaussian CMI
    of oracle/gauss.py (Methods, Vector autoregressive process: the paper's
    estimator for its VAR networks); its decisions compare the float64
    estimates themselves, and it has no neighbour count or Theiler window.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import gauss, ksg

STAGE_STANDALONE, STAGE_TARGET, STAGE_SOURCES, STAGE_PRUNE, STAGE_OMNIBUS, STAGE_SEQ = range(6)


@dataclass
class Params:
    k: int = 4
    theiler: int = 0
    max_lag_target: int = 5
    max_lag_sources: int = 5
    n_surr: int = 200
    alpha_max: float = 0.05
    alpha_min: float = 0.05
    alpha_omnibus: float = 0.05
    alpha_seq: float = 0.05
    seq_test: bool = False
    fdr: bool = False
    alpha_fdr: float = 0.05
    seed: int = 0
    indep_surr: bool = False
    n_threads: int | None = None
    estimator: str = "ksg"        # "ksg" or "gauss"


@dataclass
class TargetResult:
    target: int
    sel_target: list = field(default_factory=list)
    sel_sources: list = field(default_factory=list)
    omnibus_cmi: float = 0.0
    omnibus_p: float = 1.0
    omnibus_key: int = 0
    significant: bool = False
    omnibus_tested: bool = False
    n_estimates: int = 0
    trace: list = field(default_factory=list)   # (stage, iter, cands, keys, null, p, decision)


@dataclass
class _View:
    """What the estimates of one target read: the estimator's series, the
    target present as a variable, the first point t0, the point count N, the
    map from a (process, lag) variable to the estimator's variable, and for
    pooled replications (R trials of n points, surrogate mode) the trial
    layout."""
    series: np.ndarray
    target: int
    y: tuple
    t0: int
    N: int
    vmap: object = None
    trials: tuple | None = None


def _perms(p: Params, v: _View, stage: int, it: int, c: int = 0):
    """Surrogate permutations of a test; with independent surrogates,
    candidate c (canonical order, from 0) draws surrogate s with the counter
    s + c * 2^32 (candidate 0 keeps the shared permutations).  Pooled
    replications shuffle the trial order or the samples inside each trial."""
    off = (c << 32) if p.indep_surr else 0
    if v.trials is not None:
        R_, n, mode = v.trials
        return np.stack([ksg.permutation_trials(p.seed, v.target, stage, it, s + off, R_, n, mode)
                         for s in range(1, p.n_surr + 1)]).astype(np.int32)
    return np.stack([ksg.permutation(p.seed, v.target, stage, it, s + off, v.N)
                     for s in range(1, p.n_surr + 1)]).astype(np.int32)


def _shared_z_keys(v: _View, cand, z, p: Params, stage, it):
    """Keys of single-variable candidates that share one conditioning set."""
    if not p.indep_surr:
        return _group_keys(v, [[c] for c in cand], z, p, _perms(p, v, stage, it))
    keys = []
    for ci, c in enumerate(cand):
        keys += _group_keys(v, [[c]], z, p, _perms(p, v, stage, it, ci))
    return keys


def _group_keys(v: _View, cands_x, z, p: Params, perms):
    """Keys for every candidate (each a list of X variables of equal length)
    against Y = target present given Z, identity and every surrogate.
    Returns int array [n_cand][1 + S] of Python ints (float64 estimates
    with the Gaussian estimator)."""
    vm = v.vmap or (lambda u: tuple(u))
    if p.estimator == "gauss":
        zz = [vm(u) for u in z]
        return [list(gauss.cmi_gauss(v.series, [vm(u) for u in c], [v.y], zz, max_lag=v.t0,
                                     perms=perms)) for c in cands_x]
    n_c = len(cands_x)
    S = perms.shape[0]
    xs, pidx = [], []
    for c in cands_x:
        xs.append([vm(u) for u in c])
        pidx.append(-1)
        for s_ in range(S):
            xs.append([vm(u) for u in c])
            pidx.append(s_)
    z = [vm(u) for u in z]
    keys, _, _ = ksg.cmi_ksg_batch(v.series, xs, [v.y], z, perms=perms, perm_idx=pidx,
                                   k=p.k, theiler=p.theiler, max_lag=v.t0, n_threads=p.n_threads)
    return [keys[c * (S + 1):(c + 1) * (S + 1)] for c in range(n_c)]


def _i_from_key(key: int, q, k: int, N: int) -> float:
    return float(np.ldexp(float(q[k]), -52)) + float(key) / (4503599627370496.0 * float(N))


def max_statistic_test(keys, alpha: float):
    """keys[c][0] original, keys[c][1..S] surrogates.  Returns (argmax c, p,
    significant, null list).  Statistical tests, Maximum statistic test a-d."""
    n_c = len(keys)
    S = len(keys[0]) - 1
    orig = [keys[c][0] for c in range(n_c)]
    best = max(range(n_c), key=lambda c: (orig[c], -c))
    null = [max(keys[c][s] for c in range(n_c)) for s in range(1, S + 1)]
    cnt = sum(1 for v in null if v > orig[best])
    pval = cnt / S
    return best, pval, pval < alpha, null


def min_statistic_test(keys, alpha: float):
    """Minimum statistic: argmin over candidates, null = min over candidates
    per surrogate; p = #{null > observed}/S, significant iff p < alpha."""
    n_c = len(keys)
    S = len(keys[0]) - 1
    orig = [keys[c][0] for c in range(n_c)]
    worst = min(range(n_c), key=lambda c: (orig[c], c))
    null = [min(keys[c][s] for c in range(n_c)) for s in range(1, S + 1)]
    cnt = sum(1 for v in null if v > orig[worst])
    pval = cnt / S
    return worst, pval, pval < alpha, null


def _remove(lst, item):
    return [v for v in lst if v != item]


def _resolve_theiler(series, p: Params) -> Params:
    """A negative window means automatic: the largest autocorrelation decay
    time over the processes (Supporting Information, dynamic correlation
    exclusion)."""
    if p.estimator == "gauss":
        if p.theiler != 0:
            raise ValueError("the Gaussian estimator has no Theiler window")
        return p
    if p.theiler >= 0:
        return p
    from dataclasses import replace
    from .theiler import theiler_window
    return replace(p, theiler=theiler_window(series))


def _trial_mode(mode, R_: int, S: int) -> int:
    """0 = shuffle the trial order, 1 = shuffle inside trials; 'auto' takes
    trial shuffling when the R! trial orders cover the S surrogates."""
    if mode == "trials":
        return 0
    if mode == "within":
        return 1
    return 0 if math.factorial(R_) >= S else 1


def infer_target(series, target: int, p: Params, trials=None) -> TargetResult:
    """series: [n_proc][T], or with trials ('auto', 'trials' or 'within')
    [n_proc][R][T] replications pooled point by point, each trial embedded on
    its own."""
    t0 = max(p.max_lag_target, p.max_lag_sources)
    if trials is None:
        series = np.ascontiguousarray(series, dtype=np.float32)
        p = _resolve_theiler(series, p)
        n_proc, T = series.shape
        N = T - t0
        v = _View(series, target, (target, 0), t0, N)
    else:
        s3 = np.ascontiguousarray(series, dtype=np.float32)
        n_proc, R_, T = s3.shape
        if p.theiler != 0:
            raise ValueError("a Theiler window is not defined across pooled replications")
        n = T - t0
        N = R_ * n
        pooled = ksg.pool_trials(s3, t0)
        v = _View(pooled, target, (target * (t0 + 1), 0), 0, N,
                  vmap=lambda u: (u[0] * (t0 + 1) + u[1], 0),
                  trials=(R_, n, _trial_mode(trials, R_, p.n_surr)))
    if p.estimator not in ("ksg", "gauss"):
        raise ValueError("estimator must be 'ksg' or 'gauss'")
    q = ksg.digamma_q(N + 1)[0] if p.estimator == "ksg" else None
    res = TargetResult(target=target)

    # Step 1: target past
    cand = [(target, l) for l in range(1, p.max_lag_target + 1)]
    sel_y: list = []
    it = 0
    while cand:
        keys = _shared_z_keys(v, cand, sel_y, p, STAGE_TARGET, it)
        res.n_estimates += len(cand) * (p.n_surr + 1)
        b, pval, sig, null = max_statistic_test(keys, p.alpha_max)
        res.trace.append((STAGE_TARGET, it, list(cand), keys, null, pval, sig))
        if not sig:
            break
        sel_y.append(cand[b])
        cand = _remove(cand, cand[b])
        it += 1

    # Step 2: sources past
    cand = [(s, l) for s in range(n_proc) if s != target for l in range(1, p.max_lag_sources + 1)]
    sel_x: list = []
    it = 0
    while cand:
        keys = _shared_z_keys(v, cand, sel_y + sel_x, p, STAGE_SOURCES, it)
        res.n_estimates += len(cand) * (p.n_surr + 1)
        b, pval, sig, null = max_statistic_test(keys, p.alpha_max)
        res.trace.append((STAGE_SOURCES, it, list(cand), keys, null, pval, sig))
        if not sig:
            break
        sel_x.append(cand[b])
        cand = _remove(cand, cand[b])
        it += 1

    # Step 3: prune (each candidate has its own conditioning set)
    it = 0
    while sel_x:
        order = sorted(sel_x)
        keys = []
        for ci, c in enumerate(order):
            rest = [v for v in order if v != c]
            keys += _group_keys(v, [[c]], sel_y + rest, p, _perms(p, v, STAGE_PRUNE, it, ci))
        res.n_estimates += len(order) * (p.n_surr + 1)
        w, pval, sig, null = min_statistic_test(keys, p.alpha_min)
        res.trace.append((STAGE_PRUNE, it, list(order), keys, null, pval, sig))
        if sig:
            break
        sel_x = _remove(sel_x, order[w])
        it += 1

    # Step 4: omnibus
    if sel_x:
        order = sorted(sel_x)
        keys = _group_keys(v, [order], sel_y, p, _perms(p, v, STAGE_OMNIBUS, 0))[0]
        res.n_estimates += p.n_surr + 1
        kstar = keys[0]
        cnt = sum(1 for v in keys[1:] if v > kstar)
        pval = cnt / p.n_surr
        res.omnibus_key = kstar
        res.omnibus_cmi = float(kstar) if q is None else _i_from_key(kstar, q, p.k, N)
        res.omnibus_p = pval
        res.omnibus_tested = True
        res.significant = pval < p.alpha_omnibus
        res.trace.append((STAGE_OMNIBUS, 0, list(order), [keys], None, pval, res.significant))
        if not res.significant:
            sel_x = []

    # Optional step-down stage
    if p.seq_test and sel_x:
        order = sorted(sel_x)
        keys = []
        for ci, c in enumerate(order):
            rest = [v for v in order if v != c]
            keys += _group_keys(v, [[c]], sel_y + rest, p, _perms(p, v, STAGE_SEQ, 0, ci))
        res.n_estimates += len(order) * (p.n_surr + 1)
        S = p.n_surr
        null = [max(keys[c][s] for c in range(len(order))) for s in range(1, S + 1)]
        rank = sorted(range(len(order)), key=lambda c: (-keys[c][0], c))
        keep = []
        for c in rank:
            pv = sum(1 for v in null if v > keys[c][0]) / S
            if pv >= p.alpha_seq:
                break
            keep.append(order[c])
        res.trace.append((STAGE_SEQ, 0, list(order), keys, null, None, keep))
        sel_x = [v for v in order if v in keep]

    res.sel_target = sorted(sel_y)
    res.sel_sources = sorted(sel_x)
    res.significant = res.significant and bool(sel_x)
    return res


def decision_margin(results) -> float:
    """Smallest nonzero gap of a comparison that decided a test in the traces
    of `results`: best against runner-up and observed against every surrogate
    statistic (maximum, minimum and omnibus tests), neighbouring contributions
    and contribution against null (step-down stage).  A second evaluation
    whose estimates differ by less than half of it takes the same decisions;
    exact ties (zero gaps) are left out, as identical inputs tie on both
    sides."""
    gaps = []
    for r in results:
        for stage, _it, _c, keys, null, _p, _d in r.trace:
            orig = np.array([k[0] for k in keys], float)
            if stage in (STAGE_TARGET, STAGE_SOURCES, STAGE_PRUNE):
                srt = np.sort(orig)
                low = stage == STAGE_PRUNE
                if len(srt) > 1:
                    gaps.append(srt[1] - srt[0] if low else srt[-1] - srt[-2])
                gaps += list(np.abs(np.asarray(null, float) - (srt[0] if low else srt[-1])))
            elif stage == STAGE_OMNIBUS:
                k = np.asarray(keys[0], float)
                gaps += list(np.abs(k[1:] - k[0]))
            else:
                gaps += list(np.diff(np.sort(orig)))
                gaps += list(np.abs(np.asarray(null, float)[:, None] - orig[None, :]).ravel())
    gaps = np.asarray(gaps, float)
    gaps = gaps[gaps > 0]
    return float(gaps.min()) if gaps.size else float("inf")


def fdr_bh(pvals, alpha: float):
    """Benjamini-Hochberg step-up: boolean mask of rejected hypotheses."""
    m = len(pvals)
    if m == 0:
        return []
    order = sorted(range(m), key=lambda i: (pvals[i], i))
    last = -1
    for r, i in enumerate(order, start=1):
        if pvals[i] <= alpha * r / m:
            last = r
    rej = [False] * m
    for r, i in enumerate(order, start=1):
        if r <= last:
            rej[i] = True
    return rej


def infer_network(series, p: Params, targets=None, trials=None):
    series = np.ascontiguousarray(series, dtype=np.float32)
    if trials is None:
        p = _resolve_theiler(series, p)
    n_proc = series.shape[0]
    targets = list(range(n_proc)) if targets is None else list(targets)
    results = [infer_target(series, t, p, trials) for t in targets]
    if p.fdr:
        tested = [r for r in results if r.omnibus_tested]
        rej = fdr_bh([r.omnibus_p for r in tested], p.alpha_fdr)
        for r, ok in zip(tested, rej):
            if not ok:
                r.sel_sources = []
                r.significant = False
    adj = np.zeros((n_proc, n_proc), dtype=np.uint8)
    for r in results:
        for (src, _lag) in r.sel_sources:
            adj[src, r.target] = 1
    return adj, results
