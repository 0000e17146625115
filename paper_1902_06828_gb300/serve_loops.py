"""Greedy target loops as clients of the serving API (te_serve_*).

A loop runs one target's greedy multivariate TE inference (Methods, Inference
algorithm steps 1-4; Statistical tests: maximum statistic, minimum statistic
and omnibus tests) and emits every test as one served request: one serving job
per candidate, each with the test's S surrogates.  The jobs of a test share
the seed and the stream tag, so they draw the same permutations (one
permutation per test and surrogate, shared by its candidates), and every test
has its own tag.  Decisions compare the exact 128-bit keys the server returns:
  * target past / sources past: maximum statistic, argmax (ties to the first
    candidate in order), p = #{max over candidates of surrogate s > observed}/S,
    select while p < alpha;
  * pruning: minimum statistic over the selected sources, each conditioned on
    the others, remove the argmin while p >= alpha;
  * omnibus: the selected sources as one block, p = #{K_s > K*}/S; a failed
    test empties the selection.
Many loops over many data sets share one server: this is the request stream
of independent targets analysed concurrently (Supporting Information, Run-time
on CPU and GPU).  The module is host control only; every estimate runs in the
library.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    loop: int
    stage: int
    it: int
    jobs: list
    t_submit: float = 0.0
    t_done: float = 0.0
    keys: list = field(default_factory=list)

    @property
    def estimates(self) -> int:
        return sum(1 + j.n_surr for j in self.jobs)


class TargetLoop:
    """The greedy state of one target; next_request() gives the jobs of the
    next test (None when the target is done), decide(keys) applies it."""

    def __init__(self, te, data, n_proc, target, *, n_surr, alpha=0.05, k=4, max_lag=5,
                 seed=0, tag_base=0, loop_id=0):
        self.te, self.data, self.n_proc, self.target = te, data, n_proc, target
        self.S, self.alpha, self.k, self.L = n_surr, alpha, k, max_lag
        self.seed, self.tag, self.id = seed, tag_base, loop_id
        self.stage, self.it = 1, 0
        self.cand = [(target, l) for l in range(1, max_lag + 1)]
        self.sel_y, self.sel_x = [], []
        self.omnibus_p = None
        self.done = False
        self._order = []

    def _job(self, x, z, tag):
        return self.te.Job(self.data, list(x), [(self.target, 0)], list(z), k=self.k,
                           max_lag=self.L, n_surr=self.S, seed=self.seed, stream_tag=tag)

    def next_request(self):
        while not self.done:
            if self.stage in (1, 2):
                if self.stage == 2 and self.it == 0 and not self._order and not self.cand:
                    self.cand = [(q, l) for q in range(self.n_proc) if q != self.target
                                 for l in range(1, self.L + 1)]
                if not self.cand:
                    self._advance()
                    continue
                z = self.sel_y + (self.sel_x if self.stage == 2 else [])
                self._order = list(self.cand)
                self.tag += 1
                return Request(self.id, self.stage, self.it,
                               [self._job([c], z, self.tag) for c in self._order])
            if self.stage == 3:
                if not self.sel_x:
                    self._advance()
                    continue
                self._order = sorted(self.sel_x)
                self.tag += 1
                return Request(self.id, 3, self.it, [
                    self._job([c], self.sel_y + [v for v in self._order if v != c], self.tag)
                    for c in self._order])
            if self.stage == 4:
                if not self.sel_x:
                    self._advance()
                    continue
                self._order = sorted(self.sel_x)
                self.tag += 1
                return Request(self.id, 4, 0, [self._job(self._order, self.sel_y, self.tag)])
        return None

    def _advance(self):
        self.stage += 1
        self.it = 0
        self.cand = []
        self._order = []
        if self.stage > 4:
            self.done = True

    def decide(self, keys):
        """keys: one list of 1 + S exact keys per job of the request."""
        S = self.S
        orig = [kk[0] for kk in keys]
        if self.stage in (1, 2):
            best = max(range(len(orig)), key=lambda c: (orig[c], -c))
            null = [max(kk[s] for kk in keys) for s in range(1, S + 1)]
            p = sum(1 for v in null if v > orig[best]) / S
            if p < self.alpha:
                c = self._order[best]
                (self.sel_y if self.stage == 1 else self.sel_x).append(c)
                self.cand = [v for v in self._order if v != c]
                self.it += 1
            else:
                self.cand = []
                if self.stage == 1:   # the sources' candidates come next
                    self._advance()
                    self.cand = [(q, l) for q in range(self.n_proc) if q != self.target
                                 for l in range(1, self.L + 1)]
                    return
                self._advance()
            return
        if self.stage == 3:
            worst = min(range(len(orig)), key=lambda c: (orig[c], c))
            null = [min(kk[s] for kk in keys) for s in range(1, S + 1)]
            p = sum(1 for v in null if v > orig[worst]) / S
            if p < self.alpha:
                self._advance()
            else:
                c = self._order[worst]
                self.sel_x = [v for v in self.sel_x if v != c]
                self.it += 1
            return
        if self.stage == 4:
            p = sum(1 for v in keys[0][1:] if v > keys[0][0]) / S
            self.omnibus_p = p
            if not p < self.alpha:
                self.sel_x = []
            self._advance()

    def result(self):
        return dict(target=self.target, sel_target=sorted(self.sel_y),
                    sel_sources=sorted(self.sel_x), omnibus_p=self.omnibus_p)


def run_served(te, ctx, loops, deadline_s=None, evaluate=None):
    """Run every loop on its own thread against the server started on ctx
    (te_serve_start) until it is done or the deadline passes; a request
    already submitted is completed.  evaluate(request) may replace the server
    (then the keys come from it).  Returns the completed requests."""
    done = []
    lock = threading.Lock()
    t_end = None if deadline_s is None else time.perf_counter() + deadline_s

    def worker(loop):
        while t_end is None or time.perf_counter() < t_end:
            req = loop.next_request()
            if req is None:
                return
            req.t_submit = time.perf_counter()
            if evaluate is not None:
                req.keys = evaluate(req)
            else:
                tickets = [te.te_serve_submit(ctx, j) for j in req.jobs]
                req.keys = [te.te_serve_poll(ctx, t, j.n_surr, return_keys=True)[1]
                            for t, j in zip(tickets, req.jobs)]
            req.t_done = time.perf_counter()
            loop.decide(req.keys)
            with lock:
                done.append(req)

    ths = [threading.Thread(target=worker, args=(lp,), daemon=True) for lp in loops]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    return done
