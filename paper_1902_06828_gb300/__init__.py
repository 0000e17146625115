"""GB300 (sm_103a) KSG conditional mutual information and greedy multivariate
transfer-entropy network inference (Novelli et al., arXiv:1902.06828).

A thin Python layer over the C ABI in include/te_ksg.h: it marshals arguments
and owns handles; every estimate, permutation and test statistic is computed
by the library's CUDA kernels.  Functions carry the C names:

    ctx = Context(0)
    data = te_data_create(ctx, series)              # numpy / torch, host or device
    cmi = cmi_ksg(ctx, data, x=[(1, 1)], y=[(2, 0)], z=[(2, 1), (2, 2)],
                  k=4, max_lag=2, n_surr=200)       # float64 [1 + S]
    net = te_network_infer(ctx, data, n_surr=200, alpha_max=0.05)

Variables are (process, lag) pairs; see include/te_ksg.h for the point set,
the estimator, the surrogates and every error rule.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import _abi
from ._abi import TE_MAX_DIMS, TE_MAX_K  # noqa: F401

__all__ = ["Context", "Data", "TEError", "te_data_create", "cmi_ksg", "cmi_ksg_debug",
           "cmi_ksg_batch", "te_network_infer", "te_get_stats", "Job", "library_path",
           "cmi_ksg_static", "cmi_gauss", "te_serve_start", "te_serve_submit", "te_serve_poll",
           "te_serve_cancel", "te_serve_stop", "te_serve_get_stats", "te_autocorr_decay",
           "te_data_create_trials", "trial_var"]


class TEError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_abi.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def library_path() -> str:
    return _abi.library_path()


def _check(ctx_ptr, st):
    if st != _abi.TE_OK:
        lib = _abi.load()
        msg = lib.te_last_error(ctx_ptr) if ctx_ptr else b"no context"
        raise TEError(st, (msg or b"").decode())


def _vars(v):
    v = list(v) if v is not None else []
    arr = (_abi.TeVar * max(len(v), 1))()
    for a, (p, l) in enumerate(v):
        arr[a].proc = int(p)
        arr[a].lag = int(l)
    return arr, len(v)


class Context:
    """One CUDA device, one stream, the library's workspaces."""

    def __init__(self, device: int = 0):
        self._lib = _abi.load()
        h = C.c_void_p()
        st = self._lib.te_ctx_create(int(device), C.byref(h))
        if st != _abi.TE_OK:
            raise TEError(st, f"te_ctx_create(device={device}) failed (is a CUDA GPU visible?)")
        self._h = h
        self.device = device

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream=None):
        """stream: None (own stream), an int handle, or a torch.cuda.Stream."""
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        _check(self._h, self._lib.te_ctx_set_stream(self._h, C.c_void_p(stream or 0)))

    def set_option(self, name: str, value: int):
        """Execution options (no change to any result): "ksg_tile" (64, 128,
        256; 0 = tuning table), "ksg_members_per_lane" (1, 2; 0 = tuning
        table), "persistent" (0/1), "graph" (0/1)."""
        if name not in _abi.OPTIONS:
            raise ValueError(f"unknown option {name!r}; one of {sorted(_abi.OPTIONS)}")
        _check(self._h, self._lib.te_ctx_set_option(self._h, _abi.OPTIONS[name], int(value)))

    def set_trace(self, fn=None):
        """fn(target, stage, iter, vars, n_cand, n_surr, keys) is called by
        te_network_infer once per test, before its decision: vars a list of
        (proc, lag), keys a list of n_cand lists of n_surr + 1 Python ints
        (128-bit keys, candidate-major).  None switches tracing off."""
        if fn is None:
            self._trace_cb = None
            _check(self._h, self._lib.te_ctx_set_trace(self._h, _abi.TRACE_FN(), None))
            return

        def cb(_user, target, stage, it, vars_p, n_vars, n_cand, n_surr, keys_p):
            vs = [(vars_p[i].proc, vars_p[i].lag) for i in range(n_vars)]
            m = n_cand * (n_surr + 1)
            raw = np.ctypeslib.as_array(keys_p, shape=(2 * m,)).copy()
            flat = _keys_to_int(raw)
            keys = [flat[c * (n_surr + 1):(c + 1) * (n_surr + 1)] for c in range(n_cand)]
            fn(int(target), int(stage), int(it), vs, int(n_cand), int(n_surr), keys)

        self._trace_cb = _abi.TRACE_FN(cb)   # kept alive while the library holds it
        _check(self._h, self._lib.te_ctx_set_trace(self._h, self._trace_cb, None))

    def stats(self) -> dict:
        s = _abi.Stats()
        _check(self._h, self._lib.te_get_stats(self._h, C.byref(s)))
        return dict(estimates=s.estimates, launches=s.launches, pair_evals=s.pair_evals,
                    kernel_ms=s.kernel_ms, ksg_launches=s.ksg_launches, h2d_bytes=s.h2d_bytes,
                    d2h_bytes=s.d2h_bytes, pair_evals_bruteforce=s.pair_evals_bruteforce,
                    ksg_ops=s.ksg_ops)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.te_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Data:
    def __init__(self, ctx: Context, handle, n_proc: int, T: int):
        self.ctx, self._h, self.n_proc, self.T = ctx, handle, n_proc, T

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) and self.ctx._h:
            self.ctx._lib.te_data_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def te_data_create(ctx: Context, series) -> Data:
    """series: float32 [n_proc][T] as a numpy array or a torch tensor (CPU or
    on the context's device).  The library keeps its own device copy."""
    on_dev = 0
    keep = series
    if hasattr(series, "data_ptr"):  # torch tensor
        t = series.contiguous()
        if str(t.dtype) != "torch.float32":
            raise TEError(_abi.TE_EINVAL, "series must be float32")
        keep = t
        ptr = t.data_ptr()
        on_dev = 1 if t.is_cuda else 0
        n_proc, T = t.shape
    else:
        a = np.ascontiguousarray(series, dtype=np.float32)
        if a.ndim != 2:
            raise TEError(_abi.TE_EINVAL, "series must be 2-D [n_proc][T]")
        keep = a
        ptr = a.ctypes.data
        n_proc, T = a.shape
    h = C.c_void_p()
    st = ctx._lib.te_data_create(ctx._h, C.c_void_p(ptr), int(n_proc), int(T), on_dev, C.byref(h))
    del keep
    _check(ctx._h, st)
    return Data(ctx, h, int(n_proc), int(T))


def te_data_create_trials(ctx: Context, series, max_lag: int) -> Data:
    """series: float32 [n_proc][n_rep][T] replications (numpy).  Each trial
    is embedded with the maximum lag `max_lag` and the trials are pooled:
    row p * (max_lag + 1) + l of the result is process p at lag l."""
    a = np.ascontiguousarray(series, dtype=np.float32)
    if a.ndim != 3:
        raise TEError(_abi.TE_EINVAL, "series must be 3-D [n_proc][n_rep][T]")
    n_proc, n_rep, T = a.shape
    h = C.c_void_p()
    st = ctx._lib.te_data_create_trials(ctx._h, C.c_void_p(a.ctypes.data), int(n_proc),
                                        int(n_rep), int(T), int(max_lag), 0, C.byref(h))
    _check(ctx._h, st)
    return Data(ctx, h, int(n_proc) * (int(max_lag) + 1), int(n_rep) * (int(T) - int(max_lag)))


def trial_var(proc: int, lag: int, max_lag: int) -> tuple:
    """The row of pooled trial data holding process `proc` at `lag`, as a
    variable for the single-estimate calls (lag 0, max_lag 0)."""
    return (proc * (max_lag + 1) + lag, 0)


def _params(k, theiler, max_lag, n_surr, seed, stream_tag):
    return _abi.KsgParams(int(k), int(theiler), int(max_lag), int(n_surr), int(seed),
                          int(stream_tag))


def _default_max_lag(x, y, z):
    lags = [l for _, l in list(x) + list(y) + list(z or [])]
    return max(lags) if lags else 0


def cmi_ksg(ctx: Context, data: Data, x, y, z=(), *, k=4, theiler=0, max_lag=None, n_surr=0,
            seed=0, stream_tag=0, return_keys=False):
    """KSG I(X;Y|Z) and n_surr permutation surrogates -> float64 [1 + n_surr]
    (and int keys when return_keys)."""
    if max_lag is None:
        max_lag = _default_max_lag(x, y, z)
    xv, dx = _vars(x)
    yv, dy = _vars(y)
    zv, dz = _vars(z)
    out = np.zeros(1 + max(int(n_surr), 0), np.float64)
    keys = np.zeros(2 * out.size, np.int64)
    p = _params(k, theiler, max_lag, n_surr, seed, stream_tag)
    st = ctx._lib.cmi_ksg(ctx._h, data._h, xv, dx, yv, dy, zv if dz else None, dz, C.byref(p),
                          out.ctypes.data, keys.ctypes.data)
    _check(ctx._h, st)
    if return_keys:
        return out, _keys_to_int(keys)
    return out


def cmi_gauss(ctx: Context, data: Data, x, y, z=(), *, max_lag=None, n_surr=0, seed=0,
              stream_tag=0):
    """Linear-Gaussian CMI and n_surr permutation surrogates -> (values, error
    bounds), each float64 [1 + n_surr]."""
    if max_lag is None:
        max_lag = _default_max_lag(x, y, z)
    xv, dx = _vars(x)
    yv, dy = _vars(y)
    zv, dz = _vars(z)
    out = np.zeros(1 + max(int(n_surr), 0), np.float64)
    err = np.zeros_like(out)
    p = _params(1, 0, max_lag, n_surr, seed, stream_tag)
    st = ctx._lib.cmi_gauss(ctx._h, data._h, xv, dx, yv, dy, zv if dz else None, dz, C.byref(p),
                            out.ctypes.data, err.ctypes.data)
    _check(ctx._h, st)
    return out, err


def _keys_to_int(keys):
    res = []
    for hi, lo in keys.reshape(-1, 2):
        v = (int(hi) << 64) | (int(lo) & 0xFFFFFFFFFFFFFFFF)
        if v >= 1 << 127:
            v -= 1 << 128
        res.append(v)
    return res


def cmi_ksg_debug(ctx: Context, data: Data, x, y, z=(), *, member=0, k=4, theiler=0,
                  max_lag=None, n_surr=0, seed=0, stream_tag=0):
    """Per-point eps and counts (n_xz, n_yz, n_z) of one member."""
    if max_lag is None:
        max_lag = _default_max_lag(x, y, z)
    N = data.T - int(max_lag)
    xv, dx = _vars(x)
    yv, dy = _vars(y)
    zv, dz = _vars(z)
    eps = np.zeros(max(N, 1), np.float32)
    nxz, nyz, nz = (np.zeros(max(N, 1), np.int32) for _ in range(3))
    p = _params(k, theiler, max_lag, n_surr, seed, stream_tag)
    st = ctx._lib.cmi_ksg_debug(ctx._h, data._h, xv, dx, yv, dy, zv if dz else None, dz,
                                C.byref(p), int(member), eps.ctypes.data, nxz.ctypes.data,
                                nyz.ctypes.data, nz.ctypes.data)
    _check(ctx._h, st)
    return dict(eps=eps, n_xz=nxz, n_yz=nyz, n_z=nz)


@dataclass
class Job:
    data: Data
    x: list
    y: list
    z: list = field(default_factory=list)
    k: int = 4
    theiler: int = 0
    max_lag: int | None = None
    n_surr: int = 0
    seed: int = 0
    stream_tag: int = 0


def cmi_ksg_batch(ctx: Context, jobs, return_keys=False):
    """Evaluate many jobs in fused launches -> list of float64 arrays."""
    n = len(jobs)
    arr = (_abi.CmiJob * max(n, 1))()
    keep = []
    sizes = []
    for a, j in enumerate(jobs):
        ml = j.max_lag if j.max_lag is not None else _default_max_lag(j.x, j.y, j.z)
        xv, dx = _vars(j.x)
        yv, dy = _vars(j.y)
        zv, dz = _vars(j.z)
        keep += [xv, yv, zv]
        arr[a].data = j.data._h
        arr[a].x = C.cast(xv, C.POINTER(_abi.TeVar))
        arr[a].y = C.cast(yv, C.POINTER(_abi.TeVar))
        arr[a].z = C.cast(zv, C.POINTER(_abi.TeVar)) if dz else None
        arr[a].dx, arr[a].dy, arr[a].dz = dx, dy, dz
        arr[a].params = _params(j.k, j.theiler, ml, j.n_surr, j.seed, j.stream_tag)
        sizes.append(1 + int(j.n_surr))
    total = sum(sizes)
    out = np.zeros(max(total, 1), np.float64)
    keys = np.zeros(2 * max(total, 1), np.int64)
    st = ctx._lib.cmi_ksg_batch(ctx._h, arr, n, out.ctypes.data, keys.ctypes.data)
    _check(ctx._h, st)
    res, kres, o = [], [], 0
    allk = _keys_to_int(keys) if return_keys else None
    for s in sizes:
        res.append(out[o:o + s].copy())
        if return_keys:
            kres.append(allk[o:o + s])
        o += s
    return (res, kres) if return_keys else res


def te_network_infer(ctx: Context, data: Data, *, k=4, theiler=0, max_lag_target=5,
                     max_lag_sources=5, n_surr=200, alpha_max=0.05, alpha_min=0.05,
                     alpha_omnibus=0.05, alpha_seq=0.05, seq_test=False, fdr=False,
                     alpha_fdr=0.05, seed=0, targets=None, indep_surr=False,
                     surr_mode="auto", estimator="ksg") -> dict:
    """Greedy multivariate TE network inference; returns a dict with the
    adjacency [src, tgt], min lags, per-target selections and counters.
    estimator: "ksg" or "gauss" (the linear-Gaussian estimator of cmi_gauss;
    k is then unused and theiler must be 0)."""
    modes = {"auto": 0, "trials": 1, "within": 2}
    estimators = {"ksg": 0, "gauss": 1}
    if surr_mode not in modes:
        raise ValueError(f"surr_mode must be one of {sorted(modes)}, not {surr_mode!r}")
    if estimator not in estimators:
        raise ValueError(f"estimator must be one of {sorted(estimators)}, not {estimator!r}")
    tarr = None
    nt = 0
    if targets is not None:
        nt = len(targets)
        tarr = (C.c_int32 * max(nt, 1))(*[int(t) for t in targets])
    P = _abi.InferParams(int(k), int(theiler), int(max_lag_target), int(max_lag_sources),
                         int(n_surr), float(alpha_max), float(alpha_min), float(alpha_omnibus),
                         float(alpha_seq), int(bool(seq_test)), int(bool(fdr)), float(alpha_fdr),
                         int(seed), C.cast(tarr, C.POINTER(C.c_int32)) if tarr else None, nt,
                         int(bool(indep_surr)), modes[surr_mode], estimators[estimator])
    res = C.POINTER(_abi.NetworkResult)()
    st = ctx._lib.te_network_infer(ctx._h, data._h, C.byref(P), C.byref(res))
    _check(ctx._h, st)
    try:
        R = res.contents
        n = R.n_proc
        adj = np.ctypeslib.as_array(R.adjacency, shape=(n * n,)).reshape(n, n).copy()
        lag = np.ctypeslib.as_array(R.min_lag, shape=(n * n,)).reshape(n, n).copy()
        tlist = []
        for a in range(R.n_targets):
            t = R.targets[a]
            tlist.append(dict(
                target=t.target,
                sel_target=[(t.sel_target[i].proc, t.sel_target[i].lag)
                            for i in range(t.n_sel_target)],
                sel_sources=[(t.sel_sources[i].proc, t.sel_sources[i].lag)
                             for i in range(t.n_sel_sources)],
                omnibus_cmi=t.omnibus_cmi, omnibus_p=t.omnibus_p,
                omnibus_tested=bool(t.omnibus_tested), significant=bool(t.significant),
                n_estimates=int(t.n_estimates)))
        return dict(adjacency=adj, min_lag=lag, targets=tlist, n_estimates=int(R.n_estimates),
                    seconds=R.seconds, theiler=int(R.theiler))
    finally:
        ctx._lib.te_network_result_free(res)


def te_get_stats(ctx: Context) -> dict:
    return ctx.stats()


def te_alu_peak(ctx: Context, kind: str) -> float:
    """Measured rate (counted lane operations per second) of the KSG kernel's
    instruction pattern: kind "knn" (3 per member-pair), "count" (7 per
    member-pair) or "fadd" (plain FP32 adds, the issue limit)."""
    out = C.c_double()
    k = {"knn": 0, "count": 1, "fadd": 2}[kind]
    _check(ctx._h, ctx._lib.te_alu_peak(ctx._h, k, C.byref(out)))
    return float(out.value)


def te_autocorr_decay(ctx: Context, data: Data, proc: int = -1) -> int:
    """Autocorrelation decay time of one process (or the largest over all
    with proc = -1): the Theiler-window heuristic."""
    out = C.c_int32()
    st = ctx._lib.te_autocorr_decay(ctx._h, data._h, int(proc), C.byref(out))
    _check(ctx._h, st)
    return int(out.value)


def _job_struct(j, keep):
    ml = j.max_lag if j.max_lag is not None else _default_max_lag(j.x, j.y, j.z)
    xv, dx = _vars(j.x)
    yv, dy = _vars(j.y)
    zv, dz = _vars(j.z)
    keep += [xv, yv, zv]
    js = _abi.CmiJob()
    js.data = j.data._h
    js.x = C.cast(xv, C.POINTER(_abi.TeVar))
    js.y = C.cast(yv, C.POINTER(_abi.TeVar))
    js.z = C.cast(zv, C.POINTER(_abi.TeVar)) if dz else None
    js.dx, js.dy, js.dz = dx, dy, dz
    js.params = _params(j.k, j.theiler, ml, j.n_surr, j.seed, j.stream_tag)
    return js


def te_serve_start(ctx: Context, hbm_budget_bytes=0, max_inflight=0, max_batch_jobs=0):
    cfg = _abi.ServeConfig(int(hbm_budget_bytes), int(max_inflight), int(max_batch_jobs))
    _check(ctx._h, ctx._lib.te_serve_start(ctx._h, C.byref(cfg)))


def te_serve_submit(ctx: Context, job: "Job") -> int:
    """Queue a job (thread-safe) -> ticket."""
    keep = []
    js = _job_struct(job, keep)
    t = C.c_uint64()
    st = ctx._lib.te_serve_submit(ctx._h, C.byref(js), C.byref(t))
    if st != _abi.TE_OK:
        raise TEError(st, "te_serve_submit rejected the job")
    return int(t.value)


def te_serve_poll(ctx: Context, ticket: int, n_surr: int, timeout_ms: int = -1,
                  return_keys=False):
    """Wait for a job's results (float64 [1 + n_surr]); raises TEError with
    TE_ETIMEOUT (ticket kept) or TE_ECANCELLED."""
    out = np.zeros(1 + int(n_surr), np.float64)
    keys = np.zeros(2 * out.size, np.int64)
    st = ctx._lib.te_serve_poll(ctx._h, int(ticket), int(timeout_ms), out.ctypes.data,
                                keys.ctypes.data)
    if st != _abi.TE_OK:
        raise TEError(st, "te_serve_poll")
    return (out, _keys_to_int(keys)) if return_keys else out


def te_serve_cancel(ctx: Context, ticket: int):
    _check(ctx._h, ctx._lib.te_serve_cancel(ctx._h, int(ticket)))


def te_serve_stop(ctx: Context):
    _check(ctx._h, ctx._lib.te_serve_stop(ctx._h))


def te_serve_get_stats(ctx: Context) -> dict:
    s = _abi.ServeStats()
    _check(ctx._h, ctx._lib.te_serve_get_stats(ctx._h, C.byref(s)))
    return {f: getattr(s, f) for f, _ in s._fields_}


def cmi_ksg_static(series_dev, x, y, z=(), *, k=4, theiler=0, max_lag=None, n_surr=0, seed=0,
                   stream_tag=0, stream=None, return_keys=False):
    """cmi_ksg without any device allocation, for callers that cannot
    allocate device memory (see include/te_ksg.h).  series_dev: a CUDA float32
    tensor [n_proc][T] on the current device; stream: None, an int handle or a
    torch.cuda.Stream.  No context is involved; errors carry the status only."""
    lib = _abi.load()
    t = series_dev
    if not (hasattr(t, "is_cuda") and t.is_cuda) or str(t.dtype) != "torch.float32":
        raise TEError(_abi.TE_EINVAL, "series_dev must be a CUDA float32 tensor")
    import torch
    if t.device.index != torch.cuda.current_device():
        raise TEError(_abi.TE_EINVAL, "series_dev must live on the current CUDA device")
    if t.dim() != 2 or not t.is_contiguous():
        # a copy would allocate device memory, which this entry point promises not to do
        raise TEError(_abi.TE_EINVAL, "series_dev must be a contiguous [n_proc][T] tensor")
    n_proc, T = t.shape
    if max_lag is None:
        max_lag = _default_max_lag(x, y, z)
    if stream is not None and hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    xv, dx = _vars(x)
    yv, dy = _vars(y)
    zv, dz = _vars(z)
    out = np.zeros(1 + max(int(n_surr), 0), np.float64)
    keys = np.zeros(2 * out.size, np.int64)
    p = _params(k, theiler, max_lag, n_surr, seed, stream_tag)
    st = lib.cmi_ksg_static(C.c_void_p(t.data_ptr()), int(n_proc), int(T), xv, dx, yv, dy,
                            zv if dz else None, dz, C.byref(p), C.c_void_p(stream or 0),
                            out.ctypes.data, keys.ctypes.data)
    if st != _abi.TE_OK:
        raise TEError(st, "cmi_ksg_static failed")
    return (out, _keys_to_int(keys)) if return_keys else out
