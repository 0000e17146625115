"""ctypes wrapper over the C oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this module.  It never touches the CUDA library.

Variables are (process, lag) pairs; a point i sits at time t0 + i and the
variable's value there is series[process][t0 + i - lag] (Methods, "Definitions
and assumptions": candidate past sets up to a maximum lag; the embedding keeps
relative lags only).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = C.CDLL(path)
        i32, i64, u64, dbl = C.c_int32, C.c_int64, C.c_uint64, C.c_double
        P = C.c_void_p
        L.oracle_digamma_q.argtypes = [i32, P, P]
        L.oracle_digamma_q.restype = C.c_int
        L.oracle_digamma_plain.argtypes = [i32]
        L.oracle_digamma_plain.restype = dbl
        L.oracle_perm_key.argtypes = [u64, u64, u64, u64, u64]
        L.oracle_perm_key.restype = u64
        L.oracle_splitmix64_stream.argtypes = [u64, i32, P]
        L.oracle_splitmix64_stream.restype = None
        L.oracle_permutation.argtypes = [u64, u64, u64, u64, u64, i32, P]
        L.oracle_permutation.restype = C.c_int
        L.oracle_permutation_trials.argtypes = [u64, u64, u64, u64, u64, i32, i32, i32, P]
        L.oracle_permutation_trials.restype = C.c_int
        L.oracle_ksg_cmi.argtypes = [P, i32, i32, i32, i32, P, i32, P, i32, P, i32, P, i32, i32,
                                     P, P, P, P, P, P, P]
        L.oracle_ksg_cmi.restype = C.c_int
        L.oracle_ksg_batch.argtypes = [P, i32, i32, i32, i32, i32, P, i32, P, i32, P, i32, P, i32,
                                       P, i32, i32, i32, P, P, P]
        L.oracle_ksg_batch.restype = C.c_int
        L.oracle_max_threads.argtypes = []
        L.oracle_max_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _vars(v):
    a = np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(-1, 2))
    return a, a.shape[0]


def key_to_int(hi: int, lo: int) -> int:
    """128-bit two's-complement (hi, lo) -> Python int."""
    v = (int(hi) << 64) | (int(lo) & 0xFFFFFFFFFFFFFFFF)
    if v >= 1 << 127:
        v -= 1 << 128
    return v


def digamma_q(n_max: int):
    q = np.zeros(n_max + 1, dtype=np.int64)
    margin = C.c_double(0.0)
    st = lib().oracle_digamma_q(n_max, _ptr(q), C.byref(margin))
    if st:
        raise ValueError(f"oracle_digamma_q failed ({st})")
    return q, margin.value


def digamma_plain(n: int) -> float:
    return lib().oracle_digamma_plain(int(n))


def perm_key(seed, target, stage, it, s) -> int:
    return int(lib().oracle_perm_key(seed, target, stage, it, s))


def splitmix64_stream(state: int, n: int):
    out = np.zeros(n, dtype=np.uint64)
    lib().oracle_splitmix64_stream(state, n, _ptr(out))
    return [int(v) for v in out]


def permutation(seed: int, target: int, stage: int, it: int, s: int, n: int) -> np.ndarray:
    p = np.empty(n, dtype=np.int32)
    st = lib().oracle_permutation(seed, target, stage, it, s, n, _ptr(p))
    if st:
        raise ValueError("oracle_permutation: bad arguments")
    return p


def permutation_trials(seed: int, target: int, stage: int, it: int, s: int, R: int, n: int,
                       mode: int) -> np.ndarray:
    """Surrogate permutation of R pooled trials of n points: mode 0 shuffles
    the trial order, mode 1 the samples inside each trial."""
    p = np.empty(R * n, dtype=np.int32)
    st = lib().oracle_permutation_trials(seed, target, stage, it, s, R, n, mode, _ptr(p))
    if st:
        raise ValueError("oracle_permutation_trials: bad arguments")
    return p


def pool_trials(series3, L: int) -> np.ndarray:
    """Embedded, pooled view of a [n_proc][R][T] series for lags 0..L: row
    p * (L + 1) + l holds X_p at lag l for the points t = L .. T - 1 of every
    trial, trial by trial (R (T - L) points)."""
    s = np.asarray(series3, dtype=np.float32)
    n_proc, R, T = s.shape
    out = np.empty((n_proc * (L + 1), R * (T - L)), dtype=np.float32)
    for p in range(n_proc):
        for l in range(L + 1):
            out[p * (L + 1) + l] = s[p, :, L - l:T - l].reshape(-1)
    return out


def cmi_ksg(series, x, y, z, *, k=4, theiler=0, max_lag=None, perm=None, per_point=False):
    """One KSG CMI estimate I(X;Y|Z), X read through `perm` when given.

    Returns dict(key=int, i_key=float, i_plain=float[, eps, n_xz, n_yz, n_z]).
    `max_lag` fixes the first point's time t0; default = largest lag used.
    """
    s = np.ascontiguousarray(series, dtype=np.float32)
    n_proc, T = s.shape
    xv, dx = _vars(x)
    yv, dy = _vars(y)
    zv, dz = _vars(z) if len(z) else (np.zeros((0, 2), np.int32), 0)
    if max_lag is None:
        lags = [v[1] for v in list(xv) + list(yv) + list(zv)]
        max_lag = int(max(lags)) if lags else 0
    t0 = int(max_lag)
    N = T - t0
    pm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
    if pm is not None and pm.shape != (N,):
        raise ValueError("perm must have one entry per point")
    key2 = np.zeros(2, dtype=np.int64)
    ik, ip = C.c_double(), C.c_double()
    eps = nxz = nyz = nz = None
    if per_point:
        eps = np.zeros(N, np.float32)
        nxz, nyz, nz = (np.zeros(N, np.int32) for _ in range(3))
    st = lib().oracle_ksg_cmi(_ptr(s), n_proc, T, t0, N, _ptr(xv), dx, _ptr(yv), dy,
                              _ptr(zv) if dz else None, dz, _ptr(pm), k, theiler,
                              _ptr(key2), C.byref(ik), C.byref(ip),
                              _ptr(eps), _ptr(nxz), _ptr(nyz), _ptr(nz))
    if st:
        raise ValueError(f"oracle_ksg_cmi rejected its arguments ({st})")
    out = dict(key=key_to_int(key2[0], key2[1]), i_key=ik.value, i_plain=ip.value, N=N)
    if per_point:
        out.update(eps=eps, n_xz=nxz, n_yz=nyz, n_z=nz)
    return out


def cmi_ksg_batch(series, xs, y, z, *, perms=None, perm_idx=None, k=4, theiler=0,
                  max_lag=None, n_threads=None):
    """Many members sharing Y and Z.  xs: list of X variable lists (equal dims);
    perms: int32 [n_perm][N]; perm_idx[b] = row of perms for member b, -1 identity.
    Returns (keys list[int], i_key ndarray, i_plain ndarray)."""
    s = np.ascontiguousarray(series, dtype=np.float32)
    n_proc, T = s.shape
    nm = len(xs)
    xa = np.ascontiguousarray(np.asarray(xs, dtype=np.int32).reshape(nm, -1, 2))
    dx = xa.shape[1]
    yv, dy = _vars(y)
    zv, dz = _vars(z) if len(z) else (np.zeros((0, 2), np.int32), 0)
    if max_lag is None:
        lags = list(xa[..., 1].ravel()) + list(yv[:, 1]) + list(zv[:, 1])
        max_lag = int(max(lags))
    t0 = int(max_lag)
    N = T - t0
    if perms is None:
        pa = np.zeros((0, N), np.int32)
    else:
        pa = np.ascontiguousarray(perms, dtype=np.int32).reshape(-1, N)
    pidx = np.full(nm, -1, np.int32) if perm_idx is None else np.ascontiguousarray(perm_idx, np.int32)
    key2 = np.zeros((nm, 2), np.int64)
    ik = np.zeros(nm)
    ip = np.zeros(nm)
    nt = n_threads if n_threads else max(1, lib().oracle_max_threads())
    st = lib().oracle_ksg_batch(_ptr(s), n_proc, T, t0, N, nm, _ptr(xa), dx, _ptr(yv), dy,
                                _ptr(zv) if dz else None, dz, _ptr(pa), pa.shape[0], _ptr(pidx),
                                k, theiler, nt, _ptr(key2), _ptr(ik), _ptr(ip))
    if st:
        raise ValueError(f"oracle_ksg_batch rejected its arguments ({st})")
    keys = [key_to_int(h, l) for h, l in key2]
    return keys, ik, ip


def max_threads() -> int:
    return int(lib().oracle_max_threads())


def cpu_count() -> int:
    return os.cpu_count() or 1
