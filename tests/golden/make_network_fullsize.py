"""Write the expected greedy-inference traces of one target at T = 10^4.

Runs only the CPU oracle (oracle.network.infer_target, Methods, Inference
algorithm steps 1-4 with the maximum / minimum statistic and omnibus tests)
on the benchmark's synthetic workloads at full length and stores, per target:

  * the SHA-256 of the float32 input series (the GPU test regenerates the
    series from the same seed and checks this first),
  * every request of the greedy loop in order: stage, iteration, candidates,
    the SHA-256 of all its keys (every candidate x (original + S surrogates),
    decimal, candidate-major, comma separated) and the first keys in clear,
    the p-value and the decision,
  * the result: selected target past and sources past, omnibus estimate, key
    and p-value, significance and the number of estimates.

The sizes are those of the benchmark (T = 10^4, max lag 5, k = 4, N = 9995);
only the surrogate count is reduced (S = 20, alpha = 0.1 for every test so
that S * alpha > 1) to keep the oracle's brute-force run to hours on a
workstation.  Usage:

    python tests/golden/make_network_fullsize.py var10 0
    python tests/golden/make_network_fullsize.py clm100 5
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from oracle import network as onet  # noqa: E402

T = 10000
SEED = 1
PARAMS = dict(k=4, max_lag_target=5, max_lag_sources=5, n_surr=20, alpha_max=0.1,
              alpha_min=0.1, alpha_omnibus=0.1, seed=SEED)
N_HEAD = 4


def series_for(workload: str) -> np.ndarray:
    gen = {"var10": synth.workload_var10, "clm100": synth.workload_clm100}[workload]
    return np.ascontiguousarray(gen(T=T, seed=SEED)["series"], dtype=np.float32)


def series_sha(s: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(s, dtype=np.float32).tobytes()).hexdigest()


def keys_sha(keys) -> str:
    """keys: [n_cand][S + 1] integers, candidate-major."""
    flat = ",".join(str(int(k)) for row in keys for k in row)
    return hashlib.sha256(flat.encode()).hexdigest()


def path_for(workload: str, target: int) -> str:
    return os.path.join(HERE, f"network_{workload}_T{T}_target{target}_S20.json")


def main(workload: str, target: int, n_threads: int | None = None) -> None:
    s = series_for(workload)
    p = onet.Params(**PARAMS, n_threads=n_threads)
    t0 = time.time()
    r = onet.infer_target(s, target, p)
    dt = time.time() - t0
    trace = []
    for stage, it, cands, keys, _null, pval, dec in r.trace:
        trace.append(dict(stage=int(stage), iter=int(it), cands=[list(map(int, c)) for c in cands],
                          n_cand=len(keys), keys_sha256=keys_sha(keys),
                          keys_head=[str(int(k)) for k in keys[0][:N_HEAD]],
                          p=pval, decision=(dec if isinstance(dec, bool)
                                            else [list(map(int, v)) for v in dec])))
    out = dict(workload=workload, T=T, seed=SEED, target=target, params=PARAMS,
               series_sha256=series_sha(s),
               result=dict(sel_target=[list(map(int, v)) for v in r.sel_target],
                           sel_sources=[list(map(int, v)) for v in r.sel_sources],
                           omnibus_tested=bool(r.omnibus_tested), omnibus_p=r.omnibus_p,
                           omnibus_cmi=float(r.omnibus_cmi).hex(), omnibus_key=str(r.omnibus_key),
                           significant=bool(r.significant), n_estimates=int(r.n_estimates)),
               trace=trace, oracle_seconds=round(dt, 1))
    with open(path_for(workload, target), "w") as f:
        json.dump(out, f, indent=1)
    print(f"{workload} target {target}: {r.n_estimates} estimates in {dt:.0f} s "
          f"-> {path_for(workload, target)}")


if __name__ == "__main__":
    nt = int(sys.argv[3]) if len(sys.argv) > 3 else None
    main(sys.argv[1], int(sys.argv[2]), nt)
