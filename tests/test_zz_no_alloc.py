"""cmi_ksg_static, the allocation-free estimate, against cmi_ksg.

cmi_ksg_static exists for callers that cannot allocate device memory (a host
framework that already owns the device through its own pool allocator, a
process with a fixed device-memory budget, a loop that cannot take the device
synchronisation of cudaMalloc).  It keeps its scratch in a static device array
shared by all calls, so it is checked on consecutive calls, through the C ABI,
against the context-based entry point.  This file is collected last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REL, ABS = 1e-9, 1e-12   # the tolerance of the GPU parity tests


def _close(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.all(np.abs(a - b) <= REL * np.abs(b) + ABS)


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    import paper_1902_06828_gb300 as te
    ctx = te.Context(0)
    yield torch, te, ctx
    ctx.close()


def test_static_matches_cmi_ksg_on_consecutive_calls(env):
    torch, te, ctx = env
    w = synth.workload_chain3(T=1000, seed=1)
    data = te.te_data_create(ctx, w["series"])
    dev = torch.from_numpy(w["series"]).cuda()
    # the same call twice, then a different one: each must match cmi_ksg
    for seed in (11, 11, 12):
        kw = dict(k=4, max_lag=2, n_surr=200, seed=seed, stream_tag=5)
        ref, rkeys = te.cmi_ksg(ctx, data, w["x"], w["y"], w["z"], return_keys=True, **kw)
        got, gkeys = te.cmi_ksg_static(dev, w["x"], w["y"], w["z"], return_keys=True, **kw)
        assert gkeys == rkeys
        assert _close(got, ref)


def test_static_multidim_x_runtime_k_and_stream(env):
    torch, te, ctx = env
    rng = np.random.default_rng(3)
    s = rng.normal(size=(5, 700))
    s[1, 1:] += 0.5 * s[0, :-1]
    s = synth.standardise_jitter(s, 3)
    data = te.te_data_create(ctx, s)
    dev = torch.from_numpy(s).cuda()
    stream = torch.cuda.Stream()
    for x, k in (([(0, 1), (2, 2)], 4), ([(0, 1)], 6), ([(0, 1), (3, 1)], 5)):
        kw = dict(k=k, max_lag=3, n_surr=17, seed=2, stream_tag=9)
        ref = te.cmi_ksg(ctx, data, x, [(1, 0)], [(1, 1), (4, 3)], **kw)
        for _ in range(2):
            got = te.cmi_ksg_static(dev, x, [(1, 0)], [(1, 1), (4, 3)], stream=stream, **kw)
            assert _close(got, ref)


def test_static_rejects_sizes_beyond_its_scratch(env):
    torch, te, ctx = env
    dev = torch.zeros((3, 10000), dtype=torch.float32, device="cuda")
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.cmi_ksg_static(dev, [(0, 1)], [(1, 0)], [], k=4, max_lag=1, n_surr=5000)
    with pytest.raises(te.TEError, match="TE_EINVAL"):   # 4 S N bytes > 32 MiB
        te.cmi_ksg_static(dev, [(0, 1)], [(1, 0)], [], k=4, max_lag=1, n_surr=1000)


def test_static_rejects_series_not_on_the_current_device(env):
    torch, te, ctx = env
    import ctypes as C
    from paper_1902_06828_gb300 import _abi
    lib = _abi.load()
    host = np.zeros((3, 1000), np.float32)
    xv = (_abi.TeVar * 1)(_abi.TeVar(0, 1))
    yv = (_abi.TeVar * 1)(_abi.TeVar(1, 0))
    p = _abi.KsgParams(4, 0, 1, 3, 0, 0)
    out = np.zeros(4, np.float64)
    # a host pointer is refused by the C entry point before any launch
    st = lib.cmi_ksg_static(C.c_void_p(host.ctypes.data), 3, 1000, xv, 1, yv, 1, None, 0,
                            C.byref(p), None, out.ctypes.data, None)
    assert st == _abi.TE_EINVAL
    # a non-contiguous tensor is refused by the binding instead of being copied
    dev = torch.zeros((1000, 3), dtype=torch.float32, device="cuda").t()
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te.cmi_ksg_static(dev, [(0, 1)], [(1, 0)], [], k=4, max_lag=1, n_surr=3)
