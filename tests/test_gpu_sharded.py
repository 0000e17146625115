"""GPU: network inference through the target-sharding helper.  With one
process the helper runs every target in one shard and applies the FDR step
on the host after the gather; the result must equal te_network_infer with
its own FDR step (two implementations of the same rule)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_one_rank_sharded_inference_equals_library_fdr():
    import paper_1902_06828_gb300 as te
    from paper_1902_06828_gb300.shard import infer_network_sharded
    ctx = te.Context(0)
    try:
        x, _, _ = synth.var_er(n=5, p=0.35, T=400, seed=4, lo=0.4, hi=0.7, max_lag=3)
        s = synth.standardise_jitter(x, 4)
        data = te.te_data_create(ctx, s)
        kw = dict(k=4, max_lag_target=3, max_lag_sources=3, n_surr=30, alpha_max=0.1,
                  alpha_min=0.1, alpha_omnibus=0.1, seed=21)
        for a in (0.1, 0.01):
            lib = te.te_network_infer(ctx, data, fdr=True, alpha_fdr=a, **kw)
            sh = infer_network_sharded(ctx, data, 5, None, fdr=True, alpha_fdr=a, **kw)
            np.testing.assert_array_equal(sh["adjacency"], lib["adjacency"])
            np.testing.assert_array_equal(sh["min_lag"], lib["min_lag"])
            for u, v in zip(sh["targets"], lib["targets"]):
                assert u["target"] == v["target"]
                assert u["sel_sources"] == v["sel_sources"]
                assert u["significant"] == v["significant"]
            assert sh["n_estimates"] == lib["n_estimates"]
            assert sh["theiler"] == lib["theiler"]
    finally:
        ctx.close()
