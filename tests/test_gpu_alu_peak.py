"""GPU: the measured ceiling of the KSG kernel's counted instruction patterns
(te_alu_peak).  A probe's rate cannot exceed the FP32 issue limit of the GPU
(counted operations are at most the instructions issued), and the plain-add
probe reaches a sizeable part of that limit."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_1902_06828_gb300 as te
    ctx = te.Context(0)
    props = torch.cuda.get_device_properties(0)
    yield te, ctx, props.multi_processor_count
    ctx.close()


def test_alu_peak_rates_are_bounded_by_issue(env):
    te, ctx, sms = env
    # 4 schedulers x 32 lanes per SM per clock, at most 2.2 GHz
    issue_limit = sms * 128 * 2.2e9
    add = te.te_alu_peak(ctx, "fadd")
    knn = te.te_alu_peak(ctx, "knn")
    cnt = te.te_alu_peak(ctx, "count")
    assert 0.3 * issue_limit < add <= issue_limit
    assert 0 < knn <= 1.05 * add
    assert 0 < cnt <= 1.05 * add


def test_alu_peak_rejects_unknown_kind(env):
    import ctypes as C
    te, ctx, _ = env
    out = C.c_double()
    with pytest.raises(te.TEError, match="TE_EINVAL"):
        te._check(ctx._h, ctx._lib.te_alu_peak(ctx._h, 3, C.byref(out)))
