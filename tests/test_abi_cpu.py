"""CPU-only checks of the boundary: the library builds, loads without a GPU and
exports every symbol include/te_ksg.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "te_ksg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:te_status|void|const char \*)\s*\*?\s*(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    from paper_1902_06828_gb300 import _abi
    lib = _abi.load()
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(_abi.SIGNATURES), set(names) - set(_abi.SIGNATURES)


def test_library_is_in_tree_and_built_for_sm103a():
    from paper_1902_06828_gb300 import _abi, build
    path = _abi.library_path()
    assert path.startswith(ROOT)
    assert os.path.exists(path)
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_context_creation_fails_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    import paper_1902_06828_gb300 as te
    with pytest.raises(te.TEError):
        te.Context(0)


def test_null_arguments_rejected_without_touching_the_gpu():
    from paper_1902_06828_gb300 import _abi
    lib = _abi.load()
    assert lib.te_ctx_create(0, None) == _abi.TE_EINVAL
    assert lib.te_last_error(None) == b"no context"
    lib.te_ctx_destroy(None)
    lib.te_data_destroy(None)
    lib.te_network_result_free(None)


def test_network_infer_rejects_unknown_modes_before_any_call():
    import paper_1902_06828_gb300 as te
    for kw in (dict(estimator="kraskov"), dict(surr_mode="shuffle")):
        with pytest.raises(ValueError):
            te.te_network_infer(None, None, **kw)
