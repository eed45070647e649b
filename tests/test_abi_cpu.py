"""CPU checks of the C ABI library: it loads without a GPU and exports every
function declared in include/s2dw.h (no compute calls)."""
import os
import re

import pytest

from paper_1308_5706_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "s2dw.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(s2dw_[a-z_]+)\s*\(", txt)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("s2dw_plan", "s2dw_analysis", "s2dw_synthesis", "s2dw_kernels", "s2dw_plan_destroy",
              "s2dw_query", "s2dw_analysis_batch", "s2dw_synthesis_batch", "s2dw_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(B.LIB_PATH):
        pytest.skip("libs2dw.so not built")
    lib = B.lib()
    for n in _declared():
        assert hasattr(lib, n), n
        assert n in B._SIGNATURES, f"binding lacks {n}"


def test_strerror_and_argument_validation_without_gpu():
    if not os.path.exists(B.LIB_PATH):
        pytest.skip("libs2dw.so not built")
    assert B.s2dw_strerror(B.S2DW_OK) == "ok"
    assert B.s2dw_strerror(B.S2DW_EINVAL) == "invalid argument"
    # argument checks happen before any CUDA call
    # invalid requests: no transform exists for them
    for args in ((1, 1, 2.0, 0, B.S2DW_FP64), (32, 0, 2.0, 0, B.S2DW_FP64), (4, 5, 2.0, 0, B.S2DW_FP64),
                 (32, 3, 1.0, 0, B.S2DW_FP64), (32, 3, 2.0, 0, 0), (32, 3, 2.0, 0, B.S2DW_FP64 | B.S2DW_MIXED),
                 (32, 3, float("nan"), 0, B.S2DW_FP64), (32, 3, 2.0, 6, B.S2DW_FP64),
                 (32, 3, 2.0, -1, B.S2DW_FP64)):
        with pytest.raises(B.S2dwError) as ei:
            B.s2dw_plan(*args)
        assert ei.value.status == B.S2DW_EINVAL, args
    # valid requests beyond this build's limits (L <= 2048, N <= 8)
    for args in ((4096, 3, 2.0, 0, B.S2DW_MIXED), (32, 9, 2.0, 0, B.S2DW_FP64)):
        with pytest.raises(B.S2dwError) as ei:
            B.s2dw_plan(*args)
        assert ei.value.status == B.S2DW_ENOTSUP, args
