"""The C-ABI library loads and exports every symbol include/paro.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "paro.h")).read()
    return sorted(set(re.findall(r"^(?:int|void|const char\*)\s+(paro_[a-z_0-9]+)\s*\(", src, re.M)))


def test_header_and_binding_agree():
    from paper_1702_04045_gb300 import paro
    assert _declared() == sorted(paro.EXPORTS)


def test_library_exports_every_declared_symbol():
    from paper_1702_04045_gb300 import build, paro
    if not os.path.exists(paro.LIB_PATH):
        try:
            build.build()
        except RuntimeError as e:  # no nvcc on this machine
            pytest.skip(str(e))
    lib = paro.load_library()
    for name in _declared():
        assert hasattr(lib, name), name


def test_no_cpu_fallback_without_gpu():
    import torch
    from paper_1702_04045_gb300 import paro
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        paro.Context([10, 0, 0, 0, 10, 0, 0, 0, 10], [[0, 0, 0]], 2.0, 2, 1)
