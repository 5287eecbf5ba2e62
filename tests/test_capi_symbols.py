"""The C-ABI library builds, loads and exports every entry point of include/hho.h (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hho.h")).read()
    return sorted(set(re.findall(r"^(?:hho_status|const char\*)\s+(\w+)\s*\(", src, re.M)))


def test_header_matches_binding_list():
    from paper_2009_13840_gb300 import hho
    assert _declared() == sorted(hho.SYMBOLS)


def test_library_builds_and_exports_symbols():
    from paper_2009_13840_gb300 import build, hho
    path = build.build()
    lib = hho.load(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_null_arguments_return_status_without_gpu():
    import ctypes as C
    from paper_2009_13840_gb300 import build, hho
    lib = hho.load(build.build())
    out = C.c_void_p()
    assert lib.hho_setup(None, 1, 0, None, C.byref(out)) == 1   # HHO_ERR_ARG, context with message
    assert b"null mesh" in lib.hho_last_error(out)
    assert lib.hho_destroy(out) == 0
    assert lib.hho_ndof(None, 0, None) == 1
    assert lib.hho_destroy(None) == 0


def test_binding_refuses_mistyped_or_short_buffers():
    """The binding checks dtype and length before a pointer reaches the library."""
    torch = pytest.importorskip("torch")
    from paper_2009_13840_gb300 import hho
    x = torch.zeros(10, dtype=torch.float32)
    with pytest.raises(TypeError):
        hho._vec(x, torch.float64, 10, "x")
    with pytest.raises(ValueError):
        hho._vec(torch.zeros(9, dtype=torch.float64), torch.float64, 10, "x")
    with pytest.raises(ValueError):
        hho._vec(None, torch.float64, 10, "x")
    with pytest.raises(ValueError):  # right type and size, but not a CUDA tensor
        hho._vec(torch.zeros(10, dtype=torch.float64), torch.float64, 10, "x")
