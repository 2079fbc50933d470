"""The C-ABI library builds, loads and exports every entry point that
include/ebvisc.h declares (no compute calls: this runs without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ebvisc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ebv_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1905_07392_gb300 import build_lib
    path = build_lib.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("ebv_create", "ebv_build_geometry", "ebv_update_viscosity", "ebv_solve_viscous",
              "ebv_solve_projection", "ebv_solve_mac", "ebv_advance", "ebv_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1905_07392_gb300 import ebvisc
    assert sorted(ebvisc.EXPORTS) == _declared()


def test_create_without_device_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1905_07392_gb300 import ebvisc
    with pytest.raises(ebvisc.EbvError):
        ebvisc.Solver((8, 8, 8), 1.0 / 8, stream=type("S", (), {"cuda_stream": 0})())
