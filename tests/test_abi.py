"""The C-ABI library builds for sm_103a, loads, and exports every symbol its
header declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pwa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(pwa_[a-z_]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pwa_create", "pwa_nll", "pwa_grad", "pwa_hvp", "pwa_newton_cg_fit", "pwa_destroy",
                     "pwa_last_error"):
        assert required in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2403_09225_b300 import binding, build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(binding.EXPORTS)


def test_binding_refuses_a_missing_library(tmp_path):
    from paper_2403_09225_b300 import binding
    with pytest.raises(RuntimeError):
        binding.load_library(str(tmp_path / "nope.so"))
