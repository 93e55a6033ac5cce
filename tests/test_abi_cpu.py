"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every symbol include/shci.h declares; calls that
cannot reach a device fail with a status code instead of crashing."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "shci.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(shci_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_04600_gb300 import build_lib
    path = build_lib.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ["shci_load_integrals", "shci_build_connectivity", "shci_sigma", "shci_davidson"]:
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1809_04600_gb300 import binding
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert sorted(binding.EXPORTED) == sorted(declared_symbols())


def test_binding_loads_and_marshals(lib):
    from paper_1809_04600_gb300 import binding
    L = binding.load_library()
    assert L.shci_last_error(None) is not None


def test_no_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1809_04600_gb300 import binding
    with pytest.raises(binding.ShciError):
        binding.shci_create(0)
    # null context is rejected without touching a device
    L = binding.load_library()
    assert L.shci_sigma(None, 1, None, None, 0) == binding.SHCI_ERR_INVALID
    assert L.shci_extend_connectivity(None, 1, None, 0, 0.2, None) == binding.SHCI_ERR_INVALID
