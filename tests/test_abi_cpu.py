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


def _header_text():
    txt = open(os.path.join(ROOT, "include", "shci.h")).read()
    return re.sub(r"/\*.*?\*/", "", txt, flags=re.S)


def test_header_constants_match_binding():
    """Every enumerator of include/shci.h has the binding's value."""
    from paper_1809_04600_gb300 import binding
    txt = _header_text()
    found = 0
    for body in re.findall(r"enum\s+shci_\w+\s*\{(.*?)\}", txt, flags=re.S):
        for name, val in re.findall(r"(SHCI_\w+)\s*=\s*(-?\d+)", body):
            assert getattr(binding, name) == int(val), name
            found += 1
    assert found >= 12


_CTYPES = {"int": ctypes.c_int, "int64_t": ctypes.c_int64, "double": ctypes.c_double}


def _header_struct(name):
    """[(field, ctypes type)] of `typedef struct { ... } name;` in the header."""
    txt = _header_text()
    body = re.search(r"typedef struct\s*\{([^{}]*)\}\s*%s\s*;" % name, txt, flags=re.S).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(const\s+)?(int64_t|uint64_t|int|double)\s+(.*)$", decl, flags=re.S)
        assert m, decl
        base = m.group(2)
        for item in m.group(3).split(","):
            item = item.strip()
            ptr = item.startswith("*")
            item = item.lstrip("*").strip()
            arr = re.match(r"(\w+)\s*\[(\d+)\]$", item)
            fname = arr.group(1) if arr else item
            t = ctypes.c_void_p if ptr else _CTYPES[base]
            if arr:
                t = t * int(arr.group(2))
            fields.append((fname, t))
    return fields


@pytest.mark.parametrize("name", ["shci_stats_t", "shci_batch_stats_t", "shci_system_desc", "shci_pt2_3step_t"])
def test_header_structs_match_binding(name):
    """The ctypes mirrors of the ABI structs have the header's fields, in order,
    with the same sizes (an appended or reordered field would otherwise shift
    every later one silently)."""
    from paper_1809_04600_gb300 import binding
    ours = getattr(binding, name)._fields_
    theirs = _header_struct(name)
    assert [f for f, _ in ours] == [f for f, _ in theirs]
    for (f, a), (_, b) in zip(ours, theirs):
        assert ctypes.sizeof(a) == ctypes.sizeof(b), f
