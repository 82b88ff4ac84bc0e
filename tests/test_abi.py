"""The C-ABI library builds, loads and exports every symbol include/rsort.h
declares (no GPU needed; no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(rsort_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1606_08766_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rsort_create", "rsort_destroy", "rsort_strerror", "rsort_sort",
                 "rsort_partition", "rsort_check"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (rsort_[a-z0-9_]+)$", out, flags=re.M))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_answers_without_a_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.rsort_strerror.restype = ctypes.c_char_p
    lib.rsort_strerror.argtypes = [ctypes.c_int32]
    assert lib.rsort_strerror(0) == b"ok"
    assert b"invalid" in lib.rsort_strerror(-1)
    lib.rsort_sort.restype = ctypes.c_int32
    # a NULL context is rejected before any CUDA call
    assert lib.rsort_sort(None, 0, None, None, None, ctypes.c_uint64(0), ctypes.c_uint32(1),
                          ctypes.c_uint64(1), None, None) == -1
    lib.rsort_destroy.restype = ctypes.c_int32
    assert lib.rsort_destroy(None) == 0


def test_binding_has_no_cpu_fallback(monkeypatch, tmp_path):
    import paper_1606_08766_gb300.binding as b
    monkeypatch.setattr(b, "_lib", None)
    monkeypatch.setattr(b._build, "LIB", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        b.load_library(build_if_missing=False)
