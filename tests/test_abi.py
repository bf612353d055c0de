"""The C ABI: libluda.so builds for sm_103a, loads without a GPU, and exports every
function include/luda.h declares (no compute call is made here)."""
import ctypes as C
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "luda.h")) as f:
        text = f.read()
    return re.findall(r"LUDA_API\s+[\w\s\*]+?\b(luda_\w+)\s*\(", text)


def _lib():
    from paper_2004_03054_b300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_entry_points():
    names = set(_declared())
    for n in ("luda_compact", "luda_compact_device", "luda_batch_compact_device", "luda_plan_create",
              "luda_plan_run", "luda_plan_outputs", "luda_plan_destroy", "luda_build", "luda_build_device",
              "luda_outputs_free", "luda_strerror", "luda_last_error_detail", "luda_check_table_noalloc"):
        assert n in names, n


def test_library_exports_every_declared_symbol():
    lib = _lib()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_only_luda_symbols_are_exported():
    import subprocess
    from paper_2004_03054_b300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.build()], capture_output=True, text=True).stdout
    names = [ln.split()[-1] for ln in out.splitlines() if ln.strip()]
    ours = [n for n in names if not n.startswith("_") and n not in ("main",)]
    assert all(n.startswith("luda_") for n in ours), [n for n in ours if not n.startswith("luda_")][:10]


def test_non_compute_calls():
    lib = _lib()
    lib.luda_strerror.restype = C.c_char_p
    lib.luda_version.restype = C.c_char_p
    assert lib.luda_strerror(-2) == b"corrupt input table"
    assert b"sm_103a" in lib.luda_version()


def test_binding_fails_loudly_without_the_library(tmp_path, monkeypatch):
    from paper_2004_03054_b300 import luda
    monkeypatch.setattr(luda, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(luda, "_lib", None)
    try:
        luda.lib()
    except RuntimeError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("expected a loud failure")
