"""The C ABI: the shared library builds for sm_103a, loads, and exports every entry
point that include/*.h declares (no GPU needed, no compute calls)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(mlswe_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol(mlswe_lib):
    lib = ctypes.CDLL(mlswe_lib.LIB_PATH)
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_raises_without_library(tmp_path, monkeypatch):
    import paper_1803_01450_gb300 as pkg
    monkeypatch.setattr(pkg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    try:
        pkg.lib()
    except pkg.MLSWEError as e:
        assert e.status == 9
    else:
        raise AssertionError("loading a missing library must fail")


def test_create_rejects_bad_config_without_gpu(mlswe_lib):
    """Argument validation happens before any CUDA call."""
    L = mlswe_lib.lib()
    cfg = mlswe_lib.Config(M=3).to_c()
    dom = (mlswe_lib._Domain * 1)(mlswe_lib._Domain(0, 0, 1, 1, 10, 10))
    h = ctypes.c_void_p()
    assert L.mlswe_create_hierarchy(ctypes.byref(cfg), 1, dom, None, None, ctypes.byref(h)) == 1
