"""The C-ABI library builds for sm_103a, loads, and exports every function include/dks.h declares
(no GPU needed; no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|void|const char\s*\*)\s*(dks_\w+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_1211_1446_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_export():
    import paper_1211_1446_gb300 as P
    assert set(P.EXPORTS) == set(_declared())


def test_strerror_without_gpu():
    import paper_1211_1446_gb300 as P
    lib = P.load_library()
    assert lib.dks_strerror(-8).decode().startswith("planewave sphere")
    assert lib.dks_strerror(0).decode() == "ok"
