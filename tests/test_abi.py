"""The C-ABI library builds for sm_103a, loads, and exports every function include/mpdo.h declares
(no GPU needed: nothing here calls into CUDA)."""
import ctypes
import os
import re

from paper_2508_07610_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^\s*(?:mpdo_status|const char\s*\*|long long)\s+(\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 25
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_without_a_gpu():
    from paper_2508_07610_gb300 import mpdo as M

    L = M.lib()
    assert L.mpdo_status_string(3) == b"process matrix is not completely positive"
