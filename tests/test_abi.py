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
            names |= set(re.findall(r"^\s*(?:mpdo_status|surr_status|const char\s*\*|long long|int)\s+(\w+)\s*\(", src,
                                    flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 35 and "surr_forward" in names and "mpdo_init" in names
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_without_a_gpu():
    from paper_2508_07610_gb300 import mpdo as M

    L = M.lib()
    assert L.mpdo_status_string(3) == b"process matrix is not completely positive"


def test_headers_compile_and_link_as_plain_c(tmp_path):
    """Both headers are usable from C99 (no C++ in the declarations), and a C caller links against
    the library with every entry point it names resolved."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest

        pytest.skip("no C compiler")
    path = B.build()
    src = tmp_path / "caller.c"
    src.write_text(
        '#include "mpdo.h"\n#include "surrogate.h"\n#include <stddef.h>\n'
        "int main(int argc, char** argv) {\n"
        "  (void)argv;\n"
        "  if (argc > 99) {  /* never taken: the calls only have to link */\n"
        "    mpdo_t h = NULL; mpdo_chan_t ch = NULL; surr_t s = NULL; double u[32] = {0};\n"
        "    mpdo_init(4, 8, 2, MPDO_FP32, NULL, &h);\n"
        "    channel_from_process_matrix(h, 1, u, 1e-12, &ch, NULL);\n"
        "    apply_1q(h, 0, u, ch); apply_2q(h, 0, u, ch); truncate_kraus(h, 0, 0, NULL);\n"
        "    expect(h, MPDO_EXPECT_TRACE, NULL, 0, u); channel_free(ch); mpdo_free(h);\n"
        "    surr_create(16, 256, 3, 2, 1024, 1ull, NULL, &s); surr_free(s);\n"
        "  }\n"
        "  return 0;\n"
        "}\n")
    exe = tmp_path / "caller"
    inc = os.path.join(ROOT, "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", inc, str(src), "-o", str(exe),
                        "-L", os.path.dirname(path), "-lmpdo", "-Wl,-rpath," + os.path.dirname(path)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_checked_library_builds_with_the_same_entry_points():
    """The address-checked debug build (-DMPDO_BOUNDS) compiles from the same sources and exports
    every declared entry point; it reports itself as checked, the release library as not, and the
    release stubs touch no device (they run here without a GPU)."""
    names = _declared()
    checked = ctypes.CDLL(B.build(bounds=True))
    missing = [n for n in sorted(names) if not hasattr(checked, n)]
    assert not missing, missing
    assert checked.mpdo_bounds_enabled() == 1
    release = ctypes.CDLL(B.build())
    assert release.mpdo_bounds_enabled() == 0
    fails, line = ctypes.c_ulonglong(7), ctypes.c_int(7)
    buf = ctypes.create_string_buffer(8)
    assert release.mpdo_bounds_read(ctypes.byref(fails), buf, 8, ctypes.byref(line), None, None) == 8  # ESTATE
    assert fails.value == 0 and line.value == 0 and buf.value == b""
    release.mpdo_bounds_register.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    assert release.mpdo_bounds_register(16, 64) == 0
