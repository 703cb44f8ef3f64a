"""The C-ABI library builds, loads and exports every function include/fastmnmf.h declares
(no GPU needed: nothing here calls into the device)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fmnmf_\w+)\s*\(", src))
    return names


def test_library_exports_declared_symbols():
    from paper_1903_03237_gb300.build import build
    path = build()
    lib = ctypes.CDLL(path)
    decl = _declared()
    assert "fmnmf_init" in decl and "fmnmf_iterate" in decl and "fmnmf_separate" in decl
    missing = [n for n in sorted(decl) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf
    assert set(fastmnmf.EXPORTS) == _declared()


def test_host_side_argument_errors():
    # Argument validation happens on the host before any device call.
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf as fm
    lib = fm.lib()
    ctx = ctypes.c_void_p()
    X = (ctypes.c_float * 8)()
    assert lib.fmnmf_init(ctypes.byref(ctx), ctypes.addressof(X), 0, 2, 2, 9, 1, 1, 0, None) == fm.EINVAL
    assert b"M" in lib.fmnmf_last_error(None)
    assert lib.fmnmf_init(ctypes.byref(ctx), None, 0, 2, 2, 2, 1, 1, 0, None) == fm.EINVAL
    assert lib.fmnmf_iterate(None, 1) == fm.EINVAL
    o = fm.default_opts()
    assert o.update_mask == 15 and o.normalise == 1 and o.precision == 0
