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


def test_front_end_host_side():
    # frame count against the oracle's, and argument errors caught before any device call
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf as fm
    from oracle import fastmnmf_oracle as O
    for S, L, hop in [(1, 16, 1), (16, 16, 4), (17, 16, 4), (5000, 1024, 256), (1024, 1024, 256),
                      (164608, 1024, 256), (777, 64, 16), (10, 4096, 4096)]:
        assert fm.stft_frames(S, L, hop) == O.stft_frames(S, L, hop)
    lib = fm.lib()
    T = ctypes.c_int()
    assert lib.fmnmf_stft_frames(100, 1000, 250, ctypes.byref(T)) == fm.EINVAL      # L not a power of two
    assert lib.fmnmf_stft_frames(100, 8192, 256, ctypes.byref(T)) == fm.EINVAL      # L too large
    assert lib.fmnmf_stft_frames(100, 1024, 0, ctypes.byref(T)) == fm.EINVAL
    assert lib.fmnmf_stft_frames(100, 1024, 2048, ctypes.byref(T)) == fm.EINVAL     # hop > L
    assert lib.fmnmf_stft_frames(0, 1024, 256, ctypes.byref(T)) == fm.EINVAL
    assert lib.fmnmf_stft(None, 2, 100, 64, 16, None, None) == fm.EINVAL
    assert lib.fmnmf_istft(None, 1, 33, 4, 2, 100, 64, 16, None, None) == fm.EINVAL  # NULL
    assert lib.fmnmf_istft(None, 1, 32, 4, 2, 100, 64, 16, None, None) == fm.EINVAL  # F != L/2 + 1
    assert b"F" in lib.fmnmf_last_error(None)
    assert lib.fmnmf_istft(None, 1, 33, 4, 2, 200, 64, 16, None, None) == fm.EINVAL  # frames too short
    assert lib.fmnmf_init_spectral(None) == fm.EINVAL


def test_dp_host_side():
    # FastMNMF-DP defaults (the paper's D = 16, 30 proposals, eps = 1e-4) and the argument errors
    # the C ABI reports before it touches a device
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf as fm
    lib = fm.lib()
    o = fm.DPOpts()
    assert lib.fmnmf_dp_default_opts(ctypes.byref(o)) == fm.OK
    assert (o.D, o.Hd, o.n_proposals, o.normalise) == (16, 128, 30, 1) and o.eps == ctypes.c_float(1e-4).value
    X = (ctypes.c_float * 64)()
    dp = ctypes.c_void_p()
    for field, value, word in (("Hd", 10, b"Hd"), ("D", 0, b"D"), ("n_proposals", -1, b"n_proposals"),
                               ("eps", -1.0, b"eps")):
        bad = fm.DPOpts()
        lib.fmnmf_dp_default_opts(ctypes.byref(bad))
        setattr(bad, field, value)
        assert lib.fmnmf_dp_create(ctypes.byref(dp), ctypes.addressof(X), 0, 4, 4, 2, 2, 2, ctypes.byref(bad)) == fm.EINVAL
        assert word in lib.fmnmf_dp_last_error(None)
    assert lib.fmnmf_dp_create(ctypes.byref(dp), ctypes.addressof(X), 0, 4, 4, 2, 9, 2, None) == fm.EINVAL   # N > 8
    assert lib.fmnmf_dp_create(ctypes.byref(dp), ctypes.addressof(X), 0, 4, 4, 2, 3, 200, None) == fm.EINVAL  # (N-1)K > 256
    assert lib.fmnmf_dp_create(None, ctypes.addressof(X), 0, 4, 4, 2, 2, 2, None) == fm.EINVAL
    for call in (lambda: lib.fmnmf_dp_set_decoder(None, None, None, None, None),
                 lambda: lib.fmnmf_dp_iterate(None, 1, None, None, 0),
                 lambda: lib.fmnmf_dp_sync(None)):
        assert call() == fm.EINVAL
    assert lib.fmnmf_dp_destroy(None) == fm.OK
