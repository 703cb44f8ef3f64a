"""The float-float primitives of the IP update (csrc/fm_df64.cuh) against float64, on the GPU.

Each primitive runs on log-uniform inputs through a test-only probe (tests/df64_probe.cu,
compiled here with nvcc) and is compared with the float64 value of the same float-float
inputs.  Bounds, with u = 2^-24:
  df_add  (accurate double-word addition)   3u^2 / (1 - 4u)   relative (Joldes, Muller &
                                                               Popescu 2017, Thm. 3.1)
  df_mul  (double-word times double-word)   5u^2               relative (ibid., Alg. 11)
  df_rcp  (one Newton step on RN(1/hi))     12u^2              relative (derived: (2u)^2 from
                                                               the seed, 2u^2 the residual,
                                                               3u^2 the final addition)
  df_sqrt (s + (x - s^2)/(2s))               8u^2               relative
  df_rsqrt (hardware estimate, one Newton   1e-13 relative inside [1e-30, 1e30] (the header's
           step in float-float)                                figure); outside it (the
                                                               fallback through df_sqrt and
                                                               df_rcp) 1e-13 + 8 * 2^-149 / x:
                                                               below 1e-30 the low parts are
                                                               float subnormals, whose spacing
                                                               2^-149 limits any float-float
                                                               value there
  df_logf (logf(hi) + lo/hi)                 2^-22 |log x| + 1e-15 absolute (logf's 1 ulp)
The range fallback of df_rsqrt (outside [1e-30, 1e30] it goes through df_sqrt and df_rcp)
is exercised on both sides.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U = 2.0 ** -24
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    out = str(tmp_path_factory.mktemp("df64") / "libdf64probe.so")
    csrc = os.path.join(os.path.dirname(HERE), "paper_1903_03237_gb300", "csrc")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                    "-Xcompiler", "-fPIC", "-I" + csrc, os.path.join(HERE, "df64_probe.cu"), "-o", out],
                   check=True, capture_output=True)
    lib = ctypes.CDLL(out)
    fn = lib.df64_probe
    P = ctypes.POINTER(ctypes.c_double)
    fn.argtypes = [ctypes.c_int, P, P, ctypes.c_int, P, P, P]
    fn.restype = ctypes.c_int

    def run(op, a, b=None):
        a = np.ascontiguousarray(a, np.float64)
        b = np.ascontiguousarray(np.ones_like(a) if b is None else b, np.float64)
        o, sa, sb = np.empty_like(a), np.empty_like(a), np.empty_like(a)
        p = lambda x: x.ctypes.data_as(P)
        assert fn(op, p(a), p(b), a.size, p(o), p(sa), p(sb)) == 0
        return o, sa, sb
    return run


def _logu(rng, lo, hi, n):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def test_df_add(probe):
    rng = np.random.default_rng(1)
    a = _logu(rng, 1e-15, 1e15, 20000) * rng.choice([-1, 1], 20000)
    b = a * (1 + rng.uniform(-1e-3, 1e-3, a.size)) * rng.choice([-1, 1], a.size)   # cancellation too
    b[::3] = _logu(rng, 1e-15, 1e15, b[::3].size)
    o, sa, sb = probe(0, a, b)
    ref = sa + sb
    nz = ref != 0
    err = np.max(np.abs(o[nz] - ref[nz]) / np.abs(ref[nz]))
    print("df_add", err / U ** 2, "u^2")
    assert err <= 3 * U * U / (1 - 4 * U)


def test_df_mul(probe):
    rng = np.random.default_rng(2)
    a = _logu(rng, 1e-15, 1e15, 20000) * rng.choice([-1, 1], 20000)
    b = _logu(rng, 1e-15, 1e15, 20000)
    o, sa, sb = probe(1, a, b)
    ref = sa * sb
    err = np.max(np.abs(o - ref) / np.abs(ref))
    print("df_mul", err / U ** 2, "u^2")
    assert err <= 5 * U * U


def test_df_rcp(probe):
    rng = np.random.default_rng(3)
    a = _logu(rng, 1e-30, 1e30, 20000)
    o, sa, _ = probe(2, a)
    err = np.max(np.abs(o * sa - 1.0))
    print("df_rcp", err / U ** 2, "u^2")
    assert err <= 12 * U * U


def test_df_sqrt(probe):
    rng = np.random.default_rng(4)
    a = _logu(rng, 1e-30, 1e30, 20000)
    o, sa, _ = probe(3, a)
    ref = np.sqrt(sa)
    err = np.max(np.abs(o - ref) / ref)
    print("df_sqrt", err / U ** 2, "u^2")
    assert err <= 8 * U * U


@pytest.mark.parametrize("lo,hi", [(1e-30, 1e30), (1e-36, 1e-30), (1e30, 1e36)], ids=["inside", "below", "above"])
def test_df_rsqrt(probe, lo, hi):
    rng = np.random.default_rng(5)
    a = _logu(rng, lo, hi, 20000)
    o, sa, _ = probe(4, a)
    ref = 1.0 / np.sqrt(sa)
    rel = np.abs(o - ref) / ref
    bound = 1e-13 + 8 * 2.0 ** -149 / sa
    print("df_rsqrt", (lo, hi), rel.max(), (rel / bound).max())
    assert np.all(rel <= bound)


def test_df_logf(probe):
    rng = np.random.default_rng(6)
    a = np.concatenate([_logu(rng, 1e-30, 1e30, 20000), 1 + rng.uniform(-1e-3, 1e-3, 2000)])
    o, sa, _ = probe(5, a)
    ref = np.log(sa)
    err = np.abs(o - ref) / (2.0 ** -22 * np.abs(ref) + 1e-15)
    print("df_logf", err.max())
    assert err.max() <= 1.0
