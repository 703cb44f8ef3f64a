"""fmnmf_loglik_noalloc: the log-likelihood entry point for callers that cannot allocate
device memory (a real-time audio thread that must not block on cudaMalloc, or an
application whose device memory belongs to its own pool allocator).  It keeps its working
memory in the library's static device array instead of allocating.

Checked through the C ABI against the context entry point (fmnmf_init / fmnmf_set_state /
fmnmf_loglik) on the same state, within the log-likelihood tolerance of the parity tests
(1e-5 of the sum of |terms| of Eq. 17), on two calls in a row with different states so
that the second call runs on the scratch the first one left behind; and directly against
the float64 oracle's Eq. 17 at the sizes of the small and the paper-scale mixtures.  The
size and alignment checks run on the host before any launch.  This file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest

from oracle import fastmnmf_oracle as O
from paper_1903_03237_gb300.synth import make_mixture, make_state

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def fm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf
    return fastmnmf


def _noalloc_ll(fm, X, W, H, G, Q):
    import torch
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    Xd, Wd, Hd, Gd, Qd = d(X), d(W), d(H), d(G), d(Q)
    ll = torch.zeros(1, dtype=torch.float64, device="cuda")
    F, T, M = X.shape
    N, K = W.shape[0], W.shape[1]
    stream = torch.cuda.current_stream()
    st = fm.lib().fmnmf_loglik_noalloc(Xd.data_ptr(), Wd.data_ptr(), Hd.data_ptr(), Gd.data_ptr(), Qd.data_ptr(),
                                       F, T, M, N, K, ll.data_ptr(), ctypes.c_void_p(stream.cuda_stream))
    assert st == fm.OK, fm.lib().fmnmf_last_error(None)
    torch.cuda.synchronize()
    return float(ll.item())


@pytest.mark.parametrize("shape", [(37, 150, 3, 3, 5), (257, 200, 2, 2, 8), (20, 64, 8, 3, 4)],
                         ids=["M3", "c0", "M8"])
def test_noalloc_loglik_matches_context(fm, shape):
    F, T, M, N, K = shape
    mix = make_mixture(F, T, M, N, K, 21)
    states = [make_state(F, T, M, N, K, 21)]
    ctx = fm.Context(mix.X, N, K, seed=5)
    states.append(ctx.get_state())          # a second, different state: the seeded init
    X64 = mix.X.astype(np.complex128)
    for W, H, G, Q in states:               # two calls in a row
        ctx.set_state(W, H, G, Q)
        ref = ctx.loglik()
        got = _noalloc_ll(fm, mix.X, W, H, G, Q)
        scale = O.loglik_terms_abs(X64, W.astype(float), H.astype(float), G.astype(float), Q.astype(complex))
        assert abs(got - ref) / scale < TOL, (got, ref)


@pytest.mark.parametrize("name", ["c0", "c1"])
def test_noalloc_loglik_matches_oracle(fm, name):
    from paper_1903_03237_gb300.synth import config_mixture, CONFIGS
    c = CONFIGS[name]
    F, T, M, N, K = c["F"], c["T"], c["M"], c["N"], c["K"]
    mix = config_mixture(name, seed=3)
    X64 = mix.X.astype(np.complex128)
    for s in (3, 4):                        # two calls in a row, different states
        W, H, G, Q = make_state(F, T, M, N, K, s)
        args = (W.astype(float), H.astype(float), G.astype(float), Q.astype(complex))
        ref = O.loglik(X64, *args)
        got = _noalloc_ll(fm, mix.X, W, H, G, Q)
        err = abs(got - ref) / O.loglik_terms_abs(X64, *args)
        print(name, "noalloc vs oracle", f"{err:.2e}")
        assert err < TOL, (got, ref)


def test_noalloc_rejects_oversize(fm):
    lib = fm.lib()
    one = ctypes.c_void_p(1 << 20)  # never dereferenced: the size check comes first
    st = lib.fmnmf_loglik_noalloc(one, one, one, one, one, 20000, 4, 2, 1, 1, one, None)
    assert st == fm.EINVAL
    assert b"scratch limit" in lib.fmnmf_last_error(None)
    # within the bin limit but beyond the TF-bin limit of the per-block partial sums
    st = lib.fmnmf_loglik_noalloc(one, one, one, one, one, 16384, 8000, 2, 1, 1, one, None)
    assert st == fm.EINVAL
    assert b"TF bins" in lib.fmnmf_last_error(None)


def test_noalloc_rejects_misaligned(fm):
    lib = fm.lib()
    one = ctypes.c_void_p(1 << 20)
    odd = ctypes.c_void_p((1 << 20) + 1)  # never dereferenced: the alignment check comes first
    st = lib.fmnmf_loglik_noalloc(odd, one, one, one, one, 16, 16, 2, 1, 1, one, None)
    assert st == fm.EINVAL
    assert b"misaligned" in lib.fmnmf_last_error(None)
