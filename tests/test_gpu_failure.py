"""Failure detection without a GPU fault.

* The tensor-core kernels of the mixed form (tcgen05 GEMM, V_fm and g~ kernels) bound every
  mbarrier wait.  A test-only limit (the FMNMF_TEST_WAIT_LIMIT environment variable, read by
  fmnmf_init and fmnmf_iterate) shortens their consumer waits and sends one of them to an
  mbarrier nothing arrives at, so that the timeout path runs: the CTA leaves its loop, drains
  the copies and MMAs it issued (full bound), reports ST_TIMEOUT and frees its TMEM.  The
  context then reports FMNMF_ETIMEOUT; after fmnmf_set_state (which clears the error word)
  the same context computes a correct iteration again.
* Host-side rejections: a singular Q_f (a vanishing row; the pivot test is relative, 1e-30
  of the largest entry) gives FMNMF_ESINGULAR, a NaN in W FMNMF_EINVAL (the documented
  argument check), and both leave the context usable.
"""
import numpy as np
import pytest

from oracle import fastmnmf_oracle as O
from paper_1903_03237_gb300.synth import make_mixture, make_state

from tests._parity import rel, ll_rel, as64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf
    return fastmnmf


def _one_iteration_errors(ctx, mix, W, H, G, Q):
    ctx.set_state(W, H, G, Q)
    ctx.iterate(1)
    ll = ctx.loglik()
    Wg, Hg, Gg, Qg = ctx.get_state()
    X64 = mix.X.astype(np.complex128)
    Wr, Hr, Gr, Qr, tr = O.iterate(X64, *as64(W, H, G, Q), n_iter=1)
    return {"W": rel(Wg, Wr), "H": rel(Hg, Hr), "G": rel(Gg, Gr), "Q": rel(Qg, Qr),
            "LL": ll_rel(ll, tr[-1], X64, Wr, Hr, Gr, Qr)}


@pytest.mark.parametrize("shape", [(37, 152, 3, 3, 5), (29, 151, 3, 2, 6)], ids=["tma", "no-tma"])
def test_tensor_core_wait_timeout_reports_and_recovers(fm, monkeypatch, shape):
    # (29, 151, 3): T*M odd, so the V_fm and g~ kernels load their inputs with the threads
    # (the path whose formation warps meet at a named barrier)
    F, T, M, N, K = shape
    mix = make_mixture(F, T, M, N, K, 1)
    W, H, G, Q = make_state(F, T, M, N, K, 1)
    ctx = fm.Context(mix.X, N, K, precision=fm.PREC_BF16)
    monkeypatch.setenv("FMNMF_TEST_WAIT_LIMIT", "64")
    ctx.iterate(2)
    with pytest.raises(fm.FastMNMFError) as e:
        ctx.sync()
    assert e.value.status == fm.ETIMEOUT, str(e.value)
    assert "timed out" in str(e.value)
    # the error stays until the state is set again
    with pytest.raises(fm.FastMNMFError):
        ctx.loglik()
    monkeypatch.delenv("FMNMF_TEST_WAIT_LIMIT")
    err = _one_iteration_errors(ctx, mix, W, H, G, Q)
    print("after timeout", shape, {k: f"{v:.2e}" for k, v in err.items()})
    assert max(err.values()) < 1e-3, err
    # and a new context on the device works as well
    ctx2 = fm.Context(mix.X, N, K, precision=fm.PREC_BF16)
    err2 = _one_iteration_errors(ctx2, mix, W, H, G, Q)
    assert max(err2.values()) < 1e-3, err2


def test_singular_q_is_reported(fm):
    F, T, M, N, K = 10, 40, 3, 2, 3
    mix = make_mixture(F, T, M, N, K, 2)
    W, H, G, Q = make_state(F, T, M, N, K, 2)
    ctx = fm.Context(mix.X, N, K)
    Qs = Q.copy()
    Qs[4, 2] = 0                 # a vanishing row: Q_4 is singular
    with pytest.raises(fm.FastMNMFError) as e:
        ctx.set_state(W, H, G, Qs)
    assert e.value.status == fm.ESINGULAR
    err = _one_iteration_errors(ctx, mix, W, H, G, Q)   # a good state clears it
    assert max(err.values()) < 1e-5, err


def test_nonfinite_state_is_rejected(fm):
    F, T, M, N, K = 10, 40, 3, 2, 3
    mix = make_mixture(F, T, M, N, K, 3)
    W, H, G, Q = make_state(F, T, M, N, K, 3)
    ctx = fm.Context(mix.X, N, K)
    Wn = W.copy()
    Wn[1, 2, 3] = np.nan
    with pytest.raises(fm.FastMNMFError) as e:
        ctx.set_state(Wn, H, G, Q)
    assert e.value.status == fm.EINVAL
    err = _one_iteration_errors(ctx, mix, W, H, G, Q)
    assert max(err.values()) < 1e-5, err
