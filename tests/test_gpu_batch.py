"""Batched form: several mixtures of uneven shapes (and precisions) iterated by one CUDA
graph launch.  Each member must end bit-identical to the same context iterated alone with
the same iterations per call (the fused schedule's mu normalisation runs at the end of each
call, so call boundaries are part of the computation)."""
import numpy as np
import pytest

from paper_1903_03237_gb300.synth import make_mixture

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


CASES = [  # (F, T, M, N, K, precision)
    (65, 230, 2, 2, 16, 0), (65, 410, 4, 4, 16, 0), (33, 170, 8, 8, 16, 0),
    (65, 300, 4, 4, 16, 1), (20, 77, 3, 3, 5, 0), (65, 512, 8, 8, 16, 2),
]


def test_batch_equals_alone(fm):
    mixes = [make_mixture(F, T, M, N, K, 1000 + i) for i, (F, T, M, N, K, _) in enumerate(CASES)]
    ctxs = [fm.Context(m.X, c[3], c[4], seed=i, precision=c[5]) for i, (m, c) in enumerate(zip(mixes, CASES))]
    with fm.Batch(ctxs) as b:
        b.iterate(4)
        b.iterate(3)   # a second chunk length: a second captured graph
        b.sync()
    got = [c.get_state() + (c.loglik(),) for c in ctxs]
    for i, (m, c) in enumerate(zip(mixes, CASES)):
        alone = fm.Context(m.X, c[3], c[4], seed=i, precision=c[5])
        alone.iterate(4)
        alone.iterate(3)
        ref = alone.get_state() + (alone.loglik(),)
        for a, r in zip(got[i], ref):
            np.testing.assert_array_equal(a, r)


def test_batch_then_alone_orders(fm):
    # a member may still be used on its own between batch calls
    m = make_mixture(33, 120, 4, 3, 8, 7)
    a = fm.Context(m.X, 3, 8, seed=1)
    b2 = fm.Context(m.X, 3, 8, seed=2)
    with fm.Batch([a, b2]) as b:
        b.iterate(2)
        a.iterate(1)
        b.iterate(2)
        b.sync()
    ref = fm.Context(m.X, 3, 8, seed=1)
    ref.iterate(2)
    ref.iterate(1)
    ref.iterate(2)
    for x, y in zip(a.get_state(), ref.get_state()):
        np.testing.assert_array_equal(x, y)


def test_batch_autotune_restores_state_and_matches_tuned_alone(fm):
    mixes = [make_mixture(F, T, M, N, K, 1000 + i) for i, (F, T, M, N, K, _) in enumerate(CASES)]
    ctxs = [fm.Context(m.X, c[3], c[4], seed=i, precision=c[5]) for i, (m, c) in enumerate(zip(mixes, CASES))]
    with fm.Batch(ctxs) as b:
        b.iterate(2)
        b.sync()
        before = [c.get_state() for c in ctxs]
        sp = b.autotune(2)
        assert sp >= 1.0
        # the tuner's trials leave every member's state as it was
        for c, st in zip(ctxs, before):
            for x, y in zip(c.get_state(), st):
                np.testing.assert_array_equal(x, y)
        b.iterate(3)
        b.sync()
    for i, (m, c) in enumerate(zip(mixes, CASES)):
        alone = fm.Context(m.X, c[3], c[4], seed=i, precision=c[5])
        alone.iterate(2)                      # the planned shapes, as the batch before tuning
        alone.set_tuning(ctxs[i].get_tuning())
        alone.iterate(3)
        for x, y in zip(ctxs[i].get_state(), alone.get_state()):
            np.testing.assert_array_equal(x, y)
