"""Serving (continuous batching): requests of different lengths admitted as memory and
slots free up, advanced together, each returning exactly what the same request returns
when run alone with the same iterations per call (the server advances a request by
iters_per_step iterations per call; the fused schedule applies its mu normalisation at the
end of each call, so the call boundaries are part of the computation)."""
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


def _alone(fm, X, N, K, n_iter, seed, step):
    with fm.Context(X, N, K, seed=seed) as ctx:
        done = 0
        while done < n_iter:
            n = min(step, n_iter - done)
            ctx.iterate(n)
            done += n
        return ctx.separate(), ctx.loglik()


def test_results_same_alone_and_in_the_mix(fm):
    Ts = [120, 300, 75, 410, 200, 150, 333, 90]
    with fm.Server(max_active=4, iters_per_step=5) as srv:
        jobs = []
        for i, T in enumerate(Ts):
            mix = make_mixture(65, T, 4, 3, 16, 2000 + i)
            jobs.append((srv.submit(mix.X, 3, 16, 12, seed=2000 + i), mix, 2000 + i))
        for j, _, _ in jobs:
            assert srv.wait(j, 300.0) == fm.JOB_DONE
        for j, mix, sd in jobs:
            out, ll = srv.result(j)
            ref, ref_ll = _alone(fm, mix.X, 3, 16, 12, sd, 5)
            np.testing.assert_array_equal(out, ref)
            assert ll == ref_ll
        st = srv.stats()
        assert st["completed"] == len(Ts) and st["failed"] == 0 and st["bytes_in_use"] == 0


def test_admission_by_budget(fm):
    one = fm.footprint(65, 300, 4, 3, 16)
    with fm.Server(hbm_budget=int(1.5 * one), max_active=8, iters_per_step=3) as srv:
        mixes = [make_mixture(65, 300, 4, 3, 16, 50 + i) for i in range(4)]
        ids = [srv.submit(m.X, 3, 16, 7, seed=i) for i, m in enumerate(mixes)]
        for j in ids:
            assert srv.wait(j, 300.0) == fm.JOB_DONE
        for i, (j, m) in enumerate(zip(ids, mixes)):
            out, _ = srv.result(j)
            ref, _ = _alone(fm, m.X, 3, 16, 7, i, 3)
            np.testing.assert_array_equal(out, ref)
        big = make_mixture(65, 2000, 4, 3, 16, 9)
        with pytest.raises(fm.FastMNMFError) as e:
            srv.submit(big.X, 3, 16, 5)
        assert e.value.status == fm.ENOMEM


def test_failed_request_is_reported(fm):
    with fm.Server(max_active=2, iters_per_step=5) as srv:
        X = make_mixture(33, 100, 2, 2, 4, 3).X.copy()
        X[5, 7, 1] = np.nan
        j = srv.submit(X, 2, 4, 5)
        ok = srv.submit(make_mixture(33, 100, 2, 2, 4, 4).X, 2, 4, 5)
        assert srv.wait(j, 300.0) == fm.JOB_FAILED
        assert srv.wait(ok, 300.0) == fm.JOB_DONE
        with pytest.raises(fm.FastMNMFError) as e:
            srv.result(j)
        assert e.value.status == fm.ENONFINITE
        srv.result(ok)
