"""The bin-fused FP32 schedule and the unconstrained source model (FastFCA) against the
float64 oracle, through the C ABI.

The fused schedule runs an iteration as two launches (the H update as a GEMM whose bin
splits are the CTAs of a thread-block cluster; everything else per bin, with the W update of
the next iteration and the next H update's per-point factors at the end of the bin's kernel) and applies the mu normalisation once at the end of a call, so several iterations
in one call exercise paths one iteration does not: they are checked against the oracle's
same iterations.  Bar: 1e-5 per iteration of the plain FP32 form (per tensor and per
element, as in test_gpu_parity), scaled by the number of iterations for multi-iteration
runs.  FastFCA (Sec. III-C-1, Eq. 22) runs only in this schedule.
"""
import numpy as np
import pytest

from oracle import fastmnmf_oracle as O
from paper_1903_03237_gb300.synth import make_mixture, make_state

from tests._parity import rel, elem_rel, image_scale, q_row_scale, state_errors, ll_rel, as64

pytestmark = pytest.mark.gpu

TOL = 1e-5
TAU_Q = 1.0
TAU_IMG = 1.0


@pytest.fixture(scope="module")
def fm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf
    return fastmnmf


def _nmf_case(fm, F, T, M, N, K, n_iter, seed=1, mask=O.UPDATE_ALL, normalise=True):
    mix = make_mixture(F, T, M, N, K, seed)
    W, H, G, Q = make_state(F, T, M, N, K, seed)
    ctx = fm.Context(mix.X, N, K, update_mask=mask, normalise=normalise, schedule=fm.SCHED_FUSED)
    ctx.set_state(W, H, G, Q)
    ctx.iterate(n_iter)
    ll = ctx.loglik()
    Wg, Hg, Gg, Qg = ctx.get_state()
    ctx.close()
    X64 = mix.X.astype(np.complex128)
    Wr, Hr, Gr, Qr, tr = O.iterate(X64, *as64(W, H, G, Q), n_iter=n_iter, mask=mask, do_normalise=normalise)
    err = state_errors(Wg, Hg, Gg, Qg, Wr, Hr, Gr, Qr, TAU_Q)
    err["LL"] = ll_rel(ll, tr[-1], X64, Wr, Hr, Gr, Qr)
    print("fused", (F, T, M, N, K), n_iter, {k: f"{v:.2e}" for k, v in err.items()})
    return err


# chunked frames (T > 256), ragged frame tiles, bins beyond one H-kernel chunk, every bucket
SHAPES = [(37, 150, 3, 3, 5), (70, 300, 4, 3, 16), (20, 601, 8, 3, 4), (130, 65, 2, 4, 7), (19, 45, 1, 2, 3),
          (9, 517, 5, 2, 1), (200, 33, 6, 2, 9)]


@pytest.mark.parametrize("n_iter", [2, 3])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"F{s[0]}T{s[1]}M{s[2]}N{s[3]}K{s[4]}" for s in SHAPES])
def test_fused_iterations_match_oracle(fm, shape, n_iter):
    err = _nmf_case(fm, *shape, n_iter=n_iter)
    assert max(err.values()) < n_iter * TOL, err


# several base tiles of the H GEMM (K > 32), frames not a multiple of 4 (scalar paths) or of
# the 64-frame tile, fewer bins than splits; the split counts 8 (few tiles), 6 (40 tiles, the
# paper-scale source shape), 2 (80 tiles) and 1 (396 tiles: one CTA per tile, no cluster
# partners), with bins left over in the last chunk of 32
HG_SHAPES = [(70, 303, 4, 3, 40), (33, 128, 2, 2, 70), (5, 64, 3, 2, 33), (70, 301, 8, 3, 16),
             (100, 640, 4, 4, 32), (71, 1280, 4, 4, 32), (40, 2049, 2, 6, 40)]


@pytest.mark.parametrize("shape", HG_SHAPES, ids=[f"F{s[0]}T{s[1]}M{s[2]}N{s[3]}K{s[4]}" for s in HG_SHAPES])
def test_fused_h_gemm_tiles(fm, shape):
    err = _nmf_case(fm, *shape, n_iter=2, seed=4)
    assert max(err.values()) < 2 * TOL, err


# N*K above 256 (the W sums loop over bases in passes of 64 per warp; the H GEMM tiles K by
# 32): the large mixture's source shape (M8 N6 K64) on small F, T, and K beyond 128
LARGE_NK_SHAPES = [(20, 130, 8, 6, 64), (33, 301, 4, 5, 100), (17, 64, 2, 3, 130), (9, 257, 6, 8, 40)]


@pytest.mark.parametrize("shape", LARGE_NK_SHAPES, ids=[f"F{s[0]}T{s[1]}M{s[2]}N{s[3]}K{s[4]}" for s in LARGE_NK_SHAPES])
def test_fused_many_bases(fm, shape):
    err = _nmf_case(fm, *shape, n_iter=2, seed=6)
    assert max(err.values()) < 2 * TOL, err


def test_fused_pair_limit(fm):
    # N*M above 256: the fused schedule is refused when asked for and not chosen otherwise
    mix = make_mixture(5, 20, 8, 33, 2, 1)
    with pytest.raises(fm.FastMNMFError) as ei:
        fm.Context(mix.X, 33, 2, seed=1, schedule=fm.SCHED_FUSED)
    assert ei.value.status == fm.EINVAL
    ctx = fm.Context(mix.X, 33, 2, seed=1)
    ctx.set_timing(True)
    ctx.iterate(1)
    kt = ctx.kernel_times()
    assert kt["bin"][1] == 0 and kt["w_update"][1] > 0      # the sweep schedule ran
    assert np.isfinite(ctx.loglik())


@pytest.mark.parametrize("mask", [O.UPDATE_W, O.UPDATE_H, O.UPDATE_G, O.UPDATE_Q, O.UPDATE_W | O.UPDATE_H,
                                  O.UPDATE_G | O.UPDATE_Q], ids=["W", "H", "G", "Q", "WH", "GQ"])
@pytest.mark.parametrize("normalise", [False, True], ids=["raw", "norm"])
def test_fused_masks_over_iterations(fm, mask, normalise):
    err = _nmf_case(fm, 29, 277, 3, 3, 5, n_iter=3, seed=3, mask=mask, normalise=normalise)
    assert max(err.values()) < 3 * TOL, err


def test_fused_equals_itself_across_calls(fm):
    # three calls of one iteration = one call of three, up to the rounding of the mu
    # normalisation (applied at the end of each call)
    mix = make_mixture(37, 150, 3, 3, 5, 6)
    a = fm.Context(mix.X, 3, 5, seed=11, schedule=fm.SCHED_FUSED)
    b = fm.Context(mix.X, 3, 5, seed=11, schedule=fm.SCHED_FUSED)
    a.iterate(3)
    for _ in range(3):
        b.iterate(1)
    for x, y in zip(a.get_state(), b.get_state()):
        assert rel(x, y) < 1e-6
    assert abs(a.loglik() - b.loglik()) < 1e-7 * abs(a.loglik())


def test_fused_restart_is_bitwise(fm):
    mix = make_mixture(37, 150, 3, 3, 5, 8)
    ctx = fm.Context(mix.X, 3, 5, seed=4, schedule=fm.SCHED_FUSED)
    ctx.iterate(7)
    a = ctx.get_state() + (ctx.loglik(),)
    ctx.iterate(5)
    ctx.restart()
    ctx.iterate(7)
    b = ctx.get_state() + (ctx.loglik(),)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


# ---- FastFCA: the unconstrained source model ------------------------------------------
def _free_state(F, T, M, N, seed):
    _, _, G, Q = make_state(F, T, M, N, 2, seed)
    rng = np.random.default_rng(seed + 5)
    lam = rng.uniform(0.2, 2.0, size=(N, F, T)).astype(np.float32)     # library layout [N][F][T]
    return lam, G, Q


def _fca_case(fm, F, T, M, N, n_iter, seed=1, mask=O.UPDATE_ALL, normalise=True):
    mix = make_mixture(F, T, M, N, 2, seed)
    lam, G, Q = _free_state(F, T, M, N, seed)
    ctx = fm.Context(mix.X, N, 1, update_mask=mask, normalise=normalise, source_model=fm.SOURCE_FREE)
    ctx.set_lambda(lam, G, Q)
    ll0 = ctx.loglik()
    ctx.iterate(n_iter)
    ll = ctx.loglik()
    Lg, Gg, Qg = ctx.get_lambda()
    S = ctx.separate()
    ctx.close()
    X64 = mix.X.astype(np.complex128)
    lam64 = lam.astype(np.float64).transpose(1, 2, 0)
    ll0_ref = O.loglik_lam(X64, lam64, G.astype(float), Q.astype(complex))
    Lr, Gr, Qr, tr = O.iterate_free(X64, lam64, G.astype(float), Q.astype(complex), n_iter=n_iter, mask=mask,
                                    do_normalise=normalise)
    Sr = O.separate_lam(X64, Lr, Gr, Qr)
    sc = O.loglik_terms_abs_lam(X64, Lr, Gr, Qr)
    err = {"lambda": rel(Lg, Lr.transpose(2, 0, 1)), "lambda_el": elem_rel(Lg, Lr.transpose(2, 0, 1), 0.0, 0.0),
           "G": rel(Gg, Gr), "G_el": elem_rel(Gg, Gr, 0.0, 0.0), "Q": rel(Qg, Qr),
           "Q_el": elem_rel(Qg, Qr, q_row_scale(Qr), TAU_Q), "LL0": abs(ll0 - ll0_ref) / sc,
           "LL": abs(ll - tr[-1]) / sc, "separated": rel(S, Sr),
           "separated_el": elem_rel(S, Sr, image_scale(X64, N), TAU_IMG)}
    print("fca", (F, T, M, N), n_iter, {k: f"{v:.2e}" for k, v in err.items()})
    return err


FCA_SHAPES = [(37, 150, 3, 3), (40, 300, 4, 4), (20, 64, 8, 3), (19, 45, 1, 2), (33, 70, 2, 5)]


@pytest.mark.parametrize("n_iter", [1, 3])
@pytest.mark.parametrize("shape", FCA_SHAPES, ids=[f"F{s[0]}T{s[1]}M{s[2]}N{s[3]}" for s in FCA_SHAPES])
def test_fca_matches_oracle(fm, shape, n_iter):
    err = _fca_case(fm, *shape, n_iter=n_iter)
    assert max(err.values()) < n_iter * TOL, err


@pytest.mark.parametrize("mask", [O.UPDATE_W, O.UPDATE_G, O.UPDATE_Q], ids=["lambda", "G", "Q"])
def test_fca_each_block(fm, mask):
    err = _fca_case(fm, 29, 77, 3, 3, n_iter=2, seed=3, mask=mask)
    assert max(err.values()) < 2 * TOL, err


def test_fca_init_matches_spec(fm):
    F, T, M, N, seed = 21, 35, 3, 4, 12345
    mix = make_mixture(F, T, M, N, 2, 5)
    ctx = fm.Context(mix.X, N, 1, seed=seed, source_model=fm.SOURCE_FREE)
    L, G, Q = ctx.get_lambda()
    Lr, Gr, Qr = O.init_state_free(F, T, M, N, seed)
    np.testing.assert_array_equal(L, Lr.transpose(2, 0, 1).astype(np.float32))
    np.testing.assert_allclose(G, Gr, rtol=1e-7)
    np.testing.assert_array_equal(Q, Qr.astype(np.complex64))
    X64 = mix.X.astype(np.complex128)
    assert abs(ctx.loglik() - O.loglik_lam(X64, Lr, Gr, Qr)) / O.loglik_terms_abs_lam(X64, Lr, Gr, Qr) < TOL


def test_fca_trajectory_monotone(fm):
    mix = make_mixture(64, 200, 4, 3, 2, 9)
    ctx = fm.Context(mix.X, 3, 1, seed=3, source_model=fm.SOURCE_FREE)
    lls = [ctx.loglik()]
    for _ in range(20):
        ctx.iterate(1)
        lls.append(ctx.loglik())
    d = np.diff(lls)
    assert np.all(d >= -1e-6 * np.abs(lls).max()), d.min()
    assert lls[-1] > lls[0]


def test_fca_rejects_nmf_calls(fm):
    mix = make_mixture(10, 20, 2, 2, 2, 1)
    ctx = fm.Context(mix.X, 2, 1, source_model=fm.SOURCE_FREE)
    W = np.ones((2, 1, 10), np.float32)
    H = np.ones((2, 1, 20), np.float32)
    _, _, G, Q = ctx.get_state()
    with pytest.raises(fm.FastMNMFError) as e:
        ctx.set_state(W, H, G, Q)
    assert e.value.status == fm.EINVAL
    with pytest.raises(fm.FastMNMFError) as e:
        fm.Context(mix.X, 2, 1, source_model=fm.SOURCE_FREE, precision=fm.PREC_BF16)
    assert e.value.status == fm.EINVAL
