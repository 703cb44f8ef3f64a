"""FastMNMF-DP on the GPU (through the C ABI) against the float64 oracle (Sec. III-B-3, III-C-3).

The Metropolis decisions are integers decided by floating point.  Both sides compute log
gamma_t; the GPU in float32.  A proposal whose log gamma lies within the arithmetic's error of
log u can be decided either way, and every later value then differs.  So the acceptance draws
of these tests are made tie-free with the oracle alone: any log u within a margin of the
oracle's log gamma is moved to the same side, twice the margin away.  The margin is
1e-3 x sum_{f,m} |term|, the sum of the absolute terms of log gamma_t (the float32 sum of
F M terms, plus a decoder output with float32 rounding in each of its Hd products, stays far
inside it: test_metropolis_log_gamma measures it).  Every decision must then agree exactly.

Bars (FP32 class, as the other FP32 parity tests): z per element 1e-5 (relative to |z| + 1);
u, v, W, H, g~ per element 1e-5; Q per element 1e-5 against its row norm (tau = 1); the
log-likelihood within 1e-5 of the sum of the absolute terms of Eq. 17; log gamma within
1e-4 of its sum of absolute terms.  As in the random-shape test of FastMNMF (the same per-bin
IP kernel), an error above its bar is held to sqrt(T) times the error the oracle itself makes
when V_fm is rounded to float32 before the IP step: with few frames per channel V_fm is
ill-conditioned (cond 1.2e6 at F50 T23 M4 with the speech source alone), and the IP step
amplifies any rounding of V_fm by up to that factor.
"""
import numpy as np
import pytest

from oracle import fastmnmf_oracle as O
from oracle import fastmnmf_dp_oracle as D
from paper_1903_03237_gb300.synth import make_mixture, make_dp_state, make_decoder, make_dp_draws

from tests._parity import elem_rel, q_row_scale, rel

pytestmark = pytest.mark.gpu

MARGIN = 1e-3


@pytest.fixture(scope="module")
def fm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf
    return fastmnmf


def _problem(F, T, M, N, K, Dd, Hd, seed):
    mix = make_mixture(F, T, M, N, K, seed)
    state = make_dp_state(F, T, M, N, K, Dd, seed)
    theta = make_decoder(F, Dd, Hd, seed)
    return mix.X, state, theta


def _as64(state):
    return tuple(a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64) for a in state)


def _log_gamma_scale(xt, lam_new, lam_old, g0, y_rest):
    """sum_{f,m} |term| of log gamma_t, per frame."""
    y_new = lam_new[:, :, None] * g0[:, None, :] + y_rest
    y_old = lam_old[:, :, None] * g0[:, None, :] + y_rest
    return np.sum(np.abs(xt / y_new - xt / y_old) + np.abs(np.log(y_new / y_old)), axis=(0, 2))


def tie_free_draws(X, state, theta, eps, n_iter, S, seed):
    """Draws of n_iter iterations whose acceptance decisions are at least 2 MARGIN x scale away
    from the oracle's log gamma, following the oracle's own trajectory."""
    X = X.astype(np.complex128)
    Z, u, v, W, H, G, Q = _as64(state)
    th = tuple(a.astype(np.float64) for a in theta)
    T, Dd = Z.shape
    xi, logu = make_dp_draws(n_iter, S, T, Dd, seed)
    xi = xi.astype(np.float64)
    logu = logu.astype(np.float64)
    se = np.sqrt(np.float64(np.float32(eps)))
    for i in range(n_iter):
        xt = O.projected_power(Q, X)
        lam_rest = O.source_psd(W, H) if W.shape[0] else np.zeros(xt.shape[:2] + (0,))
        y_rest = O.model_power(lam_rest, G[1:]) if W.shape[0] else np.zeros(xt.shape)
        Zc = Z.copy()
        R = D.decoder(Zc, th)
        for s in range(S):
            Zp = Zc + se * xi[i, s]
            Rp = D.decoder(Zp, th)
            ln, lo = D.speech_psd(u, v, Rp), D.speech_psd(u, v, R)
            lg = D.log_gamma(xt, ln, lo, G[0], y_rest)
            m = MARGIN * _log_gamma_scale(xt, ln, lo, G[0], y_rest)
            near = np.abs(logu[i, s] - lg) < 2 * m
            logu[i, s][near] = np.where(logu[i, s][near] < lg[near], lg[near] - 2 * m[near], lg[near] + 2 * m[near])
            acc = logu[i, s] < lg
            Zc[acc] = Zp[acc]
            R[acc] = Rp[acc]
        Z, u, v, W, H, G, Q, _ = D.iterate_dp(X, Z, u, v, W, H, G, Q, th, xi[i:i + 1], logu[i:i + 1],
                                              float(np.float32(eps)), n_iter=1)
    return xi.astype(np.float32), logu.astype(np.float32)


def _state_errors(g, r):
    Zg, ug, vg, Wg, Hg, Gg, Qg = g
    Zr, ur, vr, Wr, Hr, Gr, Qr = r
    err = {"Z_el": float(np.max(np.abs(Zg - Zr) / (np.abs(Zr) + 1.0))),
           "u_el": elem_rel(ug, ur, 0.0, 0.0), "v_el": elem_rel(vg, vr, 0.0, 0.0),
           "G_el": elem_rel(Gg, Gr, 0.0, 0.0), "Q_el": elem_rel(Qg, Qr, q_row_scale(Qr), 1.0),
           "u": rel(ug, ur), "v": rel(vg, vr), "G": rel(Gg, Gr), "Q": rel(Qg, Qr)}
    if Wr.size:
        err.update({"W_el": elem_rel(Wg, Wr, 0.0, 0.0), "H_el": elem_rel(Hg, Hr, 0.0, 0.0),
                    "W": rel(Wg, Wr), "H": rel(Hg, Hr)})
    return err


def _round_bits(a, p):
    m, e = np.frexp(a)
    return np.ldexp(np.round(m * 2.0 ** p) / 2.0 ** p, e)


def _v_float32_floor(args, n_iter):
    """The oracle's own errors when V_fm (Eq. 18) is rounded to float32 before every IP step."""
    ref = D.iterate_dp(*args, n_iter=n_iter)
    exact = O.weighted_scm

    def rounded(X, yt):
        V = exact(X, yt)
        return _round_bits(V.real, 24) + 1j * _round_bits(V.imag, 24)

    O.weighted_scm = rounded
    try:
        per = D.iterate_dp(*args, n_iter=n_iter)
    finally:
        O.weighted_scm = exact
    return _state_errors(per[:7], ref[:7])


def _assert_within(err, bar, T, args, n_iter):
    over = {k: v for k, v in err.items() if not v < bar}
    if not over:
        return
    floor = _v_float32_floor(args, n_iter)
    for k, v in over.items():
        lim = np.sqrt(T) * floor.get(k, 0.0)
        print(f"  {k} {v:.1e} above {bar:.0e}: conditioning bar {lim:.1e}")
        assert v < lim, (k, v, lim, err)


def _ll_rel(ll, X, state, theta):
    Z, u, v, W, H, G, Q = state
    lam = D.dp_lambda(u, v, D.decoder(Z, theta), W, H)
    return abs(ll - D.loglik_dp(X, Z, u, v, W, H, G, Q, theta)) / O.loglik_terms_abs_lam(X, lam, G, Q)


def _ctx(fm, X, state, theta, N, K, S, eps=1e-4, normalise=True):
    Z = state[0]
    dp = fm.DPContext(X, N, K, D=Z.shape[1], Hd=theta[0].shape[0], n_proposals=S, eps=eps, normalise=normalise)
    dp.set_decoder(*theta)
    dp.set_state(*state)
    return dp


# F, T, M, N, K, D, Hd, S, seed: ragged T (not a multiple of 4 or 8), F beyond one CTA's 256
# threads, every channel bucket, speech alone (N = 1), several noise sources; Metropolis launches
# with clusters of 1 CTA (1, 2 and 4 frames), 5 CTAs (F300) and 8 CTAs with 16 frames (the
# paper-scale case)
SHAPES = [
    (33, 41, 2, 2, 3, 16, 128, 5, 1),
    (300, 37, 3, 3, 4, 8, 64, 4, 2),
    (64, 75, 5, 2, 16, 16, 128, 6, 3),
    (20, 30, 8, 3, 2, 4, 12, 3, 4),
    (50, 23, 4, 1, 1, 16, 32, 5, 5),
    (40, 1000, 2, 2, 2, 8, 16, 3, 6),     # 4 frames per Metropolis cluster
    (40, 600, 3, 2, 2, 8, 16, 3, 7),      # 2 frames per Metropolis cluster
]
IDS = [f"F{s[0]}T{s[1]}M{s[2]}N{s[3]}K{s[4]}D{s[5]}H{s[6]}S{s[7]}" for s in SHAPES]


@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_set_state_loglik(fm, shape):
    F, T, M, N, K, Dd, Hd, S, seed = shape
    X, state, theta = _problem(F, T, M, N, K, Dd, Hd, seed)
    with _ctx(fm, X, state, theta, N, K, S) as dp:
        e = _ll_rel(dp.loglik(), X.astype(np.complex128), _as64(state), tuple(a.astype(np.float64) for a in theta))
    print(shape, f"LL {e:.1e}")
    assert e < 1e-5


@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_metropolis_log_gamma(fm, shape):
    F, T, M, N, K, Dd, Hd, S, seed = shape
    X, state, theta = _problem(F, T, M, N, K, Dd, Hd, seed)
    eps = 1e-2
    xi, logu = tie_free_draws(X, state, theta, eps, 1, S, seed)
    X64 = X.astype(np.complex128)
    Z, u, v, W, H, G, Q = _as64(state)
    th = tuple(a.astype(np.float64) for a in theta)
    xt = O.projected_power(Q, X64)
    lam_rest = O.source_psd(W, H) if W.shape[0] else np.zeros(xt.shape[:2] + (0,))
    hist = []
    Zr, _, nr = D.metropolis(xt, Z, u, v, th, G, lam_rest, xi[0].astype(np.float64), logu[0].astype(np.float64),
                             float(np.float32(eps)), history=hist)
    with _ctx(fm, X, state, theta, N, K, S, eps=eps) as dp:
        lg, na = dp.metropolis(xi[0], logu[0])
        Zg = dp.get_state()[0]
    # log gamma of every proposal against its sum of absolute terms (recomputed along the chain)
    y_rest = O.model_power(lam_rest, G[1:]) if W.shape[0] else np.zeros(xt.shape)
    Zc, R = Z.copy(), D.decoder(Z, th)
    worst = 0.0
    for s in range(S):
        Zp = Zc + np.sqrt(np.float32(eps)) * xi[0, s]
        Rp = D.decoder(Zp, th)
        scale = _log_gamma_scale(xt, D.speech_psd(u, v, Rp), D.speech_psd(u, v, R), G[0], y_rest)
        worst = max(worst, float(np.max(np.abs(lg[s] - hist[s][0]) / scale)))
        acc = hist[s][1]
        Zc[acc] = Zp[acc]
        R[acc] = Rp[acc]
    print(shape, f"log gamma err/scale {worst:.1e}, accepted {na} of {S * T}")
    assert worst < 1e-4
    assert na == nr
    assert float(np.max(np.abs(Zg - Zr) / (np.abs(Zr) + 1.0))) < 1e-5


@pytest.mark.parametrize("shape", SHAPES, ids=IDS)
def test_one_iteration(fm, shape):
    F, T, M, N, K, Dd, Hd, S, seed = shape
    X, state, theta = _problem(F, T, M, N, K, Dd, Hd, seed)
    xi, logu = tie_free_draws(X, state, theta, 1e-4, 1, S, seed)
    X64 = X.astype(np.complex128)
    th = tuple(a.astype(np.float64) for a in theta)
    acc = []
    args = (X64, *_as64(state), th, xi.astype(np.float64), logu.astype(np.float64), float(np.float32(1e-4)))
    *ref, tr = D.iterate_dp(*args, n_iter=1, accepted=acc)
    with _ctx(fm, X, state, theta, N, K, S) as dp:
        dp.iterate(1, xi, logu)
        ll = dp.loglik()
        got = dp.get_state()
        na = dp.accepted()
    err = _state_errors(got, ref)
    print(shape, f"accepted {na} / {acc[0]}", {k: f"{v:.1e}" for k, v in err.items()})
    assert na == acc[0]
    assert _ll_rel(ll, X64, ref, th) < 1e-5
    _assert_within(err, 1e-5, T, args, 1)


@pytest.mark.parametrize("shape", SHAPES[:3], ids=IDS[:3])
def test_three_iterations(fm, shape):
    F, T, M, N, K, Dd, Hd, S, seed = shape
    X, state, theta = _problem(F, T, M, N, K, Dd, Hd, seed)
    xi, logu = tie_free_draws(X, state, theta, 1e-4, 3, S, seed + 50)
    X64 = X.astype(np.complex128)
    th = tuple(a.astype(np.float64) for a in theta)
    acc = []
    args = (X64, *_as64(state), th, xi.astype(np.float64), logu.astype(np.float64), float(np.float32(1e-4)))
    *ref, tr = D.iterate_dp(*args, n_iter=3, accepted=acc)
    with _ctx(fm, X, state, theta, N, K, S) as dp:
        dp.iterate(3, xi, logu)
        ll = dp.loglik()
        got = dp.get_state()
        na = dp.accepted()
    err = _state_errors(got, ref)
    print(shape, f"accepted {na} / {sum(acc)}", {k: f"{v:.1e}" for k, v in err.items()})
    assert na == sum(acc)
    assert _ll_rel(ll, X64, ref, th) < 3e-5
    _assert_within(err, 3e-5, T, args, 3)


def test_accept_all_and_none(fm):
    F, T, M, N, K, Dd, Hd, S, seed = SHAPES[0]
    X, state, theta = _problem(F, T, M, N, K, Dd, Hd, seed)
    xi, _ = make_dp_draws(1, S, T, Dd, seed)
    eps = 1e-2
    with _ctx(fm, X, state, theta, N, K, S, eps=eps) as dp:
        _, n = dp.metropolis(xi[0], np.full((S, T), np.inf, np.float32))
        assert n == 0 and np.array_equal(dp.get_state()[0], state[0])
        _, n = dp.metropolis(xi[0], np.full((S, T), -np.inf, np.float32))
        assert n == S * T
        Zg = dp.get_state()[0]
    expect = state[0].astype(np.float64) + np.sqrt(np.float64(np.float32(eps))) * xi[0].astype(np.float64).sum(axis=0)
    assert float(np.max(np.abs(Zg - expect) / (np.abs(expect) + 1.0))) < 1e-5


def test_images_sum_to_mixture(fm):
    F, T, M, N, K, Dd, Hd, S, seed = SHAPES[1]
    X, state, theta = _problem(F, T, M, N, K, Dd, Hd, seed)
    xi, logu = make_dp_draws(2, S, T, Dd, seed)
    with _ctx(fm, X, state, theta, N, K, S) as dp:
        dp.iterate(2, xi, logu)
        Y = dp.separate()
        Z, u, v, W, H, G, Q = _as64(dp.get_state())
    X64 = X.astype(np.complex128)
    # Eq. 3: the images add up to the mixture; each equals the oracle's filter of the GPU state
    assert elem_rel(Y.sum(axis=0), X64, np.linalg.norm(X64, axis=2, keepdims=True) * np.ones(X.shape), 1.0) < 1e-5
    lam = D.dp_lambda(u, v, D.decoder(Z, tuple(a.astype(np.float64) for a in theta)), W, H)
    ref = O.separate_lam(X64, lam, G, Q)
    assert rel(Y, ref) < 1e-4


def test_bad_arguments(fm):
    X, state, theta = _problem(10, 12, 2, 2, 2, 4, 8, 0)
    for kw in (dict(Hd=10), dict(D=0), dict(n_proposals=-1), dict(eps=-1.0)):
        with pytest.raises(fm.FastMNMFError) as e:
            fm.DPContext(X, 2, 2, **kw)
        assert e.value.status == fm.EINVAL
    with pytest.raises(fm.FastMNMFError) as e:
        fm.DPContext(X, 9, 2)
    assert e.value.status == fm.EINVAL
    with fm.DPContext(X, 2, 2, D=4, Hd=8, n_proposals=2) as dp:
        xi, logu = make_dp_draws(1, 2, 12, 4, 0)
        with pytest.raises(fm.FastMNMFError) as e:
            dp.iterate(1, xi, logu)           # no decoder, no state yet
        assert e.value.status == fm.EINVAL
        dp.set_decoder(*theta)
        bad = list(state)
        bad[1] = -bad[1]
        with pytest.raises(fm.FastMNMFError) as e:
            dp.set_state(*bad)
        assert e.value.status == fm.EINVAL


def test_paper_scale_one_iteration(fm):
    """The paper's FastMNMF-DP setting (Sec. IV-A): F = 513, 8 s at a 256-point shift (T = 500),
    M = 5, N = 2, K = 16, D = 16, 30 proposals per frame, eps = 1e-4; decoder width 128."""
    F, T, M, N, K, Dd, Hd, S = 513, 500, 5, 2, 16, 16, 128, 30
    X, state, theta = _problem(F, T, M, N, K, Dd, Hd, 7)
    xi, logu = tie_free_draws(X, state, theta, 1e-4, 1, S, 7)
    X64 = X.astype(np.complex128)
    th = tuple(a.astype(np.float64) for a in theta)
    acc = []
    args = (X64, *_as64(state), th, xi.astype(np.float64), logu.astype(np.float64), float(np.float32(1e-4)))
    *ref, tr = D.iterate_dp(*args, n_iter=1, accepted=acc)
    with _ctx(fm, X, state, theta, N, K, S) as dp:
        dp.iterate(1, xi, logu)
        ll = dp.loglik()
        got = dp.get_state()
        na = dp.accepted()
    err = _state_errors(got, ref)
    print("paper scale", f"accepted {na} / {acc[0]}", {k: f"{v:.1e}" for k, v in err.items()})
    assert na == acc[0]
    assert _ll_rel(ll, X64, ref, th) < 1e-5
    _assert_within(err, 1e-5, T, args, 1)


def test_one_iteration_without_normalisation(fm):
    F, T, M, N, K, Dd, Hd, S, seed = SHAPES[1]
    X, state, theta = _problem(F, T, M, N, K, Dd, Hd, seed)
    xi, logu = make_dp_draws(1, S, T, Dd, seed)
    logu[:] = -np.inf        # every proposal accepted: no decision depends on rounding
    X64 = X.astype(np.complex128)
    th = tuple(a.astype(np.float64) for a in theta)
    args = (X64, *_as64(state), th, xi.astype(np.float64), logu.astype(np.float64), float(np.float32(1e-4)))
    *ref, tr = D.iterate_dp(*args, n_iter=1, do_normalise=False)
    with _ctx(fm, X, state, theta, N, K, S, normalise=False) as dp:
        dp.iterate(1, xi, logu)
        ll = dp.loglik()
        got = dp.get_state()
    err = _state_errors(got, ref)
    print("raw", {k: f"{v:.1e}" for k, v in err.items()})
    assert _ll_rel(ll, X64, ref, th) < 1e-5
    for k, v in err.items():
        assert v < 1e-5, (k, v, err)


def test_device_draws_equal_host_draws(fm):
    import torch
    F, T, M, N, K, Dd, Hd, S, seed = SHAPES[0]
    X, state, theta = _problem(F, T, M, N, K, Dd, Hd, seed)
    xi, logu = make_dp_draws(6, S, T, Dd, seed)   # more than one chunk of host draws
    outs = []
    for on_device in (False, True):
        with _ctx(fm, X, state, theta, N, K, S) as dp:
            if on_device:
                dp.iterate(6, torch.from_numpy(xi).cuda(), torch.from_numpy(logu).cuda())
            else:
                dp.iterate(6, xi, logu)
            outs.append((dp.get_state(), dp.loglik(), dp.accepted()))
    (sa, la, na), (sb, lb, nb) = outs
    assert na == nb and la == lb
    for a, b in zip(sa, sb):
        assert np.array_equal(a, b)
