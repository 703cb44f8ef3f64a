"""Pins of the oracle's unconstrained source model (FastFCA: Sec. III-B-1 and III-C-1, the
lambda rule of Eq. 22) against what the paper and the mathematics fix.  CPU only."""
import numpy as np
import pytest

from oracle import fastmnmf_oracle as O
from paper_1903_03237_gb300.synth import make_mixture, make_state


def _case(F=5, T=30, M=3, N=2, seed=3):
    mix = make_mixture(F, T, M, N, 2, seed)
    _, _, G, Q = make_state(F, T, M, N, 2, seed)
    rng = np.random.default_rng(seed + 100)
    lam = rng.uniform(0.2, 2.0, size=(F, T, N))          # not of NMF form
    return mix.X.astype(np.complex128), lam, G.astype(np.float64), Q.astype(np.complex128)


def test_init_state_free_layout():
    lam, G, Q = O.init_state_free(4, 6, 3, 2, seed=11)
    assert lam.shape == (4, 6, 2)
    u = O.splitmix64_uniform(11, 0, 2 * 4 * 6)
    # lambda[f, t, n] = 0.1 + u_{(n F + f) T + t}
    assert lam[0, 0, 0] == np.float32(0.1 + u[0])
    assert lam[3, 5, 1] == np.float32(0.1 + u[(1 * 4 + 3) * 6 + 5])
    np.testing.assert_allclose(G.sum(axis=2), 1.0, rtol=1e-6)
    np.testing.assert_array_equal(Q, np.tile(np.eye(3), (4, 1, 1)))


def test_lambda_rule_terms_are_loglik_gradient():
    # d LL / d lambda_ftn = sum_m g~_nfm (x~/y~^2 - 1/y~) = num - den of Eq. 22
    X, lam, G, Q = _case(seed=5)
    xt = O.projected_power(Q, X)
    num, den = O.mu_lambda_terms(xt, lam, G)
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(10):
        i = tuple(rng.integers(0, s) for s in lam.shape)
        lp, lm = lam.copy(), lam.copy()
        lp[i] += h
        lm[i] -= h
        g = (O.loglik_lam(X, lp, G, Q) - O.loglik_lam(X, lm, G, Q)) / (2 * h)
        assert abs((num - den)[i] - g) <= 1e-5 * max(1.0, abs(g))


def test_lambda_rule_m1_n1_closed_form():
    # M = N = 1 with g~ and Q fixed: y~ = lambda, and Eq. 22 is lambda <- sqrt(lambda x~), so
    # after k steps lambda_k = x~^(1 - 2^-k) lambda_0^(2^-k) at every point.
    F, T = 4, 7
    rng = np.random.default_rng(2)
    X = rng.standard_normal((F, T, 1)) + 1j * rng.standard_normal((F, T, 1))
    lam0 = rng.uniform(0.1, 3.0, (F, T, 1))
    G = np.ones((1, F, 1))
    Q = np.ones((F, 1, 1), dtype=complex)
    for k in (1, 2, 5):
        lam, _, _, _ = O.iterate_free(X, lam0, G, Q, n_iter=k, mask=O.UPDATE_W, do_normalise=False)
        xt = np.abs(X) ** 2
        np.testing.assert_allclose(lam, xt ** (1 - 2.0 ** -k) * lam0 ** (2.0 ** -k), rtol=1e-12)


@pytest.mark.parametrize("M,N", [(1, 2), (2, 3), (3, 2), (4, 4)])
def test_loglik_lam_equals_fullrank_density(M, N):
    X, lam, G, Q = _case(F=3, T=8, M=M, N=N, seed=M * 7 + N)
    a = O.loglik_lam(X, lam, G, Q)
    b = O.loglik_fullrank_lam(X, lam, G, Q)
    assert abs(a - b) <= 1e-10 * abs(b)


def test_fca_monotone_per_block_and_iteration():
    X, lam, G, Q = _case(F=6, T=30, M=3, N=3, seed=9)
    blocks = []
    _, _, _, trace = O.iterate_free(X, lam, G, Q, n_iter=8, block_ll=blocks)
    ll0 = O.loglik_lam(X, lam, G, Q)
    seq = [ll0] + [v for _, v in blocks]
    d = np.diff(seq)
    assert np.all(d >= -1e-9 * np.abs(seq[1:])), (d.min(), blocks)
    assert np.all(np.diff([ll0] + trace) >= -1e-9 * abs(ll0))


def test_normalise_free_invariance():
    X, lam, G, Q = _case(F=5, T=12, M=3, N=3, seed=23)
    lam2, G2, Q2 = O.normalise_free(lam, G, Q)
    a, b = O.loglik_lam(X, lam, G, Q), O.loglik_lam(X, lam2, G2, Q2)
    assert abs(a - b) < 1e-12 * abs(a)
    np.testing.assert_allclose(np.einsum("fij,fij->f", Q2, Q2.conj()).real, 3.0, rtol=1e-12)
    np.testing.assert_allclose(G2.sum(axis=2), 1.0, rtol=1e-12)


def test_fca_trajectory_independent_of_normalisation():
    X, lam, G, Q = _case(F=5, T=20, M=2, N=2, seed=29)
    *_, t1 = O.iterate_free(X, lam, G, Q, n_iter=5, do_normalise=True)
    *_, t2 = O.iterate_free(X, lam, G, Q, n_iter=5, do_normalise=False)
    np.testing.assert_allclose(t1, t2, rtol=1e-10)


def test_g_and_q_blocks_agree_with_the_nmf_model():
    # With lambda of NMF form and only g~ and Q updated, both source models take the same
    # steps: the log-likelihood trajectories are equal.
    mix = make_mixture(5, 25, 3, 2, 3, 31)
    W, H, G, Q = make_state(5, 25, 3, 2, 3, 31)
    X = mix.X.astype(np.complex128)
    W, H, G, Q = W.astype(float), H.astype(float), G.astype(float), Q.astype(complex)
    mask = O.UPDATE_G | O.UPDATE_Q
    *_, t_nmf = O.iterate(X, W, H, G, Q, n_iter=4, mask=mask)
    *_, t_free = O.iterate_free(X, O.source_psd(W, H), G, Q, n_iter=4, mask=mask)
    np.testing.assert_allclose(t_free, t_nmf, rtol=1e-12)


def test_wiener_lam_sums_to_mixture_and_matches_direct():
    X, lam, G, Q = _case(F=3, T=5, M=3, N=3, seed=37)
    S = O.separate_lam(X, lam, G, Q)
    np.testing.assert_allclose(S.sum(axis=0), X, atol=1e-12 * np.abs(X).max())
    np.testing.assert_allclose(S, O.separate_direct_lam(X, lam, G, Q), atol=1e-11 * np.abs(X).max())
