"""Pins of the float64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form, an
invariant the paper guarantees, a brute-force search, a textbook special case, or a
published test vector.  They run on the CPU (no GPU marker).
"""
import os

import numpy as np
import pytest

from oracle import fastmnmf_oracle as O
from paper_1903_03237_gb300.synth import make_mixture, make_state


def _case(F=6, T=40, M=3, N=2, K=3, seed=3):
    mix = make_mixture(F, T, M, N, K, seed)
    W, H, G, Q = make_state(F, T, M, N, K, seed)
    return (mix.X.astype(np.complex128), W.astype(np.float64), H.astype(np.float64),
            G.astype(np.float64), Q.astype(np.complex128))


# --- SplitMix64 ---------------------------------------------------------------------
def test_splitmix64_published_vector():
    # published SplitMix64 outputs for seed 1234567 (fixture with its citation)
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")
    expect = [int(l) for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(expect) == 5
    u = O.splitmix64_uniform(1234567, 0, 5)
    np.testing.assert_array_equal(u, np.array([(e >> 11) / 2.0 ** 53 for e in expect]))


def test_init_state_layout():
    W, H, G, Q = O.init_state(5, 7, 3, 4, 2, seed=11)
    assert W.shape == (4, 2, 5) and H.shape == (4, 2, 7) and G.shape == (4, 5, 3)
    assert np.all(W >= 0.1) and np.all(W < 1.1) and np.all(H >= 0.1)
    np.testing.assert_allclose(G.sum(axis=2), 1.0, rtol=1e-6)
    assert np.argmax(G[3, 0]) == 3 % 3
    np.testing.assert_array_equal(Q, np.tile(np.eye(3), (5, 1, 1)))
    u = O.splitmix64_uniform(11, 0, 4 * 2 * 5 + 1)
    assert W[0, 0, 0] == np.float32(0.1 + u[0])
    assert H[0, 0, 0] == np.float32(0.1 + u[4 * 2 * 5])


# --- Log-likelihood: decorrelated form == full-rank log-density -----------------------
@pytest.mark.parametrize("M,N", [(1, 1), (2, 3), (3, 2), (4, 4)])
def test_loglik_equals_fullrank_density(M, N):
    X, W, H, G, Q = _case(F=4, T=9, M=M, N=N, K=3, seed=M * 10 + N)
    a = O.loglik(X, W, H, G, Q)
    b = O.loglik_fullrank(X, W, H, G, Q)
    assert abs(a - b) <= 1e-10 * abs(b)


def test_loglik_constant_single_gaussian():
    # M=1, N=1, K=1, Q=1, G=1: the density is that of independent CN(0, w h) scalars:
    # log p = -|x|^2/(w h) - log(pi w h)
    F, T = 3, 4
    rng = np.random.default_rng(0)
    X = (rng.standard_normal((F, T, 1)) + 1j * rng.standard_normal((F, T, 1)))
    W = rng.uniform(0.5, 2.0, (1, 1, F))
    H = rng.uniform(0.5, 2.0, (1, 1, T))
    G = np.ones((1, F, 1))
    Q = np.ones((F, 1, 1), dtype=complex)
    lam = W[0, 0][:, None] * H[0, 0][None, :]
    ref = np.sum(-np.abs(X[..., 0]) ** 2 / lam - np.log(np.pi * lam))
    assert abs(O.loglik(X, W, H, G, Q) - ref) < 1e-12 * abs(ref)


# --- MU rules: numerator - denominator == gradient of the log-likelihood --------------
def _fd_grad(fun, P, idx, h=1e-6):
    Pp = P.copy(); Pp[idx] += h
    Pm = P.copy(); Pm[idx] -= h
    return (fun(Pp) - fun(Pm)) / (2 * h)


def test_mu_terms_are_loglik_gradient():
    X, W, H, G, Q = _case(F=5, T=11, M=3, N=2, K=2, seed=5)
    xt = O.projected_power(Q, X)
    rng = np.random.default_rng(1)
    numW, denW = O.mu_W_terms(xt, W, H, G)
    numH, denH = O.mu_H_terms(xt, W, H, G)
    numG, denG = O.mu_G_terms(xt, W, H, G)
    for _ in range(6):
        i = tuple(rng.integers(0, s) for s in W.shape)
        g = _fd_grad(lambda P: O.loglik(X, P, H, G, Q), W, i)
        assert abs((numW - denW)[i] - g) <= 1e-5 * max(1.0, abs(g))
        i = tuple(rng.integers(0, s) for s in H.shape)
        g = _fd_grad(lambda P: O.loglik(X, W, P, G, Q), H, i)
        assert abs((numH - denH)[i] - g) <= 1e-5 * max(1.0, abs(g))
        i = tuple(rng.integers(0, s) for s in G.shape)
        g = _fd_grad(lambda P: O.loglik(X, W, H, P, Q), G, i)
        assert abs((numG - denG)[i] - g) <= 1e-5 * max(1.0, abs(g))


# --- Monotonicity (MM and IP guarantees) ----------------------------------------------
def test_loglik_monotone_per_block_and_iteration():
    X, W, H, G, Q = _case(F=7, T=30, M=3, N=3, K=4, seed=9)
    blocks = []
    _, _, _, _, trace = O.iterate(X, W, H, G, Q, n_iter=8, block_ll=blocks)
    ll0 = O.loglik(X, W, H, G, Q)
    seq = [ll0] + [v for _, v in blocks]
    d = np.diff(seq)
    assert np.all(d >= -1e-9 * np.abs(seq[1:])), (d.min(), blocks)
    assert np.all(np.diff([ll0] + trace) >= -1e-9 * abs(ll0))


# --- IP pins --------------------------------------------------------------------------
def test_ip_normalisation_and_projection():
    X, W, H, G, Q = _case(F=4, T=25, M=4, N=2, K=2, seed=13)
    tr = []
    O.update_Q(X, W, H, G, Q, trace=tr)
    assert len(tr) == 4 * 4
    for f, m, qvq, QVq in tr:
        assert abs(qvq - 1.0) < 1e-12
        e = np.zeros(4); e[m] = 1.0
        np.testing.assert_allclose(QVq, e, atol=1e-12)


def test_ip_row_is_brute_force_maximiser():
    # With lambda and g~ fixed, the last row updated maximises the log-likelihood over
    # that row: no random perturbation of it increases Eq. 17.
    X, W, H, G, Q = _case(F=3, T=20, M=3, N=2, K=2, seed=17)
    Qn = O.update_Q(X, W, H, G, Q)
    base = O.loglik(X, W, H, G, Qn)
    rng = np.random.default_rng(2)
    for scale in (1e-1, 1e-2, 1e-3):
        for _ in range(20):
            P = Qn.copy()
            f = rng.integers(0, 3)
            P[f, 2, :] += scale * (rng.standard_normal(3) + 1j * rng.standard_normal(3))
            assert O.loglik(X, W, H, G, P) <= base + 1e-9 * abs(base)


def test_ip_equals_closed_form_for_M1():
    # M=1: Q_f is a scalar q*; the IP rule gives |q|^2 = 1 / V_f  (V_f = mean |x|^2/y~).
    X, W, H, G, Q = _case(F=4, T=15, M=1, N=2, K=2, seed=19)
    Qn = O.update_Q(X, W, H, G, Q)
    yt = O.model_power(O.source_psd(W, H), G)
    V = np.mean(np.abs(X[..., 0]) ** 2 / yt[..., 0], axis=1)
    np.testing.assert_allclose(np.abs(Qn[:, 0, 0]) ** 2, 1.0 / V, rtol=1e-12)


# --- M = 1 reduces to IS-NMF ----------------------------------------------------------
def test_m1_reduces_to_is_nmf():
    F, T, K = 9, 13, 3
    rng = np.random.default_rng(4)
    X = (rng.standard_normal((F, T, 1)) + 1j * rng.standard_normal((F, T, 1))) * rng.uniform(0.5, 3, (F, 1, 1))
    W = rng.uniform(0.2, 1.0, (1, K, F))
    H = rng.uniform(0.2, 1.0, (1, K, T))
    G = np.ones((1, F, 1))
    Q = np.ones((F, 1, 1), dtype=complex)
    Wo, Ho, _, _, _ = O.iterate(X, W, H, G, Q, n_iter=3, mask=O.UPDATE_W | O.UPDATE_H, do_normalise=False)
    # Textbook IS-NMF multiplicative updates with the MM exponent 1/2 (Nakano et al. 2010),
    # in matrix form: V ~ Wt Ht with Wt = F x K, Ht = K x T.
    V = np.abs(X[..., 0]) ** 2
    Wt, Ht = W[0].T.copy(), H[0].copy()
    for _ in range(3):
        L = Wt @ Ht
        Wt = Wt * np.sqrt(((V / L ** 2) @ Ht.T) / ((1 / L) @ Ht.T))
        L = Wt @ Ht
        Ht = Ht * np.sqrt((Wt.T @ (V / L ** 2)) / (Wt.T @ (1 / L)))
    np.testing.assert_allclose(Wo[0].T, Wt, rtol=1e-12)
    np.testing.assert_allclose(Ho[0], Ht, rtol=1e-12)


# --- Normalisation --------------------------------------------------------------------
def test_normalise_invariance():
    X, W, H, G, Q = _case(F=5, T=12, M=3, N=3, K=2, seed=23)
    W2, H2, G2, Q2 = O.normalise(W, H, G, Q)
    a, b = O.loglik(X, W, H, G, Q), O.loglik(X, W2, H2, G2, Q2)
    assert abs(a - b) < 1e-12 * abs(a)
    np.testing.assert_allclose(O.projected_power(Q2, X) / O.model_power(O.source_psd(W2, H2), G2),
                               O.projected_power(Q, X) / O.model_power(O.source_psd(W, H), G), rtol=1e-12)
    np.testing.assert_allclose(np.einsum("fij,fij->f", Q2, Q2.conj()).real, 3.0, rtol=1e-12)
    np.testing.assert_allclose(G2.sum(axis=2), 1.0, rtol=1e-12)
    np.testing.assert_allclose(W2.sum(axis=2), 1.0, rtol=1e-12)


def test_trajectory_independent_of_normalisation():
    X, W, H, G, Q = _case(F=5, T=20, M=2, N=2, K=3, seed=29)
    *_, t1 = O.iterate(X, W, H, G, Q, n_iter=5, do_normalise=True)
    *_, t2 = O.iterate(X, W, H, G, Q, n_iter=5, do_normalise=False)
    np.testing.assert_allclose(t1, t2, rtol=1e-10)


# --- Wiener separation ----------------------------------------------------------------
def test_wiener_sums_to_mixture_and_matches_direct():
    X, W, H, G, Q = _case(F=4, T=6, M=3, N=3, K=2, seed=31)
    S = O.separate(X, W, H, G, Q)
    np.testing.assert_allclose(S.sum(axis=0), X, atol=1e-12 * np.abs(X).max())
    np.testing.assert_allclose(S, O.separate_direct(X, W, H, G, Q), atol=1e-11 * np.abs(X).max())


def test_wiener_single_source_is_identity():
    X, W, H, G, Q = _case(F=3, T=5, M=2, N=1, K=2, seed=37)
    np.testing.assert_allclose(O.separate(X, W, H, G, Q)[0], X, atol=1e-12)


# --- Generator sanity (the data model of Eq. 1-2 / Eq. 16) ----------------------------
def test_generator_covariance():
    mix = make_mixture(2, 20000, 2, 1, 1, seed=41)
    # With N=K=1 and H ~ Gamma(1,1): E[x x^H] = E[w h] Q^-1 Diag(g) Q^-H per bin.
    for f in range(2):
        Qi = np.linalg.inv(mix.Q[f])
        x = mix.X[f].astype(np.complex128)
        C = x.T @ x.conj() / x.shape[0]
        ref = mix.W[0, 0, f] * mix.H[0, 0].mean() * Qi @ np.diag(mix.G[0, f]) @ Qi.conj().T
        np.testing.assert_allclose(C, ref, atol=0.05 * np.abs(ref).max())
