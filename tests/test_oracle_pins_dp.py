"""Pins of the FastMNMF-DP oracle (Sec. II-B-3, Sec. III-B-3, Sec. III-C-3) against what the
mathematics fixes, independent of the oracle's own formulas:

* decoder r = exp(W2 tanh(W1 z + b1) + b2): constant output when the hidden layer is off,
  odd symmetry of tanh, invariance under a permutation of the hidden units, the first-order
  expansion at z = 0 (central differences), saturation of tanh to sign();
* log gamma_t equals the change of the full log-likelihood (Eq. 17, itself pinned to the
  full-rank density) when lambda_ft0 of frame t alone changes;
* Metropolis: every proposal accepted for log u = -inf, none for +inf, and the acceptance
  frequency of one proposal per frame equals sum_t min(1, gamma_t) within a binomial bound;
* MU rules of u, v and the noise W, H: numerator - denominator == finite-difference
  gradient of the log-likelihood; every block raises the log-likelihood;
* with the decoder fixed to r = 1 the model is NMF with a rank-1 speech source, so the u, v
  and noise W rules equal the pinned FastMNMF W, H rules, and a whole iteration with no
  accepted proposal equals a FastMNMF iteration (N = 1, K = 1);
* normalisation: log-likelihood and lambda g~ unchanged, sum_m g~ = 1, sum_f u = sum_f w = 1.
"""
import numpy as np
import pytest

from oracle import fastmnmf_oracle as O
from oracle import fastmnmf_dp_oracle as D
from paper_1903_03237_gb300.synth import make_mixture, make_dp_state, make_decoder, make_dp_draws

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _case(F=9, T=12, M=3, N=3, K=2, Dd=4, Hd=8, seed=5):
    mix = make_mixture(F, T, M, N, K, seed)
    X = mix.X.astype(np.complex128)
    Z, u, v, W, H, G, Q = (a.astype(np.complex128) if np.iscomplexobj(a) else a.astype(np.float64)
                           for a in make_dp_state(F, T, M, N, K, Dd, seed))
    theta = tuple(a.astype(np.float64) for a in make_decoder(F, Dd, Hd, seed))
    return X, Z, u, v, W, H, G, Q, theta


# ---- decoder -------------------------------------------------------------------------
def test_decoder_constant_without_hidden_layer():
    rng = np.random.default_rng(0)
    Dd, Hd, F = 5, 7, 11
    theta = (np.zeros((Hd, Dd)), np.zeros(Hd), rng.standard_normal((F, Hd)), rng.standard_normal(F))
    R = D.decoder(rng.standard_normal((6, Dd)), theta)
    assert np.allclose(R, np.exp(theta[3])[None, :], rtol=1e-15, atol=0)


def test_decoder_odd_symmetry():
    rng = np.random.default_rng(1)
    Dd, Hd, F = 5, 7, 11
    theta = (rng.standard_normal((Hd, Dd)), np.zeros(Hd), rng.standard_normal((F, Hd)), rng.standard_normal(F))
    Z = rng.standard_normal((6, Dd))
    s = np.log(D.decoder(Z, theta)) + np.log(D.decoder(-Z, theta))
    assert np.allclose(s, 2 * theta[3][None, :], rtol=0, atol=1e-12)


def test_decoder_hidden_permutation():
    rng = np.random.default_rng(2)
    Dd, Hd, F = 4, 9, 10
    W1, b1, W2, b2 = rng.standard_normal((Hd, Dd)), rng.standard_normal(Hd), rng.standard_normal((F, Hd)), rng.standard_normal(F)
    p = rng.permutation(Hd)
    Z = rng.standard_normal((5, Dd))
    assert np.allclose(D.decoder(Z, (W1, b1, W2, b2)), D.decoder(Z, (W1[p], b1[p], W2[:, p], b2)), rtol=1e-14)


def test_decoder_first_order_expansion():
    rng = np.random.default_rng(3)
    Dd, Hd, F = 4, 6, 8
    W1, b1, W2, b2 = rng.standard_normal((Hd, Dd)), rng.standard_normal(Hd), rng.standard_normal((F, Hd)), rng.standard_normal(F)
    jac = W2 @ np.diag(1.0 - np.tanh(b1) ** 2) @ W1          # d log r / dz at z = 0
    h = 1e-5
    for d in range(Dd):
        e = np.zeros((1, Dd))
        e[0, d] = h
        fd = (np.log(D.decoder(e, (W1, b1, W2, b2))) - np.log(D.decoder(-e, (W1, b1, W2, b2))))[0] / (2 * h)
        assert np.allclose(fd, jac[:, d], rtol=1e-7, atol=1e-8)


def test_decoder_saturation():
    rng = np.random.default_rng(4)
    Dd, Hd, F = 3, 5, 7
    W1, b1, W2, b2 = rng.standard_normal((Hd, Dd)), rng.standard_normal(Hd), rng.standard_normal((F, Hd)), rng.standard_normal(F)
    z = rng.standard_normal((1, Dd)) * 1e4
    expect = b2 + W2 @ np.sign(W1 @ z[0] + b1)
    assert np.allclose(np.log(D.decoder(z, (W1, b1, W2, b2)))[0], expect, rtol=0, atol=1e-12)


# ---- acceptance ratio ----------------------------------------------------------------
def test_log_gamma_is_loglik_change():
    X, Z, u, v, W, H, G, Q, theta = _case()
    T = X.shape[1]
    xt = O.projected_power(Q, X)
    R = D.decoder(Z, theta)
    Zp = Z + 0.3 * np.random.default_rng(9).standard_normal(Z.shape)
    Rp = D.decoder(Zp, theta)
    y_rest = O.model_power(O.source_psd(W, H), G[1:])
    lg = D.log_gamma(xt, D.speech_psd(u, v, Rp), D.speech_psd(u, v, R), G[0], y_rest)
    lam = D.dp_lambda(u, v, R, W, H)
    ll0 = O.loglik_lam(X, lam, G, Q)
    for t in range(T):
        lam_t = lam.copy()
        lam_t[:, t, 0] = D.speech_psd(u, v, Rp)[:, t]
        assert abs((O.loglik_lam(X, lam_t, G, Q) - ll0) - lg[t]) < 1e-9 * abs(ll0)


def test_metropolis_accept_all_and_none():
    X, Z, u, v, W, H, G, Q, theta = _case()
    T, Dd = Z.shape
    xt = O.projected_power(Q, X)
    xi, _ = make_dp_draws(1, 5, T, Dd, 3)
    xi = xi[0].astype(np.float64)
    lam_rest = O.source_psd(W, H)
    eps = 1e-2
    Za, Ra, na = D.metropolis(xt, Z, u, v, theta, G, lam_rest, xi, np.full((5, T), -np.inf), eps)
    assert na == 5 * T
    assert np.allclose(Za, Z + np.sqrt(eps) * xi.sum(axis=0), rtol=1e-14, atol=1e-14)
    assert np.allclose(Ra, D.decoder(Za, theta), rtol=1e-14)
    Zn, Rn, nn = D.metropolis(xt, Z, u, v, theta, G, lam_rest, xi, np.full((5, T), np.inf), eps)
    assert nn == 0 and np.array_equal(Zn, Z)


def test_metropolis_acceptance_frequency():
    # one proposal per frame; accepted with probability min(1, gamma_t)
    X, Z, u, v, W, H, G, Q, theta = _case(F=6, T=4000, M=2, N=2, K=2, Dd=3, Hd=6, seed=11)
    T, Dd = Z.shape
    xt = O.projected_power(Q, X)
    xi, logu = make_dp_draws(1, 1, T, Dd, 12)
    lam_rest = O.source_psd(W, H)
    hist = []
    _, _, na = D.metropolis(xt, Z, u, v, theta, G, lam_rest, xi[0].astype(np.float64),
                            logu[0].astype(np.float64), 0.05, history=hist)
    p = np.minimum(1.0, np.exp(hist[0][0]))
    assert 0.05 < p.mean() < 0.95                       # a case where acceptance is random
    assert abs(na - p.sum()) < 4.0 * np.sqrt(np.sum(p * (1 - p)))


# ---- multiplicative updates ----------------------------------------------------------
def _ll(X, u, v, R, W, H, G, Q):
    return O.loglik_lam(X, D.dp_lambda(u, v, R, W, H), G, Q)


def test_mu_terms_are_gradients():
    X, Z, u, v, W, H, G, Q, theta = _case()
    xt = O.projected_power(Q, X)
    R = D.decoder(Z, theta)
    h = 1e-6
    nu_, du_ = D.mu_U_terms(xt, u, v, R, W, H, G)
    nv_, dv_ = D.mu_V_terms(xt, u, v, R, W, H, G)
    nw_, dw_ = D.mu_Wn_terms(xt, u, v, R, W, H, G)
    nh_, dh_ = D.mu_Hn_terms(xt, u, v, R, W, H, G)
    for f in (0, 4, 8):
        up, um = u.copy(), u.copy()
        up[f] += h
        um[f] -= h
        g = (_ll(X, up, v, R, W, H, G, Q) - _ll(X, um, v, R, W, H, G, Q)) / (2 * h)
        assert abs(g - (nu_[f] - du_[f])) < 1e-5 * (abs(nu_[f]) + abs(du_[f]))
    for t in (0, 5, 11):
        vp, vm = v.copy(), v.copy()
        vp[t] += h
        vm[t] -= h
        g = (_ll(X, u, vp, R, W, H, G, Q) - _ll(X, u, vm, R, W, H, G, Q)) / (2 * h)
        assert abs(g - (nv_[t] - dv_[t])) < 1e-5 * (abs(nv_[t]) + abs(dv_[t]))
    for (n, k, f) in ((0, 0, 1), (1, 1, 7)):
        Wp, Wm = W.copy(), W.copy()
        Wp[n, k, f] += h
        Wm[n, k, f] -= h
        g = (_ll(X, u, v, R, Wp, H, G, Q) - _ll(X, u, v, R, Wm, H, G, Q)) / (2 * h)
        assert abs(g - (nw_[n, k, f] - dw_[n, k, f])) < 1e-5 * (abs(nw_[n, k, f]) + abs(dw_[n, k, f]))
    for (n, k, t) in ((0, 1, 2), (1, 0, 10)):
        Hp, Hm = H.copy(), H.copy()
        Hp[n, k, t] += h
        Hm[n, k, t] -= h
        g = (_ll(X, u, v, R, W, Hp, G, Q) - _ll(X, u, v, R, W, Hm, G, Q)) / (2 * h)
        assert abs(g - (nh_[n, k, t] - dh_[n, k, t])) < 1e-5 * (abs(nh_[n, k, t]) + abs(dh_[n, k, t]))


def test_every_update_block_raises_loglik():
    X, Z, u, v, W, H, G, Q, theta = _case(F=12, T=30, M=3, N=3, K=3, Dd=4, Hd=8, seed=21)
    xi, logu = make_dp_draws(3, 4, 30, 4, 21)
    bl = []
    D.iterate_dp(X, Z, u, v, W, H, G, Q, theta, xi, logu, 1e-3, n_iter=3, block_ll=bl)
    prev = None
    for name, ll in bl:
        if prev is not None and name != "Z":
            assert ll >= prev - 1e-9 * abs(prev), (name, ll - prev)
        prev = ll


# ---- reduction to FastMNMF with r = 1 ------------------------------------------------
def _unit_decoder(F, Dd, Hd):
    return (np.zeros((Hd, Dd)), np.zeros(Hd), np.zeros((F, Hd)), np.zeros(F))


def test_rules_reduce_to_nmf_rules():
    X, Z, u, v, W, H, G, Q, theta = _case(K=1, N=3)
    F = X.shape[0]
    R = D.decoder(Z, _unit_decoder(F, Z.shape[1], 8))
    assert np.all(R == 1.0)
    xt = O.projected_power(Q, X)
    Wb = np.concatenate([u[None, None, :], W], axis=0)           # speech as a rank-1 NMF source
    Hb = np.concatenate([v[None, None, :], H], axis=0)
    Wn = O.update_W(xt, Wb, Hb, G)
    Hn = O.update_H(xt, Wb, Hb, G)
    assert np.allclose(D.update_U(xt, u, v, R, W, H, G), Wn[0, 0], rtol=1e-12)
    assert np.allclose(D.update_Wn(xt, u, v, R, W, H, G), Wn[1:], rtol=1e-12)
    assert np.allclose(D.update_V(xt, u, v, R, W, H, G), Hn[0, 0], rtol=1e-12)
    assert np.allclose(D.update_Hn(xt, u, v, R, W, H, G), Hn[1:], rtol=1e-12)


def test_iteration_reduces_to_fastmnmf():
    X, Z, u, v, W, H, G, Q, theta = _case(M=3, N=1, K=1, seed=8)
    F, T, M = X.shape
    G = G[:1]
    th = _unit_decoder(F, Z.shape[1], 8)
    xi, logu = make_dp_draws(3, 2, T, Z.shape[1], 8)
    out = D.iterate_dp(X, Z, u, v, W[:0], H[:0], G, Q, th, xi, np.full_like(logu, np.inf), 1e-3, n_iter=3)
    ref = O.iterate(X, u[None, None, :], v[None, None, :], G, Q, n_iter=3)
    assert np.array_equal(out[0], Z)
    assert np.allclose(out[1], ref[0][0, 0], rtol=1e-11)
    assert np.allclose(out[2], ref[1][0, 0], rtol=1e-11)
    assert np.allclose(out[5], ref[2], rtol=1e-11)
    assert np.allclose(out[6], ref[3], rtol=1e-11, atol=1e-12)
    assert np.allclose(out[7], ref[4], rtol=1e-12)


# ---- normalisation -------------------------------------------------------------------
def test_normalise_dp_invariants():
    X, Z, u, v, W, H, G, Q, theta = _case()
    R = D.decoder(Z, theta)
    u2, v2, W2, H2, G2, Q2 = D.normalise_dp(u, v, W, H, G, Q)
    ll1 = _ll(X, u, v, R, W, H, G, Q)
    ll2 = _ll(X, u2, v2, R, W2, H2, G2, Q2)
    assert abs(ll1 - ll2) < 1e-11 * abs(ll1)
    M = Q.shape[1]
    phi = np.einsum("fij,fij->f", Q, Q.conj()).real / M
    lg1 = np.einsum("ftn,nfm->nftm", D.dp_lambda(u, v, R, W, H), G) / phi[None, :, None, None]
    lg2 = np.einsum("ftn,nfm->nftm", D.dp_lambda(u2, v2, R, W2, H2), G2)
    assert np.allclose(lg1, lg2, rtol=1e-12)
    assert np.allclose(G2.sum(axis=2), 1.0, rtol=1e-14)
    assert np.isclose(u2.sum(), 1.0, rtol=1e-14)
    assert np.allclose(W2.sum(axis=2), 1.0, rtol=1e-14)
