"""Planted mistakes in a copy of the FastMNMF-DP oracle, each caught by a check that holds for
the oracle as written (CPU only).  The checks rest on what the paper and the mathematics fix:
  * log gamma_t is the change of the log-likelihood of Eq. 17 (computed by the FastMNMF
    oracle, pinned to the full-rank density) when lambda_ft0 of frame t alone changes, both
    for the function itself and for the values the Metropolis loop decides with;
  * with log u = -inf every proposal is accepted and r follows z through the decoder;
  * num - den of each MU rule is the gradient of the log-likelihood (central differences);
  * with r = 1 the u, v rules are the FastMNMF W, H rules of a rank-1 source;
  * the normalisation leaves the log-likelihood unchanged;
  * the decoder is odd-symmetric in log r around b2 when b1 = 0 (tanh is odd, exp output).
"""
import types

import numpy as np
import pytest

import oracle.fastmnmf_oracle as O
import oracle.fastmnmf_dp_oracle as D

SRC = open(D.__file__).read()

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _mutant(old: str, new: str):
    assert SRC.count(old) == 1, old
    mod = types.ModuleType("dp_oracle_mutant")
    exec(compile(SRC.replace(old, new), "dp_oracle_mutant", "exec"), mod.__dict__)
    return mod


def _case(seed=0, F=5, T=8, M=3, N=3, K=2, Dd=3, Hd=5):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((F, T, M)) + 1j * rng.standard_normal((F, T, M))) / np.sqrt(2)
    Z = rng.standard_normal((T, Dd))
    u = rng.uniform(0.5, 1.5, F)
    v = rng.uniform(0.5, 1.5, T)
    W = rng.uniform(0.3, 1.5, (N - 1, K, F))
    H = rng.uniform(0.3, 1.5, (N - 1, K, T))
    G = rng.dirichlet(np.ones(M), size=(N, F)) + 0.05
    Q = np.eye(M)[None] + 0.3 * (rng.standard_normal((F, M, M)) + 1j * rng.standard_normal((F, M, M)))
    theta = (rng.standard_normal((Hd, Dd)), 0.1 * rng.standard_normal(Hd), rng.standard_normal((F, Hd)) / 2,
             rng.standard_normal(F) / 2)
    return X, Z, u, v, W, H, G, Q, theta


def _ll(D_, X, u, v, R, W, H, G, Q):
    return O.loglik_lam(X, D_.dp_lambda(u, v, R, W, H), G, Q)


# ---- checks ----------------------------------------------------------------------------------

def check_log_gamma(D_):
    X, Z, u, v, W, H, G, Q, theta = _case(1)
    xt = O.projected_power(Q, X)
    R = D.decoder(Z, theta)
    Rp = D.decoder(Z + 0.3, theta)
    lg = D_.log_gamma(xt, D.speech_psd(u, v, Rp), D.speech_psd(u, v, R), G[0],
                      O.model_power(O.source_psd(W, H), G[1:]))
    lam = D.dp_lambda(u, v, R, W, H)
    ll0 = O.loglik_lam(X, lam, G, Q)
    for t in range(X.shape[1]):
        lt = lam.copy()
        lt[:, t, 0] = D.speech_psd(u, v, Rp)[:, t]
        if abs(O.loglik_lam(X, lt, G, Q) - ll0 - lg[t]) > 1e-9 * abs(ll0):
            return False
    return True


def check_metropolis_decides_with_loglik_change(D_):
    X, Z, u, v, W, H, G, Q, theta = _case(2)
    T = X.shape[1]
    xt = O.projected_power(Q, X)
    xi = np.random.default_rng(5).standard_normal((1, T, Z.shape[1]))
    hist = []
    D_.metropolis(xt, Z, u, v, theta, G, O.source_psd(W, H), xi, np.full((1, T), np.inf), 0.04, history=hist)
    lam = D.dp_lambda(u, v, D.decoder(Z, theta), W, H)
    ll0 = O.loglik_lam(X, lam, G, Q)
    Rp = D.decoder(Z + 0.2 * xi[0], theta)
    for t in range(T):
        lt = lam.copy()
        lt[:, t, 0] = D.speech_psd(u, v, Rp)[:, t]
        if abs(O.loglik_lam(X, lt, G, Q) - ll0 - hist[0][0][t]) > 1e-9 * abs(ll0):
            return False
    return True


def check_accept_all(D_):
    X, Z, u, v, W, H, G, Q, theta = _case(3)
    T = X.shape[1]
    xt = O.projected_power(Q, X)
    xi = np.random.default_rng(6).standard_normal((3, T, Z.shape[1]))
    Za, Ra, na = D_.metropolis(xt, Z, u, v, theta, G, O.source_psd(W, H), xi, np.full((3, T), -np.inf), 0.01)
    return (na == 3 * T and np.allclose(Za, Z + 0.1 * xi.sum(axis=0), rtol=1e-13, atol=1e-13)
            and np.allclose(Ra, D.decoder(Za, theta), rtol=1e-13))


def _grad(D_, which):
    X, Z, u, v, W, H, G, Q, theta = _case(4)
    xt = O.projected_power(Q, X)
    R = D.decoder(Z, theta)
    h = 1e-6
    fn = {"u": D_.mu_U_terms, "v": D_.mu_V_terms, "W": D_.mu_Wn_terms, "H": D_.mu_Hn_terms}[which]
    num, den = fn(xt, u, v, R, W, H, G)
    arrs = {"u": u, "v": v, "W": W, "H": H}
    a = arrs[which]
    for idx in list(np.ndindex(a.shape))[:: max(1, a.size // 5)]:
        ap, am = a.copy(), a.copy()
        ap[idx] += h
        am[idx] -= h
        args_p = dict(arrs, **{which: ap})
        args_m = dict(arrs, **{which: am})
        g = (_ll(D, X, args_p["u"], args_p["v"], R, args_p["W"], args_p["H"], G, Q)
             - _ll(D, X, args_m["u"], args_m["v"], R, args_m["W"], args_m["H"], G, Q)) / (2 * h)
        if abs(g - (num[idx] - den[idx])) > 1e-5 * (abs(num[idx]) + abs(den[idx])):
            return False
    return True


def check_u_gradient(D_):
    return _grad(D_, "u")


def check_v_gradient(D_):
    return _grad(D_, "v")


def check_w_gradient(D_):
    return _grad(D_, "W")


def check_h_gradient(D_):
    return _grad(D_, "H")


def check_rank1_rules(D_):
    X, Z, u, v, W, H, G, Q, theta = _case(5, K=1)
    F, T = X.shape[:2]
    R = np.ones((T, F))
    xt = O.projected_power(Q, X)
    Wb = np.concatenate([u[None, None, :], W], axis=0)
    Hb = np.concatenate([v[None, None, :], H], axis=0)
    return (np.allclose(D_.update_U(xt, u, v, R, W, H, G), O.update_W(xt, Wb, Hb, G)[0, 0], rtol=1e-12)
            and np.allclose(D_.update_V(xt, u, v, R, W, H, G), O.update_H(xt, Wb, Hb, G)[0, 0], rtol=1e-12))


def check_normalise_keeps_loglik(D_):
    X, Z, u, v, W, H, G, Q, theta = _case(6)
    R = D.decoder(Z, theta)
    u2, v2, W2, H2, G2, Q2 = D_.normalise_dp(u, v, W, H, G, Q)
    a, b = _ll(D, X, u, v, R, W, H, G, Q), _ll(D, X, u2, v2, R, W2, H2, G2, Q2)
    return abs(a - b) <= 1e-11 * abs(a)


def check_decoder_odd(D_):
    rng = np.random.default_rng(7)
    th = (rng.standard_normal((5, 3)), np.zeros(5), rng.standard_normal((6, 5)), rng.standard_normal(6))
    z = rng.standard_normal((4, 3))
    with np.errstate(all="ignore"):
        s = np.log(D_.decoder(z, th)) + np.log(D_.decoder(-z, th))
    return bool(np.allclose(s, 2 * th[3][None, :], rtol=0, atol=1e-12))


MUTANTS = [
    ("log_gamma_log_sign", "            - np.sum(np.log(y_new / y_old), axis=(0, 2)))",
     "            + np.sum(np.log(y_new / y_old), axis=(0, 2)))", check_log_gamma),
    ("log_gamma_swapped_ratio", "-np.sum(xt / y_new - xt / y_old, axis=(0, 2))",
     "-np.sum(xt / y_old - xt / y_new, axis=(0, 2))", check_log_gamma),
    ("y_rest_wrong_sources", "model_power(lam_rest, G[1:])", "model_power(lam_rest, G[:-1])",
     check_metropolis_decides_with_loglik_change),
    ("old_lambda_from_proposal", "speech_psd(u, v, Rp), speech_psd(u, v, R), g0",
     "speech_psd(u, v, Rp), speech_psd(u, v, Rp), g0", check_metropolis_decides_with_loglik_change),
    ("accept_direction", "acc = logu[s] < lg", "acc = logu[s] > lg", check_accept_all),
    ("r_not_updated", "        R[acc] = Rp[acc]\n", "", check_accept_all),
    ("step_without_sqrt", "se = np.sqrt(eps)", "se = eps", check_accept_all),
    ("u_rule_uses_u", "return (P * v[None, :] * R.T).sum(axis=1), (B * v[None, :] * R.T).sum(axis=1)",
     "return (P * v[None, :] * R.T).sum(axis=1), (B * R.T).sum(axis=1)", check_u_gradient),
    ("v_rule_wrong_axis", "return (P * u[:, None] * R.T).sum(axis=0), (B * u[:, None] * R.T).sum(axis=0)",
     "return (P * u[:, None] * R.T).sum(axis=0), (B * u[:, None]).sum(axis=0)", check_v_gradient),
    ("w_rule_wrong_g", 'num = np.einsum("nkt,nfm,ftm->nkf", H, G[1:], A, optimize=True)',
     'num = np.einsum("nkt,nfm,ftm->nkf", H, G[:-1], A, optimize=True)', check_w_gradient),
    ("h_rule_no_square", "    A, B = _aux(xt, model_power(dp_lambda(u, v, R, W, H), G))\n"
     "    num = np.einsum(\"nkf,nfm,ftm->nkt\"",
     "    A, B = _aux(xt, model_power(dp_lambda(u, v, R, W, H), G))\n    A = A * model_power(dp_lambda(u, v, R, W, H), G)\n"
     "    num = np.einsum(\"nkf,nfm,ftm->nkt\"", check_h_gradient),
    ("v_rule_no_sqrt", "return v * np.sqrt(num / den)", "return v * (num / den)", check_rank1_rules),
    ("normalise_v_divided", "v = v * mu0", "v = v / mu0", check_normalise_keeps_loglik),
    ("normalise_nu_to_v", "u = u * nu[0]", "v = v * nu[0].mean()", check_normalise_keeps_loglik),
    ("decoder_relu", "hidden = np.tanh(", "hidden = np.maximum(0.0, ", check_decoder_odd),
    ("decoder_no_exp", "return np.exp(hidden @ W2.T + b2)", "return np.abs(hidden @ W2.T + b2)", check_decoder_odd),
]


@pytest.mark.parametrize("name,old,new,check", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, check):
    assert check(D), f"check {check.__name__} fails on the oracle itself"
    mod = _mutant(old, new)
    try:
        caught = not check(mod)
    except Exception:
        caught = True      # an exception (shape, domain) is a caught mistake too
    assert caught, f"planted mistake {name} not caught by {check.__name__}"
