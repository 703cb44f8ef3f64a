"""Planted mistakes in a copy of the oracle, each caught by a check that holds for the
oracle as written.  CPU only.

Every case edits one line of the oracle's source text (the mistake a restatement of the
paper could plausibly contain), loads the edited text as a separate module, and runs a check
built from what the paper and the mathematics fix, not from the oracle's own output:
  * the decorrelated log-likelihood (Eq. 17) equals the full-rank complex-Gaussian density
    built from Q_f^-1 Diag(y~) Q_f^-H (Eqs. 2, 16);
  * num - den of an MU rule is the gradient of Eq. 17 (central differences);
  * after a row update of the IP step, q^H V q = 1 and Q_f V_fm q_fm = e_m (Eqs. 19-20), with
    V_fm formed here from its definition (Eq. 18);
  * with M = 1 and g~, Q fixed the W rule is the textbook IS-NMF multiplicative update;
  * the scale normalisation leaves the log-likelihood unchanged;
  * the Wiener images add up to the mixture (Eq. 3);
  * with M = N = 1 the lambda rule (Eq. 22) has the closed form x~^(1 - 2^-k) lambda_0^(2^-k);
  * the STFT equals the DFT sum written out, its inverse recovers the signal, and the spectral
    initialisation diagonalises the average SCM with the eigenvalues largest first.
The check must pass on the oracle and fail on the mutant.
"""
import types

import numpy as np
import pytest

import oracle.fastmnmf_oracle as O

SRC = open(O.__file__).read()


def _mutant(old: str, new: str):
    assert SRC.count(old) == 1, old
    mod = types.ModuleType("oracle_mutant")
    exec(compile(SRC.replace(old, new), "oracle_mutant", "exec"), mod.__dict__)
    return mod


def _case(F=4, T=12, M=3, N=2, K=2, seed=0):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((F, T, M)) + 1j * rng.standard_normal((F, T, M))) / np.sqrt(2)
    W = rng.uniform(0.3, 1.5, (N, K, F))
    H = rng.uniform(0.3, 1.5, (N, K, T))
    G = rng.dirichlet(np.ones(M), size=(N, F)) + 0.05
    Q = np.eye(M)[None] + 0.3 * (rng.standard_normal((F, M, M)) + 1j * rng.standard_normal((F, M, M)))
    return X, W, H, G, Q


# ---- checks (each returns True when the module behaves as the paper fixes) -----------------

def check_loglik_equals_full_rank(O_):
    X, W, H, G, Q = _case(seed=1)
    a, b = O_.loglik(X, W, H, G, Q), O_.loglik_fullrank(X, W, H, G, Q)
    return abs(a - b) <= 1e-9 * abs(b)


def _grad_check(O_, which):
    X, W, H, G, Q = _case(seed=2)
    xt = O_.projected_power(Q, X)
    arrs = {"W": W, "H": H, "G": G}
    num, den = {"W": O_.mu_W_terms, "H": O_.mu_H_terms, "G": O_.mu_G_terms}[which](xt, W, H, G)
    rng = np.random.default_rng(3)
    h = 1e-6
    for _ in range(8):
        A = arrs[which]
        i = tuple(rng.integers(0, s) for s in A.shape)
        Ap, Am = A.copy(), A.copy()
        Ap[i] += h
        Am[i] -= h
        kw = dict(arrs)
        kw[which] = Ap
        lp = O.loglik(X, kw["W"], kw["H"], kw["G"], Q)      # the reference log-likelihood
        kw[which] = Am
        lm = O.loglik(X, kw["W"], kw["H"], kw["G"], Q)
        g = (lp - lm) / (2 * h)
        if abs((num - den)[i] - g) > 1e-5 * max(1.0, abs(g)):
            return False
    return True


def check_w_gradient(O_):
    return _grad_check(O_, "W")


def check_h_gradient(O_):
    return _grad_check(O_, "H")


def check_g_gradient(O_):
    return _grad_check(O_, "G")


def check_ip_rows(O_):
    # V_fm from Eq. 18 written out here; after the sweep the last row of each bin satisfies
    # q^H V q = 1 and Q_f V_fm q_fm = e_m
    X, W, H, G, Q = _case(seed=4)
    F, T, M = X.shape
    yt = np.einsum("ftn,nfm->ftm", np.einsum("nkf,nkt->ftn", W, H), G)
    Qn = O_.update_Q(X, W, H, G, Q)
    m = M - 1
    for f in range(F):
        V = sum(np.outer(X[f, t], X[f, t].conj()) / yt[f, t, m] for t in range(T)) / T
        q = Qn[f, m].conj()
        if abs(np.real(q.conj() @ V @ q) - 1.0) > 1e-9:
            return False
        e = np.zeros(M)
        e[m] = 1.0
        if np.abs(Qn[f] @ V @ q - e).max() > 1e-9:
            return False
    return True


def check_isnmf_reduction(O_):
    # M = N = 1, g~ = 1, Q = 1: Nakano's IS-NMF rule W <- W sqrt((V/L^2) H^T / ((1/L) H^T))
    rng = np.random.default_rng(5)
    F, T, K = 6, 9, 3
    X = (rng.standard_normal((F, T, 1)) + 1j * rng.standard_normal((F, T, 1)))
    W = rng.uniform(0.2, 1.2, (1, K, F))
    H = rng.uniform(0.2, 1.2, (1, K, T))
    G = np.ones((1, F, 1))
    Q = np.ones((F, 1, 1), dtype=complex)
    V = np.abs(X[:, :, 0]) ** 2
    Wm, Hm = W[0].T, H[0]                                   # [F, K], [K, T]
    L = Wm @ Hm
    ref = Wm * np.sqrt(((V / L ** 2) @ Hm.T) / ((1.0 / L) @ Hm.T))
    got = O_.update_W(O_.projected_power(Q, X), W, H, G)[0].T
    return np.allclose(got, ref, rtol=1e-12)


def check_normalise_keeps_loglik(O_):
    X, W, H, G, Q = _case(seed=6)
    a = O.loglik(X, W, H, G, Q)
    b = O.loglik(X, *O_.normalise(W, H, G, Q))
    return abs(a - b) <= 1e-10 * abs(a)


def check_wiener_sums_to_mixture(O_):
    X, W, H, G, Q = _case(seed=7)
    S = O_.separate(X, W, H, G, Q)
    return np.abs(S.sum(axis=0) - X).max() <= 1e-10 * np.abs(X).max()


def check_fca_closed_form(O_):
    # M = N = 1 with g~, Q fixed: Eq. 22 is lambda <- sqrt(lambda x~), so after k steps
    # lambda = x~^(1 - 2^-k) lambda_0^(2^-k)
    rng = np.random.default_rng(8)
    X = rng.standard_normal((3, 5, 1)) + 1j * rng.standard_normal((3, 5, 1))
    lam0 = rng.uniform(0.1, 3.0, (3, 5, 1))
    lam, _, _, _ = O_.iterate_free(X, lam0, np.ones((1, 3, 1)), np.ones((3, 1, 1), dtype=complex), n_iter=3,
                                   mask=O.UPDATE_W, do_normalise=False)
    return np.allclose(lam, (np.abs(X) ** 2) ** (1 - 2.0 ** -3) * lam0 ** (2.0 ** -3), rtol=1e-12)


def check_stft_dft_sum(O_):
    # X[f, t, m] = sum_j w_j x_m[t hop + j] exp(-2 pi i f j / L), written out
    L, hop, S = 16, 4, 30
    x = np.random.default_rng(9).standard_normal((1, S))
    X = O_.stft(x, L, hop)
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(L) / L)
    for t in range(X.shape[1]):
        seg = np.zeros(L)
        n = min(L, S - t * hop)
        seg[:n] = x[0, t * hop:t * hop + n]
        ref = np.array([np.sum(w * seg * np.exp(-2j * np.pi * f * np.arange(L) / L)) for f in range(L // 2 + 1)])
        if np.abs(X[:, t, 0] - ref).max() > 1e-12:
            return False
    return True


def check_istft_round_trip(O_):
    L, hop, S = 64, 16, 500
    x = np.random.default_rng(10).standard_normal((2, S))
    y = O_.istft(O.stft(x, L, hop)[None], S, L, hop)[0]
    return np.abs(y[:, L:-L] - x[:, L:-L]).max() < 1e-9


def check_spectral_init(O_):
    # Q_f G_1f Q_f^H = Diag(g~_1f) with g~_1f in descending order, G_1f the average SCM
    rng = np.random.default_rng(11)
    X = rng.standard_normal((3, 40, 3)) + 1j * rng.standard_normal((3, 40, 3))
    G, Q = O_.spectral_init(X, 2)
    for f in range(3):
        R = np.einsum("ti,tj->ij", X[f], X[f].conj()) / 40
        D = Q[f] @ R @ Q[f].conj().T
        if np.abs(D - np.diag(G[0, f])).max() > 1e-10 * np.abs(R).max() or np.any(np.diff(G[0, f]) > 0):
            return False
    return True


# ---- the planted mistakes -------------------------------------------------------------------

# the phi step of the NMF model's normalisation (the same lines open the unconstrained model's:
# the span runs to the line that only the NMF model has)
_i = SRC.index("    Q = Q / np.sqrt(phi)[:, None, None]", SRC.index("def normalise(W, H, G, Q):"))
_PHI_OLD = SRC[_i:SRC.index("    W = W * nu[:, None, :]", _i) + len("    W = W * nu[:, None, :]")]

MUTANTS = [
    ("no square root in the W rule", "    return W * np.sqrt(num / den)", "    return W * (num / den)",
     check_isnmf_reduction),
    ("1/T missing from V_fm", "optimize=True) / T\n\n\ndef update_Q(", "optimize=True)\n\n\ndef update_Q(",
     check_ip_rows),
    ("row of Q_f without the conjugate", "            Qn[f, m, :] = q.conj()", "            Qn[f, m, :] = q",
     check_ip_rows),
    ("V_fm Q_f instead of Q_f V_fm", "np.linalg.solve(Qn[f] @ Vfm, e)", "np.linalg.solve(Vfm @ Qn[f], e)",
     check_ip_rows),
    ("transposed Q_f in x~", 'QX = np.einsum("fmj,ftj->ftm", Q, X, optimize=True)\n    return (QX.real',
     'QX = np.einsum("fjm,ftj->ftm", Q, X, optimize=True)\n    return (QX.real', check_loglik_equals_full_rank),
    ("sign of the x~/y~ term", "np.sum(-xt / yt - np.log(yt))", "np.sum(xt / yt - np.log(yt))",
     check_loglik_equals_full_rank),
    ("T missing before the log-determinant", "+ T * float(np.sum(log_det_QQH(Q)))", "+ float(np.sum(log_det_QQH(Q)))",
     check_loglik_equals_full_rank),
    ("A = x~/y~ instead of x~/y~^2", "    return xt / yt ** 2, 1.0 / yt", "    return xt / yt, 1.0 / yt",
     check_w_gradient),
    ("wrong bin in the H numerator", 'num = np.einsum("nkf,nfm,ftm->nkt", W, G, A, optimize=True)',
     'num = np.einsum("nkf,nfm,ftm->nkt", np.roll(W, 1, axis=2), G, A, optimize=True)', check_h_gradient),
    ("perturbed g~ numerator", 'num = np.einsum("ftn,ftm->nfm", lam, A, optimize=True)',
     'num = 1.01 * np.einsum("ftn,ftm->nfm", lam, A, optimize=True)', check_g_gradient),
    ("phi applied the wrong way", _PHI_OLD, _PHI_OLD.replace("Q = Q / np.sqrt", "Q = Q * np.sqrt", 1),
     check_normalise_keeps_loglik),
    ("Q^H instead of Q^-1 in the Wiener filter", "    Qi = np.linalg.inv(Q)\n    gain",
     "    Qi = Q.conj().transpose(0, 2, 1)\n    gain", check_wiener_sums_to_mixture),
    ("no square root in the lambda rule (Eq. 22)", "    return lam * np.sqrt(num / den)", "    return lam * (num / den)",
     check_fca_closed_form),
    ("STFT frames without the window", "pad[:, t * hop:t * hop + L] * w for t", "pad[:, t * hop:t * hop + L] for t",
     check_stft_dft_sum),
    ("inverse STFT without the squared-window division", "    y[:, :, ok] /= den[ok]\n", "\n",
     check_istft_round_trip),
    ("Q_f = U_f instead of U_f^H", "    Q = U.conj().transpose(0, 2, 1)", "    Q = U.copy()", check_spectral_init),
    ("eigenvalues in ascending order", "    e, U = e[:, ::-1], U[:, :, ::-1]\n", "\n", check_spectral_init),
]


@pytest.mark.parametrize("name,old,new,check", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(name, old, new, check):
    assert check(O), f"{check.__name__} fails on the oracle itself"
    assert not check(_mutant(old, new)), f"{name}: {check.__name__} does not catch it"
