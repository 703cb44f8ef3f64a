"""Float64 CPU oracle of FastMNMF-DP (Sec. III-B-3 and Sec. III-C-3 of arXiv 1903.03237).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module; the
product path never calls it, and it imports nothing from the product package.

The model: source 0 (the paper's n = 1, speech) has the deep-prior PSD
    lambda_ft0 = u_f v_t [sigma^2_theta(z_t)]_f                           (Sec. II-B-3)
with a latent z_t in R^D per frame; sources 1..N-1 (noise) have the NMF PSD of Eq. 9.  The
spatial model is the jointly diagonalisable one of Sec. III-A, so g~, Q, x~, y~ and the
log-likelihood (Eq. 17) are the functions of ``fastmnmf_oracle`` that take lambda itself.

Steps of one iteration, in the paper's order where it gives one (readings of the rest below):
* Z: Metropolis sampling (Sec. III-B-3): per frame, a proposal z' = z + sqrt(eps) xi with
  xi ~ N(0, I) is accepted when log u < log gamma_t, u ~ U(0, 1), where log gamma_t is the
  change of the diagonalised log-likelihood when lambda_ft0 alone changes (the reconstruction
  without source 0, y~^{-0}, is held fixed).  Several proposals per iteration, all with y~^{-0},
  g~ and x~ of the iteration's start (Sec. III-B-3, "updated several times without updating Y").
  The draws xi and log u are inputs: the method's random numbers are passed in.
* u, v: the MU rules of Sec. III-B-3 (square roots of ratios of sums of
  v_t r_tf g~_0fm x~/y~^2 and v_t r_tf g~_0fm / y~ over t, m; and of u_f r_tf (...) over f, m).
* W, H of the noise sources: Eqs. 23-24 with y~ including source 0.
* g~ (Eq. 21), Q (Eqs. 18-20), normalisation.

Readings where the paper is silent:
* decoder sigma^2_theta: the two-layer perceptron of the VAE speech models the paper cites,
  r = exp(W2 tanh(W1 z + b1) + b2) (hidden width Hd, exp output so that r > 0); its weights
  are inputs (trained weights are not available; tests and benchmarks use seeded random ones);
* the acceptance ratio has no prior term: log gamma is the likelihood ratio the paper states;
* block order Z -> u -> v -> W -> H -> g~ -> Q -> normalise, each block from the current
  parameters (y~, x~ recomputed), as in ``fastmnmf_oracle.iterate``;
* normalisation: phi and nu as for FastMNMF (nu_0f scales u_f, nu_nf scales w_nkf), then
  mu_0 = sum_f u_f (u / mu_0, v * mu_0) and mu_nk = sum_f w_nkf (w / mu, h * mu); every
  lambda g~ and the log-likelihood are unchanged in exact arithmetic.

Shapes: X [F,T,M]; Z [T,D]; u [F]; v [T]; W [N-1,K,F]; H [N-1,K,T]; G [N,F,M]; Q [F,M,M];
decoder theta = (W1 [Hd,D], b1 [Hd], W2 [F,Hd], b2 [F]); xi [S,T,D] and logu [S,T] per
iteration (S proposals per frame).  lambda is [F,T,N] as in ``fastmnmf_oracle``.

Pins: tests/test_oracle_pins_dp.py.
"""
from __future__ import annotations

import numpy as np

from oracle.fastmnmf_oracle import (
    _aux, model_power, projected_power, source_psd, loglik_lam, update_G_lam, update_Q_lam)


# ---------------------------------------------------------------------------
# Source model of the speech source (Sec. II-B-3)
# ---------------------------------------------------------------------------
def decoder(Z, theta):
    """r_t = sigma^2_theta(z_t) = exp(W2 tanh(W1 z_t + b1) + b2): [T,D] -> [T,F]."""
    W1, b1, W2, b2 = (np.asarray(a, dtype=np.float64) for a in theta)
    hidden = np.tanh(np.asarray(Z, dtype=np.float64) @ W1.T + b1)   # [T,Hd]
    return np.exp(hidden @ W2.T + b2)                                # [T,F]


def speech_psd(u, v, R):
    """lambda_ft0 = u_f v_t r_tf: [F,T]."""
    return u[:, None] * v[None, :] * R.T


def dp_lambda(u, v, R, W, H):
    """lambda[f,t,n]: source 0 from the deep prior, sources 1.. from Eq. 9."""
    F, T = u.shape[0], v.shape[0]
    lam = np.empty((F, T, 1 + W.shape[0]))
    lam[:, :, 0] = speech_psd(u, v, R)
    if W.shape[0]:
        lam[:, :, 1:] = source_psd(W, H)
    return lam


# ---------------------------------------------------------------------------
# Metropolis sampling of Z (Sec. III-B-3)
# ---------------------------------------------------------------------------
def log_gamma(xt, lam0_new, lam0_old, g0, y_rest):
    """log gamma_t = - sum_{f,m} ( x~/(lam_new g~_0 + y~^{-0}) - x~/(lam_old g~_0 + y~^{-0}) )
                     - sum_{f,m} log( (lam_new g~_0 + y~^{-0}) / (lam_old g~_0 + y~^{-0}) ).
    xt, y_rest [F,T,M]; lam0_* [F,T]; g0 [F,M].  Returns [T]."""
    y_new = lam0_new[:, :, None] * g0[:, None, :] + y_rest
    y_old = lam0_old[:, :, None] * g0[:, None, :] + y_rest
    return (-np.sum(xt / y_new - xt / y_old, axis=(0, 2))
            - np.sum(np.log(y_new / y_old), axis=(0, 2)))


def metropolis(xt, Z, u, v, theta, G, lam_rest, xi, logu, eps, history=None):
    """S Metropolis proposals per frame: for s = 0..S-1, z' = z + sqrt(eps) xi[s]; accept where
    logu[s] < log gamma.  y~^{-0} = sum_{n>=1} lambda_ftn g~_nfm is held fixed (Sec. III-B-3).
    lam_rest [F,T,N-1].  Returns (Z, R, accepted count).  ``history`` (a list) receives
    (log gamma [T], accepted mask [T]) of every proposal."""
    Z = np.array(Z, dtype=np.float64)
    R = decoder(Z, theta)
    y_rest = (model_power(lam_rest, G[1:]) if lam_rest.shape[2]
              else np.zeros(xt.shape))
    g0 = G[0]
    se = np.sqrt(eps)
    n_acc = 0
    for s in range(xi.shape[0]):
        Zp = Z + se * xi[s]
        Rp = decoder(Zp, theta)
        lg = log_gamma(xt, speech_psd(u, v, Rp), speech_psd(u, v, R), g0, y_rest)
        acc = logu[s] < lg
        Z[acc] = Zp[acc]
        R[acc] = Rp[acc]
        n_acc += int(acc.sum())
        if history is not None:
            history.append((lg, acc))
    return Z, R, n_acc


# ---------------------------------------------------------------------------
# Multiplicative updates (Sec. III-B-3 for u, v; Eqs. 23-24 for the noise W, H)
# ---------------------------------------------------------------------------
def _source_terms(xt, lam, G, n):
    """P[f,t] = sum_m g~_nfm x~/y~^2 and R[f,t] = sum_m g~_nfm / y~ for source n."""
    A, B = _aux(xt, model_power(lam, G))
    return (np.einsum("fm,ftm->ft", G[n], A, optimize=True),
            np.einsum("fm,ftm->ft", G[n], B, optimize=True))


def mu_U_terms(xt, u, v, R, W, H, G):
    """num_f = sum_{t,m} v_t r_tf g~_0fm x~/y~^2,  den_f = sum_{t,m} v_t r_tf g~_0fm / y~."""
    P, B = _source_terms(xt, dp_lambda(u, v, R, W, H), G, 0)
    return (P * v[None, :] * R.T).sum(axis=1), (B * v[None, :] * R.T).sum(axis=1)


def update_U(xt, u, v, R, W, H, G):
    """u_f <- u_f sqrt(num_f / den_f)."""
    num, den = mu_U_terms(xt, u, v, R, W, H, G)
    return u * np.sqrt(num / den)


def mu_V_terms(xt, u, v, R, W, H, G):
    """num_t = sum_{f,m} u_f r_tf g~_0fm x~/y~^2,  den_t = sum_{f,m} u_f r_tf g~_0fm / y~."""
    P, B = _source_terms(xt, dp_lambda(u, v, R, W, H), G, 0)
    return (P * u[:, None] * R.T).sum(axis=0), (B * u[:, None] * R.T).sum(axis=0)


def update_V(xt, u, v, R, W, H, G):
    """v_t <- v_t sqrt(num_t / den_t)."""
    num, den = mu_V_terms(xt, u, v, R, W, H, G)
    return v * np.sqrt(num / den)


def mu_Wn_terms(xt, u, v, R, W, H, G):
    """Eq. 23 for the noise sources n = 1..N-1 with y~ including source 0:
    num[n-1,k,f] = sum_{t,m} h_nkt g~_nfm x~/y~^2,  den likewise with 1/y~."""
    A, B = _aux(xt, model_power(dp_lambda(u, v, R, W, H), G))
    num = np.einsum("nkt,nfm,ftm->nkf", H, G[1:], A, optimize=True)
    den = np.einsum("nkt,nfm,ftm->nkf", H, G[1:], B, optimize=True)
    return num, den


def update_Wn(xt, u, v, R, W, H, G):
    num, den = mu_Wn_terms(xt, u, v, R, W, H, G)
    return W * np.sqrt(num / den)


def mu_Hn_terms(xt, u, v, R, W, H, G):
    """Eq. 24 for the noise sources with y~ including source 0."""
    A, B = _aux(xt, model_power(dp_lambda(u, v, R, W, H), G))
    num = np.einsum("nkf,nfm,ftm->nkt", W, G[1:], A, optimize=True)
    den = np.einsum("nkf,nfm,ftm->nkt", W, G[1:], B, optimize=True)
    return num, den


def update_Hn(xt, u, v, R, W, H, G):
    num, den = mu_Hn_terms(xt, u, v, R, W, H, G)
    return H * np.sqrt(num / den)


# ---------------------------------------------------------------------------
# Normalisation, log-likelihood, iteration
# ---------------------------------------------------------------------------
def normalise_dp(u, v, W, H, G, Q):
    """phi_f = tr(Q_f Q_f^H)/M (Q / sqrt(phi), g~ / phi); nu_nf = sum_m g~_nfm (g~ / nu,
    u * nu_0, w_n * nu_n); mu_0 = sum_f u_f (u / mu_0, v * mu_0); mu_nk = sum_f w_nkf
    (w / mu, h * mu).  Each step leaves every lambda g~ product scaled so that y~/phi and
    x~/phi move together, and the log-likelihood unchanged."""
    M = Q.shape[1]
    phi = np.einsum("fij,fij->f", Q, Q.conj(), optimize=True).real / M
    Q = Q / np.sqrt(phi)[:, None, None]
    G = G / phi[None, :, None]
    nu = G.sum(axis=2)                                               # [N,F]
    G = G / nu[:, :, None]
    u = u * nu[0]
    W = W * nu[1:, None, :]
    mu0 = u.sum()
    u = u / mu0
    v = v * mu0
    mu = W.sum(axis=2)                                               # [N-1,K]
    W = W / mu[:, :, None]
    H = H * mu[:, :, None]
    return u, v, W, H, G, Q


def loglik_dp(X, Z, u, v, W, H, G, Q, theta):
    """Eq. 17 (with its constant) for the deep-prior + NMF source models."""
    return loglik_lam(X, dp_lambda(u, v, decoder(Z, theta), W, H), G, Q)


def iterate_dp(X, Z, u, v, W, H, G, Q, theta, xi, logu, eps, n_iter=1, do_normalise=True,
               block_ll=None, accepted=None):
    """n_iter FastMNMF-DP iterations (Sec. III-C-3).  xi [n_iter,S,T,D] and logu [n_iter,S,T]
    are the Metropolis draws of each iteration.  Block order Z -> u -> v -> W -> H -> g~ ->
    Q -> normalise; y~ and x~ from the current parameters before every block.
    Returns (Z, u, v, W, H, G, Q, ll_trace).  ``block_ll`` receives (block, LL) after every
    block; ``accepted`` (a list) the number of accepted proposals of each iteration."""
    Z = np.array(Z, dtype=np.float64)
    u = np.array(u, dtype=np.float64)
    v = np.array(v, dtype=np.float64)
    W = np.array(W, dtype=np.float64)
    H = np.array(H, dtype=np.float64)
    G = np.array(G, dtype=np.float64)
    Q = np.array(Q, dtype=np.complex128)
    X = np.asarray(X, dtype=np.complex128)

    def ll(R):
        return loglik_lam(X, dp_lambda(u, v, R, W, H), G, Q)

    trace = []
    for i in range(n_iter):
        xt = projected_power(Q, X)
        lam_rest = source_psd(W, H) if W.shape[0] else np.zeros(xt.shape[:2] + (0,))
        Z, R, n_acc = metropolis(xt, Z, u, v, theta, G, lam_rest, xi[i], logu[i], eps)
        if accepted is not None:
            accepted.append(n_acc)
        if block_ll is not None:
            block_ll.append(("Z", ll(R)))
        u = update_U(xt, u, v, R, W, H, G)
        if block_ll is not None:
            block_ll.append(("u", ll(R)))
        v = update_V(xt, u, v, R, W, H, G)
        if block_ll is not None:
            block_ll.append(("v", ll(R)))
        if W.shape[0]:
            W = update_Wn(xt, u, v, R, W, H, G)
            if block_ll is not None:
                block_ll.append(("W", ll(R)))
            H = update_Hn(xt, u, v, R, W, H, G)
            if block_ll is not None:
                block_ll.append(("H", ll(R)))
        lam = dp_lambda(u, v, R, W, H)
        G = update_G_lam(xt, lam, G)
        if block_ll is not None:
            block_ll.append(("G", ll(R)))
        Q = update_Q_lam(X, lam, G, Q)
        if block_ll is not None:
            block_ll.append(("Q", ll(R)))
        if do_normalise:
            u, v, W, H, G, Q = normalise_dp(u, v, W, H, G, Q)
        trace.append(ll(R))
    return Z, u, v, W, H, G, Q, trace
