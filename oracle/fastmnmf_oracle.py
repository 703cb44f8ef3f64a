"""Float64 CPU oracle of FastMNMF (Sekiguchi et al., EUSIPCO 2019, arXiv 1903.03237).

TEST INFRASTRUCTURE ONLY.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this module.
The product path (the CUDA library and its Python binding) never calls it, and this
module imports nothing from the product package: the two share no code.

What it computes, step by step in the paper's order and notation (NumPy float64 /
complex128; plain ``einsum`` sums, with NumPy choosing the pairwise contraction order,
and explicit Python loops for the iterative projection).  Each function cites the passage it follows:

* source model        lambda_ftn = sum_k w_nkf h_nkt                      (Sec. II-B-2, Eq. 9)
* diagonalised SCMs   Q_f G_nf Q_f^H = Diag(g~_nf),  Q_f = [q_f1..q_fM]^H   (Sec. III-A-1, Eq. 16)
* model power         y~_ftm = sum_n lambda_ftn g~_nfm                     (Sec. III-A-2, below Eq. 17)
* projected power     x~_ftm = |q_fm^H x_ft|^2                             (Sec. III-A-2, below Eq. 17)
* log-likelihood      Eq. 17, with the dropped constant -FTM log(pi) restored
* IP update of Q_f    V_fm, (Q_f V_fm)^-1 e_m, normalisation by q^H V q   (Eqs. 18-20)
* MU of g~            Eq. 21;   MU of W and H   Eqs. 23-24
* MU of lambda        Eq. 22 (unconstrained source model, Sec. III-B-1: FastFCA, Sec. III-C-1)
* Wiener separation   x_ftn = Y_ftn Y_ft^-1 x_ft                          (Sec. II-A-1, Eq. 3)
* front end           STFT with a 1024-point window and a 256-point shift, F = 513 (Sec. IV-A),
                      its inverse by weighted overlap-add, and the initialisation of g~ and Q by
                      spectral decomposition of the initial SCMs (Sec. IV-A)

The spatial-model functions take lambda[f,t,n] itself (``*_lam``); the NMF source model forms
it by Eq. 9 and calls them, the unconstrained model passes its own lambda.

Readings of points where the paper is silent (block order, scale normalisation,
initialisation, the log-likelihood constant) are fixed in ``iterate``,
``normalise`` and ``init_state`` below.

Pins (see tests/test_oracle_*.py): monotone log-likelihood per block (MM / IP
guarantee), q^H V q = 1 and Q V q = e after each IP row update, decorrelated
log-likelihood == full-rank complex-Gaussian log-density built from explicit
covariances, MU numerator minus denominator == finite-difference gradient of the
log-likelihood, IP row == brute-force row maximiser, M=1 reduction to textbook
IS-NMF, Wiener outputs summing to the mixture and equal to the direct full-rank
filter, LL invariance of the normalisation.
"""
from __future__ import annotations

import numpy as np

UPDATE_W = 1
UPDATE_H = 2
UPDATE_G = 4
UPDATE_Q = 8
UPDATE_ALL = UPDATE_W | UPDATE_H | UPDATE_G | UPDATE_Q

# ---------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014), counter form: output i (i = 0, 1, ...) of the
# stream seeded with s is mix(s + (i + 1) * 0x9E3779B97F4A7C15 mod 2^64), where
# mix(z) = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
#          z *= 0x94D049BB133111EB; z ^= z >> 31.
# The initial state of fmnmf_init draws its W, H from this stream; the library
# implements the same published definition independently.
# ---------------------------------------------------------------------------
_MASK64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def _splitmix64_mix(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def splitmix64_uniform(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1): top 53 bits of SplitMix64 outputs start..start+count-1."""
    out = np.empty(count, dtype=np.float64)
    s = seed & _MASK64
    for i in range(count):
        z = _splitmix64_mix((s + (start + i + 1) * _GAMMA) & _MASK64)
        out[i] = (z >> 11) * (1.0 / 9007199254740992.0)
    return out


def init_state(F: int, T: int, M: int, N: int, K: int, seed: int):
    """Initial state of ``fmnmf_init`` (the paper fixes an initialisation only for its
    DP experiments, Sec. IV-A; this is the library's documented one):

    * W[n,k,f] = 0.1 + u_i, i = (n*K + k)*F + f        (u_i the SplitMix64 uniforms)
    * H[n,k,t] = 0.1 + u_j, j = N*K*F + (n*K + k)*T + t
    * g~[n,f,m] = 1 if m == n mod M else 1e-2, then divided by its sum over m
    * Q_f = I (identity diagonaliser)

    Values are rounded to float32, the library's state precision.
    """
    nw, nh = N * K * F, N * K * T
    u = splitmix64_uniform(seed, 0, nw + nh)
    W = (0.1 + u[:nw]).astype(np.float32).astype(np.float64).reshape(N, K, F)
    H = (0.1 + u[nw:]).astype(np.float32).astype(np.float64).reshape(N, K, T)
    G, Q = _init_gq(F, M, N)
    return W, H, G, Q


def _init_gq(F: int, M: int, N: int):
    """g~[n,f,m] = 1 if m == n mod M else 1e-2, divided by its sum over m (float32); Q_f = I."""
    G = np.full((N, F, M), 1e-2)
    for n in range(N):
        G[n, :, n % M] = 1.0
    G = G / G.sum(axis=2, keepdims=True)
    G = G.astype(np.float32).astype(np.float64)
    Q = np.tile(np.eye(M, dtype=np.complex128), (F, 1, 1))
    return G, Q


def init_state_free(F: int, T: int, M: int, N: int, seed: int):
    """Initial state of ``fmnmf_init`` for the unconstrained source model (FastFCA):
    lambda[f,t,n] = 0.1 + u_i with i = (n F + f) T + t (the library stores lambda as
    [N][F][T]), rounded to float32; g~ and Q as in ``init_state``."""
    u = splitmix64_uniform(seed, 0, N * F * T)
    lam = (0.1 + u).astype(np.float32).astype(np.float64).reshape(N, F, T).transpose(1, 2, 0)
    G, Q = _init_gq(F, M, N)
    return np.ascontiguousarray(lam), G, Q


# ---------------------------------------------------------------------------
# Model quantities
# ---------------------------------------------------------------------------
def source_psd(W, H):
    """lambda[f,t,n] = sum_k w_nkf h_nkt  (Sec. II-B-2, Eq. 9)."""
    return np.einsum("nkf,nkt->ftn", W, H, optimize=True)


def model_power(lam, G):
    """y~[f,t,m] = sum_n lambda_ftn g~_nfm  (Sec. III-A-2, definition below Eq. 17)."""
    return np.einsum("ftn,nfm->ftm", lam, G, optimize=True)


def projected_power(Q, X):
    """x~[f,t,m] = |q_fm^H x_ft|^2 = |(Q_f x_ft)_m|^2  (Sec. III-A-2, below Eq. 17;
    row m of Q_f is q_fm^H, Eq. 16)."""
    QX = np.einsum("fmj,ftj->ftm", Q, X, optimize=True)
    return (QX.real ** 2) + (QX.imag ** 2)


def log_det_QQH(Q):
    """log |Q_f Q_f^H| = log |det Q_f|^2 per bin (the last term of Eq. 17)."""
    _, logabs = np.linalg.slogdet(Q)
    return 2.0 * logabs


def loglik_lam(X, lam, G, Q):
    """Decorrelated log-likelihood, Eq. 17:
    sum_{f,t,m} ( -x~/y~ - log y~ ) + T sum_f log|Q_f Q_f^H|  - F T M log(pi).
    The constant -FTM log(pi), dropped by the paper's "=c", is restored so that the
    value is the true log-density of Eq. 2 under the constraint of Eq. 16."""
    F, T, M = X.shape
    xt = projected_power(Q, X)
    yt = model_power(lam, G)
    return (float(np.sum(-xt / yt - np.log(yt))) + T * float(np.sum(log_det_QQH(Q)))
            - F * T * M * np.log(np.pi))


def loglik(X, W, H, G, Q):
    """Eq. 17 for the NMF source model (lambda by Eq. 9)."""
    return loglik_lam(X, source_psd(W, H), G, Q)


def loglik_terms_abs(X, W, H, G, Q):
    """Sum of the absolute values of the terms of Eq. 17 (scale for relative LL errors)."""
    return loglik_terms_abs_lam(X, source_psd(W, H), G, Q)


def loglik_terms_abs_lam(X, lam, G, Q):
    """Sum of the absolute values of the terms of Eq. 17, lambda given."""
    F, T, M = X.shape
    xt = projected_power(Q, X)
    yt = model_power(lam, G)
    return (float(np.sum(np.abs(xt / yt)) + np.sum(np.abs(np.log(yt))))
            + T * float(np.sum(np.abs(log_det_QQH(Q)))) + F * T * M * np.log(np.pi))


def full_rank_covariances(W, H, G, Q):
    """Full-rank covariances of the NMF source model (lambda by Eq. 9)."""
    return full_rank_covariances_lam(source_psd(W, H), G, Q)


def full_rank_covariances_lam(lam, G, Q):
    """Y_ftn = lambda_ftn G_nf with G_nf = Q_f^-1 Diag(g~_nf) Q_f^-H (Eq. 16 solved for
    G_nf), and Y_ft = sum_n Y_ftn (Eq. 2).  Returns (Ysrc[f,t,n,M,M], Y[f,t,M,M])."""
    Qi = np.linalg.inv(Q)                                            # [F,M,M]
    Gfull = np.einsum("fij,nfj,fkj->nfik", Qi, G, Qi.conj(), optimize=True)         # Q^-1 Diag(g) Q^-H
    Ysrc = np.einsum("ftn,nfik->ftnik", lam, Gfull, optimize=True)
    return Ysrc, Ysrc.sum(axis=2)


def loglik_fullrank(X, W, H, G, Q):
    """Full-rank log-density of the NMF source model (lambda by Eq. 9)."""
    return loglik_fullrank_lam(X, source_psd(W, H), G, Q)


def loglik_fullrank_lam(X, lam, G, Q):
    """Log-density of Eq. 2 evaluated directly: sum_{f,t} log CN(x_ft | 0, Y_ft)
    = -sum ( x^H Y^-1 x + log det(pi Y) )  (Eq. 4 with its constant), with Y_ft built
    explicitly from the full-rank SCMs.  Used only as a pin of ``loglik``."""
    _, Y = full_rank_covariances_lam(lam, G, Q)
    M = X.shape[2]
    sol = np.linalg.solve(Y, X[..., None])[..., 0]
    quad = np.einsum("ftm,ftm->ft", X.conj(), sol, optimize=True).real
    _, logabs = np.linalg.slogdet(Y)
    return float(-np.sum(quad) - np.sum(logabs) - X.shape[0] * X.shape[1] * M * np.log(np.pi))


# ---------------------------------------------------------------------------
# Update rules
# ---------------------------------------------------------------------------
def _aux(xt, yt):
    """The two ratios every MU rule is built from: A = y~^-1 x~ y~^-1 and B = y~^-1."""
    return xt / yt ** 2, 1.0 / yt


def mu_W_terms(xt, W, H, G):
    """Numerator and denominator of the W rule (Sec. III-B-2, Eq. 23):
    num[n,k,f] = sum_{t,m} h_nkt g~_nfm x~/y~^2,  den[n,k,f] = sum_{t,m} h_nkt g~_nfm / y~."""
    A, B = _aux(xt, model_power(source_psd(W, H), G))
    num = np.einsum("nkt,nfm,ftm->nkf", H, G, A, optimize=True)
    den = np.einsum("nkt,nfm,ftm->nkf", H, G, B, optimize=True)
    return num, den


def update_W(xt, W, H, G):
    """w_nkf <- w_nkf sqrt(num/den)  (Eq. 23)."""
    num, den = mu_W_terms(xt, W, H, G)
    return W * np.sqrt(num / den)


def mu_H_terms(xt, W, H, G):
    """Numerator and denominator of the H rule (Eq. 24): sums over f and m of
    w_nkf g~_nfm x~/y~^2 and of w_nkf g~_nfm / y~."""
    A, B = _aux(xt, model_power(source_psd(W, H), G))
    num = np.einsum("nkf,nfm,ftm->nkt", W, G, A, optimize=True)
    den = np.einsum("nkf,nfm,ftm->nkt", W, G, B, optimize=True)
    return num, den


def update_H(xt, W, H, G):
    """h_nkt <- h_nkt sqrt(num/den)  (Eq. 24)."""
    num, den = mu_H_terms(xt, W, H, G)
    return H * np.sqrt(num / den)


def mu_G_terms(xt, W, H, G):
    """The g~ rule's terms for the NMF source model (lambda by Eq. 9)."""
    return mu_G_terms_lam(xt, source_psd(W, H), G)


def mu_G_terms_lam(xt, lam, G):
    """Numerator and denominator of the g~ rule (Sec. III-A-2, Eq. 21):
    num[n,f,m] = sum_t lambda_ftn x~/y~^2,  den[n,f,m] = sum_t lambda_ftn / y~."""
    A, B = _aux(xt, model_power(lam, G))
    num = np.einsum("ftn,ftm->nfm", lam, A, optimize=True)
    den = np.einsum("ftn,ftm->nfm", lam, B, optimize=True)
    return num, den


def update_G(xt, W, H, G):
    """g~_nfm <- g~_nfm sqrt(num/den)  (Eq. 21)."""
    num, den = mu_G_terms(xt, W, H, G)
    return G * np.sqrt(num / den)


def update_G_lam(xt, lam, G):
    """Eq. 21 with lambda given."""
    num, den = mu_G_terms_lam(xt, lam, G)
    return G * np.sqrt(num / den)


def mu_lambda_terms(xt, lam, G):
    """Numerator and denominator of the lambda rule of the unconstrained source model
    (Sec. III-B-1, Eq. 22): num[f,t,n] = sum_m g~_nfm x~/y~^2,  den[f,t,n] = sum_m g~_nfm / y~."""
    A, B = _aux(xt, model_power(lam, G))
    num = np.einsum("nfm,ftm->ftn", G, A, optimize=True)
    den = np.einsum("nfm,ftm->ftn", G, B, optimize=True)
    return num, den


def update_lambda(xt, lam, G):
    """lambda_ftn <- lambda_ftn sqrt(num/den)  (Eq. 22)."""
    num, den = mu_lambda_terms(xt, lam, G)
    return lam * np.sqrt(num / den)


def weighted_scm(X, yt):
    """V_fm = (1/T) sum_t x_ft x_ft^H / y~_ftm  (Sec. III-A-2, Eq. 18).  Returns V[f,m,i,j]."""
    T = X.shape[1]
    return np.einsum("fti,ftj,ftm->fmij", X, X.conj(), 1.0 / yt, optimize=True) / T


def update_Q(X, W, H, G, Q, trace=None):
    """The IP update for the NMF source model (lambda by Eq. 9)."""
    return update_Q_lam(X, source_psd(W, H), G, Q, trace)


def update_Q_lam(X, lam, G, Q, trace=None):
    """Iterative projection (Eqs. 18-20), rows in order m = 1..M, each using the
    current Q_f (Eq. 19 has Q_f on the right-hand side):

        q_fm <- (Q_f V_fm)^-1 e_m ;  q_fm <- q_fm / sqrt(q_fm^H V_fm q_fm) ;
        row m of Q_f <- q_fm^H.

    V_fm depends on y~ only, which the Q update does not change, so all V_fm of a bin
    are formed once before its row loop.  ``trace`` (a list) receives, after each row
    update, (f, m, q^H V q, Q_f V_fm q_fm) for the pins."""
    F, T, M = X.shape
    yt = model_power(lam, G)
    V = weighted_scm(X, yt)
    Qn = Q.copy()
    for f in range(F):
        for m in range(M):
            Vfm = V[f, m]
            e = np.zeros(M, dtype=np.complex128)
            e[m] = 1.0
            q = np.linalg.solve(Qn[f] @ Vfm, e)                      # Eq. 19
            s = float(np.real(q.conj() @ Vfm @ q))
            q = q / np.sqrt(s)                                       # Eq. 20
            Qn[f, m, :] = q.conj()                                   # Q_f = [q_f1 .. q_fM]^H
            if trace is not None:
                trace.append((f, m, float(np.real(q.conj() @ Vfm @ q)), Qn[f] @ Vfm @ q))
    return Qn


def normalise(W, H, G, Q):
    """Scale normalisation (the paper is silent; this reading leaves every y~_ftm, every
    x~/y~ and the log-likelihood unchanged in exact arithmetic):

    1. phi_f = tr(Q_f Q_f^H)/M;  Q_f <- Q_f/sqrt(phi_f);  g~_nf <- g~_nf/phi_f
       (x~_ft and y~_ft both scale by 1/phi_f; log|Q Q^H| drops by M log phi_f, which
       the T*M log phi_f rise of -sum log y~ cancels).
    2. nu_nf = sum_m g~_nfm;  g~_nf <- g~_nf/nu_nf;  w_nkf <- w_nkf nu_nf  (lambda g~ fixed).
    3. mu_nk = sum_f w_nkf;   w_nkf <- w_nkf/mu_nk;  h_nkt <- h_nkt mu_nk  (lambda fixed).
    """
    M = Q.shape[1]
    phi = np.einsum("fij,fij->f", Q, Q.conj(), optimize=True).real / M
    Q = Q / np.sqrt(phi)[:, None, None]
    G = G / phi[None, :, None]
    nu = G.sum(axis=2)                                               # [N,F]
    G = G / nu[:, :, None]
    W = W * nu[:, None, :]
    mu = W.sum(axis=2)                                               # [N,K]
    W = W / mu[:, :, None]
    H = H * mu[:, :, None]
    return W, H, G, Q


def iterate(X, W, H, G, Q, n_iter=1, mask=UPDATE_ALL, do_normalise=True, block_ll=None):
    """n_iter FastMNMF iterations (Sec. III-C-2: the NMF source model of Sec. III-B-2
    inside the jointly diagonalisable spatial model of Sec. III-A).  Block order
    (the paper only says the method alternates NTF-style multiplicative updates and
    IP): W (Eq. 23) -> H (Eq. 24) -> g~ (Eq. 21) -> Q (Eqs. 18-20) -> normalise.
    y~ and x~ are recomputed from the current parameters before every block, so each
    block is an exact MM / IP step and the log-likelihood never decreases.

    Returns (W, H, G, Q, ll_trace) with ll_trace[i] the log-likelihood after
    iteration i.  ``block_ll`` (a list), if given, receives the log-likelihood after
    every block."""
    W = np.array(W, dtype=np.float64)
    H = np.array(H, dtype=np.float64)
    G = np.array(G, dtype=np.float64)
    Q = np.array(Q, dtype=np.complex128)
    X = np.asarray(X, dtype=np.complex128)
    trace = []
    for _ in range(n_iter):
        xt = projected_power(Q, X)
        if mask & UPDATE_W:
            W = update_W(xt, W, H, G)
            if block_ll is not None:
                block_ll.append(("W", loglik(X, W, H, G, Q)))
        if mask & UPDATE_H:
            H = update_H(xt, W, H, G)
            if block_ll is not None:
                block_ll.append(("H", loglik(X, W, H, G, Q)))
        if mask & UPDATE_G:
            G = update_G(xt, W, H, G)
            if block_ll is not None:
                block_ll.append(("G", loglik(X, W, H, G, Q)))
        if mask & UPDATE_Q:
            Q = update_Q(X, W, H, G, Q)
            if block_ll is not None:
                block_ll.append(("Q", loglik(X, W, H, G, Q)))
        if do_normalise:
            W, H, G, Q = normalise(W, H, G, Q)
        trace.append(loglik(X, W, H, G, Q))
    return W, H, G, Q, trace


def normalise_free(lam, G, Q):
    """Scale normalisation of the unconstrained source model: steps 1 and 2 of ``normalise``
    with nu_nf scaling lambda_ftn (every t) instead of w_nkf; no step 3 (there is no W, H).
    lambda g~ and the log-likelihood are unchanged in exact arithmetic."""
    M = Q.shape[1]
    phi = np.einsum("fij,fij->f", Q, Q.conj(), optimize=True).real / M
    Q = Q / np.sqrt(phi)[:, None, None]
    G = G / phi[None, :, None]
    nu = G.sum(axis=2)                                               # [N,F]
    G = G / nu[:, :, None]
    lam = lam * nu.T[:, None, :]
    return lam, G, Q


def iterate_free(X, lam, G, Q, n_iter=1, mask=UPDATE_ALL, do_normalise=True, block_ll=None):
    """n_iter FastFCA iterations (Sec. III-C-1: the unconstrained source model of Sec.
    III-B-1 in the jointly diagonalisable spatial model, with the IP update of Q).  Block
    order, as for FastMNMF: lambda (Eq. 22; mask bit UPDATE_W) -> g~ (Eq. 21) -> Q (Eqs.
    18-20) -> normalise, every block from the current parameters.
    Returns (lam, G, Q, ll_trace); lam is [F, T, N]."""
    lam = np.array(lam, dtype=np.float64)
    G = np.array(G, dtype=np.float64)
    Q = np.array(Q, dtype=np.complex128)
    X = np.asarray(X, dtype=np.complex128)
    trace = []
    for _ in range(n_iter):
        xt = projected_power(Q, X)
        if mask & UPDATE_W:
            lam = update_lambda(xt, lam, G)
            if block_ll is not None:
                block_ll.append(("lambda", loglik_lam(X, lam, G, Q)))
        if mask & UPDATE_G:
            G = update_G_lam(xt, lam, G)
            if block_ll is not None:
                block_ll.append(("G", loglik_lam(X, lam, G, Q)))
        if mask & UPDATE_Q:
            Q = update_Q_lam(X, lam, G, Q)
            if block_ll is not None:
                block_ll.append(("Q", loglik_lam(X, lam, G, Q)))
        if do_normalise:
            lam, G, Q = normalise_free(lam, G, Q)
        trace.append(loglik_lam(X, lam, G, Q))
    return lam, G, Q, trace


# ---------------------------------------------------------------------------
# Separation
# ---------------------------------------------------------------------------
def separate(X, W, H, G, Q):
    """Wiener separation for the NMF source model (lambda by Eq. 9)."""
    return separate_lam(X, source_psd(W, H), G, Q)


def separate_lam(X, lam, G, Q):
    """Multichannel Wiener filter of Eq. 3 in the diagonalised form.  Substituting
    G_nf = Q_f^-1 Diag(g~_nf) Q_f^-H (Eq. 16) into Y_ftn Y_ft^-1 gives
    Q_f^-1 Diag(lambda_ftn g~_nf / y~_ft) Q_f, so
        x_ftn = Q_f^-1 ( lambda_ftn g~_nf / y~_ft  (elementwise)  Q_f x_ft ).
    Returns out[n,f,t,m] (every channel of every source image)."""
    yt = model_power(lam, G)
    QX = np.einsum("fmj,ftj->ftm", Q, X, optimize=True)
    Qi = np.linalg.inv(Q)
    gain = np.einsum("ftn,nfm->nftm", lam, G, optimize=True) / yt[None]
    return np.einsum("fij,nftj->nfti", Qi, gain * QX[None], optimize=True)


def separate_direct(X, W, H, G, Q):
    """Direct Wiener filter for the NMF source model (lambda by Eq. 9)."""
    return separate_direct_lam(X, source_psd(W, H), G, Q)


def separate_direct_lam(X, lam, G, Q):
    """Eq. 3 evaluated literally, x_ftn = Y_ftn Y_ft^-1 x_ft with explicit full-rank
    matrices (pin of ``separate``)."""
    Ysrc, Y = full_rank_covariances_lam(lam, G, Q)
    sol = np.linalg.solve(Y, X[..., None])[..., 0]                   # Y_ft^-1 x_ft
    return np.einsum("ftnij,ftj->nfti", Ysrc, sol, optimize=True)


# ---------------------------------------------------------------------------
# Front end (Sec. IV-A): the STFT of the paper's experiments (window of 1024 points, F = 513,
# shift of 256 points), its inverse, and the initialisation of g~ and Q by spectral
# decomposition.  The paper names neither the window nor the framing: a periodic Hann window,
# frames starting at sample t * hop with zeros past the end, and synthesis with the same window
# normalised by the overlap-added squared window are this library's reading.
# ---------------------------------------------------------------------------
def stft_frames(S: int, L: int = 1024, hop: int = 256) -> int:
    """Number of frames of a signal of S samples: 1 + ceil((S - L) / hop), at least 1."""
    return 1 if S <= L else 1 + -(-(S - L) // hop)


def hann(L: int) -> np.ndarray:
    """Periodic Hann window w_j = (1 - cos(2 pi j / L)) / 2."""
    return 0.5 - 0.5 * np.cos(2.0 * np.pi * np.arange(L) / L)


def stft(x, L: int = 1024, hop: int = 256):
    """X[f, t, m] = sum_j w_j x_m[t hop + j] exp(-2 pi i f j / L), f = 0..L/2 (x: [M, S] real;
    samples past S are zero).  The DFT of each windowed frame is numpy's rfft."""
    x = np.asarray(x, dtype=np.float64)
    M, S = x.shape
    T = stft_frames(S, L, hop)
    pad = np.zeros((M, (T - 1) * hop + L))
    pad[:, :S] = x
    w = hann(L)
    frames = np.stack([pad[:, t * hop:t * hop + L] * w for t in range(T)], axis=1)   # [M, T, L]
    return np.fft.rfft(frames, axis=2).transpose(2, 1, 0)                              # [F, T, M]


def istft(Y, S: int, L: int = 1024, hop: int = 256):
    """Inverse of ``stft`` for a batch Y[b, f, t, m]: each frame's inverse real DFT (numpy's
    irfft) times the window, overlap-added, divided by the overlap-added squared window
    sum_t w_{s - t hop}^2 (samples where that sum is below 1e-10 of its largest value are
    zero).  Returns y[b, m, s], s < S."""
    Y = np.asarray(Y, dtype=np.complex128)
    B, F, T, M = Y.shape
    w = hann(L)
    frames = np.fft.irfft(Y.transpose(0, 3, 2, 1), n=L, axis=3) * w                 # [B, M, T, L]
    n_out = (T - 1) * hop + L
    y = np.zeros((B, M, n_out))
    den = np.zeros(n_out)
    for t in range(T):
        y[:, :, t * hop:t * hop + L] += frames[:, :, t]
        den[t * hop:t * hop + L] += w * w
    ok = den > 1e-10 * den.max()
    y[:, :, ok] /= den[ok]
    y[:, :, ~ok] = 0.0
    return y[:, :, :S]


def spectral_init(X, N: int):
    """Initial g~ and Q by spectral decomposition (Sec. IV-A): G_1f = (1/T) sum_t x_ft x_ft^H
    (the average observed SCM), G_nf = I for n >= 2; with G_1f = U_f Diag(e_f) U_f^H (numpy's
    eigh, eigenvalues ordered largest first), Q_f = U_f^H jointly diagonalises every G_nf:
    g~_1f = e_f and g~_nf = 1 (Q_f I Q_f^H = I).  Returns G[n, f, m] (before the nu
    normalisation) and Q[f, m, j]."""
    X = np.asarray(X, dtype=np.complex128)
    F, T, M = X.shape
    R = np.einsum("fti,ftj->fij", X, X.conj(), optimize=True) / T
    e, U = np.linalg.eigh(R)                       # ascending
    e, U = e[:, ::-1], U[:, :, ::-1]
    Q = U.conj().transpose(0, 2, 1)                # rows = conjugated eigenvectors
    G = np.ones((N, F, M))
    G[0] = e
    return G, Q


def spectral_init_state(X, W, G, Q):
    """The spectral initialisation with the library's nu normalisation: g~_nf /= sum_m g~_nfm
    and w_nkf *= that sum (lambda g~ unchanged); Q_f is unitary, so phi_f = 1."""
    nu = G.sum(axis=2)
    return W * nu[:, None, :], G / nu[:, :, None], Q
