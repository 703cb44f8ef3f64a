"""Shared helpers of the GPU parity tests (error metrics and state round-trips).

Two kinds of error are reported for every result:

* ``rel``       ||a - b||_2 / ||b||_2 over the whole tensor;
* ``elem_rel``  the largest per-element relative error, max_i |a_i - b_i| / (|b_i| + tau * s_i),
  where s_i is the natural magnitude an absolute rounding error of entry i scales with:
  - W, H, g~ (each entry is its own product of sums of positive terms): s = 0, a pure
    per-element relative error;
  - Q: the norm of the row q_fm^H the entry belongs to (Eqs. 19-20 form each row as one
    vector, so its rounding is relative to the row, not to a small entry of it);
  - separated images: the norm of the mixture x_ft at that point (Eq. 3 filters x_ft;
    a weak source's image carries rounding of the size of the mixture, not of itself).
  ``tau`` is stated beside each assertion.
"""
import numpy as np

from oracle import fastmnmf_oracle as O


def rel(a, b):
    """||a - b||_2 / ||b||_2 (per tensor)."""
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def maxrel(a, b):
    """max |a - b| / max |b|."""
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def elem_rel(a, b, scale=None, tau=0.0):
    """max_i |a_i - b_i| / (|b_i| + tau * scale_i); scale defaults to max|b| (broadcast)."""
    a = np.asarray(a)
    b = np.asarray(b)
    d = np.abs(a.astype(np.complex128) - b.astype(np.complex128))
    if scale is None:
        scale = np.max(np.abs(b))
    den = np.abs(b) + tau * np.asarray(scale, dtype=np.float64)
    return float(np.max(d / np.maximum(den, 1e-300)))


def q_row_scale(Q):
    """Per-entry scale of Q[f, m, j]: the norm of row m of Q_f."""
    return np.linalg.norm(np.asarray(Q, dtype=np.complex128), axis=2, keepdims=True) * np.ones(Q.shape)


def image_scale(X, N):
    """Per-entry scale of the separated images S[n, f, t, m]: the norm of x_ft."""
    nx = np.linalg.norm(np.asarray(X, dtype=np.complex128), axis=2, keepdims=True)   # [F, T, 1]
    return np.broadcast_to(nx[None], (N,) + X.shape)


def state_errors(Wg, Hg, Gg, Qg, Wr, Hr, Gr, Qr, tau_q):
    """Norm-wise and element-wise errors of a state against the oracle's."""
    return {"W": rel(Wg, Wr), "H": rel(Hg, Hr), "G": rel(Gg, Gr), "Q": rel(Qg, Qr),
            "W_el": elem_rel(Wg, Wr, 0.0, 0.0), "H_el": elem_rel(Hg, Hr, 0.0, 0.0),
            "G_el": elem_rel(Gg, Gr, 0.0, 0.0), "Q_el": elem_rel(Qg, Qr, q_row_scale(Qr), tau_q)}


def ll_rel(ll_gpu, ll_ref, X, W, H, G, Q):
    """|dLL| / sum |terms of Eq. 17| (the log-likelihood is a cancelling sum)."""
    return abs(ll_gpu - ll_ref) / O.loglik_terms_abs(X, W, H, G, Q)


def as64(W, H, G, Q):
    return (W.astype(np.float64), H.astype(np.float64), G.astype(np.float64), Q.astype(np.complex128))
