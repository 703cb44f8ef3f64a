"""Shared helpers of the GPU parity tests (error metrics and state round-trips)."""
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


def ll_rel(ll_gpu, ll_ref, X, W, H, G, Q):
    """|dLL| / sum |terms of Eq. 17| (the log-likelihood is a cancelling sum)."""
    return abs(ll_gpu - ll_ref) / O.loglik_terms_abs(X, W, H, G, Q)


def as64(W, H, G, Q):
    return (W.astype(np.float64), H.astype(np.float64), G.astype(np.float64), Q.astype(np.complex128))
