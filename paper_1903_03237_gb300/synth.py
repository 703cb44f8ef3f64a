"""Seeded synthetic multichannel mixtures drawn from FastMNMF's own generative model.

This module only draws data: it is the one piece that both the CUDA path's tests and
the float64 oracle consume, and it contains none of the estimation updates.  A
mixture is synthesised exactly as the generative model states it:

* source model (Sec. II-B-2, Eq. 9): lambda_ftn = sum_k w_nkf h_nkt with
  w, h ~ Gamma(1, 1) i.i.d.;
* jointly diagonalisable spatial model (Sec. III-A-1, Eq. 16): per bin a
  diagonaliser Q_f = I + 0.3 Z (Z_ij ~ CN(0, 1)) and per (n, f) a nonnegative
  g~_nf ~ Dirichlet(1_M);
* source images (Eq. 1): x_ftn = Q_f^-1 diag(sqrt(lambda_ftn g~_nf)) z_ftn with
  z_ftn ~ CN(0, I), so x_ftn ~ CN(0, lambda_ftn Q_f^-1 Diag(g~_nf) Q_f^-H);
* mixture (Eq. 2): x_ft = sum_n x_ftn;
* optional diffuse noise on a seeded 10 % of the frequency bins: x_ft += CN(0, s I).

Everything is drawn with NumPy's ``default_rng(seed)`` (PCG64) in a fixed order, and
stored as complex64 ``X[F][T][M]`` (real/imag interleaved), the library's input
layout.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Mixture:
    X: np.ndarray          # complex64 [F, T, M]
    W: np.ndarray          # float64 [N, K, F]   (truth used for the draw)
    H: np.ndarray          # float64 [N, K, T]
    G: np.ndarray          # float64 [N, F, M]
    Q: np.ndarray          # complex128 [F, M, M]
    noisy_bins: np.ndarray  # int64 indices of bins that received diffuse noise


def _cn(rng, shape):
    """Circularly-symmetric CN(0, 1): real and imaginary parts i.i.d. N(0, 1/2)."""
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * np.sqrt(0.5)


def make_mixture(F: int, T: int, M: int, N: int, K: int, seed: int,
                 diffuse_frac: float = 0.0, diffuse_var: float = 1e-3) -> Mixture:
    rng = np.random.default_rng(seed)
    W = rng.gamma(1.0, 1.0, size=(N, K, F))
    H = rng.gamma(1.0, 1.0, size=(N, K, T))
    G = rng.dirichlet(np.ones(M), size=(N, F))                      # [N, F, M]
    Q = np.eye(M)[None] + 0.3 * _cn(rng, (F, M, M))
    Z = _cn(rng, (N, F, T, M))
    Qi = np.linalg.inv(Q)
    X = np.zeros((F, T, M), dtype=np.complex128)
    for n in range(N):
        psd = W[n].T @ H[n]                                         # [F, T] source PSD
        amp = np.sqrt(psd[:, :, None] * G[n][:, None, :])           # [F, T, M]
        X += np.einsum("fij,ftj->fti", Qi, amp * Z[n])
    noisy = np.zeros(0, dtype=np.int64)
    if diffuse_frac > 0.0:
        n_noisy = int(round(diffuse_frac * F))
        noisy = np.sort(rng.choice(F, size=n_noisy, replace=False)).astype(np.int64)
        X[noisy] += np.sqrt(diffuse_var) * _cn(rng, (n_noisy, T, M))
    return Mixture(X=X.astype(np.complex64), W=W, H=H, G=G, Q=Q, noisy_bins=noisy)


def make_state(F: int, T: int, M: int, N: int, K: int, seed: int):
    """A random positive starting state (not the truth) for parity tests:
    W, H ~ U(0.2, 1.2), g~ rows ~ Dirichlet(1) + 0.05 renormalised, Q_f = I + 0.2 Z.
    Returned already rounded to the library's storage types (float32 / complex64)."""
    rng = np.random.default_rng(seed + 7919)
    W = rng.uniform(0.2, 1.2, size=(N, K, F)).astype(np.float32)
    H = rng.uniform(0.2, 1.2, size=(N, K, T)).astype(np.float32)
    G = rng.dirichlet(np.ones(M), size=(N, F)) + 0.05
    G = (G / G.sum(axis=2, keepdims=True)).astype(np.float32)
    Q = (np.eye(M)[None] + 0.2 * _cn(rng, (F, M, M))).astype(np.complex64)
    return W, H, G, Q


def make_decoder(F: int, D: int, Hd: int, seed: int):
    """Seeded random weights of the deep-prior decoder r = exp(W2 tanh(W1 z + b1) + b2)
    (trained weights are not available): W1 ~ N(0, 1/D) [Hd, D], b1 ~ N(0, 0.01) [Hd],
    W2 ~ N(0, 1/Hd) [F, Hd], b2 ~ N(0, 0.25) [F]; float32."""
    rng = np.random.default_rng(seed + 104729)
    W1 = rng.standard_normal((Hd, D)) / np.sqrt(D)
    b1 = 0.1 * rng.standard_normal(Hd)
    W2 = rng.standard_normal((F, Hd)) / np.sqrt(Hd)
    b2 = 0.5 * rng.standard_normal(F)
    return tuple(a.astype(np.float32) for a in (W1, b1, W2, b2))


def make_dp_state(F: int, T: int, M: int, N: int, K: int, D: int, seed: int):
    """A random starting state of the deep-prior model (speech source 0, NMF noise sources
    1..N-1): Z ~ N(0, I) [T, D], u ~ U(0.5, 1.5) [F], v ~ K U(0.2, 1.2) [T], and W, H, g~, Q
    as ``make_state`` draws them for the N-1 noise sources and N sources.  float32 /
    complex64."""
    W, H, G, Q = make_state(F, T, M, N, K, seed)
    rng = np.random.default_rng(seed + 15485863)
    Z = rng.standard_normal((T, D)).astype(np.float32)
    u = rng.uniform(0.5, 1.5, size=F).astype(np.float32)
    v = (K * rng.uniform(0.2, 1.2, size=T)).astype(np.float32)
    return Z, u, v, W[1:].copy(), H[1:].copy(), G, Q


def make_dp_draws(n_iter: int, S: int, T: int, D: int, seed: int):
    """The Metropolis draws of n_iter iterations with S proposals per frame:
    xi ~ N(0, I) [n_iter, S, T, D] and log u, u ~ U(0, 1) [n_iter, S, T]; float32."""
    rng = np.random.default_rng(seed + 32452843)
    xi = rng.standard_normal((n_iter, S, T, D)).astype(np.float32)
    logu = np.log(rng.uniform(np.finfo(np.float64).tiny, 1.0, size=(n_iter, S, T))).astype(np.float32)
    return xi, logu


def make_signals(M: int, S: int, n_src: int, seed: int, taps: int = 64) -> np.ndarray:
    """Seeded time-domain multichannel recordings for the front end (STFT, its inverse and
    the spectral initialisation), float32 [M, S]: n_src sources, each white Gaussian noise
    under a slowly varying nonnegative envelope (a bounded random walk, so the source power
    changes over frames as a speech or noise source does), reach every microphone through
    its own impulse response of ``taps`` samples (Gaussian taps under an exponential decay
    of time constant taps / 4, like a short room response); plus white sensor noise of
    1e-3 of the source level."""
    rng = np.random.default_rng(seed)
    x = np.zeros((M, S))
    decay = np.exp(-np.arange(taps) / (taps / 4.0))
    for _ in range(n_src):
        steps = rng.standard_normal(S // 256 + 2) * 0.3
        env = np.exp(np.clip(np.cumsum(steps), -3.0, 3.0))
        env = np.repeat(env, 256)[:S]
        src = rng.standard_normal(S) * env
        for m in range(M):
            h = rng.standard_normal(taps) * decay
            x[m] += np.convolve(src, h)[:S]
    x += 1e-3 * x.std() * rng.standard_normal((M, S))
    return x.astype(np.float32)


# Workload shapes (M channels, N sources, K bases, F bins, T frames, iterations).
CONFIGS = {
    "c0": dict(M=2, N=2, K=8, F=257, T=200, iters=20, diffuse=0.0),
    "c1": dict(M=4, N=4, K=32, F=513, T=640, iters=100, diffuse=0.1),
    "c2": dict(M=8, N=6, K=64, F=1025, T=4096, iters=1, diffuse=0.0),
}


def config_mixture(name: str, seed: int = 0) -> Mixture:
    c = CONFIGS[name]
    return make_mixture(c["F"], c["T"], c["M"], c["N"], c["K"], seed, diffuse_frac=c["diffuse"])
