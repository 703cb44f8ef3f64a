"""Pins of the oracle's front end (Sec. IV-A: STFT with a 1024-point window and a 256-point
shift, F = 513; its inverse; the initialisation of g~ and Q by spectral decomposition).  CPU."""
import numpy as np
import pytest

from oracle import fastmnmf_oracle as O
from paper_1903_03237_gb300.synth import make_mixture


def _ola_weight(T, L, hop):
    w = O.hann(L)
    den = np.zeros((T - 1) * hop + L)
    for t in range(T):
        den[t * hop:t * hop + L] += w * w
    return den


@pytest.mark.parametrize("S,L,hop", [(5000, 1024, 256), (1024, 1024, 256), (777, 64, 16), (100, 32, 8)])
def test_istft_inverts_stft(S, L, hop):
    x = np.random.default_rng(S).standard_normal((3, S))
    X = O.stft(x, L, hop)
    assert X.shape == (L // 2 + 1, O.stft_frames(S, L, hop), 3)
    y = O.istft(X[None], S, L, hop)[0]
    den = _ola_weight(X.shape[1], L, hop)[:S]
    ok = den > 1e-6 * den.max()
    assert np.abs(y[:, ok] - x[:, ok]).max() < 1e-9
    cov = den > 1e-10 * den.max()                     # every covered sample, looser
    assert np.abs(y[:, cov] - x[:, cov]).max() < 1e-4
    assert np.all(y[:, ~cov] == 0)


def test_stft_matches_the_dft_sum():
    # tiny case against the DFT written out: X[f,t,m] = sum_j w_j x_m[t hop + j] e^{-2 pi i f j / L}
    L, hop, S = 16, 4, 37
    x = np.random.default_rng(1).standard_normal((2, S))
    X = O.stft(x, L, hop)
    w = O.hann(L)
    for t in range(X.shape[1]):
        for f in range(L // 2 + 1):
            for m in range(2):
                acc = 0j
                for j in range(L):
                    s = t * hop + j
                    if s < S:
                        acc += w[j] * x[m, s] * np.exp(-2j * np.pi * f * j / L)
                assert abs(X[f, t, m] - acc) < 1e-12


def test_stft_parseval_per_frame():
    L, hop = 1024, 256
    x = np.random.default_rng(2).standard_normal((1, 4000))
    X = O.stft(x, L, hop)
    w = O.hann(L)
    for t in range(X.shape[1]):
        seg = np.zeros(L)
        n = min(L, 4000 - t * hop)
        seg[:n] = x[0, t * hop:t * hop + n]
        e_time = np.sum((w * seg) ** 2)
        P = np.abs(X[:, t, 0]) ** 2
        e_freq = (P[0] + P[-1] + 2 * P[1:-1].sum()) / L
        assert abs(e_time - e_freq) < 1e-10 * e_time


def test_stft_of_a_tone_is_the_hann_kernel():
    # x = cos(2 pi k0 s / L): in every full frame the periodic Hann window leaves three lines,
    # |X| = L/4 at k0 and L/8 at k0 +- 1, nothing elsewhere; the phase advances by
    # 2 pi k0 hop / L per frame
    L, hop, k0 = 1024, 256, 37
    s = np.arange(8 * L)
    X = O.stft(np.cos(2 * np.pi * k0 * s / L)[None], L, hop)
    for t in range(X.shape[1] - 4):
        mag = np.abs(X[:, t, 0])
        assert abs(mag[k0] - L / 4) < 1e-9 and abs(mag[k0 - 1] - L / 8) < 1e-9 and abs(mag[k0 + 1] - L / 8) < 1e-9
        rest = np.delete(mag, [k0 - 1, k0, k0 + 1])
        assert rest.max() < 1e-9
        ph = np.angle(X[k0, t + 1, 0] / X[k0, t, 0])
        assert abs(np.angle(np.exp(1j * (ph - 2 * np.pi * k0 * hop / L)))) < 1e-9


@pytest.mark.parametrize("M,N", [(1, 2), (2, 2), (4, 3), (8, 6)])
def test_spectral_init_diagonalises_the_initial_scms(M, N):
    mix = make_mixture(7, 300, M, N, 4, 5)
    X = mix.X.astype(np.complex128)
    G, Q = O.spectral_init(X, N)
    R = np.einsum("fti,ftj->fij", X, X.conj()) / X.shape[1]
    for f in range(7):
        q = Q[f]
        np.testing.assert_allclose(q @ q.conj().T, np.eye(M), atol=1e-12)           # unitary: phi = 1
        D = q @ R[f] @ q.conj().T
        np.testing.assert_allclose(D, np.diag(G[0, f]), atol=1e-10 * np.abs(R[f]).max())
        assert np.all(np.diff(G[0, f]) <= 1e-12 * G[0, f].max())                   # largest first
        # the full-rank SCMs the decorrelated model represents (Eq. 16): G_1f and I
        np.testing.assert_allclose(q.conj().T @ np.diag(G[0, f]) @ q, R[f], atol=1e-10 * np.abs(R[f]).max())
        for n in range(1, N):
            np.testing.assert_allclose(q.conj().T @ np.diag(G[n, f]) @ q, np.eye(M), atol=1e-12)


def test_spectral_init_state_keeps_the_model():
    mix = make_mixture(5, 200, 3, 2, 4, 6)
    X = mix.X.astype(np.complex128)
    W, H, _, _ = O.init_state(5, 200, 3, 2, 4, seed=3)
    G, Q = O.spectral_init(X, 2)
    W2, G2, Q2 = O.spectral_init_state(X, W, G, Q)
    np.testing.assert_allclose(G2.sum(axis=2), 1.0, rtol=1e-12)
    np.testing.assert_allclose(O.model_power(O.source_psd(W2, H), G2), O.model_power(O.source_psd(W, H), G), rtol=1e-12)
