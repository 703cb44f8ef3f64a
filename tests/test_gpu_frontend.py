"""The front end (Sec. IV-A) against the float64 oracle, through the C ABI: the STFT, its
inverse, and the spectral initialisation of g~ and Q, alone and as the first and last steps
of a whole separation (signals -> X -> estimation -> images -> signals).

Bars (float32 transforms; their error grows with the log2(L) butterfly stages):
 * STFT: |X_gpu - X_ref| <= 1e-5 x the frame's RMS spectral magnitude, per element;
 * iSTFT: an output sample y_s = sum_t w z_t / sum_t w^2 carries the frames' float32 errors
   weighted by w, so |dy_s| sum_t w^2 / sum_t w <= 1e-5 x the largest frame RMS of that
   channel (+ 1e-6 |y_s|), per sample; samples the oracle zeroes are exactly 0;
 * spectral initialisation (float64 Jacobi on the device, stored as float32 / float-float):
   g~ within 1e-6 absolute (each (n, f) row sums to 1), W (or lambda) x nu within 1e-6
   relative, Q_f unitary within 1e-6, rows of Q_f equal to the oracle's up to a phase
   (|q_gpu . q_ref^*| >= 1 - 1e-6) where the eigenvalue is separated from the others by
   1e-3 of the largest, and the log-likelihood of the new state within 1e-6 (it does not
   depend on the phases or on the basis chosen inside a repeated eigenvalue's eigenspace).
"""
import numpy as np
import pytest

from oracle import fastmnmf_oracle as O
from paper_1903_03237_gb300.synth import make_signals, make_mixture

pytestmark = pytest.mark.gpu

TOL_STFT = 1e-5
TOL_ISTFT = 1e-5
TOL_G = 1e-6
TOL_INIT = 1e-6


@pytest.fixture(scope="module")
def fm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf
    return fastmnmf


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _stft_gpu(fm, x, L, hop):
    import torch
    X = fm.stft(_dev(x), L, hop)
    torch.cuda.synchronize()
    return X.cpu().numpy()


STFT_CASES = [
    (5000, 1024, 256, 3),     # ragged last frame
    (48000, 1024, 256, 4),    # 3 s at 16 kHz, the paper's framing
    (1024, 1024, 256, 2),     # S = L: one frame
    (10, 64, 16, 1),          # S < L: one zero-padded frame
    (777, 64, 16, 2),
    (100, 32, 8, 1),
    (20000, 4096, 1024, 1),   # largest window
    (3000, 16, 16, 8),        # smallest window, no overlap, 8 channels
]


@pytest.mark.parametrize("S,L,hop,M", STFT_CASES)
def test_stft_matches_oracle(fm, S, L, hop, M):
    x = make_signals(M, S, 2, seed=S + L)
    Xg = _stft_gpu(fm, x, L, hop)
    Xr = O.stft(x.astype(np.float64), L, hop)
    assert Xg.shape == Xr.shape == (L // 2 + 1, fm.stft_frames(S, L, hop), M)
    scale = np.sqrt(np.mean(np.abs(Xr) ** 2, axis=0, keepdims=True))      # [1, T, M]
    err = np.abs(Xg - Xr) / (scale + 1e-30)
    assert err.max() <= TOL_STFT, err.max()


def test_stft_of_silence_is_zero(fm):
    x = np.zeros((2, 3000), np.float32)
    assert np.all(_stft_gpu(fm, x, 256, 64) == 0)


def _istft_check(fm, Y, S, L, hop):
    import torch
    yg = fm.istft(_dev(Y.astype(np.complex64)), S, L, hop)
    torch.cuda.synchronize()
    yg = yg.cpu().numpy().astype(np.float64)
    Y64 = Y.astype(np.complex64).astype(np.complex128)
    yr = O.istft(Y64, S, L, hop)
    B, F, T, M = Y.shape
    w = O.hann(L)
    den = np.zeros((T - 1) * hop + L)
    wsum = np.zeros_like(den)
    for t in range(T):
        den[t * hop:t * hop + L] += w * w
        wsum[t * hop:t * hop + L] += w
    ok = den > 1e-10 * den.max()
    den, wsum, ok = den[:S], wsum[:S], ok[:S]
    z = np.fft.irfft(Y64.transpose(0, 3, 2, 1), n=L, axis=3)                 # [B, M, T, L]
    zr = np.sqrt(np.mean(z ** 2, axis=3)).max(axis=2)                        # [B, M]
    assert np.all(yg[:, :, ~ok] == 0)
    e = np.abs(yg - yr)[:, :, ok] * den[ok] / wsum[ok]
    bound = TOL_ISTFT * zr[:, :, None] + 1e-6 * np.abs(yr[:, :, ok])
    assert np.all(e <= bound), (e / bound).max()
    return yg


@pytest.mark.parametrize("S,L,hop,M,B", [(5000, 1024, 256, 3, 2), (777, 64, 16, 2, 3), (1024, 1024, 256, 1, 1),
                                         (10, 64, 16, 2, 1), (3000, 16, 16, 8, 1)])
def test_istft_matches_oracle(fm, S, L, hop, M, B):
    # images of a Wiener-like filtering: the STFT times a random nonnegative mask per source,
    # with bins 0 and L/2 given imaginary parts the inverse must ignore
    x = make_signals(M, S, 2, seed=S + 7)
    X = O.stft(x.astype(np.float64), L, hop)
    rng = np.random.default_rng(S)
    Y = X[None] * rng.uniform(0.0, 1.0, size=(B,) + X.shape)
    Y[:, 0] += 1j * rng.standard_normal(Y[:, 0].shape)
    Y[:, -1] += 1j * rng.standard_normal(Y[:, -1].shape)
    _istft_check(fm, Y, S, L, hop)


def test_round_trip(fm):
    import torch
    S, L, hop, M = 20000, 1024, 256, 4
    x = make_signals(M, S, 3, seed=5)
    y = fm.istft(fm.stft(_dev(x), L, hop), S, L, hop)
    torch.cuda.synchronize()
    y = y.cpu().numpy()
    T = fm.stft_frames(S, L, hop)
    w = O.hann(L)
    den = np.zeros((T - 1) * hop + L)
    for t in range(T):
        den[t * hop:t * hop + L] += w * w
    ok = den[:S] > 1e-3 * den.max()
    assert np.abs(y[:, ok] - x[:, ok]).max() <= 1e-5 * np.abs(x).max()


# ---- spectral initialisation -----------------------------------------------------------

def _rows_match(Qg, Qr, e, f):
    """Rows of Q_f equal up to a phase where the eigenvalue is separated from the others."""
    emax = max(e[f].max(), 1e-300)
    for r in range(Qg.shape[1]):
        gap = np.min(np.abs(np.delete(e[f], r) - e[f, r])) / emax if e.shape[1] > 1 else 1.0
        if gap < 1e-3:
            continue
        ov = abs(np.vdot(Qr[f, r], Qg[f, r]))
        assert ov >= 1 - TOL_INIT, (f, r, ov)


def _check_spectral(X, N, W0, G1, Q1, W1, ll_gpu, H0, lam0=None, lam1=None):
    X64 = X.astype(np.complex128)
    Gr, Qr = O.spectral_init(X64, N)
    nu = Gr.sum(axis=2)                                                    # [N, F]
    Gref = Gr / nu[:, :, None]
    assert np.abs(G1 - Gref).max() <= TOL_G
    F, M = Q1.shape[0], Q1.shape[1]
    QQ = np.einsum("fij,fkj->fik", Q1.astype(np.complex128), Q1.conj())
    assert np.abs(QQ - np.eye(M)[None]).max() <= TOL_INIT
    for f in range(F):
        _rows_match(Q1.astype(np.complex128), Qr, Gr[0], f)
    if lam0 is None:
        Wref = W0.astype(np.float64) * nu[:, None, :]
        assert np.max(np.abs(W1 - Wref) / Wref) <= TOL_INIT
        llr = O.loglik(X64, Wref, H0.astype(np.float64), Gref, Qr)
    else:
        Lref = lam0.astype(np.float64) * nu[:, :, None]
        assert np.max(np.abs(lam1 - Lref) / Lref) <= TOL_INIT
        llr = O.loglik_lam(X64, Lref.transpose(1, 2, 0), Gref, Qr)
    assert abs(ll_gpu - llr) <= TOL_INIT * abs(llr), (ll_gpu, llr)


SPEC_CASES = [
    (65, 100, 4, 3, 4),
    (33, 2, 4, 2, 2),       # T < M: a repeated zero eigenvalue in every bin
    (129, 200, 8, 4, 4),
    (40, 50, 1, 2, 3),      # one channel: Q_f = 1
    (17, 30, 2, 5, 2),
]


@pytest.mark.parametrize("F,T,M,N,K", SPEC_CASES)
def test_spectral_init_matches_oracle(fm, F, T, M, N, K):
    mix = make_mixture(F, T, M, N, K, seed=F + T)
    ctx = fm.Context(mix.X, N, K, seed=11)
    W0, H0, _, _ = ctx.get_state()
    ctx.init_spectral()
    W1, H1, G1, Q1 = ctx.get_state()
    np.testing.assert_array_equal(H1, H0)
    _check_spectral(mix.X, N, W0, G1, Q1, W1, ctx.loglik(), H0)
    # the spectral state is the restart state
    ctx.iterate(3)
    ctx.restart()
    W2, H2, G2, Q2 = ctx.get_state()
    for a, b in ((W2, W1), (H2, H1), (G2, G1), (Q2, Q1)):
        np.testing.assert_array_equal(a, b)


def test_spectral_init_free_model(fm):
    F, T, M, N = 30, 60, 3, 2
    mix = make_mixture(F, T, M, N, 2, seed=41)
    ctx = fm.Context(mix.X, N, seed=5, source_model=fm.SOURCE_FREE)
    lam0, _, _ = ctx.get_lambda()
    ctx.init_spectral()
    lam1, G1, Q1 = ctx.get_lambda()
    _check_spectral(mix.X, N, None, G1, Q1, None, ctx.loglik(), None, lam0=lam0, lam1=lam1)


def test_spectral_init_zero_power_bin(fm):
    mix = make_mixture(9, 20, 3, 2, 2, seed=2)
    X = mix.X.copy()
    X[4] = 0
    ctx = fm.Context(X, 2, 2, seed=1)
    with pytest.raises(fm.FastMNMFError) as ei:
        ctx.init_spectral()
    assert ei.value.status == fm.ESINGULAR
    # a zero bin also leaves V_fm = 0 (the IP system of Eqs. 19-20 is singular whatever the
    # state), so recovery means a new mixture: reset clears the error word
    ctx.reset(mix.X, seed=1)
    ctx.init_spectral()
    ctx.iterate(1)
    assert np.isfinite(ctx.loglik())


def test_whole_separation_from_signals(fm):
    """Signals -> STFT -> spectral init -> 20 iterations -> Wiener images -> iSTFT at the
    paper's framing (L = 1024, shift 256) and the 4-channel, 4-source, 32-basis shape with
    640 frames: the initial state matches the oracle, the log-likelihood never decreases, and
    the separated signals add up to the recording on every covered sample."""
    import torch
    L, hop, M, N, K, T = 1024, 256, 4, 4, 32, 640
    S = (T - 1) * hop + L
    x = make_signals(M, S, N, seed=17)
    Xd = fm.stft(_dev(x), L, hop)
    torch.cuda.synchronize()
    assert tuple(Xd.shape) == (L // 2 + 1, T, M)
    ctx = fm.Context(Xd, N, K, seed=3)
    W0, H0, _, _ = ctx.get_state()
    ctx.init_spectral()
    W1, _, G1, Q1 = ctx.get_state()
    _check_spectral(Xd.cpu().numpy(), N, W0, G1, Q1, W1, ctx.loglik(), H0)
    lls = [ctx.loglik()]
    for _ in range(4):
        ctx.iterate(5)
        lls.append(ctx.loglik())
    assert np.all(np.diff(lls) >= -1e-6 * abs(lls[0])), lls
    imgs = torch.empty((N, L // 2 + 1, T, M), dtype=torch.complex64, device="cuda")
    ctx.separate(imgs)
    ctx.sync()
    ys = fm.istft(imgs, S, L, hop)                                          # [N, M, S]
    torch.cuda.synchronize()
    total = ys.sum(dim=0).cpu().numpy()
    w = O.hann(L)
    den = np.zeros((T - 1) * hop + L)
    for t in range(T):
        den[t * hop:t * hop + L] += w * w
    ok = den[:S] > 1e-3 * den.max()
    assert np.abs(total[:, ok] - x[:, ok]).max() <= 1e-4 * np.abs(x).max()
