"""Thin Python binding of libfastmnmf.so (ctypes).  Argument marshalling only: every step
of FastMNMF runs in the library's CUDA kernels.  Host arrays are NumPy; device arrays are
torch CUDA tensors (their data pointers are handed to the C ABI).

The library must have been built (``paper_1903_03237_gb300.build.build()``); importing
this module without it raises ImportError - there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

try:  # load torch first so the library binds to the same CUDA runtime instance
    import torch  # noqa: F401
except Exception:  # pragma: no cover - torch is optional for pure host use
    torch = None

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libfastmnmf.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"{_LIB_PATH} is missing: build it with paper_1903_03237_gb300.build.build()")
_lib = ctypes.CDLL(_LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ESINGULAR, ETIMEOUT, EBUSY = range(8)
UPDATE_W, UPDATE_H, UPDATE_G, UPDATE_Q, UPDATE_ALL = 1, 2, 4, 8, 15
PREC_FP32, PREC_BF16, PREC_TF32 = 0, 1, 2
SCHED_AUTO, SCHED_SWEEP, SCHED_FUSED = 0, 1, 2
SOURCE_NMF, SOURCE_FREE = 0, 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENONFINITE", 5: "ESINGULAR",
                6: "ETIMEOUT", 7: "EBUSY"}

# every symbol include/fastmnmf.h declares
EXPORTS = ["fmnmf_default_opts", "fmnmf_init", "fmnmf_reset", "fmnmf_restart", "fmnmf_iterate", "fmnmf_sync",
           "fmnmf_query",
           "fmnmf_loglik", "fmnmf_separate", "fmnmf_get_state", "fmnmf_set_state", "fmnmf_shape",
           "fmnmf_get_lambda", "fmnmf_set_lambda",
           "fmnmf_destroy", "fmnmf_last_error", "fmnmf_set_timing", "fmnmf_kernel_times",
           "fmnmf_kernel_name", "fmnmf_launch_count", "fmnmf_loglik_noalloc",
           "fmnmf_batch_create", "fmnmf_batch_iterate", "fmnmf_batch_sync", "fmnmf_batch_destroy",
           "fmnmf_autotune", "fmnmf_batch_autotune", "fmnmf_get_tuning", "fmnmf_set_tuning",
           "fmnmf_footprint", "fmnmf_server_create", "fmnmf_server_submit", "fmnmf_server_poll",
           "fmnmf_server_wait", "fmnmf_server_result", "fmnmf_server_stats", "fmnmf_server_destroy",
           "fmnmf_init_spectral", "fmnmf_stft_frames", "fmnmf_stft", "fmnmf_istft",
           "fmnmf_dp_default_opts", "fmnmf_dp_create", "fmnmf_dp_set_decoder", "fmnmf_dp_set_state",
           "fmnmf_dp_get_state", "fmnmf_dp_iterate", "fmnmf_dp_metropolis", "fmnmf_dp_sync",
           "fmnmf_dp_loglik", "fmnmf_dp_accepted", "fmnmf_dp_separate", "fmnmf_dp_destroy",
           "fmnmf_dp_last_error"]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("update_mask", ctypes.c_uint), ("normalise", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("hbm_budget", ctypes.c_size_t), ("schedule", ctypes.c_int),
                ("source_model", ctypes.c_int)]


class DPOpts(ctypes.Structure):
    _fields_ = [("D", ctypes.c_int), ("Hd", ctypes.c_int), ("n_proposals", ctypes.c_int), ("eps", ctypes.c_float),
                ("normalise", ctypes.c_int), ("stream", ctypes.c_void_p)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_S = ctypes.c_int  # fmnmf_status
_sig = {
    "fmnmf_default_opts": (_S, [ctypes.POINTER(Opts)]),
    "fmnmf_init": (_S, [ctypes.POINTER(_P), _P, _I, _I, _I, _I, _I, _I, ctypes.c_uint64, ctypes.POINTER(Opts)]),
    "fmnmf_reset": (_S, [_P, _P, _I, ctypes.c_uint64]),
    "fmnmf_restart": (_S, [_P]),
    "fmnmf_iterate": (_S, [_P, _I]),
    "fmnmf_sync": (_S, [_P]),
    "fmnmf_query": (_S, [_P]),
    "fmnmf_loglik": (_S, [_P, ctypes.POINTER(ctypes.c_double)]),
    "fmnmf_separate": (_S, [_P, _P, _I]),
    "fmnmf_get_state": (_S, [_P, _P, _P, _P, _P]),
    "fmnmf_set_state": (_S, [_P, _P, _P, _P, _P]),
    "fmnmf_get_lambda": (_S, [_P, _P, _P, _P]),
    "fmnmf_set_lambda": (_S, [_P, _P, _P, _P]),
    "fmnmf_shape": (_S, [_P] + [ctypes.POINTER(_I)] * 5),
    "fmnmf_destroy": (_S, [_P]),
    "fmnmf_last_error": (ctypes.c_char_p, [_P]),
    "fmnmf_set_timing": (_S, [_P, _I]),
    "fmnmf_kernel_times": (_S, [_P, _P, _P, ctypes.POINTER(_I)]),
    "fmnmf_kernel_name": (ctypes.c_char_p, [_I]),
    "fmnmf_launch_count": (ctypes.c_longlong, [_P]),
    "fmnmf_loglik_noalloc": (_S, [_P, _P, _P, _P, _P, _I, _I, _I, _I, _I, _P, _P]),
    "fmnmf_batch_create": (_S, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P)]),
    "fmnmf_batch_iterate": (_S, [_P, _I]),
    "fmnmf_batch_sync": (_S, [_P]),
    "fmnmf_autotune": (_S, [_P, _I, ctypes.POINTER(ctypes.c_double)]),
    "fmnmf_batch_autotune": (_S, [_P, _I, ctypes.POINTER(ctypes.c_double)]),
    "fmnmf_get_tuning": (_S, [_P, ctypes.POINTER(ctypes.c_float)]),
    "fmnmf_set_tuning": (_S, [_P, ctypes.POINTER(ctypes.c_float)]),
    "fmnmf_batch_destroy": (_S, [_P]),
    "fmnmf_footprint": (_S, [_I, _I, _I, _I, _I, ctypes.POINTER(Opts), ctypes.POINTER(ctypes.c_size_t)]),
    "fmnmf_server_create": (_S, [_P, ctypes.POINTER(_P)]),
    "fmnmf_server_submit": (_S, [_P, _P, _I, _I, _I, _I, _I, _I, ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]),
    "fmnmf_server_poll": (_S, [_P, ctypes.c_uint64, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_double)]),
    "fmnmf_server_wait": (_S, [_P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(_I)]),
    "fmnmf_server_result": (_S, [_P, ctypes.c_uint64, _P, ctypes.POINTER(ctypes.c_double)]),
    "fmnmf_server_stats": (_S, [_P] + [ctypes.POINTER(ctypes.c_longlong)] * 4 + [ctypes.POINTER(ctypes.c_size_t)]),
    "fmnmf_server_destroy": (_S, [_P]),
    "fmnmf_init_spectral": (_S, [_P]),
    "fmnmf_stft_frames": (_S, [_I, _I, _I, ctypes.POINTER(_I)]),
    "fmnmf_stft": (_S, [_P, _I, _I, _I, _I, _P, _P]),
    "fmnmf_istft": (_S, [_P, _I, _I, _I, _I, _I, _I, _I, _P, _P]),
    "fmnmf_dp_default_opts": (_S, [ctypes.POINTER(DPOpts)]),
    "fmnmf_dp_create": (_S, [ctypes.POINTER(_P), _P, _I, _I, _I, _I, _I, _I, ctypes.POINTER(DPOpts)]),
    "fmnmf_dp_set_decoder": (_S, [_P, _P, _P, _P, _P]),
    "fmnmf_dp_set_state": (_S, [_P] + [_P] * 7),
    "fmnmf_dp_get_state": (_S, [_P] + [_P] * 7),
    "fmnmf_dp_iterate": (_S, [_P, _I, _P, _P, _I]),
    "fmnmf_dp_metropolis": (_S, [_P, _P, _P, _I, _P, ctypes.POINTER(ctypes.c_longlong)]),
    "fmnmf_dp_sync": (_S, [_P]),
    "fmnmf_dp_loglik": (_S, [_P, ctypes.POINTER(ctypes.c_double)]),
    "fmnmf_dp_accepted": (_S, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    "fmnmf_dp_separate": (_S, [_P, _P, _I]),
    "fmnmf_dp_destroy": (_S, [_P]),
    "fmnmf_dp_last_error": (ctypes.c_char_p, [_P]),
}
for _name, (_res, _args) in _sig.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class FastMNMFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib() -> ctypes.CDLL:
    return _lib


def _check(st: int, ctx=None):
    if st != OK:
        msg = _lib.fmnmf_last_error(ctx)
        raise FastMNMFError(st, msg.decode() if msg else "")


def default_opts() -> Opts:
    o = Opts()
    _check(_lib.fmnmf_default_opts(ctypes.byref(o)))
    return o


def _host_ptr(a: np.ndarray, dtype) -> tuple[np.ndarray, int]:
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


class Context:
    """One mixture's device-resident FastMNMF state (wraps fmnmf_ctx)."""

    def __init__(self, X, N: int, K: int = 1, seed: int = 0, *, update_mask: int = UPDATE_ALL,
                 normalise: bool = True, precision: int = PREC_FP32, stream=None, hbm_budget: int = 0,
                 schedule: int = SCHED_AUTO, source_model: int = SOURCE_NMF):
        opts = default_opts()
        opts.update_mask = update_mask
        opts.normalise = 1 if normalise else 0
        opts.precision = precision
        opts.stream = stream
        opts.hbm_budget = hbm_budget
        opts.schedule = schedule
        opts.source_model = source_model
        self.free_model = source_model == SOURCE_FREE
        self._ctx = _P()
        self._keep = None
        if torch is not None and isinstance(X, torch.Tensor) and X.is_cuda:
            assert X.dtype == torch.complex64 and X.dim() == 3 and X.is_contiguous()
            F, T, M = X.shape
            torch.cuda.synchronize(X.device)  # the library reads X on its own stream
            ptr, on_dev = X.data_ptr(), 1
        else:
            Xh, ptr = _host_ptr(X, np.complex64)
            F, T, M = Xh.shape
            self._keep, on_dev = Xh, 0
        st = _lib.fmnmf_init(ctypes.byref(self._ctx), ptr, on_dev, F, T, M, N, K, seed, ctypes.byref(opts))
        self._keep = None
        _check(st, None)
        self.F, self.T, self.M, self.N, self.K = F, T, M, N, K

    # -- lifecycle ----------------------------------------------------------------------
    def close(self):
        if self._ctx:
            _lib.fmnmf_destroy(self._ctx)
            self._ctx = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._ctx

    # -- calls --------------------------------------------------------------------------
    def reset(self, X, seed: int = 0):
        if torch is not None and isinstance(X, torch.Tensor) and X.is_cuda:
            torch.cuda.synchronize(X.device)  # the library reads X on its own stream
            _check(_lib.fmnmf_reset(self._ctx, X.data_ptr(), 1, seed), self._ctx)
        else:
            Xh, ptr = _host_ptr(X, np.complex64)
            _check(_lib.fmnmf_reset(self._ctx, ptr, 0, seed), self._ctx)

    def restart(self):
        """Back to the state of the last init / reset / set_state (device-side, async)."""
        _check(_lib.fmnmf_restart(self._ctx), self._ctx)

    def iterate(self, n: int = 1):
        _check(_lib.fmnmf_iterate(self._ctx, n), self._ctx)

    def sync(self):
        _check(_lib.fmnmf_sync(self._ctx), self._ctx)

    def busy(self) -> bool:
        """True while work enqueued on the context stream is still running (non-blocking)."""
        st = _lib.fmnmf_query(self._ctx)
        if st == EBUSY:
            return True
        _check(st, self._ctx)
        return False

    def loglik(self) -> float:
        v = ctypes.c_double()
        _check(_lib.fmnmf_loglik(self._ctx, ctypes.byref(v)), self._ctx)
        return v.value

    def separate(self, out=None) -> np.ndarray:
        """Wiener-filtered source images [N, F, T, M] complex64.  ``out`` may be a torch
        CUDA tensor of that shape (filled asynchronously) or None (a NumPy array is returned)."""
        if out is not None and torch is not None and isinstance(out, torch.Tensor) and out.is_cuda:
            assert out.dtype == torch.complex64 and out.is_contiguous()
            assert tuple(out.shape) == (self.N, self.F, self.T, self.M)
            _check(_lib.fmnmf_separate(self._ctx, out.data_ptr(), 1), self._ctx)
            return out
        res = np.empty((self.N, self.F, self.T, self.M), dtype=np.complex64) if out is None else out
        _check(_lib.fmnmf_separate(self._ctx, res.ctypes.data, 0), self._ctx)
        return res

    def get_state(self):
        """(W, H, g~, Q); W and H are None for the unconstrained source model."""
        G = np.empty((self.N, self.F, self.M), np.float32)
        Q = np.empty((self.F, self.M, self.M), np.complex64)
        if self.free_model:
            _check(_lib.fmnmf_get_state(self._ctx, None, None, G.ctypes.data, Q.ctypes.data), self._ctx)
            return None, None, G, Q
        W = np.empty((self.N, self.K, self.F), np.float32)
        H = np.empty((self.N, self.K, self.T), np.float32)
        _check(_lib.fmnmf_get_state(self._ctx, W.ctypes.data, H.ctypes.data, G.ctypes.data, Q.ctypes.data), self._ctx)
        return W, H, G, Q

    def get_lambda(self):
        """(lambda [N, F, T], g~, Q) of the unconstrained source model."""
        L = np.empty((self.N, self.F, self.T), np.float32)
        G = np.empty((self.N, self.F, self.M), np.float32)
        Q = np.empty((self.F, self.M, self.M), np.complex64)
        _check(_lib.fmnmf_get_lambda(self._ctx, L.ctypes.data, G.ctypes.data, Q.ctypes.data), self._ctx)
        return L, G, Q

    def set_lambda(self, L, G, Q):
        L, lp = _host_ptr(L, np.float32)
        G, gp = _host_ptr(G, np.float32)
        Q, qp = _host_ptr(Q, np.complex64)
        assert L.shape == (self.N, self.F, self.T) and G.shape == (self.N, self.F, self.M)
        assert Q.shape == (self.F, self.M, self.M)
        _check(_lib.fmnmf_set_lambda(self._ctx, lp, gp, qp), self._ctx)

    def init_spectral(self):
        """g~ and Q from the eigendecomposition of the average observed SCM (Sec. IV-A), nu
        normalised with W (or lambda) scaled to match; H kept.  Becomes the restart state."""
        _check(_lib.fmnmf_init_spectral(self._ctx), self._ctx)

    def set_state(self, W, H, G, Q):
        W, wp = _host_ptr(W, np.float32)
        H, hp = _host_ptr(H, np.float32)
        G, gp = _host_ptr(G, np.float32)
        Q, qp = _host_ptr(Q, np.complex64)
        assert W.shape == (self.N, self.K, self.F) and H.shape == (self.N, self.K, self.T)
        assert G.shape == (self.N, self.F, self.M) and Q.shape == (self.F, self.M, self.M)
        _check(_lib.fmnmf_set_state(self._ctx, wp, hp, gp, qp), self._ctx)

    # -- measurement --------------------------------------------------------------------
    def set_timing(self, kinds=True):
        """True / False: time every kernel class or none; an int: bit mask of classes;
        a list of names: those classes."""
        if kinds is True:
            mask = -1
        elif kinds is False or kinds is None:
            mask = 0
        elif isinstance(kinds, int):
            mask = kinds
        else:
            names = [_lib.fmnmf_kernel_name(i).decode() for i in range(16)]
            mask = sum(1 << names.index(k) for k in kinds)
        _check(_lib.fmnmf_set_timing(self._ctx, mask), self._ctx)

    def kernel_times(self) -> dict:
        """{kernel name: (total ms, launches)} since the last call (synchronises)."""
        ms = (ctypes.c_double * 16)()
        cnt = (ctypes.c_longlong * 16)()
        n = _I(16)
        _check(_lib.fmnmf_kernel_times(self._ctx, ctypes.addressof(ms), ctypes.addressof(cnt), ctypes.byref(n)), self._ctx)
        return {_lib.fmnmf_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(n.value)}

    def launch_count(self) -> int:
        return int(_lib.fmnmf_launch_count(self._ctx))

    def autotune(self, n_iter: int = 2) -> float:
        """Times the launch-shape candidates (state restored afterwards); returns the speedup."""
        sp = ctypes.c_double()
        _check(_lib.fmnmf_autotune(self._ctx, n_iter, ctypes.byref(sp)), self._ctx)
        return sp.value

    def get_tuning(self) -> list:
        v = (ctypes.c_float * 8)()
        _check(_lib.fmnmf_get_tuning(self._ctx, v), self._ctx)
        return list(v)

    def set_tuning(self, scales):
        v = (ctypes.c_float * 8)(*scales)
        _check(_lib.fmnmf_set_tuning(self._ctx, v), self._ctx)


class Batch:
    """Several contexts iterated by one graph launch (one concurrent branch per context)."""

    def __init__(self, contexts):
        self._members = list(contexts)
        arr = (_P * len(self._members))(*[c.handle for c in self._members])
        self._b = _P()
        _check(_lib.fmnmf_batch_create(arr, len(self._members), ctypes.byref(self._b)), None)

    def iterate(self, n: int = 1):
        _check(_lib.fmnmf_batch_iterate(self._b, n), None)

    def sync(self):
        _check(_lib.fmnmf_batch_sync(self._b), None)

    def autotune(self, n_iter: int = 2) -> float:
        """One split scale for all members, timed on the whole batch; returns the speedup."""
        sp = ctypes.c_double()
        _check(_lib.fmnmf_batch_autotune(self._b, n_iter, ctypes.byref(sp)), None)
        return sp.value

    def close(self):
        if self._b:
            _lib.fmnmf_batch_destroy(self._b)
            self._b = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _check_dp(st: int, dp=None):
    if st != OK:
        msg = _lib.fmnmf_dp_last_error(dp)
        raise FastMNMFError(st, msg.decode() if msg else "")


class DPContext:
    """FastMNMF-DP (Sec. III-B-3, III-C-3): a deep-prior speech source (source 0) and NMF noise
    sources (1..N-1) for one mixture (wraps fmnmf_dp).  Host arrays are NumPy; the Metropolis
    draws may be torch CUDA tensors (kept resident on the device)."""

    def __init__(self, X, N: int, K: int, *, D: int = 16, Hd: int = 128, n_proposals: int = 30,
                 eps: float = 1e-4, normalise: bool = True, stream=None):
        o = DPOpts()
        _check_dp(_lib.fmnmf_dp_default_opts(ctypes.byref(o)))
        o.D, o.Hd, o.n_proposals, o.eps = D, Hd, n_proposals, eps
        o.normalise = 1 if normalise else 0
        o.stream = stream
        self._dp = _P()
        if torch is not None and isinstance(X, torch.Tensor) and X.is_cuda:
            assert X.dtype == torch.complex64 and X.dim() == 3 and X.is_contiguous()
            F, T, M = X.shape
            torch.cuda.synchronize(X.device)
            st = _lib.fmnmf_dp_create(ctypes.byref(self._dp), X.data_ptr(), 1, F, T, M, N, K, ctypes.byref(o))
        else:
            Xh, ptr = _host_ptr(X, np.complex64)
            F, T, M = Xh.shape
            st = _lib.fmnmf_dp_create(ctypes.byref(self._dp), ptr, 0, F, T, M, N, K, ctypes.byref(o))
        _check_dp(st, None)
        self.F, self.T, self.M, self.N, self.K = F, T, M, N, K
        self.D, self.Hd, self.S = D, Hd, n_proposals

    def close(self):
        if self._dp:
            _lib.fmnmf_dp_destroy(self._dp)
            self._dp = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_decoder(self, W1, b1, W2, b2):
        a = [_host_ptr(x, np.float32) for x in (W1, b1, W2, b2)]
        assert a[0][0].shape == (self.Hd, self.D) and a[2][0].shape == (self.F, self.Hd)
        _check_dp(_lib.fmnmf_dp_set_decoder(self._dp, *[p for _, p in a]), self._dp)

    def set_state(self, Z, u, v, W, H, G, Q):
        a = [_host_ptr(x, np.float32) for x in (Z, u, v, W, H, G)]
        q = _host_ptr(Q, np.complex64)
        assert a[0][0].shape == (self.T, self.D)
        _check_dp(_lib.fmnmf_dp_set_state(self._dp, *[p for _, p in a], q[1]), self._dp)

    def get_state(self):
        F, T, M, N, K, D = self.F, self.T, self.M, self.N, self.K, self.D
        Z = np.empty((T, D), np.float32)
        u = np.empty(F, np.float32)
        v = np.empty(T, np.float32)
        W = np.empty((N - 1, K, F), np.float32)
        H = np.empty((N - 1, K, T), np.float32)
        G = np.empty((N, F, M), np.float32)
        Q = np.empty((F, M, M), np.complex64)
        _check_dp(_lib.fmnmf_dp_get_state(self._dp, *[x.ctypes.data for x in (Z, u, v, W, H, G, Q)]), self._dp)
        return Z, u, v, W, H, G, Q

    def _draws(self, xi, logu):
        if torch is not None and isinstance(xi, torch.Tensor) and xi.is_cuda:
            assert xi.dtype == torch.float32 and logu.dtype == torch.float32
            assert xi.is_contiguous() and logu.is_contiguous()
            return xi.data_ptr(), logu.data_ptr(), 1, None
        xh, xp = _host_ptr(xi, np.float32)
        lh, lp = _host_ptr(logu, np.float32)
        return xp, lp, 0, (xh, lh)

    def iterate(self, n: int, xi, logu):
        """n iterations; xi [n][S][T][D], logu [n][S][T] (NumPy, or CUDA tensors on the device)."""
        xp, lp, dev, keep = self._draws(xi, logu)
        if not dev:
            assert keep[0].shape == (n, self.S, self.T, self.D) and keep[1].shape == (n, self.S, self.T)
        _check_dp(_lib.fmnmf_dp_iterate(self._dp, n, xp, lp, dev), self._dp)

    def metropolis(self, xi, logu):
        """The Z block alone: xi [S][T][D], logu [S][T]; returns (log gamma [S][T], accepted)."""
        xp, lp, dev, keep = self._draws(xi, logu)
        lg = np.empty((self.S, self.T), np.float32)
        n = ctypes.c_longlong(0)
        _check_dp(_lib.fmnmf_dp_metropolis(self._dp, xp, lp, dev, lg.ctypes.data, ctypes.byref(n)), self._dp)
        return lg, n.value

    def sync(self):
        _check_dp(_lib.fmnmf_dp_sync(self._dp), self._dp)

    def loglik(self) -> float:
        v = ctypes.c_double(0.0)
        _check_dp(_lib.fmnmf_dp_loglik(self._dp, ctypes.byref(v)), self._dp)
        return v.value

    def accepted(self) -> int:
        n = ctypes.c_longlong(0)
        _check_dp(_lib.fmnmf_dp_accepted(self._dp, ctypes.byref(n)), self._dp)
        return n.value

    def separate(self) -> np.ndarray:
        out = np.empty((self.N, self.F, self.T, self.M), np.complex64)
        _check_dp(_lib.fmnmf_dp_separate(self._dp, out.ctypes.data, 0), self._dp)
        return out


def stft_frames(S: int, L: int = 1024, hop: int = 256) -> int:
    """Frames of a signal of S samples: 1 if S <= L, else 1 + ceil((S - L) / hop)."""
    T = ctypes.c_int()
    _check(_lib.fmnmf_stft_frames(S, L, hop, ctypes.byref(T)))
    return T.value


def _cuda_stream(dev) -> int:
    return torch.cuda.current_stream(dev).cuda_stream


def stft(x, L: int = 1024, hop: int = 256):
    """STFT of device signals x (torch float32 CUDA tensor [M, S]) on torch's current stream:
    X[f, t, m] (complex64 [L/2 + 1, T, M]) with a periodic Hann window, frames at t * hop."""
    assert torch is not None and isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float32
    x = x.contiguous()
    M, S = x.shape
    T = stft_frames(S, L, hop)
    X = torch.empty((L // 2 + 1, T, M), dtype=torch.complex64, device=x.device)
    _check(_lib.fmnmf_stft(x.data_ptr(), M, S, L, hop, X.data_ptr(), _cuda_stream(x.device)))
    return X


def istft(Y, S: int, L: int = 1024, hop: int = 256):
    """Inverse of ``stft`` for device images Y (torch complex64 CUDA [B, F, T, M] or [F, T, M])
    on torch's current stream: y[B, M, S] float32 (weighted overlap-add)."""
    assert torch is not None and isinstance(Y, torch.Tensor) and Y.is_cuda and Y.dtype == torch.complex64
    squeeze = Y.dim() == 3
    Y = (Y[None] if squeeze else Y).contiguous()
    B, F, T, M = Y.shape
    y = torch.empty((B, M, S), dtype=torch.float32, device=Y.device)
    _check(_lib.fmnmf_istft(Y.data_ptr(), B, F, T, M, S, L, hop, y.data_ptr(), _cuda_stream(Y.device)))
    return y[0] if squeeze else y


JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_FAILED = 0, 1, 2, 3


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_active", ctypes.c_int), ("iters_per_step", ctypes.c_int),
                ("precision", ctypes.c_int)]


def footprint(F, T, M, N, K, precision=PREC_FP32) -> int:
    o = default_opts()
    o.precision = precision
    b = ctypes.c_size_t()
    _check(_lib.fmnmf_footprint(F, T, M, N, K, ctypes.byref(o), ctypes.byref(b)))
    return b.value


class Server:
    """Continuous-batching separation server (wraps fmnmf_server)."""

    def __init__(self, hbm_budget=0, max_active=16, iters_per_step=10, precision=PREC_FP32):
        o = ServerOpts(hbm_budget, max_active, iters_per_step, precision)
        self._s = _P()
        _check(_lib.fmnmf_server_create(ctypes.byref(o), ctypes.byref(self._s)))
        self._shapes = {}

    def submit(self, X, N, K, n_iter, seed=0) -> int:
        Xh, ptr = _host_ptr(X, np.complex64)
        F, T, M = Xh.shape
        job = ctypes.c_uint64()
        _check(_lib.fmnmf_server_submit(self._s, ptr, F, T, M, N, K, n_iter, seed, ctypes.byref(job)))
        self._shapes[job.value] = (N, F, T, M)
        return job.value

    def poll(self, job):
        st, lat = _I(), ctypes.c_double()
        _check(_lib.fmnmf_server_poll(self._s, job, ctypes.byref(st), ctypes.byref(lat)))
        return st.value, lat.value

    def wait(self, job, timeout=600.0) -> int:
        st = _I()
        _check(_lib.fmnmf_server_wait(self._s, job, timeout, ctypes.byref(st)))
        return st.value

    def result(self, job):
        out = np.empty(self._shapes.pop(job), np.complex64)
        ll = ctypes.c_double()
        _check(_lib.fmnmf_server_result(self._s, job, out.ctypes.data, ctypes.byref(ll)))
        return out, ll.value

    def stats(self) -> dict:
        q, a, c, f = (ctypes.c_longlong() for _ in range(4))
        b = ctypes.c_size_t()
        _check(_lib.fmnmf_server_stats(self._s, ctypes.byref(q), ctypes.byref(a), ctypes.byref(c), ctypes.byref(f), ctypes.byref(b)))
        return {"queued": q.value, "active": a.value, "completed": c.value, "failed": f.value, "bytes_in_use": b.value}

    def close(self):
        if self._s:
            _lib.fmnmf_server_destroy(self._s)
            self._s = _P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
