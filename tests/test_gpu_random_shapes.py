"""Seeded random shapes in every form against the float64 oracle (one iteration from the same
state), so that the per-bucket, per-tail and per-schedule code paths are exercised beyond the
hand-picked shapes of the other parity tests.

Shapes: F in [1, 300], T in [4 M, 700], M in [1, 8] (every channel bucket), N in [1, 6], K in
[1, 70]; inputs from the generative model.

Bars.  The base bars are those of the other parity tests: 1e-5 per tensor and per element for
the two FP32 schedules, 1e-3 for the tensor-core forms.  With few frames per channel V_fm
becomes ill-conditioned (at F270 T193 M8 its condition number reaches 7.9e4), and the IP step
(Eqs. 19-20) amplifies the rounding of V_fm by up to that factor in every form; normalisation
(phi, Sec. III-A-3) carries it into W.  Where an error is above its base bar, it is held to
the error the oracle itself makes when V_fm is rounded before the IP, to the precision the
form forms V_fm in:

* FP32 schedules: V_fm rounded to float32 (24 significant bits), times sqrt(T) -- a float32
  sum of T frames carries about sqrt(T) independent roundings where storage carries one;
* tensor-core forms: V_fm rounded to 16 significant bits, the precision of the split
  operands (hi + lo, 8 + 8 bits) its products are formed from.
"""
import functools

import numpy as np
import pytest

from oracle import fastmnmf_oracle as O
from paper_1903_03237_gb300.synth import make_mixture, make_state

from tests._parity import state_errors, ll_rel, as64


def _shapes(n=24, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        M = int(rng.integers(1, 9))
        T = int(rng.integers(4 * M, 701))
        out.append((int(rng.integers(1, 301)), T, M, int(rng.integers(1, 7)), int(rng.integers(1, 71)), 100 + i))
    return out


SHAPES = _shapes()
FORMS = ["fused", "sweep", "bf16", "tf32"]
BASE = {"fused": 1e-5, "sweep": 1e-5, "bf16": 1e-3, "tf32": 1e-3}
V_BITS = {"fused": 24, "sweep": 24, "bf16": 16, "tf32": 16}


def _round_bits(a, p):
    """a rounded to p significant bits (round to nearest)."""
    m, e = np.frexp(a)
    return np.ldexp(np.round(m * 2.0 ** p) / 2.0 ** p, e)


@functools.lru_cache(maxsize=None)
def _oracle(shape):
    F, T, M, N, K, seed = shape
    mix = make_mixture(F, T, M, N, K, seed)
    W, H, G, Q = make_state(F, T, M, N, K, seed)
    X64 = mix.X.astype(np.complex128)
    return O.iterate(X64, *as64(W, H, G, Q), n_iter=1)


@functools.lru_cache(maxsize=None)
def _rounded_v_floor(shape, p):
    """Errors of the oracle's own iteration when V_fm (Eq. 18) is rounded to p bits before the
    IP step, against the unrounded oracle: the error that rounding alone causes."""
    F, T, M, N, K, seed = shape
    mix = make_mixture(F, T, M, N, K, seed)
    W, H, G, Q = make_state(F, T, M, N, K, seed)
    X64 = mix.X.astype(np.complex128)
    exact = O.weighted_scm

    def rounded(X, yt):
        V = exact(X, yt)
        return _round_bits(V.real, p) + 1j * _round_bits(V.imag, p)

    O.weighted_scm = rounded
    try:
        Wp, Hp, Gp, Qp, _ = O.iterate(X64, *as64(W, H, G, Q), n_iter=1)
    finally:
        O.weighted_scm = exact
    Wr, Hr, Gr, Qr, _ = _oracle(shape)
    return state_errors(Wp, Hp, Gp, Qp, Wr, Hr, Gr, Qr, 1.0)


def test_rounded_v_floor_is_a_perturbation():
    """The floor helper perturbs the oracle only inside its call, and rounding to 53 bits is
    no perturbation at all."""
    shape = (7, 40, 3, 2, 4, 1)
    assert O.weighted_scm.__name__ == "weighted_scm"
    e53 = _rounded_v_floor(shape, 53)
    assert O.weighted_scm.__name__ == "weighted_scm"
    assert max(e53.values()) == 0.0
    e24 = _rounded_v_floor(shape, 24)
    assert 0.0 < e24["Q"] < 1e-5


@pytest.fixture(scope="module")
def fm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1903_03237_gb300.build import build
    build()
    from paper_1903_03237_gb300 import fastmnmf
    return fastmnmf


@pytest.mark.gpu
@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("shape", SHAPES, ids=[f"F{s[0]}T{s[1]}M{s[2]}N{s[3]}K{s[4]}" for s in SHAPES])
def test_random_shape_one_iteration(fm, shape, form):
    F, T, M, N, K, seed = shape
    mix = make_mixture(F, T, M, N, K, seed)
    W, H, G, Q = make_state(F, T, M, N, K, seed)
    kw = {"fused": dict(schedule=fm.SCHED_FUSED), "sweep": dict(schedule=fm.SCHED_SWEEP),
          "bf16": dict(precision=fm.PREC_BF16), "tf32": dict(precision=fm.PREC_TF32)}[form]
    try:
        ctx = fm.Context(mix.X, N, K, **kw)
    except fm.FastMNMFError as e:
        # a shape the form does not take (the fused schedule needs N*M <= 256; the tensor-core
        # V_fm kernel bounds N): refused at creation, never computed wrongly
        assert e.status == fm.EINVAL, e
        pytest.skip(str(e))
    ctx.set_state(W, H, G, Q)
    ctx.iterate(1)
    ll = ctx.loglik()
    Wg, Hg, Gg, Qg = ctx.get_state()
    ctx.close()
    X64 = mix.X.astype(np.complex128)
    Wr, Hr, Gr, Qr, tr = _oracle(shape)
    err = state_errors(Wg, Hg, Gg, Qg, Wr, Hr, Gr, Qr, 1.0)
    print(form, shape, {k: f"{v:.1e}" for k, v in err.items()})
    base = BASE[form]
    assert ll_rel(ll, tr[-1], X64, Wr, Hr, Gr, Qr) < base
    over = {k: v for k, v in err.items() if not v < base}
    if over:
        floor = _rounded_v_floor(shape, V_BITS[form])
        scale = np.sqrt(T) if V_BITS[form] == 24 else 1.0
        bars = {k: scale * floor[k] for k in over}
        print("  above the base bar:", {k: f"{v:.1e} (bar {bars[k]:.1e})" for k, v in over.items()})
        for k, v in over.items():
            assert v < bars[k], (k, v, bars[k], err)
