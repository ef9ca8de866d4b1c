"""Pins for the oracle's predictor (CPU only).

Each building block is pinned by a closed form or a textbook routine, and the
composed forward pass by special cases and by an independent whole-sequence
("materialised") re-derivation at tiny sizes:
* LayerNorm: closed forms for +-1 inputs, constant inputs, affine gamma/beta.
* softmax: equal logits give 1/256 (log2 = -8); one raised logit gives 3/258.
* causal depthwise conv: equals numpy.convolve with the taps reversed.
* selective scan (App. A): equals the materialised sum
      y_t = D u_t + sum_{s<=t} sum_n C_t[n] exp(sum_{q=s+1..t} Delta_q A[n]) Delta_s B_s[n] u_s,
  and, for constant Delta, B, C (the LTI case), a convolution with the kernel
  K_k = sum_n C[n] exp(Delta A[n])^k Delta B[n].
* whole model: zero out_proj reduces each block to its LayerNorms; a
  memoryless configuration makes logits depend on the current byte only; and
  the step-by-step recurrence equals a vectorised whole-sequence evaluation.
"""
import math
import os

import numpy as np
import pytest
from scipy.special import erf

from oracle import oracle as O
from paper_2511_11337_b300 import synth


# ------------------------------------------------------------- LayerNorm

def test_layernorm_closed_forms():
    y = O.layernorm([1.0, -1.0], [1.0, 1.0], [0.0, 0.0])
    assert np.allclose(y, np.array([1.0, -1.0]) / math.sqrt(1 + 1e-5), rtol=0, atol=1e-15)
    y = O.layernorm(np.full(8, 3.75), np.full(8, 2.0), np.arange(8.0))
    assert np.array_equal(y, np.arange(8.0))
    # gamma = 2, beta = 3 on x = [0, 2] (mean 1, var 1)
    y = O.layernorm([0.0, 2.0], [2.0, 2.0], [3.0, 3.0])
    s = 1 / math.sqrt(1 + 1e-5)
    assert np.allclose(y, [3 - 2 * s, 3 + 2 * s], rtol=0, atol=1e-14)


def test_layernorm_moments():
    g = np.random.default_rng(0)
    x = g.normal(5, 3, 256)
    y = O.layernorm(x, np.ones(256), np.zeros(256))
    var = x.var()
    assert abs(y.mean()) < 1e-12 and abs(y.var() - var / (var + 1e-5)) < 1e-12


# ------------------------------------------------------------- softmax

def test_softmax_closed_forms():
    assert np.allclose(O.softmax(np.zeros(256)), 1 / 256, rtol=0, atol=1e-18)
    assert np.array_equal(O.log2_softmax(np.full(256, 4.2)), np.full(256, -8.0))
    l = np.zeros(256); l[9] = math.log(3.0)
    p = O.softmax(l)
    assert abs(p[9] - 3 / 258) < 1e-16 and abs(p[0] - 1 / 258) < 1e-16
    lp = O.log2_softmax(l)
    assert abs(lp[9] - math.log2(3 / 258)) < 1e-13
    # shift invariance
    g = np.random.default_rng(1); l = g.normal(0, 5, 256)
    assert np.allclose(O.softmax(l), O.softmax(l + 123.0), rtol=1e-12, atol=0)


# ------------------------------------------------------------- conv and scan

def test_conv_equals_numpy_convolve():
    g = np.random.default_rng(2)
    T, E, K = 23, 5, 4
    x = g.normal(size=(T, E)); w = g.normal(size=(E, K)); b = g.normal(size=E)
    out = O.causal_conv(x, w, b)
    for c in range(E):
        ref = np.convolve(x[:, c], w[c, ::-1])[:T] + b[c]
        assert np.allclose(out[:, c], ref, rtol=0, atol=1e-13)


def test_conv_impulse_response():
    T, E, K = 8, 1, 4
    x = np.zeros((T, E)); x[0, 0] = 1.0
    w = np.array([[1.0, 2.0, 3.0, 4.0]])
    out = O.causal_conv(x, w, np.zeros(1))[:, 0]
    assert list(out) == [4.0, 3.0, 2.0, 1.0, 0, 0, 0, 0]


def scan_materialised(u, delta, A, B, Cm, D):
    T, E = u.shape
    N = A.shape[1]
    y = D[None, :] * u
    # S[t, c, n] = sum_{q <= t} delta[q, c] A[c, n]
    S = np.cumsum(delta[:, :, None] * A[None, :, :], axis=0)
    for t in range(T):
        for s in range(t + 1):
            decay = np.exp(S[t] - S[s])                       # prod_{q=s+1..t} exp(delta_q A)
            y[t] += np.einsum("n,cn,c,n,c->c", Cm[t], decay, delta[s], B[s], u[s])
    return y


def test_scan_equals_materialised_sum():
    g = np.random.default_rng(3)
    for T, E, N in ((1, 3, 2), (16, 8, 4), (11, 5, 16)):
        u = g.normal(size=(T, E)); delta = np.log1p(np.exp(g.normal(size=(T, E))))
        A = -np.exp(g.normal(size=(E, N))); B = g.normal(size=(T, N)); Cm = g.normal(size=(T, N))
        D = g.normal(size=E)
        assert np.allclose(O.selective_scan(u, delta, A, B, Cm, D),
                           scan_materialised(u, delta, A, B, Cm, D), rtol=1e-12, atol=1e-12)


def test_scan_lti_is_convolution():
    g = np.random.default_rng(4)
    T, E, N = 40, 3, 4
    u = g.normal(size=(T, E))
    dl = np.array([0.3, 0.9, 1.7])
    A = -np.arange(1, N + 1, dtype=float)[None].repeat(E, 0)
    Bv = g.normal(size=N); Cv = g.normal(size=N); D = g.normal(size=E)
    y = O.selective_scan(u, np.tile(dl, (T, 1)), A, np.tile(Bv, (T, 1)), np.tile(Cv, (T, 1)), D)
    for c in range(E):
        k = np.array([np.sum(Cv * np.exp(dl[c] * A[c]) ** j * dl[c] * Bv) for j in range(T)])
        ref = np.convolve(u[:, c], k)[:T] + D[c] * u[:, c]
        assert np.allclose(y[:, c], ref, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------- whole model

def _loud_weights(shape, seed):
    """Dense random weights with every term large enough to matter."""
    w = synth.init_weights(shape, seed)
    g = np.random.default_rng(seed)
    for k, a in w.items():
        if k.endswith("A_log"):
            w[k] = g.uniform(-1, 1.5, a.shape).astype(np.float32)
        else:
            scale = 0.5 / math.sqrt(a.shape[-1]) if a.ndim == 2 else 0.3
            w[k] = (g.normal(0, 1, a.shape) * scale + (1.0 if k.endswith(("ln_a.w", "ln_b.w")) else 0)).astype(np.float32)
    return w


def _np_ln(X, g, b):
    mu = X.mean(-1, keepdims=True)
    var = ((X - mu) ** 2).mean(-1, keepdims=True)
    return (X - mu) / np.sqrt(var + 1e-5) * g + b


def forward_materialised(shape, w, data):
    """Whole-sequence evaluation: every projection as one matrix product over
    all time steps, the conv as shifted sums, the scan as the materialised sum."""
    w = {k: v.astype(np.float64) for k, v in w.items()}
    tok = np.frombuffer(data, np.uint8)[:-1]
    T = len(tok)
    d, E, N, K, r = shape.d_model, shape.d_inner, shape.d_state, shape.d_conv, shape.dt_rank
    silu = lambda v: v / (1 + np.exp(-v))
    X = w["embed"][tok]
    for l in range(shape.n_layer):
        p = f"layers.{l}."
        XZ = _np_ln(X, w[p + "ln_a.w"], w[p + "ln_a.b"]) @ w[p + "in_proj.w"].T
        Xi, Z = XZ[:, :E], XZ[:, E:]
        pad = np.vstack([np.zeros((K - 1, E)), Xi])
        U = w[p + "conv.b"] + sum(w[p + "conv.w"][:, k] * pad[k:k + T] for k in range(K))
        U = silu(U)
        DBC = U @ w[p + "x_proj.w"].T
        pre = DBC[:, :r] @ w[p + "dt_proj.w"].T + w[p + "dt_proj.b"]
        Delta = np.where(pre > 20, pre, np.log1p(np.exp(pre)))
        A = -np.exp(w[p + "A_log"])
        Y = scan_materialised(U, Delta, A, DBC[:, r:r + N], DBC[:, r + N:], w[p + "D"])
        X = X + (Y * silu(Z)) @ w[p + "out_proj.w"].T
        if shape.ffn_mult:
            H = X @ w[p + "ffn.w1"].T + w[p + "ffn.b1"]
            H = 0.5 * H * (1 + erf(H / math.sqrt(2)))
            X = X + H @ w[p + "ffn.w2"].T + w[p + "ffn.b2"]
        X = _np_ln(X, w[p + "ln_b.w"], w[p + "ln_b.b"])
    return X @ w["head.w"].T + w["head.b"]


def _oracle_logits(path, data):
    m = O.Model(path)
    st = m.new_state()
    return np.array([st.step(b) for b in data[:-1]])


@pytest.mark.parametrize("ffn", [0, 4])
def test_step_recurrence_equals_materialised_forward(ffn, tmp_path):
    shape = synth.ModelShape(d_model=16, n_layer=2, d_state=4, ffn_mult=ffn)
    w = _loud_weights(shape, 7 + ffn)
    path = str(tmp_path / "m.boaw")
    synth.write_model(path, shape, w)
    data = bytes(np.random.default_rng(8).integers(0, 256, 14, dtype=np.uint8))
    got = _oracle_logits(path, data)
    ref = forward_materialised(shape, w, data)
    assert np.abs(ref).max() > 0.5          # the check is not vacuous
    assert np.allclose(got, ref, rtol=1e-10, atol=1e-10)


def test_zero_out_proj_reduces_to_layernorms(tmp_path):
    shape = synth.ModelShape(d_model=16, n_layer=3, d_state=4)
    w = _loud_weights(shape, 9)
    for l in range(shape.n_layer):
        w[f"layers.{l}.out_proj.w"][:] = 0
    path = str(tmp_path / "m.boaw")
    synth.write_model(path, shape, w)
    data = bytes([5, 200, 5, 17, 5, 99])
    got = _oracle_logits(path, data)
    w64 = {k: v.astype(np.float64) for k, v in w.items()}
    for t, b in enumerate(data[:-1]):
        x = w64["embed"][b]
        for l in range(shape.n_layer):
            x = _np_ln(x, w64[f"layers.{l}.ln_b.w"], w64[f"layers.{l}.ln_b.b"])
        ref = x @ w64["head.w"].T + w64["head.b"]
        assert np.allclose(got[t], ref, rtol=1e-12, atol=1e-12)


def test_memoryless_configuration(tmp_path):
    """Conv taps only on the newest input and exp(Delta A) = 0 make every
    step independent of history: logits equal those of a fresh stream."""
    shape = synth.ModelShape(d_model=16, n_layer=2, d_state=4)
    w = _loud_weights(shape, 10)
    for l in range(shape.n_layer):
        w[f"layers.{l}.conv.w"][:, :-1] = 0
        w[f"layers.{l}.A_log"][:] = 30.0
    path = str(tmp_path / "m.boaw")
    synth.write_model(path, shape, w)
    data = bytes([3, 9, 3, 250, 9, 3, 0])
    got = _oracle_logits(path, data)
    m = O.Model(path)
    for t, b in enumerate(data[:-1]):
        assert np.array_equal(got[t], m.new_state().step(b))


def test_causality(tiny_model_path):
    a = synth.records_stream(1, 40)
    b = a[:20] + bytes(x ^ 0x5A for x in a[20:])
    la, lb = _oracle_logits(tiny_model_path, a), _oracle_logits(tiny_model_path, b)
    assert np.array_equal(la[:20], lb[:20]) and not np.array_equal(la[20:], lb[20:])


def test_logprobs_match_steps(tiny_model_path):
    m = O.Model(tiny_model_path)
    data = synth.records_stream(2, 30)
    lp = m.logprobs(data)
    ref = np.array([O.log2_softmax(l) for l in _oracle_logits(tiny_model_path, data)])
    assert np.array_equal(lp, ref)
    assert np.allclose(np.exp2(lp).sum(1), 1.0, rtol=0, atol=1e-12)


def test_scan_gradient_matches_central_differences():
    """The oracle's reverse-mode scan gradient against central finite
    differences of the oracle's forward scan, for every input element."""
    g = np.random.default_rng(21)
    T, E, N = 7, 3, 2
    ins = {"u": g.normal(size=(T, E)), "delta": np.log1p(np.exp(g.normal(size=(T, E)))),
           "A": -np.exp(g.normal(size=(E, N))), "B": g.normal(size=(T, N)), "C": g.normal(size=(T, N)),
           "D": g.normal(size=E)}
    dy = g.normal(size=(T, E))
    grad = O.selective_scan_grad(ins["u"], ins["delta"], ins["A"], ins["B"], ins["C"], ins["D"], dy)

    def loss(v):
        y = O.selective_scan(v["u"], v["delta"], v["A"], v["B"], v["C"], v["D"])
        return float((dy * y).sum())

    h = 1e-6
    for name, arr in ins.items():
        for idx in np.ndindex(arr.shape):
            plus = {k: a.copy() for k, a in ins.items()}
            minus = {k: a.copy() for k, a in ins.items()}
            plus[name][idx] += h
            minus[name][idx] -= h
            fd = (loss(plus) - loss(minus)) / (2 * h)
            assert abs(fd - grad[name][idx]) <= 1e-6 * (1 + abs(fd)), (name, idx, fd, grad[name][idx])
