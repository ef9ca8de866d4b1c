"""Tensor-core (tcgen05) projection GEMM and the BF16 predictor path.

* The GEMM kernels against float64 products of the same (BF16-rounded or
  FP32) operands, for every epilogue and for shapes with ragged M and N.
* Row-position invariance: a row's result does not depend on the batch it
  sits in (what keeps the encoder and decoder in lockstep).
* The BF16 model: lossless round trip, identical CDFs in encoder and decoder,
  batch invariance, code length within 0.5 % of the FP64 oracle; the log2 p
  error against the oracle is reported against a stated bound.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_11337_b300 import synth

pytestmark = pytest.mark.gpu

BF16_LOG2P_TOL = 0.03    # BF16 operands: relative rounding 2^-9 per input, summed over d <= 512 terms
# E4M3 operands: 3 mantissa bits, relative rounding 2^-4 per input (each row
# and weight channel scaled to the full E4M3 range first, so no subnormal
# loss); the same accumulation as BF16 with a unit roundoff 2^5 times larger
FP8_LOG2P_TOL = BF16_LOG2P_TOL * 2.0 ** 5


def bf16_round(x):
    x = np.ascontiguousarray(x, np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def ref_gemm(A, W, bias, epi, C_in):
    acc = A.astype(np.float64) @ W.astype(np.float64).T
    if epi in (1, 3, 4):
        acc = acc + bias.astype(np.float64)
    if epi == 3:
        from scipy.special import erf
        acc = 0.5 * acc * (1 + erf(acc / np.sqrt(2)))
    if epi in (2, 4):
        acc = C_in.astype(np.float64) + acc
    return acc


@pytest.fixture(scope="module")
def api():
    from paper_2511_11337_b300 import api as A, build
    build.build()
    return A


SHAPES = [(128, 128, 64), (300, 1024, 256), (4096, 48, 512), (1000, 256, 512), (77, 64, 64), (129, 36, 64),
          (513, 256, 1024), (8500, 256, 256), (8300, 1024, 128),   # these two: compression-size 128-wide tiles
          (20000, 256, 512), (19000, 48, 512), (19000, 128, 256),  # grids that fill the GPU (BF16 / FP8
                                                                   # x_proj: split K inside one CTA's TMEM)
          (70001, 1024, 256), (30001, 256, 32)]  # 3xTF32: persistent CTAs, ~30 tiles each / one K block


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_gemm_kernels(api, shape, precision):
    M, N, K = shape
    if precision == 1 and K % 64:
        pytest.skip("BF16 K blocks are 64 wide")
    g = np.random.default_rng(M * 7 + N + K)
    A = g.normal(0, 1, (M, K)).astype(np.float32)
    W = g.normal(0, 0.05, (N, K)).astype(np.float32)
    bias = g.normal(0, 0.1, N).astype(np.float32)
    C_in = g.normal(0, 1, (M, N)).astype(np.float32)
    Ar, Wr = (bf16_round(A), bf16_round(W)) if precision == 1 else (A, W)
    mag = np.abs(Ar.astype(np.float64)) @ np.abs(Wr.astype(np.float64)).T
    for epi in range(5):
        got = api.gemm(A, W, bias, epi, C_in, precision=precision)
        ref = ref_gemm(Ar, Wr, bias, epi, C_in)
        bound = 4 * 2.0 ** -24 * (K + 2) * (mag + np.abs(bias) + np.abs(C_in) + 1e-30) + 1e-6
        if precision == 2:      # 3xTF32: each product carries ~3 x 2^-21 relative error
            bound = bound + 8 * 2.0 ** -21 * mag
        err = np.abs(got - ref)
        assert (err <= bound).all(), (epi, float(err.max()), float((err / bound).max()))


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
@pytest.mark.parametrize("NK", [(1024, 256), (48, 512), (256, 512), (256, 256), (128, 256)])
def test_gemm_rows_independent_of_batch(api, precision, NK):
    """A row's result does not depend on the batch it sits in: under split K
    (its partial sums added in an order fixed by (N, K) alone, whether the
    chunks run on the CTAs of a cluster and meet through distributed shared
    memory, as in the small slices, or sit in one CTA's TMEM, as in the BF16
    and FP8 forms' grids that fill the GPU: the 20000-row batch), and across
    tile widths
    (batches above 8192 rows run 128-wide tiles, the slices the decode-size
    64- and 48-wide ones where N calls for them), and for 3xTF32 between the
    persistent CTAs that walk the tiles of the full batch (two TMEM
    accumulators, the epilogue of one tile beside the main loop of the next)
    and the one-tile CTAs of the small slices."""
    N, K = NK
    g = np.random.default_rng(5)
    A = g.normal(0, 1, (20000, K)).astype(np.float32)
    W = g.normal(0, 0.05, (N, K)).astype(np.float32)
    full = api.gemm(A, W, precision=precision)
    for lo, hi in ((0, 1), (5, 133), (19999, 20000), (300, 428), (4000, 5000), (7000, 16000)):
        part = api.gemm(A[lo:hi], W, precision=precision)
        assert np.array_equal(part, full[lo:hi])


@pytest.fixture(scope="module")
def tiny_bf16(api, tiny_model_path):
    return api.Model(tiny_model_path, precision=api.PREC_BF16)


def test_bf16_round_trip_gap_and_logprobs(tiny_bf16, tiny_model_path):
    streams = synth.records_workload()
    comp = tiny_bf16.compress(streams)
    assert tiny_bf16.decompress(comp, [len(s) for s in streams]) == streams
    om = O.Model(tiny_model_path)
    ref = om.compress_batch(streams)
    gap = (sum(map(len, comp)) - sum(map(len, ref))) / sum(map(len, ref))
    assert abs(gap) <= 0.005, gap
    err = np.abs(tiny_bf16.logprobs(streams[0][:2000]) - om.logprobs(streams[0][:2000])).max()
    print(f"BF16 max |dlog2p| = {err:.3e}, code-length gap = {gap:+.3e}")
    assert err <= BF16_LOG2P_TOL


def test_bf16_encoder_decoder_lockstep_and_batch_invariance(tiny_bf16):
    streams = [synth.records_stream(60 + i, n) for i, n in enumerate([3000, 1, 0, 2, 777, 4096, 130])]
    n_steps = sum(max(len(s) - 1, 0) for s in streams)
    tiny_bf16.enable_cdf_trace(True)
    try:
        comp = tiny_bf16.compress(streams)
        enc = tiny_bf16.read_cdf_trace(n_steps)
        out = tiny_bf16.decompress(comp, [len(s) for s in streams])
        dec = tiny_bf16.read_cdf_trace(n_steps)
    finally:
        tiny_bf16.enable_cdf_trace(False)
    assert out == streams and np.array_equal(enc, dec)
    alone = tiny_bf16.compress([streams[0]])[0]
    assert alone == comp[0] and tiny_bf16.compress([streams[0]] * 40)[17] == alone


def test_bf16_paper_scale_batch(api, model_dir):
    path = synth.make_model_file(os.path.join(model_dir, "paper_bf16.boaw"), synth.PAPER_SCALE, seed=2)
    m = api.Model(path, precision=api.PREC_BF16)
    buf = synth.atlas_workload(300, 2048, seed=77)
    streams = synth.split_equal(buf, 300)
    comp = m.compress(streams)
    assert m.decompress(comp, [len(s) for s in streams]) == streams
    om = O.Model(path)
    ref = om.compress(streams[7])
    assert abs(len(comp[7]) - len(ref)) / len(ref) <= 0.005
    ffn = synth.make_model_file(os.path.join(model_dir, "ffn_bf16.boaw"), synth.PAPER_SHAPE_FFN, seed=5)
    mf = api.Model(ffn, precision=api.PREC_BF16)
    comp = mf.compress(streams[:50])
    assert mf.decompress(comp, [len(s) for s in streams[:50]]) == streams[:50]


@pytest.fixture(scope="module")
def tiny_t3(api, tiny_model_path):
    return api.Model(tiny_model_path, precision=api.PREC_TF32X3)


def test_tf32x3_meets_the_fp32_bounds(tiny_t3, tiny_model_path):
    """The 3xTF32 tensor-core form is held to the FP32 path's bounds."""
    streams = synth.records_workload()
    comp = tiny_t3.compress(streams)
    assert tiny_t3.decompress(comp, [len(s) for s in streams]) == streams
    om = O.Model(tiny_model_path)
    ref = om.compress_batch(streams)
    gap = (sum(map(len, comp)) - sum(map(len, ref))) / sum(map(len, ref))
    assert abs(gap) <= 0.005, gap
    worst = 0.0
    for data in streams:
        worst = max(worst, float(np.abs(tiny_t3.logprobs(data) - om.logprobs(data)).max()))
    print(f"TF32x3 max |dlog2p| = {worst:.3e}")
    assert worst <= 1e-3


def test_tf32x3_lockstep_and_batch_invariance(tiny_t3):
    streams = [synth.records_stream(90 + i, n) for i, n in enumerate([2500, 0, 1, 2, 640, 4097])]
    n_steps = sum(max(len(s) - 1, 0) for s in streams)
    tiny_t3.enable_cdf_trace(True)
    try:
        comp = tiny_t3.compress(streams)
        enc = tiny_t3.read_cdf_trace(n_steps)
        out = tiny_t3.decompress(comp, [len(s) for s in streams])
        dec = tiny_t3.read_cdf_trace(n_steps)
    finally:
        tiny_t3.enable_cdf_trace(False)
    assert out == streams and np.array_equal(enc, dec)
    assert tiny_t3.compress([streams[0]] * 33)[20] == comp[0]


def test_tf32x3_paper_scale(api, model_dir):
    path = synth.make_model_file(os.path.join(model_dir, "paper_t3.boaw"), synth.PAPER_SCALE, seed=2)
    m = api.Model(path, precision=api.PREC_TF32X3)
    buf = synth.atlas_workload(200, 2048, seed=78)
    streams = synth.split_equal(buf, 200)
    comp = m.compress(streams)
    assert m.decompress(comp, [len(s) for s in streams]) == streams
    om = O.Model(path)
    assert np.abs(m.logprobs(streams[3][:400]) - om.logprobs(streams[3][:400])).max() <= 1e-3


def test_tf32x3_paper_scale_lockstep(api, model_dir):
    """The benchmark model's shape in the 3xTF32 form: the encoder's
    (compression-size tiles, in-CTA chunks) and the decoder's (decode-size
    tiles, cluster split K) per-step CDFs are identical, with one and with
    two decode lanes."""
    path = synth.make_model_file(os.path.join(model_dir, "paper_t3l.boaw"), synth.PAPER_SCALE, seed=3)
    m = api.Model(path, precision=api.PREC_TF32X3)
    streams = synth.split_equal(synth.atlas_workload(300, 700, seed=79), 300) + [b"", b"x", b"ab"]
    n_steps = sum(max(len(s) - 1, 0) for s in streams)
    m.enable_cdf_trace(True)
    try:
        comp = m.compress(streams)
        enc = m.read_cdf_trace(n_steps)
        for lanes in (1, 2):
            m.set_tuning(1 << 18, 0, lanes)
            assert m.decompress(comp, [len(s) for s in streams]) == streams
            assert np.array_equal(m.read_cdf_trace(n_steps), enc), lanes
    finally:
        m.enable_cdf_trace(False)


# ------------------------------------------------------------------ FP8 E4M3

def e4m3_quant_rows(X):
    """Per-row scale max|x| / 448 and E4M3 values (round to nearest even,
    saturated), computed in float32 as the kernels do."""
    import torch
    X = np.ascontiguousarray(X, np.float32)
    amax = np.abs(X).max(axis=1).astype(np.float32)
    inv = np.where(amax > 0, np.float32(448.0) / np.where(amax > 0, amax, 1), 1).astype(np.float32)
    scale = np.where(amax > 0, amax / np.float32(448.0), 1).astype(np.float32)
    y = np.clip((X * inv[:, None]).astype(np.float32), -448, 448)
    q = torch.from_numpy(y).to(torch.float8_e4m3fn).float().numpy()
    return q, scale


@pytest.mark.parametrize("shape", [(128, 128, 128), (300, 1024, 256), (4096, 48, 512), (1000, 256, 512),
                                   (129, 36, 128), (513, 256, 1024), (77, 64, 64), (200, 36, 192)])
def test_fp8_gemm_kernel(api, shape):
    M, N, K = shape
    g = np.random.default_rng(M + 3 * N + K)
    A = g.normal(0, 1, (M, K)).astype(np.float32)
    W = g.normal(0, 0.05, (N, K)).astype(np.float32)
    bias = g.normal(0, 0.1, N).astype(np.float32)
    C_in = g.normal(0, 1, (M, N)).astype(np.float32)
    qa, sa = e4m3_quant_rows(A)
    qw, sw = e4m3_quant_rows(W)
    exact = (qa.astype(np.float64) @ qw.astype(np.float64).T) * sa[:, None] * sw[None, :]
    mag = (np.abs(qa.astype(np.float64)) @ np.abs(qw.astype(np.float64)).T) * sa[:, None] * sw[None, :]
    for epi in range(5):
        got = api.gemm(A, W, bias, epi, C_in, precision=api.PREC_FP8)
        ref = exact.copy()
        if epi in (1, 3, 4):
            ref = ref + bias
        if epi == 3:
            from scipy.special import erf
            ref = 0.5 * ref * (1 + erf(ref / np.sqrt(2)))
        if epi in (2, 4):
            ref = C_in + ref
        bound = 4 * 2.0 ** -24 * (K + 4) * (mag + np.abs(bias) + np.abs(C_in)) + 1e-6
        err = np.abs(got - ref)
        assert (err <= bound).all(), (epi, float(err.max()), float((err / bound).max()))


def test_fp8_model(api, model_dir):
    """FP8 projections (d_model 128, 2 layers): lossless, encoder and decoder
    in lockstep, code length within 0.5 % of the FP64 oracle."""
    shape = synth.ModelShape(d_model=128, n_layer=2)
    path = synth.make_model_file(os.path.join(model_dir, "d128.boaw"), shape, seed=11)
    m = api.Model(path, precision=api.PREC_FP8)
    streams = [synth.records_stream(300 + i, n) for i, n in enumerate([3000, 1, 0, 2, 1500, 2048])]
    n_steps = sum(max(len(s) - 1, 0) for s in streams)
    m.enable_cdf_trace(True)
    try:
        comp = m.compress(streams)
        enc = m.read_cdf_trace(n_steps)
        out = m.decompress(comp, [len(s) for s in streams])
        dec = m.read_cdf_trace(n_steps)
    finally:
        m.enable_cdf_trace(False)
    assert out == streams and np.array_equal(enc, dec)
    om = O.Model(path)
    ref = om.compress_batch(streams)
    gap = (sum(map(len, comp)) - sum(map(len, ref))) / sum(map(len, ref))
    err = np.abs(m.logprobs(streams[0][:1500]) - om.logprobs(streams[0][:1500])).max()
    print(f"FP8 max |dlog2p| = {err:.3e}, code-length gap = {gap:+.3e}")
    assert abs(gap) <= 0.005
    assert err <= FP8_LOG2P_TOL
    assert m.compress([streams[4]] * 9)[5] == comp[4]


def test_fp8_tiny_model(api, tiny_model_path):
    """d_model 64: the 64-wide K blocks are zero-padded to 128."""
    m = api.Model(tiny_model_path, precision=api.PREC_FP8)
    streams = synth.records_workload(4, 4096)
    comp = m.compress(streams)
    assert m.decompress(comp, [len(s) for s in streams]) == streams
    ref = O.Model(tiny_model_path).compress_batch(streams)
    assert abs(sum(map(len, comp)) - sum(map(len, ref))) / sum(map(len, ref)) <= 0.005
