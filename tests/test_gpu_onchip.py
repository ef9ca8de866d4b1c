"""The on-chip persistent decoder (boa_tuning.decoder = 1, FP32 form).

One launch decodes every stream: one CTA per SM runs two streams at a time
from first to last byte, their SSM state and conv windows in the SM's tensor
memory across layers and steps, the weights streamed through shared memory.
It must reproduce the FP32 form's step-kernel decoder exactly:

* lossless round trips of streams the FP32 encoder wrote, and the same CDF
  at every step (the per-step histogram hashes of encoder and decoder);
* more streams than the 2 x SM-count slots (queue refill, a slot's state
  reset between streams), lengths 0, 1, 2 and ragged;
* the benchmark model (3 blocks, d_model 256, d_inner 512) and the small one;
* truncated input flagged for that stream only;
* a form or model it does not run refused by boa_set_tuning.
"""
import os

import numpy as np
import pytest

from paper_2511_11337_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2511_11337_b300 import api as A, build
    build.build()
    return A


def onchip(m):
    t = m.tuning()
    m.set_tuning(t["max_rows"], t["scan_variant"], t["decode_lanes"], decoder=1)


def hbm(m):
    t = m.tuning()
    m.set_tuning(t["max_rows"], t["scan_variant"], t["decode_lanes"], decoder=0)


def test_round_trip_and_cdfs_match_the_encoder(api, tiny_model_path):
    m = api.Model(tiny_model_path, precision=api.PREC_FP32)
    streams = [synth.records_stream(70 + i, n) for i, n in enumerate([3000, 1, 0, 2, 777, 4096, 130, 3])]
    n_steps = sum(max(len(s) - 1, 0) for s in streams)
    m.enable_cdf_trace(True)
    try:
        comp = m.compress(streams)
        enc = m.read_cdf_trace(n_steps)
        onchip(m)
        out = m.decompress(comp, [len(s) for s in streams])
        dec = m.read_cdf_trace(n_steps)
    finally:
        m.enable_cdf_trace(False)
        hbm(m)
    assert out == streams
    assert np.array_equal(enc, dec)
    assert m.last_launch_count <= 2          # the trivial-stream kernel and the decoder


def test_benchmark_model_more_streams_than_slots(api, model_dir):
    path = synth.make_model_file(os.path.join(model_dir, "paper_onchip.boaw"), synth.PAPER_SCALE, seed=2)
    m = api.Model(path, precision=api.PREC_FP32)
    g = np.random.default_rng(9)
    lens = [int(x) for x in g.integers(2, 700, 320)] + [0, 1, 2, 5000]
    buf = synth.atlas_workload(1, sum(lens), seed=91)
    streams, at = [], 0
    for n in lens:
        streams.append(buf[at:at + n])
        at += n
    comp = m.compress(streams)
    hbm(m)
    ref = m.decompress(comp, lens)
    onchip(m)
    try:
        out = m.decompress(comp, lens)
    finally:
        hbm(m)
    assert ref == streams and out == streams


def test_truncated_stream_flagged(api, tiny_model_path):
    m = api.Model(tiny_model_path, precision=api.PREC_FP32)
    streams = [synth.records_stream(11, 2000), synth.records_stream(12, 2000), synth.records_stream(13, 900)]
    comp = m.compress(streams)
    onchip(m)
    try:
        with pytest.raises(Exception) as e:
            m.decompress([comp[0][:-9], comp[1], comp[2]], [2000, 2000, 900])
        assert getattr(e.value, "code", None) == 7
        st = m.last_stream_status(3)
        assert st[0] & 2 and st[1] == 0 and st[2] == 0
        assert m.decompress(comp, [2000, 2000, 900]) == streams
    finally:
        hbm(m)


def test_refused_where_it_does_not_run(api, tiny_model_path, model_dir):
    t3 = api.Model(tiny_model_path, precision=api.PREC_TF32X3)
    with pytest.raises(Exception) as e:
        onchip(t3)
    assert getattr(e.value, "code", None) == 1
    ffn = synth.make_model_file(os.path.join(model_dir, "ffn_onchip.boaw"), synth.PAPER_SHAPE_FFN, seed=5)
    mf = api.Model(ffn, precision=api.PREC_FP32)
    with pytest.raises(Exception):
        onchip(mf)
    assert mf.tuning()["decoder"] == 0


def test_autotune_weighs_the_onchip_decoder(api, tiny_model_path):
    """boa_autotune times the on-chip decoder beside the step kernels for an
    FP32 model (its choice is reported in the tuning) and the model decodes
    correctly with whichever it keeps; for another form it never picks it."""
    m = api.Model(tiny_model_path, precision=api.PREC_FP32)
    t = m.autotune(16, 1024)
    assert t["decoder"] in (0, 1) and m.tuning()["decoder"] == t["decoder"]
    streams = [synth.records_stream(300 + i, 1024 + 37 * i) for i in range(16)]
    comp = m.compress(streams)
    assert m.decompress(comp, [len(s) for s in streams]) == streams
    t3 = api.Model(tiny_model_path, precision=api.PREC_TF32X3)
    assert t3.autotune(16, 1024)["decoder"] == 0


@pytest.mark.parametrize("d_model,n_layer,d_conv", [(128, 3, 4), (64, 1, 2), (128, 2, 3)])
def test_other_shapes_and_conv_widths(api, model_dir, d_model, n_layer, d_conv):
    """The decoder's other shapes: d_model 128 (d_inner 256, dt_rank 8), one
    block, and conv widths 2 and 3 (a window of one or two values)."""
    shape = synth.ModelShape(d_model=d_model, n_layer=n_layer, d_conv=d_conv)
    path = synth.make_model_file(os.path.join(model_dir, f"oc_{d_model}_{n_layer}_{d_conv}.boaw"), shape, seed=11)
    m = api.Model(path, precision=api.PREC_FP32)
    streams = [synth.records_stream(500 + i, n) for i, n in enumerate([900, 2, 1, 0, 333, 1500, 64] * 3)]
    n_steps = sum(max(len(s) - 1, 0) for s in streams)
    m.enable_cdf_trace(True)
    try:
        comp = m.compress(streams)
        enc = m.read_cdf_trace(n_steps)
        onchip(m)
        out = m.decompress(comp, [len(s) for s in streams])
        dec = m.read_cdf_trace(n_steps)
    finally:
        m.enable_cdf_trace(False)
        hbm(m)
    assert out == streams and np.array_equal(enc, dec)
