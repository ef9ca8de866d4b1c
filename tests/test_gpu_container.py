"""The .boa container, the autotuner and the graph-captured decode loop."""
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


def test_pack_unpack_round_trip(api, tiny_model_path):
    m = api.Model(tiny_model_path)
    data = synth.atlas_table(50_000, seed=4)          # 3 chunks + a ragged tail at 16 KB
    box = m.pack(data, chunk_len=16384)
    assert box[:4] == b"BOA1"
    assert m.unpack(box) == data
    assert m.unpack(m.pack(b"", 4096)) == b""
    assert m.unpack(m.pack(data[:1], 4096)) == data[:1]
    small = m.pack(data[:5000], chunk_len=700)        # many short chunks
    assert m.unpack(small) == data[:5000]


def test_container_refuses_wrong_model_and_corruption(api, tiny_model_path, peaked_model_path):
    m = api.Model(tiny_model_path)
    data = synth.records_stream(5, 20_000)
    box = bytearray(m.pack(data, chunk_len=4096))
    with pytest.raises(api.BoaError) as e:
        api.Model(peaked_model_path).unpack(bytes(box))
    assert e.value.code == 8
    bad = bytearray(box); bad[56 + 3] ^= 1            # index byte
    with pytest.raises(api.BoaError) as e:
        m.unpack(bytes(bad))
    assert e.value.code == 7
    bad = bytearray(box); bad[20] ^= 1                # header byte
    with pytest.raises(api.BoaError) as e:
        m.unpack(bytes(bad))
    assert e.value.code == 7
    with pytest.raises(api.BoaError):
        m.unpack(bytes(box[:-10]))                    # truncated payload


def test_autotune_keeps_bytes(api, tiny_model_path):
    streams = [synth.records_stream(40 + i, 700 + 37 * i) for i in range(24)]
    m = api.Model(tiny_model_path)
    before = m.compress(streams)
    t = m.autotune(len(streams), 1024)
    assert t["max_rows"] in (1 << 16, 1 << 17, 1 << 18, 1 << 19) and t["scan_variant"] in (0, 1, 2, 3)
    after = m.compress(streams)
    assert after == before
    assert m.decompress(after, [len(s) for s in streams]) == streams


def test_graph_and_eager_decode_agree(api, tiny_model_path):
    """The decode step loop runs as CUDA graphs of 32 steps; with kernel
    profiling on, a timed eager step (lanes one after another) precedes each
    graph launch.  Lanes on separate streams or not, the bytes agree, and
    the step counts add up."""
    streams = [synth.records_stream(90 + i, 3000 + 11 * i) for i in range(5)]
    m = api.Model(tiny_model_path)
    comp = m.compress(streams)
    lens = [len(s) for s in streams]
    assert m.decompress(comp, lens) == streams        # graphs
    for lanes in (1, 2):
        m.set_tuning(1 << 18, 0, lanes)
        m.profile(True, 1)
        m.profile_reset()
        try:
            assert m.decompress(comp, lens) == streams
            timed, total = m.profile_steps()["decompress"]
            assert total == max(lens) - 1 and 0 < timed < total
            assert m.profile_read()["decompress"]["scan"]["launches"] == timed * lanes * 2
        finally:
            m.profile(False)


@pytest.mark.parametrize("d_model,expand,prec,d_conv", [(64, 2, 0, 4), (256, 2, 2, 4), (64, 3, 1, 4), (128, 4, 0, 4),
                                                         (64, 2, 2, 3), (64, 2, 1, 2), (64, 2, 3, 4), (128, 2, 3, 4),
                                                         (256, 2, 3, 4)])
def test_decode_scan_variants_agree(api, tmp_path, d_model, expand, prec, d_conv):
    """Every decode-step scan kernel (persistent bulk-copy fed, four channels
    per thread, one or eight streams per CTA), with the slots split into one
    to four lanes on separate streams, decodes the same bytes.  Many
    short streams: more slots than the persistent grid, so its CTAs walk
    several streams, with a ragged last round; model widths cover one to
    eight CTAs per SM and two to four ring stages; conv widths 2 to 4 and
    every precision form.  FP8 at d_model 128 and 256: in_proj's FP8 rows
    (K = d) are narrower than the FP8 scratch's per-row room (K = expand d),
    so a lane that read rows written through another lane's view would
    decode garbage."""
    shape = synth.ModelShape(d_model=d_model, n_layer=2, expand=expand, d_conv=d_conv)
    path = synth.make_model_file(str(tmp_path / "v.boaw"), shape, seed=7)
    g = np.random.default_rng(d_model + expand)
    lens = g.integers(2, 90, size=2500)
    buf = synth.atlas_table(int(lens.sum()), seed=11)
    off = np.concatenate([[0], np.cumsum(lens)])
    streams = [buf[off[i]:off[i + 1]] for i in range(len(lens))]
    m = api.Model(path, precision=prec)
    comp = m.compress(streams)
    for v, lanes in ((0, 1), (0, 3), (1, 2), (2, 1), (3, 4)):
        m.set_tuning(1 << 18, v, lanes)
        assert m.tuning() == {"max_rows": 1 << 18, "scan_variant": v, "decode_lanes": lanes, "decoder": 0}
        assert m.decompress(comp, [len(s) for s in streams]) == streams, (v, lanes)
    with pytest.raises(api.BoaError):
        m.set_tuning(1 << 18, 4)
    with pytest.raises(api.BoaError):
        m.set_tuning(1 << 18, 0, 17)
