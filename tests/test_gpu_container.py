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
    assert t["max_rows"] in (1 << 16, 1 << 17, 1 << 18, 1 << 19) and t["scan_group"] in (0, 1, 2, 4, 8, 16)
    after = m.compress(streams)
    assert after == before
    assert m.decompress(after, [len(s) for s in streams]) == streams


def test_graph_and_eager_decode_agree(api, tiny_model_path):
    """The decode step loop runs as CUDA graphs unless kernel profiling is on;
    both give the same bytes."""
    streams = [synth.records_stream(90 + i, 3000 + 11 * i) for i in range(5)]
    m = api.Model(tiny_model_path)
    comp = m.compress(streams)
    lens = [len(s) for s in streams]
    assert m.decompress(comp, lens) == streams        # graphs
    m.profile(True, 1)
    try:
        assert m.decompress(comp, lens) == streams    # eager, profiled
    finally:
        m.profile(False)
