"""The streaming pipeline (boa_stream_*, the paper's section "Streaming"):
pushed bytes cut into sets of chunks, each set compressed into one container
shard by a worker thread while the next set fills and pre-loads the device.
Shards are byte-identical to boa_pack of the same set, decode alone
(boa_unpack) and together (boa_unpack_shards), and every set after the first
is already on the device when the worker takes it."""
import os
import struct

import numpy as np
import pytest

from paper_2511_11337_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2511_11337_b300 import api as A, build
    build.build()
    return A


@pytest.fixture(scope="module")
def paper_model_path(model_dir):
    return synth.make_model_file(os.path.join(model_dir, "paper_stream.boaw"), synth.PAPER_SCALE, seed=2)


def split_shards(blob: bytes) -> list[bytes]:
    """Container boundaries read from the documented header and index."""
    out, at = [], 0
    while at < len(blob):
        n = struct.unpack_from("<Q", blob, at + 32)[0]
        idx = [struct.unpack_from("<QQ", blob, at + 56 + 16 * i) for i in range(n)]
        end = max((o + z for o, z in idx), default=0)
        size = 56 + 16 * n + end
        out.append(blob[at:at + size])
        at += size
    assert at == len(blob)
    return out


def stream_compress(api, model, data, chunk_len, set_chunks, pieces):
    with api.Stream(model, chunk_len, set_chunks) as st:
        at, out = 0, []
        for k in pieces:
            st.push(data[at:at + k])
            at += k
            out.append(st.read())                  # shards finished so far
        st.push(data[at:])
        st.finish()
        out.append(st.read())
        stats = st.stats()
    return b"".join(out), stats


@pytest.mark.parametrize("form", ["PREC_FP32", "PREC_TF32X3"])
def test_shards_equal_pack_and_round_trip(api, tiny_model_path, form):
    m = api.Model(tiny_model_path, precision=getattr(api, form))
    data = synth.records_stream(77, 300_000)
    chunk, per = 4096, 8                            # 32 KB sets: 9 full sets and a ragged one
    pieces = np.random.default_rng(3).integers(1, 50_000, 12).tolist()
    blob, stats = stream_compress(api, m, data, chunk, per, pieces)
    shards = split_shards(blob)
    set_bytes = chunk * per
    assert len(shards) == -(-len(data) // set_bytes) == stats["sets"]
    assert stats["bytes_in"] == len(data)
    for i, sh in enumerate(shards):
        part = data[i * set_bytes:(i + 1) * set_bytes]
        assert sh == m.pack(part, chunk), i
        assert m.unpack(sh) == part
    assert m.unpack_shards(blob) == data


def test_next_set_is_preloaded(api, paper_model_path):
    """Benchmark model, sets of 64 x 16 KB: the caller fills and copies the
    next set while the worker compresses the current one."""
    m = api.Model(paper_model_path, precision=api.PREC_TF32X3)
    data = synth.atlas_table(8 * 64 * 16384, seed=11)
    blob, stats = stream_compress(api, m, data, 16384, 64, [64 * 16384] * 7)
    assert stats["sets"] == 8
    assert stats["preloaded"] >= stats["sets"] - 2, stats
    assert m.unpack_shards(blob) == data


def test_empty_and_tiny_streams(api, tiny_model_path):
    m = api.Model(tiny_model_path)
    blob, stats = stream_compress(api, m, b"", 1024, 4, [])
    assert blob == b"" and stats["sets"] == 0
    assert m.unpack_shards(b"") == b""
    blob, stats = stream_compress(api, m, b"x", 1024, 4, [])
    assert stats["sets"] == 1 and m.unpack_shards(blob) == b"x"


def test_stream_errors(api, tiny_model_path, peaked_model_path):
    m = api.Model(tiny_model_path)
    with pytest.raises(api.BoaError) as e:
        api.Stream(m, 0, 4)
    assert e.value.code == 1
    st = api.Stream(m, 1024, 1)                          # one chunk per set: 3 shards
    st.push(b"abc" * 1000)
    st.finish()
    with pytest.raises(api.BoaError) as e:
        st.push(b"more")
    assert e.value.code == 1
    blob = st.read()
    st.close()
    data = b"abc" * 1000
    assert m.unpack_shards(blob) == data
    with pytest.raises(api.BoaError) as e:             # another model's shards
        api.Model(peaked_model_path).unpack_shards(blob)
    assert e.value.code == 8
    shards = split_shards(blob)
    assert len(shards) == 3
    bad = bytearray(blob)
    bad[len(shards[0]) + 20] ^= 1                       # second shard's header
    with pytest.raises(api.BoaError) as e:
        m.unpack_shards(bytes(bad))
    assert e.value.code == 7
    with pytest.raises(api.BoaError) as e:              # last shard cut short
        m.unpack_shards(blob[:-3])
    assert e.value.code == 7
