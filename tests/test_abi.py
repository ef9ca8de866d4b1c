"""The C-ABI library loads and exports every symbol include/boa.h declares
(no GPU calls here), and the host-side logic that needs no device behaves."""
import os
import re

import pytest

from paper_2511_11337_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "boa.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(boa_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_loads():
    build.build()
    lib = _lib.load()
    assert lib is not None


def test_every_declared_symbol_is_exported_and_bound():
    lib = _lib.load()
    syms = declared_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
        assert s in _lib.SIGNATURES, s
    assert set(_lib.SIGNATURES) == set(syms)


def test_max_compressed_size():
    lib = _lib.load()
    assert lib.boa_max_compressed_size(0) == 0
    assert lib.boa_max_compressed_size(1) == 1
    assert lib.boa_max_compressed_size(2) == 1 + 5 + 4
    assert lib.boa_max_compressed_size(16384) == 1 + 5 * 16383 + 4


def test_load_errors_are_reported_not_raised(tmp_path):
    from paper_2511_11337_b300 import api
    with pytest.raises(_lib.BoaError) as e:
        api.Model(str(tmp_path / "missing.boaw"))
    assert e.value.code == 2
    bad = tmp_path / "bad.boaw"
    bad.write_bytes(b"XXXX" + b"\0" * 100)
    with pytest.raises(_lib.BoaError) as e:
        api.Model(str(bad))
    assert e.value.code == 3


def test_product_path_does_not_import_oracle():
    """Nothing in the package imports, links or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_2511_11337_b300")
    pat = re.compile(r"^\s*(from\s+oracle|import\s+oracle)|liboracle|boa_oracle", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert not pat.search(open(os.path.join(dirpath, f)).read()), f


def test_container_checksum_is_crc32():
    """The container checksum is CRC-32 (IEEE 802.3): check value of
    "123456789" is 0xCBF43926, and it agrees with zlib on random data."""
    import zlib

    import numpy as np

    from paper_2511_11337_b300 import api
    assert api.crc32(b"123456789") == 0xCBF43926
    assert api.crc32(b"") == 0
    data = np.random.default_rng(0).integers(0, 256, 10007, dtype=np.uint8).tobytes()
    assert api.crc32(data) == zlib.crc32(data)


def test_container_header_checks_without_gpu():
    import ctypes as C

    import numpy as np

    from paper_2511_11337_b300 import _lib
    lib = _lib.load()
    assert lib.boa_pack_bound(0, 16) == 56
    assert lib.boa_pack_bound(33, 16) == 56 + 3 * 16 + 2 * (1 + 5 * 15 + 4) + 1
    junk = np.zeros(100, np.uint8)
    t, f = C.c_uint64(), C.c_uint64()
    assert lib.boa_unpack_info(junk.ctypes.data_as(C.c_void_p), 100, C.byref(t), C.byref(f)) == 3
    assert lib.boa_unpack_info(junk.ctypes.data_as(C.c_void_p), 10, C.byref(t), C.byref(f)) == 7


def test_stream_entry_points_check_arguments():
    """The streaming pipeline's argument checks need no GPU."""
    import ctypes as C
    lib = _lib.load()
    h = C.c_void_p()
    assert lib.boa_stream_open(None, 16, 4, C.byref(h)) == 1 and not h.value
    assert lib.boa_stream_push(None, None, 0) == 1
    assert lib.boa_stream_finish(None) == 1
    assert lib.boa_stream_available(None) == 0
    n = C.c_size_t()
    assert lib.boa_stream_read(None, None, 0, C.byref(n)) == 1
    assert lib.boa_stream_stats(None, None, None, None) == 1
    lib.boa_stream_close(None)
    assert lib.boa_unpack_shards(None, None, 0, None, 0, C.byref(n)) == 1


def test_bench_traffic_record_is_read_safely(tmp_path, monkeypatch):
    """bench.traffic_for returns the committed record only while the decode
    scan's sources hash as recorded, and None (never an exception) for a
    stale, old-format or missing record."""
    import json
    import bench
    ent = bench.traffic_for("decompress:scan")
    assert ent is None or ent["bytes_per_launch"] > 0
    assert bench.traffic_for("no such kernel") is None
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "profiles").mkdir()
    assert bench.traffic_for("decompress:scan") is None
    for rec in ({"source": "x.cuh", "source_sha256": "0"}, {"sources": ["x.cuh"], "sources_sha256": "0"}):
        (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({"decompress:scan": rec}))
        assert bench.traffic_for("decompress:scan") is None
