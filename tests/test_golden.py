"""Stored expected values (tests/golden/*.json, written by
tests/golden/make_golden.py from the FP64 oracle alone).

CPU: the oracle still reproduces every stored value, and the hand-derived
cases (uniform coder, two quantiser rows) hold as derived.
GPU: the CUDA path matches the stored values under the parity bars: coder
bytes and quantiser histograms bit-exact, log2 p within 1e-3, code length
within 0.5 %, lossless round trip.
"""
import hashlib
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_11337_b300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
LOG2P_TOL = 1e-3
GAP_TOL = 0.005


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def sha(b: bytes) -> str:
    return hashlib.sha256(b).hexdigest()


def cdfs_from(hist):
    c = np.zeros((hist.shape[0], 257), np.uint32)
    c[:, 1:] = np.cumsum(hist, axis=1)
    return c


def coder_inputs(case):
    hist, syms = synth.random_histograms(case["n"], seed=case["seed"], adversarial=case["adversarial"])
    c = cdfs_from(hist)
    assert sha(c.tobytes() + syms.tobytes()) == case["inputs_sha256"], "input generator changed"
    return c, syms


def uniform_inputs(g):
    msg = np.frombuffer(g["uniform"]["message"].encode(), np.uint8)
    return np.tile((256 * np.arange(257)).astype(np.uint32), (len(msg), 1)), msg


def quantise_inputs(q):
    return np.stack([np.frombuffer(bytes.fromhex(r["p_f32_hex"]), ">u4").astype(np.uint32).view(np.float32)
                     for r in q["rows"]])


@pytest.fixture(scope="module")
def golden_model_path(model_dir):
    g = load("model_tiny.json")
    path = synth.make_model_file(os.path.join(model_dir, "golden_tiny.boaw"), synth.TINY, seed=g["model"]["seed"])
    assert sha(open(path, "rb").read()) == g["model"]["file_sha256"], "weight generator changed"
    return path


def model_streams(g):
    out = []
    for s in g["streams"]:
        data = synth.records_stream(s["seed"], s["len"])
        assert sha(data) == s["data_sha256"], "stream generator changed"
        out.append(data)
    return out


# ------------------------------------------------------------------ CPU

def test_oracle_reproduces_coder_golden():
    g = load("coder.json")
    for case in g["cases"]:
        c, syms = coder_inputs(case)
        code, _ = O.encode_cdfs(c, syms)
        assert code.hex() == case["code_hex"], case["seed"]
        dec, ok = O.decode_cdfs(c, code, len(syms))
        assert ok and np.array_equal(dec, syms)
    c, msg = uniform_inputs(g)
    code, _ = O.encode_cdfs(c, msg)
    assert code.hex() == g["uniform"]["code_hex"]
    # the hand derivation: the message itself, then the four zero bytes of L
    assert bytes.fromhex(g["uniform"]["code_hex"]) == msg.tobytes() + bytes(4)


def test_oracle_reproduces_quantise_golden():
    q = load("quantise.json")
    p = quantise_inputs(q)
    for i, r in enumerate(q["rows"]):
        assert [int(x) for x in O.quantise_f32(p[i])] == r["f"], r["note"]
        assert sum(r["f"]) == 1 << 16 and min(r["f"]) >= 1
    by_note = {r["note"]: r["f"] for r in q["rows"]}
    a = by_note["hand case A"]
    assert a[:5] == [16322, 16321, 16321, 16193, 128] and a[5:] == [1] * 251
    b = by_note["hand case B"]
    assert b[:200] == [1] * 200 and b[200] == 1206 and b[201:] == [1166] * 55


def test_oracle_reproduces_model_golden(golden_model_path):
    g = load("model_tiny.json")
    om = O.Model(golden_model_path)
    for s, data in zip(g["streams"], model_streams(g)):
        code = om.compress(data)
        assert len(code) == s["code_len"] and sha(code) == s["code_sha256"], s["seed"]
        out, ok = om.decompress(code, len(data))
        assert ok and out == data
        if "log2p_next" in s:
            lp = om.logprobs(data)
            k = len(s["log2p_next"])
            nxt = np.frombuffer(data, np.uint8)[1:k + 1]
            np.testing.assert_allclose(lp[np.arange(k), nxt], [float(v) for v in s["log2p_next"]],
                                       rtol=0, atol=1e-12)
        if "log2p_row0" in s:
            np.testing.assert_allclose(om.logprobs(data)[0], [float(v) for v in s["log2p_row0"]], rtol=0, atol=1e-12)


# ------------------------------------------------------------------ GPU

@pytest.fixture(scope="module")
def api():
    from paper_2511_11337_b300 import api as A, build
    build.build()
    return A


@pytest.mark.gpu
def test_cuda_coder_matches_golden(api):
    g = load("coder.json")
    inputs = [coder_inputs(c) for c in g["cases"]] + [uniform_inputs(g)]
    expect = [c["code_hex"] for c in g["cases"]] + [g["uniform"]["code_hex"]]
    got = api.encode_cdfs([c for c, _ in inputs], [s for _, s in inputs])
    assert [x.hex() for x in got] == expect
    dec = api.decode_cdfs([c for c, _ in inputs], [bytes.fromhex(h) for h in expect])
    for (_, s), d in zip(inputs, dec):
        assert np.array_equal(s, d)


@pytest.mark.gpu
def test_cuda_quantiser_matches_golden(api):
    q = load("quantise.json")
    got = api.quantise(quantise_inputs(q))
    for i, r in enumerate(q["rows"]):
        assert [int(x) for x in got[i]] == r["f"], r["note"]


@pytest.mark.gpu
@pytest.mark.parametrize("form", ["PREC_FP32", "PREC_TF32X3"])
def test_cuda_model_matches_golden(api, golden_model_path, form):
    """The FP32 and 3xTF32 forms against the stored oracle values."""
    precision = getattr(api, form)
    g = load("model_tiny.json")
    streams = model_streams(g)
    m = api.Model(golden_model_path, precision=precision)
    comp = m.compress(streams)
    assert m.decompress(comp, [len(s) for s in streams]) == streams
    for s, c in zip(g["streams"], comp):
        if s["len"] <= 1:
            assert len(c) == s["code_len"]                      # raw first byte only
    total, ref = sum(map(len, comp)), sum(s["code_len"] for s in g["streams"])
    assert abs(total - ref) <= GAP_TOL * ref, (total, ref)
    for s, data in zip(g["streams"], streams):
        if "log2p_next" not in s:
            continue
        lp = m.logprobs(data)
        k = len(s["log2p_next"])
        nxt = np.frombuffer(data, np.uint8)[1:k + 1]
        assert np.abs(lp[np.arange(k), nxt] - np.array([float(v) for v in s["log2p_next"]])).max() <= LOG2P_TOL
        if "log2p_row0" in s:
            assert np.abs(lp[0] - np.array([float(v) for v in s["log2p_row0"]])).max() <= LOG2P_TOL
