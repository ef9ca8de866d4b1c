"""Writes the stored expected values in tests/golden/*.json.

Every expected value comes from the FP64 oracle (oracle/) and every input
from the seeded generators in synth or from literal values in this file;
nothing here calls the CUDA library.  The paper prints no worked example,
so these files are regression vectors: the CPU tests check that the oracle
still reproduces them, the GPU tests that the CUDA path matches them under
the same bars as the parity tests.  Two quantiser rows and the uniform
coder case also carry hand derivations (the "derivation" fields), which the
CPU tests check against the stored numbers.

Run from the repository root:  python tests/golden/make_golden.py
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O          # noqa: E402
from paper_2511_11337_b300 import synth  # noqa: E402

M = 1 << 16
UNIFORM_MESSAGE = b"BOA Constrictor: a Mamba predictor drives a range coder."

# (seed, n, adversarial) of synth.random_histograms cases
CODER_CASES = [(11, 1, False), (12, 17, False), (13, 300, True), (14, 1000, False), (15, 1000, True)]

# tiny model (synth.TINY, seed 1) and records streams (seed, length)
MODEL_SEED = 1
MODEL_STREAMS = [(4000, 0), (4001, 1), (4002, 2), (4003, 257), (4004, 3000)]
N_LOG2P = 24


def sha(b: bytes) -> str:
    return hashlib.sha256(b).hexdigest()


def cdfs_from(hist: np.ndarray) -> np.ndarray:
    c = np.zeros((hist.shape[0], 257), np.uint32)
    c[:, 1:] = np.cumsum(hist, axis=1)
    return c


def uniform_cdfs(n: int) -> np.ndarray:
    return np.tile((256 * np.arange(257)).astype(np.uint32), (n, 1))


def coder_golden() -> dict:
    cases = []
    for seed, n, adv in CODER_CASES:
        hist, syms = synth.random_histograms(n, seed=seed, adversarial=adv)
        c = cdfs_from(hist)
        code, _ = O.encode_cdfs(c, syms)
        cases.append({"generator": "synth.random_histograms", "seed": seed, "n": n, "adversarial": adv,
                      "inputs_sha256": sha(c.tobytes() + syms.tobytes()), "code_hex": code.hex()})
    msg = np.frombuffer(UNIFORM_MESSAGE, np.uint8)
    code, _ = O.encode_cdfs(uniform_cdfs(len(msg)), msg)
    return {
        "cite": "Section 'Range coding': 32-bit range coder over integer CDFs with total M = 2^16; the "
                "oracle's readings of the ring (L + R <= 2^32), the emission test, the straddle rule and "
                "the 4-byte flush",
        "cases": cases,
        "uniform": {
            "message": UNIFORM_MESSAGE.decode(),
            "code_hex": code.hex(),
            "derivation": "Uniform CDF C(s) = 256 s, f = 256. From L = 0, R = 2^32: r = R / 2^16 = 2^16, "
                          "L = r C(s) = s 2^24, R = r f = 2^24. L and L + R - 1 share the top byte s, so s "
                          "is emitted and L = 0, R = 2^32 again. The code is the message followed by the four "
                          "zero bytes of the flushed L.",
        },
    }


def quantise_rows() -> tuple[np.ndarray, list[str]]:
    g = np.random.Generator(np.random.PCG64(21))
    rows, notes = [], []
    for scale in (0.5, 3.0, 20.0):
        lg = g.normal(0, scale, 256)
        e = np.exp(lg - lg.max())
        rows.append((e / e.sum()).astype(np.float32))
        notes.append(f"softmax of N(0, {scale}^2) logits, rounded to float32")
    r = np.zeros(256, np.float32)
    r[:5] = [0.25, 0.25, 0.25, 0.25 - 2 ** -9, 2 ** -9]
    rows.append(r)
    notes.append("hand case A")
    r = np.zeros(256, np.float32)
    r[200:] = np.float32(1 / 56)
    rows.append(r)
    notes.append("hand case B")
    return np.stack(rows), notes


def quantise_golden() -> dict:
    p, notes = quantise_rows()
    rows = []
    for i in range(p.shape[0]):
        f = O.quantise_f32(p[i])
        rows.append({"note": notes[i], "p_f32_hex": p[i].view(np.uint32).astype(">u4").tobytes().hex(),
                     "f": [int(x) for x in f]})
    return {
        "cite": "Section 'Range coding': strictly positive integer frequencies summing to M = 2^16, read as "
                "f = 1 + floor(p (M - 256)) with the remainder to the argmax (lowest index on ties); float32 "
                "inputs",
        "rows": rows,
        "derivation": {
            "hand case A": "p = (1/4, 1/4, 1/4, 1/4 - 2^-9, 2^-9, 0, ...): p (M - 256) = 16320, 16320, 16320, "
                           "16192.5, 127.5, 0 -> f = 16321, 16321, 16321, 16193, 128 and 251 ones; the sum "
                           "65535 leaves 1 for symbol 0: f0 = 16322.",
            "hand case B": "p = float32(1/56) on symbols 200..255: p (M - 256) = 1165.71 -> f = 1166 there and 1 "
                           "on the 200 others; the sum 65496 leaves 40 for symbol 200: f200 = 1206.",
        },
    }


def model_golden() -> dict:
    with tempfile.TemporaryDirectory() as d:
        path = synth.make_model_file(os.path.join(d, "tiny.boaw"), synth.TINY, seed=MODEL_SEED)
        model_sha = sha(open(path, "rb").read())
        om = O.Model(path)
        streams = []
        for seed, n in MODEL_STREAMS:
            data = synth.records_stream(seed, n)
            code = om.compress(data)
            entry = {"seed": seed, "len": n, "data_sha256": sha(data), "code_len": len(code),
                     "code_sha256": sha(code)}
            if n > 1:
                lp = om.logprobs(data)
                k = min(N_LOG2P, n - 1)
                nxt = np.frombuffer(data, np.uint8)[1:k + 1]
                entry["log2p_next"] = [repr(float(v)) for v in lp[np.arange(k), nxt]]
                if n == max(m for _, m in MODEL_STREAMS):
                    entry["log2p_row0"] = [repr(float(v)) for v in lp[0]]
            streams.append(entry)
    shape = synth.TINY
    return {
        "cite": "Algorithm 1 and App. A (the Mamba predictor), section 'Range coding' (quantiser and "
                "coder); byte 0 of a stream stored raw, the model predicting bytes 1..n-1",
        "model": {"generator": "synth.make_model_file", "shape": {"d_model": shape.d_model,
                  "n_layer": shape.n_layer}, "seed": MODEL_SEED, "file_sha256": model_sha},
        "streams_generator": "synth.records_stream",
        "streams": streams,
    }


def main() -> None:
    for name, fn in (("coder.json", coder_golden), ("quantise.json", quantise_golden),
                     ("model_tiny.json", model_golden)):
        with open(os.path.join(HERE, name), "w") as f:
            json.dump(fn(), f, indent=1)
            f.write("\n")
        print("wrote", name)


if __name__ == "__main__":
    main()
