"""Pins for the oracle's quantiser and range coder (CPU only).

The paper prints no worked example, so the coder is pinned by:
* a closed form: a uniform model (f = 256 everywhere, paper "Probabilities and
  integer CDF" with p = 1/256) must emit each symbol as its own byte, then the
  4-byte flush, i.e. exactly 8 bits per symbol plus 32 bits;
* information bounds on the code length (no code beats -log2 prod f/M; the
  truncating coder loses at most a bounded amount per symbol and per straddle);
* a brute-force decoder that decodes by trial encoding (uses only the encoder
  and a membership test, never the decoder's division and search), which pins
  the decoder's target formula x = floor(((C - L + 1) M - 1) / R);
* round trips on adversarial histograms that force the straddle rule.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_11337_b300 import synth

M = 1 << 16


def cdfs_from(hist):
    c = np.zeros((hist.shape[0], 257), np.uint32)
    c[:, 1:] = np.cumsum(hist, axis=1)
    return c


# ------------------------------------------------------------- quantiser

def test_quantise_uniform_is_256_each():
    f = O.quantise(np.full(256, 1 / 256))
    assert (f == 256).all()


def test_quantise_one_hot():
    p = np.zeros(256); p[7] = 1.0
    f = O.quantise(p)
    assert f[7] == 1 + (M - 256) and (np.delete(f, 7) == 1).all() and f.sum() == M


def test_quantise_hand_cases():
    # p = [1/2, 1/4, 1/8, 1/8, 0, ...]: floors are exact, remainder 0.
    p = np.zeros(256); p[:4] = [0.5, 0.25, 0.125, 0.125]
    f = O.quantise(p)
    assert list(f[:4]) == [32641, 16321, 8161, 8161] and (f[4:] == 1).all()
    # p = [3/4, 1/4 - 2^-10, 2^-10, 0 ...]: floors 48960, 16256, 63 -> sum 65535,
    # the remainder 1 goes to the most probable symbol.
    p = np.zeros(256); p[:3] = [0.75, 0.25 - 2 ** -10, 2 ** -10]
    f = O.quantise(p)
    assert list(f[:3]) == [48962, 16257, 64] and (f[3:] == 1).all()
    # ties for the most probable symbol go to the lowest index.
    p = np.zeros(256); p[:5] = [0.25, 0.25, 0.25, 0.25 - 2 ** -9, 2 ** -9]
    f = O.quantise(p)
    assert list(f[:5]) == [16322, 16321, 16321, 16193, 128]


def test_quantise_f32_matches_f64_on_exact_cases():
    for vals in ([0.5, 0.25, 0.125, 0.125], [0.75, 0.25 - 2 ** -10, 2 ** -10]):
        p = np.zeros(256); p[:len(vals)] = vals
        assert (O.quantise(p) == O.quantise_f32(p.astype(np.float32))).all()


def test_quantise_invariants_random():
    g = np.random.default_rng(0)
    for _ in range(200):
        l = g.normal(0, g.uniform(0.1, 30), 256)
        p = np.exp(l - l.max()); p /= p.sum()
        for f in (O.quantise(p), O.quantise_f32(p.astype(np.float32))):
            assert f.min() >= 1 and int(f.sum()) == M
        c = O.cdf_from_hist(O.quantise(p))
        assert c[0] == 0 and c[256] == M and (np.diff(c.astype(np.int64)) >= 1).all()


# ------------------------------------------------------------- coder

def test_uniform_closed_form():
    g = np.random.default_rng(1)
    syms = g.integers(0, 256, 1000).astype(np.uint8)
    cdfs = np.tile((256 * np.arange(257)).astype(np.uint32), (len(syms), 1))
    out, stra = O.encode_cdfs(cdfs, syms)
    assert out == syms.tobytes() + b"\0\0\0\0"
    assert stra == 0


def _ideal_bits(hist, syms):
    return -sum(math.log2(int(hist[t, s]) / M) for t, s in enumerate(syms))


@pytest.mark.parametrize("adversarial", [False, True])
def test_code_length_bounds(adversarial):
    hist, syms = synth.random_histograms(3000, seed=11 + adversarial, adversarial=adversarial)
    out, stra = O.encode_cdfs(cdfs_from(hist), syms)
    bits = 8 * len(out)
    ideal = _ideal_bits(hist, syms)
    # Lower bound: the final interval is no wider than prod(f/M) * 2^32 and the
    # flush writes 32 bits below the last emitted byte.
    assert bits >= ideal
    # Upper bound: each truncation floor(R f / M) with R >= 2^16 before the
    # update costs at most log2(1 + M/(R f)) <= 1 bit; each straddle costs at
    # most 16 bits; the flush adds 32 bits; byte granularity adds < 8 bits.
    assert bits <= ideal + len(syms) * 1.0 + 16 * stra + 32 + 8
    if adversarial:
        assert stra > 0     # the straddle rule was exercised


@pytest.mark.parametrize("adversarial", [False, True])
def test_round_trip_random_histograms(adversarial):
    hist, syms = synth.random_histograms(5000, seed=21 + adversarial, adversarial=adversarial)
    cdfs = cdfs_from(hist)
    out, _ = O.encode_cdfs(cdfs, syms)
    dec, ok = O.decode_cdfs(cdfs, out, len(syms))
    assert ok and (dec == syms).all()


def _dyadic_hist():
    """Powers of two in decreasing order: 2^15 .. 2^8, eight 2s, 240 1s (sum 2^16).
    Every C(a) is a multiple of f(a), so with R a power of two every floor in
    the update is exact and every interval stays aligned to its width."""
    f = [1 << k for k in range(15, 7, -1)] + [2] * 8 + [1] * 240
    assert len(f) == 256 and sum(f) == M
    return np.array(f, np.uint32)


def test_dyadic_equals_exact_arithmetic_coding():
    """With dyadic histograms the truncating coder is exact, so its output read
    as a base-256 fraction must equal the textbook arithmetic-coding low end
    sum_t C_t(s_t)/M * prod_{q<t} f_q(s_q)/M, computed in exact rationals."""
    from fractions import Fraction
    f = _dyadic_hist()
    c = O.cdf_from_hist(f)
    g = np.random.default_rng(5)
    for n in (1, 2, 7, 50, 400):
        syms = g.choice(256, size=n, p=f / M).astype(np.uint8)
        out, stra = O.encode_cdfs(np.tile(c, (n, 1)), syms)
        assert stra == 0
        low, width = Fraction(0), Fraction(1)
        for s in syms:
            low += width * Fraction(int(c[s]), M)
            width *= Fraction(int(f[s]), M)
        V = Fraction(int.from_bytes(out, "big"), 256 ** len(out))
        assert V == low
        # A byte leaves as soon as 8 bits of it are fixed (R <= 2^24), so the
        # length is the whole bytes of the (integer) ideal length plus the flush.
        ideal_bits = sum(16 - int(f[s]).bit_length() + 1 for s in syms)
        assert len(out) == ideal_bits // 8 + 4


def test_truncated_stream_is_flagged():
    hist, syms = synth.random_histograms(500, seed=41)
    cdfs = cdfs_from(hist)
    out, _ = O.encode_cdfs(cdfs, syms)
    _, ok = O.decode_cdfs(cdfs, out[:-7], len(syms))
    assert not ok
    _, ok = O.decode_cdfs(cdfs, out + b"\x00", len(syms))
    assert not ok


# ------------------------------------------------------------- whole method

def test_uniform_model_closed_form(uniform_model_path):
    """A zero head gives p = 1/256 exactly, so compressing n bytes yields the
    raw first byte, the remaining n-1 bytes unchanged, then 4 zero bytes."""
    m = O.Model(uniform_model_path)
    data = synth.records_stream(7, 300)
    assert m.compress(data) == data + b"\0\0\0\0"
    assert m.compress(data[:1]) == data[:1]
    assert m.compress(b"") == b""


@pytest.mark.parametrize("which", ["tiny", "peaked"])
def test_stream_round_trip(which, tiny_model_path, peaked_model_path):
    m = O.Model(tiny_model_path if which == "tiny" else peaked_model_path)
    for n in (0, 1, 2, 3, 200):
        data = synth.records_stream(100 + n, n) if n else b""
        comp = m.compress(data)
        assert len(comp) <= O.max_compressed_size(n)
        dec, ok = m.decompress(comp, n)
        assert ok and dec == data


def test_compress_matches_cdf_encoding(tiny_model_path):
    """compress == [raw byte] + encode(teacher-forced CDFs, bytes 1..n-1)."""
    m = O.Model(tiny_model_path)
    data = synth.records_stream(9, 150)
    cd = m.cdfs(data)
    coded, _ = O.encode_cdfs(cd, np.frombuffer(data, np.uint8)[1:])
    assert m.compress(data) == data[:1] + coded


def test_batch_matches_single(tiny_model_path):
    m = O.Model(tiny_model_path)
    streams = [synth.records_stream(50 + i, 64 + 13 * i) for i in range(5)]
    assert m.compress_batch(streams, n_threads=2) == [m.compress(s) for s in streams]
