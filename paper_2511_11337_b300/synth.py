"""Seeded synthetic inputs and random-init weight files.

This module is the one piece shared by the CUDA path's tests/benchmark and the
CPU oracle: it draws random numbers and lays bytes out, and holds none of the
compressor's arithmetic (no model evaluation, no quantisation, no coding).

Inputs stand in for the CERN open datasets the paper evaluates on (paper,
section "Dataset"), which are not available here:

* ``records_stream``   32-byte structs (u32 counter, 5 x f32 Gaussian random
  walks sigma=0.01, 3 x u16 uniform on {0..15}, 2 zero pad bytes).
* ``atlas_table``      row-major jet table, rows of 5 x f32 [k, pT, eta, phi, m]
  with event multiplicity k ~ Poisson(6) (k=0 events skipped),
  pT = 20 + Exponential(mean 40), eta ~ N(0, 1.5^2), phi ~ U(-pi, pi),
  m ~ LogNormal(2, 0.5).
* ``cms_records``      24-byte structs (u32 run, u32 lumi, u64 event id,
  8 x u8 flags); run/lumi constant over blocks of floor(10^U(3,5)) records,
  event ids increasing by 1 + Poisson(2), each flag 0 with probability 0.95
  else U{1..255}.

Weights follow the Mamba-1 block layout (paper Alg. 1 and App. A): every
matrix, the embedding and the conv taps N(0, 0.02^2); biases 0; D = 1;
LayerNorm gamma = 1, beta = 0; A_log[c, n] = log(n + 1).
"""
from __future__ import annotations

import math
import struct
from dataclasses import dataclass

import numpy as np

MAGIC = b"BOAW"
VERSION = 1
HEADER_FMT = "<4sI8I"  # magic, version, vocab, d_model, n_layer, d_state, d_conv, expand, dt_rank, ffn_mult


@dataclass(frozen=True)
class ModelShape:
    d_model: int
    n_layer: int
    d_state: int = 16
    d_conv: int = 4
    expand: int = 2
    ffn_mult: int = 0
    vocab: int = 256

    @property
    def d_inner(self) -> int:
        return self.expand * self.d_model

    @property
    def dt_rank(self) -> int:
        return math.ceil(self.d_model / 16)


# Model shapes used by the workloads.
TINY = ModelShape(d_model=64, n_layer=2)             # 64 KB records workload
PAPER_SCALE = ModelShape(d_model=256, n_layer=3)     # 64 MB jet-table workload
PAPER_SHAPE_FFN = ModelShape(d_model=256, n_layer=1, ffn_mult=4)  # d_m=256, n_l=1 with FFN


def tensor_specs(shape: ModelShape):
    """(name, dims) in file order.  Both readers (library and oracle) parse
    this order independently; it is the weight file format."""
    d, E, N, K, r = shape.d_model, shape.d_inner, shape.d_state, shape.d_conv, shape.dt_rank
    F = shape.ffn_mult * d
    specs = [("embed", (shape.vocab, d))]
    for l in range(shape.n_layer):
        p = f"layers.{l}."
        specs += [
            (p + "ln_a.w", (d,)), (p + "ln_a.b", (d,)),
            (p + "in_proj.w", (2 * E, d)),
            (p + "conv.w", (E, K)), (p + "conv.b", (E,)),
            (p + "x_proj.w", (r + 2 * N, E)),
            (p + "dt_proj.w", (E, r)), (p + "dt_proj.b", (E,)),
            (p + "A_log", (E, N)),
            (p + "D", (E,)),
            (p + "out_proj.w", (d, E)),
        ]
        if F:
            specs += [(p + "ffn.w1", (F, d)), (p + "ffn.b1", (F,)),
                      (p + "ffn.w2", (d, F)), (p + "ffn.b2", (d,))]
        specs += [(p + "ln_b.w", (d,)), (p + "ln_b.b", (d,))]
    specs += [("head.w", (shape.vocab, d)), ("head.b", (shape.vocab,))]
    return specs


def init_weights(shape: ModelShape, seed: int, head_scale: float = 1.0,
                 zero_head: bool = False) -> dict[str, np.ndarray]:
    """Random-init weights as float32 arrays.

    head_scale multiplies the head matrix (a "peaked" stress model sharpens the
    next-byte distribution); zero_head zeroes head weight and bias, which makes
    every prediction exactly uniform.
    """
    g = np.random.Generator(np.random.PCG64(seed))
    out = {}
    for name, dims in tensor_specs(shape):
        leaf = name.split(".", 2)[-1] if name.startswith("layers.") else name
        if leaf in ("ln_a.w", "ln_b.w", "D"):
            a = np.ones(dims, np.float32)
        elif leaf in ("ln_a.b", "ln_b.b", "conv.b", "dt_proj.b", "ffn.b1", "ffn.b2", "head.b"):
            a = np.zeros(dims, np.float32)
        elif leaf == "A_log":
            a = np.tile(np.log(np.arange(1, dims[1] + 1, dtype=np.float64)), (dims[0], 1)).astype(np.float32)
        else:
            a = g.normal(0.0, 0.02, size=dims).astype(np.float32)
        out[name] = a
    out["head.w"] = (out["head.w"] * np.float32(head_scale)).astype(np.float32)
    if zero_head:
        out["head.w"][:] = 0
        out["head.b"][:] = 0
    return out


def write_model(path: str, shape: ModelShape, weights: dict[str, np.ndarray]) -> None:
    hdr = struct.pack(HEADER_FMT, MAGIC, VERSION, shape.vocab, shape.d_model, shape.n_layer,
                      shape.d_state, shape.d_conv, shape.expand, shape.dt_rank, shape.ffn_mult)
    with open(path, "wb") as f:
        f.write(hdr)
        for name, dims in tensor_specs(shape):
            a = np.ascontiguousarray(weights[name], dtype="<f4")
            assert a.shape == tuple(dims), (name, a.shape, dims)
            f.write(a.tobytes())


def read_model(path: str) -> tuple[ModelShape, dict[str, np.ndarray]]:
    with open(path, "rb") as f:
        buf = f.read()
    magic, ver, vocab, d, nl, N, K, ex, r, ffn = struct.unpack_from(HEADER_FMT, buf, 0)
    assert magic == MAGIC and ver == VERSION
    shape = ModelShape(d_model=d, n_layer=nl, d_state=N, d_conv=K, expand=ex, ffn_mult=ffn, vocab=vocab)
    assert shape.dt_rank == r
    off = struct.calcsize(HEADER_FMT)
    w = {}
    for name, dims in tensor_specs(shape):
        n = int(np.prod(dims))
        w[name] = np.frombuffer(buf, "<f4", n, off).reshape(dims).copy()
        off += 4 * n
    assert off == len(buf)
    return shape, w


def make_model_file(path: str, shape: ModelShape, seed: int = 0, **kw) -> str:
    write_model(path, shape, init_weights(shape, seed, **kw))
    return path


# ----------------------------------------------------------------- byte data

def records_stream(seed: int, n_bytes: int = 16384) -> bytes:
    """32-byte records: u32 counter, 5 x f32 random walks, 3 x u16 in {0..15}, 2 pad bytes."""
    g = np.random.Generator(np.random.PCG64(seed))
    n_rec = -(-n_bytes // 32)
    rec = np.zeros(n_rec, dtype=[("cnt", "<u4"), ("walk", "<f4", (5,)), ("u", "<u2", (3,)), ("pad", "u1", (2,))])
    assert rec.dtype.itemsize == 32
    rec["cnt"] = np.arange(n_rec, dtype=np.uint32)
    rec["walk"] = np.cumsum(g.normal(0.0, 0.01, size=(n_rec, 5)), axis=0).astype(np.float32)
    rec["u"] = g.integers(0, 16, size=(n_rec, 3), dtype=np.uint16)
    return rec.tobytes()[:n_bytes]


def records_workload(n_streams: int = 4, stream_len: int = 16384, seed_base: int = 1000) -> list[bytes]:
    """4 x 16 KB records streams (seed 1000 + i): the 64 KB tiny workload."""
    return [records_stream(seed_base + i, stream_len) for i in range(n_streams)]


def atlas_table(n_bytes: int, seed: int) -> bytes:
    """Row-major jet table of 5 x f32 rows [k, pT, eta, phi, m]."""
    g = np.random.Generator(np.random.PCG64(seed))
    n_rows = -(-n_bytes // 20)
    ks = []
    tot = 0
    while tot < n_rows:
        k = g.poisson(6.0, size=max(1024, (n_rows - tot) // 5))
        k = k[k > 0]
        ks.append(k)
        tot += int(k.sum())
    k = np.concatenate(ks)
    kk = np.repeat(k, k)[:n_rows].astype(np.float32)
    rows = np.empty((n_rows, 5), np.float32)
    rows[:, 0] = kk
    rows[:, 1] = 20.0 + g.exponential(40.0, n_rows)
    rows[:, 2] = g.normal(0.0, 1.5, n_rows)
    rows[:, 3] = g.uniform(-math.pi, math.pi, n_rows)
    rows[:, 4] = g.lognormal(2.0, 0.5, n_rows)
    return rows.astype("<f4").tobytes()[:n_bytes]


def atlas_workload(n_streams: int = 4096, stream_len: int = 16384, seed: int = 2000) -> bytes:
    """One contiguous buffer of n_streams * stream_len bytes (64 MiB default),
    split by the caller into equal contiguous chunks."""
    return atlas_table(n_streams * stream_len, seed)


def cms_records(n_bytes: int, seed: int) -> bytes:
    g = np.random.Generator(np.random.PCG64(seed))
    n_rec = -(-n_bytes // 24)
    rec = np.zeros(n_rec, dtype=[("run", "<u4"), ("lumi", "<u4"), ("event", "<u8"), ("flags", "u1", (8,))])
    assert rec.dtype.itemsize == 24

    def blocks(base):
        vals = np.empty(n_rec, np.uint32)
        i, v = 0, base
        while i < n_rec:
            blen = int(10 ** g.uniform(3, 5))
            vals[i:i + blen] = v
            i += blen
            v += 1
        return vals

    rec["run"] = blocks(int(g.integers(100000, 400000)))
    rec["lumi"] = blocks(1)
    rec["event"] = np.uint64(g.integers(0, 1 << 32)) + np.cumsum(1 + g.poisson(2.0, n_rec)).astype(np.uint64)
    flags = g.integers(1, 256, size=(n_rec, 8)).astype(np.uint8)
    flags[g.random((n_rec, 8)) < 0.95] = 0
    rec["flags"] = flags
    return rec.tobytes()[:n_bytes]


def mixed_lengths(n_streams: int, seed: int, lo_log2: float = 10.0, hi_log2: float = 20.0) -> np.ndarray:
    g = np.random.Generator(np.random.PCG64(seed))
    return np.floor(2.0 ** g.uniform(lo_log2, hi_log2, n_streams)).astype(np.int64)


def mixed_workload(n_streams: int = 20000, seed: int = 3000, lo_log2: float = 10.0,
                   hi_log2: float = 20.0) -> list[bytes]:
    """Uneven streams (log-uniform lengths), each ATLAS-like or CMS-like with probability 1/2."""
    lens = mixed_lengths(n_streams, seed, lo_log2, hi_log2)
    g = np.random.Generator(np.random.PCG64(seed + 1))
    kinds = g.random(n_streams) < 0.5
    out = []
    for i, (n, atlas) in enumerate(zip(lens, kinds)):
        out.append(atlas_table(int(n), seed * 100 + i) if atlas else cms_records(int(n), seed * 100 + i))
    return out


def split_equal(buf: bytes, n_streams: int) -> list[bytes]:
    step = len(buf) // n_streams
    return [buf[i * step:(i + 1) * step] for i in range(n_streams)]


def random_histograms(n: int, seed: int, adversarial: bool = False) -> tuple[np.ndarray, np.ndarray]:
    """Random strictly positive integer histograms f[n, 256] with each row
    summing to 2^16, plus one symbol drawn per row.  With adversarial=True
    most rows put almost all mass on one symbol and leave f = 1 on the rest,
    and half of those rows draw an f = 1 symbol, which drives a range coder
    into its straddle (underflow) case."""
    g = np.random.Generator(np.random.PCG64(seed))
    M = 1 << 16
    hist = np.zeros((n, 256), np.uint32)
    syms = np.zeros(n, np.uint8)
    for i in range(n):
        if adversarial and g.random() < 0.8:
            f = np.ones(256, np.int64)
            big = int(g.integers(0, 256))
            f[big] = M - 255
            s = big if g.random() < 0.5 else int(g.integers(0, 256))
        else:
            w = g.random(256) ** 4
            f = 1 + np.floor(w / w.sum() * (M - 256)).astype(np.int64)
            f[int(g.integers(0, 256))] += M - int(f.sum())
            s = int(g.choice(256, p=f / M))
        hist[i] = f
        syms[i] = s
    return hist, syms
