"""ctypes binding of the FP64 oracle (test infrastructure only).

Each function wraps one entry of boa_oracle.c; see that file for the paper
passages each one follows and the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        L = _lib
        vp, sz, i32 = C.c_void_p, C.c_size_t, C.c_int
        L.orc_model_load.argtypes = [C.c_char_p, C.POINTER(vp)]
        L.orc_model_free.argtypes = [vp]
        L.orc_model_dims.argtypes = [vp, vp]
        L.orc_state_new.argtypes = [vp]; L.orc_state_new.restype = vp
        L.orc_state_free.argtypes = [vp]
        L.orc_step.argtypes = [vp, vp, i32, vp]
        L.orc_layernorm.argtypes = [i32, vp, vp, vp, vp]
        L.orc_softmax.argtypes = [vp, vp]
        L.orc_log2_softmax.argtypes = [vp, vp]
        L.orc_selective_scan.argtypes = [i32, i32, i32, vp, vp, vp, vp, vp, vp, vp]
        L.orc_causal_conv.argtypes = [i32, i32, i32, vp, vp, vp, vp]
        L.orc_selective_scan_grad.argtypes = [i32, i32, i32] + [vp] * 13
        L.orc_quantise.argtypes = [vp, vp]
        L.orc_quantise_f32.argtypes = [vp, vp]
        L.orc_cdf_from_hist.argtypes = [vp, vp]
        L.orc_coded_bound.argtypes = [sz]; L.orc_coded_bound.restype = sz
        L.orc_encode_cdfs.argtypes = [sz, vp, vp, vp, sz, C.POINTER(sz), C.POINTER(C.c_uint64)]
        L.orc_decode_cdfs.argtypes = [sz, vp, vp, sz, vp]
        L.orc_max_compressed_size.argtypes = [sz]; L.orc_max_compressed_size.restype = sz
        L.orc_compress_stream.argtypes = [vp, vp, sz, vp, sz, C.POINTER(sz)]
        L.orc_decompress_stream.argtypes = [vp, vp, sz, sz, vp]
        L.orc_logprobs.argtypes = [vp, vp, sz, vp]
        L.orc_cdfs.argtypes = [vp, vp, sz, vp]
        L.orc_compress_batch.argtypes = [vp, sz, vp, vp, vp, vp, vp, i32]
        L.orc_decompress_batch.argtypes = [vp, sz, vp, vp, vp, vp, i32]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Model:
    """An oracle model loaded from a weight file (FP64 copy of the FP32 weights)."""

    def __init__(self, path: str):
        self.h = C.c_void_p()
        rc = lib().orc_model_load(os.fsencode(path), C.byref(self.h))
        if rc != 0:
            raise RuntimeError(f"oracle could not load {path} (code {rc})")
        dims = np.zeros(8, np.int32)
        lib().orc_model_dims(self.h, _p(dims))
        self.vocab, self.d, self.nl, self.N, self.K, self.E, self.r, self.ffn_mult = map(int, dims)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_model_free(self.h)
            self.h = None

    # -- per-step access
    def new_state(self):
        return _State(self)

    # -- whole-stream
    def logprobs(self, data: bytes) -> np.ndarray:
        n = len(data)
        out = np.zeros((max(n - 1, 0), 256), np.float64)
        if n >= 2:
            buf = np.frombuffer(data, np.uint8).copy()
            lib().orc_logprobs(self.h, _p(buf), n, _p(out))
        return out

    def cdfs(self, data: bytes) -> np.ndarray:
        n = len(data)
        out = np.zeros((max(n - 1, 0), 257), np.uint32)
        if n >= 2:
            buf = np.frombuffer(data, np.uint8).copy()
            lib().orc_cdfs(self.h, _p(buf), n, _p(out))
        return out

    def compress(self, data: bytes) -> bytes:
        n = len(data)
        cap = lib().orc_max_compressed_size(n)
        out = np.zeros(max(cap, 1), np.uint8)
        size = C.c_size_t()
        buf = np.frombuffer(data, np.uint8).copy() if n else np.zeros(1, np.uint8)
        rc = lib().orc_compress_stream(self.h, _p(buf), n, _p(out), cap, C.byref(size))
        if rc:
            raise RuntimeError("oracle compress overflow")
        return out[:size.value].tobytes()

    def decompress(self, comp: bytes, length: int) -> tuple[bytes, bool]:
        out = np.zeros(max(length, 1), np.uint8)
        buf = np.frombuffer(comp, np.uint8).copy() if comp else np.zeros(1, np.uint8)
        rc = lib().orc_decompress_stream(self.h, _p(buf), len(comp), length, _p(out))
        return out[:length].tobytes(), rc == 0

    def compress_batch(self, streams: list[bytes], n_threads: int = 0) -> list[bytes]:
        n = len(streams)
        ins = [np.frombuffer(s, np.uint8).copy() if len(s) else np.zeros(1, np.uint8) for s in streams]
        lens = np.array([len(s) for s in streams], np.uint64)
        caps = np.array([lib().orc_max_compressed_size(len(s)) for s in streams], np.uint64)
        outs = [np.zeros(max(int(c), 1), np.uint8) for c in caps]
        in_ptrs = np.array([a.ctypes.data for a in ins], np.uint64)
        out_ptrs = np.array([a.ctypes.data for a in outs], np.uint64)
        sizes = np.zeros(n, np.uint64)
        rc = lib().orc_compress_batch(self.h, n, _p(in_ptrs), _p(lens), _p(out_ptrs), _p(caps), _p(sizes), n_threads)
        if rc:
            raise RuntimeError("oracle batch compress overflow")
        return [o[:int(z)].tobytes() for o, z in zip(outs, sizes)]


    def decompress_batch(self, comps: list[bytes], lens: list[int], n_threads: int = 0) -> tuple[list[bytes], bool]:
        n = len(comps)
        ins = [np.frombuffer(c, np.uint8).copy() if len(c) else np.zeros(1, np.uint8) for c in comps]
        sizes = np.array([len(c) for c in comps], np.uint64)
        l = np.array(lens, np.uint64)
        outs = [np.zeros(max(int(x), 1), np.uint8) for x in lens]
        in_ptrs = np.array([a.ctypes.data for a in ins], np.uint64)
        out_ptrs = np.array([a.ctypes.data for a in outs], np.uint64)
        rc = lib().orc_decompress_batch(self.h, n, _p(in_ptrs), _p(sizes), _p(l), _p(out_ptrs), n_threads)
        return [o[:int(x)].tobytes() for o, x in zip(outs, lens)], rc == 0


class _State:
    def __init__(self, model: Model):
        self.model = model
        self.h = lib().orc_state_new(model.h)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_state_free(self.h)
            self.h = None

    def step(self, byte: int) -> np.ndarray:
        out = np.zeros(256, np.float64)
        lib().orc_step(self.model.h, self.h, int(byte), _p(out))
        return out


# ----------------------------------------------------------- building blocks

def layernorm(x, g, b):
    x, g, b = _f64(x), _f64(g), _f64(b)
    y = np.zeros_like(x)
    lib().orc_layernorm(x.shape[0], _p(x), _p(g), _p(b), _p(y))
    return y


def softmax(logits):
    l = _f64(logits); p = np.zeros(256)
    lib().orc_softmax(_p(l), _p(p))
    return p


def log2_softmax(logits):
    l = _f64(logits); p = np.zeros(256)
    lib().orc_log2_softmax(_p(l), _p(p))
    return p


def selective_scan(u, delta, A, B, Cm, D):
    """u, delta: [T, E]; A: [E, N]; B, C: [T, N]; D: [E] -> y [T, E] (h_0 = 0)."""
    u, delta, A, B, Cm, D = map(_f64, (u, delta, A, B, Cm, D))
    T, E = u.shape
    N = A.shape[1]
    y = np.zeros((T, E))
    lib().orc_selective_scan(T, E, N, _p(u), _p(delta), _p(A), _p(B), _p(Cm), _p(D), _p(y))
    return y


def selective_scan_grad(u, delta, A, B, Cm, D, dy):
    """Gradients of sum(dy * scan(...)) wrt u, delta, A, B, C, D."""
    u, delta, A, B, Cm, D, dy = map(_f64, (u, delta, A, B, Cm, D, dy))
    T, E = u.shape
    N = A.shape[1]
    out = [np.zeros((T, E)), np.zeros((T, E)), np.zeros((E, N)), np.zeros((T, N)), np.zeros((T, N)), np.zeros(E)]
    lib().orc_selective_scan_grad(T, E, N, _p(u), _p(delta), _p(A), _p(B), _p(Cm), _p(D), _p(dy), *[_p(o) for o in out])
    return dict(zip(["u", "delta", "A", "B", "C", "D"], out))


def causal_conv(x, w, b):
    """x: [T, E]; w: [E, K]; b: [E] -> [T, E] (zero history, no activation)."""
    x, w, b = _f64(x), _f64(w), _f64(b)
    T, E = x.shape
    K = w.shape[1]
    out = np.zeros((T, E))
    lib().orc_causal_conv(T, E, K, _p(x), _p(w), _p(b), _p(out))
    return out


def quantise(p) -> np.ndarray:
    p = _f64(p); f = np.zeros(256, np.uint32)
    lib().orc_quantise(_p(p), _p(f))
    return f


def quantise_f32(p) -> np.ndarray:
    p = np.ascontiguousarray(p, np.float32); f = np.zeros(256, np.uint32)
    lib().orc_quantise_f32(_p(p), _p(f))
    return f


def cdf_from_hist(f) -> np.ndarray:
    f = np.ascontiguousarray(f, np.uint32); c = np.zeros(257, np.uint32)
    lib().orc_cdf_from_hist(_p(f), _p(c))
    return c


def encode_cdfs(cdfs: np.ndarray, syms: np.ndarray) -> tuple[bytes, int]:
    cdfs = np.ascontiguousarray(cdfs, np.uint32)
    syms = np.ascontiguousarray(syms, np.uint8)
    n = len(syms)
    cap = lib().orc_coded_bound(n)
    out = np.zeros(cap, np.uint8)
    size = C.c_size_t(); stra = C.c_uint64()
    rc = lib().orc_encode_cdfs(n, _p(cdfs), _p(syms), _p(out), cap, C.byref(size), C.byref(stra))
    if rc:
        raise RuntimeError("oracle encoder overflow")
    return out[:size.value].tobytes(), int(stra.value)


def decode_cdfs(cdfs: np.ndarray, data: bytes, n: int) -> tuple[np.ndarray, bool]:
    cdfs = np.ascontiguousarray(cdfs, np.uint32)
    buf = np.frombuffer(data, np.uint8).copy() if data else np.zeros(1, np.uint8)
    syms = np.zeros(max(n, 1), np.uint8)
    rc = lib().orc_decode_cdfs(n, _p(cdfs), _p(buf), len(data), _p(syms))
    return syms[:n], rc == 0


def max_compressed_size(n: int) -> int:
    return int(lib().orc_max_compressed_size(n))
