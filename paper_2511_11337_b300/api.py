"""Python API over libboa.so: names follow include/boa.h; marshalling only."""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._lib import BoaError, check, load

PREC_FP32 = 0
PREC_BF16 = 1
PREC_TF32X3 = 2
PREC_FP8 = 3


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def crc32(data: bytes) -> int:
    buf = np.frombuffer(data, np.uint8) if data else np.zeros(1, np.uint8)
    return int(load().boa_crc32(_p(buf), len(data)))


def max_compressed_size(n: int) -> int:
    return int(load().boa_max_compressed_size(n))


class _Opts(C.Structure):
    _fields_ = [("device", C.c_int), ("precision", C.c_int), ("cuda_stream", C.c_void_p), ("max_rows", C.c_size_t),
                ("max_slots", C.c_size_t)]


class _Tuning(C.Structure):
    _fields_ = [("max_rows", C.c_size_t), ("scan_variant", C.c_int), ("decode_lanes", C.c_int), ("compress_ms", C.c_double),
                ("decompress_ms", C.c_double), ("decoder", C.c_int)]


class Model:
    """A predictor loaded on the GPU (boa_load_model)."""

    def __init__(self, path: str, device: int = 0, precision: int = PREC_FP32, cuda_stream: int | None = None,
                 max_rows: int = 0, max_slots: int = 0):
        self._h = C.c_void_p()
        opts = _Opts(device, precision, cuda_stream, max_rows, max_slots)
        check(load().boa_load_model(os.fsencode(path), C.byref(opts), C.byref(self._h)))

    def close(self):
        if self._h:
            load().boa_free_model(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def fingerprint(self) -> int:
        return int(load().boa_model_fingerprint(self._h))

    def last_stream_status(self, n: int) -> np.ndarray:
        """boa_last_stream_status: per-stream flags of the last call (0 = clean)."""
        out = np.zeros(max(n, 1), np.uint32)
        check(load().boa_last_stream_status(self._h, n, _p(out)))
        return out[:n]

    @property
    def last_launch_count(self) -> int:
        return int(load().boa_last_launch_count(self._h))

    # ----------------------------------------------------------- host API
    def compress(self, streams: list[bytes]) -> list[bytes]:
        n = len(streams)
        if n == 0:
            return []
        bufs = [np.frombuffer(s, np.uint8) if len(s) else np.zeros(1, np.uint8) for s in streams]
        lens = np.array([len(s) for s in streams], np.uintp)
        caps = np.array([max_compressed_size(len(s)) for s in streams], np.uintp)
        outs = [np.empty(max(int(c), 1), np.uint8) for c in caps]      # the library writes sizes[i] bytes
        in_ptrs = np.array([b.ctypes.data for b in bufs], np.uintp)
        out_ptrs = np.array([o.ctypes.data for o in outs], np.uintp)
        sizes = np.zeros(n, np.uintp)
        check(load().boa_compress(self._h, n, _p(in_ptrs), _p(lens), _p(out_ptrs), _p(caps), _p(sizes)))
        return [o[:int(z)].tobytes() for o, z in zip(outs, sizes)]

    def decompress(self, comps: list[bytes], lens: list[int]) -> list[bytes]:
        n = len(comps)
        if n == 0:
            return []
        bufs = [np.frombuffer(c, np.uint8) if len(c) else np.zeros(1, np.uint8) for c in comps]
        sizes = np.array([len(c) for c in comps], np.uintp)
        l = np.array(lens, np.uintp)
        outs = [np.empty(max(int(x), 1), np.uint8) for x in lens]      # the library writes lens[i] bytes
        in_ptrs = np.array([b.ctypes.data for b in bufs], np.uintp)
        out_ptrs = np.array([o.ctypes.data for o in outs], np.uintp)
        check(load().boa_decompress(self._h, n, _p(in_ptrs), _p(sizes), _p(l), _p(out_ptrs)))
        return [o[:int(x)].tobytes() for o, x in zip(outs, lens)]

    # ----------------------------------------------------------- device API
    def compress_device(self, d_in_ptr: int, in_offsets: np.ndarray, d_out_ptr: int,
                        out_offsets: np.ndarray) -> np.ndarray:
        """d_in_ptr / d_out_ptr: device addresses (e.g. torch tensor data_ptr())."""
        in_offsets = np.ascontiguousarray(in_offsets, np.uint64)
        out_offsets = np.ascontiguousarray(out_offsets, np.uint64)
        n = len(in_offsets) - 1
        sizes = np.zeros(max(n, 1), np.uint64)
        check(load().boa_compress_device(self._h, n, C.c_void_p(d_in_ptr), _p(in_offsets), C.c_void_p(d_out_ptr),
                                         _p(out_offsets), _p(sizes)))
        return sizes[:n]

    def decompress_device(self, d_in_ptr: int, in_offsets: np.ndarray, lens: np.ndarray, d_out_ptr: int,
                          out_offsets: np.ndarray, in_sizes: np.ndarray | None = None) -> None:
        """in_sizes: coded bytes at the start of each input slot (None = whole slot)."""
        in_offsets = np.ascontiguousarray(in_offsets, np.uint64)
        out_offsets = np.ascontiguousarray(out_offsets, np.uint64)
        lens = np.ascontiguousarray(lens, np.uint64)
        n = len(in_offsets) - 1
        sz = None
        if in_sizes is not None:
            in_sizes = np.ascontiguousarray(in_sizes, np.uint64)
            sz = _p(in_sizes)
        check(load().boa_decompress_device(self._h, n, C.c_void_p(d_in_ptr), _p(in_offsets), sz, _p(lens),
                                           C.c_void_p(d_out_ptr), _p(out_offsets)))

    # ----------------------------------------------------------- container
    def pack(self, data: bytes, chunk_len: int = 16384) -> bytes:
        """boa_pack: one buffer -> .boa container (chunks of chunk_len bytes)."""
        cap = int(load().boa_pack_bound(len(data), chunk_len))
        out = np.zeros(max(cap, 1), np.uint8)
        buf = np.frombuffer(data, np.uint8) if data else np.zeros(1, np.uint8)
        size = C.c_size_t()
        check(load().boa_pack(self._h, _p(buf), len(data), chunk_len, _p(out), cap, C.byref(size)))
        return out[:size.value].tobytes()

    def unpack(self, container: bytes) -> bytes:
        """boa_unpack: .boa container -> original bytes."""
        buf = np.frombuffer(container, np.uint8) if container else np.zeros(1, np.uint8)
        total, fp = C.c_uint64(), C.c_uint64()
        check(load().boa_unpack_info(_p(buf), len(container), C.byref(total), C.byref(fp)))
        out = np.zeros(max(int(total.value), 1), np.uint8)
        n = C.c_size_t()
        check(load().boa_unpack(self._h, _p(buf), len(container), _p(out), int(total.value), C.byref(n)))
        return out[:n.value].tobytes()

    def unpack_shards(self, data: bytes) -> bytes:
        """boa_unpack_shards: containers laid end to end -> original bytes."""
        buf = np.frombuffer(data, np.uint8) if data else np.zeros(1, np.uint8)
        n = C.c_size_t()
        check(load().boa_unpack_shards(self._h, _p(buf), len(data), None, 0, C.byref(n)))
        out = np.zeros(max(n.value, 1), np.uint8)
        check(load().boa_unpack_shards(self._h, _p(buf), len(data), _p(out), n.value, C.byref(n)))
        return out[:n.value].tobytes()

    def autotune(self, n_streams: int, stream_len: int) -> dict:
        """boa_autotune: pick the chunk size and the decode scan kernel for this shape."""
        t = _Tuning()
        check(load().boa_autotune(self._h, n_streams, stream_len, C.byref(t)))
        return {"max_rows": int(t.max_rows), "scan_variant": int(t.scan_variant),
                "decode_lanes": int(t.decode_lanes), "decoder": int(t.decoder), "compress_ms_est": t.compress_ms,
                "decompress_ms_est": t.decompress_ms}

    # ----------------------------------------------------------- training
    @property
    def param_count(self) -> int:
        return int(load().boa_model_param_count(self._h))

    def train_step(self, batch: np.ndarray, lr: float) -> float:
        """boa_train_step on a [n_seq, seqlen] uint8 batch; returns the loss
        (bytes per byte) before the update."""
        b = np.ascontiguousarray(batch, np.uint8)
        loss = C.c_float()
        check(load().boa_train_step(self._h, _p(b), b.shape[0], b.shape[1], C.c_float(lr), C.byref(loss)))
        return float(loss.value)

    def train_grad(self, batch: np.ndarray) -> tuple[float, np.ndarray]:
        """boa_debug_train_grad: (loss, gradient in the weight file's layout)."""
        b = np.ascontiguousarray(batch, np.uint8)
        g = np.zeros(self.param_count, np.float32)
        loss = C.c_float()
        check(load().boa_debug_train_grad(self._h, _p(b), b.shape[0], b.shape[1], _p(g), C.byref(loss)))
        return float(loss.value), g

    def save(self, path: str) -> None:
        """boa_save_model: write the current weights as a weight file."""
        check(load().boa_save_model(self._h, os.fsencode(path)))

    def set_tuning(self, max_rows: int, scan_variant: int, decode_lanes: int = 0, decoder: int = 0) -> None:
        """boa_set_tuning: apply a launch configuration (results do not depend on it).
        decoder 1: the on-chip persistent decoder (FP32 form)."""
        t = _Tuning(max_rows, scan_variant, decode_lanes, 0.0, 0.0, decoder)
        check(load().boa_set_tuning(self._h, C.byref(t)))

    def tuning(self) -> dict:
        """boa_get_tuning: the configuration in use."""
        t = _Tuning()
        check(load().boa_get_tuning(self._h, C.byref(t)))
        return {"max_rows": int(t.max_rows), "scan_variant": int(t.scan_variant),
                "decode_lanes": int(t.decode_lanes), "decoder": int(t.decoder)}

    # ----------------------------------------------------------- benchmark hooks
    KERNEL_CLASSES = ["embed_ln", "gemm_in_proj", "conv_silu", "gemm_x_proj", "scan", "gemm_out_proj",
                      "gemm_ffn", "layernorm", "gemm_head", "encode", "decode", "other"]

    def profile(self, on: bool = True, decode_step_stride: int = 1) -> None:
        check(load().boa_profile_enable(self._h, int(on), int(decode_step_stride)))

    def profile_reset(self) -> None:
        check(load().boa_profile_reset(self._h))

    def profile_read(self) -> dict:
        """{phase: {class: {launches, ms, flops, bytes}}} for the timed launches."""
        out = {}
        for ph, pname in enumerate(("compress", "decompress")):
            d = {}
            for i, name in enumerate(self.KERNEL_CLASSES):
                n, ms, fl, by = C.c_uint64(), C.c_double(), C.c_double(), C.c_double()
                check(load().boa_profile_read(self._h, ph, i, C.byref(n), C.byref(ms), C.byref(fl), C.byref(by)))
                if n.value:
                    d[name] = {"launches": int(n.value), "ms": ms.value, "flops": fl.value, "bytes": by.value}
            out[pname] = d
        return out

    def profile_steps(self) -> dict:
        """{phase: (timed steps, all steps)} since the last profile_reset."""
        out = {}
        for ph, pname in enumerate(("compress", "decompress")):
            a, b = C.c_uint64(), C.c_uint64()
            check(load().boa_profile_steps(self._h, ph, C.byref(a), C.byref(b)))
            out[pname] = (int(a.value), int(b.value))
        return out

    # ----------------------------------------------------------- test hooks
    def logprobs(self, data: bytes) -> np.ndarray:
        n = len(data)
        out = np.zeros((max(n - 1, 1), 256), np.float32)
        buf = np.frombuffer(data, np.uint8) if n else np.zeros(1, np.uint8)
        check(load().boa_debug_logprobs(self._h, _p(buf), n, _p(out)))
        return out[:max(n - 1, 0)]

    def enable_cdf_trace(self, on: bool = True) -> None:
        check(load().boa_debug_enable_cdf_trace(self._h, int(on)))

    def read_cdf_trace(self, n: int) -> np.ndarray:
        out = np.zeros(max(n, 1), np.uint64)
        check(load().boa_debug_read_cdf_trace(self._h, _p(out), n))
        return out[:n]


def encode_cdfs(cdf_list: list[np.ndarray], sym_list: list[np.ndarray]) -> list[bytes]:
    """GPU range encoder fed caller CDFs ([n][257] u32 per sequence)."""
    n_seq = len(cdf_list)
    n_syms = np.array([len(s) for s in sym_list], np.uintp)
    cdfs = np.ascontiguousarray(np.concatenate([np.asarray(c, np.uint32).reshape(-1, 257) for c in cdf_list]), np.uint32)
    syms = np.ascontiguousarray(np.concatenate([np.asarray(s, np.uint8) for s in sym_list]), np.uint8)
    stride = int(5 * max(n_syms.max(initial=0), 1) + 4)
    out = np.zeros(n_seq * stride, np.uint8)
    sizes = np.zeros(n_seq, np.uintp)
    check(load().boa_debug_encode_cdfs(n_seq, _p(n_syms), _p(cdfs), _p(syms), _p(out), stride, _p(sizes)))
    return [out[i * stride:i * stride + int(sizes[i])].tobytes() for i in range(n_seq)]


def decode_cdfs(cdf_list: list[np.ndarray], coded: list[bytes]) -> list[np.ndarray]:
    n_seq = len(cdf_list)
    n_syms = np.array([np.asarray(c).reshape(-1, 257).shape[0] for c in cdf_list], np.uintp)
    cdfs = np.ascontiguousarray(np.concatenate([np.asarray(c, np.uint32).reshape(-1, 257) for c in cdf_list]), np.uint32)
    stride = max(max(len(c) for c in coded), 1)
    inb = np.zeros(n_seq * stride, np.uint8)
    for i, c in enumerate(coded):
        inb[i * stride:i * stride + len(c)] = np.frombuffer(c, np.uint8)
    in_sizes = np.array([len(c) for c in coded], np.uintp)
    syms = np.zeros(max(int(n_syms.sum()), 1), np.uint8)
    check(load().boa_debug_decode_cdfs(n_seq, _p(n_syms), _p(cdfs), _p(inb), stride, _p(in_sizes), _p(syms)))
    out, o = [], 0
    for k in n_syms:
        out.append(syms[o:o + int(k)].copy())
        o += int(k)
    return out


def decode_cdfs_static(n_syms, d_cdfs_ptr: int, d_in_ptr: int, in_stride: int, in_sizes, d_syms_ptr: int,
                       cuda_stream: int | None = None) -> None:
    """Allocation-free decoder (boa_decode_cdfs_static): device inputs and
    outputs, scratch in the library's static device array."""
    n = np.ascontiguousarray(n_syms, np.uintp)
    sz = np.ascontiguousarray(in_sizes, np.uintp)
    check(load().boa_decode_cdfs_static(len(n), _p(n), C.c_void_p(d_cdfs_ptr), C.c_void_p(d_in_ptr), in_stride,
                                        _p(sz), C.c_void_p(d_syms_ptr), C.c_void_p(cuda_stream)))


def gemm(A: np.ndarray, W: np.ndarray, bias=None, epilogue: int = 0, C_in=None, precision: int = PREC_FP32):
    """One projection GEMM on the GPU (boa_debug_gemm): epi(A . W^T)."""
    A = np.ascontiguousarray(A, np.float32); W = np.ascontiguousarray(W, np.float32)
    M, K = A.shape
    N = W.shape[0]
    out = np.zeros((M, N), np.float32)
    b = np.ascontiguousarray(bias, np.float32) if bias is not None else None
    ci = np.ascontiguousarray(C_in, np.float32) if C_in is not None else None
    check(load().boa_debug_gemm(precision, M, N, K, _p(A), _p(W), _p(b) if b is not None else None, epilogue,
                                _p(ci) if ci is not None else None, _p(out)))
    return out


def quantise(p: np.ndarray) -> np.ndarray:
    p = np.ascontiguousarray(p, np.float32).reshape(-1, 256)
    f = np.zeros_like(p, dtype=np.uint32)
    check(load().boa_debug_quantise(p.shape[0], _p(p), _p(f)))
    return f


def pack(streams: list[bytes]) -> tuple[np.ndarray, np.ndarray]:
    """Concatenate streams into one byte array plus n+1 offsets."""
    offs = np.zeros(len(streams) + 1, np.uint64)
    offs[1:] = np.cumsum([len(s) for s in streams], dtype=np.uint64)
    flat = np.frombuffer(b"".join(streams), np.uint8) if offs[-1] else np.zeros(0, np.uint8)
    return flat, offs


def slot_offsets(caps) -> np.ndarray:
    """n+1 offsets of consecutive output slots with the given capacities."""
    offs = np.zeros(len(caps) + 1, np.uint64)
    offs[1:] = np.cumsum(np.asarray(caps, np.uint64), dtype=np.uint64)
    return offs


def compressed_slot_offsets(lens) -> np.ndarray:
    return slot_offsets([max_compressed_size(int(n)) for n in lens])


__all__ = ["decode_cdfs_static", "pack", "slot_offsets", "compressed_slot_offsets", "Model", "BoaError", "encode_cdfs", "decode_cdfs", "quantise", "max_compressed_size", "PREC_FP32", "PREC_BF16", "PREC_TF32X3", "PREC_FP8", "gemm"]


class Stream:
    """boa_stream_*: the double-buffered streaming compressor.  Pushed bytes
    are cut into sets of set_chunks chunks of chunk_len bytes; each set
    becomes one container shard.  The model belongs to the pipeline until
    close()."""

    def __init__(self, model: Model, chunk_len: int = 16384, set_chunks: int = 256):
        self._model = model
        self._h = C.c_void_p()
        check(load().boa_stream_open(model._h, chunk_len, set_chunks, C.byref(self._h)))

    def push(self, data: bytes) -> None:
        buf = np.frombuffer(data, np.uint8) if data else np.zeros(1, np.uint8)
        check(load().boa_stream_push(self._h, _p(buf), len(data)))

    def finish(self) -> None:
        check(load().boa_stream_finish(self._h))

    def read(self) -> bytes:
        n = int(load().boa_stream_available(self._h))
        out = np.zeros(max(n, 1), np.uint8)
        got = C.c_size_t()
        check(load().boa_stream_read(self._h, _p(out), n, C.byref(got)))
        return out[:got.value].tobytes()

    def stats(self) -> dict:
        b, s, p = C.c_uint64(), C.c_uint64(), C.c_uint64()
        check(load().boa_stream_stats(self._h, C.byref(b), C.byref(s), C.byref(p)))
        return {"bytes_in": int(b.value), "sets": int(s.value), "preloaded": int(p.value)}

    def close(self) -> None:
        if self._h:
            load().boa_stream_close(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
