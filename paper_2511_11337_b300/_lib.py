"""ctypes loader for libboa.so (argument marshalling only).

The library is the product: there is no Python or CPU fallback.  If the
shared object is missing or no GPU is usable, calls fail loudly.
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(_PKG, "libboa.so")

# Every symbol include/boa.h declares, with its ctypes signature.
vp, sz, u64, i32 = C.c_void_p, C.c_size_t, C.c_uint64, C.c_int
SIGNATURES = {
    "boa_load_model": (i32, [C.c_char_p, vp, C.POINTER(vp)]),
    "boa_free_model": (None, [vp]),
    "boa_model_fingerprint": (u64, [vp]),
    "boa_max_compressed_size": (sz, [sz]),
    "boa_compress": (i32, [vp, sz, vp, vp, vp, vp, vp]),
    "boa_decompress": (i32, [vp, sz, vp, vp, vp, vp]),
    "boa_compress_device": (i32, [vp, sz, vp, vp, vp, vp, vp]),
    "boa_decompress_device": (i32, [vp, sz, vp, vp, vp, vp, vp, vp]),
    "boa_last_launch_count": (u64, [vp]),
    "boa_last_stream_status": (i32, [vp, sz, vp]),
    "boa_last_error": (C.c_char_p, []),
    "boa_train_step": (i32, [vp, vp, sz, sz, C.c_float, vp]),
    "boa_save_model": (i32, [vp, C.c_char_p]),
    "boa_model_param_count": (sz, [vp]),
    "boa_debug_train_grad": (i32, [vp, vp, sz, sz, vp, vp]),
    "boa_autotune": (i32, [vp, sz, sz, vp]),
    "boa_set_tuning": (i32, [vp, vp]),
    "boa_get_tuning": (i32, [vp, vp]),
    "boa_pack_bound": (sz, [sz, sz]),
    "boa_pack": (i32, [vp, vp, sz, sz, vp, sz, C.POINTER(sz)]),
    "boa_unpack_info": (i32, [vp, sz, C.POINTER(u64), C.POINTER(u64)]),
    "boa_unpack": (i32, [vp, vp, sz, vp, sz, C.POINTER(sz)]),
    "boa_crc32": (C.c_uint32, [vp, sz]),
    "boa_unpack_shards": (i32, [vp, vp, sz, vp, sz, C.POINTER(sz)]),
    "boa_stream_open": (i32, [vp, sz, sz, C.POINTER(vp)]),
    "boa_stream_push": (i32, [vp, vp, sz]),
    "boa_stream_finish": (i32, [vp]),
    "boa_stream_available": (sz, [vp]),
    "boa_stream_read": (i32, [vp, vp, sz, C.POINTER(sz)]),
    "boa_stream_stats": (i32, [vp, C.POINTER(u64), C.POINTER(u64), C.POINTER(u64)]),
    "boa_stream_close": (None, [vp]),
    "boa_scan_train_fwd": (i32, [sz, sz, sz, sz, sz] + [vp] * 9),
    "boa_scan_train_bwd": (i32, [sz, sz, sz, sz, sz] + [vp] * 16),
    "boa_profile_enable": (i32, [vp, i32, i32]),
    "boa_profile_reset": (i32, [vp]),
    "boa_profile_read": (i32, [vp, i32, i32, vp, vp, vp, vp]),
    "boa_profile_steps": (i32, [vp, i32, vp, vp]),
    "boa_debug_encode_cdfs": (i32, [sz, vp, vp, vp, vp, sz, vp]),
    "boa_debug_decode_cdfs": (i32, [sz, vp, vp, vp, sz, vp, vp]),
    "boa_debug_quantise": (i32, [sz, vp, vp]),
    "boa_debug_gemm": (i32, [i32, sz, sz, sz, vp, vp, vp, i32, vp, vp]),
    "boa_debug_logprobs": (i32, [vp, vp, sz, vp]),
    "boa_debug_enable_cdf_trace": (i32, [vp, i32]),
    "boa_debug_read_cdf_trace": (i32, [vp, vp, sz]),
    "boa_decode_cdfs_static": (i32, [sz, vp, vp, vp, sz, vp, vp, vp]),
    "boa_microbench": (i32, [i32, i32, i32, i32, i32, i32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
}

STATUS = {0: "BOA_OK", 1: "BOA_ERR_ARG", 2: "BOA_ERR_IO", 3: "BOA_ERR_FORMAT", 4: "BOA_ERR_CUDA",
          5: "BOA_ERR_OOM", 6: "BOA_ERR_OUTPUT_TOO_SMALL", 7: "BOA_ERR_CORRUPT", 8: "BOA_ERR_FINGERPRINT"}

_lib = None


class BoaError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def load() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(SO_PATH):
            raise ImportError(f"libboa.so is not built ({SO_PATH}); run paper_2511_11337_b300.build.build()")
        lib = C.CDLL(SO_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(code: int) -> None:
    if code != 0:
        raise BoaError(code, load().boa_last_error().decode(errors="replace"))
