"""B300-native BOA Constrictor: batched Mamba next-byte prediction fused with
integer-CDF range coding over many independent byte streams (arXiv 2511.11337).

The compute path is libboa.so (hand-written sm_103a CUDA behind the C-ABI in
include/boa.h); this package only marshals arguments to it.  Submodules load
lazily so that `synth` (seeded inputs) imports without the CUDA library.
"""
import importlib

__all__ = ["api", "synth", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
