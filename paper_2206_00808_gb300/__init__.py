"""GB300-native spinor RPA polarizability chi0_GG'(q, i omega).

The compute path is the C-ABI library `libbgwchi.so` (CUDA, sm_103a) built
from `csrc/`; `binding` is its thin ctypes wrapper.  Importing this package
does not load the library: `from paper_2206_00808_gb300 import binding` does,
and fails loudly if the library has not been built.
"""
__all__ = ["binding", "synthetic", "build"]
