"""GB300-native blocked GEMM, C := beta*C + alpha*A*B, after the family of blocked
algorithms of "Automatic Generators for a Family of Matrix Multiplication
Routines with Apache TVM" (Alaejos et al.).

The compute lives in libg3gemm.so (CUDA for sm_103a, C ABI in include/g3gemm.h);
``_lib`` is its ctypes binding and ``torch_api`` a convenience layer that takes
torch CUDA tensors.  ``synth`` holds the seeded input generators.
Importing the package loads nothing; the library is loaded on first use.
"""
from ._lib import (G3_BF16, G3_F32, G3_F32_3XBF16, G3_FP16, G3_FP8_E4M3, G3_INT8, G3_TF32, DTYPES,  # noqa: F401
                   G3_F32_3XTF32, G3_F64, G3_INT16, G3_SPLIT_STREAM_K, G3Error, load)


def build(force: bool = False, verbose: bool = False) -> str:
    from . import nvcc_build
    return nvcc_build.build(force=force, verbose=verbose)
