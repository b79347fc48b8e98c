"""GB300-native saliency-progressive point-source hologram generation.

The compute path is libcgh.so (CUDA for sm_103a, C ABI in include/cgh.h); this
package holds its sources, its in-tree build and a thin ctypes binding.
"""
from .cgh import (CghError, Plan, lib, FORMS, FORM_DIRECT_LUT, FORM_TC_BF16X3,  # noqa: F401
                  FORM_TC_FP16X3)

__all__ = ["CghError", "Plan", "lib", "FORMS"]
