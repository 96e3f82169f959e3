"""GB300-native screened periodic LRI exchange build (arXiv:2009.12505).

The compute path is the CUDA library ``libhfx`` (C ABI in ``include/hfx.h``);
``paper_2009_12505_gb300.hfx`` is a thin ctypes binding with the same names.
There is no CPU fallback: loading fails loudly if the library cannot be built
or loaded.
"""
from .hfx import (HFX_BF16X3, HFX_FP64, HFX_OZAKI, Context, ExchangeEnergy, HfxError,
                  build_batch, build_library, load_library)

__all__ = ["Context", "ExchangeEnergy", "HfxError", "HFX_FP64", "HFX_BF16X3", "HFX_OZAKI", "build_batch",
           "build_library", "load_library"]
