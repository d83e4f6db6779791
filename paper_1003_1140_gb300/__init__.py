"""GB300-native in-situ radiation-spectrum accumulator (sm_103a CUDA + C ABI).

The hot path -- per-step ingest of leapfrog states, the FP32 split-phase and
FP64 accumulation of the Lienard-Wiechert far-field amplitude, the window
close and the finalize -- runs in ``_build/librad.so`` built from ``csrc/``.
``rad`` is a ctypes binding with the same entry points as ``include/rad.h``.
"""
from .rad import (RAD_COHERENT, RAD_FP32_SPLIT, RAD_FP64, RAD_INCOHERENT, RAD_VARIANT_AUTO,
                  RAD_VARIANT_MIX, RAD_VARIANT_PRECISE, RAD_VARIANT_SFU, RadError, Radiation, load,
                  spectrum_from_sums)

__all__ = ["Radiation", "RadError", "load", "RAD_COHERENT", "RAD_INCOHERENT", "RAD_FP32_SPLIT",
           "RAD_FP64", "RAD_VARIANT_AUTO", "RAD_VARIANT_SFU", "RAD_VARIANT_MIX",
           "RAD_VARIANT_PRECISE", "spectrum_from_sums"]
