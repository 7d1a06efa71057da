"""GB300-native Kadanoff-Baym time stepping (arXiv 2505.19467) on one GPU.

The numerical work runs in ``libkbe.so`` (hand-written CUDA for sm_103a,
C ABI in ``include/kbe.h``); this package is its thin Python binding.
"""
from ._binding import (KBE, KBEError, KBE_PREC_FP64, KBE_PREC_DF64, KBE_PREC_C64, KBE_PREC_F16X2, PRECISIONS,
                       EXPORTS, collision_row_workspace, pack, LIB_PATH, load, collision_row,
                       propagators, sigma_row, sigma_row_noalloc, sigma_row_workspace, update_row,
                       NOALLOC_SCRATCH_BYTES, KBEBatch, memory_bytes, backward_memory_bytes,
                       system_config, device_info, measure_fma_peaks,
                       set_sweep_choice, history_bytes)
from .builder import build

__all__ = ["KBE", "KBEError", "KBE_PREC_FP64", "KBE_PREC_DF64", "KBE_PREC_C64", "KBE_PREC_F16X2", "PRECISIONS",
           "collision_row_workspace", "pack", "EXPORTS", "LIB_PATH", "load", "build",
           "sigma_row", "sigma_row_noalloc", "sigma_row_workspace", "NOALLOC_SCRATCH_BYTES", "collision_row", "propagators", "update_row",
           "KBEBatch", "memory_bytes", "backward_memory_bytes", "system_config", "device_info", "measure_fma_peaks", "set_sweep_choice", "history_bytes", "occupations",
           "KBEFunction"]


def __getattr__(name):   # the torch.autograd wrapper is imported on first use
    if name in ("occupations", "KBEFunction"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
