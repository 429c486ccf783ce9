"""GB300 (sm_103a) implementation of the FIRLS hot path (arXiv 1411.5057).

The compute lives in the CUDA library ``libfirls.so`` (C ABI in
``include/firls.h``); this package holds its sources (``csrc/``), the build
step (``build.py``) and a thin ctypes binding (``binding.py``).
"""
from .binding import (Cnn, DenseContext, PSI_DB4, PSI_HAAR, PSI_TV, PSI_TV_ANISO, Context, FirlsError, Params, Stats, lib,
                      make_params, serve, size_supported, solve_multi)

__all__ = ["Cnn", "DenseContext", "PSI_DB4", "PSI_HAAR", "PSI_TV", "PSI_TV_ANISO", "Context", "FirlsError", "Params", "Stats", "lib", "make_params",
           "serve", "size_supported", "solve_multi"]
