"""GB300-native signature-kernel library (sm_103a): the tile-centred local
Neumann/power-series solver of arXiv 2502.20392 as a persistent CUDA
wavefront kernel behind the C-ABI in include/sigk.h.

Import is light: the CUDA library is loaded on first use by ``sigk``.
"""
__all__ = ["sigk", "synth", "build"]
