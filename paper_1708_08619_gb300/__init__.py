"""GB300-native multiple-time-origin time correlation (MSD / autocorrelation).

The compute path is the CUDA library ``libtcorr.so`` (built from ``csrc/``);
``tcorr`` is its Python binding.  Importing this package loads nothing: the
library is opened on first use by ``paper_1708_08619_gb300.tcorr``.
"""
__all__ = ["tcorr", "synth", "build"]
