"""GB300-native embedded-boundary viscoplastic flow solver (arXiv:1905.07392).

The compute path is the CUDA library ``libebvisc.so`` (sources in ``csrc/``,
C-ABI in ``include/ebvisc.h``); ``ebvisc`` is its thin ctypes binding.  Import
of this package is light: the library is loaded on first use.
"""
__all__ = ["workloads"]
