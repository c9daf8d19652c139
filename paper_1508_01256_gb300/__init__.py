"""GB300-native Parallel-l0 expander decoding (Mendoza-Smith & Tanner,
"Expander l0-decoding", 2015).

The compute path is the CUDA library ``libccs.so`` (sources in ``csrc/``,
C ABI in ``include/ccs.h``); ``ccs`` is its thin ctypes binding and
``inputs`` draws seeded synthetic problems.
"""
__all__ = ["ccs", "inputs"]
