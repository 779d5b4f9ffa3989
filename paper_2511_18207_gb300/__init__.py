"""GB300-native ProHD hot path (arxiv 2511.18207): a CUDA library for sm_103a
behind a C ABI (``include/prohd.h``), with a thin ctypes binding.

Importing the package loads nothing; the CUDA library is loaded on first use
by :mod:`paper_2511_18207_gb300.prohd`.
"""
