"""GB300-native Gray-Scott 7-point stencil (arxiv 2309.10292, Eq. 1-3).

The compute path is the CUDA library ``libgs.so`` built from ``csrc/``; the
ctypes binding in :mod:`paper_2309_10292_gb300.gs` exposes its C-ABI under
the same names.  Importing this package does not load the library; the
binding raises when it is missing.
"""
